"""Non-orthogonal cells (App., non-orthogonal lattices) on the GPU against the oracle:
pair tables bit for bit, level densities, the Fock build and the Hxc gradient within
the tolerances of the orthorhombic path (1e-10 relative for rho and V, 1e-8 Ha, 1e-7
Ha/Bohr), the sheared description of a cubic crystal against the cubic one, batches."""
import numpy as np
import pytest

import oracle
import systems
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-10


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def gpw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_24881_gb300 as g
    g.load()
    return g


CASES = {
    "skewed_spd": lambda: systems.skewed(shells=((0, 1), (1, 1), (2, 1)), natm=2),
    "skewed_f": lambda: systems.skewed(seed=8, shells=((0, 1), (1, 1), (2, 1), (3, 1)), natm=3),
    "sheared": lambda: systems.sheared(systems.resolved(seed=7, shells=((0, 1), (1, 1), (2, 1)), natm=2)),
    # third row orthogonal to the first two: the kernels' R01-only path
    "hexagonal": lambda: systems.skewed(seed=9, shells=((0, 1), (1, 1), (2, 1), (3, 1)), natm=2,
                                        lattice=6.0 * workloads.HEXAGONAL),
    # a triclinic cell turned by a seeded rotation: no lattice row on an axis
    "rotated": lambda: systems.rotated(systems.skewed(seed=6, shells=((0, 1), (1, 1), (2, 1), (3, 1)),
                                                      natm=2), systems.rotation(12)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_skew_parity(gpw, name):
    s = CASES[name]()
    op = oracle.Plan(s)
    gp = gpw.Plan(s)
    assert np.array_equal(gp.pair_table(), op.pair_table())
    rl = [x.cpu().numpy() for x in gp.eval_rho_levels(s.D)]
    ref = op.rho_levels(s.D)
    scale = max(np.max(np.abs(r)) for r in ref)
    for x, y in zip(rl, ref):
        assert np.max(np.abs(x - y)) <= RTOL * scale, name
    out = gp.fock_grad(s.D)
    r = op.fock(s.D)
    assert abs(out["EH"] - r["EH"]) <= 1e-8 and abs(out["Ex"] - r["Ex"]) <= 1e-8
    assert _rel(out["V"].cpu().numpy(), r["V"]) <= RTOL
    g = op.grad_levels(s.D, r["v_levels"])
    assert np.max(np.abs(out["grad"].cpu().numpy() - g)) <= 1e-7
    f = gp.fock(s.D, want_v=True)
    assert _rel(f["V"].cpu().numpy(), r["V"]) <= RTOL
    assert _rel(f["v"].cpu().numpy(), r["v_fine"]) <= RTOL
    assert gp.check_device() == 0


def test_skew_mat_plane_waves(gpw):
    s = CASES["skewed_f"]()
    op = oracle.Plan(s)
    gp = gpw.Plan(s)
    vf = s.potential.sample(op.meshes[0])
    assert _rel(gp.eval_mat(vf).cpu().numpy(), op.mat_levels(op.restrict(vf))) <= RTOL
    got = gp.eval_mat_ip1(s.D, vf).cpu().numpy()
    assert np.max(np.abs(got - op.grad_levels(s.D, op.restrict(vf)))) <= 1e-7


def test_triclinic_water_sampled(gpw):
    # realistic exponents in a triclinic cell: sampled points of every level density
    # and two Fock blocks against the oracle
    s = workloads.config("water4_triclinic")
    op = oracle.Plan(s)
    gp = gpw.Plan(s)
    assert np.array_equal(gp.pair_table(), op.pair_table())
    rl = [x.cpu().numpy() for x in gp.eval_rho_levels(s.D)]
    rng = np.random.default_rng(1)
    for k, m in enumerate(op.meshes):
        pts = np.stack([rng.integers(0, int(n), 64) for n in m], axis=1)
        ref = op.rho_points(s.D, k, pts)
        got = rl[k][pts[:, 0], pts[:, 1], pts[:, 2]]
        assert np.max(np.abs(got - ref)) <= RTOL * max(np.max(np.abs(rl[k])), 1e-300), k
    vf = s.potential.sample(op.meshes[0])
    V = gp.eval_mat(vf).cpu().numpy()
    vl = op.restrict(vf)
    off = s.ao_offsets()
    for sa, sb in [(0, 6), (3, 10)]:
        blk = op.mat_block(vl, sa, sb)
        got = V[off[sa]:off[sa + 1], off[sb]:off[sb + 1]]
        assert np.max(np.abs(got - blk)) <= 1e-10 * max(1.0, np.max(np.abs(V)))


def test_sheared_equals_cubic_on_gpu(gpw):
    s = systems.resolved(seed=7, shells=((0, 1), (1, 1), (2, 1)), natm=2, nlevels=2)
    m = oracle.Plan(s).meshes
    s.meshes = np.array([[oracle._smooth7_even(int(1.6 * x)) for x in row] for row in m])
    s.cutoff_ha = 0.0
    s.rel_cutoff = 100.0
    a = gpw.Plan(s).fock_grad(s.D)
    b = gpw.Plan(systems.sheared(s)).fock_grad(s.D)
    assert b["EH"] == pytest.approx(a["EH"], rel=1e-9)
    assert b["Ex"] == pytest.approx(a["Ex"], rel=1e-9)
    assert _rel(b["V"].cpu().numpy(), a["V"].cpu().numpy()) <= 1e-9
    assert np.max(np.abs(b["grad"].cpu().numpy() - a["grad"].cpu().numpy())) <= 1e-8


def test_skew_batch_and_limits(gpw):
    ss = [CASES["skewed_spd"](), CASES["skewed_f"](), CASES["hexagonal"]()]
    plans = [gpw.Plan(s) for s in ss]
    alone = [p.fock_grad(s.D) for p, s in zip(plans, ss)]
    batch = gpw.Batch(3).set(plans)
    Ds = [torch.as_tensor(s.D, device="cuda") for s in ss]
    Vs = [torch.empty((p.nao, p.nao), dtype=torch.float64, device="cuda") for p in plans]
    gs = [torch.empty((p.natm, 3), dtype=torch.float64, device="cuda") for p in plans]
    E = torch.empty(6, dtype=torch.float64, device="cuda")
    batch.fock_grad_async(Ds, Vs, gs, E)
    torch.cuda.synchronize()
    for i, a in enumerate(alone):
        assert float(E[2 * i]) == pytest.approx(a["EH"], rel=1e-12, abs=1e-13)
        assert _rel(Vs[i].cpu().numpy(), a["V"].cpu().numpy()) <= 1e-12
    # a batch does not mix orthorhombic and non-orthogonal cells
    with pytest.raises(gpw.GpwError):
        gpw.Batch(2).set([plans[0], gpw.Plan(systems.resolved())])
    batch.close()


def test_skew_gga_parity(gpw):
    # PBE exchange in a triclinic cell: Cartesian Fourier derivatives from the
    # reciprocal rows, against the oracle
    s = CASES["skewed_spd"]()
    op = oracle.Plan(s)
    gp = gpw.Plan(s, xc="pbe_x")
    out = gp.fock_grad(s.D)
    r = op.fock(s.D, xc="pbe_x")
    assert abs(out["EH"] - r["EH"]) <= 1e-8 and abs(out["Ex"] - r["Ex"]) <= 1e-8
    assert _rel(out["V"].cpu().numpy(), r["V"]) <= RTOL
    assert np.max(np.abs(out["grad"].cpu().numpy() - op.grad_levels(s.D, r["v_levels"]))) <= 1e-7
    f = gp.fock(s.D, want_v=True)
    assert _rel(f["v"].cpu().numpy(), r["v_fine"]) <= RTOL


def test_skew_edge_cases(gpw):
    # no screened pair in a triclinic cell: zero density, V and energies
    s = CASES["skewed_spd"]().with_tau(1e6)
    gp = gpw.Plan(s)
    assert gp.stats()["npairs"] == 0
    out = gp.fock(s.D, want_rho=True)
    assert float(out["rho"].abs().max()) == 0.0 and float(out["V"].abs().max()) == 0.0
    assert out["EH"] == 0.0 and out["Ex"] == 0.0
    # one level with odd, unequal explicit meshes (ragged sub-boxes on every axis)
    s = CASES["skewed_spd"]()
    s.nlevels = 1
    s.meshes = np.array([[45, 39, 51]])
    s.cutoff_ha = 0.0
    op = oracle.Plan(s)
    gp = gpw.Plan(s)
    assert np.array_equal(gp.pair_table(), op.pair_table())
    out = gp.fock_grad(s.D)
    r = op.fock(s.D)
    assert abs(out["EH"] - r["EH"]) <= 1e-8 and abs(out["Ex"] - r["Ex"]) <= 1e-8
    assert _rel(out["V"].cpu().numpy(), r["V"]) <= RTOL
    assert np.max(np.abs(out["grad"].cpu().numpy() - op.grad_levels(s.D, r["v_levels"]))) <= 1e-7


def test_skew_gradient_matches_gpu_finite_differences(gpw):
    # central differences of the GPU energy with the plan frozen (gpw_plan_update_coords
    # moves the centres: images along the lattice rows, tables and cross factors rebuilt)
    s = CASES["skewed_spd"]()
    gp = gpw.Plan(s)
    g = gp.fock_grad(s.D)["grad"].cpu().numpy()
    h = 1e-4
    for atom, d in [(0, 0), (1, 2)]:
        e = []
        for sgn in (1, -1):
            c = s.coords.copy()
            c[atom, d] += sgn * h
            gp.update_coords(c)
            o = gp.fock(s.D)
            e.append(o["EH"] + o["Ex"])
        gp.update_coords(s.coords)
        fd = (e[0] - e[1]) / (2 * h)
        assert abs(fd - g[atom, d]) <= 1e-6 * max(1.0, abs(g[atom, d]))
