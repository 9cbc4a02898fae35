"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: 1e-10 relative (max-norm over
the array) for rho and V, 1e-8 Ha for energies, 1e-7 Ha/Bohr for gradients.
Integer plan data (pair sets, images, levels, boxes) must match exactly.
"""
import numpy as np
import pytest

import oracle
import workloads
import systems

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-10


def _rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def gpw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_24881_gb300 as g
    g.load()
    return g


def _cases():
    return {
        "tiny": workloads.tiny(),
        "tiny14": systems.tiny14(),
        "resolved": systems.resolved(),
        "water4": workloads.config("water4"),
    }


@pytest.fixture(scope="module")
def cases():
    out = {}
    for k, s in _cases().items():
        out[k] = (s, oracle.Plan(s))
    return out


@pytest.mark.parametrize("name", ["tiny", "tiny14", "resolved", "water4"])
def test_plan_pairs_identical(gpw, cases, name):
    s, op = cases[name]
    gp = gpw.Plan(s)
    a = gp.pair_table()
    b = op.pair_table()
    assert a.shape == b.shape
    assert np.array_equal(a, b)
    st = gp.stats()
    assert st["pair_points"] == op.pair_points()
    assert [tuple(m) for m in op.meshes.tolist()] == [tuple(m) for m in st["meshes"]]


@pytest.mark.parametrize("name", ["tiny", "tiny14", "resolved", "water4"])
def test_rho_levels(gpw, cases, name):
    s, op = cases[name]
    gp = gpw.Plan(s)
    got = [x.cpu().numpy() for x in gp.eval_rho_levels(s.D)]
    ref = op.rho_levels(s.D)
    scale = max(np.max(np.abs(r)) for r in ref)
    for k, (x, y) in enumerate(zip(got, ref)):
        assert np.max(np.abs(x - y)) <= RTOL * scale, (name, k)
    assert gp.check_device() == 0


@pytest.mark.parametrize("name", ["tiny", "resolved", "water4"])
def test_rho_fine(gpw, cases, name):
    s, op = cases[name]
    gp = gpw.Plan(s)
    got = gp.eval_rho(s.D).cpu().numpy()
    ref = op.combine(op.rho_levels(s.D))
    assert _rel(got, ref) <= RTOL


@pytest.mark.parametrize("name", ["tiny", "resolved", "water4"])
def test_mat_plane_waves(gpw, cases, name):
    s, op = cases[name]
    gp = gpw.Plan(s)
    vf = s.potential.sample(op.meshes[0])
    got = gp.eval_mat(vf).cpu().numpy()
    ref = op.mat_levels(op.restrict(vf))
    assert _rel(got, ref) <= RTOL
    assert np.max(np.abs(got - got.T)) <= 1e-12 * np.max(np.abs(got))


@pytest.mark.parametrize("name", ["tiny", "resolved"])
def test_mat_levels_random(gpw, cases, name):
    s, op = cases[name]
    gp = gpw.Plan(s)
    rng = np.random.default_rng(5)
    vl = [rng.standard_normal(tuple(m)) for m in op.meshes]
    got = gp.eval_mat_levels(vl).cpu().numpy()
    ref = op.mat_levels(vl)
    assert _rel(got, ref) <= RTOL


@pytest.mark.parametrize("name", ["tiny", "resolved", "water4"])
def test_fock(gpw, cases, name):
    s, op = cases[name]
    gp = gpw.Plan(s)
    out = gp.fock(s.D, want_rho=True, want_v=True)
    ref = op.fock(s.D)
    assert abs(out["EH"] - ref["EH"]) <= 1e-8
    assert abs(out["Ex"] - ref["Ex"]) <= 1e-8
    assert _rel(out["rho"].cpu().numpy(), ref["rho_fine"]) <= RTOL
    assert _rel(out["v"].cpu().numpy(), ref["v_fine"]) <= RTOL
    assert _rel(out["V"].cpu().numpy(), ref["V"]) <= RTOL


@pytest.mark.parametrize("name", ["tiny", "resolved", "water4"])
def test_ip1(gpw, cases, name):
    s, op = cases[name]
    gp = gpw.Plan(s)
    vf = s.potential.sample(op.meshes[0])
    got = gp.eval_mat_ip1(s.D, vf).cpu().numpy()
    ref = op.grad_levels(s.D, op.restrict(vf))
    assert np.max(np.abs(got - ref)) <= 1e-7
    assert _rel(got, ref) <= 1e-9


def test_fock_gradient_matches_oracle_and_fd(gpw, cases):
    s, op = cases["resolved"]
    gp = gpw.Plan(s)
    out = gp.fock(s.D, want_v=True)
    g = gp.eval_mat_ip1(s.D, out["v"]).cpu().numpy()
    ref = op.fock(s.D)
    gref = op.grad_levels(s.D, ref["v_levels"])
    assert np.max(np.abs(g - gref)) <= 1e-7
    # central differences of the GPU energy with frozen plan boxes
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


def test_adjoint_identity_gpu(gpw, cases):
    s, op = cases["water4"]
    gp = gpw.Plan(s)
    rng = np.random.default_rng(9)
    D = rng.standard_normal((s.nao, s.nao))
    D = D + D.T
    v = rng.standard_normal(tuple(op.meshes[0]))
    rho = gp.eval_rho(D).cpu().numpy()
    V = gp.eval_mat(v).cpu().numpy()
    omega = float(np.prod(np.diag(s.lattice)))
    lhs = omega / rho.size * float(np.sum(v * rho))
    rhs = float(np.sum(D * V))
    assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), 1.0)


def test_repeatable_and_independent_plans(gpw, cases):
    s, _ = cases["water4"]
    a = gpw.Plan(s)
    b = gpw.Plan(s)
    r1 = a.fock(s.D)
    r2 = b.fock(s.D)
    r3 = a.fock(s.D)
    assert r1["EH"] == r2["EH"] == r3["EH"]
    assert torch.equal(r1["V"], r3["V"])
    assert torch.equal(r1["V"], r2["V"])


def test_empty_screening(gpw):
    # tau so large that every primitive is dropped: zero density, zero V, zero energy
    s = workloads.tiny().with_tau(1e6)
    gp = gpw.Plan(s)
    assert gp.stats()["npairs"] == 0
    out = gp.fock(s.D, want_rho=True)
    assert float(out["rho"].abs().max()) == 0.0
    assert float(out["V"].abs().max()) == 0.0
    assert out["EH"] == 0.0 and out["Ex"] == 0.0


def test_invalid_inputs(gpw):
    s = workloads.tiny()
    bad = s.with_coords(s.coords)
    bad.lattice = np.array([[5.0, 0.0, 0.0], [5.0, 0.0, 0.0], [0.0, 0.0, 5.0]])  # dependent rows
    with pytest.raises(gpw.GpwError) as e:
        gpw.Plan(bad)
    assert e.value.code == -1
    bad2 = s.with_coords(s.coords)
    bad2.shell_l = s.shell_l.copy()
    bad2.shell_l[0] = 4
    with pytest.raises(gpw.GpwError):
        gpw.Plan(bad2)


@pytest.mark.parametrize("name", ["tiny", "resolved", "water4"])
def test_fock_grad_fused(gpw, cases, name):
    # one integration pass at degree L+1 gives V and the gradient
    s, op = cases[name]
    gp = gpw.Plan(s)
    out = gp.fock_grad(s.D)
    ref = op.fock(s.D)
    gref = op.grad_levels(s.D, ref["v_levels"])
    assert abs(out["EH"] - ref["EH"]) <= 1e-8
    assert abs(out["Ex"] - ref["Ex"]) <= 1e-8
    assert _rel(out["V"].cpu().numpy(), ref["V"]) <= RTOL
    assert np.max(np.abs(out["grad"].cpu().numpy() - gref)) <= 1e-7


@pytest.mark.parametrize("tile", [(8, 8, 16), (4, 8, 32), (8, 8, 32), (4, 8, 64)])
def test_tile_shapes(gpw, cases, tile):
    s, op = cases["water4"]
    gp = gpw.Plan(s, tile=tile, tile_integ=tile)
    assert gp.stats()["tile"] == tile and gp.stats()["tile_integ"] == tile
    rl = [x.cpu().numpy() for x in gp.eval_rho_levels(s.D)]
    ref = op.rho_levels(s.D)
    scale = max(np.max(np.abs(r)) for r in ref)
    for x, y in zip(rl, ref):
        assert np.max(np.abs(x - y)) <= RTOL * scale
    out = gp.fock_grad(s.D)
    r = op.fock(s.D)
    assert _rel(out["V"].cpu().numpy(), r["V"]) <= RTOL
    assert np.max(np.abs(out["grad"].cpu().numpy() - op.grad_levels(s.D, r["v_levels"]))) <= 1e-7
    assert gp.check_device() == 0


@pytest.mark.parametrize("tile_integ", [(8, 8, 64), (8, 4, 64)])
def test_integration_only_tiles(gpw, cases, tile_integ):
    s, op = cases["water4"]
    gp = gpw.Plan(s, tile_integ=tile_integ)
    assert gp.stats()["tile_integ"] == tile_integ
    out = gp.fock_grad(s.D)
    r = op.fock(s.D)
    assert _rel(out["V"].cpu().numpy(), r["V"]) <= RTOL
    assert np.max(np.abs(out["grad"].cpu().numpy() - op.grad_levels(s.D, r["v_levels"]))) <= 1e-7
    assert gp.check_device() == 0


def test_integration_z_windows(gpw, cases):
    # 8x8x16 integration sub-boxes whose blocks stage overlapping 48-point z windows: a
    # pair box is cut where a window ends (fewer tasks than at every sub-box end, and
    # windows clipped at the period on meshes that are not a multiple of 48); the V tensor
    # sums are the same in another order
    s, op = cases["water4"]
    gw = gpw.Plan(s, tile_integ=(8, 8, 16), integ_zwin=48)
    gp = gpw.Plan(s, tile_integ=(8, 8, 16))
    assert gw.stats()["integ_zwin"] == 48 and gp.stats()["integ_zwin"] == 16
    assert gw.stats()["nentries_integ"] < gp.stats()["nentries_integ"]
    a = gw.fock_grad(s.D)
    b = gp.fock_grad(s.D)
    r = op.fock(s.D)
    assert _rel(a["V"].cpu().numpy(), r["V"]) <= RTOL
    assert np.max(np.abs(a["grad"].cpu().numpy() - op.grad_levels(s.D, r["v_levels"]))) <= 1e-7
    assert _rel(a["V"].cpu().numpy(), b["V"].cpu().numpy()) <= 1e-13
    assert np.max(np.abs(a["grad"].cpu().numpy() - b["grad"].cpu().numpy())) <= 1e-12
    assert gw.check_device() == 0
    with pytest.raises(gpw.GpwError):  # windows only where a kernel exists for them
        gpw.Plan(s, tile_integ=(8, 8, 32), integ_zwin=48)


def test_real_transforms_odd_and_even_meshes(gpw):
    # the real FFTs of the combine and the restriction run as half-length complex
    # transforms where the z extent is even and the grid 16-byte aligned, and as cuFFT's
    # real transforms otherwise: here level 0 and 1 have odd z extents (so level 2's grid
    # starts at an odd offset too) and the result is the oracle's all the same
    import dataclasses
    s = dataclasses.replace(workloads.tiny(),
                            meshes=np.array([[40, 40, 41], [20, 20, 21], [10, 10, 10]], np.int32))
    op = oracle.Plan(s)
    gp = gpw.Plan(s)
    out = gp.fock(s.D, want_rho=True, want_v=True)
    ref = op.fock(s.D)
    assert abs(out["EH"] - ref["EH"]) <= 1e-8 and abs(out["Ex"] - ref["Ex"]) <= 1e-8
    assert _rel(out["rho"].cpu().numpy(), ref["rho_fine"]) <= RTOL
    assert _rel(out["v"].cpu().numpy(), ref["v_fine"]) <= RTOL
    assert _rel(out["V"].cpu().numpy(), ref["V"]) <= RTOL


def test_real_transforms_keep_their_inputs(gpw, cases):
    # the forward transform of a caller's potential (eval_mat) leaves it unchanged
    s, op = cases["water4"]
    gp = gpw.Plan(s)
    vf = torch.as_tensor(s.potential.sample(op.meshes[0]), device="cuda")
    v0 = vf.clone()
    V = gp.eval_mat(vf)
    torch.cuda.synchronize()
    assert torch.equal(vf, v0)
    assert _rel(V.cpu().numpy(), op.mat_levels(op.restrict(v0.cpu().numpy()))) <= RTOL


def test_unsupported_tile(gpw):
    with pytest.raises(gpw.GpwError):
        gpw.Plan(workloads.tiny(), tile=(3, 8, 16))
    with pytest.raises(gpw.GpwError):  # an integration-only shape as collocation tile
        gpw.Plan(workloads.tiny(), tile=(8, 8, 64))


def test_mixed_tiles_carbon_like_f_shells(gpw):
    # f shells (L up to 6 per pair) with different collocation and integration tiles
    s = systems.resolved(seed=8, shells=((0, 1), (1, 1), (2, 1), (3, 1)), natm=3)
    op = oracle.Plan(s)
    gp = gpw.Plan(s, tile=(4, 8, 32), tile_integ=(8, 8, 32))
    out = gp.fock_grad(s.D)
    r = op.fock(s.D)
    assert _rel(out["V"].cpu().numpy(), r["V"]) <= RTOL
    assert abs(out["EH"] - r["EH"]) <= 1e-8 and abs(out["Ex"] - r["Ex"]) <= 1e-8
    assert np.max(np.abs(out["grad"].cpu().numpy() - op.grad_levels(s.D, r["v_levels"]))) <= 1e-7


def test_fock_grad_from_host_buffers(gpw):
    # gpw_fock_grad_host (host D in, host V / gradient / energies out, through the C ABI)
    # runs the same build as the device-pointer call: identical results, pinned or
    # pageable host memory, and repeated calls on the plan's kept device copies
    s = workloads.config("water4")
    p = gpw.Plan(s)
    ref = p.fock_grad(s.D)
    for pinned in (True, False):
        Dh = torch.as_tensor(np.ascontiguousarray(s.D))
        if pinned:
            Dh = Dh.pin_memory()
        for _ in range(2):
            out = p.fock_grad_host(Dh)
            assert torch.equal(out["V"], ref["V"].cpu())
            assert torch.equal(out["grad"], ref["grad"].cpu())
            assert float(out["E"][0]) == ref["EH"] and float(out["E"][1]) == ref["Ex"]
    assert p.check_device() == 0
    p.close()


@pytest.mark.parametrize("host_tasks", [False, True])
def test_debug_checks(gpw, host_tasks):
    # GPW_DEBUG_CHECKS: the task lists pass their validation at commit, the results are
    # those of a plain plan bit for bit, and an output that is not finite is reported
    # through the device error word (code 16) without disturbing the plan
    s = workloads.config("water4")
    dbg = gpw.Plan(s, debug_checks=True, host_tasks=host_tasks)
    assert dbg.check_device() == 0
    ref = gpw.Plan(s).fock_grad(s.D)
    out = dbg.fock_grad(s.D)
    assert torch.equal(out["V"], ref["V"]) and torch.equal(out["grad"], ref["grad"])
    assert out["EH"] == ref["EH"] and out["Ex"] == ref["Ex"]
    assert dbg.check_device() == 0
    bad = s.D.copy()
    bad[0, 0] = float("nan")
    dbg.fock_grad(bad)
    assert dbg.check_device() == 16
    assert dbg.check_device() == 0  # read and cleared
    out = dbg.fock_grad(s.D)
    assert torch.equal(out["V"], ref["V"]) and dbg.check_device() == 0
    dbg.close()


def test_permuting_atoms_permutes_V_and_gradient_gpu(gpw):
    # the 4-water box with its atoms in another seeded order (shells and D reindexed):
    # the GPU gives the same energies, and V and the gradient reindexed, to the parity
    # tolerances, and each of the two agrees with the oracle
    s = workloads.config("water4").with_tau(1e-12)
    perm = np.random.default_rng(17).permutation(s.natm)
    r, ao = systems.permuted_atoms(s, perm)
    outs = []
    for sys_ in (s, r):
        gp = gpw.Plan(sys_)
        o = gp.fock_grad(sys_.D)
        outs.append(dict(EH=o["EH"], Ex=o["Ex"], V=o["V"].cpu().numpy(), g=o["grad"].cpu().numpy()))
        gp.close()
    a, b = outs
    assert abs(a["EH"] - b["EH"]) <= 1e-8 and abs(a["Ex"] - b["Ex"]) <= 1e-8
    assert _rel(b["V"], a["V"][np.ix_(ao, ao)]) <= RTOL
    assert np.max(np.abs(b["g"] - a["g"][perm])) <= 1e-7
    ref = oracle.Plan(r).fock(r.D)
    assert abs(b["EH"] - ref["EH"]) <= 1e-8 and _rel(b["V"], ref["V"]) <= RTOL
