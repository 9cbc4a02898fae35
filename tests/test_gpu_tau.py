"""Kinetic-energy-density (meta-GGA) kernels on the GPU against the oracle: tau on the
levels and the finest grid, its Fock term (1/2) int v grad phi . grad phi, and the nuclear
gradient of <v, tau(D)> (Sec. II meta-GGA, Eq. J_metaGGA).  Tolerances as for rho, V
and the Hxc gradient: 1e-10 relative, 1e-7 Ha/Bohr."""
import numpy as np
import pytest

import oracle
import workloads
import systems

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-10


@pytest.fixture(scope="module")
def gpw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_24881_gb300 as g
    g.load()
    return g


SPDF = ((0, 1), (1, 1), (2, 1), (3, 1))


@pytest.fixture(scope="module", params=["tiny", "resolved_d", "triclinic_d", "resolved_f",
                                        "triclinic_f", "rotated_f"])
def case(request):
    s = {"tiny": workloads.tiny,
         "resolved_d": lambda: systems.resolved(seed=6, shells=((0, 1), (1, 1), (2, 1)),
                                                cutoff=100.0),
         # a non-orthogonal cell: the cross-factor kernels at degree L+2 / L+3
         "triclinic_d": lambda: systems.skewed(seed=6, shells=((0, 1), (1, 1), (2, 1)),
                                               cutoff=100.0),
         # f shells: (f|f) pairs reach degree 8 (tau) and 9 (its gradient)
         "resolved_f": lambda: systems.resolved(seed=6, shells=SPDF, cutoff=100.0),
         "triclinic_f": lambda: systems.skewed(seed=7, shells=SPDF, cutoff=100.0),
         "rotated_f": lambda: systems.rotated(systems.skewed(seed=8, shells=SPDF, cutoff=100.0),
                                              systems.rotation(13))}[request.param]()
    return request.param, s, oracle.Plan(s)


def test_tau_levels_and_fine(gpw, case):
    name, s, op = case
    gp = gpw.Plan(s, tau=True)
    ref = op.tau_levels(s.D)
    got = [x.cpu().numpy() for x in gp.eval_tau_levels(s.D)]
    scale = max(np.max(np.abs(r)) for r in ref)
    for k, (x, y) in enumerate(zip(got, ref)):
        assert np.max(np.abs(x - y)) <= RTOL * scale, (name, k)
    fine = gp.eval_tau(s.D).cpu().numpy()
    fref = op.combine(ref)
    assert np.max(np.abs(fine - fref)) <= RTOL * np.max(np.abs(fref)), name
    assert gp.check_device() == 0


def test_mat_tau(gpw, case):
    name, s, op = case
    gp = gpw.Plan(s, tau=True)
    vl = [s.potential.sample(m) for m in op.meshes]
    ref = op.mat_tau_levels(vl)
    got = gp.eval_mat_tau_levels(vl).cpu().numpy()
    assert np.max(np.abs(got - ref)) <= RTOL * np.max(np.abs(ref)), name
    # through the finest grid: restriction of v_fine to the levels first
    vf = s.potential.sample(op.meshes[0])
    ref2 = op.mat_tau_levels(op.restrict(vf))
    got2 = gp.eval_mat_tau(vf).cpu().numpy()
    assert np.max(np.abs(got2 - ref2)) <= RTOL * np.max(np.abs(ref2)), name


def test_tau_gradient(gpw, case):
    name, s, op = case
    gp = gpw.Plan(s, tau=True)
    vl = [s.potential.sample(m) for m in op.meshes]
    ref = op.grad_tau_levels(s.D, vl)
    got = gp.eval_mat_tau_ip1_levels(s.D, vl).cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-7, name
    vf = s.potential.sample(op.meshes[0])
    got2 = gp.eval_mat_tau_ip1(s.D, vf).cpu().numpy()
    ref2 = op.grad_tau_levels(s.D, op.restrict(vf))
    assert np.max(np.abs(got2 - ref2)) <= 1e-7, name


def test_tau_plan_keeps_the_density_path(gpw, case):
    # the larger tables and per-pair buffers of a GPW_TAU plan change no other result
    name, s, op = case
    a = gpw.Plan(s, tau=True).fock_grad(s.D)
    b = gpw.Plan(s).fock_grad(s.D)
    assert float((a["V"] - b["V"]).abs().max()) <= 1e-13 * float(b["V"].abs().max())
    assert abs(a["EH"] - b["EH"]) <= 1e-12 and abs(a["Ex"] - b["Ex"]) <= 1e-12
    assert float((a["grad"] - b["grad"]).abs().max()) <= 1e-12


def test_tau_needs_the_flag(gpw):
    s = workloads.tiny()
    with pytest.raises(gpw.GpwError):
        gpw.Plan(s).eval_tau(s.D)
