"""autograd wrappers: hand-written backward = eval_mat / eval_mat_ip1, checked against
the oracle's analytic gradient and against central finite differences of the oracle
energy with the plan boxes frozen (h = 1e-4 Bohr, 3 seeded atoms)."""
import numpy as np
import pytest

import oracle
import workloads
import systems

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_24881_gb300 as g
    g.load()
    return g


def _rotated():
    # a triclinic cell turned by a seeded rotation: no row of the lattice is triangular,
    # so the cell volume is not the product of the lattice's diagonal
    return systems.rotated(systems.skewed(shells=((0, 1), (1, 1), (2, 1)), natm=2),
                           systems.rotation(12))


@pytest.mark.parametrize("name", ["resolved", "water4", "triclinic", "rotated"])
def test_energy_backward_matches_oracle_and_fd(gpw, name):
    from paper_2603_24881_gb300 import autograd as ag
    s = {"resolved": systems.resolved, "water4": lambda: workloads.config("water4"),
         "triclinic": lambda: systems.skewed(shells=((0, 1), (1, 1), (2, 1)), natm=2),
         "rotated": _rotated}[name]()
    plan = gpw.Plan(s)
    op = oracle.Plan(s)
    D = torch.as_tensor(s.D, device="cuda").requires_grad_(True)
    R = torch.as_tensor(s.coords, device="cuda").requires_grad_(True)
    E = ag.energy(D, R, plan)
    E.backward()
    ref = op.fock(s.D)
    assert abs(float(E) - (ref["EH"] + ref["Ex"])) <= 1e-8
    gref = op.grad_levels(s.D, ref["v_levels"])
    assert float(np.max(np.abs(R.grad.cpu().numpy() - gref))) <= 1e-7
    Vref = ref["V"]
    assert float(np.max(np.abs(D.grad.cpu().numpy() - Vref))) <= 1e-10 * np.max(np.abs(Vref))
    # central differences of the ORACLE energy with frozen boxes
    rng = np.random.default_rng(31)
    h = 1e-4
    for at in rng.choice(s.natm, size=min(3, s.natm), replace=False):
        d = int(rng.integers(0, 3))
        cp, cm = s.coords.copy(), s.coords.copy()
        cp[at, d] += h
        cm[at, d] -= h
        fd = (op.with_coords(cp).energy(s.D) - op.with_coords(cm).energy(s.D)) / (2 * h)
        assert abs(fd - float(R.grad[at, d])) <= 1e-6 * max(1.0, abs(fd))


@pytest.mark.parametrize("name", ["water4", "rotated"])
def test_rho_backward_is_the_adjoint(gpw, name):
    from paper_2603_24881_gb300 import autograd as ag
    s = workloads.config("water4") if name == "water4" else _rotated()
    plan = gpw.Plan(s)
    D = torch.as_tensor(s.D, device="cuda").requires_grad_(True)
    R = torch.as_tensor(s.coords, device="cuda").requires_grad_(True)
    rho = ag.rho(D, R, plan)
    w = torch.randn(rho.shape, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    L = (w * rho).sum()
    L.backward()
    # directional derivative along a symmetric D perturbation
    X = torch.randn(D.shape, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(6))
    X = X + X.T
    h = 1e-3
    Lp = float((w * plan.eval_rho(D.detach() + h * X)).sum())
    Lm = float((w * plan.eval_rho(D.detach() - h * X)).sum())
    fd = (Lp - Lm) / (2 * h)
    assert abs(fd - float((D.grad * X).sum())) <= 1e-8 * max(1.0, abs(fd))
    # coordinate derivative with frozen boxes
    at, d, hr = min(2, s.natm - 1), 1, 1e-4
    c = s.coords.copy()
    c[at, d] += hr
    plan.update_coords(c)
    Lp = float((w * plan.eval_rho(D.detach())).sum())
    c[at, d] -= 2 * hr
    plan.update_coords(c)
    Lm = float((w * plan.eval_rho(D.detach())).sum())
    plan.update_coords(s.coords)
    fd = (Lp - Lm) / (2 * hr)
    assert abs(fd - float(R.grad[at, d])) <= 1e-6 * max(1.0, abs(fd))


def test_tau_backward_is_the_adjoint(gpw):
    # the tau wrapper: gradients with respect to D and the atoms from the tau integration
    # directions, against central differences of the forward (boxes frozen)
    from paper_2603_24881_gb300 import autograd as ag
    s = systems.resolved(seed=6, shells=((0, 1), (1, 1), (2, 1), (3, 1)), cutoff=100.0)
    plan = gpw.Plan(s, tau=True)
    D = torch.as_tensor(s.D, device="cuda").requires_grad_(True)
    R = torch.as_tensor(s.coords, device="cuda").requires_grad_(True)
    t = ag.tau(D, R, plan)
    w = torch.randn(t.shape, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(7))
    (w * t).sum().backward()
    X = torch.randn(D.shape, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(8))
    X = X + X.T
    h = 1e-3
    fd = (float((w * plan.eval_tau(D.detach() + h * X)).sum()) -
          float((w * plan.eval_tau(D.detach() - h * X)).sum())) / (2 * h)
    assert abs(fd - float((D.grad * X).sum())) <= 1e-8 * max(1.0, abs(fd))
    at, d, hr = 1, 2, 1e-4
    c = s.coords.copy()
    c[at, d] += hr
    plan.update_coords(c)
    Lp = float((w * plan.eval_tau(D.detach())).sum())
    c[at, d] -= 2 * hr
    plan.update_coords(c)
    Lm = float((w * plan.eval_tau(D.detach())).sum())
    plan.update_coords(s.coords)
    fd = (Lp - Lm) / (2 * hr)
    assert abs(fd - float(R.grad[at, d])) <= 1e-6 * max(1.0, abs(fd))


def test_energy_backward_pbe_exchange(gpw):
    # the energy wrapper with a GGA plan (PBE exchange): dE/dD = V and dE/dR against the
    # oracle's PBE build and its analytic gradient
    from paper_2603_24881_gb300 import autograd as ag
    s = systems.resolved(seed=5, shells=((0, 1), (1, 1), (2, 1)), natm=2)
    plan = gpw.Plan(s, xc="pbe_x")
    op = oracle.Plan(s)
    D = torch.as_tensor(s.D, device="cuda").requires_grad_(True)
    R = torch.as_tensor(s.coords, device="cuda").requires_grad_(True)
    E = ag.energy(D, R, plan)
    E.backward()
    ref = op.fock(s.D, xc="pbe_x")
    assert abs(float(E.detach()) - (ref["EH"] + ref["Ex"])) <= 1e-8
    assert float(np.max(np.abs(D.grad.cpu().numpy() - ref["V"]))) <= 1e-10 * np.max(np.abs(ref["V"]))
    g = op.grad_levels(s.D, ref["v_levels"])
    assert float(np.max(np.abs(R.grad.cpu().numpy() - g))) <= 1e-7
