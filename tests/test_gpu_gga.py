"""GGA exchange (PBE exchange, GPW_XC_PBE_X) on the GPU against the oracle: the same
collocation and integration, Fourier gradients of the density and the divergence of
de/d grad rho folded into the potential (Sec. II, GGA).  Tolerances as for LDA: 1e-10
relative in V and potentials, 1e-8 Ha in energies, 1e-7 Ha/Bohr in gradients."""
import numpy as np
import pytest

import oracle
import workloads
import systems

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


@pytest.fixture(scope="module", params=["tiny", "resolved", "water4"])
def case(request):
    s = {"tiny": workloads.tiny, "resolved": systems.resolved,
         "water4": lambda: workloads.config("water4")}[request.param]()
    op = oracle.Plan(s)
    return request.param, s, op, op.fock(s.D, xc="pbe_x")


def test_fock_and_potential(gpw, case):
    name, s, op, ref = case
    gp = gpw.Plan(s, xc="pbe_x")
    assert gp.stats()["xc"] == "pbe_x"
    out = gp.fock(s.D, want_rho=True, want_v=True)
    assert abs(out["EH"] - ref["EH"]) <= 1e-8, name
    assert abs(out["Ex"] - ref["Ex"]) <= 1e-8, name
    assert _rel(out["rho"].cpu().numpy(), ref["rho_fine"]) <= RTOL, name
    assert _rel(out["v"].cpu().numpy(), ref["v_fine"]) <= RTOL, name
    assert _rel(out["V"].cpu().numpy(), ref["V"]) <= RTOL, name
    # the gradient correction is not negligible on these cells
    lda = op.fock(s.D)
    assert abs(ref["Ex"] - lda["Ex"]) > 1e-4 * abs(lda["Ex"])
    assert gp.check_device() == 0


def test_fock_grad(gpw, case):
    name, s, op, ref = case
    gp = gpw.Plan(s, xc="pbe_x")
    out = gp.fock_grad(s.D)
    assert abs(out["EH"] - ref["EH"]) <= 1e-8 and abs(out["Ex"] - ref["Ex"]) <= 1e-8
    assert _rel(out["V"].cpu().numpy(), ref["V"]) <= RTOL
    g = op.grad_levels(s.D, ref["v_levels"])
    assert np.max(np.abs(out["grad"].cpu().numpy() - g)) <= 1e-7, name


def test_batch_mixes_functionals(gpw):
    # one batch: a PBE plan and an LDA plan, each equal to its own run alone
    s1, s2 = workloads.config("water4"), workloads.small_water(4, seed=13)
    alone = []
    for s, xc in [(s1, "pbe_x"), (s2, "lda_x")]:
        p = gpw.Plan(s, xc=xc)
        r = p.fock_grad(s.D)
        alone.append(r)
    plans = [gpw.Plan(s1, xc="pbe_x"), gpw.Plan(s2, xc="lda_x")]
    b = gpw.Batch(2).set(plans)
    Ds = [torch.as_tensor(s.D, device="cuda") for s in (s1, s2)]
    Vs = [torch.empty((p.nao, p.nao), dtype=torch.float64, device="cuda") for p in plans]
    gs = [torch.empty((p.natm, 3), dtype=torch.float64, device="cuda") for p in plans]
    E = torch.empty(4, dtype=torch.float64, device="cuda")
    b.fock_grad_async(Ds, Vs, gs, E)
    torch.cuda.synchronize()
    e = E.cpu().numpy()
    for i, r in enumerate(alone):
        assert abs(e[2 * i] - r["EH"]) <= 1e-8 and abs(e[2 * i + 1] - r["Ex"]) <= 1e-8
        assert _rel(Vs[i].cpu().numpy(), r["V"].cpu().numpy()) <= RTOL
        assert np.max(np.abs(gs[i].cpu().numpy() - r["grad"].cpu().numpy())) <= 1e-7
    b.close()


def test_unknown_functional(gpw):
    with pytest.raises(ValueError):
        gpw.Plan(workloads.tiny(), xc="b88")
