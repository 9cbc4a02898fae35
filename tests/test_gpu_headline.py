"""The headline workload against the oracle in full: the 256-water box (28 functions per
water, 280 Ha, 4 levels) as bench.py times it, one gpw_fock_grad in the plan's default
launch configuration.

* E_H and E_x of the whole Fock build to 1e-8 Ha, all of V to 1e-10 relative, the
  finest-grid potential v_Hxc to 1e-10 relative: the oracle builds the whole Fock matrix
  (every pair, every grid point, numpy's FFT for the spectral steps) on the host cores.
* The gradient of 3 seeded atoms against the oracle's analytic gradient (Alg. 3) taken
  with the oracle's own level potentials, to 1e-7 Ha/Bohr.
* Central finite differences of the GPU energy on the same atoms, all three directions
  (h = 1e-4 Bohr, pair set and boxes frozen through gpw_plan_update_coords), against the
  GPU gradient to 1e-7 Ha/Bohr.  At h = 1e-4 the quotient's truncation error h^2 E'''/6
  and its rounding error (the ~3e4 Ha energy is summed over 2.4e7 points, a few 1e-12
  Ha, divided by 2h) both stay near 1e-8; a smaller h would trade the first for more of
  the second.
"""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-10


@pytest.fixture(scope="module")
def water256():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_24881_gb300 as gpw
    gpw.load()
    s = workloads.config("water256")
    gp = gpw.Plan(s)
    out = gp.fock_grad(s.D)
    res = dict(EH=out["EH"], Ex=out["Ex"], V=out["V"].cpu().numpy(),
               grad=out["grad"].cpu().numpy())
    res["v"] = gp.fock(s.D, want_v=True)["v"].cpu().numpy()
    op = oracle.Plan(s)
    ref = op.fock(s.D)
    yield s, gp, op, res, ref
    gp.close()
    torch.cuda.empty_cache()


def test_energies_and_V(water256):
    s, gp, op, res, ref = water256
    assert np.array_equal(gp.pair_table(), op.pair_table())
    assert abs(res["EH"] - ref["EH"]) <= 1e-8, (res["EH"], ref["EH"])
    assert abs(res["Ex"] - ref["Ex"]) <= 1e-8, (res["Ex"], ref["Ex"])
    Vref = ref["V"]
    assert float(np.max(np.abs(res["V"] - Vref))) <= RTOL * float(np.max(np.abs(Vref)))
    vref = ref["v_fine"]
    assert float(np.max(np.abs(res["v"] - vref))) <= RTOL * float(np.max(np.abs(vref)))


def _atoms(s):
    return np.random.default_rng(41).choice(s.natm, size=3, replace=False)


def test_gradient_against_oracle(water256):
    s, gp, op, res, ref = water256
    pa = op.prims["atom"]
    for at in _atoms(s):
        sel = np.nonzero((pa[op.ab[:, 0]] == at) | (pa[op.ab[:, 1]] == at))[0]
        g = op.grad_levels(s.D, ref["v_levels"], sel=sel)[at]
        assert np.max(np.abs(res["grad"][at] - g)) <= 1e-7, (at, res["grad"][at], g)


def test_gradient_against_finite_differences(water256):
    s, gp, op, res, ref = water256

    def energy(coords):
        gp.update_coords(coords)
        o = gp.fock(s.D)
        return o["EH"] + o["Ex"]

    def quotient(at, d, h):
        cp, cm = s.coords.copy(), s.coords.copy()
        cp[at, d] += h
        cm[at, d] -= h
        return (energy(cp) - energy(cm)) / (2 * h)

    h = 1e-4
    try:
        for at in _atoms(s):
            for d in range(3):
                fd = quotient(at, d, h)
                g = float(res["grad"][at, d])
                assert abs(fd - g) <= 1e-7, (at, d, fd, g)
    finally:
        gp.update_coords(s.coords)
    assert gp.check_device() == 0
