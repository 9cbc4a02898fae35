"""Pins of the oracle's screening against the definition it restates, with no planner in
the loop (Eq. cut and Sec. III A; App. Alg. 4 for the pair rule):

* r_cut of a primitive is the largest root of f(r) = |cN| r^(l+2) exp(-alpha r^2) = tau,
  found here by an independent root finder (scipy's brentq) bracketed at the analytic
  maximum of f; f stays below tau beyond it; the primitive is dropped exactly when the
  maximum of f is below tau.
* R_p of a kept pair is the largest root of
  h(r) = |c_aN_a c_bN_b| K_ab (r+|P-A|)^la (r+|P-B|)^lb r^2 exp(-alpha_p r^2) = tau;
  a pair that passes the distance rule but is dropped has h < tau for every r.
* Brute force on grid points, from the Cartesian Gaussians themselves (no h): at every
  point outside a kept pair's integer box, r^2 |phi_mu phi_nu| < tau (r the distance from
  P); for a pair dropped by the distance rule |A - B - T| >= r_a + r_b, at every point
  one of the two primitives is below its own threshold, |r-X|^2 |phi| < tau (what the
  distance rule guarantees); the integer box is the tightest one holding P +- R_p.

These fail for a wrong power of r, a wrong branch of the root, a swapped ceil/floor or a
wrong N/L scaling of the box, in the oracle or in any code that matches it bit for bit.
"""
import itertools
import math

import numpy as np
import pytest
from scipy.optimize import brentq, minimize_scalar

import oracle
import systems
import workloads


def _f(cn, l, a, r):
    return abs(cn) * r ** (l + 2) * math.exp(-a * r * r)


def _largest_root(fun, rmax, tau, scale):
    """Largest root of fun(r) = tau for a function that decreases beyond rmax."""
    hi = rmax + scale
    while fun(hi) >= tau:
        hi = rmax + 2.0 * (hi - rmax)
    return brentq(lambda r: fun(r) - tau, rmax, hi, xtol=1e-300, rtol=8.9e-16, maxiter=500)


@pytest.mark.parametrize("l", [0, 1, 2, 3])
@pytest.mark.parametrize("alpha", [0.11, 0.9, 6.5, 40.0])
@pytest.mark.parametrize("tau", [1e-6, 1e-10, 1e-14])
def test_rcut_is_largest_root(l, alpha, tau):
    lib = oracle._lib()
    cn = oracle.prim_norm(l, alpha) * 0.7
    r = lib.orc_rcut(cn, l, alpha, tau)
    rmax = math.sqrt((l + 2) / (2.0 * alpha))          # f'(r) = 0
    if _f(cn, l, alpha, rmax) < tau:
        assert r == -1.0
        return
    root = _largest_root(lambda x: _f(cn, l, alpha, x), rmax, tau, 1.0 / math.sqrt(alpha))
    assert abs(r - root) <= 1e-12 * root
    assert _f(cn, l, alpha, r) < tau * (1 + 1e-13)
    assert _f(cn, l, alpha, r * (1 - 1e-11)) >= tau
    beyond = r * (1.0 + np.geomspace(1e-12, 20.0, 4000))
    assert max(_f(cn, l, alpha, x) for x in beyond) < tau


@pytest.mark.parametrize("l", [0, 2, 3])
def test_rcut_drops_exactly_below_threshold(l):
    lib = oracle._lib()
    alpha, tau = 1.7, 1e-8
    rmax = math.sqrt((l + 2) / (2.0 * alpha))
    peak_per_cn = rmax ** (l + 2) * math.exp(-alpha * rmax * rmax)
    assert lib.orc_rcut(tau * (1 - 1e-9) / peak_per_cn, l, alpha, tau) == -1.0
    r = lib.orc_rcut(tau * (1 + 1e-9) / peak_per_cn, l, alpha, tau)
    assert r > 0 and abs(r - rmax) < 1e-3 * rmax


# ------------------------------------------------------------------ pairs ---------

def _cells():
    tiny = workloads.tiny()
    skew = systems.skewed(seed=5).with_tau(1e-6)
    water4 = workloads.config("water4")
    return {"tiny": tiny, "skewed": skew, "water4": water4}


@pytest.fixture(scope="module", params=["tiny", "skewed", "water4"])
def cell(request):
    s = _cells()[request.param]
    op = oracle.Plan(s)
    return request.param, s, op


def _pair_geometry(op, p, lat):
    pr = op.prims
    a, b = int(op.ab[p, 0]), int(op.ab[p, 1])
    A = pr["center"][a]
    B = pr["center"][b] + op.img[p].astype(np.float64) @ lat
    aa, ab = float(pr["alpha"][a]), float(pr["alpha"][b])
    ap = aa + ab
    P = (aa * A + ab * B) / ap
    K = math.exp(-aa * ab * float(np.sum((A - B) ** 2)) / ap)
    C = abs(float(pr["cn"][a] * pr["cn"][b]))
    return a, b, A, B, P, ap, C * K, int(pr["l"][a]), int(pr["l"][b])


def _h(CK, la, lb, dA, dB, ap):
    return lambda r: CK * (r + dA) ** la * (r + dB) ** lb * r * r * math.exp(-ap * r * r)


def _hmax(h, ap, la, lb):
    r0 = math.sqrt((la + lb + 2) / (2.0 * ap))
    m = minimize_scalar(lambda r: -h(r), bounds=(0.0, r0), method="bounded",
                        options={"xatol": 1e-14 * r0})
    return max(-m.fun, h(r0), h(m.x)), m.x


def test_pair_extent_is_largest_root(cell):
    name, s, op = cell
    lat = np.asarray(s.lattice, dtype=np.float64)
    rng = np.random.default_rng(17)
    idx = np.arange(op.npairs)
    if op.npairs > 3000:
        idx = np.sort(rng.choice(op.npairs, 3000, replace=False))
    for p in idx:
        a, b, A, B, P, ap, CK, la, lb = _pair_geometry(op, p, lat)
        h = _h(CK, la, lb, float(np.linalg.norm(P - A)), float(np.linalg.norm(P - B)), ap)
        R = float(op.R[p])
        hm, rpk = _hmax(h, ap, la, lb)
        assert hm >= s.tau
        root = _largest_root(h, max(rpk, 1e-300), s.tau, 1.0 / math.sqrt(ap))
        assert abs(R - root) <= 1e-10 * root, (name, p, R, root)
        assert h(R) < s.tau * (1 + 1e-12)
        beyond = R * (1.0 + np.geomspace(1e-10, 20.0, 400))
        assert max(h(x) for x in beyond) < s.tau


def _grid_points(lat, N, lo, hi):
    """Cartesian positions of the unwrapped integer points lo..hi (inclusive) of an
    N-point mesh: sum_d (i_d / N_d) R_d."""
    ax = [np.arange(lo[d], hi[d] + 1) for d in range(3)]
    I = np.stack(np.meshgrid(*ax, indexing="ij"), axis=-1).reshape(-1, 3)
    return I, (I / np.asarray(N, dtype=np.float64)) @ lat


def _max_pair_value(r, A, B, la, lb, aa, ab, C):
    """max over the Cartesian components mu of a, nu of b of |phi_mu(r) phi_nu(r)|
    (the largest monomial |x^i y^j z^k| with i+j+k = l is max(|x|,|y|,|z|)^l)."""
    va, vb = r - A, r - B
    ma = np.max(np.abs(va), axis=1) ** la
    mb = np.max(np.abs(vb), axis=1) ** lb
    return C * ma * mb * np.exp(-aa * np.sum(va * va, axis=1) - ab * np.sum(vb * vb, axis=1))


def test_points_outside_each_box_are_below_tau(cell):
    name, s, op = cell
    lat = np.asarray(s.lattice, dtype=np.float64)
    pr = op.prims
    rng = np.random.default_rng(23)
    idx = np.arange(op.npairs)
    if op.npairs > 400:
        idx = np.sort(rng.choice(op.npairs, 400, replace=False))
    worst = 0.0
    for p in idx:
        a, b, A, B, P, ap, CK, la, lb = _pair_geometry(op, p, lat)
        N = op.meshes[int(op.lev[p])]
        lo, hi = op.lo[p], op.hi[p]
        m = np.maximum(2, (0.3 * (hi - lo + 1)).astype(int))
        I, r = _grid_points(lat, N, lo - m, hi + m)
        out = np.any((I < lo) | (I > hi), axis=1)
        r = r[out]
        C = abs(float(pr["cn"][a] * pr["cn"][b]))
        val = _max_pair_value(r, A, B, la, lb, float(pr["alpha"][a]), float(pr["alpha"][b]), C)
        u = val * np.sum((r - P) ** 2, axis=1)
        worst = max(worst, float(u.max()) / s.tau)
        assert u.max() < s.tau * (1 + 1e-9), (name, p, float(u.max()))
    assert worst > 1e-3  # the margin reaches points near the threshold


def test_box_is_tightest_around_extent(cell):
    name, s, op = cell
    lat = np.asarray(s.lattice, dtype=np.float64)
    rec = np.linalg.inv(lat).T          # rows b_d with b_d . R_e = delta
    for p in range(op.npairs):
        *_, P, ap, CK, la, lb = _pair_geometry(op, p, lat)
        N = op.meshes[int(op.lev[p])].astype(np.float64)
        R = float(op.R[p])
        for d in range(3):
            f = float(rec[d] @ P)
            w = R * float(np.linalg.norm(rec[d]))
            x_lo, x_hi = (f - w) * N[d], (f + w) * N[d]
            # lo is the first grid index at or beyond P - R along row d, hi the last
            for x, i, side in ((x_lo, op.lo[p, d], 1), (x_hi, op.hi[p, d], -1)):
                if abs(x - round(x)) < 1e-9:
                    continue  # exactly on a grid plane: either rounding is a valid box
                if side == 1:
                    assert i - 1 < x <= i, (name, p, d)
                else:
                    assert i <= x < i + 1, (name, p, d)


def test_dropped_candidates_are_below_tau(cell):
    """Every (a <= b, T) with |n_d| <= 3 cells that the oracle does not keep."""
    name, s, op = cell
    if name == "water4":
        pytest.skip("brute force over all candidates on the two-atom cells only")
    lat = np.asarray(s.lattice, dtype=np.float64)
    pr = op.prims
    npr = len(pr["l"])
    kept = {(int(a), int(b), *map(int, n)) for (a, b), n in zip(op.ab, op.img)}
    coarse = op.meshes[-1]   # the distance-rule check needs points, not resolution
    n_dist = n_ext = 0
    for a in range(npr):
        for b in range(a, npr):
            ra, rb = float(op.rcut[a]), float(op.rcut[b])
            for n in itertools.product(range(-3, 4), repeat=3):
                if (a, b, *n) in kept:
                    continue
                A = pr["center"][a]
                B = pr["center"][b] + np.asarray(n, dtype=np.float64) @ lat
                dist = float(np.linalg.norm(A - B))
                aa, ab = float(pr["alpha"][a]), float(pr["alpha"][b])
                la, lb = int(pr["l"][a]), int(pr["l"][b])
                if ra < 0 or rb < 0 or dist >= ra + rb:
                    if ra < 0 or rb < 0 or dist > ra + rb + 1.0 or n_dist >= 60:
                        continue  # far apart: covered by the r_cut pins
                    # distance rule: at every point one primitive is below its threshold
                    n_dist += 1
                    c = 0.5 * (A + B)
                    ext = 0.5 * dist + max(ra, rb)
                    f = (c[None, :] + np.array([[-ext], [ext]])) @ np.linalg.inv(lat)
                    lo = np.floor(f.min(axis=0) * coarse).astype(int)
                    hi = np.ceil(f.max(axis=0) * coarse).astype(int)
                    _, r = _grid_points(lat, coarse, lo, hi)
                    for X, al, l, rc, cn in ((A, aa, la, ra, pr["cn"][a]), (B, ab, lb, rb, pr["cn"][b])):
                        v = r - X
                        u = abs(float(cn)) * np.max(np.abs(v), axis=1) ** l * \
                            np.exp(-al * np.sum(v * v, axis=1)) * np.sum(v * v, axis=1)
                        if X is A:
                            ua = u
                        else:
                            ub = u
                    assert np.minimum(ua, ub).max() < s.tau * (1 + 1e-9)
                    continue
                # passed the distance rule, dropped by the pair extent: h < tau everywhere
                n_ext += 1
                ap = aa + ab
                P = (aa * A + ab * B) / ap
                CK = abs(float(pr["cn"][a] * pr["cn"][b])) * math.exp(-aa * ab * dist * dist / ap)
                h = _h(CK, la, lb, float(np.linalg.norm(P - A)), float(np.linalg.norm(P - B)), ap)
                hm, _ = _hmax(h, ap, la, lb)
                assert hm < s.tau, (name, a, b, n, hm)
    assert n_dist + n_ext > 0


def test_every_pair_within_reach_is_kept_or_peaks_below_tau(cell):
    """All (a <= b, T) that pass the distance rule |A - B - T| < r_a + r_b: kept, or
    max_r h(r) < tau (the maximum of h can lie inside sqrt((la+lb+2)/(2 alpha_p)), where
    r^2 exp(-alpha_p r^2) alone peaks, when P is away from A or B)."""
    name, s, op = cell
    lat = np.asarray(s.lattice, dtype=np.float64)
    pr = op.prims
    npr = len(pr["l"])
    kept = {(int(a), int(b), *map(int, n)) for (a, b), n in zip(op.ab, op.img)}
    reach = 1 + int(2.0 * float(op.rcut.max()) / min(np.linalg.norm(lat, axis=1)))
    imgs = np.array(list(itertools.product(range(-reach, reach + 1), repeat=3)), dtype=np.float64)
    T = imgs @ lat
    n_checked = n_kept = 0
    for a in range(npr):
        if op.rcut[a] < 0:
            continue
        for b in range(a, npr):
            if op.rcut[b] < 0:
                continue
            A = pr["center"][a]
            B = pr["center"][b][None, :] + T
            dist = np.linalg.norm(A[None, :] - B, axis=1)
            for t in np.nonzero(dist < op.rcut[a] + op.rcut[b])[0]:
                n = tuple(int(x) for x in imgs[t])
                if (a, b, *n) in kept:
                    n_kept += 1
                    continue
                n_checked += 1
                aa, ab = float(pr["alpha"][a]), float(pr["alpha"][b])
                la, lb = int(pr["l"][a]), int(pr["l"][b])
                ap = aa + ab
                P = (aa * A + ab * B[t]) / ap
                CK = abs(float(pr["cn"][a] * pr["cn"][b])) * math.exp(-aa * ab * float(dist[t]) ** 2 / ap)
                h = _h(CK, la, lb, float(np.linalg.norm(P - A)), float(np.linalg.norm(P - B[t])), ap)
                hm, _ = _hmax(h, ap, la, lb)
                assert hm < s.tau, (name, a, b, n, hm / s.tau)
    assert n_kept == op.npairs
