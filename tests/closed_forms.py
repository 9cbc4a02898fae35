"""Closed forms and brute-force references that pin the oracle.

None of this code is shared with ``oracle/``: the integrals below are the
textbook Gaussian-product / Hermite forms over all space, and the brute force
evaluates the double lattice sum of Eq. (rho) with periodised orbitals.
"""
from __future__ import annotations

import math

import numpy as np


def _cart(l):
    return [(ix, iy, l - ix - iy) for ix in range(l, -1, -1) for iy in range(l - ix, -1, -1)]


def norm(l, a):
    # N^2 * int x^(2l) e^(-2 a x^2) dx * (int e^(-2 a y^2) dy)^2 = 1
    dfac = 1.0
    for k in range(2 * l - 1, 0, -2):
        dfac *= k
    mom = dfac / (4.0 * a) ** l * math.sqrt(math.pi / (2.0 * a))
    return 1.0 / math.sqrt(mom * (math.pi / (2.0 * a)))


def gauss_moment(n, p):
    """int_{-inf}^{inf} u^n exp(-p u^2) du."""
    if n % 2:
        return 0.0
    dfac = 1.0
    for k in range(n - 1, 0, -2):
        dfac *= k
    return dfac / (2.0 * p) ** (n // 2) * math.sqrt(math.pi / p)


def overlap_1d(i, j, a, b, A, B):
    """int (x-A)^i (x-B)^j exp(-a (x-A)^2 - b (x-B)^2) dx, by expanding both
    factors about the product centre P."""
    p = a + b
    P = (a * A + b * B) / p
    K = math.exp(-a * b * (A - B) ** 2 / p)
    s = 0.0
    for k1 in range(i + 1):
        c1 = math.comb(i, k1) * (P - A) ** (i - k1)
        for k2 in range(j + 1):
            c2 = math.comb(j, k2) * (P - B) ** (j - k2)
            s += c1 * c2 * gauss_moment(k1 + k2, p)
    return K * s


def pw_1d(i, j, a, b, A, B, G):
    """int (x-A)^i (x-B)^j exp(-a (x-A)^2 - b (x-B)^2) exp(i G x) dx (complex)."""
    p = a + b
    P = (a * A + b * B) / p
    K = math.exp(-a * b * (A - B) ** 2 / p)
    nmax = i + j
    # I_n = int u^n exp(-p u^2 + i G u) du; I_{n+1} = (i G I_n + n I_{n-1}) / (2p)
    I = [0j] * (nmax + 2)
    I[0] = math.sqrt(math.pi / p) * math.exp(-G * G / (4.0 * p)) + 0j
    if nmax >= 1:
        I[1] = (1j * G * I[0]) / (2.0 * p)
    for n in range(1, nmax):
        I[n + 1] = (1j * G * I[n] + n * I[n - 1]) / (2.0 * p)
    s = 0j
    for k1 in range(i + 1):
        c1 = math.comb(i, k1) * (P - A) ** (i - k1)
        for k2 in range(j + 1):
            c2 = math.comb(j, k2) * (P - B) ** (j - k2)
            s += c1 * c2 * I[k1 + k2]
    return K * s * complex(math.cos(G * P), math.sin(G * P))


def _contracted(sys):
    """List of AOs: (atom, comps, [(alpha, coef*N)], l) in AO order."""
    aos = []
    for s in range(sys.nshell):
        l = int(sys.shell_l[s])
        o = int(sys.shell_prim_off[s])
        prims = [(float(sys.exponents[o + k]), float(sys.coeffs[o + k]) * norm(l, float(sys.exponents[o + k])))
                 for k in range(int(sys.shell_nprim[s]))]
        for c in _cart(l):
            aos.append((int(sys.shell_atom[s]), c, prims))
    return aos


def _images(L, reach):
    """Integer image triples covering |T| <= reach; L = the lattice's reach per index
    step along each axis (its lengths for an orthorhombic cell, 1 / |b_d| otherwise)."""
    n = [int(math.ceil(reach / L[d])) + 1 for d in range(3)]
    return [(i, j, k) for i in range(-n[0], n[0] + 1) for j in range(-n[1], n[1] + 1)
            for k in range(-n[2], n[2] + 1)]


def _shell_pair_sum(sys, reach, one_d):
    """Sum over images T and primitive pairs of a shell pair of products of 1-D
    factors one_d(i, j, a, b, A_d, B_d, d) -> matrix [nao, nao]."""
    lat = np.asarray(sys.lattice, dtype=float)
    # images T = n . lat; along axis d, |n_d| <= |T| |b_d| with b_d the reciprocal rows
    step = 1.0 / np.linalg.norm(np.linalg.inv(lat).T, axis=1)
    off = sys.ao_offsets()
    nao = int(off[-1])
    out = np.zeros((nao, nao))
    imgs = np.array(_images(step, reach), dtype=float) @ lat  # Cartesian image vectors
    for sa in range(sys.nshell):
        la = int(sys.shell_l[sa])
        ca = _cart(la)
        A = sys.coords[int(sys.shell_atom[sa])]
        oa = int(sys.shell_prim_off[sa])
        for sb in range(sys.nshell):
            lb = int(sys.shell_l[sb])
            cb = _cart(lb)
            ob = int(sys.shell_prim_off[sb])
            B0 = sys.coords[int(sys.shell_atom[sb])]
            blk = np.zeros((len(ca), len(cb)), dtype=complex)
            for T in imgs:
                B = B0 + T
                if np.sum((A - B) ** 2) > reach * reach:
                    continue
                for ka in range(int(sys.shell_nprim[sa])):
                    a = float(sys.exponents[oa + ka])
                    na = float(sys.coeffs[oa + ka]) * norm(la, a)
                    for kb in range(int(sys.shell_nprim[sb])):
                        b = float(sys.exponents[ob + kb])
                        nb = float(sys.coeffs[ob + kb]) * norm(lb, b)
                        t = [[[one_d(i, j, a, b, A[d], B[d], d) for j in range(lb + 1)]
                              for i in range(la + 1)] for d in range(3)]
                        for m, cm in enumerate(ca):
                            for n, cn in enumerate(cb):
                                blk[m, n] += na * nb * t[0][cm[0]][cn[0]] * t[1][cm[1]][cn[1]] * t[2][cm[2]][cn[2]]
            out[off[sa]:off[sa + 1], off[sb]:off[sb + 1]] = blk.real
    return out


def lattice_overlap(sys, reach=40.0):
    """S_mu,nu = sum_T int phi_mu(r) phi_nu(r - T) dr over all space."""
    return _shell_pair_sum(sys, reach, lambda i, j, a, b, A, B, d: overlap_1d(i, j, a, b, A, B))


def lattice_pw_matrix(sys, waves, reach=40.0):
    """V_mu,nu = sum_T int phi_mu(r) v(r) phi_nu(r - T) dr for
    v(r) = sum_k a_k cos(G_k . r), G_k = 2 pi sum_d n_kd b_d with the reciprocal rows b_d
    (2 pi n_k / L for an orthorhombic cell; one wave at a time: the 3-D integral of
    exp(i G.r) factorises over Cartesian axes, and cos is its real part)."""
    lat = np.asarray(sys.lattice, dtype=float)
    ortho = bool(np.all(lat == np.diag(np.diag(lat))))
    rec = np.linalg.inv(lat).T
    tot = 0.0
    for nk, amp in zip(waves.n, waves.a):
        if ortho:
            G = 2 * np.pi * np.asarray(nk, dtype=float) / np.diag(lat)
        else:
            G = 2 * np.pi * (np.asarray(nk, dtype=float) @ rec)
        tot = tot + amp * _shell_pair_sum(
            sys, reach, lambda i, j, a, b, A, B, d, G=G: pw_1d(i, j, a, b, A, B, G[d]))
    return tot


def periodic_aos(sys, mesh, reach=30.0):
    """Periodised AOs Phi_mu(r) = sum_S phi_mu(r - S) on a grid (Eq. 1 at k = 0),
    shape (nao, N0, N1, N2)."""
    L = np.diag(sys.lattice)
    x = [np.arange(mesh[d]) * (L[d] / mesh[d]) for d in range(3)]
    aos = _contracted(sys)
    out = np.zeros((len(aos),) + tuple(int(m) for m in mesh))
    imgs = _images(L, reach)
    for m, (am, c, prims) in enumerate(aos):
        for img in imgs:
            A = sys.coords[am] + np.array(img) * L
            u = [x[d] - A[d] for d in range(3)]
            if min(np.min(np.abs(u[d])) for d in range(3)) > reach:
                continue
            for (a, ca) in prims:
                f = [u[d] ** c[d] * np.exp(-a * u[d] ** 2) for d in range(3)]
                out[m] += ca * f[0][:, None, None] * f[1][None, :, None] * f[2][None, None, :]
    return out


def brute_rho(sys, mesh, D=None, reach=30.0):
    """rho(r) = sum_ST sum_mu,nu D phi_mu(r-S) phi_nu(r-T) (Eq. rho), untruncated."""
    D = sys.D if D is None else D
    Phi = periodic_aos(sys, mesh, reach)
    return np.einsum("mn,mxyz,nxyz->xyz", D, Phi, Phi, optimize=True)


def gaussian_charge_hartree(alpha_charge, L, gcut=None):
    """E_H of a unit Gaussian charge (exponent alpha') in a cubic cell with a
    neutralising background: (2 pi / Omega) sum_{0<|G|<gcut} exp(-G^2/(2 a'))/G^2."""
    omega = L ** 3
    nmax = int(math.ceil((gcut if gcut else 12 * math.sqrt(alpha_charge)) * L / (2 * math.pi))) + 1
    r = np.arange(-nmax, nmax + 1)
    g = 2 * np.pi * r / L
    G2 = g[:, None, None] ** 2 + g[None, :, None] ** 2 + g[None, None, :] ** 2
    mask = G2 > 0
    if gcut:
        mask &= G2 < gcut * gcut
    return 2 * np.pi / omega * float(np.sum(np.exp(-G2[mask] / (2 * alpha_charge)) / G2[mask]))


def madelung_cubic_background(L, eta=None, nreal=6, nrec=12):
    """Ewald energy per unit point charge on a simple cubic lattice of edge L with
    a neutralising background (computed, not a remembered constant)."""
    from scipy.special import erfc
    eta = eta or 2.5 / L
    omega = L ** 3
    r = np.arange(-nreal, nreal + 1)
    R = L * np.sqrt(r[:, None, None] ** 2 + r[None, :, None] ** 2 + r[None, None, :] ** 2)
    Rm = R[R > 0]
    real = float(np.sum(erfc(eta * Rm) / Rm))
    k = np.arange(-nrec, nrec + 1)
    g = 2 * np.pi * k / L
    G2 = g[:, None, None] ** 2 + g[None, :, None] ** 2 + g[None, None, :] ** 2
    G2 = G2[G2 > 0]
    rec = 4 * np.pi / omega * float(np.sum(np.exp(-G2 / (4 * eta * eta)) / G2))
    return 0.5 * (real + rec - 2 * eta / math.sqrt(math.pi) - math.pi / (eta * eta * omega))


def dov_1d(i, j, a, b, A, B):
    """int d/dx[(x-A)^i e^(-a (x-A)^2)] d/dx[(x-B)^j e^(-b (x-B)^2)] dx: each derivative
    is i (x-A)^(i-1) - 2a (x-A)^(i+1) (times the exponential), expanded into overlaps."""
    s = 4.0 * a * b * overlap_1d(i + 1, j + 1, a, b, A, B)
    if i > 0:
        s -= 2.0 * b * i * overlap_1d(i - 1, j + 1, a, b, A, B)
    if j > 0:
        s -= 2.0 * a * j * overlap_1d(i + 1, j - 1, a, b, A, B)
    if i > 0 and j > 0:
        s += i * j * overlap_1d(i - 1, j - 1, a, b, A, B)
    return s


def dpw_1d(i, j, a, b, A, B, G):
    """The same with a plane wave exp(i G x) (complex)."""
    s = 4.0 * a * b * pw_1d(i + 1, j + 1, a, b, A, B, G)
    if i > 0:
        s -= 2.0 * b * i * pw_1d(i - 1, j + 1, a, b, A, B, G)
    if j > 0:
        s -= 2.0 * a * j * pw_1d(i + 1, j - 1, a, b, A, B, G)
    if i > 0 and j > 0:
        s += i * j * pw_1d(i - 1, j - 1, a, b, A, B, G)
    return s


def lattice_grad_overlap(sys, reach=40.0):
    """T_mu,nu = sum_T int grad phi_mu(r) . grad phi_nu(r - T) dr over all space (the
    kinetic matrix times 2), one dimension differentiated at a time."""
    out = 0.0
    for dd in range(3):
        out = out + _shell_pair_sum(
            sys, reach, lambda i, j, a, b, A, B, d, dd=dd:
            dov_1d(i, j, a, b, A, B) if d == dd else overlap_1d(i, j, a, b, A, B))
    return out


def lattice_grad_pw_matrix(sys, waves, reach=40.0):
    """T_mu,nu[v] = sum_T int grad phi_mu(r) . grad phi_nu(r - T) v(r) dr for
    v(r) = sum_k a_k cos(G_k . r) (as lattice_pw_matrix, one dimension differentiated at
    a time)."""
    lat = np.asarray(sys.lattice, dtype=float)
    ortho = bool(np.all(lat == np.diag(np.diag(lat))))
    rec = np.linalg.inv(lat).T
    tot = 0.0
    for nk, amp in zip(waves.n, waves.a):
        if ortho:
            G = 2 * np.pi * np.asarray(nk, dtype=float) / np.diag(lat)
        else:
            G = 2 * np.pi * (np.asarray(nk, dtype=float) @ rec)
        for dd in range(3):
            tot = tot + amp * _shell_pair_sum(
                sys, reach, lambda i, j, a, b, A, B, d, G=G, dd=dd:
                dpw_1d(i, j, a, b, A, B, G[d]) if d == dd else pw_1d(i, j, a, b, A, B, G[d]))
    return tot
