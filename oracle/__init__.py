"""Plain FP64 CPU oracle for the multigrid GPW Fock build (arXiv 2603.24881).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s ``cpu_baseline``/reference leg may import this package.  It shares
no code with the CUDA path (``paper_2603_24881_gb300``) and never imports it.

Layout
------
* ``gpw_oracle.c`` (plain C, built by :func:`build`): screening, collocation,
  integration and the gradient contraction, point by point.
* this module: primitive normalisation, multigrid meshes and level cutoffs,
  the spectral steps (Fourier interpolation between levels, Poisson, LDA and
  PBE exchange) written with numpy's FFT, and the assembly of V and the gradient.

Readings of the paper that this oracle fixes (the CUDA path follows the same
ones) are listed in the docstring of each function.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = None
_LOCK = threading.Lock()


def build(force: bool = False) -> str:
    """Compile gpw_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP, no FMA
    contraction) and return its path."""
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_HERE, "gpw_oracle.c")
    out = os.path.join(_BUILD, "liboracle.so")
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            L = ctypes.CDLL(build())
            L.orc_rcut.restype = ctypes.c_double
            L.orc_rcut.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double]
            L.orc_pairs.restype = ctypes.c_long
            L.orc_pairs_lat.restype = ctypes.c_long
            L.orc_volume.restype = ctypes.c_double
            L.orc_volume.argtypes = [ctypes.c_void_p]
            L.orc_collocate.restype = None
            L.orc_integrate.restype = None
            L.orc_rho_points.restype = None
            L.orc_collocate_tau.restype = None
            L.orc_integrate_tau.restype = None
            _LIB = L
    return _LIB


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------- basis ----

def cart_components(l: int):
    """Cartesian exponents of a shell, x^l first (d: xx, xy, xz, yy, yz, zz)."""
    out = []
    for ix in range(l, -1, -1):
        for iy in range(l - ix, -1, -1):
            out.append((ix, iy, l - ix - iy))
    return out


def _dfact(n: int) -> float:
    r = 1.0
    while n > 1:
        r *= n
        n -= 2
    return r


def prim_norm(l: int, alpha: float) -> float:
    """N_l(alpha) = [(2 alpha/pi)^(3/2) (4 alpha)^l / (2l-1)!!]^(1/2): unit
    self-overlap of the x^l component of a primitive (a reading; the paper does
    not state its normalisation)."""
    ipow = 1.0
    for _ in range(l):
        ipow *= 4.0 * alpha
    return math.sqrt(math.pow(2.0 * alpha / math.pi, 1.5) * ipow / _dfact(2 * l - 1))


def primitives(sys):
    """Flatten the shells into primitives (global order = shell order, then
    primitive order).  Returns dict of arrays: centre, l, alpha, cn = c*N,
    ao (first AO of the shell), atom, shell."""
    ao_off = sys.ao_offsets()
    cen, ls, al, cn, ao, atom, shell = [], [], [], [], [], [], []
    for s in range(sys.nshell):
        l = int(sys.shell_l[s])
        a = int(sys.shell_atom[s])
        o = int(sys.shell_prim_off[s])
        for k in range(int(sys.shell_nprim[s])):
            alpha = float(sys.exponents[o + k])
            cen.append(sys.coords[a])
            ls.append(l)
            al.append(alpha)
            cn.append(float(sys.coeffs[o + k]) * prim_norm(l, alpha))
            ao.append(int(ao_off[s]))
            atom.append(a)
            shell.append(s)
    return dict(center=np.ascontiguousarray(np.array(cen, dtype=np.float64).reshape(-1, 3)),
                l=np.array(ls, dtype=np.int32), alpha=np.array(al, dtype=np.float64),
                cn=np.array(cn, dtype=np.float64), ao=np.array(ao, dtype=np.int64),
                atom=np.array(atom, dtype=np.int32), shell=np.array(shell, dtype=np.int32))


# ---------------------------------------------------------------- grids ----

def _smooth7_even(n: int) -> int:
    m = max(2, n)
    while True:
        if m % 2 == 0:
            r = m
            for f in (2, 3, 5, 7):
                while r % f == 0:
                    r //= f
            if r == 1:
                return m
        m += 1


def is_orthorhombic(lattice) -> bool:
    lat = np.asarray(lattice, dtype=np.float64)
    return bool(np.all(lat == np.diag(np.diag(lat))))


def lattice_lengths(lattice):
    """|R_d| of the lattice rows (the diagonal of an orthorhombic lattice, exactly),
    sqrt(x^2 + y^2 + z^2) summed in that order."""
    lat = np.asarray(lattice, dtype=np.float64)
    if is_orthorhombic(lat):
        return np.diag(lat).astype(np.float64)
    return np.array([math.sqrt(float(r[0]) * float(r[0]) + float(r[1]) * float(r[1]) +
                               float(r[2]) * float(r[2])) for r in lat])


def reciprocal(lattice):
    """Rows b_d with b_d . R_e = delta_de (no 2 pi): b_0 = R_1 x R_2 / V, b_1 = R_2 x R_0 / V,
    b_2 = R_0 x R_1 / V, V = R_0 . (R_1 x R_2), each operation in double in that order, so
    that the fractional coordinate b_d . r of a screening decision is reproducible."""
    R = [[float(x) for x in row] for row in np.asarray(lattice, dtype=np.float64)]
    cr = []
    for d in range(3):
        a, b = R[(d + 1) % 3], R[(d + 2) % 3]
        cr.append([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]])
    V = R[0][0] * cr[0][0] + R[0][1] * cr[0][1] + R[0][2] * cr[0][2]
    return np.ascontiguousarray(np.array([[c / V for c in row] for row in cr]))


def level_grids(sys):
    """Level meshes and cutoffs (Sec. II multigrid; constants are readings).

    With explicit meshes: E_k = G_k^2 / 2 with G_k = min_d 2 pi floor((N_kd - 1)/2) / |R_d|.
    Otherwise E_k = E_cut / ratio^k and N_kd = smallest even 7-smooth integer
    >= 2 ceil(G_k |R_d| / 2 pi) + 1, G_k = sqrt(2 E_k): every plane wave with |G| < G_k,
    G = 2 pi sum_d m_d b_d, has |m_d| = |G . R_d| / 2 pi <= (N_kd - 1) / 2.  For an
    orthorhombic cell |R_d| = L_d.  Returns (meshes (K,3), E (K,), G (K,)).
    """
    L = lattice_lengths(sys.lattice)
    K = int(sys.nlevels)
    meshes = np.zeros((K, 3), dtype=np.int32)
    E = np.zeros(K)
    if sys.meshes is not None:
        meshes[:] = np.asarray(sys.meshes, dtype=np.int32)
        for k in range(K):
            G = min(2.0 * math.pi * ((int(meshes[k, d]) - 1) // 2) / L[d] for d in range(3))
            E[k] = 0.5 * G * G
    else:
        for k in range(K):
            div = 1.0
            for _ in range(k):
                div *= sys.level_ratio
            E[k] = sys.cutoff_ha / div
            G = math.sqrt(2.0 * E[k])
            for d in range(3):
                meshes[k, d] = _smooth7_even(2 * math.ceil(G * L[d] / (2.0 * math.pi)) + 1)
    G = np.sqrt(2.0 * E)
    return meshes, E, G


def gvectors(mesh, lattice):
    """|G|^2 on the full FFT grid of `mesh` (numpy fftfreq order).  `lattice` is the
    3 x 3 lattice (rows R_d) or, for an orthorhombic cell, its three lengths:
    G = 2 pi sum_d m_d b_d with the reciprocal rows b_d."""
    lat = np.asarray(lattice, dtype=np.float64)
    if lat.ndim == 1 or is_orthorhombic(lat):
        L = lat if lat.ndim == 1 else np.diag(lat)
        g = [2.0 * np.pi * np.fft.fftfreq(int(mesh[d]), d=1.0 / int(mesh[d])) / L[d] for d in range(3)]
        return (g[0][:, None, None] ** 2 + g[1][None, :, None] ** 2 + g[2][None, None, :] ** 2)
    B = reciprocal(lat)
    m = [np.fft.fftfreq(int(mesh[d]), d=1.0 / int(mesh[d])) for d in range(3)]
    G = [2.0 * np.pi * (m[0][:, None, None] * B[0, c] + m[1][None, :, None] * B[1, c] +
                        m[2][None, None, :] * B[2, c]) for c in range(3)]
    return G[0] ** 2 + G[1] ** 2 + G[2] ** 2


def _freq_index(mesh):
    return [np.fft.fftfreq(int(m), d=1.0 / int(m)).astype(np.int64) for m in mesh]


# PBE exchange (Perdew, Burke, Ernzerhof 1996): enhancement factor
# F_x(s) = 1 + kappa - kappa / (1 + mu s^2 / kappa), kappa = 0.804 (Lieb-Oxford bound
# F_x <= 1.804), mu = beta pi^2 / 3 with beta = 0.06672455060314922.
PBE_KAPPA = 0.804
PBE_MU = 0.06672455060314922 * math.pi ** 2 / 3.0
# below this density the exchange energy density and potential are set to zero
GGA_RHO_MIN = 1e-12


def pbe_x_point(rho, sigma):
    """Spin-unpolarised PBE exchange at points: rho (>= 0 used), sigma = |grad rho|^2.
    Returns (e, de/drho, de/dsigma) with e the energy per volume,
    e = e_x^LDA(rho) F_x(s), e_x^LDA = -(3/4)(3/pi)^(1/3) rho^(4/3),
    s^2 = sigma / (4 k_F^2 rho^2), k_F = (3 pi^2 rho)^(1/3)."""
    rho = np.asarray(rho, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    ok = rho > GGA_RHO_MIN
    r = np.where(ok, rho, 1.0)
    cx = (3.0 / math.pi) ** (1.0 / 3.0)
    r13 = np.cbrt(r)
    elda = -0.75 * cx * r * r13            # e_x^LDA
    delda = -cx * r13                      # d e_x^LDA / d rho
    kf2 = (3.0 * math.pi ** 2 * r) ** (2.0 / 3.0)
    ds2_dsigma = 1.0 / (4.0 * kf2 * r * r)
    s2 = sigma * ds2_dsigma
    den = 1.0 + PBE_MU * s2 / PBE_KAPPA
    F = 1.0 + PBE_KAPPA - PBE_KAPPA / den
    dF = PBE_MU / (den * den)              # dF / d(s^2)
    e = elda * F
    dedr = delda * F + elda * dF * (-8.0 / 3.0) * s2 / r
    deds = elda * dF * ds2_dsigma
    z = np.zeros_like(e)
    return np.where(ok, e, z), np.where(ok, dedr, z), np.where(ok, deds, z)


# ---------------------------------------------------------------- plan -----

class Plan:
    """Oracle-side screening of one system (Sec. III A and Eq. cut).

    Pairs are stored as arrays: ab (npairs,2) primitive indices with a <= b,
    img (npairs,3) image integers n of T = n . L, lev, lo/hi (npairs,3) integer
    box on the level mesh, R (extent).
    """

    def __init__(self, sys, prims=None):
        self.sys = sys
        self.lat = np.ascontiguousarray(np.asarray(sys.lattice, dtype=np.float64).reshape(3, 3))
        self.ortho = is_orthorhombic(self.lat)
        # lattice lengths along the rows of an orthorhombic cell
        self.L = np.ascontiguousarray(np.diag(self.lat).astype(np.float64))
        self.omega = float(np.prod(self.L)) if self.ortho else float(_lib().orc_volume(_p(self.lat)))
        self.prims = prims or primitives(sys)
        self.meshes, self.E, self.G = level_grids(sys)
        self.nlev = len(self.E)
        lib = _lib()
        pr = self.prims
        self.rcut = np.array([lib.orc_rcut(float(abs(c)), int(l), float(a), float(sys.tau))
                              for c, l, a in zip(pr["cn"], pr["l"], pr["alpha"])])
        self._enumerate()
        self.grid_off = np.zeros(self.nlev + 1, dtype=np.int64)
        for k in range(self.nlev):
            self.grid_off[k + 1] = self.grid_off[k] + int(np.prod(self.meshes[k]))

    def _enumerate(self):
        lib = _lib()
        pr = self.prims
        cap = 1 << 16
        while True:
            ab = np.zeros((cap, 2), np.int32)
            img = np.zeros((cap, 3), np.int32)
            lev = np.zeros(cap, np.int32)
            lo = np.zeros((cap, 3), np.int32)
            hi = np.zeros((cap, 3), np.int32)
            R = np.zeros(cap)
            if self.ortho:
                n = lib.orc_pairs(ctypes.c_int(len(pr["l"])), _p(pr["center"]), _p(pr["l"]),
                                  _p(pr["alpha"]), _p(pr["cn"]), _p(self.rcut), _p(self.L),
                                  ctypes.c_int(self.nlev), _p(self.meshes), _p(self.E),
                                  ctypes.c_double(self.sys.rel_cutoff),
                                  ctypes.c_double(self.sys.tau), ctypes.c_long(cap), _p(ab),
                                  _p(img), _p(lev), _p(lo), _p(hi), _p(R))
            else:
                rec = reciprocal(self.lat)
                n = lib.orc_pairs_lat(ctypes.c_int(len(pr["l"])), _p(pr["center"]), _p(pr["l"]),
                                      _p(pr["alpha"]), _p(pr["cn"]), _p(self.rcut), _p(self.lat),
                                      _p(rec), ctypes.c_int(self.nlev), _p(self.meshes),
                                      _p(self.E), ctypes.c_double(self.sys.rel_cutoff),
                                      ctypes.c_double(self.sys.tau), ctypes.c_long(cap), _p(ab),
                                      _p(img), _p(lev), _p(lo), _p(hi), _p(R))
            if n <= cap:
                break
            cap = int(n)
        self.ab, self.img, self.lev = ab[:n].copy(), img[:n].copy(), lev[:n].copy()
        self.lo, self.hi, self.R = lo[:n].copy(), hi[:n].copy(), R[:n].copy()

    @property
    def npairs(self) -> int:
        return int(self.ab.shape[0])

    def pair_points(self) -> int:
        return int(np.prod(self.hi - self.lo + 1, axis=1).sum())

    def pair_table(self):
        """Integer pair table sorted lexicographically: (a, b, n0, n1, n2, level,
        lo0, lo1, lo2, hi0, hi1, hi2)."""
        t = np.concatenate([self.ab, self.img, self.lev[:, None], self.lo, self.hi], axis=1)
        order = np.lexsort(t[:, ::-1].T)
        return t[order].astype(np.int64)

    def _args(self):
        """Pair arrays for the C oracle, with the lattice rows."""
        pr = self.prims
        return (_p(self.ab), _p(self.img), _p(self.lev), _p(self.lo), _p(self.hi),
                _p(pr["center"]), _p(pr["l"]), _p(pr["alpha"]), _p(pr["cn"]), _p(pr["ao"]),
                _p(self.lat), _p(self.meshes))

    def _ortho_only(self, what):
        if not self.ortho:
            raise ValueError(f"{what}: orthorhombic cells only")

    # -------------------------------------------------- eval_rho (Alg. 1) --
    def rho_levels(self, D, mode: str = "separable", nthreads: int = 0, pairs=None):
        """Raw level densities rho_k (Eq. rho_wrap), each pair on its own level.

        ``pairs``: optional index array restricting the sum to a subset.
        """
        lib = _lib()
        D = np.ascontiguousarray(D, dtype=np.float64)
        total = int(self.grid_off[-1])
        grids = np.zeros(total)
        sub = self if pairs is None else self.subset(pairs)
        if not self.ortho:
            mode = "plain"  # the separable factorisation holds for orthorhombic cells only
        lib.orc_collocate(ctypes.c_int(0 if mode == "plain" else 1), ctypes.c_long(sub.npairs),
                          *sub._args(), _p(self.grid_off), ctypes.c_long(total), _p(D),
                          ctypes.c_long(D.shape[0]), _p(grids), ctypes.c_int(nthreads))
        return [grids[self.grid_off[k]:self.grid_off[k + 1]].reshape(tuple(self.meshes[k]))
                for k in range(self.nlev)]

    # -------------------------------------------------- meta-GGA (Sec. II) --
    def tau_levels(self, D, nthreads: int = 0):
        """Kinetic energy density of each level, tau_k = (1/2) sum D_mu,nu grad phi_mu .
        grad phi_nu over the pairs of that level (point by point, like Eq. rho_wrap)."""
        lib = _lib()
        D = np.ascontiguousarray(D, dtype=np.float64)
        total = int(self.grid_off[-1])
        grids = np.zeros(total)
        lib.orc_collocate_tau(ctypes.c_long(self.npairs), *self._args(), _p(self.grid_off),
                              ctypes.c_long(total), _p(D), ctypes.c_long(D.shape[0]), _p(grids),
                              ctypes.c_int(nthreads))
        return [grids[self.grid_off[k]:self.grid_off[k + 1]].reshape(tuple(self.meshes[k]))
                for k in range(self.nlev)]

    def _tau_blocks(self, v_levels, grad_D=None, nthreads: int = 0):
        lib = _lib()
        v = np.ascontiguousarray(np.concatenate([np.ascontiguousarray(x).ravel() for x in v_levels]))
        pr = self.prims
        na = np.array([(l + 1) * (l + 2) // 2 for l in pr["l"]], dtype=np.int64)
        if grad_D is None:
            sizes = na[self.ab[:, 0]] * na[self.ab[:, 1]]
            xoff = np.zeros(self.npairs + 1, dtype=np.int64)
            xoff[1:] = np.cumsum(sizes)
            xout = np.zeros(int(xoff[-1]))
            gd, nao = None, 0
        else:
            xoff = np.zeros(1, dtype=np.int64)
            xout = np.zeros(6 * self.npairs)
            gd = np.ascontiguousarray(grad_D, dtype=np.float64)
            nao = gd.shape[0]
        lib.orc_integrate_tau(ctypes.c_long(self.npairs), None, ctypes.c_long(self.npairs),
                              *self._args(), _p(self.grid_off), _p(v),
                              None if gd is None else _p(gd), ctypes.c_long(nao), _p(xoff),
                              _p(xout), ctypes.c_int(nthreads))
        return xoff, xout, na

    def mat_tau_levels(self, v_levels, nthreads: int = 0):
        """Fock term of a kinetic-energy-density potential (Eq. J_metaGGA):
        V_mu,nu = sum over pairs (Omega/N_k) sum_r v_k (1/2) grad phi_mu . grad phi_nu,
        mirror blocks as for eval_mat."""
        nao = self.sys.nao
        xoff, xout, na = self._tau_blocks(v_levels, nthreads=nthreads)
        V = np.zeros((nao, nao))
        ao = self.prims["ao"]
        for p in range(self.npairs):
            a, b = int(self.ab[p, 0]), int(self.ab[p, 1])
            X = xout[xoff[p]:xoff[p + 1]].reshape(na[a], na[b])
            ia, ib = int(ao[a]), int(ao[b])
            V[ia:ia + na[a], ib:ib + na[b]] += X
            if a < b:
                V[ib:ib + na[b], ia:ia + na[a]] += X.T
        return V

    def grad_tau_levels(self, D, v_levels, nthreads: int = 0):
        """Nuclear gradient of <v, tau(D)> at fixed level potentials v (frozen boxes)."""
        _, xout, _ = self._tau_blocks(v_levels, grad_D=D, nthreads=nthreads)
        g = np.zeros((self.sys.natm, 3))
        atom = self.prims["atom"]
        for p in range(self.npairs):
            a, b = int(self.ab[p, 0]), int(self.ab[p, 1])
            g[atom[a]] += xout[6 * p:6 * p + 3]
            g[atom[b]] += xout[6 * p + 3:6 * p + 6]
        return g

    def subset(self, idx):
        import copy
        out = copy.copy(self)
        idx = np.asarray(idx, dtype=np.int64)
        for name in ("ab", "img", "lev", "lo", "hi", "R"):
            setattr(out, name, np.ascontiguousarray(getattr(self, name)[idx]))
        return out

    def rho_points(self, D, level: int, pts, nthreads: int = 0):
        """rho_level at integer grid points pts (n,3), by direct summation."""
        lib = _lib()
        D = np.ascontiguousarray(D, dtype=np.float64)
        pts = np.ascontiguousarray(pts, dtype=np.int32)
        out = np.zeros(len(pts))
        lib.orc_rho_points(ctypes.c_long(self.npairs), *self._args(), ctypes.c_int(level),
                           ctypes.c_long(len(pts)), _p(pts), _p(D), ctypes.c_long(D.shape[0]),
                           _p(out), ctypes.c_int(nthreads))
        return out

    # -------------------------------------------------- spectral steps -----
    def combine(self, rho_levels):
        """Fourier interpolation onto the finest grid (Sec. II, multigrid):
        rho~(G) = sum_k rho~_k(G) for |G| < G_k, each level's unnormalised DFT
        scaled by N_fine/N_k (a reading: it makes interpolation and restriction
        exact adjoints).  Returns rho on the finest mesh (real)."""
        fine = tuple(int(m) for m in self.meshes[0])
        Nf = float(np.prod(fine))
        spec = np.zeros(fine, dtype=np.complex128)
        for k in range(self.nlev):
            mesh = self.meshes[k]
            Nk = float(np.prod(mesh))
            rk = np.fft.fftn(rho_levels[k])
            g2 = gvectors(mesh, self.lat)
            mask = g2 < self.G[k] ** 2
            f = _freq_index(mesh)
            idx = np.nonzero(mask)
            fi = tuple(np.mod(f[d][idx[d]], fine[d]) for d in range(3))
            np.add.at(spec, fi, (Nf / Nk) * rk[idx])
        self._last_spec = spec
        return np.real(np.fft.ifftn(spec))

    def restrict(self, v_fine):
        """Potential on each level (Sec. II, per-level back-transform): keep
        |G| < G_k of the fine spectrum, scale by N_k/N_fine, inverse FFT."""
        fine = tuple(int(m) for m in self.meshes[0])
        Nf = float(np.prod(fine))
        vs = np.fft.fftn(v_fine)
        out = []
        for k in range(self.nlev):
            mesh = tuple(int(m) for m in self.meshes[k])
            Nk = float(np.prod(mesh))
            g2 = gvectors(mesh, self.lat)
            mask = g2 < self.G[k] ** 2
            f = _freq_index(mesh)
            idx = np.nonzero(mask)
            fi = tuple(np.mod(f[d][idx[d]], fine[d]) for d in range(3))
            sk = np.zeros(mesh, dtype=np.complex128)
            sk[idx] = (Nk / Nf) * vs[fi]
            out.append(np.real(np.fft.ifftn(sk)))
        return out

    def poisson(self, rho_fine):
        """Hartree potential, Eqs. (vH) and (vHG): v~(G) = 4 pi rho~(G)/|G|^2 for
        G != 0, 0 at G = 0.  E_H = (1/2)(Omega/N) sum_r rho v_H."""
        fine = self.meshes[0]
        g2 = gvectors(fine, self.lat)
        rs = np.fft.fftn(rho_fine)
        with np.errstate(divide="ignore", invalid="ignore"):
            k = np.where(g2 > 0, 4.0 * np.pi / np.where(g2 > 0, g2, 1.0), 0.0)
        vH = np.real(np.fft.ifftn(rs * k))
        omega = self.omega
        EH = 0.5 * omega / float(np.prod(fine)) * float(np.sum(rho_fine * vH))
        return vH, EH

    def lda_x(self, rho_fine):
        """Spin-unpolarised Slater exchange (Sec. II, LDA): with rho+ = max(rho, 0),
        e_x = -(3/4)(3/pi)^(1/3) rho+^(4/3), v_x = -(3/pi)^(1/3) rho+^(1/3),
        E_x = (Omega/N) sum_r e_x."""
        rp = np.maximum(rho_fine, 0.0)
        cx = (3.0 / np.pi) ** (1.0 / 3.0)
        vx = -cx * np.cbrt(rp)
        ex = -0.75 * cx * rp * np.cbrt(rp)
        omega = self.omega
        return vx, omega / float(np.prod(self.meshes[0])) * float(np.sum(ex))

    def _deriv(self, spec, d):
        """Fourier derivative along Cartesian axis d of a full (numpy-order) spectrum:
        i G_d spec, with the Nyquist plane of an even axis set to zero (a reading: the
        derivative of a real field stays real)."""
        mesh = tuple(int(m) for m in self.meshes[0])
        if self.ortho:
            f = np.fft.fftfreq(mesh[d], d=1.0 / mesh[d])
            g = 2.0 * np.pi * f / self.L[d]
            if mesh[d] % 2 == 0:
                g[mesh[d] // 2] = 0.0
            shape = [1, 1, 1]
            shape[d] = mesh[d]
            return spec * (1j * g).reshape(shape)
        # non-orthogonal cell: Cartesian component d of G = 2 pi sum_e m_e b_e, with the
        # Nyquist frequency of an even mesh axis taken as zero (as above, per axis)
        B = reciprocal(self.lat)
        m = []
        for e in range(3):
            f = np.fft.fftfreq(mesh[e], d=1.0 / mesh[e])
            if mesh[e] % 2 == 0:
                f[mesh[e] // 2] = 0.0
            m.append(f)
        g = 2.0 * np.pi * (m[0][:, None, None] * B[0, d] + m[1][None, :, None] * B[1, d] +
                           m[2][None, None, :] * B[2, d])
        return spec * (1j * g)

    def pbe_x(self, rho_fine):
        """GGA exchange (Sec. II, GGA; PBE exchange): the density gradient from the
        Fourier derivative of rho (grad rho = F^-1(i G rho~)), e and its derivatives at
        every point (pbe_x_point with rho+ = max(rho, 0)), and the potential
        v = de/drho - div(2 de/dsigma grad rho), the divergence again a Fourier
        derivative (the integration by parts that folds the GGA term into the local
        potential).  E_x = (Omega/N) sum_r e.  Returns (v_x, E_x)."""
        rs = np.fft.fftn(rho_fine)
        grad = [np.real(np.fft.ifftn(self._deriv(rs, d))) for d in range(3)]
        sigma = grad[0] ** 2 + grad[1] ** 2 + grad[2] ** 2
        e, dedr, deds = pbe_x_point(np.maximum(rho_fine, 0.0), sigma)
        div = np.zeros_like(rho_fine)
        for d in range(3):
            div += np.real(np.fft.ifftn(self._deriv(np.fft.fftn(2.0 * deds * grad[d]), d)))
        omega = self.omega
        return dedr - div, omega / float(np.prod(self.meshes[0])) * float(np.sum(e))

    def xc(self, rho_fine, xc: str = "lda_x"):
        """Exchange potential and energy of the named functional ("lda_x", "pbe_x")."""
        if xc == "lda_x":
            return self.lda_x(rho_fine)
        if xc == "pbe_x":
            return self.pbe_x(rho_fine)
        raise ValueError(f"unknown functional {xc!r}")

    # -------------------------------------------------- eval_mat (Alg. 2) --
    def _pair_blocks(self, v_levels, grad_D=None, sel=None, nthreads: int = 0):
        lib = _lib()
        v = np.ascontiguousarray(np.concatenate([np.ascontiguousarray(x).ravel() for x in v_levels]))
        pr = self.prims
        na = np.array([(l + 1) * (l + 2) // 2 for l in pr["l"]], dtype=np.int64)
        nsel = self.npairs if sel is None else len(sel)
        selp = None if sel is None else np.ascontiguousarray(sel, dtype=np.int64)
        if grad_D is None:
            sizes = na[self.ab[:, 0]] * na[self.ab[:, 1]]
            xoff = np.zeros(self.npairs + 1, dtype=np.int64)
            xoff[1:] = np.cumsum(sizes)
            xout = np.zeros(int(xoff[-1]))
            gd = None
            nao = 0
        else:
            xoff = np.zeros(1, dtype=np.int64)
            xout = np.zeros(6 * nsel)
            gd = np.ascontiguousarray(grad_D, dtype=np.float64)
            nao = gd.shape[0]
        lib.orc_integrate(ctypes.c_long(self.npairs),
                          None if selp is None else _p(selp), ctypes.c_long(nsel),
                          *self._args(), _p(self.grid_off), _p(v),
                          None if gd is None else _p(gd), ctypes.c_long(nao), _p(xoff),
                          _p(xout), ctypes.c_int(nthreads))
        return xoff, xout, na

    def mat_levels(self, v_levels, nthreads: int = 0):
        """V_mu,nu = sum over pairs (Eq. J_wrap, weight Omega/N_k); a pair with
        a < b also fills its mirror block (the (b, a, -T) term).  Sum in pair
        order, so the result is deterministic."""
        nao = self.sys.nao
        xoff, xout, na = self._pair_blocks(v_levels, nthreads=nthreads)
        V = np.zeros((nao, nao))
        ao = self.prims["ao"]
        for p in range(self.npairs):
            a, b = int(self.ab[p, 0]), int(self.ab[p, 1])
            X = xout[xoff[p]:xoff[p + 1]].reshape(na[a], na[b])
            ia, ib = int(ao[a]), int(ao[b])
            V[ia:ia + na[a], ib:ib + na[b]] += X
            if a < b:
                V[ib:ib + na[b], ia:ia + na[a]] += X.T
        return V

    def mat_block(self, v_levels, sa: int, sb: int):
        """One contracted block V[shell sa, shell sb] (sampled check for big cells)."""
        sh = self.prims["shell"]
        sel = np.nonzero(((sh[self.ab[:, 0]] == sa) & (sh[self.ab[:, 1]] == sb)) |
                         ((sh[self.ab[:, 0]] == sb) & (sh[self.ab[:, 1]] == sa)))[0]
        xoff, xout, na = self._pair_blocks(v_levels, sel=sel if len(sel) else np.zeros(0, np.int64))
        ao_off = self.sys.ao_offsets()
        la, lb = int(self.sys.shell_l[sa]), int(self.sys.shell_l[sb])
        nA, nB = (la + 1) * (la + 2) // 2, (lb + 1) * (lb + 2) // 2
        out = np.zeros((nA, nB))
        for p in sel:
            a, b = int(self.ab[p, 0]), int(self.ab[p, 1])
            X = xout[xoff[p]:xoff[p + 1]].reshape(na[a], na[b])
            if sh[a] == sa and sh[b] == sb:
                out += X
            if a < b and sh[b] == sa and sh[a] == sb:
                out += X.T
        return out

    def grad_levels(self, D, v_levels, nthreads: int = 0, sel=None):
        """dE/dR_atom = sum over pairs of the Algorithm-3 contraction of D, v and
        the centre derivatives of the two primitives (frozen boxes)."""
        _, xout, _ = self._pair_blocks(v_levels, grad_D=D, sel=sel, nthreads=nthreads)
        g = np.zeros((self.sys.natm, 3))
        atom = self.prims["atom"]
        pairs = range(self.npairs) if sel is None else sel
        for s, p in enumerate(pairs):
            a, b = int(self.ab[p, 0]), int(self.ab[p, 1])
            g[atom[a]] += xout[6 * s:6 * s + 3]
            g[atom[b]] += xout[6 * s + 3:6 * s + 6]
        return g

    # -------------------------------------------------- whole build ---------
    def fock(self, D, nthreads: int = 0, xc: str = "lda_x"):
        """One Fock build: rho -> combine -> Poisson + exchange (LDA or PBE) -> restrict
        -> V.  Returns dict(V, EH, Ex, rho_fine, v_fine, v_levels)."""
        rl = self.rho_levels(D, nthreads=nthreads)
        rho = self.combine(rl)
        vH, EH = self.poisson(rho)
        vx, Ex = self.xc(rho, xc)
        v = vH + vx
        vl = self.restrict(v)
        V = self.mat_levels(vl, nthreads=nthreads)
        return dict(V=V, EH=EH, Ex=Ex, rho_fine=rho, v_fine=v, v_levels=vl, rho_levels=rl)

    def energy(self, D, nthreads: int = 0, xc: str = "lda_x") -> float:
        rho = self.combine(self.rho_levels(D, nthreads=nthreads))
        return self.poisson(rho)[1] + self.xc(rho, xc)[1]

    def with_coords(self, coords):
        """Frozen plan at new atom positions: same pairs, images, levels and boxes;
        only the Gaussian centres move (the FD reading of the gradient)."""
        import copy
        out = copy.copy(self)
        out.sys = self.sys.with_coords(coords)
        pr = dict(self.prims)
        pr["center"] = np.ascontiguousarray(np.asarray(coords, dtype=np.float64)[pr["atom"]])
        out.prims = pr
        return out


def fock(sys, D=None, nthreads: int = 0):
    plan = Plan(sys)
    return plan.fock(sys.D if D is None else D, nthreads=nthreads)
