"""Small seeded systems for the oracle pins and parity tests (inputs only)."""
from __future__ import annotations

import numpy as np

import workloads
from workloads import System, ncart, _plane_waves, _finish_shells, _log_uniform


def resolved(seed: int = 5, L: float = 6.0, cutoff: float = 150.0, nlevels: int = 3,
             tau: float = 1e-14, amin: float = 0.25, amax: float = 1.5,
             shells=((0, 2), (1, 1), (2, 1), (3, 1)), natm: int = 2) -> System:
    """Cubic cell whose pair exponents are all resolved by their level grid
    (alpha_p h^2 < 0.1), so grid sums equal integrals to ~1e-15 and the closed
    forms apply.  `shells` lists (l, nprim) per atom; contraction coefficients
    are 1, 0.5, 0.25, ..."""
    rng = np.random.default_rng(seed)
    coords = rng.uniform(0.0, L, size=(natm, 3))
    sa, sl, se, sc = [], [], [], []
    for a in range(natm):
        for l, npr in shells:
            sa.append(a)
            sl.append(l)
            se.append(_log_uniform(rng, amin, amax, npr))
    shell_atom, shell_l, nprim, off, ex, _ = _finish_shells(sa, sl, se)
    co = np.concatenate([0.5 ** np.arange(len(e)) for e in se])
    nao = sum(ncart(l) for l in sl)
    C = rng.standard_normal((nao, 3))
    D = C @ C.T
    return System("resolved", np.eye(3) * L, coords, shell_atom, shell_l, nprim, off, ex, co,
                  D, cutoff_ha=cutoff, nlevels=nlevels, level_ratio=3.0, meshes=None,
                  rel_cutoff=40.0, tau=tau, nocc=3, potential=_plane_waves(rng, 6, 2))


def single_gaussian(alpha: float, L: float, cutoff: float = 200.0, nlevels: int = 3,
                    pos=(0.3, 0.1, 0.7)) -> System:
    """One s primitive (unit coefficient) in a cubic box, D = [[1]]."""
    coords = np.array([pos], dtype=float) * L
    return System("gauss", np.eye(3) * L, coords, np.array([0], np.int32),
                  np.array([0], np.int32), np.array([1], np.int32), np.array([0], np.int32),
                  np.array([alpha]), np.array([1.0]), np.array([[1.0]]), cutoff_ha=cutoff,
                  nlevels=nlevels, level_ratio=3.0, meshes=None, rel_cutoff=40.0, tau=1e-14)


def tiny14() -> System:
    """The tiny workload at tau = 1e-14."""
    return workloads.tiny().with_tau(1e-14)


TRICLINIC = workloads.TRICLINIC


def skewed(seed: int = 5, L: float = 6.0, lattice=None, **kw) -> System:
    """The `resolved` system in a non-orthogonal cell: lattice rows L * TRICLINIC (or
    `lattice`), atoms at the same fractional positions."""
    s = resolved(seed=seed, L=L, **kw)
    lat = np.asarray(lattice if lattice is not None else L * TRICLINIC, dtype=np.float64)
    frac = s.coords / L
    s.lattice = lat
    s.coords = np.ascontiguousarray(frac @ lat)
    s.name = "skewed"
    return s


def sheared(s: System) -> System:
    """The same crystal as the orthorhombic (cubic-mesh) system s, described with the
    lattice rows (R0, R0 + R1, R2): the same lattice, so the same images and, with
    N0 = N1, the same grid points (skewed point (i, j, k) = cubic point (i + j, j, k))."""
    import copy
    out = copy.copy(s)
    lat = np.asarray(s.lattice, dtype=np.float64)
    out.lattice = np.ascontiguousarray(np.array([lat[0], lat[0] + lat[1], lat[2]]))
    out.name = s.name + "-sheared"
    return out


def rotation(seed: int) -> np.ndarray:
    """A seeded rotation, uniform on SO(3)."""
    return workloads._rotation(np.random.default_rng(seed))


def rotated(s: System, Q: np.ndarray) -> System:
    """The crystal s turned by the rotation Q: lattice rows R_d -> Q R_d and atoms
    A -> Q A (so no row stays on an axis), same meshes and fractional grid points.  The
    Cartesian shell components are those of the new frame, so the density matrix is the
    one of the turned frame only after cart_rotation(); D is kept as it is here."""
    import copy
    out = copy.copy(s)
    Q = np.asarray(Q, dtype=np.float64)
    out.lattice = np.ascontiguousarray(np.asarray(s.lattice, dtype=np.float64) @ Q.T)
    out.coords = np.ascontiguousarray(np.asarray(s.coords, dtype=np.float64) @ Q.T)
    out.name = s.name + "-rotated"
    return out


def cart_rotation(l: int, Q: np.ndarray) -> np.ndarray:
    """M with old monomial mu = sum_kappa M[mu, kappa] new monomial kappa, for the
    degree-l Cartesian monomials (x^l first) of a frame turned by Q (u_new = Q u_old,
    so u_old_c = sum_e Q[e, c] u_new_e): expanded by polynomial multiplication."""
    comps = [(ix, iy, l - ix - iy) for ix in range(l, -1, -1) for iy in range(l - ix, -1, -1)]
    index = {c: i for i, c in enumerate(comps)}
    M = np.zeros((len(comps), len(comps)))
    for mu, m in enumerate(comps):
        poly = {(0, 0, 0): 1.0}
        for c in range(3):
            for _ in range(m[c]):
                nxt = {}
                for e_, coef in poly.items():
                    for e in range(3):
                        k = list(e_)
                        k[e] += 1
                        k = tuple(k)
                        nxt[k] = nxt.get(k, 0.0) + coef * Q[e, c]
                poly = nxt
        for k, coef in poly.items():
            M[mu, index[k]] += coef
    return M


def basis_rotation(s: System, Q: np.ndarray) -> np.ndarray:
    """Block-diagonal nao x nao matrix of cart_rotation over the shells of s:
    phi_old = M phi_new, so D_new = M^T D M gives the same density and
    V_old = M V_new M^T."""
    blocks = [cart_rotation(int(l), Q) for l in s.shell_l]
    n = sum(b.shape[0] for b in blocks)
    M = np.zeros((n, n))
    o = 0
    for b in blocks:
        M[o:o + b.shape[0], o:o + b.shape[0]] = b
        o += b.shape[0]
    return M


def permuted_atoms(s: System, perm) -> tuple:
    """The same crystal with its atoms listed in another order: new atom i is old atom
    perm[i], its shells keep their order and are listed atom by atom in the new order, D
    is reindexed to the new AO order.  Returns (system, ao) with ao[new AO] = old AO, so
    that quantities indexed by AOs or atoms of the new system are the old ones taken at
    ao and perm."""
    import copy
    perm = np.asarray(perm, dtype=np.int64)
    off = s.ao_offsets()
    shells = [sh for a in perm for sh in range(s.nshell) if s.shell_atom[sh] == a]
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    ao = np.concatenate([np.arange(off[sh], off[sh + 1]) for sh in shells]).astype(np.int64)
    exps, coefs, nprim, poff = [], [], [], []
    k = 0
    for sh in shells:
        o, n = int(s.shell_prim_off[sh]), int(s.shell_nprim[sh])
        exps.append(s.exponents[o:o + n])
        coefs.append(s.coeffs[o:o + n])
        nprim.append(n)
        poff.append(k)
        k += n
    out = copy.copy(s)
    out.coords = np.ascontiguousarray(s.coords[perm])
    out.shell_atom = np.ascontiguousarray(inv[s.shell_atom[shells]].astype(np.int32))
    out.shell_l = np.ascontiguousarray(s.shell_l[shells].astype(np.int32))
    out.shell_nprim = np.array(nprim, dtype=np.int32)
    out.shell_prim_off = np.array(poff, dtype=np.int32)
    out.exponents = np.ascontiguousarray(np.concatenate(exps))
    out.coeffs = np.ascontiguousarray(np.concatenate(coefs))
    out.D = np.ascontiguousarray(s.D[np.ix_(ao, ao)])
    out.name = s.name + "-permuted"
    return out, ao
