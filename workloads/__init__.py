"""Seeded synthetic inputs for the multigrid GPW collocation/integration path.

This module only draws random numbers and lays out the inputs (cells, atoms,
Gaussian shells, density matrices, band-limited test potentials).  It holds none
of the method's arithmetic: no normalisation, screening, grids or integrals.
Both the CPU oracle (``oracle/``) and the CUDA path
(``paper_2603_24881_gb300``) consume these objects; neither imports the other.

The workloads stand in for the paper's CP2K water clusters, diamond supercells
and GTH basis sets (Sec. IV), which are not available: every geometry, exponent
and density matrix is drawn from ``numpy.random.default_rng(seed)``.

Conventions
-----------
* Bohr and Hartree.  ``lattice`` rows are the cell vectors a1, a2, a3.
* Shells are Cartesian, angular momentum l <= 3; within a shell the components
  are ordered lexicographically with x^l first (d: xx, xy, xz, yy, yz, zz).
* ``shell_prim_off``/``shell_nprim`` index the flat ``exponents``/``coeffs``.
* Atom coordinates are wrapped into the home cell [0, L).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

__all__ = [
    "System", "PlaneWaves", "ncart", "tiny", "water_box", "carbon", "water32",
    "water256", "stream_requests", "small_water", "config",
]


def ncart(l: int) -> int:
    """Number of Cartesian components of a shell of angular momentum l."""
    return (l + 1) * (l + 2) // 2


@dataclass
class PlaneWaves:
    """A real band-limited field v(s) = sum_k a_k cos(2 pi n_k . s), s fractional.

    ``sample(mesh)`` returns it on an N0 x N1 x N2 grid (C order, index 2 fastest),
    the grid point (i0, i1, i2) sitting at fractional position (i0/N0, i1/N1, i2/N2).
    """
    n: np.ndarray      # (K, 3) integer G indices
    a: np.ndarray      # (K,) amplitudes

    def sample(self, mesh) -> np.ndarray:
        n0, n1, n2 = (int(m) for m in mesh)
        s0 = np.arange(n0) / n0
        s1 = np.arange(n1) / n1
        s2 = np.arange(n2) / n2
        out = np.zeros((n0, n1, n2))
        for (k0, k1, k2), amp in zip(self.n.tolist(), self.a.tolist()):
            ph = (2 * np.pi * (k0 * s0[:, None, None] + k1 * s1[None, :, None]
                               + k2 * s2[None, None, :]))
            out += amp * np.cos(ph)
        return out


@dataclass
class System:
    name: str
    lattice: np.ndarray                 # (3, 3)
    coords: np.ndarray                  # (natm, 3)
    shell_atom: np.ndarray              # (nshell,) int32
    shell_l: np.ndarray                 # (nshell,) int32
    shell_nprim: np.ndarray             # (nshell,) int32
    shell_prim_off: np.ndarray          # (nshell,) int32
    exponents: np.ndarray               # (nprim_total,)
    coeffs: np.ndarray                  # (nprim_total,)
    D: np.ndarray                       # (nao, nao) symmetric
    cutoff_ha: float = 0.0              # 0 => explicit meshes
    nlevels: int = 1
    level_ratio: float = 3.0
    meshes: np.ndarray | None = None    # (nlevels, 3) or None
    rel_cutoff: float = 40.0
    tau: float = 1e-6
    nocc: int = 0
    potential: PlaneWaves | None = None
    extra: dict = field(default_factory=dict)

    @property
    def natm(self) -> int:
        return int(self.coords.shape[0])

    @property
    def nshell(self) -> int:
        return int(self.shell_l.shape[0])

    @property
    def nao(self) -> int:
        return int(sum(ncart(int(l)) for l in self.shell_l))

    def ao_offsets(self) -> np.ndarray:
        off = np.zeros(self.nshell + 1, dtype=np.int64)
        for s, l in enumerate(self.shell_l):
            off[s + 1] = off[s] + ncart(int(l))
        return off

    def with_coords(self, coords) -> "System":
        """Same system with other atom positions (not re-wrapped)."""
        import copy
        out = copy.copy(self)
        out.coords = np.ascontiguousarray(np.asarray(coords, dtype=np.float64))
        return out

    def with_tau(self, tau: float) -> "System":
        import copy
        out = copy.copy(self)
        out.tau = float(tau)
        return out


def _log_uniform(rng, lo, hi, size=None):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


def _finish_shells(shell_atom, shell_l, shell_exps):
    nprim = np.array([len(e) for e in shell_exps], dtype=np.int32)
    off = np.zeros(len(shell_exps), dtype=np.int32)
    if len(shell_exps) > 1:
        off[1:] = np.cumsum(nprim)[:-1]
    exps = np.concatenate([np.asarray(e, dtype=np.float64) for e in shell_exps])
    return (np.asarray(shell_atom, dtype=np.int32), np.asarray(shell_l, dtype=np.int32),
            nprim, off, exps, np.ones_like(exps))


def _density(rng, nao, nocc, literal: bool):
    """D = s C C^T with C (nao x nocc) standard normal.

    literal=True keeps s = 1; otherwise s = 2*nocc / tr(C C^T), which fixes tr(D)
    to the electron count 2*nocc and keeps energies O(10^2) Hartree.
    """
    C = rng.standard_normal((nao, nocc))
    D = C @ C.T
    if not literal:
        D *= 2.0 * nocc / np.trace(D)
    return np.ascontiguousarray(0.5 * (D + D.T))


def _plane_waves(rng, count=8, nmax=3):
    pts = []
    r = range(-nmax, nmax + 1)
    for a in r:
        for b in r:
            for c in r:
                if (a, b, c) != (0, 0, 0) and a * a + b * b + c * c <= nmax * nmax:
                    pts.append((a, b, c))
    pts = np.array(pts, dtype=np.int64)
    pick = rng.choice(len(pts), size=count, replace=False)
    return PlaneWaves(n=pts[pick], a=rng.standard_normal(count))


def tiny(seed: int = 0) -> System:
    """Cubic L=6 cell, 2 atoms, each with s, s, p, d single primitives.

    Exponents log-uniform in [0.2, 20], unit coefficients, 22 functions,
    D = C C^T with C 22x3 N(0,1), meshes 40^3/20^3/10^3 and a potential built
    from 8 plane waves with |n| <= 3.
    """
    rng = np.random.default_rng(seed)
    L = 6.0
    coords = rng.uniform(0.0, L, size=(2, 3))
    shell_atom, shell_l, shell_exps = [], [], []
    for a in range(2):
        for l in (0, 0, 1, 2):
            shell_atom.append(a)
            shell_l.append(l)
            shell_exps.append([_log_uniform(rng, 0.2, 20.0)])
    sa, sl, npr, off, ex, co = _finish_shells(shell_atom, shell_l, shell_exps)
    nao = sum(ncart(l) for l in shell_l)
    D = _density(rng, nao, 3, literal=True)
    pw = _plane_waves(rng)
    return System("tiny", np.eye(3) * L, coords, sa, sl, npr, off, ex, co, D,
                  cutoff_ha=0.0, nlevels=3, level_ratio=3.0,
                  meshes=np.array([[40] * 3, [20] * 3, [10] * 3], dtype=np.int32),
                  rel_cutoff=40.0, tau=1e-6, nocc=3, potential=pw)


def _rotation(rng):
    # uniform random rotation from a uniform unit quaternion
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def water_box(nwat: int, L: float, seed: int, *, cutoff_ha: float = 280.0,
              nlevels: int = 4, level_ratio: float = 3.0, tau: float = 1e-6,
              name: str | None = None, max_tries: int = 2_000_000) -> System:
    """Rigid waters by random sequential placement in a cubic cell of edge L.

    O uniform in the cell, orientation uniform on SO(3), O-H 1.81 Bohr,
    HOH 104.5 deg, minimum-image O-O >= 4.8 Bohr.  Per O: 3 s, 3 p, 1 d shells,
    exponents log-uniform in [0.15, 12]; per H: 2 s, 1 p, exponents in [0.1, 4];
    1-3 primitives per shell, unit coefficients.  D from 4 occupied columns per
    water (the valence pairs).
    """
    rng = np.random.default_rng(seed)
    roh, th = 1.81, math.radians(104.5)
    h1 = roh * np.array([math.sin(th / 2), 0.0, math.cos(th / 2)])
    h2 = roh * np.array([-math.sin(th / 2), 0.0, math.cos(th / 2)])
    oxy = []
    tries = 0
    while len(oxy) < nwat:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("water placement did not converge")
        o = rng.uniform(0.0, L, 3)
        ok = True
        for p in oxy:
            d = o - p
            d -= L * np.round(d / L)
            if d @ d < 4.8 * 4.8:
                ok = False
                break
        if ok:
            oxy.append(o)
    coords = []
    for o in oxy:
        R = _rotation(rng)
        coords += [o, o + R @ h1, o + R @ h2]
    coords = np.mod(np.array(coords), L)
    shell_atom, shell_l, shell_exps = [], [], []
    for a in range(3 * nwat):
        if a % 3 == 0:
            ls, lo, hi = (0, 0, 0, 1, 1, 1, 2), 0.15, 12.0
        else:
            ls, lo, hi = (0, 0, 1), 0.1, 4.0
        for l in ls:
            npr = int(rng.integers(1, 4))
            shell_atom.append(a)
            shell_l.append(l)
            shell_exps.append(_log_uniform(rng, lo, hi, npr))
    sa, sl, npr, off, ex, co = _finish_shells(shell_atom, shell_l, shell_exps)
    nao = sum(ncart(l) for l in shell_l)
    nocc = 4 * nwat
    D = _density(rng, nao, nocc, literal=False)
    pw = _plane_waves(rng)
    return System(name or f"water{nwat}", np.eye(3) * L, coords, sa, sl, npr, off,
                  ex, co, D, cutoff_ha=cutoff_ha, nlevels=nlevels,
                  level_ratio=level_ratio, meshes=None, rel_cutoff=40.0, tau=tau,
                  nocc=nocc, potential=pw)


def water32(seed: int = 1) -> System:
    """32 waters, L = 18.64 Bohr (1 g/cm^3), 896 functions, 280 Ha, 4 levels."""
    return water_box(32, 18.64, seed, name="water32")


def water256(seed: int = 3) -> System:
    """256 waters, L = 37.3 Bohr, 7168 functions, 280 Ha, 4 levels."""
    return water_box(256, 37.3, seed, name="water256")


# a triclinic cell shape (rows; angles about 74, 103 and 79 degrees), volume 0.912 L^3
TRICLINIC = np.array([[1.0, 0.0, 0.0], [0.28, 0.96, 0.0], [-0.21, 0.17, 0.95]])


# a hexagonal cell shape (rows a, b at 120 degrees, c orthogonal to both, c/a = 1.1),
# volume (sqrt(3)/2) 1.1 L^3
HEXAGONAL = np.array([[1.0, 0.0, 0.0], [-0.5, math.sqrt(3.0) / 2.0, 0.0], [0.0, 0.0, 1.1]])


def hexagonal(s: System) -> System:
    """The cubic system s moved into a hexagonal cell of the same volume (as triclinic)."""
    return _reshape_cell(s, HEXAGONAL, "hexagonal")


def _reshape_cell(s: System, shape, name) -> System:
    import copy
    L = float(s.lattice[0, 0])
    scale = L / float(np.linalg.det(shape)) ** (1.0 / 3.0)
    out = copy.copy(s)
    out.lattice = np.ascontiguousarray(scale * np.asarray(shape, dtype=np.float64))
    out.coords = np.ascontiguousarray((s.coords / L) @ out.lattice)
    out.name = s.name + "-" + name
    return out


def triclinic(s: System) -> System:
    """The cubic system s moved into a triclinic cell of the same volume: lattice rows
    L' TRICLINIC with L'^3 det(TRICLINIC) = L^3, every atom at the same fractional
    position (molecules are sheared with the cell: a synthetic non-orthogonal input)."""
    return _reshape_cell(s, TRICLINIC, "triclinic")


def small_water(nwat: int = 4, seed: int = 11, **kw) -> System:
    """A water box at the 32-water density: L = 18.64 (n/32)^(1/3)."""
    return water_box(nwat, 18.64 * (nwat / 32.0) ** (1.0 / 3.0), seed, **kw)


def carbon(seed: int = 2, reps: int = 3) -> System:
    """Diamond, conventional cubic cell a = 20.2/3 Bohr, reps^3 cells, jitter 0.05.

    Per C: 2 s, 2 p, 2 d and 1 f single primitives, exponents log-uniform in
    [0.2, 10]; 30 functions per atom; 2 occupied columns per atom; 400 Ha, 5 levels.
    """
    rng = np.random.default_rng(seed)
    a = 20.2 / 3.0
    base = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]], dtype=float)
    base = np.concatenate([base, base + 0.25])
    pos = []
    for i in range(reps):
        for j in range(reps):
            for k in range(reps):
                for b in base:
                    pos.append((np.array([i, j, k]) + b) * a)
    pos = np.array(pos) + rng.normal(0.0, 0.05, size=(len(pos), 3))
    L = a * reps
    coords = np.mod(pos, L)
    shell_atom, shell_l, shell_exps = [], [], []
    for at in range(len(coords)):
        for l in (0, 0, 1, 1, 2, 2, 3):
            shell_atom.append(at)
            shell_l.append(l)
            shell_exps.append([_log_uniform(rng, 0.2, 10.0)])
    sa, sl, npr, off, ex, co = _finish_shells(shell_atom, shell_l, shell_exps)
    nao = sum(ncart(l) for l in shell_l)
    nocc = 2 * len(coords)
    D = _density(rng, nao, nocc, literal=False)
    pw = _plane_waves(rng)
    return System(f"carbon{reps}", np.eye(3) * L, coords, sa, sl, npr, off, ex, co,
                  D, cutoff_ha=400.0, nlevels=5, level_ratio=3.0, meshes=None,
                  rel_cutoff=40.0, tau=1e-6, nocc=nocc, potential=pw)


@dataclass
class Request:
    rid: int
    nwat: int
    seed: int
    want_grad: bool
    arrival: float = 0.0

    def system(self) -> System:
        return small_water(self.nwat, seed=self.seed, name=f"req{self.rid}-w{self.nwat}")


def stream_requests(count: int = 400, seed: int = 4, rate: float | None = None):
    """The served stream: n in {4..128} with p ~ 1/n, 10% gradients.

    With ``rate`` (requests/s) arrivals are Poisson; otherwise all arrive at t=0.
    """
    rng = np.random.default_rng(seed)
    sizes = np.array([4, 8, 16, 32, 64, 128])
    p = (1.0 / sizes) / np.sum(1.0 / sizes)
    n = rng.choice(sizes, size=count, p=p)
    grad = rng.uniform(size=count) < 0.10
    seeds = rng.integers(0, 2**31 - 1, size=count)
    gaps = rng.exponential(1.0, size=count)
    t = np.cumsum(gaps) / rate if rate else np.zeros(count)
    return [Request(i, int(n[i]), int(seeds[i]), bool(grad[i]), float(t[i]))
            for i in range(count)]


def config(name: str) -> System:
    """Named workloads: tiny, water32, carbon, water256, water4, water8 and the triclinic
    water4, water32 and water256 and the hexagonal water32 and water256 (non-orthogonal
    cells)."""
    return {
        "tiny": tiny, "water32": water32, "carbon": carbon, "water256": water256,
        "water4": lambda: small_water(4, seed=11),
        "water8": lambda: small_water(8, seed=12),
        "water4_triclinic": lambda: triclinic(small_water(4, seed=11)),
        "water32_triclinic": lambda: triclinic(water32()),
        "water256_triclinic": lambda: triclinic(water256()),
        "water32_hexagonal": lambda: hexagonal(water32()),
        "water256_hexagonal": lambda: hexagonal(water256()),
    }[name]()
