"""Pins of the CPU oracle against mathematics it does not itself contain.

The paper prints no values of rho, V, energies or forces (only timings), so every
pin here is a closed form, a brute-force evaluation, an identity or an invariance:

* normalisation: unit self-overlap from Gaussian moments (Sec. II basis);
* integral of rho over the cell = tr(D S), S the lattice-summed analytic overlap
  (Eq. rho integrated; resolved exponents so the grid sum is exact);
* eval_mat(constant) = c S and eval_mat(plane waves) = closed-form Gaussian x
  plane-wave integrals (Eq. J);
* each level density equals the untruncated double lattice sum of Eq. (rho),
  built from periodised orbitals, on the pairs of that level;
* adjoint identity <v, rho(D)> = tr(D V(v)) through the multigrid Fourier
  interpolation and restriction;
* Hartree energy of one Gaussian charge against the analytic G sum and the
  Ewald-corrected isolated self-energy (Eqs. vH, vHG);
* LDA exchange of a uniform density against Dirac's -(3/4 pi) k_F per electron;
* PBE exchange (GGA): Dirac exchange for a uniform density, the enhancement factor's
  limits (1, the Lieb-Oxford 1.804, the gradient-expansion coefficient), the potential
  as the functional derivative through the Fourier gradient and divergence, and exact
  uniform-scaling of exchange (E[l^3 rho(l r)] = l E[rho]);
* gradient contraction (Algorithm 3) against central finite differences;
* kinetic energy density (meta-GGA): the integral of tau against (1/2) tr(D T) with the
  analytic lattice-summed grad-phi overlaps T, its Fock term for a constant and for
  plane-wave potentials against closed forms, the adjoint identity, and its gradient
  against finite differences;
* invariance under lattice translations and whole-grid shifts.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
import closed_forms as cf
import systems


@pytest.fixture(scope="module")
def res():
    s = systems.resolved()
    return s, oracle.Plan(s)


@pytest.fixture(scope="module")
def overlap(res):
    return cf.lattice_overlap(res[0], reach=20.0)


def test_normalisation_unit_self_overlap():
    for l in range(4):
        for a in (0.1, 0.7, 3.0, 25.0):
            assert oracle.prim_norm(l, a) == pytest.approx(cf.norm(l, a), rel=1e-14)


def test_cartesian_order():
    assert oracle.cart_components(2) == [(2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)]
    assert len(oracle.cart_components(3)) == 10


def test_meshes_from_cutoff():
    # 32-water: 280 Ha, L = 18.64, ratio 3 -> 144/84/50/30 (smallest even 7-smooth)
    m, E, G = oracle.level_grids(workloads.water_box(1, 18.64, 0))
    assert m[:, 0].tolist() == [144, 84, 50, 30]
    for k in range(4):
        # the strict cutoff sphere never reaches the Nyquist planes
        assert G[k] * 18.64 / (2 * math.pi) < (m[k, 0] - 1) / 2
    m, E, G = oracle.level_grids(workloads.tiny())
    assert E[0] == pytest.approx(0.5 * (2 * math.pi * 19 / 6) ** 2)


def test_integrated_density_is_trace_DS(res, overlap):
    s, p = res
    S = overlap
    rho = p.combine(p.rho_levels(s.D))
    omega = float(np.prod(np.diag(s.lattice)))
    tot = omega / rho.size * rho.sum()
    ref = float(np.sum(s.D * S))
    assert tot == pytest.approx(ref, rel=1e-11, abs=1e-12)
    # each level separately integrates to its share (sum over levels)
    parts = [omega / r.size * r.sum() for r in p.rho_levels(s.D)]
    assert sum(parts) == pytest.approx(ref, rel=1e-11)


def test_mat_of_constant_is_overlap(res, overlap):
    s, p = res
    S = overlap
    c = 0.37
    V = p.mat_levels([np.full(tuple(m), c) for m in p.meshes])
    assert np.max(np.abs(V - c * S)) < 1e-11 * np.max(np.abs(S))
    assert np.max(np.abs(V - V.T)) < 1e-14 * np.max(np.abs(V))


def test_mat_of_plane_waves_closed_form(res):
    s, p = res
    pw = s.potential
    vf = pw.sample(p.meshes[0])
    vl = p.restrict(vf)
    # band-limited inside every level sphere: restriction reproduces the waves
    for k in range(p.nlev):
        assert np.max(np.abs(vl[k] - pw.sample(p.meshes[k]))) < 1e-12
    V = p.mat_levels(vl)
    ref = cf.lattice_pw_matrix(s, pw, reach=20.0)
    assert np.max(np.abs(V - ref)) < 1e-10 * max(1.0, np.max(np.abs(ref)))


def _periodic_prims(sys, mesh, reach=30.0):
    """Per (AO, primitive): periodised primitive values on `mesh`."""
    L = np.diag(sys.lattice)
    x = [np.arange(mesh[d]) * (L[d] / mesh[d]) for d in range(3)]
    n = [int(math.ceil(reach / L[d])) + 1 for d in range(3)]
    out = []
    ao = 0
    for sh in range(sys.nshell):
        l = int(sys.shell_l[sh])
        o = int(sys.shell_prim_off[sh])
        for c in oracle.cart_components(l):
            for k in range(int(sys.shell_nprim[sh])):
                a = float(sys.exponents[o + k])
                cn = float(sys.coeffs[o + k]) * cf.norm(l, a)
                f = np.zeros(tuple(int(m) for m in mesh))
                for i in range(-n[0], n[0] + 1):
                    for j in range(-n[1], n[1] + 1):
                        for kk in range(-n[2], n[2] + 1):
                            A = sys.coords[int(sys.shell_atom[sh])] + np.array([i, j, kk]) * L
                            u = [x[d] - A[d] for d in range(3)]
                            g = [u[d] ** c[d] * np.exp(-a * u[d] ** 2) for d in range(3)]
                            f += cn * g[0][:, None, None] * g[1][None, :, None] * g[2][None, None, :]
                out.append((ao, a, f))
            ao += 1
    return out


@pytest.mark.parametrize("name", ["tiny14", "resolved"])
def test_levels_match_untruncated_double_lattice_sum(name):
    s = systems.tiny14() if name == "tiny14" else systems.resolved()
    p = oracle.Plan(s)
    rl = p.rho_levels(s.D, mode="plain")
    for k in range(p.nlev):
        mesh = p.meshes[k]
        prims = _periodic_prims(s, mesh)
        ref = np.zeros(tuple(int(m) for m in mesh))
        for (m, am, fm) in prims:
            for (n, an, fn) in prims:
                ap = am + an
                lev = 0
                for kk in range(p.nlev - 1, -1, -1):
                    if p.E[kk] >= 40.0 * ap:
                        lev = kk
                        break
                if lev == k:
                    ref += s.D[m, n] * fm * fn
        scale = max(1.0, np.max(np.abs(ref)))
        assert np.max(np.abs(rl[k] - ref)) < 1e-11 * scale, (name, k)


def test_plain_equals_separable():
    s = systems.tiny14()
    p = oracle.Plan(s)
    a = p.rho_levels(s.D, mode="plain")
    b = p.rho_levels(s.D, mode="separable")
    for x, y in zip(a, b):
        assert np.max(np.abs(x - y)) <= 1e-12 * max(1.0, np.max(np.abs(x)))


def test_screening_error_is_tau_sized():
    s = workloads.tiny()        # tau = 1e-6
    p6 = oracle.Plan(s)
    p14 = oracle.Plan(s.with_tau(1e-14))
    assert p14.npairs > p6.npairs
    a = p6.rho_levels(s.D)
    b = p14.rho_levels(s.D)
    nd = float(np.max(np.abs(s.D)))
    for x, y in zip(a, b):
        # every dropped or clipped piece is below tau per unit D element
        assert np.max(np.abs(x - y)) < 200 * 1e-6 * nd


def test_adjoint_identity(res):
    s, p = res
    rng = np.random.default_rng(7)
    D = rng.standard_normal((s.nao, s.nao))
    D = D + D.T
    v = rng.standard_normal(tuple(p.meshes[0]))
    rho = p.combine(p.rho_levels(D))
    omega = float(np.prod(np.diag(s.lattice)))
    lhs = omega / rho.size * float(np.sum(v * rho))
    V = p.mat_levels(p.restrict(v))
    rhs = float(np.sum(D * V))
    assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("alpha,L", [(0.8, 10.0), (2.5, 8.0)])
def test_hartree_of_gaussian_charge(alpha, L):
    s = systems.single_gaussian(alpha, L)
    p = oracle.Plan(s)
    rho = p.combine(p.rho_levels(s.D))
    _, EH = p.poisson(rho)
    k = int(p.lev[0])
    ref = cf.gaussian_charge_hartree(2 * alpha, L, gcut=p.G[k])
    assert EH == pytest.approx(ref, rel=1e-11)


def test_hartree_isolated_limit_with_ewald():
    # unit Gaussian charge exponent a' = 2 alpha in a large cube:
    # E_per = E_self + E_Madelung(L) + pi/(a' Omega) up to erfc tails
    alpha, L = 1.2, 16.0
    s = systems.single_gaussian(alpha, L, cutoff=160.0)
    p = oracle.Plan(s)
    _, EH = p.poisson(p.combine(p.rho_levels(s.D)))
    ap = 2 * alpha
    e_self = math.sqrt(ap / (2 * math.pi))
    ref = e_self + cf.madelung_cubic_background(L) + math.pi / (ap * L ** 3)
    assert EH == pytest.approx(ref, rel=1e-10)


def test_lda_uniform_gas():
    s = systems.resolved()
    p = oracle.Plan(s)
    c = 0.0123
    rho = np.full(tuple(p.meshes[0]), c)
    vx, Ex = p.lda_x(rho)
    omega = float(np.prod(np.diag(s.lattice)))
    kF = (3 * math.pi ** 2 * c) ** (1.0 / 3.0)
    assert Ex == pytest.approx(-(3.0 / (4 * math.pi)) * kF * c * omega, rel=1e-13)
    # v_x is the functional derivative: dE_x / d rho(r) = (Omega/N) v_x(r)
    h = 1e-7
    ep = p.lda_x(rho + h)[1]
    em = p.lda_x(rho - h)[1]
    assert (ep - em) / (2 * h) == pytest.approx(omega / rho.size * float(np.sum(vx)), rel=1e-7)
    # negative density is clipped (continuous at 0)
    vx0, E0 = p.lda_x(np.full(tuple(p.meshes[0]), -1.0))
    assert E0 == 0.0 and np.all(vx0 == 0.0)


def test_gradient_matches_finite_differences_of_bilinear_form(res):
    s, p = res
    v = [s.potential.sample(m) for m in p.meshes]
    g = p.grad_levels(s.D, v)
    omega = float(np.prod(np.diag(s.lattice)))

    def form(coords):
        q = p.with_coords(coords)
        rl = q.rho_levels(s.D)
        return sum(omega / r.size * float(np.sum(r * vv)) for r, vv in zip(rl, v))

    h = 1e-4
    for atom, d in [(0, 0), (0, 2), (1, 1)]:
        cp = s.coords.copy()
        cm = s.coords.copy()
        cp[atom, d] += h
        cm[atom, d] -= h
        fd = (form(cp) - form(cm)) / (2 * h)
        assert g[atom, d] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_energy_gradient_matches_finite_differences(res):
    s, p = res
    out = p.fock(s.D)
    g = p.grad_levels(s.D, out["v_levels"])
    h = 1e-4
    for atom, d in [(0, 1), (1, 0), (1, 2)]:
        cp = s.coords.copy()
        cm = s.coords.copy()
        cp[atom, d] += h
        cm[atom, d] -= h
        fd = (p.with_coords(cp).energy(s.D) - p.with_coords(cm).energy(s.D)) / (2 * h)
        assert g[atom, d] == pytest.approx(fd, rel=1e-6, abs=1e-7)


def test_energy_derivative_wrt_density_matrix_is_V(res):
    # dE/dD_mu,nu = V_mu,nu (symmetric perturbation)
    s, p = res
    out = p.fock(s.D)
    rng = np.random.default_rng(3)
    X = rng.standard_normal(s.D.shape)
    X = X + X.T
    h = 1e-5
    fd = (p.energy(s.D + h * X) - p.energy(s.D - h * X)) / (2 * h)
    assert fd == pytest.approx(float(np.sum(X * out["V"])), rel=1e-7)


def test_lattice_translation_invariance():
    s = systems.tiny14()
    p = oracle.Plan(s)
    c2 = s.coords.copy()
    c2[1] += np.array([6.0, -6.0, 12.0])
    q = oracle.Plan(s.with_coords(c2))
    assert q.npairs == p.npairs
    for x, y in zip(p.rho_levels(s.D), q.rho_levels(s.D)):
        assert np.max(np.abs(x - y)) < 1e-11 * max(1.0, np.max(np.abs(x)))


def test_whole_grid_shift():
    s = systems.tiny14()
    p = oracle.Plan(s)
    # 4 finest-grid spacings = 2 on the 20^3 level = 1 on the 10^3 level
    shift = 4 * 6.0 / 40
    q = oracle.Plan(s.with_coords(s.coords + np.array([shift, 0, 0])))
    a = p.rho_levels(s.D)
    b = q.rho_levels(s.D)
    for k, (x, y) in enumerate(zip(a, b)):
        n = 4 * int(p.meshes[k][0]) // 40
        assert np.max(np.abs(np.roll(x, n, axis=0) - y)) < 1e-11 * max(1.0, np.max(np.abs(x)))


def test_rho_points_match_full_grid():
    s = workloads.tiny()
    p = oracle.Plan(s)
    rl = p.rho_levels(s.D)
    rng = np.random.default_rng(1)
    for k in range(2):
        pts = rng.integers(0, p.meshes[k][0], size=(20, 3))
        got = p.rho_points(s.D, k, pts)
        ref = rl[k][pts[:, 0], pts[:, 1], pts[:, 2]]
        assert np.max(np.abs(got - ref)) < 1e-12 * max(1.0, np.max(np.abs(rl[k])))


def test_mat_block_matches_full(res):
    s, p = res
    vl = [s.potential.sample(m) for m in p.meshes]
    V = p.mat_levels(vl)
    off = s.ao_offsets()
    for sa, sb in [(0, 3), (2, 2), (4, 1)]:
        blk = p.mat_block(vl, sa, sb)
        ref = V[off[sa]:off[sa + 1], off[sb]:off[sb + 1]]
        assert np.max(np.abs(blk - ref)) < 1e-13 * max(1.0, np.max(np.abs(V)))


# ---------------------------------------------------------------- GGA (PBE exchange) --

def _smooth_density(p, seed=5, floor=0.02):
    """A positive, band-limited density on the finest mesh (random Fourier components
    inside half the cutoff sphere plus a constant)."""
    mesh = tuple(int(m) for m in p.meshes[0])
    rng = np.random.default_rng(seed)
    g2 = oracle.gvectors(mesh, p.L)
    spec = (rng.standard_normal(mesh) + 1j * rng.standard_normal(mesh)) * (g2 < 0.25 * p.G[0] ** 2)
    f = np.real(np.fft.ifftn(spec))
    f = f / np.max(np.abs(f))
    return floor + 0.01 * (1.0 + f), spec


def test_pbe_x_uniform_density_is_dirac_exchange():
    s = systems.resolved()
    p = oracle.Plan(s)
    c = 0.0123
    rho = np.full(tuple(p.meshes[0]), c)
    vx, Ex = p.pbe_x(rho)
    omega = float(np.prod(np.diag(s.lattice)))
    kF = (3 * math.pi ** 2 * c) ** (1.0 / 3.0)
    assert Ex == pytest.approx(-(3.0 / (4 * math.pi)) * kF * c * omega, rel=1e-13)
    assert np.allclose(vx, -kF / math.pi, rtol=1e-13, atol=0)  # v_x = -k_F/pi
    vl, El = p.lda_x(rho)
    assert Ex == pytest.approx(El, rel=1e-14)


def test_pbe_x_enhancement_factor_limits():
    # F_x(0) = 1, F_x -> 1 + kappa = 1.804 (Lieb-Oxford bound) for s -> infinity,
    # F_x = 1 + mu s^2 + O(s^4) with mu = beta pi^2/3 = 0.21951 (gradient expansion)
    rho = 0.3
    kf = (3 * math.pi ** 2 * rho) ** (1.0 / 3.0)
    elda = -(3.0 / (4 * math.pi)) * kf * rho
    for s_val, ref, tol in [(0.0, 1.0, 1e-15), (1e6, 1.804, 1e-9)]:
        sigma = (s_val * 2 * kf * rho) ** 2
        e, _, _ = oracle.pbe_x_point(rho, sigma)
        assert float(e) / elda == pytest.approx(ref, rel=tol)
    s_small = 1e-4
    e, _, _ = oracle.pbe_x_point(rho, (s_small * 2 * kf * rho) ** 2)
    assert (float(e) / elda - 1.0) / s_small ** 2 == pytest.approx(0.2195149727645171, rel=1e-6)


def test_pbe_x_potential_is_functional_derivative():
    # (E[rho + h d] - E[rho - h d]) / 2h = (Omega/N) sum_r v(r) d(r), through the Fourier
    # gradient and divergence
    s = systems.resolved()
    p = oracle.Plan(s)
    rho, _ = _smooth_density(p)
    dlt, _ = _smooth_density(p, seed=9, floor=0.0)
    dlt -= dlt.mean()
    v, E = p.pbe_x(rho)
    h = 1e-4  # central differences converge as h^2 (1e-2: 2.5e-6, 1e-3: 2.5e-8 relative)
    fd = (p.pbe_x(rho + h * dlt)[1] - p.pbe_x(rho - h * dlt)[1]) / (2 * h)
    omega = float(np.prod(np.diag(s.lattice)))
    assert fd == pytest.approx(omega / rho.size * float(np.sum(v * dlt)), rel=1e-8)
    # and the gradient term matters: PBE differs from LDA for this density
    assert abs(E - p.lda_x(rho)[1]) > 1e-3 * abs(E)


def test_pbe_x_uniform_scaling():
    # exchange under uniform scaling rho_l(r) = l^3 rho(l r): E_x[rho_l] = l E_x[rho],
    # v_l(r) = l v(l r) (a cell shrunk by l with the same mesh samples l^3 rho)
    import copy
    s = systems.resolved()
    p = oracle.Plan(s)
    rho, _ = _smooth_density(p)
    v, E = p.pbe_x(rho)
    lam = 1.7
    q = copy.copy(p)
    q.L = p.L / lam
    q.lat = p.lat / lam
    q.omega = float(np.prod(q.L))
    vq, Eq = q.pbe_x(lam ** 3 * rho)
    assert Eq == pytest.approx(lam * E, rel=1e-12)
    assert np.max(np.abs(vq - lam * v)) <= 1e-12 * np.max(np.abs(lam * v))


@pytest.mark.parametrize("xc", ["pbe_x"])
def test_energy_derivative_wrt_density_matrix_is_V_gga(res, xc):
    s, p = res
    out = p.fock(s.D, xc=xc)
    rng = np.random.default_rng(4)
    X = rng.standard_normal(s.D.shape)
    X = X + X.T
    h = 1e-5
    fd = (p.energy(s.D + h * X, xc=xc) - p.energy(s.D - h * X, xc=xc)) / (2 * h)
    assert fd == pytest.approx(float(np.sum(X * out["V"])), rel=1e-7)


def test_energy_gradient_matches_finite_differences_gga(res):
    s, p = res
    out = p.fock(s.D, xc="pbe_x")
    g = p.grad_levels(s.D, out["v_levels"])
    h = 1e-4
    for atom, d in [(0, 2), (1, 1)]:
        cp = s.coords.copy()
        cm = s.coords.copy()
        cp[atom, d] += h
        cm[atom, d] -= h
        fd = (p.with_coords(cp).energy(s.D, xc="pbe_x") -
              p.with_coords(cm).energy(s.D, xc="pbe_x")) / (2 * h)
        assert g[atom, d] == pytest.approx(fd, rel=1e-6, abs=1e-7)


# ---------------------------------------------------------------- meta-GGA (tau) ----

@pytest.fixture(scope="module")
def res_tau():
    # shells up to f (the kinetic-energy-density kernels' range), resolved exponents
    s = systems.resolved(seed=6, shells=((0, 1), (1, 1), (2, 1), (3, 1)), cutoff=100.0)
    return s, oracle.Plan(s)


@pytest.fixture(scope="module")
def gradov(res_tau):
    return cf.lattice_grad_overlap(res_tau[0], reach=20.0)


def test_integrated_tau_is_half_trace_DT(res_tau, gradov):
    # int tau = (1/2) tr(D T), T_mu,nu = sum_T int grad phi_mu . grad phi_nu (analytic)
    s, p = res_tau
    tl = p.tau_levels(s.D)
    omega = float(np.prod(np.diag(s.lattice)))
    tot = sum(omega / t.size * float(np.sum(t)) for t in tl)
    assert tot == pytest.approx(0.5 * float(np.sum(s.D * gradov)), rel=1e-10)
    assert tot > 0  # D = C C^T is positive semidefinite


def test_mat_tau_of_constant_is_half_T(res_tau, gradov):
    s, p = res_tau
    c = 0.37
    V = p.mat_tau_levels([np.full(tuple(m), c) for m in p.meshes])
    assert np.max(np.abs(V - 0.5 * c * gradov)) <= 1e-10 * np.max(np.abs(gradov))


def test_mat_tau_of_plane_waves_closed_form(res_tau):
    s, p = res_tau
    waves = workloads.PlaneWaves(s.potential.n[:2], s.potential.a[:2])  # two waves suffice
    V = p.mat_tau_levels([waves.sample(m) for m in p.meshes])
    ref = 0.5 * cf.lattice_grad_pw_matrix(s, waves, reach=20.0)
    assert np.max(np.abs(V - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_tau_adjoint_identity(res_tau):
    # <v, tau(D)> = tr(D V_tau(v)) level by level
    s, p = res_tau
    v = [s.potential.sample(m) for m in p.meshes]
    tl = p.tau_levels(s.D)
    omega = float(np.prod(np.diag(s.lattice)))
    lhs = sum(omega / t.size * float(np.sum(t * vv)) for t, vv in zip(tl, v))
    rhs = float(np.sum(s.D * p.mat_tau_levels(v)))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_tau_gradient_matches_finite_differences(res_tau):
    s, p = res_tau
    v = [s.potential.sample(m) for m in p.meshes]
    g = p.grad_tau_levels(s.D, v)
    omega = float(np.prod(np.diag(s.lattice)))

    def form(coords):
        tl = p.with_coords(coords).tau_levels(s.D)
        return sum(omega / t.size * float(np.sum(t * vv)) for t, vv in zip(tl, v))

    h = 1e-4
    for atom, d in [(0, 2), (1, 0)]:
        cp = s.coords.copy()
        cm = s.coords.copy()
        cp[atom, d] += h
        cm[atom, d] -= h
        fd = (form(cp) - form(cm)) / (2 * h)
        assert g[atom, d] == pytest.approx(fd, rel=1e-6, abs=1e-8)


# ------------------------------------------- non-orthogonal cells (App., lattices) --
@pytest.fixture(scope="module")
def res_skew():
    s = systems.skewed(shells=((0, 1), (1, 1), (2, 1)), natm=2)
    return s, oracle.Plan(s)


def test_skew_integrated_density_is_trace_DS(res_skew):
    # a triclinic cell: the level densities integrate to Tr(D S), S the lattice sum of
    # the analytic overlaps over Cartesian image vectors T = n . R
    s, p = res_skew
    rl = p.rho_levels(s.D)
    N = sum(p.omega / float(np.prod(m)) * float(r.sum()) for m, r in zip(p.meshes, rl))
    S = cf.lattice_overlap(s, reach=30.0)
    assert N == pytest.approx(float(np.sum(s.D * S)), rel=1e-11)


def test_skew_mat_of_plane_waves_closed_form(res_skew):
    # v(r) = sum a cos(G . r) with G = 2 pi n . B (reciprocal rows B): the fractional
    # samples of the waves on every level, and V against the analytic lattice sums
    s, p = res_skew
    pw = s.potential
    vl = p.restrict(pw.sample(p.meshes[0]))
    for k in range(p.nlev):
        assert np.max(np.abs(vl[k] - pw.sample(p.meshes[k]))) < 1e-12
    V = p.mat_levels(vl)
    ref = cf.lattice_pw_matrix(s, pw, reach=20.0)
    assert np.max(np.abs(V - ref)) < 1e-10 * max(1.0, np.max(np.abs(ref)))


def test_skew_energy_gradient_matches_finite_differences(res_skew):
    s, p = res_skew
    out = p.fock(s.D)
    g = p.grad_levels(s.D, out["v_levels"])
    h = 1e-4
    for atom, d in [(0, 0), (1, 1), (1, 2)]:
        cp = s.coords.copy()
        cm = s.coords.copy()
        cp[atom, d] += h
        cm[atom, d] -= h
        fd = (p.with_coords(cp).energy(s.D) - p.with_coords(cm).energy(s.D)) / (2 * h)
        assert g[atom, d] == pytest.approx(fd, rel=1e-6, abs=1e-7)


def test_sheared_description_of_a_cubic_cell():
    # one cubic crystal described by rows (R0, R1, R2) and by (R0, R0 + R1, R2), with the
    # same explicit meshes: the same lattice, images and grid points (skewed point
    # (i, j, k) is cubic point (i + j mod N, j, k)).  The longer row R0 + R1 gives the
    # sheared description level spheres sqrt(2) smaller (Sec. II multigrid: the sphere
    # must fit the mesh along every row), so the meshes are taken 1.6 times finer than
    # the cutoff asks, which leaves the resolved densities' spectra below 1e-11 outside
    # either sphere; the two descriptions then agree up to that and the pair boxes.
    s = systems.resolved(seed=7, shells=((0, 1), (1, 1), (2, 1)), natm=2, nlevels=2)
    p = oracle.Plan(s)
    s.meshes = np.array([[oracle._smooth7_even(int(1.6 * m)) for m in row] for row in p.meshes])
    s.cutoff_ha = 0.0
    # the sheared levels' cutoffs are half the cubic ones, so pairs may sit on other
    # levels: a level keeps a pair's spectrum down to exp(-E_k / (2 alpha_p)) <=
    # exp(-rel / 2), made negligible here by rel = 100
    s.rel_cutoff = 100.0
    p = oracle.Plan(s)
    q = oracle.Plan(systems.sheared(s))
    a, b = p.fock(s.D), q.fock(s.D)
    N = int(p.meshes[0][0])
    i = np.arange(N)
    perm = (i[:, None] + i[None, :]) % N  # cubic x index of skewed (i, j)
    rho_b_on_a = np.empty_like(a["rho_fine"])
    rho_b_on_a[perm, i[None, :], :] = b["rho_fine"]
    scale = np.max(np.abs(a["rho_fine"]))
    assert np.max(np.abs(rho_b_on_a - a["rho_fine"])) <= 1e-9 * scale
    assert b["EH"] == pytest.approx(a["EH"], rel=1e-9)
    assert b["Ex"] == pytest.approx(a["Ex"], rel=1e-9)
    assert np.max(np.abs(b["V"] - a["V"])) <= 1e-9 * np.max(np.abs(a["V"]))
    ga = p.grad_levels(s.D, a["v_levels"])
    gb = q.grad_levels(s.D, b["v_levels"])
    assert np.max(np.abs(gb - ga)) <= 1e-8


def test_skew_gga_energy_derivatives(res_skew):
    # PBE exchange in a triclinic cell: dE/dD = V and the energy gradient against
    # central differences (the Cartesian Fourier derivatives from the reciprocal rows)
    s, p = res_skew
    out = p.fock(s.D, xc="pbe_x")
    rng = np.random.default_rng(4)
    X = rng.standard_normal(s.D.shape)
    X = X + X.T
    h = 1e-5
    fd = (p.energy(s.D + h * X, xc="pbe_x") - p.energy(s.D - h * X, xc="pbe_x")) / (2 * h)
    assert fd == pytest.approx(float(np.sum(X * out["V"])), rel=1e-7)
    g = p.grad_levels(s.D, out["v_levels"])
    h = 1e-4
    for atom, d in [(0, 2), (1, 0)]:
        cp = s.coords.copy()
        cm = s.coords.copy()
        cp[atom, d] += h
        cm[atom, d] -= h
        fd = (p.with_coords(cp).energy(s.D, xc="pbe_x") -
              p.with_coords(cm).energy(s.D, xc="pbe_x")) / (2 * h)
        assert g[atom, d] == pytest.approx(fd, rel=1e-6, abs=1e-7)


def test_sheared_description_gga():
    # PBE exchange of the sheared description against the cubic one (odd meshes, so no
    # Nyquist plane: the two descriptions' derivatives are the same functions)
    s = systems.resolved(seed=7, shells=((0, 1), (1, 1), (2, 1)), natm=2, nlevels=2)
    p = oracle.Plan(s)
    s.meshes = np.array([[oracle._smooth7_even(int(1.6 * m)) + 1 for m in row] for row in p.meshes])
    s.cutoff_ha = 0.0
    s.rel_cutoff = 100.0
    a = oracle.Plan(s).fock(s.D, xc="pbe_x")
    b = oracle.Plan(systems.sheared(s)).fock(s.D, xc="pbe_x")
    assert b["Ex"] == pytest.approx(a["Ex"], rel=1e-9)
    assert b["EH"] == pytest.approx(a["EH"], rel=1e-9)
    assert np.max(np.abs(b["V"] - a["V"])) <= 1e-9 * np.max(np.abs(a["V"]))


def test_skew_tau_closed_forms(res_skew):
    # kinetic-energy density in a triclinic cell: int tau = (1/2) tr(D T) and the tau
    # Fock term of plane waves, against the analytic lattice sums over Cartesian images
    s, p = res_skew
    tl = p.tau_levels(s.D)
    tot = sum(p.omega / t.size * float(np.sum(t)) for t in tl)
    T = cf.lattice_grad_overlap(s, reach=20.0)
    assert tot == pytest.approx(0.5 * float(np.sum(s.D * T)), rel=1e-10)
    waves = workloads.PlaneWaves(s.potential.n[:2], s.potential.a[:2])
    V = p.mat_tau_levels([waves.sample(m) for m in p.meshes])
    ref = 0.5 * cf.lattice_grad_pw_matrix(s, waves, reach=20.0)
    assert np.max(np.abs(V - ref)) <= 1e-9 * np.max(np.abs(ref))


@pytest.mark.parametrize("base", ["triclinic", "cubic"])
def test_rotated_cell_is_the_same_crystal(base):
    # A crystal turned by a seeded rotation Q (lattice rows and atoms), so that no row of
    # the lattice is triangular: with the same fractional meshes every level density on
    # the grid, E_H and E_x are those of the unturned crystal once D is expressed in the
    # turned Cartesian components (D' = M^T D M), V transforms back as V = M V' M^T and
    # the gradient turns with the atoms (g' = g Q^T).  The cubic cell goes through the
    # separable orthorhombic evaluation and its rotation through the point-by-point one.
    if base == "triclinic":
        s = systems.skewed(seed=6, shells=((0, 1), (1, 1), (2, 1), (3, 1)), natm=2)
    else:
        s = systems.resolved(seed=6, shells=((0, 1), (1, 1), (2, 1), (3, 1)), natm=2)
    Q = systems.rotation(12)
    r = systems.rotated(s, Q)
    assert np.all(np.abs(r.lattice[np.triu_indices(3, 1)]) > 1e-3)
    M = systems.basis_rotation(s, Q)
    p, q = oracle.Plan(s), oracle.Plan(r)
    assert np.array_equal(p.meshes, q.meshes)
    Dr = M.T @ s.D @ M
    a, b = p.fock(s.D), q.fock(Dr)
    for x, y in zip(a["rho_levels"], b["rho_levels"]):
        assert np.max(np.abs(x - y)) <= 1e-10 * np.max(np.abs(x))
    assert b["EH"] == pytest.approx(a["EH"], rel=1e-10)
    assert b["Ex"] == pytest.approx(a["Ex"], rel=1e-10)
    assert np.max(np.abs(M @ b["V"] @ M.T - a["V"])) <= 1e-10 * np.max(np.abs(a["V"]))
    ga = p.grad_levels(s.D, a["v_levels"])
    gb = q.grad_levels(Dr, b["v_levels"])
    assert np.max(np.abs(gb - ga @ Q.T)) <= 1e-9 * max(1.0, np.max(np.abs(ga)))


def test_collocation_is_reproducible_bit_for_bit():
    # the oracle sums per-thread grids over a fixed pair-to-thread map
    s = workloads.tiny()
    p = oracle.Plan(s)
    for nt in (1, 3):
        a = p.rho_levels(s.D, nthreads=nt)
        b = p.rho_levels(s.D, nthreads=nt)
        assert all(np.array_equal(x, y) for x, y in zip(a, b))
    t = p.tau_levels(s.D, nthreads=3)
    u = p.tau_levels(s.D, nthreads=3)
    assert all(np.array_equal(x, y) for x, y in zip(t, u))


def test_permuting_atoms_permutes_V_and_gradient():
    # the atoms of a cell listed in another order (shells and D reindexed with them): the
    # same level densities and energies, V and the gradient reindexed (tau small enough
    # that a last-bit change of a pair centre cannot move a box edge across a grid point)
    s = systems.resolved(seed=9, shells=((0, 1), (1, 1), (2, 1)), natm=3).with_tau(1e-14)
    perm = np.array([2, 0, 1])
    r, ao = systems.permuted_atoms(s, perm)
    p, q = oracle.Plan(s), oracle.Plan(r)
    a, b = p.fock(s.D), q.fock(r.D)
    for x, y in zip(a["rho_levels"], b["rho_levels"]):
        assert np.max(np.abs(x - y)) <= 1e-12 * np.max(np.abs(x))
    assert b["EH"] == pytest.approx(a["EH"], rel=1e-12)
    assert b["Ex"] == pytest.approx(a["Ex"], rel=1e-12)
    assert np.max(np.abs(b["V"] - a["V"][np.ix_(ao, ao)])) <= 1e-12 * np.max(np.abs(a["V"]))
    ga = p.grad_levels(s.D, a["v_levels"])
    gb = q.grad_levels(r.D, b["v_levels"])
    assert np.max(np.abs(gb - ga[perm])) <= 1e-11 * max(1.0, np.max(np.abs(ga)))
