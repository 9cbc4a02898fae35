"""The host planner of libgpw (gpw_plan_prepare: screening, levels, boxes, task counts)
on the CPU, no GPU needed: integer pair tables identical to the oracle's independent
screening, the work counts it reports, and the validation of plan descriptions."""
import numpy as np
import pytest

import oracle
import workloads
import systems
from paper_2603_24881_gb300 import binding
from paper_2603_24881_gb300.binding import GpwError


@pytest.fixture(scope="module")
def lib():
    return binding.load()


@pytest.mark.parametrize("name", ["tiny", "tiny14", "resolved", "water4", "water32", "skewed",
                                  "sheared", "water4_triclinic"])
def test_pair_table_and_counts_match_oracle(lib, name):
    s = {"tiny": workloads.tiny, "tiny14": systems.tiny14, "resolved": systems.resolved,
         "water4": lambda: workloads.config("water4"),
         "water32": lambda: workloads.config("water32"),
         "skewed": systems.skewed,
         "sheared": lambda: systems.sheared(systems.resolved(seed=7)),
         "water4_triclinic": lambda: workloads.config("water4_triclinic")}[name]()
    p = binding.Plan(s, commit=False)
    op = oracle.Plan(s)
    a, b = p.pair_table(), op.pair_table()
    assert a.shape == b.shape and np.array_equal(a, b), name
    st = p.stats()
    assert st["npairs"] == op.npairs and st["pair_points"] == op.pair_points()
    assert [tuple(m) for m in st["meshes"]] == [tuple(m) for m in op.meshes.tolist()]
    # model FLOPs: 2 (L+1) per pair-point for rho, 2 (L+2) for the degree-(L+1) pass
    pts_L = st["pair_points_L"]
    assert st["flops_rho"] == pytest.approx(sum(2.0 * (L + 1) * n for L, n in enumerate(pts_L)))
    assert st["flops_ip1"] == pytest.approx(sum(2.0 * (L + 2) * n for L, n in enumerate(pts_L)))
    assert st["device_bytes"] > 0 and not p.committed
    p.close()
    # the host-built task lists (GPW_HOST_TASKS) count the same tasks as the per-pair
    # counts the device build starts from
    h = binding.Plan(s, commit=False, host_tasks=True)
    sh = h.stats()
    h.close()
    for k in ("nentries", "nentries_integ", "integ_chunk", "npairs", "pair_points"):
        assert sh[k] == st[k], (name, k)


def test_plan_independent_of_thread_count(lib, monkeypatch):
    # the planner threads over pairs for large cells; its result must not depend on it
    s = workloads.config("water32")
    p1 = binding.Plan(s, commit=False)
    t1, st1 = p1.pair_table(), p1.stats()
    p1.close()
    import ctypes.util
    omp = ctypes.CDLL(ctypes.util.find_library("gomp") or "libgomp.so.1")
    omp.omp_set_num_threads(1)
    try:
        p2 = binding.Plan(s, commit=False)
        t2, st2 = p2.pair_table(), p2.stats()
        p2.close()
    finally:
        import os
        omp.omp_set_num_threads(os.cpu_count() or 1)
    p3 = binding.Plan(s, commit=False, host_threads=2)  # the per-plan cap of a server
    t3, st3 = p3.pair_table(), p3.stats()
    p3.close()
    assert np.array_equal(t1, t2) and np.array_equal(t1, t3)
    for k in ("nentries", "nentries_integ", "integ_chunk", "device_bytes", "pair_points"):
        assert st1[k] == st2[k] == st3[k], k


def _expect_error(s, **kw):
    with pytest.raises((GpwError, ValueError)):
        binding.Plan(s, commit=False, **kw)


def test_validation(lib):
    s = workloads.tiny()
    _expect_error(s, tile=(3, 8, 16))                 # no kernels for this shape
    _expect_error(s, tile=(8, 8, 64))                 # integration-only shape
    _expect_error(s, colloc_warps=5)
    _expect_error(s, xc="b88")
    _expect_error(s, host_threads=-1)
    sk = systems.skewed()
    binding.Plan(sk, commit=False).close()           # a triclinic cell plans (LDA, PBE, tau)
    binding.Plan(sk, commit=False, xc="pbe_x").close()
    binding.Plan(systems.skewed(shells=((0, 1), (2, 1))), commit=False, tau=True).close()
    _expect_error(sk, tile=(8, 8, 32))                # and the 4x8x16 sub-boxes
    # integration z windows: only for shapes compiled with them, and only with an
    # explicit tile_integ; non-orthogonal cells keep plain windows
    _expect_error(s, tile_integ=(8, 8, 16), integ_zwin=32)
    _expect_error(s, tile_integ=(8, 8, 32), integ_zwin=48)
    _expect_error(s, integ_zwin=48)
    _expect_error(sk, tile_integ=(8, 8, 16), integ_zwin=48)
    binding.Plan(s, commit=False, tile_integ=(8, 8, 16), integ_zwin=48).close()
    binding.Plan(s, commit=False, tile_integ=(8, 8, 16), integ_zwin=16).close()
    flat = sk.with_tau(sk.tau)
    flat.lattice = np.array([[6.0, 0.0, 0.0], [6.0, 0.0, 0.0], [0.0, 0.0, 6.0]])
    _expect_error(flat)                               # dependent rows
    bad = s.with_tau(s.tau)
    bad.lattice = bad.lattice.copy()
    bad.lattice[1, 1] = -bad.lattice[1, 1]            # negative length of an orthorhombic cell
    _expect_error(bad)
    neg = s.with_tau(s.tau)
    neg.exponents = -np.abs(neg.exponents)            # exponents must be positive
    _expect_error(neg)
    f = systems.resolved(seed=8, shells=((0, 1), (3, 1)), natm=2)
    binding.Plan(f, commit=False).close()             # f shells are fine,
    binding.Plan(f, commit=False, tau=True).close()   # also for the tau kernels
    # the opt-in flags plan; an unknown flag bit does not
    binding.Plan(s, commit=False, fast_prune=True, debug_checks=True).close()
    binding.Plan(sk, commit=False, fast_prune=True).close()


def test_tau_plan_sizes(lib):
    # GPW_TAU plans carry tables to degree L+3 and larger per-pair buffers
    s = workloads.tiny()
    a = binding.Plan(s, commit=False).stats()["device_bytes"]
    b = binding.Plan(s, commit=False, tau=True).stats()["device_bytes"]
    assert b > a


@pytest.mark.parametrize("name", ["water32", "many_primitives"])
def test_pair_order_is_shell_pair_primitives_image(lib, name):
    # the plan's own pair order (the pair index of the task records) is by contracted
    # shell pair, then primitives, then image; the 17-primitive shell takes the planner's
    # general sort instead of its packed 64-bit keys, and both give that order and the
    # oracle's pair set
    s = (workloads.config("water32") if name == "water32" else
         systems.resolved(seed=3, shells=((0, 17), (1, 2)), natm=2, tau=1e-8))
    p = binding.Plan(s, commit=False)
    t = p.pair_table(sort=False)
    p.close()
    sh = oracle.primitives(s)["shell"]
    key = np.column_stack([sh[t[:, 0]], sh[t[:, 1]], t[:, 0], t[:, 1], t[:, 2], t[:, 3], t[:, 4]])
    order = np.lexsort(key[:, ::-1].T)
    assert np.array_equal(order, np.arange(len(t)))
    ref = oracle.Plan(s).pair_table()
    assert np.array_equal(t[np.lexsort(t[:, ::-1].T)], ref)


def _pieces(lo, hi, N, T, W):
    """Segments of the unwrapped grid range [lo, hi] along an axis of N points with
    sub-boxes of T whose windows span W points from their start (W = T: plain tiling):
    each segment runs from where the previous one ended to the end of the window of the
    sub-box it starts in (clipped at the period)."""
    n, i = 0, lo
    while i <= hi:
        k = i // N
        j = (i - k * N) // T
        i = k * N + min(j * T + W, N)
        n += 1
    return n


@pytest.mark.parametrize("name,kw,win", [
    ("water4", {}, (8, 8, 16, 48)),                                   # the default
    ("water4", dict(tile_integ=(8, 8, 16), integ_zwin=48), (8, 8, 16, 48)),
    ("water4", dict(tile_integ=(8, 8, 32)), (8, 8, 32, 32)),
    ("tiny", {}, (8, 8, 16, 48)),                                     # windows clipped at N
    ("water4_triclinic", {}, (4, 8, 16, 16)),                         # plain 4x8x16
])
def test_integration_task_count_follows_the_windows(lib, name, kw, win):
    # the planner's integration task count is the product over the three axes of the
    # segments each pair box is cut into, counted here from the pair table alone
    s = workloads.config(name) if name != "tiny" else workloads.tiny()
    p = binding.Plan(s, commit=False, **kw)
    st = p.stats()
    assert tuple(st["tile_integ"]) + (st["integ_zwin"],) == win
    t = p.pair_table(sort=False)
    T0, T1, T2, W2 = win
    want = 0
    for r in t:
        N = st["meshes"][r[5]]
        want += (_pieces(r[6], r[9], N[0], T0, T0) * _pieces(r[7], r[10], N[1], T1, T1) *
                 _pieces(r[8], r[11], N[2], T2, W2))
    assert st["nentries_integ"] == want
    # and the collocation lists are plain 4x8x16 sub-boxes
    T = st["tile"]
    want_c = sum(_pieces(r[6], r[9], st["meshes"][r[5]][0], T[0], T[0]) *
                 _pieces(r[7], r[10], st["meshes"][r[5]][1], T[1], T[1]) *
                 _pieces(r[8], r[11], st["meshes"][r[5]][2], T[2], T[2]) for r in t)
    assert st["nentries"] == want_c
    p.close()
