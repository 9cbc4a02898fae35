"""Thin ctypes binding of libgpw (include/gpw.h): argument marshalling only.

Every step of the computation runs in libgpw's CUDA kernels and cuFFT on the device.
Tensors are torch tensors on the current CUDA device (float64, contiguous); the
calls are enqueued on torch's current stream.  There is no CPU fallback: loading
fails loudly when the library is missing or cannot be built.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

GPW_MAX_LEVELS = 8
_LOCK = threading.Lock()
_LIB = None

ERRORS = {0: "GPW_OK", -1: "GPW_EINVAL", -2: "GPW_ENOMEM", -3: "GPW_ECUDA", -4: "GPW_ECUFFT",
          -5: "GPW_ETIMEDOUT", -6: "GPW_EDEVICE", -7: "GPW_ERANGE"}

EXPORTS = ["gpw_plan", "gpw_plan_query", "gpw_plan_update_coords", "gpw_plan_pairs",
           "gpw_plan_task_lists",
           "gpw_eval_rho", "gpw_eval_rho_levels", "gpw_eval_mat", "gpw_eval_mat_levels",
           "gpw_eval_mat_ip1", "gpw_eval_mat_ip1_levels", "gpw_eval_tau", "gpw_eval_tau_levels",
           "gpw_eval_mat_tau", "gpw_eval_mat_tau_levels", "gpw_eval_mat_tau_ip1",
           "gpw_eval_mat_tau_ip1_levels", "gpw_plan_destroy_async", "gpw_fock", "gpw_fock_async",
           "gpw_fock_grad", "gpw_fock_grad_async", "gpw_fock_grad_host", "gpw_tile_supported",
           "gpw_integ_zwin_supported",
           "gpw_plan_prepare", "gpw_plan_commit", "gpw_batch_create", "gpw_batch_set",
           "gpw_batch_fock_grad_async", "gpw_batch_generation", "gpw_batch_destroy",
           "gpw_check_device", "gpw_profile", "gpw_profile_read", "gpw_plan_destroy",
           "gpw_stream_wait", "gpw_strerror", "gpw_last_error"]
PHASES = ["coef", "collocate", "spectral", "integrate", "assemble", "integrate_ip1", "grad"]


class GpwError(RuntimeError):
    def __init__(self, code, where, msg):
        super().__init__(f"{where}: {ERRORS.get(code, code)}: {msg}")
        self.code = code


class Desc(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_double * 9), ("natm", ctypes.c_int),
                ("coords", ctypes.c_void_p), ("nshell", ctypes.c_int),
                ("shell_atom", ctypes.c_void_p), ("shell_l", ctypes.c_void_p),
                ("shell_nprim", ctypes.c_void_p), ("shell_prim_off", ctypes.c_void_p),
                ("exponents", ctypes.c_void_p), ("coeffs", ctypes.c_void_p),
                ("cutoff_ha", ctypes.c_double), ("nlevels", ctypes.c_int),
                ("level_ratio", ctypes.c_double), ("meshes", ctypes.c_void_p),
                ("rel_cutoff", ctypes.c_double), ("tau", ctypes.c_double),
                ("flags", ctypes.c_int), ("tile", ctypes.c_int * 3),
                ("tile_integ", ctypes.c_int * 3), ("colloc_warps", ctypes.c_int),
                ("integ_chunk", ctypes.c_int), ("xc", ctypes.c_int),
                ("host_threads", ctypes.c_int), ("integ_zwin", ctypes.c_int)]

GPW_TAU = 1  # gpw_desc.flags: kinetic-energy-density kernels
GPW_HOST_TASKS = 2  # gpw_desc.flags: task records built on the host (default: device)
GPW_FAST_BLOCK_PRUNE = 4  # gpw_desc.flags: per-block value screening of the collocation tasks
GPW_DEBUG_CHECKS = 8  # gpw_desc.flags: task-list validation at commit, finite-output checks

# exchange functionals (gpw_desc.xc)
XC = {"lda_x": 0, "pbe_x": 1}

# sub-box shapes with compiled kernels (gpw_tile_supported): collocation, integration
TILES = [(8, 8, 16), (4, 8, 32), (8, 8, 32), (4, 8, 64), (4, 8, 16), (4, 4, 16), (2, 8, 16),
         (4, 4, 32)]
TILES_INTEG = TILES + [(8, 8, 64), (8, 4, 64)]
# integration sub-boxes with overlapping z windows (gpw_integ_zwin_supported):
# (t0, t1, t2, zwin)
TILES_INTEG_ZWIN = [(8, 8, 16, 48)]


class Info(ctypes.Structure):
    _fields_ = [("nao", ctypes.c_int), ("natm", ctypes.c_int), ("nlevels", ctypes.c_int),
                ("lmax", ctypes.c_int), ("meshes", (ctypes.c_int * 3) * GPW_MAX_LEVELS),
                ("level_cutoff", ctypes.c_double * GPW_MAX_LEVELS),
                ("npairs", ctypes.c_longlong),
                ("npairs_level", ctypes.c_longlong * GPW_MAX_LEVELS),
                ("pair_points", ctypes.c_longlong),
                ("pair_points_level", ctypes.c_longlong * GPW_MAX_LEVELS),
                ("pair_points_L", ctypes.c_longlong * 8), ("nentries", ctypes.c_longlong),
                ("device_bytes", ctypes.c_longlong), ("flops_rho", ctypes.c_double),
                ("flops_mat", ctypes.c_double), ("flops_ip1", ctypes.c_double),
                ("tile", ctypes.c_int * 3), ("tile_integ", ctypes.c_int * 3),
                ("nentries_integ", ctypes.c_longlong), ("colloc_warps", ctypes.c_int),
                ("integ_chunk", ctypes.c_int), ("xc", ctypes.c_int),
                ("volume", ctypes.c_double), ("weight", ctypes.c_double * GPW_MAX_LEVELS),
                ("integ_zwin", ctypes.c_int)]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libgpw.so (building it in-tree with nvcc if absent).  Raises if it cannot."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"libgpw not built: {path}")
            _build.build()
        L = ctypes.CDLL(path)
        vp, ci, cd = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.gpw_plan.argtypes = [ctypes.POINTER(Desc), vp, ctypes.POINTER(vp)]
        L.gpw_plan_query.argtypes = [vp, ctypes.POINTER(Info)]
        L.gpw_plan_update_coords.argtypes = [vp, vp, vp]
        L.gpw_plan_pairs.argtypes = [vp, vp, vp, vp, vp, vp]
        L.gpw_plan_task_lists.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, vp, vp]
        L.gpw_eval_rho.argtypes = [vp, vp, vp, vp]
        L.gpw_eval_rho_levels.argtypes = [vp, vp, vp, vp]
        L.gpw_eval_mat.argtypes = [vp, vp, vp, vp]
        L.gpw_eval_mat_levels.argtypes = [vp, vp, vp, vp]
        L.gpw_eval_mat_ip1.argtypes = [vp, vp, vp, vp, vp]
        L.gpw_eval_mat_ip1_levels.argtypes = [vp, vp, vp, vp, vp]
        L.gpw_eval_tau.argtypes = [vp, vp, vp, vp]
        L.gpw_eval_tau_levels.argtypes = [vp, vp, vp, vp]
        L.gpw_eval_mat_tau.argtypes = [vp, vp, vp, vp]
        L.gpw_eval_mat_tau_levels.argtypes = [vp, vp, vp, vp]
        L.gpw_eval_mat_tau_ip1.argtypes = [vp, vp, vp, vp, vp]
        L.gpw_eval_mat_tau_ip1_levels.argtypes = [vp, vp, vp, vp, vp]
        L.gpw_fock.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.gpw_fock_async.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.gpw_fock_grad.argtypes = [vp, vp, vp, vp, vp, vp]
        L.gpw_fock_grad_async.argtypes = [vp, vp, vp, vp, vp, vp]
        L.gpw_fock_grad_host.argtypes = [vp, vp, vp, vp, vp, vp]
        L.gpw_tile_supported.argtypes = [ci, ci, ci]
        L.gpw_integ_zwin_supported.argtypes = [ci, ci, ci, ci]
        L.gpw_plan_prepare.argtypes = [ctypes.POINTER(Desc), ctypes.POINTER(vp)]
        L.gpw_plan_commit.argtypes = [vp, vp]
        L.gpw_batch_create.argtypes = [ci, ctypes.POINTER(vp)]
        L.gpw_batch_set.argtypes = [vp, ci, vp, vp]
        L.gpw_batch_fock_grad_async.argtypes = [vp, vp, vp, vp, vp, vp]
        L.gpw_batch_destroy.argtypes = [vp]
        L.gpw_batch_generation.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
        L.gpw_stream_wait.argtypes = [vp, cd]
        L.gpw_batch_destroy.restype = None
        L.gpw_check_device.argtypes = [vp, ctypes.POINTER(ci), vp]
        L.gpw_profile.argtypes = [vp, ci]
        L.gpw_profile_read.argtypes = [vp, vp, vp, ci, vp]
        L.gpw_plan_destroy.argtypes = [vp]
        L.gpw_plan_destroy.restype = None
        L.gpw_plan_destroy_async.argtypes = [vp, vp]
        L.gpw_plan_destroy_async.restype = None
        L.gpw_strerror.argtypes = [ci]
        L.gpw_strerror.restype = ctypes.c_char_p
        L.gpw_last_error.argtypes = []
        L.gpw_last_error.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name not in ("gpw_plan_destroy", "gpw_plan_destroy_async", "gpw_strerror",
                            "gpw_last_error", "gpw_batch_destroy"):
                getattr(L, name).restype = ci
        _LIB = L
        return L


def check(rc: int, where: str):
    if rc != 0:
        msg = load().gpw_last_error().decode(errors="replace")
        raise GpwError(rc, where, msg)


def _ptr(t) -> int:
    return int(t.data_ptr()) if t is not None else 0


def _stream(stream=None) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def stream_wait(stream, timeout_s: float) -> bool:
    """Bounded host wait on a CUDA stream (gpw_stream_wait): True once its work so far has
    finished, False when timeout_s passed first (the work keeps running)."""
    rc = load().gpw_stream_wait(ctypes.c_void_p(_stream(stream)), float(timeout_s))
    if rc == -5:
        return False
    check(rc, "gpw_stream_wait")
    return True


def _dev_f64(x, shape=None):
    import torch
    if not isinstance(x, torch.Tensor):
        x = torch.as_tensor(np.asarray(x, dtype=np.float64))
    if x.device.type != "cuda" or x.dtype != torch.float64 or not x.is_contiguous():
        x = x.to(device="cuda", dtype=torch.float64).contiguous()
    if shape is not None and tuple(x.shape) != tuple(shape):
        x = x.reshape(shape)
    return x


class Plan:
    """A libgpw plan for one cell (Sec. II / III A of the paper): screened pairs,
    levels, task lists, grids and FFT plans live on the current CUDA device."""

    def __init__(self, system, stream=None, tile=None, tile_integ=None, commit=True,
                 colloc_warps=None, integ_chunk=None, xc="lda_x", tau=False, host_threads=0,
                 host_tasks=False, fast_prune=False, debug_checks=False, integ_zwin=None):
        """Prepare the plan on the host (screening, levels, task lists) and, unless
        commit=False, commit it to the current device.  An uncommitted plan reports its
        exact device footprint in stats()["device_bytes"].  tile, tile_integ,
        colloc_warps, integ_chunk: launch shape (library defaults if None); xc: exchange
        functional, "lda_x" (Slater) or "pbe_x" (PBE exchange, a GGA); tau: also build the
        kinetic-energy-density (meta-GGA) kernels' data; host_threads: most planner
        threads (0 = all cores); host_tasks: build the sub-box task lists on the host
        instead of on the device at commit (identical lists); fast_prune: leave out of
        the collocation lists the (pair, sub-box) tasks wholly beyond the pair's extent
        (GPW_FAST_BLOCK_PRUNE: tau-sized changes, outside the strict definition);
        debug_checks: validate the task lists at commit and every output for values that
        are not finite (GPW_DEBUG_CHECKS, read with check_device()); integ_zwin: z window
        of the integration sub-boxes tile_integ (a multiple of tile_integ[2]; None = the
        library default)."""
        self._lib = load()
        s = system
        self.system = s
        self._keep = []

        def arr(a, dt):
            a = np.ascontiguousarray(np.asarray(a, dtype=dt))
            self._keep.append(a)
            return a.ctypes.data_as(ctypes.c_void_p)

        d = Desc()
        lat = np.asarray(s.lattice, dtype=np.float64).ravel()
        for i in range(9):
            d.lattice[i] = float(lat[i])
        d.natm = int(s.coords.shape[0])
        d.coords = arr(s.coords, np.float64)
        d.nshell = int(len(s.shell_l))
        d.shell_atom = arr(s.shell_atom, np.int32)
        d.shell_l = arr(s.shell_l, np.int32)
        d.shell_nprim = arr(s.shell_nprim, np.int32)
        d.shell_prim_off = arr(s.shell_prim_off, np.int32)
        d.exponents = arr(s.exponents, np.float64)
        d.coeffs = arr(s.coeffs, np.float64)
        d.cutoff_ha = float(s.cutoff_ha)
        d.nlevels = int(s.nlevels)
        d.level_ratio = float(s.level_ratio)
        d.meshes = arr(s.meshes, np.int32) if s.meshes is not None else None
        d.rel_cutoff = float(s.rel_cutoff)
        d.tau = float(s.tau)
        d.flags = ((GPW_TAU if tau else 0) | (GPW_HOST_TASKS if host_tasks else 0) |
                   (GPW_FAST_BLOCK_PRUNE if fast_prune else 0) |
                   (GPW_DEBUG_CHECKS if debug_checks else 0))
        if tile is not None:
            for i in range(3):
                d.tile[i] = int(tile[i])
        if tile_integ is not None:
            for i in range(3):
                d.tile_integ[i] = int(tile_integ[i])
        d.colloc_warps = int(colloc_warps or 0)
        d.integ_chunk = int(integ_chunk or 0)
        d.integ_zwin = int(integ_zwin or 0)
        if xc not in XC:
            raise ValueError(f"unknown exchange functional {xc!r} (one of {sorted(XC)})")
        d.xc = XC[xc]
        d.host_threads = int(host_threads)
        h = ctypes.c_void_p()
        check(self._lib.gpw_plan_prepare(ctypes.byref(d), ctypes.byref(h)), "gpw_plan_prepare")
        self._h = h
        self._keep = []
        self.committed = False
        self._query()
        if commit:
            self.commit(stream)

    def _query(self):
        info = Info()
        check(self._lib.gpw_plan_query(self._h, ctypes.byref(info)), "gpw_plan_query")
        self.info = info
        self.nao = info.nao
        self.natm = info.natm
        self.nlevels = info.nlevels
        self.meshes = [tuple(info.meshes[k][i] for i in range(3)) for k in range(info.nlevels)]
        self.fine_mesh = self.meshes[0]

    def commit(self, stream=None):
        """Allocate and upload the plan on the current device (gpw_plan_commit)."""
        import torch
        if self.committed:
            return self
        torch.cuda.init()
        check(self._lib.gpw_plan_commit(self._h, ctypes.c_void_p(_stream(stream))), "gpw_plan_commit")
        self.committed = True
        self._query()
        return self

    # -- housekeeping -------------------------------------------------------
    def close(self, stream=None):
        """Release the plan.  With a stream: in stream order on it, without synchronising
        the device (all work using the plan must have finished or be ordered before it)."""
        if getattr(self, "_h", None) is not None and self._h.value:
            if stream is None:
                self._lib.gpw_plan_destroy(self._h)
            else:
                self._lib.gpw_plan_destroy_async(self._h, ctypes.c_void_p(_stream(stream)))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stats(self) -> dict:
        i = self.info
        return dict(nao=i.nao, natm=i.natm, nlevels=i.nlevels, lmax=i.lmax,
                    meshes=self.meshes, npairs=i.npairs,
                    npairs_level=[i.npairs_level[k] for k in range(i.nlevels)],
                    pair_points=i.pair_points,
                    pair_points_level=[i.pair_points_level[k] for k in range(i.nlevels)],
                    pair_points_L=[i.pair_points_L[l] for l in range(8)],
                    nentries=i.nentries, device_bytes=i.device_bytes,
                    flops_rho=i.flops_rho, flops_mat=i.flops_mat, flops_ip1=i.flops_ip1,
                    level_cutoff=[i.level_cutoff[k] for k in range(i.nlevels)],
                    tile=tuple(i.tile), tile_integ=tuple(i.tile_integ),
                    integ_zwin=i.integ_zwin,
                    nentries_integ=i.nentries_integ, colloc_warps=i.colloc_warps,
                    integ_chunk=i.integ_chunk,
                    xc={v: k for k, v in XC.items()}.get(i.xc, i.xc),
                    volume=i.volume, weight=[i.weight[k] for k in range(i.nlevels)])

    def task_lists(self, integ: bool = False):
        """One task list of the committed plan (gpw_plan_task_lists): the task records
        (nent x 8 int32), the sub-box CSR offsets (nsub + 1) and the work items
        (nwork x 4 int32)."""
        n, ns, nw = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        it = 1 if integ else 0
        check(self._lib.gpw_plan_task_lists(self._h, it, ctypes.byref(n), ctypes.byref(ns),
                                            ctypes.byref(nw), None, None, None),
              "gpw_plan_task_lists")
        tasks = np.zeros((n.value, 8), np.int32)
        sub = np.zeros(ns.value + 1, np.int64)
        work = np.zeros((nw.value, 4), np.int32)
        P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        check(self._lib.gpw_plan_task_lists(self._h, it, ctypes.byref(n), ctypes.byref(ns),
                                            ctypes.byref(nw), P(tasks), P(sub), P(work)),
              "gpw_plan_task_lists")
        return tasks, sub, work

    def pair_table(self, sort: bool = True) -> np.ndarray:
        """Screened pairs as int64 rows (a, b, n0, n1, n2, level, lo0..2, hi0..2),
        sorted lexicographically (sort=False: in the plan's pair order, the pair index of
        the task records)."""
        n = int(self.info.npairs)
        ab = np.zeros((n, 2), np.int32)
        img = np.zeros((n, 3), np.int32)
        lev = np.zeros(n, np.int32)
        lo = np.zeros((n, 3), np.int32)
        hi = np.zeros((n, 3), np.int32)
        P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        check(self._lib.gpw_plan_pairs(self._h, P(ab), P(img), P(lev), P(lo), P(hi)), "gpw_plan_pairs")
        t = np.concatenate([ab, img, lev[:, None], lo, hi], axis=1).astype(np.int64)
        return t[np.lexsort(t[:, ::-1].T)] if sort else t

    def update_coords(self, coords, stream=None):
        c = np.ascontiguousarray(np.asarray(coords, dtype=np.float64))
        check(self._lib.gpw_plan_update_coords(self._h, c.ctypes.data_as(ctypes.c_void_p),
                                               ctypes.c_void_p(_stream(stream))),
              "gpw_plan_update_coords")

    def check_device(self, stream=None) -> int:
        code = ctypes.c_int(0)
        rc = self._lib.gpw_check_device(self._h, ctypes.byref(code), ctypes.c_void_p(_stream(stream)))
        if rc not in (0, -6):
            check(rc, "gpw_check_device")
        return int(code.value)

    def profile(self, enable: bool = True):
        """Start (clearing totals) or stop per-phase CUDA-event timing of later calls."""
        check(self._lib.gpw_profile(self._h, 1 if enable else 0), "gpw_profile")

    def profile_read(self) -> dict:
        """Per-phase summed device milliseconds and interval counts, plus the number of
        libgpw kernels launched on this plan so far."""
        n = len(PHASES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_longlong * n)()
        launches = ctypes.c_longlong(0)
        check(self._lib.gpw_profile_read(self._h, ms, cnt, n, ctypes.byref(launches)),
              "gpw_profile_read")
        return dict(ms={PHASES[i]: ms[i] for i in range(n)},
                    count={PHASES[i]: cnt[i] for i in range(n)}, launches=int(launches.value))

    def launches(self) -> int:
        launches = ctypes.c_longlong(0)
        check(self._lib.gpw_profile_read(self._h, None, None, 0, ctypes.byref(launches)),
              "gpw_profile_read")
        return int(launches.value)

    # -- evaluations (device tensors) ----------------------------------------
    def _levels_out(self, dtype=None):
        import torch
        return [torch.empty(m, dtype=torch.float64, device="cuda") for m in self.meshes]

    def eval_rho(self, D, out=None, stream=None):
        import torch
        D = _dev_f64(D, (self.nao, self.nao))
        if out is None:
            out = torch.empty(self.fine_mesh, dtype=torch.float64, device="cuda")
        check(self._lib.gpw_eval_rho(self._h, _ptr(D), _ptr(out), _stream(stream)), "gpw_eval_rho")
        return out

    def eval_rho_levels(self, D, stream=None):
        D = _dev_f64(D, (self.nao, self.nao))
        outs = self._levels_out()
        ptrs = (ctypes.c_void_p * len(outs))(*[_ptr(o) for o in outs])
        check(self._lib.gpw_eval_rho_levels(self._h, _ptr(D), ptrs, _stream(stream)),
              "gpw_eval_rho_levels")
        return outs

    def eval_mat(self, v_fine, out=None, stream=None):
        import torch
        v = _dev_f64(v_fine, self.fine_mesh)
        if out is None:
            out = torch.empty((self.nao, self.nao), dtype=torch.float64, device="cuda")
        check(self._lib.gpw_eval_mat(self._h, _ptr(v), _ptr(out), _stream(stream)), "gpw_eval_mat")
        return out

    def eval_mat_levels(self, v_levels, out=None, stream=None):
        import torch
        vs = [_dev_f64(v, m) for v, m in zip(v_levels, self.meshes)]
        if out is None:
            out = torch.empty((self.nao, self.nao), dtype=torch.float64, device="cuda")
        ptrs = (ctypes.c_void_p * len(vs))(*[_ptr(v) for v in vs])
        check(self._lib.gpw_eval_mat_levels(self._h, ptrs, _ptr(out), _stream(stream)),
              "gpw_eval_mat_levels")
        return out

    def eval_mat_ip1(self, D, v_fine, out=None, stream=None):
        import torch
        D = _dev_f64(D, (self.nao, self.nao))
        v = _dev_f64(v_fine, self.fine_mesh)
        if out is None:
            out = torch.empty((self.natm, 3), dtype=torch.float64, device="cuda")
        check(self._lib.gpw_eval_mat_ip1(self._h, _ptr(D), _ptr(v), _ptr(out), _stream(stream)),
              "gpw_eval_mat_ip1")
        return out

    def eval_mat_ip1_levels(self, D, v_levels, out=None, stream=None):
        import torch
        D = _dev_f64(D, (self.nao, self.nao))
        vs = [_dev_f64(v, m) for v, m in zip(v_levels, self.meshes)]
        if out is None:
            out = torch.empty((self.natm, 3), dtype=torch.float64, device="cuda")
        ptrs = (ctypes.c_void_p * len(vs))(*[_ptr(v) for v in vs])
        check(self._lib.gpw_eval_mat_ip1_levels(self._h, _ptr(D), ptrs, _ptr(out), _stream(stream)),
              "gpw_eval_mat_ip1_levels")
        return out

    # -- kinetic energy density (meta-GGA; plans built with tau=True) ----------
    def eval_tau(self, D, out=None, stream=None):
        import torch
        D = _dev_f64(D, (self.nao, self.nao))
        if out is None:
            out = torch.empty(self.fine_mesh, dtype=torch.float64, device="cuda")
        check(self._lib.gpw_eval_tau(self._h, _ptr(D), _ptr(out), _stream(stream)), "gpw_eval_tau")
        return out

    def eval_tau_levels(self, D, stream=None):
        D = _dev_f64(D, (self.nao, self.nao))
        outs = self._levels_out()
        ptrs = (ctypes.c_void_p * len(outs))(*[_ptr(o) for o in outs])
        check(self._lib.gpw_eval_tau_levels(self._h, _ptr(D), ptrs, _stream(stream)),
              "gpw_eval_tau_levels")
        return outs

    def eval_mat_tau(self, v_fine, out=None, stream=None):
        import torch
        v = _dev_f64(v_fine, self.fine_mesh)
        if out is None:
            out = torch.empty((self.nao, self.nao), dtype=torch.float64, device="cuda")
        check(self._lib.gpw_eval_mat_tau(self._h, _ptr(v), _ptr(out), _stream(stream)),
              "gpw_eval_mat_tau")
        return out

    def eval_mat_tau_levels(self, v_levels, out=None, stream=None):
        import torch
        vs = [_dev_f64(v, m) for v, m in zip(v_levels, self.meshes)]
        if out is None:
            out = torch.empty((self.nao, self.nao), dtype=torch.float64, device="cuda")
        ptrs = (ctypes.c_void_p * len(vs))(*[_ptr(v) for v in vs])
        check(self._lib.gpw_eval_mat_tau_levels(self._h, ptrs, _ptr(out), _stream(stream)),
              "gpw_eval_mat_tau_levels")
        return out

    def eval_mat_tau_ip1(self, D, v_fine, out=None, stream=None):
        import torch
        D = _dev_f64(D, (self.nao, self.nao))
        v = _dev_f64(v_fine, self.fine_mesh)
        if out is None:
            out = torch.empty((self.natm, 3), dtype=torch.float64, device="cuda")
        check(self._lib.gpw_eval_mat_tau_ip1(self._h, _ptr(D), _ptr(v), _ptr(out),
                                             _stream(stream)), "gpw_eval_mat_tau_ip1")
        return out

    def eval_mat_tau_ip1_levels(self, D, v_levels, out=None, stream=None):
        import torch
        D = _dev_f64(D, (self.nao, self.nao))
        vs = [_dev_f64(v, m) for v, m in zip(v_levels, self.meshes)]
        if out is None:
            out = torch.empty((self.natm, 3), dtype=torch.float64, device="cuda")
        ptrs = (ctypes.c_void_p * len(vs))(*[_ptr(v) for v in vs])
        check(self._lib.gpw_eval_mat_tau_ip1_levels(self._h, _ptr(D), ptrs, _ptr(out),
                                                    _stream(stream)), "gpw_eval_mat_tau_ip1_levels")
        return out

    def fock(self, D, want_rho=False, want_v=False, stream=None):
        """One Fock build.  Returns dict(V, EH, Ex[, rho, v]) (energies as floats)."""
        import torch
        D = _dev_f64(D, (self.nao, self.nao))
        V = torch.empty((self.nao, self.nao), dtype=torch.float64, device="cuda")
        rho = torch.empty(self.fine_mesh, dtype=torch.float64, device="cuda") if want_rho else None
        v = torch.empty(self.fine_mesh, dtype=torch.float64, device="cuda") if want_v else None
        e = (ctypes.c_double * 2)()
        check(self._lib.gpw_fock(self._h, _ptr(D), _ptr(V), e, _ptr(rho), _ptr(v), _stream(stream)),
              "gpw_fock")
        out = dict(V=V, EH=float(e[0]), Ex=float(e[1]))
        if want_rho:
            out["rho"] = rho
        if want_v:
            out["v"] = v
        return out

    def fock_grad_host(self, D_host, out=None, stream=None):
        """End-to-end Fock build plus Hxc gradient from HOST memory through the C ABI
        (gpw_fock_grad_host: D copied in, the build on the stream, V, the gradient and the
        two energies copied back, synchronised).  D_host: a contiguous float64 host tensor
        (pinned for full-rate copies).  Returns dict(V, grad, E) of host tensors."""
        import torch
        if out is None:
            out = dict(V=torch.empty((self.nao, self.nao), dtype=torch.float64, pin_memory=True),
                       grad=torch.empty((self.natm, 3), dtype=torch.float64, pin_memory=True),
                       E=torch.empty(2, dtype=torch.float64, pin_memory=True))
        for t in (D_host, out["V"], out["grad"], out["E"]):
            if t.device.type != "cpu" or t.dtype != torch.float64 or not t.is_contiguous():
                raise ValueError("fock_grad_host takes contiguous float64 host tensors")
        check(self._lib.gpw_fock_grad_host(self._h, _ptr(D_host), _ptr(out["V"]), _ptr(out["grad"]),
                                           _ptr(out["E"]), _stream(stream)), "gpw_fock_grad_host")
        return out

    def fock_grad(self, D, stream=None):
        """Fock build and Hxc gradient in one pass (gpw_fock_grad).
        Returns dict(V, grad, EH, Ex)."""
        import torch
        D = _dev_f64(D, (self.nao, self.nao))
        V = torch.empty((self.nao, self.nao), dtype=torch.float64, device="cuda")
        g = torch.empty((self.natm, 3), dtype=torch.float64, device="cuda")
        e = (ctypes.c_double * 2)()
        check(self._lib.gpw_fock_grad(self._h, _ptr(D), _ptr(V), _ptr(g), e, _stream(stream)),
              "gpw_fock_grad")
        return dict(V=V, grad=g, EH=float(e[0]), Ex=float(e[1]))

    def fock_grad_async(self, D, V, grad, energies, stream=None):
        """Enqueue gpw_fock_grad_async: V, grad and energies (device, 2 doubles)."""
        check(self._lib.gpw_fock_grad_async(self._h, _ptr(D), _ptr(V), _ptr(grad), _ptr(energies),
                                            _stream(stream)), "gpw_fock_grad_async")

    def fock_async(self, D, V, energies, rho=None, v=None, stream=None):
        """Enqueue a Fock build writing V and energies (device, 2 doubles) only."""
        check(self._lib.gpw_fock_async(self._h, _ptr(D), _ptr(V), _ptr(energies), _ptr(rho),
                                       _ptr(v), _stream(stream)), "gpw_fock_async")


class Batch:
    """Several committed plans whose collocation and integration tasks run in one launch
    each (gpw_batch_*).  set() attaches plans; fock_grad_async() enqueues one Fock build
    plus gradient for every plan without allocating or synchronising."""

    def __init__(self, max_plans: int):
        self._lib = load()
        h = ctypes.c_void_p()
        check(self._lib.gpw_batch_create(int(max_plans), ctypes.byref(h)), "gpw_batch_create")
        self._h = h
        self.max_plans = int(max_plans)
        self.plans = []

    def set(self, plans, stream=None):
        arr = (ctypes.c_void_p * len(plans))(*[p._h.value for p in plans])
        check(self._lib.gpw_batch_set(self._h, len(plans), arr, ctypes.c_void_p(_stream(stream))),
              "gpw_batch_set")
        self.plans = list(plans)
        return self

    @property
    def generation(self) -> int:
        """Successful set() calls so far: a CUDA graph captured from fock_grad_async is
        valid only while this is unchanged (gpw_batch_generation)."""
        g = ctypes.c_longlong()
        check(self._lib.gpw_batch_generation(self._h, ctypes.byref(g)), "gpw_batch_generation")
        return int(g.value)

    def fock_grad_async(self, Ds, Vs, grads, energies, stream=None):
        n = len(self.plans)
        P = lambda ts: (ctypes.c_void_p * n)(*[_ptr(t) for t in ts])
        g = P(grads) if grads is not None else None
        check(self._lib.gpw_batch_fock_grad_async(self._h, P(Ds), P(Vs), g, _ptr(energies),
                                                  ctypes.c_void_p(_stream(stream))),
              "gpw_batch_fock_grad_async")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.gpw_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
