"""Autotuner for the launch shape of the grid kernels.

Four knobs decide how the (pair, sub-box) tasks are cut and spread over the GPU:
the collocation sub-box and its warps per thread block, and the integration sub-box (with
its z window: (t0, t1, t2) stages the sub-box itself, (t0, t1, t2, zwin) overlapping
windows of zwin points) and its tasks per work item (how many pair tasks one thread
block takes).  The fastest
setting depends on the workload (pair box sizes against the sub-box, the mix of angular
momenta, tasks per sub-box, one large cell or a batch of small ones), so it is measured:
every candidate is planned, committed and timed with the library's per-phase CUDA-event
timers (gpw_profile) over a few Fock + gradient builds, for one cell (gpw_fock_grad) or
for a batch of cells (gpw_batch_fock_grad_async, one launch per grid pass for all).
Collocation and integration are separate kernels with separate task lists, so their
knobs are tuned one after the other: collocation sub-box, then its warps; integration
sub-box, then its chunk.

Choices are cached in a JSON file keyed by the GPU name and a signature of the workload
(cell sizes, atoms, shells, cutoff, levels, screening threshold), so each workload class
is measured once.  The cache file is GPW_AUTOTUNE_CACHE, else
~/.cache/gpw_autotune.json.
"""
from __future__ import annotations

import hashlib
import json
import os
import tempfile
from dataclasses import asdict, dataclass, field

import numpy as np

from .binding import TILES, TILES_INTEG, TILES_INTEG_ZWIN, Batch, GpwError, Plan

WARPS = (0, 8, 6, 4)             # 0 = the library's occupancy choice
CHUNKS = (0, 64, 256, 1024, 4096)  # 0 = the library's default


@dataclass
class Choice:
    tile: tuple
    tile_integ: tuple
    colloc_warps: int
    integ_chunk: int
    timings: dict = field(default_factory=dict)  # candidate -> ms per build (phase)

    def plan_kwargs(self) -> dict:
        return dict(tile=tuple(self.tile), colloc_warps=int(self.colloc_warps),
                    integ_chunk=int(self.integ_chunk), **integ_kwargs(self.tile_integ))


def integ_kwargs(t) -> dict:
    """Plan arguments of an integration candidate (t0, t1, t2) or (t0, t1, t2, zwin)."""
    t = tuple(int(x) for x in t)
    return dict(tile_integ=t[:3], integ_zwin=t[3] if len(t) > 3 else None)


def signature(systems) -> str:
    """Workload class of a cell or a list of cells (order-independent)."""
    items = []
    for s in systems:
        # the cell by its metric R R^T (so the shape, not the orientation) and whether
        # the rows are axis-aligned (which selects the orthorhombic kernels)
        lat = np.asarray(s.lattice, dtype=np.float64)
        L = [np.round(lat @ lat.T, 6).tolist(), bool(np.all(lat == np.diag(np.diag(lat))))]
        lcount = np.bincount(np.asarray(s.shell_l, dtype=np.int64), minlength=4).tolist()
        items.append(json.dumps([L, int(np.asarray(s.coords).shape[0]), lcount,
                                 int(np.asarray(s.exponents).size), float(s.cutoff_ha),
                                 int(s.nlevels), float(s.level_ratio), float(s.tau),
                                 None if s.meshes is None else np.asarray(s.meshes).tolist()]))
    return hashlib.sha256("\n".join(sorted(items)).encode()).hexdigest()[:24]


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def _cache_path(path=None) -> str:
    return path or os.environ.get("GPW_AUTOTUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "gpw_autotune.json")


def _load_cache(path) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, key, choice: Choice):
    data = _load_cache(path)
    data[key] = asdict(choice)
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=d, prefix=".gpw_autotune")
    with os.fdopen(fd, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def measure_builds(systems, kwargs, steps=2, warmup=1) -> dict:
    """Device milliseconds per Fock + gradient build of the collocation and integration
    passes (gpw_profile phases) for the given plan settings; a list of more than one
    cell is run as one batch."""
    import torch
    plans = [Plan(s, **kwargs) for s in systems]
    try:
        Ds = [torch.as_tensor(np.ascontiguousarray(s.D), device="cuda") for s in systems]
        if len(plans) == 1:
            def run():
                plans[0].fock_grad(Ds[0])
        else:
            batch = Batch(len(plans)).set(plans)
            Vs = [torch.empty((p.nao, p.nao), dtype=torch.float64, device="cuda") for p in plans]
            gs = [torch.empty((p.natm, 3), dtype=torch.float64, device="cuda") for p in plans]
            E = torch.empty(2 * len(plans), dtype=torch.float64, device="cuda")

            def run():
                batch.fock_grad_async(Ds, Vs, gs, E)
        for _ in range(warmup):
            run()
        torch.cuda.synchronize()
        for p in plans:
            p.profile(True)
        for _ in range(steps):
            run()
        torch.cuda.synchronize()
        colloc = integ = 0.0
        for p in plans:
            ms = p.profile_read()["ms"]
            p.profile(False)
            colloc += ms["collocate"]
            integ += ms["integrate_ip1"]
        used = plans[0].stats()
        if len(plans) > 1:
            batch.close()  # its grid passes were timed on the first plan's phase events
        return {"collocate": colloc / steps, "integrate": integ / steps,
                "colloc_warps": used["colloc_warps"], "integ_chunk": used["integ_chunk"]}
    finally:
        for p in plans:
            p.close()
        torch.cuda.empty_cache()


def tune(systems, *, tiles=None, tiles_integ=None, warps=None, chunks=None, steps=2,
         cache_path=None, refresh=False, measure=None) -> Choice:
    """Pick the collocation sub-box and warps and the integration sub-box and chunk for a
    cell (or a list of cells run as one batch).  Uses the cache unless refresh;
    `measure(systems, plan_kwargs) -> {"collocate": ms, "integrate": ms}` may replace the
    GPU measurement."""
    if not isinstance(systems, (list, tuple)):
        systems = [systems]
    tiles = list(tiles or TILES)
    tiles_integ = list(tiles_integ or (TILES_INTEG + TILES_INTEG_ZWIN))
    warps = list(WARPS if warps is None else warps)
    chunks = list(CHUNKS if chunks is None else chunks)
    meas = measure or (lambda ss, kw: measure_builds(ss, kw, steps=steps))
    path = _cache_path(cache_path)
    key = f"{_gpu_name() if measure is None else 'model'}|{signature(systems)}"
    if not refresh:
        hit = _load_cache(path).get(key)
        if hit is not None:
            return Choice(tuple(hit["tile"]), tuple(hit["tile_integ"]), int(hit["colloc_warps"]),
                          int(hit["integ_chunk"]), hit.get("timings", {}))
    timings = {}

    def best(label, cands, phase, make):
        res = {}
        for c in cands:
            try:
                r = meas(systems, make(c))
            except GpwError:  # a shape this workload cannot use (e.g. shared memory)
                continue
            res[c] = float(r[phase])
            timings[f"{label}={c}"] = res[c]
        if not res:
            raise GpwError(-1, "autotune", f"no usable candidate for {label}")
        return min(res, key=res.get)

    tile = best("tile", [tuple(t) for t in tiles], "collocate", lambda t: dict(tile=t))
    nw = best("colloc_warps", warps, "collocate", lambda w: dict(tile=tile, colloc_warps=w))
    ti = best("tile_integ", [tuple(t) for t in tiles_integ], "integrate", integ_kwargs)
    ch = best("integ_chunk", chunks, "integrate",
              lambda c: dict(integ_kwargs(ti), integ_chunk=c))
    choice = Choice(tile, ti, int(nw), int(ch), timings)
    _store(path, key, choice)
    return choice
