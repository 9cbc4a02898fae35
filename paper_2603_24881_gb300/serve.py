"""Continuous-batching server for Fock builds (and Hxc gradients) of many cells.

Requests (a cell + its density matrix, optionally asking for the gradient) arrive at any
time.  Each one is planned on a host thread (gpw_plan_prepare: screening and task lists
on the CPU, which also yields the exact device footprint).  A GPU thread admits prepared
requests in arrival order while their footprints fit the device-memory budget, commits
their plans, and launches them together as one batch (gpw_batch_fock_grad_async: one
collocation and one integration launch for all cells of the batch).  Up to `streams`
batches are in flight at once on separate CUDA streams, so requests that arrive while
others run are admitted into the next batch as soon as slots and memory free up, and
their work overlaps on the device.  Each request's plan, pair lists and grids stay on the
device until its result has been copied back; then the memory is released.

Per-request results are those of the request run alone (the same tasks, in the same
order per sub-box, with the same reductions); the tests check this within the stated
tolerances.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import os
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from .binding import Batch, Plan


@dataclass
class Result:
    rid: int
    EH: float
    Ex: float
    V: np.ndarray
    grad: np.ndarray | None
    t_submit: float
    t_done: float
    batch: int
    batch_size: int
    t_prepared: float = 0.0  # host planning finished
    t_launch: float = 0.0    # its batch was enqueued on the GPU

    @property
    def latency(self) -> float:
        return self.t_done - self.t_submit


@dataclass
class _Req:
    rid: int
    system: object
    want_grad: bool
    future: cf.Future
    t_submit: float
    plan: Plan | None = None
    bytes: int = 0
    error: BaseException | None = None
    t_prepared: float = 0.0
    t_launch: float = 0.0


@dataclass
class _Flight:
    bid: int
    reqs: list
    stream: object
    event: object
    bufs: dict
    batch: Batch
    nbytes: int


class Server:
    """Continuous-batching Fock/gradient server on one GPU.

    hbm_budget: device bytes the plans and buffers of admitted requests may use at once
    (default: 70% of the free device memory at start).  max_batch: most requests per
    batch.  streams: batches in flight.  host_workers: planning threads.  tile,
    tile_integ, colloc_warps, integ_chunk: launch shape of every plan (library defaults
    if None); tune_with: a list of sample cells to run the autotuner on (as one batch)
    instead, its choice (cached per GPU and workload class) then serves every request.
    """

    def __init__(self, hbm_budget: int | None = None, max_batch: int = 32, streams: int = 2,
                 host_workers: int | None = None, tile=None, tile_integ=None,
                 colloc_warps=None, integ_chunk=None, tune_with=None, fail_prepare=None):
        import torch
        self.torch = torch
        torch.cuda.init()
        free, _ = torch.cuda.mem_get_info()
        self.budget = int(hbm_budget if hbm_budget is not None else 0.7 * free)
        self.max_batch = int(max_batch)
        self.plan_kwargs = dict(tile=tile, tile_integ=tile_integ, colloc_warps=colloc_warps,
                                integ_chunk=integ_chunk)
        self.choice = None
        if tune_with:
            from .autotune import tune
            self.choice = tune(list(tune_with))
            self.plan_kwargs = self.choice.plan_kwargs()
        self._fail_prepare = fail_prepare  # test hook: callable(system) -> bool
        self._pool = cf.ThreadPoolExecutor(host_workers or max(2, (os.cpu_count() or 4)))
        self._streams = [torch.cuda.Stream() for _ in range(max(1, streams))]
        self._batches = [Batch(self.max_batch) for _ in self._streams]
        self._ready = collections.deque()
        self._flights: list[_Flight] = []
        self._used = 0
        self._rid = 0
        self._bid = 0
        self._cv = threading.Condition()
        self._stop = False
        self.stats = dict(batches=0, admitted=0, rejected=0, max_in_flight=0, peak_bytes=0)
        self._gpu = threading.Thread(target=self._gpu_loop, name="gpw-serve", daemon=True)
        self._gpu.start()

    # ------------------------------------------------------------------ API --
    def submit(self, system, want_grad: bool = False) -> cf.Future:
        """Queue one Fock build (plus gradient if want_grad); returns a Future[Result]."""
        fut: cf.Future = cf.Future()
        with self._cv:
            rid = self._rid
            self._rid += 1
        req = _Req(rid, system, bool(want_grad), fut, time.perf_counter())
        self._pool.submit(self._prepare, req)
        return fut

    def close(self):
        """Finish every submitted request, then stop."""
        self._pool.shutdown(wait=True)  # all preparations have reached the ready queue
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        self._gpu.join()
        for b in self._batches:
            b.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------- host side --
    def _prepare(self, req: _Req):
        try:
            if self._fail_prepare and self._fail_prepare(req.system):
                raise RuntimeError("plan preparation failed (injected)")
            req.plan = Plan(req.system, commit=False, **self.plan_kwargs)
            nao, natm = req.plan.nao, req.plan.natm
            req.bytes = int(req.plan.stats()["device_bytes"]) + 8 * (2 * nao * nao + 3 * natm + 2)
            if req.bytes > self.budget:
                raise MemoryError(f"request needs {req.bytes} device bytes, budget is {self.budget}")
        except BaseException as ex:  # the request fails alone; the server keeps serving
            req.error = ex
        req.t_prepared = time.perf_counter()
        with self._cv:
            self._ready.append(req)
            self._cv.notify_all()

    # -------------------------------------------------------------- GPU side --
    def _admit(self):
        """Take prepared requests in arrival order while they fit the memory budget."""
        out = []
        while self._ready and len(out) < self.max_batch:
            req = self._ready[0]
            if req.error is not None:
                self._ready.popleft()
                self.stats["rejected"] += 1
                req.future.set_exception(req.error)
                continue
            if self._used + req.bytes > self.budget and (out or self._flights):
                break
            self._ready.popleft()
            self._used += req.bytes
            out.append(req)
        return out

    def _launch(self, reqs, slot: int):
        torch = self.torch
        stream = self._streams[slot]
        batch = self._batches[slot]
        bufs = dict(D=[], V=[], g=[], E=None)
        t = time.perf_counter()
        for r in reqs:
            r.t_launch = t
        with torch.cuda.stream(stream):
            for r in reqs:
                r.plan.commit(stream)
                bufs["D"].append(torch.as_tensor(np.ascontiguousarray(r.system.D), device="cuda"))
                bufs["V"].append(torch.empty((r.plan.nao, r.plan.nao), dtype=torch.float64, device="cuda"))
                bufs["g"].append(torch.empty((r.plan.natm, 3), dtype=torch.float64, device="cuda")
                                 if r.want_grad else None)
            bufs["E"] = torch.empty(2 * len(reqs), dtype=torch.float64, device="cuda")
            batch.set([r.plan for r in reqs], stream)
            batch.fock_grad_async(bufs["D"], bufs["V"], bufs["g"], bufs["E"], stream)
            ev = torch.cuda.Event()
            ev.record(stream)
        self.stats["batches"] += 1
        self.stats["admitted"] += len(reqs)
        bid = self._bid
        self._bid += 1
        return _Flight(bid, reqs, stream, ev, bufs, batch, sum(r.bytes for r in reqs))

    def _complete(self, fl: _Flight):
        fl.event.synchronize()
        E = fl.bufs["E"].cpu().numpy()
        t = time.perf_counter()
        for i, r in enumerate(fl.reqs):
            V = fl.bufs["V"][i].cpu().numpy()
            g = fl.bufs["g"][i].cpu().numpy() if fl.bufs["g"][i] is not None else None
            res = Result(r.rid, float(E[2 * i]), float(E[2 * i + 1]), V, g, r.t_submit, t,
                         fl.bid, len(fl.reqs), r.t_prepared, r.t_launch)
            r.plan.close(stream=fl.stream)  # its batch has finished: no device sync
            r.plan = None
            r.future.set_result(res)
        with self._cv:
            self._used -= fl.nbytes
            self._cv.notify_all()

    def _free_slot(self):
        busy = {id(f.stream) for f in self._flights}
        for i, s in enumerate(self._streams):
            if id(s) not in busy:
                return i
        return None

    def _gpu_loop(self):
        torch = self.torch
        while True:
            # retire finished batches first: frees memory and slots for new arrivals
            done = [f for f in self._flights if f.event.query()]
            for f in done:
                self._flights.remove(f)
                self._complete(f)
            with self._cv:
                slot = self._free_slot()
                reqs = self._admit() if slot is not None else []
                if not reqs:
                    if self._stop and not self._ready and not self._flights:
                        return
                    if not self._flights:
                        self._cv.wait(timeout=0.05)
                        continue
            if reqs:
                self.stats["peak_bytes"] = max(self.stats["peak_bytes"], self._used)
                try:
                    fl = self._launch(reqs, slot)
                    self._flights.append(fl)
                    self.stats["max_in_flight"] = max(self.stats["max_in_flight"], len(self._flights))
                except BaseException as ex:
                    with self._cv:
                        self._used -= sum(r.bytes for r in reqs)
                    for r in reqs:
                        if r.plan is not None:
                            r.plan.close()
                        r.future.set_exception(ex)
            elif self._flights:
                # wait for the oldest batch (with a bound, to keep admitting arrivals)
                t0 = time.perf_counter()
                while not self._flights[0].event.query() and time.perf_counter() - t0 < 0.002:
                    time.sleep(0.0002)


def run_plain(systems, want_grads):
    """Baseline: one plain, un-batched launch sequence per request, serially (plan,
    Fock build [+ gradient], copy back, release).  Returns (results, seconds)."""
    import torch
    out = []
    t0 = time.perf_counter()
    for s, wg in zip(systems, want_grads):
        ts = time.perf_counter()
        p = Plan(s)
        D = torch.as_tensor(np.ascontiguousarray(s.D), device="cuda")
        if wg:
            r = p.fock_grad(D)
            g = r["grad"].cpu().numpy()
        else:
            r = p.fock(D)
            g = None
        V = r["V"].cpu().numpy()
        p.close()
        out.append(Result(len(out), r["EH"], r["Ex"], V, g, ts, time.perf_counter(), -1, 1))
    return out, time.perf_counter() - t0
