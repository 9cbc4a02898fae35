"""Continuous-batching server for Fock builds (and Hxc gradients) of many cells.

Requests (a cell + its density matrix, optionally asking for the gradient) arrive at any
time.  Each one is planned on a host thread (gpw_plan_prepare: screening and task lists
on the CPU, which also yields the exact device footprint).  A GPU thread admits prepared
requests in arrival order while their footprints fit the device-memory budget; commit
threads upload each admitted plan and its density matrix on their own streams; the GPU
thread launches committed requests together as one batch (gpw_batch_fock_grad_async:
one collocation and one integration launch for all cells of the batch), and a finisher
thread copies results back and releases each plan in stream order.  Up to `streams`
batches are in flight at once on separate CUDA streams, so requests that arrive while
others run are admitted into the next batch as soon as slots and memory free up, and
their work overlaps on the device.  Each request's plan, pair lists and grids stay on the
device until its result has been copied back; then the memory is released.

Per-request results are those of the request run alone (the same tasks, in the same
order per sub-box, with the same reductions); the tests check this within the stated
tolerances.

Batches are formed by :class:`BatchPolicy` (host-only, tested without a GPU): the oldest
waiting request opens a batch, which takes later requests of the same kind of cell in
arrival order while the batch's estimated work (pair-points) stays under a cap, so that
small cells are not held behind a large one.  A request may carry a deadline: if it has
not been launched by then it fails with GPW_ETIMEDOUT, and if its batch is still running
then its future fails with GPW_ETIMEDOUT at once (the batch finishes and its memory is
released as usual).  A request whose future is cancelled before launch is dropped.

An optional priority lane (Server(priority_lane=True)) adds a stream of high CUDA priority
that takes batches of small requests only, so that they need not wait for a free batch
slot or for the blocks of a large batch: it halves the median latency of a mixed stream
and costs the large cells' tail (their blocks yield the SMs to the lane's), so it is off
by default.

Batches are launched directly, not through CUDA graphs: every batch holds a different set
of plans, so a captured graph would be replayed exactly once and its capture and
instantiation would cost what the launches cost.  A caller that repeats one batch (the
same cells with new density matrices, as in SCF iterations) can capture
Batch.fock_grad_async once and replay it (gpw_batch_generation tells when it is stale).
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import os
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from .binding import Batch, GpwError, Plan, stream_wait

GPW_ETIMEDOUT = -5


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
    deadline: float | None = None  # absolute time (perf_counter) or None
    plan: Plan | None = None
    bytes: int = 0
    cost: float = 0.0  # estimated GPU work: pair-points of the plan
    kind: object = False  # what a batch must share: cell kind and integration sub-boxes
    error: BaseException | None = None
    t_prepared: float = 0.0
    t_launch: float = 0.0
    bufs: dict | None = None  # device D, V, grad of the request (after commit)
    done: bool = False  # its future has been resolved


class BatchPolicy:
    """Which staged requests go into the next batch (host-only: no CUDA, so it is tested
    on the CPU).  A request is anything with the attributes kind, cost and deadline.

    max_batch: most requests per batch.  batch_cost: cap on a batch's summed cost
    (pair-points); a request costlier than the cap opens a batch of its own, and the
    oldest request always opens the next batch, so no request starves.  small_cost: the
    most a request may cost to ride in a small-request batch (form(small_only=True)),
    which the server launches on a high-priority stream; lane_cost: the cap on such a
    batch's summed cost (None: batch_cost), which keeps the high-priority batches short."""

    def __init__(self, max_batch: int = 32, batch_cost: float = 1.5e9,
                 small_cost: float = 4.0e8, lane_cost: float | None = None):
        self.max_batch = int(max_batch)
        self.batch_cost = float(batch_cost)
        self.small_cost = float(small_cost)
        self.lane_cost = float(batch_cost if lane_cost is None else lane_cost)

    @staticmethod
    def expired(req, now: float) -> bool:
        return req.deadline is not None and now > req.deadline

    def form(self, staged, now: float, small_only: bool = False):
        """Split `staged` (oldest first) into (batch, keep, expired): expired requests are
        past their deadline; the batch is the oldest live request (the oldest small one
        with small_only) plus later ones of its kind (small ones with small_only), in
        order, while the count stays <= max_batch and the summed cost <= max(cap, cost of
        its first request), cap = lane_cost with small_only, else batch_cost; keep is the
        rest, in order."""
        expired = [r for r in staged if self.expired(r, now)]
        live = [r for r in staged if not self.expired(r, now)]
        fits = (lambda r: r.cost <= self.small_cost) if small_only else (lambda r: True)
        i0 = next((i for i, r in enumerate(live) if fits(r)), None)
        if i0 is None:
            return [], live, expired
        first = live[i0]
        cap = max(self.lane_cost if small_only else self.batch_cost, first.cost)
        batch, keep, total = [first], live[:i0], first.cost
        for r in live[i0 + 1:]:
            if (r.kind == first.kind and fits(r) and len(batch) < self.max_batch and
                    total + r.cost <= cap):
                batch.append(r)
                total += r.cost
            else:
                keep.append(r)
        return batch, keep, expired


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
    batch.  streams: batches in flight.  host_workers: planning threads (default half
    the cores; each plan uses its share of the cores among the plans being made).  tile,
    tile_integ, colloc_warps, integ_chunk: launch shape of every plan (library defaults
    if None); tune_with: a list of sample cells to run the autotuner on (as one batch)
    instead, its choice (cached per GPU and workload class) then serves every request.
    Non-orthogonal cells plan with 4x8x16 sub-boxes for both passes, so a request of that
    kind fails alone under another explicit shape; batches hold one kind of cell, and
    only plans with the same integration sub-boxes (by default they follow a plan's
    largest degree: cells with f shells take plain 8x8x32 sub-boxes).
    batch_cost: most pair-points (estimated GPU work) per batch, beyond its first
    request; small_cost: the most a request may cost to ride the priority lane;
    lane_cost: the cap on a priority-lane batch's work (default batch_cost);
    priority_lane: one more stream for batches of small requests; lane_priority: its
    CUDA stream priority (-1 high: its blocks take the SMs first; 0 the same as the
    regular streams: its blocks queue with theirs, so the lane only spares small requests
    the wait for a free batch slot).
    """

    def __init__(self, hbm_budget: int | None = None, max_batch: int = 32, streams: int = 3,
                 host_workers: int | None = None, tile=None, tile_integ=None,
                 colloc_warps=None, integ_chunk=None, tune_with=None, fail_prepare=None,
                 batch_cost: float = 1.5e9, small_cost: float = 4.0e8,
                 priority_lane: bool = False, lane_priority: int = -1,
                 lane_cost: float | None = None):
        import torch
        self.torch = torch
        torch.cuda.init()
        free, _ = torch.cuda.mem_get_info()
        self.budget = int(hbm_budget if hbm_budget is not None else 0.7 * free)
        self.max_batch = int(max_batch)
        self.policy = BatchPolicy(self.max_batch, batch_cost, small_cost, lane_cost)
        self.plan_kwargs = dict(tile=tile, tile_integ=tile_integ, colloc_warps=colloc_warps,
                                integ_chunk=integ_chunk)
        self.choice = None
        if tune_with:
            from .autotune import tune
            self.choice = tune(list(tune_with))
            self.plan_kwargs = self.choice.plan_kwargs()
        self._fail_prepare = fail_prepare  # test hook: callable(system) -> bool
        # planning threads; each plan takes an equal share of the cores among the plans
        # being made at its start, so that the planners' thread teams do not oversubscribe
        # the host the GPU threads run on, and a large cell planned alone gets them all
        self._cores = os.cpu_count() or 4
        workers = host_workers or max(2, self._cores // 2)
        self._planning = 0
        self._pool = cf.ThreadPoolExecutor(workers, thread_name_prefix="gpw-plan")
        self._commits = cf.ThreadPoolExecutor(4, thread_name_prefix="gpw-commit")
        self._finisher = cf.ThreadPoolExecutor(2, thread_name_prefix="gpw-finish")
        self._tls = threading.local()
        self._streams = [torch.cuda.Stream() for _ in range(max(1, streams))]
        # the priority lane: one more stream, of high priority, for batches of small
        # requests only; the block scheduler gives its blocks the SMs as soon as blocks of
        # the running large batches retire, so small cells do not queue behind them
        self._lane = len(self._streams) if priority_lane else None
        if priority_lane:
            self._streams.append(torch.cuda.Stream(priority=int(lane_priority)))
        self._batches = [Batch(self.max_batch) for _ in self._streams]
        self._ready = collections.deque()    # prepared, waiting for admission
        self._staged = collections.deque()   # committed, waiting for a batch
        self._committing = 0
        self._finishing = 0
        self._flights: list[_Flight] = []
        self._used = 0
        self._rid = 0
        self._bid = 0
        self._cv = threading.Condition()
        self._stop = False
        self.stats = dict(batches=0, admitted=0, rejected=0, max_in_flight=0, peak_bytes=0,
                          timed_out=0, cancelled=0)
        self._gpu = threading.Thread(target=self._gpu_loop, name="gpw-serve", daemon=True)
        self._gpu.start()

    # ------------------------------------------------------------------ API --
    def submit(self, system, want_grad: bool = False, deadline_s: float | None = None) -> cf.Future:
        """Queue one Fock build (plus gradient if want_grad); returns a Future[Result].
        deadline_s: seconds from now; past it the future fails with GpwError
        (GPW_ETIMEDOUT).  Cancelling the future before its batch is launched drops it."""
        fut: cf.Future = cf.Future()
        with self._cv:
            rid = self._rid
            self._rid += 1
        t = time.perf_counter()
        req = _Req(rid, system, bool(want_grad), fut, t,
                   None if deadline_s is None else t + float(deadline_s))
        self._pool.submit(self._prepare, req)
        return fut

    def close(self, timeout_s: float | None = None):
        """Finish every submitted request, then stop.  With timeout_s, the wait for the
        batches still on the GPU is bounded (gpw_stream_wait) and a TimeoutError is raised
        if they have not finished."""
        self._pool.shutdown(wait=True)  # all preparations have reached the ready queue
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        if timeout_s is not None:
            t_end = time.perf_counter() + float(timeout_s)
            while self._gpu.is_alive():
                for f in list(self._flights):
                    if not stream_wait(f.stream, max(0.0, t_end - time.perf_counter())):
                        raise TimeoutError("batches still running on the GPU at the timeout")
                self._gpu.join(timeout=0.01)
                if time.perf_counter() > t_end and self._gpu.is_alive():
                    raise TimeoutError("server did not drain within the timeout")
        self._gpu.join()
        self._commits.shutdown(wait=True)
        self._finisher.shutdown(wait=True)
        for b in self._batches:
            b.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------- host side --
    def _prepare(self, req: _Req):
        with self._cv:
            self._planning += 1
            share = max(1, self._cores // self._planning)
        try:
            if self._fail_prepare and self._fail_prepare(req.system):
                raise RuntimeError("plan preparation failed (injected)")
            req.plan = Plan(req.system, commit=False, host_threads=share, **self.plan_kwargs)
            nao, natm = req.plan.nao, req.plan.natm
            st = req.plan.stats()
            req.bytes = int(st["device_bytes"]) + 8 * (2 * nao * nao + 3 * natm + 2)
            req.cost = float(st["pair_points"])
            # plans batch only with plans of the same kernels: orthorhombic or not, and the
            # same integration sub-boxes (the library default depends on a plan's degrees)
            req.kind = (_skewed(req.system), tuple(st["tile_integ"]), st["integ_zwin"])
            if req.bytes > self.budget:
                raise MemoryError(f"request needs {req.bytes} device bytes, budget is {self.budget}")
        except BaseException as ex:  # the request fails alone; the server keeps serving
            req.error = ex
        req.t_prepared = time.perf_counter()
        with self._cv:
            self._planning -= 1
            self._ready.append(req)
            self._cv.notify_all()

    # -------------------------------------------------------------- GPU side --
    def _admit(self):
        """Admit prepared requests in arrival order while they fit the memory budget and
        hand them to the commit threads (called with the lock held)."""
        now = time.perf_counter()
        while self._ready:
            req = self._ready[0]
            if req.error is None and req.future.cancelled():
                self._ready.popleft()
                self.stats["cancelled"] += 1
                req.plan.close()
                req.plan = None
                continue
            if req.error is None and self.policy.expired(req, now):
                req.error = GpwError(GPW_ETIMEDOUT, "serve", "deadline passed before launch")
                self.stats["timed_out"] += 1
                req.plan.close()
                req.plan = None
            if req.error is not None:
                self._ready.popleft()
                self.stats["rejected"] += 1
                if not req.future.cancelled():
                    req.future.set_exception(req.error)
                continue
            busy = self._flights or self._staged or self._committing or self._finishing
            if self._used + req.bytes > self.budget and busy:
                break
            self._ready.popleft()
            self._used += req.bytes
            self.stats["peak_bytes"] = max(self.stats["peak_bytes"], self._used)
            self._committing += 1
            self._commits.submit(self._commit, req)

    def _commit(self, req: _Req):
        """Commit thread: the plan and the request's buffers on this thread's stream."""
        torch = self.torch
        st = getattr(self._tls, "stream", None)
        if st is None:
            # high priority: the plan's table kernel takes SMs as soon as blocks of the
            # running batches retire instead of queueing behind them
            st = self._tls.stream = torch.cuda.Stream(priority=-1)
        try:
            with torch.cuda.stream(st):
                req.plan.commit(st)
                D = torch.as_tensor(np.ascontiguousarray(req.system.D), device="cuda")
                V = torch.empty((req.plan.nao, req.plan.nao), dtype=torch.float64, device="cuda")
                g = (torch.empty((req.plan.natm, 3), dtype=torch.float64, device="cuda")
                     if req.want_grad else None)
            st.synchronize()
            req.bufs = dict(D=D, V=V, g=g)
            ok = True
        except BaseException as ex:
            ok = False
            err = ex
        with self._cv:
            self._committing -= 1
            if ok:
                self._staged.append(req)
            else:
                self._used -= req.bytes
                self.stats["rejected"] += 1
            self._cv.notify_all()
        if not ok:
            if req.plan is not None:
                req.plan.close()
                req.plan = None
            if not req.future.cancelled():
                req.future.set_exception(err)

    def _launch(self, reqs, slot: int):
        torch = self.torch
        stream = self._streams[slot]
        batch = self._batches[slot]
        t = time.perf_counter()
        for r in reqs:
            r.t_launch = t
            for x in r.bufs.values():
                if x is not None:
                    x.record_stream(stream)  # the allocator keeps them until this batch ends
        with torch.cuda.stream(stream):
            E = torch.empty(2 * len(reqs), dtype=torch.float64, device="cuda")
            batch.set([r.plan for r in reqs], stream)
            batch.fock_grad_async([r.bufs["D"] for r in reqs], [r.bufs["V"] for r in reqs],
                                  [r.bufs["g"] for r in reqs], E, stream)
            ev = torch.cuda.Event()
            ev.record(stream)
        self.stats["batches"] += 1
        self.stats["admitted"] += len(reqs)
        bid = self._bid
        self._bid += 1
        return _Flight(bid, reqs, stream, ev, dict(E=E), batch, sum(r.bytes for r in reqs))

    def _complete(self, fl: _Flight):
        """Finisher thread: copy the results of a finished batch back and release plans."""
        E = fl.bufs["E"].cpu().numpy()
        t = time.perf_counter()
        for i, r in enumerate(fl.reqs):
            with self._cv:
                late = r.done  # its deadline passed while the batch ran
                r.done = True
            if not late:
                V = r.bufs["V"].cpu().numpy()
                g = r.bufs["g"].cpu().numpy() if r.bufs["g"] is not None else None
                res = Result(r.rid, float(E[2 * i]), float(E[2 * i + 1]), V, g, r.t_submit, t,
                             fl.bid, len(fl.reqs), r.t_prepared, r.t_launch)
            r.plan.close(stream=fl.stream)  # its batch has finished: no device sync
            r.plan = None
            r.bufs = None
            if not late:
                r.future.set_result(res)
        with self._cv:
            self._used -= fl.nbytes
            self._finishing -= 1
            self._cv.notify_all()

    def _launchable(self) -> bool:
        """A batch could be launched now (lock held): staged requests and a free regular
        slot, or the priority lane free and a small request staged."""
        if not self._staged:
            return False
        if self._free_slot() is not None:
            return True
        return (self._lane is not None and self._free_slot(lane=True) is not None and
                any(r.cost <= self.policy.small_cost for r in self._staged))

    def _free_slot(self, lane: bool = False):
        """A free stream slot: a regular one, or with lane=True the priority lane."""
        busy = {id(f.stream) for f in self._flights}
        for i, s in enumerate(self._streams):
            if (i == self._lane) == lane and id(s) not in busy:
                return i
        return None

    def _drop(self, r: _Req, err: BaseException | None):
        """Release a staged request that will not run (expired or cancelled)."""
        self._used -= r.bytes
        if r.plan is not None:
            r.plan.close()
            r.plan = None
        r.bufs = None
        r.done = True
        if err is not None and not r.future.cancelled():
            r.future.set_exception(err)

    def _expire_in_flight(self, now: float):
        """Futures of running requests past their deadline fail now (lock held)."""
        for f in self._flights:
            for r in f.reqs:
                if not r.done and self.policy.expired(r, now):
                    r.done = True
                    self.stats["timed_out"] += 1
                    r.future.set_exception(GpwError(GPW_ETIMEDOUT, "serve",
                                                    "deadline passed while its batch ran"))

    def _gpu_loop(self):
        while True:
            # hand finished batches to the finisher: frees their stream slots at once
            done = [f for f in self._flights if f.event.query()]
            with self._cv:
                for f in done:
                    self._flights.remove(f)
                    self._finishing += 1
            for f in done:
                self._finisher.submit(self._complete, f)
            reqs, slot = [], None
            with self._cv:
                now = time.perf_counter()
                self._expire_in_flight(now)
                self._admit()
                slot, small = None, False
                if self._staged:
                    slot = self._free_slot()
                    if slot is None and self._lane is not None:
                        slot, small = self._free_slot(lane=True), True
                if slot is not None:
                    # the policy picks the batch: one kind of cell, oldest first, its work
                    # capped (small requests only on the priority lane); expired and
                    # cancelled requests leave here
                    batch, keep, expired = self.policy.form(list(self._staged), now,
                                                            small_only=small)
                    self._staged = collections.deque(keep)
                    for r in expired:
                        self.stats["timed_out"] += 1
                        self._drop(r, GpwError(GPW_ETIMEDOUT, "serve", "deadline passed before launch"))
                    for r in batch:
                        if r.future.set_running_or_notify_cancel():
                            reqs.append(r)
                        else:
                            self.stats["cancelled"] += 1
                            self._drop(r, None)
                if not reqs:
                    idle = not (self._ready or self._staged or self._committing or
                                self._flights or self._finishing)
                    if self._stop and idle:
                        return
                    if not self._flights:
                        self._cv.wait(timeout=0.005)
                        continue
            if reqs:
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
                # wait briefly for the oldest batch, staying responsive to new arrivals
                t0 = time.perf_counter()
                while not self._flights[0].event.query() and time.perf_counter() - t0 < 0.002:
                    with self._cv:
                        if self._launchable():
                            break
                    time.sleep(0.0002)


def _skewed(system) -> bool:
    """Non-orthogonal cell (a non-diagonal lattice): its plans batch only with their kind."""
    lat = np.asarray(system.lattice, dtype=np.float64)
    return bool(np.any(lat != np.diag(np.diag(lat))))


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
