#!/usr/bin/env python
"""Throughput of the multigrid GPW hot path on GB300 (one JSON line on rank 0).

One step = one full pass of the path over the 256-water workload: gpw_fock_grad (pair
D tensors, collocation on every level, Fourier interpolation, Poisson, Slater exchange,
restriction, one integration pass at degree L+1 per pair, V assembly and the Hxc
gradient contraction).
The plan (screening, task lists, 1-D tables) is built once per geometry before the
timed region, as the method prescribes; its time is reported as plan_ms.

value = model FP64 FLOPs of the two grid passes (2(L+1) per pair-point for eval_rho,
2(L+2) for the integration that serves eval_mat and eval_mat_ip1) per second, summed
over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank runs an independent replica of the workload on its own GPU
(weak scaling, no collective on the data path).  --impl reference times the CPU
oracle on a bounded sample of the same workload, on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "eval_rho+eval_mat FP64 TFLOP/s (% of peak); served builds/s, p50/p99 latency"
# FP64 peak of one GB300: 152 SMs x 4 FLOP/clk/SM (the nominal 1.25 TFLOP/s at the
# 2070 MHz maximum SM clock is 3.97 FLOP/clk/SM) x 2.070 GHz.
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12
WORKLOAD = "water256"
WORKLOAD_DESC = ("256 H2O, cubic L=37.3 Bohr, 7168 Cartesian AOs, 280 Ha, 4 levels "
                 "(288/168/96/60), tau=1e-6; step = gpw_fock_grad (V, energies, Hxc gradient)")


def _workload_desc(name: str, system, stats) -> str:
    """What one step computes on the named workload (sizes from the system and plan)."""
    if name == WORKLOAD:
        return WORKLOAD_DESC
    import numpy as np
    lat = np.asarray(system.lattice, dtype=float)
    mesh = "/".join("x".join(str(int(x)) for x in m) for m in stats["meshes"])
    if np.all(lat == np.diag(np.diag(lat))):
        cell = f"orthorhombic L={'/'.join(f'{x:.2f}' for x in np.diag(lat))} Bohr"
    else:
        cell = ("triclinic rows " + " ".join("(" + ",".join(f"{x:.2f}" for x in r) + ")" for r in lat)
                + " Bohr")
    return (f"{name}: {cell}, {system.natm} atoms, {system.nao} Cartesian AOs, "
            f"{system.cutoff_ha:g} Ha, {stats['nlevels']} levels ({mesh}), tau={system.tau:g}; "
            f"step = gpw_fock_grad (V, energies, Hxc gradient)")


# DRAM bytes per launch of the dominant kernel from one ncu capture (of a smaller case,
# scaled by the work it processes), valid while the kernels and the plan (task lists,
# work order) are unchanged: sha256 of csrc/kernels.cu + csrc/plan.cpp at capture time.
TRAFFIC = {
    # integration at degree L+1 (8x8x16 sub-boxes, 48-point z windows): read + write of
    # one 32-water launch (1.393 GB) scaled by pair-points to the 256-water launch
    "integrate_ip1": {"bytes_per_launch": 1.0124e+10, "src_sha": "f56b93e800c9ee4f",
                      "capture": "profiles/integrate_traffic_water32.md"},
}


def _kernels_sha() -> str:
    h = hashlib.sha256()
    for f in ("kernels.cu", "plan.cpp"):
        h.update(open(os.path.join(ROOT, "paper_2603_24881_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpw", choices=["gpw", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-stride", type=int, default=8)
    ap.add_argument("--served", type=int, default=400,
                    help="also run the served request stream with this many requests")
    ap.add_argument("--tile", default=None, help="collocation sub-box t0,t1,t2")
    ap.add_argument("--tile-integ", default=None,
                    help="integration sub-box t0,t1,t2 or, with overlapping z windows, t0,t1,t2,zwin")
    ap.add_argument("--xc", default="lda_x", choices=["lda_x", "pbe_x"],
                    help="exchange functional (LDA Slater or PBE exchange, a GGA)")
    ap.add_argument("--configs", action="store_true",
                    help="per-call timings of eval_rho / eval_mat / eval_mat_ip1 / fock_grad "
                         "on every config (one JSON line each) instead of the bench step")
    ap.add_argument("--tau", action="store_true",
                    help="also time the kinetic-energy-density (meta-GGA) kernels")
    ap.add_argument("--autotune", action="store_true",
                    help="pick the launch shape with the autotuner (cached per GPU/workload)")
    ap.add_argument("--fast-prune", action="store_true",
                    help="GPW_FAST_BLOCK_PRUNE: per-block value screening of the collocation "
                         "tasks (tau-sized changes, outside the strict definition)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks -----
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", gpu_id], stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        rows = [l.strip().split(",") for l in open(self.file.name) if l.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def _gpu_id(torch) -> str:
    try:
        u = torch.cuda.get_device_properties(torch.cuda.current_device()).uuid
        return "GPU-" + str(u)
    except Exception:
        return str(torch.cuda.current_device())


# ------------------------------------------------------------------ oracle -----
def oracle_sample(sys_, stride: int, offset: int = 0, threads: int = 0, ops=None):
    """Time the CPU oracle (as it stands) on every stride-th pair of the workload:
    separable collocation, integration and the gradient contraction.  Returns
    (model flops, seconds, pairs, pair-points, threads); `ops`, if a dict, receives the
    seconds of each of the three."""
    import numpy as np
    import oracle
    p = oracle.Plan(sys_)
    idx = np.arange(offset % stride, p.npairs, stride)
    sub = p.subset(idx)
    L = (p.prims["l"][sub.ab[:, 0]] + p.prims["l"][sub.ab[:, 1]]).astype(np.float64)
    pts = np.prod(sub.hi - sub.lo + 1, axis=1).astype(np.float64)
    flops = float(np.sum(2 * (L + 1) * pts) * 2 + np.sum(2 * (L + 2) * pts))
    rng = np.random.default_rng(0)
    vl = [rng.standard_normal(tuple(m)) for m in p.meshes]
    nthr = threads or os.cpu_count() or 1
    t0 = time.perf_counter()
    sub.rho_levels(sys_.D, mode="separable", nthreads=nthr)
    t1 = time.perf_counter()
    sub._pair_blocks(vl, nthreads=nthr)
    t2 = time.perf_counter()
    sub._pair_blocks(vl, grad_D=sys_.D, nthreads=nthr)
    t3 = time.perf_counter()
    if ops is not None:
        ops.update(eval_rho=t1 - t0, eval_mat=t2 - t1, eval_mat_ip1=t3 - t2)
    return flops, t3 - t0, len(idx), float(pts.sum()), nthr


def cpu_baseline(sys_, stride: int) -> dict:
    """The oracle on all host threads, and on one thread over a 16 times smaller sample:
    model TFLOP/s, seconds and pair-points/s of each operation."""
    ops = {}
    f, dt, n, pts, nthr = oracle_sample(sys_, stride, ops=ops)
    ops1 = {}
    f1, dt1, n1, pts1, _ = oracle_sample(sys_, 16 * stride, threads=1, ops=ops1)
    per = lambda o, p: {k: {"s": v, "pair_points_per_s": p / v} for k, v in o.items()}
    return {"value": f / dt / 1e12, "unit": "TFLOP/s", "cores": nthr, "kind": "oracle",
            "sample": f"every {stride}th screened pair of {WORKLOAD} ({n} pairs, {pts:.3e} "
                      f"pair-points): separable collocation + integration + gradient "
                      f"contraction, {dt:.1f} s on {nthr} threads",
            "ops": per(ops, pts),
            "single_thread": {"value": f1 / dt1 / 1e12, "unit": "TFLOP/s", "cores": 1,
                              "sample": f"every {16 * stride}th pair ({n1} pairs, {pts1:.3e} "
                                        f"pair-points), {dt1:.1f} s",
                              "ops": per(ops1, pts1)}}


def run_reference(a, rank, world):
    """Reference arm: the CPU oracle, timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import workloads
    s = workloads.config(a.workload)
    stride = max(a.cpu_stride * 4, 64)
    for i in range(a.warmup):
        oracle_sample(s, stride * 4, offset=i)
    tot_f, tot_t, nthr = 0.0, 0.0, 0
    for i in range(a.steps):
        f, dt, n, pts, nthr = oracle_sample(s, stride, offset=i)
        tot_f += f
        tot_t += dt
    val = tot_f / tot_t / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s",
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * tot_t / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC, "sample": f"every {stride}th pair per step"},
            "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": nthr, "kind": "oracle",
                             "sample": f"every {stride}th screened pair of {a.workload} per step"},
            "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def fp64_dgemm_tflops(torch, n: int = 6144, reps: int = 3) -> float:
    """cuBLAS DGEMM rate on this GPU in this run (context for the FP64 peak): best of
    `reps` n x n x n products after one warm-up, CUDA events."""
    g = torch.Generator(device="cuda").manual_seed(0)
    a = torch.rand((n, n), dtype=torch.float64, device="cuda", generator=g)
    b = torch.rand((n, n), dtype=torch.float64, device="cuda", generator=g)
    c = a @ b
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b, c
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


# ------------------------------------------------------------------ served -----
def served_bench(nreq: int) -> dict:
    """The served stream (water boxes of 4..128 molecules, p ~ 1/n, 10% gradients):
    saturated builds/s of the continuous-batching server, then a replay with Poisson
    arrivals at 80% of it for p50/p99 latency, against one plain launch sequence per
    request, and the largest per-request disagreement between the two; the same two
    runs with the optional priority lane for small cells, for comparison."""
    import numpy as np
    import workloads
    from paper_2603_24881_gb300.serve import Server, run_plain
    reqs = workloads.stream_requests(nreq, seed=4)
    systems = [r.system() for r in reqs]
    grads = [r.want_grad for r in reqs]
    # warm-up (untimed): one request of every cell size in the stream, so that the CUDA
    # modules of every kernel and FFT size are loaded and the allocator has seen them
    first = {}
    for i, s in enumerate(systems):
        first.setdefault(int(s.natm), i)
    warm = sorted(first.values())
    with Server() as srv:
        [f.result() for f in [srv.submit(systems[i], True) for i in warm]]

    def saturated(**kw):
        with Server(**kw) as srv:
            t0 = time.perf_counter()
            futs = [srv.submit(s, g) for s, g in zip(systems, grads)]
            res = [f.result() for f in futs]
            return res, time.perf_counter() - t0, dict(srv.stats)

    def poisson(rate, **kw):
        arr = [r.arrival for r in workloads.stream_requests(nreq, seed=4, rate=rate)]
        with Server(**kw) as srv:
            t0 = time.perf_counter()
            futs = []
            for s, g, ta in zip(systems, grads, arr):
                dt = ta - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                futs.append(srv.submit(s, g))
            res = [f.result() for f in futs]
            return res, max(r.t_done for r in res) - t0

    sat, t_sat, st_sat = saturated()
    rate = 0.8 * nreq / t_sat
    pois, t_pois = poisson(rate)
    _, t_sat_l, _ = saturated(priority_lane=True)
    pois_l, _ = poisson(0.8 * nreq / t_sat_l, priority_lane=True)
    lat_l = np.array([r.latency for r in pois_l])
    lat = np.array([r.latency for r in pois])
    nwat = np.array([int(sy.natm) // 3 for sy in systems])
    by_size = {int(n): {"requests": int(np.sum(nwat == n)),
                        "p50_ms": 1e3 * float(np.percentile(lat[nwat == n], 50)),
                        "p99_ms": 1e3 * float(np.percentile(lat[nwat == n], 99))}
               for n in sorted(set(nwat.tolist()))}
    plan_ms = np.array([r.t_prepared - r.t_submit for r in pois]) * 1e3
    wait_ms = np.array([r.t_launch - r.t_prepared for r in pois]) * 1e3
    run_ms = np.array([r.t_done - r.t_launch for r in pois]) * 1e3
    plain, t_plain = run_plain(systems, grads)
    plat = np.array([r.latency for r in plain])
    dE = max(max(abs(a.EH - b.EH), abs(a.Ex - b.Ex)) for a, b in zip(sat, plain))
    dV = max(float(np.max(np.abs(a.V - b.V)) / max(np.max(np.abs(b.V)), 1e-300))
             for a, b in zip(sat, plain))
    dg = max((float(np.max(np.abs(a.grad - b.grad))) for a, b in zip(sat, plain)
              if a.grad is not None), default=0.0)
    return {"requests": nreq, "builds_per_s_saturated": nreq / t_sat,
            "builds_per_s_poisson": nreq / t_pois, "poisson_rate_per_s": rate,
            "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "plain_builds_per_s": nreq / t_plain,
            "plain_p50_ms": 1e3 * float(np.percentile(plat, 50)),
            "plain_p99_ms": 1e3 * float(np.percentile(plat, 99)),
            "speedup_vs_plain": t_plain / t_sat, "batches": st_sat["batches"],
            "poisson_p50_ms_split": {"host_plan": float(np.percentile(plan_ms, 50)),
                                     "admission_wait": float(np.percentile(wait_ms, 50)),
                                     "gpu_batch_and_copy": float(np.percentile(run_ms, 50))},
            "poisson_p99_ms_split": {"host_plan": float(np.percentile(plan_ms, 99)),
                                     "admission_wait": float(np.percentile(wait_ms, 99)),
                                     "gpu_batch_and_copy": float(np.percentile(run_ms, 99))},
            "poisson_latency_by_waters": by_size,
            "max_abs_dE_Ha": dE, "max_rel_dV": dV, "max_abs_dgrad": dg,
            "with_priority_lane": {"builds_per_s_saturated": nreq / t_sat_l,
                                   "p50_ms": 1e3 * float(np.percentile(lat_l, 50)),
                                   "p99_ms": 1e3 * float(np.percentile(lat_l, 99))},
            "stream": "water boxes n in {4,8,16,32,64,128}, p ~ 1/n, 10% gradients, seed 4"}


# ------------------------------------------------------------------ main -------
def per_config(a):
    """Per call, on every config: eval_rho, eval_mat, eval_mat_ip1 (finest-grid potential)
    and gpw_fock_grad, CUDA events, median of 10 after 3 warm-up calls; model FLOPs
    (2(L+1) per pair-point for rho and V, 2(L+2) for the gradient pass) per second and
    pair-points per second."""
    import numpy as np
    import torch
    import workloads
    import paper_2603_24881_gb300 as gpw
    gpw.load()
    for name in ("tiny", "water32", "carbon", "water256", "water32_triclinic", "water256_triclinic",
                 "water32_hexagonal", "water256_hexagonal"):
        s = workloads.config(name)
        plan = gpw.Plan(s)
        st = plan.stats()
        D = torch.as_tensor(s.D, device="cuda")
        v = plan.fock(D, want_v=True)["v"]
        V = torch.empty((plan.nao, plan.nao), dtype=torch.float64, device="cuda")
        g = torch.empty((plan.natm, 3), dtype=torch.float64, device="cuda")
        rho = torch.empty(plan.fine_mesh, dtype=torch.float64, device="cuda")
        E = torch.empty(2, dtype=torch.float64, device="cuda")
        calls = {"eval_rho": (lambda: plan.eval_rho(D, out=rho), st["flops_rho"]),
                 "eval_mat": (lambda: plan.eval_mat(v, out=V), st["flops_mat"]),
                 "eval_mat_ip1": (lambda: plan.eval_mat_ip1(D, v, out=g), st["flops_ip1"]),
                 "fock_grad": (lambda: plan.fock_grad_async(D, V, g, E),
                               st["flops_rho"] + st["flops_ip1"])}
        res = {}
        for cname, (fn, fl) in calls.items():
            for _ in range(3):
                fn()
            ts = []
            for _ in range(10):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                fn()
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            ms = float(np.median(ts))
            res[cname] = {"ms": ms, "model_tflops": fl / ms / 1e9,
                          "pct_fp64_peak": 100.0 * fl / ms / 1e9 / FP64_PEAK_TFLOPS,
                          "pair_points_per_s": st["pair_points"] / (ms * 1e-3)}
        err = plan.check_device()
        print(json.dumps({"config": name, "pairs": st["npairs"], "pair_points": st["pair_points"],
                          "nao": plan.nao, "meshes": [list(m) for m in st["meshes"]],
                          "calls": res, "device_check": err}), flush=True)
        plan.close()
        torch.cuda.empty_cache()


def main():
    from paper_2603_24881_gb300 import replicas
    a = _args()
    rank, world, local = replicas.ranks_from_env()
    if a.impl == "reference":
        run_reference(a, rank, world)
        return
    if a.configs:
        if rank == 0:
            per_config(a)
        return
    import numpy as np
    import torch
    import workloads
    import paper_2603_24881_gb300 as gpw

    torch.cuda.set_device(local)
    dist = replicas.init(world, "nccl", torch.device("cuda", local))
    gpw.load()
    s = workloads.config(a.workload)
    t0 = time.perf_counter()
    tile = tuple(int(x) for x in a.tile.split(",")) if a.tile else None
    tile_i = tuple(int(x) for x in a.tile_integ.split(",")) if a.tile_integ else None
    shape = dict(tile=tile, tile_integ=tile_i[:3] if tile_i else None,
                 integ_zwin=tile_i[3] if tile_i and len(tile_i) > 3 else None)
    if a.autotune:
        from paper_2603_24881_gb300.autotune import tune
        shape = tune(s).plan_kwargs()
    plan = gpw.Plan(s, xc=a.xc, tau=a.tau, fast_prune=a.fast_prune, **shape)
    torch.cuda.synchronize()
    plan_ms = 1e3 * (time.perf_counter() - t0)
    st = plan.stats()
    flops_step = st["flops_rho"] + st["flops_ip1"]

    D = torch.as_tensor(s.D, device="cuda")
    V = torch.empty((plan.nao, plan.nao), dtype=torch.float64, device="cuda")
    E = torch.empty(2, dtype=torch.float64, device="cuda")
    v = torch.empty(plan.fine_mesh, dtype=torch.float64, device="cuda")
    g = torch.empty((plan.natm, 3), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        plan.fock_grad_async(D, V, g, E, stream=stream)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    plan.check_device()
    plan.profile(True)
    l0 = plan.launches()
    clk = Clocks(_gpu_id(torch)) if rank == 0 else None
    replicas.barrier(dist)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    replicas.barrier(dist)
    clocks = clk.stop() if clk else None
    launches = plan.launches() - l0
    prof = plan.profile_read()
    plan.profile(False)
    ms = replicas.max_over_ranks(dist, e0.elapsed_time(e1), device="cuda")
    err = plan.check_device()
    if err:
        raise RuntimeError(f"device bounds check fired: code {err}")
    value = replicas.whole_job_rate(flops_step * a.steps, world, ms * 1e-3) / 1e12

    # dominant kernel: the grid pass with the largest share of device time
    ph_flops = {"collocate": st["flops_rho"], "integrate_ip1": st["flops_ip1"]}
    dom = max(ph_flops, key=lambda k: prof["ms"][k])
    per_launch_ms = prof["ms"][dom] / max(prof["count"][dom], 1)
    achieved = ph_flops[dom] / (per_launch_ms * 1e-3) / 1e12
    tr = TRAFFIC.get(dom) if a.workload == WORKLOAD else None
    traffic = tr["bytes_per_launch"] if tr and tr.get("src_sha") == _kernels_sha() else None
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                "peak_source": "FP64 pipe: 152 SMs x 4 FLOP/clk x 2.07 GHz (no FP64 figure in "
                               "MEASURED_PEAKS.json)",
                "dgemm_tflops_measured": fp64_dgemm_tflops(torch)}

    e2e = None
    if not a.no_e2e:
        Dh = torch.as_tensor(s.D).pin_memory()
        out = dict(V=torch.empty((plan.nao, plan.nao), dtype=torch.float64, pin_memory=True),
                   grad=torch.empty((plan.natm, 3), dtype=torch.float64, pin_memory=True),
                   E=torch.empty(2, dtype=torch.float64, pin_memory=True))
        for _ in range(2):
            plan.fock_grad_host(Dh, out=out)
        eclk = Clocks(_gpu_id(torch)) if rank == 0 else None
        replicas.barrier(dist)
        # per step: the host lap and, from events on the call's stream around it, the
        # device span of its copies and kernels
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(a.steps)]
        t1 = time.perf_counter()
        laps = []
        for i in range(a.steps):
            tl = time.perf_counter()
            evs[i][0].record()
            plan.fock_grad_host(Dh, out=out)
            evs[i][1].record()
            laps.append(1e3 * (time.perf_counter() - tl))
        e2e_s = replicas.max_over_ranks(dist, time.perf_counter() - t1, device="cuda")
        eclocks = eclk.stop() if eclk else None
        dev = [b.elapsed_time(c) for b, c in evs]
        e2e = {"value": replicas.whole_job_rate(flops_step * a.steps, world, e2e_s) / 1e12,
               "unit": "TFLOP/s",
               "h2d_bytes_per_step": int(Dh.numel() * 8),
               "d2h_bytes_per_step": int((out["V"].numel() + out["grad"].numel() + 2) * 8),
               "api": "gpw_fock_grad_host through the C ABI (pinned host D in; V, gradient, "
                      "energies out; copies inside the timed region)",
               "ms_per_step": 1e3 * e2e_s / a.steps,
               "ms_min_max": [min(laps), max(laps)],
               "device_ms_min_max": [min(dev), max(dev)], "clocks": eclocks}

    tau = None
    if a.tau:
        # tau on the finest grid, its Fock term and the gradient for a fixed potential
        # (the fine Hxc potential of this density), CUDA events, same steps
        vt = plan.fock(D, want_v=True)["v"]
        Vt = torch.empty_like(V)
        tt = torch.empty(plan.fine_mesh, dtype=torch.float64, device="cuda")
        calls = {"eval_tau": lambda: plan.eval_tau(D, out=tt),
                 "eval_mat_tau": lambda: plan.eval_mat_tau(vt, out=Vt),
                 "eval_mat_tau_ip1": lambda: plan.eval_mat_tau_ip1(D, vt, out=g)}
        tau = {}
        for name, fn in calls.items():
            for _ in range(max(1, a.warmup)):
                fn()
            ta, tb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ta.record()
            for _ in range(a.steps):
                fn()
            tb.record()
            torch.cuda.synchronize()
            tau[name + "_ms"] = ta.elapsed_time(tb) / a.steps
        pp = st["pair_points_L"]
        tau["model_tflops"] = {
            "eval_tau": sum(2.0 * (l + 3) * n for l, n in enumerate(pp)) / tau["eval_tau_ms"] / 1e9,
            "eval_mat_tau": sum(2.0 * (l + 3) * n for l, n in enumerate(pp)) / tau["eval_mat_tau_ms"] / 1e9,
            "eval_mat_tau_ip1": sum(2.0 * (l + 4) * n for l, n in enumerate(pp)) / tau["eval_mat_tau_ip1_ms"] / 1e9}
        if plan.check_device():
            raise RuntimeError("device bounds check fired in the tau kernels")

    if rank == 0:
        cpu = None
        if not a.no_cpu:
            try:
                cpu = cpu_baseline(s, a.cpu_stride)
            except Exception as ex:  # the CPU oracle is a reported baseline only
                cpu = {"value": None, "unit": "TFLOP/s", "cores": os.cpu_count(),
                       "kind": "oracle", "sample": f"failed: {ex}"}
        served = served_bench(a.served) if a.served > 0 else None
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": _workload_desc(a.workload, s, st), "pairs": st["npairs"],
                           "pair_points": st["pair_points"], "tasks": st["nentries"],
                           "l2": "no flush: plan tables, tasks and grids (>2 GB) exceed L2",
                           "tile": list(st["tile"]), "tile_integ": list(st["tile_integ"]),
                           "integ_zwin": st["integ_zwin"],
                           "colloc_warps": st["colloc_warps"], "integ_chunk": st["integ_chunk"],
                           "launch_shape": "autotuned" if a.autotune else "library defaults",
                           "xc": a.xc, **({"screening": "GPW_FAST_BLOCK_PRUNE"} if a.fast_prune else {}),
                           "parallelism": f"replicas x{world}"},
                "pct_of_fp64_peak": 100.0 * value / world / FP64_PEAK_TFLOPS,
                **({"tau": tau} if tau else {}),
                "pair_points_per_s": st["pair_points"] * a.steps * world / (ms * 1e-3),
                "plan_ms": plan_ms, "phase_ms_per_step": {k: v / a.steps for k, v in prof["ms"].items()},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clocks, "served": served}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
