"""Batched launches and the continuous-batching server: every result equals the same
request run alone (1e-10 relative in V, 1e-8 Ha in energies, 1e-7 Ha/Bohr in gradients),
admission respects the device-memory budget, and failures stay with their request."""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-10


@pytest.fixture(scope="module")
def gpw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_24881_gb300 as g
    g.load()
    return g


def _systems():
    return [workloads.small_water(4, seed=101), workloads.small_water(8, seed=102),
            workloads.tiny(), workloads.small_water(4, seed=103),
            workloads.small_water(16, seed=104)]


@pytest.fixture(scope="module")
def alone(gpw):
    out = []
    for s in _systems():
        p = gpw.Plan(s)
        r = p.fock_grad(s.D)
        out.append(dict(V=r["V"].cpu().numpy(), grad=r["grad"].cpu().numpy(), EH=r["EH"], Ex=r["Ex"]))
        p.close()
    return out


def _same(res, ref, grad=True):
    assert abs(res["EH"] - ref["EH"]) <= 1e-8 and abs(res["Ex"] - ref["Ex"]) <= 1e-8
    V = np.asarray(res["V"])
    assert np.max(np.abs(V - ref["V"])) <= RTOL * np.max(np.abs(ref["V"]))
    if grad:
        assert np.max(np.abs(np.asarray(res["grad"]) - ref["grad"])) <= 1e-7


def test_prepare_reports_footprint(gpw):
    s = workloads.small_water(8, seed=102)
    p = gpw.Plan(s, commit=False)
    est = p.stats()["device_bytes"]
    assert not p.committed and est > 0
    p.commit()
    act = p.stats()["device_bytes"]
    assert 0.8 * act <= est <= 1.25 * act
    r = p.fock(s.D)
    assert np.isfinite(r["EH"])


def test_batch_matches_alone(gpw, alone):
    systems = _systems()
    plans = [gpw.Plan(s) for s in systems]
    b = gpw.Batch(8).set(plans)
    Ds = [torch.as_tensor(s.D, device="cuda") for s in systems]
    Vs = [torch.empty((p.nao, p.nao), dtype=torch.float64, device="cuda") for p in plans]
    gs = [torch.empty((p.natm, 3), dtype=torch.float64, device="cuda") for p in plans]
    E = torch.empty(2 * len(plans), dtype=torch.float64, device="cuda")
    for _ in range(2):  # the batch is reusable
        b.fock_grad_async(Ds, Vs, gs, E)
        torch.cuda.synchronize()
        e = E.cpu().numpy()
        for i, ref in enumerate(alone):
            _same(dict(V=Vs[i].cpu().numpy(), grad=gs[i].cpu().numpy(), EH=e[2 * i], Ex=e[2 * i + 1]), ref)
    for p in plans:
        assert p.check_device() == 0
        p.close()
    b.close()


def test_batch_in_cuda_graph(gpw, alone):
    systems = _systems()[:3]
    plans = [gpw.Plan(s) for s in systems]
    b = gpw.Batch(4).set(plans)
    Ds = [torch.as_tensor(s.D, device="cuda") for s in systems]
    Vs = [torch.empty((p.nao, p.nao), dtype=torch.float64, device="cuda") for p in plans]
    gs = [torch.empty((p.natm, 3), dtype=torch.float64, device="cuda") for p in plans]
    E = torch.empty(2 * len(plans), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.fock_grad_async(Ds, Vs, gs, E, stream=s)  # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.fock_grad_async(Ds, Vs, gs, E, stream=s)
    for V in Vs:
        V.zero_()
    g.replay()
    torch.cuda.synchronize()
    e = E.cpu().numpy()
    for i in range(len(plans)):
        _same(dict(V=Vs[i].cpu().numpy(), grad=gs[i].cpu().numpy(), EH=e[2 * i], Ex=e[2 * i + 1]), alone[i])
    # a later set (here a smaller plan set) invalidates the graph: the generation tells,
    # and a graph captured again runs the new set
    gen = b.generation
    assert gen == 1
    b.set(plans[1:])
    assert b.generation == gen + 1
    g2 = torch.cuda.CUDAGraph()
    E2 = torch.empty(2 * (len(plans) - 1), dtype=torch.float64, device="cuda")
    with torch.cuda.graph(g2, stream=s):
        b.fock_grad_async(Ds[1:], Vs[1:], gs[1:], E2, stream=s)
    for V in Vs:
        V.zero_()
    g2.replay()
    torch.cuda.synchronize()
    e = E2.cpu().numpy()
    for j, i in enumerate(range(1, len(plans))):
        _same(dict(V=Vs[i].cpu().numpy(), grad=gs[i].cpu().numpy(), EH=e[2 * j], Ex=e[2 * j + 1]), alone[i])
    assert float(Vs[0].abs().max()) == 0.0
    del g, g2
    b.close()
    for p in plans:
        p.close()


def test_server_results_equal_alone(gpw, alone):
    from paper_2603_24881_gb300.serve import Server
    systems = _systems()
    with Server(max_batch=3, streams=2) as srv:
        futs = [srv.submit(s, want_grad=True) for s in systems]
        # a second wave arrives while the first is in flight
        futs += [srv.submit(s, want_grad=(i % 2 == 0)) for i, s in enumerate(systems)]
        res = [f.result(timeout=300) for f in futs]
        stats = dict(srv.stats)
    for i, r in enumerate(res):
        ref = alone[i % len(systems)]
        _same(dict(V=r.V, grad=r.grad, EH=r.EH, Ex=r.Ex), ref, grad=r.grad is not None)
    assert stats["admitted"] == len(futs)
    assert stats["batches"] >= 4  # at most 3 per batch


def test_server_with_priority_lane_equals_alone(gpw, alone):
    # the optional priority lane (small requests on a high-priority stream) changes where
    # and when batches run, not their results
    from paper_2603_24881_gb300.serve import Server
    systems = _systems()
    with Server(max_batch=3, streams=1, priority_lane=True) as srv:
        futs = [srv.submit(s, want_grad=True) for s in systems + systems]
        res = [f.result(timeout=300) for f in futs]
        stats = dict(srv.stats)
    for i, r in enumerate(res):
        _same(dict(V=r.V, grad=r.grad, EH=r.EH, Ex=r.Ex), alone[i % len(systems)])
    assert stats["admitted"] == len(futs)


def test_server_memory_budget_and_failures(gpw, alone):
    from paper_2603_24881_gb300.serve import Server
    systems = _systems()
    probe = gpw.Plan(systems[4], commit=False)
    big = probe.stats()["device_bytes"]
    probe.close()
    # budget fits the largest request but not two of them at once
    budget = int(1.5 * big)
    huge = workloads.small_water(64, seed=7)
    fail = lambda s: s is systems[3]
    with Server(hbm_budget=budget, max_batch=8, streams=2, fail_prepare=fail) as srv:
        futs = [srv.submit(s, want_grad=True) for s in systems]
        fh = srv.submit(huge)
        out = []
        for i, f in enumerate(futs):
            if i == 3:
                with pytest.raises(RuntimeError):
                    f.result(timeout=300)
                continue
            out.append((i, f.result(timeout=300)))
        with pytest.raises(MemoryError):
            fh.result(timeout=300)
        stats = dict(srv.stats)
    for i, r in out:
        _same(dict(V=r.V, grad=r.grad, EH=r.EH, Ex=r.Ex), alone[i])
    assert stats["peak_bytes"] <= budget
    assert stats["rejected"] == 2


def test_server_mixes_cell_kinds(gpw):
    # orthorhombic and triclinic requests in one stream: batches hold one kind each and
    # every result equals its request run alone
    from paper_2603_24881_gb300.serve import Server
    systems = [workloads.small_water(4, seed=111), workloads.triclinic(workloads.small_water(4, seed=112)),
               workloads.small_water(4, seed=113), workloads.triclinic(workloads.small_water(4, seed=114))]
    ref = []
    for s in systems:
        p = gpw.Plan(s)
        r = p.fock_grad(s.D)
        ref.append(dict(V=r["V"].cpu().numpy(), grad=r["grad"].cpu().numpy(), EH=r["EH"], Ex=r["Ex"]))
        p.close()
    with Server(max_batch=4, streams=2) as srv:
        res = [f.result(timeout=300) for f in [srv.submit(s, want_grad=True) for s in systems]]
    for r, a in zip(res, ref):
        _same(dict(V=r.V, grad=r.grad, EH=r.EH, Ex=r.Ex), a)


def test_deadlines_and_cancellation(gpw, alone):
    from paper_2603_24881_gb300.serve import Server
    systems = _systems()
    with Server(max_batch=3, streams=2) as srv:
        late = srv.submit(systems[0], deadline_s=0.0)          # expired before launch
        keep = [srv.submit(s, want_grad=True, deadline_s=300.0) for s in systems]
        gone = srv.submit(systems[1])
        gone.cancel()                                           # cancelled while planning
        res = [f.result(timeout=300) for f in keep]
        with pytest.raises(gpw.GpwError) as ei:
            late.result(timeout=300)
        assert ei.value.code == -5
        assert gone.cancelled()
        stats = dict(srv.stats)
    for i, r in enumerate(res):
        _same(dict(V=r.V, grad=r.grad, EH=r.EH, Ex=r.Ex), alone[i])
    assert stats["timed_out"] >= 1 and stats["cancelled"] == 1


def test_stream_wait_is_bounded(gpw):
    from paper_2603_24881_gb300.binding import stream_wait
    s = torch.cuda.Stream()
    a = torch.ones((6144, 6144), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        b = a @ a  # about half a second of FP64 work
    assert stream_wait(s, 0.0) is False                       # still running: gives up
    assert stream_wait(s, 120.0) is True                      # then finishes
    assert stream_wait(s, 0.0) is True                        # nothing left
    assert float(b[0, 0]) == 6144.0
    with pytest.raises(gpw.GpwError):
        stream_wait(s, -1.0)


def test_server_mixes_integration_shapes(gpw):
    # cells whose plans take different default integration sub-boxes (f shells: plain
    # 8x8x32; waters: 8x8x16 with 48-point z windows) are served together: each batch
    # holds plans of one shape, and every result is the request's alone-run result
    import systems
    from paper_2603_24881_gb300.serve import Server
    cells = [systems.resolved(seed=8, shells=((0, 1), (1, 1), (2, 1), (3, 1)), natm=3),
             workloads.small_water(4, seed=101),
             systems.resolved(seed=9, shells=((0, 1), (1, 1), (2, 1), (3, 1)), natm=3),
             workloads.small_water(4, seed=103)]
    shapes = set()
    ref = []
    for c in cells:
        p = gpw.Plan(c)
        st = p.stats()
        shapes.add((tuple(st["tile_integ"]), st["integ_zwin"]))
        r = p.fock_grad(c.D)
        ref.append(dict(V=r["V"].cpu().numpy(), grad=r["grad"].cpu().numpy(), EH=r["EH"], Ex=r["Ex"]))
        p.close()
    assert shapes == {((8, 8, 32), 32), ((8, 8, 16), 48)}
    with Server(max_batch=4, streams=2) as srv:
        futs = [srv.submit(c, want_grad=True) for c in cells]
        res = [f.result(timeout=300) for f in futs]
    for r, want in zip(res, ref):
        _same(dict(V=r.V, grad=r.grad, EH=r.EH, Ex=r.Ex), want)
