"""The replica path of bench.py (one process per GPU, no collective on the data) with two
gloo ranks on the CPU: barriers, the maximum of the per-rank times, the whole-job rate,
and the reference arm doing no work on ranks other than 0."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    from paper_2603_24881_gb300 import replicas
    r, w, loc = replicas.ranks_from_env()
    dist = replicas.init(w, "gloo")
    replicas.barrier(dist)
    # each rank "timed" a different interval; all must agree on the maximum
    t = replicas.max_over_ranks(dist, 1.0 + r)
    rate = replicas.whole_job_rate(100.0, w, t)
    replicas.barrier(dist)
    dist.destroy_process_group()
    q.put((r, w, loc, t, rate))


def test_two_gloo_ranks_agree_on_max_time_and_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[3] == 2.0 for o in out)             # max over ranks of 1.0, 2.0
    assert all(o[4] == pytest.approx(100.0) for o in out)  # 2 ranks x 100 units / 2 s


def test_single_process_needs_no_group(monkeypatch):
    from paper_2603_24881_gb300 import replicas
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert replicas.ranks_from_env() == (0, 1, 0)
    assert replicas.init(1, "gloo") is None
    assert replicas.max_over_ranks(None, 3.5) == 3.5
    assert replicas.whole_job_rate(10.0, 1, 2.0) == 5.0


def test_reference_arm_idles_on_other_ranks(capsys):
    sys.path.insert(0, ROOT)
    import bench
    # rank 1 of 2 returns at once without output (rank 0 alone runs the oracle)
    class A:
        steps, warmup, workload, cpu_stride, gpus = 1, 0, "water256", 8, 2
    assert bench.run_reference(A(), 1, 2) is None
    assert capsys.readouterr().out == ""
