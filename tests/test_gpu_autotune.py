"""The autotuner on the GPU: a measured choice among the candidates, cached, and a plan
built with it gives the same Fock build as the default plan."""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_24881_gb300 as g
    g.load()
    return g


def test_tune_single_and_batch(gpw, tmp_path):
    from paper_2603_24881_gb300 import autotune
    cache = str(tmp_path / "tune.json")
    s = workloads.small_water(4, seed=11)
    kw = dict(tiles=[(4, 8, 16), (4, 4, 32)], tiles_integ=[(8, 8, 32), (4, 8, 64)],
              warps=(0, 4), chunks=(0, 64), cache_path=cache, steps=1)
    ch = autotune.tune(s, **kw)
    assert ch.tile in kw["tiles"] and ch.tile_integ in kw["tiles_integ"]
    assert ch.colloc_warps in kw["warps"] and ch.integ_chunk in kw["chunks"]
    assert all(v > 0 for v in ch.timings.values()) and len(ch.timings) == 8
    p = gpw.Plan(s, **ch.plan_kwargs())
    st = p.stats()
    assert st["tile"] == ch.tile and st["tile_integ"] == ch.tile_integ
    if ch.colloc_warps:
        assert st["colloc_warps"] == ch.colloc_warps
    if ch.integ_chunk:
        assert st["integ_chunk"] == ch.integ_chunk
    r = p.fock_grad(s.D)
    p.close()
    q = gpw.Plan(s)
    r0 = q.fock_grad(s.D)
    q.close()
    V, V0 = r["V"].cpu().numpy(), r0["V"].cpu().numpy()
    assert np.max(np.abs(V - V0)) <= 1e-10 * np.max(np.abs(V0))
    assert abs(r["EH"] - r0["EH"]) <= 1e-8 and abs(r["Ex"] - r0["Ex"]) <= 1e-8
    assert np.max(np.abs(r["grad"].cpu().numpy() - r0["grad"].cpu().numpy())) <= 1e-7
    # a batch of two cells is its own workload class
    chb = autotune.tune([s, workloads.tiny()], **kw)
    assert chb.tile in kw["tiles"]
    import json
    assert len(json.load(open(cache))) == 2


def test_explicit_warps_and_chunk(gpw):
    s = workloads.small_water(4, seed=11)
    p = gpw.Plan(s, colloc_warps=4, integ_chunk=32)
    st = p.stats()
    assert st["colloc_warps"] == 4 and st["integ_chunk"] == 32
    r = p.fock_grad(s.D)
    p.close()
    q = gpw.Plan(s)
    r0 = q.fock_grad(s.D)
    q.close()
    assert np.max(np.abs(r["V"].cpu().numpy() - r0["V"].cpu().numpy())) <= \
        1e-10 * float(r0["V"].abs().max())
    with pytest.raises(gpw.GpwError):
        gpw.Plan(s, colloc_warps=5)


def test_server_with_tuned_shapes(gpw, tmp_path, monkeypatch):
    from paper_2603_24881_gb300 import autotune
    from paper_2603_24881_gb300.serve import Server
    monkeypatch.setenv("GPW_AUTOTUNE_CACHE", str(tmp_path / "srv.json"))
    monkeypatch.setattr(autotune, "TILES", [(4, 8, 16), (8, 8, 16)])
    monkeypatch.setattr(autotune, "TILES_INTEG", [(8, 8, 32), (4, 8, 64)])
    monkeypatch.setattr(autotune, "WARPS", (0,))
    monkeypatch.setattr(autotune, "CHUNKS", (0, 128))
    systems = [workloads.small_water(4, seed=101), workloads.small_water(8, seed=102)]
    with Server(max_batch=4, tune_with=systems) as srv:
        assert srv.choice is not None
        futs = [srv.submit(x, want_grad=True) for x in systems]
        res = [f.result(timeout=300) for f in futs]
    for x, r in zip(systems, res):
        p = gpw.Plan(x)
        ref = p.fock_grad(x.D)
        p.close()
        assert abs(r.EH - ref["EH"]) <= 1e-8
        assert np.max(np.abs(r.V - ref["V"].cpu().numpy())) <= 1e-10 * float(ref["V"].abs().max())
