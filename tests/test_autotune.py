"""Autotuner selection and cache logic, with a model measurement (no GPU)."""
import json

import pytest

import workloads
from paper_2603_24881_gb300 import autotune
from paper_2603_24881_gb300.binding import GpwError


def _model(calls):
    # collocation time depends on tile and warps, integration on its tile and chunk;
    # minima at (4, 4, 32) / 6 warps and (8, 4, 64) / chunk 256; (2, 8, 16) "fails"
    def m(systems, kw):
        calls.append(dict(kw))
        t = kw.get("tile") or (4, 8, 16)
        if t == (2, 8, 16):
            raise GpwError(-1, "model", "unusable")
        ti = kw.get("tile_integ") or (8, 8, 32)
        c = 10.0 + sum(abs(a - b) for a, b in zip(t, (4, 4, 32))) + abs(kw.get("colloc_warps", 0) - 6)
        i = 20.0 + sum(abs(a - b) for a, b in zip(ti, (8, 4, 64))) + abs(kw.get("integ_chunk", 0) - 256) / 100
        return {"collocate": c, "integrate": i}
    return m


def test_tune_picks_minima_and_caches(tmp_path):
    calls = []
    cache = str(tmp_path / "tune.json")
    s = workloads.small_water(4, seed=11)
    ch = autotune.tune(s, cache_path=cache, measure=_model(calls))
    assert ch.tile == (4, 4, 32) and ch.colloc_warps == 6
    assert ch.tile_integ == (8, 4, 64) and ch.integ_chunk == 256
    n = len(calls)
    assert n == len(autotune.TILES) - 1 + len(autotune.WARPS) + len(autotune.TILES_INTEG) + \
        len(autotune.TILES_INTEG_ZWIN) + len(autotune.CHUNKS) + 1  # the failing one once
    data = json.load(open(cache))
    assert len(data) == 1 and "tile=(2, 8, 16)" not in next(iter(data.values()))["timings"]
    # cache hit: no new measurements, same choice
    ch2 = autotune.tune(s, cache_path=cache, measure=_model(calls))
    assert len(calls) == n and ch2.plan_kwargs() == ch.plan_kwargs()
    # refresh measures again
    autotune.tune(s, cache_path=cache, measure=_model(calls), refresh=True)
    assert len(calls) == 2 * n


def test_signature_is_per_workload_class():
    a = workloads.small_water(4, seed=11)
    b = workloads.small_water(8, seed=12)
    assert autotune.signature([a, b]) == autotune.signature([b, a])
    assert autotune.signature([a]) != autotune.signature([b])
    assert autotune.signature([a]) == autotune.signature([workloads.small_water(4, seed=11)])


def test_no_usable_candidate_raises(tmp_path):
    def m(systems, kw):
        raise GpwError(-1, "model", "unusable")
    with pytest.raises(GpwError):
        autotune.tune(workloads.tiny(), cache_path=str(tmp_path / "t.json"), measure=m,
                      tiles=[(4, 8, 16)])


def test_signature_tells_cell_shapes_apart():
    import numpy as np
    import systems
    s = systems.resolved(seed=5)
    t = systems.skewed(seed=5)
    r = systems.rotated(t, systems.rotation(12))
    # the triclinic cell differs from the cubic one; turning a cell keeps its metric, but
    # a cubic cell turned off the axes runs the non-orthogonal kernels
    assert autotune.signature([s]) != autotune.signature([t])
    assert autotune.signature([t]) == autotune.signature([r])
    rc = systems.rotated(s, systems.rotation(12))
    assert not np.all(rc.lattice == np.diag(np.diag(rc.lattice)))
    assert autotune.signature([s]) != autotune.signature([rc])


def test_tune_windowed_integration_candidate(tmp_path):
    # an integration candidate with overlapping z windows is passed to the plan as
    # tile_integ + integ_zwin, and a choice of it round-trips through the cache
    seen = []

    def m(systems, kw):
        seen.append(dict(kw))
        zw = kw.get("integ_zwin")
        i = 5.0 if (kw.get("tile_integ"), zw) == ((8, 8, 16), 48) else 9.0
        return {"collocate": 1.0, "integrate": i}

    cache = str(tmp_path / "tune.json")
    s = workloads.small_water(4, seed=11)
    ch = autotune.tune(s, cache_path=cache, measure=m, tiles=[(4, 8, 16)], warps=[0],
                       chunks=[0], tiles_integ=[(8, 8, 32), (8, 8, 16, 48)])
    assert ch.tile_integ == (8, 8, 16, 48)
    kw = ch.plan_kwargs()
    assert kw["tile_integ"] == (8, 8, 16) and kw["integ_zwin"] == 48
    assert any(k.get("integ_zwin") is None and k.get("tile_integ") == (8, 8, 32) for k in seen)
    ch2 = autotune.tune(s, cache_path=cache, measure=m, tiles=[(4, 8, 16)], warps=[0],
                        chunks=[0], tiles_integ=[(8, 8, 32), (8, 8, 16, 48)])
    assert ch2.plan_kwargs() == kw
