"""The server's batch formation and deadlines on the host (no GPU): the policy the GPU
thread applies to its staged requests."""
from dataclasses import dataclass

from paper_2603_24881_gb300.serve import BatchPolicy


@dataclass
class R:
    name: str
    cost: float
    kind: bool = False
    deadline: float | None = None


def names(rs):
    return [r.name for r in rs]


def test_oldest_opens_the_batch_and_order_is_kept():
    p = BatchPolicy(max_batch=8, batch_cost=10.0)
    staged = [R("a", 3), R("b", 3), R("c", 3), R("d", 3)]
    batch, keep, exp = p.form(staged, now=0.0)
    assert names(batch) == ["a", "b", "c"] and names(keep) == ["d"] and exp == []


def test_large_request_runs_alone_and_small_ones_pass_it():
    p = BatchPolicy(max_batch=8, batch_cost=10.0)
    staged = [R("s1", 1), R("big", 50), R("s2", 1), R("s3", 1)]
    batch, keep, _ = p.form(staged, now=0.0)
    assert names(batch) == ["s1", "s2", "s3"] and names(keep) == ["big"]
    batch, keep, _ = p.form(keep + [R("s4", 1)], now=0.0)
    # the oldest (large) request opens its own batch, over the cap
    assert names(batch) == ["big"] and names(keep) == ["s4"]


def test_one_kind_of_cell_per_batch_and_max_batch():
    p = BatchPolicy(max_batch=2, batch_cost=100.0)
    staged = [R("o1", 1), R("k1", 1, kind=True), R("o2", 1), R("o3", 1)]
    batch, keep, _ = p.form(staged, now=0.0)
    assert names(batch) == ["o1", "o2"] and names(keep) == ["k1", "o3"]


def test_expired_requests_leave_before_the_batch_is_formed():
    p = BatchPolicy(max_batch=8, batch_cost=100.0)
    staged = [R("late", 1, deadline=1.0), R("ok", 1, deadline=5.0), R("free", 1)]
    batch, keep, exp = p.form(staged, now=2.0)
    assert names(exp) == ["late"] and names(batch) == ["ok", "free"] and keep == []
    assert BatchPolicy.expired(staged[0], 2.0) and not BatchPolicy.expired(staged[1], 2.0)
    assert p.form([R("x", 1, deadline=0.5)], now=1.0) == ([], [], [staged[0].__class__("x", 1, deadline=0.5)])


def test_every_request_is_placed_exactly_once():
    import random
    rng = random.Random(3)
    p = BatchPolicy(max_batch=5, batch_cost=7.0)
    staged = [R(str(i), rng.choice([0.5, 1, 2, 4, 9]), kind=rng.random() < 0.3,
                deadline=rng.choice([None, 3.0, 10.0])) for i in range(60)]
    seen = []
    now = 0.0
    while staged:
        batch, keep, exp = p.form(staged, now)
        assert len(batch) <= 5 and len({r.kind for r in batch}) <= 1
        if len(batch) > 1:
            assert sum(r.cost for r in batch) <= max(7.0, batch[0].cost)
        seen += batch + exp
        staged = keep
        now += 0.25
    assert sorted(int(r.name) for r in seen) == list(range(60))


def test_small_only_batches_for_the_priority_lane():
    p = BatchPolicy(max_batch=8, batch_cost=10.0, small_cost=2.0)
    staged = [R("big", 5), R("s1", 1), R("mid", 3), R("s2", 1), R("k", 1, kind=True)]
    batch, keep, _ = p.form(staged, now=0.0, small_only=True)
    assert names(batch) == ["s1", "s2"] and names(keep) == ["big", "mid", "k"]
    batch, keep, _ = p.form([R("big", 5)], now=0.0, small_only=True)
    assert batch == [] and names(keep) == ["big"]


def test_lane_batches_have_their_own_cap():
    p = BatchPolicy(max_batch=8, batch_cost=10.0, small_cost=2.0, lane_cost=3.0)
    staged = [R("s1", 1), R("s2", 1), R("s3", 1), R("s4", 1)]
    batch, keep, _ = p.form(staged, now=0.0, small_only=True)
    assert names(batch) == ["s1", "s2", "s3"] and names(keep) == ["s4"]
    batch, keep, _ = p.form(staged, now=0.0)            # the regular cap
    assert names(batch) == ["s1", "s2", "s3", "s4"] and keep == []
    assert BatchPolicy(batch_cost=7.0).lane_cost == 7.0   # default: the regular cap


def test_kinds_with_integration_shapes_batch_apart():
    # the server's kind of a request: (non-orthogonal cell, integration sub-boxes, z
    # window); plans of different kernels never share a batch, while those of one kind do
    water = (False, (8, 8, 16), 48)
    f_shells = (False, (8, 8, 32), 32)
    skew = (True, (4, 8, 16), 16)
    p = BatchPolicy(max_batch=8, batch_cost=100.0)
    staged = [R("w1", 1, kind=water), R("f1", 1, kind=f_shells), R("w2", 1, kind=water),
              R("s1", 1, kind=skew), R("f2", 1, kind=f_shells), R("w3", 1, kind=water)]
    out = []
    while staged:
        batch, staged, _ = p.form(staged, now=0.0)
        assert len({r.kind for r in batch}) == 1
        out.append(names(batch))
    assert out == [["w1", "w2", "w3"], ["f1", "f2"], ["s1"]]
