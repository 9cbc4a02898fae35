"""GPW_FAST_BLOCK_PRUNE, the per-block value screening of App. Alg. 5, outside the strict
definition: the device-built collocation lists equal the host builder's; every task the
screening leaves out lies, point by point, farther than the pair's extent R_p from its
centre P (R_p from the oracle); the integration lists are untouched; and the densities,
energies, V and gradients stay within 1e-6 relative of the oracle's strict build."""
import numpy as np
import pytest

import oracle
import systems
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "water4": lambda: workloads.config("water4"),
    "water4_triclinic": lambda: workloads.config("water4_triclinic"),
    "f_shells": lambda: systems.resolved(seed=8, shells=((0, 1), (1, 1), (2, 1), (3, 1)), natm=3,
                                         tau=1e-6),
}


@pytest.fixture(scope="module")
def gpw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_24881_gb300 as g
    g.load()
    return g


def _records(tasks):
    """(pair, box lo offsets t, extents m) of every task record (8 int32 per task)."""
    r = tasks.astype(np.int64)
    pair = r[:, 0]
    m = np.stack([r[:, 1] & 255, (r[:, 1] >> 8) & 255, (r[:, 1] >> 16) & 255], axis=1)
    t = np.stack([r[:, 4] & 0xffff, r[:, 5] & 0xffff, r[:, 6] & 0xffff], axis=1)
    rank = r[:, 3]
    return pair, t, m, rank


@pytest.mark.parametrize("name", list(CASES))
def test_pruned_lists(gpw, name):
    s = CASES[name]()
    dev = gpw.Plan(s, fast_prune=True)
    host = gpw.Plan(s, fast_prune=True, host_tasks=True)
    full = gpw.Plan(s)
    for integ in (False, True):
        a, b = dev.task_lists(integ), host.task_lists(integ)
        for x, y in zip(a, b):
            assert x.shape == y.shape and np.array_equal(x, y), (name, integ)
    # integration lists are those of the strict plan
    for x, y in zip(dev.task_lists(True), full.task_lists(True)):
        assert np.array_equal(x, y)
    kept = dev.task_lists(False)[0]
    allt = full.task_lists(False)[0]
    assert 0 < len(kept) <= len(allt)
    # every left-out task lies wholly beyond R_p (the oracle's extent of its pair)
    kp, _, _, kr = _records(kept)
    keyk = set(zip(kp.tolist(), kr.tolist()))
    pair, t, m, rank = _records(allt)
    gone = np.array([(p, r) not in keyk for p, r in zip(pair.tolist(), rank.tolist())])
    assert len(kept) + int(gone.sum()) == len(allt)
    op = oracle.Plan(s)
    ext = {tuple(row[:5]): R for row, R in zip(np.concatenate([op.ab, op.img], axis=1).tolist(), op.R)}
    pt = dev.pair_table(sort=False)
    lat = np.asarray(s.lattice, dtype=np.float64)
    pr = op.prims
    for i in np.nonzero(gone)[0]:
        p = int(pair[i])
        a_, b_, n0, n1, n2, lev = (int(x) for x in pt[p, :6])
        A = pr["center"][a_]
        B = pr["center"][b_] + np.array([n0, n1, n2], dtype=np.float64) @ lat
        al, bl = float(pr["alpha"][a_]), float(pr["alpha"][b_])
        P = (al * A + bl * B) / (al + bl)
        lo = pt[p, 6:9] + t[i]
        ax = [np.arange(lo[d], lo[d] + m[i, d]) for d in range(3)]
        I = np.stack(np.meshgrid(*ax, indexing="ij"), axis=-1).reshape(-1, 3)
        r = (I / op.meshes[lev].astype(np.float64)) @ lat
        assert np.min(np.linalg.norm(r - P, axis=1)) > ext[(a_, b_, n0, n1, n2)], (name, i)
    for p in (dev, host, full):
        p.close()


@pytest.mark.parametrize("name", list(CASES))
def test_pruned_results_within_1e6(gpw, name):
    s = CASES[name]()
    op = oracle.Plan(s)
    ref = op.fock(s.D)
    gp = gpw.Plan(s, fast_prune=True)
    out = gp.fock_grad(s.D)
    f = gp.fock(s.D, want_rho=True)
    rho_ref = ref["rho_fine"]
    assert np.max(np.abs(f["rho"].cpu().numpy() - rho_ref)) <= 1e-6 * np.max(np.abs(rho_ref))
    for k in ("EH", "Ex"):
        assert abs(out[k] - ref[k]) <= 1e-6 * abs(ref[k]), k
    V = out["V"].cpu().numpy()
    assert np.max(np.abs(V - ref["V"])) <= 1e-6 * np.max(np.abs(ref["V"]))
    g = op.grad_levels(s.D, ref["v_levels"])
    assert np.max(np.abs(out["grad"].cpu().numpy() - g)) <= 1e-6 * max(1.0, np.max(np.abs(g)))
    assert gp.check_device() == 0
    gp.close()
