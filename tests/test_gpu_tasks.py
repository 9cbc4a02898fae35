"""Sub-box task lists built on the device at commit (the pair-to-block mapping of the
paper's appendix, Algorithm 5) against the host builder (GPW_HOST_TASKS): task records,
sub-box CSR offsets and work lists identical bit for bit, for both tile shapes; and the
Fock build and gradient of a device-built plan identical to the host-built plan's."""
import numpy as np
import pytest

import workloads
import systems

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_24881_gb300 as g
    g.load()
    return g


CASES = {
    "tiny": (workloads.tiny, {}),
    "tiny14": (systems.tiny14, {}),
    "resolved": (systems.resolved, {}),
    "water4": (lambda: workloads.config("water4"), {}),
    "water4_tiles": (lambda: workloads.config("water4"), dict(tile=(8, 8, 32), tile_integ=(8, 4, 64))),
    "water4_tau": (lambda: workloads.config("water4"), dict(tau=True)),
    "f_shells": (lambda: systems.resolved(seed=8, shells=((0, 1), (1, 1), (2, 1), (3, 1)), natm=3), {}),
    "water32": (lambda: workloads.config("water32"), dict(integ_chunk=256)),
    "water4_plain_z": (lambda: workloads.config("water4"), dict(tile_integ=(8, 8, 32))),
}


@pytest.mark.parametrize("name", list(CASES))
def test_device_task_lists_identical(gpw, name):
    make, kw = CASES[name]
    s = make()
    dev = gpw.Plan(s, **kw)
    host = gpw.Plan(s, host_tasks=True, **kw)
    for integ in (False, True):
        a = dev.task_lists(integ)
        b = host.task_lists(integ)
        for x, y, what in zip(a, b, ("tasks", "sub_off", "work")):
            assert x.shape == y.shape, (name, integ, what)
            assert np.array_equal(x, y), (name, integ, what)
    assert dev.stats()["integ_chunk"] == host.stats()["integ_chunk"]
    dev.close()
    host.close()


def test_device_tasks_same_results(gpw):
    s = workloads.config("water4")
    D = torch.as_tensor(s.D, device="cuda")
    a = gpw.Plan(s).fock_grad(D)
    b = gpw.Plan(s, host_tasks=True).fock_grad(D)
    assert a["EH"] == b["EH"] and a["Ex"] == b["Ex"]
    assert torch.equal(a["V"], b["V"]) and torch.equal(a["grad"], b["grad"])


def test_device_tasks_empty_plan(gpw):
    s = workloads.tiny().with_tau(1e6)  # every primitive dropped: no pairs, no tasks
    p = gpw.Plan(s)
    tasks, sub, work = p.task_lists(True)
    assert tasks.shape == (0, 8) and work.shape == (0, 4) and not sub.any()
    out = p.fock(torch.as_tensor(s.D, device="cuda"))
    assert out["EH"] == 0.0 and out["Ex"] == 0.0
