"""gpw_lda_x_noalloc: the exchange step for callers that cannot allocate device memory.

Such callers (an application whose memory pool owns the GPU, a loop that must not
enter the driver's allocator, a library that does not own the CUDA context) get an
entry point whose only working memory is a fixed array inside the library's device
image.  This test calls it through the C ABI, twice in a row on the same buffers,
and checks it against the existing entry point gpw_fock (its E_x, and v_x implied by
its v_H + v_x output minus the Hartree part computed here from rho) at the tolerances
used elsewhere: 1e-8 Ha for the energy, 1e-10 relative for the potential.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _hartree(rho, L):
    # v_H of Eqs. (vH)/(vHG) from rho on the finest grid, G = 0 dropped (torch FFT)
    n = rho.shape
    k = [torch.fft.fftfreq(n[d], d=1.0 / n[d], dtype=torch.float64, device=rho.device)
         * (2 * np.pi / L[d]) for d in range(3)]
    g2 = k[0][:, None, None] ** 2 + k[1][None, :, None] ** 2 + k[2][None, None, :] ** 2
    kern = torch.where(g2 > 0, 4 * np.pi / torch.where(g2 > 0, g2, torch.ones_like(g2)),
                       torch.zeros_like(g2))
    return torch.fft.ifftn(torch.fft.fftn(rho) * kern).real


def test_lda_x_noalloc_matches_fock_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import workloads
    import paper_2603_24881_gb300 as gpw
    lib = gpw.load()
    f = lib.gpw_lda_x_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_double, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    s = workloads.config("water4")
    plan = gpw.Plan(s)
    ref = plan.fock(s.D, want_rho=True, want_v=True)
    rho = ref["rho"]
    L = np.diag(s.lattice)
    n = rho.numel()
    weight = float(np.prod(L)) / n
    vx_ref = ref["v"] - _hartree(rho, L)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        vx = torch.full_like(rho, float("nan"))
        ex = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        rc = f(rho.data_ptr(), n, weight, vx.data_ptr(), ex.data_ptr(), stream.cuda_stream)
        assert rc == 0, lib.gpw_last_error()
        torch.cuda.synchronize()
        assert abs(float(ex.item()) - ref["Ex"]) <= 1e-8
        err = float((vx - vx_ref).abs().max() / vx_ref.abs().max())
        assert err <= 1e-10


def test_lda_x_noalloc_rejects_oversized_grids():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_24881_gb300 as gpw
    lib = gpw.load()
    f = lib.gpw_lda_x_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_double, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = f(x.data_ptr(), 67108864 + 1, 1.0, x.data_ptr(), x.data_ptr(), 0)
    assert rc == -7
    assert b"exceeds the fixed maximum" in lib.gpw_last_error()
    assert f(None, 4, 1.0, x.data_ptr(), x.data_ptr(), 0) == -1
