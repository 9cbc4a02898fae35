"""The C-ABI library loads and exports every entry point that include/gpw.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import paper_2603_24881_gb300 as gpw
from paper_2603_24881_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:int|void|const char\*)\s+(gpw_\w+)\s*\(", src, flags=re.M)
    return names


def test_header_declares_the_path():
    names = _declared()
    for n in ["gpw_plan", "gpw_eval_rho", "gpw_eval_mat", "gpw_eval_mat_ip1", "gpw_fock"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    gpw.load()  # builds the library in-tree when it is missing
    lib = ctypes.CDLL(gpw.lib_path())
    for n in _declared():
        assert hasattr(lib, n), n
    assert set(binding.EXPORTS) <= set(_declared())


def test_strerror_without_gpu():
    lib = gpw.load()
    assert lib.gpw_strerror(0) == b"ok"
    assert lib.gpw_strerror(-1) == b"invalid argument"
    assert lib.gpw_strerror(-7) == b"size beyond a fixed limit"


def test_tile_support_mask_without_gpu():
    # host-only query: collocation shapes are integration shapes too; two shapes exist
    # for integration only; anything else has no kernels
    lib = gpw.load()
    for t in binding.TILES:
        assert lib.gpw_tile_supported(*t) == 3, t
    for t in set(binding.TILES_INTEG) - set(binding.TILES):
        assert lib.gpw_tile_supported(*t) == 2, t
    assert lib.gpw_tile_supported(3, 8, 16) == 0
    assert lib.gpw_tile_supported(0, 0, 0) == 0
    # z windows: every integration shape with its own height, and the overlapping ones
    for t in binding.TILES_INTEG:
        assert lib.gpw_integ_zwin_supported(*t, t[2]) == 1, t
    for t in binding.TILES_INTEG_ZWIN:
        assert lib.gpw_integ_zwin_supported(*t) == 1, t
    assert lib.gpw_integ_zwin_supported(8, 8, 16, 32) == 0
    assert lib.gpw_integ_zwin_supported(3, 8, 16, 16) == 0


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # no CPU fallback: without the built library (and without building it) loading raises
    monkeypatch.setattr(binding, "_LIB", None)
    monkeypatch.setattr(binding._build, "LIB", str(tmp_path / "libgpw.so"))
    import pytest
    with pytest.raises(RuntimeError):
        binding.load(build_if_missing=False)
