"""CPU-only checks of the native library: it builds for sm_103a, loads, exports every
function that include/dv_api.h declares, and rejects bad arguments on the host
before touching the GPU. No kernel runs here."""
import ctypes
import re
from pathlib import Path

import pytest

from paper_2407_11272_b300 import build as dvbuild

HEADER = Path(__file__).resolve().parents[1] / "include" / "dv_api.h"


def _declared_functions():
    text = re.sub(r"/\*.*?\*/", "", HEADER.read_text(), flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(dv_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    path = dvbuild.build()
    return ctypes.CDLL(str(path))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("dv_mesh_create", "dv_mesh_destroy", "dv_mesh_update_verts", "dv_winding", "dv_voxelize_grid",
                     "dv_winding_backward", "dv_status_string", "dv_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_built_for_sm103a():
    log = (dvbuild.BUILD / "ptxas.log").read_text()
    assert "sm_103a" in log
    assert "arch=compute_103a,code=sm_103a" in " ".join(dvbuild.ARCH)


def test_abi_version_and_status_strings(lib):
    lib.dv_abi_version.restype = ctypes.c_int
    assert lib.dv_abi_version() == 1
    lib.dv_status_string.restype = ctypes.c_char_p
    lib.dv_status_string.argtypes = [ctypes.c_int]
    assert lib.dv_status_string(0) == b"DV_OK"
    assert lib.dv_status_string(5) == b"DV_ERR_TIMEOUT"
    assert lib.dv_status_string(99) == b"DV_ERR_UNKNOWN"


def test_host_side_argument_checks(lib):
    """Invalid arguments are rejected synchronously, before any CUDA call."""
    P, I64 = ctypes.c_void_p, ctypes.c_int64
    lib.dv_mesh_create.argtypes = [P, I64, P, I64, P, ctypes.POINTER(P)]
    lib.dv_mesh_create.restype = ctypes.c_int
    out = P()
    assert lib.dv_mesh_create(None, 10, None, 4, None, ctypes.byref(out)) == 1
    assert lib.dv_mesh_create(P(16), 2, P(16), 4, None, ctypes.byref(out)) == 1  # nv < 3
    assert lib.dv_mesh_create(P(16), 10, P(16), 0, None, ctypes.byref(out)) == 1  # nf < 1
    assert lib.dv_mesh_create(P(16), 10, P(16), 4, None, None) == 1
    lib.dv_last_error.restype = ctypes.c_char_p
    assert b"out is NULL" in lib.dv_last_error()
    lib.dv_winding.argtypes = [P, P, I64, P, P, ctypes.c_int, P]
    lib.dv_winding.restype = ctypes.c_int
    assert lib.dv_winding(None, None, 0, None, None, 0, None) == 1
    lib.dv_winding_backward.restype = ctypes.c_int
    lib.dv_winding_backward.argtypes = [P, P, I64, P, P, P, P]
    assert lib.dv_winding_backward(None, None, 0, None, None, None, None) == 1
    lib.dv_voxelize_grid.restype = ctypes.c_int
    lib.dv_voxelize_grid.argtypes = [P, P, P, P, ctypes.c_int, P, P]
    assert lib.dv_voxelize_grid(None, None, None, None, 0, None, None) == 1
    lib.dv_mesh_destroy.argtypes = [P]
    lib.dv_mesh_destroy(None)  # no-op


def test_binding_names_match_abi():
    from paper_2407_11272_b300 import dv

    for name in ("dv_mesh_create", "dv_mesh_update_verts", "dv_mesh_reserve", "dv_mesh_check", "dv_winding",
                 "dv_voxelize_grid", "dv_winding_backward", "dv_abi_version"):
        assert callable(getattr(dv, name))
    assert dv.dv_abi_version() == 1


def test_binding_rejects_cpu_tensors():
    import torch

    from paper_2407_11272_b300 import dv

    with pytest.raises(TypeError):
        dv.dv_mesh_create(torch.zeros(4, 3), torch.zeros(2, 3, dtype=torch.int32))


def test_oracle_and_product_are_independent():
    """The product package never imports the oracle, and the oracle never imports the product."""
    root = Path(__file__).resolve().parents[1]
    for p in (root / "paper_2407_11272_b300").rglob("*.py"):
        txt = p.read_text()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, flags=re.M), p
    for p in (root / "paper_2407_11272_b300" / "csrc").iterdir():
        if p.is_file():
            assert "oracle" not in p.read_text().lower() or p.suffix == ".py", p
    for p in (root / "oracle").glob("*"):
        if p.suffix == ".py":
            assert not re.search(r"^\s*(import|from)\s+paper_2407_11272_b300", p.read_text(), flags=re.M), p
        if p.suffix in (".c", ".h"):
            assert not re.search(r'#include\s+"', p.read_text()), p  # system headers only


def test_debug_library_exports_the_same_symbols_and_release_has_no_checks(lib):
    """libdv_debug.so (the bounds-checked build) exports every declared symbol; the release
    library answers dv_debug_report with DV_ERR_UNSUPPORTED without touching the GPU."""
    dbg = ctypes.CDLL(str(dvbuild.build(debug=True)))
    missing = [n for n in _declared_functions() if not hasattr(dbg, n)]
    assert not missing, f"debug build misses: {missing}"
    assert "sm_103a" in (dvbuild.BUILD / "debug" / "ptxas.log").read_text()
    I64 = ctypes.c_int64
    c, site, idx, bound = I64(7), ctypes.c_int32(7), I64(7), I64(7)
    lib.dv_debug_report.restype = ctypes.c_int
    lib.dv_debug_report.argtypes = [ctypes.POINTER(I64), ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(I64),
                                    ctypes.POINTER(I64), ctypes.c_int]
    assert lib.dv_debug_report(ctypes.byref(c), ctypes.byref(site), ctypes.byref(idx), ctypes.byref(bound), 0) == 6
    assert c.value == 0


def test_run_batch_rejects_the_default_stream(lib):
    """dv_run_batch captures a CUDA graph on its stream; the legacy default stream (0) cannot be
    captured and is rejected on the host before any CUDA call."""
    buf = (ctypes.c_byte * 256)()  # one request slot; only the stream is examined before the error
    lib.dv_run_batch.restype = ctypes.c_int
    lib.dv_run_batch.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    assert lib.dv_run_batch(ctypes.cast(buf, ctypes.c_void_p), 1, 2, None) == 1
    lib.dv_last_error.restype = ctypes.c_char_p
    assert b"default stream" in lib.dv_last_error()
