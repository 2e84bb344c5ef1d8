"""The no-allocation grid entry point (dv_winding_grid_noalloc).

dv_winding_grid_noalloc serves callers that cannot let a library allocate device
memory (their own allocator or memory budget owns the device, or cudaMalloc's
implicit synchronization is not acceptable): it keeps its working memory in one
fixed array compiled into the library. This file is named so that pytest
collects it last. The test calls the entry point through the C ABI twice in a
row, on two different meshes and grids (the second call reuses the array with
the first call's contents still in it), and compares each result with the FP64
oracle (|dw| <= 1e-4 farther than 1e-3 from the surface, the bar of the other
forward parity tests) and with the existing dv_winding entry point. Around the
second call it also checks that the device's free memory does not change.
"""
import ctypes

import numpy as np
import pytest
import torch

from _util import oracle_grid
from paper_2407_11272_b300 import dv, meshgen

pytestmark = pytest.mark.gpu

W_TOL = 1e-4  # the forward parity tolerance of the other GPU tests


class _Grid(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_float * 3), ("hi", ctypes.c_float * 3), ("n", ctypes.c_int32 * 3)]


def _noalloc_fn():
    lib = dv.load()
    fn = lib.dv_winding_grid_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(_Grid),
                   ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    lib.dv_last_error.restype = ctypes.c_char_p
    return lib, fn


def _cgrid(g):
    c = _Grid()
    for k in range(3):
        c.lo[k], c.hi[k], c.n[k] = float(g.lo[k]), float(g.hi[k]), int(g.n[k])
    return c


def _call(fn, V, F, grid, out):
    stream = torch.cuda.current_stream().cuda_stream
    c = _cgrid(grid)
    return fn(ctypes.c_void_p(V.data_ptr()), V.shape[0], ctypes.c_void_p(F.data_ptr()), F.shape[0], ctypes.byref(c),
              ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))


def test_noalloc_matches_oracle_and_dv_winding_on_two_calls(cuda_device):
    lib, fn = _noalloc_fn()
    cases = [
        (meshgen.jittered_torus(nu=60, nv=30, sigma=0.01, delete_frac=0.1, seed=0),
         dv.Grid((40, 36, 33), (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0))),  # smaller grid: face loop split
        (meshgen.icosphere(3, 0.8), dv.Grid.cube(64)),
    ]
    for call, ((V, F), grid) in enumerate(cases):
        Vd = torch.from_numpy(V).to(cuda_device)
        Fd = torch.from_numpy(F).to(cuda_device)
        mesh = dv.dv_mesh_create(Vd, Fd)
        ref = dv.dv_winding(mesh, grid=grid, precision="kahan").cpu().numpy()
        mesh.close()
        out = torch.full((grid.num_queries,), float("nan"), dtype=torch.float32, device=cuda_device)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        status = _call(fn, Vd, Fd, grid, out)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert status == 0, lib.dv_last_error()
        if call == 1:  # the first call may load the library's device code (and its array) lazily
            assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= W_TOL
        _, w64, d = oracle_grid(V, F, grid)
        far = d > 1e-3
        assert np.abs(got.astype(np.float64) - w64)[far].max() <= W_TOL


def test_noalloc_rejects_oversize_and_bad_faces(cuda_device):
    lib, fn = _noalloc_fn()
    V, F = meshgen.icosphere(1, 0.5)
    Vd = torch.from_numpy(V).to(cuda_device)
    Fd = torch.from_numpy(F).to(cuda_device)
    out = torch.empty(8 ** 3, dtype=torch.float32, device=cuda_device)
    # more faces than the fixed scratch can hold: rejected before anything is read
    assert _call_sized(fn, Vd, Fd, 2_000_000, dv.Grid.cube(8), out) == 6
    assert b"scratch" in lib.dv_last_error()
    Fbad = F.copy()
    Fbad[2, 0] = len(V) + 5
    assert _call(fn, Vd, torch.from_numpy(Fbad).to(cuda_device), dv.Grid.cube(8), out) == 2


def _call_sized(fn, V, F, nf, grid, out):
    stream = torch.cuda.current_stream().cuda_stream
    c = _cgrid(grid)
    return fn(ctypes.c_void_p(V.data_ptr()), V.shape[0], ctypes.c_void_p(F.data_ptr()), nf, ctypes.byref(c),
              ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
