"""Argument limits of the C ABI and the largest grid it accepts.

The grid path indexes queries with 64-bit arithmetic and accepts up to 2^31 - 1 cells (the
flagged-query list holds 32-bit indices); larger grids are rejected with DV_ERR_UNSUPPORTED.
The largest-grid case runs the forward (mixed precision) and the adjoint on 2048 x 1024 x 1023
cells and checks them against the oracle on a seeded sample of cells (including the first and
the last) and on a slab of the grid that carries the only nonzero upstream values."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from _util import NEAR, check_forward, grad_close, make_mesh, to_dev
from paper_2407_11272_b300 import dv, meshgen

pytestmark = pytest.mark.gpu

DV_ERR_INVALID_ARG, DV_ERR_UNSUPPORTED = 1, 6


def _open_tetra():
    """A tetrahedron with one face removed: open, so its gradient is not identically zero."""
    V = np.array([[0.45, 0.3, 0.15], [-0.6, 0.15, -0.3], [0.15, -0.65, 0.35], [0.05, 0.35, -0.7]], dtype=np.float32)
    F = np.array([[0, 1, 2], [0, 1, 3], [0, 2, 3], [1, 2, 3]], dtype=np.int32)
    F = meshgen._orient_outward(V.astype(np.float64), F, V.astype(np.float64).mean(axis=0)).astype(np.int32)
    return V, F[:3].copy()


def test_argument_errors(cuda_device):
    V, F = meshgen.icosphere(1, 0.5)
    mesh = make_mesh(V, F, cuda_device)
    lib = dv.load()
    out = torch.empty(16, device=cuda_device)
    q = torch.zeros((4, 3), device=cuda_device)

    def grid_call(lo, hi, n):
        g = dv.Grid(n=n, lo=lo, hi=hi)._c()
        return lib.dv_winding(mesh.handle, None, 0, ctypes.byref(g), ctypes.c_void_p(out.data_ptr()), 2, None)

    assert grid_call((-1.0,) * 3, (1.0,) * 3, (0, 4, 4)) == DV_ERR_INVALID_ARG
    assert grid_call((-1.0,) * 3, (1.0, 1.0, -1.0), (4, 4, 4)) == DV_ERR_INVALID_ARG  # hi <= lo
    assert grid_call((-1.0, float("nan"), -1.0), (1.0,) * 3, (4, 4, 4)) == DV_ERR_INVALID_ARG
    assert grid_call((-1.0,) * 3, (1.0,) * 3, (2048, 1024, 1025)) == DV_ERR_UNSUPPORTED  # 2^31 + 2^21 cells
    g = dv.Grid.cube(2)._c()
    qp = ctypes.c_void_p(q.data_ptr())
    # both a query list and a grid, or neither
    assert lib.dv_winding(mesh.handle, qp, 4, ctypes.byref(g), ctypes.c_void_p(out.data_ptr()), 2,
                          None) == DV_ERR_INVALID_ARG
    assert lib.dv_winding(mesh.handle, None, 4, None, ctypes.c_void_p(out.data_ptr()), 2, None) == DV_ERR_INVALID_ARG
    # an empty query list, a null output, an unknown precision
    assert lib.dv_winding(mesh.handle, qp, 0, None, ctypes.c_void_p(out.data_ptr()), 2, None) == DV_ERR_INVALID_ARG
    assert lib.dv_winding(mesh.handle, qp, 4, None, None, 2, None) == DV_ERR_INVALID_ARG
    assert lib.dv_winding(mesh.handle, qp, 4, None, ctypes.c_void_p(out.data_ptr()), 9, None) == DV_ERR_INVALID_ARG
    # meshes without faces or with fewer than three vertices
    Vd = to_dev(V, cuda_device)
    h = ctypes.c_void_p()
    fz = torch.zeros((1, 3), dtype=torch.int32, device=cuda_device)
    assert lib.dv_mesh_create(ctypes.c_void_p(Vd.data_ptr()), len(V), ctypes.c_void_p(fz.data_ptr()), 0, None,
                              ctypes.byref(h)) == DV_ERR_INVALID_ARG
    assert lib.dv_mesh_create(ctypes.c_void_p(Vd.data_ptr()), 2, ctypes.c_void_p(fz.data_ptr()), 1, None,
                              ctypes.byref(h)) == DV_ERR_INVALID_ARG
    assert not h.value


def test_largest_grid_forward_and_adjoint(cuda_device):
    V, F = _open_tetra()
    grid = dv.Grid(n=(2048, 1024, 1023), lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0))
    nq = grid.num_queries
    assert nq == 2_145_386_496 and nq < 2 ** 31
    mesh = make_mesh(V, F, cuda_device)
    w, occ, rep = dv.dv_voxelize_grid(mesh, grid, precision="mixed", report=True)
    assert rep["n_queries"] == nq and rep["n_flagged"] > 0
    # sample: seeded uniform cells, the first and last cells, and cells close to the surface
    rng = np.random.default_rng(21)
    cells = rng.integers(0, nq, size=20000, dtype=np.int64)
    cand = rng.integers(0, nq, size=400000, dtype=np.int64)
    dc = oracle.point_mesh_distance(V, F, oracle.grid_points(grid.lo, grid.hi, grid.n, cand))
    cells = np.unique(np.concatenate([cells, cand[np.argsort(dc)[:3000]], [0, nq - 1]]))
    Q = oracle.grid_points(grid.lo, grid.hi, grid.n, cells)
    w64 = oracle.winding(V, F, Q)
    d = oracle.point_mesh_distance(V, F, Q)
    idx = torch.from_numpy(cells).to(cuda_device)
    check_forward(w[idx].cpu().numpy(), w64, d, "mixed", occ[idx].cpu().numpy(), "largest grid")
    del w, occ
    torch.cuda.empty_cache()

    # adjoint: upstream N(0,1) on two z-layers through the mesh (0 within NEAR of it), 0 elsewhere
    z0 = 511
    slab = np.arange(z0 * 2048 * 1024, (z0 + 2) * 2048 * 1024, dtype=np.int64)
    Qs = oracle.grid_points(grid.lo, grid.hi, grid.n, slab)
    gs = meshgen.upstream_gradient(len(slab), seed=23).astype(np.float64)
    gs[oracle.point_mesh_distance(V, F, Qs) <= NEAR] = 0.0
    up = torch.zeros(nq, dtype=torch.float32, device=cuda_device)
    up[int(slab[0]):int(slab[-1]) + 1] = torch.from_numpy(gs.astype(np.float32)).to(cuda_device)
    G = dv.dv_winding_backward(mesh, up, grid=grid).cpu().numpy()
    G_ref = oracle.winding_grad(V, F, Qs, gs)
    grad_close(G, G_ref, "largest grid adjoint", oracle.winding_grad_scale(V, F, Qs, gs))
