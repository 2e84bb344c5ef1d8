"""Eq. (4) dipole surrogate (forward and adjoint), the autograd wrapper, and a small morphing run.

The dipole forward is compared with the oracle's Eq. (4); its adjoint with FP64 central
differences of the oracle's Eq. (4) (only the faces incident to a perturbed vertex change,
so only those are re-evaluated); the autograd path with the oracle's exact gradient."""
import numpy as np
import pytest
import torch

import oracle
from _util import NEAR, grad_close, make_mesh, oracle_grid, to_dev
from paper_2407_11272_b300 import dv, meshgen
from paper_2407_11272_b300.autograd import WindingNumber
from paper_2407_11272_b300.morph import ellipsoid_union_target, morph

pytestmark = pytest.mark.gpu


def _dipole_fd(V, F, Q, g, ids, h=1e-5):
    V = V.astype(np.float64)
    out = np.zeros((len(ids), 3))
    for t, vid in enumerate(ids):
        inc = np.any(F == vid, axis=1)
        for k in range(3):
            Vp, Vm = V.copy(), V.copy()
            Vp[vid, k] += h
            Vm[vid, k] -= h
            out[t, k] = g @ (oracle.dipole_winding(Vp, F[inc], Q) - oracle.dipole_winding(Vm, F[inc], Q)) / (2 * h)
    return out


@pytest.mark.parametrize("mesh_kind", ["icosphere", "torus"])
def test_dipole_forward_matches_oracle(cuda_device, mesh_kind):
    V, F = (meshgen.icosphere(3, 0.6) if mesh_kind == "icosphere"
            else meshgen.jittered_torus(nu=40, nv=20, sigma=0.01, delete_frac=0.1, seed=2))
    grid = dv.Grid.cube(24)
    Q = oracle.grid_queries(grid.lo, grid.hi, grid.n)
    w64 = oracle.dipole_winding(V, F, Q)
    d = oracle.point_mesh_distance(V, F, Q)
    mesh = make_mesh(V, F, cuda_device)
    w = dv.dv_dipole_winding(mesh, grid=grid).cpu().numpy().astype(np.float64)
    far = d > 0.05
    assert np.abs(w - w64)[far].max() < 1e-4
    # list path on the same points (rounded to FP32): same bar against the oracle
    wl = dv.dv_dipole_winding(mesh, queries=to_dev(Q.astype(np.float32), cuda_device)).cpu().numpy()
    assert np.abs(wl.astype(np.float64) - w64)[far].max() < 1e-4


def test_dipole_backward_matches_fd(cuda_device):
    V, F = meshgen.icosphere(2, 0.6)
    grid = dv.Grid.cube(16)
    Q = oracle.grid_queries(grid.lo, grid.hi, grid.n)
    d = oracle.point_mesh_distance(V, F, Q)
    g = meshgen.upstream_gradient(len(Q), seed=3).astype(np.float64)
    g[d < 0.05] = 0.0  # terms near a centroid grow like 1/r^3: keep FD meaningful
    mesh = make_mesh(V, F, cuda_device)
    G = dv.dv_dipole_backward(mesh, to_dev(g.astype(np.float32), cuda_device), grid=grid).cpu().numpy()
    ids = meshgen.random_vertex_ids(len(V), 24, seed=5)
    grad_close(G[ids], _dipole_fd(V, F, Q, g, ids), "dipole adjoint vs FD")


@pytest.mark.parametrize("n", [(16, 12, 10), (15, 9, 7)])
def test_dipole_backward_grid_matches_list_path(cuda_device, n):
    """The grid adjoint (row sharing, packed pairs; odd rows are padded) and the list adjoint
    (per query) are independent kernels: on the same points they agree to FP32 rounding, and
    both match the oracle's FD on the grid case above."""
    V, F = meshgen.jittered_torus(nu=24, nv=12, sigma=0.01, delete_frac=0.1, seed=4)
    grid = dv.Grid(n=n, lo=(-1.0, -0.9, -1.1), hi=(1.0, 1.1, 0.9))
    Q = oracle.grid_queries(grid.lo, grid.hi, grid.n).astype(np.float32)
    mesh = make_mesh(V, F, cuda_device)
    g = to_dev(meshgen.upstream_gradient(grid.num_queries, seed=12), cuda_device)
    Gg = dv.dv_dipole_backward(mesh, g, grid=grid).cpu().numpy().astype(np.float64)
    Gl = dv.dv_dipole_backward(mesh, g, queries=to_dev(Q, cuda_device)).cpu().numpy().astype(np.float64)
    assert np.linalg.norm(Gg - Gl) <= 1e-4 * np.linalg.norm(Gl)
    wg = dv.dv_dipole_winding(mesh, grid=grid).cpu().numpy()
    wl = dv.dv_dipole_winding(mesh, queries=to_dev(Q, cuda_device)).cpu().numpy()
    # the two paths round the query coordinates differently (FP32 fma vs FP64 then FP32); near a
    # centroid the 1/r^2 dipole term amplifies that relative to |w|
    assert np.all(np.abs(wg - wl) <= 1e-4 * np.maximum(np.abs(wl), 1.0))


def test_autograd_exact_matches_oracle_gradient(cuda_device):
    V, F = meshgen.jittered_torus(nu=60, nv=30, sigma=0.01, delete_frac=0.1, seed=0)
    grid = dv.Grid.cube(24)
    Q, _, d = oracle_grid(V, F, grid)
    g = meshgen.upstream_gradient(len(Q), seed=1).astype(np.float64)
    g[d <= NEAR] = 0.0
    Vd = to_dev(V, cuda_device).requires_grad_(True)
    field = WindingNumber(Vd, to_dev(F, cuda_device), grid=grid, kind="exact", precision="mixed")
    w = field(Vd)
    (w * to_dev(g.astype(np.float32), cuda_device)).sum().backward()
    G_ref = oracle.winding_grad(V, F, Q, g)
    grad_close(Vd.grad.cpu().numpy(), G_ref, "autograd exact", oracle.winding_grad_scale(V, F, Q, g))
    # the forward of the module is the library's winding number
    w2 = dv.dv_winding(make_mesh(V, F, cuda_device), grid=grid, precision="mixed")
    assert torch.equal(w.detach(), w2)


def test_autograd_dipole_matches_library_adjoint(cuda_device):
    V, F = meshgen.icosphere(3, 0.5)
    grid = dv.Grid.cube(20)
    Vd = to_dev(V, cuda_device).requires_grad_(True)
    field = WindingNumber(Vd, to_dev(F, cuda_device), grid=grid, kind="dipole")
    g = to_dev(meshgen.upstream_gradient(grid.num_queries, seed=9), cuda_device)
    (field(Vd) * g).sum().backward()
    ref = dv.dv_dipole_backward(make_mesh(V, F, cuda_device), g, grid=grid)
    assert torch.equal(Vd.grad, ref)


def test_small_morph_dipole_improves_iou(cuda_device):
    V0, F = meshgen.icosphere(3, 0.5)
    grid = dv.Grid.cube(32)
    target = ellipsoid_union_target(grid)
    res = morph(V0, F, target, grid, steps=60, lr=5e-3, surrogate="dipole", device=cuda_device)
    assert res["final_iou"] > res["initial_iou"] + 0.02, res
    ex = morph(V0, F, target, grid, steps=10, lr=5e-3, surrogate="exact", device=cuda_device)
    assert np.isfinite(ex["final_loss"])

