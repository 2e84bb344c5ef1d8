"""The grid forward and the FP64 re-evaluation walk the faces in strip order (consecutive faces
share two vertices). These cases stress that order against the oracle: meshes whose strips are
all singletons (triangle soup), meshes with degenerate, duplicated and non-manifold faces, long
strips cut by face splits (small grids split the face loop across CTAs, so a split starts in
the middle of a strip and must warm up on the two events before it), and a ragged grid."""
import numpy as np
import pytest
import torch

import oracle
from _util import check_forward, make_mesh, oracle_grid
from paper_2407_11272_b300 import dv, meshgen

pytestmark = pytest.mark.gpu


def _soup(n, seed):
    """n independent random triangles in [-0.8, 0.8]^3 (every strip is one face)."""
    rng = np.random.default_rng(seed)
    V = rng.uniform(-0.8, 0.8, size=(3 * n, 3)).astype(np.float32)
    F = np.arange(3 * n, dtype=np.int32).reshape(n, 3)
    return V, F


def _odd_topology():
    """Icosphere plus a fin sharing an edge with it (a non-manifold edge), a repeated face, a
    face with a repeated vertex index, and an unused vertex."""
    V, F = meshgen.icosphere(2, 0.6)
    a, b = F[0, 0], F[0, 1]
    V = np.vstack([V, [[0.9, 0.9, 0.9], [0.05, 0.02, 0.03]]]).astype(np.float32)
    fin = len(V) - 2
    extra = np.array([[a, b, fin], F[5], [F[7, 0], F[7, 0], F[7, 1]]], dtype=np.int32)
    return V, np.vstack([F, extra]).astype(np.int32)


@pytest.mark.parametrize("kind", ["soup", "odd", "long_strips_split"])
@pytest.mark.parametrize("prec", ["fp32", "kahan", "mixed"])
def test_strip_order_forward_matches_oracle(cuda_device, kind, prec):
    if kind == "soup":
        V, F = _soup(300, seed=11)
        grid = dv.Grid.cube(20)
    elif kind == "odd":
        V, F = _odd_topology()
        grid = dv.Grid.cube(24)
    else:
        V, F = meshgen.icosphere(4, 0.7)  # strips of hundreds of faces; 12^3 grid -> many splits
        grid = dv.Grid.cube(12)
    ev_vert, ev_face = dv.dv_build_strips(F, len(V))
    if kind == "soup":
        assert len(ev_vert) == 3 * len(F)
    if kind == "long_strips_split":
        assert len(ev_vert) < 1.1 * len(F)
    _, w64, d = oracle_grid(V, F, grid)
    mesh = make_mesh(V, F, cuda_device)
    w, occ, _ = dv.dv_voxelize_grid(mesh, grid, precision=prec)
    check_forward(w.cpu().numpy(), w64, d, prec, occ.cpu().numpy(), f"{kind}/{prec}")


def test_strip_order_ragged_grid(cuda_device):
    """Grid sizes that are not multiples of the per-thread query tile (4 x 2)."""
    V, F = meshgen.jittered_torus(nu=30, nv=15, sigma=0.01, delete_frac=0.2, seed=4)
    grid = dv.Grid(lo=(-1.0, -0.9, -1.1), hi=(1.0, 1.2, 0.9), n=(13, 7, 5))
    Q = oracle.grid_queries(grid.lo, grid.hi, grid.n)
    w64 = oracle.winding(V, F, Q)
    d = oracle.point_mesh_distance(V, F, Q)
    mesh = make_mesh(V, F, cuda_device)
    for prec in ("fp32", "mixed"):
        w, occ, _ = dv.dv_voxelize_grid(mesh, grid, precision=prec)
        check_forward(w.cpu().numpy(), w64, d, prec, occ.cpu().numpy(), f"ragged/{prec}")


@pytest.mark.parametrize("kind", ["torus", "soup"])
def test_list_path_near_surface_queries(cuda_device, kind):
    """Query lists in strip order, with many queries within 1e-3 of a face (centroids pushed
    off the face by 1e-6 .. 9e-4, and points next to edges and vertices) among uniform ones:
    every near query must come back at FP64 accuracy (the binned near-surface selection must
    find all of them), far ones within the FP32 bar."""
    if kind == "torus":
        V, F = meshgen.jittered_torus(nu=80, nv=40, sigma=0.01, delete_frac=0.1, seed=5)
    else:
        V, F = _soup(400, seed=13)
    rng = np.random.default_rng(17)
    V64 = V.astype(np.float64)
    P = V64[F]
    cen = P.mean(axis=1)
    n = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    pick = rng.choice(len(F), size=1500, replace=True)
    off = rng.uniform(1e-6, 9e-4, size=len(pick)) * rng.choice([-1.0, 1.0], size=len(pick))
    near_c = cen[pick] + off[:, None] * n[pick]
    t = rng.uniform(0.05, 0.95, size=len(pick))[:, None]
    near_e = P[pick, 0] * t + P[pick, 1] * (1 - t) + rng.normal(scale=3e-4, size=(len(pick), 3))
    near_v = P[pick, 2] + rng.normal(scale=3e-4, size=(len(pick), 3))
    far = rng.uniform(-1, 1, size=(6000, 3))
    Q = np.vstack([near_c, near_e, near_v, far]).astype(np.float32)
    w64 = oracle.winding(V, F, Q)
    d = oracle.point_mesh_distance(V, F, Q)
    assert (d <= 1e-3).sum() > 3000
    mesh = make_mesh(V, F, cuda_device)
    Qd = torch.from_numpy(Q).to(cuda_device)
    for prec in ("kahan", "mixed"):
        w = dv.dv_winding(mesh, queries=Qd, precision=prec).cpu().numpy()
        check_forward(w, w64, d, prec, None, f"list/{kind}/{prec}")
