"""The boundary form of the adjoint (dv_winding_backward_boundary): the same dL/dV as the
face-by-face adjoint, evaluated on the directed edges with nonzero net multiplicity. Checked
against the oracle's FP64 face-by-face gradient (grid and list queries, open, closed,
non-manifold and degenerate meshes) and against the face-by-face GPU adjoint."""
import numpy as np
import pytest
import torch

import oracle
from _util import NEAR, grad_close, make_mesh, oracle_grid, to_dev
from paper_2407_11272_b300 import dv, meshgen

pytestmark = pytest.mark.gpu


def _net_boundary_count(F):
    """Reference count of undirected edges whose directed uses do not cancel."""
    net = {}
    for t in F:
        for k in range(3):
            u, v = int(t[k]), int(t[(k + 1) % 3])
            if u == v:
                continue
            key = (min(u, v), max(u, v))
            net[key] = net.get(key, 0) + (1 if u < v else -1)
    return sum(1 for m in net.values() if m != 0)


def _masked(n, d, seed):
    g = meshgen.upstream_gradient(n, seed=seed).astype(np.float64)
    g[d <= NEAR] = 0.0
    return g


@pytest.mark.parametrize("n", [24, (25, 17, 9)])
def test_boundary_adjoint_grid_matches_oracle(cuda_device, n):
    V, F = meshgen.jittered_torus(nu=60, nv=30, sigma=0.01, delete_frac=0.1, seed=0)
    grid = dv.Grid.cube(n) if isinstance(n, int) else dv.Grid(n=n, lo=(-1.0, -0.9, -1.1), hi=(1.0, 1.1, 0.9))
    Q, _, d = oracle_grid(V, F, grid)
    g = _masked(len(Q), d, seed=1)
    mesh = make_mesh(V, F, cuda_device)
    assert dv.dv_mesh_num_boundary_edges(mesh) == _net_boundary_count(F) > 0
    gd = to_dev(g.astype(np.float32), cuda_device)
    G = dv.dv_winding_backward_boundary(mesh, gd, grid=grid).cpu().numpy()
    G_ref = oracle.winding_grad(V, F, Q, g)
    grad_close(G, G_ref, f"boundary grid {n}", oracle.winding_grad_scale(V, F, Q, g))
    # vertices off the boundary get exactly 0
    bverts = set()
    for t in F:
        for k in range(3):
            bverts.add((int(t[k]), int(t[(k + 1) % 3])))
    on = np.zeros(len(V), bool)
    for (u, v) in bverts:
        if (v, u) not in bverts:
            on[u] = on[v] = True
    assert np.all(G[~on] == 0.0)
    # and the face-by-face GPU adjoint agrees
    Gf = dv.dv_winding_backward(mesh, gd, grid=grid).cpu().numpy()
    grad_close(G, Gf.astype(np.float64), "boundary vs faces", oracle.winding_grad_scale(V, F, Q, g))


def test_boundary_adjoint_list_matches_oracle(cuda_device):
    V, F = meshgen.jittered_torus(nu=40, nv=20, sigma=0.01, delete_frac=0.15, seed=4)
    rng = np.random.default_rng(41)
    Q = np.vstack([rng.uniform(-1, 1, size=(4001, 3)),
                   V[F[:5, 0]]]).astype(np.float32)  # odd count, and queries on vertices
    d = oracle.point_mesh_distance(V, F, Q)
    g = _masked(len(Q), d, seed=2)
    mesh = make_mesh(V, F, cuda_device)
    G = dv.dv_winding_backward_boundary(mesh, to_dev(g.astype(np.float32), cuda_device),
                                        queries=to_dev(Q, cuda_device)).cpu().numpy()
    assert np.all(np.isfinite(G))
    grad_close(G, oracle.winding_grad(V, F, Q, g), "boundary list", oracle.winding_grad_scale(V, F, Q, g))


def test_boundary_adjoint_closed_mesh_is_exactly_zero(cuda_device):
    V, F = meshgen.icosphere(3, 0.6)
    grid = dv.Grid.cube(20)
    mesh = make_mesh(V, F, cuda_device)
    assert dv.dv_mesh_num_boundary_edges(mesh) == 0
    g = to_dev(meshgen.upstream_gradient(grid.num_queries, seed=3), cuda_device)
    G = dv.dv_winding_backward_boundary(mesh, g, grid=grid)
    assert torch.count_nonzero(G).item() == 0


def test_boundary_adjoint_odd_topology(cuda_device):
    """A fin on a non-manifold edge, a duplicated face (multiplicity 2 edges), a degenerate face."""
    V, F = meshgen.icosphere(2, 0.6)
    a, b = F[0, 0], F[0, 1]
    V = np.vstack([V, [[0.9, 0.9, 0.9]]]).astype(np.float32)
    F = np.vstack([F, [[a, b, len(V) - 1]], F[5:6], [[F[7, 0], F[7, 0], F[7, 1]]]]).astype(np.int32)
    grid = dv.Grid.cube(22)
    Q, _, d = oracle_grid(V, F, grid)
    g = _masked(len(Q), d, seed=5)
    mesh = make_mesh(V, F, cuda_device)
    assert dv.dv_mesh_num_boundary_edges(mesh) == _net_boundary_count(F)
    G = dv.dv_winding_backward_boundary(mesh, to_dev(g.astype(np.float32), cuda_device), grid=grid).cpu().numpy()
    grad_close(G, oracle.winding_grad(V, F, Q, g), "boundary odd topology", oracle.winding_grad_scale(V, F, Q, g))


def test_boundary_adjoint_after_update_verts(cuda_device):
    """The boundary records follow dv_mesh_update_verts like the face records."""
    V, F = meshgen.jittered_torus(nu=30, nv=15, sigma=0.0, delete_frac=0.2, seed=7)
    V2 = (V * 1.1 + np.array([0.02, -0.03, 0.01], dtype=np.float32)).astype(np.float32)
    grid = dv.Grid.cube(16)
    Q, _, d = oracle_grid(V2, F, grid)
    g = _masked(len(Q), d, seed=6)
    mesh = make_mesh(V, F, cuda_device)
    dv.dv_mesh_update_verts(mesh, to_dev(V2, cuda_device))
    G = dv.dv_winding_backward_boundary(mesh, to_dev(g.astype(np.float32), cuda_device), grid=grid).cpu().numpy()
    grad_close(G, oracle.winding_grad(V2, F, Q, g), "boundary after update", oracle.winding_grad_scale(V2, F, Q, g))


def test_autograd_boundary_adjoint_matches_face_adjoint(cuda_device):
    from paper_2407_11272_b300.autograd import WindingNumber

    V, F = meshgen.jittered_torus(nu=40, nv=20, sigma=0.01, delete_frac=0.1, seed=8)
    grid = dv.Grid.cube(20)
    Q, _, d = oracle_grid(V, F, grid)
    g = to_dev(_masked(len(Q), d, seed=7).astype(np.float32), cuda_device)
    grads = {}
    for adj in ("faces", "boundary"):
        Vd = to_dev(V, cuda_device).requires_grad_(True)
        field = WindingNumber(Vd, to_dev(F, cuda_device), grid=grid, kind="exact", adjoint=adj)
        (field(Vd) * g).sum().backward()
        grads[adj] = Vd.grad.cpu().numpy().astype(np.float64)
    Q64, gq = Q, g.cpu().numpy().astype(np.float64)
    grad_close(grads["boundary"], grads["faces"], "autograd boundary vs faces",
               oracle.winding_grad_scale(V, F, Q64, gq))


def test_boundary_adjoint_repacked_after_first_use(cuda_device):
    """The boundary records are built on the first call; a later dv_mesh_update_verts repacks
    them, so a second call sees the new vertices."""
    V, F = meshgen.jittered_torus(nu=30, nv=15, sigma=0.0, delete_frac=0.2, seed=8)
    V2 = (V * 0.9 + np.array([-0.01, 0.02, 0.03], dtype=np.float32)).astype(np.float32)
    grid = dv.Grid.cube(16)
    mesh = make_mesh(V, F, cuda_device)
    Q, _, d1 = oracle_grid(V, F, grid)
    g1 = _masked(len(Q), d1, seed=9)
    G1 = dv.dv_winding_backward_boundary(mesh, to_dev(g1.astype(np.float32), cuda_device), grid=grid).cpu().numpy()
    grad_close(G1, oracle.winding_grad(V, F, Q, g1), "boundary first use", oracle.winding_grad_scale(V, F, Q, g1))
    dv.dv_mesh_update_verts(mesh, to_dev(V2, cuda_device))
    _, _, d2 = oracle_grid(V2, F, grid)
    g2 = _masked(len(Q), d2, seed=10)
    G2 = dv.dv_winding_backward_boundary(mesh, to_dev(g2.astype(np.float32), cuda_device), grid=grid).cpu().numpy()
    grad_close(G2, oracle.winding_grad(V2, F, Q, g2), "boundary after repack", oracle.winding_grad_scale(V2, F, Q, g2))
