"""Adjoint parity: dL/dV from the CUDA path against the FP64 oracle's analytic
gradient and against FP64 central finite differences.

Upstream values are masked to 0 for queries within 1e-3 of the surface in every
gradient comparison (there the terms grow like 1/d^2 and finite differences
lose meaning); closed meshes, whose exact gradient is 0, are compared in
absolute terms."""
import numpy as np
import pytest

import oracle
from _util import NEAR, grad_close, make_mesh, oracle_grid, to_dev
from paper_2407_11272_b300 import dv, meshgen

pytestmark = pytest.mark.gpu


def _masked_upstream(n, d, seed=1):
    g = meshgen.upstream_gradient(n, seed=seed).astype(np.float64)
    g[d <= NEAR] = 0.0
    return g


@pytest.mark.parametrize("n", [24, 33])
def test_small_torus_grid_gradient(cuda_device, n):
    V, F = meshgen.jittered_torus(nu=60, nv=30, sigma=0.01, delete_frac=0.1, seed=0)
    grid = dv.Grid.cube(n)
    Q, _, d = oracle_grid(V, F, grid)
    g = _masked_upstream(len(Q), d)
    G_ref = oracle.winding_grad(V, F, Q, g)
    mesh = make_mesh(V, F, cuda_device)
    G = dv.dv_winding_backward(mesh, to_dev(g.astype(np.float32), cuda_device), grid=grid).cpu().numpy()
    grad_close(G, G_ref, f"torus grid {n}", oracle.winding_grad_scale(V, F, Q, g))


def test_ragged_faces_odd_grid_gradient(cuda_device):
    V, F = meshgen.jittered_torus(nu=20, nv=10, sigma=0.01, delete_frac=0.0, seed=1)
    F = F[:129]
    grid = dv.Grid((37, 23, 11), (-0.9, -1.1, -0.7), (1.2, 0.8, 0.9))
    Q, _, d = oracle_grid(V, F, grid)
    g = _masked_upstream(len(Q), d, seed=7)
    G_ref = oracle.winding_grad(V, F, Q, g)
    mesh = make_mesh(V, F, cuda_device)
    G = dv.dv_winding_backward(mesh, to_dev(g.astype(np.float32), cuda_device), grid=grid).cpu().numpy()
    used = np.unique(F)
    grad_close(G[used], G_ref[used], "ragged", oracle.winding_grad_scale(V, F, Q, g)[used])
    unused = np.setdiff1d(np.arange(len(V)), used)
    assert np.all(G[unused] == 0.0)


@pytest.mark.parametrize("grid_n", [(24, 24, 24), (25, 19, 7)])
def test_grid_gradient_face_pairs_mixed_orientation(cuda_device, grid_n):
    """The grid adjoint walks edge-sharing face pairs (dv_build_face_pairs): with 30 % of the
    faces reversed, pairs whose second face runs against (p2, p1, p3) occur beside consistent
    ones, and on an even and an odd row length (packed and guarded paths) the gradient matches
    the oracle's for the mesh as given."""
    V, F = meshgen.jittered_torus(nu=40, nv=20, sigma=0.01, delete_frac=0.1, seed=2)
    flip = np.random.default_rng(5).random(len(F)) < 0.3
    F[flip] = F[flip][:, ::-1]
    pairs, singles = dv.dv_build_face_pairs(F, len(V))
    rev = (pairs[:, 6] >> 12) & 1
    assert 0 < rev.sum() < len(pairs) and len(singles) > 0
    grid = dv.Grid(grid_n, (-1.0, -0.9, -1.05), (1.0, 1.1, 0.95))
    Q, _, d = oracle_grid(V, F, grid)
    g = _masked_upstream(len(Q), d, seed=11)
    G_ref = oracle.winding_grad(V, F, Q, g)
    mesh = make_mesh(V, F, cuda_device)
    G = dv.dv_winding_backward(mesh, to_dev(g.astype(np.float32), cuda_device), grid=grid).cpu().numpy()
    grad_close(G, G_ref, f"pairs mixed orientation {grid_n}", oracle.winding_grad_scale(V, F, Q, g))


def test_grid_gradient_rows_longer_than_the_window(cuda_device):
    """Rows of 2101 and 4100 voxels (longer than the 2048-query staging window): they go through
    the kernel in pieces on the guarded path, for paired and single faces alike."""
    V, F = meshgen.jittered_torus(nu=24, nv=12, sigma=0.01, delete_frac=0.1, seed=3)
    for n in ((2101, 3, 2), (4100, 2, 1)):
        grid = dv.Grid(n, (-1.0, -0.3, -0.05), (1.0, 0.3, 0.05))
        Q, _, d = oracle_grid(V, F, grid)
        g = _masked_upstream(len(Q), d, seed=13)
        G_ref = oracle.winding_grad(V, F, Q, g)
        mesh = make_mesh(V, F, cuda_device)
        G = dv.dv_winding_backward(mesh, to_dev(g.astype(np.float32), cuda_device), grid=grid).cpu().numpy()
        grad_close(G, G_ref, f"long rows {n}", oracle.winding_grad_scale(V, F, Q, g))


def test_grid_gradient_vertices_on_cell_centres(cuda_device):
    """Mesh vertices placed exactly on voxel centres (as the kernels compute them in FP32): the
    packed sums of those rows are not finite, so paired and single faces alike take the guarded
    path for them; upstream is 0 within 1e-3 of the surface, so the oracle's gradient is the
    reference."""
    V, F = meshgen.jittered_torus(nu=30, nv=15, sigma=0.01, delete_frac=0.1, seed=9)
    n, lo, hi = 24, -1.0, 1.0
    h = np.float32((hi - lo) / n)
    idx = np.clip(np.floor((V.astype(np.float64) - lo) / h), 0, n - 1)
    centre = ((idx + 0.5) * np.float64(h) + lo).astype(np.float32)  # fmaf((float)i + 0.5f, h, lo)
    pick = np.random.default_rng(3).choice(len(V), size=40, replace=False)
    V = V.copy()
    V[pick] = centre[pick]
    pairs, singles = dv.dv_build_face_pairs(F, len(V))
    grid = dv.Grid.cube(n)
    Q, _, d = oracle_grid(V, F, grid)
    assert (d < 1e-6).sum() >= 40  # the oracle's FP64 centres sit within 1e-7 of the FP32 ones
    g = _masked_upstream(len(Q), d, seed=12)
    G_ref = oracle.winding_grad(V, F, Q, g)
    mesh = make_mesh(V, F, cuda_device)
    G = dv.dv_winding_backward(mesh, to_dev(g.astype(np.float32), cuda_device), grid=grid).cpu().numpy()
    assert np.all(np.isfinite(G))
    grad_close(G, G_ref, "vertices on cell centres", oracle.winding_grad_scale(V, F, Q, g))


def test_list_gradient(cuda_device):
    V, F = meshgen.jittered_torus(nu=40, nv=20, sigma=0.01, delete_frac=0.1, seed=2)
    rng = np.random.default_rng(31)
    Q = rng.uniform(-1, 1, size=(5000, 3)).astype(np.float32)
    d = oracle.point_mesh_distance(V, F, Q)
    g = _masked_upstream(len(Q), d, seed=8)
    G_ref = oracle.winding_grad(V, F, Q, g)
    mesh = make_mesh(V, F, cuda_device)
    G = dv.dv_winding_backward(mesh, to_dev(g.astype(np.float32), cuda_device),
                               queries=to_dev(Q, cuda_device)).cpu().numpy()
    grad_close(G, G_ref, "list", oracle.winding_grad_scale(V, F, Q, g))


def test_list_gradient_odd_count_and_queries_on_the_mesh(cuda_device):
    """Odd query count (the packed pairs are padded), and queries exactly on vertices and on an
    edge's midpoint: their packed sums are not finite, so their chunks take the guarded path."""
    V, F = meshgen.jittered_torus(nu=30, nv=15, sigma=0.01, delete_frac=0.1, seed=6)
    rng = np.random.default_rng(37)
    on = np.vstack([V[F[3]], V[F[40, :1]], 0.5 * (V[F[7, 0]] + V[F[7, 1]])]).astype(np.float32)
    Q = np.vstack([rng.uniform(-1, 1, size=(1000, 3)).astype(np.float32), on])
    Q = Q[rng.permutation(len(Q))]
    assert len(Q) % 2 == 1
    d = oracle.point_mesh_distance(V, F, Q)
    g = _masked_upstream(len(Q), d, seed=9)
    G_ref = oracle.winding_grad(V, F, Q, g)
    mesh = make_mesh(V, F, cuda_device)
    G = dv.dv_winding_backward(mesh, to_dev(g.astype(np.float32), cuda_device),
                               queries=to_dev(Q, cuda_device)).cpu().numpy()
    assert np.all(np.isfinite(G))
    grad_close(G, G_ref, "list odd/on-mesh", oracle.winding_grad_scale(V, F, Q, g))


def _long_edge_mesh(y0, z0):
    """Two faces sharing the edge A-C, with the long boundary edge A-B along x at height (y0, z0)."""
    A, B = (-0.8, y0, z0), (0.8, y0, z0)
    C, D = (0.1, y0 + 0.5, z0 - 0.4), (-0.5, y0 - 0.3, z0 + 0.6)
    return np.array([A, B, C, D], dtype=np.float32), np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)


_H64 = 2.0 / 64
_Y0, _Z0 = -1 + 40.5 * _H64 + 0.002, -1 + 20.5 * _H64 + 0.001  # 2.2e-3 from a row of the 64^2 (y, z) grid


def _backward_form(form):
    return dv.dv_winding_backward if form == "faces" else dv.dv_winding_backward_boundary


@pytest.mark.parametrize("form", ["faces", "boundary"])
def test_gradient_queries_near_long_edges(cuda_device, form):
    """List queries 1.5e-3 to 3e-2 from the interior of edges 1.2 to 1.6 long: there |a||b| + a.b
    cancels in FP32 (relative error ~ eps (L / dist)^2), so the kernels take the guarded path with
    t = |a x b|^2 / (|a||b| - a.b). Both adjoint forms: face pairs and the boundary curve."""
    V, F = _long_edge_mesh(_Y0, _Z0)
    mesh = make_mesh(V, F, cuda_device)
    rng = np.random.default_rng(41)
    Vd = V.astype(np.float64)
    pts = []
    for i, j in ((0, 1), (1, 2), (2, 0), (2, 3), (3, 0)):
        e = Vd[j] - Vd[i]
        s = rng.uniform(0.1, 0.9, size=300)
        u = rng.normal(size=(300, 3))
        u -= np.outer(u @ e, e) / (e @ e)
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        dist = np.exp(rng.uniform(np.log(1.5e-3), np.log(3e-2), size=300))
        pts.append(Vd[i] + s[:, None] * e + dist[:, None] * u)
    Q = np.vstack(pts + [rng.uniform(-1, 1, size=(500, 3))]).astype(np.float32)
    d = oracle.point_mesh_distance(V, F, Q)
    g = _masked_upstream(len(Q), d, seed=14)
    assert (g[:1500] != 0).sum() > 1000
    G_ref = oracle.winding_grad(V, F, Q, g)
    G = _backward_form(form)(mesh, to_dev(g.astype(np.float32), cuda_device),
                             queries=to_dev(Q, cuda_device)).cpu().numpy()
    grad_close(G, G_ref, f"{form} list near long edges", oracle.winding_grad_scale(V, F, Q, g))


@pytest.mark.parametrize("form", ["faces", "boundary"])
@pytest.mark.parametrize("nx", [64, 65])
def test_gradient_grid_row_near_a_long_edge(cuda_device, form, nx):
    """A grid row parallel to the edge A-B (length 1.6) at 2.2e-3 from it, even and odd row
    lengths (an odd row is padded in the adjoint's window). Upstream on the 3 x 3 rows around it
    only: random upstream over the whole grid would let the far rows' terms, which cancel among
    themselves, set the error instead."""
    V, F = _long_edge_mesh(_Y0, _Z0)
    mesh = make_mesh(V, F, cuda_device)
    grid = dv.Grid(n=(nx, 64, 64), lo=(-1.0,) * 3, hi=(1.0,) * 3)
    Qg, _, dg = oracle_grid(V, F, grid)
    g = _masked_upstream(len(Qg), dg, seed=15)
    row = (np.abs(Qg[:, 1] - (_Y0 - 0.002)) < 1e-6) & (np.abs(Qg[:, 2] - (_Z0 - 0.001)) < 1e-6)
    block = (np.abs(Qg[:, 1] - (_Y0 - 0.002)) < 1.5 * _H64) & (np.abs(Qg[:, 2] - (_Z0 - 0.001)) < 1.5 * _H64)
    g[~block] = 0.0
    assert row.sum() == nx and block.sum() == 9 * nx and (g[row] != 0).sum() >= 40
    G_ref = oracle.winding_grad(V, F, Qg, g)
    G = _backward_form(form)(mesh, to_dev(g.astype(np.float32), cuda_device), grid=grid).cpu().numpy()
    grad_close(G, G_ref, f"{form} grid row near a long edge (nx={nx})", oracle.winding_grad_scale(V, F, Qg, g))


@pytest.mark.parametrize("form", ["faces", "boundary"])
@pytest.mark.parametrize("n", [(1, 1, 1), (1, 7, 9), (3, 5, 2), (2049, 2, 2)])
def test_grid_gradient_degenerate_shapes(cuda_device, n, form):
    """Grids one cell wide (every row is one query and one g = 0 padding entry), tiny grids, and
    rows of 2049 queries (a full window piece and an odd piece of one), on an open mesh."""
    V, F = meshgen.icosphere(2, 0.6)
    F = F[7:]
    grid = dv.Grid(n, (-0.9, -0.8, -0.7), (0.8, 0.9, 0.6))
    Q, _, d = oracle_grid(V, F, grid)
    g = _masked_upstream(len(Q), d, seed=16)
    assert (g != 0).any()
    G_ref = oracle.winding_grad(V, F, Q, g)
    mesh = make_mesh(V, F, cuda_device)
    G = _backward_form(form)(mesh, to_dev(g.astype(np.float32), cuda_device), grid=grid).cpu().numpy()
    assert np.all(np.isfinite(G))
    grad_close(G, G_ref, f"{form} grid {n}", oracle.winding_grad_scale(V, F, Q, g))


def test_closed_mesh_gradient_is_cancellation_noise(cuda_device):
    """Closed icosphere: exact dL/dV = 0. Remove one face and the same vertices get O(1) gradients;
    the closed-mesh values must be orders of magnitude below those."""
    V, F = meshgen.icosphere(3, 0.6)
    grid = dv.Grid.cube(32)
    Q, _, d = oracle_grid(V, F, grid, with_distance=True)
    g = to_dev(_masked_upstream(len(Q), d).astype(np.float32), cuda_device)
    Gc = dv.dv_winding_backward(make_mesh(V, F, cuda_device), g, grid=grid).cpu().numpy()
    Go = dv.dv_winding_backward(make_mesh(V, F[1:], cuda_device), g, grid=grid).cpu().numpy()
    hole = F[0]
    assert np.abs(Gc).max() < 1e-4 * np.abs(Go[hole]).max()


def test_deterministic_gradient(cuda_device):
    V, F = meshgen.jittered_torus(nu=50, nv=25, sigma=0.01, delete_frac=0.1, seed=3)
    grid = dv.Grid.cube(32)
    mesh = make_mesh(V, F, cuda_device)
    g = to_dev(meshgen.upstream_gradient(grid.num_queries), cuda_device)
    a = dv.dv_winding_backward(mesh, g, grid=grid).cpu().numpy()
    b = dv.dv_winding_backward(mesh, g, grid=grid).cpu().numpy()
    assert np.array_equal(a, b)


def test_torus128_full_size_64_vertices(cuda_device):
    """Open irregular torus, 128^3 grid, N(0,1) upstream: dL/dV on 64 seeded vertices against the
    oracle's analytic gradient (all 2.1M queries), and against FP64 central differences (h = 1e-4)
    on a seeded 20 000-query subsample through the list path."""
    V, F = meshgen.jittered_torus()
    grid = dv.Grid.cube(128)
    mesh = make_mesh(V, F, cuda_device)
    Q = oracle.grid_queries(grid.lo, grid.hi, grid.n)
    g32 = meshgen.upstream_gradient(len(Q), seed=1)
    # Only the faces incident to the 64 vertices enter their gradient, so the upstream is masked to
    # 0 within 1e-3 of those faces (the near-surface radius of the gradient bar), by the oracle's
    # exact distance to them.
    ids = meshgen.random_vertex_ids(len(V), 64, seed=2)
    used = np.isin(ids, np.unique(F))
    ids = ids[used]
    inc = np.isin(F, ids).any(axis=1)
    sub_d = oracle.point_mesh_distance(V, F[inc], Q)
    g = g32.astype(np.float64)
    g[sub_d <= 1e-3] = 0.0
    G = dv.dv_winding_backward(mesh, to_dev(g.astype(np.float32), cuda_device), grid=grid).cpu().numpy()[ids]
    G_ref = oracle.vertex_grad_subset(V, F, Q, g, ids)
    # per-vertex cancellation scale (sum of |face contributions|) from the incident faces, which are
    # all the faces the 64 vertices have: vertices away from the holes have an exact gradient of 0
    # that FP32 reaches only up to a fraction of the terms that cancel
    scale = oracle.winding_grad_scale(V, F[inc], Q, g)[ids]
    grad_close(G, G_ref, "torus128 analytic", scale)
    # finite differences on a query subsample (list path); central differences with h = 1e-4 have a
    # truncation error ~ (h/d)^2, so here the upstream is masked within 1e-2 of the incident faces
    sub = meshgen.query_subsample(len(Q), 20000, seed=5)
    Qs = Q[sub].astype(np.float32)
    gs = g[sub].copy()
    gs[sub_d[sub] <= 1e-2] = 0.0
    Gs = dv.dv_winding_backward(mesh, to_dev(gs.astype(np.float32), cuda_device),
                                queries=to_dev(Qs, cuda_device)).cpu().numpy()[ids]
    fd = oracle.fd_vertex_grad(V, F, Qs, gs, ids, h=1e-4)
    grad_close(Gs, fd, "torus128 finite differences")


def test_shsphere256_full_size_open_adjoint_sampled(cuda_device):
    """The 204 020-face sphere with a cap cut away (an open mesh, so dL/dV is not identically 0)
    on the full 256^3 grid, in the launch configuration of the bench's adjoint (face pairs on
    nearly every face): dL/dV on 6 vertices of the cut's rim and 2 away from it against the
    oracle's analytic gradient over all 16.8M queries."""
    V, F = meshgen.sh_sphere()
    cz = V[F].mean(axis=1)[:, 2]
    F = F[cz < 0.55].copy()
    pairs, singles = dv.dv_build_face_pairs(F, len(V))
    assert 2 * len(pairs) > 0.99 * len(F)
    grid = dv.Grid.cube(256)
    mesh = make_mesh(V, F, cuda_device)
    # rim vertices: endpoints of edges used by one face only
    und = np.sort(np.stack([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]], axis=1).reshape(-1, 2), axis=1)
    key, cnt = np.unique(und[:, 0].astype(np.int64) * len(V) + und[:, 1], return_counts=True)
    rim = np.unique(np.concatenate([key[cnt == 1] // len(V), key[cnt == 1] % len(V)]))
    rng = np.random.default_rng(8)
    inner = np.setdiff1d(np.unique(F), rim)
    ids = np.concatenate([rng.choice(rim, 6, replace=False), rng.choice(inner, 2, replace=False)])
    Q = oracle.grid_queries(grid.lo, grid.hi, grid.n)
    g = meshgen.upstream_gradient(len(Q), seed=1).astype(np.float64)
    inc = np.isin(F, ids).any(axis=1)
    g[oracle.point_mesh_distance(V, F[inc], Q) <= 1e-3] = 0.0  # the gradient bar's near-surface radius
    G = dv.dv_winding_backward(mesh, to_dev(g.astype(np.float32), cuda_device), grid=grid).cpu().numpy()[ids]
    G_ref = oracle.vertex_grad_subset(V, F, Q, g, ids)
    assert np.linalg.norm(G_ref[:6], axis=1).min() > 0.0
    scale = oracle.winding_grad_scale(V, F[inc], Q, g)[ids]  # exact for these vertices (all their faces)
    grad_close(G, G_ref, "shsphere256 open, analytic", scale)


def test_forward_and_adjoint_concurrently_on_two_streams(cuda_device):
    """A forward (mixed precision) and an adjoint of the same mesh, reserved, launched on two
    streams at once (the header allows it): both equal the same calls made one after the other,
    bit for bit."""
    import torch

    V, F = meshgen.jittered_torus(nu=60, nv=30, sigma=0.01, delete_frac=0.1, seed=0)
    grid = dv.Grid.cube(40)
    mesh = make_mesh(V, F, cuda_device)
    dv.dv_mesh_reserve(mesh, grid)
    g = to_dev(meshgen.upstream_gradient(grid.num_queries, seed=4), cuda_device)
    w0, occ0, _ = dv.dv_voxelize_grid(mesh, grid, precision="mixed")
    G0 = dv.dv_winding_backward(mesh, g, grid=grid)
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    ev = torch.cuda.Event()
    ev.record()
    s1.wait_event(ev)
    s2.wait_event(ev)
    with torch.cuda.stream(s1):
        w1, occ1, _ = dv.dv_voxelize_grid(mesh, grid, precision="mixed", stream=s1)
    with torch.cuda.stream(s2):
        G1 = dv.dv_winding_backward(mesh, g, grid=grid, stream=s2)
    torch.cuda.synchronize()
    assert torch.equal(w0, w1) and torch.equal(occ0, occ1)
    assert torch.equal(G0, G1)
