"""Forward parity: CUDA path (through the C ABI) against the FP64 oracle.

Sizes where the oracle evaluates every query in seconds span several face
tiles (64 faces), ragged tails, split and unsplit face loops; the full-size
workloads are checked on seeded query samples the oracle computes one by one.
"""
import numpy as np
import pytest

import oracle
from _util import NEAR, check_forward, grad_close, make_mesh, oracle_grid, to_dev
from paper_2407_11272_b300 import dv, meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def icosphere32():
    V, F = meshgen.icosphere(3, 0.8)
    grid = dv.Grid.cube(32)
    Q, w64, d = oracle_grid(V, F, grid)
    return V, F, grid, w64, d


@pytest.mark.parametrize("prec", ["fp32", "kahan", "mixed"])
def test_icosphere32_full_grid(cuda_device, icosphere32, prec):
    V, F, grid, w64, d = icosphere32
    mesh = make_mesh(V, F, cuda_device)
    w, occ, rep = dv.dv_voxelize_grid(mesh, grid, precision=prec, report=True)
    check_forward(w.cpu().numpy(), w64, d, prec, occ.cpu().numpy(), "icosphere32")
    # closed mesh: w is 0 or 1 away from the surface
    far = d > NEAR
    assert np.abs(w.cpu().numpy()[far] - np.round(w64[far])).max() < 1e-4
    if prec == "mixed":
        assert rep["n_flagged"] >= int(np.sum(d < NEAR))


def test_small_torus_all_precisions(cuda_device):
    V, F = meshgen.jittered_torus(nu=60, nv=30, sigma=0.01, delete_frac=0.1, seed=0)
    grid = dv.Grid.cube(40)
    Q, w64, d = oracle_grid(V, F, grid)
    mesh = make_mesh(V, F, cuda_device)
    for prec in ("fp32", "kahan", "mixed"):
        w, occ, _ = dv.dv_voxelize_grid(mesh, grid, precision=prec, report=True)
        check_forward(w.cpu().numpy(), w64, d, prec, occ.cpu().numpy(), "torus40")
    # dv_winding on the same grid gives the same w as dv_voxelize_grid
    w2 = dv.dv_winding(mesh, grid=grid, precision="mixed")
    assert np.array_equal(w2.cpu().numpy(), w.cpu().numpy())


@pytest.mark.parametrize("nfaces", [1, 63, 64, 65, 129])
def test_ragged_face_counts_and_odd_grid(cuda_device, nfaces):
    V, F = meshgen.jittered_torus(nu=20, nv=10, sigma=0.01, delete_frac=0.0, seed=1)
    F = F[:nfaces]
    grid = dv.Grid((37, 23, 11), (-0.9, -1.1, -0.7), (1.2, 0.8, 0.9))
    Q, w64, d = oracle_grid(V, F, grid)
    mesh = make_mesh(V, F, cuda_device)
    for prec in ("fp32", "mixed"):
        w, occ, _ = dv.dv_voxelize_grid(mesh, grid, precision=prec)
        check_forward(w.cpu().numpy(), w64, d, prec, occ.cpu().numpy(), f"ragged{nfaces}")


@pytest.mark.parametrize("nfaces", [1, 2, 63, 65, 129])
def test_ragged_face_counts_list_path(cuda_device, nfaces):
    """Query lists (odd count) against meshes whose strip events end mid-tile and mid-step of the
    software-pipelined event loop, and the list adjoint on the same inputs."""
    V, F = meshgen.jittered_torus(nu=20, nv=10, sigma=0.01, delete_frac=0.0, seed=1)
    F = F[:nfaces]
    rng = np.random.default_rng(nfaces)
    Q = rng.uniform(-1, 1, size=(1001, 3)).astype(np.float32)
    w64 = oracle.winding(V, F, Q)
    d = oracle.point_mesh_distance(V, F, Q)
    mesh = make_mesh(V, F, cuda_device)
    for prec in ("fp32", "kahan", "mixed"):
        w = dv.dv_winding(mesh, queries=to_dev(Q, cuda_device), precision=prec)
        check_forward(w.cpu().numpy(), w64, d, prec, None, f"list ragged{nfaces}")
    g = meshgen.upstream_gradient(len(Q), seed=3).astype(np.float64)
    g[d <= NEAR] = 0.0
    G = dv.dv_winding_backward(mesh, to_dev(g.astype(np.float32), cuda_device), queries=to_dev(Q, cuda_device))
    grad_close(G.cpu().numpy(), oracle.winding_grad(V, F, Q, g), f"list ragged{nfaces} adjoint",
               oracle.winding_grad_scale(V, F, Q, g))


@pytest.mark.parametrize("n", [(1, 1, 1), (2, 3, 5), (9, 1, 7), (130, 3, 2)])
def test_degenerate_grid_shapes(cuda_device, n):
    V, F = meshgen.icosphere(2, 0.6)
    grid = dv.Grid(n, (-1, -1, -1), (1, 1, 1))
    Q, w64, d = oracle_grid(V, F, grid)
    mesh = make_mesh(V, F, cuda_device)
    w, occ, _ = dv.dv_voxelize_grid(mesh, grid, precision="mixed")
    check_forward(w.cpu().numpy(), w64, d, "mixed", occ.cpu().numpy(), f"grid{n}")


@pytest.mark.parametrize("prec", ["fp32", "kahan", "mixed"])
def test_query_list_path(cuda_device, prec):
    V, F = meshgen.jittered_torus(nu=40, nv=20, sigma=0.01, delete_frac=0.1, seed=2)
    rng = np.random.default_rng(21)
    Q = np.concatenate([rng.uniform(-1, 1, size=(3000, 3)),
                        V[rng.choice(len(V), 300)] + rng.normal(0, 2e-3, size=(300, 3))]).astype(np.float32)
    w64 = oracle.winding(V, F, Q)
    d = oracle.point_mesh_distance(V, F, Q)
    mesh = make_mesh(V, F, cuda_device)
    w = dv.dv_winding(mesh, queries=to_dev(Q, cuda_device), precision=prec)
    check_forward(w.cpu().numpy(), w64, d, prec, None, "list")


def test_exact_conventions_vertex_edge_face(cuda_device):
    """Queries exactly on a vertex, on an edge and inside a face (Eq. (8) zero cases)."""
    r2 = np.sqrt(2.0)
    V = np.array([[-1, 0, 0], [1, 0, 0], [0, -1, r2], [0, 1, r2]], dtype=np.float32) * 0.5
    F = meshgen._orient_outward(V.astype(np.float64), np.array([[0, 1, 2], [0, 1, 3], [0, 2, 3], [1, 2, 3]]),
                                V.astype(np.float64).mean(axis=0)).astype(np.int32)
    Vc = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float32) * 0.5
    Fc = meshgen._orient_outward(Vc.astype(np.float64), np.array([[0, 1, 2], [0, 1, 3], [0, 2, 3], [1, 2, 3]]),
                                 Vc.astype(np.float64).mean(axis=0)).astype(np.int32)
    for VV, FF, Q in ((V, F, np.array([V[2], [0, 0, 0], V[0]], dtype=np.float32)),
                      (Vc, Fc, np.array([[0.125, 0.125, 0.0], Vc[3], [0.25, 0.0, 0.0]], dtype=np.float32))):
        w64 = oracle.winding(VV, FF, Q)
        mesh = make_mesh(VV, FF, cuda_device)
        w = dv.dv_winding(mesh, queries=to_dev(Q, cuda_device), precision="mixed").cpu().numpy()
        np.testing.assert_allclose(w, w64, atol=1e-7)
        wf = dv.dv_winding(mesh, queries=to_dev(Q, cuda_device), precision="fp32").cpu().numpy()
        assert np.all(np.isfinite(wf))


def test_split_and_unsplit_agree(cuda_device):
    """Small grids split the face loop across CTAs; a list of the same points does not."""
    V, F = meshgen.jittered_torus(nu=50, nv=25, sigma=0.01, delete_frac=0.1, seed=3)
    grid = dv.Grid.cube(16)
    mesh = make_mesh(V, F, cuda_device)
    wg = dv.dv_winding(mesh, grid=grid, precision="kahan").cpu().numpy()
    Q = oracle.grid_queries(grid.lo, grid.hi, grid.n).astype(np.float32)
    wl = dv.dv_winding(mesh, queries=to_dev(Q, cuda_device), precision="kahan").cpu().numpy()
    assert np.abs(wg - wl).max() < 2e-6


def test_deterministic(cuda_device):
    V, F = meshgen.jittered_torus(nu=50, nv=25, sigma=0.01, delete_frac=0.1, seed=3)
    grid = dv.Grid.cube(24)
    mesh = make_mesh(V, F, cuda_device)
    a = dv.dv_voxelize_grid(mesh, grid, precision="mixed")
    b = dv.dv_voxelize_grid(mesh, grid, precision="mixed")
    assert np.array_equal(a[0].cpu().numpy(), b[0].cpu().numpy())
    assert np.array_equal(a[1].cpu().numpy(), b[1].cpu().numpy())


def test_invalid_mesh_is_rejected(cuda_device):
    V, F = meshgen.icosphere(1, 0.5)
    F = F.copy()
    F[3, 1] = len(V)
    with pytest.raises(dv.DvError) as e:
        make_mesh(V, F, cuda_device)
    assert e.value.status == 2
    V2 = V.copy()
    V2[0, 0] = np.nan
    with pytest.raises(dv.DvError):
        make_mesh(V2, meshgen.icosphere(1, 0.5)[1], cuda_device)


def _sample_with_near(V, F, Q, n_rand, n_near, n_cand, seed):
    """Seeded sample: n_rand uniform grid queries plus n_near queries within 2*NEAR of the
    surface, chosen from n_cand seeded candidates by the oracle's exact distance."""
    rand = meshgen.query_subsample(len(Q), n_rand, seed=seed)
    cand = meshgen.query_subsample(len(Q), n_cand, seed=seed + 1)
    dc = oracle.point_mesh_distance(V, F, Q[cand])
    near = cand[np.argsort(dc)[:n_near]]
    return np.unique(np.concatenate([rand, near]))


def test_torus128_full_size_sampled(cuda_device):
    """Open irregular torus (36 000 faces) on the 128^3 grid, mixed precision, sampled check."""
    V, F = meshgen.jittered_torus()
    grid = dv.Grid.cube(128)
    mesh = make_mesh(V, F, cuda_device)
    w, occ, rep = dv.dv_voxelize_grid(mesh, grid, precision="mixed", report=True)
    w, occ = w.cpu().numpy(), occ.cpu().numpy()
    Q = oracle.grid_queries(grid.lo, grid.hi, grid.n)
    idx = _sample_with_near(V, F, Q, 1500, 400, 30000, seed=4)
    w64 = oracle.winding(V, F, Q[idx])
    d = oracle.point_mesh_distance(V, F, Q[idx])
    check_forward(w[idx], w64, d, "mixed", occ[idx], "torus128")
    assert rep["n_flagged"] > 0


def test_shsphere256_full_size_sampled(cuda_device):
    """Large closed mesh (204 020 faces) on the 256^3 grid: FP32 bulk + FP64 re-evaluation."""
    V, F = meshgen.sh_sphere()
    grid = dv.Grid.cube(256)
    mesh = make_mesh(V, F, cuda_device)
    w, occ, rep = dv.dv_voxelize_grid(mesh, grid, precision="mixed", report=True)
    w, occ = w.cpu().numpy(), occ.cpu().numpy()
    Q = oracle.grid_queries(grid.lo, grid.hi, grid.n)
    idx = _sample_with_near(V, F, Q, 3000, 1000, 20000, seed=4)
    w64 = oracle.winding(V, F, Q[idx])
    d = oracle.point_mesh_distance(V, F, Q[idx])
    stats = check_forward(w[idx], w64, d, "mixed", occ[idx], "shsphere256")
    assert rep["n_flagged"] > 10000
    print(stats, rep)


@pytest.mark.parametrize("scale", [1e-3, 1e3])
def test_scaled_meshes_mixed_precision(cuda_device, scale):
    """The winding number is scale invariant; meshes and grids scaled by 1e-3 and 1e3 exercise the
    FP32 fast path and the FP64 pass (whose running product of small-angle factors is rescaled by
    exact powers of two) far from unit size. At 1e-3 every voxel centre lies within the absolute
    1e-3 band and goes through FP64."""
    V, F = meshgen.jittered_torus(nu=30, nv=15, sigma=0.01, delete_frac=0.1, seed=5)
    V = (V.astype(np.float64) * scale).astype(np.float32)
    grid = dv.Grid((20, 17, 9), tuple(-scale * x for x in (1.0, 0.9, 0.4)), tuple(scale * x for x in (1.0, 0.9, 0.4)))
    Q, w64, d = oracle_grid(V, F, grid)
    mesh = make_mesh(V, F, cuda_device)
    w, occ, rep = dv.dv_voxelize_grid(mesh, grid, precision="mixed", report=True)
    check_forward(w.cpu().numpy(), w64, d, "mixed", occ.cpu().numpy(), f"scale {scale}")
    if scale < 1:
        assert rep["n_flagged"] == grid.num_queries


@pytest.mark.parametrize("case", ["shsphere_256", "closed_torus_128"])
def test_whole_grid_occupancy_matches_ray_crossings(cuda_device, case):
    """Every voxel of the grid (16.8M on the 204 020-face sphere at 256^3; the 40 000-face torus
    with no face deleted at 128^3): mixed-precision occupancy equals the occupancy from signed ray
    crossings of the closed mesh (the oracle's check that evaluates no solid angle), wherever that
    count is decided. A slip in any tile, split or row of the grid would show here."""
    if case == "shsphere_256":
        V, F = meshgen.sh_sphere()
        grid = dv.Grid.cube(256)
    else:
        V, F = meshgen.jittered_torus(delete_frac=0.0, seed=0)
        grid = dv.Grid.cube(128)
    mesh = make_mesh(V, F, cuda_device)
    w, occ, rep = dv.dv_voxelize_grid(mesh, grid, precision="mixed", report=True)
    w_ray, und = oracle.ray_winding_grid(V, F, grid.lo, grid.hi, grid.n)
    if case == "shsphere_256":
        assert set(np.unique(w_ray[~und]).tolist()) == {0, 1}
    # (the jittered torus folds over itself in places: integer winding numbers -1 and 2 occur)
    assert und.sum() < 1e-5 * grid.num_queries
    # off the surface w is an integer: every decided voxel within the forward bar of it, and its
    # occupancy (w > 0.5) that of the integer (w >= 1)
    err = np.abs(w.cpu().numpy().astype(np.float64) - w_ray)[~und]
    assert err.max() <= 1e-4, f"max |w - ray count| over the whole grid {err.max():.3e}"
    bad = (occ.cpu().numpy().astype(bool) != (w_ray >= 1)) & ~und
    assert not bad.any(), f"{bad.sum()} occupancy mismatches over the whole grid"
    assert (w_ray >= 1).sum() > 0.05 * grid.num_queries and rep["n_flagged"] > 0
