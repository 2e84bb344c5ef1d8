"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

Each test checks the oracle against a closed form, an independent
formulation (Girard's spherical excess, plane-side tests for convex
polyhedra, brute-force finite differences, dense sampling), or an
invariant of the mathematics. A plausible slip in the oracle (a dropped
term of beta in Eq. (7), a wrong sign of the determinant, a wrong ATAN2
quadrant, a transposed index, a wrong chain-rule factor) fails at least one.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2407_11272_b300 import meshgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            rows[parts[0]] = float(parts[1])
    return rows


def _tri(V, F, f):
    return V[F[f, 0]], V[F[f, 1]], V[F[f, 2]]


# ---------------------------------------------------------------- Eq. (8)

def test_atan2_table_cases():
    with open(os.path.join(GOLDEN, "atan2_table.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            y, x, want = (float(t) for t in line.split()[:3])
            assert oracle.atan2_table(y, x) == pytest.approx(want, abs=1e-15), (y, x)


def test_atan2_table_matches_quadrant_geometry():
    # Away from the table's boundaries ATAN2 is the polar angle of (x, y):
    # check that (cos, sin) of the result points along (x, y).
    rng = np.random.default_rng(11)
    for y, x in rng.normal(size=(200, 2)):
        t = oracle.atan2_table(y, x)
        r = math.hypot(x, y)
        assert math.cos(t) * r == pytest.approx(x, abs=1e-12)
        assert math.sin(t) * r == pytest.approx(y, abs=1e-12)
        assert -math.pi < t <= math.pi


# ---------------------------------------------------------------- Eq. (7)

def test_octant_triangle_is_one_eighth_of_sphere():
    g = _golden("closed_forms.txt")
    om = oracle.solid_angle([1, 0, 0], [0, 1, 0], [0, 0, 1], [0, 0, 0])
    assert om == pytest.approx(g["octant_triangle_from_origin"], abs=1e-14)
    # reversed orientation flips the sign
    om2 = oracle.solid_angle([1, 0, 0], [0, 0, 1], [0, 1, 0], [0, 0, 0])
    assert om2 == pytest.approx(-g["octant_triangle_from_origin"], abs=1e-14)


def test_regular_tetrahedron_faces_from_centre():
    g = _golden("closed_forms.txt")
    V, F = meshgen.regular_tetrahedron(0.5)
    V = V.astype(np.float64)
    for f in range(4):
        assert oracle.solid_angle(*_tri(V, F, f), [0, 0, 0]) == pytest.approx(g["tetra_face_from_centre"], abs=1e-13)


def test_cube_triangles_from_centre():
    g = _golden("closed_forms.txt")
    V, F = meshgen.cube(0.5)
    V = V.astype(np.float64)
    for f in range(12):
        assert oracle.solid_angle(*_tri(V, F, f), [0, 0, 0]) == pytest.approx(g["cube_triangle_from_centre"],
                                                                           abs=1e-13)


def _girard(v0, v1, v2, q):
    """Spherical excess A + B + C - pi of the triangle's central projection (Girard)."""
    p = [np.asarray(v, float) - np.asarray(q, float) for v in (v0, v1, v2)]
    p = [x / np.linalg.norm(x) for x in p]
    ang = 0.0
    for i in range(3):
        a, b, c = p[i], p[(i + 1) % 3], p[(i + 2) % 3]
        tb = b - np.dot(a, b) * a
        tc = c - np.dot(a, c) * a
        ang += math.acos(np.clip(np.dot(tb, tc) / (np.linalg.norm(tb) * np.linalg.norm(tc)), -1, 1))
    sign = np.sign(np.dot(p[0], np.cross(p[1], p[2])))
    return sign * (ang - math.pi)


def test_solid_angle_equals_spherical_excess():
    rng = np.random.default_rng(5)
    n = 0
    while n < 300:
        q = rng.normal(size=3)
        v = q + rng.normal(size=(3, 3)) * rng.uniform(0.1, 3.0, size=(3, 1))
        ex = _girard(v[0], v[1], v[2], q)
        if abs(abs(ex) - 2 * math.pi) < 1e-3:
            continue
        assert oracle.solid_angle(v[0], v[1], v[2], q) == pytest.approx(ex, abs=1e-9)
        n += 1


def test_solid_angle_invariant_along_rays():
    # Moving each vertex along its ray from q does not change the central projection.
    rng = np.random.default_rng(6)
    for _ in range(100):
        q = rng.normal(size=3)
        v = q + rng.normal(size=(3, 3))
        lam = rng.uniform(0.05, 20.0, size=(3, 1))
        w = q + lam * (v - q)
        assert oracle.solid_angle(*w, q) == pytest.approx(oracle.solid_angle(*v, q), abs=1e-11)


# ---------------------------------------------------------------- Eq. (5) / Algorithm 1

def _inside_convex(V, F, Q):
    """q inside a convex outward mesh iff it is on the inner side of every face plane."""
    V = V.astype(np.float64)
    p0, p1, p2 = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    n = np.cross(p1 - p0, p2 - p0)
    s = np.einsum("fk,qfk->qf", n, Q[:, None, :] - p0[None])
    return np.all(s < 0, axis=1), np.min(np.abs(s) / np.linalg.norm(n, axis=1), axis=1)


@pytest.mark.parametrize("mesh", ["tetra", "cube", "ico2"])
def test_closed_convex_mesh_winding_is_indicator(mesh):
    V, F = {"tetra": lambda: meshgen.regular_tetrahedron(0.5),
            "cube": lambda: meshgen.cube(0.5),
            "ico2": lambda: meshgen.icosphere(2, 0.8)}[mesh]()
    Q = np.random.default_rng(7).uniform(-1.0, 1.0, size=(3000, 3))
    inside, dplane = _inside_convex(V, F, Q)
    keep = dplane > 1e-6
    w = oracle.winding(V, F, Q[keep])
    np.testing.assert_allclose(w, inside[keep].astype(float), atol=1e-11)
    assert inside[keep].any() and (~inside[keep]).any()


def test_winding_rigid_motion_and_scale_invariant():
    V, F = meshgen.icosphere(2, 0.6)
    rng = np.random.default_rng(8)
    Q = rng.uniform(-1, 1, size=(500, 3))
    torus_v, torus_f = meshgen.jittered_torus(nu=24, nv=12, sigma=0.01, delete_frac=0.1, seed=3)
    for VV, FF in ((V, F), (torus_v, torus_f)):
        w0 = oracle.winding(VV, FF, Q)
        Rm = np.linalg.qr(rng.normal(size=(3, 3)))[0]
        if np.linalg.det(Rm) < 0:
            Rm[:, 0] *= -1
        t = rng.normal(size=3)
        s = 1.7
        V2 = s * (VV.astype(np.float64) @ Rm.T) + t
        Q2 = s * (Q @ Rm.T) + t
        np.testing.assert_allclose(oracle.winding(V2, FF, Q2), w0, atol=1e-10)


def test_reflection_flips_sign():
    V, F = meshgen.jittered_torus(nu=24, nv=12, sigma=0.01, delete_frac=0.1, seed=3)
    Q = np.random.default_rng(9).uniform(-1, 1, size=(300, 3))
    M = np.diag([-1.0, 1.0, 1.0])
    np.testing.assert_allclose(oracle.winding(V.astype(np.float64) @ M, F, Q @ M), -oracle.winding(V, F, Q),
                               atol=1e-12)


def test_conventions_on_vertex_edge_and_face():
    # Configurations where alpha and beta of Eq. (7) come out exactly zero in
    # floating point, so the ATAN2 conventions of Eq. (8) decide the result.
    g = _golden("closed_forms.txt")
    r2 = math.sqrt(2.0)
    V = np.array([[-1, 0, 0], [1, 0, 0], [0, -1, r2], [0, 1, r2]], dtype=np.float64)
    F = meshgen._orient_outward(V, np.array([[0, 1, 2], [0, 1, 3], [0, 2, 3], [1, 2, 3]]), V.mean(axis=0))
    w = oracle.winding(V, F, np.stack([V[2], [0.0, 0.0, 0.0]]))
    assert w[0] == pytest.approx(g["tetra_w_at_vertex"], abs=1e-13)
    assert w[1] == pytest.approx(g["tetra_w_at_edge_midpoint"], abs=1e-13)
    Vc = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)
    Fc = meshgen._orient_outward(Vc, np.array([[0, 1, 2], [0, 1, 3], [0, 2, 3], [1, 2, 3]]), Vc.mean(axis=0))
    w = oracle.winding(Vc, Fc, np.array([[0.25, 0.25, 0.0]]))
    assert w[0] == pytest.approx(g["corner_tetra_w_on_face_interior"], abs=1e-13)


def test_single_face_in_plane_conventions():
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=np.float64)
    # interior of the face: Omega = +2pi (negative zero in alpha must not give -2pi)
    for q in ([0.25, 0.25, 0.0], [0.25, 0.25, -0.0]):
        assert oracle.solid_angle(*v, q) == pytest.approx(2 * math.pi, abs=1e-13)
    # in the plane, outside the face: Omega = 0
    assert oracle.solid_angle(*v, [2.0, 2.0, 0.0]) == pytest.approx(0.0, abs=1e-13)
    # on an edge and on a vertex: ATAN2(0, 0) = 0
    assert oracle.solid_angle(*v, [0.5, 0.0, 0.0]) == 0.0
    assert oracle.solid_angle(*v, [1.0, 0.0, 0.0]) == 0.0


def test_grid_queries_cell_centred_x_fastest():
    Q = oracle.grid_queries([-1, -1, -1], [1, 1, 1], [4, 3, 2])
    assert Q.shape == (24, 3)
    np.testing.assert_allclose(Q[0], [-0.75, -2 / 3, -0.5])
    np.testing.assert_allclose(Q[1], [-0.25, -2 / 3, -0.5])
    np.testing.assert_allclose(Q[4], [-0.75, 0.0, -0.5])
    np.testing.assert_allclose(Q[-1], [0.75, 2 / 3, 0.5])


def test_grid_points_selected_cells():
    """Cells picked by linear index (x fastest): closed-form centres, and agreement with the
    full listing on a grid small enough to list."""
    P = oracle.grid_points([-1, -1, -1], [1, 1, 1], [4, 3, 2], [0, 5, 23])
    np.testing.assert_allclose(P, [[-0.75, -2 / 3, -0.5], [-0.25, 0.0, -0.5], [0.75, 2 / 3, 0.5]])
    Q = oracle.grid_queries([-1, 0, -2], [1, 2, 1], [5, 7, 3])
    cells = np.array([0, 4, 5, 34, 35, 70, 104])
    np.testing.assert_array_equal(oracle.grid_points([-1, 0, -2], [1, 2, 1], [5, 7, 3], cells), Q[cells])


# ---------------------------------------------------------------- gradient

def _brute_fd(V, F, Q, g, h=1e-6):
    V = V.astype(np.float64)
    G = np.zeros_like(V)
    for i in range(len(V)):
        for k in range(3):
            Vp, Vm = V.copy(), V.copy()
            Vp[i, k] += h
            Vm[i, k] -= h
            G[i, k] = (g @ oracle.winding(Vp, F, Q) - g @ oracle.winding(Vm, F, Q)) / (2 * h)
    return G


def _open_patch():
    V = np.array([[0, 0, 0], [1, 0, 0.1], [0, 1, -0.1], [1, 1, 0.3], [-0.5, 0.7, 0.2]], dtype=np.float64) * 0.6
    F = np.array([[0, 1, 2], [1, 3, 2], [0, 2, 4]], dtype=np.int32)
    return V, F


def test_gradient_matches_brute_force_fd():
    V, F = _open_patch()
    rng = np.random.default_rng(10)
    Q = rng.uniform(-1, 1, size=(40, 3))
    g = rng.normal(size=40)
    G = oracle.winding_grad(V, F, Q, g)
    np.testing.assert_allclose(G, _brute_fd(V, F, Q, g), rtol=1e-6, atol=1e-8)


def test_fd_driver_matches_brute_force():
    V, F = _open_patch()
    rng = np.random.default_rng(12)
    Q = rng.uniform(-1, 1, size=(30, 3))
    g = rng.normal(size=30)
    ids = np.array([0, 2, 4])
    fd = oracle.fd_vertex_grad(V, F, Q, g, ids, h=1e-5)
    np.testing.assert_allclose(fd, _brute_fd(V, F, Q, g, h=1e-5)[ids], rtol=1e-9, atol=1e-12)


def test_vertex_subset_gradient_equals_full_gradient_rows():
    V, F = meshgen.jittered_torus(nu=16, nv=8, sigma=0.01, delete_frac=0.1, seed=4)
    rng = np.random.default_rng(16)
    Q = rng.uniform(-1, 1, size=(300, 3))
    g = rng.normal(size=300)
    ids = np.array([0, 5, 17, 60, 127])
    np.testing.assert_allclose(oracle.vertex_grad_subset(V, F, Q, g, ids), oracle.winding_grad(V, F, Q, g)[ids],
                               rtol=1e-12, atol=1e-14)


def test_gradient_scale_bounds_gradient():
    V, F = meshgen.jittered_torus(nu=16, nv=8, sigma=0.01, delete_frac=0.1, seed=4)
    rng = np.random.default_rng(17)
    Q = rng.uniform(-1, 1, size=(300, 3))
    g = rng.normal(size=300)
    G = oracle.winding_grad(V, F, Q, g)
    S = oracle.winding_grad_scale(V, F, Q, g)
    assert np.all(np.linalg.norm(G, axis=1) <= S * (1 + 1e-12) + 1e-300)
    # a vertex with a single incident face: the scale equals the gradient norm
    counts = np.bincount(F.ravel(), minlength=len(V))
    one = np.where(counts == 1)[0]
    if len(one):
        np.testing.assert_allclose(np.linalg.norm(G[one], axis=1), S[one], rtol=1e-12)


def test_closed_mesh_gradient_vanishes():
    V, F = meshgen.icosphere(1, 0.6)
    rng = np.random.default_rng(13)
    Q = rng.uniform(-1, 1, size=(200, 3))
    G = oracle.winding_grad(V, F, Q, rng.normal(size=200))
    assert np.abs(G).max() < 1e-12


def test_gradient_translation_and_scale_identities():
    # w(V + t, q + t) = w(V, q)  =>  sum_j dw/dv_j = -dw/dq
    # w(s V, s q) = w(V, q)      =>  sum_j v_j . dw/dv_j + q . dw/dq = 0
    V, F = _open_patch()
    rng = np.random.default_rng(14)
    h = 1e-6
    for _ in range(10):
        q = rng.uniform(-1, 1, size=3)
        G = oracle.winding_grad(V, F, q[None], [1.0])
        dq = np.array([(oracle.winding(V, F, (q + h * e)[None])[0] - oracle.winding(V, F, (q - h * e)[None])[0])
                       / (2 * h) for e in np.eye(3)])
        np.testing.assert_allclose(G.sum(axis=0), -dq, rtol=1e-6, atol=1e-8)
        assert np.sum(V * G) + q @ dq == pytest.approx(0.0, abs=1e-7)


# ---------------------------------------------------------------- distance

def test_point_triangle_distance_against_dense_sampling():
    rng = np.random.default_rng(15)
    tri = rng.normal(size=(3, 3))
    F = np.array([[0, 1, 2]], dtype=np.int32)
    Q = rng.normal(size=(60, 3)) * 1.5
    d = oracle.point_mesh_distance(tri, F, Q)
    m = 400
    i, j = np.meshgrid(np.arange(m + 1), np.arange(m + 1), indexing="ij")
    keep = i + j <= m
    u, v = i[keep] / m, j[keep] / m
    P = tri[0] + u[:, None] * (tri[1] - tri[0]) + v[:, None] * (tri[2] - tri[0])
    edge = max(np.linalg.norm(tri[1] - tri[0]), np.linalg.norm(tri[2] - tri[0]))
    for k, q in enumerate(Q):
        ds = np.sqrt(((P - q) ** 2).sum(axis=1)).min()
        assert d[k] <= ds + 1e-12
        assert ds - d[k] <= 2 * edge / m


def test_point_triangle_distance_regions():
    tri = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=np.float64)
    F = np.array([[0, 1, 2]], dtype=np.int32)
    Q = np.array([[0.2, 0.2, 0.5], [-1, -1, 0], [2, 0, 1], [0.5, -1, 0]], dtype=np.float64)
    np.testing.assert_allclose(oracle.point_mesh_distance(tri, F, Q), [0.5, math.sqrt(2), math.sqrt(2), 1.0],
                               atol=1e-14)


# ---------------------------------------------------------------- Eq. (4) and Algorithm 2

def test_dipole_discretization_converges_far_from_surface():
    Q = np.array([[0.0, 0.0, 0.0], [0.1, -0.2, 0.05], [1.5, 0.0, 0.0], [0.0, 2.0, 1.0]])
    errs = []
    for k in (2, 3, 4):
        V, F = meshgen.icosphere(k, 0.8)
        errs.append(np.abs(oracle.dipole_winding(V, F, Q) - np.array([1.0, 1.0, 0.0, 0.0])).max())
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 5e-3


def _rotated_face(scale, seed):
    """One triangle (0,0,0), (s,0,0), (0,1.3s,0) under a seeded rotation and shift, with its exact
    area, unit normal (counter-clockwise side) and centroid, and an in-plane unit vector."""
    rng = np.random.default_rng(seed)
    R, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(R) < 0:
        R[:, 0] = -R[:, 0]
    shift = rng.uniform(-0.3, 0.3, size=3)
    P = np.array([[0.0, 0, 0], [scale, 0, 0], [0, 1.3 * scale, 0]])
    V = P @ R.T + shift
    area = 0.5 * 1.3 * scale * scale
    n = R @ np.array([0.0, 0, 1])
    u = R @ np.array([0.6, 0.8, 0.0])
    return V, np.array([[0, 1, 2]], dtype=np.int32), area, n, V.mean(axis=0), u


def test_dipole_single_face_closed_forms():
    # Eq. (4) for one face: W = (1/4pi) <n, E_q(c)> area with E_q(r) = (r - q)/|r - q|^3. For q at
    # distance d behind the centroid along the normal, c - q = d n, so W = area / (4 pi d^2); moved
    # by t inside the plane, W = area d / (4 pi (d^2 + t^2)^(3/2)); in front of the face the sign
    # flips. The area is not 1/2, d is not 1 and the evaluation point matters, so dropping the
    # area, an unnormalized normal, a wrong power of |r - q| or evaluating at a vertex all fail.
    for seed, s, d, t in ((0, 0.7, 0.37, 0.23), (1, 1.6, 2.5, -1.1), (2, 0.05, 0.011, 0.004)):
        V, F, area, n, c, u = _rotated_face(s, seed)
        Q = np.stack([c - d * n, c - d * n + t * u, c + d * n])
        want = np.array([area / (4 * math.pi * d * d),
                         area * d / (4 * math.pi * (d * d + t * t) ** 1.5),
                         -area / (4 * math.pi * d * d)])
        got = oracle.dipole_winding(V, F, Q)
        assert np.allclose(got, want, rtol=1e-12, atol=0), (seed, got, want)


def test_dipole_sums_faces_and_skips_degenerate_ones():
    # Eq. (4) is a plain sum over faces: two separate faces give the sum of their single-face
    # closed forms, and a zero-area face adds nothing.
    V1, F1, a1, n1, c1, _ = _rotated_face(0.4, 5)
    V2, F2, a2, n2, c2, _ = _rotated_face(0.9, 6)
    V2 = V2 + np.array([1.5, 0.0, 0.0])
    c2 = c2 + np.array([1.5, 0.0, 0.0])
    Vd = np.array([[0.2, 0.2, 0.2], [0.4, 0.4, 0.4], [0.8, 0.8, 0.8]])  # collinear: zero area
    V = np.concatenate([V1, V2, Vd])
    F = np.concatenate([F1, F2 + 3, np.array([[6, 7, 8]], dtype=np.int32)])
    q = c1 - 0.3 * n1
    r = c2 - q
    want = (a1 / (4 * math.pi * 0.09)
            + a2 * float(np.dot(n2, r)) / (4 * math.pi * float(np.linalg.norm(r)) ** 3))
    assert abs(oracle.dipole_winding(V, F, q[None])[0] - want) <= 1e-13 * abs(want)


def test_flipped_duplication_closes_open_cap():
    V, F = meshgen.open_cap(freq=6, radius=0.5, max_polar=1.0)
    V2, F2 = oracle.flipped_duplication(V, F, eps=0.01)
    assert len(V2) == 2 * len(V) and len(F2) == 2 * len(F)
    # Copied faces are reversed: same vertex set, opposite orientation.
    n1 = np.cross(V2[F2[0, 1]] - V2[F2[0, 0]], V2[F2[0, 2]] - V2[F2[0, 0]])
    j = len(F)
    n2 = np.cross(V2[F2[j, 1]] - V2[F2[j, 0]], V2[F2[j, 2]] - V2[F2[j, 0]])
    assert np.dot(n1, n2) < 0
    # A point inside the slit (between the layers, under the cap's apex) is occupied; points
    # well away are not.
    apex = V[np.argmax(V[:, 2])].astype(np.float64)
    qs = np.stack([apex * (1 - 0.005 / np.linalg.norm(apex)), [0, 0, 0.0], [0, 0, 0.9], [0.8, 0, 0]])
    w = oracle.winding(V2, F2, qs)
    # The rim of the slit stays open, so the shell is only almost closed (§2.3):
    # the slit point is near 1, not exactly 1.
    assert w[0] > 0.95
    assert np.all(np.abs(w[1:]) < 0.05)
    # without the duplication the open cap leaves that point far from binary
    w1 = oracle.winding(V, F, qs[:1])[0]
    assert 0.1 < w1 < 0.9


# ---------------------------------------------------------------- closed meshes by ray crossings

@pytest.mark.parametrize("mesh", ["tetra", "cube", "ico2"])
def test_ray_winding_of_convex_mesh_is_indicator(mesh):
    # a closed convex mesh: the signed ray-crossing count is the plane-side indicator, on an
    # anisotropic grid over an off-centre box; reversing every face negates it
    V, F = {"tetra": lambda: meshgen.regular_tetrahedron(0.5, centre=(0.03, -0.02, 0.05)),
            "cube": lambda: meshgen.cube(0.45, centre=(0.02, 0.01, -0.03)),
            "ico2": lambda: meshgen.icosphere(2, 0.8)}[mesh]()
    lo, hi, n = (-0.97, -1.01, -0.93), (1.03, 0.99, 1.07), (23, 19, 17)
    w, und = oracle.ray_winding_grid(V, F, lo, hi, n)
    Q = oracle.grid_queries(lo, hi, n)
    inside, dplane = _inside_convex(V, F, Q)
    keep = (dplane > 1e-6) & ~und
    assert keep.sum() > 0.95 * len(Q)
    assert np.array_equal(w[keep], inside[keep].astype(np.int32))
    wr, undr = oracle.ray_winding_grid(V, F[:, ::-1], lo, hi, n)
    assert np.array_equal(wr[keep & ~undr], -w[keep & ~undr])


def test_ray_winding_marks_rays_through_a_vertex_undecided():
    # a vertex placed exactly on a row's ray: that row's counts are undecided, the others are not
    # (a generically rotated tetrahedron, so that no other row or centre meets an edge or face)
    V, F = meshgen.regular_tetrahedron(0.5)
    R, _ = np.linalg.qr(np.random.default_rng(21).normal(size=(3, 3)))
    V = V.astype(np.float64) @ R.T
    lo, hi, n = (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), (16, 16, 16)
    h = 2.0 / 16
    V = V + np.array([0.0137, (-1.0 + 10.5 * h) - V[0, 1], (-1.0 + 5.5 * h) - V[0, 2]])
    w, und = oracle.ray_winding_grid(V, F, lo, hi, n)
    rows = und.reshape(16, 16, 16).any(axis=2)  # [iz, iy]
    assert rows[5, 10] and rows.sum() == 1
    inside, _ = _inside_convex(V, F, oracle.grid_queries(lo, hi, n))
    assert np.array_equal(w[~und], inside[~und].astype(np.int32))


def test_ray_winding_matches_solid_angles_on_closed_nonconvex_mesh():
    # closed jittered torus (no faces deleted): the signed crossing count equals the solid-angle
    # winding number of Eq. (5) rounded, wherever the count is decided
    V, F = meshgen.jittered_torus(nu=40, nv=20, sigma=0.01, delete_frac=0.0, seed=2)
    lo, hi, n = (-1.0, -1.0, -0.5), (1.0, 1.0, 0.5), (26, 24, 13)
    w, und = oracle.ray_winding_grid(V, F, lo, hi, n)
    w64 = oracle.winding(V, F, oracle.grid_queries(lo, hi, n))
    assert np.abs(w64[~und] - w[~und]).max() < 1e-9
    assert (w == 1).sum() > 100 and (w == 0).sum() > 100
