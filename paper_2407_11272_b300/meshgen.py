"""Seeded synthetic inputs: triangle meshes, grids, upstream gradients.

This module only builds inputs. It holds none of the winding-number
arithmetic (no solid angles, no sums over faces, no query generation), so
both the CUDA path and the FP64 oracle may consume what it produces.

Every mesh is returned as ``(verts float32 [V,3], faces int32 [F,3])`` with
faces ordered counter-clockwise when seen from outside, so that the
generalized winding number of Eq. (5) is +1 inside a closed surface.

The shapes stand in for the paper's test meshes (public scan meshes with
828 to 268 686 faces, normalized to [-1, 1], §3 and §3.1), which are not
available here:

* ``icosphere(3, 0.8)``            small closed mesh, 1280 faces
* ``jittered_torus(...)``          open irregular mesh (holes), ~36 000 faces
* ``sh_sphere(101, 0.7, ...)``     large closed mesh, 204 020 faces
* ``ellipsoid_union(...)``         overlapping components, 500 .. 100 000 faces
* ``open_cap(...)``                an open surface for Algorithm 2
"""
from __future__ import annotations

import functools
import math

import numpy as np

__all__ = [
    "icosahedron", "icosphere", "geodesic_sphere", "sh_sphere", "jittered_torus",
    "ellipsoid", "ellipsoid_union", "random_ellipsoids", "open_cap", "octant_triangle",
    "regular_tetrahedron", "cube", "upstream_gradient", "query_subsample",
    "random_vertex_ids", "normalize_unit_box", "face_count", "CONFIGS",
]


def _orient_outward(verts: np.ndarray, faces: np.ndarray, centre=None) -> np.ndarray:
    """Flip faces whose normal points towards ``centre`` (star-shaped meshes only)."""
    c = np.zeros(3) if centre is None else np.asarray(centre, dtype=np.float64)
    v = verts.astype(np.float64)
    p0, p1, p2 = v[faces[:, 0]], v[faces[:, 1]], v[faces[:, 2]]
    n = np.cross(p1 - p0, p2 - p0)
    cen = (p0 + p1 + p2) / 3.0 - c
    flip = np.einsum("ij,ij->i", n, cen) < 0
    out = faces.copy()
    out[flip] = out[flip][:, [0, 2, 1]]
    return out


def icosahedron():
    """12 vertices on the unit sphere, 20 outward-oriented faces."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([
        [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
        [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
        [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1],
    ], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
    ], dtype=np.int64)
    return v, _orient_outward(v, f)


def icosphere(subdivisions: int, radius: float = 1.0, centre=(0.0, 0.0, 0.0)):
    """Recursive midpoint subdivision of the icosahedron, re-projected each level.

    ``subdivisions=3`` gives 642 vertices / 1280 faces; ``6`` gives 40 962 / 81 920.
    """
    v, f = icosahedron()
    verts = [tuple(p) for p in v]
    faces = f
    for _ in range(subdivisions):
        cache: dict[tuple[int, int], int] = {}

        def mid(i: int, j: int) -> int:
            key = (i, j) if i < j else (j, i)
            k = cache.get(key)
            if k is None:
                p = (np.asarray(verts[i]) + np.asarray(verts[j])) * 0.5
                p /= np.linalg.norm(p)
                k = len(verts)
                verts.append(tuple(p))
                cache[key] = k
            return k

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = np.asarray(nf, dtype=np.int64)
    vv = np.asarray(verts, dtype=np.float64) * radius + np.asarray(centre, dtype=np.float64)
    return vv.astype(np.float32), faces.astype(np.int32)


@functools.lru_cache(maxsize=128)
def _unit_geodesic(freq: int):
    v, f = icosahedron()
    n = int(freq)
    I, J = [], []
    for i in range(n + 1):
        for j in range(n + 1 - i):
            I.append(i)
            J.append(j)
    I = np.asarray(I, dtype=np.int64)
    J = np.asarray(J, dtype=np.int64)
    P = len(I)
    pid = lambda i, j: i * (n + 1) - (i * (i - 1)) // 2 + j  # noqa: E731  (index of (i, j) in I, J)
    # Key of every point of every face: its (icosahedron vertex, integer weight) pairs, zero weights
    # dropped, sorted by vertex; points shared along edges and corners get equal keys.
    W = np.stack([np.broadcast_to(n - I - J, (20, P)), np.broadcast_to(I, (20, P)), np.broadcast_to(J, (20, P))],
                 axis=-1)
    Vid = np.broadcast_to(f[:, None, :], (20, P, 3)).copy()
    Vid[W == 0] = -1
    order = np.argsort(Vid, axis=-1)
    key = np.concatenate([np.take_along_axis(Vid, order, -1), np.take_along_axis(W, order, -1)], axis=-1)
    key = key.reshape(20 * P, 6)
    uniq, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
    inv = inv.reshape(20, P)
    Wf = W.reshape(20 * P, 3)[first].astype(np.float64)
    Vf = np.broadcast_to(f[:, None, :], (20, P, 3)).reshape(20 * P, 3)[first]
    pos = (Wf[:, :1] * v[Vf[:, 0]] + Wf[:, 1:2] * v[Vf[:, 1]] + Wf[:, 2:] * v[Vf[:, 2]]) / n
    pos /= np.linalg.norm(pos, axis=1, keepdims=True)
    tris = []
    for i in range(n):
        for j in range(n - i):
            tris.append((pid(i, j), pid(i + 1, j), pid(i, j + 1)))
            if i + j < n - 1:
                tris.append((pid(i + 1, j), pid(i + 1, j + 1), pid(i, j + 1)))
    tris = np.asarray(tris, dtype=np.int64)
    faces = inv[:, tris].reshape(-1, 3)
    return pos, faces


def geodesic_sphere(freq: int, radius: float = 1.0):
    """Class-I geodesic sphere: each icosahedron face split into ``freq**2`` triangles.

    ``freq=101`` gives 102 012 vertices and 20 * 101**2 = 204 020 faces.
    Points are shared between faces by their exact barycentric key.
    """
    pos, faces = _unit_geodesic(int(freq))
    return (pos * radius).astype(np.float32), faces.astype(np.int32)


def _real_sh(lmax: int, theta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Real orthonormal spherical harmonics, shape [(lmax+1)**2, n]; theta polar, phi azimuth."""
    from scipy.special import sph_harm_y  # noqa: PLC0415

    rows = []
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            y = sph_harm_y(l, abs(m), theta, phi)
            if m == 0:
                rows.append(y.real)
            elif m > 0:
                rows.append(math.sqrt(2.0) * (-1) ** m * y.real)
            else:
                rows.append(math.sqrt(2.0) * (-1) ** m * y.imag)
    return np.asarray(rows)


def sh_sphere(freq: int = 101, radius: float = 0.7, lmax: int = 8, sigma: float = 0.02,
              seed: int = 3):
    """Geodesic sphere with radius ``radius + sum c_lm Y_lm``, c_lm ~ N(0, sigma^2)."""
    v, f = geodesic_sphere(freq, 1.0)
    d = v.astype(np.float64)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    theta = np.arccos(np.clip(d[:, 2], -1.0, 1.0))
    phi = np.arctan2(d[:, 1], d[:, 0])
    rng = np.random.default_rng(seed)
    coef = rng.normal(0.0, sigma, size=(lmax + 1) ** 2)
    r = radius + coef @ _real_sh(lmax, theta, phi)
    return (d * r[:, None]).astype(np.float32), f


def jittered_torus(R: float = 0.6, r: float = 0.25, nu: int = 200, nv: int = 100,
                   sigma: float = 0.01, delete_frac: float = 0.10, seed: int = 0):
    """Torus grid ``nu x nv`` (2*nu*nv triangles), Gaussian vertex jitter, faces deleted.

    With the defaults: 20 000 vertices, 40 000 triangles before deletion,
    36 000 after deleting 10 % uniformly at random: an open, irregular mesh.
    """
    i = np.arange(nu)[:, None]
    j = np.arange(nv)[None, :]
    u = 2.0 * np.pi * i / nu
    w = 2.0 * np.pi * j / nv
    x = (R + r * np.cos(w)) * np.cos(u)
    y = (R + r * np.cos(w)) * np.sin(u)
    z = r * np.sin(w) * np.ones_like(u)
    verts = np.stack([x, y, z], axis=-1).reshape(-1, 3)
    vid = lambda a, b: (a % nu) * nv + (b % nv)  # noqa: E731
    faces = []
    for a in range(nu):
        for b in range(nv):
            p00, p10, p11, p01 = vid(a, b), vid(a + 1, b), vid(a + 1, b + 1), vid(a, b + 1)
            faces.append((p00, p10, p11))
            faces.append((p00, p11, p01))
    faces = np.asarray(faces, dtype=np.int64)
    # orient outward: normal must point away from the tube centre line
    p0, p1, p2 = verts[faces[:, 0]], verts[faces[:, 1]], verts[faces[:, 2]]
    n = np.cross(p1 - p0, p2 - p0)
    cen = (p0 + p1 + p2) / 3.0
    rad = np.stack([cen[:, 0], cen[:, 1], np.zeros(len(cen))], axis=1)
    rad = R * rad / np.linalg.norm(rad, axis=1, keepdims=True)
    flip = np.einsum("ij,ij->i", n, cen - rad) < 0
    faces[flip] = faces[flip][:, [0, 2, 1]]
    rng = np.random.default_rng(seed)
    verts = verts + rng.normal(0.0, sigma, size=verts.shape)
    keep = np.sort(rng.permutation(len(faces))[: len(faces) - int(round(delete_frac * len(faces)))])
    return verts.astype(np.float32), faces[keep].astype(np.int32)


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    q, rr = np.linalg.qr(rng.normal(size=(3, 3)))
    q *= np.sign(np.diag(rr))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def ellipsoid(semi_axes, centre=(0.0, 0.0, 0.0), rotation=None, freq: int = 8):
    """Geodesic sphere mapped affinely onto an ellipsoid (orientation preserved)."""
    v, f = geodesic_sphere(freq, 1.0)
    p = v.astype(np.float64) * np.asarray(semi_axes, dtype=np.float64)
    if rotation is not None:
        p = p @ np.asarray(rotation, dtype=np.float64).T
    p += np.asarray(centre, dtype=np.float64)
    return p.astype(np.float32), f


def random_ellipsoids(n: int, rng: np.random.Generator, axis_lo=0.15, axis_hi=0.45,
                      centre_lo=-0.5, centre_hi=0.5):
    """Parameters (semi_axes, centre, rotation) of ``n`` random ellipsoids."""
    out = []
    for _ in range(n):
        out.append((rng.uniform(axis_lo, axis_hi, size=3), rng.uniform(centre_lo, centre_hi, size=3),
                    _random_rotation(rng)))
    return out


def ellipsoid_union(target_faces: int, n_components: int, seed: int, jitter: float = 0.002,
                    axis_lo=0.15, axis_hi=0.45):
    """Union (concatenation, no boolean) of ``n_components`` jittered ellipsoids.

    Components overlap, so the winding number reaches 2 or more inside overlaps;
    occupancy w > 0.5 is still the union. The face count is close to
    ``target_faces`` (each component a geodesic sphere of frequency ~sqrt(F/20n)).
    """
    rng = np.random.default_rng(seed)
    per = max(20, target_faces // max(1, n_components))
    freq = max(1, int(round(math.sqrt(per / 20.0))))
    vs, fs, off = [], [], 0
    for axes, c, rot in random_ellipsoids(n_components, rng, axis_lo, axis_hi):
        v, f = ellipsoid(axes, c, rot, freq)
        v = v + rng.normal(0.0, jitter, size=v.shape).astype(np.float32)
        vs.append(v)
        fs.append(f + off)
        off += len(v)
    return np.concatenate(vs).astype(np.float32), np.concatenate(fs).astype(np.int32)


def open_cap(freq: int = 8, radius: float = 0.5, max_polar: float = 1.2):
    """Open spherical cap: faces of a geodesic sphere whose centroid polar angle < max_polar."""
    v, f = geodesic_sphere(freq, radius)
    c = v[f].mean(axis=1)
    pol = np.arccos(np.clip(c[:, 2] / np.linalg.norm(c, axis=1), -1, 1))
    f = f[pol < max_polar]
    used = np.unique(f)
    remap = -np.ones(len(v), dtype=np.int64)
    remap[used] = np.arange(len(used))
    return v[used].astype(np.float32), remap[f].astype(np.int32)


def octant_triangle():
    """The triangle (1,0,0),(0,1,0),(0,0,1): seen from the origin it covers one octant."""
    v = np.eye(3, dtype=np.float32)
    f = np.array([[0, 1, 2]], dtype=np.int32)
    return v, f


def regular_tetrahedron(scale: float = 0.5, centre=(0.0, 0.0, 0.0)):
    """Regular tetrahedron centred at ``centre``, outward faces."""
    v = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64) * scale
    v += np.asarray(centre, dtype=np.float64)
    f = np.array([[0, 1, 2], [0, 1, 3], [0, 2, 3], [1, 2, 3]], dtype=np.int64)
    return v.astype(np.float32), _orient_outward(v, f, centre).astype(np.int32)


def cube(half: float = 0.5, centre=(0.0, 0.0, 0.0)):
    """Axis-aligned cube, 8 vertices, 12 outward triangles."""
    s = np.array([[x, y, z] for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)], dtype=np.float64)
    v = s * half + np.asarray(centre, dtype=np.float64)
    quads = [(0, 1, 3, 2), (4, 6, 7, 5), (0, 4, 5, 1), (2, 3, 7, 6), (0, 2, 6, 4), (1, 5, 7, 3)]
    f = []
    for a, b, c, d in quads:
        f += [(a, b, c), (a, c, d)]
    f = np.asarray(f, dtype=np.int64)
    return v.astype(np.float32), _orient_outward(v, f, centre).astype(np.int32)


def normalize_unit_box(verts: np.ndarray, margin: float = 0.0) -> np.ndarray:
    """Affine rescale of a vertex array into [-1+margin, 1-margin]^3 (§3.1: normalized to [-1,1])."""
    v = verts.astype(np.float64)
    lo, hi = v.min(axis=0), v.max(axis=0)
    c = (lo + hi) / 2.0
    s = (hi - lo).max() / 2.0
    return ((v - c) / s * (1.0 - margin)).astype(np.float32)


def upstream_gradient(n: int, seed: int = 1) -> np.ndarray:
    """dL/dw ~ N(0, 1) per query (float32)."""
    return np.random.default_rng(seed).standard_normal(n).astype(np.float32)


def query_subsample(n_total: int, n: int, seed: int = 4) -> np.ndarray:
    """Sorted seeded sample of ``n`` distinct query indices out of ``n_total``."""
    n = min(n, n_total)
    return np.sort(np.random.default_rng(seed).choice(n_total, size=n, replace=False)).astype(np.int64)


def random_vertex_ids(nv: int, n: int = 64, seed: int = 2) -> np.ndarray:
    return np.sort(np.random.default_rng(seed).choice(nv, size=min(n, nv), replace=False)).astype(np.int64)


def face_count(faces: np.ndarray) -> int:
    return int(faces.shape[0])


# Workloads used by the tests and the benchmark. Grids are cell-centred over
# [lo, hi]^3 with ``n`` cells per axis.
CONFIGS = {
    "icosphere_32": dict(mesh=lambda: icosphere(3, 0.8), n=32, lo=-1.0, hi=1.0),
    "torus_128": dict(mesh=lambda: jittered_torus(), n=128, lo=-1.0, hi=1.0),
    "shsphere_256": dict(mesh=lambda: sh_sphere(), n=256, lo=-1.0, hi=1.0),
}
