"""FP64 CPU oracle (ctypes wrapper around ``oracle.c``).

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this package. The product path (the
``paper_2407_11272_b300`` package and its CUDA library) never imports,
links or runs anything here, and nothing here imports the product.

Functions (each follows the passage named in ``oracle.c``):

* ``solid_angle(v0, v1, v2, q)``      Eq. (7), Omega = 2 ATAN2(alpha, beta)
* ``atan2_table(y, x)``               Eq. (8)
* ``winding(V, F, Q)``                Eq. (5) / Algorithm 1, W = (1/4pi) sum Omega
* ``grid_queries(lo, hi, n)``         cell-centred voxel grid (§3), x fastest
* ``grid_points(lo, hi, n, cells)``   the same centres for selected linear cell indices
* ``winding_grad(V, F, Q, g)``        sum_q g_q dW(q)/dV, chain rule through Eq. (7)
* ``point_mesh_distance(V, F, Q)``    exact Euclidean distance to the nearest face
* ``vertex_grad_subset(V, F, Q, g, ids)``  rows of winding_grad for selected vertices
* ``winding_grad_scale(V, F, Q, g)``  per-vertex sum of |face contributions| (cancellation scale)
* ``fd_vertex_grad(V, F, Q, g, ids)`` FP64 central differences of sum_q g_q W(q)
* ``dipole_winding(V, F, Q)``         Eq. (4), naive dipole discretization
* ``ray_winding_grid(V, F, lo, hi, n)``  closed meshes: w on a grid by signed ray crossings (Eq. (3))
* ``flipped_duplication(V, F, eps)``  Algorithm 2, open mesh to thin closed shell

All arrays are converted to float64 / int32 before the call; vertex inputs
given as float32 are widened exactly.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "oracle.c"
_LIB = _HERE / "liboracle.so"
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_f = ctypes.POINTER(ctypes.c_float)
_i32 = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.POINTER(ctypes.c_int64)
_I64 = ctypes.c_int64


def build(force: bool = False) -> Path:
    """Compile ``oracle.c`` with gcc (OpenMP, IEEE semantics, no FP contraction)."""
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB.with_suffix(f".so.tmp{os.getpid()}")
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC",
                        str(_SRC), "-o", str(tmp), "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(str(build()))
        lib.atan2_table.restype = ctypes.c_double
        lib.atan2_table.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.orc_solid_angle.restype = ctypes.c_double
        lib.orc_solid_angle.argtypes = [_d, _d, _d, _d]
        lib.orc_max_threads.restype = ctypes.c_int
        mesh_q = [_d, _I64, _i32, _I64, _d, _I64]
        lib.orc_winding.argtypes = mesh_q + [_d, ctypes.c_int]
        lib.orc_dipole_winding.argtypes = mesh_q + [_d, ctypes.c_int]
        lib.orc_point_mesh_distance.argtypes = mesh_q + [_d, ctypes.c_int]
        lib.orc_winding_grad.argtypes = mesh_q + [_d, _d, ctypes.c_int]
        lib.orc_fd_vertex_grad.argtypes = mesh_q + [_d, _i64, _I64, ctypes.c_double, _d, ctypes.c_int]
        lib.orc_vertex_grad_subset.argtypes = mesh_q + [_d, _i64, _I64, _d, ctypes.c_int]
        lib.orc_winding_grad_scale.argtypes = mesh_q + [_d, _d, ctypes.c_int]
        lib.orc_grid_queries.argtypes = [_f, _f, _i32, _d]
        lib.orc_grid_points.argtypes = [_f, _f, _i32, _i64, _I64, _d]
        lib.orc_ray_winding_grid.argtypes = [_d, _I64, _i32, _I64, _f, _f, _i32, ctypes.c_double, ctypes.c_double,
                                             _i32, ctypes.POINTER(ctypes.c_uint8), ctypes.c_int]
        lib.orc_ray_winding_grid.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_d)


def _mesh(V, F):
    V = np.ascontiguousarray(np.asarray(V, dtype=np.float64).reshape(-1, 3))
    F = np.ascontiguousarray(np.asarray(F, dtype=np.int32).reshape(-1, 3))
    if F.size and (F.min() < 0 or F.max() >= len(V)):
        raise ValueError("face index out of range")
    return V, F


def _q(Q):
    return np.ascontiguousarray(np.asarray(Q, dtype=np.float64).reshape(-1, 3))


def max_threads() -> int:
    return int(_load().orc_max_threads())


def atan2_table(y: float, x: float) -> float:
    return float(_load().atan2_table(float(y), float(x)))


def solid_angle(v0, v1, v2, q) -> float:
    a = [np.ascontiguousarray(np.asarray(t, dtype=np.float64).reshape(3)) for t in (v0, v1, v2, q)]
    return float(_load().orc_solid_angle(*[_dp(t) for t in a]))


def winding(V, F, Q, threads: int = 0) -> np.ndarray:
    V, F = _mesh(V, F)
    Q = _q(Q)
    out = np.empty(len(Q), dtype=np.float64)
    _load().orc_winding(_dp(V), len(V), F.ctypes.data_as(_i32), len(F), _dp(Q), len(Q), _dp(out), threads)
    return out


def dipole_winding(V, F, Q, threads: int = 0) -> np.ndarray:
    V, F = _mesh(V, F)
    Q = _q(Q)
    out = np.empty(len(Q), dtype=np.float64)
    _load().orc_dipole_winding(_dp(V), len(V), F.ctypes.data_as(_i32), len(F), _dp(Q), len(Q), _dp(out), threads)
    return out


def point_mesh_distance(V, F, Q, threads: int = 0) -> np.ndarray:
    V, F = _mesh(V, F)
    Q = _q(Q)
    out = np.empty(len(Q), dtype=np.float64)
    _load().orc_point_mesh_distance(_dp(V), len(V), F.ctypes.data_as(_i32), len(F), _dp(Q), len(Q), _dp(out),
                                    threads)
    return out


def winding_grad(V, F, Q, upstream, threads: int = 0) -> np.ndarray:
    V, F = _mesh(V, F)
    Q = _q(Q)
    g = np.ascontiguousarray(np.asarray(upstream, dtype=np.float64).reshape(-1))
    if len(g) != len(Q):
        raise ValueError("upstream must have one value per query")
    out = np.zeros((len(V), 3), dtype=np.float64)
    _load().orc_winding_grad(_dp(V), len(V), F.ctypes.data_as(_i32), len(F), _dp(Q), len(Q), _dp(g), _dp(out),
                             threads)
    return out


def winding_grad_scale(V, F, Q, upstream, threads: int = 0) -> np.ndarray:
    """Per vertex: sum over incident faces of the norm of that face's gradient contribution."""
    V, F = _mesh(V, F)
    Q = _q(Q)
    g = np.ascontiguousarray(np.asarray(upstream, dtype=np.float64).reshape(-1))
    out = np.zeros(len(V), dtype=np.float64)
    _load().orc_winding_grad_scale(_dp(V), len(V), F.ctypes.data_as(_i32), len(F), _dp(Q), len(Q), _dp(g),
                                   _dp(out), threads)
    return out


def fd_vertex_grad(V, F, Q, upstream, vertex_ids, h: float = 1e-4, threads: int = 0) -> np.ndarray:
    V, F = _mesh(V, F)
    Q = _q(Q)
    g = np.ascontiguousarray(np.asarray(upstream, dtype=np.float64).reshape(-1))
    ids = np.ascontiguousarray(np.asarray(vertex_ids, dtype=np.int64).reshape(-1))
    out = np.zeros((len(ids), 3), dtype=np.float64)
    _load().orc_fd_vertex_grad(_dp(V), len(V), F.ctypes.data_as(_i32), len(F), _dp(Q), len(Q), _dp(g),
                               ids.ctypes.data_as(_i64), len(ids), float(h), _dp(out), threads)
    return out


def vertex_grad_subset(V, F, Q, upstream, vertex_ids, threads: int = 0) -> np.ndarray:
    """Rows of ``winding_grad`` for the selected vertices only (incident faces, all queries)."""
    V, F = _mesh(V, F)
    Q = _q(Q)
    g = np.ascontiguousarray(np.asarray(upstream, dtype=np.float64).reshape(-1))
    ids = np.ascontiguousarray(np.asarray(vertex_ids, dtype=np.int64).reshape(-1))
    out = np.zeros((len(ids), 3), dtype=np.float64)
    _load().orc_vertex_grad_subset(_dp(V), len(V), F.ctypes.data_as(_i32), len(F), _dp(Q), len(Q), _dp(g),
                                   ids.ctypes.data_as(_i64), len(ids), _dp(out), threads)
    return out


def grid_queries(lo, hi, n) -> np.ndarray:
    lo = np.ascontiguousarray(np.broadcast_to(np.asarray(lo, dtype=np.float32), (3,)))
    hi = np.ascontiguousarray(np.broadcast_to(np.asarray(hi, dtype=np.float32), (3,)))
    nn = np.ascontiguousarray(np.broadcast_to(np.asarray(n, dtype=np.int32), (3,)))
    out = np.empty((int(np.prod(nn.astype(np.int64))), 3), dtype=np.float64)
    _load().orc_grid_queries(lo.ctypes.data_as(_f), hi.ctypes.data_as(_f), nn.ctypes.data_as(_i32), _dp(out))
    return out


def grid_points(lo, hi, n, cells) -> np.ndarray:
    """Centres of the grid cells with the given linear indices (x fastest), FP64 [m, 3]."""
    lo = np.ascontiguousarray(np.broadcast_to(np.asarray(lo, dtype=np.float32), (3,)))
    hi = np.ascontiguousarray(np.broadcast_to(np.asarray(hi, dtype=np.float32), (3,)))
    nn = np.ascontiguousarray(np.broadcast_to(np.asarray(n, dtype=np.int32), (3,)))
    c = np.ascontiguousarray(np.asarray(cells, dtype=np.int64).ravel())
    out = np.empty((len(c), 3), dtype=np.float64)
    _load().orc_grid_points(lo.ctypes.data_as(_f), hi.ctypes.data_as(_f), nn.ctypes.data_as(_i32),
                            c.ctypes.data_as(_i64), len(c), _dp(out))
    return out


def ray_winding_grid(V, F, lo, hi, n, eps_bary: float = 1e-12, eps_x: float = 1e-9, threads: int = 0):
    """Winding number of a CLOSED, consistently oriented mesh at every cell centre of the grid
    (x fastest), by signed crossings of rays along +x (Eq. (3)), and a mask of the cells whose
    count is undecided (a ray grazing an edge or vertex, or a centre within eps_x of a crossing).
    Returns (w int32 [nx*ny*nz], undecided bool [nx*ny*nz])."""
    V, F = _mesh(V, F)
    lo = np.ascontiguousarray(lo, dtype=np.float32)
    hi = np.ascontiguousarray(hi, dtype=np.float32)
    nn = np.ascontiguousarray(n, dtype=np.int32)
    total = int(nn[0]) * int(nn[1]) * int(nn[2])
    w = np.empty(total, dtype=np.int32)
    amb = np.empty(total, dtype=np.uint8)
    st = _load().orc_ray_winding_grid(_dp(V), len(V), F.ctypes.data_as(_i32), len(F), lo.ctypes.data_as(_f),
                                      hi.ctypes.data_as(_f), nn.ctypes.data_as(_i32), eps_bary, eps_x,
                                      w.ctypes.data_as(_i32), amb.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                      threads)
    if st != 0:
        raise MemoryError("orc_ray_winding_grid: out of host memory")
    return w, amb.astype(bool)


def occupancy(w: np.ndarray) -> np.ndarray:
    """Binarised occupancy, w > 0.5 (the paper states no threshold; this is the reading used)."""
    return (np.asarray(w) > 0.5).astype(np.uint8)


def flipped_duplication(V, F, eps: float = 0.01):
    """Algorithm 2: duplicate an open mesh, push the copy along -N_v by eps, flip its faces.

    Vertex normals N_v are the normalized sums of the incident faces' area
    vectors (the paper does not say how N_v is computed; area weighting is
    the reading used). "Flip" reverses each copied face's orientation:
    (v0', v1', v2') becomes (v0', v2', v1').
    """
    V = np.asarray(V, dtype=np.float64).reshape(-1, 3)
    F = np.asarray(F, dtype=np.int64).reshape(-1, 3)
    nvert = np.zeros_like(V)
    for f in F:
        a, b, c = V[f[0]], V[f[1]], V[f[2]]
        m = np.cross(b - a, c - a)
        for k in f:
            nvert[k] += m
    ln = np.linalg.norm(nvert, axis=1, keepdims=True)
    ln[ln == 0] = 1.0
    nvert = nvert / ln
    V2 = V - eps * nvert
    F2 = F[:, [0, 2, 1]] + len(V)
    return np.concatenate([V, V2]), np.concatenate([F, F2]).astype(np.int32)
