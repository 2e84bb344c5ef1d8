"""Python binding of the C ABI in ``include/dv_api.h`` (ctypes).

Argument marshalling only: every computation runs in ``libdv.so``'s CUDA
kernels. The functions keep the C names. Tensors must be CUDA tensors on the
current device (PyTorch supplies memory and streams; nothing here computes).
If the library is missing or cannot be loaded, every call raises
``DvError``: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

from . import build as _build

__all__ = [
    "DvError", "Grid", "Mesh", "PRECISION", "dv_abi_version", "dv_mesh_create", "dv_mesh_update_verts",
    "dv_mesh_reserve", "dv_mesh_check", "dv_winding", "dv_voxelize_grid", "dv_winding_backward",
    "dv_winding_backward_boundary", "dv_mesh_num_boundary_edges", "dv_mesh_num_strip_events",
    "dv_run_batch", "dv_dipole_winding", "dv_dipole_backward", "dv_flipped_duplication", "dv_build_strips", "dv_build_face_pairs", "dv_selftest_bounded_wait", "dv_selftest_forward_timeout", "dv_debug_report", "dv_profile_enable", "dv_profile_reset", "dv_profile_read", "dv_launch_count", "library_path", "load",
]

PRECISION = {"fp32": 0, "kahan": 1, "mixed": 2, "fp16": 3}
STATUS = {0: "DV_OK", 1: "DV_ERR_INVALID_ARG", 2: "DV_ERR_INVALID_MESH", 3: "DV_ERR_OOM", 4: "DV_ERR_CUDA",
          5: "DV_ERR_TIMEOUT", 6: "DV_ERR_UNSUPPORTED"}


class DvError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))


class _Grid(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_float * 3), ("hi", ctypes.c_float * 3), ("n", ctypes.c_int32 * 3)]


class _Request(ctypes.Structure):
    _fields_ = [("mesh", ctypes.c_void_p), ("grid", _Grid), ("d_out_w", ctypes.c_void_p),
                ("d_out_occ", ctypes.c_void_p), ("d_upstream", ctypes.c_void_p), ("d_dverts", ctypes.c_void_p)]


class _Report(ctypes.Structure):
    _fields_ = [("n_queries", ctypes.c_int64), ("n_faces", ctypes.c_int64), ("n_flagged", ctypes.c_int64),
                ("n_occ_changed", ctypes.c_int64), ("max_abs_fp32_vs_fp64", ctypes.c_double)]


@dataclass(frozen=True)
class Grid:
    """Cell-centred voxel grid over [lo, hi]^3 (per axis), x fastest."""
    n: tuple
    lo: tuple = (-1.0, -1.0, -1.0)
    hi: tuple = (1.0, 1.0, 1.0)

    @staticmethod
    def cube(n: int, lo: float = -1.0, hi: float = 1.0) -> "Grid":
        return Grid((n, n, n), (lo, lo, lo), (hi, hi, hi))

    @property
    def num_queries(self) -> int:
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])

    @property
    def shape_zyx(self):
        return (int(self.n[2]), int(self.n[1]), int(self.n[0]))

    def _c(self) -> _Grid:
        g = _Grid()
        for k in range(3):
            g.lo[k] = float(self.lo[k])
            g.hi[k] = float(self.hi[k])
            g.n[k] = int(self.n[k])
        return g


_lib = None
_P = ctypes.c_void_p
_I64 = ctypes.c_int64


def library_path():
    """libdv.so, or its bounds-checked debug build libdv_debug.so when DV_DEBUG=1 is set."""
    import os

    return _build.LIB_DEBUG if os.environ.get("DV_DEBUG") == "1" else _build.LIB


def load():
    """Load libdv.so (built in-tree by ``paper_2407_11272_b300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not path.exists():
        flag = " --debug" if path == _build.LIB_DEBUG else ""
        raise DvError(4, "load", f"{path} is missing; run `python -m paper_2407_11272_b300.build{flag}`")
    import torch  # noqa: F401  (loads the CUDA runtime the library links against)

    lib = ctypes.CDLL(str(path))
    lib.dv_abi_version.restype = ctypes.c_int
    lib.dv_status_string.restype = ctypes.c_char_p
    lib.dv_status_string.argtypes = [ctypes.c_int]
    lib.dv_last_error.restype = ctypes.c_char_p
    lib.dv_mesh_create.argtypes = [_P, _I64, _P, _I64, _P, ctypes.POINTER(_P)]
    lib.dv_mesh_update_verts.argtypes = [_P, _P, _P]
    lib.dv_mesh_reserve.argtypes = [_P, ctypes.POINTER(_Grid), _I64]
    lib.dv_mesh_num_verts.argtypes = [_P]
    lib.dv_mesh_num_verts.restype = _I64
    lib.dv_mesh_num_faces.argtypes = [_P]
    lib.dv_mesh_num_faces.restype = _I64
    lib.dv_mesh_check.argtypes = [_P, _P]
    lib.dv_mesh_destroy.argtypes = [_P]
    lib.dv_mesh_destroy.restype = None
    lib.dv_winding.argtypes = [_P, _P, _I64, ctypes.POINTER(_Grid), _P, ctypes.c_int, _P]
    lib.dv_voxelize_grid.argtypes = [_P, ctypes.POINTER(_Grid), _P, _P, ctypes.c_int, ctypes.POINTER(_Report), _P]
    lib.dv_winding_backward.argtypes = [_P, _P, _I64, ctypes.POINTER(_Grid), _P, _P, _P]
    lib.dv_winding_backward_boundary.argtypes = [_P, _P, _I64, ctypes.POINTER(_Grid), _P, _P, _P]
    lib.dv_winding_backward_boundary.restype = ctypes.c_int
    lib.dv_mesh_num_boundary_edges.argtypes = [_P]
    lib.dv_mesh_num_boundary_edges.restype = _I64
    lib.dv_mesh_num_strip_events.argtypes = [_P]
    lib.dv_mesh_num_strip_events.restype = _I64
    lib.dv_run_batch.argtypes = [ctypes.POINTER(_Request), ctypes.c_int, ctypes.c_int, _P]
    lib.dv_run_batch.restype = ctypes.c_int
    lib.dv_dipole_winding.argtypes = [_P, _P, _I64, ctypes.POINTER(_Grid), _P, _P]
    lib.dv_dipole_winding.restype = ctypes.c_int
    lib.dv_dipole_backward.argtypes = [_P, _P, _I64, ctypes.POINTER(_Grid), _P, _P, _P]
    lib.dv_dipole_backward.restype = ctypes.c_int
    lib.dv_flipped_duplication.argtypes = [_P, _P, ctypes.c_float, _P, _P, _P]
    lib.dv_flipped_duplication.restype = ctypes.c_int
    lib.dv_debug_report.argtypes = [ctypes.POINTER(_I64), ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(_I64),
                                    ctypes.POINTER(_I64), ctypes.c_int]
    lib.dv_debug_report.restype = ctypes.c_int
    lib.dv_selftest_bounded_wait.argtypes = [_I64, ctypes.c_int, _P]
    lib.dv_selftest_bounded_wait.restype = ctypes.c_int
    lib.dv_selftest_forward_timeout.argtypes = [_P, ctypes.POINTER(_Grid), _P, _I64, _I64, _P]
    lib.dv_selftest_forward_timeout.restype = ctypes.c_int
    lib.dv_build_strips.argtypes = [_P, _I64, _I64, _P, _P, _I64, ctypes.POINTER(_I64)]
    lib.dv_build_strips.restype = ctypes.c_int
    lib.dv_build_face_pairs.argtypes = [_P, _I64, _I64, _P, _P, _I64, _I64, ctypes.POINTER(_I64),
                                        ctypes.POINTER(_I64)]
    lib.dv_build_face_pairs.restype = ctypes.c_int
    lib.dv_profile_enable.argtypes = [ctypes.c_int]
    lib.dv_profile_enable.restype = None
    lib.dv_profile_reset.restype = None
    lib.dv_profile_read.argtypes = [ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(_I64), ctypes.c_int]
    lib.dv_profile_read.restype = ctypes.c_int
    lib.dv_launch_count.restype = _I64
    for name in ("dv_mesh_create", "dv_mesh_update_verts", "dv_mesh_reserve", "dv_mesh_check", "dv_winding",
                 "dv_voxelize_grid", "dv_winding_backward"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != 0:
        raise DvError(status, where, load().dv_last_error().decode(errors="replace"))


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _tensor(t, dtype, shape_tail, name):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if shape_tail is not None and tuple(t.shape[-len(shape_tail):]) != tuple(shape_tail):
        raise ValueError(f"{name} must have trailing shape {shape_tail}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def dv_abi_version() -> int:
    return int(load().dv_abi_version())


class Mesh:
    """Resident mesh handle (``dv_mesh``): packed faces, adjacency and scratch on the GPU."""

    def __init__(self, handle: int, device):
        self._h = ctypes.c_void_p(handle)
        self.device = device

    @property
    def handle(self):
        return self._h

    @property
    def num_verts(self) -> int:
        return int(load().dv_mesh_num_verts(self._h))

    @property
    def num_faces(self) -> int:
        return int(load().dv_mesh_num_faces(self._h))

    def close(self):
        if self._h:
            load().dv_mesh_destroy(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 (interpreter shutdown)
            pass


def dv_mesh_create(verts, faces, stream=None) -> Mesh:
    import torch

    verts = _tensor(verts, torch.float32, (3,), "verts")
    faces = _tensor(faces, torch.int32, (3,), "faces")
    out = ctypes.c_void_p()
    _check(load().dv_mesh_create(ctypes.c_void_p(verts.data_ptr()), verts.shape[0],
                                 ctypes.c_void_p(faces.data_ptr()), faces.shape[0], _stream(stream),
                                 ctypes.byref(out)), "dv_mesh_create")
    return Mesh(out.value, verts.device)


def dv_mesh_update_verts(mesh: Mesh, verts, stream=None) -> None:
    import torch

    verts = _tensor(verts, torch.float32, (3,), "verts")
    if verts.shape[0] != mesh.num_verts:
        raise ValueError("vertex count differs from the mesh")
    _check(load().dv_mesh_update_verts(mesh.handle, ctypes.c_void_p(verts.data_ptr()), _stream(stream)),
           "dv_mesh_update_verts")


def dv_mesh_reserve(mesh: Mesh, grid: Grid | None = None, max_list_queries: int = 0) -> None:
    g = grid._c() if grid is not None else None
    _check(load().dv_mesh_reserve(mesh.handle, ctypes.byref(g) if g is not None else None, int(max_list_queries)),
           "dv_mesh_reserve")


def dv_mesh_check(mesh: Mesh, stream=None) -> None:
    _check(load().dv_mesh_check(mesh.handle, _stream(stream)), "dv_mesh_check")


def _queries_or_grid(queries, grid):
    import torch

    if (queries is None) == (grid is None):
        raise ValueError("pass exactly one of queries or grid")
    if queries is not None:
        q = _tensor(queries, torch.float32, (3,), "queries")
        return ctypes.c_void_p(q.data_ptr()), q.shape[0], None, q.shape[0], q.device
    g = grid._c()
    return None, 0, g, grid.num_queries, None


def dv_winding(mesh: Mesh, queries=None, grid: Grid | None = None, out=None, precision: str = "mixed",
               stream=None):
    """w(q) for a query list [nq,3] or the voxel centres of ``grid`` (flat, x fastest)."""
    import torch

    qp, nq_arg, g, nq, _ = _queries_or_grid(queries, grid)
    if out is None:
        out = torch.empty(nq, dtype=torch.float32, device=mesh.device)
    out = _tensor(out, torch.float32, None, "out")
    if out.numel() != nq:
        raise ValueError("out has the wrong size")
    _check(load().dv_winding(mesh.handle, qp, nq_arg, ctypes.byref(g) if g is not None else None,
                             ctypes.c_void_p(out.data_ptr()), PRECISION[precision], _stream(stream)), "dv_winding")
    return out


def dv_voxelize_grid(mesh: Mesh, grid: Grid, out_w=None, out_occ=None, precision: str = "mixed",
                     report: bool = False, want_w: bool = True, stream=None):
    """Occupancy (uint8, w > 0.5) and w over ``grid``; returns (w or None, occ, report dict or None)."""
    import torch

    nq = grid.num_queries
    if out_w is None and want_w:
        out_w = torch.empty(nq, dtype=torch.float32, device=mesh.device)
    if out_occ is None:
        out_occ = torch.empty(nq, dtype=torch.uint8, device=mesh.device)
    _tensor(out_occ, torch.uint8, None, "out_occ")
    if out_w is not None:
        _tensor(out_w, torch.float32, None, "out_w")
    g = grid._c()
    rep = _Report() if report else None
    _check(load().dv_voxelize_grid(mesh.handle, ctypes.byref(g),
                                   ctypes.c_void_p(out_w.data_ptr()) if out_w is not None else None,
                                   ctypes.c_void_p(out_occ.data_ptr()), PRECISION[precision],
                                   ctypes.byref(rep) if rep is not None else None, _stream(stream)),
           "dv_voxelize_grid")
    rd = None
    if rep is not None:
        rd = {k: getattr(rep, k) for k, _ in _Report._fields_}
    return out_w, out_occ, rd


def dv_winding_backward(mesh: Mesh, upstream, queries=None, grid: Grid | None = None, out=None, stream=None):
    """dL/dV [nv,3] = sum_q upstream[q] dw(q)/dV."""
    import torch

    qp, nq_arg, g, nq, _ = _queries_or_grid(queries, grid)
    up = _tensor(upstream, torch.float32, None, "upstream")
    if up.numel() != nq:
        raise ValueError("upstream must have one value per query")
    if out is None:
        out = torch.empty((mesh.num_verts, 3), dtype=torch.float32, device=mesh.device)
    out = _tensor(out, torch.float32, (3,), "out")
    _check(load().dv_winding_backward(mesh.handle, qp, nq_arg, ctypes.byref(g) if g is not None else None,
                                      ctypes.c_void_p(up.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                      _stream(stream)), "dv_winding_backward")
    return out


def dv_winding_backward_boundary(mesh: Mesh, upstream, queries=None, grid: Grid | None = None, out=None,
                                 stream=None):
    """The same dL/dV as ``dv_winding_backward``, evaluated from the mesh's boundary edges."""
    import torch

    qp, nq_arg, g, nq, _ = _queries_or_grid(queries, grid)
    up = _tensor(upstream, torch.float32, None, "upstream")
    if up.numel() != nq:
        raise ValueError("upstream must have one value per query")
    if out is None:
        out = torch.empty((mesh.num_verts, 3), dtype=torch.float32, device=mesh.device)
    out = _tensor(out, torch.float32, (3,), "out")
    _check(load().dv_winding_backward_boundary(mesh.handle, qp, nq_arg, ctypes.byref(g) if g is not None else None,
                                               ctypes.c_void_p(up.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                               _stream(stream)), "dv_winding_backward_boundary")
    return out


def dv_mesh_num_strip_events(mesh: Mesh) -> int:
    """Number of strip events of the mesh's face visiting order."""
    return int(load().dv_mesh_num_strip_events(mesh.handle))


def dv_mesh_num_boundary_edges(mesh: Mesh) -> int:
    return int(load().dv_mesh_num_boundary_edges(mesh.handle))


def dv_run_batch(requests, precision: str = "mixed", stream=None) -> None:
    """Launch independent requests as one CUDA graph (one branch per request) on ``stream``.

    ``requests``: iterable of dicts with keys mesh (Mesh), grid (Grid), occ (uint8 CUDA tensor),
    and optionally w (float32), upstream (float32) and dverts (float32 [nv,3]). Returns at once."""
    import torch

    reqs = list(requests)
    arr = (_Request * max(1, len(reqs)))()
    for i, r in enumerate(reqs):
        mesh, grid = r["mesh"], r["grid"]
        arr[i].mesh = mesh.handle
        arr[i].grid = grid._c()
        occ = _tensor(r["occ"], torch.uint8, None, "occ")
        if occ.numel() != grid.num_queries:
            raise ValueError("occ has the wrong size")
        arr[i].d_out_occ = occ.data_ptr()
        w = r.get("w")
        arr[i].d_out_w = _tensor(w, torch.float32, None, "w").data_ptr() if w is not None else None
        up = r.get("upstream")
        if up is not None:
            _tensor(up, torch.float32, None, "upstream")
            dV = _tensor(r["dverts"], torch.float32, (3,), "dverts")
            arr[i].d_upstream = up.data_ptr()
            arr[i].d_dverts = dV.data_ptr()
    _check(load().dv_run_batch(arr, len(reqs), PRECISION[precision], _stream(stream)), "dv_run_batch")


def dv_dipole_winding(mesh: Mesh, queries=None, grid: Grid | None = None, out=None, stream=None):
    """Eq. (4) dipole approximation of w for a query list or the voxel centres of ``grid``."""
    import torch

    qp, nq_arg, g, nq, _ = _queries_or_grid(queries, grid)
    if out is None:
        out = torch.empty(nq, dtype=torch.float32, device=mesh.device)
    out = _tensor(out, torch.float32, None, "out")
    _check(load().dv_dipole_winding(mesh.handle, qp, nq_arg, ctypes.byref(g) if g is not None else None,
                                    ctypes.c_void_p(out.data_ptr()), _stream(stream)), "dv_dipole_winding")
    return out


def dv_dipole_backward(mesh: Mesh, upstream, queries=None, grid: Grid | None = None, out=None, stream=None):
    """dL/dV [nv,3] = sum_q upstream[q] dW_dip(q)/dV."""
    import torch

    qp, nq_arg, g, nq, _ = _queries_or_grid(queries, grid)
    up = _tensor(upstream, torch.float32, None, "upstream")
    if up.numel() != nq:
        raise ValueError("upstream must have one value per query")
    if out is None:
        out = torch.empty((mesh.num_verts, 3), dtype=torch.float32, device=mesh.device)
    out = _tensor(out, torch.float32, (3,), "out")
    _check(load().dv_dipole_backward(mesh.handle, qp, nq_arg, ctypes.byref(g) if g is not None else None,
                                     ctypes.c_void_p(up.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                     _stream(stream)), "dv_dipole_backward")
    return out


def dv_selftest_bounded_wait(limit_us: int, arrive: bool, stream=None) -> int:
    """Status code of one bounded wait on the GPU (0 = DV_OK, 5 = DV_ERR_TIMEOUT); no exception."""
    return int(load().dv_selftest_bounded_wait(int(limit_us), 1 if arrive else 0, _stream(stream)))


def dv_debug_report(clear: bool = False):
    """Bounds-check report of the debug build: dict(count, site, index, bound) of the accesses it
    rejected since the last clear; None with the release library (which has no checks)."""
    c, site, idx, bound = _I64(0), ctypes.c_int32(0), _I64(0), _I64(0)
    st = load().dv_debug_report(ctypes.byref(c), ctypes.byref(site), ctypes.byref(idx), ctypes.byref(bound),
                                1 if clear else 0)
    if st == 6:  # DV_ERR_UNSUPPORTED: release build
        return None
    _check(st, "dv_debug_report")
    return {"count": c.value, "site": site.value, "index": idx.value, "bound": bound.value}


def dv_selftest_forward_timeout(mesh: Mesh, grid: Grid, out, skip_tile: int, limit_us: int, stream=None) -> int:
    """Status code of the grid forward run with tile `skip_tile` of every CTA never issued and
    every wait limited to limit_us (0 = DV_OK, 5 = DV_ERR_TIMEOUT); no exception."""
    import torch

    out = _tensor(out, torch.float32, None, "out")
    if out.numel() != grid.num_queries:
        raise ValueError("out must have one value per grid cell")
    g = grid._c()
    return int(load().dv_selftest_forward_timeout(mesh.handle, ctypes.byref(g), ctypes.c_void_p(out.data_ptr()),
                                                  int(skip_tile), int(limit_us), _stream(stream)))


def dv_build_strips(faces, nv: int):
    """Strip order of the faces (host call, no GPU): returns (ev_vert, ev_face) int32 numpy arrays."""
    import numpy as np

    f = np.ascontiguousarray(faces, dtype=np.int32)
    nf = f.shape[0]
    lib = load()
    n = _I64(0)
    ptr = ctypes.c_void_p(f.ctypes.data)
    _check(lib.dv_build_strips(ptr, nf, int(nv), None, None, 0, ctypes.byref(n)), "dv_build_strips")
    ev_vert = np.empty(n.value, dtype=np.int32)
    ev_face = np.empty(n.value, dtype=np.int32)
    _check(lib.dv_build_strips(ptr, nf, int(nv), ctypes.c_void_p(ev_vert.ctypes.data),
                               ctypes.c_void_p(ev_face.ctypes.data), n.value, ctypes.byref(n)), "dv_build_strips")
    return ev_vert, ev_face


def dv_build_face_pairs(faces, nv: int):
    """Edge-sharing face pairs of the adjoint (host call, no GPU): returns (pairs [n, 8],
    singles [m]) int32 numpy arrays; see dv_build_face_pairs in dv_api.h for the record layout."""
    import numpy as np

    f = np.ascontiguousarray(faces, dtype=np.int32)
    nf = f.shape[0]
    lib = load()
    n_p, n_s = _I64(0), _I64(0)
    ptr = ctypes.c_void_p(f.ctypes.data)
    _check(lib.dv_build_face_pairs(ptr, nf, int(nv), None, None, 0, 0, ctypes.byref(n_p), ctypes.byref(n_s)),
           "dv_build_face_pairs")
    pairs = np.empty((n_p.value, 8), dtype=np.int32)
    singles = np.empty(n_s.value, dtype=np.int32)
    _check(lib.dv_build_face_pairs(ptr, nf, int(nv), ctypes.c_void_p(pairs.ctypes.data),
                                   ctypes.c_void_p(singles.ctypes.data), n_p.value, n_s.value, ctypes.byref(n_p),
                                   ctypes.byref(n_s)), "dv_build_face_pairs")
    return pairs, singles


def dv_flipped_duplication(mesh: Mesh, verts, eps: float = 0.01, stream=None):
    """Algorithm 2: (V u V', F u F') as new CUDA tensors [2nv,3] float32 and [2nf,3] int32."""
    import torch

    verts = _tensor(verts, torch.float32, (3,), "verts")
    if verts.shape[0] != mesh.num_verts:
        raise ValueError("vertex count differs from the mesh")
    ov = torch.empty((2 * mesh.num_verts, 3), dtype=torch.float32, device=verts.device)
    of = torch.empty((2 * mesh.num_faces, 3), dtype=torch.int32, device=verts.device)
    _check(load().dv_flipped_duplication(mesh.handle, ctypes.c_void_p(verts.data_ptr()), float(eps),
                                         ctypes.c_void_p(ov.data_ptr()), ctypes.c_void_p(of.data_ptr()),
                                         _stream(stream)), "dv_flipped_duplication")
    return ov, of


def dv_profile_enable(on: bool = True) -> None:
    load().dv_profile_enable(1 if on else 0)


def dv_profile_reset() -> None:
    load().dv_profile_reset()


def dv_profile_read() -> dict:
    """{kernel name: (total ms, launches)} for the library's launches since the last reset."""
    lib = load()
    cap = 64
    names = (ctypes.c_char_p * cap)()
    ms = (ctypes.c_double * cap)()
    cnt = (_I64 * cap)()
    n = lib.dv_profile_read(names, ms, cnt, cap)
    return {names[i].decode(): (ms[i], int(cnt[i])) for i in range(min(n, cap))}


def dv_launch_count() -> int:
    return int(load().dv_launch_count())
