"""Planted mistakes in the oracle must fail its pins.

Each case copies ``oracle/oracle.c`` to a temporary directory, plants one
plausible slip by text replacement, compiles it, and checks that at least
one closed-form pin rejects the mutant. The real oracle is never modified.
"""
import ctypes
import math
import subprocess

import numpy as np
import pytest

from paper_2407_11272_b300 import meshgen

SRC = __import__("pathlib").Path(__file__).resolve().parents[1] / "oracle" / "oracle.c"

MUTANTS = {
    "beta_drops_term": ("dot3(e[1], e[2]) + dot3(e[2], e[0]);\n    return", "dot3(e[1], e[2]);\n    return"),
    "alpha_sign": ("double alpha = dot3(e[0], c12);                                   /* det",
                   "double alpha = -dot3(e[0], c12);                                   /* det"),
    "atan2_strict_y": ("if (x < 0 && y >= 0)", "if (x < 0 && y > 0)"),
    "atan2_minus_pi": ("return atan(y / x) - ORC_PI;", "return atan(y / x) + ORC_PI;"),
    "no_factor_two": ("return 2.0 * half_solid_angle(v0, v1, v2, q);", "return half_solid_angle(v0, v1, v2, q);"),
    "winding_norm": ("w_out[i] = s / (2.0 * ORC_PI);", "w_out[i] = s / (4.0 * ORC_PI);"),
    "wrong_vertex_index": ("vtx(V, F, f, 1), vtx(V, F, f, 2), Q + 3 * i);\n        w_out",
                           "vtx(V, F, f, 2), vtx(V, F, f, 1), Q + 3 * i);\n        w_out"),
    "grad_db_sign": ("db = -2.0 * alpha / den", "db = 2.0 * alpha / den"),
    "grad_projection": ("(t[k] - e[j][k] * et)", "(t[k] + e[j][k] * et)"),
    "grad_len": ("/ len[j];\n    }\n}", "/ (len[j] * len[j]);\n    }\n}"),
    "grid_corner": ("((double)ix + 0.5)", "((double)ix)"),
    "grid_points_index": ("(c / n[0]) % n[1], c / ((int64_t)n[0] * n[1])", "(c / n[0]) % n[1], c / n[1]"),
    # Eq. (4): the dipole evaluated at a vertex instead of the face centre, an unnormalized face
    # normal (2 x area), and the field's denominator |r - q|^2 instead of |r - q|^3
    "dipole_centroid_to_v0": ("x[k] = (a[k] + b[k] + c[k]) / 3.0 - Q[3 * i + k];", "x[k] = a[k] - Q[3 * i + k];"),
    "dipole_unnormalized_normal": ("double nrm[3] = {m[0] / (2 * area), m[1] / (2 * area), m[2] / (2 * area)};",
                                   "double nrm[3] = {m[0], m[1], m[2]};"),
    "dipole_r_squared": ("/ (r * r * r) * area", "/ (r * r) * area"),
    # ray crossings of a closed mesh: the crossing's sign from the wrong normal component's sign
    "ray_sign": ("cr[slot].sign = d > 0 ? 1 : -1;", "cr[slot].sign = d < 0 ? 1 : -1;"),
    "ray_beyond_side": ("while (k > 0 && c[k - 1].x > x)", "while (k > 0 && c[k - 1].x < x)"),
}

_d = ctypes.POINTER(ctypes.c_double)


def _build(tmp_path, name, old, new):
    src = SRC.read_text()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    p = tmp_path / f"{name}.c"
    p.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", str(p), "-o", str(so), "-lm"],
                   check=True)
    lib = ctypes.CDLL(str(so))
    lib.orc_solid_angle.restype = ctypes.c_double
    lib.orc_solid_angle.argtypes = [_d] * 4
    return lib


def _winding(lib, V, F, Q):
    V = np.ascontiguousarray(V, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.int32)
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    out = np.empty(len(Q))
    lib.orc_winding(V.ctypes.data_as(_d), ctypes.c_int64(len(V)), F.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                    ctypes.c_int64(len(F)), Q.ctypes.data_as(_d), ctypes.c_int64(len(Q)), out.ctypes.data_as(_d),
                    ctypes.c_int(1))
    return out


def _grad(lib, V, F, Q, g):
    V = np.ascontiguousarray(V, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.int32)
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    out = np.zeros((len(V), 3))
    lib.orc_winding_grad(V.ctypes.data_as(_d), ctypes.c_int64(len(V)),
                         F.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.c_int64(len(F)),
                         Q.ctypes.data_as(_d), ctypes.c_int64(len(Q)), g.ctypes.data_as(_d), out.ctypes.data_as(_d),
                         ctypes.c_int(1))
    return out


def _dipole(lib, V, F, Q):
    V = np.ascontiguousarray(V, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.int32)
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    out = np.empty(len(Q))
    lib.orc_dipole_winding(V.ctypes.data_as(_d), ctypes.c_int64(len(V)),
                           F.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.c_int64(len(F)),
                           Q.ctypes.data_as(_d), ctypes.c_int64(len(Q)), out.ctypes.data_as(_d), ctypes.c_int(1))
    return out


def _ray(lib, V, F, lo, hi, n):
    V = np.ascontiguousarray(V, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.int32)
    lo, hi = np.asarray(lo, np.float32), np.asarray(hi, np.float32)
    nn = np.asarray(n, np.int32)
    w = np.empty(int(np.prod(nn)), np.int32)
    amb = np.empty(int(np.prod(nn)), np.uint8)
    lib.orc_ray_winding_grid(V.ctypes.data_as(_d), ctypes.c_int64(len(V)), F.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                             ctypes.c_int64(len(F)), lo.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                             hi.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                             nn.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.c_double(1e-12),
                             ctypes.c_double(1e-9), w.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                             amb.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), ctypes.c_int(1))
    return w, amb.astype(bool)


def _grid(lib, n):
    lo = np.full(3, -1, np.float32)
    hi = np.full(3, 1, np.float32)
    nn = np.full(3, n, np.int32)
    out = np.empty((n ** 3, 3))
    lib.orc_grid_queries(lo.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                         hi.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                         nn.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), out.ctypes.data_as(_d))
    return out


def _pins_pass(lib) -> bool:
    """A condensed copy of the closed-form pins (octant, tetra, conventions, FD, grid)."""
    ok = True
    v = [np.ascontiguousarray(x, dtype=np.float64) for x in ([1, 0, 0], [0, 1, 0], [0, 0, 1], [0, 0, 0])]
    ok &= abs(lib.orc_solid_angle(*[x.ctypes.data_as(_d) for x in v]) - math.pi / 2) < 1e-12
    V, F = meshgen.regular_tetrahedron(0.5)
    V64 = V.astype(np.float64)
    c0 = V64[F[0]].mean(axis=0)
    n0 = np.cross(V64[F[0, 1]] - V64[F[0, 0]], V64[F[0, 2]] - V64[F[0, 0]])
    n0 /= np.linalg.norm(n0)
    # centre, far outside, inside, and just outside / just inside face 0 (large |Omega| of both signs)
    Q = np.array([[0.0, 0, 0], [0.9, 0.9, 0.9], [0.05, -0.1, 0.02], c0 + 0.01 * n0, c0 - 0.01 * n0])
    ok &= np.allclose(_winding(lib, V, F, Q), [1, 0, 1, 0, 1], atol=1e-12)
    Vc = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)
    Fc = meshgen._orient_outward(Vc, np.array([[0, 1, 2], [0, 1, 3], [0, 2, 3], [1, 2, 3]]), Vc.mean(axis=0))
    ok &= abs(_winding(lib, Vc, Fc, np.array([[0.25, 0.25, 0.0]]))[0] - 1.0) < 1e-12
    # gradient against brute-force central differences of the same library
    Vp = np.array([[0, 0, 0], [1, 0, 0.1], [0, 1, -0.1], [1, 1, 0.3]], dtype=np.float64) * 0.6
    Fp = np.array([[0, 1, 2], [1, 3, 2]], dtype=np.int32)
    rng = np.random.default_rng(3)
    Qp = rng.uniform(-1, 1, size=(12, 3))
    g = rng.normal(size=12)
    G = _grad(lib, Vp, Fp, Qp, g)
    h = 1e-6
    fd = np.zeros_like(Vp)
    for i in range(len(Vp)):
        for k in range(3):
            a, b = Vp.copy(), Vp.copy()
            a[i, k] += h
            b[i, k] -= h
            fd[i, k] = (g @ _winding(lib, a, Fp, Qp) - g @ _winding(lib, b, Fp, Qp)) / (2 * h)
    ok &= np.allclose(G, fd, rtol=1e-5, atol=1e-7)
    # Eq. (4) on one face: q at distance d behind the centroid along the unit normal gives
    # area / (4 pi d^2), and shifted by t inside the plane area d / (4 pi (d^2 + t^2)^1.5)
    Vt = np.array([[0.1, -0.2, 0.05], [0.8, -0.2, 0.05], [0.1, 0.71, 0.05]])
    area, d, t = 0.5 * 0.7 * 0.91, 0.37, 0.23
    ct = Vt.mean(axis=0)
    Qt = np.array([ct - [0, 0, d], ct - [0, 0, d] + [t, 0, 0]])
    ok &= np.allclose(_dipole(lib, Vt, np.array([[0, 1, 2]]), Qt),
                      [area / (4 * math.pi * d * d), area * d / (4 * math.pi * (d * d + t * t) ** 1.5)],
                      rtol=1e-12, atol=0)
    # closed convex mesh by ray crossings: 1 inside, 0 outside (the cube's plane-side indicator)
    Vq, Fq = meshgen.cube(0.45, centre=(0.02, 0.01, -0.03))
    wq, uq = _ray(lib, Vq, Fq, (-1, -1, -1), (1, 1, 1), (9, 8, 7))
    Qq = _grid_any(lib, (9, 8, 7))
    inq = np.all(np.abs(Qq - np.array([0.02, 0.01, -0.03])) < 0.45, axis=1)
    ok &= bool(np.array_equal(wq[~uq], inq[~uq].astype(np.int32))) and not uq.any()  # generic: all decided
    ok &= np.allclose(_grid(lib, 4)[0], [-0.75, -0.75, -0.75])
    ok &= np.allclose(_grid_points(lib, (4, 2, 8), [4 * 2 * 8 - 1]), [[0.75, 0.5, 0.875]])
    return bool(ok)


def _grid_any(lib, n):
    lo = np.full(3, -1, np.float32)
    hi = np.full(3, 1, np.float32)
    nn = np.asarray(n, np.int32)
    out = np.empty((int(np.prod(nn)), 3))
    lib.orc_grid_queries(lo.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                         hi.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                         nn.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), out.ctypes.data_as(_d))
    return out


def _grid_points(lib, n, cells):
    lo = np.full(3, -1, np.float32)
    hi = np.full(3, 1, np.float32)
    nn = np.asarray(n, np.int32)
    c = np.asarray(cells, np.int64)
    out = np.empty((len(c), 3))
    lib.orc_grid_points(lo.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                        hi.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                        nn.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                        c.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ctypes.c_int64(len(c)),
                        out.ctypes.data_as(_d))
    return out


def test_unmutated_oracle_passes_condensed_pins(tmp_path):
    lib = _build(tmp_path, "identity", "#define ORC_PI", "#define ORC_PI")
    assert _pins_pass(lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_rejected(tmp_path, name):
    old, new = MUTANTS[name]
    assert not _pins_pass(_build(tmp_path, name, old, new)), f"mutant {name} survived the pins"
