"""Fit the minimax polynomial used by the FP32 kernels' arctangent fast path.

The FP32 forward kernel evaluates ATAN2(N, D) for the common case |N| < D/8
(a face seen under a solid angle below about 0.25 sr). It stores the face
normal pre-multiplied by 8, so it holds v = 8N/D in [-1, 1] and needs

    atan(v / 8) ~= v * P(v^2),   P of degree ``DEG32`` in s = v^2,

with a small *relative* error, so that the error of a sum over faces stays
proportional to the sum of |terms| (the faces far from a query have tiny
solid angles).

P is fitted by the Remez exchange algorithm (E. Remez, 1934) on the reduced
variable in [0, 1] with weight 1/g (relative error), carried out in 50-digit
arithmetic with mpmath; the float32 coefficients are then checked by
evaluating the float32 Horner scheme exactly as the kernel does.

Run ``python gen_atan_poly.py`` to regenerate ``atan_poly.h``.
"""
from __future__ import annotations

from pathlib import Path

import mpmath as mp
import numpy as np

T = 0.125      # fast-path bound on |N/D|
DEG32 = 2

mp.mp.dps = 50


def g_mp(s, scale):
    """atan(scale * sqrt(s)) / sqrt(s), the function P must match (s in [0, 1])."""
    s = mp.mpf(s)
    if s == 0:
        return mp.mpf(scale)
    r = mp.sqrt(s)
    return mp.atan(scale * r) / r


def remez(deg: int, scale: float, iters: int = 30, ngrid: int = 4000):
    """Weighted (relative) minimax polynomial P(s) ~ g(s) on [0, 1]; returns mpf coefficients c0..c_deg."""
    n = deg + 2
    x = [mp.mpf(1) / 2 - mp.cos(mp.pi * k / (n - 1)) / 2 for k in range(n)]
    grid = [mp.mpf(k) / ngrid for k in range(ngrid + 1)]
    gg = [g_mp(t, scale) for t in grid]
    coef = None
    for _ in range(iters):
        A = mp.matrix(n, n)
        b = mp.matrix(n, 1)
        for i in range(n):
            gi = g_mp(x[i], scale)
            for k in range(deg + 1):
                A[i, k] = x[i] ** k
            A[i, deg + 1] = (-1) ** i * gi
            b[i] = gi
        sol = mp.lu_solve(A, b)
        coef = [sol[k] for k in range(deg + 1)]
        err = [(mp.polyval(coef[::-1], t) - gv) / gv for t, gv in zip(grid, gg)]
        # one extremum per run of equal sign
        idx, start = [], 0
        for k in range(1, len(grid) + 1):
            if k == len(grid) or mp.sign(err[k]) != mp.sign(err[start]):
                idx.append(max(range(start, k), key=lambda j: abs(err[j])))
                start = k
        if len(idx) < n:
            break
        while len(idx) > n:
            if abs(err[idx[0]]) < abs(err[idx[-1]]):
                idx.pop(0)
            else:
                idx.pop()
        x = [grid[j] for j in idx]
    return coef


def max_rel_err_mp(coef, scale, npts=4001):
    worst = mp.mpf(0)
    for k in range(npts):
        s = mp.mpf(k) / (npts - 1)
        gv = g_mp(s, scale)
        worst = max(worst, abs((mp.polyval(coef[::-1], s) - gv) / gv))
    return worst


def eval_f32(coef32, v):
    """Horner in float32 exactly as the kernel: P = c_n; P = fma(P, s, c_k); out = v * P."""
    v = np.asarray(v, dtype=np.float32)
    s = (v * v).astype(np.float32)
    p = np.full_like(v, coef32[-1])
    for c in coef32[-2::-1]:
        p = (p.astype(np.float64) * s + np.float64(c)).astype(np.float32)  # fma: one rounding
    return (v * p).astype(np.float32)


def main():
    c32 = remez(DEG32, T)
    c32f = np.asarray([float(c) for c in c32], dtype=np.float32)
    v = np.linspace(-1.0, 1.0, 2000001)[1:-1]
    v = v[v != 0]
    ref = np.arctan(T * v.astype(np.float64))
    rel32 = float((np.abs(eval_f32(c32f, v).astype(np.float64) - ref) / np.abs(ref)).max())
    e32 = max_rel_err_mp(c32, T)
    lines = [
        "// Generated by gen_atan_poly.py (Remez minimax fit, relative error). Do not edit.",
        f"// FP32: atan(v * {T}) ~= v * P(v*v) for |v| <= 1, P of degree {DEG32};",
        f"//       max relative error of the polynomial itself: {float(e32):.3e},",
        f"//       of its float32 evaluation: {rel32:.3e}",
        "#pragma once",
        f"#define DV_ATAN_FAST_T {T}f",
        f"#define DV_ATAN_FAST_DEG {DEG32}",
    ]
    for k, c in enumerate(c32f):
        lines.append(f"#define DV_ATAN_C{k} {float(c)!r}f")
    Path(__file__).with_name("atan_poly.h").write_text("\n".join(lines) + "\n")
    print("\n".join(lines))


if __name__ == "__main__":
    main()
