"""Fit the minimax polynomial used by the kernels' arctangent fast path.

The forward kernel evaluates ATAN2(N, D) for the common case |N| < D/4
(a face seen under a solid angle below about 0.49 sr). It stores the face
normal pre-multiplied by 4, so it holds v = 4N/D in [-1, 1] and needs

    atan(v / 4) ~= v * P(v^2),   P of degree ``DEG`` in s = v^2,

with a small *relative* error, so that the error of a sum over faces stays
proportional to the sum of |terms| (the faces far from a query have tiny
solid angles). ``P`` is fitted here by the Remez exchange algorithm
(E. Remez, 1934) on s in [0, 1] with weight 1/g(s), g(s) = atan(sqrt(s)/4)/sqrt(s),
in float64 with numpy, then rounded to float32 and checked by evaluating the
float32 Horner scheme exactly as the kernel does.

Run ``python gen_atan_poly.py`` to regenerate ``atan_poly.h``.
"""
from __future__ import annotations

import math
from pathlib import Path

import numpy as np

T = 0.25
DEG = 3


def g(s):
    s = np.asarray(s, dtype=np.float64)
    r = np.sqrt(s)
    out = np.empty_like(s)
    small = r < 1e-8
    out[small] = T
    out[~small] = np.arctan(T * r[~small]) / r[~small]
    return out


def remez(deg: int, iters: int = 60):
    n = deg + 2
    # Chebyshev extrema as the first reference
    x = 0.5 - 0.5 * np.cos(np.pi * np.arange(n) / (n - 1))
    grid = np.linspace(0.0, 1.0, 200001)
    coef = None
    for _ in range(iters):
        A = np.zeros((n, n))
        for i in range(n):
            A[i, : deg + 1] = x[i] ** np.arange(deg + 1)
            A[i, deg + 1] = (-1) ** i * g(x[i : i + 1])[0]
        sol = np.linalg.solve(A, g(x))
        coef = sol[: deg + 1]
        err = (np.polyval(coef[::-1], grid) - g(grid)) / g(grid)
        # new reference: one extremum per sign-alternating segment
        sgn = np.sign(err)
        idx, start = [], 0
        for k in range(1, len(grid) + 1):
            if k == len(grid) or sgn[k] != sgn[start]:
                seg = slice(start, k)
                idx.append(start + int(np.argmax(np.abs(err[seg]))))
                start = k
        if len(idx) < n:
            break
        # keep the n largest consecutive alternating extrema
        while len(idx) > n:
            e = np.abs(err[idx])
            if e[0] < e[-1]:
                idx.pop(0)
            else:
                idx.pop()
        x = grid[idx]
    return coef


def eval_f32(coef32, v):
    """Horner in float32 exactly as the kernel: P = c_n; P = fma(P, s, c_k); out = v * P."""
    v = np.asarray(v, dtype=np.float32)
    s = (v * v).astype(np.float32)
    p = np.full_like(v, coef32[-1])
    for c in coef32[-2::-1]:
        p = (p.astype(np.float64) * s + np.float64(c)).astype(np.float32)  # fma: one rounding
    return (v * p).astype(np.float32)


def main():
    coef = remez(DEG)
    c32 = np.asarray(coef, dtype=np.float32)
    v = np.linspace(-1.0, 1.0, 2000001)[1:-1]
    v = v[v != 0]
    ref = np.arctan(T * v.astype(np.float64))
    rel = np.abs(eval_f32(c32, v).astype(np.float64) - ref) / np.abs(ref)
    lines = [
        "// Generated by gen_atan_poly.py (Remez minimax fit, relative error). Do not edit.",
        f"// atan(v * {T}) ~= v * P(v*v) for |v| <= 1, P of degree {DEG};",
        f"// measured max relative error of the float32 evaluation: {rel.max():.3e}",
        "#pragma once",
        f"#define DV_ATAN_FAST_T {T}f",
        f"#define DV_ATAN_FAST_DEG {DEG}",
    ]
    for k, c in enumerate(c32):
        lines.append(f"#define DV_ATAN_C{k} {float(c)!r}f")
    Path(__file__).with_name("atan_poly.h").write_text("\n".join(lines) + "\n")
    print("\n".join(lines))


if __name__ == "__main__":
    main()
