// Generated by gen_atan_poly.py (Remez minimax fit, relative error). Do not edit.
// FP32: atan(v * 0.125) ~= v * P(v*v) for |v| <= 1, P of degree 2;
//       max relative error of the polynomial itself: 1.667e-08,
//       of its float32 evaluation: 1.695e-07
#pragma once
#define DV_ATAN_FAST_T 0.125f
#define DV_ATAN_FAST_DEG 2
#define DV_ATAN_C0 0.125f
#define DV_ATAN_C1 -0.0006510040839202702f
#define DV_ATAN_C2 6.0027723520761356e-06f
