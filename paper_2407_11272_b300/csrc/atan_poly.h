// Generated by gen_atan_poly.py (Remez minimax fit, relative error). Do not edit.
// atan(v * 0.25) ~= v * P(v*v) for |v| <= 1, P of degree 3;
// measured max relative error of the float32 evaluation: 1.576e-07
#pragma once
#define DV_ATAN_FAST_T 0.25f
#define DV_ATAN_FAST_DEG 3
#define DV_ATAN_C0 0.25f
#define DV_ATAN_C1 -0.005208238027989864f
#define DV_ATAN_C2 0.0001948303251992911f
#define DV_ATAN_C3 -7.929056664579548e-06f
