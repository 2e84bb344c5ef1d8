// Generated by gen_atan_poly.py (Remez minimax fits, relative error). Do not edit.
// FP32: atan(v * 0.125) ~= v * P(v*v) for |v| <= 1, P of degree 2;
//       max relative error of the float32 evaluation: 1.695e-07
// FP64: atan(u) ~= u * Q(u*u) for |u| <= 0.125, Q of degree 6;
//       max relative error of the polynomial itself: 1.756e-18
#pragma once
#define DV_ATAN_FAST_T 0.125f
#define DV_ATAN_FAST_DEG 2
#define DV_ATAN_C0 0.125f
#define DV_ATAN_C1 -0.0006510040839202702f
#define DV_ATAN_C2 6.0027723520761356e-06f
#define DV_ATAN64_FAST_T 0.125
#define DV_ATAN64_DEG 6
#define DV_ATAN64_C0 0.9999999999999999982438001
#define DV_ATAN64_C1 -0.3333333333333223044163845
#define DV_ATAN64_C2 0.1999999999886886655282764
#define DV_ATAN64_C3 -0.1428571385044880033355607
#define DV_ATAN64_C4 0.1111103127639539156827746
#define DV_ATAN64_C5 -0.09083377682733414998057317
#define DV_ATAN64_C6 0.07338265110376805502736929
