// Eq. (4): the naive dipole discretization of the winding number,
//     W_dip(q) = (1/4pi) sum_f <n_f, (c_f - q) / |c_f - q|^3> Delta_f
//              = (1/4pi) sum_f (m_f . r) / (2 |r|^3),   r = c_f - q,  m_f = (v1-v0) x (v2-v0),
// with c_f the face centroid and Delta_f its area (m_f = 2 Delta_f n_f). The paper uses it for
// mesh morphing (§2.4) because it is smooth where the exact winding number is almost binary.
// Its adjoint with respect to the vertices: with G_m = sum_q g r / (2|r|^3) and
// G_r = sum_q g [m / (2|r|^3) - 3 (m.r) r / (2|r|^5)],
//     dL/dv0 = (e1 - e2) x G_m + G_r / 3,  dL/dv1 = e2 x G_m + G_r / 3,  dL/dv2 = -e1 x G_m + G_r / 3
// (e1 = v1 - v0, e2 = v2 - v0), all times 1/(4pi). A query at a centroid contributes 0.
// FP32 terms, plain FP32 sums within a tile of faces (forward) or a window of queries or a grid
// row (adjoint), Kahan across them; the adjoint writes per-face partials for the FP64 vertex
// gather. Grid queries share the (y, z) parts per row and pair x-adjacent queries in packed
// FP32x2 instructions.
#include <math.h>

#include <type_traits>

#include "dv_internal.cuh"

namespace dv {

constexpr int kDipThreads = 256;
constexpr int kDipQ = 4;         // queries per thread (forward)
constexpr int kDipTile = 128;    // faces per shared-memory tile (forward)
constexpr int kDipBwdThreads = 128;
constexpr int kDipWin = 2048;    // queries per staged window (adjoint)
constexpr float kInv4Pi = 0.07957747154594767f;

struct DipFace {
    float4 c;  // centroid, w unused
    float4 m;  // m_f / 2 (= area * unit normal), w unused
};

__device__ __forceinline__ DipFace dip_face(const FaceRec &r) {
    const float s = 0.5f / kNormalScale;  // records hold 8 m_f
    DipFace d;
    d.c = make_float4((r.r0.x + r.r1.x + r.r2.x) * (1.0f / 3.0f), (r.r0.y + r.r1.y + r.r2.y) * (1.0f / 3.0f),
                      (r.r0.z + r.r1.z + r.r2.z) * (1.0f / 3.0f), 0.f);
    d.m = make_float4(r.r0.w * s, r.r1.w * s, r.r2.w * s, 0.f);
    return d;
}

__device__ __forceinline__ void query_point(const GridF &g, const float *queries, int64_t idx, float &x, float &y,
                                            float &z) {
    if (queries) {
        x = queries[3 * idx];
        y = queries[3 * idx + 1];
        z = queries[3 * idx + 2];
    } else {
        const int ix = (int)(idx % g.n[0]);
        const int iy = (int)((idx / g.n[0]) % g.n[1]);
        const int iz = (int)(idx / ((int64_t)g.n[0] * g.n[1]));
        x = __fmaf_rn((float)ix + 0.5f, g.h[0], g.lo[0]);
        y = __fmaf_rn((float)iy + 0.5f, g.h[1], g.lo[1]);
        z = __fmaf_rn((float)iz + 0.5f, g.h[2], g.lo[2]);
    }
}

// Face gradient from the 7 compensated sums S0 = sum g/|r|^3, V1 = sum g r/|r|^3,
// V2 = sum g (m.r) r/|r|^5 (FP64 combination), written as 9 floats (v0, v1, v2).
__device__ void dip_face_grad(const FaceRec &r, const DipFace &d, const float (&s)[7], const float (&c)[7],
                              float *out) {
    double S[7];
    for (int k = 0; k < 7; ++k) S[k] = (double)s[k] - (double)c[k];
    const double kk = 1.0 / (4.0 * 3.14159265358979323846);
    // G_m = sum g dterm/dm_f = V1 / 2;  G_r = sum g dterm/dr = (m_f / 2) S0 - 3 V2
    const double Gm[3] = {0.5 * S[1], 0.5 * S[2], 0.5 * S[3]};
    const double mh[3] = {d.m.x, d.m.y, d.m.z};  // m_f / 2
    const double Gr[3] = {mh[0] * S[0] - 3.0 * S[4], mh[1] * S[0] - 3.0 * S[5], mh[2] * S[0] - 3.0 * S[6]};
    const double e1[3] = {(double)r.r1.x - r.r0.x, (double)r.r1.y - r.r0.y, (double)r.r1.z - r.r0.z};
    const double e2[3] = {(double)r.r2.x - r.r0.x, (double)r.r2.y - r.r0.y, (double)r.r2.z - r.r0.z};
    const double dd[3] = {e1[0] - e2[0], e1[1] - e2[1], e1[2] - e2[2]};
    auto cross = [](const double *a, const double *b, double *o) {
        o[0] = a[1] * b[2] - a[2] * b[1];
        o[1] = a[2] * b[0] - a[0] * b[2];
        o[2] = a[0] * b[1] - a[1] * b[0];
    };
    double c0[3], c1[3], c2[3];
    cross(dd, Gm, c0);
    cross(e2, Gm, c1);
    cross(e1, Gm, c2);
    for (int k = 0; k < 3; ++k) {
        out[k] = (float)(kk * (c0[k] + Gr[k] / 3.0));
        out[3 + k] = (float)(kk * (c1[k] + Gr[k] / 3.0));
        out[6 + k] = (float)(kk * (-c2[k] + Gr[k] / 3.0));
    }
}

__global__ void __launch_bounds__(kDipThreads) dipole_fwd_kernel(const FaceRec *__restrict__ rec, int64_t nf, GridF g,
                                                                 const float *__restrict__ queries, int64_t nq,
                                                                 float *__restrict__ w_out) {
    __shared__ DipFace tile[kDipTile];
    const int64_t base = (int64_t)blockIdx.x * kDipThreads * kDipQ + threadIdx.x;
    float qx[kDipQ], qy[kDipQ], qz[kDipQ], acc[kDipQ], ks[kDipQ], kc[kDipQ];
#pragma unroll
    for (int j = 0; j < kDipQ; ++j) {
        int64_t idx = base + (int64_t)j * kDipThreads;
        if (idx >= nq) idx = nq - 1;
        query_point(g, queries, idx, qx[j], qy[j], qz[j]);
        acc[j] = ks[j] = kc[j] = 0.f;
    }
    for (int64_t f0 = 0; f0 < nf; f0 += kDipTile) {
        const int cnt = (int)(nf - f0 < kDipTile ? nf - f0 : kDipTile);
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += kDipThreads) tile[i] = dip_face(rec[f0 + i]);
        __syncthreads();
        for (int k = 0; k < cnt; ++k) {
            const DipFace d = tile[k];
#pragma unroll
            for (int j = 0; j < kDipQ; ++j) {
                const float rx = d.c.x - qx[j], ry = d.c.y - qy[j], rz = d.c.z - qz[j];
                const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                const float ir = rsqrt_approx(r2);
                const float ir3 = r2 > 0.f ? ir * ir * ir : 0.f;
                const float mr = fmaf(d.m.x, rx, fmaf(d.m.y, ry, d.m.z * rz));
                acc[j] = fmaf(mr, ir3, acc[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < kDipQ; ++j) {  // Kahan across tiles
            const float y = acc[j] - kc[j];
            const float t = ks[j] + y;
            kc[j] = (t - ks[j]) - y;
            ks[j] = t;
            acc[j] = 0.f;
        }
    }
#pragma unroll
    for (int j = 0; j < kDipQ; ++j) {
        const int64_t idx = base + (int64_t)j * kDipThreads;
        if (idx < nq) w_out[idx] = (ks[j] - kc[j]) * kInv4Pi;
    }
}

__global__ void __launch_bounds__(kDipBwdThreads) dipole_bwd_kernel(const FaceRec *__restrict__ rec, int64_t nf,
                                                                    GridF g, const float *__restrict__ queries,
                                                                    int64_t nq, const float *__restrict__ upstream,
                                                                    int64_t per_split, float *__restrict__ face_grad) {
    __shared__ float4 win[kDipWin];  // (x, y, z, g)
    const int64_t f = (int64_t)blockIdx.x * kDipBwdThreads + threadIdx.x;
    const FaceRec r = rec[f < nf ? f : nf - 1];
    const DipFace d = dip_face(r);
    const int64_t q0 = (int64_t)blockIdx.y * per_split;
    const int64_t q1 = q0 + per_split < nq ? q0 + per_split : nq;
    // face sums with Kahan compensation: S0 = sum g/|r|^3, V1 = sum g r/|r|^3, V2 = sum g (m.r) r/|r|^5
    float s[7] = {0, 0, 0, 0, 0, 0, 0}, c[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int64_t w0 = q0; w0 < q1; w0 += kDipWin) {
        const int len = (int)(q1 - w0 < kDipWin ? q1 - w0 : kDipWin);
        __syncthreads();
        for (int i = threadIdx.x; i < len; i += kDipBwdThreads) {
            float x, y, z;
            query_point(g, queries, w0 + i, x, y, z);
            win[i] = make_float4(x, y, z, upstream[w0 + i]);
        }
        __syncthreads();
        float p[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int i = 0; i < len; ++i) {
            const float4 q = win[i];
            const float rx = d.c.x - q.x, ry = d.c.y - q.y, rz = d.c.z - q.z;
            const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
            const float ir = rsqrt_approx(r2);
            const float ir2 = ir * ir;
            const bool at_c = !(r2 > 0.f);  // a query at the centroid contributes 0 (not 0 * inf)
            const float gi3 = at_c ? 0.f : q.w * ir2 * ir;
            const float t = at_c ? 0.f : gi3 * fmaf(d.m.x, rx, fmaf(d.m.y, ry, d.m.z * rz)) * ir2;
            p[0] += gi3;
            p[1] = fmaf(gi3, rx, p[1]);
            p[2] = fmaf(gi3, ry, p[2]);
            p[3] = fmaf(gi3, rz, p[3]);
            p[4] = fmaf(t, rx, p[4]);
            p[5] = fmaf(t, ry, p[5]);
            p[6] = fmaf(t, rz, p[6]);
        }
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            const float y = p[k] - c[k];
            const float tt = s[k] + y;
            c[k] = (tt - s[k]) - y;
            s[k] = tt;
        }
    }
    if (f >= nf) return;
    dip_face_grad(r, d, s, c, face_grad + ((int64_t)blockIdx.y * nf + f) * 9);
}

// ---------------------------------------------------------------------------------------------
// Grid versions. On a grid row (fixed y, z) the y and z parts of r = c_f - q are constant, so per
// pair only rx, |r|^2 = rx^2 + (ry^2 + rz^2) and m.r = m_x rx + (m_y ry + m_z rz) vary; two
// x-adjacent queries go through one packed FP32x2 instruction.
constexpr int kDipGX = 4, kDipGY = 2;  // queries per thread: 4 along x (two pairs) x 2 rows

__global__ void __launch_bounds__(kDipThreads, 2) dipole_fwd_grid_kernel(const FaceRec *__restrict__ rec, int64_t nf,
                                                                         GridF g, float *__restrict__ w_out) {
    __shared__ DipFace tile[kDipTile];
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int tiles_x = (nx + kDipGX - 1) / kDipGX, tiles_y = (ny + kDipGY - 1) / kDipGY;
    const int64_t t = (int64_t)blockIdx.x * kDipThreads + threadIdx.x;
    const int tx = (int)(t % tiles_x);
    const int64_t t2 = t / tiles_x;
    const int ty = (int)(t2 % tiles_y);
    const int64_t zz = t2 / tiles_y;
    const bool valid = zz < nz;
    const int z = valid ? (int)zz : nz - 1;
    float2 nqx[kDipGX / 2];
#pragma unroll
    for (int j = 0; j < kDipGX / 2; ++j)
        nqx[j] = make_float2(-__fmaf_rn((float)(tx * kDipGX + 2 * j) + 0.5f, g.h[0], g.lo[0]),
                             -__fmaf_rn((float)(tx * kDipGX + 2 * j + 1) + 0.5f, g.h[0], g.lo[0]));
    float qy[kDipGY];
#pragma unroll
    for (int i = 0; i < kDipGY; ++i) qy[i] = __fmaf_rn((float)(ty * kDipGY + i) + 0.5f, g.h[1], g.lo[1]);
    const float qz = __fmaf_rn((float)z + 0.5f, g.h[2], g.lo[2]);
    float2 acc[kDipGY][kDipGX / 2], ks[kDipGY][kDipGX / 2], kc[kDipGY][kDipGX / 2];
#pragma unroll
    for (int i = 0; i < kDipGY; ++i)
#pragma unroll
        for (int j = 0; j < kDipGX / 2; ++j) acc[i][j] = ks[i][j] = kc[i][j] = make_float2(0.f, 0.f);
    for (int64_t f0 = 0; f0 < nf; f0 += kDipTile) {
        const int cnt = (int)(nf - f0 < kDipTile ? nf - f0 : kDipTile);
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += kDipThreads) tile[i] = dip_face(rec[f0 + i]);
        __syncthreads();
#pragma unroll 1
        for (int k = 0; k < cnt; ++k) {
            const DipFace d = tile[k];
            const float rz = d.c.z - qz;
            const float rz2 = rz * rz, mzrz = d.m.z * rz;
            const float2 cx = make_float2(d.c.x, d.c.x), mx = make_float2(d.m.x, d.m.x);
#pragma unroll
            for (int i = 0; i < kDipGY; ++i) {
                const float ry = d.c.y - qy[i];
                // + 1e-24 keeps |r|^2 > 0 at the centroid itself, where m.r = 0 exactly and
                // |r|^-3 = 1e36 stays finite, so the term is 0 as before
                const float Lyz = fmaf(ry, ry, rz2) + 1e-24f, Myz = fmaf(d.m.y, ry, mzrz);
#pragma unroll
                for (int j = 0; j < kDipGX / 2; ++j) {
                    const float2 rx = __fadd2_rn(cx, nqx[j]);
                    const float2 r2 = __ffma2_rn(rx, rx, make_float2(Lyz, Lyz));
                    const float2 ir = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
                    const float2 ir3 = __fmul2_rn(__fmul2_rn(ir, ir), ir);
                    const float2 mr = __ffma2_rn(mx, rx, make_float2(Myz, Myz));
                    acc[i][j] = __ffma2_rn(mr, ir3, acc[i][j]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < kDipGY; ++i)
#pragma unroll
            for (int j = 0; j < kDipGX / 2; ++j) {  // Kahan across tiles
                const float2 y = make_float2(acc[i][j].x - kc[i][j].x, acc[i][j].y - kc[i][j].y);
                const float2 tt = make_float2(ks[i][j].x + y.x, ks[i][j].y + y.y);
                kc[i][j] = make_float2((tt.x - ks[i][j].x) - y.x, (tt.y - ks[i][j].y) - y.y);
                ks[i][j] = tt;
                acc[i][j] = make_float2(0.f, 0.f);
            }
    }
    if (!valid) return;
#pragma unroll
    for (int i = 0; i < kDipGY; ++i) {
        const int iy = ty * kDipGY + i;
        if (iy >= ny) continue;
#pragma unroll
        for (int j = 0; j < kDipGX; ++j) {
            const int ix = tx * kDipGX + j;
            if (ix >= nx) continue;
            const float s0 = j % 2 ? ks[i][j / 2].y : ks[i][j / 2].x, c0 = j % 2 ? kc[i][j / 2].y : kc[i][j / 2].x;
            w_out[((int64_t)z * ny + iy) * nx + ix] = (s0 - c0) * kInv4Pi;
        }
    }
}

// Adjoint on a grid: face-parallel over a split of the grid's rows. Per pair only
// gi3 = g / |r|^3 and t = gi3 (m.r) / |r|^2 are computed; the row sums of gi3, gi3 rx, t and
// t rx are folded per row with the row's ry, rz into the 7 Kahan face sums.
__global__ void __launch_bounds__(kDipBwdThreads) dipole_bwd_grid_kernel(const FaceRec *__restrict__ rec, int64_t nf,
                                                                        GridF g, const float *__restrict__ upstream,
                                                                        int64_t rows_per_split,
                                                                        float *__restrict__ face_grad) {
    __shared__ __align__(16) float4 win[kDipWin / 2];  // pairs: (-x_i, -x_i+1, g_i, g_i+1)
    const int64_t f = (int64_t)blockIdx.x * kDipBwdThreads + threadIdx.x;
    const FaceRec r = rec[f < nf ? f : nf - 1];
    const DipFace d = dip_face(r);
    const int nx = g.n[0], ny = g.n[1];
    const int64_t nrows = (int64_t)g.n[1] * g.n[2];
    const int64_t r0 = (int64_t)blockIdx.y * rows_per_split;
    const int64_t r1 = r0 + rows_per_split < nrows ? r0 + rows_per_split : nrows;
    const bool whole = nx <= kDipWin && nx % 2 == 0;
    const int rows_per_win = whole ? kDipWin / nx : 1;
    const float2 cx = make_float2(d.c.x, d.c.x), mx = make_float2(d.m.x, d.m.x);
    float s[7] = {0, 0, 0, 0, 0, 0, 0}, c[7] = {0, 0, 0, 0, 0, 0, 0};
    auto kahan = [&](int k, float x) {
        const float y = x - c[k];
        const float tt = s[k] + y;
        c[k] = (tt - s[k]) - y;
        s[k] = tt;
    };
    for (int64_t rw = r0; rw < r1; rw += rows_per_win) {
        const int64_t rend = rw + rows_per_win < r1 ? rw + rows_per_win : r1;
        for (int x0 = 0; x0 < nx; x0 += kDipWin) {
            const int xlen = whole ? nx : (nx - x0 < kDipWin ? nx - x0 : kDipWin);
            const int64_t len = whole ? (rend - rw) * nx : xlen;
            const int64_t base = rw * nx + (whole ? 0 : x0);
            __syncthreads();
            float *wf = reinterpret_cast<float *>(win);
            for (int64_t i = threadIdx.x; i < len; i += kDipBwdThreads) {
                const int ix = whole ? (int)(i % nx) : x0 + (int)i;
                wf[4 * (i >> 1) + (i & 1)] = -__fmaf_rn((float)ix + 0.5f, g.h[0], g.lo[0]);
                wf[4 * (i >> 1) + 2 + (i & 1)] = upstream[base + i];
            }
            if (!whole && (len & 1) && threadIdx.x == 0) {  // pad an odd piece with g = 0
                wf[4 * (len >> 1) + 1] = -__fmaf_rn((float)(x0 + len - 1) + 0.5f, g.h[0], g.lo[0]);
                wf[4 * (len >> 1) + 3] = 0.f;
            }
            __syncthreads();
            const int64_t nr = whole ? rend - rw : 1;
            for (int64_t rr = 0; rr < nr; ++rr) {
                const int64_t row = rw + rr;
                const int iy = (int)(row % ny), iz = (int)(row / ny);
                const float ry = d.c.y - __fmaf_rn((float)iy + 0.5f, g.h[1], g.lo[1]);
                const float rz = d.c.z - __fmaf_rn((float)iz + 0.5f, g.h[2], g.lo[2]);
                const float2 L2 = make_float2(fmaf(ry, ry, rz * rz), fmaf(ry, ry, rz * rz));
                const float myz = fmaf(d.m.y, ry, d.m.z * rz);
                const float2 M2 = make_float2(myz, myz);
                const int64_t p0 = whole ? rr * nx / 2 : 0;
                const int np = whole ? nx / 2 : (int)((len + 1) / 2);
                // sums of gi3, gi3 rx, t, t rx over the row: unguarded first; a query exactly at the
                // centroid (|r| = 0) makes them non-finite, and then the row is summed again with
                // that query's term set to 0
                auto row_sums = [&](auto guard, float2 &A, float2 &B, float2 &T, float2 &E) {
                    A = B = T = E = make_float2(0.f, 0.f);
#pragma unroll 2
                    for (int p = 0; p < np; ++p) {
                        const float4 q = win[p0 + p];
                        const float2 rx = __fadd2_rn(cx, make_float2(q.x, q.y));
                        const float2 r2 = __ffma2_rn(rx, rx, L2);
                        const float2 ir = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
                        const float2 ir2 = __fmul2_rn(ir, ir);
                        float2 gi3 = __fmul2_rn(__fmul2_rn(make_float2(q.z, q.w), ir2), ir);
                        if (decltype(guard)::value) {  // |r| = 0: the term is 0 (not 0 * inf)
                            gi3.x = r2.x > 0.f ? gi3.x : 0.f;
                            gi3.y = r2.y > 0.f ? gi3.y : 0.f;
                        }
                        float2 tt = __fmul2_rn(__fmul2_rn(gi3, __ffma2_rn(mx, rx, M2)), ir2);
                        if (decltype(guard)::value) {
                            tt.x = r2.x > 0.f ? tt.x : 0.f;
                            tt.y = r2.y > 0.f ? tt.y : 0.f;
                        }
                        A = __fadd2_rn(A, gi3);
                        B = __ffma2_rn(gi3, rx, B);
                        T = __fadd2_rn(T, tt);
                        E = __ffma2_rn(tt, rx, E);
                    }
                };
                float2 A, B, T, E;
                row_sums(std::false_type{}, A, B, T, E);
                if (!isfinite((A.x + A.y) + (B.x + B.y) + (T.x + T.y) + (E.x + E.y)))
                    row_sums(std::true_type{}, A, B, T, E);
                const float a = A.x + A.y, b = B.x + B.y, t = T.x + T.y, e = E.x + E.y;
                kahan(0, a);
                kahan(1, b);
                kahan(2, a * ry);
                kahan(3, a * rz);
                kahan(4, e);
                kahan(5, t * ry);
                kahan(6, t * rz);
            }
            if (whole) break;
        }
    }
    if (f >= nf) return;
    dip_face_grad(r, d, s, c, face_grad + ((int64_t)blockIdx.y * nf + f) * 9);
}

int dipole_bwd_splits(int64_t nq, int64_t nf, int num_sms) {
    const int64_t fblocks = (nf + kDipBwdThreads - 1) / kDipBwdThreads;
    int64_t ns = (20LL * num_sms + fblocks - 1) / fblocks;
    if (ns < 1) ns = 1;
    if (ns > nq) ns = nq;
    if (ns > 1024) ns = 1024;
    const int64_t per = (nq + ns - 1) / ns;
    return (int)((nq + per - 1) / per);
}

cudaError_t launch_dipole_forward(const FaceRec *rec, int64_t nf, const GridF *g, const float *queries, int64_t nq,
                                  float *w_out, cudaStream_t s) {
    GridF gf{};
    if (g) gf = *g;
    prof_begin("dipole_fwd", s);
    if (queries) {
        const int64_t blocks = (nq + (int64_t)kDipThreads * kDipQ - 1) / ((int64_t)kDipThreads * kDipQ);
        dipole_fwd_kernel<<<(unsigned)blocks, kDipThreads, 0, s>>>(rec, nf, gf, queries, nq, w_out);
    } else {
        const int64_t tiles = (int64_t)((gf.n[0] + kDipGX - 1) / kDipGX) * ((gf.n[1] + kDipGY - 1) / kDipGY) * gf.n[2];
        dipole_fwd_grid_kernel<<<(unsigned)((tiles + kDipThreads - 1) / kDipThreads), kDipThreads, 0, s>>>(rec, nf, gf,
                                                                                                         w_out);
    }
    count_launch();
    prof_end("dipole_fwd", s);
    return cudaGetLastError();
}

cudaError_t launch_dipole_backward(const FaceRec *rec, int64_t nf, const GridF *g, const float *queries, int64_t nq,
                                   const float *upstream, int nsplit, float *face_grad, cudaStream_t s) {
    GridF gf{};
    if (g) gf = *g;
    dim3 grid((unsigned)((nf + kDipBwdThreads - 1) / kDipBwdThreads), (unsigned)nsplit);
    prof_begin("dipole_bwd", s);
    if (queries) {
        const int64_t per = (nq + nsplit - 1) / nsplit;
        dipole_bwd_kernel<<<grid, kDipBwdThreads, 0, s>>>(rec, nf, gf, queries, nq, upstream, per, face_grad);
    } else {
        // the same nsplit slices of the grid's rows (a slice past the last row writes zeros)
        const int64_t nrows = (int64_t)gf.n[1] * gf.n[2];
        const int64_t per_rows = (nrows + nsplit - 1) / nsplit;
        dipole_bwd_grid_kernel<<<grid, kDipBwdThreads, 0, s>>>(rec, nf, gf, upstream, per_rows, face_grad);
    }
    count_launch();
    prof_end("dipole_bwd", s);
    return cudaGetLastError();
}

}  // namespace dv
