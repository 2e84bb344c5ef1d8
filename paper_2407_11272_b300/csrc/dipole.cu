// Eq. (4): the naive dipole discretization of the winding number,
//     W_dip(q) = (1/4pi) sum_f <n_f, (c_f - q) / |c_f - q|^3> Delta_f
//              = (1/4pi) sum_f (m_f . r) / (2 |r|^3),   r = c_f - q,  m_f = (v1-v0) x (v2-v0),
// with c_f the face centroid and Delta_f its area (m_f = 2 Delta_f n_f). The paper uses it for
// mesh morphing (§2.4) because it is smooth where the exact winding number is almost binary.
// Its adjoint with respect to the vertices: with G_m = sum_q g r / (2|r|^3) and
// G_r = sum_q g [m / (2|r|^3) - 3 (m.r) r / (2|r|^5)],
//     dL/dv0 = (e1 - e2) x G_m + G_r / 3,  dL/dv1 = e2 x G_m + G_r / 3,  dL/dv2 = -e1 x G_m + G_r / 3
// (e1 = v1 - v0, e2 = v2 - v0), all times 1/(4pi). A query at a centroid contributes 0.
// FP32 terms, plain FP32 sums within a tile of faces (forward) or a window of queries (adjoint),
// Kahan across tiles/windows; the adjoint writes per-face partials for the FP64 vertex gather.
#include <math.h>

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
            const float ir2 = r2 > 0.f ? ir * ir : 0.f;
            const float gi3 = q.w * ir2 * ir;
            const float t = gi3 * fmaf(d.m.x, rx, fmaf(d.m.y, ry, d.m.z * rz)) * ir2;
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
    float *out = face_grad + ((int64_t)blockIdx.y * nf + f) * 9;
    for (int k = 0; k < 3; ++k) {
        out[k] = (float)(kk * (c0[k] + Gr[k] / 3.0));
        out[3 + k] = (float)(kk * (c1[k] + Gr[k] / 3.0));
        out[6 + k] = (float)(kk * (-c2[k] + Gr[k] / 3.0));
    }
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
    const int64_t blocks = (nq + (int64_t)kDipThreads * kDipQ - 1) / ((int64_t)kDipThreads * kDipQ);
    prof_begin("dipole_fwd", s);
    dipole_fwd_kernel<<<(unsigned)blocks, kDipThreads, 0, s>>>(rec, nf, gf, queries, nq, w_out);
    count_launch();
    prof_end("dipole_fwd", s);
    return cudaGetLastError();
}

cudaError_t launch_dipole_backward(const FaceRec *rec, int64_t nf, const GridF *g, const float *queries, int64_t nq,
                                   const float *upstream, int nsplit, float *face_grad, cudaStream_t s) {
    GridF gf{};
    if (g) gf = *g;
    const int64_t per = (nq + nsplit - 1) / nsplit;
    dim3 grid((unsigned)((nf + kDipBwdThreads - 1) / kDipBwdThreads), (unsigned)nsplit);
    prof_begin("dipole_bwd", s);
    dipole_bwd_kernel<<<grid, kDipBwdThreads, 0, s>>>(rec, nf, gf, queries, nq, upstream, per, face_grad);
    count_launch();
    prof_end("dipole_bwd", s);
    return cudaGetLastError();
}

}  // namespace dv
