// Adjoint of the winding number from the mesh's boundary curve.
//
// The solid angle a surface subtends at q depends only on the surface's boundary curve (for q
// off the surface), so the derivative of Eq. (5) with respect to the vertices collects only on
// boundary vertices. Summing the per-face derivative of Eq. (7) over all faces, every edge shared
// by two consistently oriented faces cancels, and what remains is a sum over the directed edges
// u -> v with nonzero net multiplicity m (count of u -> v minus count of v -> u over all faces).
// For one directed edge p -> r, with a = p - q, b = r - q (varying the curve linearly along the
// edge and integrating the variation of the solid angle in closed form):
//   dOmega/dp = (b x a) / (|a| (|a||b| + a.b)),   dOmega/dr = (b x a) / (|b| (|a||b| + a.b)).
// The result is the same quantity as the face-by-face adjoint (winding_bwd.cu) up to rounding,
// with exact zeros on closed meshes and on vertices away from the boundary, and it needs one pair
// evaluation per (boundary edge, query) instead of per (face, query).
//
// Because b x a = r x p - e x q (e = r - p) is linear in q, per edge only
//   S_p = sum g c_p, Q_p = sum g c_p q, S_r = sum g c_r, Q_r = sum g c_r q
// (c_p = 1 / (|a| (|a||b| + a.b)), c_r likewise with |b|) are accumulated; the gather forms
//   dL/dp += m/(4 pi) [(r x p) S_p - e x Q_p],  dL/dr += m/(4 pi) [(r x p) S_r - e x Q_r]
// in FP64. On a grid row the y and z parts of a, b are constant; two x-adjacent queries share
// one packed FP32x2 instruction. Sums are FP32 per row (grid) or per chunk (list), Kahan across
// rows in shared memory. A pair with |a||b| + a.b = 0 (q on the edge segment, i.e. on the mesh)
// has no derivative; such rows are recomputed by a guarded path that skips those pairs.
#include <math.h>

#include "dv_internal.cuh"

namespace dv {

constexpr int kBndThreads = 128;
constexpr int kBndWin = 2048;   // grid: queries staged per window; list: 2 x (x, y, z, g) float4s
constexpr int kBndSlots = 8;    // S_p, S_r, Q_p (3), Q_r (3)
constexpr int kBndChunk = 128;  // list path: queries per plain FP32 partial sum

struct BndArgs {
    const BndRec *rec;
    int64_t nb;
    GridF g;
    const float *queries;
    int64_t nq;
    const float *upstream;
    int64_t per_split;  // grid: rows per split; list: queries per split
    float *part;        // [nsplit][nb][8]
};

__device__ __forceinline__ void kahan_slot(float2 *slot, float x) {
    float2 k = *slot;
    const float y = __fsub_rn(x, k.y);
    const float t = __fadd_rn(k.x, y);
    k.y = __fsub_rn(__fsub_rn(t, k.x), y);
    k.x = t;
    *slot = k;
}

// Scalar guarded pair: skips q at an endpoint or on the edge segment.
__device__ __forceinline__ void bnd_pair_guarded(float ax, float ay, float az, float bx, float by, float bz, float g,
                                                 float &sp, float &sr, float &cpq, float &crq) {
    const float la2 = fmaf(ax, ax, fmaf(ay, ay, az * az));
    const float lb2 = fmaf(bx, bx, fmaf(by, by, bz * bz));
    if (!(la2 > 0.f) || !(lb2 > 0.f)) return;
    const float la = sqrtf(la2), lb = sqrtf(lb2);
    const float De = fmaf(la, lb, fmaf(ax, bx, fmaf(ay, by, az * bz)));
    if (!(De > 1e-30f * la * lb)) return;
    const float gr = g / De;
    cpq = gr / la;
    crq = gr / lb;
    sp += cpq;
    sr += crq;
}

__global__ void __launch_bounds__(kBndThreads, 4) bnd_grid_kernel(const BndArgs a) {
    __shared__ __align__(16) float wf[2 * kBndWin];  // pairs: (-x_i, -x_i+1, g_i, g_i+1)
    __shared__ float2 ks[kBndSlots][kBndThreads];
    const int64_t e = (int64_t)blockIdx.x * kBndThreads + threadIdx.x;
    const BndRec R = a.rec[e < a.nb ? e : a.nb - 1];
    const float2 px = make_float2(R.p.x, R.p.x), rx = make_float2(R.r.x, R.r.x);
    const int nx = a.g.n[0], ny = a.g.n[1];
    const int64_t nrows = (int64_t)a.g.n[1] * a.g.n[2];
    const int64_t r0 = (int64_t)blockIdx.y * a.per_split;
    const int64_t r1 = r0 + a.per_split < nrows ? r0 + a.per_split : nrows;
#pragma unroll
    for (int k = 0; k < kBndSlots; ++k) ks[k][threadIdx.x] = make_float2(0.f, 0.f);
    const bool whole = nx <= kBndWin && nx % 2 == 0;
    const int rows_per_win = whole ? kBndWin / nx : 1;
    for (int64_t rw = r0; rw < r1; rw += rows_per_win) {
        const int64_t rend = rw + rows_per_win < r1 ? rw + rows_per_win : r1;
        for (int x0 = 0; x0 < nx; x0 += kBndWin) {
            const int xlen = whole ? nx : (nx - x0 < kBndWin ? nx - x0 : kBndWin);
            const int64_t len = whole ? (rend - rw) * nx : xlen;
            const int64_t base = rw * nx + (whole ? 0 : x0);
            __syncthreads();
            for (int64_t i = threadIdx.x; i < len; i += kBndThreads) {
                const int ix = whole ? (int)(i % nx) : x0 + (int)i;
                wf[4 * (i >> 1) + (i & 1)] = -__fmaf_rn((float)ix + 0.5f, a.g.h[0], a.g.lo[0]);
                wf[4 * (i >> 1) + 2 + (i & 1)] = a.upstream[base + i];
            }
            if (!whole && (len & 1) && threadIdx.x == 0) {  // pad an odd piece with g = 0
                wf[4 * (len >> 1) + 1] = -__fmaf_rn((float)(x0 + len - 1) + 0.5f, a.g.h[0], a.g.lo[0]);
                wf[4 * (len >> 1) + 3] = 0.f;
            }
            __syncthreads();
            const int64_t nr = whole ? rend - rw : 1;
            for (int64_t rr = 0; rr < nr; ++rr) {
                const int64_t row = rw + rr;
                const int iy = (int)(row % ny), iz = (int)(row / ny);
                const float qy = __fmaf_rn((float)iy + 0.5f, a.g.h[1], a.g.lo[1]);
                const float qz = __fmaf_rn((float)iz + 0.5f, a.g.h[2], a.g.lo[2]);
                const float ay = R.p.y - qy, az = R.p.z - qz, by = R.r.y - qy, bz = R.r.z - qz;
                const float La = fmaf(ay, ay, az * az), Lb = fmaf(by, by, bz * bz), Pab = fmaf(ay, by, az * bz);
                const float2 La2 = make_float2(La, La), Lb2 = make_float2(Lb, Lb), Pab2 = make_float2(Pab, Pab);
                float2 Sp = make_float2(0.f, 0.f), Sr = Sp, Xp = Sp, Xr = Sp;  // X = sum g c (-x)
                const int64_t p0 = whole ? rr * nx / 2 : 0;
                const int np = whole ? nx / 2 : (int)((len + 1) / 2);
                const float4 *wp = reinterpret_cast<const float4 *>(wf) + p0;
#pragma unroll 4
                for (int p = 0; p < np; ++p) {
                    const float4 q = wp[p];
                    const float2 nqx = make_float2(q.x, q.y);
                    const float2 ax = __fadd2_rn(px, nqx), bx = __fadd2_rn(rx, nqx);
                    const float2 la2 = __ffma2_rn(ax, ax, La2), lb2 = __ffma2_rn(bx, bx, Lb2);
                    const float2 ia = make_float2(rsqrt_approx(la2.x), rsqrt_approx(la2.y));
                    const float2 ib = make_float2(rsqrt_approx(lb2.x), rsqrt_approx(lb2.y));
                    const float2 De = __ffma2_rn(__fmul2_rn(la2, ia), __fmul2_rn(lb2, ib), __ffma2_rn(ax, bx, Pab2));
                    const float2 gr = __fmul2_rn(make_float2(q.z, q.w), make_float2(rcp_approx(De.x), rcp_approx(De.y)));
                    const float2 cp = __fmul2_rn(gr, ia), cr = __fmul2_rn(gr, ib);
                    Sp = __fadd2_rn(Sp, cp);
                    Sr = __fadd2_rn(Sr, cr);
                    Xp = __ffma2_rn(cp, nqx, Xp);
                    Xr = __ffma2_rn(cr, nqx, Xr);
                }
                float sp = Sp.x + Sp.y, sr = Sr.x + Sr.y, xp = Xp.x + Xp.y, xr = Xr.x + Xr.y;
                if (!isfinite(sp + sr + xp + xr)) {
                    // a query on an endpoint or on the edge segment: skip those pairs
                    sp = sr = xp = xr = 0.f;
                    const int cnt = whole ? nx : (int)len;
                    for (int i = 0; i < cnt; ++i) {
                        const int64_t wi = 2 * p0 + i;
                        const float nqxs = wf[4 * (wi >> 1) + (wi & 1)], gs = wf[4 * (wi >> 1) + 2 + (wi & 1)];
                        float cpq = 0.f, crq = 0.f;
                        bnd_pair_guarded(R.p.x + nqxs, ay, az, R.r.x + nqxs, by, bz, gs, sp, sr, cpq, crq);
                        xp = fmaf(cpq, nqxs, xp);
                        xr = fmaf(crq, nqxs, xr);
                    }
                }
                const int t = threadIdx.x;
                kahan_slot(&ks[0][t], sp);
                kahan_slot(&ks[1][t], sr);
                kahan_slot(&ks[2][t], -xp);  // Q_p.x = sum g c_p x
                kahan_slot(&ks[3][t], qy * sp);
                kahan_slot(&ks[4][t], qz * sp);
                kahan_slot(&ks[5][t], -xr);
                kahan_slot(&ks[6][t], qy * sr);
                kahan_slot(&ks[7][t], qz * sr);
            }
            if (whole) break;
        }
    }
    if (e >= a.nb) return;
    float *out = a.part + ((int64_t)blockIdx.y * a.nb + e) * kBndSlots;
#pragma unroll
    for (int k = 0; k < kBndSlots; ++k) out[k] = ks[k][threadIdx.x].x - ks[k][threadIdx.x].y;
}

// List path: queries staged as (x, y, z, g); no row sharing, two queries per packed instruction.
__global__ void __launch_bounds__(kBndThreads, 4) bnd_list_kernel(const BndArgs a) {
    __shared__ float4 win[kBndWin / 2];
    __shared__ float2 ks[kBndSlots][kBndThreads];
    const int64_t e = (int64_t)blockIdx.x * kBndThreads + threadIdx.x;
    const BndRec R = a.rec[e < a.nb ? e : a.nb - 1];
    const float2 px = make_float2(R.p.x, R.p.x), py = make_float2(R.p.y, R.p.y), pz = make_float2(R.p.z, R.p.z);
    const float2 rx = make_float2(R.r.x, R.r.x), ry = make_float2(R.r.y, R.r.y), rz = make_float2(R.r.z, R.r.z);
    const int64_t q0 = (int64_t)blockIdx.y * a.per_split;
    const int64_t q1 = q0 + a.per_split < a.nq ? q0 + a.per_split : a.nq;
#pragma unroll
    for (int k = 0; k < kBndSlots; ++k) ks[k][threadIdx.x] = make_float2(0.f, 0.f);
    for (int64_t w0 = q0; w0 < q1; w0 += kBndWin / 2) {
        const int len = (int)(q1 - w0 < kBndWin / 2 ? q1 - w0 : kBndWin / 2);
        const int len2 = (len + 1) & ~1;
        __syncthreads();
        for (int i = threadIdx.x; i < len2; i += kBndThreads) {
            const int64_t k = w0 + (i < len ? i : len - 1);
            win[i] = make_float4(-a.queries[3 * k], -a.queries[3 * k + 1], -a.queries[3 * k + 2],
                                 i < len ? a.upstream[k] : 0.0f);
        }
        __syncthreads();
        for (int c0 = 0; c0 < len2; c0 += kBndChunk) {
            const int c1 = c0 + kBndChunk < len2 ? c0 + kBndChunk : len2;
            float2 Sp = make_float2(0.f, 0.f), Sr = Sp, Qp[3] = {Sp, Sp, Sp}, Qr[3] = {Sp, Sp, Sp};  // Q: sum g c (-q)
#pragma unroll 2
            for (int i = c0; i < c1; i += 2) {
                const float4 u = win[i], v = win[i + 1];
                const float2 nx2 = make_float2(u.x, v.x), ny2 = make_float2(u.y, v.y), nz2 = make_float2(u.z, v.z);
                const float2 ax = __fadd2_rn(px, nx2), ay = __fadd2_rn(py, ny2), az = __fadd2_rn(pz, nz2);
                const float2 bx = __fadd2_rn(rx, nx2), by = __fadd2_rn(ry, ny2), bz = __fadd2_rn(rz, nz2);
                const float2 la2 = __ffma2_rn(az, az, __ffma2_rn(ay, ay, __fmul2_rn(ax, ax)));
                const float2 lb2 = __ffma2_rn(bz, bz, __ffma2_rn(by, by, __fmul2_rn(bx, bx)));
                const float2 ia = make_float2(rsqrt_approx(la2.x), rsqrt_approx(la2.y));
                const float2 ib = make_float2(rsqrt_approx(lb2.x), rsqrt_approx(lb2.y));
                const float2 ab = __ffma2_rn(az, bz, __ffma2_rn(ay, by, __fmul2_rn(ax, bx)));
                const float2 De = __ffma2_rn(__fmul2_rn(la2, ia), __fmul2_rn(lb2, ib), ab);
                const float2 gr = __fmul2_rn(make_float2(u.w, v.w), make_float2(rcp_approx(De.x), rcp_approx(De.y)));
                const float2 cp = __fmul2_rn(gr, ia), cr = __fmul2_rn(gr, ib);
                Sp = __fadd2_rn(Sp, cp);
                Sr = __fadd2_rn(Sr, cr);
                Qp[0] = __ffma2_rn(cp, nx2, Qp[0]);
                Qp[1] = __ffma2_rn(cp, ny2, Qp[1]);
                Qp[2] = __ffma2_rn(cp, nz2, Qp[2]);
                Qr[0] = __ffma2_rn(cr, nx2, Qr[0]);
                Qr[1] = __ffma2_rn(cr, ny2, Qr[1]);
                Qr[2] = __ffma2_rn(cr, nz2, Qr[2]);
            }
            float v[kBndSlots] = {Sp.x + Sp.y,       Sr.x + Sr.y,       -(Qp[0].x + Qp[0].y), -(Qp[1].x + Qp[1].y),
                                  -(Qp[2].x + Qp[2].y), -(Qr[0].x + Qr[0].y), -(Qr[1].x + Qr[1].y), -(Qr[2].x + Qr[2].y)};
            float t = 0.f;
#pragma unroll
            for (int k = 0; k < kBndSlots; ++k) t += v[k];
            if (!isfinite(t)) {
                // a query on an endpoint or on the edge segment: skip those pairs
#pragma unroll
                for (int k = 0; k < kBndSlots; ++k) v[k] = 0.f;
                const int ce = c1 < len ? c1 : len;
                for (int i = c0; i < ce; ++i) {
                    const float4 q = win[i];
                    float cpq = 0.f, crq = 0.f;
                    bnd_pair_guarded(R.p.x + q.x, R.p.y + q.y, R.p.z + q.z, R.r.x + q.x, R.r.y + q.y, R.r.z + q.z,
                                     q.w, v[0], v[1], cpq, crq);
                    v[2] = fmaf(cpq, -q.x, v[2]);
                    v[3] = fmaf(cpq, -q.y, v[3]);
                    v[4] = fmaf(cpq, -q.z, v[4]);
                    v[5] = fmaf(crq, -q.x, v[5]);
                    v[6] = fmaf(crq, -q.y, v[6]);
                    v[7] = fmaf(crq, -q.z, v[7]);
                }
            }
            // slots: S_p, S_r, Q_p (x, y, z), Q_r (x, y, z)
            const float sl[kBndSlots] = {v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7]};
#pragma unroll
            for (int k = 0; k < kBndSlots; ++k) kahan_slot(&ks[k][threadIdx.x], sl[k]);
        }
    }
    if (e >= a.nb) return;
    float *out = a.part + ((int64_t)blockIdx.y * a.nb + e) * kBndSlots;
#pragma unroll
    for (int k = 0; k < kBndSlots; ++k) out[k] = ks[k][threadIdx.x].x - ks[k][threadIdx.x].y;
}

// dverts[v] = sum over the boundary endpoints at v (CSR, fixed order) of
//   m/(4 pi) [(r x p) S - e x Q]   (S, Q of that endpoint, summed over the splits in FP64).
__global__ void bnd_gather_kernel(int64_t nv, const BndRec *__restrict__ rec, int64_t nb,
                                  const float *__restrict__ part, int nsplit, const int32_t *__restrict__ vptr,
                                  const int32_t *__restrict__ vend, float *__restrict__ dverts) {
    const double k4 = 1.0 / (4.0 * 3.14159265358979323846);
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
        double G[3] = {0.0, 0.0, 0.0};
        for (int32_t c = vptr[v]; c < vptr[v + 1]; ++c) {
            const int32_t code = vend[c];
            const int64_t e = code >> 1;
            const int end = code & 1;  // 0: v is p (the edge's start), 1: v is r
            const BndRec b = rec[e];
            const double m = (double)b.p.w;
            double S = 0.0, Q[3] = {0.0, 0.0, 0.0};
            for (int s = 0; s < nsplit; ++s) {
                const float *pp = part + ((int64_t)s * nb + e) * kBndSlots;
                S += (double)pp[end];
                for (int k = 0; k < 3; ++k) Q[k] += (double)pp[2 + 3 * end + k];
            }
            const double p[3] = {b.p.x, b.p.y, b.p.z};
            const double r[3] = {b.r.x, b.r.y, b.r.z};
            const double ed[3] = {r[0] - p[0], r[1] - p[1], r[2] - p[2]};
            const double rxp[3] = {r[1] * p[2] - r[2] * p[1], r[2] * p[0] - r[0] * p[2], r[0] * p[1] - r[1] * p[0]};
            const double exq[3] = {ed[1] * Q[2] - ed[2] * Q[1], ed[2] * Q[0] - ed[0] * Q[2], ed[0] * Q[1] - ed[1] * Q[0]};
            for (int k = 0; k < 3; ++k) G[k] += m * (rxp[k] * S - exq[k]);
        }
        for (int k = 0; k < 3; ++k) dverts[3 * v + k] = (float)(k4 * G[k]);
    }
}

// Endpoint coordinates come from the packed face records (the first (face, corner) of each
// vertex in the vertex CSR): the same FP32 values as the vertex array they were packed from.
__device__ __forceinline__ float4 vertex_from_rec(const FaceRec *__restrict__ frec, const int32_t *__restrict__ vptr,
                                                  const int32_t *__restrict__ vcorner, int64_t v) {
    const int32_t c = vcorner[vptr[v]];
    const FaceRec r = frec[c / 3];
    const int k = c - 3 * (c / 3);
    return k == 0 ? r.r0 : (k == 1 ? r.r1 : r.r2);
}

__global__ void pack_bnd_kernel(const FaceRec *__restrict__ frec, const int32_t *__restrict__ vptr,
                                const int32_t *__restrict__ vcorner, const int32_t *__restrict__ edges, int64_t nb,
                                BndRec *__restrict__ rec) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nb; e += (int64_t)gridDim.x * blockDim.x) {
        const float4 p = vertex_from_rec(frec, vptr, vcorner, edges[3 * e]);
        const float4 r = vertex_from_rec(frec, vptr, vcorner, edges[3 * e + 1]);
        BndRec b;
        b.p = make_float4(p.x, p.y, p.z, (float)edges[3 * e + 2]);
        b.r = make_float4(r.x, r.y, r.z, 0.f);
        rec[e] = b;
    }
}

static int grid_blocks(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (1 << 20)) b = 1 << 20;
    return (int)b;
}

cudaError_t launch_pack_boundary(const FaceRec *frec, const int32_t *vptr, const int32_t *vcorner,
                                 const int32_t *edges, int64_t nb, BndRec *rec, cudaStream_t s) {
    if (nb == 0) return cudaSuccess;
    prof_begin("pack_boundary", s);
    pack_bnd_kernel<<<grid_blocks(nb, 256), 256, 0, s>>>(frec, vptr, vcorner, edges, nb, rec);
    count_launch();
    prof_end("pack_boundary", s);
    return cudaGetLastError();
}

BndPlan plan_boundary(int64_t nq, int64_t nb, bool grid, const GridF *g, int num_sms) {
    BndPlan p{};
    p.eblocks = (nb + kBndThreads - 1) / kBndThreads;
    if (p.eblocks < 1) p.eblocks = 1;
    const int64_t units = grid ? (int64_t)g->n[1] * g->n[2] : nq;  // rows or queries
    const int64_t target = 16LL * num_sms;  // about 4 resident CTAs per SM, >= 4 waves
    int64_t ns = (target + p.eblocks - 1) / p.eblocks;
    if (ns < 1) ns = 1;
    if (ns > units) ns = units > 0 ? units : 1;
    if (ns > 4096) ns = 4096;
    p.per_split = (units + ns - 1) / ns;
    p.nsplit = (int)((units + p.per_split - 1) / p.per_split);
    if (p.nsplit < 1) p.nsplit = 1;
    return p;
}

cudaError_t launch_boundary_backward(const BndPlan &p, const BndRec *rec, int64_t nb, const GridF *g,
                                     const float *queries, int64_t nq, const float *upstream, float *part,
                                     cudaStream_t s) {
    if (nb == 0) return cudaSuccess;
    BndArgs a{};
    a.rec = rec;
    a.nb = nb;
    if (g) a.g = *g;
    a.queries = queries;
    a.nq = nq;
    a.upstream = upstream;
    a.per_split = p.per_split;
    a.part = part;
    dim3 grid((unsigned)p.eblocks, (unsigned)p.nsplit);
    prof_begin(queries ? "bnd_list" : "bnd_grid", s);
    if (queries)
        bnd_list_kernel<<<grid, kBndThreads, 0, s>>>(a);
    else
        bnd_grid_kernel<<<grid, kBndThreads, 0, s>>>(a);
    count_launch();
    prof_end(queries ? "bnd_list" : "bnd_grid", s);
    return cudaGetLastError();
}

cudaError_t launch_boundary_gather(int64_t nv, const BndRec *rec, int64_t nb, const float *part, int nsplit,
                                   const int32_t *vptr, const int32_t *vend, float *dverts, cudaStream_t s) {
    prof_begin("bnd_gather", s);
    bnd_gather_kernel<<<grid_blocks(nv, 256), 256, 0, s>>>(nv, rec, nb, part, nsplit, vptr, vend, dverts);
    count_launch();
    prof_end("bnd_gather", s);
    return cudaGetLastError();
}

}  // namespace dv
