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
// With d = r - p, b x a = d x a = d x b, so the term at either endpoint is its c times d x (its own
// offset from q): per edge only
//   V_p = sum g c_p a,   V_r = sum g c_r b
// (c_p = 1 / (|a| (|a||b| + a.b)), c_r likewise with |b|) are accumulated, and the gather forms
//   dL/dp += m/(4 pi) d x V_p,  dL/dr += m/(4 pi) d x V_r
// in FP64 (offsets, not absolute coordinates: the sums do not depend on where the mesh sits). On
// a grid row the y and z parts of a, b are constant (V_p = (sum g c_p a_x, a_y S_p, a_z S_p)); two
// x-adjacent queries share one packed FP32x2 instruction. Sums are FP32 per row (grid) or per
// chunk (list), Kahan across
// rows in shared memory. A pair with |a||b| + a.b = 0 (q on the edge segment, i.e. on the mesh)
// has no derivative; such rows are recomputed by a guarded path that skips those pairs. Rows (grid)
// or chunks (list) with a query near the segment, where the packed sum |a||b| + a.b cancels, take
// the same guarded path with t from edge_t.
#include <math.h>

#include "dv_internal.cuh"

namespace dv {

constexpr int kBndThreads = 128;
constexpr int kBndWin = 2048;   // grid: queries staged per window; list: 2 x (x, y, z, g) float4s
constexpr int kBndSlots = kBndPartFloats;  // V_p (3), V_r (3)
constexpr int kBndChunk = 128;  // list path: queries per plain FP32 partial sum

struct BndArgs {
    const BndRec *rec;
    int64_t nb;
    GridF g;
    const float *queries;
    int64_t nq;
    const float *upstream;
    int64_t per_split;  // grid: rows per split; list: queries per split
    float *part;        // [nsplit][nb][6]
};

__device__ __forceinline__ void kahan_slot(float2 *slot, float x) {
    float2 k = *slot;
    const float y = __fsub_rn(x, k.y);
    const float t = __fadd_rn(k.x, y);
    k.y = __fsub_rn(__fsub_rn(t, k.x), y);
    k.x = t;
    *slot = k;
}

// Scalar guarded pair (t from edge_t, d = r - p): skips q at an endpoint or on the edge segment.
__device__ __forceinline__ void bnd_pair_guarded(float ax, float ay, float az, float bx, float by, float bz, float dx,
                                                 float dy, float dz, float g, float &sp, float &sr, float &cpq,
                                                 float &crq) {
    const float la2 = fmaf(ax, ax, fmaf(ay, ay, az * az));
    const float lb2 = fmaf(bx, bx, fmaf(by, by, bz * bz));
    float ia, ib, gr;
    if (!edge_coeffs(ax, ay, az, bx, by, bz, la2, lb2, dx, dy, dz, g, ia, ib, gr)) return;
    cpq = gr * ia;
    crq = gr * ib;
    sp += cpq;
    sr += crq;
}

__global__ void __launch_bounds__(kBndThreads, 4) bnd_grid_kernel(const BndArgs a) {
    __shared__ __align__(16) float wf[2 * kBndWin];  // pairs: (-x_i, -x_i+1, g_i, g_i+1)
    __shared__ float2 ks[kBndSlots][kBndThreads];
    const int64_t e = (int64_t)blockIdx.x * kBndThreads + threadIdx.x;
    const BndRec R = a.rec[e < a.nb ? e : a.nb - 1];
    const float2 px = make_float2(R.p.x, R.p.x), rx = make_float2(R.r.x, R.r.x);
    const float dx = R.r.x - R.p.x, dy = R.r.y - R.p.y, dz = R.r.z - R.p.z;
    const float L2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const int nx = a.g.n[0], ny = a.g.n[1];
    const int64_t nrows = (int64_t)a.g.n[1] * a.g.n[2];
    const int64_t r0 = (int64_t)blockIdx.y * a.per_split;
    const int64_t r1 = r0 + a.per_split < nrows ? r0 + a.per_split : nrows;
#pragma unroll
    for (int k = 0; k < kBndSlots; ++k) ks[k][threadIdx.x] = make_float2(0.f, 0.f);
    // Whole rows per window when a row fits, else pieces of up to kBndWin queries; each row (or
    // piece) takes an even number of entries, an odd one padded with a copy of its last query
    // carrying g = 0, so every row runs the packed loop.
    const bool whole = nx <= kBndWin;
    const int nxe = (nx + 1) & ~1;
    const int rows_per_win = whole ? kBndWin / nxe : 1;
    for (int64_t rw = r0; rw < r1; rw += rows_per_win) {
        const int64_t rend = rw + rows_per_win < r1 ? rw + rows_per_win : r1;
        for (int x0 = 0; x0 < nx; x0 += kBndWin) {
            const int xlen = whole ? nx : (nx - x0 < kBndWin ? nx - x0 : kBndWin);
            const int xle = (xlen + 1) & ~1;
            const int len = whole ? (int)(rend - rw) * nxe : xle;
            __syncthreads();
            for (int i = threadIdx.x; i < len; i += kBndThreads) {
                const int rr = whole ? i / nxe : 0;
                const int k = i - rr * nxe;
                const bool pad = k >= xlen;
                const int ix = x0 + (pad ? xlen - 1 : k);
                wf[4 * (i >> 1) + (i & 1)] = -__fmaf_rn((float)ix + 0.5f, a.g.h[0], a.g.lo[0]);
                wf[4 * (i >> 1) + 2 + (i & 1)] = pad ? 0.f : a.upstream[(rw + rr) * nx + ix];
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
                float2 Sp = make_float2(0.f, 0.f), Sr = Sp, Xp = Sp, Xr = Sp;  // X = sum g c a_x (b_x)
                const int64_t p0 = whole ? rr * nxe / 2 : 0;
                const int np = xle / 2;
                const float4 *wp = reinterpret_cast<const float4 *>(wf) + p0;
                // a row close to the edge segment goes through the guarded path (edge_t)
                const bool near = row_near_edge(ay, az, by, bz, L2);
                if (!near) {
#pragma unroll 4
                    for (int p = 0; p < np; ++p) {
                        const float4 q = wp[p];
                        const float2 nqx = make_float2(q.x, q.y);
                        const float2 ax = __fadd2_rn(px, nqx), bx = __fadd2_rn(rx, nqx);
                        const float2 la2 = __ffma2_rn(ax, ax, La2), lb2 = __ffma2_rn(bx, bx, Lb2);
                        const float2 ia = make_float2(rsqrt_approx(la2.x), rsqrt_approx(la2.y));
                        const float2 ib = make_float2(rsqrt_approx(lb2.x), rsqrt_approx(lb2.y));
                        const float2 De =
                            __ffma2_rn(__fmul2_rn(la2, ia), __fmul2_rn(lb2, ib), __ffma2_rn(ax, bx, Pab2));
                        const float2 gr =
                            __fmul2_rn(make_float2(q.z, q.w), make_float2(rcp_approx(De.x), rcp_approx(De.y)));
                        const float2 cp = __fmul2_rn(gr, ia), cr = __fmul2_rn(gr, ib);
                        Sp = __fadd2_rn(Sp, cp);
                        Sr = __fadd2_rn(Sr, cr);
                        Xp = __ffma2_rn(cp, ax, Xp);
                        Xr = __ffma2_rn(cr, bx, Xr);
                    }
                }
                float sp = Sp.x + Sp.y, sr = Sr.x + Sr.y, xp = Xp.x + Xp.y, xr = Xr.x + Xr.y;
                if (near || !isfinite(sp + sr + xp + xr)) {
                    // near the segment, or a query on an endpoint or on the segment (those pairs
                    // are skipped)
                    sp = sr = xp = xr = 0.f;
                    const int cnt = xle;  // the padding entries carry g = 0
                    for (int i = 0; i < cnt; ++i) {
                        const int64_t wi = 2 * p0 + i;
                        const float nqxs = wf[4 * (wi >> 1) + (wi & 1)], gs = wf[4 * (wi >> 1) + 2 + (wi & 1)];
                        float cpq = 0.f, crq = 0.f;
                        bnd_pair_guarded(R.p.x + nqxs, ay, az, R.r.x + nqxs, by, bz, dx, dy, dz, gs, sp, sr, cpq,
                                         crq);
                        xp = fmaf(cpq, R.p.x + nqxs, xp);
                        xr = fmaf(crq, R.r.x + nqxs, xr);
                    }
                }
                const int t = threadIdx.x;
                kahan_slot(&ks[0][t], xp);  // V_p = (sum g c_p a_x, a_y S_p, a_z S_p)
                kahan_slot(&ks[1][t], ay * sp);
                kahan_slot(&ks[2][t], az * sp);
                kahan_slot(&ks[3][t], xr);  // V_r likewise with b
                kahan_slot(&ks[4][t], by * sr);
                kahan_slot(&ks[5][t], bz * sr);
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
    const float dx = R.r.x - R.p.x, dy = R.r.y - R.p.y, dz = R.r.z - R.p.z;
    const float2 kn = make_float2(kNearCos, kNearCos);
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
            const float2 z2 = make_float2(0.f, 0.f);
            float2 Vp[3] = {z2, z2, z2}, Vr[3] = {z2, z2, z2};  // sum g c_p a, sum g c_r b
            uint32_t near = 0;  // sign bit: a query near the segment (t < kNearCos |a.b|)
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
                const float2 chk = __ffma2_rn(kn, ab, De);
                near |= __float_as_uint(chk.x) | __float_as_uint(chk.y);
                const float2 gr = __fmul2_rn(make_float2(u.w, v.w), make_float2(rcp_approx(De.x), rcp_approx(De.y)));
                const float2 cp = __fmul2_rn(gr, ia), cr = __fmul2_rn(gr, ib);
                Vp[0] = __ffma2_rn(cp, ax, Vp[0]);
                Vp[1] = __ffma2_rn(cp, ay, Vp[1]);
                Vp[2] = __ffma2_rn(cp, az, Vp[2]);
                Vr[0] = __ffma2_rn(cr, bx, Vr[0]);
                Vr[1] = __ffma2_rn(cr, by, Vr[1]);
                Vr[2] = __ffma2_rn(cr, bz, Vr[2]);
            }
            float v[kBndSlots] = {Vp[0].x + Vp[0].y, Vp[1].x + Vp[1].y, Vp[2].x + Vp[2].y,
                                  Vr[0].x + Vr[0].y, Vr[1].x + Vr[1].y, Vr[2].x + Vr[2].y};
            float t = 0.f;
#pragma unroll
            for (int k = 0; k < kBndSlots; ++k) t += v[k];
            if ((near >> 31) || !isfinite(t)) {
                // a query near the segment (guarded t), or on an endpoint or on the segment (those
                // pairs are skipped)
#pragma unroll
                for (int k = 0; k < kBndSlots; ++k) v[k] = 0.f;
                const int ce = c1 < len ? c1 : len;
                for (int i = c0; i < ce; ++i) {
                    const float4 q = win[i];
                    const float ax = R.p.x + q.x, ay = R.p.y + q.y, az = R.p.z + q.z;
                    const float bx = R.r.x + q.x, by = R.r.y + q.y, bz = R.r.z + q.z;
                    float sp = 0.f, sr = 0.f, cpq = 0.f, crq = 0.f;
                    bnd_pair_guarded(ax, ay, az, bx, by, bz, dx, dy, dz, q.w, sp, sr, cpq, crq);
                    v[0] = fmaf(cpq, ax, v[0]);
                    v[1] = fmaf(cpq, ay, v[1]);
                    v[2] = fmaf(cpq, az, v[2]);
                    v[3] = fmaf(crq, bx, v[3]);
                    v[4] = fmaf(crq, by, v[4]);
                    v[5] = fmaf(crq, bz, v[5]);
                }
            }
            // slots: V_p (x, y, z), V_r (x, y, z)
#pragma unroll
            for (int k = 0; k < kBndSlots; ++k) kahan_slot(&ks[k][threadIdx.x], v[k]);
        }
    }
    if (e >= a.nb) return;
    float *out = a.part + ((int64_t)blockIdx.y * a.nb + e) * kBndSlots;
#pragma unroll
    for (int k = 0; k < kBndSlots; ++k) out[k] = ks[k][threadIdx.x].x - ks[k][threadIdx.x].y;
}

// dverts[v] = sum over the boundary endpoints at v (CSR, fixed order) of
//   m/(4 pi) d x V   (V of that endpoint, summed over the splits in FP64; d = r - p).
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
            double V[3] = {0.0, 0.0, 0.0};
            for (int s = 0; s < nsplit; ++s) {
                const float *pp = part + ((int64_t)s * nb + e) * kBndSlots;
                for (int k = 0; k < 3; ++k) V[k] += (double)pp[3 * end + k];
            }
            const double ed[3] = {(double)b.r.x - (double)b.p.x, (double)b.r.y - (double)b.p.y,
                                  (double)b.r.z - (double)b.p.z};
            G[0] += m * (ed[1] * V[2] - ed[2] * V[1]);
            G[1] += m * (ed[2] * V[0] - ed[0] * V[2]);
            G[2] += m * (ed[0] * V[1] - ed[1] * V[0]);
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
