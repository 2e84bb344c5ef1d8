// Adjoint of the winding number: dL/dV = sum_q g_q dw(q)/dV over every (query, face) pair, with
// w = (1/4pi) sum_f Omega_f (Eq. (5)) and Omega_f the solid angle of Eq. (7).
//
// The solid angle of a triangle depends only on its boundary, so the derivative of Omega_f with
// respect to the face's vertices is a sum over its three directed edges: for an edge p -> r of the
// face, with a = p - q and b = r - q,
//   dOmega/dp += (b x a) / (|a| (|a||b| + a.b)),   dOmega/dr += (b x a) / (|b| (|a||b| + a.b)),
// which is the chain rule through Eq. (7) rearranged (q off the face). No arctangent is needed.
// The kernels are face-parallel: a thread owns two faces that share an edge (consecutive faces of
// a strip, paired on the host) or one face left unpaired, streams the queries (uniform across the
// warp) through shared memory, and for the pair evaluates the quad's four edges (the shared edge's
// terms from the two faces cancel; details at bwd_grid_pairs_edges). Per-edge sums are FP32 with
// Kahan compensation in shared memory; per-split face gradients are summed over splits and
// incident faces in FP64 by the gather kernel (pack.cu), in a fixed order.
// With d = r - p, b x a = d x a = d x b, so each edge keeps only the sums of g c times the
// endpoint's offset from q, V_p = sum g c_p a and V_r = sum g c_r b, and forms d x V in FP64.
//   * Grid queries (bwd_grid_kernel): the y, z parts of a, b are constant along a row, so each edge
//     keeps two packed row sums per endpoint (g c and g c a_x).
//   * Query lists (bwd_list_kernel): three packed sums per endpoint (the components of V).
// Where q is near an edge segment, |a||b| + a.b cancels in FP32; rows (grid) or chunks (list) with
// such queries take a guarded scalar path that forms it as |a x b|^2 / (|a||b| - a.b) (edge_t).
#include <math.h>

#include <atomic>

#include "dv_internal.cuh"

namespace dv {

constexpr int kBwdThreads = 128;
constexpr int kBwdWin = 2048;  // queries staged per window

struct BwdArgs {
    const FaceRec *rec;
    int64_t nf;
    GridF g;
    const float *queries;
    int64_t nq;
    const float *upstream;
    int64_t rows_per_split;  // grid: rows; list: queries
    float *face_grad;        // [nsplit][nf][9]
    int *err;
    // grid path: edge-sharing pairs (CTAs [0, pblocks)) and unpaired faces (null: all faces)
    const PairRec *prec;
    const int32_t *ptopo;
    int64_t np;
    const int32_t *singles;
    int64_t nsingle;
    int64_t pblocks;
};

// Packed FP32x2 helpers (Blackwell FFMA2/FADD2/FMUL2 take two queries per instruction; the MUFU
// reciprocal square roots and reciprocals stay scalar).
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 rsqrt2(float2 v) { return make_float2(rsqrt_approx(v.x), rsqrt_approx(v.y)); }

__device__ __forceinline__ void kahan_sm(float2 *slot, float x) {
    float2 k = *slot;
    const float y = __fsub_rn(x, k.y);
    const float t = __fadd_rn(k.x, y);
    k.y = __fsub_rn(__fsub_rn(t, k.x), y);
    k.x = t;
    *slot = k;
}

// Corner codes: canonical corner j of a face goes to its input corner (code >> 2j) & 3.
constexpr int kCornersIdentity = 0 | 1 << 2 | 2 << 4;

// Staged queries of a window, in pairs: for query i (pair p = i/2, k = i%2) the window holds
// -x_i at wf[4p + k] and the upstream g_i at wf[4p + 2 + k], so one 16-byte load gives the
// packed (-x, -x') and (g, g') operands of two consecutive queries.
__device__ __forceinline__ float win_nqx(const float *wf, int64_t i) { return wf[4 * (i >> 1) + (i & 1)]; }
__device__ __forceinline__ float win_g(const float *wf, int64_t i) { return wf[4 * (i >> 1) + 2 + (i & 1)]; }

// Rows of the grid are processed in windows of whole rows when a row fits the window, longer
// rows in pieces of up to kBwdWin queries. Each row (or piece) takes an even number of window
// entries: an odd one is padded with a copy of its last query carrying g = 0, so every row runs
// the packed path. visit(qy, qz, i0, xlen) handles one row (or piece) whose entries sit at window
// indices i0 .. i0 + xlen - 1 (xlen even).
template <typename RowFn>
__device__ __forceinline__ void for_each_row(const BwdArgs &a, float *wf, RowFn &&visit) {
    const int nx = a.g.n[0], ny = a.g.n[1];
    const int64_t nrows = (int64_t)a.g.n[1] * a.g.n[2];
    const int64_t r0 = (int64_t)blockIdx.y * a.rows_per_split;
    const int64_t r1 = r0 + a.rows_per_split < nrows ? r0 + a.rows_per_split : nrows;
    const bool whole = nx <= kBwdWin;
    const int nxe = (nx + 1) & ~1;  // a whole row's entries (<= kBwdWin)
    const int rows_per_win = whole ? kBwdWin / nxe : 1;
    for (int64_t rw = r0; rw < r1; rw += rows_per_win) {
        const int64_t rend = rw + rows_per_win < r1 ? rw + rows_per_win : r1;
        for (int x0 = 0; x0 < nx; x0 += kBwdWin) {
            const int xlen = whole ? nx : (nx - x0 < kBwdWin ? nx - x0 : kBwdWin);
            const int xle = (xlen + 1) & ~1;
            const int len = whole ? (int)(rend - rw) * nxe : xle;
            __syncthreads();
            for (int i = threadIdx.x; i < len; i += kBwdThreads) {
                const int rr = whole ? i / nxe : 0;
                const int k = i - rr * nxe;  // entry within the row (piece)
                const bool pad = k >= xlen;
                const int ix = x0 + (pad ? xlen - 1 : k);
                const int64_t q = (rw + rr) * nx + ix;
                wf[4 * (i >> 1) + (i & 1)] = -__fmaf_rn((float)ix + 0.5f, a.g.h[0], a.g.lo[0]);
                wf[4 * (i >> 1) + 2 + (i & 1)] = !pad && DV_INB(q, a.nq, kSiteBwdUpstream) ? a.upstream[q] : 0.f;
            }
            __syncthreads();
            const int64_t nr = whole ? rend - rw : 1;
            for (int64_t rr = 0; rr < nr; ++rr) {
                const int64_t row = rw + rr;
                const int iy = (int)(row % ny), iz = (int)(row / ny);
                const float qy = __fmaf_rn((float)iy + 0.5f, a.g.h[1], a.g.lo[1]);
                const float qz = __fmaf_rn((float)iz + 0.5f, a.g.h[2], a.g.lo[2]);
                visit(qy, qz, whole ? rr * nxe : (int64_t)0, xle);
            }
            if (whole) break;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Grid adjoint from the faces' edges. The derivative of one face's solid angle (Eq. (7)) with
// respect to its vertices depends only on the face's boundary, its three directed edges: for an
// edge p -> r of the face, with a = p - q and b = r - q,
//   dOmega/dp += (b x a) / (|a| (|a||b| + a.b)),   dOmega/dr += (b x a) / (|b| (|a||b| + a.b))
// (the closed form of winding_bnd.cu applied to one triangle, equal to the chain rule through
// Eq. (7) for q off the face). For the two faces of an edge-sharing pair, A = (p0, p1, p2) and
// B = (p2, p1, p3) in the canonical orientation, the shared edge is p1 -> p2 in A and p2 -> p1 in
// B, whose terms are exact negatives: the pair's derivative is the sum over the quad's four edges
// p0 -> p1, p2 -> p0 (A) and p1 -> p3, p3 -> p2 (B, times B's orientation sign sB = +-1) plus the
// shared edge p1 -> p2 with multiplicity 1 - sB (0 unless B's input orientation is reversed).
// Every (pair, query) is still evaluated; per one the four distances (one MUFU reciprocal square
// root each) serve four edges, each one dot, |a||b| + a.b, one MUFU reciprocal and four sums.
// With d = r - p, b x a = d x a = d x b, so the term at either endpoint is its c times d x (its own
// offset from q), and an edge needs only V_p = sum g c_p a and V_r = sum g c_r b
// (c_p = 1/(|a| (|a||b| + a.b)), c_r with |b|): per grid row the packed sums of g c and g c a_x for
// two x-adjacent queries at a time (a_y, a_z are constant along the row and enter as a_y S, a_z S),
// folded per row into Kahan sums in shared memory (offsets from the endpoint, not absolute
// coordinates, so the sums do not depend on where the mesh sits). At the end the thread forms in FP64
// dL/dp = m/(4 pi) d x V_p, dL/dr = m/(4 pi) d x V_r and writes each vertex's
// share into the gradient slots of the pair's faces (A's slot gets A's edges and the shared edge,
// B's slot B's edges); the gather sums the slots per vertex, so the per-vertex sums are the
// derivative, while a single slot is not that face's own derivative.
constexpr int kEdgeSlots = 6;  // per directed edge: V_p (3), V_r (3)

// Edge tables: pair (4 points, edges 0-3 the quad, 4 the shared edge) and single face (3 edges).
template <int NP>
__device__ __forceinline__ constexpr int edge_start(int k) {
    return NP == 4 ? (k == 0 ? 0 : k == 1 ? 2 : k == 2 ? 1 : k == 3 ? 3 : 1) : (k == 0 ? 0 : k == 1 ? 1 : 2);
}
template <int NP>
__device__ __forceinline__ constexpr int edge_end(int k) {
    return NP == 4 ? (k == 0 ? 1 : k == 1 ? 0 : k == 2 ? 3 : k == 3 ? 2 : 2) : (k == 0 ? 1 : k == 1 ? 2 : 0);
}

// Packed per-row sums of one directed edge: g c and g c o_x (o = P - q, the endpoint's offset) at
// its start (p) and its end (r).
struct EdgeRow2 {
    float2 Sp, Xp, Sr, Xr;
};

// The NP points of a pair or face, their per-row (y, z) parts and the edges' per-row dot parts.
template <int NP, int NE>
struct EdgeRowConst {
    float2 px[NP];  // point x, broadcast to both halves
    float2 L[NP];   // (y - qy)^2 + (z - qz)^2
    float2 P[NE];   // (y_p - qy)(y_r - qy) + (z_p - qz)(z_r - qz) of each edge
};

// One row (or piece) of packed query pairs from the window: every edge's four sums. Software
// pipelined: the next pair's offsets, squared distances and MUFU reciprocal square roots are
// issued before the current pair's edge work.
template <int NP, int NE>
__device__ __forceinline__ void edges_row2(const EdgeRowConst<NP, NE> &C, const float *wf, int64_t i0, int xlen,
                                           EdgeRow2 (&R)[NE]) {
#pragma unroll
    for (int k = 0; k < NE; ++k) R[k].Sp = R[k].Xp = R[k].Sr = R[k].Xr = make_float2(0.f, 0.f);
    const float4 *wp = reinterpret_cast<const float4 *>(wf) + (i0 >> 1);
    const int n = xlen / 2;
    float2 x[NP], m[NP], iv[NP], g;
    {
        const float4 q = wp[0];
        const float2 nqx = make_float2(q.x, q.y);
        g = make_float2(q.z, q.w);
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            x[k] = __fadd2_rn(C.px[k], nqx);
            m[k] = __ffma2_rn(x[k], x[k], C.L[k]);
            iv[k] = make_float2(rsqrt_approx(m[k].x), rsqrt_approx(m[k].y));
        }
    }
#pragma unroll 1
    for (int p = 0; p < n; ++p) {
        // next pair (the last iteration recomputes its own pair; its results are not used)
        const float4 qn = wp[p + 1 < n ? p + 1 : p];
        const float2 nqxn = make_float2(qn.x, qn.y), gn = make_float2(qn.z, qn.w);
        float2 xn[NP], mn[NP], ivn[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            xn[k] = __fadd2_rn(C.px[k], nqxn);
            mn[k] = __ffma2_rn(xn[k], xn[k], C.L[k]);
            ivn[k] = make_float2(rsqrt_approx(mn[k].x), rsqrt_approx(mn[k].y));
        }
        float2 l[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) l[k] = __fmul2_rn(m[k], iv[k]);
#pragma unroll
        for (int k = 0; k < NE; ++k) {
            const int s = edge_start<NP>(k), e = edge_end<NP>(k);
            const float2 t = __ffma2_rn(l[s], l[e], __ffma2_rn(x[s], x[e], C.P[k]));  // |a||b| + a.b
            const float2 c = __fmul2_rn(g, make_float2(rcp_approx(t.x), rcp_approx(t.y)));
            const float2 cp = __fmul2_rn(c, iv[s]), cr = __fmul2_rn(c, iv[e]);
            R[k].Sp = __fadd2_rn(R[k].Sp, cp);
            R[k].Xp = __ffma2_rn(cp, x[s], R[k].Xp);
            R[k].Sr = __fadd2_rn(R[k].Sr, cr);
            R[k].Xr = __ffma2_rn(cr, x[e], R[k].Xr);
        }
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            x[k] = xn[k];
            m[k] = mn[k];
            iv[k] = ivn[k];
        }
        g = gn;
    }
}

// The guarded scalar path of one row (or piece) and one edge: rows that pass close to one of the
// thread's edges (t from edge_t) and rows whose packed sums are not finite (a query at an endpoint
// or on the edge segment, where the derivative does not exist: those pairs are skipped). Returns
// the row's S_p, sum g c_p a_x, S_r, sum g c_r b_x.
__device__ __noinline__ float4 edge_row_guarded(float px, float py, float pz, float rx, float ry, float rz, float qy,
                                               float qz, const float *wf, int64_t i0, int xlen) {
    const float ay = py - qy, az = pz - qz, by = ry - qy, bz = rz - qz;
    const float dx = rx - px, dy = ry - py, dz = rz - pz;
    float sp = 0.f, sr = 0.f, xp = 0.f, xr = 0.f;
    for (int ix = 0; ix < xlen; ++ix) {
        const float nqx = win_nqx(wf, i0 + ix), g = win_g(wf, i0 + ix);
        const float ax = px + nqx, bx = rx + nqx;
        const float la2 = fmaf(ax, ax, fmaf(ay, ay, az * az)), lb2 = fmaf(bx, bx, fmaf(by, by, bz * bz));
        if (!(la2 > 0.f) || !(lb2 > 0.f)) continue;
        const float la = sqrtf(la2), lb = sqrtf(lb2);
        const float t = edge_t(ax, ay, az, la, lb, fmaf(ax, bx, fmaf(ay, by, az * bz)), dx, dy, dz);
        if (!(t > 1e-30f * la * lb)) continue;
        const float c = g / t, cp = c / la, cr = c / lb;
        sp += cp;
        sr += cr;
        xp = fmaf(cp, ax, xp);
        xr = fmaf(cr, bx, xr);
    }
    return make_float4(sp, xp, sr, xr);
}

// Fold one edge's row sums into its 6 Kahan slots V_p = sum g c_p a and V_r = sum g c_r b, whose y
// and z parts are the row's constant offsets times S: (sum g c_p a_x, a_y S_p, a_z S_p), ...
__device__ __forceinline__ void fold_edge(float2 (*ks)[kBwdThreads], int edge, float sp, float xp, float sr, float xr,
                                          float ay, float az, float by, float bz) {
    const int t = threadIdx.x;
    float2 (*k)[kBwdThreads] = ks + kEdgeSlots * edge;
    kahan_sm(&k[0][t], xp);
    kahan_sm(&k[1][t], ay * sp);
    kahan_sm(&k[2][t], az * sp);
    kahan_sm(&k[3][t], xr);
    kahan_sm(&k[4][t], by * sr);
    kahan_sm(&k[5][t], bz * sr);
}

// m/(4 pi) (r - p) x V for both endpoints of edge `edge` (FP64, from its Kahan slots): with
// d = r - p, b x a = d x a = d x b, so the start gets d x V_p and the end d x V_r.
__device__ __forceinline__ void edge_grad(float2 (*ks)[kBwdThreads], int edge, const double (&p)[3],
                                          const double (&r)[3], double m, double (&gp)[3], double (&gr)[3]) {
    const int t = threadIdx.x;
    float2 (*k)[kBwdThreads] = ks + kEdgeSlots * edge;
    double v[kEdgeSlots];
#pragma unroll
    for (int i = 0; i < kEdgeSlots; ++i) v[i] = (double)k[i][t].x - (double)k[i][t].y;
    const double w = m * (0.5 * kInv2PiD);
    const double d[3] = {r[0] - p[0], r[1] - p[1], r[2] - p[2]};
    const double *Vp = v, *Vr = v + 3;
    gp[0] += w * (d[1] * Vp[2] - d[2] * Vp[1]);
    gp[1] += w * (d[2] * Vp[0] - d[0] * Vp[2]);
    gp[2] += w * (d[0] * Vp[1] - d[1] * Vp[0]);
    gr[0] += w * (d[1] * Vr[2] - d[2] * Vr[1]);
    gr[1] += w * (d[2] * Vr[0] - d[0] * Vr[2]);
    gr[2] += w * (d[0] * Vr[1] - d[1] * Vr[0]);
}

// Every row of the CTA's split for the NP points and NE edges of this thread: packed rows, the
// guarded path for the others, folded into the edges' Kahan slots.
template <int NP, int NE>
__device__ __forceinline__ void edges_all_rows(const BwdArgs &a, float *wf, float2 (*ks)[kBwdThreads],
                                               const float (&X)[NP], const float (&Y)[NP], const float (&Z)[NP]) {
#pragma unroll
    for (int k = 0; k < kEdgeSlots * NE; ++k) ks[k][threadIdx.x] = make_float2(0.f, 0.f);
    for_each_row(a, wf, [&](float qy, float qz, int64_t i0, int xlen) {
        float y[NP], z[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            y[k] = Y[k] - qy;
            z[k] = Z[k] - qz;
        }
        bool near = false;
#pragma unroll
        for (int k = 0; k < NE; ++k) {
            const int s = edge_start<NP>(k), e = edge_end<NP>(k);
            const float dx = X[e] - X[s], dy = Y[e] - Y[s], dz = Z[e] - Z[s];
            near |= row_near_edge(y[s], z[s], y[e], z[e], fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        }
        bool ok = false;
        if (!near) {
            EdgeRowConst<NP, NE> C;
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                C.px[k] = bc2(X[k]);
                C.L[k] = bc2(fmaf(y[k], y[k], z[k] * z[k]));
            }
#pragma unroll
            for (int k = 0; k < NE; ++k) {
                const int s = edge_start<NP>(k), e = edge_end<NP>(k);
                C.P[k] = bc2(fmaf(y[s], y[e], z[s] * z[e]));
            }
            EdgeRow2 R[NE];
            edges_row2<NP, NE>(C, wf, i0, xlen, R);
            float t = 0.f;
#pragma unroll
            for (int k = 0; k < NE; ++k)
                t += ((R[k].Sp.x + R[k].Sp.y) + (R[k].Xp.x + R[k].Xp.y)) + ((R[k].Sr.x + R[k].Sr.y) + (R[k].Xr.x + R[k].Xr.y));
            ok = isfinite(t);
            if (ok) {
                // the row offsets again, from an opaque copy of (qy, qz): the compiler would
                // otherwise keep all 2 NP of them live through the packed loop
                float qy2 = qy, qz2 = qz;
                asm volatile("" : "+f"(qy2), "+f"(qz2));
#pragma unroll
                for (int k = 0; k < NE; ++k) {
                    const int s = edge_start<NP>(k), e = edge_end<NP>(k);
                    fold_edge(ks, k, R[k].Sp.x + R[k].Sp.y, R[k].Xp.x + R[k].Xp.y, R[k].Sr.x + R[k].Sr.y,
                              R[k].Xr.x + R[k].Xr.y, Y[s] - qy2, Z[s] - qz2, Y[e] - qy2, Z[e] - qz2);
                }
            }
        }
        if (!ok) {
            float qy2 = qy, qz2 = qz;
            asm volatile("" : "+f"(qy2), "+f"(qz2));
#pragma unroll
            for (int k = 0; k < NE; ++k) {
                const int s = edge_start<NP>(k), e = edge_end<NP>(k);
                const float4 v = edge_row_guarded(X[s], Y[s], Z[s], X[e], Y[e], Z[e], qy2, qz2, wf, i0, xlen);
                fold_edge(ks, k, v.x, v.y, v.z, v.w, Y[s] - qy2, Z[s] - qz2, Y[e] - qy2, Z[e] - qz2);
            }
        }
    });
}

__device__ __forceinline__ void write_pair_edges(const BwdArgs &a, float2 (*ks)[kBwdThreads], const PairRec &P,
                                                 const int32_t *tp, bool five);
__device__ __forceinline__ void write_single_edges(const BwdArgs &a, float2 (*ks)[kBwdThreads], const FaceRec &r,
                                                   int64_t f);

// A CTA of edge-sharing face pairs, edge form: thread t owns pair t. When a pair of the warp has
// B reversed, the warp also evaluates the shared edge (multiplicity 1 - sB: 2 for that pair, 0 for
// the others); otherwise the four quad edges suffice.
__device__ __forceinline__ void bwd_grid_pairs_edges(const BwdArgs &a, float *wf, float2 (*ks)[kBwdThreads]) {
    const int64_t idx = (int64_t)blockIdx.x * kBwdThreads + threadIdx.x;
    const int64_t ic = idx < a.np ? idx : a.np - 1;
    const PairRec P = a.prec[DV_INB(ic, a.np, kSiteBwdRecord) ? ic : 0];
    const int32_t *tp = a.ptopo + 8 * ic;
    const int code = tp[6];
    const bool rev = (code >> 12) & 1;
    const float X[4] = {P.r0.x, P.r1.x, P.r2.x, P.r3.x};
    const float Y[4] = {P.r0.y, P.r1.y, P.r2.y, P.r3.y};
    const float Z[4] = {P.r0.z, P.r1.z, P.r2.z, P.r3.z};
    const bool five = __syncthreads_or(rev) != 0;  // CTA-uniform: the row loop has barriers
    if (five)
        edges_all_rows<4, 5>(a, wf, ks, X, Y, Z);
    else
        edges_all_rows<4, 4>(a, wf, ks, X, Y, Z);
    if (idx < a.np) write_pair_edges(a, ks, P, tp, five);
}

// The gradient of a pair (edge form) from its edges' Kahan slots, FP64, into the slots of its
// two faces in face_grad (split blockIdx.y).
__device__ __forceinline__ void write_pair_edges(const BwdArgs &a, float2 (*ks)[kBwdThreads], const PairRec &P,
                                                 const int32_t *tp, bool five) {
    const int code = tp[6];
    const bool rev = (code >> 12) & 1;
    const double p[4][3] = {{P.r0.x, P.r0.y, P.r0.z}, {P.r1.x, P.r1.y, P.r1.z},
                            {P.r2.x, P.r2.y, P.r2.z}, {P.r3.x, P.r3.y, P.r3.z}};
    const double sB = rev ? -1.0 : 1.0;
    // slot A: canonical corners (p0, p1, p2); slot B: (p2, p1, p3)
    double gA[3][3] = {}, gB[3][3] = {};
    edge_grad(ks, 0, p[0], p[1], 1.0, gA[0], gA[1]);  // p0 -> p1
    edge_grad(ks, 1, p[2], p[0], 1.0, gA[2], gA[0]);  // p2 -> p0
    edge_grad(ks, 2, p[1], p[3], sB, gB[1], gB[2]);   // p1 -> p3
    edge_grad(ks, 3, p[3], p[2], sB, gB[2], gB[0]);   // p3 -> p2
    if (five && rev) edge_grad(ks, 4, p[1], p[2], 1.0 - sB, gA[1], gA[2]);  // shared p1 -> p2
    float *out = a.face_grad + (int64_t)blockIdx.y * a.nf * 9;
    const int cA = code & 63, cB = (code >> 6) & 63;
    if (DV_INB(tp[4], a.nf, kSiteBwdFaceGrad)) {
        float *o = out + (int64_t)tp[4] * 9;
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int c = 0; c < 3; ++c) o[3 * ((cA >> (2 * j)) & 3) + c] = (float)gA[j][c];
    }
    if (DV_INB(tp[5], a.nf, kSiteBwdFaceGrad)) {
        float *o = out + (int64_t)tp[5] * 9;
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int c = 0; c < 3; ++c) o[3 * ((cB >> (2 * j)) & 3) + c] = (float)gB[j][c];
    }
}

// A CTA of single faces, edge form: thread t owns one face (unpaired list, or face index order).
__device__ __forceinline__ void bwd_grid_singles_edges(const BwdArgs &a, float *wf, float2 (*ks)[kBwdThreads]) {
    const int64_t count = a.singles ? a.nsingle : a.nf;
    const int64_t idx = ((int64_t)blockIdx.x - a.pblocks) * kBwdThreads + threadIdx.x;
    const int64_t ic = idx < count ? idx : count - 1;
    int64_t f = a.singles ? (DV_INB(ic, a.nsingle, kSiteBwdRecord) ? (int64_t)a.singles[ic] : 0) : ic;
    if (!DV_INB(f, a.nf, kSiteBwdRecord)) f = 0;
    const FaceRec r = a.rec[f];
    const float X[3] = {r.r0.x, r.r1.x, r.r2.x}, Y[3] = {r.r0.y, r.r1.y, r.r2.y}, Z[3] = {r.r0.z, r.r1.z, r.r2.z};
    edges_all_rows<3, 3>(a, wf, ks, X, Y, Z);
    if (idx < count && DV_INB(f, a.nf, kSiteBwdFaceGrad)) write_single_edges(a, ks, r, f);
}

// The gradient of a single face (edge form) from its edges' Kahan slots, FP64, into its slot.
__device__ __forceinline__ void write_single_edges(const BwdArgs &a, float2 (*ks)[kBwdThreads], const FaceRec &r,
                                                   int64_t f) {
    const double p[3][3] = {{r.r0.x, r.r0.y, r.r0.z}, {r.r1.x, r.r1.y, r.r1.z}, {r.r2.x, r.r2.y, r.r2.z}};
    double g[3][3] = {};
    edge_grad(ks, 0, p[0], p[1], 1.0, g[0], g[1]);
    edge_grad(ks, 1, p[1], p[2], 1.0, g[1], g[2]);
    edge_grad(ks, 2, p[2], p[0], 1.0, g[2], g[0]);
    float *o = a.face_grad + ((int64_t)blockIdx.y * a.nf + f) * 9;
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int c = 0; c < 3; ++c) o[3 * j + c] = (float)g[j][c];
}

// Grid adjoint (edge form): CTAs [0, pblocks) take edge-sharing face pairs, the rest single faces.
// Dynamic shared memory: the query window, then 5 edges x 6 Kahan slots per thread.
constexpr size_t kBwdGridSmem = sizeof(float) * 2 * kBwdWin + sizeof(float2) * 5 * kEdgeSlots * kBwdThreads;

__global__ void __launch_bounds__(kBwdThreads, 3) bwd_grid_kernel(const BwdArgs a) {
    extern __shared__ __align__(16) float bwd_smem[];
    float *wf = bwd_smem;
    float2(*ks)[kBwdThreads] = reinterpret_cast<float2(*)[kBwdThreads]>(bwd_smem + 2 * kBwdWin);
    if ((int64_t)blockIdx.x < a.pblocks)
        bwd_grid_pairs_edges(a, wf, ks);
    else
        bwd_grid_singles_edges(a, wf, ks);
}

// Query lists: queries staged in windows, taken in chunks of kListChunk (plain FP32 sums within a
// chunk, Kahan across chunks).
constexpr int kListChunk = 128;

__device__ __forceinline__ float2 dot2(float2 ax, float2 ay, float2 az, float2 bx, float2 by, float2 bz) {
    return __ffma2_rn(az, bz, __ffma2_rn(ay, by, __fmul2_rn(ax, bx)));
}

// Query i of a window laid out in pairs: (-x, -y, -z, g).
__device__ __forceinline__ float4 list_query(const float4 *win, int i) {
    const float *wf = reinterpret_cast<const float *>(win) + 8 * (i >> 1) + (i & 1);
    return make_float4(wf[0], wf[2], wf[4], wf[6]);
}

// Query windows of a split (padded to an even count with g = 0), in chunks of kListChunk
// queries: visit(c0, c1, len) for window entries c0 .. c1 - 1 (entries >= len are padding).
template <typename ChunkFn>
__device__ __forceinline__ void for_each_chunk(const BwdArgs &a, float4 *win, ChunkFn &&visit) {
    const int64_t q0 = (int64_t)blockIdx.y * a.rows_per_split;
    const int64_t q1 = q0 + a.rows_per_split < a.nq ? q0 + a.rows_per_split : a.nq;
    for (int64_t w0 = q0; w0 < q1; w0 += kBwdWin / 2) {
        const int len = (int)(q1 - w0 < kBwdWin / 2 ? q1 - w0 : kBwdWin / 2);
        const int len2 = (len + 1) & ~1;
        __syncthreads();
        for (int i = threadIdx.x; i < len2; i += kBwdThreads) {
            int64_t k = w0 + (i < len ? i : len - 1);
            if (!DV_INB(k, a.nq, kSiteBwdUpstream)) k = 0;
            float *wf = reinterpret_cast<float *>(win) + 8 * (i >> 1) + (i & 1);
            wf[0] = -a.queries[3 * k];
            wf[2] = -a.queries[3 * k + 1];
            wf[4] = -a.queries[3 * k + 2];
            wf[6] = i < len ? a.upstream[k] : 0.0f;
        }
        __syncthreads();
        for (int c0 = 0; c0 < len2; c0 += kListChunk)
            visit(c0, c0 + kListChunk < len2 ? c0 + kListChunk : len2, len);
    }
}

// List adjoint from the faces' edges: the same edge terms as the grid path, with the full q of each
// query (no row sharing). With d = r - p, b x a = d x a = d x b, so the term at either endpoint is
// its c times d x (its own offset from q): per edge and endpoint only the vector sum V = sum c o of
// the endpoint's offsets o = P - q is kept (3 packed sums), and d x V is formed at the end in FP64.
// Per chunk the sums fold into 6 Kahan slots per edge.

struct EdgeList2 {
    float2 Vp[3], Vr[3];
};

// Returns the OR of the bit patterns of every t + kNearCos a.b: its sign bit is set when a query
// of the chunk is near one of the edges (or a sum is NaN).
template <int NP, int NE>
__device__ __forceinline__ uint32_t edges_list_chunk(const float2 (&X)[NP], const float2 (&Y)[NP], const float2 (&Z)[NP],
                                                     const float4 *win, int c0, int c1, EdgeList2 (&R)[NE]) {
    uint32_t near = 0;
    const float2 kn = bc2(kNearCos);
#pragma unroll
    for (int k = 0; k < NE; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) R[k].Vp[c] = R[k].Vr[c] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int i = c0; i < c1; i += 2) {
        // window entries of a pair of queries: (-x0, -x1, -y0, -y1), (-z0, -z1, g0, g1)
        const float4 q0 = win[i], q1 = win[i + 1];
        const float2 nqx = make_float2(q0.x, q0.y), nqy = make_float2(q0.z, q0.w), nqz = make_float2(q1.x, q1.y);
        const float2 g = make_float2(q1.z, q1.w);
        float2 x[NP], y[NP], z[NP], l[NP], iv[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            x[k] = __fadd2_rn(X[k], nqx);
            y[k] = __fadd2_rn(Y[k], nqy);
            z[k] = __fadd2_rn(Z[k], nqz);
            const float2 m = dot2(x[k], y[k], z[k], x[k], y[k], z[k]);
            iv[k] = rsqrt2(m);
            l[k] = __fmul2_rn(m, iv[k]);
        }
#pragma unroll
        for (int k = 0; k < NE; ++k) {
            const int s = edge_start<NP>(k), e = edge_end<NP>(k);
            const float2 ab = dot2(x[s], y[s], z[s], x[e], y[e], z[e]);
            const float2 t = __ffma2_rn(l[s], l[e], ab);  // |a||b| + a.b
            const float2 chk = __ffma2_rn(kn, ab, t);
            near |= __float_as_uint(chk.x) | __float_as_uint(chk.y);
            const float2 c = __fmul2_rn(g, make_float2(rcp_approx(t.x), rcp_approx(t.y)));
            const float2 cp = __fmul2_rn(c, iv[s]), cr = __fmul2_rn(c, iv[e]);
            R[k].Vp[0] = __ffma2_rn(cp, x[s], R[k].Vp[0]);
            R[k].Vp[1] = __ffma2_rn(cp, y[s], R[k].Vp[1]);
            R[k].Vp[2] = __ffma2_rn(cp, z[s], R[k].Vp[2]);
            R[k].Vr[0] = __ffma2_rn(cr, x[e], R[k].Vr[0]);
            R[k].Vr[1] = __ffma2_rn(cr, y[e], R[k].Vr[1]);
            R[k].Vr[2] = __ffma2_rn(cr, z[e], R[k].Vr[2]);
        }
    }
    return near;
}

struct Edge6 {
    float v[kEdgeSlots];  // V_p (3), V_r (3)
};

// Guarded scalar recompute of one chunk for one edge (t from edge_t): chunks with a query near one
// of the thread's edges or with sums that are not finite. Skips queries at an endpoint or on the
// edge segment (no derivative there).
__device__ __noinline__ Edge6 edge_chunk_guarded(float px, float py, float pz, float rx, float ry, float rz,
                                                 const float4 *win, int c0, int ce) {
    Edge6 o;
#pragma unroll
    for (int k = 0; k < kEdgeSlots; ++k) o.v[k] = 0.f;
    const float dx = rx - px, dy = ry - py, dz = rz - pz;
    for (int i = c0; i < ce; ++i) {
        const float4 q = list_query(win, i);  // (-x, -y, -z, g)
        const float ax = px + q.x, ay = py + q.y, az = pz + q.z, bx = rx + q.x, by = ry + q.y, bz = rz + q.z;
        const float la2 = fmaf(ax, ax, fmaf(ay, ay, az * az)), lb2 = fmaf(bx, bx, fmaf(by, by, bz * bz));
        float ia, ib, c;
        if (!edge_coeffs(ax, ay, az, bx, by, bz, la2, lb2, dx, dy, dz, q.w, ia, ib, c)) continue;
        const float cp = c * ia, cr = c * ib;
        o.v[0] = fmaf(cp, ax, o.v[0]);
        o.v[1] = fmaf(cp, ay, o.v[1]);
        o.v[2] = fmaf(cp, az, o.v[2]);
        o.v[3] = fmaf(cr, bx, o.v[3]);
        o.v[4] = fmaf(cr, by, o.v[4]);
        o.v[5] = fmaf(cr, bz, o.v[5]);
    }
    return o;
}

// Every chunk of the CTA's split for this thread's NP points and NE edges, folded into the edges'
// Kahan slots (the guarded path for chunks with a query near an edge or sums that are not finite).
template <int NP, int NE>
__device__ __forceinline__ void edges_list_all(const BwdArgs &a, float4 *win, float2 (*ks)[kBwdThreads],
                                               const float (&X)[NP], const float (&Y)[NP], const float (&Z)[NP]) {
#pragma unroll
    for (int k = 0; k < kEdgeSlots * NE; ++k) ks[k][threadIdx.x] = make_float2(0.f, 0.f);
    float2 X2[NP], Y2[NP], Z2[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        X2[k] = bc2(X[k]);
        Y2[k] = bc2(Y[k]);
        Z2[k] = bc2(Z[k]);
    }
    for_each_chunk(a, win, [&](int c0, int c1, int len) {
        EdgeList2 R[NE];
        const uint32_t near = edges_list_chunk<NP, NE>(X2, Y2, Z2, win, c0, c1, R);
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < NE; ++k)
#pragma unroll
            for (int j = 0; j < 3; ++j) t += (R[k].Vp[j].x + R[k].Vp[j].y) + (R[k].Vr[j].x + R[k].Vr[j].y);
        const bool ok = isfinite(t) && !(near >> 31);
        const int th = threadIdx.x;
#pragma unroll
        for (int k = 0; k < NE; ++k) {
            float v[kEdgeSlots];
            if (ok) {
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    v[j] = R[k].Vp[j].x + R[k].Vp[j].y;
                    v[3 + j] = R[k].Vr[j].x + R[k].Vr[j].y;
                }
            } else {
                const int s = edge_start<NP>(k), e = edge_end<NP>(k);
                const Edge6 gv = edge_chunk_guarded(X[s], Y[s], Z[s], X[e], Y[e], Z[e], win, c0, c1 < len ? c1 : len);
#pragma unroll
                for (int j = 0; j < kEdgeSlots; ++j) v[j] = gv.v[j];
            }
#pragma unroll
            for (int j = 0; j < kEdgeSlots; ++j) kahan_sm(&ks[kEdgeSlots * k + j][th], v[j]);
        }
    });
}

// Store the 3 x 3 gradient g (canonical corners) of a face into its slot, corner j at input corner
// (code >> 2j) & 3.
__device__ __forceinline__ void store_face_grad(float *o, const double (&g)[3][3], int code) {
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int c = 0; c < 3; ++c) o[3 * ((code >> (2 * j)) & 3) + c] = (float)g[j][c];
}

__device__ __forceinline__ void bwd_list_pairs_edges(const BwdArgs &a, float4 *win, float2 (*ks)[kBwdThreads]) {
    const int64_t idx = (int64_t)blockIdx.x * kBwdThreads + threadIdx.x;
    const int64_t ic = idx < a.np ? idx : a.np - 1;
    const PairRec P = a.prec[DV_INB(ic, a.np, kSiteBwdRecord) ? ic : 0];
    const int32_t *tp = a.ptopo + 8 * ic;
    const int code = tp[6];
    const bool rev = (code >> 12) & 1;
    const float X[4] = {P.r0.x, P.r1.x, P.r2.x, P.r3.x};
    const float Y[4] = {P.r0.y, P.r1.y, P.r2.y, P.r3.y};
    const float Z[4] = {P.r0.z, P.r1.z, P.r2.z, P.r3.z};
    const bool five = __syncthreads_or(rev) != 0;  // CTA-uniform: the chunk loop has barriers
    if (five)
        edges_list_all<4, 5>(a, win, ks, X, Y, Z);
    else
        edges_list_all<4, 4>(a, win, ks, X, Y, Z);
    if (idx >= a.np) return;
    const double p[4][3] = {{P.r0.x, P.r0.y, P.r0.z}, {P.r1.x, P.r1.y, P.r1.z},
                            {P.r2.x, P.r2.y, P.r2.z}, {P.r3.x, P.r3.y, P.r3.z}};
    const double sB = rev ? -1.0 : 1.0;
    double gA[3][3] = {}, gB[3][3] = {};  // A: (p0, p1, p2), B: (p2, p1, p3)
    edge_grad(ks, 0, p[0], p[1], 1.0, gA[0], gA[1]);
    edge_grad(ks, 1, p[2], p[0], 1.0, gA[2], gA[0]);
    edge_grad(ks, 2, p[1], p[3], sB, gB[1], gB[2]);
    edge_grad(ks, 3, p[3], p[2], sB, gB[2], gB[0]);
    if (five && rev) edge_grad(ks, 4, p[1], p[2], 1.0 - sB, gA[1], gA[2]);
    float *out = a.face_grad + (int64_t)blockIdx.y * a.nf * 9;
    if (DV_INB(tp[4], a.nf, kSiteBwdFaceGrad)) store_face_grad(out + (int64_t)tp[4] * 9, gA, code & 63);
    if (DV_INB(tp[5], a.nf, kSiteBwdFaceGrad)) store_face_grad(out + (int64_t)tp[5] * 9, gB, (code >> 6) & 63);
}

__device__ __forceinline__ void bwd_list_singles_edges(const BwdArgs &a, float4 *win, float2 (*ks)[kBwdThreads]) {
    const int64_t count = a.singles ? a.nsingle : a.nf;
    const int64_t idx = ((int64_t)blockIdx.x - a.pblocks) * kBwdThreads + threadIdx.x;
    const int64_t ic = idx < count ? idx : count - 1;
    int64_t f = a.singles ? (DV_INB(ic, a.nsingle, kSiteBwdRecord) ? (int64_t)a.singles[ic] : 0) : ic;
    if (!DV_INB(f, a.nf, kSiteBwdRecord)) f = 0;
    const FaceRec r = a.rec[f];
    const float X[3] = {r.r0.x, r.r1.x, r.r2.x}, Y[3] = {r.r0.y, r.r1.y, r.r2.y}, Z[3] = {r.r0.z, r.r1.z, r.r2.z};
    edges_list_all<3, 3>(a, win, ks, X, Y, Z);
    if (idx >= count || !DV_INB(f, a.nf, kSiteBwdFaceGrad)) return;
    const double p[3][3] = {{r.r0.x, r.r0.y, r.r0.z}, {r.r1.x, r.r1.y, r.r1.z}, {r.r2.x, r.r2.y, r.r2.z}};
    double g[3][3] = {};
    edge_grad(ks, 0, p[0], p[1], 1.0, g[0], g[1]);
    edge_grad(ks, 1, p[1], p[2], 1.0, g[1], g[2]);
    edge_grad(ks, 2, p[2], p[0], 1.0, g[2], g[0]);
    store_face_grad(a.face_grad + ((int64_t)blockIdx.y * a.nf + f) * 9, g, kCornersIdentity);
}

// List adjoint (edge form): CTAs [0, pblocks) take edge-sharing face pairs, the rest single faces.
// Dynamic shared memory: the query window (consecutive queries in pairs, each pair as (-x0, -x1,
// -y0, -y1), (-z0, -z1, g0, g1), so two 16-byte loads give the packed operands), then 5 edges x 6
// Kahan slots per thread.
constexpr size_t kBwdListSmem = sizeof(float4) * (kBwdWin / 2) + sizeof(float2) * 5 * kEdgeSlots * kBwdThreads;

__global__ void __launch_bounds__(kBwdThreads, 3) bwd_list_kernel(const BwdArgs a) {
    extern __shared__ __align__(16) float4 bwd_list_smem[];
    float4 *win = bwd_list_smem;
    float2(*ks)[kBwdThreads] = reinterpret_cast<float2(*)[kBwdThreads]>(bwd_list_smem + kBwdWin / 2);
    if ((int64_t)blockIdx.x < a.pblocks)
        bwd_list_pairs_edges(a, win, ks);
    else
        bwd_list_singles_edges(a, win, ks);
}

// Once per device (mesh creation calls it, outside any stream capture): the adjoint kernels'
// dynamic shared memory exceeds the 48 KB default.
// CTAs of the grid adjoint resident per SM on each device (from the occupancy calculator, set by
// prepare_backward_kernels; 0 = not known yet).
static std::atomic<int> g_bwd_resident[64];

cudaError_t prepare_backward_kernels() {
    static std::atomic<uint64_t> smem_set{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if (smem_set.load() & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(bwd_grid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdGridSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(bwd_list_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdListSmem);
    int resident = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, bwd_grid_kernel, kBwdThreads, kBwdGridSmem);
    if (e == cudaSuccess) {
        g_bwd_resident[dev & 63].store(resident);
        smem_set.fetch_or(bit);
    }
    return e;
}

// Fraction of the CTA slots the last wave leaves busy: total CTAs / (waves x slots).
static double wave_efficiency(int64_t ctas, int64_t slots) {
    const int64_t waves = (ctas + slots - 1) / slots;
    return (double)ctas / (double)(waves * slots);
}

BwdPlan plan_backward(int64_t nq, const BwdFaces &fc, bool grid, const GridF *g, int num_sms) {
    BwdPlan p{};
    p.threads = kBwdThreads;
    if (fc.prec) {
        p.pblocks = (fc.np + kBwdThreads - 1) / kBwdThreads;
        p.fblocks = p.pblocks + (fc.nsingle + kBwdThreads - 1) / kBwdThreads;
    } else {
        p.pblocks = 0;
        p.fblocks = (fc.nf + kBwdThreads - 1) / kBwdThreads;
    }
    const int64_t units = grid ? (int64_t)g->n[1] * g->n[2] : nq;  // rows or queries
    // 3 to 5 CTAs of 128 threads are resident per SM; aim for >= 4 waves in total.
    const int64_t target = 20LL * num_sms;
    int64_t ns = (target + p.fblocks - 1) / p.fblocks;
    // at least 16 rows (grid) or 512 queries (list) per split: on small problems more splits only
    // lengthen the per-vertex gather over splits
    const int64_t per_min = grid ? 16 : 512;
    if (ns > units / per_min) ns = units / per_min;
    if (ns < 1) ns = 1;
    if (ns > 4096) ns = 4096;
    // Every CTA carries the same work, so a last wave that fills few of the GPU's CTA slots
    // idles most SMs for a whole CTA time. Among up to 4x as many splits, take the fewest whose
    // waves fill at least 98 % of the slots (else the best filled), e.g. 799 face CTAs on 148 SMs
    // x 3: 4 splits fill 90 % (7.2 waves), 5 splits 99.97 % (9.0 waves).
    int dev = 0;
    cudaGetDevice(&dev);
    const int resident = g_bwd_resident[dev & 63].load();
    if (resident > 0) {
        const int64_t slots = (int64_t)resident * num_sms;
        int64_t hi = 4 * ns;
        if (hi > units / per_min) hi = units / per_min;
        if (hi > 4096) hi = 4096;
        int64_t best = ns;
        for (int64_t k = ns; k <= hi && wave_efficiency(p.fblocks * best, slots) < 0.98; ++k)
            if (wave_efficiency(p.fblocks * k, slots) > wave_efficiency(p.fblocks * best, slots)) best = k;
        ns = best;
    }
    p.rows_per_split = (units + ns - 1) / ns;
    p.nsplit = (int)((units + p.rows_per_split - 1) / p.rows_per_split);
    if (p.nsplit < 1) p.nsplit = 1;
    return p;
}

cudaError_t launch_backward(const BwdPlan &p, const BwdFaces &fc, const GridF *g, const float *queries, int64_t nq,
                            const float *upstream, float *face_grad, const LaunchCtx &ctx) {
    BwdArgs a{};
    a.rec = fc.rec;
    a.nf = fc.nf;
    if (g) a.g = *g;
    a.queries = queries;
    a.nq = nq;
    a.upstream = upstream;
    a.rows_per_split = p.rows_per_split;
    a.face_grad = face_grad;
    a.err = ctx.d_err;
    a.pblocks = p.pblocks;
    if (p.pblocks > 0) {
        a.prec = fc.prec;
        a.ptopo = fc.ptopo;
        a.np = fc.np;
        a.singles = fc.singles;
        a.nsingle = fc.nsingle;
    }
    dim3 grid((unsigned)p.fblocks, (unsigned)p.nsplit);
    const char *name = queries ? "bwd_list" : "bwd_grid";
    const cudaError_t e = prepare_backward_kernels();
    if (e != cudaSuccess) return e;
    prof_begin(name, ctx.stream);
    if (queries)
        bwd_list_kernel<<<grid, kBwdThreads, kBwdListSmem, ctx.stream>>>(a);
    else
        bwd_grid_kernel<<<grid, kBwdThreads, kBwdGridSmem, ctx.stream>>>(a);
    count_launch();
    prof_end(name, ctx.stream);
    return cudaGetLastError();
}

}  // namespace dv
