// Adjoint of the winding number: dL/dV = sum_q g_q dw(q)/dV, every (query, face) pair.
//
// Two exact formulations of the per-face derivative of Eq. (7), w = (1/4pi) sum Omega:
//
// Grid queries (bwd_grid_kernel) -- from each face's edges. The solid angle of a triangle depends
// only on its boundary, so for an edge p -> r of the face (a = p - q, b = r - q)
//   dOmega/dp += (b x a) / (|a| (|a||b| + a.b)),   dOmega/dr += (b x a) / (|b| (|a||b| + a.b)).
// A thread owns two faces that share an edge (consecutive faces of a strip, paired on the host);
// their shared edge's terms cancel, leaving the quad's four edges: per query four distances, four
// dots and four reciprocals serve both faces, and every edge keeps four packed row sums (details at
// bwd_grid_pairs_edges). Faces left unpaired run alone (three edges).
//
// Query lists (bwd_list_kernel) -- the chain rule through N and D. With a = v0 - q, b = v1 - q,
// c = v2 - q, N = a.n (n = (v1-v0)x(v2-v0)), D as in the forward and Omega = 2 ATAN2(N, D):
//   dw = (1/2pi) (D dN - N dD) / (N^2 + D^2)
//   dN/da = b x c,  dN/db = c x a,  dN/dc = a x b
//   dD/da = (a/|a|)(|b||c| + b.c) + b|c| + c|b|   (and cyclically)
// Writing b = e1 + a, c = e2 + a (e1 = v1 - v0, e2 = v2 - v0), every per-query vector term is
// (scalar) x a or a constant vector, so per face only these sums are needed:
//   T_cD = sum cD, T_P = sum cN|a|, T_Q = sum cN|b|, T_R = sum cN|c|,
//   T_ab = sum alpha_b, T_ac = sum alpha_c,
//   U_cD = sum cD a, U_a = sum W_a a, U_b = sum W_b a, U_c = sum W_c a,
// with cD = g D/(N^2+D^2), cN = g N/(N^2+D^2), alpha_a = cN (|b||c| + b.c)/|a| (cyclic),
// W_a = alpha_a + T_R-term + T_Q-term etc. Then
//   dL/dv0 = k [T_cD n + (e1 - e2) x U_cD - T_R e1 - T_Q e2 - U_a]
//   dL/dv1 = k [e2 x U_cD - T_ab e1 - T_P e2 - U_b]
//   dL/dv2 = k [-e1 x U_cD - T_P e1 - T_ac e2 - U_c],   k = 1/(2 pi).
// Edge-sharing face pairs share the four distances and five edge dots here too.
//
// Both kernels are face-parallel: a thread owns its faces, streams the queries (uniform across the
// warp) through shared memory, keeps per-face (per-edge) sums in FP32 with Kahan compensation in
// shared memory, and writes per-split face gradients that the gather kernel (pack.cu) sums over
// splits and incident faces in FP64, in a fixed order.
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

struct FaceF {
    float v0x, v0y, v0z, v1x, v1y, v1z, v2x, v2y, v2z, nx, ny, nz;
};

struct RowB {
    float ay, az, La, Lb, Lc, Pab, Pbc, Pca, Nyz;
};

__device__ __forceinline__ RowB row_b(const FaceF &F, float qy, float qz) {
    RowB r;
    r.ay = F.v0y - qy;
    r.az = F.v0z - qz;
    const float by = F.v1y - qy, bz = F.v1z - qz, cy = F.v2y - qy, cz = F.v2z - qz;
    r.La = fmaf(r.ay, r.ay, r.az * r.az);
    r.Lb = fmaf(by, by, bz * bz);
    r.Lc = fmaf(cy, cy, cz * cz);
    r.Pab = fmaf(r.ay, by, r.az * bz);
    r.Pbc = fmaf(by, cy, bz * cz);
    r.Pca = fmaf(cy, r.ay, cz * r.az);
    r.Nyz = fmaf(r.ay, F.ny, r.az * F.nz);
    return r;
}

// One pair: accumulate the 7 row scalars S and their x-weighted versions X.
template <bool GUARD>
__device__ __forceinline__ void bwd_pair(const FaceF &F, const RowB &R, float qx, float g, float (&S)[7],
                                         float (&X)[7]) {
    const float ax = F.v0x - qx, bx = F.v1x - qx, cx = F.v2x - qx;
    float la2 = fmaf(ax, ax, R.La), lb2 = fmaf(bx, bx, R.Lb), lc2 = fmaf(cx, cx, R.Lc);
    if (GUARD) {
        la2 = fmaxf(la2, 1e-30f);
        lb2 = fmaxf(lb2, 1e-30f);
        lc2 = fmaxf(lc2, 1e-30f);
    }
    const float ia = rsqrt_approx(la2), ib = rsqrt_approx(lb2), ic = rsqrt_approx(lc2);
    const float la = la2 * ia, lb = lb2 * ib, lc = lc2 * ic;  // multiply, not a second MUFU op per vertex
    const float ab = fmaf(ax, bx, R.Pab), bc = fmaf(bx, cx, R.Pbc), ca = fmaf(cx, ax, R.Pca);
    const float N = fmaf(ax, F.nx, R.Nyz);
    const float tc = fmaf(la, lb, ab);  // |a||b| + a.b, also the numerator of alpha_c
    float D = tc * lc;
    D = fmaf(la, bc, D);
    D = fmaf(lb, ca, D);
    const float den = fmaf(N, N, D * D);
    float r = rcp_approx(den);
    if (GUARD) r = den >= 1.17549435e-38f ? r : 0.0f;
    const float gr = g * r;
    const float cD = gr * D, cN = gr * N;
    const float P = cN * la, Qb = cN * lb, Rc = cN * lc;
    const float alA = cN * (fmaf(lb, lc, bc) * ia);
    const float alB = cN * (fmaf(lc, la, ca) * ib);
    const float alC = cN * (tc * ic);
    S[0] += cD;
    S[1] += P;
    S[2] += Qb;
    S[3] += Rc;
    S[4] += alA;
    S[5] += alB;
    S[6] += alC;
    X[0] = fmaf(cD, ax, X[0]);
    X[1] = fmaf(P, ax, X[1]);
    X[2] = fmaf(Qb, ax, X[2]);
    X[3] = fmaf(Rc, ax, X[3]);
    X[4] = fmaf(alA, ax, X[4]);
    X[5] = fmaf(alB, ax, X[5]);
    X[6] = fmaf(alC, ax, X[6]);
}

// Packed FP32x2 helpers (Blackwell FFMA2/FADD2/FMUL2 take two queries per instruction; the MUFU
// reciprocal square roots and reciprocals stay scalar).
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 rsqrt2(float2 v) { return make_float2(rsqrt_approx(v.x), rsqrt_approx(v.y)); }

// Face A (which = 0) or B (which = 1) of a pair as a face alone, in its canonical corner order.
__device__ __forceinline__ FaceF pair_face(const PairRec &P, int which) {
    FaceF F;
    const float4 a = which ? P.r2 : P.r0, c = which ? P.r3 : P.r2;
    F.v0x = a.x; F.v0y = a.y; F.v0z = a.z;
    F.v1x = P.r1.x; F.v1y = P.r1.y; F.v1z = P.r1.z;
    F.v2x = c.x; F.v2y = c.y; F.v2z = c.z;
    F.nx = which ? P.r3.w : P.r0.w;
    F.ny = which ? P.r4.x : P.r1.w;
    F.nz = which ? P.r4.y : P.r2.w;
    return F;
}

// Per-face sums, kept in shared memory (touched once per row or chunk of queries, so the
// registers of the pair loop stay free): slot k of thread t is ks[k][t] = (sum, compensation),
// k = 0..5 for T_cD, T_P, T_Q, T_R, T_ab, T_ac and 6 + 3i + j for U_i component j
// (U_cD, U_a, U_b, U_c).
constexpr int kFaceSlots = 18;

__device__ __forceinline__ void kahan_sm(float2 *slot, float x) {
    float2 k = *slot;
    const float y = __fsub_rn(x, k.y);
    const float t = __fadd_rn(k.x, y);
    k.y = __fsub_rn(__fsub_rn(t, k.x), y);
    k.x = t;
    *slot = k;
}

__device__ __forceinline__ void fold_sm(float2 (*ks)[kBwdThreads], const float (&S)[7], const float (&X)[7], float ay,
                                        float az) {
    const int t = threadIdx.x;
    kahan_sm(&ks[0][t], S[0]);
    kahan_sm(&ks[1][t], S[1]);
    kahan_sm(&ks[2][t], S[2]);
    kahan_sm(&ks[3][t], S[3]);
    kahan_sm(&ks[4][t], S[5]);
    kahan_sm(&ks[5][t], S[6]);
    const float ws[4] = {S[0], S[4] + S[3] + S[2], S[5] + S[1] + S[3], S[6] + S[2] + S[1]};
    const float wx[4] = {X[0], X[4] + X[3] + X[2], X[5] + X[1] + X[3], X[6] + X[2] + X[1]};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        kahan_sm(&ks[6 + 3 * i][t], wx[i]);
        kahan_sm(&ks[7 + 3 * i][t], ay * ws[i]);
        kahan_sm(&ks[8 + 3 * i][t], az * ws[i]);
    }
}

__device__ __forceinline__ FaceF load_face(const FaceRec *rec, int64_t f) {
    const FaceRec r = rec[f];
    FaceF F;
    F.v0x = r.r0.x; F.v0y = r.r0.y; F.v0z = r.r0.z;
    F.v1x = r.r1.x; F.v1y = r.r1.y; F.v1z = r.r1.z;
    F.v2x = r.r2.x; F.v2y = r.r2.y; F.v2z = r.r2.z;
    F.nx = r.r0.w * (1.0f / kNormalScale);
    F.ny = r.r1.w * (1.0f / kNormalScale);
    F.nz = r.r2.w * (1.0f / kNormalScale);
    return F;
}

// Combine the face sums (T, U as compensated FP64 values) into the 9 gradient components (FP64
// arithmetic) and store them: corner c of F goes to the input corner (code >> 2c) & 3 of the face,
// times sign (-1 when F is the face with its orientation reversed).
constexpr int kCornersIdentity = 0 | 1 << 2 | 2 << 4;

__device__ __forceinline__ void write_face_grad_d(const FaceF &F, const double (&T)[6], const double (&U)[4][3],
                                                  float *out, int code = kCornersIdentity, double sign = 1.0) {
    const double e1[3] = {(double)F.v1x - F.v0x, (double)F.v1y - F.v0y, (double)F.v1z - F.v0z};
    const double e2[3] = {(double)F.v2x - F.v0x, (double)F.v2y - F.v0y, (double)F.v2z - F.v0z};
    const double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const double *u = U[0];
    const double d[3] = {e1[0] - e2[0], e1[1] - e2[1], e1[2] - e2[2]};
    const double dxu[3] = {d[1] * u[2] - d[2] * u[1], d[2] * u[0] - d[0] * u[2], d[0] * u[1] - d[1] * u[0]};
    const double e2xu[3] = {e2[1] * u[2] - e2[2] * u[1], e2[2] * u[0] - e2[0] * u[2], e2[0] * u[1] - e2[1] * u[0]};
    const double e1xu[3] = {e1[1] * u[2] - e1[2] * u[1], e1[2] * u[0] - e1[0] * u[2], e1[0] * u[1] - e1[1] * u[0]};
    for (int k = 0; k < 3; ++k) {
        const double g0 = T[0] * n[k] + dxu[k] - T[3] * e1[k] - T[2] * e2[k] - U[1][k];
        const double g1 = e2xu[k] - T[4] * e1[k] - T[1] * e2[k] - U[2][k];
        const double g2 = -e1xu[k] - T[1] * e1[k] - T[5] * e2[k] - U[3][k];
        const double k2 = sign * kInv2PiD;
        out[3 * (code & 3) + k] = (float)(g0 * k2);
        out[3 * ((code >> 2) & 3) + k] = (float)(g1 * k2);
        out[3 * ((code >> 4) & 3) + k] = (float)(g2 * k2);
    }
}

__device__ __forceinline__ void write_face_grad_sm(const FaceF &F, float2 (*ks)[kBwdThreads], float *out,
                                                   int code = kCornersIdentity, double sign = 1.0) {
    const int t = threadIdx.x;
    double T[6], U[4][3];
    for (int i = 0; i < 6; ++i) T[i] = (double)ks[i][t].x - (double)ks[i][t].y;
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 3; ++k) U[i][k] = (double)ks[6 + 3 * i + k][t].x - (double)ks[6 + 3 * i + k][t].y;
    write_face_grad_d(F, T, U, out, code, sign);
}

// Staged queries of a window, in pairs: for query i (pair p = i/2, k = i%2) the window holds
// -x_i at wf[4p + k] and the upstream g_i at wf[4p + 2 + k], so one 16-byte load gives the
// packed (-x, -x') and (g, g') operands of two consecutive queries.
__device__ __forceinline__ float win_nqx(const float *wf, int64_t i) { return wf[4 * (i >> 1) + (i & 1)]; }
__device__ __forceinline__ float win_g(const float *wf, int64_t i) { return wf[4 * (i >> 1) + 2 + (i & 1)]; }

// Rows of the grid are processed in windows of whole rows when a row fits the window (packed
// pairs of queries when the row length is even); longer rows go in pieces through the guarded
// path. visit(qy, qz, i0, xlen, packed) handles one row (or piece) whose queries sit at window
// indices i0 .. i0 + xlen - 1.
template <typename RowFn>
__device__ __forceinline__ void for_each_row(const BwdArgs &a, float *wf, RowFn &&visit) {
    const int nx = a.g.n[0], ny = a.g.n[1];
    const int64_t nrows = (int64_t)a.g.n[1] * a.g.n[2];
    const int64_t r0 = (int64_t)blockIdx.y * a.rows_per_split;
    const int64_t r1 = r0 + a.rows_per_split < nrows ? r0 + a.rows_per_split : nrows;
    const bool whole = nx <= kBwdWin;
    const bool packed = whole && (nx % 2 == 0);
    const int rows_per_win = whole ? kBwdWin / nx : 1;
    for (int64_t rw = r0; rw < r1; rw += rows_per_win) {
        const int64_t rend = rw + rows_per_win < r1 ? rw + rows_per_win : r1;
        for (int x0 = 0; x0 < nx; x0 += kBwdWin) {
            const int xlen = whole ? nx : (nx - x0 < kBwdWin ? nx - x0 : kBwdWin);
            const int64_t len = whole ? (rend - rw) * nx : xlen;
            const int64_t base = rw * nx + (whole ? 0 : x0);
            __syncthreads();
            for (int64_t i = threadIdx.x; i < len; i += kBwdThreads) {
                const int ix = whole ? (int)(i % nx) : x0 + (int)i;
                wf[4 * (i >> 1) + (i & 1)] = -__fmaf_rn((float)ix + 0.5f, a.g.h[0], a.g.lo[0]);
                wf[4 * (i >> 1) + 2 + (i & 1)] = DV_INB(base + i, a.nq, kSiteBwdUpstream) ? a.upstream[base + i] : 0.f;
            }
            __syncthreads();
            const int64_t nr = whole ? rend - rw : 1;
            for (int64_t rr = 0; rr < nr; ++rr) {
                const int64_t row = rw + rr;
                const int iy = (int)(row % ny), iz = (int)(row / ny);
                const float qy = __fmaf_rn((float)iy + 0.5f, a.g.h[1], a.g.lo[1]);
                const float qz = __fmaf_rn((float)iz + 0.5f, a.g.h[2], a.g.lo[2]);
                visit(qy, qz, whole ? rr * nx : (int64_t)0, xlen, packed);
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
// Because b x a = r x p - (r - p) x q is linear in q, an edge needs only
//   S_p = sum g c_p, Q_p = sum g c_p q, S_r, Q_r   (c_p = 1/(|a| (|a||b| + a.b)), c_r with |b|):
// per grid row the packed sums of g c and g c (-x) for two x-adjacent queries at a time, folded
// per row into Kahan sums in shared memory (y and z enter as qy S, qz S). At the end the thread
// forms in FP64 dL/dp = m/(4 pi) [(r x p) S_p - (r - p) x Q_p] (r likewise) and writes each vertex's
// share into the gradient slots of the pair's faces (A's slot gets A's edges and the shared edge,
// B's slot B's edges); the gather sums the slots per vertex, so only the per-vertex sum is that of
// the face formula, not each slot.
constexpr int kEdgeSlots = 8;  // per directed edge: S_p, Q_p (3), S_r, Q_r (3)

// Edge tables: pair (4 points, edges 0-3 the quad, 4 the shared edge) and single face (3 edges).
template <int NP>
__device__ __forceinline__ constexpr int edge_start(int k) {
    return NP == 4 ? (k == 0 ? 0 : k == 1 ? 2 : k == 2 ? 1 : k == 3 ? 3 : 1) : (k == 0 ? 0 : k == 1 ? 1 : 2);
}
template <int NP>
__device__ __forceinline__ constexpr int edge_end(int k) {
    return NP == 4 ? (k == 0 ? 1 : k == 1 ? 0 : k == 2 ? 3 : k == 3 ? 2 : 2) : (k == 0 ? 1 : k == 1 ? 2 : 0);
}

// Packed per-row sums of one directed edge: g c and g c (-x) at its start (p) and its end (r).
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

// One row (or piece) of packed query pairs from the window: every edge's four sums.
template <int NP, int NE>
__device__ __forceinline__ void edges_row2(const EdgeRowConst<NP, NE> &C, const float *wf, int64_t i0, int xlen,
                                           EdgeRow2 (&R)[NE]) {
#pragma unroll
    for (int k = 0; k < NE; ++k) R[k].Sp = R[k].Xp = R[k].Sr = R[k].Xr = make_float2(0.f, 0.f);
    const float4 *wp = reinterpret_cast<const float4 *>(wf) + (i0 >> 1);
#pragma unroll 2
    for (int p = 0; p < xlen / 2; ++p) {
        const float4 q = wp[p];
        const float2 nqx = make_float2(q.x, q.y), g = make_float2(q.z, q.w);
        float2 x[NP], l[NP], iv[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            x[k] = __fadd2_rn(C.px[k], nqx);
            const float2 m = __ffma2_rn(x[k], x[k], C.L[k]);
            iv[k] = make_float2(rsqrt_approx(m.x), rsqrt_approx(m.y));
            l[k] = __fmul2_rn(m, iv[k]);
        }
#pragma unroll
        for (int k = 0; k < NE; ++k) {
            const int s = edge_start<NP>(k), e = edge_end<NP>(k);
            const float2 t = __ffma2_rn(l[s], l[e], __ffma2_rn(x[s], x[e], C.P[k]));  // |a||b| + a.b
            const float2 c = __fmul2_rn(g, make_float2(rcp_approx(t.x), rcp_approx(t.y)));
            const float2 cp = __fmul2_rn(c, iv[s]), cr = __fmul2_rn(c, iv[e]);
            R[k].Sp = __fadd2_rn(R[k].Sp, cp);
            R[k].Xp = __ffma2_rn(cp, nqx, R[k].Xp);
            R[k].Sr = __fadd2_rn(R[k].Sr, cr);
            R[k].Xr = __ffma2_rn(cr, nqx, R[k].Xr);
        }
    }
}

// The guarded scalar path of one row (or piece) and one edge: rows with an odd number of queries,
// pieces of long rows, and rows whose packed sums are not finite (a query at an endpoint or on the
// edge segment, where the derivative does not exist: those pairs are skipped). Returns the row's
// S_p, sum g c_p (-x), S_r, sum g c_r (-x).
__device__ __noinline__ float4 edge_row_guarded(float px, float py, float pz, float rx, float ry, float rz, float qy,
                                               float qz, const float *wf, int64_t i0, int xlen) {
    const float ay = py - qy, az = pz - qz, by = ry - qy, bz = rz - qz;
    float sp = 0.f, sr = 0.f, xp = 0.f, xr = 0.f;
    for (int ix = 0; ix < xlen; ++ix) {
        const float nqx = win_nqx(wf, i0 + ix), g = win_g(wf, i0 + ix);
        const float ax = px + nqx, bx = rx + nqx;
        const float la2 = fmaf(ax, ax, fmaf(ay, ay, az * az)), lb2 = fmaf(bx, bx, fmaf(by, by, bz * bz));
        if (!(la2 > 0.f) || !(lb2 > 0.f)) continue;
        const float la = sqrtf(la2), lb = sqrtf(lb2);
        const float t = fmaf(la, lb, fmaf(ax, bx, fmaf(ay, by, az * bz)));
        if (!(t > 1e-30f * la * lb)) continue;
        const float c = g / t, cp = c / la, cr = c / lb;
        sp += cp;
        sr += cr;
        xp = fmaf(cp, nqx, xp);
        xr = fmaf(cr, nqx, xr);
    }
    return make_float4(sp, xp, sr, xr);
}

// Fold one edge's row sums into its 8 Kahan slots: S_p, Q_p = (sum g c_p x, qy S_p, qz S_p), S_r, Q_r.
__device__ __forceinline__ void fold_edge(float2 (*ks)[kBwdThreads], int edge, float sp, float nxp, float sr,
                                          float nxr, float qy, float qz) {
    const int t = threadIdx.x;
    float2 (*k)[kBwdThreads] = ks + kEdgeSlots * edge;
    kahan_sm(&k[0][t], sp);
    kahan_sm(&k[1][t], -nxp);
    kahan_sm(&k[2][t], qy * sp);
    kahan_sm(&k[3][t], qz * sp);
    kahan_sm(&k[4][t], sr);
    kahan_sm(&k[5][t], -nxr);
    kahan_sm(&k[6][t], qy * sr);
    kahan_sm(&k[7][t], qz * sr);
}

// m/(4 pi) [(r x p) S - (r - p) x Q] for both endpoints of edge `edge` (FP64, from its Kahan slots),
// added to gp (the start p) and gr (the end r).
__device__ __forceinline__ void edge_grad(float2 (*ks)[kBwdThreads], int edge, const double (&p)[3],
                                          const double (&r)[3], double m, double (&gp)[3], double (&gr)[3]) {
    const int t = threadIdx.x;
    float2 (*k)[kBwdThreads] = ks + kEdgeSlots * edge;
    double v[kEdgeSlots];
#pragma unroll
    for (int i = 0; i < kEdgeSlots; ++i) v[i] = (double)k[i][t].x - (double)k[i][t].y;
    const double w = m * (0.5 * kInv2PiD);
    const double d[3] = {r[0] - p[0], r[1] - p[1], r[2] - p[2]};
    const double rxp[3] = {r[1] * p[2] - r[2] * p[1], r[2] * p[0] - r[0] * p[2], r[0] * p[1] - r[1] * p[0]};
    const double *Qp = v + 1, *Qr = v + 5;
    const double dxp[3] = {d[1] * Qp[2] - d[2] * Qp[1], d[2] * Qp[0] - d[0] * Qp[2], d[0] * Qp[1] - d[1] * Qp[0]};
    const double dxr[3] = {d[1] * Qr[2] - d[2] * Qr[1], d[2] * Qr[0] - d[0] * Qr[2], d[0] * Qr[1] - d[1] * Qr[0]};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        gp[c] += w * (rxp[c] * v[0] - dxp[c]);
        gr[c] += w * (rxp[c] * v[4] - dxr[c]);
    }
}

// Every row of the CTA's split for the NP points and NE edges of this thread: packed rows, the
// guarded path for the others, folded into the edges' Kahan slots.
template <int NP, int NE>
__device__ __forceinline__ void edges_all_rows(const BwdArgs &a, float *wf, float2 (*ks)[kBwdThreads],
                                               const float (&X)[NP], const float (&Y)[NP], const float (&Z)[NP]) {
#pragma unroll
    for (int k = 0; k < kEdgeSlots * NE; ++k) ks[k][threadIdx.x] = make_float2(0.f, 0.f);
    for_each_row(a, wf, [&](float qy, float qz, int64_t i0, int xlen, bool packed) {
        float y[NP], z[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            y[k] = Y[k] - qy;
            z[k] = Z[k] - qz;
        }
        bool ok = false;
        if (packed) {
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
#pragma unroll
                for (int k = 0; k < NE; ++k)
                    fold_edge(ks, k, R[k].Sp.x + R[k].Sp.y, R[k].Xp.x + R[k].Xp.y, R[k].Sr.x + R[k].Sr.y,
                              R[k].Xr.x + R[k].Xr.y, qy, qz);
            }
        }
        if (!ok) {
#pragma unroll
            for (int k = 0; k < NE; ++k) {
                const int s = edge_start<NP>(k), e = edge_end<NP>(k);
                const float4 v = edge_row_guarded(X[s], Y[s], Z[s], X[e], Y[e], Z[e], qy, qz, wf, i0, xlen);
                fold_edge(ks, k, v.x, v.y, v.z, v.w, qy, qz);
            }
        }
    });
}

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
    if (idx >= a.np) return;
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
    if (idx >= count || !DV_INB(f, a.nf, kSiteBwdFaceGrad)) return;
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
// Dynamic shared memory: the query window, then 5 edges x 8 Kahan slots per thread.
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

// List path: arbitrary queries, so no row sharing. Two queries per packed FP32x2 instruction;
// per pair of queries the adjoint terms go straight into the 6 T sums and the 4 a-weighted
// combinations U_i = sum W_i a (12 FMAs), plain FP32 over chunks of kListChunk queries, folded
// per chunk into the Kahan face sums (shared memory). A chunk whose sums are not finite (a query
// on a vertex or an edge line) is recomputed by the guarded scalar path.
constexpr int kListChunk = 128;

struct FaceL2 {
    float2 v0x, v0y, v0z, v1x, v1y, v1z, v2x, v2y, v2z, nx, ny, nz;
};

// The list-path adjoint terms of one face for two queries, from the distances, their reciprocals,
// the edge dots, N and the offsets (ax, ay, az) of the face's first vertex.
__device__ __forceinline__ void list_face2(float2 la, float2 lb, float2 lc, float2 ia, float2 ib, float2 ic,
                                           float2 ab, float2 bcd, float2 ca, float2 N, float2 ax, float2 ay,
                                           float2 az, float2 g, float2 (&T)[6], float2 (&U)[4][3]) {
    // |a||b| + a.b written lb * la, so that for the two faces of a pair the shared edge's term
    // (the other face's lb * lc + b.c) is the same expression, computed once
    const float2 tc = __ffma2_rn(lb, la, ab);
    float2 D = __fmul2_rn(tc, lc);
    D = __ffma2_rn(la, bcd, D);
    D = __ffma2_rn(lb, ca, D);
    const float2 den = __ffma2_rn(N, N, __fmul2_rn(D, D));
    const float2 gr = __fmul2_rn(g, make_float2(rcp_approx(den.x), rcp_approx(den.y)));
    const float2 cD = __fmul2_rn(gr, D), cN = __fmul2_rn(gr, N);
    const float2 kA = __fmul2_rn(__ffma2_rn(lb, lc, bcd), ia);
    const float2 kB = __fmul2_rn(__ffma2_rn(lc, la, ca), ib);
    const float2 kC = __fmul2_rn(tc, ic);
    T[0] = __fadd2_rn(T[0], cD);
    T[1] = __ffma2_rn(cN, la, T[1]);
    T[2] = __ffma2_rn(cN, lb, T[2]);
    T[3] = __ffma2_rn(cN, lc, T[3]);
    T[4] = __ffma2_rn(cN, kB, T[4]);
    T[5] = __ffma2_rn(cN, kC, T[5]);
    // W_a = alpha_a + cN |c| + cN |b| = cN (k_a + |b| + |c|), cyclically
    const float2 W[4] = {cD, __fmul2_rn(cN, __fadd2_rn(kA, __fadd2_rn(lc, lb))),
                         __fmul2_rn(cN, __fadd2_rn(kB, __fadd2_rn(la, lc))),
                         __fmul2_rn(cN, __fadd2_rn(kC, __fadd2_rn(lb, la)))};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        U[i][0] = __ffma2_rn(W[i], ax, U[i][0]);
        U[i][1] = __ffma2_rn(W[i], ay, U[i][1]);
        U[i][2] = __ffma2_rn(W[i], az, U[i][2]);
    }
}

__device__ __forceinline__ void bwd_list_pair2(const FaceL2 &F, float4 q0, float4 q1, float2 (&T)[6],
                                               float2 (&U)[4][3]) {
    // window entries of a pair of queries: (-x0, -x1, -y0, -y1), (-z0, -z1, g0, g1)
    const float2 nqx = make_float2(q0.x, q0.y), nqy = make_float2(q0.z, q0.w), nqz = make_float2(q1.x, q1.y);
    const float2 g = make_float2(q1.z, q1.w);
    const float2 ax = __fadd2_rn(F.v0x, nqx), ay = __fadd2_rn(F.v0y, nqy), az = __fadd2_rn(F.v0z, nqz);
    const float2 bx = __fadd2_rn(F.v1x, nqx), by = __fadd2_rn(F.v1y, nqy), bz = __fadd2_rn(F.v1z, nqz);
    const float2 cx = __fadd2_rn(F.v2x, nqx), cy = __fadd2_rn(F.v2y, nqy), cz = __fadd2_rn(F.v2z, nqz);
    const float2 la2 = __ffma2_rn(az, az, __ffma2_rn(ay, ay, __fmul2_rn(ax, ax)));
    const float2 lb2 = __ffma2_rn(bz, bz, __ffma2_rn(by, by, __fmul2_rn(bx, bx)));
    const float2 lc2 = __ffma2_rn(cz, cz, __ffma2_rn(cy, cy, __fmul2_rn(cx, cx)));
    const float2 ia = rsqrt2(la2), ib = rsqrt2(lb2), ic = rsqrt2(lc2);
    const float2 la = __fmul2_rn(la2, ia), lb = __fmul2_rn(lb2, ib), lc = __fmul2_rn(lc2, ic);
    const float2 ab = __ffma2_rn(az, bz, __ffma2_rn(ay, by, __fmul2_rn(ax, bx)));
    const float2 bcd = __ffma2_rn(bz, cz, __ffma2_rn(by, cy, __fmul2_rn(bx, cx)));
    const float2 ca = __ffma2_rn(cz, az, __ffma2_rn(cy, ay, __fmul2_rn(cx, ax)));
    const float2 N = __ffma2_rn(az, F.nz, __ffma2_rn(ay, F.ny, __fmul2_rn(ax, F.nx)));
    list_face2(la, lb, lc, ia, ib, ic, ab, bcd, ca, N, ax, ay, az, g, T, U);
}

// Two edge-sharing faces (A = (p0, p1, p2), B = (p2, p1, p3)) against two queries: four distances
// and five dots for both faces.
struct PairL2 {
    float2 x[4], y[4], z[4];
    float2 nA[3], nB[3];
};

__device__ __forceinline__ PairL2 pair_l2(const PairRec &P) {
    PairL2 Q;
    const float4 r[4] = {P.r0, P.r1, P.r2, P.r3};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        Q.x[i] = bc2(r[i].x);
        Q.y[i] = bc2(r[i].y);
        Q.z[i] = bc2(r[i].z);
    }
    Q.nA[0] = bc2(P.r0.w);
    Q.nA[1] = bc2(P.r1.w);
    Q.nA[2] = bc2(P.r2.w);
    Q.nB[0] = bc2(P.r3.w);
    Q.nB[1] = bc2(P.r4.x);
    Q.nB[2] = bc2(P.r4.y);
    return Q;
}

__device__ __forceinline__ float2 dot2(float2 ax, float2 ay, float2 az, float2 bx, float2 by, float2 bz) {
    return __ffma2_rn(az, bz, __ffma2_rn(ay, by, __fmul2_rn(ax, bx)));
}

__device__ __forceinline__ void bwd_list_quad2(const PairL2 &P, float4 q0, float4 q1, float2 (&TA)[6],
                                               float2 (&UA)[4][3], float2 (&TB)[6], float2 (&UB)[4][3]) {
    const float2 nqx = make_float2(q0.x, q0.y), nqy = make_float2(q0.z, q0.w), nqz = make_float2(q1.x, q1.y);
    const float2 g = make_float2(q1.z, q1.w);
    float2 x[4], y[4], z[4], l[4], r[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        x[i] = __fadd2_rn(P.x[i], nqx);
        y[i] = __fadd2_rn(P.y[i], nqy);
        z[i] = __fadd2_rn(P.z[i], nqz);
        const float2 m = dot2(x[i], y[i], z[i], x[i], y[i], z[i]);
        r[i] = rsqrt2(m);
        l[i] = __fmul2_rn(m, r[i]);
    }
    const float2 d01 = dot2(x[0], y[0], z[0], x[1], y[1], z[1]);
    const float2 d12 = dot2(x[1], y[1], z[1], x[2], y[2], z[2]);
    const float2 d20 = dot2(x[2], y[2], z[2], x[0], y[0], z[0]);
    const float2 d13 = dot2(x[1], y[1], z[1], x[3], y[3], z[3]);
    const float2 d32 = dot2(x[3], y[3], z[3], x[2], y[2], z[2]);
    const float2 NA = dot2(x[0], y[0], z[0], P.nA[0], P.nA[1], P.nA[2]);
    const float2 NB = dot2(x[2], y[2], z[2], P.nB[0], P.nB[1], P.nB[2]);
    list_face2(l[0], l[1], l[2], r[0], r[1], r[2], d01, d12, d20, NA, x[0], y[0], z[0], g, TA, UA);
    list_face2(l[2], l[1], l[3], r[2], r[1], r[3], d12, d13, d32, NB, x[2], y[2], z[2], g, TB, UB);
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

__device__ __forceinline__ bool finite_tu(const float2 (&T)[6], const float2 (&U)[4][3]) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 6; ++k) t += T[k].x + T[k].y;
#pragma unroll
    for (int i = 0; i < 4; ++i) t += U[i][0].x + U[i][0].y + U[i][1].x + U[i][1].y + U[i][2].x + U[i][2].y;
    return isfinite(t);
}

__device__ __forceinline__ void fold_list(float2 (*ks)[kBwdThreads], const float2 (&T)[6], const float2 (&U)[4][3]) {
    const int th = threadIdx.x;
#pragma unroll
    for (int k = 0; k < 6; ++k) kahan_sm(&ks[k][th], T[k].x + T[k].y);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) kahan_sm(&ks[6 + 3 * i + j][th], U[i][j].x + U[i][j].y);
}

// Guarded scalar recompute of one chunk for one face, one query at a time (a chunk whose packed
// sums are not finite: a query on a vertex or an edge line).
__device__ __noinline__ void list_guarded(const FaceF F, const float4 *win, int c0, int ce,
                                          float2 (*ks)[kBwdThreads]) {
    for (int i = c0; i < ce; ++i) {
        const float4 q = list_query(win, i);
        const RowB R = row_b(F, -q.y, -q.z);
        float S[7], X[7];
#pragma unroll
        for (int k = 0; k < 7; ++k) S[k] = X[k] = 0.f;
        bwd_pair<true>(F, R, -q.x, q.w, S, X);
        fold_sm(ks, S, X, R.ay, R.az);
    }
}

__device__ __forceinline__ void bwd_list_singles(const BwdArgs &a, float4 *win, float2 (*ks)[kBwdThreads]) {
    const int64_t count = a.singles ? a.nsingle : a.nf;
    const int64_t idx = ((int64_t)blockIdx.x - a.pblocks) * kBwdThreads + threadIdx.x;
    const int64_t ic = idx < count ? idx : count - 1;
    int64_t f = a.singles ? (DV_INB(ic, a.nsingle, kSiteBwdRecord) ? (int64_t)a.singles[ic] : 0) : ic;
    if (!DV_INB(f, a.nf, kSiteBwdRecord)) f = 0;
    const FaceF F = load_face(a.rec, f);
    FaceL2 F2;
    F2.v0x = bc2(F.v0x); F2.v0y = bc2(F.v0y); F2.v0z = bc2(F.v0z);
    F2.v1x = bc2(F.v1x); F2.v1y = bc2(F.v1y); F2.v1z = bc2(F.v1z);
    F2.v2x = bc2(F.v2x); F2.v2y = bc2(F.v2y); F2.v2z = bc2(F.v2z);
    F2.nx = bc2(F.nx); F2.ny = bc2(F.ny); F2.nz = bc2(F.nz);
#pragma unroll
    for (int k = 0; k < kFaceSlots; ++k) ks[k][threadIdx.x] = make_float2(0.f, 0.f);
    for_each_chunk(a, win, [&](int c0, int c1, int len) {
        float2 T[6], U[4][3];
#pragma unroll
        for (int k = 0; k < 6; ++k) T[k] = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < 4; ++i) U[i][0] = U[i][1] = U[i][2] = make_float2(0.f, 0.f);
#pragma unroll 2
        for (int i = c0; i < c1; i += 2) bwd_list_pair2(F2, win[i], win[i + 1], T, U);  // i even: one pair
        if (finite_tu(T, U))
            fold_list(ks, T, U);
        else
            list_guarded(F, win, c0, c1 < len ? c1 : len, ks);
    });
    if (idx < count && DV_INB(f, a.nf, kSiteBwdFaceGrad))
        write_face_grad_sm(F, ks, a.face_grad + ((int64_t)blockIdx.y * a.nf + f) * 9);
}

__device__ __forceinline__ void bwd_list_pairs(const BwdArgs &a, float4 *win, float2 (*ks)[kBwdThreads]) {
    const int64_t idx = (int64_t)blockIdx.x * kBwdThreads + threadIdx.x;
    const int64_t ic = idx < a.np ? idx : a.np - 1;
    const PairRec P = a.prec[DV_INB(ic, a.np, kSiteBwdRecord) ? ic : 0];
    const PairL2 P2 = pair_l2(P);
    float2(*ksB)[kBwdThreads] = ks + kFaceSlots;
#pragma unroll
    for (int k = 0; k < 2 * kFaceSlots; ++k) ks[k][threadIdx.x] = make_float2(0.f, 0.f);
    for_each_chunk(a, win, [&](int c0, int c1, int len) {
        float2 TA[6], UA[4][3], TB[6], UB[4][3];
#pragma unroll
        for (int k = 0; k < 6; ++k) TA[k] = TB[k] = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < 4; ++i) UA[i][0] = UA[i][1] = UA[i][2] = UB[i][0] = UB[i][1] = UB[i][2] = make_float2(0.f, 0.f);
        for (int i = c0; i < c1; i += 2) bwd_list_quad2(P2, win[i], win[i + 1], TA, UA, TB, UB);
        const int ce = c1 < len ? c1 : len;
        if (finite_tu(TA, UA))
            fold_list(ks, TA, UA);
        else
            list_guarded(pair_face(P, 0), win, c0, ce, ks);
        if (finite_tu(TB, UB))
            fold_list(ksB, TB, UB);
        else
            list_guarded(pair_face(P, 1), win, c0, ce, ksB);
    });
    if (idx < a.np) {
        const int32_t *t = a.ptopo + 8 * idx;
        const int code = t[6];
        float *out = a.face_grad + (int64_t)blockIdx.y * a.nf * 9;
        if (DV_INB(t[4], a.nf, kSiteBwdFaceGrad))
            write_face_grad_sm(pair_face(P, 0), ks, out + (int64_t)t[4] * 9, code & 63, 1.0);
        if (DV_INB(t[5], a.nf, kSiteBwdFaceGrad))
            write_face_grad_sm(pair_face(P, 1), ksB, out + (int64_t)t[5] * 9, (code >> 6) & 63,
                               (code >> 12) & 1 ? -1.0 : 1.0);
    }
}

// List adjoint: CTAs [0, pblocks) take edge-sharing face pairs, the rest single faces. Dynamic
// shared memory: the query window (consecutive queries in pairs, each pair as (-x0, -x1, -y0,
// -y1), (-z0, -z1, g0, g1), so two 16-byte loads give the packed operands), then 2 x 18
// face-sum slots per thread.
constexpr size_t kBwdListSmem = sizeof(float4) * (kBwdWin / 2) + sizeof(float2) * 2 * kFaceSlots * kBwdThreads;

__global__ void __launch_bounds__(kBwdThreads, 3) bwd_list_kernel(const BwdArgs a) {
    extern __shared__ __align__(16) float4 bwd_list_smem[];
    float4 *win = bwd_list_smem;
    float2(*ks)[kBwdThreads] = reinterpret_cast<float2(*)[kBwdThreads]>(bwd_list_smem + kBwdWin / 2);
    if ((int64_t)blockIdx.x < a.pblocks)
        bwd_list_pairs(a, win, ks);
    else
        bwd_list_singles(a, win, ks);
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
