// Forward pass: generalized winding number over all (query, face) pairs, FP32.
//
// Per pair (Eq. (7) in unnormalized form, Eq. (8) for the quadrant):
//   a = v0 - q, b = v1 - q, c = v2 - q
//   N = a . n_f                    (= det(a, b, c), n_f = (v1 - v0) x (v2 - v0))
//   D = |a||b||c| + (a.b)|c| + (b.c)|a| + (c.a)|b|
//   sum += ATAN2(N, D)             (= Omega / 2)
// and w = sum / (2 pi)  (Eq. (5)).
//
// Design for sm_103a:
//   * Main path (grid and list queries, FP32 / Kahan): the faces are visited in the
//     vertex-sharing strip order of strips.cu. Strip events (32 B: vertex + face normal) stream
//     through shared memory in tiles of 96 moved by 1-D TMA bulk copies (cp.async.bulk +
//     mbarrier, 4-stage ring, bounded waits); every warp reads each event as a broadcast. Each
//     event brings one vertex: |v - q| (one MUFU square root) and the dot with the previous
//     vertex are computed once and kept in three rotating register slots, so a face costs one
//     square root, two dots and D = (|V||P1| + V.P1)|P2| + |V|(P1.P2) + |P1|(V.P2).
//   * Voxel-centre queries are generated in registers from the grid index; each thread owns
//     QX consecutive x positions (paired into packed FP32x2 instructions) on QY rows at one z;
//     the (y, z) parts of offsets, lengths, dots and N are computed once per event per row.
//   * ATAN2 fast path: with the normal pre-scaled by 8, the test D > |8N| selects |N/D| < 1/8,
//     where atan(N/D) = v P(v^2), v = 8N/D, P a degree-2 Remez polynomial (atan_poly.h). Terms
//     failing the test contribute 0 on the fast path; if any lane of the warp has such a term
//     for the current face, a slow path recomputes N and D with the same operations and adds
//     ATAN2 via atan2f for exactly those terms.
//   * Compensated summation: plain FP32 within a tile, Kahan across tiles (state in shared
//     memory).
//   * Split over the event range (grid.y) for small query counts, each split starting with two
//     warm-up events; partial sums (sum, -compensation) go to a scratch buffer and are reduced
//     in FP64, in fixed order, by split_reduce_kernel.
//   * Face order (48 B face records, tiles of 64) remains for the FP16 ablation and the
//     allocation-free entry point (noalloc.cu), which build no strip order.
#include <cuda_fp16.h>
#include <math.h>
#include <string.h>

#include "dv_internal.cuh"

namespace dv {

constexpr int kFwdThreads = 256;
constexpr int kTileFaces = 64;
constexpr int kStages = 4;

struct FwdArgs {
    const FaceRec *rec;
    int64_t nf;
    const StripRec *srec;  // strip events (grid FP32 path); null: face order
    int64_t ne;
    GridF g;
    const float *queries;  // list path: [nq][3]; grid path: null
    int64_t nq;
    int64_t faces_per_split;
    int nsplit;
    float2 *partial;  // [nsplit][nq] when nsplit > 1
    float *w_out;
    uint8_t *occ_out;
    const uint8_t *near_flag;  // null unless re-evaluation is on
    int *flag_list;
    int *flag_count;
    int *err;
    int skip_tile;     // self-test: tile (per CTA) that thread 0 never issues; -1 = none
    uint64_t wait_ns;  // limit of each bounded wait
};

// ---------------------------------------------------------------------------------------------
// Per-pair arithmetic. Inputs are the x components of a, b, c plus the (y,z) partial sums.
struct PairOut {
    float N8, D;  // 8 det(a, b, c) and D
};

__device__ __forceinline__ PairOut pair_terms(float ax, float bx, float cx, float La, float Lb, float Lc, float Pab,
                                              float Pbc, float Pca, float Nyz, float n8x, float &la2_min) {
    const float la2 = __fmaf_rn(ax, ax, La);
    const float lb2 = __fmaf_rn(bx, bx, Lb);
    const float lc2 = __fmaf_rn(cx, cx, Lc);
    const float la = sqrt_approx(la2);
    const float lb = sqrt_approx(lb2);
    const float lc = sqrt_approx(lc2);
    const float ab = __fmaf_rn(ax, bx, Pab);
    const float bc = __fmaf_rn(bx, cx, Pbc);
    const float ca = __fmaf_rn(cx, ax, Pca);
    PairOut o;
    o.N8 = __fmaf_rn(ax, n8x, Nyz);
    float D = __fmul_rn(__fmaf_rn(la, lb, ab), lc);
    D = __fmaf_rn(la, bc, D);
    o.D = __fmaf_rn(lb, ca, D);
    la2_min = fminf(la2, fminf(lb2, lc2));
    return o;
}

// Slow-path term for a pair the fast path skipped: ATAN2(N, D) per Eq. (8) (-0 treated as +0,
// the table's y >= 0 case), and 0 when q coincides with a vertex (ATAN2(0,0)).
__device__ __forceinline__ float slow_term(const PairOut &o, float la2_min) {
    if (o.D > fabsf(o.N8)) return 0.0f;  // already added by the fast path
    if (!(la2_min >= 1.17549435e-38f)) return 0.0f;
    return atan2f(__fadd_rn(o.N8, 0.0f), __fmul_rn(kNormalScale, o.D));
}

// (y, z) partial sums of one row for one face.
struct RowPart {
    float La, Lb, Lc, Pab, Pbc, Pca, Nyz;
};

__device__ __forceinline__ RowPart row_part(const FaceRec &r, float qy, float Laz, float Lbz, float Lcz, float Pabz,
                                            float Pbcz, float Pcaz, float Nz) {
    const float ay = __fsub_rn(r.r0.y, qy), by = __fsub_rn(r.r1.y, qy), cy = __fsub_rn(r.r2.y, qy);
    RowPart p;
    p.La = __fmaf_rn(ay, ay, Laz);
    p.Lb = __fmaf_rn(by, by, Lbz);
    p.Lc = __fmaf_rn(cy, cy, Lcz);
    p.Pab = __fmaf_rn(ay, by, Pabz);
    p.Pbc = __fmaf_rn(by, cy, Pbcz);
    p.Pca = __fmaf_rn(cy, ay, Pcaz);
    p.Nyz = __fmaf_rn(ay, r.r1.w, Nz);
    return p;
}

// One face against the thread's QY x QX grid queries, x-adjacent queries paired: every FP32
// operation of the fast path is one packed FP32x2 instruction (Blackwell FFMA2/FADD2/FMUL2) for
// two queries; MUFU square roots and reciprocals stay scalar. nqx holds the negated query x
// coordinates in pairs. Returns true if every pair took the fast path. The SLOW variant adds
// ATAN2 for exactly the pairs the fast path skipped, recomputing N and D with scalar _rn
// operations in the same order (bit-identical to the packed ones).
template <int QX, int QY, bool SLOW>
__device__ __forceinline__ bool face_grid(const FaceRec &r, const float2 (&nqx)[QX / 2], const float (&qy)[QY],
                                          float qz, float2 (&acc)[QY][QX / 2]) {
    static_assert(QX % 2 == 0, "queries are paired along x");
    const float az = __fsub_rn(r.r0.z, qz), bz = __fsub_rn(r.r1.z, qz), cz = __fsub_rn(r.r2.z, qz);
    const float Laz = __fmul_rn(az, az), Lbz = __fmul_rn(bz, bz), Lcz = __fmul_rn(cz, cz);
    const float Pabz = __fmul_rn(az, bz), Pbcz = __fmul_rn(bz, cz), Pcaz = __fmul_rn(cz, az);
    const float Nz = __fmul_rn(az, r.r2.w);
    const float2 v0x = make_float2(r.r0.x, r.r0.x), v1x = make_float2(r.r1.x, r.r1.x), v2x = make_float2(r.r2.x, r.r2.x);
    float2 ax[QX / 2], bx[QX / 2], cx[QX / 2];
#pragma unroll
    for (int j = 0; j < QX / 2; ++j) {
        ax[j] = __fadd2_rn(v0x, nqx[j]);
        bx[j] = __fadd2_rn(v1x, nqx[j]);
        cx[j] = __fadd2_rn(v2x, nqx[j]);
    }
    bool ok = true;
#pragma unroll
    for (int i = 0; i < QY; ++i) {
        const RowPart p = row_part(r, qy[i], Laz, Lbz, Lcz, Pabz, Pbcz, Pcaz, Nz);
        if (!SLOW) {
            const float2 La = make_float2(p.La, p.La), Lb = make_float2(p.Lb, p.Lb), Lc = make_float2(p.Lc, p.Lc);
            const float2 Pab = make_float2(p.Pab, p.Pab), Pbc = make_float2(p.Pbc, p.Pbc);
            const float2 Pca = make_float2(p.Pca, p.Pca), Nyz = make_float2(p.Nyz, p.Nyz);
            const float2 n8x = make_float2(r.r0.w, r.r0.w);
            const float2 C0 = make_float2(DV_ATAN_C0, DV_ATAN_C0), C1 = make_float2(DV_ATAN_C1, DV_ATAN_C1);
            const float2 C2 = make_float2(DV_ATAN_C2, DV_ATAN_C2);
#pragma unroll
            for (int j = 0; j < QX / 2; ++j) {
                const float2 la2 = __ffma2_rn(ax[j], ax[j], La);
                const float2 lb2 = __ffma2_rn(bx[j], bx[j], Lb);
                const float2 lc2 = __ffma2_rn(cx[j], cx[j], Lc);
                const float2 la = make_float2(sqrt_approx(la2.x), sqrt_approx(la2.y));
                const float2 lb = make_float2(sqrt_approx(lb2.x), sqrt_approx(lb2.y));
                const float2 lc = make_float2(sqrt_approx(lc2.x), sqrt_approx(lc2.y));
                const float2 ab = __ffma2_rn(ax[j], bx[j], Pab);
                const float2 bc = __ffma2_rn(bx[j], cx[j], Pbc);
                const float2 ca = __ffma2_rn(cx[j], ax[j], Pca);
                const float2 N8 = __ffma2_rn(ax[j], n8x, Nyz);
                float2 D = __fmul2_rn(__ffma2_rn(la, lb, ab), lc);
                D = __ffma2_rn(la, bc, D);
                D = __ffma2_rn(lb, ca, D);
                const bool p0 = D.x > fabsf(N8.x), p1 = D.y > fabsf(N8.y);
                ok = ok && p0 && p1;
                float2 v = __fmul2_rn(N8, make_float2(rcp_approx(D.x), rcp_approx(D.y)));
                v.x = p0 ? v.x : 0.0f;
                v.y = p1 ? v.y : 0.0f;
                const float2 sq = __fmul2_rn(v, v);
                const float2 P = __ffma2_rn(__ffma2_rn(C2, sq, C1), sq, C0);
                acc[i][j] = __ffma2_rn(v, P, acc[i][j]);
            }
        } else {
#pragma unroll
            for (int j = 0; j < QX / 2; ++j) {
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const float axs = k ? ax[j].y : ax[j].x, bxs = k ? bx[j].y : bx[j].x, cxs = k ? cx[j].y : cx[j].x;
                    float m;
                    const PairOut o = pair_terms(axs, bxs, cxs, p.La, p.Lb, p.Lc, p.Pab, p.Pbc, p.Pca, p.Nyz, r.r0.w, m);
                    const float t = slow_term(o, m);
                    if (k)
                        acc[i][j].y = __fadd_rn(acc[i][j].y, t);
                    else
                        acc[i][j].x = __fadd_rn(acc[i][j].x, t);
                }
            }
        }
    }
    return ok;
}

// FP16 ablation of face_grid (the paper computed in half precision, §3.1): offsets and their
// (y,z) partial sums in FP32 as above, then every per-pair operation in packed half2 arithmetic
// (two x-adjacent queries per instruction), the fast-path arctangent in half, and the term
// accumulated in FP32. Pairs failing the half fast-path test are added by the SLOW variant
// through the FP32 formula and atan2f. Quantifies half precision; not an accurate mode.
__device__ __forceinline__ unsigned h2_bits(__half2 v) {
    unsigned u;
    memcpy(&u, &v, sizeof(u));
    return u;
}
__device__ __forceinline__ __half2 bits_h2(unsigned u) {
    __half2 v;
    memcpy(&v, &u, sizeof(u));
    return v;
}

template <int QX, int QY, bool SLOW>
__device__ __forceinline__ bool face_grid_h(const FaceRec &r, const float (&qx)[QX], const float (&qy)[QY], float qz,
                                            float (&acc)[QY][QX]) {
    static_assert(QX % 2 == 0, "half2 path pairs x-adjacent queries");
    const float az = __fsub_rn(r.r0.z, qz), bz = __fsub_rn(r.r1.z, qz), cz = __fsub_rn(r.r2.z, qz);
    const float Laz = __fmul_rn(az, az), Lbz = __fmul_rn(bz, bz), Lcz = __fmul_rn(cz, cz);
    const float Pabz = __fmul_rn(az, bz), Pbcz = __fmul_rn(bz, cz), Pcaz = __fmul_rn(cz, az);
    const float Nz = __fmul_rn(az, r.r2.w);
    float ax[QX], bx[QX], cx[QX];
#pragma unroll
    for (int j = 0; j < QX; ++j) {
        ax[j] = __fsub_rn(r.r0.x, qx[j]);
        bx[j] = __fsub_rn(r.r1.x, qx[j]);
        cx[j] = __fsub_rn(r.r2.x, qx[j]);
    }
    __half2 ax2[QX / 2], bx2[QX / 2], cx2[QX / 2];
#pragma unroll
    for (int j = 0; j < QX / 2; ++j) {
        ax2[j] = __floats2half2_rn(ax[2 * j], ax[2 * j + 1]);
        bx2[j] = __floats2half2_rn(bx[2 * j], bx[2 * j + 1]);
        cx2[j] = __floats2half2_rn(cx[2 * j], cx[2 * j + 1]);
    }
    const __half2 n8x = __float2half2_rn(r.r0.w);
    const __half2 Dmin = __float2half2_rn(6.103515625e-05f);
    const __half2 C0 = __float2half2_rn(DV_ATAN_C0), C1 = __float2half2_rn(DV_ATAN_C1),
                  C2 = __float2half2_rn(DV_ATAN_C2);
    bool ok = true;
#pragma unroll
    for (int i = 0; i < QY; ++i) {
        const RowPart p = row_part(r, qy[i], Laz, Lbz, Lcz, Pabz, Pbcz, Pcaz, Nz);
        const __half2 La = __float2half2_rn(p.La), Lb = __float2half2_rn(p.Lb), Lc = __float2half2_rn(p.Lc);
        const __half2 Pab = __float2half2_rn(p.Pab), Pbc = __float2half2_rn(p.Pbc), Pca = __float2half2_rn(p.Pca);
        const __half2 Nyz = __float2half2_rn(p.Nyz);
#pragma unroll
        for (int j = 0; j < QX / 2; ++j) {
            const __half2 la = h2sqrt(__hfma2(ax2[j], ax2[j], La));
            const __half2 lb = h2sqrt(__hfma2(bx2[j], bx2[j], Lb));
            const __half2 lc = h2sqrt(__hfma2(cx2[j], cx2[j], Lc));
            const __half2 ab = __hfma2(ax2[j], bx2[j], Pab);
            const __half2 bc = __hfma2(bx2[j], cx2[j], Pbc);
            const __half2 ca = __hfma2(cx2[j], ax2[j], Pca);
            const __half2 N8 = __hfma2(ax2[j], n8x, Nyz);
            __half2 D = __hmul2(__hfma2(la, lb, ab), lc);
            D = __hfma2(la, bc, D);
            D = __hfma2(lb, ca, D);
            // fast path needs D > |8N| and D > 2^-14, so that 1/D stays finite in half precision
            const unsigned m = __hgt2_mask(D, __hmax2(__habs2(N8), Dmin));
            if (!SLOW) {
                ok = ok && m == 0xffffffffu;
                const __half2 v = bits_h2(h2_bits(__hmul2(N8, h2rcp(D))) & m);
                const __half2 sq = __hmul2(v, v);
                const __half2 t = __hmul2(v, __hfma2(__hfma2(C2, sq, C1), sq, C0));
                acc[i][2 * j] = __fadd_rn(acc[i][2 * j], __low2float(t));
                acc[i][2 * j + 1] = __fadd_rn(acc[i][2 * j + 1], __high2float(t));
            } else {
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if ((m >> (16 * k)) & 0xffffu) continue;  // taken by the half fast path
                    float mn;
                    const PairOut o = pair_terms(ax[2 * j + k], bx[2 * j + k], cx[2 * j + k], p.La, p.Lb, p.Lc, p.Pab,
                                                 p.Pbc, p.Pca, p.Nyz, r.r0.w, mn);
                    if (mn >= 1.17549435e-38f)
                        acc[i][2 * j + k] = __fadd_rn(acc[i][2 * j + k], atan2f(__fadd_rn(o.N8, 0.0f),
                                                                                __fmul_rn(kNormalScale, o.D)));
                }
            }
        }
    }
    return ok;
}

// Kahan step: (s, c) += x.
__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// Final per-query write: w, occupancy, and the re-evaluation flag.
__device__ __forceinline__ void epilogue(const FwdArgs &a, int64_t idx, float w) {
    if (!DV_INB(idx, a.nq, kSiteFwdOut)) return;
    a.w_out[idx] = w;
    if (a.occ_out) a.occ_out[idx] = w > 0.5f ? 1 : 0;
    if (a.flag_list) {
        const bool flagged = a.near_flag[idx] != 0 || fabsf(__fsub_rn(w, 0.5f)) < kThreshBand;
        if (flagged) {
            const int pos = atomicAdd(a.flag_count, 1);
            if (DV_INB(pos, a.nq, kSiteFwdFlagList)) a.flag_list[pos] = (int)idx;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Shared TMA tile pipeline over an array of 16-byte-multiple records (faces or strip events).
// `Body` processes one tile: body(const Rec* tile, int count).
template <typename Rec, int kT = kTileFaces>
struct TilePipe {
    Rec (*sm)[kT];
    uint64_t *full;
    const Rec *src;
    int64_t f0;
    int64_t nfaces;
    int ntiles;
    int skip_tile;     // self-test hook: this tile is never issued (-1: none)
    uint64_t wait_ns;  // limit of each bounded wait
    int64_t total;     // records in the source array (bounds check of the debug build)

    __device__ __forceinline__ int tile_count(int t) const {
        const int64_t left = nfaces - (int64_t)t * kT;
        return left < kT ? (int)left : kT;
    }
    __device__ __forceinline__ void issue(int t) const {
        if (t == skip_tile) return;
        const int s = t % kStages;
        const uint32_t bytes = (uint32_t)tile_count(t) * (uint32_t)sizeof(Rec);
        // debug build: a tile reaching outside the records is not copied (its wait then runs out)
        if (!DV_INB(f0 + (int64_t)t * kT, total, kSiteFwdTile) ||
            !DV_INB(f0 + (int64_t)t * kT + tile_count(t) - 1, total, kSiteFwdTile))
            return;
        mbar_arrive_expect_tx(&full[s], bytes);
        tma_load_1d(&sm[s][0], src + f0 + (int64_t)t * kT, bytes, &full[s]);
    }
};

// Every thread waits (bounded) for tile t, processes it, and the barrier that ends the tile
// combines the threads' verdicts, so the CTA decides as one whether a wait ran out. On a timeout
// the CTA stops: no further copies are issued, the sticky error word gets DV_ERR_TIMEOUT, and
// thread 0 waits (bounded again) for the copies already issued and not yet seen complete, tiles
// t .. min(ntiles, t + kStages) - 1, before the CTA leaves. The results of such a CTA are not
// meaningful; the error word says so.
template <typename Rec, int kT, typename Body, typename TileEnd>
__device__ __forceinline__ bool run_face_tiles(TilePipe<Rec, kT> &pp, int *err, Body &&body, TileEnd &&tile_end) {
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&pp.full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int pre = pp.ntiles < kStages ? pp.ntiles : kStages;
        for (int t = 0; t < pre; ++t) pp.issue(t);
    }
    int t = 0;
    bool timed_out = false;
    for (; t < pp.ntiles; ++t) {
        const int s = t % kStages;
        const bool ok = mbar_wait_bounded(&pp.full[s], (uint32_t)((t / kStages) & 1), pp.wait_ns);
        body(&pp.sm[s][0], pp.tile_count(t));
        tile_end();
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        if (threadIdx.x == 0 && t + kStages < pp.ntiles) {
            fence_proxy_async_smem();
            pp.issue(t + kStages);
        }
    }
    if (timed_out) {  // the same value in every thread of the CTA
        if (threadIdx.x == 0) {
            set_error(err, 5);
            const int last = t + kStages < pp.ntiles ? t + kStages : pp.ntiles;
            for (int u = t; u < last; ++u)
                if (u != pp.skip_tile) mbar_wait_bounded(&pp.full[u % kStages], (uint32_t)((u / kStages) & 1), pp.wait_ns);
        }
        __syncthreads();
    }
    return !timed_out;
}

// ---------------------------------------------------------------------------------------------
template <int QX, int QY, bool KAHAN, bool HALF>
__global__ void __launch_bounds__(kFwdThreads, 3) fwd_grid_kernel(const FwdArgs a) {
    __shared__ __align__(128) FaceRec sm[kStages][kTileFaces];
    __shared__ __align__(8) uint64_t full[kStages];
    // Kahan state (sum, compensation) of every query of every thread, touched once per tile:
    // kept in shared memory so that the hot loop's registers hold only the tile sums.
    __shared__ float2 kst[KAHAN ? QX * QY : 1][kFwdThreads];

    const int nx = a.g.n[0], ny = a.g.n[1], nz = a.g.n[2];
    const int tiles_x = (nx + QX - 1) / QX, tiles_y = (ny + QY - 1) / QY;
    const int64_t tile = (int64_t)blockIdx.x * kFwdThreads + threadIdx.x;
    const int tx = (int)(tile % tiles_x);
    const int64_t t2 = tile / tiles_x;
    const int ty = (int)(t2 % tiles_y);
    const int64_t zz = t2 / tiles_y;
    const bool valid_t = zz < nz;
    const int z = valid_t ? (int)zz : nz - 1;

    float qx[QX], qy[QY];
#pragma unroll
    for (int j = 0; j < QX; ++j) qx[j] = __fmaf_rn((float)(tx * QX + j) + 0.5f, a.g.h[0], a.g.lo[0]);
    float2 nqx[QX / 2];
#pragma unroll
    for (int j = 0; j < QX / 2; ++j) nqx[j] = make_float2(-qx[2 * j], -qx[2 * j + 1]);
#pragma unroll
    for (int i = 0; i < QY; ++i) qy[i] = __fmaf_rn((float)(ty * QY + i) + 0.5f, a.g.h[1], a.g.lo[1]);
    const float qz = __fmaf_rn((float)z + 0.5f, a.g.h[2], a.g.lo[2]);

    // acc2: packed per pair of x-adjacent queries (FP32 path); acc: per query (FP16 path)
    float2 acc2[QY][QX / 2];
    float acc[QY][QX];
#pragma unroll
    for (int i = 0; i < QY; ++i)
#pragma unroll
        for (int j = 0; j < QX; ++j) {
            acc[i][j] = 0.0f;
            if (j % 2 == 0) acc2[i][j / 2] = make_float2(0.0f, 0.0f);
            if (KAHAN) kst[i * QX + j][threadIdx.x] = make_float2(0.0f, 0.0f);
        }

    TilePipe<FaceRec> pp;
    pp.sm = sm;
    pp.full = full;
    pp.src = a.rec;
    pp.f0 = (int64_t)blockIdx.y * a.faces_per_split;
    const int64_t f1 = pp.f0 + a.faces_per_split < a.nf ? pp.f0 + a.faces_per_split : a.nf;
    pp.nfaces = f1 - pp.f0;
    pp.ntiles = (int)((pp.nfaces + kTileFaces - 1) / kTileFaces);
    pp.skip_tile = a.skip_tile;
    pp.wait_ns = a.wait_ns;
    pp.total = a.nf;

    run_face_tiles(
        pp, a.err,
        [&](const FaceRec *tilep, int cnt) {
#pragma unroll 1
            for (int k = 0; k < cnt; ++k) {
                const FaceRec r = tilep[k];
                if (HALF) {
                    const bool ok = face_grid_h<QX, QY, false>(r, qx, qy, qz, acc);
                    if (__any_sync(kFull, !ok)) face_grid_h<QX, QY, true>(r, qx, qy, qz, acc);
                } else {
                    const bool ok = face_grid<QX, QY, false>(r, nqx, qy, qz, acc2);
                    if (__any_sync(kFull, !ok)) face_grid<QX, QY, true>(r, nqx, qy, qz, acc2);
                }
            }
        },
        [&]() {
            if (KAHAN) {
#pragma unroll
                for (int i = 0; i < QY; ++i)
#pragma unroll
                    for (int j = 0; j < QX; ++j) {
                        float2 k = kst[i * QX + j][threadIdx.x];
                        const float t = HALF ? acc[i][j] : (j % 2 ? acc2[i][j / 2].y : acc2[i][j / 2].x);
                        kahan_add(k.x, k.y, t);
                        kst[i * QX + j][threadIdx.x] = k;
                        acc[i][j] = 0.0f;
                        if (j % 2) acc2[i][j / 2] = make_float2(0.0f, 0.0f);
                    }
            }
        });

    if (!valid_t) return;
#pragma unroll
    for (int i = 0; i < QY; ++i) {
        const int iy = ty * QY + i;
        if (iy >= ny) continue;
#pragma unroll
        for (int j = 0; j < QX; ++j) {
            const int ix = tx * QX + j;
            if (ix >= nx) continue;
            const int64_t idx = ((int64_t)z * ny + iy) * nx + ix;
            const float plain = HALF ? acc[i][j] : (j % 2 ? acc2[i][j / 2].y : acc2[i][j / 2].x);
            const float2 k = KAHAN ? kst[i * QX + j][threadIdx.x] : make_float2(plain, 0.0f);
            const float s = k.x, c = k.y;
            if (a.nsplit > 1) {
                if (DV_INB((int64_t)blockIdx.y * a.nq + idx, (int64_t)a.nsplit * a.nq, kSiteFwdPartial))
                    a.partial[(int64_t)blockIdx.y * a.nq + idx] = make_float2(s, -c);
            } else
                epilogue(a, idx, __fmul_rn(__fsub_rn(s, c), kInv2Pi));
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Grid forward over the vertex-sharing strip order (strips.cu). Each event brings a vertex V; an
// event flagged as a face completes the face {P2, P1, V} of the two vertices before it. Per
// thread and query the state carried from event to event is, for P1 and P2, the offset from the
// query, the distance |P - q| and the dot (P - q).(P' - q) with the vertex before it, so a face
// costs one MUFU square root, two dots and D:
//   D = (|V||P1| + V.P1)|P2| + |V|(P1.P2) + |P1|(V.P2)      (offsets relative to q)
//   N = (V - q) . n_f                                       (any vertex of the face gives det)
// then the ATAN2 fast path / slow path of face_grid. (y, z) parts are shared per row as before.
// Three state slots rotate through the roles (P2, P1, V), so the event loop is unrolled by
// three and no state is copied; strip tiles hold a multiple of three events.
constexpr int kStripThreads = 128;
constexpr int kTileEvents = 96;

template <int QX, int QY>
struct StripSlot {
    float2 ax[QX / 2];     // vertex x - query x, pairs of x-adjacent queries
    float ay[QY], az;      // vertex y - query y per row, vertex z - query z
    float2 l[QY][QX / 2];  // |vertex - query|
    float2 e[QY][QX / 2];  // (vertex - query).(previous vertex - query)
};

// Slow-path term for a strip face (same conventions as slow_term): 0 if the fast path took it,
// 0 when q coincides with one of the face's vertices (a distance that is 0 after the flush to
// zero of a subnormal |.|^2), else ATAN2(N, D) per Eq. (8).
__device__ __forceinline__ float strip_slow_term(float N8, float D, float lmin) {
    if (D > fabsf(N8)) return 0.0f;
    if (!(lmin > 0.0f)) return 0.0f;
    return atan2f(__fadd_rn(N8, 0.0f), __fmul_rn(kNormalScale, D));
}

// Vertex part of a strip event: offsets of the event's vertex V from the thread's queries,
// |V - q| (MUFU square root) and the dot with the previous vertex P1.
template <int QX, int QY>
__device__ __forceinline__ void strip_vertex(const StripRec &r, const float2 (&nqx)[QX / 2], const float (&qy)[QY],
                                             float qz, const StripSlot<QX, QY> &P1, StripSlot<QX, QY> &V) {
    V.az = __fsub_rn(r.p.z, qz);
    const float2 vx = make_float2(r.p.x, r.p.x);
#pragma unroll
    for (int j = 0; j < QX / 2; ++j) V.ax[j] = __fadd2_rn(vx, nqx[j]);
    const float azz = __fmul_rn(V.az, V.az), az1 = __fmul_rn(V.az, P1.az);
#pragma unroll
    for (int i = 0; i < QY; ++i) {
        V.ay[i] = __fsub_rn(r.p.y, qy[i]);
        const float Lyz = __fmaf_rn(V.ay[i], V.ay[i], azz);
        const float d1yz = __fmaf_rn(V.ay[i], P1.ay[i], az1);
#pragma unroll
        for (int j = 0; j < QX / 2; ++j) {
            const float2 l2 = __ffma2_rn(V.ax[j], V.ax[j], make_float2(Lyz, Lyz));
            V.l[i][j] = make_float2(sqrt_approx(l2.x), sqrt_approx(l2.y));
            V.e[i][j] = __ffma2_rn(V.ax[j], P1.ax[j], make_float2(d1yz, d1yz));  // (V - q).(P1 - q)
        }
    }
}

// N and D of the face {P2, P1, V} for pair (i, j) of the thread's queries.
template <int QX, int QY>
__device__ __forceinline__ void strip_nd(const StripRec &r, const StripSlot<QX, QY> &P2, const StripSlot<QX, QY> &P1,
                                         const StripSlot<QX, QY> &V, int i, int j, float2 &N8, float2 &D) {
    const float d2yz = __fmaf_rn(V.ay[i], P2.ay[i], __fmul_rn(V.az, P2.az));
    const float Nyz = __fmaf_rn(V.ay[i], r.q.x, __fmul_rn(V.az, r.q.y));
    const float2 d2 = __ffma2_rn(V.ax[j], P2.ax[j], make_float2(d2yz, d2yz));  // (V - q).(P2 - q)
    N8 = __ffma2_rn(V.ax[j], make_float2(r.p.w, r.p.w), make_float2(Nyz, Nyz));
    D = __fmul2_rn(__ffma2_rn(V.l[i][j], P1.l[i][j], V.e[i][j]), P2.l[i][j]);
    D = __ffma2_rn(V.l[i][j], P1.e[i][j], D);
    D = __ffma2_rn(P1.l[i][j], d2, D);
}

// Face part of a strip event: the ATAN2 fast path for the thread's queries; if any lane of the
// warp has a pair outside it, the slow path recomputes N and D (same operations, same values)
// and adds ATAN2 for exactly those pairs.
template <int QX, int QY>
__device__ __forceinline__ void strip_face(const StripRec &r, const StripSlot<QX, QY> &P2,
                                           const StripSlot<QX, QY> &P1, const StripSlot<QX, QY> &V,
                                           float2 (&acc)[QY][QX / 2]) {
    const float2 C0 = make_float2(DV_ATAN_C0, DV_ATAN_C0), C1 = make_float2(DV_ATAN_C1, DV_ATAN_C1);
    const float2 C2 = make_float2(DV_ATAN_C2, DV_ATAN_C2);
    bool ok = true;
#pragma unroll
    for (int i = 0; i < QY; ++i)
#pragma unroll
        for (int j = 0; j < QX / 2; ++j) {
            float2 N8, D;
            strip_nd(r, P2, P1, V, i, j, N8, D);
            const bool p0 = D.x > fabsf(N8.x), p1 = D.y > fabsf(N8.y);
            ok = ok && p0 && p1;
            float2 v = __fmul2_rn(N8, make_float2(rcp_approx(D.x), rcp_approx(D.y)));
            v.x = p0 ? v.x : 0.0f;
            v.y = p1 ? v.y : 0.0f;
            const float2 sq = __fmul2_rn(v, v);
            const float2 P = __ffma2_rn(__ffma2_rn(C2, sq, C1), sq, C0);
            acc[i][j] = __ffma2_rn(v, P, acc[i][j]);
        }
    if (__any_sync(kFull, !ok)) {
#pragma unroll
        for (int i = 0; i < QY; ++i)
#pragma unroll
            for (int j = 0; j < QX / 2; ++j) {
                float2 N8, D;
                strip_nd(r, P2, P1, V, i, j, N8, D);
                const float lx = fminf(V.l[i][j].x, fminf(P1.l[i][j].x, P2.l[i][j].x));
                const float ly = fminf(V.l[i][j].y, fminf(P1.l[i][j].y, P2.l[i][j].y));
                acc[i][j].x = __fadd_rn(acc[i][j].x, strip_slow_term(N8.x, D.x, lx));
                acc[i][j].y = __fadd_rn(acc[i][j].y, strip_slow_term(N8.y, D.y, ly));
            }
    }
}

// One software-pipelined step: the face part of event k (if it completes a face) and the vertex
// part of event k + 1 in one basic block, so the compiler can overlap the next vertex's square
// roots with this face's arithmetic. The next vertex goes into P2's slot, which this face reads
// first (the scheduler renames registers where it overlaps the two).
template <int QX, int QY>
__device__ __forceinline__ void strip_step(const StripRec &r, bool face, const StripRec &rn,
                                           const float2 (&nqx)[QX / 2], const float (&qy)[QY], float qz,
                                           StripSlot<QX, QY> &P2, const StripSlot<QX, QY> &P1,
                                           const StripSlot<QX, QY> &V, float2 (&acc)[QY][QX / 2]) {
    if (face) {
        strip_face<QX, QY>(r, P2, P1, V, acc);
        strip_vertex<QX, QY>(rn, nqx, qy, qz, V, P2);
    } else {
        strip_vertex<QX, QY>(rn, nqx, qy, qz, V, P2);
    }
}

template <int QX, int QY, bool KAHAN>
__global__ void __launch_bounds__(kStripThreads, 4) fwd_grid_strip_kernel(const FwdArgs a) {
    __shared__ __align__(128) StripRec sm[kStages][kTileEvents];
    __shared__ __align__(8) uint64_t full[kStages];
    __shared__ float2 kst[KAHAN ? QX * QY : 1][kStripThreads];

    const int nx = a.g.n[0], ny = a.g.n[1], nz = a.g.n[2];
    const int tiles_x = (nx + QX - 1) / QX, tiles_y = (ny + QY - 1) / QY;
    const int64_t tile = (int64_t)blockIdx.x * kStripThreads + threadIdx.x;
    const int tx = (int)(tile % tiles_x);
    const int64_t t2 = tile / tiles_x;
    const int ty = (int)(t2 % tiles_y);
    const int64_t zz = t2 / tiles_y;
    const bool valid_t = zz < nz;
    const int z = valid_t ? (int)zz : nz - 1;

    float qy[QY];
    float2 nqx[QX / 2];
#pragma unroll
    for (int j = 0; j < QX / 2; ++j)
        nqx[j] = make_float2(-__fmaf_rn((float)(tx * QX + 2 * j) + 0.5f, a.g.h[0], a.g.lo[0]),
                             -__fmaf_rn((float)(tx * QX + 2 * j + 1) + 0.5f, a.g.h[0], a.g.lo[0]));
#pragma unroll
    for (int i = 0; i < QY; ++i) qy[i] = __fmaf_rn((float)(ty * QY + i) + 0.5f, a.g.h[1], a.g.lo[1]);
    const float qz = __fmaf_rn((float)z + 0.5f, a.g.h[2], a.g.lo[2]);

    float2 acc[QY][QX / 2];
    StripSlot<QX, QY> S0, S1, S2;
#pragma unroll
    for (int i = 0; i < QY; ++i) {
        S0.ay[i] = S1.ay[i] = S2.ay[i] = 0.0f;
#pragma unroll
        for (int j = 0; j < QX / 2; ++j) {
            acc[i][j] = make_float2(0.0f, 0.0f);
            S0.l[i][j] = S1.l[i][j] = S2.l[i][j] = S0.e[i][j] = S1.e[i][j] = S2.e[i][j] = make_float2(0.0f, 0.0f);
            if (KAHAN) {
                kst[i * QX + 2 * j][threadIdx.x] = make_float2(0.0f, 0.0f);
                kst[i * QX + 2 * j + 1][threadIdx.x] = make_float2(0.0f, 0.0f);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < QX / 2; ++j) S0.ax[j] = S1.ax[j] = S2.ax[j] = make_float2(0.0f, 0.0f);
    S0.az = S1.az = S2.az = 0.0f;

    // Events [e0, e1) of this split, preceded by up to two warm-up events (vertex part only)
    // that supply the first faces' earlier vertices. Splits hold whole tiles of events.
    const int64_t e0 = (int64_t)blockIdx.y * a.faces_per_split;
    const int64_t e1 = e0 + a.faces_per_split < a.ne ? e0 + a.faces_per_split : a.ne;
    const int warm = (int)(e0 < 2 ? e0 : 2);
    TilePipe<StripRec, kTileEvents> pp;
    pp.sm = sm;
    pp.full = full;
    pp.src = a.srec;
    pp.f0 = e0 - warm;
    pp.nfaces = e1 - pp.f0;
    pp.ntiles = (int)((pp.nfaces + kTileEvents - 1) / kTileEvents);
    pp.skip_tile = a.skip_tile;
    pp.wait_ns = a.wait_ns;
    pp.total = a.ne;

    int first = warm;  // leading events of the current tile that are warm-up only
    run_face_tiles(
        pp, a.err,
        [&](const StripRec *tilep, int cnt) {
            // On entry S1, S2 hold the vertex parts of the two events before this tile (older,
            // newer). Event k of the tile goes to slot k mod 3; step k finishes event k's face
            // and computes event k + 1's vertex part.
            strip_vertex<QX, QY>(tilep[0], nqx, qy, qz, S2, S0);
            int k = 0;
#pragma unroll 1
            for (; k + 3 < cnt; k += 3) {
                strip_step<QX, QY>(tilep[k], tilep[k].q.z != 0.0f && k >= first, tilep[k + 1], nqx, qy, qz, S1,
                                   S2, S0, acc);
                strip_step<QX, QY>(tilep[k + 1], tilep[k + 1].q.z != 0.0f && k + 1 >= first, tilep[k + 2], nqx, qy,
                                   qz, S2, S0, S1, acc);
                strip_step<QX, QY>(tilep[k + 2], tilep[k + 2].q.z != 0.0f, tilep[k + 3], nqx, qy, qz, S0, S1, S2,
                                   acc);
            }
            // last one to three events of the tile; the vertex part after the tile's last event
            // belongs to the next tile
            {
                const StripRec r = tilep[k];
                const bool face = r.q.z != 0.0f && k >= first;
                if (k + 1 < cnt)
                    strip_step<QX, QY>(r, face, tilep[k + 1], nqx, qy, qz, S1, S2, S0, acc);
                else if (face)
                    strip_face<QX, QY>(r, S1, S2, S0, acc);
            }
            if (k + 1 < cnt) {
                const StripRec r = tilep[k + 1];
                const bool face = r.q.z != 0.0f && k + 1 >= first;
                if (k + 2 < cnt)
                    strip_step<QX, QY>(r, face, tilep[k + 2], nqx, qy, qz, S2, S0, S1, acc);
                else if (face)
                    strip_face<QX, QY>(r, S2, S0, S1, acc);
            }
            if (k + 2 < cnt) {
                const StripRec r = tilep[k + 2];
                if (r.q.z != 0.0f) strip_face<QX, QY>(r, S0, S1, S2, acc);
            }
            first = 0;
        },
        [&]() {
            if (KAHAN) {
#pragma unroll
                for (int i = 0; i < QY; ++i)
#pragma unroll
                    for (int j = 0; j < QX; ++j) {
                        float2 k = kst[i * QX + j][threadIdx.x];
                        kahan_add(k.x, k.y, j % 2 ? acc[i][j / 2].y : acc[i][j / 2].x);
                        kst[i * QX + j][threadIdx.x] = k;
                        if (j % 2) acc[i][j / 2] = make_float2(0.0f, 0.0f);
                    }
            }
        });

    if (!valid_t) return;
#pragma unroll
    for (int i = 0; i < QY; ++i) {
        const int iy = ty * QY + i;
        if (iy >= ny) continue;
#pragma unroll
        for (int j = 0; j < QX; ++j) {
            const int ix = tx * QX + j;
            if (ix >= nx) continue;
            const int64_t idx = ((int64_t)z * ny + iy) * nx + ix;
            const float plain = j % 2 ? acc[i][j / 2].y : acc[i][j / 2].x;
            const float2 k = KAHAN ? kst[i * QX + j][threadIdx.x] : make_float2(plain, 0.0f);
            if (a.nsplit > 1) {
                if (DV_INB((int64_t)blockIdx.y * a.nq + idx, (int64_t)a.nsplit * a.nq, kSiteFwdPartial))
                    a.partial[(int64_t)blockIdx.y * a.nq + idx] = make_float2(k.x, -k.y);
            } else
                epilogue(a, idx, __fmul_rn(__fsub_rn(k.x, k.y), kInv2Pi));
        }
    }
}

// ---------------------------------------------------------------------------------------------
// List forward over the strip order: arbitrary queries, so no (y, z) sharing; each thread
// holds QP pairs of queries (packed FP32x2) and, per pair and strip slot, the vertex offsets,
// |v - q| and the dot with the previous vertex. Same N, D, fast path and slow path as the grid
// strip kernel; Kahan state in shared memory.
template <int QP>
struct ListSlot {
    float2 ax[QP], ay[QP], az[QP];  // vertex - query
    float2 l[QP];                   // |vertex - query|
    float2 e[QP];                   // (vertex - query).(previous vertex - query)
};

template <int QP>
__device__ __forceinline__ void list_nd(const StripRec &r, const ListSlot<QP> &P2, const ListSlot<QP> &P1,
                                        const ListSlot<QP> &V, int j, float2 &N8, float2 &D) {
    float2 d2 = __fmul2_rn(V.ax[j], P2.ax[j]);
    d2 = __ffma2_rn(V.ay[j], P2.ay[j], d2);
    d2 = __ffma2_rn(V.az[j], P2.az[j], d2);
    N8 = __fmul2_rn(V.ax[j], make_float2(r.p.w, r.p.w));
    N8 = __ffma2_rn(V.ay[j], make_float2(r.q.x, r.q.x), N8);
    N8 = __ffma2_rn(V.az[j], make_float2(r.q.y, r.q.y), N8);
    D = __fmul2_rn(__ffma2_rn(V.l[j], P1.l[j], V.e[j]), P2.l[j]);
    D = __ffma2_rn(V.l[j], P1.e[j], D);
    D = __ffma2_rn(P1.l[j], d2, D);
}

// Vertex part of a list event (offsets, |V - q|, dot with the previous vertex P1).
template <int QP>
__device__ __forceinline__ void list_vertex(const StripRec &r, const float2 (&nq)[QP][3], const ListSlot<QP> &P1,
                                            ListSlot<QP> &V) {
    const float2 vx = make_float2(r.p.x, r.p.x), vy = make_float2(r.p.y, r.p.y), vz = make_float2(r.p.z, r.p.z);
#pragma unroll
    for (int j = 0; j < QP; ++j) {
        V.ax[j] = __fadd2_rn(vx, nq[j][0]);
        V.ay[j] = __fadd2_rn(vy, nq[j][1]);
        V.az[j] = __fadd2_rn(vz, nq[j][2]);
        float2 l2 = __fmul2_rn(V.ax[j], V.ax[j]);
        l2 = __ffma2_rn(V.ay[j], V.ay[j], l2);
        l2 = __ffma2_rn(V.az[j], V.az[j], l2);
        V.l[j] = make_float2(sqrt_approx(l2.x), sqrt_approx(l2.y));
        float2 e = __fmul2_rn(V.ax[j], P1.ax[j]);
        e = __ffma2_rn(V.ay[j], P1.ay[j], e);
        V.e[j] = __ffma2_rn(V.az[j], P1.az[j], e);
    }
}

// Face part of a list event: fast path, and the slow path when any lane needs it.
template <int QP>
__device__ __forceinline__ void list_face(const StripRec &r, const ListSlot<QP> &P2, const ListSlot<QP> &P1,
                                          const ListSlot<QP> &V, float2 (&acc)[QP]) {
    const float2 C0 = make_float2(DV_ATAN_C0, DV_ATAN_C0), C1 = make_float2(DV_ATAN_C1, DV_ATAN_C1);
    const float2 C2 = make_float2(DV_ATAN_C2, DV_ATAN_C2);
    bool ok = true;
#pragma unroll
    for (int j = 0; j < QP; ++j) {
        float2 N8, D;
        list_nd<QP>(r, P2, P1, V, j, N8, D);
        const bool p0 = D.x > fabsf(N8.x), p1 = D.y > fabsf(N8.y);
        ok = ok && p0 && p1;
        float2 v = __fmul2_rn(N8, make_float2(rcp_approx(D.x), rcp_approx(D.y)));
        v.x = p0 ? v.x : 0.0f;
        v.y = p1 ? v.y : 0.0f;
        const float2 sq = __fmul2_rn(v, v);
        const float2 P = __ffma2_rn(__ffma2_rn(C2, sq, C1), sq, C0);
        acc[j] = __ffma2_rn(v, P, acc[j]);
    }
    if (__any_sync(kFull, !ok)) {
#pragma unroll
        for (int j = 0; j < QP; ++j) {
            float2 N8, D;
            list_nd<QP>(r, P2, P1, V, j, N8, D);
            const float lx = fminf(V.l[j].x, fminf(P1.l[j].x, P2.l[j].x));
            const float ly = fminf(V.l[j].y, fminf(P1.l[j].y, P2.l[j].y));
            acc[j].x = __fadd_rn(acc[j].x, strip_slow_term(N8.x, D.x, lx));
            acc[j].y = __fadd_rn(acc[j].y, strip_slow_term(N8.y, D.y, ly));
        }
    }
}

// Software-pipelined step: face part of event r (if it completes a face), then the vertex part
// of the next event rn into P2's slot.
template <int QP>
__device__ __forceinline__ void list_pstep(const StripRec &r, bool face, const StripRec &rn,
                                           const float2 (&nq)[QP][3], ListSlot<QP> &P2, const ListSlot<QP> &P1,
                                           const ListSlot<QP> &V, float2 (&acc)[QP]) {
    if (face) {
        list_face<QP>(r, P2, P1, V, acc);
        list_vertex<QP>(rn, nq, V, P2);
    } else {
        list_vertex<QP>(rn, nq, V, P2);
    }
}

template <int QP, bool KAHAN>
__global__ void __launch_bounds__(kStripThreads, 4) fwd_list_strip_kernel(const FwdArgs a) {
    __shared__ __align__(128) StripRec sm[kStages][kTileEvents];
    __shared__ __align__(8) uint64_t full[kStages];
    __shared__ float2 kst[KAHAN ? 2 * QP : 1][kStripThreads];

    // query j of this thread: base + j * blockDim (coalesced loads); pairs (2p, 2p + 1)
    const int64_t base = (int64_t)blockIdx.x * kStripThreads * 2 * QP + threadIdx.x;
    float2 nq[QP][3];
#pragma unroll
    for (int p = 0; p < QP; ++p) {
        int64_t i0 = base + (int64_t)(2 * p) * kStripThreads, i1 = i0 + kStripThreads;
        if (i0 >= a.nq) i0 = a.nq - 1;
        if (i1 >= a.nq) i1 = a.nq - 1;
#pragma unroll
        for (int c = 0; c < 3; ++c) nq[p][c] = make_float2(-a.queries[3 * i0 + c], -a.queries[3 * i1 + c]);
    }
    float2 acc[QP];
    ListSlot<QP> S0, S1, S2;
#pragma unroll
    for (int p = 0; p < QP; ++p) {
        acc[p] = make_float2(0.0f, 0.0f);
        S0.ax[p] = S0.ay[p] = S0.az[p] = S0.l[p] = S0.e[p] = make_float2(0.0f, 0.0f);
        S1.ax[p] = S1.ay[p] = S1.az[p] = S1.l[p] = S1.e[p] = make_float2(0.0f, 0.0f);
        S2.ax[p] = S2.ay[p] = S2.az[p] = S2.l[p] = S2.e[p] = make_float2(0.0f, 0.0f);
        if (KAHAN) {
            kst[2 * p][threadIdx.x] = make_float2(0.0f, 0.0f);
            kst[2 * p + 1][threadIdx.x] = make_float2(0.0f, 0.0f);
        }
    }

    const int64_t e0 = (int64_t)blockIdx.y * a.faces_per_split;
    const int64_t e1 = e0 + a.faces_per_split < a.ne ? e0 + a.faces_per_split : a.ne;
    const int warm = (int)(e0 < 2 ? e0 : 2);
    TilePipe<StripRec, kTileEvents> pp;
    pp.sm = sm;
    pp.full = full;
    pp.src = a.srec;
    pp.f0 = e0 - warm;
    pp.nfaces = e1 - pp.f0;
    pp.ntiles = (int)((pp.nfaces + kTileEvents - 1) / kTileEvents);
    pp.skip_tile = a.skip_tile;
    pp.wait_ns = a.wait_ns;
    pp.total = a.ne;

    int first = warm;
    run_face_tiles(
        pp, a.err,
        [&](const StripRec *tilep, int cnt) {
            // roles on entry: S1 = P2, S2 = P1 (the two most recent vertices); event k goes to
            // slot k mod 3, and step k finishes event k's face and computes event k + 1's vertex
            list_vertex<QP>(tilep[0], nq, S2, S0);
            int k = 0;
#pragma unroll 1
            for (; k + 3 < cnt; k += 3) {
                list_pstep<QP>(tilep[k], tilep[k].q.z != 0.0f && k >= first, tilep[k + 1], nq, S1, S2, S0, acc);
                list_pstep<QP>(tilep[k + 1], tilep[k + 1].q.z != 0.0f && k + 1 >= first, tilep[k + 2], nq, S2, S0,
                               S1, acc);
                list_pstep<QP>(tilep[k + 2], tilep[k + 2].q.z != 0.0f, tilep[k + 3], nq, S0, S1, S2, acc);
            }
            {
                const StripRec r = tilep[k];
                const bool face = r.q.z != 0.0f && k >= first;
                if (k + 1 < cnt)
                    list_pstep<QP>(r, face, tilep[k + 1], nq, S1, S2, S0, acc);
                else if (face)
                    list_face<QP>(r, S1, S2, S0, acc);
            }
            if (k + 1 < cnt) {
                const StripRec r = tilep[k + 1];
                const bool face = r.q.z != 0.0f && k + 1 >= first;
                if (k + 2 < cnt)
                    list_pstep<QP>(r, face, tilep[k + 2], nq, S2, S0, S1, acc);
                else if (face)
                    list_face<QP>(r, S2, S0, S1, acc);
            }
            if (k + 2 < cnt) {
                const StripRec r = tilep[k + 2];
                if (r.q.z != 0.0f) list_face<QP>(r, S0, S1, S2, acc);
            }
            first = 0;
        },
        [&]() {
            if (KAHAN) {
#pragma unroll
                for (int j = 0; j < 2 * QP; ++j) {
                    float2 k = kst[j][threadIdx.x];
                    kahan_add(k.x, k.y, j % 2 ? acc[j / 2].y : acc[j / 2].x);
                    kst[j][threadIdx.x] = k;
                    if (j % 2) acc[j / 2] = make_float2(0.0f, 0.0f);
                }
            }
        });

#pragma unroll
    for (int j = 0; j < 2 * QP; ++j) {
        const int64_t idx = base + (int64_t)j * kStripThreads;
        if (idx >= a.nq) continue;
        const float plain = j % 2 ? acc[j / 2].y : acc[j / 2].x;
        const float2 k = KAHAN ? kst[j][threadIdx.x] : make_float2(plain, 0.0f);
        if (a.nsplit > 1) {
            if (DV_INB((int64_t)blockIdx.y * a.nq + idx, (int64_t)a.nsplit * a.nq, kSiteFwdPartial))
                a.partial[(int64_t)blockIdx.y * a.nq + idx] = make_float2(k.x, -k.y);
        } else
            epilogue(a, idx, __fmul_rn(__fsub_rn(k.x, k.y), kInv2Pi));
    }
}

// Sum the face-split partials of each query in FP64, in split order, then the epilogue.
__global__ void split_reduce_kernel(const float2 *__restrict__ partial, int nsplit, FwdArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < a.nq; idx += stride) {
        double s = 0.0;
        for (int k = 0; k < nsplit; ++k) {
            if (!DV_INB((int64_t)k * a.nq + idx, (int64_t)nsplit * a.nq, kSiteFwdPartial)) break;
            const float2 p = partial[(int64_t)k * a.nq + idx];
            s += (double)p.x;
            s += (double)p.y;
        }
        epilogue(a, idx, (float)(s * kInv2PiD));
    }
}

// ---------------------------------------------------------------------------------------------
// Host side.
constexpr int kGridQX = 4, kGridQY = 2;  // 8 queries per thread on the grid path (3 CTAs per SM)
constexpr int kStripQX = 4, kStripQY = 2;  // 8 queries per thread on the strip grid path
constexpr int kListQP = 2;                 // 2 packed pairs (4 queries) per thread, strip list path

FwdPlan plan_forward(int64_t nq, int64_t nf, bool grid, const GridF *g, int num_sms, int64_t n_events) {
    FwdPlan p{};
    p.strips = n_events > 0;
    int64_t nrec = nf, tile = kTileFaces, per_sm = grid ? 3 : 2;
    if (p.strips) {
        p.threads = kStripThreads;
        p.qx = grid ? kStripQX : 2 * kListQP;
        p.qy = grid ? kStripQY : 1;
        nrec = n_events;
        tile = kTileEvents;
        per_sm = 4;
    } else {
        // face order: the grid kernel only (the FP16 ablation and the allocation-free entry);
        // query lists always run in strip order
        p.threads = kFwdThreads;
        p.qx = kGridQX;
        p.qy = kGridQY;
    }
    if (grid) {
        const int64_t tiles = (int64_t)((g->n[0] + p.qx - 1) / p.qx) * ((g->n[1] + p.qy - 1) / p.qy) * g->n[2];
        p.qblocks = (tiles + p.threads - 1) / p.threads;
    } else {
        p.qblocks = (nq + (int64_t)p.threads * p.qx - 1) / ((int64_t)p.threads * p.qx);
    }
    // per_sm CTAs fit on an SM. Split the face (event) loop when the query CTAs alone would leave
    // the GPU under-filled (fewer than ~4 waves), keeping at least 2 tiles per split.
    const int64_t slots = per_sm * num_sms;
    int nsplit = 1;
    if (p.qblocks < 4 * slots) {
        const int64_t want = (4 * slots + p.qblocks - 1) / p.qblocks;
        const int64_t maxs = (nrec + 2 * tile - 1) / (2 * tile);
        nsplit = (int)(want < maxs ? want : maxs);
        if (nsplit < 1) nsplit = 1;
        if (nsplit > 65535) nsplit = 65535;
    }
    int64_t fps = (nrec + nsplit - 1) / nsplit;
    fps = ((fps + tile - 1) / tile) * tile;  // whole tiles per split
    p.faces_per_split = fps;
    p.nsplit = (int)((nrec + fps - 1) / fps);
    return p;
}

cudaError_t launch_forward(const FwdPlan &p, const FaceRec *rec, int64_t nf, const StripRec *srec, int64_t ne,
                           const GridF *g, const float *queries, int64_t nq, int arith, float2 *partial, float *w_out,
                           uint8_t *occ_out, const uint8_t *near_flag, int *flag_list, int *flag_count,
                           const LaunchCtx &ctx) {
    FwdArgs a{};
    a.rec = rec;
    a.nf = nf;
    a.srec = srec;
    a.ne = ne;
    if (g) a.g = *g;
    a.queries = queries;
    a.nq = nq;
    a.faces_per_split = p.faces_per_split;
    a.nsplit = p.nsplit;
    a.partial = partial;
    a.w_out = w_out;
    a.occ_out = occ_out;
    a.near_flag = near_flag;
    a.flag_list = flag_list;
    a.flag_count = flag_count;
    a.err = ctx.d_err;
    a.skip_tile = ctx.test_skip_tile;
    a.wait_ns = ctx.wait_ns;
    dim3 grid((unsigned)p.qblocks, (unsigned)p.nsplit);
    const bool kahan = arith != kArithFP32;
    if (arith == kArithFP16 && queries) return cudaErrorNotSupported;
    if (queries && !p.strips) return cudaErrorInvalidValue;  // lists run in strip order only
    if (p.strips && (arith == kArithFP16 || !srec || ne < 1)) return cudaErrorInvalidValue;
    const char *name = queries    ? (kahan ? "fwd_list_strip_kahan" : "fwd_list_strip")
                       : p.strips ? (kahan ? "fwd_strip_kahan" : "fwd_strip")
                                  : (arith == kArithFP16 ? "fwd_grid_fp16" : (kahan ? "fwd_grid_kahan" : "fwd_grid"));
    prof_begin(name, ctx.stream);
    if (queries) {
        if (kahan)
            fwd_list_strip_kernel<kListQP, true><<<grid, kStripThreads, 0, ctx.stream>>>(a);
        else
            fwd_list_strip_kernel<kListQP, false><<<grid, kStripThreads, 0, ctx.stream>>>(a);
    } else {
        if (p.strips) {
            if (kahan)
                fwd_grid_strip_kernel<kStripQX, kStripQY, true><<<grid, kStripThreads, 0, ctx.stream>>>(a);
            else
                fwd_grid_strip_kernel<kStripQX, kStripQY, false><<<grid, kStripThreads, 0, ctx.stream>>>(a);
        } else if (arith == kArithFP16)
            fwd_grid_kernel<kGridQX, kGridQY, true, true><<<grid, kFwdThreads, 0, ctx.stream>>>(a);
        else if (kahan)
            fwd_grid_kernel<kGridQX, kGridQY, true, false><<<grid, kFwdThreads, 0, ctx.stream>>>(a);
        else
            fwd_grid_kernel<kGridQX, kGridQY, false, false><<<grid, kFwdThreads, 0, ctx.stream>>>(a);
    }
    count_launch();
    prof_end(name, ctx.stream);
    return cudaGetLastError();
}

cudaError_t launch_split_reduce(const FwdPlan &p, const float2 *partial, int64_t nq, float *w_out, uint8_t *occ_out,
                                const uint8_t *near_flag, int *flag_list, int *flag_count, cudaStream_t s) {
    FwdArgs a{};
    a.nq = nq;
    a.w_out = w_out;
    a.occ_out = occ_out;
    a.near_flag = near_flag;
    a.flag_list = flag_list;
    a.flag_count = flag_count;
    int64_t blocks = (nq + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    prof_begin("split_reduce", s);
    split_reduce_kernel<<<(unsigned)blocks, 256, 0, s>>>(partial, p.nsplit, a);
    count_launch();
    prof_end("split_reduce", s);
    return cudaGetLastError();
}

}  // namespace dv
