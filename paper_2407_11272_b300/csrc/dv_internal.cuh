// Internal declarations shared by the CUDA sources of libdv (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "atan_poly.h"

#include "dv_api.h"

namespace dv {

constexpr float kInv2Pi = 0.15915494309189535f;  // w = (1/4pi) sum Omega = (1/2pi) sum ATAN2
constexpr double kInv2PiD = 0.15915494309189533576888;
constexpr double kTwoPiD = 6.283185307179586476925;
constexpr float kNearDist = 1e-3f;    // re-evaluate queries within this distance of a triangle
constexpr float kThreshBand = 1e-3f;  // ... or with |w - 0.5| below this
constexpr unsigned kFull = 0xffffffffu;
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // bounded mbarrier waits: give up after 2 s

// Per-face FP32 record, 48 bytes = 3 x float4:
//   r0 = (v0.x, v0.y, v0.z, 8 n.x), r1 = (v1.x, v1.y, v1.z, 8 n.y), r2 = (v2.x, v2.y, v2.z, 8 n.z)
// with n = (v1 - v0) x (v2 - v0). The factor 8 (exact) lets the forward kernel test
// |N| < D/8 as one comparison and feed 8N/D straight into its arctangent polynomial.
constexpr float kNormalScale = 8.0f;
struct FaceRec {
    float4 r0, r1, r2;
};
static_assert(sizeof(FaceRec) == 48, "face record must be 48 bytes (TMA bulk copies need 16B multiples)");

// Per-face FP64 record for the re-evaluation pass: v0, v1, v2, n (12 doubles, 96 bytes).
struct FaceRec64 {
    double v[12];
};

// One event of the vertex-sharing strip order (strips.cu), FP32: the event's vertex and, if the
// event completes a face, that face's normal n_f pre-scaled by kNormalScale and flag = 1 (else
// n = 0, flag = 0). 32 bytes: TMA bulk copies of any run of events stay 16-byte aligned.
struct StripRec {
    float4 p;  // vx, vy, vz, 8 n.x
    float4 q;  // 8 n.y, 8 n.z, flag, 0
};
static_assert(sizeof(StripRec) == 32, "strip record must be 32 bytes");

// FP64 strip event for the re-evaluation pass: vertex, unscaled normal, flag (64 bytes).
struct StripRec64 {
    double v[3];
    double n[3];
    double flag;
    double pad;
};

// Two faces sharing an edge, for the grid adjoint (winding_bwd.cu; pairing in strips.cu):
// face A = (p0, p1, p2), face B = (p2, p1, p3), each with its unit-free normal n = e1 x e2 in
// that canonical orientation (FP32, the face record's 8 n / 8, negated for B when its input
// orientation is reversed). 80 bytes.
struct PairRec {
    float4 r0;  // p0, nA.x
    float4 r1;  // p1, nA.y
    float4 r2;  // p2, nA.z
    float4 r3;  // p3, nB.x
    float4 r4;  // nB.y, nB.z, 0, 0
};
static_assert(sizeof(PairRec) == 80, "pair record must be 80 bytes");

// One directed boundary edge p -> r of the mesh (net multiplicity m != 0 over all faces), for the
// boundary form of the adjoint (winding_bnd.cu). 32 bytes.
struct BndRec {
    float4 p;  // start vertex, m (as float)
    float4 r;  // end vertex, 0
};

// Cell-centred grid, FP32 form used by the FP32 kernels: x = lo + (i + 0.5) * h.
struct GridF {
    float lo[3];
    float h[3];
    int n[3];
};

// FP64 form for the re-evaluation: x = lo + (i + 0.5) * (hi - lo) / n in double.
struct GridD {
    double lo[3];
    double h[3];
    int n[3];
};

// ------------------------------------------------------------------------------------------
// Inline PTX: mbarrier + bulk async copy (TMA, non-tensor form) into this CTA's shared memory.

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of `bar`, giving up after kWaitLimitNs (or limit_ns if smaller than
// that). Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  uint64_t limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        for (int k = 0; k < 64; ++k)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_timer_ns() - t0 > limit_ns) return false;
    }
}

// 1-D bulk copy global -> shared, completion signalled on `bar` as transaction bytes.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ------------------------------------------------------------------------------------------
// FP32 special-function approximations (MUFU): reciprocal, reciprocal square root, square root.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ------------------------------------------------------------------------------------------
// Edge terms of the adjoint, shared by the face-pair and the boundary-curve forms: for a directed
// edge p -> r seen from q (a = p - q, b = r - q, d = r - p), dOmega/dp = (b x a) / (|a| t) with
// t = |a||b| + a.b. Where a and b point apart (q near the segment) that sum cancels: its FP32
// relative error grows like eps / (1 + cos(a, b)). There edge_t takes t = |a x b|^2 / (|a||b| - a.b)
// with a x b = a x d, whose denominator does not cancel and whose cross product has relative error
// ~ eps |a| / dist(q, edge).
__device__ __forceinline__ float edge_t(float ax, float ay, float az, float la, float lb, float ab, float dx, float dy,
                                        float dz) {
    if (ab >= 0.f) return fmaf(la, lb, ab);
    const float wx = fmaf(ay, dz, -az * dy), wy = fmaf(az, dx, -ax * dz), wz = fmaf(ax, dy, -ay * dx);
    return fmaf(wx, wx, fmaf(wy, wy, wz * wz)) / fmaf(la, lb, -ab);
}

// edge_t with a MUFU reciprocal in place of the division.
__device__ __forceinline__ float edge_t_approx(float ax, float ay, float az, float la, float lb, float ab, float dx,
                                               float dy, float dz) {
    if (ab >= 0.f) return fmaf(la, lb, ab);
    const float wx = fmaf(ay, dz, -az * dy), wy = fmaf(az, dx, -ax * dz), wz = fmaf(ax, dy, -ay * dx);
    return fmaf(wx, wx, fmaf(wy, wy, wz * wz)) * rcp_approx(fmaf(la, lb, -ab));
}

// Per-pair coefficients of the guarded paths of the list and boundary-form adjoints, from MUFU
// approximations (the cancellation near the segment is handled by edge_t's form, not by IEEE
// rounding): for a = p - q, b = r - q with squared lengths la2, lb2, sets ia = 1/|a|, ib = 1/|b|
// and c = g / t; returns false (skip the pair) for q within 1e-15 of an endpoint or on the
// segment, where the derivative does not exist. (The grid adjoint's guarded path keeps IEEE
// square roots and divisions: the same change there slowed that kernel's packed path.)
__device__ __forceinline__ bool edge_coeffs(float ax, float ay, float az, float bx, float by, float bz, float la2,
                                            float lb2, float dx, float dy, float dz, float g, float &ia, float &ib,
                                            float &c) {
    if (!(la2 > 1e-30f) || !(lb2 > 1e-30f)) return false;
    ia = rsqrt_approx(la2);
    ib = rsqrt_approx(lb2);
    const float la = la2 * ia, lb = lb2 * ib;
    const float t = edge_t_approx(ax, ay, az, la, lb, fmaf(ax, bx, fmaf(ay, by, az * bz)), dx, dy, dz);
    if (!(t > 1e-30f * la * lb) || !(t >= 1.2e-38f)) return false;
    c = g * rcp_approx(t);
    return true;
}

// Whether the grid row through (qy, qz) passes within kNearEdge |r - p| of the segment p -> r, from
// the row's offsets (ys, zs) = (p_y - qy, p_z - qz), (ye, ze) likewise for r, and the edge's squared
// length L2: the row is a line along x, so its distance to the segment is the distance from the
// origin to the segment's projection on the (y, z) plane. Beyond that distance every query of the
// row has 1 + cos(a, b) >= 7e-3, so the packed t's relative error stays below ~4e-5.
constexpr float kNearEdge = 0.03f;
__device__ __forceinline__ bool row_near_edge(float ys, float zs, float ye, float ze, float L2) {
    const float dy = ye - ys, dz = ze - zs;
    const float K = kNearEdge * kNearEdge * L2;
    const float sn = -fmaf(ys, dy, zs * dz), den = fmaf(dy, dy, dz * dz);
    if (sn <= 0.f) return fmaf(ys, ys, zs * zs) < K;
    if (sn >= den) return fmaf(ye, ye, ze * ze) < K;
    const float cr = fmaf(ys, dz, -zs * dy);  // distance to the projected line times sqrt(den)
    return cr * cr < K * den;
}

// Query lists: a query whose t = |a||b| + a.b falls below kNearCos |a.b| for some edge
// (1 + cos(a, b) < ~0.01: q near the segment, where the packed t cancels) sends its chunk through
// the guarded path; for the others the packed t's relative error stays below ~3e-5. The test is the
// sign of t + kNearCos a.b.
constexpr float kNearCos = 0.01f;

// Sticky error word: first error code wins.
__device__ __forceinline__ void set_error(int *err, int code) {
    if (err) atomicCAS(err, 0, code);
}

// ------------------------------------------------------------------------------------------
// Bounds checks of the debug build (libdv_debug.so, compiled with -DDV_DEBUG). The indexed global
// accesses of the hot kernels go through DV_INB(index, length, site). In the debug build an index
// outside [0, length) is counted, the first one is recorded with its site and length in this
// translation unit's device record, and the access is skipped: a wrong index shows up as a
// report (dv_debug_report), never as a memory fault or a trap. Release builds compile every check
// to `true`.
enum DebugSite : int {
    kSiteFwdTile = 1,      // forward: copy of a tile of face / strip records
    kSiteFwdOut = 2,       // forward epilogue: w, occupancy, near flag of a query
    kSiteFwdFlagList = 3,  // forward epilogue: slot of the flagged-query list
    kSiteFwdPartial = 4,   // forward: per-split partial sums
    kSiteReevalEvent = 5,  // FP64 pass: strip event record
    kSiteReevalQuery = 6,  // FP64 pass: flagged-list entry and the query it names
    kSiteBwdRecord = 7,    // adjoint: pair or face record, unpaired-face list
    kSiteBwdUpstream = 8,  // adjoint: upstream value of a query
    kSiteBwdFaceGrad = 9,  // adjoint: per-split face gradient
    kSiteGather = 10,      // vertex gather: CSR entry, face gradient, dL/dV
    kSiteNear = 11,        // near-surface flag of a grid query
    kSitePack = 12,        // packing: vertex of a face or of a strip event
};

struct DebugRecord {
    unsigned long long count;
    long long site, index, bound;
};
using DebugFetchFn = cudaError_t (*)(DebugRecord *out, bool clear);
// Registers one translation unit's record reader (dv_api.cu); returns the count so far.
int debug_register(DebugFetchFn fn);

#ifdef DV_DEBUG
namespace {
__device__ DebugRecord g_debug_record;  // this translation unit's record

__device__ __forceinline__ bool in_bounds(long long i, long long n, int site) {
    if (i >= 0 && i < n) return true;
    if (atomicAdd(&g_debug_record.count, 1ull) == 0ull) {
        g_debug_record.site = site;
        g_debug_record.index = i;
        g_debug_record.bound = n;
    }
    return false;
}

cudaError_t debug_fetch(DebugRecord *out, bool clear) {
    cudaError_t e = cudaMemcpyFromSymbol(out, g_debug_record, sizeof(DebugRecord));
    if (e == cudaSuccess && clear) {
        const DebugRecord z{};
        e = cudaMemcpyToSymbol(g_debug_record, &z, sizeof(DebugRecord));
    }
    return e;
}

[[maybe_unused]] const int g_debug_registered = debug_register(debug_fetch);
}  // namespace
#define DV_INB(i, n, site) (::dv::in_bounds((long long)(i), (long long)(n), (int)(site)))
#else
#define DV_INB(i, n, site) true
#endif

}  // namespace dv

// ------------------------------------------------------------------------------------------
// Host-side launch wrappers implemented in the .cu files (C++ linkage, internal).
namespace dv {

struct LaunchCtx {
    cudaStream_t stream;
    int *d_err;  // sticky device error word (may be null)
    // Self-test hooks of the forward's copy pipeline (dv_selftest_forward_timeout): a tile index
    // that no CTA issues (-1: none) and the limit of every bounded wait.
    int test_skip_tile = -1;
    uint64_t wait_ns = kWaitLimitNs;
};

// Kernel-profiling hooks (dv_api.cu): bracket one launch with events when enabled.
void prof_begin(const char *name, cudaStream_t s);
void prof_end(const char *name, cudaStream_t s);
void count_launch();
// Record `msg` as the calling thread's dv_last_error() text and return `s` (dv_api.cu).
dv_status report_error(dv_status s, const char *msg);

// pack.cu
cudaError_t launch_validate(const float *verts, int64_t nv, const int32_t *faces, int64_t nf, int *d_bad,
                            cudaStream_t s);
cudaError_t launch_pack(const float *verts, int64_t nv, const int32_t *faces, int64_t nf, FaceRec *rec,
                        FaceRec64 *rec64, cudaStream_t s);
// Strip events from the vertices and the packed face records (normals copied from rec/rec64, so
// both orders see the same n_f). Runs after launch_pack on the same stream.
cudaError_t launch_pack_strips(const float *verts, int64_t nv, int64_t nf, const int32_t *ev_vert,
                               const int32_t *ev_face, int64_t ne, const FaceRec *rec, const FaceRec64 *rec64,
                               StripRec *srec, StripRec64 *srec64, cudaStream_t s);

// winding_bnd.cu: the adjoint from the mesh's boundary edges.
constexpr int kBndPartFloats = 6;  // per (split, boundary edge): V_p (3), V_r (3)
struct BndPlan {
    int64_t eblocks;    // CTAs over boundary edges
    int nsplit;         // query (row) splits (grid dimension y)
    int64_t per_split;  // grid: rows per split; list: queries per split
};
BndPlan plan_boundary(int64_t nq, int64_t nb, bool grid, const GridF *g, int num_sms);
// Boundary records from the packed face records (vertex coordinates through the vertex CSR).
cudaError_t launch_pack_boundary(const FaceRec *frec, const int32_t *vptr, const int32_t *vcorner,
                                 const int32_t *edges, int64_t nb, BndRec *rec, cudaStream_t s);
// Per-split edge sums into part [nsplit][nb][8]; nothing to do when nb == 0.
cudaError_t launch_boundary_backward(const BndPlan &p, const BndRec *rec, int64_t nb, const GridF *g,
                                     const float *queries, int64_t nq, const float *upstream, float *part,
                                     cudaStream_t s);
// dverts [nv][3] (overwritten; 0 off the boundary) from the split sums, FP64, fixed order.
cudaError_t launch_boundary_gather(int64_t nv, const BndRec *rec, int64_t nb, const float *part, int nsplit,
                                   const int32_t *vptr, const int32_t *vend, float *dverts, cudaStream_t s);
// Directed edges with nonzero net multiplicity as (u, v, m) triples, and per vertex the list of
// (edge << 1 | endpoint) codes in edge order (CSR: vptr [nv + 1], vend [2 nb]); host.
void build_boundary(const int32_t *faces, int64_t nf, int64_t nv, std::vector<int32_t> &edges,
                    std::vector<int32_t> &vptr, std::vector<int32_t> &vend);

// strips.cu: vertex-sharing strip order of the faces (host, once per mesh).
void build_strips(const int32_t *faces, int64_t nf, int64_t nv, std::vector<int32_t> &ev_vert,
                  std::vector<int32_t> &ev_face);
// Edge-sharing face pairs from the strip order: pairs [np][8] = p0, p1, p2, p3, fA, fB, code, 0
// and the faces left unpaired (host).
void build_pairs(const int32_t *faces, int64_t nf, const std::vector<int32_t> &ev_vert,
                 const std::vector<int32_t> &ev_face, std::vector<int32_t> &pairs, std::vector<int32_t> &singles);
// Pair records from the packed face records (after launch_pack).
cudaError_t launch_pack_pairs(const FaceRec *rec, const int32_t *ptopo, int64_t np, PairRec *prec, cudaStream_t s);
cudaError_t launch_flipped_duplication(const float *verts, int64_t nv, const int32_t *faces, int64_t nf,
                                       const FaceRec64 *rec64, const int32_t *vtx_ptr, const int32_t *vtx_corner,
                                       double eps, float *out_verts, int32_t *out_faces, cudaStream_t s);
cudaError_t launch_gather_dverts(const double *unused, const float *face_grad, int nsplit, int64_t nf,
                                 const int32_t *vtx_ptr, const int32_t *vtx_corner, int64_t nv, float *dverts,
                                 cudaStream_t s);

// winding_fwd.cu
struct FwdPlan {
    int qx, qy;          // queries per thread along x and along y (grid kernels)
    int threads;         // CTA size
    int64_t qblocks;     // CTAs over queries
    int nsplit;          // face splits (grid dimension y); 1 = no split
    int64_t faces_per_split;  // faces, or strip events when strips is set
    bool strips;         // over the strip events (FP32 / Kahan arithmetic)
};
// n_events > 0 selects the strip-order kernels (FP32 or Kahan arithmetic, grid or list).
FwdPlan plan_forward(int64_t nq, int64_t nf, bool grid, const GridF *g, int num_sms, int64_t n_events = 0);
// Per-pair arithmetic of the forward: FP32 with a plain sum, FP32 with Kahan across face tiles,
// or the FP16 ablation (half2 per-pair terms, FP32 Kahan sums; grid queries only).
constexpr int kArithFP32 = 0, kArithKahan = 1, kArithFP16 = 2;
cudaError_t launch_forward(const FwdPlan &p, const FaceRec *rec, int64_t nf, const StripRec *srec, int64_t ne,
                           const GridF *g, const float *queries, int64_t nq, int arith, float2 *partial, float *w_out,
                           uint8_t *occ_out, const uint8_t *near_flag, int *flag_list, int *flag_count,
                           const LaunchCtx &ctx);
cudaError_t launch_split_reduce(const FwdPlan &p, const float2 *partial, int64_t nq, float *w_out, uint8_t *occ_out,
                                const uint8_t *near_flag, int *flag_list, int *flag_count, cudaStream_t s);

// near_surface.cu
// Near-surface flags (distance <= 1e-3, conservative). The list path needs `scratch` of
// near_list_scratch_ints(nq) ints (query bins); the grid path ignores it.
cudaError_t launch_near_surface(const FaceRec *rec, int64_t nf, const GridF *g, const float *queries, int64_t nq,
                                uint8_t *near_flag, int *scratch, cudaStream_t s);
int64_t near_list_scratch_ints(int64_t nq);

// winding_fp64.cu
// FP64 re-evaluation of the flagged queries over the strip events.
cudaError_t launch_reeval_fp64(const StripRec64 *srec64, int64_t ne, const GridD *g, const float *queries,
                               const int *flag_list, const int *flag_count, int64_t max_flagged, float *w_out,
                               uint8_t *occ_out, unsigned *stat_maxdiff_bits, int *stat_occ_changed, int num_sms,
                               cudaStream_t s);

// dipole.cu (Eq. (4) surrogate)
int dipole_bwd_splits(int64_t nq, int64_t nf, int num_sms);
cudaError_t launch_dipole_forward(const FaceRec *rec, int64_t nf, const GridF *g, const float *queries, int64_t nq,
                                  float *w_out, cudaStream_t s);
cudaError_t launch_dipole_backward(const FaceRec *rec, int64_t nf, const GridF *g, const float *queries, int64_t nq,
                                   const float *upstream, int nsplit, float *face_grad, cudaStream_t s);

// winding_bwd.cu
// The faces as the adjoint sees them: the face records, and for grid queries the edge-sharing
// pairs (records + topology) and the unpaired faces (prec == nullptr: every face alone).
struct BwdFaces {
    const FaceRec *rec;
    int64_t nf;
    const PairRec *prec;
    const int32_t *ptopo;  // [np][8]
    int64_t np;
    const int32_t *singles;  // [nsingle]
    int64_t nsingle;
};
struct BwdPlan {
    int threads;
    int64_t fblocks;         // CTAs along x: pair CTAs first (grid), then single-face CTAs
    int64_t pblocks;         // of which take pairs
    int nsplit;
    int64_t rows_per_split;  // grid: rows (z,y) per split; list: queries per split
};
// Kernel attributes of the adjoint on the current device (once; outside stream capture).
cudaError_t prepare_backward_kernels();
BwdPlan plan_backward(int64_t nq, const BwdFaces &fc, bool grid, const GridF *g, int num_sms);
cudaError_t launch_backward(const BwdPlan &p, const BwdFaces &fc, const GridF *g, const float *queries, int64_t nq,
                            const float *upstream, float *face_grad, const LaunchCtx &ctx);

}  // namespace dv
