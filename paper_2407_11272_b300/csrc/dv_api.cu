// Host side of the C ABI declared in include/dv_api.h: argument checks, the resident mesh
// (packed face records + vertex adjacency + scratch), launch planning, error reporting and the
// optional per-kernel event timing used by measurement tools.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/dv_api.h"
#include "dv_internal.cuh"

// An NVTX range around each host entry point, named after it, so that a timeline tool (Nsight
// Systems, ncu --nvtx) shows which call issued which kernels. NVTX is header-only: without a tool
// attached a range costs a few nanoseconds.
namespace {
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace
#define DV_NVTX_RANGE(name) const NvtxRange dv_nvtx_range_(name)

// ------------------------------------------------------------------------------------------
// Errors
static thread_local std::string g_last_error;

static dv_status fail(dv_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

#define DV_CUDA(call)                                                                                  \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess)                                                                         \
            return fail(e_ == cudaErrorMemoryAllocation ? DV_ERR_OOM : DV_ERR_CUDA, "%s: %s (%s:%d)", #call, \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                                   \
    } while (0)

// ------------------------------------------------------------------------------------------
// Launch counting and optional event timing
namespace dv {

static std::atomic<int64_t> g_launches{0};
static bool g_prof_on = false;
struct ProfRec {
    const char *name;
    cudaEvent_t a, b;
};
static std::vector<ProfRec> g_prof_pending;
struct ProfTot {
    const char *name;
    double ms;
    int64_t n;
};
static std::vector<ProfTot> g_prof_tot;
static std::mutex g_prof_mu;

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Readers of the debug build's per-translation-unit bounds records (registered at load time).
static std::vector<DebugFetchFn> &debug_fetchers() {
    static std::vector<DebugFetchFn> v;
    return v;
}

int debug_register(DebugFetchFn fn) {
    debug_fetchers().push_back(fn);
    return (int)debug_fetchers().size();
}

dv_status report_error(dv_status s, const char *msg) { return fail(s, "%s", msg); }

void prof_begin(const char *name, cudaStream_t s) {
    if (!g_prof_on) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    ProfRec r{name, nullptr, nullptr};
    cudaEventCreate(&r.a);
    cudaEventCreate(&r.b);
    cudaEventRecord(r.a, s);
    g_prof_pending.push_back(r);
}

void prof_end(const char *name, cudaStream_t s) {
    if (!g_prof_on) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto it = g_prof_pending.rbegin(); it != g_prof_pending.rend(); ++it)
        if (it->name == name) {
            cudaEventRecord(it->b, s);
            return;
        }
}

}  // namespace dv

// ------------------------------------------------------------------------------------------
// Mesh
struct dv_mesh {
    int device = 0;
    cudaStream_t last_stream = nullptr;  // stream of the most recent call (frees are ordered on it)
    int num_sms = 148;
    int64_t nv = 0, nf = 0;
    int32_t *faces = nullptr;       // device copy [nf][3]
    dv::FaceRec *rec = nullptr;     // [nf]
    dv::FaceRec64 *rec64 = nullptr; // [nf]
    int32_t *vtx_ptr = nullptr;     // [nv+1]
    int32_t *vtx_corner = nullptr;  // [3 nf]
    int64_t ne = 0;                       // strip events (strips.cu)
    int32_t *ev_vert = nullptr;           // [ne]
    int32_t *ev_face = nullptr;           // [ne], -1 for a strip's first two events
    dv::StripRec *srec = nullptr;         // [ne]
    dv::StripRec64 *srec64 = nullptr;     // [ne]
    int64_t np = 0, nsingle = 0;          // edge-sharing face pairs and unpaired faces (grid adjoint)
    int32_t *ptopo = nullptr;             // [np][8]
    dv::PairRec *prec = nullptr;          // [np]
    int32_t *singles = nullptr;           // [nsingle]
    // boundary edges (net multiplicity != 0), built on first use: host topology, then device copies
    std::vector<int32_t> hfaces;          // host copy of the faces [nf][3]
    bool bnd_host = false, bnd_dev = false;
    std::vector<int32_t> hb_edges, hb_vptr, hb_vend;
    int64_t nb = 0;
    int32_t *bnd_edges = nullptr;         // [nb][3]: u, v, m
    dv::BndRec *bnd_rec = nullptr;        // [nb]
    int32_t *bnd_vptr = nullptr;          // [nv + 1]
    int32_t *bnd_vend = nullptr;          // [2 nb]
    int *err = nullptr;             // sticky error word + small counters: [0]=err [1]=flag_count [2]=occ_changed [3]=maxdiff bits
    // scratch, grown on demand
    int64_t cap_q = 0;
    float *ws_w = nullptr;
    uint8_t *ws_near = nullptr;
    int *ws_list = nullptr;
    int64_t cap_partial = 0;  // float2 elements
    float2 *ws_partial = nullptr;
    int64_t cap_fg = 0;       // floats
    float *ws_fg = nullptr;
    int64_t cap_bins = 0;     // ints: query bins of the list path's near-surface selection
    int *ws_bins = nullptr;
    int64_t cap_bpart = 0;    // floats: per-split boundary-edge sums
    float *ws_bpart = nullptr;
};

namespace {

dv::BwdFaces bwd_faces(const dv_mesh *m) {
    return dv::BwdFaces{m->rec, m->nf, m->prec, m->ptopo, m->np, m->singles, m->nsingle};
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// All device memory of a mesh comes from the stream-ordered allocator (cudaMallocAsync /
// cudaFreeAsync on the calling stream): growing or releasing scratch never waits for the
// whole device, so meshes can come and go while other work runs (the request server).
template <typename T>
dv_status grow(T *&p, int64_t &cap, int64_t need, cudaStream_t s) {
    if (need <= cap) return DV_OK;
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMallocAsync((void **)&p, (size_t)need * sizeof(T), s);
    if (e != cudaSuccess) {
        p = nullptr;
        return fail(DV_ERR_OOM, "cudaMallocAsync(%lld bytes) failed: %s", (long long)(need * (int64_t)sizeof(T)),
                    cudaGetErrorString(e));
    }
    cap = need;
    return DV_OK;
}

dv_status reserve_queries(dv_mesh *m, int64_t nq, cudaStream_t s) {
    if (nq <= m->cap_q) return DV_OK;
    if (m->ws_w) cudaFreeAsync(m->ws_w, s);
    if (m->ws_near) cudaFreeAsync(m->ws_near, s);
    if (m->ws_list) cudaFreeAsync(m->ws_list, s);
    m->ws_w = nullptr;
    m->ws_near = nullptr;
    m->ws_list = nullptr;
    m->cap_q = 0;
    cudaError_t e = cudaMallocAsync((void **)&m->ws_w, (size_t)nq * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&m->ws_near, (size_t)nq, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&m->ws_list, (size_t)nq * sizeof(int), s);
    if (e != cudaSuccess) return fail(DV_ERR_OOM, "scratch for %lld queries: %s", (long long)nq, cudaGetErrorString(e));
    m->cap_q = nq;
    return DV_OK;
}

dv_status check_grid(const dv_grid *g) {
    for (int k = 0; k < 3; ++k) {
        if (g->n[k] < 1) return fail(DV_ERR_INVALID_ARG, "grid n[%d] = %d < 1", k, g->n[k]);
        if (!std::isfinite(g->lo[k]) || !std::isfinite(g->hi[k]) || !(g->hi[k] > g->lo[k]))
            return fail(DV_ERR_INVALID_ARG, "grid axis %d needs finite lo < hi", k);
    }
    const int64_t q = (int64_t)g->n[0] * g->n[1] * g->n[2];
    if (q > (int64_t)INT32_MAX) return fail(DV_ERR_UNSUPPORTED, "grid has %lld cells (max 2^31-1)", (long long)q);
    return DV_OK;
}

dv::GridF to_gridf(const dv_grid *g) {
    dv::GridF f{};
    for (int k = 0; k < 3; ++k) {
        f.lo[k] = g->lo[k];
        f.h[k] = (g->hi[k] - g->lo[k]) / (float)g->n[k];
        f.n[k] = g->n[k];
    }
    return f;
}

dv::GridD to_gridd(const dv_grid *g) {
    dv::GridD d{};
    for (int k = 0; k < 3; ++k) {
        d.lo[k] = (double)g->lo[k];
        d.h[k] = ((double)g->hi[k] - (double)g->lo[k]) / (double)g->n[k];
        d.n[k] = g->n[k];
    }
    return d;
}

// Shared argument checks for the query-list / grid choice. Sets *nq_out.
dv_status check_queries(const dv_mesh *m, const float *q, int64_t nq, const dv_grid *g, int64_t *nq_out) {
    if (!m) return fail(DV_ERR_INVALID_ARG, "mesh is NULL");
    if ((q == nullptr) == (g == nullptr)) return fail(DV_ERR_INVALID_ARG, "pass exactly one of d_queries or grid");
    if (g) {
        dv_status s = check_grid(g);
        if (s) return s;
        const int64_t n = (int64_t)g->n[0] * g->n[1] * g->n[2];
        if (nq != 0 && nq != n) return fail(DV_ERR_INVALID_ARG, "nq = %lld but the grid has %lld cells", (long long)nq,
                                            (long long)n);
        *nq_out = n;
    } else {
        if (nq < 1) return fail(DV_ERR_INVALID_ARG, "nq = %lld < 1", (long long)nq);
        if (nq > (int64_t)INT32_MAX) return fail(DV_ERR_UNSUPPORTED, "nq = %lld exceeds 2^31-1", (long long)nq);
        *nq_out = nq;
    }
    return DV_OK;
}

dv_status run_forward(dv_mesh *m, const float *queries, int64_t nq, const dv_grid *grid, float *w, uint8_t *occ,
                      dv_precision prec, dv_report *report, cudaStream_t s) {
    if (prec != DV_PREC_FP32 && prec != DV_PREC_FP32_KAHAN && prec != DV_PREC_MIXED && prec != DV_PREC_FP16)
        return fail(DV_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    if (prec == DV_PREC_FP16 && queries)
        return fail(DV_ERR_UNSUPPORTED, "the FP16 ablation is implemented for grid queries only");
    dv::GridF gf{};
    if (grid) gf = to_gridf(grid);
    const int64_t nev = prec != DV_PREC_FP16 ? m->ne : 0;  // strip order (all but the FP16 ablation)
    const dv::FwdPlan plan = dv::plan_forward(nq, m->nf, grid != nullptr, grid ? &gf : nullptr, m->num_sms, nev);
    const bool mixed = prec == DV_PREC_MIXED;
    dv_status st;
    m->last_stream = s;
    if (plan.nsplit > 1 && (st = grow(m->ws_partial, m->cap_partial, (int64_t)plan.nsplit * nq, s))) return st;
    if ((mixed || w == nullptr) && (st = reserve_queries(m, nq, s))) return st;
    if (w == nullptr) w = m->ws_w;
    const dv::LaunchCtx ctx{s, m->err};
    if (mixed) {
        DV_CUDA(cudaMemsetAsync(m->err + 1, 0, 3 * sizeof(int), s));
        DV_CUDA(cudaMemsetAsync(m->ws_near, 0, (size_t)nq, s));  // the near kernels only set flags
        if (queries && (st = grow(m->ws_bins, m->cap_bins, dv::near_list_scratch_ints(nq), s))) return st;
        DV_CUDA(dv::launch_near_surface(m->rec, m->nf, grid ? &gf : nullptr, queries, nq, m->ws_near, m->ws_bins,
                                        s));
    }
    int *list = mixed ? m->ws_list : nullptr;
    int *count = mixed ? m->err + 1 : nullptr;
    const uint8_t *nearf = mixed ? m->ws_near : nullptr;
    const int arith = prec == DV_PREC_FP16 ? dv::kArithFP16 : (prec == DV_PREC_FP32 ? dv::kArithFP32 : dv::kArithKahan);
    DV_CUDA(dv::launch_forward(plan, m->rec, m->nf, m->srec, m->ne, grid ? &gf : nullptr, queries, nq, arith,
                               m->ws_partial, w, occ, nearf, list, count, ctx));
    if (plan.nsplit > 1)
        DV_CUDA(dv::launch_split_reduce(plan, m->ws_partial, nq, w, occ, nearf, list, count, s));
    if (mixed) {
        dv::GridD gd{};
        if (grid) gd = to_gridd(grid);
        DV_CUDA(dv::launch_reeval_fp64(m->srec64, m->ne, grid ? &gd : nullptr, queries, list, count, nq, w, occ,
                                       (unsigned *)(m->err + 3), m->err + 2, m->num_sms, s));
    }
    if (report) {
        int h[4] = {0, 0, 0, 0};
        if (mixed) DV_CUDA(cudaMemcpyAsync(h, m->err, sizeof(h), cudaMemcpyDeviceToHost, s));
        DV_CUDA(cudaStreamSynchronize(s));
        report->n_queries = nq;
        report->n_faces = m->nf;
        report->n_flagged = h[1];
        report->n_occ_changed = h[2];
        float md;
        std::memcpy(&md, &h[3], sizeof(md));
        report->max_abs_fp32_vs_fp64 = mixed ? (double)md : 0.0;
    }
    return DV_OK;
}

}  // namespace

// ------------------------------------------------------------------------------------------
extern "C" {

int dv_abi_version(void) { return DV_ABI_VERSION; }

dv_status dv_debug_report(int64_t *count, int32_t *site, int64_t *index, int64_t *bound, int clear) {
    if (!count || !site || !index || !bound) return fail(DV_ERR_INVALID_ARG, "null output pointer");
    *count = 0;
    *site = 0;
    *index = *bound = 0;
#ifdef DV_DEBUG
    for (dv::DebugFetchFn fn : dv::debug_fetchers()) {
        dv::DebugRecord r{};
        const cudaError_t e = fn(&r, clear != 0);
        if (e != cudaSuccess) return fail(DV_ERR_CUDA, "debug record: %s", cudaGetErrorString(e));
        if (r.count && *count == 0) {
            *site = (int32_t)r.site;
            *index = r.index;
            *bound = r.bound;
        }
        *count += (int64_t)r.count;
    }
    return DV_OK;
#else
    (void)clear;
    return fail(DV_ERR_UNSUPPORTED, "bounds checks exist only in the debug build (libdv_debug.so)");
#endif
}

const char *dv_status_string(dv_status s) {
    switch (s) {
        case DV_OK: return "DV_OK";
        case DV_ERR_INVALID_ARG: return "DV_ERR_INVALID_ARG";
        case DV_ERR_INVALID_MESH: return "DV_ERR_INVALID_MESH";
        case DV_ERR_OOM: return "DV_ERR_OOM";
        case DV_ERR_CUDA: return "DV_ERR_CUDA";
        case DV_ERR_TIMEOUT: return "DV_ERR_TIMEOUT";
        case DV_ERR_UNSUPPORTED: return "DV_ERR_UNSUPPORTED";
    }
    return "DV_ERR_UNKNOWN";
}

const char *dv_last_error(void) { return g_last_error.c_str(); }

void dv_mesh_destroy(dv_mesh *m) {
    if (!m) return;
    DeviceGuard dg(m->device);
    void *bufs[] = {m->faces,   m->rec,     m->rec64, m->vtx_ptr, m->vtx_corner, m->ev_vert,    m->ev_face,
                    m->srec,    m->srec64,  m->err,   m->ws_w,    m->ws_near,    m->ws_list,    m->ws_partial,
                    m->ws_fg,   m->ws_bins, m->bnd_edges, m->bnd_rec, m->bnd_vptr, m->bnd_vend, m->ws_bpart,
                    m->ptopo,   m->prec,    m->singles};
    for (void *b : bufs)
        if (b) cudaFreeAsync(b, m->last_stream);
    delete m;
}

namespace {
// The body of dv_mesh_create; `m` is set as soon as the mesh object exists so that the caller
// can release it if a host allocation throws.
dv_status mesh_create_impl(const float *d_verts, int64_t nv, const int32_t *d_faces, int64_t nf, void *stream,
                           dv_mesh **out, dv_mesh *&held) {
    if (!out) return fail(DV_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!d_verts || !d_faces) return fail(DV_ERR_INVALID_ARG, "vertex or face pointer is NULL");
    if (nv < 3) return fail(DV_ERR_INVALID_ARG, "nv = %lld < 3", (long long)nv);
    if (nf < 1) return fail(DV_ERR_INVALID_ARG, "nf = %lld < 1", (long long)nf);
    if (nv > (int64_t)INT32_MAX || 3 * nf > (int64_t)INT32_MAX)
        return fail(DV_ERR_UNSUPPORTED, "mesh too large (nv %lld, nf %lld)", (long long)nv, (long long)nf);
    cudaStream_t s = (cudaStream_t)stream;
    dv_mesh *m = new dv_mesh();
    held = m;
    m->nv = nv;
    m->nf = nf;
    cudaGetDevice(&m->device);
    cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, m->device);
    auto bail = [&](dv_status st) {
        dv_mesh_destroy(m);
        return st;
    };
    cudaError_t e = cudaSuccess;
    m->last_stream = s;
    e = cudaMallocAsync((void **)&m->faces, (size_t)nf * 3 * sizeof(int32_t), s);
    if (!e) e = cudaMallocAsync((void **)&m->rec, (size_t)nf * sizeof(dv::FaceRec), s);
    if (!e) e = cudaMallocAsync((void **)&m->rec64, (size_t)nf * sizeof(dv::FaceRec64), s);
    if (!e) e = cudaMallocAsync((void **)&m->vtx_ptr, (size_t)(nv + 1) * sizeof(int32_t), s);
    if (!e) e = cudaMallocAsync((void **)&m->vtx_corner, (size_t)nf * 3 * sizeof(int32_t), s);
    if (!e) e = cudaMallocAsync((void **)&m->err, 4 * sizeof(int), s);
    if (e) return bail(fail(DV_ERR_OOM, "mesh storage: %s", cudaGetErrorString(e)));
    if ((e = cudaMemsetAsync(m->err, 0, 4 * sizeof(int), s))) return bail(fail(DV_ERR_CUDA, "%s", cudaGetErrorString(e)));
    if ((e = dv::launch_validate(d_verts, nv, d_faces, nf, m->err, s)))
        return bail(fail(DV_ERR_CUDA, "validate: %s", cudaGetErrorString(e)));
    int bad = 0;
    std::vector<int32_t> hf((size_t)nf * 3);
    if ((e = cudaMemcpyAsync(&bad, m->err, sizeof(int), cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemcpyAsync(hf.data(), d_faces, hf.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s)))
        return bail(fail(DV_ERR_CUDA, "mesh create: %s", cudaGetErrorString(e)));
    if (bad == 1) return bail(fail(DV_ERR_INVALID_MESH, "a face index is outside [0, %lld)", (long long)nv));
    if (bad == 2) return bail(fail(DV_ERR_INVALID_MESH, "a vertex coordinate is not finite"));
    // Host topology: the vertex -> (face, corner) CSR (deterministic gather), the strip order of
    // the faces (forward passes) and the adjoint's face pairs. The boundary edges (boundary form
    // of the adjoint) are built on first use from the host copy of the faces kept here.
    std::vector<int32_t> ptr((size_t)nv + 1, 0), corner((size_t)nf * 3);
    for (int64_t i = 0; i < 3 * nf; ++i) ptr[(size_t)hf[i] + 1]++;
    for (int64_t v = 0; v < nv; ++v) ptr[v + 1] += ptr[v];
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    for (int64_t i = 0; i < 3 * nf; ++i) corner[(size_t)fill[hf[i]]++] = (int32_t)i;
    std::vector<int32_t> ev_vert, ev_face, p_topo, p_singles;
    dv::build_strips(hf.data(), nf, nv, ev_vert, ev_face);
    dv::build_pairs(hf.data(), nf, ev_vert, ev_face, p_topo, p_singles);
    m->ne = (int64_t)ev_vert.size();
    e = cudaMallocAsync((void **)&m->ev_vert, (size_t)m->ne * sizeof(int32_t), s);
    if (!e) e = cudaMallocAsync((void **)&m->ev_face, (size_t)m->ne * sizeof(int32_t), s);
    if (!e) e = cudaMallocAsync((void **)&m->srec, (size_t)m->ne * sizeof(dv::StripRec), s);
    if (!e) e = cudaMallocAsync((void **)&m->srec64, (size_t)m->ne * sizeof(dv::StripRec64), s);
    if (e) return bail(fail(DV_ERR_OOM, "strip storage: %s", cudaGetErrorString(e)));
    m->np = (int64_t)p_topo.size() / 8;
    m->nsingle = (int64_t)p_singles.size();
    if (m->np > 0) e = cudaMallocAsync((void **)&m->ptopo, p_topo.size() * sizeof(int32_t), s);
    if (!e && m->np > 0) e = cudaMallocAsync((void **)&m->prec, (size_t)m->np * sizeof(dv::PairRec), s);
    if (!e && m->nsingle > 0) e = cudaMallocAsync((void **)&m->singles, p_singles.size() * sizeof(int32_t), s);
    if (e) return bail(fail(DV_ERR_OOM, "face pair storage: %s", cudaGetErrorString(e)));
    if ((m->np > 0 && (e = cudaMemcpyAsync(m->ptopo, p_topo.data(), p_topo.size() * sizeof(int32_t),
                                           cudaMemcpyHostToDevice, s))) ||
        (m->nsingle > 0 && (e = cudaMemcpyAsync(m->singles, p_singles.data(), p_singles.size() * sizeof(int32_t),
                                                cudaMemcpyHostToDevice, s))))
        return bail(fail(DV_ERR_CUDA, "face pair upload: %s", cudaGetErrorString(e)));
    if ((e = cudaMemcpyAsync(m->vtx_ptr, ptr.data(), ptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(m->vtx_corner, corner.data(), corner.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                             s)) ||
        (e = cudaMemcpyAsync(m->ev_vert, ev_vert.data(), ev_vert.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                             s)) ||
        (e = cudaMemcpyAsync(m->ev_face, ev_face.data(), ev_face.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                             s)) ||
        (e = cudaMemcpyAsync(m->faces, d_faces, (size_t)nf * 3 * sizeof(int32_t), cudaMemcpyDeviceToDevice, s)))
        return bail(fail(DV_ERR_CUDA, "mesh upload: %s", cudaGetErrorString(e)));
    if ((e = dv::prepare_backward_kernels()))
        return bail(fail(DV_ERR_CUDA, "kernel attributes: %s", cudaGetErrorString(e)));
    if ((e = dv::launch_pack(d_verts, nv, m->faces, nf, m->rec, m->rec64, s)) ||
        (e = dv::launch_pack_strips(d_verts, nv, nf, m->ev_vert, m->ev_face, m->ne, m->rec, m->rec64, m->srec,
                                         m->srec64, s)) ||
        (e = dv::launch_pack_pairs(m->rec, m->ptopo, m->np, m->prec, s)))
        return bail(fail(DV_ERR_CUDA, "pack: %s", cudaGetErrorString(e)));
    // the host vectors above must outlive the async uploads
    if ((e = cudaStreamSynchronize(s))) return bail(fail(DV_ERR_CUDA, "mesh create: %s", cudaGetErrorString(e)));
    m->hfaces.swap(hf);
    *out = m;
    return DV_OK;
}
}  // namespace

dv_status dv_mesh_create(const float *d_verts, int64_t nv, const int32_t *d_faces, int64_t nf, void *stream,
                         dv_mesh **out) {
    DV_NVTX_RANGE("dv_mesh_create");
    g_last_error.clear();
    dv_mesh *held = nullptr;
    try {
        return mesh_create_impl(d_verts, nv, d_faces, nf, stream, out, held);
    } catch (const std::bad_alloc &) {
        // a host vector could not grow; the device buffers made so far are released in stream order
        if (out) *out = nullptr;
        if (held) dv_mesh_destroy(held);
        return fail(DV_ERR_OOM, "host memory while building the mesh");
    }
}

dv_status dv_mesh_update_verts(dv_mesh *m, const float *d_verts, void *stream) {
    DV_NVTX_RANGE("dv_mesh_update_verts");
    if (!m || !d_verts) return fail(DV_ERR_INVALID_ARG, "mesh or vertex pointer is NULL");
    DeviceGuard dg(m->device);
    m->last_stream = (cudaStream_t)stream;
    DV_CUDA(dv::launch_pack(d_verts, m->nv, m->faces, m->nf, m->rec, m->rec64, (cudaStream_t)stream));
    DV_CUDA(dv::launch_pack_strips(d_verts, m->nv, m->nf, m->ev_vert, m->ev_face, m->ne, m->rec, m->rec64, m->srec,
                                   m->srec64, (cudaStream_t)stream));
    DV_CUDA(dv::launch_pack_pairs(m->rec, m->ptopo, m->np, m->prec, (cudaStream_t)stream));
    if (m->bnd_dev)
        DV_CUDA(dv::launch_pack_boundary(m->rec, m->vtx_ptr, m->vtx_corner, m->bnd_edges, m->nb, m->bnd_rec,
                                         (cudaStream_t)stream));
    return DV_OK;
}

dv_status dv_mesh_reserve(dv_mesh *m, const dv_grid *grid, int64_t max_list_queries) {
    DV_NVTX_RANGE("dv_mesh_reserve");
    if (!m || max_list_queries < 0) return fail(DV_ERR_INVALID_ARG, "bad reserve arguments");
    DeviceGuard dg(m->device);
    dv_status st;
    int64_t nq = max_list_queries, part = 0, fg = 0;
    if (max_list_queries > 0) {
        const dv::FwdPlan fp = dv::plan_forward(max_list_queries, m->nf, false, nullptr, m->num_sms, m->ne);
        const dv::BwdPlan bp = dv::plan_backward(max_list_queries, bwd_faces(m), false, nullptr, m->num_sms);
        part = fp.nsplit > 1 ? (int64_t)fp.nsplit * max_list_queries : 0;
        fg = (int64_t)bp.nsplit * m->nf * 9;
    }
    if (grid) {
        if ((st = check_grid(grid))) return st;
        const dv::GridF gf = to_gridf(grid);
        const int64_t gq = (int64_t)grid->n[0] * grid->n[1] * grid->n[2];
        // the strip plan (FP32 / Kahan / mixed) and the face plan (FP16 ablation)
        const dv::FwdPlan fp = dv::plan_forward(gq, m->nf, true, &gf, m->num_sms, m->ne);
        const dv::FwdPlan fp16 = dv::plan_forward(gq, m->nf, true, &gf, m->num_sms);
        const dv::BwdPlan bp = dv::plan_backward(gq, bwd_faces(m), true, &gf, m->num_sms);
        nq = std::max(nq, gq);
        part = std::max(part, fp.nsplit > 1 ? (int64_t)fp.nsplit * gq : (int64_t)0);
        part = std::max(part, fp16.nsplit > 1 ? (int64_t)fp16.nsplit * gq : (int64_t)0);
        fg = std::max(fg, (int64_t)bp.nsplit * m->nf * 9);
    }
    cudaStream_t s = m->last_stream;
    if ((st = reserve_queries(m, nq, s))) return st;
    if (part > 0 && (st = grow(m->ws_partial, m->cap_partial, part, s))) return st;
    if (fg > 0 && (st = grow(m->ws_fg, m->cap_fg, fg, s))) return st;
    if (max_list_queries > 0 &&
        (st = grow(m->ws_bins, m->cap_bins, dv::near_list_scratch_ints(max_list_queries), s)))
        return st;
    DV_CUDA(cudaStreamSynchronize(s));
    return DV_OK;
}

int64_t dv_mesh_num_verts(const dv_mesh *m) { return m ? m->nv : -1; }
int64_t dv_mesh_num_faces(const dv_mesh *m) { return m ? m->nf : -1; }

dv_status dv_mesh_check(dv_mesh *m, void *stream) {
    if (!m) return fail(DV_ERR_INVALID_ARG, "mesh is NULL");
    DeviceGuard dg(m->device);
    int code = 0;
    DV_CUDA(cudaMemcpyAsync(&code, m->err, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    DV_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    if (code) {
        DV_CUDA(cudaMemsetAsync(m->err, 0, sizeof(int), (cudaStream_t)stream));
        DV_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
        return fail((dv_status)code, "device error word was %d", code);
    }
    return DV_OK;
}

dv_status dv_selftest_forward_timeout(dv_mesh *m, const dv_grid *grid, float *d_out_w, int64_t skip_tile,
                                      int64_t limit_us, void *stream) {
    int64_t n = 0;
    if (!grid) return fail(DV_ERR_INVALID_ARG, "grid is NULL");
    dv_status st = check_queries(m, nullptr, 0, grid, &n);
    if (st) return st;
    if (!d_out_w) return fail(DV_ERR_INVALID_ARG, "d_out_w is NULL");
    if (skip_tile < 0 || skip_tile > (int64_t)INT32_MAX)
        return fail(DV_ERR_INVALID_ARG, "skip_tile = %lld outside [0, 2^31-1]", (long long)skip_tile);
    if (limit_us < 1 || limit_us > 10000000)
        return fail(DV_ERR_INVALID_ARG, "limit_us = %lld outside [1, 1e7]", (long long)limit_us);
    DeviceGuard dg(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    const dv::GridF gf = to_gridf(grid);
    const dv::FwdPlan plan = dv::plan_forward(n, m->nf, true, &gf, m->num_sms, m->ne);
    m->last_stream = s;
    if (plan.nsplit > 1 && (st = grow(m->ws_partial, m->cap_partial, (int64_t)plan.nsplit * n, s))) return st;
    dv::LaunchCtx ctx{s, m->err};
    ctx.test_skip_tile = (int)skip_tile;
    ctx.wait_ns = (uint64_t)limit_us * 1000ull;
    DV_CUDA(dv::launch_forward(plan, m->rec, m->nf, m->srec, m->ne, &gf, nullptr, n, dv::kArithKahan, m->ws_partial,
                               d_out_w, nullptr, nullptr, nullptr, nullptr, ctx));
    if (plan.nsplit > 1)
        DV_CUDA(dv::launch_split_reduce(plan, m->ws_partial, n, d_out_w, nullptr, nullptr, nullptr, nullptr, s));
    int code = 0;
    DV_CUDA(cudaMemcpyAsync(&code, m->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    DV_CUDA(cudaStreamSynchronize(s));
    if (code) return fail((dv_status)code, "device error word is %d after the self-test forward", code);
    return DV_OK;
}

dv_status dv_winding(const dv_mesh *mesh, const float *d_queries, int64_t nq, const dv_grid *grid, float *d_out_w,
                     dv_precision prec, void *stream) {
    DV_NVTX_RANGE("dv_winding");
    int64_t n = 0;
    dv_status st = check_queries(mesh, d_queries, nq, grid, &n);
    if (st) return st;
    if (!d_out_w) return fail(DV_ERR_INVALID_ARG, "d_out_w is NULL");
    dv_mesh *m = const_cast<dv_mesh *>(mesh);
    DeviceGuard dg(m->device);
    return run_forward(m, d_queries, n, grid, d_out_w, nullptr, prec, nullptr, (cudaStream_t)stream);
}

dv_status dv_voxelize_grid(const dv_mesh *mesh, const dv_grid *grid, float *d_out_w, uint8_t *d_out_occ,
                           dv_precision prec, dv_report *report, void *stream) {
    DV_NVTX_RANGE("dv_voxelize_grid");
    int64_t n = 0;
    if (!grid) return fail(DV_ERR_INVALID_ARG, "grid is NULL");
    dv_status st = check_queries(mesh, nullptr, 0, grid, &n);
    if (st) return st;
    if (!d_out_occ) return fail(DV_ERR_INVALID_ARG, "d_out_occ is NULL");
    dv_mesh *m = const_cast<dv_mesh *>(mesh);
    DeviceGuard dg(m->device);
    return run_forward(m, nullptr, n, grid, d_out_w, d_out_occ, prec, report, (cudaStream_t)stream);
}

dv_status dv_winding_backward(const dv_mesh *mesh, const float *d_queries, int64_t nq, const dv_grid *grid,
                              const float *d_upstream, float *d_dverts, void *stream) {
    DV_NVTX_RANGE("dv_winding_backward");
    int64_t n = 0;
    dv_status st = check_queries(mesh, d_queries, nq, grid, &n);
    if (st) return st;
    if (!d_upstream || !d_dverts) return fail(DV_ERR_INVALID_ARG, "d_upstream or d_dverts is NULL");
    dv_mesh *m = const_cast<dv_mesh *>(mesh);
    DeviceGuard dg(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    dv::GridF gf{};
    if (grid) gf = to_gridf(grid);
    const dv::BwdPlan plan = dv::plan_backward(n, bwd_faces(m), grid != nullptr, grid ? &gf : nullptr, m->num_sms);
    m->last_stream = s;
    if ((st = grow(m->ws_fg, m->cap_fg, (int64_t)plan.nsplit * m->nf * 9, s))) return st;
    const dv::LaunchCtx ctx{s, m->err};
    DV_CUDA(dv::launch_backward(plan, bwd_faces(m), grid ? &gf : nullptr, d_queries, n, d_upstream, m->ws_fg, ctx));
    DV_CUDA(dv::launch_gather_dverts(nullptr, m->ws_fg, plan.nsplit, m->nf, m->vtx_ptr, m->vtx_corner, m->nv, d_dverts,
                                     s));
    return DV_OK;
}

namespace {
// Boundary edges of the mesh on the host (once).
dv_status boundary_host(dv_mesh *m) {
    if (m->bnd_host) return DV_OK;
    try {
        dv::build_boundary(m->hfaces.data(), m->nf, m->nv, m->hb_edges, m->hb_vptr, m->hb_vend);
    } catch (const std::bad_alloc &) {
        return fail(DV_ERR_OOM, "host memory while building the boundary edges");
    }
    m->nb = (int64_t)m->hb_edges.size() / 3;
    m->bnd_host = true;
    return DV_OK;
}

// ... and on the device, packed from the current face records (once; dv_mesh_update_verts
// repacks them from then on).
dv_status boundary_device(dv_mesh *m, cudaStream_t s) {
    dv_status st = boundary_host(m);
    if (st || m->bnd_dev) return st;
    cudaError_t e = cudaMallocAsync((void **)&m->bnd_vptr, m->hb_vptr.size() * sizeof(int32_t), s);
    if (!e && m->nb > 0) e = cudaMallocAsync((void **)&m->bnd_edges, m->hb_edges.size() * sizeof(int32_t), s);
    if (!e && m->nb > 0) e = cudaMallocAsync((void **)&m->bnd_rec, (size_t)m->nb * sizeof(dv::BndRec), s);
    if (!e && m->nb > 0) e = cudaMallocAsync((void **)&m->bnd_vend, m->hb_vend.size() * sizeof(int32_t), s);
    auto release = [&] {  // a later call starts over
        for (void **p : {(void **)&m->bnd_vptr, (void **)&m->bnd_edges, (void **)&m->bnd_rec, (void **)&m->bnd_vend})
            if (*p) {
                cudaFreeAsync(*p, s);
                *p = nullptr;
            }
    };
    if (e) {
        release();
        return fail(DV_ERR_OOM, "boundary storage: %s", cudaGetErrorString(e));
    }
    if ((e = cudaMemcpyAsync(m->bnd_vptr, m->hb_vptr.data(), m->hb_vptr.size() * sizeof(int32_t),
                             cudaMemcpyHostToDevice, s)) ||
        (m->nb > 0 && (e = cudaMemcpyAsync(m->bnd_edges, m->hb_edges.data(), m->hb_edges.size() * sizeof(int32_t),
                                           cudaMemcpyHostToDevice, s))) ||
        (m->nb > 0 && (e = cudaMemcpyAsync(m->bnd_vend, m->hb_vend.data(), m->hb_vend.size() * sizeof(int32_t),
                                           cudaMemcpyHostToDevice, s))) ||
        (e = dv::launch_pack_boundary(m->rec, m->vtx_ptr, m->vtx_corner, m->bnd_edges, m->nb, m->bnd_rec, s))) {
        release();
        return fail(DV_ERR_CUDA, "boundary upload: %s", cudaGetErrorString(e));
    }
    m->bnd_dev = true;
    return DV_OK;
}
}  // namespace

dv_status dv_winding_backward_boundary(const dv_mesh *mesh, const float *d_queries, int64_t nq, const dv_grid *grid,
                                       const float *d_upstream, float *d_dverts, void *stream) {
    DV_NVTX_RANGE("dv_winding_backward_boundary");
    int64_t n = 0;
    dv_status st = check_queries(mesh, d_queries, nq, grid, &n);
    if (st) return st;
    if (!d_upstream || !d_dverts) return fail(DV_ERR_INVALID_ARG, "d_upstream or d_dverts is NULL");
    dv_mesh *m = const_cast<dv_mesh *>(mesh);
    DeviceGuard dg(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    dv::GridF gf{};
    if (grid) gf = to_gridf(grid);
    m->last_stream = s;
    if ((st = boundary_device(m, s))) return st;
    const dv::BndPlan plan = dv::plan_boundary(n, m->nb, grid != nullptr, grid ? &gf : nullptr, m->num_sms);
    const int64_t bpart = (int64_t)plan.nsplit * m->nb * dv::kBndPartFloats;
    if (m->nb > 0 && (st = grow(m->ws_bpart, m->cap_bpart, bpart, s))) return st;
    DV_CUDA(dv::launch_boundary_backward(plan, m->bnd_rec, m->nb, grid ? &gf : nullptr, d_queries, n, d_upstream,
                                         m->ws_bpart, s));
    DV_CUDA(dv::launch_boundary_gather(m->nv, m->bnd_rec, m->nb, m->ws_bpart, plan.nsplit, m->bnd_vptr, m->bnd_vend,
                                       d_dverts, s));
    return DV_OK;
}

int64_t dv_mesh_num_strip_events(const dv_mesh *mesh) { return mesh ? mesh->ne : -1; }

int64_t dv_mesh_num_boundary_edges(const dv_mesh *mesh) {
    if (!mesh) return -1;
    dv_mesh *m = const_cast<dv_mesh *>(mesh);
    return boundary_host(m) == DV_OK ? m->nb : -1;
}

// ------------------------------------------------------------------------------------------
// Batches of independent requests as one CUDA graph (request server).
namespace {

constexpr int kBranches = 16;
struct BatchRes {
    bool ready = false;
    cudaStream_t branch[kBranches];
    cudaEvent_t fork, join[kBranches];
    std::vector<std::pair<cudaEvent_t, cudaGraphExec_t>> pending;  // launched graphs, freed once done
};
std::mutex g_batch_mu;
BatchRes g_batch[64];

cudaError_t batch_resources(int dev, BatchRes **out) {
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    BatchRes &r = g_batch[dev];
    if (!r.ready) {
        cudaError_t e = cudaEventCreateWithFlags(&r.fork, cudaEventDisableTiming);
        for (int i = 0; i < kBranches && e == cudaSuccess; ++i) {
            e = cudaStreamCreateWithFlags(&r.branch[i], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r.join[i], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return e;
        r.ready = true;
    }
    // release the executable graphs of batches that have finished
    for (auto it = r.pending.begin(); it != r.pending.end();) {
        if (cudaEventQuery(it->first) == cudaSuccess) {
            cudaGraphExecDestroy(it->second);
            cudaEventDestroy(it->first);
            it = r.pending.erase(it);
        } else {
            ++it;
        }
    }
    *out = &r;
    return cudaSuccess;
}

// Scratch a forward / adjoint of this request will use, allocated in stream order on s.
dv_status reserve_request(dv_mesh *m, const dv_request &r, dv_precision prec, cudaStream_t s) {
    const int64_t nq = (int64_t)r.grid.n[0] * r.grid.n[1] * r.grid.n[2];
    const dv::GridF gf = to_gridf(&r.grid);
    const dv::FwdPlan fp = dv::plan_forward(nq, m->nf, true, &gf, m->num_sms, prec != DV_PREC_FP16 ? m->ne : 0);
    dv_status st;
    m->last_stream = s;
    if (fp.nsplit > 1 && (st = grow(m->ws_partial, m->cap_partial, (int64_t)fp.nsplit * nq, s))) return st;
    if ((prec == DV_PREC_MIXED || r.d_out_w == nullptr) && (st = reserve_queries(m, nq, s))) return st;
    if (r.d_upstream) {
        const dv::BwdPlan bp = dv::plan_backward(nq, bwd_faces(m), true, &gf, m->num_sms);
        if ((st = grow(m->ws_fg, m->cap_fg, (int64_t)bp.nsplit * m->nf * 9, s))) return st;
    }
    return DV_OK;
}

dv_status backward_on(dv_mesh *m, const dv_grid *grid, int64_t nq, const float *up, float *dverts, cudaStream_t s) {
    const dv::GridF gf = to_gridf(grid);
    const dv::BwdPlan plan = dv::plan_backward(nq, bwd_faces(m), true, &gf, m->num_sms);
    dv_status st;
    if ((st = grow(m->ws_fg, m->cap_fg, (int64_t)plan.nsplit * m->nf * 9, s))) return st;
    const dv::LaunchCtx ctx{s, m->err};
    DV_CUDA(dv::launch_backward(plan, bwd_faces(m), &gf, nullptr, nq, up, m->ws_fg, ctx));
    DV_CUDA(dv::launch_gather_dverts(nullptr, m->ws_fg, plan.nsplit, m->nf, m->vtx_ptr, m->vtx_corner, m->nv, dverts,
                                     s));
    return DV_OK;
}

}  // namespace

dv_status dv_run_batch(const dv_request *reqs, int n, dv_precision prec, void *stream) {
    DV_NVTX_RANGE("dv_run_batch");
    if (n < 0 || (n > 0 && !reqs)) return fail(DV_ERR_INVALID_ARG, "bad request array");
    if (n == 0) return DV_OK;
    if (prec != DV_PREC_FP32 && prec != DV_PREC_FP32_KAHAN && prec != DV_PREC_MIXED && prec != DV_PREC_FP16)
        return fail(DV_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    if (stream == nullptr || (cudaStream_t)stream == cudaStreamLegacy || (cudaStream_t)stream == cudaStreamPerThread)
        return fail(DV_ERR_INVALID_ARG, "dv_run_batch captures a CUDA graph on `stream`: pass a created stream, "
                                        "not the default stream");
    int dev = -1;
    for (int i = 0; i < n; ++i) {
        const dv_request &r = reqs[i];
        if (!r.mesh || !r.d_out_occ) return fail(DV_ERR_INVALID_ARG, "request %d: mesh and d_out_occ are required", i);
        if (r.d_upstream && !r.d_dverts) return fail(DV_ERR_INVALID_ARG, "request %d: d_dverts is required", i);
        dv_status st = check_grid(&r.grid);
        if (st) return st;
        if (dev < 0) dev = r.mesh->device;
        if (r.mesh->device != dev) return fail(DV_ERR_INVALID_ARG, "all meshes of a batch must be on one device");
        for (int j = 0; j < i; ++j)
            if (reqs[j].mesh == r.mesh) return fail(DV_ERR_INVALID_ARG, "a mesh appears twice in one batch");
    }
    DeviceGuard dg(dev);
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_batch_mu);
    BatchRes *br = nullptr;
    DV_CUDA(batch_resources(dev, &br));
    for (int i = 0; i < n; ++i) {
        dv_status st = reserve_request(const_cast<dv_mesh *>(reqs[i].mesh), reqs[i], prec, s);
        if (st) return st;
    }
    // Capture: fork one branch per request (round-robin over the branch streams), join all.
    DV_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    dv_status st = DV_OK;
    cudaError_t e = cudaEventRecord(br->fork, s);
    const int nb = n < kBranches ? n : kBranches;
    for (int b = 0; b < nb && e == cudaSuccess; ++b) e = cudaStreamWaitEvent(br->branch[b], br->fork, 0);
    for (int i = 0; i < n && e == cudaSuccess && st == DV_OK; ++i) {
        const dv_request &r = reqs[i];
        dv_mesh *m = const_cast<dv_mesh *>(r.mesh);
        cudaStream_t b = br->branch[i % nb];
        const int64_t nq = (int64_t)r.grid.n[0] * r.grid.n[1] * r.grid.n[2];
        st = run_forward(m, nullptr, nq, &r.grid, r.d_out_w, r.d_out_occ, prec, nullptr, b);
        if (st == DV_OK && r.d_upstream) st = backward_on(m, &r.grid, nq, r.d_upstream, r.d_dverts, b);
    }
    for (int b = 0; b < nb && e == cudaSuccess; ++b) {
        e = cudaEventRecord(br->join[b], br->branch[b]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, br->join[b], 0);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(s, &graph);
    if (st != DV_OK || e != cudaSuccess || ee != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (st != DV_OK) return st;
        return fail(DV_ERR_CUDA, "batch capture: %s", cudaGetErrorString(e != cudaSuccess ? e : ee));
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(DV_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    e = cudaGraphLaunch(exec, s);
    if (e != cudaSuccess) {
        cudaGraphExecDestroy(exec);
        return fail(DV_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
    }
    cudaEvent_t done;
    DV_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    DV_CUDA(cudaEventRecord(done, s));
    br->pending.emplace_back(done, exec);
    for (int i = 0; i < n; ++i) const_cast<dv_mesh *>(reqs[i].mesh)->last_stream = s;
    return DV_OK;
}

dv_status dv_dipole_winding(const dv_mesh *mesh, const float *d_queries, int64_t nq, const dv_grid *grid,
                            float *d_out_w, void *stream) {
    DV_NVTX_RANGE("dv_dipole_winding");
    int64_t n = 0;
    dv_status st = check_queries(mesh, d_queries, nq, grid, &n);
    if (st) return st;
    if (!d_out_w) return fail(DV_ERR_INVALID_ARG, "d_out_w is NULL");
    DeviceGuard dg(mesh->device);
    const_cast<dv_mesh *>(mesh)->last_stream = (cudaStream_t)stream;
    dv::GridF gf{};
    if (grid) gf = to_gridf(grid);
    DV_CUDA(dv::launch_dipole_forward(mesh->rec, mesh->nf, grid ? &gf : nullptr, d_queries, n, d_out_w,
                                      (cudaStream_t)stream));
    return DV_OK;
}

dv_status dv_dipole_backward(const dv_mesh *mesh, const float *d_queries, int64_t nq, const dv_grid *grid,
                             const float *d_upstream, float *d_dverts, void *stream) {
    DV_NVTX_RANGE("dv_dipole_backward");
    int64_t n = 0;
    dv_status st = check_queries(mesh, d_queries, nq, grid, &n);
    if (st) return st;
    if (!d_upstream || !d_dverts) return fail(DV_ERR_INVALID_ARG, "d_upstream or d_dverts is NULL");
    dv_mesh *m = const_cast<dv_mesh *>(mesh);
    DeviceGuard dg(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    dv::GridF gf{};
    if (grid) gf = to_gridf(grid);
    const int ns = dv::dipole_bwd_splits(n, m->nf, m->num_sms);
    m->last_stream = s;
    if ((st = grow(m->ws_fg, m->cap_fg, (int64_t)ns * m->nf * 9, s))) return st;
    DV_CUDA(dv::launch_dipole_backward(m->rec, m->nf, grid ? &gf : nullptr, d_queries, n, d_upstream, ns, m->ws_fg, s));
    DV_CUDA(dv::launch_gather_dverts(nullptr, m->ws_fg, ns, m->nf, m->vtx_ptr, m->vtx_corner, m->nv, d_dverts, s));
    return DV_OK;
}

dv_status dv_flipped_duplication(const dv_mesh *mesh, const float *d_verts, float eps, float *d_out_verts,
                                 int32_t *d_out_faces, void *stream) {
    DV_NVTX_RANGE("dv_flipped_duplication");
    if (!mesh || !d_verts || !d_out_verts || !d_out_faces)
        return fail(DV_ERR_INVALID_ARG, "mesh, d_verts, d_out_verts and d_out_faces must be non-NULL");
    if (!std::isfinite(eps)) return fail(DV_ERR_INVALID_ARG, "eps must be finite");
    if (2 * mesh->nv > (int64_t)INT32_MAX || 6 * mesh->nf > (int64_t)INT32_MAX)
        return fail(DV_ERR_UNSUPPORTED, "duplicated mesh exceeds the 32-bit index range");
    dv_mesh *m = const_cast<dv_mesh *>(mesh);
    DeviceGuard dg(m->device);
    m->last_stream = (cudaStream_t)stream;
    DV_CUDA(dv::launch_flipped_duplication(d_verts, m->nv, m->faces, m->nf, m->rec64, m->vtx_ptr, m->vtx_corner,
                                           (double)eps, d_out_verts, d_out_faces, (cudaStream_t)stream));
    return DV_OK;
}

void dv_profile_enable(int on) { dv::g_prof_on = on != 0; }

void dv_profile_reset(void) {
    std::lock_guard<std::mutex> lk(dv::g_prof_mu);
    for (auto &r : dv::g_prof_pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    dv::g_prof_pending.clear();
    dv::g_prof_tot.clear();
}

int dv_profile_read(const char **names, double *total_ms, int64_t *launches, int cap) {
    std::lock_guard<std::mutex> lk(dv::g_prof_mu);
    for (auto &r : dv::g_prof_pending) {
        cudaEventSynchronize(r.b);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) ms = 0.f;
        auto it = std::find_if(dv::g_prof_tot.begin(), dv::g_prof_tot.end(),
                               [&](const dv::ProfTot &t) { return std::strcmp(t.name, r.name) == 0; });
        if (it == dv::g_prof_tot.end())
            dv::g_prof_tot.push_back({r.name, (double)ms, 1});
        else {
            it->ms += ms;
            it->n += 1;
        }
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    dv::g_prof_pending.clear();
    const int n = (int)dv::g_prof_tot.size();
    for (int i = 0; i < n && i < cap; ++i) {
        if (names) names[i] = dv::g_prof_tot[i].name;
        if (total_ms) total_ms[i] = dv::g_prof_tot[i].ms;
        if (launches) launches[i] = dv::g_prof_tot[i].n;
    }
    return n;
}

int64_t dv_launch_count(void) { return dv::g_launches.load(); }

}  // extern "C"
