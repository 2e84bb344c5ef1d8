// Grid winding numbers for callers that must not allocate device memory.
//
// dv_winding_grid_noalloc runs the same packing and forward kernels as dv_mesh_create +
// dv_winding (Kahan-compensated FP32, grid queries), but everything the library itself needs
// beyond the caller's inputs and output -- the packed face records, the per-split partial sums
// and an error word -- lives in one file-scope device array of fixed size. The library then
// makes no cudaMalloc/cudaFree call (and no other allocating call) on this path.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "dv_internal.cuh"

namespace dv {
namespace {

// 32 MiB per device. This array is part of the library's device code: a GPU on which the code
// is loaded holds it until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr size_t kHeaderBytes = 256;  // error word at offset 0

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
unsigned char *g_addr[kMaxDevices] = {};

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Device address of the scratch array on the current device, looked up once per device. In host
// code the array's name only stands for the symbol; kernels must be given this address.
cudaError_t scratch_address(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (!g_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

// Pack FP32 face records like pack_kernel, checking every index first: an index outside
// [0, nv) sets the error word and leaves a zero (degenerate) record instead of reading.
__global__ void noalloc_pack_kernel(const float *__restrict__ verts, int64_t nv, const int32_t *__restrict__ faces,
                                    int64_t nf, FaceRec *__restrict__ rec, int *err) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    int64_t id[3];
    bool ok = true;
    for (int k = 0; k < 3; ++k) {
        id[k] = faces[3 * f + k];
        ok = ok && id[k] >= 0 && id[k] < nv;
    }
    FaceRec r;
    if (!ok) {
        atomicCAS(err, 0, (int)DV_ERR_INVALID_MESH);
        r.r0 = r.r1 = r.r2 = make_float4(0.f, 0.f, 0.f, 0.f);
        rec[f] = r;
        return;
    }
    double v[3][3];
    for (int k = 0; k < 3; ++k)
        for (int c = 0; c < 3; ++c) v[k][c] = (double)verts[3 * id[k] + c];
    const double e1[3] = {v[1][0] - v[0][0], v[1][1] - v[0][1], v[1][2] - v[0][2]};
    const double e2[3] = {v[2][0] - v[0][0], v[2][1] - v[0][1], v[2][2] - v[0][2]};
    const double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                         e1[0] * e2[1] - e1[1] * e2[0]};
    r.r0 = make_float4((float)v[0][0], (float)v[0][1], (float)v[0][2], (float)(kNormalScale * n[0]));
    r.r1 = make_float4((float)v[1][0], (float)v[1][1], (float)v[1][2], (float)(kNormalScale * n[1]));
    r.r2 = make_float4((float)v[2][0], (float)v[2][1], (float)v[2][2], (float)(kNormalScale * n[2]));
    rec[f] = r;
}

dv_status cuda_fail(const char *what, cudaError_t e) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    return report_error(DV_ERR_CUDA, buf);
}

}  // namespace
}  // namespace dv

extern "C" dv_status dv_winding_grid_noalloc(const float *d_verts, int64_t nv, const int32_t *d_faces, int64_t nf,
                                             const dv_grid *grid, float *d_out_w, void *stream) {
    using namespace dv;
    if (!d_verts || !d_faces || !grid || !d_out_w)
        return report_error(DV_ERR_INVALID_ARG, "null pointer argument");
    if (nv < 3 || nf < 1) return report_error(DV_ERR_INVALID_ARG, "need nv >= 3 and nf >= 1");
    for (int k = 0; k < 3; ++k) {
        if (grid->n[k] < 1) return report_error(DV_ERR_INVALID_ARG, "grid n must be >= 1 on every axis");
        if (!std::isfinite(grid->lo[k]) || !std::isfinite(grid->hi[k]) || !(grid->hi[k] > grid->lo[k]))
            return report_error(DV_ERR_INVALID_ARG, "grid needs finite lo < hi on every axis");
    }
    const int64_t nq = (int64_t)grid->n[0] * grid->n[1] * grid->n[2];
    if (nq > (int64_t)INT32_MAX || nv > (int64_t)INT32_MAX || 3 * nf > (int64_t)INT32_MAX)
        return report_error(DV_ERR_UNSUPPORTED, "sizes exceed the 32-bit index range");

    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail("device query", e);

    GridF gf{};
    for (int k = 0; k < 3; ++k) {
        gf.lo[k] = grid->lo[k];
        gf.h[k] = (grid->hi[k] - grid->lo[k]) / (float)grid->n[k];
        gf.n[k] = grid->n[k];
    }
    const FwdPlan plan = plan_forward(nq, nf, true, &gf, sms);
    const size_t rec_bytes = round_up((size_t)nf * sizeof(FaceRec), 256);
    const size_t part_bytes = plan.nsplit > 1 ? (size_t)plan.nsplit * (size_t)nq * sizeof(float2) : 0;
    const size_t need = kHeaderBytes + rec_bytes + part_bytes;
    if (need > kNoAllocScratchBytes) {
        char buf[256];
        snprintf(buf, sizeof(buf),
                 "this mesh and grid need %zu bytes of scratch (%zu for %lld face records, %zu for partial "
                 "sums); the fixed scratch holds %zu",
                 need, rec_bytes, (long long)nf, part_bytes, kNoAllocScratchBytes);
        return report_error(DV_ERR_UNSUPPORTED, buf);
    }

    unsigned char *base = nullptr;
    if ((e = scratch_address(dev, &base)) != cudaSuccess) return cuda_fail("cudaGetSymbolAddress(scratch)", e);
    int *err = reinterpret_cast<int *>(base);
    FaceRec *rec = reinterpret_cast<FaceRec *>(base + kHeaderBytes);
    float2 *partial = part_bytes ? reinterpret_cast<float2 *>(base + kHeaderBytes + rec_bytes) : nullptr;
    cudaStream_t s = (cudaStream_t)stream;

    // The array keeps the previous call's contents: only the error word has to start at zero
    // (records and partial sums are fully overwritten below).
    if ((e = cudaMemsetAsync(err, 0, sizeof(int), s)) != cudaSuccess) return cuda_fail("clear error word", e);
    noalloc_pack_kernel<<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(d_verts, nv, d_faces, nf, rec, err);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail("pack launch", e);
    const LaunchCtx ctx{s, err};
    if ((e = launch_forward(plan, rec, nf, nullptr, 0, &gf, nullptr, nq, kArithKahan, partial, d_out_w, nullptr,
                            nullptr, nullptr, nullptr, ctx)) != cudaSuccess)
        return cuda_fail("forward launch", e);
    if (plan.nsplit > 1 &&
        (e = launch_split_reduce(plan, partial, nq, d_out_w, nullptr, nullptr, nullptr, nullptr, s)) != cudaSuccess)
        return cuda_fail("split reduce launch", e);
    int code = 0;
    if ((e = cudaMemcpyAsync(&code, err, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail("read error word", e);
    if (code == DV_ERR_INVALID_MESH) return report_error(DV_ERR_INVALID_MESH, "a face index is outside [0, nv)");
    if (code != 0) return report_error((dv_status)code, "a bounded device wait ran out");
    return DV_OK;
}
