// Self-test of the bounded waits that every TMA pipeline in this library uses (no counterpart in
// the paper). One CTA waits on an mbarrier phase with a short time limit; with `arrive` set,
// thread 0 arrives first and the wait succeeds, otherwise nothing ever arrives, the wait gives up
// after limit_ns and the kernel records DV_ERR_TIMEOUT in an error word and returns. The host
// reads the word. This exercises the give-up path of mbar_wait_bounded without a fault: no bulk
// copy is issued, so nothing is left in flight when the kernel exits.
#include "dv_internal.cuh"

namespace dv {

__device__ int g_selftest_err;

__global__ void selftest_wait_kernel(uint64_t limit_ns, int arrive) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (arrive && threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
    }
    if (!mbar_wait_bounded(&bar, 0u, limit_ns)) set_error(&g_selftest_err, (int)DV_ERR_TIMEOUT);
}

}  // namespace dv

extern "C" dv_status dv_selftest_bounded_wait(int64_t limit_us, int arrive, void *stream) {
    if (limit_us < 1 || limit_us > 10000000)
        return dv::report_error(DV_ERR_INVALID_ARG, "dv_selftest_bounded_wait: limit_us outside [1, 1e7]");
    cudaStream_t s = (cudaStream_t)stream;
    const int zero = 0;
    int err = 0;
    cudaError_t e = cudaMemcpyToSymbolAsync(dv::g_selftest_err, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        dv::selftest_wait_kernel<<<1, 64, 0, s>>>((uint64_t)limit_us * 1000ull, arrive);
        dv::count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyFromSymbolAsync(&err, dv::g_selftest_err, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return dv::report_error(DV_ERR_CUDA, cudaGetErrorString(e));
    return err == 0 ? DV_OK : (dv_status)err;
}
