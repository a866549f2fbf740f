// k_wait_check.cu -- gsb_wait_check: runs one of the library's bounded
// device-side waits on a condition that nothing will satisfy (or, as a
// control, on one that already holds), so a caller can see a wait give up with
// GSB_ETIMEOUT and the CUDA context stay usable. The tensor-core kernels use
// the same wait helpers for their barriers and their replica-column counters.
#include "gsb_internal.cuh"
#include "tc_ptx.cuh"

namespace gsb {

namespace {

using namespace tc;

// kind 0: an mbarrier of count 1 that nobody arrives on; kind 1: a counter in
// global memory waited on for a value nobody adds; kind 2: the counter already
// at its target (completes at once).
__global__ void k_wait_check(int kind, uint64_t limit_cycles, const uint32_t* ctr, int* status) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    if (kind == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
        mbar_wait(&bar, 0, status, limit_cycles);
    } else {
        wait_counter(ctr, kind == 1 ? 1u : 0u, status, limit_cycles);
    }
}

}  // namespace

}  // namespace gsb

using namespace gsb;

extern "C" gsb_status gsb_wait_check(int32_t kind, int64_t limit_ns, void* stream) {
    if (kind < 0 || kind > 2) return set_error(GSB_EINVAL, "kind must be 0, 1 or 2");
    if (limit_ns < 1000 || limit_ns > 10000000000ll)
        return set_error(GSB_EINVAL, "limit_ns must be in [1 us, 10 s]");
    cudaStream_t s = (cudaStream_t)stream;
    // the waits count SM clock cycles: the limit at the device's rated clock
    int dev = 0, khz = 0;
    GSB_CUDA_TRY(cudaGetDevice(&dev));
    GSB_CUDA_TRY(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
    const uint64_t limit_cycles = (uint64_t)((double)limit_ns * (double)khz * 1e-6) + 1;
    uint32_t* ctr = nullptr;
    int* status = nullptr;
    GSB_CUDA_TRY(cudaMalloc(&ctr, sizeof(uint32_t)));
    if (cudaMalloc(&status, sizeof(int)) != cudaSuccess) {
        cudaFree(ctr);
        return cuda_error(cudaGetLastError(), "cudaMalloc");
    }
    gsb_status st = GSB_OK;
    int h = 0;
    do {
        if (cudaMemsetAsync(ctr, 0, sizeof(uint32_t), s) != cudaSuccess ||
            cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) {
            st = cuda_error(cudaGetLastError(), "memset");
            break;
        }
        k_wait_check<<<1, 32, 0, s>>>(kind, limit_cycles, ctr, status);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            st = cuda_error(e, "k_wait_check");
            break;
        }
        if (h & kDevTimeout) st = set_error(GSB_ETIMEOUT, "the device-side wait timed out");
    } while (0);
    cudaFree(ctr);
    cudaFree(status);
    return st;
}
