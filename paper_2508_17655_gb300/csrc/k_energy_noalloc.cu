// k_energy_noalloc.cu -- Ising energies of caller spin vectors with no device
// allocation: the per-replica accumulators live in a fixed array that is part
// of the library image instead of memory from cudaMalloc.
//
// Who needs it: programs that must not call cudaMalloc / cudaFree once they
// are running -- a steady-state loop that cannot afford the blocking those
// calls may do (cudaFree waits for the device), or an application whose own
// allocator has reserved the device memory and forbids allocations behind its
// back. They pass device buffers for J, the spins and the energies; this
// entry point only launches kernels on their stream.
//
// Limits and sharing: at most kMaxReplicas spin vectors of at most kMaxN
// spins per call. The scratch array is one per device and is shared by every
// call on that device; it keeps the last call's partial sums, so each call
// clears it first, and two calls whose work overlaps on the GPU (different
// streams, no ordering) race on it.
#include "gsb_internal.cuh"

namespace gsb {

namespace {

constexpr int kMaxReplicas = 65536;  // 512 KiB of doubles, held by every device that loads the library
constexpr int kReplicasPerBlock = 8;
// The spins of kReplicasPerBlock replicas are staged in shared memory, one byte
// each: 8 x 29,000 = 232,000 bytes, within the 227 KiB (232,448 bytes) a block
// may opt in to on this GPU.
constexpr int kMaxN = 29000;
constexpr int kRowsPerBlock = 64;

__device__ __align__(256) double g_energy_scratch[kMaxReplicas];

__global__ void k_scratch_clear(double* acc, int R) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < R) acc[r] = 0.0;
}

// acc[r] += sum_{i in block} s_ri sum_j J_ij s_rj for 8 replicas and 64 rows:
// the replicas' spins are staged in shared memory, each warp walks 8 rows with
// coalesced reads of J and reduces over j with shuffles.
__global__ void __launch_bounds__(256) k_energy_partial(const float* __restrict__ J, int N,
                                                        const int8_t* __restrict__ spins, int R,
                                                        double* __restrict__ acc) {
    extern __shared__ int8_t s_sh[];  // [kReplicasPerBlock][N]
    const int rb = blockIdx.x * kReplicasPerBlock;
    const int nrep = min(kReplicasPerBlock, R - rb);
    for (int k = threadIdx.x; k < kReplicasPerBlock * N; k += blockDim.x) {
        const int q = k / N, j = k - q * N;
        s_sh[k] = q < nrep ? spins[(size_t)(rb + q) * N + j] : (int8_t)0;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double part[kReplicasPerBlock];
#pragma unroll
    for (int q = 0; q < kReplicasPerBlock; ++q) part[q] = 0.0;
    const int row0 = blockIdx.y * kRowsPerBlock + warp * (kRowsPerBlock / 8);
    for (int rr = 0; rr < kRowsPerBlock / 8; ++rr) {
        const int i = row0 + rr;
        if (i >= N) break;
        float f[kReplicasPerBlock];
#pragma unroll
        for (int q = 0; q < kReplicasPerBlock; ++q) f[q] = 0.f;
        for (int j = lane; j < N; j += 32) {
            const float w = J[(size_t)i * N + j];
#pragma unroll
            for (int q = 0; q < kReplicasPerBlock; ++q) f[q] = fmaf(w, (float)s_sh[q * N + j], f[q]);
        }
#pragma unroll
        for (int q = 0; q < kReplicasPerBlock; ++q) {
            float v = f[q];
            for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            part[q] += (double)s_sh[q * N + i] * (double)v;
        }
    }
    if (lane == 0)
        for (int q = 0; q < nrep; ++q) atomicAdd(&acc[rb + q], part[q]);
}

__global__ void k_energy_finish(const double* __restrict__ acc, double* __restrict__ e, int R) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < R) e[r] = -0.5 * acc[r];
}

// Device address of the scratch array on the current device. In host code the
// symbol's name is only a host-side handle, not a device address. The lookup
// is a host-side table query that allocates nothing; doing it on every call
// (rather than caching one address per device number) keeps the address right
// when the caller resets a device, after which the module is loaded again and
// the array may sit elsewhere. The first call on a device may load the
// library's module there, which is why it should come before any stream
// capture.
gsb_status scratch_for_current_device(double** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_energy_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_energy_scratch)");
    *out = (double*)p;
    return GSB_OK;
}

}  // namespace

}  // namespace gsb

using namespace gsb;

extern "C" gsb_status gsb_energy_noalloc(const float* J, int32_t N, const int8_t* spins,
                                         int32_t R, double* energies, void* stream) {
    if (!J || !spins || !energies) return set_error(GSB_EINVAL, "NULL device pointer");
    if (N < 1 || N > kMaxN)
        return set_error(GSB_EINVAL, "gsb_energy_noalloc takes 1 to " + std::to_string(kMaxN) +
                                         " spins");
    if (R < 1 || R > kMaxReplicas)
        return set_error(GSB_EINVAL, "gsb_energy_noalloc takes 1 to " +
                                         std::to_string(kMaxReplicas) + " spin vectors per call");
    const size_t smem = (size_t)kReplicasPerBlock * N;
    double* acc = nullptr;
    gsb_status st = scratch_for_current_device(&acc);
    if (st != GSB_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (smem > 48 * 1024)
        GSB_CUDA_TRY(cudaFuncSetAttribute(k_energy_partial,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_scratch_clear<<<(R + 255) / 256, 256, 0, s>>>(acc, R);
    GSB_LAUNCH_CHECK("k_scratch_clear");
    dim3 grid((R + kReplicasPerBlock - 1) / kReplicasPerBlock, (N + kRowsPerBlock - 1) / kRowsPerBlock);
    k_energy_partial<<<grid, 256, smem, s>>>(J, N, spins, R, acc);
    GSB_LAUNCH_CHECK("k_energy_partial");
    k_energy_finish<<<(R + 255) / 256, 256, 0, s>>>(acc, energies, R);
    GSB_LAUNCH_CHECK("k_energy_finish");
    return GSB_OK;
}
