// k_csr.cu -- one sparse time step: the many-body term f_i = sum_k val_k v_{col_k}
// over all replicas at once (CSR SpMM against the spin-major state), with
// Eqs. 3-7 fused into its epilogue; and the Ising energy (Eq. 1) of sgn x.
//
// Mapping: one warp per (row i, 128 replicas); each lane owns 4 consecutive
// replicas, so every gathered row of v is one coalesced 512-byte (x) or
// 128-byte (sgn x, int8) access. The warp loads up to 32 nonzeros of its row at
// once (one per lane) and broadcasts them with __shfl_sync.
//
// With integer J the x coupling is exact: each gathered x_j becomes the 32-bit
// fixed-point integer q_j = rint(x_j 2^30) (equal to x_j 2^30 for
// |x_j| >= 2^-7), sum_k J_ik q_k is accumulated in int64, and 2^-30 times it is
// rounded once to FP32. The sgn x coupling of integer J is an integer sum
// already (exact in FP32).
#include "gsb_update.cuh"

namespace gsb {

namespace {

constexpr int kWarpsPerBlock = 8;
constexpr int kReplicasPerWarp = 128;

template <bool SIGN, bool EXACT>
__device__ __forceinline__ float4 row_coupling(const int32_t* __restrict__ rowptr,
                                               const int32_t* __restrict__ col,
                                               const float* __restrict__ val,
                                               const float* __restrict__ xv,
                                               const int8_t* __restrict__ sv, int Rp, int i,
                                               int rlane) {
    const int lane = threadIdx.x & 31;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    long long qa[4] = {0, 0, 0, 0};
    const int beg = rowptr[i], end = rowptr[i + 1];
    for (int kb = beg; kb < end; kb += 32) {
        const int k = kb + lane;
        const int cj = k < end ? col[k] : 0;
        const float wj = k < end ? val[k] : 0.f;
        const int cnt = min(32, end - kb);
        for (int t = 0; t < cnt; ++t) {
            const int j = __shfl_sync(0xffffffffu, cj, t);
            const float w = __shfl_sync(0xffffffffu, wj, t);
            if (SIGN) {
                const char4 s = *reinterpret_cast<const char4*>(sv + (size_t)j * Rp + rlane);
                acc.x = fmaf(w, (float)s.x, acc.x);
                acc.y = fmaf(w, (float)s.y, acc.y);
                acc.z = fmaf(w, (float)s.z, acc.z);
                acc.w = fmaf(w, (float)s.w, acc.w);
            } else if (EXACT) {
                const float4 v = *reinterpret_cast<const float4*>(xv + (size_t)j * Rp + rlane);
                const long long wi = (long long)__float2int_rn(w);
                qa[0] += wi * __float2int_rn(v.x * 1073741824.0f);
                qa[1] += wi * __float2int_rn(v.y * 1073741824.0f);
                qa[2] += wi * __float2int_rn(v.z * 1073741824.0f);
                qa[3] += wi * __float2int_rn(v.w * 1073741824.0f);
            } else {
                const float4 v = *reinterpret_cast<const float4*>(xv + (size_t)j * Rp + rlane);
                acc.x = fmaf(w, v.x, acc.x);
                acc.y = fmaf(w, v.y, acc.y);
                acc.z = fmaf(w, v.z, acc.z);
                acc.w = fmaf(w, v.w, acc.w);
            }
        }
    }
    if (!SIGN && EXACT) {
        // one correctly rounded int64 -> FP32 conversion, then the exact 2^-30
        const float s = 9.313225746154785e-10f;
        acc = make_float4(__ll2float_rn(qa[0]) * s, __ll2float_rn(qa[1]) * s,
                          __ll2float_rn(qa[2]) * s, __ll2float_rn(qa[3]) * s);
    }
    return acc;
}

template <bool SIGN, bool CONTROL, bool EXACT>
__global__ void __launch_bounds__(256) k_csr_step(
    const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const float* __restrict__ val, int N, int Rp, const float* __restrict__ xc,
    const int8_t* __restrict__ sc, float* __restrict__ xn, int8_t* __restrict__ sn,
    float* __restrict__ y, float* __restrict__ p, const float* __restrict__ A, float c, float dt,
    float p_shared, float inv_rem) {
    // launched with programmatic dependent launch: the next step may be
    // scheduled once every block of this one has started; everything below
    // reads or writes state the previous step touched, so it waits for it
    griddep_trigger();
    griddep_wait();
    const int i = blockIdx.y * kWarpsPerBlock + (threadIdx.x >> 5);
    if (i >= N) return;
    const int rlane = blockIdx.x * kReplicasPerWarp + (threadIdx.x & 31) * 4;
    const float4 f = row_coupling<SIGN, EXACT>(rowptr, col, val, xc, sc, Rp, i, rlane);
    const size_t o = (size_t)i * Rp + rlane;
    float4 x4 = *reinterpret_cast<const float4*>(xc + o);
    float4 y4 = *reinterpret_cast<const float4*>(y + o);
    float4 p4 = make_float4(0.f, 0.f, 0.f, 0.f), a4 = p4;
    if (CONTROL) {
        p4 = *reinterpret_cast<const float4*>(p + o);
        a4 = *reinterpret_cast<const float4*>(A + rlane);
    }
    float* xs = &x4.x; float* ys = &y4.x; float* ps = &p4.x;
    const float* fs = &f.x; const float* as = &a4.x;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        sb_update<CONTROL>(xs[q], ys[q], ps[q], fs[q], as[q], c, dt, p_shared, inv_rem);
    *reinterpret_cast<float4*>(xn + o) = x4;
    *reinterpret_cast<float4*>(y + o) = y4;
    if (CONTROL) *reinterpret_cast<float4*>(p + o) = p4;
    if (SIGN) {
        char4 s;
        s.x = x4.x >= 0.f ? 1 : -1;
        s.y = x4.y >= 0.f ? 1 : -1;
        s.z = x4.z >= 0.f ? 1 : -1;
        s.w = x4.w >= 0.f ? 1 : -1;
        *reinterpret_cast<char4*>(sn + o) = s;
    }
}

// e_acc[r] += sum_i s_i (J s)_i. Each warp walks kRowsPerWarp rows; partial
// sums are combined across the block's warps in shared memory, then one
// double atomic per replica and block.
constexpr int kRowsPerWarp = 16;

__global__ void __launch_bounds__(256) k_csr_energy(const int32_t* __restrict__ rowptr,
                                                    const int32_t* __restrict__ col,
                                                    const float* __restrict__ val, int N,
                                                    int Rp, const float* __restrict__ x,
                                                    double* __restrict__ e_acc) {
    __shared__ float red[kWarpsPerBlock][kReplicasPerWarp];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rlane = blockIdx.x * kReplicasPerWarp + lane * 4;
    const int row0 = (blockIdx.y * kWarpsPerBlock + warp) * kRowsPerWarp;
    float4 part = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int rr = 0; rr < kRowsPerWarp; ++rr) {
        const int i = row0 + rr;
        if (i >= N) break;
        float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
        const int beg = rowptr[i], end = rowptr[i + 1];
        for (int kb = beg; kb < end; kb += 32) {
            const int k = kb + lane;
            const int cj = k < end ? col[k] : 0;
            const float wj = k < end ? val[k] : 0.f;
            const int cnt = min(32, end - kb);
            for (int t = 0; t < cnt; ++t) {
                const int j = __shfl_sync(0xffffffffu, cj, t);
                const float w = __shfl_sync(0xffffffffu, wj, t);
                const float4 v = *reinterpret_cast<const float4*>(x + (size_t)j * Rp + rlane);
                f.x = fmaf(w, sgnf(v.x), f.x);
                f.y = fmaf(w, sgnf(v.y), f.y);
                f.z = fmaf(w, sgnf(v.z), f.z);
                f.w = fmaf(w, sgnf(v.w), f.w);
            }
        }
        const float4 xi = *reinterpret_cast<const float4*>(x + (size_t)i * Rp + rlane);
        part.x = fmaf(sgnf(xi.x), f.x, part.x);
        part.y = fmaf(sgnf(xi.y), f.y, part.y);
        part.z = fmaf(sgnf(xi.z), f.z, part.z);
        part.w = fmaf(sgnf(xi.w), f.w, part.w);
    }
    red[warp][lane * 4 + 0] = part.x;
    red[warp][lane * 4 + 1] = part.y;
    red[warp][lane * 4 + 2] = part.z;
    red[warp][lane * 4 + 3] = part.w;
    __syncthreads();
    if (threadIdx.x < kReplicasPerWarp) {
        double s = 0.0;
        for (int w = 0; w < kWarpsPerBlock; ++w) s += (double)red[w][threadIdx.x];
        atomicAdd(&e_acc[blockIdx.x * kReplicasPerWarp + threadIdx.x], s);
    }
}

}  // namespace

gsb_status launch_csr_step(gsb_run_state* run, const StepScalars& sc) {
    const gsb_problem* P = run->prob;
    dim3 grid(run->Rp / kReplicasPerWarp, (run->N + kWarpsPerBlock - 1) / kWarpsPerBlock);
    const int cur = run->cur;
    const float inv_rem = 1.0f / (float)(sc.M - sc.m);
#define GSB_CSR_LAUNCH(S, C, E)                                                              \
    GSB_CUDA_TRY(launch_pdl(k_csr_step<S, C, E>, grid, dim3(256), 0, run->stream, P->rowptr,   \
                            P->col, P->val, run->N, run->Rp, (const float*)run->x[cur],      \
                            (const int8_t*)run->s8[cur], run->x[cur ^ 1], run->s8[cur ^ 1],  \
                            run->y, run->p, (const float*)run->A, sc.c, sc.dt, sc.p_next,    \
                            inv_rem))
    // exact fixed-point x coupling when J is integer and 2^30 sum_k |J_ik| fits in int64
    const bool exact = P->integer_J && P->max_row_abs < 4294967296.0;
    if (run->sign_coupling) {
        if (run->control) GSB_CSR_LAUNCH(true, true, false); else GSB_CSR_LAUNCH(true, false, false);
    } else if (exact) {
        if (run->control) GSB_CSR_LAUNCH(false, true, true); else GSB_CSR_LAUNCH(false, false, true);
    } else {
        if (run->control) GSB_CSR_LAUNCH(false, true, false); else GSB_CSR_LAUNCH(false, false, false);
    }
#undef GSB_CSR_LAUNCH
    GSB_LAUNCH_CHECK("k_csr_step");
    run->cur ^= 1;
    return GSB_OK;
}

gsb_status launch_csr_energy(const gsb_problem* P, const float* x, int Rp, double* e_acc,
                             cudaStream_t s) {
    const int rows_per_block = kWarpsPerBlock * kRowsPerWarp;
    dim3 grid(Rp / kReplicasPerWarp, (P->N + rows_per_block - 1) / rows_per_block);
    k_csr_energy<<<grid, 256, 0, s>>>(P->rowptr, P->col, P->val, P->N, Rp, x, e_acc);
    GSB_LAUNCH_CHECK("k_csr_energy");
    return GSB_OK;
}

}  // namespace gsb
