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
#include "tc_ptx.cuh"

#include <algorithm>
#include <vector>

namespace gsb {

namespace {

constexpr int kWarpsPerBlock = 8;
constexpr int kReplicasPerWarp = 128;

// Gathered loads of the coupled state. CG: through L2 only (ld.global.cg), for
// the fused multi-step kernel, whose gathered rows were written by other SMs
// during the launch and may sit stale in this SM's L1.
template <bool CG>
__device__ __forceinline__ float4 load_x4(const float* p) {
    return CG ? __ldcg(reinterpret_cast<const float4*>(p)) : *reinterpret_cast<const float4*>(p);
}
template <bool CG>
__device__ __forceinline__ char4 load_s4(const int8_t* p) {
    if (CG) {
        const int w = __ldcg(reinterpret_cast<const int*>(p));
        return *reinterpret_cast<const char4*>(&w);
    }
    return *reinterpret_cast<const char4*>(p);
}

template <bool SIGN, bool EXACT, bool CG, bool MLP4>
__device__ __forceinline__ float4 row_coupling(const int32_t* __restrict__ rowptr,
                                               const int32_t* __restrict__ col,
                                               const float* __restrict__ val,
                                               const float* __restrict__ xv,
                                               const int8_t* __restrict__ sv, int Rp, int i,
                                               int rlane, int N, int* status) {
    const int lane = threadIdx.x & 31;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    long long qa[4] = {0, 0, 0, 0};
    const int beg = rowptr[i], end = rowptr[i + 1];
#ifdef GSB_DEBUG
    // the row's nonzeros within col / val (one warp, one row: a uniform return)
    if (!GSB_DOK(beg >= 0 && beg <= end && end <= rowptr[N], status)) return acc;
#endif
    for (int kb = beg; kb < end; kb += 32) {
        const int k = kb + lane;
        int cj = k < end ? col[k] : 0;
        float wj = k < end ? val[k] : 0.f;
        // debug build: an out-of-range column reads row 0 with weight 0
        if (!GSB_DOK(cj >= 0 && cj < N, status)) {
            cj = 0;
            wj = 0.f;
        }
        const int cnt = min(32, end - kb);
        int t0 = 0;
        if (MLP4 && !SIGN) {
            // four gathers in flight at once (MLP4): the loads first,
            // then the sums in the nonzeros' order, so the result is the
            // one-at-a-time loop's bit for bit
            for (; t0 + 4 <= cnt; t0 += 4) {
                float4 v[4];
                float w[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int j = __shfl_sync(0xffffffffu, cj, t0 + q);
                    w[q] = __shfl_sync(0xffffffffu, wj, t0 + q);
                    v[q] = load_x4<CG>(xv + (size_t)j * Rp + rlane);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (EXACT) {
                        const long long wi = (long long)__float2int_rn(w[q]);
                        qa[0] += wi * __float2int_rn(v[q].x * 1073741824.0f);
                        qa[1] += wi * __float2int_rn(v[q].y * 1073741824.0f);
                        qa[2] += wi * __float2int_rn(v[q].z * 1073741824.0f);
                        qa[3] += wi * __float2int_rn(v[q].w * 1073741824.0f);
                    } else {
                        acc.x = fmaf(w[q], v[q].x, acc.x);
                        acc.y = fmaf(w[q], v[q].y, acc.y);
                        acc.z = fmaf(w[q], v[q].z, acc.z);
                        acc.w = fmaf(w[q], v[q].w, acc.w);
                    }
                }
            }
        }
        for (int t = t0; t < cnt; ++t) {
            const int j = __shfl_sync(0xffffffffu, cj, t);
            const float w = __shfl_sync(0xffffffffu, wj, t);
            if (SIGN) {
                const char4 s = load_s4<CG>(sv + (size_t)j * Rp + rlane);
                acc.x = fmaf(w, (float)s.x, acc.x);
                acc.y = fmaf(w, (float)s.y, acc.y);
                acc.z = fmaf(w, (float)s.z, acc.z);
                acc.w = fmaf(w, (float)s.w, acc.w);
            } else if (EXACT) {
                const float4 v = load_x4<CG>(xv + (size_t)j * Rp + rlane);
                const long long wi = (long long)__float2int_rn(w);
                qa[0] += wi * __float2int_rn(v.x * 1073741824.0f);
                qa[1] += wi * __float2int_rn(v.y * 1073741824.0f);
                qa[2] += wi * __float2int_rn(v.z * 1073741824.0f);
                qa[3] += wi * __float2int_rn(v.w * 1073741824.0f);
            } else {
                const float4 v = load_x4<CG>(xv + (size_t)j * Rp + rlane);
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

// Row i, replicas rlane .. rlane + 3 of one step: the coupling, then Eqs. 7,
// 3, 4, 5 on the four oscillators, written to the next buffers.
template <bool SIGN, bool CONTROL, bool EXACT, bool CG, bool MLP4>
__device__ __forceinline__ void csr_task(const int32_t* __restrict__ rowptr,
                                         const int32_t* __restrict__ col,
                                         const float* __restrict__ val, int Rp,
                                         const float* __restrict__ xc,
                                         const int8_t* __restrict__ sc, float* __restrict__ xn,
                                         int8_t* __restrict__ sn, float* __restrict__ y,
                                         float* __restrict__ p, const float* __restrict__ A,
                                         float c, float dt, float p_shared, float inv_rem, int i,
                                         int rlane, int N, int* status) {
    const float4 f = row_coupling<SIGN, EXACT, CG, MLP4>(rowptr, col, val, xc, sc, Rp, i, rlane, N,
                                                         status);
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

// MLP4: four gathers of a row in flight at once (more registers, fewer
// resident warps); taken when the state fits in half the L2, where the gathers'
// latency bounds the step: 12.7 -> 11.4 us per step at N = 2000, R = 512, and
// 90 -> 92 us at N = 20000, where the state streams from HBM.
template <bool SIGN, bool CONTROL, bool EXACT, bool MLP4>
__global__ void __launch_bounds__(256) k_csr_step(
    const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const float* __restrict__ val, int N, int Rp, const float* __restrict__ xc,
    const int8_t* __restrict__ sc, float* __restrict__ xn, int8_t* __restrict__ sn,
    float* __restrict__ y, float* __restrict__ p, const float* __restrict__ A, float c, float dt,
    float p_shared, float inv_rem, int* status) {
    // launched with programmatic dependent launch: the next step may be
    // scheduled once every block of this one has started; everything below
    // reads or writes state the previous step touched, so it waits for it
    griddep_trigger();
    griddep_wait();
    const int i = blockIdx.y * kWarpsPerBlock + (threadIdx.x >> 5);
    if (i >= N) return;
    const int rlane = blockIdx.x * kReplicasPerWarp + (threadIdx.x & 31) * 4;
    csr_task<SIGN, CONTROL, EXACT, false, MLP4>(rowptr, col, val, Rp, xc, sc, xn, sn, y, p, A, c,
                                                dt, p_shared, inv_rem, i, rlane, N, status);
}

// Fused multi-step form (the steps of Sec. II repeated, one cooperative launch
// per stretch of steps between energy evaluations): every warp takes the
// (row, 128-replica) tasks w, w + W, ... of each step -- the same tasks every
// step, so a task's y and p stay with one SM -- and the CTAs meet at a grid
// barrier between steps (release add / acquire poll on a counter, bounded).
// The gathered rows of x (or sgn x) were written by other SMs the step before,
// so they are read through L2 (ld.global.cg), never from a stale L1 line. The
// buffers alternate with the step's parity from the run's current one.
template <bool SIGN, bool CONTROL, bool EXACT>
__global__ void __launch_bounds__(256) k_csr_persist(
    const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const float* __restrict__ val, int N, int Rp, float* __restrict__ xa, float* __restrict__ xb,
    int8_t* __restrict__ sa, int8_t* __restrict__ sb, float* __restrict__ y,
    float* __restrict__ p, const float* __restrict__ A, float c, float dt,
    const float* __restrict__ p_sched, int M, int m0, int nsteps, uint32_t* __restrict__ bar,
    int* status) {
    __shared__ int abort_flag;
    if (threadIdx.x == 0) abort_flag = 0;
    __syncthreads();
    const int w0 = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int W = (int)((gridDim.x * blockDim.x) >> 5);
    const int nrb = Rp / kReplicasPerWarp;
    const int ntask = N * nrb;
    const int lane = threadIdx.x & 31;
    for (int s = 0; s < nsteps; ++s) {
        const int m = m0 + s;
        const bool odd = s & 1;
        const float* xc = odd ? xb : xa;
        float* xn = odd ? xa : xb;
        const int8_t* sc = odd ? sb : sa;
        int8_t* sn = odd ? sa : sb;
        const float inv_rem = __frcp_rn((float)(M - m));
        const float p_shared = CONTROL ? 0.f : p_sched[m];
        for (int t = w0; t < ntask; t += W) {
            const int i = t / nrb;
            const int rlane = (t - i * nrb) * kReplicasPerWarp + lane * 4;
            csr_task<SIGN, CONTROL, EXACT, true, true>(rowptr, col, val, Rp, xc, sc, xn, sn, y, p,
                                                       A, c, dt, p_shared, inv_rem, i, rlane, N,
                                                       status);
        }
        if (s + 1 == nsteps) break;
        // grid barrier: every CTA's writes of this step before any read of the next
        __syncthreads();
        if (threadIdx.x == 0) {
            tc::red_release_add(bar, 1u);
            const uint32_t target = (uint32_t)(s + 1) * gridDim.x;
            if (!tc::bounded_wait([&] { return tc::ld_acquire(bar) >= target; }, status,
                                  tc::kWaitLimitCycles))
                abort_flag = 1;
        }
        __syncthreads();
        if (abort_flag) break;
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
                                                    double* __restrict__ e_acc, int* status) {
    __shared__ float red[kWarpsPerBlock][kReplicasPerWarp];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rlane = blockIdx.x * kReplicasPerWarp + lane * 4;
    const int row0 = (blockIdx.y * kWarpsPerBlock + warp) * kRowsPerWarp;
    float4 part = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int rr = 0; rr < kRowsPerWarp; ++rr) {
        const int i = row0 + rr;
        if (i >= N) break;
        float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
        int beg = rowptr[i], end = rowptr[i + 1];
#ifdef GSB_DEBUG
        if (!GSB_DOK(beg >= 0 && beg <= end && end <= rowptr[N], status)) end = beg = 0;
#endif
        for (int kb = beg; kb < end; kb += 32) {
            const int k = kb + lane;
            int cj = k < end ? col[k] : 0;
            float wj = k < end ? val[k] : 0.f;
            if (!GSB_DOK(cj >= 0 && cj < N, status)) {
                cj = 0;
                wj = 0.f;
            }
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
    GSB_CUDA_TRY(launch_pdl(run->csr_mlp4 ? k_csr_step<S, C, E, true> : k_csr_step<S, C, E, false>, \
                            grid, dim3(256), 0, run->stream, P->rowptr,                        \
                            P->col, P->val, run->N, run->Rp, (const float*)run->x[cur],      \
                            (const int8_t*)run->s8[cur], run->x[cur ^ 1], run->s8[cur ^ 1],  \
                            run->y, run->p, (const float*)run->A, sc.c, sc.dt, sc.p_next,    \
                            inv_rem, run->status))
    // exact fixed-point x coupling when J is integer and 2^30 sum_k |J_ik| fits in
    // int64, unless FP32 sums were asked for
    const bool exact = P->integer_J && P->max_row_abs < 4294967296.0 &&
                       run->params.precision != GSB_PREC_FP32;
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

namespace {

// The fused kernel for the run's coupling, control and exactness.
const void* csr_persist_kernel(const gsb_run_state* run) {
    const gsb_problem* P = run->prob;
    const bool exact = P->integer_J && P->max_row_abs < 4294967296.0 &&
                       run->params.precision != GSB_PREC_FP32;
    if (run->sign_coupling)
        return run->control ? (const void*)k_csr_persist<true, true, false>
                            : (const void*)k_csr_persist<true, false, false>;
    if (exact)
        return run->control ? (const void*)k_csr_persist<false, true, true>
                            : (const void*)k_csr_persist<false, false, true>;
    return run->control ? (const void*)k_csr_persist<false, true, false>
                        : (const void*)k_csr_persist<false, false, false>;
}

}  // namespace

// Fused multi-step launches, asked for with GSB_RUN_FUSED_CSR (one step per
// launch with programmatic dependent launch measured faster on the ER
// workloads: 12.6 against 13.7 us per step at N = 2000, R = 512, 90 against
// 93 us at N = 20000; the grid barrier costs about what the overlapped launch
// gap did): the cooperative grid is every block that fits at once, at most one
// warp per task; its barrier counter and the shared p(t_{m+1}) of every step.
gsb_status csr_setup(gsb_run_state* run) {
    run->csr_grid = 0;
    {
        // the per-step kernel's gathers: four in flight while the state (x
        // twice, y, p) fits in half the L2
        int dev = 0, l2 = 0;
        GSB_CUDA_TRY(cudaGetDevice(&dev));
        GSB_CUDA_TRY(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
        run->csr_mlp4 = 16.0 * run->Np * run->Rp <= 0.5 * l2;
    }
    if (!(run->params.flags & GSB_RUN_FUSED_CSR) || run->params.steps_per_launch == 1)
        return GSB_OK;
    int dev = 0, sms = 0, coop = 0, per_sm = 0;
    GSB_CUDA_TRY(cudaGetDevice(&dev));
    GSB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    GSB_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) return GSB_OK;
    GSB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, csr_persist_kernel(run),
                                                               kWarpsPerBlock * 32, 0));
    if (per_sm < 1) return GSB_OK;
    const long ntask = (long)run->N * (run->Rp / kReplicasPerWarp);
    const long want = (ntask + kWarpsPerBlock - 1) / kWarpsPerBlock;
    gsb_status st;
    if ((st = dev_alloc(&run->csr_bar, 1))) return st;
    if ((st = dev_alloc(&run->csr_psched, (size_t)run->params.M))) return st;
    std::vector<float> ps(run->params.M);
    for (int m = 0; m < run->params.M; ++m) ps[m] = run_p_shared(run, m + 1);
    GSB_CUDA_TRY(cudaMemcpy(run->csr_psched, ps.data(), sizeof(float) * run->params.M,
                            cudaMemcpyHostToDevice));
    run->csr_grid = (int)std::min<long>((long)per_sm * sms, want);
    return GSB_OK;
}

// Steps [m0, m0 + nsteps) of a CSR run on the fused kernel: one launch per
// stretch of steps between energy evaluations (at most steps_per_launch).
gsb_status csr_steps(gsb_run_state* run, int m0, int nsteps) {
    const gsb_problem* P = run->prob;
    const void* kern = csr_persist_kernel(run);
    const int end = m0 + nsteps;
    const int spl = run->params.steps_per_launch;
    int m = m0;
    while (m < end) {
        int stop = end;
        for (int k = m + 1; k <= end; ++k)
            if (run_is_eval_step(run, k)) {
                stop = k;
                break;
            }
        if (spl > 0 && stop - m > spl) stop = m + spl;
        int n = stop - m, N = run->N, Rp = run->Rp, M = run->params.M;
        const int cur = run->cur;
        float c = run->c, dt = run->dt;
        GSB_CUDA_TRY(cudaMemsetAsync(run->csr_bar, 0, sizeof(uint32_t), run->stream));
        void* args[] = {(void*)&P->rowptr, (void*)&P->col,      (void*)&P->val,
                        &N,                &Rp,                  (void*)&run->x[cur],
                        (void*)&run->x[cur ^ 1], (void*)&run->s8[cur], (void*)&run->s8[cur ^ 1],
                        (void*)&run->y,    (void*)&run->p,       (void*)&run->A,
                        &c,                &dt,                  (void*)&run->csr_psched,
                        &M,                &m,                   &n,
                        (void*)&run->csr_bar, (void*)&run->status};
        gsb_status st = prof_begin(run);
        if (st != GSB_OK) return st;
        GSB_CUDA_TRY(cudaLaunchCooperativeKernel(kern, dim3(run->csr_grid), dim3(kWarpsPerBlock * 32),
                                                 args, 0, run->stream));
        count_launch();
        if ((st = prof_end(run, n)) != GSB_OK) return st;
        if (n & 1) run->cur ^= 1;
        m = stop;
        if (run_is_eval_step(run, m))
            if ((st = run_evaluate(run, m)) != GSB_OK) return st;
    }
    return GSB_OK;
}

// Debug build: the CSR energy kernel on a 4-row matrix whose third row names
// column 9; its check must skip that gather and report it.
gsb_status csr_debug_selftest(int* status, cudaStream_t s) {
#ifndef GSB_DEBUG
    // the release kernel has no check: it must never see this matrix
    (void)status;
    (void)s;
    return set_error(GSB_EUNSUPPORTED, "built without GSB_DEBUG");
#endif
    const int N = 4, Rp = kReplicasPerWarp;
    const int32_t rowptr_h[N + 1] = {0, 1, 2, 3, 4};
    const int32_t col_h[N] = {1, 0, 9, 2};
    const float val_h[N] = {1.f, 1.f, 1.f, 1.f};
    gsb_problem P;
    P.N = N;
    float* x = nullptr;
    double* e = nullptr;
    gsb_status st = GSB_OK;
    if ((st = dev_alloc(&P.rowptr, N + 1)) || (st = dev_alloc(&P.col, N)) ||
        (st = dev_alloc(&P.val, N)) || (st = dev_alloc(&x, (size_t)N * Rp)) ||
        (st = dev_alloc(&e, Rp))) {
    } else if (cudaMemcpyAsync(P.rowptr, rowptr_h, sizeof(rowptr_h), cudaMemcpyHostToDevice, s) ||
               cudaMemcpyAsync(P.col, col_h, sizeof(col_h), cudaMemcpyHostToDevice, s) ||
               cudaMemcpyAsync(P.val, val_h, sizeof(val_h), cudaMemcpyHostToDevice, s) ||
               cudaMemsetAsync(x, 0, sizeof(float) * N * Rp, s) ||
               cudaMemsetAsync(e, 0, sizeof(double) * Rp, s)) {
        st = cuda_error(cudaGetLastError(), "debug self-test set-up");
    } else {
        st = launch_csr_energy(&P, x, Rp, e, s, status);
        if (st == GSB_OK && cudaStreamSynchronize(s) != cudaSuccess)
            st = cuda_error(cudaGetLastError(), "debug self-test");
    }
    if (cudaStreamSynchronize(s) != cudaSuccess && st == GSB_OK)
        st = cuda_error(cudaGetLastError(), "debug self-test");
    dev_free(P.rowptr);
    dev_free(P.col);
    dev_free(P.val);
    P.rowptr = nullptr;
    P.col = nullptr;
    P.val = nullptr;
    dev_free(x);
    dev_free(e);
    return st;
}

gsb_status launch_csr_energy(const gsb_problem* P, const float* x, int Rp, double* e_acc,
                             cudaStream_t s, int* status) {
    const int rows_per_block = kWarpsPerBlock * kRowsPerWarp;
    dim3 grid(Rp / kReplicasPerWarp, (P->N + rows_per_block - 1) / rows_per_block);
    k_csr_energy<<<grid, 256, 0, s>>>(P->rowptr, P->col, P->val, P->N, Rp, x, e_acc, status);
    GSB_LAUNCH_CHECK("k_csr_energy");
    return GSB_OK;
}

}  // namespace gsb
