// k_common.cu -- state initialisation (App. A), layout transposes, energy
// best-keeping, and the power iteration that sets c and dt (App. A, Eq. 13).
#include "gsb_internal.cuh"

namespace gsb {

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of the 4x32 S-box, key
// bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 ctr, uint2 key) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round) {
            key.x += 0x9E3779B9u;
            key.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * ctr.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, ctr.x);
        const uint32_t lo1 = 0xCD9E8D57u * ctr.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, ctr.z);
        ctr = make_uint4(hi1 ^ ctr.y ^ key.x, lo1, hi0 ^ ctr.w ^ key.y, lo0);
    }
    return ctr;
}

// Uniform value in [-range, range): k = top 24 bits - 2^23, times range 2^-23,
// one FP32 rounding. Counter (i, r, stream, 0), key = seed.
__device__ __forceinline__ float uniform_draw(int i, int r, uint32_t stream, uint2 key,
                                              float scale) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)r, stream, 0u), key);
    const int k = (int)(w.x >> 8) - 8388608;
    return __fmul_rn((float)k, scale);
}

// x(0), y(0), p(0) = 1 in the spin-major [Np][Rp] layout; padded spins and
// replicas start (and, with y = 0, stay) at zero.
__global__ void k_init_state(float* __restrict__ x, float* __restrict__ y, float* __restrict__ p,
                             int N, int R, int Np, int Rp, uint2 key, float scale, int y_uniform,
                             const float* __restrict__ x0_rm, const float* __restrict__ y0_rm) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (r >= Rp || i >= Np) return;
    const size_t o = (size_t)i * Rp + r;
    float xv = 0.f, yv = 0.f;
    if (i < N && r < R) {
        xv = x0_rm ? x0_rm[(size_t)r * N + i] : uniform_draw(i, r, 0u, key, scale);
        if (y0_rm)
            yv = y0_rm[(size_t)r * N + i];
        else if (y_uniform)
            yv = uniform_draw(i, r, 1u, key, scale);
    }
    x[o] = xv;
    y[o] = yv;
    if (p) p[o] = 1.f;
}

// Twin initial conditions of the chaos measure (Sec. IV): pair q = 0..Q-1 runs as
// replicas q and Q + q. x^(1)_i = +-0.1 and x^(2)_i = x^(1)_i +- 2e-6, each sign
// drawn independently (Philox streams 2 and 3 at counter (i, q, stream, 0); a
// draw >= 0 gives +); x^(2) is the FP64 sum rounded once to FP32. y = 0, p = 1.
__global__ void k_twin_init(float* __restrict__ x, float* __restrict__ y, float* __restrict__ p,
                            int N, int Q, int Np, int Rp, uint2 key) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (r >= Rp || i >= Np) return;
    const size_t o = (size_t)i * Rp + r;
    float xv = 0.f;
    if (i < N && r < 2 * Q) {
        const int q = r < Q ? r : r - Q;
        const double x1 = uniform_draw(i, q, 2u, key, 1.f) >= 0.f ? 0.1 : -0.1;
        if (r < Q) {
            xv = __double2float_rn(x1);
        } else {
            const double e = uniform_draw(i, q, 3u, key, 1.f) >= 0.f ? 2e-6 : -2e-6;
            xv = __double2float_rn(x1 + e);
        }
    }
    x[o] = xv;
    y[o] = 0.f;
    if (p) p[o] = 1.f;
}

__global__ void k_sign_extract(const float* __restrict__ x, int8_t* __restrict__ s, size_t n) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) s[k] = x[k] >= 0.f ? (int8_t)1 : (int8_t)-1;
}

// [Np][Rp] spin-major -> [R][N] replica-major, through a 32 x 33 tile.
template <typename T>
__global__ void k_transpose_out(const T* __restrict__ src, T* __restrict__ dst, int Rp, int N,
                                int R) {
    __shared__ T tile[32][33];
    const int r0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int i = i0 + k, r = r0 + threadIdx.x;
        tile[k][threadIdx.x] = (i < N && r < R) ? src[(size_t)i * Rp + r] : T(0);
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, i = i0 + threadIdx.x;
        if (r < R && i < N) dst[(size_t)r * N + i] = tile[threadIdx.x][k];
    }
}

// Caller spins [R][N] int8 -> x state [Np][Rp] float +-1 (zero padding).
__global__ void k_spins_in(const int8_t* __restrict__ s, float* __restrict__ x, int N, int R,
                           int Rp) {
    __shared__ float tile[32][33];
    const int i0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, i = i0 + threadIdx.x;
        tile[k][threadIdx.x] = (r < R && i < N) ? (float)s[(size_t)r * N + i] : 0.f;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int i = i0 + k, r = r0 + threadIdx.x;
        x[(size_t)i * Rp + r] = tile[threadIdx.x][k];
    }
}

gsb_status launch_init_state(gsb_run_state* run, const float* x0_rm, const float* y0_rm) {
    const gsb_params& P = run->params;
    const float range = P.x0_range > 0.f ? P.x0_range : 0.1f;
    const float scale = range * 1.1920928955078125e-07f;  // times 2^-23, exact
    const uint2 key = make_uint2((uint32_t)P.seed, (uint32_t)(P.seed >> 32));
    dim3 grid((run->Rp + 127) / 128, run->Np);
    if (run->twin_pairs > 0) {
        k_twin_init<<<grid, 128, 0, run->stream>>>(run->x[0], run->y, run->p, run->N,
                                                   run->twin_pairs, run->Np, run->Rp, key);
        GSB_LAUNCH_CHECK("k_twin_init");
    } else {
        k_init_state<<<grid, 128, 0, run->stream>>>(run->x[0], run->y, run->p, run->N, run->R,
                                                    run->Np, run->Rp, key, scale, P.y0_uniform,
                                                    x0_rm, y0_rm);
        GSB_LAUNCH_CHECK("k_init_state");
    }
    run->cur = 0;
    if (run->s8[0]) return launch_sign_extract(run);
    return GSB_OK;
}

gsb_status launch_sign_extract(gsb_run_state* run) {
    const size_t n = (size_t)run->Np * run->Rp;
    k_sign_extract<<<(unsigned)((n + 255) / 256), 256, 0, run->stream>>>(run->x[run->cur],
                                                                          run->s8[run->cur], n);
    GSB_LAUNCH_CHECK("k_sign_extract");
    return GSB_OK;
}

gsb_status launch_transpose_to_host_layout(const float* src, float* dst, int Np, int Rp, int N,
                                           int R, cudaStream_t s) {
    (void)Np;
    dim3 grid((R + 31) / 32, (N + 31) / 32), block(32, 8);
    k_transpose_out<float><<<grid, block, 0, s>>>(src, dst, Rp, N, R);
    GSB_LAUNCH_CHECK("k_transpose_out<float>");
    return GSB_OK;
}

gsb_status launch_transpose_i8_to_host_layout(const int8_t* src, int8_t* dst, int Np, int Rp,
                                              int N, int R, cudaStream_t s) {
    (void)Np;
    dim3 grid((R + 31) / 32, (N + 31) / 32), block(32, 8);
    k_transpose_out<int8_t><<<grid, block, 0, s>>>(src, dst, Rp, N, R);
    GSB_LAUNCH_CHECK("k_transpose_out<int8>");
    return GSB_OK;
}

gsb_status launch_spins_to_state(const int8_t* spins_rm, float* x_sm, int N, int R, int Np,
                                 int Rp, cudaStream_t s) {
    dim3 grid(Np / 32, Rp / 32), block(32, 8);
    k_spins_in<<<grid, block, 0, s>>>(spins_rm, x_sm, N, R, Rp);
    GSB_LAUNCH_CHECK("k_spins_in");
    return GSB_OK;
}

// ---------------------------------------------------------------- best keeping
// E = -1/2 sum_i s_i (J s)_i (Eq. 1). Strict improvement: the earliest
// evaluated step wins a tie.
__global__ void k_best_decide(const double* __restrict__ e_acc, double* __restrict__ best_e,
                              int32_t* __restrict__ best_step, int32_t* __restrict__ flag, int R,
                              int step, int* status) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const double e = -0.5 * e_acc[r];
    int f = 0;
    if (e < best_e[r]) {
        best_e[r] = e;
        best_step[r] = step;
        f = 1;
    }
    flag[r] = f;
    if (!isfinite(e)) atomicOr(status, kDevNumeric);
}

__global__ void k_best_copy(const float* __restrict__ x, int8_t* __restrict__ best_s,
                            const int32_t* __restrict__ flag, int N, int R, int Rp,
                            int* status) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (r >= R || i >= N) return;
    const float v = x[(size_t)i * Rp + r];
    if (!isfinite(v)) atomicOr(status, kDevNumeric);
    if (flag[r]) best_s[(size_t)i * Rp + r] = v >= 0.f ? (int8_t)1 : (int8_t)-1;
}

gsb_status launch_best_keep(gsb_run_state* run, int step) {
    k_best_decide<<<(run->R + 255) / 256, 256, 0, run->stream>>>(
        run->e_acc, run->best_e, run->best_step, run->flag, run->R, step, run->status);
    GSB_LAUNCH_CHECK("k_best_decide");
    dim3 grid((run->R + 127) / 128, run->N);
    k_best_copy<<<grid, 128, 0, run->stream>>>(run->x[run->cur], run->best_s, run->flag, run->N,
                                               run->R, run->Rp, run->status);
    GSB_LAUNCH_CHECK("k_best_copy");
    return GSB_OK;
}

// ---------------------------------------------------------------- power iteration
// Extreme eigenvalues of J (App. A): spectral radius rho from J^2, then the
// dominant eigenvalues of J + sigma I and sigma I - J with sigma = 1.01 rho.

// w = J v, one warp per row (dense FP32 or CSR).
__global__ void k_gemv_dense(const float* __restrict__ J, const double* __restrict__ v,
                             double* __restrict__ w, int N, int Np) {
    const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x % 32;
    if (row >= N) return;
    double acc = 0.0;
    for (int j = lane; j < N; j += 32) acc += (double)J[(size_t)row * Np + j] * v[j];
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (!lane) w[row] = acc;
}

__global__ void k_gemv_csr(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                           const float* __restrict__ val, const double* __restrict__ v,
                           double* __restrict__ w, int N) {
    const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x % 32;
    if (row >= N) return;
    double acc = 0.0;
    for (int k = rowptr[row] + lane; k < rowptr[row + 1]; k += 32) acc += (double)val[k] * v[col[k]];
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (!lane) w[row] = acc;
}

// acc[0] += v.w', acc[1] += w'.w' with w' = sigma v + sgn w.
__global__ void k_pi_dots(const double* __restrict__ v, double* __restrict__ w, int N,
                          double sigma, double sgn, double* acc) {
    __shared__ double s0[8], s1[8];
    double a = 0.0, b = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const double wi = sigma * v[i] + sgn * w[i];
        w[i] = wi;
        a += v[i] * wi;
        b += wi * wi;
    }
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (threadIdx.x % 32 == 0) {
        s0[threadIdx.x / 32] = a;
        s1[threadIdx.x / 32] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x / 32); ++k) {
            a += s0[k];
            b += s1[k];
        }
        atomicAdd(&acc[0], a);
        atomicAdd(&acc[1], b);
    }
}

// v = w / |w|, records the Rayleigh quotient v.w' (v unit) in rq[it].
__global__ void k_pi_normalize(double* __restrict__ v, const double* __restrict__ w, int N,
                               double* acc, double* rq, int it) {
    const double nrm = sqrt(acc[1]);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        v[i] = nrm > 0.0 ? w[i] / nrm : 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) rq[it] = acc[0];
}

__global__ void k_pi_init(double* v, int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint4 w = philox4x32_10(make_uint4((uint32_t)i, 0u, 77u, 0u), make_uint2(2718u, 0u));
    v[i] = ((double)(w.x >> 8) + 0.5) / 16777216.0 - 0.5;
}

__global__ void k_pi_zero(double* acc) {
    acc[0] = 0.0;
    acc[1] = 0.0;
}

__global__ void k_pi_unit(double* v, int N, double* acc) {
    // normalise the start vector: acc[1] must hold |v|^2
    const double nrm = sqrt(acc[1]);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        v[i] /= nrm;
}

__global__ void k_pi_sqnorm(const double* v, int N, double* acc) {
    double b = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        b += v[i] * v[i];
    for (int o = 16; o; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
    if (threadIdx.x % 32 == 0) atomicAdd(&acc[1], b);
}

// One power iteration phase on the GPU. mode 0: J^2 (returns rho^2);
// mode 1: J + sigma I; mode 2: sigma I - J. Returns the converged Rayleigh
// quotient of the iterated operator.
static gsb_status power_phase(gsb_problem* P, cudaStream_t s, int mode, double sigma,
                              double* result) {
    const int N = P->N;
    double *v = nullptr, *w = nullptr, *w2 = nullptr, *acc = nullptr, *rq = nullptr;
    const int kChunk = 64, kMaxIt = 20000;
    GSB_CUDA_TRY(cudaMalloc(&v, sizeof(double) * N));
    GSB_CUDA_TRY(cudaMalloc(&w, sizeof(double) * N));
    GSB_CUDA_TRY(cudaMalloc(&w2, sizeof(double) * N));
    GSB_CUDA_TRY(cudaMalloc(&acc, sizeof(double) * 2));
    GSB_CUDA_TRY(cudaMalloc(&rq, sizeof(double) * kChunk));
    gsb_status st = GSB_OK;
    const int gb = (N + 255) / 256 < 256 ? (N + 255) / 256 : 256;
    auto gemv = [&](const double* in, double* out) {
        const int blocks = (N + 7) / 8;
        if (P->csr)
            k_gemv_csr<<<blocks, 256, 0, s>>>(P->rowptr, P->col, P->val, in, out, N);
        else
            k_gemv_dense<<<blocks, 256, 0, s>>>(P->J32, in, out, N, P->Np);
        count_launch();
    };
    k_pi_init<<<(N + 255) / 256, 256, 0, s>>>(v, N);
    k_pi_zero<<<1, 1, 0, s>>>(acc);
    k_pi_sqnorm<<<gb, 256, 0, s>>>(v, N, acc);
    k_pi_unit<<<gb, 256, 0, s>>>(v, N, acc);
    count_launch(4);
    double prev = 0.0, cur = 0.0;
    double host_rq[kChunk];
    for (int it0 = 0; it0 < kMaxIt; it0 += kChunk) {
        for (int it = 0; it < kChunk; ++it) {
            gemv(v, w);
            double sg = -1.0;
            if (mode == 0) {
                gemv(w, w2);
                std::swap(w, w2);
                sg = 1.0;
            } else if (mode == 1) {
                sg = 1.0;
            }
            k_pi_zero<<<1, 1, 0, s>>>(acc);
            k_pi_dots<<<gb, 256, 0, s>>>(v, w, N, mode == 0 ? 0.0 : sigma, sg, acc);
            k_pi_normalize<<<gb, 256, 0, s>>>(v, w, N, acc, rq, it);
            count_launch(3);
        }
        cudaError_t e = cudaMemcpyAsync(host_rq, rq, sizeof(host_rq), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            st = cuda_error(e, "power iteration");
            break;
        }
        cur = host_rq[kChunk - 1];
        prev = host_rq[kChunk - 2];
        if (it0 > 0 && fabs(cur - prev) <= 1e-12 * fabs(cur)) break;
    }
    *result = cur;
    cudaFree(v);
    cudaFree(w);
    cudaFree(w2);
    cudaFree(acc);
    cudaFree(rq);
    return st;
}

gsb_status compute_lambda(gsb_problem* P, cudaStream_t s) {
    if (P->have_lambda) return GSB_OK;
    double rho2 = 0.0, top = 0.0, bot = 0.0;
    gsb_status st = power_phase(P, s, 0, 0.0, &rho2);
    if (st != GSB_OK) return st;
    const double sigma = 1.01 * sqrt(rho2 > 0.0 ? rho2 : 0.0) + 1e-300;
    if ((st = power_phase(P, s, 1, sigma, &top)) != GSB_OK) return st;
    if ((st = power_phase(P, s, 2, sigma, &bot)) != GSB_OK) return st;
    P->lambda_max = top - sigma;
    P->lambda_min = sigma - bot;
    P->have_lambda = true;
    return GSB_OK;
}

}  // namespace gsb
