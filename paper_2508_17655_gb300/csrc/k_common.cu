// k_common.cu -- state initialisation (App. A), layout transposes, energy
// best-keeping, and the Lanczos iteration that sets c and dt (App. A, Eq. 13).
#include "gsb_internal.cuh"
#include "philox.cuh"

namespace gsb {


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

// Host-layout [R][ncols] (replica-major) to the spin-major state layout
// [Np][Rp]: rows ncols .. N-1 (the auxiliary spin of the h augmentation) get
// `aux`, padded spins and replicas get 0.
template <typename T>
__global__ void k_rm_to_sm(const T* __restrict__ src, T* __restrict__ dst, int ncols, int N, int R,
                           int Rp, T aux) {
    __shared__ T tile[32][33];
    const int i0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, i = i0 + threadIdx.x;
        T v = T(0);
        if (r < R && i < ncols) v = src[(size_t)r * ncols + i];
        else if (r < R && i < N) v = aux;
        tile[k][threadIdx.x] = v;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int i = i0 + k, r = r0 + threadIdx.x;
        dst[(size_t)i * Rp + r] = tile[threadIdx.x][k];
    }
}

gsb_status launch_rm_to_sm(const float* src, float* dst, int ncols, int N, int R, int Np, int Rp,
                           cudaStream_t s) {
    dim3 grid(Np / 32, Rp / 32), block(32, 8);
    k_rm_to_sm<float><<<grid, block, 0, s>>>(src, dst, ncols, N, R, Rp, 0.f);
    GSB_LAUNCH_CHECK("k_rm_to_sm");
    return GSB_OK;
}

gsb_status launch_rm_to_sm_i8(const int8_t* src, int8_t* dst, int ncols, int N, int R, int Np,
                              int Rp, int8_t aux, cudaStream_t s) {
    dim3 grid(Np / 32, Rp / 32), block(32, 8);
    k_rm_to_sm<int8_t><<<grid, block, 0, s>>>(src, dst, ncols, N, R, Rp, aux);
    GSB_LAUNCH_CHECK("k_rm_to_sm");
    return GSB_OK;
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

// ---------------------------------------------------------------- extreme eigenvalues
// lambda_max and lambda_min of J (App. A) by the Lanczos method: from a random
// unit v_0, w = J v_j - beta_j v_{j-1}, alpha_j = v_j . w, w -= alpha_j v_j
// (and once more against v_j, the local correction), beta_{j+1} = |w|,
// v_{j+1} = w / beta_{j+1}, all on the GPU in FP64. The extreme eigenvalues of
// the tridiagonal matrix T (alpha on the diagonal, beta beside it) converge to
// those of J from inside; the loss of orthogonality of the plain recurrence
// only adds copies of converged Ritz values, not wrong extremes. The host
// bisects T's Sturm sequence for them every kCheck steps and stops once both
// stand still (or the Krylov space is invariant). Every sum is a block
// reduction added in a fixed order: the result does not vary run to run.

// w = J v, one warp per row (dense FP32 or CSR), FP64 accumulation.
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

constexpr int kLzThreads = 256;

// part[block] = sum over the block's grid-stride slice of a_i b_i, added in a
// fixed order (warp shuffles, then the warps in order).
__global__ void __launch_bounds__(kLzThreads) k_lz_dot(const double* __restrict__ a,
                                                       const double* __restrict__ b, int N,
                                                       double* __restrict__ part) {
    __shared__ double ws[kLzThreads / 32];
    double t = 0.0;
    for (int i = blockIdx.x * kLzThreads + threadIdx.x; i < N; i += gridDim.x * kLzThreads)
        t += a[i] * b[i];
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x % 32 == 0) ws[threadIdx.x / 32] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0.0;
        for (int k = 0; k < kLzThreads / 32; ++k) u += ws[k];
        part[blockIdx.x] = u;
    }
}

// The sum of the parts, in block order (every block computes the same value).
__device__ __forceinline__ double parts_sum(const double* __restrict__ part, int nparts) {
    __shared__ double t;
    if (threadIdx.x == 0) {
        double u = 0.0;
        for (int k = 0; k < nparts; ++k) u += part[k];
        t = u;
    }
    __syncthreads();
    return t;
}

// w -= coef v with coef = the dot product in part; alpha[j] = coef (set) or
// += coef (accumulate), written by block 0.
__global__ void k_lz_remove(const double* __restrict__ part, int nparts,
                            const double* __restrict__ v, int N, double* __restrict__ w,
                            double* __restrict__ alpha, int j, int accumulate) {
    const double coef = parts_sum(part, nparts);
    if (blockIdx.x == 0 && threadIdx.x == 0) alpha[j] = accumulate ? alpha[j] + coef : coef;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        w[i] -= coef * v[i];
}

// w -= beta[j] vprev
__global__ void k_lz_axpy(const double* __restrict__ beta, int j, const double* __restrict__ vprev,
                          int N, double* __restrict__ w) {
    const double bj = beta[j];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        w[i] -= bj * vprev[i];
}

// nrm = sqrt(<w, w>) from part; beta[j] = nrm; dst = w / nrm (0 if nrm is 0)
__global__ void k_lz_normalize(const double* __restrict__ part, int nparts,
                               const double* __restrict__ w, int N, double* __restrict__ dst,
                               double* __restrict__ beta, int j) {
    const double nrm = sqrt(parts_sum(part, nparts));
    if (blockIdx.x == 0 && threadIdx.x == 0) beta[j] = nrm;
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        dst[i] = w[i] * inv;
}

__global__ void k_lz_start(double* v, int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint4 w = philox4x32_10(make_uint4((uint32_t)i, 0u, 77u, 0u), make_uint2(2718u, 0u));
    v[i] = ((double)(w.x >> 8) + 0.5) / 16777216.0 - 0.5;
}

// Number of eigenvalues below x of the symmetric tridiagonal matrix with
// diagonal a[0..n-1] and off-diagonal b[1..n-1] (signs of the LDL^T pivots).
int sturm_below(const std::vector<double>& a, const std::vector<double>& b, int n, double x) {
    int c = 0;
    double q = 1.0;
    for (int k = 0; k < n; ++k) {
        q = a[k] - x - (k ? b[k] * b[k] / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++c;
    }
    return c;
}

// Smallest and largest eigenvalue of that matrix: bisection on the count
// inside the Gershgorin interval.
void tridiag_extremes(const std::vector<double>& a, const std::vector<double>& b, int n,
                      double* lmin, double* lmax) {
    double lo = INFINITY, hi = -INFINITY;
    for (int k = 0; k < n; ++k) {
        const double r = (k ? fabs(b[k]) : 0.0) + (k + 1 < n ? fabs(b[k + 1]) : 0.0);
        lo = fmin(lo, a[k] - r);
        hi = fmax(hi, a[k] + r);
    }
    auto bisect = [&](int target) {  // the x where the count reaches target
        double l = lo - (fabs(lo) + 1.0) * 1e-12, h = hi + (fabs(hi) + 1.0) * 1e-12;
        for (int it = 0; it < 300; ++it) {
            const double mid = 0.5 * (l + h);
            if (mid <= l || mid >= h) break;
            if (sturm_below(a, b, n, mid) >= target) h = mid; else l = mid;
        }
        return 0.5 * (l + h);
    };
    *lmin = bisect(1);
    *lmax = bisect(n);
}

gsb_status compute_lambda(gsb_problem* P, cudaStream_t s) {
    if (P->have_lambda) return GSB_OK;
    const int N = P->N;
    const int mmax = N < 2000 ? N : 2000;  // steps at most
    constexpr int kCheck = 16;
    const int eb = (N + kLzThreads - 1) / kLzThreads;
    const int nparts = eb < 256 ? eb : 256;
    double *v[3] = {nullptr, nullptr, nullptr}, *w = nullptr, *part = nullptr, *alpha = nullptr,
           *beta = nullptr;
    auto release = [&]() {
        for (double* q : v) cudaFree(q);
        cudaFree(w);
        cudaFree(part);
        cudaFree(alpha);
        cudaFree(beta);
    };
    bool ok = true;
    for (double*& q : v) ok = ok && cudaMalloc(&q, sizeof(double) * N) == cudaSuccess;
    ok = ok && cudaMalloc(&w, sizeof(double) * N) == cudaSuccess &&
         cudaMalloc(&part, sizeof(double) * nparts) == cudaSuccess &&
         cudaMalloc(&alpha, sizeof(double) * (mmax + 1)) == cudaSuccess &&
         cudaMalloc(&beta, sizeof(double) * (mmax + 2)) == cudaSuccess;
    if (!ok) {
        release();
        return set_error(GSB_ENOMEM, "eigenvalue workspace");
    }
    auto gemv = [&](const double* in, double* out) {
        const int blocks = (N + 7) / 8;
        if (P->csr)
            k_gemv_csr<<<blocks, 256, 0, s>>>(P->rowptr, P->col, P->val, in, out, N);
        else
            k_gemv_dense<<<blocks, 256, 0, s>>>(P->J32, in, out, N, P->Np);
    };
    // v_0: random, unit (beta[0] holds its norm before scaling; unused after)
    k_lz_start<<<eb, kLzThreads, 0, s>>>(w, N);
    k_lz_dot<<<nparts, kLzThreads, 0, s>>>(w, w, N, part);
    k_lz_normalize<<<nparts, kLzThreads, 0, s>>>(part, nparts, w, N, v[0], beta, 0);
    count_launch(3);
    std::vector<double> a(mmax + 1), b(mmax + 2);
    double pmin = 0.0, pmax = 0.0, lmin = 0.0, lmax = 0.0;
    gsb_status st = GSB_OK;
    int prev = 2, cur = 0, next = 1;  // v[prev] = v_{j-1}, v[cur] = v_j
    for (int j = 0; j < mmax; ++j) {
        gemv(v[cur], w);
        if (j > 0) k_lz_axpy<<<nparts, kLzThreads, 0, s>>>(beta, j, v[prev], N, w);
        k_lz_dot<<<nparts, kLzThreads, 0, s>>>(v[cur], w, N, part);
        k_lz_remove<<<nparts, kLzThreads, 0, s>>>(part, nparts, v[cur], N, w, alpha, j, 0);
        k_lz_dot<<<nparts, kLzThreads, 0, s>>>(v[cur], w, N, part);
        k_lz_remove<<<nparts, kLzThreads, 0, s>>>(part, nparts, v[cur], N, w, alpha, j, 1);
        k_lz_dot<<<nparts, kLzThreads, 0, s>>>(w, w, N, part);
        k_lz_normalize<<<nparts, kLzThreads, 0, s>>>(part, nparts, w, N, v[next], beta, j + 1);
        count_launch(j > 0 ? 8 : 7);
        const int t = prev;
        prev = cur;
        cur = next;
        next = t;
        const int n = j + 1;
        if (n % kCheck != 0 && n != mmax) continue;
        if (cudaMemcpyAsync(a.data(), alpha, sizeof(double) * n, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(b.data(), beta, sizeof(double) * (n + 1), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            st = cuda_error(cudaGetLastError(), "eigenvalue iteration");
            break;
        }
        tridiag_extremes(a, b, n, &lmin, &lmax);
        const double scale = fmax(fabs(lmin), fabs(lmax)) + 1e-300;
        // the Krylov space is invariant (b[n] = 0), or both Ritz values stand still
        if (b[n] <= 1e-12 * scale ||
            (n > kCheck && fabs(lmax - pmax) <= 1e-14 * scale && fabs(lmin - pmin) <= 1e-14 * scale))
            break;
        pmin = lmin;
        pmax = lmax;
    }
    release();
    if (st != GSB_OK) return st;
    P->lambda_max = lmax;
    P->lambda_min = lmin;
    P->have_lambda = true;
    return GSB_OK;
}

}  // namespace gsb
