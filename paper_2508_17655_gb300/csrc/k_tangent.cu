// k_tangent.cu -- tangent-linear propagation through the time step and the
// largest Lyapunov exponent (gsb_lyapunov).
//
// Linearising one step (Sec. II, Eqs. 3-7) in the state (x, y, p):
//   dp' = dp - [(1 - A x^2) dp - 2 A x dx p] / (M - m)   (individual control; 0 otherwise)
//   dy' = dy - [dp' x + p' dx - c (J dx)] dt              (sgn-x coupling: no J dx term)
//   dx' = dx + dy' dt;  where Eq. 5 clamps x', also dx' = dy' = 0.
// Each replica's tangent rides next to it: the state arrays hold column pairs
// (x_r, dx_r), so one FP32 SGEMM tile over 2R columns yields J x and J dx for
// the same thread, and the epilogue advances both. Every renorm_every steps
// (and at the end) the tangent is renormalised; the log of its norm is
// accumulated in FP64 per replica.
#include "gsb_update.cuh"
#include "philox.cuh"
#include "sgemm_f32.cuh"

namespace gsb {

namespace {

using namespace f32;

// State [Np][C] with C = 2 Rq columns, column 2r = replica r, 2r+1 = its tangent.
template <bool SIGN, bool CONTROL>
__global__ void __launch_bounds__(256) k_tangent_step(const float* __restrict__ J, int Np, int C,
                                                      const float* __restrict__ xc,
                                                      float* __restrict__ xn,
                                                      float* __restrict__ y,
                                                      float* __restrict__ p,
                                                      const float* __restrict__ A, float c,
                                                      float dt, float p_shared, float inv_rem) {
    __shared__ __align__(16) F32Smem sm;
    const int i0 = blockIdx.y * BM, r0 = blockIdx.x * BN;
    float acc[8][8];
    sgemm_tile<SIGN>(J, xc, Np, C, i0, r0, acc, sm);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int cols[2] = {r0 + tx * 4, r0 + 64 + tx * 4};
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const size_t rowoff = (size_t)(i0 + row_of(a, ty)) * C;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const size_t o = rowoff + cols[h];
            float4 x4 = *reinterpret_cast<const float4*>(xc + o);
            float4 y4 = *reinterpret_cast<float4*>(y + o);
            float4 p4 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (CONTROL) p4 = *reinterpret_cast<float4*>(p + o);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                float* xs = &x4.x + 2 * k;
                float* ys = &y4.x + 2 * k;
                float* ps = &p4.x + 2 * k;
                const float av = CONTROL ? A[(cols[h] >> 1) + k] : 0.f;
                sb_tangent_update<CONTROL, SIGN>(xs[0], ys[0], ps[0], xs[1], ys[1], ps[1],
                                                 acc[a][h * 4 + 2 * k], acc[a][h * 4 + 2 * k + 1],
                                                 av, c, dt, p_shared, inv_rem);
            }
            *reinterpret_cast<float4*>(xn + o) = x4;
            *reinterpret_cast<float4*>(y + o) = y4;
            if (CONTROL) *reinterpret_cast<float4*>(p + o) = p4;
        }
    }
}

// Initial state: replica r of the run draws x(0) (and y(0)) exactly as gsb_run
// does for replica r; its tangent starts at dx uniform in [-1, 1) (Philox
// stream 4), dy = dp = 0, normalised before the first step.

__global__ void k_tangent_init(float* x, float* y, float* p, int N, int R, int Np, int C,
                               uint2 key, float scale, int y_uniform) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (col >= C || i >= Np) return;
    const int r = col >> 1;
    const bool tangent = col & 1;
    const size_t o = (size_t)i * C + col;
    float xv = 0.f, yv = 0.f;
    if (i < N && r < R) {
        if (tangent) {
            xv = uniform_draw(i, r, 4u, key, 1.1920928955078125e-07f);  // uniform [-1, 1)
        } else {
            xv = uniform_draw(i, r, 0u, key, scale);
            if (y_uniform) yv = uniform_draw(i, r, 1u, key, scale);
        }
    }
    x[o] = xv;
    y[o] = yv;
    if (p) p[o] = tangent ? 0.f : 1.f;
}

// part[b][r] = sum over row block b (kNormRows rows) of dx^2 + dy^2 + dp^2, in
// FP64; the blocks are added in order by k_tangent_log (deterministic).
constexpr int kNormRows = 64;
__global__ void k_tangent_norm(const float* __restrict__ x, const float* __restrict__ y,
                               const float* __restrict__ p, int N, int C, int R,
                               double* __restrict__ part) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int i0 = blockIdx.y * kNormRows;
    const int i1 = min(N, i0 + kNormRows);
    double s = 0.0;
    for (int i = i0; i < i1; ++i) {
        const size_t o = (size_t)i * C + 2 * r + 1;
        const double a = x[o], b = y[o], d = p ? p[o] : 0.f;
        s += a * a + b * b + d * d;
    }
    part[(size_t)blockIdx.y * R + r] = s;
}

__global__ void k_tangent_log(const double* __restrict__ part, int nblk,
                              double* __restrict__ log_sum, float* __restrict__ scale, int R,
                              int accumulate) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    double s2 = 0.0;
    for (int b = 0; b < nblk; ++b) s2 += part[(size_t)b * R + r];
    if (accumulate) log_sum[r] += 0.5 * log(s2);
    scale[r] = s2 > 0.0 ? (float)(1.0 / sqrt(s2)) : 0.f;
}

__global__ void k_tangent_scale(float* x, float* y, float* p, int N, int C, int R,
                                const float* __restrict__ scale) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (r >= R || i >= N) return;
    const size_t o = (size_t)i * C + 2 * r + 1;
    const float s = scale[r];
    x[o] *= s;
    y[o] *= s;
    if (p) p[o] *= s;
}

struct TangentBuffers {
    float* x[2] = {nullptr, nullptr};
    float* y = nullptr;
    float* p = nullptr;
    float* A = nullptr;
    double* nrm2 = nullptr;
    double* log_sum = nullptr;
    float* scale = nullptr;
    ~TangentBuffers() {
        cudaFree(x[0]);
        cudaFree(x[1]);
        cudaFree(y);
        cudaFree(p);
        cudaFree(A);
        cudaFree(nrm2);
        cudaFree(log_sum);
        cudaFree(scale);
    }
};

}  // namespace

}  // namespace gsb

using namespace gsb;

extern "C" gsb_status gsb_lyapunov(gsb_problem* P, const gsb_params* prm, int32_t nA,
                                   const float* A_values, int32_t renorm_every, int32_t nsteps,
                                   double* mle_out, void* stream) {
    if (!P || !prm || !mle_out || nA < 1 || !A_values)
        return set_error(GSB_EINVAL, "NULL argument or nA < 1");
    const gsb_params& Q = *prm;
    if (P->csr) return set_error(GSB_EUNSUPPORTED, "gsb_lyapunov takes dense problems");
    if (Q.variant < GSB_BSB || Q.variant > GSB_GDSB) return set_error(GSB_EINVAL, "unknown variant");
    if (Q.M < 1 || Q.R < 1) return set_error(GSB_EINVAL, "M and R must be >= 1");
    if (renorm_every < 1) return set_error(GSB_EINVAL, "renorm_every must be >= 1");
    if (nsteps == 0) nsteps = Q.M;
    if (nsteps < 1 || nsteps > Q.M) return set_error(GSB_EINVAL, "nsteps must be in 1..M");
    if (Q.schedule) return set_error(GSB_EUNSUPPORTED, "gsb_lyapunov uses the Eq. 6 schedule");
    const long long Rtot = (long long)nA * Q.R;
    if (Rtot > (1 << 21)) return set_error(GSB_EINVAL, "nA * R too large");
    cudaStream_t s = (cudaStream_t)stream;
    double c = Q.c, dt = Q.dt;
    if (c == 0.0 || dt == 0.0) {
        gsb_status st = compute_lambda(P, s);
        if (st != GSB_OK) return st;
        if (c == 0.0) c = 1.0 / P->lambda_max;
        if (dt == 0.0) dt = 1.25 * sqrt(2.0 / (1.0 - P->lambda_min / P->lambda_max));
    }
    const bool sign = Q.variant == GSB_DSB || Q.variant == GSB_GDSB;
    const bool control = Q.variant == GSB_GBSB || Q.variant == GSB_GDSB;
    const int R = (int)Rtot;
    const float range = Q.x0_range > 0.f ? Q.x0_range : 0.1f;
    if (Q.precision == GSB_PREC_BF16X3) {
        // J x and J dx on the tensor cores (split bf16)
        std::vector<float> Ar((size_t)R);
        for (int k = 0; k < nA; ++k)
            for (int r = 0; r < Q.R; ++r) Ar[(size_t)k * Q.R + r] = A_values[k];
        std::vector<double> ls((size_t)R);
        gsb_status st = tangent_bf16x3(P, sign, control, R, Ar.data(), (float)c, (float)dt, Q.M,
                                       nsteps, renorm_every, Q.seed, range, Q.y0_uniform != 0,
                                       ls.data(), s);
        if (st != GSB_OK) return st;
        const double T = (double)nsteps * (double)(float)dt;
        for (int r = 0; r < R; ++r) mle_out[r] = ls[r] / T;
        return GSB_OK;
    }
    if (Q.precision != GSB_PREC_AUTO && Q.precision != GSB_PREC_FP32)
        return set_error(GSB_EUNSUPPORTED, "gsb_lyapunov takes FP32 or BF16X3 coupling");
    const int Rq = round_up(R, BN / 2);  // pairs, padded so 2 Rq is a multiple of the tile
    const int C = 2 * Rq;
    const int Np = P->Np;
    TangentBuffers B;
    const size_t nst = (size_t)Np * C;
    GSB_CUDA_TRY(cudaMalloc(&B.x[0], nst * sizeof(float)));
    GSB_CUDA_TRY(cudaMalloc(&B.x[1], nst * sizeof(float)));
    GSB_CUDA_TRY(cudaMalloc(&B.y, nst * sizeof(float)));
    if (control) GSB_CUDA_TRY(cudaMalloc(&B.p, nst * sizeof(float)));
    GSB_CUDA_TRY(cudaMalloc(&B.A, Rq * sizeof(float)));
    const int nblk = (P->N + kNormRows - 1) / kNormRows;
    GSB_CUDA_TRY(cudaMalloc(&B.nrm2, (size_t)nblk * R * sizeof(double)));
    GSB_CUDA_TRY(cudaMalloc(&B.log_sum, Rq * sizeof(double)));
    GSB_CUDA_TRY(cudaMalloc(&B.scale, Rq * sizeof(float)));
    std::vector<float> Ah(Rq, 0.f);
    for (int k = 0; k < nA; ++k)
        for (int r = 0; r < Q.R; ++r) Ah[(size_t)k * Q.R + r] = A_values[k];
    GSB_CUDA_TRY(cudaMemcpyAsync(B.A, Ah.data(), Rq * sizeof(float), cudaMemcpyHostToDevice, s));
    GSB_CUDA_TRY(cudaMemsetAsync(B.log_sum, 0, Rq * sizeof(double), s));
    const uint2 key = make_uint2((uint32_t)Q.seed, (uint32_t)(Q.seed >> 32));
    k_tangent_init<<<dim3((C + 127) / 128, Np), 128, 0, s>>>(
        B.x[0], B.y, B.p, P->N, R, Np, C, key, range * 1.1920928955078125e-07f, Q.y0_uniform);
    GSB_LAUNCH_CHECK("k_tangent_init");
    auto renorm = [&](int cur, int accumulate) -> gsb_status {
        k_tangent_norm<<<dim3((R + 127) / 128, nblk), 128, 0, s>>>(B.x[cur], B.y, B.p, P->N, C, R,
                                                                  B.nrm2);
        GSB_LAUNCH_CHECK("k_tangent_norm");
        k_tangent_log<<<(R + 255) / 256, 256, 0, s>>>(B.nrm2, nblk, B.log_sum, B.scale, R,
                                                      accumulate);
        GSB_LAUNCH_CHECK("k_tangent_log");
        k_tangent_scale<<<dim3((R + 127) / 128, P->N), 128, 0, s>>>(B.x[cur], B.y, B.p, P->N, C,
                                                                    R, B.scale);
        GSB_LAUNCH_CHECK("k_tangent_scale");
        return GSB_OK;
    };
    gsb_status st = renorm(0, 0);  // unit start vector
    if (st != GSB_OK) return st;
    int cur = 0;
    const dim3 grid(C / BN, Np / BM);
    call_prof_reset();
    for (int m = 0; m < nsteps; ++m) {
        const float p_shared = (float)(1.0 - (double)(m + 1) / (double)Q.M);
        const float inv_rem = 1.0f / (float)(Q.M - m);
#define GSB_TAN_LAUNCH(S, CT)                                                                  \
    k_tangent_step<S, CT><<<grid, 256, 0, s>>>(P->J32, Np, C, B.x[cur], B.x[cur ^ 1], B.y, B.p, \
                                               B.A, (float)c, (float)dt, p_shared, inv_rem)
        if ((st = call_prof_begin(s)) != GSB_OK) return st;
        if (sign) {
            if (control) GSB_TAN_LAUNCH(true, true); else GSB_TAN_LAUNCH(true, false);
        } else {
            if (control) GSB_TAN_LAUNCH(false, true); else GSB_TAN_LAUNCH(false, false);
        }
#undef GSB_TAN_LAUNCH
        GSB_LAUNCH_CHECK("k_tangent_step");
        if ((st = call_prof_end(s, 1)) != GSB_OK) return st;
        cur ^= 1;
        if ((m + 1) % renorm_every == 0 || m + 1 == nsteps)
            if ((st = renorm(cur, 1)) != GSB_OK) return st;
    }
    std::vector<double> ls(R);
    GSB_CUDA_TRY(cudaMemcpyAsync(ls.data(), B.log_sum, R * sizeof(double), cudaMemcpyDeviceToHost, s));
    GSB_CUDA_TRY(cudaStreamSynchronize(s));
    if ((st = call_prof_collect()) != GSB_OK) return st;
    const double T = (double)nsteps * (double)(float)dt;
    for (int r = 0; r < R; ++r) mle_out[r] = ls[r] / T;
    return GSB_OK;
}
