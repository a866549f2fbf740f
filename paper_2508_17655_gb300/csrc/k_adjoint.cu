// k_adjoint.cu -- gradient of the relaxed energy E = -1/2 x(t_W)^T J x(t_W)
// after W steps (not in the paper) with respect to x(0), the control strength A
// and the time step dt, by a hand-written reverse sweep with checkpointed
// recomputation (gsb_relaxed_energy_grad).
//
// Forward: W steps of Sec. II (FP32 SGEMM coupling, the same update as the
// plain form), a checkpoint of (x, y, p) every K steps. Backward, segment by
// segment from the last: recompute the segment from its checkpoint, keeping
// every state and the momentum before the wall test, then undo its steps in
// reverse. One reverse step, for lx, ly, lp the adjoints of the step's outputs:
//   wall: clamped components: lx~ = ly~ = 0; else lx~ = lx, ly~ = ly
//   FY  (x~ = x + y~ dt):          ly~ += lx~ dt,   gdt += lx~ y~
//   FX  (y~ = y - (p' x - c f) dt): ly = ly~, lp' = lp - ly~ x dt,
//                                   lx = lx~ - ly~ p' dt, lf = ly~ c dt,
//                                   gdt -= ly~ (p' x - c f) = ly~ (y~ - y) / dt
//   JX  (f = J x, J symmetric):     lx += J lf  (no term for the sgn coupling)
//   FP  (p' = p - g p / (M - m), g = 1 - A x^2):
//                                   lp = lp' (1 - g / (M - m)), lg = -lp' p / (M - m),
//                                   gA -= lg x^2, lx -= 2 A x lg
// Each reverse step is an elementwise pass writing lf, then an SGEMM J lf whose
// epilogue finishes the step and reduces gA, gdt per replica. Under
// GSB_PREC_BF16X3 every product J v is taken as K-split partial sums from the
// tensor cores (split bf16, k_gemm_tc.cu), which the same step kernels add in
// their fixed order.
#include <vector>

#include "sgemm_f32.cuh"

namespace gsb {

namespace {

using namespace f32;

// MODE selects how a kernel gets its SGEMM: 128 or 64 -- a fused T x T tile;
// kSplitK -- the products' K split kSplitK ways (by k_adj_gemm_part on CUDA
// cores or k_gemm_tc on the tensor cores; more CTAs when few replicas leave
// SMs idle), the step kernel adding the partial sums in a fixed order
// (deterministic: a recomputed step is bit-identical) over 32 x 32 tiles,
// four times as many blocks as 64 x 64 ones (the kernel only streams memory).
constexpr int kSplitK = 4;
template <int MODE>
struct Mode {
    static constexpr int T = MODE == 128 ? 128 : (MODE == 64 ? 64 : 32);
    static constexpr bool split = MODE == kSplitK;
};

// F_s = J[:, K_s] X[K_s, :] for the K slice s = blockIdx.z of kSplitK, 64 x 64
// tiles, into Fp[s] ([Np][Rp] each).
template <bool SIGN>
__global__ void __launch_bounds__(256) k_adj_gemm_part(const float* __restrict__ J,
                                                       const float* __restrict__ X, int Np, int Rp,
                                                       float* __restrict__ Fp) {
    __shared__ __align__(16) Smem64 sm;
    const int i0 = blockIdx.y * 64, r0 = blockIdx.x * 64, sl = blockIdx.z;
    const int klen = Np / kSplitK;
    float acc[4][4];
    sgemm_tile64<SIGN>(J, X, Np, Rp, i0, r0, acc, sm, sl * klen, klen);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float* F = Fp + (size_t)sl * Np * Rp;
#pragma unroll
    for (int a = 0; a < 4; ++a)
        *reinterpret_cast<float4*>(F + (size_t)(i0 + ty * 4 + a) * Rp + r0 + tx * 4) =
            make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
}

// acc = the tile's SGEMM, fused or from the split-K partials.
template <int MODE, bool SIGN>
__device__ __forceinline__ void adj_gemm(const float* J, const float* X, int Np, int Rp, int i0,
                                         int r0, const float* Fp,
                                         float (&acc)[Tile<Mode<MODE>::T>::NA][Tile<Mode<MODE>::T>::NB],
                                         typename Tile<Mode<MODE>::T>::Smem& sm) {
    using TT = Tile<Mode<MODE>::T>;
    if constexpr (!Mode<MODE>::split) {
        TT::template gemm<SIGN>(J, X, Np, Rp, i0, r0, acc, sm);
    } else {
        static_assert(TT::NB == 2, "the split mode's tile holds two replicas a thread");
        const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
        const size_t nst = (size_t)Np * Rp;
#pragma unroll
        for (int a = 0; a < TT::NA; ++a) {
            const size_t o = (size_t)(i0 + TT::row(a, ty)) * Rp + r0 + TT::col(0, tx);
            float2 v = *reinterpret_cast<const float2*>(Fp + o);
#pragma unroll
            for (int sl = 1; sl < kSplitK; ++sl) {
                const float2 w = *reinterpret_cast<const float2*>(Fp + sl * nst + o);
                v.x += w.x, v.y += w.y;
            }
            acc[a][0] = v.x, acc[a][1] = v.y;
        }
    }
}

// One forward step that also records y~ (the momentum before the wall test).
template <bool SIGN, bool CONTROL, int MODE>
__global__ void __launch_bounds__(256) k_adj_fwd(const float* __restrict__ J, int Np, int Rp,
                                                 const float* __restrict__ x, const float* __restrict__ y,
                                                 const float* __restrict__ p, float* __restrict__ xn,
                                                 float* __restrict__ yn, float* __restrict__ pn,
                                                 float* __restrict__ yt_out,
                                                 const float* __restrict__ A, float c, float dt,
                                                 float p_shared, float inv_rem,
                                                 const float* __restrict__ Fp) {
    constexpr int T = Mode<MODE>::T;
    using TT = Tile<T>;
    __shared__ __align__(16) typename TT::Smem sm;
    const int i0 = blockIdx.y * T, r0 = blockIdx.x * T;
    float acc[TT::NA][TT::NB];
    adj_gemm<MODE, SIGN>(J, x, Np, Rp, i0, r0, Fp, acc, sm);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int a = 0; a < TT::NA; ++a) {
        const size_t rowoff = (size_t)(i0 + TT::row(a, ty)) * Rp;
#pragma unroll
        for (int b = 0; b < TT::NB; ++b) {
            const int col = r0 + TT::col(b, tx);
            const size_t o = rowoff + col;
            const float xo = x[o];
            float pv = CONTROL ? p[o] : 0.f;
            const float g = 1.f - (CONTROL ? A[col] : 0.f) * xo * xo;
            const float pnv = CONTROL ? pv - g * pv * inv_rem : p_shared;
            const float ytv = y[o] - (pnv * xo - c * acc[a][b]) * dt;
            float xt = xo + ytv * dt, yv = ytv;
            if (fabsf(xt) > 1.f) {
                xt = sgnf(xt);
                yv = 0.f;
            }
            xn[o] = xt;
            yn[o] = yv;
            if (CONTROL) pn[o] = pnv;
            yt_out[o] = ytv;
        }
    }
}

// Seed: G = J x(t_W); lx = -G, ly = lp = 0, e_acc[b][r] += sum_i x_i G_i over the
// rows of block row b. Per-replica sums are kept per block row (one writer a
// slot) and added in order by k_finish, so every run gives the same bits.
template <int MODE>
__global__ void __launch_bounds__(256) k_adj_seed(const float* __restrict__ J, int Np, int Rp,
                                                  const float* __restrict__ x, float* __restrict__ lx,
                                                  float* __restrict__ ly, float* __restrict__ lp,
                                                  double* __restrict__ e_acc,
                                                  const float* __restrict__ Fp) {
    constexpr int T = Mode<MODE>::T;
    using TT = Tile<T>;
    __shared__ __align__(16) typename TT::Smem sm;
    __shared__ float red[16][T + 1];
    const int i0 = blockIdx.y * T, r0 = blockIdx.x * T;
    float acc[TT::NA][TT::NB];
    adj_gemm<MODE, false>(J, x, Np, Rp, i0, r0, Fp, acc, sm);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int b = 0; b < TT::NB; ++b) {
        const int col = TT::col(b, tx);
        float part = 0.f;
#pragma unroll
        for (int a = 0; a < TT::NA; ++a) {
            const size_t o = (size_t)(i0 + TT::row(a, ty)) * Rp + r0 + col;
            part = fmaf(x[o], acc[a][b], part);
            lx[o] = -acc[a][b];
            ly[o] = 0.f;
            if (lp) lp[o] = 0.f;
        }
        red[ty][col] = part;
    }
    __syncthreads();
    if (threadIdx.x < T) {
        double s = 0.0;
        for (int t = 0; t < 16; ++t) s += (double)red[t][threadIdx.x];
        e_acc[(size_t)blockIdx.y * Rp + r0 + threadIdx.x] += s;
    }
}

// Elementwise first half of a reverse step: lf = ly~ c dt (ly~ after FY).
__global__ void k_adj_pre(const float* __restrict__ x, const float* __restrict__ yt,
                          const float* __restrict__ lx, const float* __restrict__ ly,
                          float* __restrict__ lf, size_t n, float c, float dt) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float ytv = yt[k];
    const bool clamped = fabsf(x[k] + ytv * dt) > 1.f;
    const float lxt = clamped ? 0.f : lx[k];
    const float lyt = (clamped ? 0.f : ly[k]) + lxt * dt;
    lf[k] = lyt * c * dt;
}

// Second half: G = J lf (skipped for the sgn coupling), then every adjoint of
// the step's inputs and the per-replica gA, gdt sums.
template <bool SIGN, bool CONTROL, int MODE>
__global__ void __launch_bounds__(256) k_adj_post(const float* __restrict__ J, int Np, int Rp,
                                                  const float* __restrict__ lf,
                                                  const float* __restrict__ x,
                                                  const float* __restrict__ y,
                                                  const float* __restrict__ p,
                                                  const float* __restrict__ pnext,
                                                  const float* __restrict__ yt,
                                                  float* __restrict__ lx, float* __restrict__ ly,
                                                  float* __restrict__ lp,
                                                  const float* __restrict__ A, float c, float dt,
                                                  float p_shared, float inv_rem,
                                                  double* __restrict__ gA,
                                                  double* __restrict__ gdt,
                                                  const float* __restrict__ Fp) {
    constexpr int T = Mode<MODE>::T;
    using TT = Tile<T>;
    __shared__ __align__(16) typename TT::Smem sm;
    __shared__ float redA[16][T + 1], redT[16][T + 1];
    const int i0 = blockIdx.y * T, r0 = blockIdx.x * T;
    float acc[TT::NA][TT::NB];
    if (!SIGN) {
        adj_gemm<MODE, false>(J, lf, Np, Rp, i0, r0, Fp, acc, sm);
    } else {
#pragma unroll
        for (int a = 0; a < TT::NA; ++a)
#pragma unroll
            for (int b = 0; b < TT::NB; ++b) acc[a][b] = 0.f;
    }
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int b = 0; b < TT::NB; ++b) {
        const int col = TT::col(b, tx);
        const float a_r = CONTROL ? A[r0 + col] : 0.f;
        float sA = 0.f, sT = 0.f;
#pragma unroll
        for (int a = 0; a < TT::NA; ++a) {
            const size_t o = (size_t)(i0 + TT::row(a, ty)) * Rp + r0 + col;
            const float xo = x[o], ytv = yt[o];
            const bool clamped = fabsf(xo + ytv * dt) > 1.f;
            const float lxt = clamped ? 0.f : lx[o];
            const float lyt = (clamped ? 0.f : ly[o]) + lxt * dt;
            const float pnv = CONTROL ? pnext[o] : p_shared;
            sT = fmaf(lxt, ytv, sT);
            sT = fmaf(lyt, (ytv - y[o]) / dt, sT);
            float lxi = lxt - lyt * pnv * dt + acc[a][b];
            if (CONTROL) {
                const float lpn = lp[o] - lyt * xo * dt;
                const float pv = p[o];
                const float g = 1.f - a_r * xo * xo;
                const float lg = -lpn * pv * inv_rem;
                sA = fmaf(-lg, xo * xo, sA);
                lxi = fmaf(-2.f * a_r * xo, lg, lxi);
                lp[o] = lpn * (1.f - g * inv_rem);
            }
            lx[o] = lxi;
            ly[o] = lyt;
        }
        redA[ty][col] = sA;
        redT[ty][col] = sT;
    }
    __syncthreads();
    if (threadIdx.x < T) {
        double a = 0.0, t = 0.0;
        for (int k = 0; k < 16; ++k) {
            a += (double)redA[k][threadIdx.x];
            t += (double)redT[k][threadIdx.x];
        }
        // one slot per block row and replica, each written by one block a step
        // (stream order between steps): no atomics, a fixed order of additions
        const size_t slot = (size_t)blockIdx.y * Rp + r0 + threadIdx.x;
        if (CONTROL) gA[slot] += a;
        gdt[slot] += t;
    }
}

// caller layout [R][N] <-> state layout [Np][Rp]
__global__ void k_rm_to_sm(const float* __restrict__ src, float* __restrict__ dst, int N, int R,
                           int Rp) {
    __shared__ float tile[32][33];
    const int i0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, i = i0 + threadIdx.x;
        tile[k][threadIdx.x] = (r < R && i < N) ? src[(size_t)r * N + i] : 0.f;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y)
        dst[(size_t)(i0 + k) * Rp + r0 + threadIdx.x] = tile[threadIdx.x][k];
}

__global__ void k_fill(float* p, float v, size_t n) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) p[k] = v;
}

// The per-block-row sums added in block-row order.
__global__ void k_finish(const double* e_acc, double* E, const double* gA, double* gA_out,
                         const double* gdt, double* gdt_out, int R, int Rp, int nby) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    double e = 0.0, a = 0.0, t = 0.0;
    for (int b = 0; b < nby; ++b) {
        const size_t o = (size_t)b * Rp + r;
        e += e_acc[o];
        a += gA[o];
        t += gdt[o];
    }
    E[r] = -0.5 * e;
    if (gA_out) gA_out[r] = a;
    if (gdt_out) gdt_out[r] = t;
}

struct SplitGemmGuard {
    SplitGemm* g = nullptr;
    ~SplitGemmGuard() { split_gemm_destroy(g); }
};

struct DevBuf {
    std::vector<void*> ptrs;
    ~DevBuf() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <typename T>
    gsb_status alloc(T** p, size_t n) {
        *p = nullptr;
        cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (n ? n : 1));
        if (e != cudaSuccess) return cuda_error(e, "cudaMalloc (adjoint)");
        ptrs.push_back(*p);
        return GSB_OK;
    }
};

}  // namespace

}  // namespace gsb

using namespace gsb;

extern "C" gsb_status gsb_relaxed_energy_grad(gsb_problem* P, const gsb_params* prm,
                                              int32_t window, int32_t ckpt_every,
                                              const float* x0, double* energy, float* grad_x0,
                                              double* grad_A, double* grad_dt, void* stream) {
    if (!P || !prm || !x0 || !energy) return set_error(GSB_EINVAL, "NULL argument");
    const gsb_params& Q = *prm;
    if (P->csr) return set_error(GSB_EUNSUPPORTED, "gsb_relaxed_energy_grad takes dense problems");
    if (P->has_h) return set_error(GSB_EUNSUPPORTED, "gsb_relaxed_energy_grad takes problems without h");
    if (Q.variant < GSB_BSB || Q.variant > GSB_GDSB) return set_error(GSB_EINVAL, "unknown variant");
    if (Q.M < 1 || Q.R < 1) return set_error(GSB_EINVAL, "M and R must be >= 1");
    if (window < 1 || window > Q.M) return set_error(GSB_EINVAL, "window must be in 1..M");
    if (ckpt_every < 1) return set_error(GSB_EINVAL, "ckpt_every must be >= 1");
    if (!(Q.c > 0.0) || !(Q.dt > 0.0)) return set_error(GSB_EINVAL, "c and dt must be > 0");
    if (Q.schedule) return set_error(GSB_EUNSUPPORTED, "the Eq. 6 schedule only");
    if (Q.precision != GSB_PREC_AUTO && Q.precision != GSB_PREC_FP32 &&
        Q.precision != GSB_PREC_BF16X3)
        return set_error(GSB_EUNSUPPORTED, "gsb_relaxed_energy_grad takes FP32 or BF16X3 coupling");
    cudaStream_t s = (cudaStream_t)stream;
    const bool sign = Q.variant == GSB_DSB || Q.variant == GSB_GDSB;
    const bool control = Q.variant == GSB_GBSB || Q.variant == GSB_GDSB;
    const int N = P->N, Np = P->Np, R = Q.R, Rp = round_up(R, kTile);
    const int K = ckpt_every < window ? ckpt_every : window;
    const int nseg = (window + K - 1) / K;
    const size_t nst = (size_t)Np * Rp;
    const float c = (float)Q.c, dt = (float)Q.dt;
    DevBuf B;
    float *ck = nullptr, *sx = nullptr, *sy = nullptr, *sp = nullptr, *syt = nullptr;
    float *lx = nullptr, *ly = nullptr, *lp = nullptr, *lf = nullptr, *Ad = nullptr, *tmp = nullptr;
    double *e_acc = nullptr, *gA = nullptr, *gdt = nullptr;
    gsb_status st;
    // checkpoints: (x, y, p) at the start of each segment
    if ((st = B.alloc(&ck, 3 * nst * nseg)) || (st = B.alloc(&sx, nst * (K + 1))) ||
        (st = B.alloc(&sy, nst * (K + 1))) || (st = B.alloc(&sp, nst * (K + 1))) ||
        (st = B.alloc(&syt, nst * K)) || (st = B.alloc(&lx, nst)) || (st = B.alloc(&ly, nst)) ||
        (st = B.alloc(&lp, nst)) || (st = B.alloc(&lf, nst)) || (st = B.alloc(&Ad, Rp)) ||
        (st = B.alloc(&tmp, nst)) || (st = B.alloc(&e_acc, (size_t)Np / 32 * Rp)) ||
        (st = B.alloc(&gA, (size_t)Np / 32 * Rp)) || (st = B.alloc(&gdt, (size_t)Np / 32 * Rp)))
        return st;
    {
        std::vector<float> Ah(Rp, 0.f);
        for (int r = 0; r < R; ++r) Ah[r] = Q.A_per_replica ? Q.A_per_replica[r] : Q.A;
        GSB_CUDA_TRY(cudaMemcpyAsync(Ad, Ah.data(), sizeof(float) * Rp, cudaMemcpyHostToDevice, s));
        GSB_CUDA_TRY(cudaStreamSynchronize(s));
    }
    call_prof_reset();
    // per-block-row sums: at most Np / 32 block rows (32-row tiles)
    GSB_CUDA_TRY(cudaMemsetAsync(e_acc, 0, sizeof(double) * Rp * (Np / 32), s));
    GSB_CUDA_TRY(cudaMemsetAsync(gA, 0, sizeof(double) * Rp * (Np / 32), s));
    GSB_CUDA_TRY(cudaMemsetAsync(gdt, 0, sizeof(double) * Rp * (Np / 32), s));
    // initial state into segment slot 0
    k_rm_to_sm<<<dim3(Np / 32, Rp / 32), dim3(32, 8), 0, s>>>(x0, sx, N, R, Rp);
    GSB_LAUNCH_CHECK("k_rm_to_sm");
    GSB_CUDA_TRY(cudaMemsetAsync(sy, 0, sizeof(float) * nst, s));
    k_fill<<<(unsigned)((nst + 255) / 256), 256, 0, s>>>(sp, 1.f, nst);
    GSB_LAUNCH_CHECK("k_fill");
    // 64 x 64 tiles when 128 x 128 ones would leave SMs idle (few replicas),
    // and K split kSplitK ways when even those give fewer than two CTAs per SM
    int sms = 0, dev = 0;
    GSB_CUDA_TRY(cudaGetDevice(&dev));
    GSB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long tiles64 = (long)(Rp / 64) * (Np / 64);
    // the split-bf16 form takes its partial products from the tensor cores
    const bool tensor = Q.precision == GSB_PREC_BF16X3;
    const int mode = tensor ? kSplitK
                            : (long)(Rp / 128) * (Np / 128) >= sms ? 128
                                                                   : (tiles64 >= 2L * sms ? 64 : kSplitK);
    const int T = mode == 128 ? 128 : (mode == 64 ? 64 : 32);
    const dim3 grid(Rp / T, Np / T);
    float* Fp = nullptr;  // split-K partial sums
    if (mode == kSplitK && (st = B.alloc(&Fp, kSplitK * nst))) return st;
    SplitGemmGuard tg;
    if (tensor && (st = split_gemm_create(P, Rp, &tg.g, s))) return st;
    // the partial sums of J X for a kernel in the split mode
    auto gemm_part = [&](const float* X, bool sgn) -> gsb_status {
        if (tensor) return split_gemm_partials(tg.g, X, sgn, kSplitK, Fp, s);
        const dim3 g(Rp / 64, Np / 64, kSplitK);
        if (sgn)
            k_adj_gemm_part<true><<<g, 256, 0, s>>>(P->J32, X, Np, Rp, Fp);
        else
            k_adj_gemm_part<false><<<g, 256, 0, s>>>(P->J32, X, Np, Rp, Fp);
        GSB_LAUNCH_CHECK("k_adj_gemm_part");
        return GSB_OK;
    };
    auto fwd = [&](int m, int slot) -> gsb_status {
        const size_t a = (size_t)slot * nst, b = (size_t)(slot + 1) * nst;
        const float p_shared = (float)(1.0 - (double)(m + 1) / (double)Q.M);
        const float inv_rem = 1.0f / (float)(Q.M - m);
        gsb_status pst = call_prof_begin(s);
        if (pst != GSB_OK) return pst;
        if (mode == kSplitK) {
            gsb_status g = gemm_part(sx + a, sign);
            if (g != GSB_OK) return g;
        }
#define GSB_ADJ_FWD(S, C, MD)                                                                     \
    k_adj_fwd<S, C, MD><<<grid, 256, 0, s>>>(P->J32, Np, Rp, sx + a, sy + a, sp + a, sx + b,     \
                                             sy + b, sp + b, syt + a, Ad, c, dt, p_shared, inv_rem, \
                                             Fp)
#define GSB_ADJ_FWD_T(S, C)                                               \
    if (mode == 128) GSB_ADJ_FWD(S, C, 128);                              \
    else if (mode == 64) GSB_ADJ_FWD(S, C, 64);                           \
    else GSB_ADJ_FWD(S, C, kSplitK)
        if (sign) {
            if (control) { GSB_ADJ_FWD_T(true, true); } else { GSB_ADJ_FWD_T(true, false); }
        } else {
            if (control) { GSB_ADJ_FWD_T(false, true); } else { GSB_ADJ_FWD_T(false, false); }
        }
#undef GSB_ADJ_FWD_T
#undef GSB_ADJ_FWD
        GSB_LAUNCH_CHECK("k_adj_fwd");
        return call_prof_end(s, 1);
    };
    auto save_ckpt = [&](int seg) -> gsb_status {
        for (int q = 0; q < 3; ++q) {
            const float* src = q == 0 ? sx : (q == 1 ? sy : sp);
            GSB_CUDA_TRY(cudaMemcpyAsync(ck + ((size_t)seg * 3 + q) * nst, src, sizeof(float) * nst,
                                         cudaMemcpyDeviceToDevice, s));
        }
        return GSB_OK;
    };
    auto load_ckpt = [&](int seg) -> gsb_status {
        for (int q = 0; q < 3; ++q) {
            float* dst = q == 0 ? sx : (q == 1 ? sy : sp);
            GSB_CUDA_TRY(cudaMemcpyAsync(dst, ck + ((size_t)seg * 3 + q) * nst, sizeof(float) * nst,
                                         cudaMemcpyDeviceToDevice, s));
        }
        return GSB_OK;
    };
    auto seg_len = [&](int seg) { return seg == nseg - 1 ? window - seg * K : K; };
    // forward pass with checkpoints
    for (int seg = 0; seg < nseg; ++seg) {
        if ((st = save_ckpt(seg))) return st;
        const int L = seg_len(seg);
        for (int k = 0; k < L; ++k)
            if ((st = fwd(seg * K + k, k))) return st;
        if (seg < nseg - 1) {
            // the next segment starts from slot L
            for (int q = 0; q < 3; ++q) {
                float* buf = q == 0 ? sx : (q == 1 ? sy : sp);
                GSB_CUDA_TRY(cudaMemcpyAsync(buf, buf + (size_t)L * nst, sizeof(float) * nst,
                                             cudaMemcpyDeviceToDevice, s));
            }
        }
    }
    // seed from x(t_W) (slot of the last segment's end)
    const int Llast = seg_len(nseg - 1);
    if ((st = call_prof_begin(s))) return st;
    {
        const float* xW = sx + (size_t)Llast * nst;
        if (mode == kSplitK && (st = gemm_part(xW, false))) return st;
        if (mode == 128)
            k_adj_seed<128><<<grid, 256, 0, s>>>(P->J32, Np, Rp, xW, lx, ly, control ? lp : nullptr,
                                                 e_acc, Fp);
        else if (mode == 64)
            k_adj_seed<64><<<grid, 256, 0, s>>>(P->J32, Np, Rp, xW, lx, ly, control ? lp : nullptr,
                                                e_acc, Fp);
        else
            k_adj_seed<kSplitK><<<grid, 256, 0, s>>>(P->J32, Np, Rp, xW, lx, ly,
                                                     control ? lp : nullptr, e_acc, Fp);
    }
    GSB_LAUNCH_CHECK("k_adj_seed");
    if ((st = call_prof_end(s, 1))) return st;
    // reverse sweep, segment by segment; the last segment is still in the slots
    for (int seg = nseg - 1; seg >= 0; --seg) {
        const int L = seg_len(seg);
        if (seg < nseg - 1) {
            if ((st = load_ckpt(seg))) return st;
            for (int k = 0; k < L; ++k)
                if ((st = fwd(seg * K + k, k))) return st;
        }
        for (int k = L - 1; k >= 0; --k) {
            const int m = seg * K + k;
            const size_t a = (size_t)k * nst, b = (size_t)(k + 1) * nst;
            const float p_shared = (float)(1.0 - (double)(m + 1) / (double)Q.M);
            const float inv_rem = 1.0f / (float)(Q.M - m);
            if ((st = call_prof_begin(s))) return st;
            if (!sign) {
                k_adj_pre<<<(unsigned)((nst + 255) / 256), 256, 0, s>>>(sx + a, syt + a, lx, ly, lf,
                                                                         nst, c, dt);
                GSB_LAUNCH_CHECK("k_adj_pre");
            }
            if (mode == kSplitK && !sign && (st = gemm_part(lf, false))) return st;
#define GSB_ADJ_POST(S, C, MD)                                                                  \
    k_adj_post<S, C, MD><<<grid, 256, 0, s>>>(P->J32, Np, Rp, lf, sx + a, sy + a, sp + a, sp + b, \
                                              syt + a, lx, ly, lp, Ad, c, dt, p_shared, inv_rem,  \
                                              gA, gdt, Fp)
#define GSB_ADJ_POST_T(S, C)                                              \
    if (mode == 128) GSB_ADJ_POST(S, C, 128);                             \
    else if (mode == 64) GSB_ADJ_POST(S, C, 64);                          \
    else GSB_ADJ_POST(S, C, kSplitK)
            if (sign) {
                if (control) { GSB_ADJ_POST_T(true, true); } else { GSB_ADJ_POST_T(true, false); }
            } else {
                if (control) { GSB_ADJ_POST_T(false, true); } else { GSB_ADJ_POST_T(false, false); }
            }
#undef GSB_ADJ_POST_T
#undef GSB_ADJ_POST
            GSB_LAUNCH_CHECK("k_adj_post");
            if ((st = call_prof_end(s, 1))) return st;
        }
    }
    k_finish<<<(R + 255) / 256, 256, 0, s>>>(e_acc, energy, gA, grad_A, gdt, grad_dt, R, Rp,
                                             (int)grid.y);
    GSB_LAUNCH_CHECK("k_finish");
    if (grad_x0) {
        st = launch_transpose_to_host_layout(lx, grad_x0, Np, Rp, N, R, s);
        if (st != GSB_OK) return st;
    }
    GSB_CUDA_TRY(cudaStreamSynchronize(s));  // buffers are freed on return
    if (tensor && (st = split_gemm_status(tg.g, s))) return st;
    return call_prof_collect();
}
