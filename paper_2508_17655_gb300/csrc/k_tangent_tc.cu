// k_tangent_tc.cu -- the tangent-linear steps of gsb_lyapunov with J x and
// J dx on the tensor cores, in the split-bf16 form (GSB_PREC_BF16X3).
//
// The step is k_tangent_step's (the linearisation of Eqs. 3-7 in
// sb_tangent_update); only the two products differ. With J = J_hi + J_lo and
// v = v_hi + v_lo split into bf16 terms (each the rounding of what the terms
// before it leave), F = J x is accumulated in FP32 in TMEM as
// J_hi x_hi + J_hi x_lo + J_lo x_hi (three tcgen05 kind::f16 MMAs per K
// slice) and G = J dx alike; the sgn coupling takes J_hi s + J_lo s for F (s
// is exact in bf16) and has no J dx term. The error against FP64 is at most
// about 3 2^-16 of each product's magnitude sum_j |J_ij v_j| (the splits'
// residues and the J_lo v_lo term left out) plus the FP32 accumulation.
//
// One launch per time step. The tiles of a step (128 spins x 128 replicas)
// do not wait on one another -- each reads the step's operand planes and
// writes only its own state and its part of the next step's planes -- so CTA
// b of G takes tiles b, b + G, ..., and two accumulators in TMEM let one
// tile's MMAs run while the previous tile's epilogue reads the other.
//
// The MMAs take J as the A operand (M = 128 spins: TMEM lane = spin) and the
// planes as B with x and dx side by side (N = 256: the tile's 128 replicas,
// then their 128 tangents), so one MMA serves both products:
//   D = J_hi [x_hi | dx_hi] + J_lo [x_hi | dx_hi] + J_hi [x_lo | dx_lo],
// F = D[:, 0:128], G = D[:, 128:256]. Three MMAs per 16 K elements, each
// reading 12 KB of shared memory for 128 x 256 x 16 -- a third less operand
// traffic than six 128 x 128 MMAs; shared-memory bandwidth (128 bytes a
// cycle per SM) is what bounds this loop. The sgn coupling: D = J_hi s +
// J_lo s, N = 128.
//
// Layout: state x, y, p, dx, dy, dp in FP32, replica-major [Rp][Np] (a warp's
// 32 spins of one replica are 128 contiguous bytes); operand planes bf16,
// replica-major [planes][Rp][Np] -- x_hi, x_lo, dx_hi, dx_lo, or sgn x alone
// for the sgn coupling -- double-buffered by the parity of the step.
// TMEM (512 columns): accumulator b at 256 b (F at +0, G at +128).
// Shared memory: 2 stages x (J_hi, J_lo, x_hi, dx_hi, x_lo, dx_lo atoms; J_hi,
// J_lo, s for the sgn coupling), each atom 64 K elements x 128 rows, 128-byte
// swizzled; x_hi, dx_hi (and x_lo, dx_lo) are adjacent, one 256-row operand.
// Warps: 0 TMA producer, 1 TMEM owner + MMA issuer, 2-9 epilogue (warp w
// reads TMEM lanes 32 (w % 4).. -- its 32 spins -- and columns
// 64 ((w - 2) / 4) .. +63 of F and of G -- 64 replicas of the tile).
#include <cudaTypedefs.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "gsb_update.cuh"
#include "philox.cuh"
#include "tc_ptx.cuh"

namespace gsb {

namespace {

using namespace tc;

constexpr int kT = 128;          // spins and replicas per tile
constexpr int kKB = 128;         // bytes of K per atom
constexpr int kElems = kKB / 2;  // bf16 elements of K per atom
constexpr int kAtom = kT * kKB;  // one 128-row atom (16 KB)
constexpr int kThreads = 320;
constexpr int kEpiThreads = 256;
constexpr int kStages = 2;
constexpr int kStageBytes = 6 * kAtom;
constexpr int kSmem = 1024 + kStages * kStageBytes + 256;

struct TanArgs {
    CUtensorMap tmJ[2];  // J_hi, J_lo: [Np][Np]
    CUtensorMap tmV[2];  // operand planes of even / odd steps: [planes x Rp][Np]
    float* x;
    float* y;
    float* p;
    float* dx;
    float* dy;
    float* dp;
    const float* A;      // control strength per replica [Rp]
    __nv_bfloat16* v[2];
    int* status;
    int Np, Rp;
    int m;               // the step taken, t_m -> t_{m+1}
    float c, dt, p_shared, inv_rem;
};

template <bool SIGN, bool CONTROL>
__global__ void __launch_bounds__(kThreads, 1) k_tangent_tc(const __grid_constant__ TanArgs P) {
    constexpr int S = kStages;
    constexpr int NPLANE = SIGN ? 1 : 4;
    constexpr uint32_t kStageTx = (uint32_t)(2 + NPLANE) * kAtom;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + S * kStageBytes);
    uint64_t* empty = full + S;
    uint64_t* accf = empty + S;  // [2]
    uint64_t* acce = accf + 2;   // [2]
    uint64_t* drain = acce + 2;
    uint32_t* tmem_slot = (uint32_t*)(drain + 1);
    // stage st: J_hi, J_lo, then the planes
    auto atom = [&](uint32_t st, int q) { return smem + st * kStageBytes + q * kAtom; };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // tile j: replica block j / nsb, spin block j % nsb -- the CTAs at work at
    // once share few replica blocks, so each block's planes are read from L2
    // by all its spin blocks while they are hot
    const int nsb = P.Np / kT, nk = P.Np / kElems;
    const int ntiles = nsb * (P.Rp / kT);
    // debug build: whole tiles on both axes (parameters alone: a uniform
    // return before any barrier)
    if (!GSB_DOK(P.Np % kT == 0 && P.Rp % kT == 0 && P.Np > 0 && P.Rp > 0, P.status)) return;

    if (threadIdx.x == 0) {
        for (int st = 0; st < S; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 1);
        }
        mbar_init(drain, 1);
        tmem_slot[1] = 0u;  // epilogue abort flag
        fence_barrier_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, 512);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            const CUtensorMap* tv = &P.tmV[P.m & 1];
            uint32_t g = 0;
            bool ok = true;
            for (int j = blockIdx.x; j < ntiles && ok; j += gridDim.x) {
                const int i0 = (j % nsb) * kT, r0 = (j / nsb) * kT;
                for (int u = 0; u < nk; ++u, ++g) {
                    const uint32_t st = g % S, ph = (g / S) & 1u;
                    if (g >= (uint32_t)S && !mbar_wait(&empty[st], ph ^ 1u, P.status)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[st], kStageTx);
                    tma_load_2d(atom(st, 0), &P.tmJ[0], &full[st], u * kElems, i0);
                    tma_load_2d(atom(st, 1), &P.tmJ[1], &full[st], u * kElems, i0);
                    // atoms 2.. hold the planes x_hi, dx_hi, x_lo, dx_lo (stored as
                    // x_hi, x_lo, dx_hi, dx_lo), so that each hi and each lo pair
                    // is one 256-row B operand
#pragma unroll
                    for (int q = 0; q < NPLANE; ++q)
                        tma_load_2d(atom(st, 2 + q), tv, &full[st], u * kElems,
                                    ((q >> 1) | ((q & 1) << 1)) * P.Rp + r0);
                }
            }
            // no copy is in flight when the CTA leaves
            for (uint32_t gg = g > (uint32_t)S ? g - S : 0u; gg < g; ++gg)
                mbar_wait(&full[gg % S], (gg / S) & 1u, P.status, kDrainLimitCycles);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_make(1u, kT, SIGN ? kT : 2 * kT);
            uint32_t g = 0, n = 0;
            bool ok = true;
            for (int j = blockIdx.x; j < ntiles && ok; j += gridDim.x, ++n) {
                const uint32_t b = n & 1u;
                // the epilogue has read this accumulator's previous tile
                if (n >= 2 && !mbar_wait(&acce[b], ((n - 2) >> 1) & 1u, P.status)) break;
                fence_after_sync();
                const uint32_t d = tmem + 256u * b;
                for (int u = 0; u < nk; ++u, ++g) {
                    const uint32_t st = g % S, ph = (g / S) & 1u;
                    if (!mbar_wait(&full[st], ph, P.status)) {
                        ok = false;
                        break;
                    }
                    fence_after_sync();
                    const uint32_t jh = smem_u32(atom(st, 0)), jl = smem_u32(atom(st, 1));
                    const uint32_t vh = smem_u32(atom(st, 2)), vl = smem_u32(atom(st, 4));
#pragma unroll
                    for (int k = 0; k < kKB / 32; ++k) {  // 16 bf16 of K per MMA
                        const uint32_t acc = (u | k) != 0;
                        const uint64_t ah = sdesc_sw128(jh + k * 32), al = sdesc_sw128(jl + k * 32);
                        const uint64_t bh = sdesc_sw128(vh + k * 32);
                        mma_f16(d, ah, bh, idesc, acc);
                        mma_f16(d, al, bh, idesc, 1u);
                        if (!SIGN) mma_f16(d, ah, sdesc_sw128(vl + k * 32), idesc, 1u);
                    }
                    mma_commit(&empty[st]);
                }
                if (!ok) break;
                mma_commit(&accf[b]);
            }
            // every MMA issued has finished before TMEM is released
            mma_commit(drain);
            mbar_wait(drain, 0, P.status, kDrainLimitCycles);
        }
    } else {
        const int ew = warp - 2;
        const int quarter = warp & 3;
        const int c0 = (ew >> 2) * 64;
        const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
        volatile uint32_t* abort_flag = tmem_slot + 1;
        const int Np = P.Np;
        const size_t plane = (size_t)P.Rp * Np;
        const float c = P.c, dt = P.dt, p_shared = P.p_shared, inv_rem = P.inv_rem;
        float* __restrict__ x = P.x;
        float* __restrict__ y = P.y;
        float* __restrict__ p = P.p;
        float* __restrict__ dx = P.dx;
        float* __restrict__ dy = P.dy;
        float* __restrict__ dp = P.dp;
        uint16_t* __restrict__ vout = reinterpret_cast<uint16_t*>(P.v[(P.m + 1) & 1]);
        uint32_t n = 0;
        for (int j = blockIdx.x; j < ntiles; j += gridDim.x, ++n) {
            const int i0 = (j % nsb) * kT, r0 = (j / nsb) * kT;
            const uint32_t b = n & 1u;
            bool ok = *abort_flag == 0u;
            if (ok) ok = __all_sync(0xffffffffu, mbar_wait(&accf[b], (n >> 1) & 1u, P.status));
            if (!ok) {
                *abort_flag = 1u;
                named_barrier_sync(1, kEpiThreads);
                break;
            }
            fence_after_sync();
            const int i = i0 + quarter * 32 + lane;  // this thread's spin (TMEM lane)
            const uint32_t ta = tl + 256u * b;
            // chunks of 8 replicas in two register buffers taken in turn: while
            // one chunk is updated in place, the next one's state (six arrays,
            // from HBM) is in flight; the state is read and written with the
            // evict-first hint, so that it streams past the planes and J in L2
            constexpr int CW = 8;
            float qa[6][CW], qb[6][CW];
            auto load_state = [&](int cb, float (&q)[6][CW]) {
                const size_t o = (size_t)(r0 + cb) * Np + i;
#pragma unroll
                for (int k = 0; k < CW; ++k) {
                    const size_t e = o + (size_t)k * Np;
                    q[0][k] = __ldcs(x + e);
                    q[1][k] = __ldcs(y + e);
                    q[2][k] = CONTROL ? __ldcs(p + e) : 0.f;
                    q[3][k] = __ldcs(dx + e);
                    q[4][k] = __ldcs(dy + e);
                    q[5][k] = CONTROL ? __ldcs(dp + e) : 0.f;
                }
            };
            load_state(c0, qa);
            load_state(c0 + CW, qb);
            auto chunk = [&](int cb, float (&s)[6][CW]) {
                uint32_t rf[CW], rg[CW];
                tmem_ld8_async(ta + cb, rf);
                if (!SIGN) tmem_ld8_async(ta + 128u + cb, rg);
                float a_r[CW];
#pragma unroll
                for (int k = 0; k < CW; ++k) a_r[k] = CONTROL ? __ldg(P.A + r0 + cb + k) : 0.f;
                tmem_wait_ld8(rf);
                if (!SIGN) tmem_wait_ld8(rg);
#pragma unroll
                for (int k = 0; k < CW; ++k)
                    sb_tangent_update<CONTROL, SIGN>(s[0][k], s[1][k], s[2][k], s[3][k], s[4][k],
                                                     s[5][k], __uint_as_float(rf[k]),
                                                     SIGN ? 0.f : __uint_as_float(rg[k]), a_r[k], c,
                                                     dt, p_shared, inv_rem);
                const size_t o = (size_t)(r0 + cb) * Np + i;
#pragma unroll
                for (int k = 0; k < CW; ++k) {
                    const size_t e = o + (size_t)k * Np;
                    __stcs(x + e, s[0][k]);
                    __stcs(y + e, s[1][k]);
                    if (CONTROL) __stcs(p + e, s[2][k]);
                    __stcs(dx + e, s[3][k]);
                    __stcs(dy + e, s[4][k]);
                    if (CONTROL) __stcs(dp + e, s[5][k]);
                    // next step's operand planes (a warp writes 64 contiguous bytes of each)
                    if (SIGN) {
                        vout[e] = s[0][k] >= 0.f ? (uint16_t)0x3F80 : (uint16_t)0xBF80;
                    } else {
                        uint32_t h, l;
                        bf16_split_bits(s[0][k], h, l);
                        vout[e] = (uint16_t)h;
                        vout[plane + e] = (uint16_t)l;
                        bf16_split_bits(s[3][k], h, l);
                        vout[2 * plane + e] = (uint16_t)h;
                        vout[3 * plane + e] = (uint16_t)l;
                    }
                }
                if (cb + 2 * CW < c0 + 64) load_state(cb + 2 * CW, s);
            };
#pragma unroll 1
            for (int cb = c0; cb < c0 + 64; cb += 2 * CW) {
                chunk(cb, qa);
                chunk(cb + CW, qb);
            }
            // every epilogue thread has read its F and G before the accumulator
            // is handed back
            fence_before_sync();
            named_barrier_sync(1, kEpiThreads);
            if (*abort_flag) break;
            if (ew == 0 && lane == 0) mbar_arrive(&acce[b]);
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        fence_after_sync();
        tmem_dealloc(tmem, 512);
    }
}

// x(0), y(0), p(0) = 1 as gsb_run draws them for replica r, and the tangent's
// dx(0) uniform in [-1, 1) (Philox stream 4), dy = dp = 0; replica-major
// [Rp][Np], padded spins and replicas at zero (p = 1).
__global__ void k_tan_tc_init(float* x, float* y, float* p, float* dx, float* dy, float* dp, int N,
                              int R, int Np, uint2 key, float scale, int y_uniform) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (i >= Np) return;
    const size_t o = (size_t)r * Np + i;
    const bool real = i < N && r < R;
    x[o] = real ? uniform_draw(i, r, 0u, key, scale) : 0.f;
    y[o] = real && y_uniform ? uniform_draw(i, r, 1u, key, scale) : 0.f;
    dx[o] = real ? uniform_draw(i, r, 4u, key, 1.1920928955078125e-07f) : 0.f;
    dy[o] = 0.f;
    if (p) {
        p[o] = 1.f;
        dp[o] = 0.f;
    }
}

// nrm2[r] = sum over the spins of dx^2 + dy^2 + dp^2 (FP64), one warp per
// replica, partial sums added in a fixed order (deterministic).
__global__ void k_tan_tc_norm(const float* __restrict__ dx, const float* __restrict__ dy,
                              const float* __restrict__ dp, int N, int R, int Np,
                              double* __restrict__ nrm2) {
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= R) return;
    const size_t o = (size_t)r * Np;
    double s = 0.0;
    for (int i = lane; i < N; i += 32) {
        const double a = dx[o + i], b = dy[o + i], d = dp ? dp[o + i] : 0.f;
        s += a * a + b * b + d * d;
    }
    for (int k = 16; k; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
    if (lane == 0) nrm2[r] = s;
}

// log_sum[r] += log |delta| (when accumulating); scale[r] = 1 / |delta|.
__global__ void k_tan_tc_log(const double* __restrict__ nrm2, double* __restrict__ log_sum,
                             float* __restrict__ scale, int R, int accumulate) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const double s2 = nrm2[r];
    if (accumulate) log_sum[r] += 0.5 * log(s2);
    scale[r] = s2 > 0.0 ? (float)(1.0 / sqrt(s2)) : 0.f;
}

// The tangent of every replica scaled by scale[r] (scale[r] = 0 on padded
// replicas), then the step's operand planes written from x and dx.
__global__ void k_tan_tc_planes(const float* __restrict__ x, float* __restrict__ dx,
                                float* __restrict__ dy, float* __restrict__ dp,
                                const float* __restrict__ scale, uint16_t* __restrict__ v, int Np,
                                int Rp, int sign) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (i >= Np || r >= Rp) return;
    const size_t o = (size_t)r * Np + i, plane = (size_t)Rp * Np;
    const float s = scale[r];
    const float d = dx[o] * s;
    dx[o] = d;
    dy[o] *= s;
    if (dp) dp[o] *= s;
    const float xv = x[o];
    if (sign) {
        v[o] = xv >= 0.f ? (uint16_t)0x3F80 : (uint16_t)0xBF80;
    } else {
        uint32_t h, l;
        bf16_split_bits(xv, h, l);
        v[o] = (uint16_t)h;
        v[plane + o] = (uint16_t)l;
        bf16_split_bits(d, h, l);
        v[2 * plane + o] = (uint16_t)h;
        v[3 * plane + o] = (uint16_t)l;
    }
}

template <bool SIGN, bool CONTROL>
gsb_status set_attr_once() {
    static std::atomic<uint64_t> seen{0};
    if (first_on_device(seen))
        GSB_CUDA_TRY(cudaFuncSetAttribute(k_tangent_tc<SIGN, CONTROL>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
    return GSB_OK;
}

template <bool SIGN, bool CONTROL>
gsb_status launch_step(const TanArgs& a, int grid, cudaStream_t s) {
    gsb_status st = set_attr_once<SIGN, CONTROL>();
    if (st != GSB_OK) return st;
    k_tangent_tc<SIGN, CONTROL><<<grid, kThreads, kSmem, s>>>(a);
    GSB_LAUNCH_CHECK("k_tangent_tc");
    return GSB_OK;
}

struct TcBuffers {
    float* st[6] = {};  // x, y, p, dx, dy, dp
    __nv_bfloat16* v[2] = {};
    float* A = nullptr;
    double* nrm2 = nullptr;
    double* log_sum = nullptr;
    float* scale = nullptr;
    int* status = nullptr;
    ~TcBuffers() {
        for (float* q : st) dev_free(q);
        dev_free(v[0]);
        dev_free(v[1]);
        dev_free(A);
        dev_free(nrm2);
        dev_free(log_sum);
        dev_free(scale);
        dev_free(status);
    }
};

}  // namespace

gsb_status tangent_bf16x3(gsb_problem* P, bool sign, bool control, int R, const float* A_rep,
                          float c, float dt, int M, int nsteps, int renorm_every, uint64_t seed,
                          float x0_range, bool y0_uniform, double* log_sum, cudaStream_t s) {
    gsb_status st = bf16_ensure_planes(P, s);
    if (st != GSB_OK) return st;
    const int N = P->N, Np = P->Np;
    const int Rp = round_up(R, kT);
    const int planes = sign ? 1 : 4;
    const size_t nst = (size_t)Np * Rp;
    TcBuffers B;
    for (int a = 0; a < 6; ++a) {
        if (!control && (a == 2 || a == 5)) continue;
        if ((st = dev_alloc(&B.st[a], nst)) != GSB_OK) return st;
    }
    for (int b = 0; b < 2; ++b)
        if ((st = dev_alloc(&B.v[b], nst * planes)) != GSB_OK) return st;
    if ((st = dev_alloc(&B.A, (size_t)Rp)) || (st = dev_alloc(&B.nrm2, (size_t)Rp)) ||
        (st = dev_alloc(&B.log_sum, (size_t)Rp)) || (st = dev_alloc(&B.scale, (size_t)Rp)) ||
        (st = dev_alloc(&B.status, 1)))
        return st;
    std::vector<float> Ah(Rp, 0.f);
    std::copy(A_rep, A_rep + R, Ah.begin());
    GSB_CUDA_TRY(cudaMemcpyAsync(B.A, Ah.data(), Rp * sizeof(float), cudaMemcpyHostToDevice, s));
    GSB_CUDA_TRY(cudaMemsetAsync(B.log_sum, 0, Rp * sizeof(double), s));
    GSB_CUDA_TRY(cudaMemsetAsync(B.scale, 0, Rp * sizeof(float), s));
    GSB_CUDA_TRY(cudaMemsetAsync(B.status, 0, sizeof(int), s));

    TanArgs a;
    memset(&a, 0, sizeof(a));
    if ((st = bf16_tensor_map(&a.tmJ[0], P->Jhi, Np, Np)) ||
        (st = bf16_tensor_map(&a.tmJ[1], P->Jlo, Np, Np)))
        return st;
    for (int b = 0; b < 2; ++b)
        if ((st = bf16_tensor_map(&a.tmV[b], B.v[b], Np, (uint64_t)planes * Rp))) return st;
    a.x = B.st[0];
    a.y = B.st[1];
    a.p = B.st[2];
    a.dx = B.st[3];
    a.dy = B.st[4];
    a.dp = B.st[5];
    a.A = B.A;
    a.v[0] = B.v[0];
    a.v[1] = B.v[1];
    a.status = B.status;
    a.Np = Np;
    a.Rp = Rp;
    a.c = c;
    a.dt = dt;

    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    k_tan_tc_init<<<dim3(Np / 128, Rp), 128, 0, s>>>(
        a.x, a.y, a.p, a.dx, a.dy, a.dp, N, R, Np, key, x0_range * 1.1920928955078125e-07f,
        y0_uniform ? 1 : 0);
    GSB_LAUNCH_CHECK("k_tan_tc_init");
    // the tangents renormalised (the log of the norm accumulated when asked)
    // and the operand planes of step m written into buffer m & 1
    auto renorm = [&](int m, int accumulate) -> gsb_status {
        k_tan_tc_norm<<<(R + 7) / 8, 256, 0, s>>>(a.dx, a.dy, a.dp, N, R, Np, B.nrm2);
        GSB_LAUNCH_CHECK("k_tan_tc_norm");
        k_tan_tc_log<<<(R + 255) / 256, 256, 0, s>>>(B.nrm2, B.log_sum, B.scale, R, accumulate);
        GSB_LAUNCH_CHECK("k_tan_tc_log");
        k_tan_tc_planes<<<dim3(Np / 128, Rp), 128, 0, s>>>(
            a.x, a.dx, a.dy, a.dp, B.scale, reinterpret_cast<uint16_t*>(B.v[m & 1]), Np, Rp,
            sign ? 1 : 0);
        GSB_LAUNCH_CHECK("k_tan_tc_planes");
        return GSB_OK;
    };
    if ((st = renorm(0, 0)) != GSB_OK) return st;  // unit start vectors

    int sms = 0, dev = 0;
    GSB_CUDA_TRY(cudaGetDevice(&dev));
    GSB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int ntiles = (Np / kT) * (Rp / kT);
    const int grid = std::max(1, std::min(ntiles, sms));
    call_prof_reset();
    for (int m = 0; m < nsteps; ++m) {
        a.m = m;
        a.p_shared = (float)(1.0 - (double)(m + 1) / (double)M);
        a.inv_rem = 1.0f / (float)(M - m);
        if ((st = call_prof_begin(s)) != GSB_OK) return st;
        if (sign)
            st = control ? launch_step<true, true>(a, grid, s) : launch_step<true, false>(a, grid, s);
        else
            st = control ? launch_step<false, true>(a, grid, s) : launch_step<false, false>(a, grid, s);
        if (st != GSB_OK) return st;
        if ((st = call_prof_end(s, 1)) != GSB_OK) return st;
        if ((m + 1) % renorm_every == 0 || m + 1 == nsteps)
            if ((st = renorm(m + 1, 1)) != GSB_OK) return st;
    }
    int dst = 0;
    GSB_CUDA_TRY(cudaMemcpyAsync(log_sum, B.log_sum, R * sizeof(double), cudaMemcpyDeviceToHost, s));
    GSB_CUDA_TRY(cudaMemcpyAsync(&dst, B.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    GSB_CUDA_TRY(cudaStreamSynchronize(s));
    if (dst & kDevTimeout)
        return set_error(GSB_ETIMEOUT, "k_tangent_tc: a barrier wait exceeded its bound");
    if (dst & kDevBounds) return set_error(GSB_ECUDA, "a kernel detected an out-of-range index");
    return call_prof_collect();
}

}  // namespace gsb
