// k_dense_tc.cu -- dense time step on the sm_103a tensor cores.
//
// The many-body term F = J V over the full K = Np is a chain of tcgen05.mma
// into FP32 TMEM accumulators, fed by a TMA ring of 128-byte-swizzled K
// slices of J and V; epilogue warps read F back with tcgen05.ld, apply
// Eqs. 7, 3, 4, 5 and write the next step's V operand. Two exact forms:
//
//   FP8  (GSB_PREC_FP8):  J and V = sgn x in e4m3, kind::f8f6f4. Products are
//                         +-J_ij and partial sums integers far below 2^24
//                         (|J| <= 16, N < 2^20): exact in any order.
//                         k_tc_step (one step per launch, the reference form)
//                         and k_tc_persist (many steps per launch).
//   FX32 (GSB_PREC_FX32): J in bf16 (integer) and x as the 32-bit fixed
//                         point integer q = rint(x 2^30), written as four
//                         signed base-256 digits d_0..d_3 (bf16, exact).
//                         Digit plane k accumulates D_k = J d_k in its own
//                         128-column TMEM accumulator; every partial sum is an
//                         integer below 2^24 (128 sum_j |J_ij| < 2^24), so D_k
//                         is exact whatever order the tensor core adds in. The
//                         epilogue forms sum_k 256^k D_k exactly in int64 and
//                         rounds 2^-30 times it once to FP32: f is the
//                         correctly rounded J x_q, and x_q = x for
//                         |x| >= 2^-7. k_fx32_step.
#include <cudaTypedefs.h>

#include "gsb_update.cuh"
#include "tc_ptx.cuh"

namespace gsb {

namespace {

using namespace tc;

constexpr int BM = 128;   // spins per tile
constexpr int BN = 128;   // replicas per tile
constexpr int KB = 128;   // bytes of K per pipeline stage (one swizzle row)
// k_tc_step: warp 0 lane 0 issues TMA, warp 1 owns TMEM and its lane 0 issues
// MMAs, warps 2-5 run the epilogue (warp w reads TMEM lanes 32 (w % 4) ..
// +31, as tcgen05.ld requires).
constexpr int kThreads = 192;
constexpr int kStagesS = 6;

__host__ __device__ constexpr int smem_bytes_step() {
    return 1024 /*alignment slack*/ + kStagesS * (BM * KB + BN * KB) + 256;
}

__device__ __forceinline__ uint8_t e4m3_sign(float x) { return x >= 0.f ? 0x38 : 0xB8; }  // +-1.0

// bf16 bits of the integer n - 128 for 0 <= n <= 255, without a conversion
// instruction: the float with exponent 2^23 and n in its mantissa is 2^23 + n;
// subtracting 2^23 + 128 leaves n - 128 exactly, whose at most 8 significant
// bits make its top 16 bits its bf16 encoding.
__device__ __forceinline__ uint16_t small_int_bf16(int n) {
    const float f = __int_as_float(0x4B000000 | n) - 8388736.0f;  // 2^23 + 128
    return (uint16_t)(__float_as_uint(f) >> 16);
}

// x as four signed base-256 digits of q = rint(x 2^30), |x| <= 1:
// q = d0 + 256 d1 + 65536 d2 + 16777216 d3, d0..d2 in [-128, 127], |d3| <= 64.
// x 2^30 is exact in FP32 (a power-of-two scaling), so q = x 2^30 exactly
// whenever |x| >= 2^-7. With u = q + 0x808080 = q + 128 (1 + 256 + 65536):
// d_k = byte_k(u) - 128 for k < 3 and d_3 = u >> 24 (arithmetic); returned as
// bf16 bit patterns (each digit is exact in bf16).
__device__ __forceinline__ void fx32_digit_bits(float x, uint16_t (&d)[4]) {
    const int u = __float2int_rn(x * 1073741824.0f) + 0x808080;
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = small_int_bf16((u >> (8 * k)) & 255);
    d[3] = small_int_bf16((u >> 24) + 128);  // the top digit, in [-64, 64]
}

// f = 2^-30 sum_k 256^k D_k, from exact integer accumulators (|D_k| < 2^24,
// so each converts to int32 exactly), rounded once: the int64 sum is rounded
// to FP32 by one conversion and the power-of-two scale is exact. No FP64 (a
// slow pipe on this part).
__device__ __forceinline__ float fx32_combine(float d0, float d1, float d2, float d3) {
    const long long v = (long long)__float2int_rn(d0) + ((long long)__float2int_rn(d1) << 8) +
                        ((long long)__float2int_rn(d2) << 16) +
                        ((long long)__float2int_rn(d3) << 24);
    return __ll2float_rn(v) * 9.313225746154785e-10f;  // 2^-30
}

// One FP8 step per launch. One CTA owns 128 spins (rows of J, TMEM lanes) x
// 128 replicas (TMEM columns); the epilogue thread of a spin updates its 128
// oscillators.
template <bool CONTROL>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_step(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              int Np, int Rp, float* __restrict__ x, float* __restrict__ y,
              float* __restrict__ p, const float* __restrict__ A, uint8_t* __restrict__ vnext,
              float c, float dt, float p_shared, float inv_rem, int* status) {
    // debug build: the grid covers the padded shape exactly (a uniform return)
    if (!GSB_DOK(Np > 0 && Np % KB == 0 && Rp % BN == 0 && (int)gridDim.x * BN == Rp &&
                     (int)gridDim.y * BM == Np,
                 status))
        return;
    constexpr int S = kStagesS;
    constexpr int SA = BM * KB;
    constexpr int SB = BN * KB;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sB = smem + S * SA;
    uint64_t* full = (uint64_t*)(sB + S * SB);
    uint64_t* empty = full + S;
    uint64_t* accf = empty + S;
    uint64_t* drain = accf + 1;  // the MMA issuer's last commit (all its MMAs done)
    uint32_t* tmem_slot = (uint32_t*)(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i0 = blockIdx.y * BM, r0 = blockIdx.x * BN;
    const int nk = Np / KB;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accf, 1);
        mbar_init(drain, 1);
        fence_barrier_init();
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
    }
    constexpr uint32_t kTmemCols = 128;
    if (warp == 1) tmem_alloc(tmem_slot, kTmemCols);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int armed = 0;
            for (int kc = 0; kc < nk; ++kc) {
                const int s = kc % S;
                const uint32_t ph = (uint32_t)(kc / S) & 1u;
                if (kc >= S && !mbar_wait(&empty[s], ph ^ 1u, status)) break;
                mbar_arrive_expect_tx(&full[s], SA + SB);
                tma_load_2d(sA + s * SA, &tmA, &full[s], kc * KB, i0);
                tma_load_2d(sB + s * SB, &tmB, &full[s], kc * KB, r0);
                armed = kc + 1;
            }
            // no copy in flight when the CTA leaves
            for (int kc = armed > S ? armed - S : 0; kc < armed; ++kc)
                mbar_wait(&full[kc % S], (uint32_t)(kc / S) & 1u, status, kDrainLimitCycles);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_make(0u, BM, BN);
            bool ok = true;
            for (int kc = 0; kc < nk && ok; ++kc) {
                const int s = kc % S;
                const uint32_t ph = (uint32_t)(kc / S) & 1u;
                if (!mbar_wait(&full[s], ph, status)) {
                    ok = false;
                    break;
                }
                fence_after_sync();
                const uint32_t a0 = smem_u32(sA + s * SA);
                const uint32_t b0 = smem_u32(sB + s * SB);
#pragma unroll
                for (int k = 0; k < KB / 32; ++k)  // 32 bytes of K per MMA
                    mma_f8f6f4(tmem, sdesc_sw128(a0 + k * 32), sdesc_sw128(b0 + k * 32), idesc,
                               (kc | k) != 0);
                mma_commit(&empty[s]);
            }
            if (ok) mma_commit(accf);
            // every MMA issued has finished before TMEM is released
            mma_commit(drain);
            mbar_wait(drain, 0, status, kDrainLimitCycles);
        }
    } else {
        // epilogue: warp w owns TMEM lanes 32 (w % 4) .. +31
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        const int i = i0 + row;
        // tcgen05.ld is warp-collective: proceed only if every lane saw the accumulator
        const bool ready = __all_sync(0xffffffffu, mbar_wait(accf, 0, status));
        if (ready) {
            fence_after_sync();
            const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
            for (int cb = 0; cb < BN; cb += 16) {
                float f[16];
                tmem_ld16(taddr + cb, f);
                const size_t o = (size_t)i * Rp + r0 + cb;
                float xs[16], ys[16], ps[16], as[16];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 a = *reinterpret_cast<const float4*>(x + o + 4 * q);
                    const float4 b = *reinterpret_cast<const float4*>(y + o + 4 * q);
                    xs[4 * q] = a.x; xs[4 * q + 1] = a.y; xs[4 * q + 2] = a.z; xs[4 * q + 3] = a.w;
                    ys[4 * q] = b.x; ys[4 * q + 1] = b.y; ys[4 * q + 2] = b.z; ys[4 * q + 3] = b.w;
                    if (CONTROL) {
                        const float4 pp = *reinterpret_cast<const float4*>(p + o + 4 * q);
                        const float4 aa = *reinterpret_cast<const float4*>(A + r0 + cb + 4 * q);
                        ps[4 * q] = pp.x; ps[4 * q + 1] = pp.y; ps[4 * q + 2] = pp.z; ps[4 * q + 3] = pp.w;
                        as[4 * q] = aa.x; as[4 * q + 1] = aa.y; as[4 * q + 2] = aa.z; as[4 * q + 3] = aa.w;
                    } else {
                        ps[4 * q] = ps[4 * q + 1] = ps[4 * q + 2] = ps[4 * q + 3] = 0.f;
                        as[4 * q] = as[4 * q + 1] = as[4 * q + 2] = as[4 * q + 3] = 0.f;
                    }
                }
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    sb_update<CONTROL>(xs[k], ys[k], ps[k], f[k], as[k], c, dt, p_shared, inv_rem);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    *reinterpret_cast<float4*>(x + o + 4 * q) =
                        make_float4(xs[4 * q], xs[4 * q + 1], xs[4 * q + 2], xs[4 * q + 3]);
                    *reinterpret_cast<float4*>(y + o + 4 * q) =
                        make_float4(ys[4 * q], ys[4 * q + 1], ys[4 * q + 2], ys[4 * q + 3]);
                    if (CONTROL)
                        *reinterpret_cast<float4*>(p + o + 4 * q) =
                            make_float4(ps[4 * q], ps[4 * q + 1], ps[4 * q + 2], ps[4 * q + 3]);
                }
                // next step's operand, replica-major [Rp][Np]
#pragma unroll
                for (int k = 0; k < 16; ++k) vnext[(size_t)(r0 + cb + k) * Np + i] = e4m3_sign(xs[k]);
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        fence_after_sync();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// Ising energies (Eq. 1) on the FP8 tensor cores, for the sgn coupling's runs:
// e_acc[r] += sum_i s_ri (J s_r)_i over the CTA's 128 spins, with
// s = sgn x(t_m) read from the e4m3 operand V(t_m) that the step kernels leave
// in the buffer of the step's parity. The tile is transposed as in
// k_tc_persist (a TMEM lane is a replica), so each epilogue thread reduces its
// replica's products over the spins in registers; the products and sums are
// integers (exact), added in FP64 across the CTAs of a replica column.
// Warps: 0 TMA producer, 1 TMEM owner + MMA issuer, 2-5 epilogue.
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_energy(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                const uint8_t* __restrict__ v, int Np, double* __restrict__ e_acc, int* status) {
    if (!GSB_DOK(Np > 0 && Np % KB == 0 && (int)gridDim.y * BM == Np, status)) return;
    constexpr int S = kStagesS;
    constexpr int SA = BM * KB;
    constexpr int SB = BN * KB;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sB = smem + S * SA;
    uint64_t* full = (uint64_t*)(sB + S * SB);
    uint64_t* empty = full + S;
    uint64_t* accf = empty + S;
    uint64_t* drain = accf + 1;
    uint32_t* tmem_slot = (uint32_t*)(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = blockIdx.x * BN, i0 = blockIdx.y * BM;
    const int nk = Np / KB;

    if (threadIdx.x == 0) {
        for (int st = 0; st < S; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], 1);
        }
        mbar_init(accf, 1);
        mbar_init(drain, 1);
        fence_barrier_init();
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
    }
    constexpr uint32_t kTmemCols = 128;
    if (warp == 1) tmem_alloc(tmem_slot, kTmemCols);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int armed = 0;
            for (int kc = 0; kc < nk; ++kc) {
                const int st = kc % S;
                const uint32_t ph = (uint32_t)(kc / S) & 1u;
                if (kc >= S && !mbar_wait(&empty[st], ph ^ 1u, status)) break;
                mbar_arrive_expect_tx(&full[st], SA + SB);
                tma_load_2d(sA + st * SA, &tmA, &full[st], kc * KB, i0);
                tma_load_2d(sB + st * SB, &tmB, &full[st], kc * KB, r0);
                armed = kc + 1;
            }
            for (int kc = armed > S ? armed - S : 0; kc < armed; ++kc)
                mbar_wait(&full[kc % S], (uint32_t)(kc / S) & 1u, status, kDrainLimitCycles);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_make(0u, BN, BM);
            bool ok = true;
            for (int kc = 0; kc < nk && ok; ++kc) {
                const int st = kc % S;
                const uint32_t ph = (uint32_t)(kc / S) & 1u;
                if (!mbar_wait(&full[st], ph, status)) {
                    ok = false;
                    break;
                }
                fence_after_sync();
                const uint32_t a0 = smem_u32(sA + st * SA);
                const uint32_t b0 = smem_u32(sB + st * SB);
#pragma unroll
                for (int k = 0; k < KB / 32; ++k)
                    mma_f8f6f4(tmem, sdesc_sw128(b0 + k * 32), sdesc_sw128(a0 + k * 32), idesc,
                               (kc | k) != 0);
                mma_commit(&empty[st]);
            }
            if (ok) mma_commit(accf);
            mma_commit(drain);
            mbar_wait(drain, 0, status, kDrainLimitCycles);
        }
    } else {
        const int quarter = warp & 3;
        const int r = r0 + quarter * 32 + lane;  // this thread's replica (TMEM lane)
        const bool ready = __all_sync(0xffffffffu, mbar_wait(accf, 0, status));
        if (ready) {
            fence_after_sync();
            const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
            const uint8_t* srow = v + (size_t)r * Np + i0;
            // each (J s)_i is an exact integer in FP32 (the FP8 path's condition);
            // the products with s_i = +-1 are summed in int64
            long long part = 0;
#pragma unroll 1
            for (int cb = 0; cb < BM; cb += 16) {
                float f[16];
                tmem_ld16(tl + cb, f);
                const uint4 b = *reinterpret_cast<const uint4*>(srow + cb);
                const uint32_t w[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    // e4m3 +-1: the sign bit of each byte
                    const bool neg = (w[k >> 2] >> (8 * (k & 3) + 7)) & 1u;
                    const int fi = __float2int_rn(f[k]);
                    part += neg ? -fi : fi;
                }
            }
            atomicAdd(&e_acc[r], (double)part);
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        fence_after_sync();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// ---------------------------------------------------------------------------
// Persistent form of the FP8 step: one launch runs many steps.
// The tile is transposed against k_tc_step: the MMA forms F^T = V J^T, so a
// TMEM lane is a replica and a column a spin. Each CTA keeps its tile's x and
// y in TMEM next to the accumulator (columns [0,128) F; [128,384) x and y of
// each 16 spins side by side, 32 columns per chunk, so one 32-column load or
// store moves both) and p (individual control) in the registers of the
// epilogue thread that owns the oscillator, 64 per thread -- a third less
// TMEM traffic per step than with p in TMEM -- so a step moves no state
// through global memory: only the 16 KB of the next V tile leave the SM, each
// thread writing 16 consecutive bytes of its replica's row of V at a time. The
// products are +-J_ij and the sums integers, so F is bit-identical to
// k_tc_step's whatever the order of the K slices.
//
// The CTAs that share a replica block (a column) exchange those V tiles
// between steps in one of two ways:
//   CLUSTER = true (Np <= 16 x 128): the column is one thread-block cluster.
//     After its epilogue each CTA arrives (release, cluster scope) on the
//     step's barrier (count: the CTAs of the column) in every CTA of the
//     cluster, and a producer waits on its own copy before it loads the step's
//     V, the K slices in rotated order from its own. Columns are independent
//     clusters, so no grid-wide co-residency is needed. Two barriers,
//     alternating with the step's parity: a writer can run at most one step
//     ahead of a reader, so a reader's parity wait is never two phases behind.
//   CLUSTER = false (any Np): a cooperative launch; the column meets at a
//     counter in global memory (release add / acquire poll, bounded) before
//     any of its CTAs loads the column's next V.
// J does not change, so the producer issues the first ring stages' J tiles
// before it waits.
//
// FORM: kFormCluster is the cluster form above, kFormGrid the grid form, and
// kFormPair the grid form on SM pairs: the CTAs of replica blocks 2q and
// 2q + 1 (same spin block) are a cluster of two whose MMAs (cta_group::2,
// M = 256) the even CTA issues. Each CTA stages its own 128 rows of V and
// half of the spin block's J rows (64), so a K slice costs an SM 24 KB of
// shared memory and of L2 reads instead of 32 KB, for the same 128 x 128
// tile per SM (but the peer's tensor core reads the other half of B out of
// this SM's shared memory, and each step waits for two replica columns). The even CTA's
// full barriers count both CTAs' bytes (the odd CTA's loads signal them
// across the pair), the MMA issuer's commits arrive on both CTAs' barriers,
// and both epilogues release the accumulator on the even CTA's barrier. The
// exchange of V between steps is the grid form's, per replica block.
//
// Warps: 0 TMA producer, 1 TMEM owner + MMA issuer, 2-9 epilogue (warp w
// reads TMEM lanes 32 (w % 4).. -- its 32 replicas -- and columns 64 ((w - 2)
// / 4) .. +63 -- 64 spins).
constexpr int kThreadsP = 320;
constexpr int kEpiThreadsP = 256;
// A ring stage holds kAtomsP consecutive 128-byte K slices of J and of V. The
// K loop costs about 3.3 us per MB that passes through shared memory (TMA
// writes plus tensor-core operand reads: 1 MB per step for a 128 x 128 tile
// at K = 2048) plus about 0.1 us per ring stage (barrier round trip and
// commit), and neither the number of slices in flight nor the MMA's N moves
// it (measured: one-slice stages, seven in flight, 4.86 us; two-slice stages,
// three in flight, 4.10 us; N = 64, 3.84 us): three-slice stages, two in
// flight, take the fewest stages that fit.
constexpr int kAtomsP = 3;
constexpr int kStagesP = 2;
constexpr int kMaxClusterP = 16;  // the largest (non-portable) cluster
constexpr int kStagesQ = 3;       // ring stages of the pair form
enum : int { kFormGrid = 0, kFormCluster = 1, kFormPair = 2 };

__host__ __device__ constexpr int smem_bytes_persist(int form = kFormGrid, int bs = BM) {
    return form == kFormPair ? 1024 + kStagesQ * kAtomsP * (BN + BM / 2) * KB + 512
                             : 1024 + kStagesP * kAtomsP * (BN + bs) * KB + 512;
}

// TMEM moves of an epilogue chunk of CH spins: F (CH columns at cf) and x, y
// (2 CH columns at cxy, x first), the loads in flight together with one wait;
// and the store of x, y.
template <int CH>
__device__ __forceinline__ void tmem_ld_fxy(uint32_t cf, uint32_t cxy, float (&f)[CH],
                                            float (&xs)[CH], float (&ys)[CH]) {
    if constexpr (CH == 16) {
        uint32_t rf[16], rx[16], ry[16];
        tmem_ld16_async(cf, rf);
        tmem_ld32_async(cxy, rx, ry);
        tmem_wait_ld(rf);
        tmem_wait_ld(rx);
        tmem_wait_ld(ry);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            f[k] = __uint_as_float(rf[k]);
            xs[k] = __uint_as_float(rx[k]);
            ys[k] = __uint_as_float(ry[k]);
        }
    } else {
        static_assert(CH == 8, "chunk");
        uint32_t rf[8], rxy[16];
        tmem_ld8_async(cf, rf);
        tmem_ld16_async(cxy, rxy);
        tmem_wait_ld8(rf);
        tmem_wait_ld(rxy);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            f[k] = __uint_as_float(rf[k]);
            xs[k] = __uint_as_float(rxy[k]);
            ys[k] = __uint_as_float(rxy[8 + k]);
        }
    }
}
template <int CH>
__device__ __forceinline__ void tmem_st_xy(uint32_t cxy, const float (&v)[2 * CH]) {
    if constexpr (CH == 16) {
        float lo[16], hi[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            lo[k] = v[k];
            hi[k] = v[16 + k];
        }
        tmem_st32(cxy, lo, hi);
    } else {
        tmem_st16(cxy, v);
    }
}

// BS: spins per CTA (the MMA's N and the epilogue's width). 128, or 112 in the
// grid form, where ceil(N / 112) spin blocks put more SMs to work on the same
// step (N = 2000, R = 1024: 144 CTAs instead of 128, each with 6 % less
// shared-memory traffic in its K loop and 56 instead of 64 oscillators per
// epilogue thread). The spins past the last block (up to N_p) are padding:
// J is zero there, so their V bytes never reach F.
template <bool CONTROL, int FORM, int BS = BM>
__global__ void __launch_bounds__(kThreadsP, 1)
    k_tc_persist(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmV0,
                 const __grid_constant__ CUtensorMap tmV1, int Np, int Rp, float* __restrict__ x,
                 float* __restrict__ y, float* __restrict__ p, const float* __restrict__ A,
                 uint8_t* __restrict__ v0, uint8_t* __restrict__ v1, float c, float dt,
                 const float* __restrict__ p_sched, int M, int m0, int nsteps,
                 uint32_t* __restrict__ counters, int* status) {
    // debug build: the grid and the steps match the shape and the run (checked
    // by every thread alike, before any barrier: a uniform return)
    if (!GSB_DOK(Np > 0 && Np % KB == 0 && Rp % BN == 0 && m0 >= 0 && nsteps >= 0 &&
                     m0 + nsteps <= M &&
                     (FORM == kFormCluster
                          ? ((int)gridDim.x * BM == Np && (int)gridDim.y * BN == Rp &&
                             Np / BM <= kMaxClusterP)
                          : ((int)gridDim.x * BN == Rp &&
                             (BS == BM ? (int)gridDim.y * BM == Np : (int)gridDim.y * BS <= Np) &&
                             (FORM != kFormPair || gridDim.x % 2 == 0))),
                 status))
        return;
    constexpr bool CLUSTER = FORM == kFormCluster, PAIR = FORM == kFormPair;
    static_assert(BS == BM || FORM == kFormGrid, "narrow spin blocks: grid form only");
    static_assert(BS % 16 == 0 && BS <= BM, "MMA N");
    constexpr int S = PAIR ? kStagesQ : kStagesP;
    constexpr int JR = PAIR ? BM / 2 : BS;       // J rows this CTA stages
    // epilogue: CH spins per chunk, NCH chunks per thread (half the block)
    constexpr int CH = BS == BM ? 16 : 8;
    constexpr int HW = BS / 2, NCH = HW / CH;
    static_assert(NCH * CH == HW, "epilogue chunks");
    constexpr int SA1 = JR * KB, SB1 = BN * KB;  // one K atom of J / of V
    constexpr int SA = kAtomsP * SA1, SB = kAtomsP * SB1;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sB = smem + S * SA;
    uint64_t* full = (uint64_t*)(sB + S * SB);
    uint64_t* empty = full + S;
    uint64_t* accf = empty + S;
    uint64_t* acce = accf + 1;
    uint64_t* vready = acce + 1;  // [2]: the column's V of a step, one arrival per writer
    uint64_t* drain = vready + 2;  // the MMA issuer's last commit (all its MMAs done)
    uint32_t* tmem_slot = (uint32_t*)(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = Np / KB;                       // K atoms per step == spin blocks
    const int ns = (nk + kAtomsP - 1) / kAtomsP;  // ring stages per step
    // spin block (the CTA's own K slice) and replica block
    const int own = CLUSTER ? (int)blockIdx.x : (int)blockIdx.y;
    const int rb = CLUSTER ? (int)blockIdx.y : (int)blockIdx.x;
    const int i0 = own * BS, r0 = rb * BN;
    uint32_t* ctr = counters + rb;
    // pair form: this CTA's rank in its pair (0 issues the MMAs)
    const uint32_t rank = PAIR ? cluster_ctarank() : 0u;
    const bool leader = rank == 0u;
    // the k-th K atom of a step: rotated from the CTA's own slice in the cluster form
    auto atom = [&](int k) { return CLUSTER ? (own + k) % nk : k; };

    if (threadIdx.x == 0) {
        for (int st = 0; st < S; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], 1);
        }
        mbar_init(accf, 1);
        mbar_init(acce, PAIR ? 2u : 1u);  // pair form: both epilogues, on the even CTA
        mbar_init(&vready[0], (uint32_t)nk);
        mbar_init(&vready[1], (uint32_t)nk);
        mbar_init(drain, 1);
        tmem_slot[1] = 0u;  // epilogue abort flag
        fence_barrier_init();
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmV0);
        tma_prefetch_desc(&tmV1);
    }
    if (warp == 1) {
        if (PAIR)
            tmem_alloc_pair(tmem_slot, 512);
        else
            tmem_alloc(tmem_slot, 512);
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    // every CTA's barriers (and, in pairs, both TMEM allocations) exist before
    // any CTA arrives on them or issues an MMA
    if (CLUSTER || PAIR) cluster_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t g = 0;  // ring stage counter across steps
            const int pre = ns < S ? ns : S;
            bool ok = true;
            // K atoms u kAtomsP .. of a step go to stage u
            auto atoms = [&](int u) { return nk - u * kAtomsP < kAtomsP ? nk - u * kAtomsP : kAtomsP; };
            // pair form: every load signals the even CTA's full barrier,
            // which expects both CTAs' bytes
            const uint32_t full_pair = PAIR ? mapa_u32(smem_u32(full), 0u) : 0u;
            auto load_j = [&](int u, uint32_t st) {
                if (!PAIR) {
                    mbar_arrive_expect_tx(&full[st], (uint32_t)atoms(u) * (SA1 + SB1));
                    for (int a = 0; a < atoms(u); ++a)
                        tma_load_2d(sA + st * SA + a * SA1, &tmA, &full[st],
                                    atom(u * kAtomsP + a) * KB, i0);
                } else {
                    if (leader)
                        mbar_arrive_expect_tx(&full[st], 2u * (uint32_t)atoms(u) * (SA1 + SB1));
                    for (int a = 0; a < atoms(u); ++a)
                        tma_load_2d_pair(sA + st * SA + a * SA1, &tmA, full_pair + 8u * st,
                                         atom(u * kAtomsP + a) * KB, i0 + (int)rank * JR);
                }
            };
            auto load_v = [&](int u, uint32_t st, const CUtensorMap* tv) {
                for (int a = 0; a < atoms(u); ++a) {
                    if (PAIR)
                        tma_load_2d_pair(sB + st * SB + a * SB1, tv, full_pair + 8u * st,
                                         atom(u * kAtomsP + a) * KB, r0);
                    else
                        tma_load_2d(sB + st * SB + a * SB1, tv, &full[st],
                                    atom(u * kAtomsP + a) * KB, r0);
                }
            };
            uint32_t armed = 0;  // ring positions whose full barrier has been armed
            for (int s = 0; s < nsteps && ok; ++s) {
                const CUtensorMap* tv = ((m0 + s) & 1) ? &tmV1 : &tmV0;
                // J for the first ring stages: independent of the other CTAs
                int nj = 0;
                for (int u = 0; u < pre; ++u) {
                    const uint32_t gg = g + u, st = gg % S, ph = (gg / S) & 1u;
                    if (gg >= (uint32_t)S && !mbar_wait(&empty[st], ph ^ 1u, status)) {
                        ok = false;
                        break;
                    }
                    load_j(u, st);
                    armed = gg + 1;
                    ++nj;
                }
                // V of this step is complete once every CTA of the replica block
                // published it: all nk arrivals on this step's barrier (cluster
                // form), or the counter at nk per step (grid form)
                if (ok && s > 0) {
                    ok = CLUSTER ? mbar_wait_cluster(&vready[(s - 1) & 1],
                                                     (uint32_t)((s - 1) >> 1) & 1u, status)
                                 : wait_counter(ctr, gridDim.y * (uint32_t)s, status);
                    if (ok) fence_proxy_async();
                }
                // V of the stages whose J is out -- after a failed wait too, so that
                // every armed barrier completes its phase (the step's results are
                // void then; the status word says so)
                for (int u = 0; u < nj; ++u) load_v(u, (g + u) % S, tv);
                if (!ok) break;
                for (int u = pre; u < ns; ++u) {
                    const uint32_t gg = g + u, st = gg % S, ph = (gg / S) & 1u;
                    if (gg >= (uint32_t)S && !mbar_wait(&empty[st], ph ^ 1u, status)) {
                        ok = false;
                        break;
                    }
                    load_j(u, st);
                    load_v(u, st, tv);
                    armed = gg + 1;
                }
                g += ns;
            }
            // no copy is in flight when the CTA leaves: the last phase armed on
            // every stage has landed (in pairs, the even CTA's full barriers
            // count the odd CTA's copies too, and both leave together)
            if (leader)
                for (uint32_t gg = armed > (uint32_t)S ? armed - S : 0u; gg < armed; ++gg)
                    mbar_wait(&full[gg % S], (gg / S) & 1u, status, kDrainLimitCycles);
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            constexpr uint32_t idesc = idesc_make(0u, PAIR ? 2 * BN : BN, PAIR ? BM : BS);
            uint32_t g = 0;
            bool ok = true;
            for (int s = 0; s < nsteps && ok; ++s) {
                // pair form: the odd CTA's epilogue arrives from across the pair
                if (s > 0 && !(PAIR ? mbar_wait_cluster(acce, (uint32_t)(s - 1) & 1u, status)
                                    : mbar_wait(acce, (uint32_t)(s - 1) & 1u, status)))
                    break;
                fence_after_sync();
                for (int u = 0; u < ns; ++u, ++g) {
                    const uint32_t st = g % S, ph = (g / S) & 1u;
                    if (!mbar_wait(&full[st], ph, status)) {
                        ok = false;
                        break;
                    }
                    fence_after_sync();
                    const int na = nk - u * kAtomsP < kAtomsP ? nk - u * kAtomsP : kAtomsP;
                    for (int a = 0; a < na; ++a) {
                        const uint32_t a0 = smem_u32(sA + st * SA + a * SA1);
                        const uint32_t b0 = smem_u32(sB + st * SB + a * SB1);
#pragma unroll
                        for (int k = 0; k < KB / 32; ++k) {
                            if (PAIR)
                                mma_f8f6f4_pair(tmem, sdesc_sw128(b0 + k * 32),
                                                sdesc_sw128(a0 + k * 32), idesc, (u | a | k) != 0);
                            else
                                mma_f8f6f4(tmem, sdesc_sw128(b0 + k * 32), sdesc_sw128(a0 + k * 32),
                                           idesc, (u | a | k) != 0);
                        }
                    }
                    if (PAIR)
                        mma_commit_pair(&empty[st]);
                    else
                        mma_commit(&empty[st]);
                }
                if (ok) {
                    if (PAIR)
                        mma_commit_pair(accf);
                    else
                        mma_commit(accf);
                }
            }
            // every MMA issued has finished before TMEM is released
            if (PAIR)
                mma_commit_pair(drain);
            else
                mma_commit(drain);
            mbar_wait(drain, 0, status, kDrainLimitCycles);
        }
    } else {
        const int ew = warp - 2;
        const int quarter = warp & 3;
        const int c0 = (ew >> 2) * HW;
        const int r = r0 + quarter * 32 + lane;  // this thread's replica (TMEM lane)
        const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
        const float a_r = CONTROL ? A[r] : 0.f;
        // state of this thread's replica, spins i0 + c0 .. + HW - 1: x and y
        // into TMEM (x and y of each chunk side by side, 2 CH columns), p
        // (individual control) into registers -- a step's TMEM traffic is then
        // F, x, y in and x, y out
        float pr[CONTROL ? HW : 1];
#pragma unroll 1
        for (int cb = c0; cb < c0 + HW; cb += CH) {
            const size_t o = (size_t)(i0 + cb) * Rp + r;
            float v[2 * CH];
#pragma unroll
            for (int k = 0; k < CH; ++k) {
                v[k] = x[o + (size_t)k * Rp];
                v[CH + k] = y[o + (size_t)k * Rp];
            }
            tmem_st_xy<CH>(tl + 128 + 2 * cb, v);
        }
        if (CONTROL) {
#pragma unroll
            for (int k = 0; k < HW; ++k) pr[k] = p[(size_t)(i0 + c0 + k) * Rp + r];
        }
        tmem_wait_st();
        // Every epilogue warp passes the same named barriers: a timeout in one of
        // them is published in *abort and all of them leave after the barrier.
        volatile uint32_t* abort_flag = tmem_slot + 1;
        for (int s = 0; s < nsteps; ++s) {
            const int m = m0 + s;
            bool ok = *abort_flag == 0u;
            if (ok) ok = __all_sync(0xffffffffu, mbar_wait(accf, (uint32_t)s & 1u, status));
            if (!ok) {
                *abort_flag = 1u;
                named_barrier_sync(1, kEpiThreadsP);
                break;
            }
            fence_after_sync();
            const float inv_rem = __frcp_rn((float)(M - m));
            const float p_shared = CONTROL ? 0.f : p_sched[s];
            // V(t_{m+1}) goes to buffer (m + 1) & 1; this thread's CH spins of a
            // chunk are CH consecutive bytes of its replica's row
            uint8_t* vrow = ((m & 1) ? v0 : v1) + (size_t)r * Np + i0;
            uint2 pend = make_uint2(0u, 0u);  // an 8-spin chunk's bytes held for its neighbour
#pragma unroll
            for (int j = 0; j < NCH; ++j) {
                const int cb = c0 + CH * j;
                float f[CH], xs[CH], ys[CH], ps[CH];
                // the loads in flight together, one wait
                tmem_ld_fxy<CH>(tl + cb, tl + 128 + 2 * cb, f, xs, ys);
#pragma unroll
                for (int k = 0; k < CH; ++k) ps[k] = CONTROL ? pr[CH * j + k] : 0.f;
#pragma unroll
                for (int k = 0; k < CH; k += 2) {
                    float2 x2 = make_float2(xs[k], xs[k + 1]), y2 = make_float2(ys[k], ys[k + 1]);
                    float2 p2 = make_float2(ps[k], ps[k + 1]);
                    sb_update2<CONTROL>(x2, y2, p2, make_float2(f[k], f[k + 1]), a_r, c, dt,
                                        p_shared, inv_rem);
                    xs[k] = x2.x, xs[k + 1] = x2.y, ys[k] = y2.x, ys[k + 1] = y2.y;
                    ps[k] = p2.x, ps[k + 1] = p2.y;
                }
                {
                    float v[2 * CH];
#pragma unroll
                    for (int k = 0; k < CH; ++k) {
                        v[k] = xs[k];
                        v[CH + k] = ys[k];
                    }
                    tmem_st_xy<CH>(tl + 128 + 2 * cb, v);
                }
                if (CONTROL) {
#pragma unroll
                    for (int k = 0; k < CH; ++k) pr[CH * j + k] = ps[k];
                }
                // e4m3 sgn x, 0x38 (+1) or 0xB8 (-1): the sign bit of x + 0 (which
                // turns -0 into +0, so sgn 0 = +1) in the top byte of each word,
                // four gathered per word
                uint32_t b[CH], w[CH / 4];
#pragma unroll
                for (int k = 0; k < CH; k += 2) {
                    const float2 z = __fadd2_rn(make_float2(xs[k], xs[k + 1]), make_float2(0.f, 0.f));
                    b[k] = __float_as_uint(z.x);
                    b[k + 1] = __float_as_uint(z.y);
                }
#pragma unroll
                for (int q = 0; q < CH / 4; ++q) {
                    const uint32_t lo = __byte_perm(b[4 * q], b[4 * q + 1], 0x0073);
                    const uint32_t hi = __byte_perm(b[4 * q + 2], b[4 * q + 3], 0x0073);
                    w[q] = (__byte_perm(lo, hi, 0x5410) & 0x80808080u) | 0x38383838u;
                }
                if constexpr (CH == 16) {
                    *reinterpret_cast<uint4*>(vrow + cb) = make_uint4(w[0], w[1], w[2], w[3]);
                } else {
                    // 8-spin chunks: two neighbours go out as one 16-byte store
                    // where the pair starts on a 16-byte boundary (fewer stores
                    // for the release after the epilogue to wait for)
                    if (((cb >> 3) & 1) == 0) {
                        if (j + 1 < NCH)
                            pend = make_uint2(w[0], w[1]);
                        else
                            *reinterpret_cast<uint2*>(vrow + cb) = make_uint2(w[0], w[1]);
                    } else if (j > 0) {
                        *reinterpret_cast<uint4*>(vrow + cb - 8) =
                            make_uint4(pend.x, pend.y, w[0], w[1]);
                    } else {
                        *reinterpret_cast<uint2*>(vrow + cb) = make_uint2(w[0], w[1]);
                    }
                }
            }
            // The block barrier orders every thread's V bytes before the one
            // release (add or remote arrivals), which is cumulative over them;
            // the readers' TMA loads (async proxy) are ordered after them by the
            // proxy fence each producer issues after its acquire -- one proxy
            // fence on the release/acquire path suffices, none is needed here.
            tmem_wait_st();
            fence_before_sync();
            named_barrier_sync(1, kEpiThreadsP);
            if (*abort_flag) break;
            if (ew == 0) {
                if (lane == 0) {
                    if (PAIR && !leader)
                        mbar_arrive_remote(acce, 0u);
                    else
                        mbar_arrive(acce);
                }
                if (!CLUSTER) {
                    if (lane == 0) red_release_add(ctr, 1u);
                } else if (s + 1 < nsteps && lane < nk) {
                    // this CTA's slice of V(t_{m+1}) is out: lane q tells reader q
                    // (one warp instruction; each lane passed the block barrier,
                    // so each release covers every thread's V bytes)
                    mbar_arrive_remote(&vready[s & 1], (uint32_t)lane);
                }
            }
        }
        // state back to global memory
#pragma unroll 1
        for (int cb = c0; cb < c0 + HW; cb += CH) {
            const size_t o = (size_t)(i0 + cb) * Rp + r;
            float f[CH], xs[CH], ys[CH];
            tmem_ld_fxy<CH>(tl + cb, tl + 128 + 2 * cb, f, xs, ys);
#pragma unroll
            for (int k = 0; k < CH; ++k) {
                x[o + (size_t)k * Rp] = xs[k];
                y[o + (size_t)k * Rp] = ys[k];
            }
        }
        if (CONTROL) {
#pragma unroll
            for (int k = 0; k < HW; ++k) p[(size_t)(i0 + c0 + k) * Rp + r] = pr[k];
        }
    }
    fence_before_sync();
    __syncthreads();
    if (PAIR) {
        // the even CTA's MMAs have written this CTA's TMEM for the last time
        // (its own MMA warp waited for the same commit), and neither CTA
        // releases TMEM or leaves while the other may still use it
        if (!leader && warp == 1) {
            if (lane == 0) mbar_wait(drain, 0, status, kDrainLimitCycles);
            __syncwarp();
        }
        cluster_sync();
    }
    if (warp == 1) {
        fence_after_sync();
        if (PAIR)
            tmem_dealloc_pair(tmem, 512);
        else
            tmem_dealloc(tmem, 512);
    }
    // no CTA leaves while another may still arrive on its barriers
    if (CLUSTER) cluster_sync();
}

// ---------------------------------------------------------------------------
// FX16 (GSB_PREC_FX16): the x coupling with x on the 16-bit fixed-point grid of
// the paper's JX module (Sec. VI, Fig. 2 caption), q = rint(x 2^15), written
// as four signed base-16 digits q = d0 + 16 d1 + 256 d2 + 4096 d3 with
// d0..d2 in [-8, 7] and d3 in [-8, 8]. The planes hold d0, 16 d1, d2, 16 d3 in
// e4m3 (integers of at most four significant bits times a power of two:
// exact), and the pairs share an FP32 accumulator: A0 = J (d0 + 16 d1),
// A1 = J (d2 + 16 d3), every partial sum an integer below
// 136 max_i sum_j |J_ij| < 2^24, exact in any order. The epilogue forms
// A0 + 256 A1 in int32 and rounds 2^-15 times it once: f is the correctly
// rounded J x_q.
//
// Persistent over many steps like k_tc_persist's grid form (cooperative
// launch, a replica-column counter between steps): TMEM holds the two
// accumulators and x, y ([0,128) A0, [128,256) A1, [256,512) x and y of each 16
// spins side by side); p lives in shared memory. A ring stage is one 128-byte
// K atom of J and of the four digit planes (80 KB), two stages.
constexpr int kStagesX = 2;
constexpr int kStageBytesX = 5 * BM * KB;
__host__ __device__ constexpr int smem_bytes_fx16() {
    return 1024 + kStagesX * kStageBytesX + BM * BN * 4 /* p */ + 512;
}

// e4m3 bytes of two small integers of at most four significant bits (exact).
// (float)n for |n| < 2^22 without a conversion instruction: 1.5 2^23 + n lies
// in [2^23, 2^24), where the float's last mantissa bit is worth 1, so its bit
// pattern is that of 1.5 2^23 plus n, and subtracting 1.5 2^23 leaves n exactly.
__device__ __forceinline__ float small_int_to_float(int n) {
    return __fsub_rn(__int_as_float(0x4B400000 + n), 12582912.0f);
}
__device__ __forceinline__ uint32_t e4m3x2(int lo, int hi) {
    return (uint32_t)__nv_cvt_float2_to_fp8x2(
        make_float2(small_int_to_float(lo), small_int_to_float(hi)), __NV_SATFINITE, __NV_E4M3);
}

// The four digit-plane bytes of x: d0, 16 d1, d2, 16 d3 of q = rint(x 2^15).
// With u = q + 0x888 (8 (1 + 16 + 256)), d_k = nibble_k(u) - 8 for k < 3 and
// d3 = u >> 12 (arithmetic), in [-8, 8] for |x| <= 1. q is rounded by adding
// 1.5 2^23 (x 2^15 is exact, |x 2^15| <= 2^15 < 2^22, so the sum's last
// mantissa bits hold the integer, rounded to nearest even like rint) -- an
// FP32 add instead of a conversion instruction.
__device__ __forceinline__ void fx16_digits(float x, int (&d)[4]) {
    const float t = __fadd_rn(x * 32768.0f, 12582912.0f);
    const int u = __float_as_int(t) - 0x4B400000 + 0x888;
    d[0] = (u & 15) - 8;
    d[1] = 16 * (((u >> 4) & 15) - 8);
    d[2] = ((u >> 8) & 15) - 8;
    d[3] = 16 * (u >> 12);
}

template <bool CONTROL>
__global__ void __launch_bounds__(kThreadsP, 1)
    k_fx16_persist(const __grid_constant__ CUtensorMap tmJ, const __grid_constant__ CUtensorMap tmV0,
                   const __grid_constant__ CUtensorMap tmV1, int Np, int Rp,
                   float* __restrict__ x, float* __restrict__ y, float* __restrict__ p,
                   const float* __restrict__ A, uint8_t* __restrict__ v0,
                   uint8_t* __restrict__ v1, float c, float dt,
                   const float* __restrict__ p_sched, int M, int m0, int nsteps,
                   uint32_t* __restrict__ counters, int* status) {
    if (!GSB_DOK(Np > 0 && Np % KB == 0 && Rp % BN == 0 && m0 >= 0 && nsteps >= 0 &&
                     m0 + nsteps <= M && (int)gridDim.x * BN == Rp && (int)gridDim.y * BM == Np,
                 status))
        return;
    constexpr int S = kStagesX;
    constexpr int A1 = BM * KB;  // one K atom of 128 rows
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    float* ps_sh = (float*)(smem + S * kStageBytesX);  // p [128 spins][128 replicas]
    uint64_t* full = (uint64_t*)(ps_sh + BM * BN);
    uint64_t* empty = full + S;
    uint64_t* accf = empty + S;
    uint64_t* acce = accf + 1;
    uint64_t* drain = acce + 1;
    uint32_t* tmem_slot = (uint32_t*)(drain + 1);
    // stage st: J atom, then the four digit-plane atoms
    auto stage = [&](uint32_t st, int q) { return smem + st * kStageBytesX + q * A1; };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = Np / KB;
    const int rb = blockIdx.x, own = blockIdx.y;
    const int i0 = own * BM, r0 = rb * BN;
    uint32_t* ctr = counters + rb;

    if (threadIdx.x == 0) {
        for (int st = 0; st < S; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], 1);
        }
        mbar_init(accf, 1);
        mbar_init(acce, 1);
        mbar_init(drain, 1);
        tmem_slot[1] = 0u;  // epilogue abort flag
        fence_barrier_init();
        tma_prefetch_desc(&tmJ);
        tma_prefetch_desc(&tmV0);
        tma_prefetch_desc(&tmV1);
    }
    if (warp == 1) tmem_alloc(tmem_slot, 512);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t g = 0, armed = 0;
            bool ok = true;
            constexpr uint32_t bytes = 5 * A1;
            for (int s = 0; s < nsteps && ok; ++s) {
                const CUtensorMap* tv = ((m0 + s) & 1) ? &tmV1 : &tmV0;
                const int pre = nk < S ? nk : S;
                // J of the first stages does not depend on the other CTAs
                for (int u = 0; u < pre; ++u) {
                    const uint32_t gg = g + u, st = gg % S, ph = (gg / S) & 1u;
                    if (gg >= (uint32_t)S && !mbar_wait(&empty[st], ph ^ 1u, status)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[st], bytes);
                    tma_load_2d(stage(st, 0), &tmJ, &full[st], u * KB, i0);
                    armed = gg + 1;
                }
                // V(t_m) of the column is complete once its counter reached nk per step
                if (ok && s > 0) {
                    ok = wait_counter(ctr, (uint32_t)nk * (uint32_t)s, status);
                    if (ok) fence_proxy_async();
                }
                // the planes of the stages armed above -- after a failed wait too, so
                // every armed barrier completes its phase (the results are void then)
                for (uint32_t gg = g; gg < armed; ++gg)
                    for (int q = 0; q < 4; ++q)
                        tma_load_2d(stage(gg % S, 1 + q), tv, &full[gg % S], (int)(gg - g) * KB,
                                    q * Rp + r0);
                if (!ok) break;
                for (int u = pre; u < nk; ++u) {
                    const uint32_t gg = g + u, st = gg % S, ph = (gg / S) & 1u;
                    if (gg >= (uint32_t)S && !mbar_wait(&empty[st], ph ^ 1u, status)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[st], bytes);
                    tma_load_2d(stage(st, 0), &tmJ, &full[st], u * KB, i0);
                    for (int q = 0; q < 4; ++q)
                        tma_load_2d(stage(st, 1 + q), tv, &full[st], u * KB, q * Rp + r0);
                    armed = gg + 1;
                }
                g += (uint32_t)nk;
            }
            // no copy is in flight when the CTA leaves
            for (uint32_t gg = armed > (uint32_t)S ? armed - S : 0u; gg < armed; ++gg)
                mbar_wait(&full[gg % S], (gg / S) & 1u, status, kDrainLimitCycles);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_make(0u, BM, BN);
            uint32_t g = 0;
            bool ok = true;
            for (int s = 0; s < nsteps && ok; ++s) {
                if (s > 0 && !mbar_wait(acce, (uint32_t)(s - 1) & 1u, status)) break;
                fence_after_sync();
                for (int u = 0; u < nk; ++u, ++g) {
                    const uint32_t st = g % S, ph = (g / S) & 1u;
                    if (!mbar_wait(&full[st], ph, status)) {
                        ok = false;
                        break;
                    }
                    fence_after_sync();
                    const uint32_t jb = smem_u32(stage(st, 0));
#pragma unroll
                    for (int k = 0; k < KB / 32; ++k) {  // 32 bytes of K per MMA
                        const uint64_t jd = sdesc_sw128(jb + k * 32);
                        const uint32_t first = (u | k) != 0;
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            mma_f8f6f4(tmem + (q >> 1) * 128,
                                       sdesc_sw128(smem_u32(stage(st, 1 + q)) + k * 32), jd, idesc,
                                       (q & 1) ? 1u : first);
                    }
                    mma_commit(&empty[st]);
                }
                if (ok) mma_commit(accf);
            }
            mma_commit(drain);
            mbar_wait(drain, 0, status, kDrainLimitCycles);
        }
    } else {
        const int ew = warp - 2;
        const int quarter = warp & 3;
        const int c0 = (ew >> 2) * 64;
        const int rl = quarter * 32 + lane;  // the thread's replica in the tile (TMEM lane)
        const int r = r0 + rl;
        const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
        const float a_r = CONTROL ? A[r] : 0.f;
        // state of this thread's replica, spins i0 + c0 .. +63: x, y into TMEM, p
        // into shared memory
#pragma unroll 1
        for (int cb = c0; cb < c0 + 64; cb += 16) {
            const size_t o = (size_t)(i0 + cb) * Rp + r;
            float v[16], w[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                v[k] = x[o + (size_t)k * Rp];
                w[k] = y[o + (size_t)k * Rp];
                if (CONTROL) ps_sh[(cb + k) * BN + rl] = p[o + (size_t)k * Rp];
            }
            tmem_st32(tl + 256 + 2 * cb, v, w);
        }
        tmem_wait_st();
        volatile uint32_t* abort_flag = tmem_slot + 1;
        for (int s = 0; s < nsteps; ++s) {
            const int m = m0 + s;
            bool ok = *abort_flag == 0u;
            if (ok) ok = __all_sync(0xffffffffu, mbar_wait(accf, (uint32_t)s & 1u, status));
            if (!ok) {
                *abort_flag = 1u;
                named_barrier_sync(1, kEpiThreadsP);
                break;
            }
            fence_after_sync();
            const float inv_rem = __frcp_rn((float)(M - m));
            const float p_shared = CONTROL ? 0.f : p_sched[s];
            // V(t_{m+1}) goes to buffer (m + 1) & 1: four planes [4][Rp][Np]
            uint8_t* vrow = ((m & 1) ? v0 : v1) + (size_t)r * Np + i0;
            const size_t plane = (size_t)Rp * Np;
#pragma unroll 1
            for (int cb = c0; cb < c0 + 64; cb += 16) {
                float f[16], xs[16], ys[16], ps[16];
                {
                    uint32_t ra[16], rb2[16], rx[16], ry[16];
                    tmem_ld16_async(tl + cb, ra);
                    tmem_ld16_async(tl + 128 + cb, rb2);
                    tmem_ld32_async(tl + 256 + 2 * cb, rx, ry);
#pragma unroll
                    for (int k = 0; k < 16; ++k)
                        ps[k] = CONTROL ? ps_sh[(cb + k) * BN + rl] : 0.f;
                    tmem_wait_ld(ra);
                    tmem_wait_ld(rb2);
                    tmem_wait_ld(rx);
                    tmem_wait_ld(ry);
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        // A0, A1: exact integers below 2^24 in FP32. f = 2^-15 (A0 +
                        // 256 A1) rounded once: one FMA of the exactly scaled terms
                        // (2^-15 A0 and 2^-7 are exact), no conversion instruction
                        f[k] = __fmaf_rn(__uint_as_float(rb2[k]), 0.0078125f,
                                         __uint_as_float(ra[k]) * 3.0517578125e-05f);
                        xs[k] = __uint_as_float(rx[k]);
                        ys[k] = __uint_as_float(ry[k]);
                    }
                }
#pragma unroll
                for (int k = 0; k < 16; k += 2) {
                    float2 x2 = make_float2(xs[k], xs[k + 1]), y2 = make_float2(ys[k], ys[k + 1]);
                    float2 p2 = make_float2(ps[k], ps[k + 1]);
                    sb_update2<CONTROL>(x2, y2, p2, make_float2(f[k], f[k + 1]), a_r, c, dt,
                                        p_shared, inv_rem);
                    xs[k] = x2.x, xs[k + 1] = x2.y, ys[k] = y2.x, ys[k + 1] = y2.y;
                    ps[k] = p2.x, ps[k + 1] = p2.y;
                }
                tmem_st32(tl + 256 + 2 * cb, xs, ys);
                if (CONTROL) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) ps_sh[(cb + k) * BN + rl] = ps[k];
                }
                // the next step's digit planes, 16 bytes of the replica's row each
                uint32_t w[4][4];
#pragma unroll
                for (int k = 0; k < 16; k += 4) {
                    int da[4], db[4], dc[4], dd[4];
                    fx16_digits(xs[k], da);
                    fx16_digits(xs[k + 1], db);
                    fx16_digits(xs[k + 2], dc);
                    fx16_digits(xs[k + 3], dd);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        w[q][k / 4] = e4m3x2(da[q], db[q]) | (e4m3x2(dc[q], dd[q]) << 16);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    *reinterpret_cast<uint4*>(vrow + q * plane + cb) =
                        make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
            }
            tmem_wait_st();
            fence_before_sync();
            named_barrier_sync(1, kEpiThreadsP);
            if (*abort_flag) break;
            if (ew == 0 && lane == 0) {
                mbar_arrive(acce);
                red_release_add(ctr, 1u);
            }
        }
        // state back to global memory
#pragma unroll 1
        for (int cb = c0; cb < c0 + 64; cb += 16) {
            const size_t o = (size_t)(i0 + cb) * Rp + r;
            float v[16];
            tmem_ld16(tl + 256 + 2 * cb, v);
#pragma unroll
            for (int k = 0; k < 16; ++k) x[o + (size_t)k * Rp] = v[k];
            tmem_ld16(tl + 256 + 2 * cb + 16, v);
#pragma unroll
            for (int k = 0; k < 16; ++k) y[o + (size_t)k * Rp] = v[k];
            if (CONTROL) {
#pragma unroll
                for (int k = 0; k < 16; ++k) p[o + (size_t)k * Rp] = ps_sh[(cb + k) * BN + rl];
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        fence_after_sync();
        tmem_dealloc(tmem, 512);
    }
}

// V(t_0) from x(t_0): spin-major x [Np][Rp] -> replica-major operand planes.
template <int KIND>
__global__ void k_tc_prep(const float* __restrict__ x, void* __restrict__ v, int Np, int Rp) {
    __shared__ float tile[32][33];
    const int i0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y)
        tile[k][threadIdx.x] = x[(size_t)(i0 + k) * Rp + r0 + threadIdx.x];
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, i = i0 + threadIdx.x;
        const float xv = tile[threadIdx.x][k];
        const size_t vo = (size_t)r * Np + i;
        if (KIND == 0) {
            reinterpret_cast<uint8_t*>(v)[vo] = e4m3_sign(xv);
        } else if (KIND == 2) {
            int d[4];
            fx16_digits(xv, d);
            uint8_t* vb = reinterpret_cast<uint8_t*>(v);
            const size_t plane = (size_t)Rp * Np;
#pragma unroll
            for (int q = 0; q < 4; ++q) vb[q * plane + vo] = (uint8_t)(e4m3x2(d[q], 0) & 0xFFu);
        } else {
            uint16_t d[4];
            fx32_digit_bits(xv, d);
            uint16_t* vb = reinterpret_cast<uint16_t*>(v);
            const size_t plane = (size_t)Rp * Np;
#pragma unroll
            for (int q = 0; q < 4; ++q) vb[q * plane + vo] = d[q];
        }
    }
}

struct TcState {
    CUtensorMap tmA;
    CUtensorMap tmB[2];
    int vcur = 0;
    int kind = 0;
    bool persistent = false;     // a multi-step kernel runs this shape
    bool cluster = false;        // ... in its cluster form (else the cooperative grid form)
    bool pair = false;           // ... in the grid form on SM pairs
    int bs = BM;                 // spins per CTA of the grid form (128, or 112: more CTAs)
    CUtensorMap tmA_half;        // J in tiles of 64 rows (the pair form)
    CUtensorMap tmA_bs;          // J in tiles of bs rows (the narrow grid form)
    uint32_t* counters = nullptr;  // one per replica block
    float* p_sched = nullptr;      // p(t_{m+1}) for m = 0..M-1 (shared schedule)
};

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 2D K-major tensor map: inner dimension K (contiguous), outer rows; box of
// one 128-byte K slice by 128 rows, 128-byte swizzle.
gsb_status make_map(CUtensorMap* map, const void* base, CUtensorMapDataType dtype, int elem_bytes,
                    uint64_t inner, uint64_t outer, uint32_t box_rows = 128u) {
    auto encode = get_encode();
    if (!encode) return set_error(GSB_ECUDA, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {inner * (cuuint64_t)elem_bytes};
    cuuint32_t box[2] = {(cuuint32_t)(KB / elem_bytes), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1u, 1u};
    CUresult r = encode(map, dtype, 2, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return set_error(GSB_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return GSB_OK;
}

// ---------------------------------------------------------------------------
// FX32 step (one step per launch), with the tile transposed as in k_tc_persist:
// digit plane q of V (x as rint(x 2^30) in four base-256 digits) is the A
// operand, so D_q = V_q J^T lands with a replica per TMEM lane and a spin per
// column, in columns [128 q, 128 q + 128). Each epilogue thread then owns a
// replica: it reads and writes x, y, p coalesced across the warp, holds its
// control strength in a register, and writes the next step's four digit
// planes 32 contiguous bytes at a time. The digit sums are exact integers, so
// f is the same as k_tc_step<1>'s in any order.
// Warps: 0 TMA producer, 1 TMEM owner + MMA issuer, 2-9 epilogue (warp w: TMEM
// lanes 32 (w % 4).., spins 64 ((w - 2) / 4) .. +63 of the tile).
constexpr int kThreadsF = 320;
constexpr int kStagesF = 2;
__host__ __device__ constexpr int smem_bytes_fx32() {
    return 1024 + kStagesF * (4 * BN * KB + BM * KB) + 256;
}

template <bool CONTROL>
__global__ void __launch_bounds__(kThreadsF, 1)
    k_fx32_step(const __grid_constant__ CUtensorMap tmJ, const __grid_constant__ CUtensorMap tmV,
                int Np, int Rp, float* __restrict__ x, float* __restrict__ y,
                float* __restrict__ p, const float* __restrict__ A,
                __nv_bfloat16* __restrict__ vnext, float c, float dt, float p_shared,
                float inv_rem, int* status) {
    if (!GSB_DOK(Np > 0 && Np % (KB / 2) == 0 && Rp % BN == 0 && (int)gridDim.x * BN == Rp &&
                     (int)gridDim.y * BM == Np,
                 status))
        return;
    constexpr int S = kStagesF;
    constexpr int SV1 = BN * KB, SV = 4 * SV1, SJ = BM * KB;  // bytes per stage
    constexpr int kElems = KB / 2;                          // bf16 elements of K per stage
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sV = smem;
    uint8_t* sJ = smem + S * SV;
    uint64_t* full = (uint64_t*)(sJ + S * SJ);
    uint64_t* empty = full + S;
    uint64_t* accf = empty + S;
    uint64_t* drain = accf + 1;  // the MMA issuer's last commit (all its MMAs done)
    uint32_t* tmem_slot = (uint32_t*)(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = blockIdx.x * BN, i0 = blockIdx.y * BM;
    const int nk = Np / kElems;

    if (threadIdx.x == 0) {
        for (int st = 0; st < S; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], 1);
        }
        mbar_init(accf, 1);
        mbar_init(drain, 1);
        fence_barrier_init();
        tma_prefetch_desc(&tmJ);
        tma_prefetch_desc(&tmV);
    }
    if (warp == 1) tmem_alloc(tmem_slot, 512);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    griddep_trigger();  // every CTA of this step is resident: the next may be scheduled
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int armed = 0;
            // J of the first stages does not depend on the previous step: it is
            // requested before the wait for that step, V after it
            const int pre = nk < S ? nk : S;
            for (int kc = 0; kc < pre; ++kc) {
                mbar_arrive_expect_tx(&full[kc], SV + SJ);
                tma_load_2d(sJ + kc * SJ, &tmJ, &full[kc], kc * kElems, i0);
            }
            griddep_wait();
            for (int kc = 0; kc < pre; ++kc) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    tma_load_2d(sV + kc * SV + q * SV1, &tmV, &full[kc], kc * kElems, q * Rp + r0);
                armed = kc + 1;
            }
            for (int kc = pre; kc < nk; ++kc) {
                const int st = kc % S;
                const uint32_t ph = (uint32_t)(kc / S) & 1u;
                if (kc >= S && !mbar_wait(&empty[st], ph ^ 1u, status)) break;
                mbar_arrive_expect_tx(&full[st], SV + SJ);
                tma_load_2d(sJ + st * SJ, &tmJ, &full[st], kc * kElems, i0);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    tma_load_2d(sV + st * SV + q * SV1, &tmV, &full[st], kc * kElems, q * Rp + r0);
                armed = kc + 1;
            }
            // no copy in flight when the CTA leaves
            for (int kc = armed > S ? armed - S : 0; kc < armed; ++kc)
                mbar_wait(&full[kc % S], (uint32_t)(kc / S) & 1u, status, kDrainLimitCycles);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_make(1u, BN, BM);
            bool ok = true;
            for (int kc = 0; kc < nk && ok; ++kc) {
                const int st = kc % S;
                const uint32_t ph = (uint32_t)(kc / S) & 1u;
                if (!mbar_wait(&full[st], ph, status)) {
                    ok = false;
                    break;
                }
                fence_after_sync();
                const uint32_t j0 = smem_u32(sJ + st * SJ);
                const uint32_t v0 = smem_u32(sV + st * SV);
#pragma unroll
                for (int k = 0; k < KB / 32; ++k) {  // 16 bf16 of K per MMA
                    const uint64_t jd = sdesc_sw128(j0 + k * 32);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        mma_f16(tmem + q * BN, sdesc_sw128(v0 + q * SV1 + k * 32), jd, idesc,
                                (kc | k) != 0);
                }
                mma_commit(&empty[st]);
            }
            if (ok) mma_commit(accf);
            // every MMA issued has finished before TMEM is released
            mma_commit(drain);
            mbar_wait(drain, 0, status, kDrainLimitCycles);
        }
    } else {
        const int ew = warp - 2;
        const int quarter = warp & 3;
        const int c0 = (ew >> 2) * 64;
        const int r = r0 + quarter * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
        const float a_r = CONTROL ? A[r] : 0.f;
        const size_t plane = (size_t)Rp * Np;
        __nv_bfloat16* vrow = vnext + (size_t)r * Np + i0;
        // Chunks of 8 spins; the state of the next chunk is loaded while this one
        // is processed (the first before the accumulator is ready), so the L2
        // latency of the loads overlaps work.
        constexpr int CW = 8;
        float xn[CW], yn[CW], pn[CW];
        auto load_state = [&](int cb) {
            const size_t o = (size_t)(i0 + cb) * Rp + r;
#pragma unroll
            for (int k = 0; k < CW; ++k) {
                xn[k] = x[o + (size_t)k * Rp];
                yn[k] = y[o + (size_t)k * Rp];
                pn[k] = CONTROL ? p[o + (size_t)k * Rp] : 0.f;
            }
        };
        // x, y, p and the V buffer written below are the previous step's
        griddep_wait();
        load_state(c0);
        // tcgen05.ld is warp-collective: proceed only if every lane saw the accumulator
        const bool ready = __all_sync(0xffffffffu, mbar_wait(accf, 0, status));
        if (ready) {
            fence_after_sync();
#pragma unroll 1
            for (int cb = c0; cb < c0 + 64; cb += CW) {
                uint32_t d0[CW], d1[CW], d2[CW], d3[CW];
                tmem_ld8_async(tl + cb, d0);
                tmem_ld8_async(tl + BN + cb, d1);
                tmem_ld8_async(tl + 2 * BN + cb, d2);
                tmem_ld8_async(tl + 3 * BN + cb, d3);
                float xs[CW], ys[CW], ps[CW];
#pragma unroll
                for (int k = 0; k < CW; ++k) xs[k] = xn[k], ys[k] = yn[k], ps[k] = pn[k];
                if (cb + CW < c0 + 64) load_state(cb + CW);
                tmem_wait_ld8(d0);
                tmem_wait_ld8(d1);
                tmem_wait_ld8(d2);
                tmem_wait_ld8(d3);
                float f[CW];
#pragma unroll
                for (int k = 0; k < CW; ++k)
                    f[k] = fx32_combine(__uint_as_float(d0[k]), __uint_as_float(d1[k]),
                                        __uint_as_float(d2[k]), __uint_as_float(d3[k]));
#pragma unroll
                for (int k = 0; k < CW; k += 2) {
                    float2 x2 = make_float2(xs[k], xs[k + 1]), y2 = make_float2(ys[k], ys[k + 1]);
                    float2 p2 = make_float2(ps[k], ps[k + 1]);
                    sb_update2<CONTROL>(x2, y2, p2, make_float2(f[k], f[k + 1]), a_r, c, dt,
                                        p_shared, inv_rem);
                    xs[k] = x2.x, xs[k + 1] = x2.y, ys[k] = y2.x, ys[k + 1] = y2.y;
                    ps[k] = p2.x, ps[k + 1] = p2.y;
                }
                const size_t o = (size_t)(i0 + cb) * Rp + r;
#pragma unroll
                for (int k = 0; k < CW; ++k) {
                    x[o + (size_t)k * Rp] = xs[k];
                    y[o + (size_t)k * Rp] = ys[k];
                    if (CONTROL) p[o + (size_t)k * Rp] = ps[k];
                }
                // next step's digit planes: 8 bf16 (16 bytes) of this replica's row each
                uint32_t w[4][CW / 2];
#pragma unroll
                for (int k = 0; k < CW; k += 2) {
                    uint16_t da[4], db[4];
                    fx32_digit_bits(xs[k], da);
                    fx32_digit_bits(xs[k + 1], db);
#pragma unroll
                    for (int q = 0; q < 4; ++q) w[q][k / 2] = (uint32_t)da[q] | ((uint32_t)db[q] << 16);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    *reinterpret_cast<uint4*>(vrow + q * plane + cb) =
                        make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        fence_after_sync();
        tmem_dealloc(tmem, 512);
    }
}

template <int KIND, bool CONTROL>
gsb_status launch_step(gsb_run_state* run, TcState* T, float p_shared, float inv_rem) {
    dim3 grid(run->Rp / BN, run->Np / BM);
    static std::atomic<uint64_t> attr_seen{0};
    if constexpr (KIND == 1) {
        if (first_on_device(attr_seen))
            GSB_CUDA_TRY(cudaFuncSetAttribute(k_fx32_step<CONTROL>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              smem_bytes_fx32()));
        GSB_CUDA_TRY(launch_pdl(k_fx32_step<CONTROL>, grid, dim3(kThreadsF), smem_bytes_fx32(),
                                run->stream, T->tmA, T->tmB[T->vcur], run->Np, run->Rp,
                                run->x[0], run->y, run->p, run->A, run->v16[T->vcur ^ 1], run->c,
                                run->dt, p_shared, inv_rem, run->status));
        GSB_LAUNCH_CHECK("k_fx32_step");
    } else {
        if (first_on_device(attr_seen))
            GSB_CUDA_TRY(cudaFuncSetAttribute(k_tc_step<CONTROL>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              smem_bytes_step()));
        k_tc_step<CONTROL><<<grid, kThreads, smem_bytes_step(), run->stream>>>(
            T->tmA, T->tmB[T->vcur], run->Np, run->Rp, run->x[0], run->y, run->p, run->A,
            run->v8[T->vcur ^ 1], run->c, run->dt, p_shared, inv_rem, run->status);
        GSB_LAUNCH_CHECK("k_tc_step");
    }
    T->vcur ^= 1;
    return GSB_OK;
}

// Pair form: grid (replica blocks, spin blocks), clusters of two replica
// blocks, launched cooperatively (the column counters need the whole grid
// resident).
void pair_config(const gsb_run_state* run, cudaLaunchConfig_t* cfg, cudaLaunchAttribute* at) {
    cfg->gridDim = dim3(run->Rp / BN, run->Np / BM);
    cfg->blockDim = dim3(kThreadsP);
    cfg->dynamicSmemBytes = smem_bytes_persist(kFormPair);
    cfg->stream = run->stream;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeCooperative;
    at[1].val.cooperative = 1;
    cfg->attrs = at;
    cfg->numAttrs = 2;
}

// Cluster form: grid (spin blocks, replica blocks), one cluster per replica block.
void cluster_config(const gsb_run_state* run, cudaLaunchConfig_t* cfg, cudaLaunchAttribute* at) {
    const int nk = run->Np / BM;
    cfg->gridDim = dim3(nk, run->Rp / BN);
    cfg->blockDim = dim3(kThreadsP);
    cfg->dynamicSmemBytes = smem_bytes_persist();
    cfg->stream = run->stream;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = nk;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg->attrs = at;
    cfg->numAttrs = 1;
}

}  // namespace

bool tc_available() { return true; }

const char* tc_kernel_name(const gsb_run_state* run) {
    if (run->path == kPathTcBf16) return "k_bf16_multi";
    const TcState* T = (const TcState*)run->tc;
    if (!T) return "none";
    if (T->kind == 1) return "k_fx32_step";
    if (T->kind == 2) return "k_fx16_persist";
    if (T->persistent)
        return T->cluster ? "k_tc_persist<cluster>"
               : T->pair  ? "k_tc_persist<pair>"
               : T->bs != BM ? "k_tc_persist<grid112>"
                             : "k_tc_persist<grid>";
    return "k_tc_step<e4m3>";
}

gsb_status tc_setup(gsb_run_state* run) {
    if (run->path == kPathTcBf16) return bf16_setup(run);
    const gsb_problem* P = run->prob;
    TcState* T = new TcState();
    run->tc = T;
    T->kind = run->path == kPathTcFp8 ? 0 : (run->path == kPathTcFx16 ? 2 : 1);
    const size_t n = (size_t)run->Np * run->Rp;
    gsb_status st;
    if (T->kind == 0) {
        for (int b = 0; b < 2; ++b) {
            if ((st = dev_alloc(&run->v8[b], n))) return st;
            // zero (e4m3 0): spins past a narrow grid's last block keep this in
            // the buffer the steps write, and their J columns are zero
            GSB_CUDA_TRY(cudaMemsetAsync(run->v8[b], 0, n, run->stream));
        }
        if ((st = make_map(&T->tmA, P->J8, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, P->Np, P->Np))) return st;
        for (int b = 0; b < 2; ++b)
            if ((st = make_map(&T->tmB[b], run->v8[b], CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, run->Np,
                               run->Rp)))
                return st;
    } else if (T->kind == 2) {
        for (int b = 0; b < 2; ++b)
            if ((st = dev_alloc(&run->v8[b], 4 * n))) return st;
        if ((st = make_map(&T->tmA, P->J8, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, P->Np, P->Np))) return st;
        for (int b = 0; b < 2; ++b)
            if ((st = make_map(&T->tmB[b], run->v8[b], CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, run->Np,
                               4 * (uint64_t)run->Rp)))
                return st;
        // persistent grid form only: the whole grid resident at once
        int dev = 0, sms = 0, per_sm = 0, coop = 0;
        GSB_CUDA_TRY(cudaGetDevice(&dev));
        GSB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        GSB_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        auto kern = run->control ? (const void*)k_fx16_persist<true> : (const void*)k_fx16_persist<false>;
        GSB_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          smem_bytes_fx16()));
        GSB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreadsP,
                                                                   smem_bytes_fx16()));
        const int nrb = run->Rp / BN;
        if (!coop || per_sm < 1 || (long)nrb * (run->Np / BM) > (long)per_sm * sms)
            return set_error(GSB_EUNSUPPORTED,
                             "FX16 runs as one cooperative grid of (N/128) x (R/128) CTAs, "
                             "which must fit on the GPU at once");
        if ((st = dev_alloc(&T->counters, (size_t)nrb))) return st;
        T->persistent = true;
    } else {
        for (int b = 0; b < 2; ++b)
            if ((st = dev_alloc(&run->v16[b], 4 * n))) return st;
        if ((st = make_map(&T->tmA, P->J16, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, P->Np, P->Np)))
            return st;
        for (int b = 0; b < 2; ++b)
            if ((st = make_map(&T->tmB[b], run->v16[b], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                               run->Np, 4 * (uint64_t)run->Rp)))
                return st;
    }
    if (T->kind == 0 && run->params.steps_per_launch != 1) {
        // Three multi-step forms. The cluster form (one cluster of Np/128 CTAs
        // per replica block, Np <= 16 x 128) runs in waves when not every
        // cluster fits at once; the grid form and its SM-pair variant need the
        // whole grid co-resident. Take the cluster form if all its clusters fit
        // (its exchange is cheaper), else -- with GSB_RUN_SM_PAIRS -- the pair
        // form if it fits (an even number of replica blocks), else the grid
        // form if it fits, else the cluster form in waves.
        const int nrb = run->Rp / BN;
        int nclusters = 0;
        if (run->Np / BM <= kMaxClusterP) {
            auto kern = run->control ? k_tc_persist<true, kFormCluster> : k_tc_persist<false, kFormCluster>;
            GSB_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              smem_bytes_persist()));
            if (run->Np / BM > 8)
                GSB_CUDA_TRY(
                    cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            cluster_config(run, &cfg, at);
            if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess) {
                cudaGetLastError();
                nclusters = 0;
            }
        }
        bool grid_fits = false, pair_fits = false, narrow_fits = false;
        // the narrow grid form: ceil(N / 112) spin blocks of 112, when that is
        // more CTAs than the 128-wide grid and they are all resident at once
        constexpr int kNarrow = 112;
        const int nsb_narrow = (run->N + kNarrow - 1) / kNarrow;
        {
            int dev = 0, sms = 0, per_sm = 0, coop = 0;
            GSB_CUDA_TRY(cudaGetDevice(&dev));
            GSB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            GSB_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
            auto kern = run->control ? (const void*)k_tc_persist<true, kFormGrid>
                                     : (const void*)k_tc_persist<false, kFormGrid>;
            GSB_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              smem_bytes_persist()));
            GSB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreadsP,
                                                                       smem_bytes_persist()));
            grid_fits = coop && per_sm >= 1 && (long)nrb * (run->Np / BM) <= (long)per_sm * sms;
            if (coop && nsb_narrow > run->Np / BM && nsb_narrow * kNarrow <= run->Np) {
                auto kn = run->control ? (const void*)k_tc_persist<true, kFormGrid, kNarrow>
                                       : (const void*)k_tc_persist<false, kFormGrid, kNarrow>;
                const int sm_n = smem_bytes_persist(kFormGrid, kNarrow);
                int per_sm_n = 0;
                GSB_CUDA_TRY(cudaFuncSetAttribute(kn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  sm_n));
                GSB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_n, kn, kThreadsP,
                                                                           sm_n));
                narrow_fits = per_sm_n >= 1 && (long)nrb * nsb_narrow <= (long)per_sm_n * sms;
            }
            if (coop && nrb % 2 == 0 && (run->params.flags & GSB_RUN_SM_PAIRS)) {
                auto kp = run->control ? k_tc_persist<true, kFormPair> : k_tc_persist<false, kFormPair>;
                GSB_CUDA_TRY(cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  smem_bytes_persist(kFormPair)));
                cudaLaunchConfig_t cfg = {};
                cudaLaunchAttribute at[2];
                pair_config(run, &cfg, at);
                cfg.numAttrs = 1;  // the occupancy query takes the cluster shape only
                int npairs = 0;
                if (cudaOccupancyMaxActiveClusters(&npairs, kp, &cfg) != cudaSuccess) {
                    cudaGetLastError();
                    npairs = 0;
                }
                pair_fits = 2L * npairs >= (long)nrb * (run->Np / BM);
            }
        }
        if (nclusters >= nrb || (nclusters >= 1 && !grid_fits && !pair_fits)) {
            T->persistent = T->cluster = true;
        } else if (pair_fits) {
            T->persistent = T->pair = true;
            if ((st = make_map(&T->tmA_half, P->J8, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, P->Np, P->Np,
                               BM / 2)))
                return st;
            if ((st = dev_alloc(&T->counters, (size_t)nrb))) return st;
        } else if (narrow_fits) {
            T->persistent = true;
            T->bs = kNarrow;
            if ((st = make_map(&T->tmA_bs, P->J8, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, P->Np, P->Np,
                               kNarrow)))
                return st;
            if ((st = dev_alloc(&T->counters, (size_t)nrb))) return st;
        } else if (grid_fits) {
            T->persistent = true;
            if ((st = dev_alloc(&T->counters, (size_t)nrb))) return st;
        }
    }
    if (T->persistent) {
        std::vector<float> ps(run->params.M);
        for (int m = 0; m < run->params.M; ++m) ps[m] = run_p_shared(run, m + 1);
        if ((st = dev_alloc(&T->p_sched, (size_t)run->params.M))) return st;
        GSB_CUDA_TRY(cudaMemcpy(T->p_sched, ps.data(), sizeof(float) * run->params.M,
                                cudaMemcpyHostToDevice));
    }
    return tc_prepare(run);
}

// V(t_0) from the current x (after the initial state is drawn).
gsb_status tc_prepare(gsb_run_state* run) {
    if (run->path == kPathTcBf16) return bf16_prepare(run);
    TcState* T = (TcState*)run->tc;
    dim3 grid(run->Np / 32, run->Rp / 32), block(32, 8);
    // V(t_m) for the run's current step m goes to buffer m & 1: the persistent
    // kernels pick the buffer by the parity of the step, and the one-step
    // kernels start from vcur
    const int b = run->steps_done & 1;
    if (T->kind == 0)
        k_tc_prep<0><<<grid, block, 0, run->stream>>>(run->x[0], run->v8[b], run->Np, run->Rp);
    else if (T->kind == 2)
        k_tc_prep<2><<<grid, block, 0, run->stream>>>(run->x[0], run->v8[b], run->Np, run->Rp);
    else
        k_tc_prep<1><<<grid, block, 0, run->stream>>>(run->x[0], run->v16[b], run->Np, run->Rp);
    GSB_LAUNCH_CHECK("k_tc_prep");
    T->vcur = b;
    return GSB_OK;
}

// Persistent launch over steps [m0, m0 + n), one CTA per tile: in clusters
// (one per replica block) or cooperative.
template <bool CONTROL>
gsb_status launch_persist(gsb_run_state* run, TcState* T, int m0, int n) {
    int Np = run->Np, Rp = run->Rp, M = run->params.M;
    float c = run->c, dt = run->dt;
    const float* ps = T->p_sched + m0;
    if (T->kind == 2) {
        const int nrb = run->Rp / BN;
        GSB_CUDA_TRY(cudaMemsetAsync(T->counters, 0, sizeof(uint32_t) * nrb, run->stream));
        dim3 grid(nrb, run->Np / BM);
        void* args[] = {(void*)&T->tmA, (void*)&T->tmB[0], (void*)&T->tmB[1], &Np, &Rp,
                        (void*)&run->x[0], (void*)&run->y, (void*)&run->p, (void*)&run->A,
                        (void*)&run->v8[0], (void*)&run->v8[1], &c, &dt, (void*)&ps, &M, &m0, &n,
                        (void*)&T->counters, (void*)&run->status};
        GSB_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_fx16_persist<CONTROL>, grid,
                                                 dim3(kThreadsP), args, smem_bytes_fx16(),
                                                 run->stream));
    } else if (T->pair) {
        const int nrb = run->Rp / BN;
        GSB_CUDA_TRY(cudaMemsetAsync(T->counters, 0, sizeof(uint32_t) * nrb, run->stream));
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[2];
        pair_config(run, &cfg, at);
        GSB_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_tc_persist<CONTROL, kFormPair>, T->tmA_half,
                                        T->tmB[0], T->tmB[1], Np, Rp, run->x[0], run->y, run->p,
                                        (const float*)run->A, run->v8[0], run->v8[1], c, dt, ps, M,
                                        m0, n, T->counters, run->status));
    } else if (T->cluster) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        cluster_config(run, &cfg, at);
        GSB_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_tc_persist<CONTROL, kFormCluster>, T->tmA, T->tmB[0],
                                        T->tmB[1], Np, Rp, run->x[0], run->y, run->p,
                                        (const float*)run->A, run->v8[0], run->v8[1], c, dt, ps, M,
                                        m0, n, (uint32_t*)nullptr, run->status));
    } else if (T->bs != BM) {
        const int nrb = run->Rp / BN;
        GSB_CUDA_TRY(cudaMemsetAsync(T->counters, 0, sizeof(uint32_t) * nrb, run->stream));
        dim3 grid(nrb, (run->N + T->bs - 1) / T->bs);
        void* args[] = {(void*)&T->tmA_bs, (void*)&T->tmB[0], (void*)&T->tmB[1], &Np, &Rp,
                        (void*)&run->x[0], (void*)&run->y, (void*)&run->p, (void*)&run->A,
                        (void*)&run->v8[0], (void*)&run->v8[1], &c, &dt, (void*)&ps, &M, &m0, &n,
                        (void*)&T->counters, (void*)&run->status};
        GSB_CUDA_TRY(cudaLaunchCooperativeKernel(
            (const void*)k_tc_persist<CONTROL, kFormGrid, 112>, grid, dim3(kThreadsP), args,
            smem_bytes_persist(kFormGrid, 112), run->stream));
    } else {
        const int nrb = run->Rp / BN;
        GSB_CUDA_TRY(cudaMemsetAsync(T->counters, 0, sizeof(uint32_t) * nrb, run->stream));
        dim3 grid(nrb, run->Np / BM);
        void* args[] = {(void*)&T->tmA, (void*)&T->tmB[0], (void*)&T->tmB[1], &Np, &Rp,
                        (void*)&run->x[0], (void*)&run->y, (void*)&run->p, (void*)&run->A,
                        (void*)&run->v8[0], (void*)&run->v8[1], &c, &dt, (void*)&ps, &M, &m0, &n,
                        (void*)&T->counters, (void*)&run->status};
        GSB_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_tc_persist<CONTROL, kFormGrid>, grid,
                                                 dim3(kThreadsP), args, smem_bytes_persist(),
                                                 run->stream));
    }
    count_launch();
    T->vcur = (m0 + n) & 1;
    return GSB_OK;
}

gsb_status tc_steps(gsb_run_state* run, int m0, int nsteps) {
    if (run->path == kPathTcBf16) return bf16_steps(run, m0, nsteps);
    TcState* T = (TcState*)run->tc;
    if (T->persistent) {
        // one launch per stretch of steps between energy evaluations
        int m = m0;
        const int end = m0 + nsteps;
        const int spl = run->params.steps_per_launch;
        while (m < end) {
            int stop = end;
            for (int k = m + 1; k <= end; ++k)
                if (run_is_eval_step(run, k)) {
                    stop = k;
                    break;
                }
            if (spl > 0 && stop - m > spl) stop = m + spl;
            gsb_status st = prof_begin(run);
            if (st != GSB_OK) return st;
            st = run->control ? launch_persist<true>(run, T, m, stop - m)
                              : launch_persist<false>(run, T, m, stop - m);
            if (st != GSB_OK) return st;
            if ((st = prof_end(run, stop - m)) != GSB_OK) return st;
            m = stop;
            if (run_is_eval_step(run, m))
                if ((st = run_evaluate(run, m)) != GSB_OK) return st;
        }
        return GSB_OK;
    }
    for (int m = m0; m < m0 + nsteps; ++m) {
        const float p_shared = run_p_shared(run, m + 1);
        const float inv_rem = 1.0f / (float)(run->params.M - m);
        gsb_status st = prof_begin(run);
        if (st != GSB_OK) return st;
        if (T->kind == 0)
            st = run->control ? launch_step<0, true>(run, T, p_shared, inv_rem)
                              : launch_step<0, false>(run, T, p_shared, inv_rem);
        else
            st = run->control ? launch_step<1, true>(run, T, p_shared, inv_rem)
                              : launch_step<1, false>(run, T, p_shared, inv_rem);
        if (st != GSB_OK) return st;
        if ((st = prof_end(run, 1)) != GSB_OK) return st;
        if (run_is_eval_step(run, m + 1))
            if ((st = run_evaluate(run, m + 1)) != GSB_OK) return st;
    }
    return GSB_OK;
}

// Debug build: the FP8 energy kernel on a grid of two spin blocks over a
// 128-spin matrix; its entry check must return before any barrier, copy or
// MMA (the tensor maps are empty and the pointers null: nothing may touch them).
gsb_status tc_debug_selftest(int* status, cudaStream_t s) {
#ifndef GSB_DEBUG
    // the release kernel has no check: it must never see this launch
    (void)status;
    (void)s;
    return set_error(GSB_EUNSUPPORTED, "built without GSB_DEBUG");
#else
    CUtensorMap empty_map;
    memset(&empty_map, 0, sizeof(empty_map));
    GSB_CUDA_TRY(cudaFuncSetAttribute(k_tc_energy, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      smem_bytes_step()));
    k_tc_energy<<<dim3(1, 2), kThreads, smem_bytes_step(), s>>>(empty_map, empty_map, nullptr, BM,
                                                                 nullptr, status);
    GSB_LAUNCH_CHECK("k_tc_energy");
    GSB_CUDA_TRY(cudaStreamSynchronize(s));
    return GSB_OK;
#endif
}

gsb_status tc_energy(gsb_run_state* run, int step) {
    GSB_CUDA_TRY(cudaMemsetAsync(run->e_acc, 0, sizeof(double) * run->Rp, run->stream));
    const TcState* T = (const TcState*)run->tc;
    if (run->path == kPathTcFp8 && T) {
        // sgn x(t_step) is the e4m3 operand the steps left in buffer step & 1
        const int b = step & 1;
        static std::atomic<uint64_t> attr_seen{0};
        if (first_on_device(attr_seen))
            GSB_CUDA_TRY(cudaFuncSetAttribute(k_tc_energy, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              smem_bytes_step()));
        dim3 grid(run->Rp / BN, run->Np / BM);
        k_tc_energy<<<grid, kThreads, smem_bytes_step(), run->stream>>>(
            T->tmA, T->tmB[b], run->v8[b], run->Np, run->e_acc, run->status);
        GSB_LAUNCH_CHECK("k_tc_energy");
        return GSB_OK;
    }
    return launch_dense_f32_energy(run->prob, run->x[0], run->Rp, run->e_acc, run->e_part,
                                   run->stream);
}

void tc_free(gsb_run_state* run) {
    if (run->path == kPathTcBf16) return bf16_free(run);
    TcState* T = (TcState*)run->tc;
    if (T) {
        dev_free(T->counters);
        dev_free(T->p_sched);
    }
    delete T;
    run->tc = nullptr;
}

}  // namespace gsb
