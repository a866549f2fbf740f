// k_bf16.cu -- the coupling of real-valued J on the tensor cores, and many
// instances of uneven size in one persistent launch.
//
// Split-bf16 form (GSB_PREC_BF16X3): J = J_hi + J_lo and x = x_hi + x_lo, each
// term the bf16 rounding of what the terms before it leave, so every pair
// holds 16 significant bits. The coupling F = J v is accumulated in FP32 in
// TMEM as J_hi x_hi + J_hi x_lo + J_lo x_hi (three tcgen05 kind::f16 MMAs per
// K slice; the J_lo x_lo term, at most 2^-16 of |J_ij x_j|, is left out), and
// J_hi s + J_lo s for the sgn coupling, whose +-1 operand is exact in bf16.
// Each product is exact; the error against FP64 is at most about 3 2^-16 of
// sum_j |J_ij v_j| (the two splits' residues, 2^-17 each, and the term left
// out) plus the tensor core's FP32 accumulation.
//
// One kernel serves a single run and a batch of instances: it walks a work
// list of items (step, tile), a tile being 128 spins x 128 replicas of one
// instance, in a fixed global order (step-major within a launch). CTA b of G
// takes items b, b + G, ... (a cooperative launch, so every CTA is resident:
// an item waits only for items that precede it in the order, so the earliest
// unfinished item can always proceed). Before it loads the V operand of step
// s of instance k, an item waits for k's counter to show every tile of step
// s - 1 done; the epilogue counts its tile (release) after its state and V
// stores. State x, y, p lives in global memory (L2) between items; V(t_m) is
// double-buffered by the parity of m. The accumulator is double-buffered in
// TMEM so that one item's MMAs run while the previous item's epilogue reads
// its F. Every tile of a step sums over K in the same order, so an instance
// follows the same trajectory alone or in a batch, whatever the schedule.
//
// Warps: 0 TMA producer, 1 TMEM owner + MMA issuer, 2-9 epilogue (warp w
// reads TMEM lanes 32 (w % 4).. -- its 32 replicas -- and columns
// 64 ((w - 2) / 4) .. +63 -- 64 spins of the tile).
#include <cudaTypedefs.h>

#include <string.h>

#include <algorithm>
#include <vector>

#include "gsb_update.cuh"
#include "tc_ptx.cuh"

namespace gsb {

namespace {

using namespace tc;

constexpr int kT = 128;          // spins and replicas per tile
constexpr int kKB = 128;         // bytes of K per atom (64 bf16)
constexpr int kElems = kKB / 2;  // bf16 elements of K per atom
constexpr int kAtom = kT * kKB;  // bytes of one 128-row atom (16 KB)
constexpr int kThreadsM = 320;
constexpr int kEpiThreadsM = 256;
constexpr int kStagesM = 3;
constexpr int kStageBytesM = 4 * kAtom;  // J_hi, J_lo, V_hi, V_lo
constexpr int kSmemM = 1024 + kStagesM * kStageBytesM + 256;

struct MInst {  // aligned as its CUtensorMap members require
    CUtensorMap tmJ[2];  // J_hi, J_lo: [Np][Np] bf16, boxes of 64 elements x 128 rows
    CUtensorMap tmV[2];  // V(t_m), m even / odd: [planes x Rp][Np] bf16, same boxes
    float* x;
    float* y;
    float* p;
    const float* A;
    __nv_bfloat16* v[2];
    const float* p_sched;  // p(t_{m+1}) at [m], m = 0..M-1 (shared schedule)
    int* status;           // the run's status word
    int Np, Rp, M;
    int m0;     // the instance's step when the launch starts
    int stop;   // the launch advances it to this step
    int tiles;  // tiles of the instance in the launch's list
    int flags;  // 1: sgn coupling, 2: individual control (Eq. 7)
    float c, dt;
};

struct MTile {
    int inst, i0, r0, pad;
};

// The epilogue of the resident form: this CTA's one tile, its state in TMEM.
// Per step: F from TMEM, Eqs. 7, 3, 4, 5 in the order of sb_update2, x, y, p
// back to TMEM, the next step's operand planes to global memory; then the
// accumulator is released and the instance's counter advanced.
__device__ __forceinline__ void bf16_res_epilogue(const MInst* __restrict__ insts,
                                                  const MTile* __restrict__ tiles, int ntiles,
                                                  long nitems, long G, uint32_t* counters,
                                                  int* status, uint32_t tmem, uint32_t* tmem_slot,
                                                  uint64_t* accf, uint64_t* acce, int warp,
                                                  int lane) {
    const int ew = warp - 2;
    const int quarter = warp & 3;
    const int c0 = (ew >> 2) * 64;
    const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
    volatile uint32_t* abort_flag = tmem_slot + 1;
    const MTile T = tiles[blockIdx.x % ntiles];
    const MInst* I = insts + T.inst;
    const int Np = I->Np, Rp = I->Rp;
    const bool sign = I->flags & 1, control = I->flags & 2;
    const float c = I->c, dt = I->dt;
    float* __restrict__ x = I->x;
    float* __restrict__ y = I->y;
    float* __restrict__ p = I->p;
    const int r = T.r0 + quarter * 32 + lane;
    const float a_r = control ? I->A[r] : 0.f;
    const size_t plane = (size_t)Rp * Np;
    // the tile's state into TMEM
#pragma unroll 1
    for (int cb = c0; cb < c0 + 64; cb += 16) {
        const size_t o = (size_t)(T.i0 + cb) * Rp + r;
        float v[16], w[16], q[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            v[k] = x[o + (size_t)k * Rp];
            w[k] = y[o + (size_t)k * Rp];
            q[k] = control ? p[o + (size_t)k * Rp] : 0.f;
        }
        tmem_st32(tl + 128 + 2 * cb, v, w);
        tmem_st16(tl + 384 + cb, q);
    }
    tmem_wait_st();
    uint32_t n = 0;
    for (long j = blockIdx.x; j < nitems; j += G) {
        const int s = (int)(j / ntiles);
        const int m = I->m0 + s;
        if (m >= I->stop) continue;
        bool ok = *abort_flag == 0u;
        if (ok) ok = __all_sync(0xffffffffu, mbar_wait(&accf[0], n & 1u, status));
        if (!ok) {
            *abort_flag = 1u;
            named_barrier_sync(1, kEpiThreadsM);
            break;
        }
        fence_after_sync();
        const float inv_rem = __frcp_rn((float)(I->M - m));
        const float p_shared = control ? 0.f : I->p_sched[m];
        uint16_t* vrow = reinterpret_cast<uint16_t*>(I->v[(m + 1) & 1]) + (size_t)r * Np + T.i0;
#pragma unroll 1
        for (int cb = c0; cb < c0 + 64; cb += 16) {
            float f[16], xs[16], ys[16], ps[16];
            {
                uint32_t rf[16], rx[16], ry[16], rq[16];
                tmem_ld16_async(tl + cb, rf);
                tmem_ld32_async(tl + 128 + 2 * cb, rx, ry);
                tmem_ld16_async(tl + 384 + cb, rq);
                tmem_wait_ld(rf);
                tmem_wait_ld(rx);
                tmem_wait_ld(ry);
                tmem_wait_ld(rq);
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    f[k] = __uint_as_float(rf[k]);
                    xs[k] = __uint_as_float(rx[k]);
                    ys[k] = __uint_as_float(ry[k]);
                    ps[k] = __uint_as_float(rq[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < 16; k += 2) {
                float2 x2 = make_float2(xs[k], xs[k + 1]), y2 = make_float2(ys[k], ys[k + 1]);
                float2 p2 = make_float2(ps[k], ps[k + 1]);
                const float2 f2 = make_float2(f[k], f[k + 1]);
                if (control)
                    sb_update2<true>(x2, y2, p2, f2, a_r, c, dt, p_shared, inv_rem);
                else
                    sb_update2<false>(x2, y2, p2, f2, a_r, c, dt, p_shared, inv_rem);
                xs[k] = x2.x, xs[k + 1] = x2.y, ys[k] = y2.x, ys[k + 1] = y2.y;
                ps[k] = p2.x, ps[k + 1] = p2.y;
            }
            tmem_st32(tl + 128 + 2 * cb, xs, ys);
            tmem_st16(tl + 384 + cb, ps);
            // next step's operand planes, 16 bf16 (32 bytes) of the replica's row each
            uint32_t hi[8], lo[8];
#pragma unroll
            for (int k = 0; k < 16; k += 2) {
                if (sign) {
                    hi[k / 2] = (xs[k] >= 0.f ? 0x3F80u : 0xBF80u) |
                                ((xs[k + 1] >= 0.f ? 0x3F80u : 0xBF80u) << 16);
                    lo[k / 2] = 0u;
                } else {
                    uint32_t h0, l0, h1, l1;
                    bf16_split_bits(xs[k], h0, l0);
                    bf16_split_bits(xs[k + 1], h1, l1);
                    hi[k / 2] = h0 | (h1 << 16);
                    lo[k / 2] = l0 | (l1 << 16);
                }
            }
            *reinterpret_cast<uint4*>(vrow + cb) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4*>(vrow + cb + 8) = make_uint4(hi[4], hi[5], hi[6], hi[7]);
            if (!sign) {
                *reinterpret_cast<uint4*>(vrow + plane + cb) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                *reinterpret_cast<uint4*>(vrow + plane + cb + 8) =
                    make_uint4(lo[4], lo[5], lo[6], lo[7]);
            }
        }
        // the block barrier orders every thread's F reads and V stores before
        // the one release; readers acquire the counter
        tmem_wait_st();
        fence_before_sync();
        named_barrier_sync(1, kEpiThreadsM);
        if (*abort_flag) break;
        if (ew == 0 && lane == 0) {
            mbar_arrive(&acce[0]);
            red_release_add(counters + T.inst, 1u);
        }
        ++n;
    }
    // state back to global memory
#pragma unroll 1
    for (int cb = c0; cb < c0 + 64; cb += 16) {
        const size_t o = (size_t)(T.i0 + cb) * Rp + r;
        float v[16];
        tmem_ld16(tl + 128 + 2 * cb, v);
#pragma unroll
        for (int k = 0; k < 16; ++k) x[o + (size_t)k * Rp] = v[k];
        tmem_ld16(tl + 128 + 2 * cb + 16, v);
#pragma unroll
        for (int k = 0; k < 16; ++k) y[o + (size_t)k * Rp] = v[k];
        if (control) {
            tmem_ld16(tl + 384 + cb, v);
#pragma unroll
            for (int k = 0; k < 16; ++k) p[o + (size_t)k * Rp] = v[k];
        }
    }
}

// RES (resident form): launched with one CTA per tile (grid == ntiles), so the
// item loop gives every CTA the same tile each step; its x, y, p stay in TMEM
// for the whole launch (columns 128..383 x and y of each 16 spins side by
// side, 384..511 p; one accumulator at 0..127) and cross global memory only at
// the launch's start and end. Without RES the tiles of a step are spread over
// the CTAs round robin and the state goes through L2 every step (two
// accumulators for overlap across items).
template <bool RES>
__global__ void __launch_bounds__(kThreadsM, 1)
    k_bf16_multi(const MInst* __restrict__ insts, const MTile* __restrict__ tiles, int ntiles,
                 int nsteps, uint32_t* __restrict__ counters, int ninst, int* __restrict__ status) {
    constexpr int S = kStagesM;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + S * kStageBytesM);
    uint64_t* empty = full + S;
    uint64_t* accf = empty + S;  // [2]
    uint64_t* acce = accf + 2;   // [2]
    uint64_t* drain = acce + 2;
    uint32_t* tmem_slot = (uint32_t*)(drain + 1);
    // stage st: J_hi atom, J_lo atom, V_hi atom, V_lo atom
    auto stage = [&](uint32_t st, int q) { return smem + st * kStageBytesM + q * kAtom; };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long nitems = (long)nsteps * ntiles;
    const long G = gridDim.x;
#ifdef GSB_DEBUG
    // debug build: every tile of the list names an instance of the batch and a
    // whole 128 x 128 tile of it, and every instance's steps lie within its run
    // (the whole list, checked alike by every CTA before any barrier: a
    // uniform return)
    {
        int bad = 0;
        for (int k = threadIdx.x; k < ntiles; k += blockDim.x) {
            const MTile T = tiles[k];
            if (T.inst < 0 || T.inst >= ninst) {
                bad = 1;
                continue;
            }
            const MInst* I = insts + T.inst;
            bad |= !(T.i0 >= 0 && T.r0 >= 0 && T.i0 % kT == 0 && T.r0 % kT == 0 &&
                     T.i0 < I->Np && T.r0 < I->Rp && I->Np % kT == 0 && I->Rp % kT == 0 &&
                     I->m0 >= 0 && I->m0 <= I->stop && I->stop <= I->M);
        }
        if (__syncthreads_or(bad)) {
            GSB_DOK(false, status);
            return;
        }
    }
#endif

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
    if (warp == 1) tmem_alloc(tmem_slot, RES ? 512 : 256);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t g = 0, armed = 0;
            bool ok = true;
            for (long j = blockIdx.x; j < nitems && ok; j += G) {
                const int s = (int)(j / ntiles);
                const MTile T = tiles[j % ntiles];
                const MInst* I = insts + T.inst;
                const int m = I->m0 + s;
                if (m >= I->stop) continue;
                const int nk = I->Np / kElems;
                const int planes = (I->flags & 1) ? 1 : 2;
                const uint32_t bytes = (uint32_t)((2 + planes) * kAtom);
                const CUtensorMap* tv = &I->tmV[m & 1];
                const int pre = nk < S ? nk : S;
                // J of the first stages does not depend on the previous step
                for (int u = 0; u < pre; ++u) {
                    const uint32_t gg = g + u, st = gg % S, ph = (gg / S) & 1u;
                    if (gg >= (uint32_t)S && !mbar_wait(&empty[st], ph ^ 1u, status)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[st], bytes);
                    tma_load_2d(stage(st, 0), &I->tmJ[0], &full[st], u * kElems, T.i0);
                    tma_load_2d(stage(st, 1), &I->tmJ[1], &full[st], u * kElems, T.i0);
                    armed = gg + 1;
                }
                // V(t_m) is complete once every tile of step m - 1 counted itself
                if (ok && s > 0) {
                    ok = wait_counter(counters + T.inst, (uint32_t)I->tiles * (uint32_t)s, status);
                    if (ok) fence_proxy_async();
                }
                // V of the stages armed above -- after a failed wait too, so every
                // armed barrier completes its phase (the results are void then)
                for (uint32_t gg = g; gg < armed; ++gg) {
                    const int u = (int)(gg - g);
                    for (int q = 0; q < planes; ++q)
                        tma_load_2d(stage(gg % S, 2 + q), tv, &full[gg % S], u * kElems,
                                    q * I->Rp + T.r0);
                }
                if (!ok) break;
                for (int u = pre; u < nk; ++u) {
                    const uint32_t gg = g + u, st = gg % S, ph = (gg / S) & 1u;
                    if (gg >= (uint32_t)S && !mbar_wait(&empty[st], ph ^ 1u, status)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[st], bytes);
                    tma_load_2d(stage(st, 0), &I->tmJ[0], &full[st], u * kElems, T.i0);
                    tma_load_2d(stage(st, 1), &I->tmJ[1], &full[st], u * kElems, T.i0);
                    for (int q = 0; q < planes; ++q)
                        tma_load_2d(stage(st, 2 + q), tv, &full[st], u * kElems, q * I->Rp + T.r0);
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
            constexpr uint32_t idesc = idesc_make(1u, kT, kT);
            uint32_t g = 0, n = 0;
            bool ok = true;
            for (long j = blockIdx.x; j < nitems && ok; j += G) {
                const int s = (int)(j / ntiles);
                const MTile T = tiles[j % ntiles];
                const MInst* I = insts + T.inst;
                if (I->m0 + s >= I->stop) continue;
                const int nk = I->Np / kElems;
                const bool xc = !(I->flags & 1);
                const uint32_t b = RES ? 0u : n & 1u;
                // the epilogue has read this accumulator's previous item
                if (RES ? (n >= 1 && !mbar_wait(&acce[0], (n - 1) & 1u, status))
                        : (n >= 2 && !mbar_wait(&acce[b], ((n - 2) >> 1) & 1u, status)))
                    break;
                fence_after_sync();
                const uint32_t d = tmem + 128u * b;
                for (int u = 0; u < nk; ++u, ++g) {
                    const uint32_t st = g % S, ph = (g / S) & 1u;
                    if (!mbar_wait(&full[st], ph, status)) {
                        ok = false;
                        break;
                    }
                    fence_after_sync();
                    const uint32_t jh = smem_u32(stage(st, 0)), jl = smem_u32(stage(st, 1));
                    const uint32_t vh = smem_u32(stage(st, 2)), vl = smem_u32(stage(st, 3));
#pragma unroll
                    for (int k = 0; k < kKB / 32; ++k) {  // 16 bf16 of K per MMA
                        const uint64_t ah = sdesc_sw128(vh + k * 32);
                        mma_f16(d, ah, sdesc_sw128(jh + k * 32), idesc, (u | k) != 0);
                        mma_f16(d, ah, sdesc_sw128(jl + k * 32), idesc, 1u);
                        if (xc) mma_f16(d, sdesc_sw128(vl + k * 32), sdesc_sw128(jh + k * 32), idesc, 1u);
                    }
                    mma_commit(&empty[st]);
                }
                if (!ok) break;
                mma_commit(&accf[b]);
                ++n;
            }
            // every MMA issued has finished before TMEM is released
            mma_commit(drain);
            mbar_wait(drain, 0, status, kDrainLimitCycles);
        }
    } else if (RES) {
        bf16_res_epilogue(insts, tiles, ntiles, nitems, G, counters, status, tmem, tmem_slot, accf,
                          acce, warp, lane);
    } else {
        const int ew = warp - 2;
        const int quarter = warp & 3;
        const int c0 = (ew >> 2) * 64;
        const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
        volatile uint32_t* abort_flag = tmem_slot + 1;
        uint32_t n = 0;
        for (long j = blockIdx.x; j < nitems; j += G) {
            const int s = (int)(j / ntiles);
            const MTile T = tiles[j % ntiles];
            const MInst* I = insts + T.inst;
            const int m = I->m0 + s;
            if (m >= I->stop) continue;
            const uint32_t b = n & 1u;
            bool ok = *abort_flag == 0u;
            if (ok) ok = __all_sync(0xffffffffu, mbar_wait(&accf[b], (n >> 1) & 1u, status));
            // the state of this tile was written by another CTA's item of step s - 1:
            // acquire that step's completion (already reached) before reading it
            if (ok && s > 0) {
                if (lane == 0)
                    ok = wait_counter(counters + T.inst, (uint32_t)I->tiles * (uint32_t)s, status);
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            }
            __syncwarp();
            if (!ok) {
                *abort_flag = 1u;
                named_barrier_sync(1, kEpiThreadsM);
                break;
            }
            fence_after_sync();
            const int Np = I->Np, Rp = I->Rp;
            const bool sign = I->flags & 1, control = I->flags & 2;
            const float c = I->c, dt = I->dt;
            float* __restrict__ x = I->x;
            float* __restrict__ y = I->y;
            float* __restrict__ p = I->p;
            const int r = T.r0 + quarter * 32 + lane;
            const float a_r = control ? I->A[r] : 0.f;
            const float inv_rem = __frcp_rn((float)(I->M - m));
            const float p_shared = control ? 0.f : I->p_sched[m];
            __nv_bfloat16* vout = I->v[(m + 1) & 1];
            const size_t plane = (size_t)Rp * Np;
            uint16_t* vrow = reinterpret_cast<uint16_t*>(vout) + (size_t)r * Np + T.i0;
            const uint32_t ta = tl + 128u * b;
            // chunks of 8 spins; the state is loaded two chunks ahead (two register
            // buffers in turn), so the L2 latency of the loads -- the epilogue's
            // bound when only one chunk was in flight -- overlaps the work
            constexpr int CW = 8;
            float xa[CW], ya[CW], pa[CW], xb[CW], yb[CW], pb[CW];
            auto load_state = [&](int cb, float (&xq)[CW], float (&yq)[CW], float (&pq)[CW]) {
                const size_t o = (size_t)(T.i0 + cb) * Rp + r;
#pragma unroll
                for (int k = 0; k < CW; ++k) {
                    xq[k] = x[o + (size_t)k * Rp];
                    yq[k] = y[o + (size_t)k * Rp];
                    pq[k] = control ? p[o + (size_t)k * Rp] : 0.f;
                }
            };
            load_state(c0, xa, ya, pa);
            load_state(c0 + CW, xb, yb, pb);
            auto chunk = [&](int cb, float (&xq)[CW], float (&yq)[CW], float (&pq)[CW]) {
                uint32_t rf[CW];
                tmem_ld8_async(ta + cb, rf);
                float xs[CW], ys[CW], ps[CW];
#pragma unroll
                for (int k = 0; k < CW; ++k) xs[k] = xq[k], ys[k] = yq[k], ps[k] = pq[k];
                if (cb + 2 * CW < c0 + 64) load_state(cb + 2 * CW, xq, yq, pq);
                tmem_wait_ld8(rf);
#pragma unroll
                for (int k = 0; k < CW; k += 2) {
                    float2 x2 = make_float2(xs[k], xs[k + 1]), y2 = make_float2(ys[k], ys[k + 1]);
                    float2 p2 = make_float2(ps[k], ps[k + 1]);
                    const float2 f2 = make_float2(__uint_as_float(rf[k]), __uint_as_float(rf[k + 1]));
                    if (control)
                        sb_update2<true>(x2, y2, p2, f2, a_r, c, dt, p_shared, inv_rem);
                    else
                        sb_update2<false>(x2, y2, p2, f2, a_r, c, dt, p_shared, inv_rem);
                    xs[k] = x2.x, xs[k + 1] = x2.y, ys[k] = y2.x, ys[k + 1] = y2.y;
                    ps[k] = p2.x, ps[k + 1] = p2.y;
                }
                const size_t o = (size_t)(T.i0 + cb) * Rp + r;
#pragma unroll
                for (int k = 0; k < CW; ++k) {
                    x[o + (size_t)k * Rp] = xs[k];
                    y[o + (size_t)k * Rp] = ys[k];
                    if (control) p[o + (size_t)k * Rp] = ps[k];
                }
                // next step's operand planes, 8 bf16 (16 bytes) of the replica's row each
                uint32_t hi[CW / 2], lo[CW / 2];
#pragma unroll
                for (int k = 0; k < CW; k += 2) {
                    if (sign) {
                        hi[k / 2] = (xs[k] >= 0.f ? 0x3F80u : 0xBF80u) |
                                    ((xs[k + 1] >= 0.f ? 0x3F80u : 0xBF80u) << 16);
                        lo[k / 2] = 0u;
                    } else {
                        uint32_t h0, l0, h1, l1;
                        bf16_split_bits(xs[k], h0, l0);
                        bf16_split_bits(xs[k + 1], h1, l1);
                        hi[k / 2] = h0 | (h1 << 16);
                        lo[k / 2] = l0 | (l1 << 16);
                    }
                }
                *reinterpret_cast<uint4*>(vrow + cb) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                if (!sign)
                    *reinterpret_cast<uint4*>(vrow + plane + cb) =
                        make_uint4(lo[0], lo[1], lo[2], lo[3]);
            };
#pragma unroll 1
            for (int cb = c0; cb < c0 + 64; cb += 2 * CW) {
                chunk(cb, xa, ya, pa);
                chunk(cb + CW, xb, yb, pb);
            }
            // the block barrier orders every thread's F reads and its state and V
            // stores before the one release; readers acquire the counter
            fence_before_sync();
            named_barrier_sync(1, kEpiThreadsM);
            if (*abort_flag) break;
            if (ew == 0 && lane == 0) {
                mbar_arrive(&acce[b]);
                red_release_add(counters + T.inst, 1u);
            }
            ++n;
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        fence_after_sync();
        tmem_dealloc(tmem, RES ? 512 : 256);
    }
}

// J_hi = bf16(J), J_lo = bf16(J - J_hi) from the padded FP32 copy.
__global__ void k_split_J(const float* __restrict__ J, __nv_bfloat16* __restrict__ hi,
                          __nv_bfloat16* __restrict__ lo, size_t n) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float v = J[k];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[k] = h;
    lo[k] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// V(t_m) planes from x (spin-major [Np][Rp]) -> replica-major [planes][Rp][Np]:
// sgn x in one plane, or x_hi, x_lo in two.
__global__ void k_bf16_prep(const float* __restrict__ x, __nv_bfloat16* __restrict__ v, int Np,
                            int Rp, int sign) {
    __shared__ float tile[32][33];
    const int i0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y)
        tile[k][threadIdx.x] = x[(size_t)(i0 + k) * Rp + r0 + threadIdx.x];
    __syncthreads();
    const size_t plane = (size_t)Rp * Np;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, i = i0 + threadIdx.x;
        const float xv = tile[threadIdx.x][k];
        const size_t vo = (size_t)r * Np + i;
        if (sign) {
            v[vo] = __ushort_as_bfloat16(xv >= 0.f ? (uint16_t)0x3F80 : (uint16_t)0xBF80);
        } else {
            uint32_t h, l;
            bf16_split_bits(xv, h, l);
            v[vo] = __ushort_as_bfloat16((uint16_t)h);
            v[plane + vo] = __ushort_as_bfloat16((uint16_t)l);
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

// bf16 [outer][inner] (inner contiguous), boxes of one 128-byte K atom x 128
// rows, 128-byte swizzle (the layout sdesc_sw128 describes).
gsb_status bf16_map(CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer) {
    auto encode = encode_fn();
    if (!encode) return set_error(GSB_ECUDA, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {inner * 2};
    cuuint32_t box[2] = {(cuuint32_t)kElems, (cuuint32_t)kT};
    cuuint32_t estr[2] = {1u, 1u};
    CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return set_error(GSB_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return GSB_OK;
}

// Per-run state of the split-bf16 path.
struct Bf16State {
    MInst host;                  // the run's instance descriptor (host copy)
    MInst* dev = nullptr;        // its device copy (single runs)
    MTile* tiles = nullptr;      // the run's tiles (single runs)
    int ntiles = 0;
    uint32_t* counter = nullptr;
    float* p_sched = nullptr;
    int grid = 0;                // CTAs of a single-run launch
};

int device_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

gsb_status set_smem_attr() {
    static std::atomic<uint64_t> seen{0};
    if (first_on_device(seen)) {
        GSB_CUDA_TRY(cudaFuncSetAttribute(k_bf16_multi<false>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemM));
        GSB_CUDA_TRY(cudaFuncSetAttribute(k_bf16_multi<true>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemM));
    }
    return GSB_OK;
}

// Largest cooperative grid: one CTA per SM (the kernel's shared memory admits
// one), never more CTAs than items.
gsb_status coop_grid(long items, int* grid) {
    gsb_status st = set_smem_attr();
    if (st != GSB_OK) return st;
    int per_sm = 0;
    GSB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bf16_multi<false>,
                                                               kThreadsM, kSmemM));
    const long cap = (long)std::max(per_sm, 0) * device_sms();
    if (cap < 1) return set_error(GSB_ECUDA, "k_bf16_multi cannot be resident");
    *grid = (int)std::max(1L, std::min(cap, items));
    return GSB_OK;
}

// grid: the CTAs the launch may take. When every tile can have its own CTA
// (grid >= ntiles) the launch takes exactly one per tile and the resident form.
gsb_status launch_multi(const MInst* insts, const MTile* tiles, int ntiles, int nsteps,
                        uint32_t* counters, int ninst, int* status, int grid, cudaStream_t s) {
    const bool res = grid >= ntiles;
    if (res) grid = ntiles;
    GSB_CUDA_TRY(cudaMemsetAsync(counters, 0, sizeof(uint32_t) * ninst, s));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreadsM);
    cfg.dynamicSmemBytes = kSmemM;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeCooperative;  // every CTA resident at once
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (res)
        GSB_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_bf16_multi<true>, insts, tiles, ntiles, nsteps,
                                        counters, ninst, status));
    else
        GSB_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_bf16_multi<false>, insts, tiles, ntiles, nsteps,
                                        counters, ninst, status));
    count_launch();
    return GSB_OK;
}

}  // namespace

gsb_status bf16_tensor_map(CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer) {
    return bf16_map(map, base, inner, outer);
}

// J_hi / J_lo of a dense problem, made on first use.
gsb_status bf16_ensure_planes(gsb_problem* P, cudaStream_t s) {
    if (P->Jhi) return GSB_OK;
    const size_t n = (size_t)P->Np * P->Np;
    gsb_status st;
    if ((st = dev_alloc(&P->Jhi, n)) != GSB_OK) return st;
    if ((st = dev_alloc(&P->Jlo, n)) != GSB_OK) {
        dev_free(P->Jhi);
        P->Jhi = nullptr;
        return st;
    }
    k_split_J<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P->J32, P->Jhi, P->Jlo, n);
    GSB_LAUNCH_CHECK("k_split_J");
    return GSB_OK;
}

gsb_status bf16_setup(gsb_run_state* run) {
    gsb_problem* P = run->prob;
    gsb_status st = bf16_ensure_planes(P, run->stream);
    if (st != GSB_OK) return st;
    Bf16State* B = new Bf16State();
    run->tc = B;
    const int planes = run->sign_coupling ? 1 : 2;
    const size_t n = (size_t)run->Np * run->Rp * planes;
    for (int b = 0; b < 2; ++b)
        if ((st = dev_alloc(&run->v16[b], n))) return st;
    MInst& I = B->host;
    memset(&I, 0, sizeof(I));
    if ((st = bf16_map(&I.tmJ[0], P->Jhi, P->Np, P->Np)) ||
        (st = bf16_map(&I.tmJ[1], P->Jlo, P->Np, P->Np)))
        return st;
    for (int b = 0; b < 2; ++b)
        if ((st = bf16_map(&I.tmV[b], run->v16[b], run->Np, (uint64_t)planes * run->Rp))) return st;
    if (!run->control) {
        std::vector<float> ps(run->params.M);
        for (int m = 0; m < run->params.M; ++m) ps[m] = run_p_shared(run, m + 1);
        if ((st = dev_alloc(&B->p_sched, (size_t)run->params.M))) return st;
        GSB_CUDA_TRY(cudaMemcpy(B->p_sched, ps.data(), sizeof(float) * run->params.M,
                                cudaMemcpyHostToDevice));
    }
    I.x = run->x[0];
    I.y = run->y;
    I.p = run->p;
    I.A = run->A;
    I.v[0] = run->v16[0];
    I.v[1] = run->v16[1];
    I.p_sched = B->p_sched;
    I.status = run->status;
    I.Np = run->Np;
    I.Rp = run->Rp;
    I.M = run->params.M;
    I.flags = (run->sign_coupling ? 1 : 0) | (run->control ? 2 : 0);
    I.c = run->c;
    I.dt = run->dt;
    // the tiles that hold a real spin and a real replica
    std::vector<MTile> tl;
    for (int i0 = 0; i0 < run->N; i0 += kT)
        for (int r0 = 0; r0 < run->R; r0 += kT) tl.push_back({0, i0, r0, 0});
    B->ntiles = (int)tl.size();
    I.tiles = B->ntiles;
    if ((st = dev_alloc(&B->dev, 1)) || (st = dev_alloc(&B->tiles, tl.size())) ||
        (st = dev_alloc(&B->counter, 1)))
        return st;
    GSB_CUDA_TRY(cudaMemcpy(B->tiles, tl.data(), sizeof(MTile) * tl.size(), cudaMemcpyHostToDevice));
    if ((st = coop_grid(B->ntiles, &B->grid))) return st;
    return bf16_prepare(run);
}

gsb_status bf16_prepare(gsb_run_state* run) {
    dim3 grid(run->Np / 32, run->Rp / 32), block(32, 8);
    const int sign = run->sign_coupling ? 1 : 0;
    // V(t_m) for the run's current step m lives in buffer m & 1
    k_bf16_prep<<<grid, block, 0, run->stream>>>(run->x[0], run->v16[run->steps_done & 1],
                                                 run->Np, run->Rp, sign);
    GSB_LAUNCH_CHECK("k_bf16_prep");
    return GSB_OK;
}

gsb_status bf16_steps(gsb_run_state* run, int m0, int nsteps) {
    Bf16State* B = (Bf16State*)run->tc;
    int m = m0;
    const int end = m0 + nsteps;
    const int spl = run->params.steps_per_launch;
    while (m < end) {
        // one persistent launch per stretch of steps between energy evaluations
        int stop = end;
        for (int k = m + 1; k <= end; ++k)
            if (run_is_eval_step(run, k)) {
                stop = k;
                break;
            }
        if (spl > 0 && stop - m > spl) stop = m + spl;
        B->host.m0 = m;
        B->host.stop = stop;
        GSB_CUDA_TRY(cudaMemcpyAsync(B->dev, &B->host, sizeof(MInst), cudaMemcpyHostToDevice,
                                     run->stream));
        gsb_status st = prof_begin(run);
        if (st != GSB_OK) return st;
        if ((st = launch_multi(B->dev, B->tiles, B->ntiles, stop - m, B->counter, 1, run->status,
                               B->grid, run->stream)))
            return st;
        if ((st = prof_end(run, stop - m)) != GSB_OK) return st;
        // the descriptor's host copy changes for the next launch: the copy above
        // must have been taken (a pageable-source copy is staged before it returns)
        m = stop;
        if (run_is_eval_step(run, m))
            if ((st = run_evaluate(run, m)) != GSB_OK) return st;
    }
    return GSB_OK;
}

void bf16_free(gsb_run_state* run) {
    Bf16State* B = (Bf16State*)run->tc;
    if (B) {
        dev_free(B->dev);
        dev_free(B->tiles);
        dev_free(B->counter);
        dev_free(B->p_sched);
    }
    delete B;
    run->tc = nullptr;
}

// ---------------------------------------------------------------------------
// Batched runs on the split-bf16 path: every instance's run was set up by
// gsb_run (deferred); the instances are packed into windows of about `per_cta`
// tiles per CTA, largest first, and each window runs all its remaining steps
// in one persistent launch. Returns through *grid_out the CTAs per launch.
gsb_status bf16_batch(gsb_run_state* const* runs, int n, const int* stop, int per_cta,
                      double max_mb, bool graph, int* windows_out, int* grid_out,
                      int* graphed_out, cudaStream_t s) {
    gsb_status st = set_smem_attr();
    if (st != GSB_OK) return st;
    int per_sm = 0;
    GSB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bf16_multi<false>, kThreadsM,
                                                               kSmemM));
    const int G = std::max(per_sm, 0) * device_sms();
    if (G < 1) return set_error(GSB_ECUDA, "k_bf16_multi cannot be resident");
    // largest K first, so that windows hold tiles of similar cost
    std::vector<int> order(n);
    for (int k = 0; k < n; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return runs[a]->Np > runs[b]->Np;
    });
    std::vector<MInst> insts(n);
    std::vector<std::vector<MTile>> win;
    std::vector<int> win_steps;
    std::vector<MTile> cur;
    int cur_steps = 0;
    double cur_bytes = 0.0;
    const size_t budget = (size_t)G * std::max(1, per_cta);
    for (int idx = 0; idx < n; ++idx) {
        const int k = order[idx];
        gsb_run_state* r = runs[k];
        Bf16State* B = (Bf16State*)r->tc;
        insts[k] = B->host;
        insts[k].m0 = r->steps_done;
        insts[k].stop = stop[k];
        std::vector<MTile> t;
        for (int i0 = 0; i0 < r->N; i0 += kT)
            for (int r0 = 0; r0 < r->R; r0 += kT) t.push_back({k, i0, r0, 0});
        insts[k].tiles = (int)t.size();
        // the bytes a step of the instance touches: J_hi and J_lo, x, y, p, and
        // both V buffers -- a window is kept within max_mb so that it stays in L2
        const double Np = r->Np, Rp = r->Rp;
        const double bytes = 4.0 * Np * Np + (r->control ? 12.0 : 8.0) * Np * Rp +
                             2.0 * 2.0 * (r->sign_coupling ? 1.0 : 2.0) * Np * Rp;
        if (!cur.empty() &&
            (cur.size() + t.size() > budget || cur_bytes + bytes > max_mb * 1048576.0)) {
            win.push_back(cur);
            win_steps.push_back(cur_steps);
            cur.clear();
            cur_steps = 0;
            cur_bytes = 0.0;
        }
        cur_bytes += bytes;
        cur.insert(cur.end(), t.begin(), t.end());
        cur_steps = std::max(cur_steps, stop[k] - r->steps_done);
    }
    if (!cur.empty()) {
        win.push_back(cur);
        win_steps.push_back(cur_steps);
    }
    MInst* d_inst = nullptr;
    MTile* d_tiles = nullptr;
    uint32_t* d_ctr = nullptr;
    int* d_status = nullptr;
    size_t ntot = 0;
    for (auto& w : win) ntot += w.size();
    if ((st = dev_alloc(&d_inst, (size_t)n)) || (st = dev_alloc(&d_tiles, std::max<size_t>(ntot, 1))) ||
        (st = dev_alloc(&d_ctr, (size_t)n)) || (st = dev_alloc(&d_status, 1))) {
        dev_free(d_inst);
        dev_free(d_tiles);
        dev_free(d_ctr);
        return st;
    }
    // every instance reports a timeout into the batch's status word here, and
    // the word is folded into each run's own afterwards
    for (int k = 0; k < n; ++k) insts[k].status = d_status;
    do {
        if (cudaMemcpyAsync(d_inst, insts.data(), sizeof(MInst) * n, cudaMemcpyHostToDevice, s) !=
                cudaSuccess ||
            cudaMemsetAsync(d_status, 0, sizeof(int), s) != cudaSuccess) {
            st = cuda_error(cudaGetLastError(), "batch descriptors");
            break;
        }
        std::vector<MTile> all;
        for (auto& w : win) all.insert(all.end(), w.begin(), w.end());
        if (!all.empty() && cudaMemcpyAsync(d_tiles, all.data(), sizeof(MTile) * all.size(),
                                            cudaMemcpyHostToDevice, s) != cudaSuccess) {
            st = cuda_error(cudaGetLastError(), "batch tiles");
            break;
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            st = cuda_error(cudaGetLastError(), "batch set-up");
            break;
        }
        // the windows' launches, in order; as one CUDA graph when asked for
        auto issue = [&](cudaStream_t q) -> gsb_status {
            size_t o = 0;
            for (size_t w = 0; w < win.size(); ++w) {
                const int nt = (int)win[w].size();
                const int grid = (int)std::min<long>(G, (long)nt * win_steps[w]);
                if (grid_out) *grid_out = std::max(*grid_out, grid);
                gsb_status e = launch_multi(d_inst, d_tiles + o, nt, win_steps[w], d_ctr, n,
                                            d_status, grid, q);
                if (e != GSB_OK) return e;
                o += nt;
            }
            return GSB_OK;
        };
        int total_steps = 0;
        for (int v : win_steps) total_steps += v;
        cudaGraphExec_t exec = nullptr;
        if (graph && !win.empty()) {
            cudaGraph_t gr = nullptr;
            bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                const gsb_status e = issue(s);
                ok = cudaStreamEndCapture(s, &gr) == cudaSuccess && e == GSB_OK;
            }
            if (ok && cudaGraphInstantiate(&exec, gr, 0) != cudaSuccess) {
                exec = nullptr;
                ok = false;
            }
            if (gr) cudaGraphDestroy(gr);
            if (!ok) cudaGetLastError();  // capture not available: launch directly below
        }
        if (graphed_out) *graphed_out = exec != nullptr;
        if ((st = call_prof_begin(s))) break;
        if (exec) {
            const cudaError_t e = cudaGraphLaunch(exec, s);
            cudaGraphExecDestroy(exec);
            if (e != cudaSuccess) {
                st = cuda_error(e, "cudaGraphLaunch");
                break;
            }
        } else if ((st = issue(s))) {
            break;
        }
        if ((st = call_prof_end(s, total_steps))) break;
        // fold the batch's status word into every run's
        for (int k = 0; k < n && st == GSB_OK; ++k) {
            if (cudaMemcpyAsync(runs[k]->status, d_status, sizeof(int), cudaMemcpyDeviceToDevice,
                                s) != cudaSuccess)
                st = cuda_error(cudaGetLastError(), "batch status");
        }
        if (st == GSB_OK && cudaStreamSynchronize(s) != cudaSuccess)
            st = cuda_error(cudaGetLastError(), "batch launch");
    } while (0);
    cudaStreamSynchronize(s);
    dev_free(d_inst);
    dev_free(d_tiles);
    dev_free(d_ctr);
    dev_free(d_status);
    if (windows_out) *windows_out = (int)win.size();
    return st;
}

}  // namespace gsb
