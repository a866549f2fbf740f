// k_gemm_tc.cu -- K-split partial products J V on the tensor cores in the
// split-bf16 form (the adjoint's steps under GSB_PREC_BF16X3).
//
// Fp[s] = J[:, K_s] V[K_s, :] for K slice s of S, with V and every Fp[s]
// spin-major [Np][Rp] FP32: the layout the adjoint's step kernels read and add
// in a fixed order. V is first split into bf16 planes, replica-major
// [2][Rp][Np]: V_hi = bf16(V), V_lo = bf16(V - V_hi), or sgn V alone for the
// sgn coupling. Then each CTA computes one 128 x 128 tile of one K slice,
//   D = V_hi J_hi^T + V_hi J_lo^T + V_lo J_hi^T   (sgn: s J_hi^T + s J_lo^T)
// as tcgen05 kind::f16 MMAs accumulated in FP32 in TMEM (lane = replica,
// column = spin), and writes it out, a warp's 32 replicas of one spin as 128
// contiguous bytes. Splitting K gives the few-replica products of the adjoint
// (R = 256: 32 output tiles) enough CTAs to fill the GPU.
//
// Warps: 0 TMA producer, 1 TMEM owner + MMA issuer, 2-9 epilogue (warp w
// reads TMEM lanes 32 (w % 4).. -- its 32 replicas -- and columns
// 64 ((w - 2) / 4) .. +63 -- 64 spins of the tile).
#include <cudaTypedefs.h>
#include <string.h>

#include "gsb_update.cuh"
#include "tc_ptx.cuh"

namespace gsb {

namespace {

using namespace tc;

constexpr int kT = 128;          // spins and replicas per tile
constexpr int kKB = 128;         // bytes of K per atom
constexpr int kElems = kKB / 2;  // bf16 elements of K per atom
constexpr int kAtom = kT * kKB;  // one 128-row atom (16 KB)
constexpr int kThreads = 320;
constexpr int kStages = 3;
constexpr int kStageBytes = 4 * kAtom;  // J_hi, J_lo, V_hi, V_lo
constexpr int kSmem = 1024 + kStages * kStageBytes + 256;

struct GemmArgs {
    CUtensorMap tmJ[2];  // J_hi, J_lo: [Np][Np]
    CUtensorMap tmV;     // planes: [2 x Rp][Np]
    float* Fp;           // [S][Np][Rp]
    int* status;
    int Np, Rp, S;
};

template <bool SIGN>
__global__ void __launch_bounds__(kThreads, 1) k_gemm_tc(const __grid_constant__ GemmArgs G) {
    constexpr int S = kStages;
    constexpr int NPLANE = SIGN ? 1 : 2;
    constexpr uint32_t kStageTx = (uint32_t)(2 + NPLANE) * kAtom;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + S * kStageBytes);
    uint64_t* empty = full + S;
    uint64_t* accf = empty + S;
    uint64_t* drain = accf + 1;
    uint32_t* tmem_slot = (uint32_t*)(drain + 1);
    auto atom = [&](uint32_t st, int q) { return smem + st * kStageBytes + q * kAtom; };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = blockIdx.x * kT, i0 = blockIdx.y * kT, sl = blockIdx.z;
    // debug build: the grid covers whole tiles of the padded shape (parameters
    // and grid alone: a uniform return before any barrier)
    if (!GSB_DOK(G.Np % kT == 0 && G.Rp % kT == 0 && (int)gridDim.x * kT == G.Rp &&
                     (int)gridDim.y * kT == G.Np && (int)gridDim.z == G.S,
                 G.status))
        return;
    // this CTA's K atoms: slice sl of S, ceil-divided (the last may be short or empty)
    const int natoms = G.Np / kElems, per = (natoms + G.S - 1) / G.S;
    const int a0 = sl * per, a1 = min(natoms, a0 + per);
    const int nk = a1 > a0 ? a1 - a0 : 0;

    if (threadIdx.x == 0) {
        for (int st = 0; st < S; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], 1);
        }
        mbar_init(accf, 1);
        mbar_init(drain, 1);
        fence_barrier_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, 128);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int u = 0;
            for (; u < nk; ++u) {
                const uint32_t st = u % S, ph = (u / S) & 1u;
                if (u >= S && !mbar_wait(&empty[st], ph ^ 1u, G.status)) break;
                mbar_arrive_expect_tx(&full[st], kStageTx);
                const int kx = (a0 + u) * kElems;
                tma_load_2d(atom(st, 0), &G.tmJ[0], &full[st], kx, i0);
                tma_load_2d(atom(st, 1), &G.tmJ[1], &full[st], kx, i0);
#pragma unroll
                for (int q = 0; q < NPLANE; ++q)
                    tma_load_2d(atom(st, 2 + q), &G.tmV, &full[st], kx, q * G.Rp + r0);
            }
            // no copy is in flight when the CTA leaves
            for (int v = u > S ? u - S : 0; v < u; ++v)
                mbar_wait(&full[v % S], (uint32_t)(v / S) & 1u, G.status, kDrainLimitCycles);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_make(1u, kT, kT);
            bool ok = true;
            for (int u = 0; u < nk; ++u) {
                const uint32_t st = u % S, ph = (u / S) & 1u;
                if (!mbar_wait(&full[st], ph, G.status)) {
                    ok = false;
                    break;
                }
                fence_after_sync();
                const uint32_t jh = smem_u32(atom(st, 0)), jl = smem_u32(atom(st, 1));
                const uint32_t vh = smem_u32(atom(st, 2)), vl = smem_u32(atom(st, 3));
#pragma unroll
                for (int k = 0; k < kKB / 32; ++k) {  // 16 bf16 of K per MMA
                    const uint64_t ah = sdesc_sw128(vh + k * 32);
                    const uint64_t bh = sdesc_sw128(jh + k * 32);
                    mma_f16(tmem, ah, bh, idesc, (u | k) != 0);
                    mma_f16(tmem, ah, sdesc_sw128(jl + k * 32), idesc, 1u);
                    if (!SIGN) mma_f16(tmem, sdesc_sw128(vl + k * 32), bh, idesc, 1u);
                }
                mma_commit(&empty[st]);
            }
            if (ok && nk > 0) mma_commit(accf);
            // every MMA issued has finished before TMEM is released
            mma_commit(drain);
            mbar_wait(drain, 0, G.status, kDrainLimitCycles);
        }
    } else {
        const int ew = warp - 2;
        const int quarter = warp & 3;
        const int c0 = (ew >> 2) * 64;
        const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
        const int r = r0 + quarter * 32 + lane;  // this thread's replica (TMEM lane)
        bool ok = true;
        if (nk > 0) ok = __all_sync(0xffffffffu, mbar_wait(accf, 0u, G.status));
        fence_after_sync();
        float* F = G.Fp + (size_t)sl * G.Np * G.Rp + (size_t)(i0 + c0) * G.Rp + r;
#pragma unroll 1
        for (int cb = 0; cb < 64; cb += 16) {
            float v[16];
            if (nk > 0 && ok) {
                tmem_ld16(tl + c0 + cb, v);
            } else {
#pragma unroll
                for (int k = 0; k < 16; ++k) v[k] = 0.f;  // an empty K slice adds nothing
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) F[(size_t)(cb + k) * G.Rp] = v[k];
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        fence_after_sync();
        tmem_dealloc(tmem, 128);
    }
}

// V (spin-major [Np][Rp]) -> its operand planes, replica-major [2][Rp][Np]:
// sgn V in plane 0, or V_hi, V_lo (32 x 32 tiles through shared memory).
__global__ void k_gemm_planes(const float* __restrict__ V, uint16_t* __restrict__ v, int Np,
                              int Rp, int sign) {
    __shared__ float tile[32][33];
    const int i0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y)
        tile[k][threadIdx.x] = V[(size_t)(i0 + k) * Rp + r0 + threadIdx.x];
    __syncthreads();
    const size_t plane = (size_t)Rp * Np;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, i = i0 + threadIdx.x;
        const float xv = tile[threadIdx.x][k];
        const size_t o = (size_t)r * Np + i;
        if (sign) {
            v[o] = xv >= 0.f ? (uint16_t)0x3F80 : (uint16_t)0xBF80;
        } else {
            uint32_t h, l;
            bf16_split_bits(xv, h, l);
            v[o] = (uint16_t)h;
            v[plane + o] = (uint16_t)l;
        }
    }
}

template <bool SIGN>
gsb_status set_attr_once() {
    static std::atomic<uint64_t> seen{0};
    if (first_on_device(seen))
        GSB_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc<SIGN>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
    return GSB_OK;
}

}  // namespace

struct SplitGemm {
    GemmArgs args;
    __nv_bfloat16* planes = nullptr;
    int* status = nullptr;
};

gsb_status split_gemm_create(gsb_problem* P, int Rp, SplitGemm** out, cudaStream_t s) {
    *out = nullptr;
    if (Rp % kT != 0 || P->Np % kT != 0) return set_error(GSB_EINVAL, "split_gemm: unpadded shape");
    gsb_status st = bf16_ensure_planes(P, s);
    if (st != GSB_OK) return st;
    SplitGemm* g = new SplitGemm();
    memset(&g->args, 0, sizeof(g->args));
    if ((st = dev_alloc(&g->planes, (size_t)2 * Rp * P->Np)) || (st = dev_alloc(&g->status, 1)) ||
        (st = bf16_tensor_map(&g->args.tmJ[0], P->Jhi, P->Np, P->Np)) ||
        (st = bf16_tensor_map(&g->args.tmJ[1], P->Jlo, P->Np, P->Np)) ||
        (st = bf16_tensor_map(&g->args.tmV, g->planes, P->Np, (uint64_t)2 * Rp))) {
        split_gemm_destroy(g);
        return st;
    }
    if (cudaMemsetAsync(g->status, 0, sizeof(int), s) != cudaSuccess) {
        split_gemm_destroy(g);
        return cuda_error(cudaGetLastError(), "split_gemm status");
    }
    g->args.status = g->status;
    g->args.Np = P->Np;
    g->args.Rp = Rp;
    *out = g;
    return GSB_OK;
}

gsb_status split_gemm_partials(SplitGemm* g, const float* V, bool sign, int nslices, float* Fp,
                               cudaStream_t s) {
    GemmArgs& a = g->args;
    // more slices than K atoms leave the last ones empty (they write zeros)
    if (nslices < 1 || nslices > 64) return set_error(GSB_EINVAL, "split_gemm: K slices out of range");
    k_gemm_planes<<<dim3(a.Np / 32, a.Rp / 32), dim3(32, 8), 0, s>>>(
        V, reinterpret_cast<uint16_t*>(g->planes), a.Np, a.Rp, sign ? 1 : 0);
    GSB_LAUNCH_CHECK("k_gemm_planes");
    a.Fp = Fp;
    a.S = nslices;
    const dim3 grid(a.Rp / kT, a.Np / kT, nslices);
    gsb_status st = sign ? set_attr_once<true>() : set_attr_once<false>();
    if (st != GSB_OK) return st;
    if (sign)
        k_gemm_tc<true><<<grid, kThreads, kSmem, s>>>(a);
    else
        k_gemm_tc<false><<<grid, kThreads, kSmem, s>>>(a);
    GSB_LAUNCH_CHECK("k_gemm_tc");
    return GSB_OK;
}

gsb_status split_gemm_status(SplitGemm* g, cudaStream_t s) {
    int dst = 0;
    GSB_CUDA_TRY(cudaMemcpyAsync(&dst, g->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    GSB_CUDA_TRY(cudaStreamSynchronize(s));
    if (dst & kDevTimeout)
        return set_error(GSB_ETIMEOUT, "k_gemm_tc: a barrier wait exceeded its bound");
    if (dst & kDevBounds) return set_error(GSB_ECUDA, "a kernel detected an out-of-range index");
    return GSB_OK;
}

void split_gemm_destroy(SplitGemm* g) {
    if (!g) return;
    dev_free(g->planes);
    dev_free(g->status);
    delete g;
}

}  // namespace gsb
