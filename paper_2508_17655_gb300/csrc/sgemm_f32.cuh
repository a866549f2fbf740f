// sgemm_f32.cuh -- the FP32 CUDA-core SGEMM tile shared by the plain step,
// energy and tangent-linear kernels: F[i][r] = sum_k J[i][k] v[k][r] for one
// 128-spin x 128-column tile, K = Np, 256 threads with 8 x 8 accumulators
// (rows {4ty..4ty+3, 64+4ty..}, columns {4tx.., 64+4tx..}).
#pragma once
#include "gsb_update.cuh"

namespace gsb {
namespace f32 {

constexpr int BM = 128, BN = 128, BK = 8;

struct F32Smem {
    float A[2][BK][BM + 4];  // J tile, transposed (k-major)
    float B[2][BK][BN];      // v tile
};

template <bool SIGN>
__device__ __forceinline__ float4 vload(const float* p) {
    float4 v = *reinterpret_cast<const float4*>(p);
    if (SIGN) {
        v.x = sgnf(v.x);
        v.y = sgnf(v.y);
        v.z = sgnf(v.z);
        v.w = sgnf(v.w);
    }
    return v;
}

// acc[a][b] += sum_k J[row_a][k] v[k][col_b] over the full K = Np.
template <bool SIGN>
__device__ __forceinline__ void sgemm_tile(const float* __restrict__ J,
                                           const float* __restrict__ X, int Np, int Rp, int i0,
                                           int r0, float (&acc)[8][8], F32Smem& sm) {
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int a_row = tid >> 1, a_k = (tid & 1) * 4;
    const int b_k = tid >> 5, b_c = (tid & 31) * 4;
    const float* Ap = J + (size_t)(i0 + a_row) * Np + a_k;
    const float* Bp = X + (size_t)b_k * Rp + r0 + b_c;
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;

    float4 ra = *reinterpret_cast<const float4*>(Ap);
    float4 rb = vload<SIGN>(Bp);
    auto stash = [&](int buf) {
        sm.A[buf][a_k + 0][a_row] = ra.x;
        sm.A[buf][a_k + 1][a_row] = ra.y;
        sm.A[buf][a_k + 2][a_row] = ra.z;
        sm.A[buf][a_k + 3][a_row] = ra.w;
        *reinterpret_cast<float4*>(&sm.B[buf][b_k][b_c]) = rb;
    };
    stash(0);
    __syncthreads();
    const int nk = Np / BK;
    for (int kt = 0; kt < nk; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nk) {
            ra = *reinterpret_cast<const float4*>(Ap + (size_t)(kt + 1) * BK);
            rb = vload<SIGN>(Bp + (size_t)(kt + 1) * BK * Rp);
        }
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4*>(&sm.A[buf][k][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&sm.A[buf][k][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&sm.B[buf][k][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&sm.B[buf][k][64 + tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
        }
        if (kt + 1 < nk) stash(buf ^ 1);
        __syncthreads();
    }
}

__device__ __forceinline__ int row_of(int a, int ty) { return a < 4 ? ty * 4 + a : 64 + ty * 4 + (a - 4); }

// 64 x 64 tile: 256 threads, 4 x 4 accumulators each (rows 4ty.., columns 4tx..).
struct Smem64 {
    float A[2][BK][64 + 4];
    float B[2][BK][64];
};

// K = Np, J rows Np apart; or, with ldj and k0/klen, the K range [k0, k0 + klen).
template <bool SIGN>
__device__ __forceinline__ void sgemm_tile64(const float* __restrict__ J, const float* __restrict__ X,
                                             int Np, int Rp, int i0, int r0, float (&acc)[4][4],
                                             Smem64& sm, int k0 = 0, int klen = -1) {
    const int ldj = Np;
    if (klen < 0) klen = Np;
    J += k0;
    X += (size_t)k0 * Rp;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int a_row = tid >> 2, a_k = (tid & 3) * 2;
    const int b_k = tid >> 5, b_c = (tid & 31) * 2;
    const float* Ap = J + (size_t)(i0 + a_row) * ldj + a_k;
    const float* Bp = X + (size_t)b_k * Rp + r0 + b_c;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    auto ldb = [&](const float* q) {
        float2 v = *reinterpret_cast<const float2*>(q);
        if (SIGN) {
            v.x = sgnf(v.x);
            v.y = sgnf(v.y);
        }
        return v;
    };
    float2 ra = *reinterpret_cast<const float2*>(Ap);
    float2 rb = ldb(Bp);
    auto stash = [&](int buf) {
        sm.A[buf][a_k + 0][a_row] = ra.x;
        sm.A[buf][a_k + 1][a_row] = ra.y;
        *reinterpret_cast<float2*>(&sm.B[buf][b_k][b_c]) = rb;
    };
    stash(0);
    __syncthreads();
    const int nk = klen / BK;
    for (int kt = 0; kt < nk; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nk) {
            ra = *reinterpret_cast<const float2*>(Ap + (size_t)(kt + 1) * BK);
            rb = ldb(Bp + (size_t)(kt + 1) * BK * Rp);
        }
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            const float4 a = *reinterpret_cast<const float4*>(&sm.A[buf][k][ty * 4]);
            const float4 b = *reinterpret_cast<const float4*>(&sm.B[buf][k][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w};
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (kt + 1 < nk) stash(buf ^ 1);
        __syncthreads();
    }
}


// Shape of an SGEMM tile for kernels written for both sizes: T x T outputs
// over 256 threads; thread (tx, ty) holds acc[a][b] for row(a, ty), col(b, tx).
// Both tiles sum K in the same order, so an output is the same either way.
template <int T>
struct Tile;
template <>
struct Tile<128> {
    static constexpr int NA = 8, NB = 8;
    using Smem = F32Smem;
    __device__ static int row(int a, int ty) { return row_of(a, ty); }
    __device__ static int col(int b, int tx) { return b < 4 ? tx * 4 + b : 64 + tx * 4 + (b - 4); }
    template <bool SIGN>
    __device__ static void gemm(const float* J, const float* X, int Np, int Rp, int i0, int r0,
                                float (&acc)[NA][NB], Smem& sm) {
        sgemm_tile<SIGN>(J, X, Np, Rp, i0, r0, acc, sm);
    }
};
template <>
struct Tile<64> {
    static constexpr int NA = 4, NB = 4;
    using Smem = Smem64;
    __device__ static int row(int a, int ty) { return ty * 4 + a; }
    __device__ static int col(int b, int tx) { return tx * 4 + b; }
    template <bool SIGN>
    __device__ static void gemm(const float* J, const float* X, int Np, int Rp, int i0, int r0,
                                float (&acc)[NA][NB], Smem& sm) {
        sgemm_tile64<SIGN>(J, X, Np, Rp, i0, r0, acc, sm);
    }
};

// 32 x 32 elementwise tile (no SGEMM of its own: for kernels whose products
// come precomputed, e.g. as K-split partial sums): 16 x 16 threads, 2 x 2
// elements each (two consecutive replicas of two consecutive rows).
template <>
struct Tile<32> {
    static constexpr int NA = 2, NB = 2;
    struct Smem {};
    __device__ static int row(int a, int ty) { return ty * 2 + a; }
    __device__ static int col(int b, int tx) { return tx * 2 + b; }
};

}  // namespace f32
}  // namespace gsb
