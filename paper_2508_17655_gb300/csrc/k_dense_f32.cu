// k_dense_f32.cu -- the plain FP32 form of one dense time step: the many-body
// term f = J v (v = x or sgn x) as a CUDA-core SGEMM over all replicas at once,
// with Eqs. 3-7 fused into its epilogue; and the Ising energy (Eq. 1) of sgn x
// by the same SGEMM with a reducing epilogue.
//
// Layouts: J row-major [Np][Np] (zero padded), state spin-major [Np][Rp].
// One CTA computes a 128-spin x 128-replica tile; 256 threads, 8 x 8
// accumulators each (rows {4ty..4ty+3, 64+4ty..}, columns {4tx.., 64+4tx..}).
#include "sgemm_f32.cuh"

namespace gsb {

namespace {

using namespace f32;

template <bool SIGN, bool CONTROL>
__global__ void __launch_bounds__(256) k_dense_f32_step(
    const float* __restrict__ J, int Np, int Rp, const float* __restrict__ xc,
    float* __restrict__ xn, float* __restrict__ y, float* __restrict__ p,
    const float* __restrict__ A, float c, float dt, float p_shared, float inv_rem, int* status) {
    __shared__ __align__(16) F32Smem sm;
    // debug build: the grid covers the padded shape exactly (a uniform return)
    if (!GSB_DOK(Np % BM == 0 && Rp % BN == 0 && (int)gridDim.x * BN == Rp &&
                     (int)gridDim.y * BM == Np,
                 status))
        return;
    const int i0 = blockIdx.y * BM, r0 = blockIdx.x * BN;
    float acc[8][8];
    sgemm_tile<SIGN>(J, xc, Np, Rp, i0, r0, acc, sm);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int cols[2] = {r0 + tx * 4, r0 + 64 + tx * 4};
    float av[8];
    if (CONTROL) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float4 t = *reinterpret_cast<const float4*>(A + cols[h]);
            av[h * 4 + 0] = t.x; av[h * 4 + 1] = t.y; av[h * 4 + 2] = t.z; av[h * 4 + 3] = t.w;
        }
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const size_t rowoff = (size_t)(i0 + row_of(a, ty)) * Rp;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const size_t o = rowoff + cols[h];
            float4 x4 = *reinterpret_cast<const float4*>(xc + o);
            float4 y4 = *reinterpret_cast<float4*>(y + o);
            float4 p4 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (CONTROL) p4 = *reinterpret_cast<float4*>(p + o);
            float* xs = &x4.x; float* ys = &y4.x; float* ps = &p4.x;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                sb_update<CONTROL>(xs[q], ys[q], ps[q], acc[a][h * 4 + q],
                                   CONTROL ? av[h * 4 + q] : 0.f, c, dt, p_shared, inv_rem);
            *reinterpret_cast<float4*>(xn + o) = x4;
            *reinterpret_cast<float4*>(y + o) = y4;
            if (CONTROL) *reinterpret_cast<float4*>(p + o) = p4;
        }
    }
}

// part[b][r] = sum_i s_i (J s)_i over the 128 spins of row block b (s = sgn x).
__global__ void __launch_bounds__(256) k_dense_f32_energy(const float* __restrict__ J, int Np,
                                                          int Rp, const float* __restrict__ x,
                                                          double* __restrict__ part) {
    __shared__ __align__(16) F32Smem sm;
    __shared__ float red[16][BN + 1];
    const int i0 = blockIdx.y * BM, r0 = blockIdx.x * BN;
    float acc[8][8];
    sgemm_tile<true>(J, x, Np, Rp, i0, r0, acc, sm);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const int col = b < 4 ? tx * 4 + b : 64 + tx * 4 + (b - 4);
        float part = 0.f;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const float si = sgnf(x[(size_t)(i0 + row_of(a, ty)) * Rp + r0 + col]);
            part = fmaf(si, acc[a][b], part);
        }
        red[ty][col] = part;
    }
    __syncthreads();
    if (threadIdx.x < BN) {
        double s = 0.0;
        for (int t = 0; t < 16; ++t) s += (double)red[t][threadIdx.x];
        part[(size_t)blockIdx.y * Rp + r0 + threadIdx.x] = s;
    }
}

// e_acc[r] += the row blocks' partials, in row-block order.
__global__ void k_energy_parts_sum(const double* __restrict__ part, int nblk, int Rp,
                                   double* __restrict__ e_acc) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= Rp) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(size_t)b * Rp + r];
    e_acc[r] += s;
}

}  // namespace

gsb_status launch_dense_f32_step(gsb_run_state* run, const StepScalars& sc) {
    const gsb_problem* P = run->prob;
    dim3 grid(run->Rp / BN, run->Np / BM);
    const float* xc = run->x[run->cur];
    float* xn = run->x[run->cur ^ 1];
    const float inv_rem = 1.0f / (float)(sc.M - sc.m);
#define GSB_F32_LAUNCH(S, C)                                                                  \
    k_dense_f32_step<S, C><<<grid, 256, 0, run->stream>>>(P->J32, run->Np, run->Rp, xc, xn,   \
                                                          run->y, run->p, run->A, sc.c, sc.dt, \
                                                          sc.p_next, inv_rem, run->status)
    if (run->sign_coupling) {
        if (run->control) GSB_F32_LAUNCH(true, true); else GSB_F32_LAUNCH(true, false);
    } else {
        if (run->control) GSB_F32_LAUNCH(false, true); else GSB_F32_LAUNCH(false, false);
    }
#undef GSB_F32_LAUNCH
    GSB_LAUNCH_CHECK("k_dense_f32_step");
    run->cur ^= 1;
    return GSB_OK;
}

gsb_status launch_dense_f32_energy(const gsb_problem* P, const float* x, int Rp, double* e_acc,
                                   double* e_part, cudaStream_t s) {
    dim3 grid(Rp / BN, P->Np / BM);
    k_dense_f32_energy<<<grid, 256, 0, s>>>(P->J32, P->Np, Rp, x, e_part);
    GSB_LAUNCH_CHECK("k_dense_f32_energy");
    k_energy_parts_sum<<<(Rp + 255) / 256, 256, 0, s>>>(e_part, P->Np / BM, Rp, e_acc);
    GSB_LAUNCH_CHECK("k_energy_parts_sum");
    return GSB_OK;
}

}  // namespace gsb
