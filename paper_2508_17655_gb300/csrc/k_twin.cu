// k_twin.cu -- the chaos measure of Sec. IV: two trajectories started a distance
// delta(0) = 1e-6 apart, and their normalised distance (Eq. 8)
//   delta(t_m) = sqrt( sum_i [x^(1)_i(t_m) - x^(2)_i(t_m)]^2 / (4N) ).
// A twin run is an ordinary run of 2Q replicas (pair q = replicas q and Q + q,
// both with the same control strength), so the twins advance in the same step
// kernel as any other replicas; the initial state comes from k_twin_init.
//
// The distance is reduced in FP64 in a fixed order: one thread per pair sums
// kChunk spins (the difference of two FP32 values is exact in FP64), then one
// thread per pair adds the chunk sums in chunk order. Results do not depend on
// the launch configuration.
#include "gsb_internal.cuh"

namespace gsb {

namespace {

constexpr int kChunk = 64;
constexpr int kThreads = 128;

__global__ void __launch_bounds__(kThreads) k_twin_part(const float* __restrict__ x, int N,
                                                        int Rp, int Q,
                                                        double* __restrict__ part) {
    const int q = blockIdx.x * kThreads + threadIdx.x;
    if (q >= Q) return;
    const int i0 = blockIdx.y * kChunk;
    const int i1 = min(N, i0 + kChunk);
    double s = 0.0;
    for (int i = i0; i < i1; ++i) {
        const double d = (double)x[(size_t)i * Rp + q] - (double)x[(size_t)i * Rp + Q + q];
        s = fma(d, d, s);
    }
    part[(size_t)blockIdx.y * Q + q] = s;
}

__global__ void __launch_bounds__(kThreads) k_twin_finish(const double* __restrict__ part,
                                                          int chunks, int Q, int N,
                                                          double* __restrict__ delta) {
    const int q = blockIdx.x * kThreads + threadIdx.x;
    if (q >= Q) return;
    double s = 0.0;
    for (int k = 0; k < chunks; ++k) s += part[(size_t)k * Q + q];
    delta[q] = sqrt(s / (4.0 * (double)N));
}

int twin_chunks(int N) { return (N + kChunk - 1) / kChunk; }

}  // namespace

}  // namespace gsb

using namespace gsb;

extern "C" gsb_status gsb_twin_run(gsb_problem* P, const gsb_params* prm, int32_t nA,
                                   const float* A_values, gsb_run_state** out, void* stream) {
    if (!P || !prm || !out || !A_values || nA < 1)
        return set_error(GSB_EINVAL, "NULL argument or nA < 1");
    *out = nullptr;
    const gsb_params& Q = *prm;
    if (P->has_h) return set_error(GSB_EUNSUPPORTED, "twin runs take problems without h");
    if (Q.x0 || Q.y0 || Q.A_per_replica)
        return set_error(GSB_EINVAL, "twin runs draw their own x(0), y(0) and take A from A_values");
    if (Q.R < 1) return set_error(GSB_EINVAL, "R must be >= 1");
    const long long pairs = (long long)nA * Q.R;
    if (2 * pairs > (1 << 22)) return set_error(GSB_EINVAL, "2 nA R out of range");
    const int npairs = (int)pairs;
    std::vector<float> Ah(2 * (size_t)npairs);
    for (int a = 0; a < nA; ++a)
        for (int r = 0; r < Q.R; ++r)
            Ah[(size_t)a * Q.R + r] = Ah[(size_t)npairs + (size_t)a * Q.R + r] = A_values[a];
    gsb_params T = Q;
    T.R = 2 * npairs;
    T.A_per_replica = Ah.data();
    T.flags = Q.flags | GSB_RUN_DEFER;
    gsb_run_state* run = nullptr;
    gsb_status st = gsb_run(P, &T, &run, stream);
    if (st != GSB_OK) return st;
    // gsb_run drew the ordinary initial state; redraw it as twins
    run->params.A_per_replica = nullptr;
    run->twin_pairs = npairs;
    const size_t nbuf = ((size_t)twin_chunks(run->N) + 1) * npairs;
    if ((st = dev_alloc(&run->twin_part, nbuf)) != GSB_OK) {
        gsb_run_destroy(run);
        return st;
    }
    st = launch_init_state(run, nullptr, nullptr);
    if (st == GSB_OK && is_tc_path(run->path)) st = tc_prepare(run);
    if (st == GSB_OK && !(Q.flags & GSB_RUN_DEFER)) st = gsb_run_steps(run, Q.M);
    if (st != GSB_OK) {
        gsb_run_destroy(run);
        return st;
    }
    *out = run;
    return GSB_OK;
}

extern "C" gsb_status gsb_twin_delta(gsb_run_state* run, double* delta_out) {
    if (!run || !delta_out) return set_error(GSB_EINVAL, "NULL argument");
    if (run->twin_pairs < 1) return set_error(GSB_EINVAL, "not a twin run (gsb_twin_run)");
    const int Q = run->twin_pairs, chunks = twin_chunks(run->N);
    double* part = run->twin_part;
    double* delta = part + (size_t)chunks * Q;
    dim3 grid((Q + kThreads - 1) / kThreads, chunks);
    k_twin_part<<<grid, kThreads, 0, run->stream>>>(run->x[run->cur], run->N, run->Rp, Q, part);
    GSB_LAUNCH_CHECK("k_twin_part");
    k_twin_finish<<<grid.x, kThreads, 0, run->stream>>>(part, chunks, Q, run->N, delta);
    GSB_LAUNCH_CHECK("k_twin_finish");
    GSB_CUDA_TRY(cudaMemcpyAsync(delta_out, delta, sizeof(double) * Q, cudaMemcpyDeviceToHost,
                                 run->stream));
    GSB_CUDA_TRY(cudaStreamSynchronize(run->stream));
    return GSB_OK;
}
