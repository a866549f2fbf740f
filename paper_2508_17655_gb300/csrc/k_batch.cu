// k_batch.cu -- many independent instances of uneven size stepped together
// (gsb_batch_run). The paper runs several instances per machine at once and
// keeps the better result (N_batch, Sec. VI); here every instance is an
// ordinary run (its own J, replicas, parameters, state buffers).
//
// Split-bf16 form (precision AUTO or BF16X3): the tensor-core kernel of
// k_bf16.cu runs windows of instances, each window all its steps in one
// persistent launch over a device work list; batch_bf16 below sets the runs
// up and times the window size.
//
// FP32 form (precision FP32): one launch per time step covers all instances
// through a device work list of tiles (instance, spin block, replica block).
// Tiles that only hold padding are never listed. Each tile is the plain FP32
// SGEMM tile with Eqs. 3-7 in its epilogue, summing over K in the same order as
// the single-run kernel, so a batched instance follows exactly the trajectory
// it would follow alone. The step index lives in device memory and a
// one-thread kernel advances it, so a chunk of steps is captured once as a CUDA
// graph and replayed. An autotuner times the two tile sizes (128 and 64 spins x
// replicas) and the graph chunk lengths on the run's first steps and keeps the
// fastest.
#include <algorithm>
#include <vector>

#include "sgemm_f32.cuh"

namespace gsb {

namespace {

using namespace f32;

struct BatchInst {
    const float* J;
    float* x0;
    float* x1;
    float* y;
    float* p;
    const float* A;
    int Np, Rp, M, flags;  // flags: 1 = sgn-x coupling, 2 = individual control
    int stop;              // steps this batch advances the instance (<= M)
    float c, dt;
    const float* sched;    // p(t_m), m = 0..M (device) or null
    int* status;           // the instance's run status word
};

struct BatchTile {
    int inst, i0, r0, work;
};


__device__ __forceinline__ void batch_update4(const BatchInst& I, const float* xc, float* xn,
                                              size_t o, int r, const float* f, bool control,
                                              float p_shared, float inv_rem) {
    float4 x4 = *reinterpret_cast<const float4*>(xc + o);
    float4 y4 = *reinterpret_cast<float4*>(I.y + o);
    float4 p4 = control ? *reinterpret_cast<float4*>(I.p + o) : make_float4(0.f, 0.f, 0.f, 0.f);
    float* xs = &x4.x;
    float* ys = &y4.x;
    float* ps = &p4.x;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (control)
            sb_update<true>(xs[q], ys[q], ps[q], f[q], I.A[r + q], I.c, I.dt, p_shared, inv_rem);
        else
            sb_update<false>(xs[q], ys[q], ps[q], f[q], 0.f, I.c, I.dt, p_shared, inv_rem);
    }
    *reinterpret_cast<float4*>(xn + o) = x4;
    *reinterpret_cast<float4*>(I.y + o) = y4;
    if (control) *reinterpret_cast<float4*>(I.p + o) = p4;
}

template <int T>
__global__ void __launch_bounds__(256) k_batch_step(const BatchInst* __restrict__ insts,
                                                    const BatchTile* __restrict__ tiles,
                                                    const int* __restrict__ m_dev, int ninst) {
    const int m = *m_dev;
    const BatchTile t = tiles[blockIdx.x];
    // debug build: the tile names an instance of the batch and a whole T x T
    // tile of it (one tile per block: a uniform return)
    if (!GSB_DOK(t.inst >= 0 && t.inst < ninst, insts[0].status)) return;
    const BatchInst I = insts[t.inst];
    if (!GSB_DOK(t.i0 >= 0 && t.r0 >= 0 && t.i0 + T <= I.Np && t.r0 + T <= I.Rp && I.stop <= I.M,
                 I.status))
        return;
    if (m >= I.stop) return;  // this instance has finished its steps
    const bool odd = m & 1;
    const float* xc = odd ? I.x1 : I.x0;
    float* xn = odd ? I.x0 : I.x1;
    const bool sign = I.flags & 1, control = I.flags & 2;
    // same scalars as the single-run path: p(t_{m+1}) from the caller schedule
    // or Eq. 6 (double, rounded once), 1/(M - m) rounded once
    const float p_shared =
        I.sched ? I.sched[m + 1] : (float)(1.0 - (double)(m + 1) / (double)I.M);
    const float inv_rem = __frcp_rn((float)(I.M - m));
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    if (T == 128) {
        __shared__ __align__(16) F32Smem sm;
        float acc[8][8];
        if (sign)
            sgemm_tile<true>(I.J, xc, I.Np, I.Rp, t.i0, t.r0, acc, sm);
        else
            sgemm_tile<false>(I.J, xc, I.Np, I.Rp, t.i0, t.r0, acc, sm);
        const int cols[2] = {t.r0 + tx * 4, t.r0 + 64 + tx * 4};
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const size_t rowoff = (size_t)(t.i0 + row_of(a, ty)) * I.Rp;
#pragma unroll
            for (int h = 0; h < 2; ++h)
                batch_update4(I, xc, xn, rowoff + cols[h], cols[h], &acc[a][h * 4], control,
                              p_shared, inv_rem);
        }
    } else {
        __shared__ __align__(16) Smem64 sm;
        float acc[4][4];
        if (sign)
            sgemm_tile64<true>(I.J, xc, I.Np, I.Rp, t.i0, t.r0, acc, sm);
        else
            sgemm_tile64<false>(I.J, xc, I.Np, I.Rp, t.i0, t.r0, acc, sm);
        const int col = t.r0 + tx * 4;
#pragma unroll
        for (int a = 0; a < 4; ++a)
            batch_update4(I, xc, xn, (size_t)(t.i0 + ty * 4 + a) * I.Rp + col, col, acc[a],
                          control, p_shared, inv_rem);
    }
}

__global__ void k_batch_advance(int* m_dev) { *m_dev += 1; }

struct BatchState {
    int n = 0;
    BatchInst* d_inst = nullptr;
    BatchTile* d_tiles[2] = {nullptr, nullptr};  // tile lists for T = 128, 64
    int ntiles[2] = {0, 0};
    float** d_sched = nullptr;
    std::vector<float*> scheds;
    int* d_m = nullptr;
    ~BatchState() {
        cudaFree(d_inst);
        cudaFree(d_tiles[0]);
        cudaFree(d_tiles[1]);
        cudaFree(d_m);
        for (float* s : scheds) cudaFree(s);
    }
};

// One batched time step: every tile of every instance, then the step counter.
gsb_status launch_batch_step_raw(BatchState& B, int which, cudaStream_t s) {
    if (B.ntiles[which] == 0) return GSB_OK;
    if (which == 0)
        k_batch_step<128><<<B.ntiles[0], 256, 0, s>>>(B.d_inst, B.d_tiles[0], B.d_m, B.n);
    else
        k_batch_step<64><<<B.ntiles[1], 256, 0, s>>>(B.d_inst, B.d_tiles[1], B.d_m, B.n);
    GSB_LAUNCH_CHECK("k_batch_step");
    k_batch_advance<<<1, 1, 0, s>>>(B.d_m);
    GSB_LAUNCH_CHECK("k_batch_advance");
    return GSB_OK;
}

// The same, with the call-profile events around it (outside graph capture).
gsb_status launch_batch_step(BatchState& B, int which, cudaStream_t s) {
    gsb_status st = call_prof_begin(s);
    if (st == GSB_OK) st = launch_batch_step_raw(B, which, s);
    if (st == GSB_OK) st = call_prof_end(s, 1);
    return st;
}

}  // namespace

}  // namespace gsb

using namespace gsb;

namespace gsb {
namespace {

// The split-bf16 form of gsb_batch_run (see include/gsb.h): every instance an
// ordinary deferred run on the BF16X3 path, then persistent launches over
// windows of instances; tiles per CTA picked by timing real steps.
gsb_status batch_bf16(int n, gsb_problem* const* problems, const gsb_params* params,
                      gsb_run_state** runs_out, gsb_batch_info* info, cudaStream_t s) {
    auto cleanup = [&](gsb_status e) {
        for (int k = 0; k < n; ++k) {
            gsb_run_destroy(runs_out[k]);
            runs_out[k] = nullptr;
        }
        return e;
    };
    gsb_status st = GSB_OK;
    std::vector<int> stop(n);
    int M_max = 0;
    for (int k = 0; k < n; ++k) {
        if (!problems[k] || problems[k]->csr)
            return cleanup(set_error(GSB_EUNSUPPORTED, "gsb_batch_run takes dense problems"));
        if (params[k].eval_every != 0)
            return cleanup(set_error(GSB_EUNSUPPORTED, "batched runs evaluate at t_M only"));
        gsb_params q = params[k];
        q.precision = GSB_PREC_BF16X3;
        q.flags |= GSB_RUN_DEFER;
        q.steps_per_launch = 0;
        if ((st = gsb_run(problems[k], &q, &runs_out[k], s)) != GSB_OK) return cleanup(st);
        stop[k] = (info && info->max_steps > 0) ? std::min(q.M, info->max_steps) : q.M;
        M_max = std::max(M_max, stop[k]);
    }
    GSB_CUDA_TRY(cudaStreamSynchronize(s));
    call_prof_reset();
    const int force = info ? info->force_tiles_per_cta : 0;
    // Window budgets the autotuner tries, in this order until one is slower than
    // the one before: tiles per CTA per step (1: the resident form), and the MB
    // of working set (J, state, V) a window may hold -- within the 129 MB L2 it
    // stays resident across its steps, beyond it more tiles run at once.
    constexpr int kCands[4] = {1, 2, 4, 8};
    constexpr double kCandMB[4] = {80.0, 120.0, 160.0, 240.0};
    constexpr int kProbe = 16;
    int cand = force == 2 ? 1 : force == 4 ? 2 : force == 8 ? 3 : 0;
    int per_cta = kCands[cand];
    double window_mb = kCandMB[cand];
    double ms_probe[4] = {-1.0, -1.0, -1.0, -1.0};
    int windows = 0, grid = 0, graphed = 0;
    if (per_cta != force && M_max >= 8 * kProbe) {
        // real steps of the whole batch under each window size; the instances'
        // trajectories do not depend on the schedule
        cudaEvent_t e0, e1;
        GSB_CUDA_TRY(cudaEventCreate(&e0));
        GSB_CUDA_TRY(cudaEventCreate(&e1));
        double best = 1e300;
        for (int w = 0; w < 4 && st == GSB_OK; ++w) {
            std::vector<int> to(n);
            for (int k = 0; k < n; ++k) to[k] = std::min(stop[k], runs_out[k]->steps_done + kProbe);
            GSB_CUDA_TRY(cudaEventRecord(e0, s));
            st = bf16_batch(runs_out, n, to.data(), kCands[w], kCandMB[w], false, &windows, &grid,
                            &graphed, s);
            GSB_CUDA_TRY(cudaEventRecord(e1, s));
            GSB_CUDA_TRY(cudaEventSynchronize(e1));
            float t = 0.f;
            GSB_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
            ms_probe[w] = t / kProbe;
            for (int k = 0; k < n; ++k) runs_out[k]->steps_done = to[k];
            if (ms_probe[w] < best) {
                best = ms_probe[w];
                per_cta = kCands[w];
                window_mb = kCandMB[w];
            } else {
                // larger windows only lengthened the step: stop probing
                break;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (st != GSB_OK) return cleanup(st);
    }
    windows = grid = graphed = 0;
    if ((st = bf16_batch(runs_out, n, stop.data(), per_cta, window_mb, true, &windows, &grid,
                         &graphed, s)))
        return cleanup(st);
    if ((st = call_prof_collect())) return cleanup(st);
    int tiles = 0, most = 0;
    for (int k = 0; k < n; ++k) {
        gsb_run_state* r = runs_out[k];
        most = std::max(most, stop[k] - r->steps_done);
        r->steps_done = stop[k];
        tiles += ((r->N + 127) / 128) * ((r->R + 127) / 128);
        if (stop[k] == r->params.M)
            if ((st = run_evaluate(r, r->params.M)) != GSB_OK) return cleanup(st);
    }
    GSB_CUDA_TRY(cudaStreamSynchronize(s));
    if (info) {
        info->tile = 128;
        info->steps_per_graph = most;
        info->tiles = tiles;
        info->ms_step_tile128 = -1.0;
        info->ms_step_tile64 = -1.0;
        info->tiles_per_cta = per_cta;
        info->windows = windows;
        info->ctas = grid;
        for (int w = 0; w < 4; ++w) info->ms_step_probe[w] = ms_probe[w];
        info->graphed = graphed;
    }
    return GSB_OK;
}

}  // namespace
}  // namespace gsb

extern "C" gsb_status gsb_batch_run(int32_t n, gsb_problem* const* problems,
                                    const gsb_params* params, gsb_run_state** runs_out,
                                    gsb_batch_info* info, void* stream) {
    if (n < 1 || !problems || !params || !runs_out) return set_error(GSB_EINVAL, "NULL argument or n < 1");
    for (int k = 0; k < n; ++k) runs_out[k] = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    // the form follows the instances' precision, which must agree
    int prec = -1;
    for (int k = 0; k < n; ++k) {
        const int q = params[k].precision == GSB_PREC_FP32 ? GSB_PREC_FP32 : params[k].precision;
        if (q != GSB_PREC_AUTO && q != GSB_PREC_BF16X3 && q != GSB_PREC_FP32)
            return set_error(GSB_EUNSUPPORTED, "batched runs use BF16X3 (or AUTO) or FP32 coupling");
        const int form = q == GSB_PREC_FP32 ? GSB_PREC_FP32 : GSB_PREC_BF16X3;
        if (prec >= 0 && form != prec)
            return set_error(GSB_EINVAL, "batched instances must share one precision form");
        prec = form;
    }
    if (prec == GSB_PREC_BF16X3) return batch_bf16(n, problems, params, runs_out, info, s);
    // the batched steps run (and are captured) on a stream of their own, after
    // everything already queued on the caller's stream
    struct OwnStream {
        cudaStream_t s = nullptr;
        ~OwnStream() {
            if (s) cudaStreamDestroy(s);
        }
    } own;
    GSB_CUDA_TRY(cudaStreamCreateWithFlags(&own.s, cudaStreamNonBlocking));
    gsb_status st = GSB_OK;
    int M_max = 0;
    auto cleanup = [&](gsb_status e) {
        for (int k = 0; k < n; ++k) {
            gsb_run_destroy(runs_out[k]);
            runs_out[k] = nullptr;
        }
        return e;
    };
    for (int k = 0; k < n; ++k) {
        if (!problems[k] || problems[k]->csr)
            return cleanup(set_error(GSB_EUNSUPPORTED, "gsb_batch_run takes dense problems"));
        if (params[k].eval_every != 0)
            return cleanup(set_error(GSB_EUNSUPPORTED, "batched runs evaluate at t_M only"));
        gsb_params q = params[k];
        q.precision = GSB_PREC_FP32;
        q.flags |= GSB_RUN_DEFER;
        if ((st = gsb_run(problems[k], &q, &runs_out[k], stream)) != GSB_OK) return cleanup(st);
        M_max = std::max(M_max, (info && info->max_steps > 0) ? std::min(q.M, info->max_steps) : q.M);
    }
    BatchState B;
    B.n = n;
    std::vector<BatchInst> insts(n);
    std::vector<BatchTile> tiles[2];
    for (int k = 0; k < n; ++k) {
        gsb_run_state* r = runs_out[k];
        BatchInst& I = insts[k];
        I.J = r->prob->J32;
        I.x0 = r->x[0];
        I.x1 = r->x[1];
        I.y = r->y;
        I.p = r->p;
        I.A = r->A;
        I.Np = r->Np;
        I.Rp = r->Rp;
        I.M = r->params.M;
        I.stop = (info && info->max_steps > 0 && info->max_steps < I.M) ? info->max_steps : I.M;
        I.flags = (r->sign_coupling ? 1 : 0) | (r->control ? 2 : 0);
        I.c = r->c;
        I.dt = r->dt;
        I.sched = nullptr;
        I.status = r->status;
        if (!r->sched_host.empty()) {
            float* d = nullptr;
            GSB_CUDA_TRY(cudaMalloc(&d, sizeof(float) * r->sched_host.size()));
            B.scheds.push_back(d);
            GSB_CUDA_TRY(cudaMemcpyAsync(d, r->sched_host.data(), sizeof(float) * r->sched_host.size(),
                                         cudaMemcpyHostToDevice, s));
            I.sched = d;
        }
        for (int w = 0; w < 2; ++w) {
            const int T = w == 0 ? 128 : 64;
            for (int i0 = 0; i0 < r->N; i0 += T)
                for (int r0 = 0; r0 < r->R; r0 += T) tiles[w].push_back({k, i0, r0, r->Np});
        }
    }
    for (int w = 0; w < 2; ++w) {
        // longest K first, so the big tiles start early
        std::stable_sort(tiles[w].begin(), tiles[w].end(),
                         [](const BatchTile& a, const BatchTile& b) { return a.work > b.work; });
        B.ntiles[w] = (int)tiles[w].size();
        GSB_CUDA_TRY(cudaMalloc(&B.d_tiles[w], sizeof(BatchTile) * tiles[w].size()));
        GSB_CUDA_TRY(cudaMemcpyAsync(B.d_tiles[w], tiles[w].data(), sizeof(BatchTile) * tiles[w].size(),
                                     cudaMemcpyHostToDevice, s));
    }
    GSB_CUDA_TRY(cudaMalloc(&B.d_inst, sizeof(BatchInst) * n));
    GSB_CUDA_TRY(cudaMemcpyAsync(B.d_inst, insts.data(), sizeof(BatchInst) * n,
                                 cudaMemcpyHostToDevice, s));
    GSB_CUDA_TRY(cudaMalloc(&B.d_m, sizeof(int)));
    GSB_CUDA_TRY(cudaMemsetAsync(B.d_m, 0, sizeof(int), s));
    GSB_CUDA_TRY(cudaStreamSynchronize(s));
    cudaStream_t caller = s;
    s = own.s;
    call_prof_reset();

    // autotune the tile on the first steps (both sizes give the same bits)
    const int force = info ? info->force_tile : 0;
    cudaEvent_t e0, e1;
    GSB_CUDA_TRY(cudaEventCreate(&e0));
    GSB_CUDA_TRY(cudaEventCreate(&e1));
    int m = 0;
    double ms_tile[2] = {-1.0, -1.0};
    int which = force == 64 ? 1 : 0;
    const int probe = 2;
    if (!force && M_max >= 2 * probe + 2) {
        for (int w = 0; w < 2; ++w) {
            GSB_CUDA_TRY(cudaEventRecord(e0, s));
            for (int k = 0; k < probe; ++k)
                if ((st = launch_batch_step(B, w, s))) return cleanup(st);
            GSB_CUDA_TRY(cudaEventRecord(e1, s));
            GSB_CUDA_TRY(cudaEventSynchronize(e1));
            float t = 0.f;
            GSB_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
            ms_tile[w] = t / probe;
            m += probe;
        }
        which = ms_tile[1] >= 0 && ms_tile[1] < ms_tile[0] ? 1 : 0;
    }
    // graph chunk length: capture G steps once, replay; G tuned among a few sizes
    int chunk = 1;
    double best_ms = 1e300;
    const int cands[3] = {16, 64, 256};
    cudaGraphExec_t exec = nullptr;
    for (int ci = 0; ci < 3 && m < M_max; ++ci) {
        const int G = std::min(cands[ci], M_max - m);
        cudaGraph_t g;
        GSB_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        for (int k = 0; k < G; ++k)
            if ((st = launch_batch_step_raw(B, which, s))) {
                cudaStreamEndCapture(s, &g);
                return cleanup(st);
            }
        GSB_CUDA_TRY(cudaStreamEndCapture(s, &g));
        cudaGraphExec_t ex;
        GSB_CUDA_TRY(cudaGraphInstantiate(&ex, g, 0));
        cudaGraphDestroy(g);
        if ((st = call_prof_begin(s))) return cleanup(st);
        GSB_CUDA_TRY(cudaEventRecord(e0, s));
        GSB_CUDA_TRY(cudaGraphLaunch(ex, s));
        GSB_CUDA_TRY(cudaEventRecord(e1, s));
        if ((st = call_prof_end(s, G))) return cleanup(st);
        GSB_CUDA_TRY(cudaEventSynchronize(e1));
        float t = 0.f;
        GSB_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
        m += G;
        if (t / G < best_ms) {
            best_ms = t / G;
            chunk = G;
            if (exec) cudaGraphExecDestroy(exec);
            exec = ex;
        } else {
            cudaGraphExecDestroy(ex);
        }
        if (G < cands[ci]) break;
    }
    // the remaining steps: full chunks by graph replay, the tail step by step
    while (exec && m + chunk <= M_max) {
        if ((st = call_prof_begin(s))) return cleanup(st);
        GSB_CUDA_TRY(cudaGraphLaunch(exec, s));
        if ((st = call_prof_end(s, chunk))) return cleanup(st);
        m += chunk;
    }
    if (exec) cudaGraphExecDestroy(exec);
    while (m < M_max) {
        if ((st = launch_batch_step(B, which, s))) return cleanup(st);
        ++m;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    GSB_CUDA_TRY(cudaStreamSynchronize(s));
    if ((st = call_prof_collect())) return cleanup(st);
    s = caller;
    // record how far each run got; evaluate the ones that reached t_M
    for (int k = 0; k < n; ++k) {
        gsb_run_state* r = runs_out[k];
        const int stop = insts[k].stop;
        r->steps_done = stop;
        r->cur = stop & 1;
        if (stop == r->params.M)
            if ((st = run_evaluate(r, r->params.M)) != GSB_OK) return cleanup(st);
    }
    if (info) {
        info->tile = which == 0 ? 128 : 64;
        info->steps_per_graph = chunk;
        info->ms_step_tile128 = ms_tile[0];
        info->ms_step_tile64 = ms_tile[1];
        info->tiles = B.ntiles[which];
    }
    GSB_CUDA_TRY(cudaStreamSynchronize(s));
    return GSB_OK;
}
