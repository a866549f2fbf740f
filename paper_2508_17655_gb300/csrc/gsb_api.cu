// gsb_api.cu -- the C ABI declared in include/gsb.h: problem set-up and
// validation, run state, the host loop over time steps, results.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <limits>
#include <string>
#include <vector>
#include <map>
#include <mutex>
#include <unordered_map>

#include "gsb_internal.cuh"

namespace gsb {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};

gsb_status set_error(gsb_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

gsb_status cuda_error(cudaError_t err, const char* what) {
    return set_error(err == cudaErrorMemoryAllocation ? GSB_ENOMEM : GSB_ECUDA,
                     std::string(what) + ": " + cudaGetErrorString(err));
}

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {

// ---- device block cache (see cache_alloc in gsb_internal.cuh)
struct BlockCache {
    std::mutex mu;
    std::map<std::pair<int, size_t>, std::vector<void*>> free;  // (device, bytes) -> blocks
    std::unordered_map<void*, std::pair<int, size_t>> live;      // blocks handed out
    size_t cached = 0;
    size_t in_use = 0;  // bytes handed out
    size_t limit = 0;   // cap on in_use (0: none)
};
BlockCache& block_cache() {
    static BlockCache* c = new BlockCache();  // never destroyed: outlives every handle
    return *c;
}
constexpr size_t kCacheCap = (size_t)1 << 30;

}  // namespace

void* cache_alloc(size_t bytes) {
    if (bytes == 0) return nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    const size_t b = (bytes + 511) & ~(size_t)511;
    BlockCache& c = block_cache();
    {
        std::lock_guard<std::mutex> g(c.mu);
        if (c.limit && c.in_use + b > c.limit) return nullptr;
        // counted before the lock is released, so that two threads allocating
        // at once cannot both pass the cap
        c.in_use += b;
        auto it = c.free.find({dev, b});
        if (it != c.free.end() && !it->second.empty()) {
            void* p = it->second.back();
            it->second.pop_back();
            c.cached -= b;
            c.live[p] = {dev, b};
            return p;
        }
    }
    void* p = nullptr;
    const bool ok = cudaMalloc(&p, b) == cudaSuccess;
    if (!ok) cudaGetLastError();  // the caller reports GSB_ENOMEM; no sticky error remains
    std::lock_guard<std::mutex> g(c.mu);
    if (!ok) {
        c.in_use -= b;
        return nullptr;
    }
    c.live[p] = {dev, b};
    return p;
}

void cache_free(void* p) {
    if (!p) return;
    BlockCache& c = block_cache();
    std::lock_guard<std::mutex> g(c.mu);
    auto it = c.live.find(p);
    if (it == c.live.end()) {
        cudaFree(p);
        return;
    }
    const std::pair<int, size_t> key = it->second;
    c.live.erase(it);
    c.in_use -= key.second;
    if (c.cached + key.second <= kCacheCap) {
        c.free[key].push_back(p);
        c.cached += key.second;
    } else {
        cudaFree(p);
    }
}

gsb_status cache_release() {
    BlockCache& c = block_cache();
    std::lock_guard<std::mutex> g(c.mu);
    int cur = 0;
    cudaGetDevice(&cur);
    cudaError_t err = cudaSuccess;
    for (auto& kv : c.free) {
        if (kv.second.empty()) continue;
        cudaSetDevice(kv.first.first);
        for (void* q : kv.second) {
            const cudaError_t e = cudaFree(q);
            if (e != cudaSuccess) err = e;
        }
    }
    if (!c.free.empty()) cudaSetDevice(cur);
    c.free.clear();
    c.cached = 0;
    return err == cudaSuccess ? GSB_OK : cuda_error(err, "cudaFree");
}

namespace {

gsb_status check_device(int* dev_out) {
    int dev = 0;
    GSB_CUDA_TRY(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    GSB_CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
    if (prop.major != 10 || prop.minor != 3)
        return set_error(GSB_ENODEV, "libgsb is built for sm_103a (GB300); device " +
                                         std::string(prop.name) + " is sm_" +
                                         std::to_string(prop.major) + std::to_string(prop.minor));
    *dev_out = dev;
    return GSB_OK;
}

// J32 -> e4m3 and bf16 copies (exact for the integer ranges they are made for).
__global__ void k_convert_J(const float* __restrict__ J, uint8_t* __restrict__ J8,
                            __nv_bfloat16* __restrict__ J16, size_t n) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float v = J[k];
    if (J8) J8[k] = (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
    if (J16) J16[k] = __float2bfloat16_rn(v);
}

__global__ void k_fill_f64(double* p, double v, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) p[k] = v;
}
__global__ void k_fill_i32(int32_t* p, int32_t v, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) p[k] = v;
}

bool is_integer(float v) { return v == nearbyintf(v); }

void free_problem(gsb_problem* P) {
    if (!P) return;
    // runs on any stream of the problem's device may still read J: the blocks
    // are reused only once that device is idle (as a cudaFree would have
    // waited), whichever device the caller has made current
    int cur = -1;
    const bool switched = cudaGetDevice(&cur) == cudaSuccess && cur != P->device &&
                          cudaSetDevice(P->device) == cudaSuccess;
    cudaDeviceSynchronize();
    dev_free(P->J32);
    dev_free(P->J8);
    dev_free(P->J16);
    dev_free(P->Jhi);
    dev_free(P->Jlo);
    dev_free(P->rowptr);
    dev_free(P->col);
    dev_free(P->val);
    if (switched) cudaSetDevice(cur);
    delete P;
}

// Dense J on the device: padding to Np, the auxiliary spin of h, and per-row
// statistics in one pass, one block per row. Row sums of |J| and of J are
// FP64 in a fixed reduction order; flags[0] collects the largest |J| (as its
// bits), flags[1] bit 0 "not an integer", bit 1 "not finite", bit 2 "nonzero
// diagonal", bit 3 "not symmetric" (bits 1-3 only when validating).
template <typename T>
__global__ void __launch_bounds__(256) k_prepare_J(const T* __restrict__ Jr,
                                                   const float* __restrict__ h, int Nu, int N,
                                                   int Np, int validate, float* __restrict__ J32,
                                                   double* __restrict__ row_abs,
                                                   double* __restrict__ row_sum,
                                                   unsigned* __restrict__ flags) {
    const int i = blockIdx.x;
    auto value = [&](int a, int b) -> float {
        if (a < Nu && b < Nu) return (float)Jr[(size_t)a * Nu + b];
        if (a < Nu) return b == Nu ? h[a] : 0.f;  // column of the auxiliary spin
        return b < Nu ? h[b] : 0.f;               // its row
    };
    double sa = 0.0, ss = 0.0;
    float mx = 0.f;
    unsigned fl = 0u;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const float v = value(i, j);
        J32[(size_t)i * Np + j] = v;
        sa += fabs((double)v);
        ss += (double)v;
        mx = fmaxf(mx, fabsf(v));
        if (v != nearbyintf(v)) fl |= 1u;
        if (validate) {
            if (!isfinite(v)) fl |= 2u;
            if (i == j && v != 0.f) fl |= 4u;
            if (j > i && v != value(j, i)) fl |= 8u;
        }
    }
    __shared__ double ra[256], rs[256];
    ra[threadIdx.x] = sa;
    rs[threadIdx.x] = ss;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            ra[threadIdx.x] += ra[threadIdx.x + w];
            rs[threadIdx.x] += rs[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        row_abs[i] = ra[0];
        row_sum[i] = rs[0];
    }
    const unsigned mfl = __reduce_or_sync(0xffffffffu, fl);
    const unsigned mmx = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));  // mx >= 0
    if ((threadIdx.x & 31) == 0) {
        if (mfl) atomicOr(&flags[1], mfl);
        atomicMax(&flags[0], mmx);
    }
}

// Jr: N_user x N_user row-major (int8 or FP32), on the device; h: N_user
// floats on the device or NULL.
template <typename T>
gsb_status create_dense(gsb_problem* P, const T* Jr, const float* h, bool validate, cudaStream_t s) {
    const int Nu = P->N_user;
    const int N = P->N;
    const int Np = P->Np;
    const size_t n = (size_t)Np * Np;
    gsb_status st;
    if ((st = dev_alloc(&P->J32, n)) != GSB_OK) return st;
    double* stats = nullptr;  // row_abs [N], row_sum [N], then 2 flag words
    if ((st = dev_alloc(&stats, 2 * (size_t)N + 1)) != GSB_OK) return st;
    unsigned* flags = reinterpret_cast<unsigned*>(stats + 2 * (size_t)N);
    std::vector<double> hs(2 * (size_t)N + 1);
    cudaError_t e = cudaMemsetAsync(P->J32, 0, n * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, 2 * sizeof(unsigned), s);
    if (e == cudaSuccess) {
        k_prepare_J<T><<<N, 256, 0, s>>>(Jr, h, Nu, N, Np, validate ? 1 : 0, P->J32, stats,
                                         stats + N, flags);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) count_launch();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hs.data(), stats, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaStreamSynchronize(s);
    dev_free(stats);
    if (e != cudaSuccess) return set_error(GSB_ECUDA, std::string("preparing J: ") + cudaGetErrorString(e));
    unsigned fw[2];
    memcpy(fw, &hs[2 * (size_t)N], sizeof(fw));
    if (fw[1] & 2u) return set_error(GSB_EINVAL, "J has a non-finite entry");
    if (fw[1] & 4u) return set_error(GSB_EINVAL, "J has a nonzero diagonal entry (Eq. 1 needs J_ii = 0)");
    if (fw[1] & 8u) return set_error(GSB_EINVAL, "J is not symmetric (Eq. 1 needs J_ij = J_ji)");
    double max_row = 0.0, sum = 0.0;
    for (int i = 0; i < N; ++i) {
        max_row = std::max(max_row, hs[i]);
        sum += hs[N + i];
    }
    float mx;
    memcpy(&mx, &fw[0], sizeof(mx));
    const bool integer = !(fw[1] & 1u);
    P->integer_J = integer;
    P->max_abs_J = mx;
    P->max_row_abs = max_row;
    P->W_tot = -0.5 * sum;
    if (integer && mx <= 16.f)
        if ((st = dev_alloc(&P->J8, n)) != GSB_OK) return st;
    // FX32 digit planes: every partial sum |sum_j J_ij d_j| <= 128 max row sum stays
    // an exact FP32 integer
    if (integer && mx <= 256.f && 128.0 * max_row < 16777216.0)
        if ((st = dev_alloc(&P->J16, n)) != GSB_OK) return st;
    if (P->J8 || P->J16) {
        k_convert_J<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P->J32, P->J8, P->J16, n);
        GSB_LAUNCH_CHECK("k_convert_J");
    }
    return GSB_OK;
}

// Host-side checks of a CSR matrix (Eq. 1 form): rowptr from 0 to nnz and
// monotone (checked in full before any row is read), column indices in range
// and strictly increasing within each row; with validate also finite values,
// a zero diagonal and the symmetric partner (j, i) of every entry with the same
// value. Needs no GPU.
gsb_status check_csr(int Nu, const int32_t* rp, const int32_t* ci, const float* vv, int64_t nnz,
                     bool validate) {
    if (nnz < 0) return set_error(GSB_EINVAL, "nnz must be >= 0");
    if (rp[0] != 0 || rp[Nu] != nnz) return set_error(GSB_EINVAL, "rowptr must run from 0 to nnz");
    for (int i = 0; i < Nu; ++i)
        if (rp[i + 1] < rp[i]) return set_error(GSB_EINVAL, "rowptr is not monotone");
    for (int i = 0; i < Nu; ++i) {
        int prev = -1;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
            const int j = ci[k];
            if (j < 0 || j >= Nu) return set_error(GSB_EINVAL, "column index out of range");
            if (j <= prev) return set_error(GSB_EINVAL, "column indices must increase within a row");
            prev = j;
        }
    }
    if (!validate) return GSB_OK;
    for (int i = 0; i < Nu; ++i)
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
            const int j = ci[k];
            if (!isfinite(vv[k])) return set_error(GSB_EINVAL, "J has a non-finite entry");
            if (j == i && vv[k] != 0.f)
                return set_error(GSB_EINVAL, "J has a nonzero diagonal entry (Eq. 1 needs J_ii = 0)");
            const int32_t* b = ci + rp[j];
            const int32_t* e = ci + rp[j + 1];
            const int32_t* f = std::lower_bound(b, e, i);
            if (f == e || *f != i || vv[rp[j] + (f - b)] != vv[k])
                return set_error(GSB_EINVAL, "J is not symmetric (Eq. 1 needs J_ij = J_ji)");
        }
    return GSB_OK;
}

// checked: check_csr already ran on these arrays (host input, in gsb_create)
gsb_status create_csr(gsb_problem* P, const int32_t* rp, const int32_t* ci, const float* vv,
                      int64_t nnz, const float* hh, bool validate, bool checked, cudaStream_t s) {
    const int Nu = P->N_user;
    const int N = P->N;
    if (!checked) {
        gsb_status cst = check_csr(Nu, rp, ci, vv, nnz, validate);
        if (cst != GSB_OK) return cst;
    }
    std::vector<int32_t> rowptr(N + 1, 0), col;
    std::vector<float> val;
    col.reserve(nnz + (hh ? 2 * Nu : 0));
    val.reserve(col.capacity());
    for (int i = 0; i < Nu; ++i) {
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
            col.push_back(ci[k]);
            val.push_back(vv[k]);
        }
        if (hh && hh[i] != 0.f) {
            col.push_back(Nu);
            val.push_back(hh[i]);
        }
        rowptr[i + 1] = (int32_t)col.size();
    }
    if (hh) {
        for (int j = 0; j < Nu; ++j)
            if (hh[j] != 0.f) {
                col.push_back(j);
                val.push_back(hh[j]);
            }
        rowptr[N] = (int32_t)col.size();
    }
    bool integer = true;
    float mx = 0.f;
    double sum = 0.0, max_row = 0.0;
    for (float v : val) {
        integer = integer && is_integer(v);
        mx = std::max(mx, fabsf(v));
        sum += v;
    }
    for (int i = 0; i < N; ++i) {
        double row = 0.0;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) row += fabs((double)val[k]);
        max_row = std::max(max_row, row);
    }
    P->integer_J = integer;
    P->max_abs_J = mx;
    P->max_row_abs = max_row;
    P->W_tot = -0.5 * sum;
    P->nnz = (int64_t)col.size();
    gsb_status st;
    if ((st = dev_alloc(&P->rowptr, (size_t)N + 1)) != GSB_OK) return st;
    if ((st = dev_alloc(&P->col, std::max<size_t>(1, col.size()))) != GSB_OK) return st;
    if ((st = dev_alloc(&P->val, std::max<size_t>(1, val.size()))) != GSB_OK) return st;
    GSB_CUDA_TRY(cudaMemcpyAsync(P->rowptr, rowptr.data(), sizeof(int32_t) * (N + 1),
                                 cudaMemcpyHostToDevice, s));
    if (!col.empty()) {
        GSB_CUDA_TRY(cudaMemcpyAsync(P->col, col.data(), sizeof(int32_t) * col.size(),
                                     cudaMemcpyHostToDevice, s));
        GSB_CUDA_TRY(cudaMemcpyAsync(P->val, val.data(), sizeof(float) * val.size(),
                                     cudaMemcpyHostToDevice, s));
    }
    GSB_CUDA_TRY(cudaStreamSynchronize(s));
    return GSB_OK;
}

template <typename T>
std::vector<T> fetch(const T* p, size_t n, bool device) {
    std::vector<T> v(n);
    if (n == 0) return v;
    if (device)
        cudaMemcpy(v.data(), p, sizeof(T) * n, cudaMemcpyDeviceToHost);
    else
        memcpy(v.data(), p, sizeof(T) * n);
    return v;
}

void free_run(gsb_run_state* r) {
    if (!r) return;
    cudaStreamSynchronize(r->stream);  // nothing of the run is in flight
    if (r->tc) tc_free(r);
    for (int b = 0; b < 2; ++b) {
        dev_free(r->x[b]);
        dev_free(r->s8[b]);
        dev_free(r->v8[b]);
        dev_free(r->v16[b]);
    }
    dev_free(r->y);
    dev_free(r->p);
    dev_free(r->A);
    dev_free(r->twin_part);
    dev_free(r->sched);
    dev_free(r->csr_bar);
    dev_free(r->csr_psched);
    dev_free(r->e_acc);
    dev_free(r->best_e);
    dev_free(r->best_step);
    dev_free(r->e_part);
    dev_free(r->best_s);
    dev_free(r->best_out);
    dev_free(r->flag);
    dev_free(r->status);
    for (cudaEvent_t e : r->prof_events) cudaEventDestroy(e);
    delete r;
}

gsb_status evaluate(gsb_run_state* run, int step) {
    if (is_tc_path(run->path)) {
        gsb_status st = tc_energy(run, step);
        if (st != GSB_OK) return st;
        return launch_best_keep(run, step);
    }
    GSB_CUDA_TRY(cudaMemsetAsync(run->e_acc, 0, sizeof(double) * run->Rp, run->stream));
    gsb_status st = run->path == kPathCsr
                        ? launch_csr_energy(run->prob, run->x[run->cur], run->Rp, run->e_acc,
                                            run->stream, run->status)
                        : launch_dense_f32_energy(run->prob, run->x[run->cur], run->Rp,
                                                  run->e_acc, run->e_part, run->stream);
    if (st != GSB_OK) return st;
    return launch_best_keep(run, step);
}

// Clear the status word and the best-state record; zero the profile.
gsb_status reset_bookkeeping(gsb_run_state* run) {
    cudaStream_t s = run->stream;
    GSB_CUDA_TRY(cudaMemsetAsync(run->status, 0, sizeof(int), s));
    GSB_CUDA_TRY(cudaMemsetAsync(run->best_s, 0, (size_t)run->Np * run->Rp, s));
    k_fill_f64<<<(run->Rp + 255) / 256, 256, 0, s>>>(run->best_e,
                                                     std::numeric_limits<double>::infinity(),
                                                     run->Rp);
    k_fill_i32<<<(run->Rp + 255) / 256, 256, 0, s>>>(run->best_step, -1, run->Rp);
    GSB_LAUNCH_CHECK("k_fill");
    run->prof_used = 0;
    run->prof_steps = 0;
    run->steps_done = 0;
    return GSB_OK;
}

bool is_eval_step(const gsb_run_state* run, int step) {
    const int k = run->params.eval_every;
    return step == run->params.M || (k > 0 && step % k == 0);
}

// Shared bifurcation parameter p(t_step) of bSB / dSB: the caller's schedule,
// else Eq. 6, p(t_m) = 1 - m/M (evaluated in double, rounded once).
float p_shared_at(const gsb_run_state* run, int step) {
    if (!run->sched_host.empty()) return run->sched_host[step];
    return (float)(1.0 - (double)step / (double)run->params.M);
}

}  // namespace

gsb_status prof_begin(gsb_run_state* run) {
    if (!(run->params.flags & GSB_RUN_PROFILE)) return GSB_OK;
    if (run->prof_used + 2 > run->prof_events.size()) {
        for (int k = 0; k < 2; ++k) {
            cudaEvent_t e;
            GSB_CUDA_TRY(cudaEventCreate(&e));
            run->prof_events.push_back(e);
        }
    }
    GSB_CUDA_TRY(cudaEventRecord(run->prof_events[run->prof_used], run->stream));
    return GSB_OK;
}

gsb_status prof_end(gsb_run_state* run, int steps) {
    if (!(run->params.flags & GSB_RUN_PROFILE)) return GSB_OK;
    GSB_CUDA_TRY(cudaEventRecord(run->prof_events[run->prof_used + 1], run->stream));
    run->prof_used += 2;
    run->prof_steps += steps;
    return GSB_OK;
}

namespace {
struct CallProfile {
    bool on = false;
    std::vector<cudaEvent_t> ev;
    size_t used = 0;
    double ms = 0.0;
    int64_t launches = 0;
    int64_t steps = 0;
};
thread_local CallProfile g_call_prof;
}  // namespace

void call_prof_reset() {
    g_call_prof.used = 0;
    g_call_prof.ms = 0.0;
    g_call_prof.launches = 0;
    g_call_prof.steps = 0;
}

gsb_status call_prof_begin(cudaStream_t s) {
    CallProfile& c = g_call_prof;
    if (!c.on) return GSB_OK;
    while (c.used + 2 > c.ev.size()) {
        cudaEvent_t e;
        GSB_CUDA_TRY(cudaEventCreate(&e));
        c.ev.push_back(e);
    }
    GSB_CUDA_TRY(cudaEventRecord(c.ev[c.used], s));
    return GSB_OK;
}

gsb_status call_prof_end(cudaStream_t s, int steps) {
    CallProfile& c = g_call_prof;
    if (!c.on) return GSB_OK;
    GSB_CUDA_TRY(cudaEventRecord(c.ev[c.used + 1], s));
    c.used += 2;
    c.launches += 1;
    c.steps += steps;
    return GSB_OK;
}

gsb_status call_prof_collect() {
    CallProfile& c = g_call_prof;
    if (!c.on) return GSB_OK;
    double total = 0.0;
    for (size_t k = 0; k + 1 < c.used; k += 2) {
        GSB_CUDA_TRY(cudaEventSynchronize(c.ev[k + 1]));
        float t = 0.f;
        GSB_CUDA_TRY(cudaEventElapsedTime(&t, c.ev[k], c.ev[k + 1]));
        total += t;
    }
    c.ms = total;
    c.used = 0;
    return GSB_OK;
}

bool run_is_eval_step(const gsb_run_state* run, int step) { return is_eval_step(run, step); }
float run_p_shared(const gsb_run_state* run, int step) { return p_shared_at(run, step); }
gsb_status run_evaluate(gsb_run_state* run, int step) { return evaluate(run, step); }

}  // namespace gsb

using namespace gsb;

extern "C" {

const char* gsb_last_error(void) { return g_last_error.c_str(); }

gsb_status gsb_set_call_profiling(int32_t on) {
    g_call_prof.on = on != 0;
    call_prof_reset();
    return GSB_OK;
}

gsb_status gsb_last_call_profile(double* kernel_ms, int64_t* launches, int64_t* steps) {
    if (kernel_ms) *kernel_ms = g_call_prof.ms;
    if (launches) *launches = g_call_prof.launches;
    if (steps) *steps = g_call_prof.steps;
    return GSB_OK;
}
int32_t gsb_version(void) { return 100; }
int64_t gsb_launch_count(void) { return g_launches.load(); }

gsb_status gsb_create(gsb_problem** out, int32_t N, int32_t format, const void* J,
                      const int32_t* rowptr, const int32_t* col, const float* val, int64_t nnz,
                      const float* h, uint32_t flags, void* stream) {
    if (!out) return set_error(GSB_EINVAL, "out is NULL");
    *out = nullptr;
    if (N < 1) return set_error(GSB_EINVAL, "N must be >= 1");
    if (N > (1 << 20)) return set_error(GSB_EINVAL, "N too large");
    // a host CSR matrix is checked before anything touches the device
    if (format == GSB_J_CSR_F32 && !(flags & GSB_CREATE_DEVICE_INPUT)) {
        if (J || !rowptr || (nnz > 0 && (!col || !val)) || nnz < 0)
            return set_error(GSB_EINVAL, "CSR format takes rowptr, col, val");
        gsb_status cst = check_csr(N, rowptr, col, val, nnz, !(flags & GSB_CREATE_NO_VALIDATE));
        if (cst != GSB_OK) return cst;
    }
    int dev = 0;
    gsb_status st = check_device(&dev);
    if (st != GSB_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const bool device_in = flags & GSB_CREATE_DEVICE_INPUT;
    const bool validate = !(flags & GSB_CREATE_NO_VALIDATE);
    gsb_problem* P = new gsb_problem();
    P->device = dev;
    P->N_user = N;
    P->has_h = h != nullptr;
    P->N = N + (h ? 1 : 0);
    P->Np = round_up(P->N, kTile);
    std::vector<float> hv;
    if (h) hv = fetch(h, (size_t)N, device_in);
    if (format == GSB_J_DENSE_I8 || format == GSB_J_DENSE_F32) {
        if (!J || rowptr || col || val || nnz) {
            free_problem(P);
            return set_error(GSB_EINVAL, "dense formats take J only");
        }
        if ((int64_t)P->Np * P->Np > (int64_t)1 << 32) {
            free_problem(P);
            return set_error(GSB_EINVAL, "dense J too large; use CSR");
        }
        // the raw J (and h) on the device, then padding and checks there
        const size_t eb = format == GSB_J_DENSE_I8 ? 1 : sizeof(float);
        const size_t nb = (size_t)N * N * eb;
        void* Jd = nullptr;
        float* hd = nullptr;
        cudaError_t e = cudaSuccess;
        if (!device_in) {
            Jd = cache_alloc(nb);
            e = Jd ? cudaMemcpyAsync(Jd, J, nb, cudaMemcpyHostToDevice, s) : cudaErrorMemoryAllocation;
        }
        if (e == cudaSuccess && h) {
            hd = (float*)cache_alloc(sizeof(float) * N);
            e = hd ? cudaMemcpyAsync(hd, hv.data(), sizeof(float) * N, cudaMemcpyHostToDevice, s)
                   : cudaErrorMemoryAllocation;
        }
        if (e != cudaSuccess) {
            cudaStreamSynchronize(s);
            dev_free(Jd);
            dev_free(hd);
            free_problem(P);
            return set_error(e == cudaErrorMemoryAllocation ? GSB_ENOMEM : GSB_ECUDA,
                             std::string("uploading J: ") + cudaGetErrorString(e));
        }
        const void* Jsrc = device_in ? J : Jd;
        if (format == GSB_J_DENSE_I8)
            st = create_dense(P, (const int8_t*)Jsrc, hd, validate, s);
        else
            st = create_dense(P, (const float*)Jsrc, hd, validate, s);
        cudaStreamSynchronize(s);  // the temporaries may be in use by the conversion
        dev_free(Jd);
        dev_free(hd);
    } else if (format == GSB_J_CSR_F32) {
        if (J || !rowptr || (nnz > 0 && (!col || !val)) || nnz < 0) {
            free_problem(P);
            return set_error(GSB_EINVAL, "CSR format takes rowptr, col, val");
        }
        auto rp = fetch(rowptr, (size_t)N + 1, device_in);
        auto ci = fetch(col, (size_t)nnz, device_in);
        auto vv = fetch(val, (size_t)nnz, device_in);
        P->csr = true;
        st = create_csr(P, rp.data(), ci.data(), vv.data(), nnz, h ? hv.data() : nullptr,
                        validate, !device_in, s);
    } else {
        free_problem(P);
        return set_error(GSB_EINVAL, "unknown J format");
    }
    if (st != GSB_OK) {
        free_problem(P);
        return st;
    }
    *out = P;
    return GSB_OK;
}

// QUBO f(b) = sum_ij Q_ij b_i b_j, b in {0,1}^N, as an Ising problem (Eq. 1
// with a local field) under s = 2b - 1. With Qs = (Q + Q^T)/2,
//   f = 1/4 sum_{i!=j} Qs_ij s_i s_j + 1/2 sum_i s_i sum_j Qs_ij
//       + 1/4 sum_ij Q_ij + 1/4 sum_i Q_ii,
// so J_ij = -Qs_ij / 2 (i != j), h_i = -sum_j Qs_ij / 2 give f = E(s) + const.
// Everything is scaled by 4 so that integer Q gives integer J and h:
// J'_ij = -(Q_ij + Q_ji), h'_i = -sum_j (Q_ij + Q_ji), f = E'/4 + offset.
gsb_status gsb_qubo_to_ising(int32_t N, const float* Q, float* J, float* h, double* scale,
                             double* offset) {
    if (N < 1 || N > (1 << 16)) return set_error(GSB_EINVAL, "N must be in 1..65536");
    if (!Q || !J || !h) return set_error(GSB_EINVAL, "Q, J and h are required");
    const size_t n = (size_t)N;
    double total = 0.0, diag = 0.0;
    for (size_t i = 0; i < n; ++i) {
        double hs = 0.0;
        for (size_t j = 0; j < n; ++j) {
            const double a = Q[i * n + j], b = Q[j * n + i];
            if (!isfinite(a)) return set_error(GSB_EINVAL, "Q has a non-finite entry");
            total += a;
            hs += a + b;
            J[i * n + j] = i == j ? 0.f : (float)(-(a + b));
        }
        diag += Q[i * n + i];
        h[i] = (float)(-hs);
    }
    if (scale) *scale = 0.25;
    if (offset) *offset = 0.25 * (total + diag);
    return GSB_OK;
}

gsb_status gsb_create_qubo(gsb_problem** out, int32_t N, const float* Q, uint32_t flags,
                           double* scale, double* offset, void* stream) {
    if (!out) return set_error(GSB_EINVAL, "out is NULL");
    *out = nullptr;
    if (N < 1 || N > (1 << 16)) return set_error(GSB_EINVAL, "N must be in 1..65536");
    if (!Q) return set_error(GSB_EINVAL, "Q is NULL");
    if (flags & ~(uint32_t)GSB_CREATE_DEVICE_INPUT)
        return set_error(GSB_EINVAL, "gsb_create_qubo takes GSB_CREATE_DEVICE_INPUT only");
    const size_t n = (size_t)N * N;
    std::vector<float> q = fetch(Q, n, (flags & GSB_CREATE_DEVICE_INPUT) != 0);
    std::vector<float> J(n), h((size_t)N);
    gsb_status st = gsb_qubo_to_ising(N, q.data(), J.data(), h.data(), scale, offset);
    if (st != GSB_OK) return st;
    // J is symmetric with a zero diagonal by construction
    return gsb_create(out, N, GSB_J_DENSE_F32, J.data(), nullptr, nullptr, nullptr, 0, h.data(),
                      0u, stream);
}

gsb_status gsb_destroy(gsb_problem* problem) {
    free_problem(problem);
    return GSB_OK;
}

gsb_status gsb_release_cached_memory(void) { return cache_release(); }

gsb_status gsb_set_memory_limit(int64_t bytes) {
    if (bytes < 0) return set_error(GSB_EINVAL, "bytes must be >= 0");
    BlockCache& c = block_cache();
    std::lock_guard<std::mutex> g(c.mu);
    c.limit = (size_t)bytes;
    return GSB_OK;
}

gsb_status gsb_memory_usage(int64_t* in_use, int64_t* kept) {
    BlockCache& c = block_cache();
    std::lock_guard<std::mutex> g(c.mu);
    if (in_use) *in_use = (int64_t)c.in_use;
    if (kept) *kept = (int64_t)c.cached;
    return GSB_OK;
}

gsb_status gsb_problem_info(gsb_problem* P, int32_t* n_spins, double* lmax, double* lmin,
                            void* stream) {
    if (!P) return set_error(GSB_EINVAL, "problem is NULL");
    if (n_spins) *n_spins = P->N;
    if (lmax || lmin) {
        gsb_status st = compute_lambda(P, (cudaStream_t)stream);
        if (st != GSB_OK) return st;
        if (lmax) *lmax = P->lambda_max;
        if (lmin) *lmin = P->lambda_min;
    }
    return GSB_OK;
}

gsb_status gsb_run(gsb_problem* P, const gsb_params* prm, gsb_run_state** out, void* stream) {
    if (!P || !prm || !out) return set_error(GSB_EINVAL, "NULL argument");
    *out = nullptr;
    const gsb_params& Q = *prm;
    if (Q.variant < GSB_BSB || Q.variant > GSB_GDSB) return set_error(GSB_EINVAL, "unknown variant");
    if (Q.M < 1) return set_error(GSB_EINVAL, "M must be >= 1");
    if (Q.R < 1 || Q.R > (1 << 22)) return set_error(GSB_EINVAL, "R out of range");
    if (Q.c < 0 || Q.dt < 0 || !isfinite(Q.c) || !isfinite(Q.dt))
        return set_error(GSB_EINVAL, "c and dt must be >= 0 and finite");
    if (Q.eval_every < 0) return set_error(GSB_EINVAL, "eval_every must be >= 0");
    if (Q.x0_range < 0) return set_error(GSB_EINVAL, "x0_range must be >= 0");
    const bool sign = Q.variant == GSB_DSB || Q.variant == GSB_GDSB;
    const bool control = Q.variant == GSB_GBSB || Q.variant == GSB_GDSB;
    if (Q.schedule && control)
        return set_error(GSB_EINVAL, "a schedule applies to bSB / dSB only (GbSB uses Eq. 7)");
    int path = kPathDenseF32;
    if (P->csr) {
        if (Q.precision != GSB_PREC_AUTO && Q.precision != GSB_PREC_FP32)
            return set_error(GSB_EUNSUPPORTED,
                             "CSR problems take GSB_PREC_AUTO or GSB_PREC_FP32 (the CSR path)");
        path = kPathCsr;
    } else {
        switch (Q.precision) {
            case GSB_PREC_AUTO:
                if (!tc_available())
                    path = kPathDenseF32;
                else if (sign && P->J8)
                    path = kPathTcFp8;
                else if (!sign && P->J16)
                    path = kPathTcFx32;
                else if (!P->integer_J)
                    path = kPathTcBf16;  // real-valued J: split bf16
                else
                    path = kPathDenseF32;
                break;
            case GSB_PREC_FP32: path = kPathDenseF32; break;
            case GSB_PREC_FP8:
                if (!sign)
                    return set_error(GSB_EUNSUPPORTED, "FP8 serves the sgn-x coupling (dSB, GdSB)");
                if (!P->J8)
                    return set_error(GSB_EUNSUPPORTED, "FP8 needs integer J with |J| <= 16");
                path = kPathTcFp8;
                break;
            case GSB_PREC_FX32:
                if (!P->J16)
                    return set_error(GSB_EUNSUPPORTED,
                                     "FX32 needs integer J with 128 max_i sum_j |J_ij| < 2^24");
                path = kPathTcFx32;
                break;
            case GSB_PREC_BF16X3: path = kPathTcBf16; break;
            case GSB_PREC_FX16:
                if (sign)
                    return set_error(GSB_EUNSUPPORTED, "FX16 serves the x coupling (bSB, GbSB)");
                if (!P->J8 || !(136.0 * P->max_row_abs < 16777216.0))
                    return set_error(GSB_EUNSUPPORTED,
                                     "FX16 needs integer J with |J| <= 16 and "
                                     "136 max_i sum_j |J_ij| < 2^24");
                path = kPathTcFx16;
                break;
            default: return set_error(GSB_EINVAL, "unknown precision");
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    double c = Q.c, dt = Q.dt;
    if (c == 0.0 || dt == 0.0) {
        gsb_status st = compute_lambda(P, s);
        if (st != GSB_OK) return st;
        if (!(P->lambda_max > 0.0))
            return set_error(GSB_EINVAL, "lambda_max <= 0: set c and dt explicitly");
        if (c == 0.0) c = 1.0 / P->lambda_max;  // App. A
        if (dt == 0.0) dt = 1.25 * sqrt(2.0 / (1.0 - P->lambda_min / P->lambda_max));  // Eq. 13
    }
    gsb_run_state* run = new gsb_run_state();
    run->prob = P;
    run->params = Q;
    run->params.A_per_replica = nullptr;
    run->params.schedule = nullptr;
    run->params.x0 = nullptr;
    run->params.y0 = nullptr;
    run->path = path;
    run->stream = s;
    run->N = P->N;
    run->Np = P->Np;
    run->R = Q.R;
    run->Rp = round_up(Q.R, kTile);
    run->c = (float)c;
    run->dt = (float)dt;
    run->sign_coupling = sign;
    run->control = control;
    const size_t nst = (size_t)run->Np * run->Rp;
    gsb_status st = GSB_OK;
    auto fail = [&](gsb_status e) {
        free_run(run);
        return e;
    };
    if ((st = dev_alloc(&run->x[0], nst)) || (st = dev_alloc(&run->y, nst))) return fail(st);
    if (!is_tc_path(path))
        if ((st = dev_alloc(&run->x[1], nst))) return fail(st);
    if (control)
        if ((st = dev_alloc(&run->p, nst))) return fail(st);
    if (path == kPathCsr && sign)
        if ((st = dev_alloc(&run->s8[0], nst)) || (st = dev_alloc(&run->s8[1], nst)))
            return fail(st);
    if (!P->csr && (st = dev_alloc(&run->e_part, (size_t)(run->Np / kTile) * run->Rp)))
        return fail(st);
    if ((st = dev_alloc(&run->A, run->Rp)) || (st = dev_alloc(&run->e_acc, run->Rp)) ||
        (st = dev_alloc(&run->best_e, run->Rp)) || (st = dev_alloc(&run->best_step, run->Rp)) ||
        (st = dev_alloc(&run->flag, run->Rp)) || (st = dev_alloc(&run->best_s, nst)) ||
        (st = dev_alloc(&run->status, 1)))
        return fail(st);
    {
        std::vector<float> Ah(run->Rp, 0.f);
        for (int r = 0; r < Q.R; ++r) Ah[r] = Q.A_per_replica ? Q.A_per_replica[r] : Q.A;
        if (cudaMemcpyAsync(run->A, Ah.data(), sizeof(float) * run->Rp, cudaMemcpyHostToDevice,
                            s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "copy A"));
    }
    if (Q.schedule) run->sched_host.assign(Q.schedule, Q.schedule + Q.M + 1);
    if ((st = reset_bookkeeping(run))) return fail(st);
    // initial state
    float *x0d = nullptr, *y0d = nullptr;
    const size_t nrm = (size_t)Q.R * P->N;
    if (Q.x0 || Q.y0) {
        if (P->has_h) return fail(set_error(GSB_EINVAL, "explicit x0/y0 with h: pass N+1 columns is unsupported"));
    }
    if (Q.x0) {
        if ((st = dev_alloc(&x0d, nrm))) return fail(st);
        GSB_CUDA_TRY(cudaMemcpyAsync(x0d, Q.x0, sizeof(float) * nrm, cudaMemcpyHostToDevice, s));
    }
    if (Q.y0) {
        if ((st = dev_alloc(&y0d, nrm))) return fail(st);
        GSB_CUDA_TRY(cudaMemcpyAsync(y0d, Q.y0, sizeof(float) * nrm, cudaMemcpyHostToDevice, s));
    }
    st = launch_init_state(run, x0d, y0d);
    if (x0d || y0d) {
        cudaStreamSynchronize(s);
        dev_free(x0d);
        dev_free(y0d);
    }
    if (st != GSB_OK) return fail(st);
    if (is_tc_path(path)) {
        if ((st = tc_setup(run)) != GSB_OK) return fail(st);
    } else if (path == kPathCsr) {
        if ((st = csr_setup(run)) != GSB_OK) return fail(st);
    }
    *out = run;
    if (!(Q.flags & GSB_RUN_DEFER)) {
        st = gsb_run_steps(run, Q.M);
        if (st != GSB_OK) {
            *out = nullptr;
            gsb_run_destroy(run);
            return st;
        }
    }
    return GSB_OK;
}

gsb_status gsb_run_steps(gsb_run_state* run, int32_t nsteps) {
    if (!run) return set_error(GSB_EINVAL, "run is NULL");
    if (nsteps < 0 || run->steps_done + nsteps > run->params.M)
        return set_error(GSB_EINVAL, "nsteps exceeds the remaining steps of the run");
    const int M = run->params.M;
    if (is_tc_path(run->path) || (run->path == kPathCsr && run->csr_grid > 0)) {
        gsb_status st = is_tc_path(run->path) ? tc_steps(run, run->steps_done, nsteps)
                                              : csr_steps(run, run->steps_done, nsteps);
        if (st == GSB_OK) run->steps_done += nsteps;
        return st;
    }
    for (int k = 0; k < nsteps; ++k) {
        const int m = run->steps_done;
        StepScalars sc;
        sc.m = m;
        sc.M = M;
        sc.c = run->c;
        sc.dt = run->dt;
        sc.p_next = p_shared_at(run, m + 1);
        gsb_status st = prof_begin(run);
        if (st != GSB_OK) return st;
        st = run->path == kPathCsr ? launch_csr_step(run, sc) : launch_dense_f32_step(run, sc);
        if (st != GSB_OK) return st;
        if ((st = prof_end(run, 1)) != GSB_OK) return st;
        run->steps_done = m + 1;
        if (is_eval_step(run, m + 1)) {
            if ((st = evaluate(run, m + 1)) != GSB_OK) return st;
        }
    }
    return GSB_OK;
}


static gsb_status check_status_word(gsb_run_state* run) {
    int st = 0;
    GSB_CUDA_TRY(cudaMemcpyAsync(&st, run->status, sizeof(int), cudaMemcpyDeviceToHost, run->stream));
    GSB_CUDA_TRY(cudaStreamSynchronize(run->stream));
    if (st & kDevTimeout) return set_error(GSB_ETIMEOUT, "a device-side wait timed out");
    if (st & kDevBounds) return set_error(GSB_ECUDA, "a kernel detected an out-of-range index");
    if (st & kDevNumeric) return set_error(GSB_ENUMERIC, "NaN or Inf in the state");
    return GSB_OK;
}

gsb_status gsb_best(gsb_run_state* run, int8_t* spins, double* energies, double* cuts,
                    int32_t* step_found) {
    if (!run) return set_error(GSB_EINVAL, "run is NULL");
    gsb_status st = check_status_word(run);
    if (st != GSB_OK) return st;
    const int R = run->R, N = run->N, Nu = run->prob->N_user;
    std::vector<double> e(R);
    std::vector<int32_t> stp(R);
    GSB_CUDA_TRY(cudaMemcpyAsync(e.data(), run->best_e, sizeof(double) * R, cudaMemcpyDeviceToHost,
                                 run->stream));
    GSB_CUDA_TRY(cudaMemcpyAsync(stp.data(), run->best_step, sizeof(int32_t) * R,
                                 cudaMemcpyDeviceToHost, run->stream));
    // spins: transposed on the device into the host layout, then copied straight
    // into the caller's array (no auxiliary spin), or staged for the gauge fix
    std::vector<int8_t> s;
    const bool direct = !run->prob->has_h;
    if (spins) {
        if (!run->best_out && (st = dev_alloc(&run->best_out, (size_t)R * N))) return st;
        if ((st = launch_transpose_i8_to_host_layout(run->best_s, run->best_out, run->Np,
                                                     run->Rp, N, R, run->stream)))
            return st;
        int8_t* dst = spins;
        if (!direct) {
            s.resize((size_t)R * N);
            dst = s.data();
        }
        GSB_CUDA_TRY(cudaMemcpyAsync(dst, run->best_out, (size_t)R * N, cudaMemcpyDeviceToHost,
                                     run->stream));
    }
    GSB_CUDA_TRY(cudaStreamSynchronize(run->stream));
    for (int r = 0; r < R; ++r) {
        if (energies) energies[r] = e[r];
        if (cuts) cuts[r] = isfinite(e[r]) ? 0.5 * (run->prob->W_tot - e[r]) : -INFINITY;
        if (step_found) step_found[r] = stp[r];
        if (spins && !direct) {
            const int8_t* src = &s[(size_t)r * N];
            // gauge-fix the auxiliary spin of the h augmentation to +1
            const int8_t g = (run->prob->has_h && src[Nu] < 0) ? -1 : 1;
            for (int i = 0; i < Nu; ++i) spins[(size_t)r * Nu + i] = (int8_t)(g * src[i]);
        }
    }
    return GSB_OK;
}

gsb_status gsb_get_state(gsb_run_state* run, float* x, float* y, float* p, int32_t* steps_done) {
    if (!run) return set_error(GSB_EINVAL, "run is NULL");
    gsb_status st = GSB_OK;
    const int R = run->R, N = run->N;
    if (is_tc_path(run->path)) {
        // the fused path keeps x, y, p in its own buffers; they are synced after every call
    }
    float* tmp = nullptr;
    if ((st = dev_alloc(&tmp, (size_t)R * N))) return st;
    struct Item {
        const float* src;
        float* dst;
    } items[3] = {{run->x[run->cur], x}, {run->y, y}, {run->control ? run->p : nullptr, p}};
    for (auto& it : items) {
        if (!it.dst) continue;
        if (it.src) {
            st = launch_transpose_to_host_layout(it.src, tmp, run->Np, run->Rp, N, R, run->stream);
            if (st != GSB_OK) break;
            if (cudaMemcpyAsync(it.dst, tmp, sizeof(float) * R * N, cudaMemcpyDeviceToHost,
                                run->stream) != cudaSuccess ||
                cudaStreamSynchronize(run->stream) != cudaSuccess) {
                st = cuda_error(cudaGetLastError(), "copy state");
                break;
            }
        } else {
            const float pv = run->steps_done == 0 ? 1.f : run_p_shared(run, run->steps_done);
            for (size_t k = 0; k < (size_t)R * N; ++k) it.dst[k] = pv;
        }
    }
    cudaStreamSynchronize(run->stream);
    dev_free(tmp);
    if (st != GSB_OK) return st;
    if (steps_done) *steps_done = run->steps_done;
    return check_status_word(run);
}

gsb_status gsb_run_set_state(gsb_run_state* run, const float* x, const float* y, const float* p,
                             int32_t steps_done, const int8_t* best_spins,
                             const double* best_energies, const int32_t* best_step) {
    if (!run || !x || !y) return set_error(GSB_EINVAL, "run, x and y are required");
    if (steps_done < 0 || steps_done > run->params.M)
        return set_error(GSB_EINVAL, "steps_done must be in 0..M");
    if (run->control && !p) return set_error(GSB_EINVAL, "p is required for GbSB / GdSB");
    const bool best = best_spins && best_energies && best_step;
    if (!best && (best_spins || best_energies || best_step))
        return set_error(GSB_EINVAL, "best records: all three or none");
    const int R = run->R, N = run->N, Nu = run->prob->N_user;
    cudaStream_t s = run->stream;
    gsb_status st;
    GSB_CUDA_TRY(cudaStreamSynchronize(s));
    if ((st = reset_bookkeeping(run))) return st;
    float* tmp = nullptr;
    int8_t* tmp8 = nullptr;
    if ((st = dev_alloc(&tmp, (size_t)R * N))) return st;
    struct Item {
        const float* src;
        float* dst;
    } items[3] = {{x, run->x[0]}, {y, run->y}, {run->control ? p : nullptr, run->p}};
    do {
        for (const Item& it : items) {
            if (!it.src) continue;
            if (cudaMemcpyAsync(tmp, it.src, sizeof(float) * (size_t)R * N,
                                cudaMemcpyHostToDevice, s) != cudaSuccess) {
                st = cuda_error(cudaGetLastError(), "copy state");
                break;
            }
            if ((st = launch_rm_to_sm(tmp, it.dst, N, N, R, run->Np, run->Rp, s))) break;
            // the stage is reused by the next array only after this transpose
            if (cudaStreamSynchronize(s) != cudaSuccess) {
                st = cuda_error(cudaGetLastError(), "copy state");
                break;
            }
        }
        if (st != GSB_OK || !best) break;
        // best records: spins in the user layout (the auxiliary spin of h is +1)
        if ((st = dev_alloc(&tmp8, (size_t)R * Nu))) break;
        if (cudaMemcpyAsync(tmp8, best_spins, (size_t)R * Nu, cudaMemcpyHostToDevice, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(run->best_e, best_energies, sizeof(double) * R,
                            cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(run->best_step, best_step, sizeof(int32_t) * R,
                            cudaMemcpyHostToDevice, s) != cudaSuccess) {
            st = cuda_error(cudaGetLastError(), "copy best records");
            break;
        }
        st = launch_rm_to_sm_i8(tmp8, run->best_s, Nu, N, R, run->Np, run->Rp, (int8_t)1, s);
    } while (0);
    cudaStreamSynchronize(s);
    dev_free(tmp);
    dev_free(tmp8);
    if (st != GSB_OK) return st;
    run->cur = 0;
    run->steps_done = steps_done;
    // operands derived from x: sgn x for the CSR sign coupling, V for the tensor cores
    if (run->s8[0] && (st = launch_sign_extract(run))) return st;
    if (is_tc_path(run->path) && (st = tc_prepare(run))) return st;
    return GSB_OK;
}

gsb_status gsb_energy(gsb_problem* P, int32_t R, const int8_t* spins, double* energies,
                      void* stream) {
    if (!P || !spins || !energies || R < 1) return set_error(GSB_EINVAL, "bad argument");
    if (P->has_h) return set_error(GSB_EUNSUPPORTED, "gsb_energy takes problems without h");
    cudaStream_t s = (cudaStream_t)stream;
    const int Rp = round_up(R, kTile);
    const size_t nst = (size_t)P->Np * Rp;
    int8_t* sd = nullptr;
    float* xd = nullptr;
    double* acc = nullptr;
    gsb_status st = GSB_OK;
    // acc: the Rp sums, then (dense) the per-row-block partials they are made from
    if ((st = dev_alloc(&sd, (size_t)R * P->N)) || (st = dev_alloc(&xd, nst)) ||
        (st = dev_alloc(&acc, (size_t)Rp * (1 + P->Np / kTile)))) {
        dev_free(sd);
        dev_free(xd);
        dev_free(acc);
        return st;
    }
    std::vector<double> h(R);
    do {
        if (cudaMemcpyAsync(sd, spins, (size_t)R * P->N, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            st = cuda_error(cudaGetLastError(), "copy spins");
            break;
        }
        if ((st = launch_spins_to_state(sd, xd, P->N, R, P->Np, Rp, s)) != GSB_OK) break;
        if (cudaMemsetAsync(acc, 0, sizeof(double) * Rp, s) != cudaSuccess) {
            st = cuda_error(cudaGetLastError(), "memset");
            break;
        }
        st = P->csr ? launch_csr_energy(P, xd, Rp, acc, s)
                    : launch_dense_f32_energy(P, xd, Rp, acc, acc + Rp, s);
        if (st != GSB_OK) break;
        if (cudaMemcpyAsync(h.data(), acc, sizeof(double) * R, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            st = cuda_error(cudaGetLastError(), "copy energies");
            break;
        }
        for (int r = 0; r < R; ++r) energies[r] = -0.5 * h[r];
    } while (0);
    cudaStreamSynchronize(s);
    dev_free(sd);
    dev_free(xd);
    dev_free(acc);
    return st;
}

gsb_status gsb_run_restart(gsb_run_state* run, uint64_t seed, uint32_t flags) {
    if (!run) return set_error(GSB_EINVAL, "run is NULL");
    run->params.seed = seed;
    gsb_status st = reset_bookkeeping(run);
    if (st != GSB_OK) return st;
    if ((st = launch_init_state(run, nullptr, nullptr)) != GSB_OK) return st;
    if (is_tc_path(run->path))
        if ((st = tc_prepare(run)) != GSB_OK) return st;
    if (flags & GSB_RUN_DEFER) return GSB_OK;
    return gsb_run_steps(run, run->params.M);
}

const char* gsb_run_kernel(const gsb_run_state* run) {
    if (!run) return "";
    if (run->path == kPathDenseF32) return "k_dense_f32_step";
    if (run->path == kPathCsr) return run->csr_grid > 0 ? "k_csr_persist" : "k_csr_step";
    return tc_kernel_name(run);
}

gsb_status gsb_kernel_time(gsb_run_state* run, double* ms, int64_t* launches, int64_t* steps) {
    if (!run) return set_error(GSB_EINVAL, "run is NULL");
    GSB_CUDA_TRY(cudaStreamSynchronize(run->stream));
    double total = 0.0;
    for (size_t k = 0; k + 1 < run->prof_used; k += 2) {
        float t = 0.f;
        GSB_CUDA_TRY(cudaEventElapsedTime(&t, run->prof_events[k], run->prof_events[k + 1]));
        total += t;
    }
    if (ms) *ms = total;
    if (launches) *launches = (int64_t)(run->prof_used / 2);
    if (steps) *steps = run->prof_steps;
    return GSB_OK;
}

gsb_status gsb_run_destroy(gsb_run_state* run) {
    if (!run) return GSB_OK;
    cudaStreamSynchronize(run->stream);
    free_run(run);
    return GSB_OK;
}

int32_t gsb_debug_build(void) {
#ifdef GSB_DEBUG
    return 1;
#else
    return 0;
#endif
}

gsb_status gsb_debug_selftest(void) {
#ifndef GSB_DEBUG
    return set_error(GSB_EUNSUPPORTED, "gsb_debug_selftest needs the GSB_DEBUG build");
#else
    cudaStream_t s = nullptr;
    int* status = nullptr;
    gsb_status st = dev_alloc(&status, 1);
    if (st != GSB_OK) return st;
    int got[2] = {0, 0};
    for (int k = 0; k < 2 && st == GSB_OK; ++k) {
        if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) {
            st = cuda_error(cudaGetLastError(), "debug self-test");
            break;
        }
        st = k == 0 ? csr_debug_selftest(status, s) : tc_debug_selftest(status, s);
        if (st == GSB_OK &&
            cudaMemcpy(&got[k], status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            st = cuda_error(cudaGetLastError(), "debug self-test");
    }
    dev_free(status);
    if (st != GSB_OK) return st;
    if (!(got[0] & kDevBounds))
        return set_error(GSB_ECUDA, "the CSR column check did not fire");
    if (!(got[1] & kDevBounds))
        return set_error(GSB_ECUDA, "the FP8 energy kernel's grid check did not fire");
    return GSB_OK;
#endif
}

}  // extern "C"
