// gsb_internal.cuh -- types and helpers shared by the libgsb translation units.
#pragma once

#include <atomic>
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gsb.h"

namespace gsb {

// Padding unit of the spin (row) dimension and of the replica dimension: one
// tcgen05 accumulator tile is 128 spins (TMEM lanes) by 128 replicas (columns).
constexpr int kTile = 128;

inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

enum Path : int {
    kPathDenseF32 = 0,  // FP32 CUDA-core coupling (the plain form)
    kPathCsr = 1,       // CSR coupling
    kPathTcFp8 = 2,     // tcgen05 e4m3, sgn x coupling
    kPathTcFx32 = 3,    // tcgen05 bf16, x as 32-bit fixed point in four digit planes
    kPathTcBf16 = 4,    // tcgen05 bf16, J and x split into hi + lo bf16 terms
    kPathTcFx16 = 5,    // tcgen05 e4m3, x on the 16-bit fixed-point grid in four digit planes
};

inline bool is_tc_path(int path) {
    return path == kPathTcFp8 || path == kPathTcFx32 || path == kPathTcBf16 ||
           path == kPathTcFx16;
}

// Device status word bits (written by kernels, read by the host).
enum DevStatus : int {
    kDevOk = 0,
    kDevTimeout = 1,
    kDevNumeric = 2,
    kDevBounds = 4,
};

// Device-side bounds checks of the debug build (-DGSB_DEBUG, built beside the
// release library as _build_debug/libgsb.so). GSB_DOK(cond, status) is cond,
// and when cond is false the kDevBounds bit goes into *status; the caller skips
// the access the check guards, without changing its control flow, so every
// barrier is still reached by every thread. Checks made on kernel parameters
// and the grid alone (the same in every thread) may return at a kernel's
// entry, before its first barrier. Without GSB_DEBUG, GSB_DOK is the constant
// true and compiles away.
#ifdef GSB_DEBUG
__device__ __forceinline__ bool gsb_dok(bool cond, int* status) {
    if (!cond && status) atomicOr(status, (int)kDevBounds);
    return cond;
}
#define GSB_DOK(cond, status) ::gsb::gsb_dok((cond), (status))
#else
#define GSB_DOK(cond, status) true
#endif

// Per-step scalars of Eqs. 3-7 shared by every kernel of a step.
struct StepScalars {
    int m;        // step index; the step produces t_{m+1}
    int M;        // total steps
    float c;      // coupling constant
    float dt;     // time step
    float p_next; // shared p(t_{m+1}) for bSB / dSB (ignored with individual control)
};

}  // namespace gsb

struct gsb_problem {
    int device = 0;
    int N = 0;       // spins, including the auxiliary spin when h was given
    int N_user = 0;  // caller's N
    bool has_h = false;
    bool csr = false;
    int Np = 0;      // N padded to kTile
    bool integer_J = false;
    float max_abs_J = 0.f;
    double max_row_abs = 0.0;  // max_i sum_j |J_ij|
    double W_tot = 0.0;  // sum_{i<j} W_ij with W = -J (Sec. III)
    // dense device copies, Np x Np row-major, zero padded
    float* J32 = nullptr;
    uint8_t* J8 = nullptr;         // e4m3, when integer and |J| <= 16
    __nv_bfloat16* J16 = nullptr;  // bf16, when integer and 128 max row sum |J| < 2^24
    __nv_bfloat16* Jhi = nullptr;  // bf16(J) and bf16(J - Jhi): the split-bf16 path,
    __nv_bfloat16* Jlo = nullptr;  // made on first use
    // CSR device copy (N rows)
    int32_t* rowptr = nullptr;
    int32_t* col = nullptr;
    float* val = nullptr;
    int64_t nnz = 0;
    // App. A setup
    bool have_lambda = false;
    double lambda_max = 0.0, lambda_min = 0.0;
};

struct gsb_run_state {
    gsb_problem* prob = nullptr;
    gsb_params params{};
    int path = 0;
    cudaStream_t stream = nullptr;
    int R = 0, Rp = 0, Np = 0, N = 0;
    int steps_done = 0;
    float c = 0.f, dt = 0.f;
    bool sign_coupling = false;
    bool control = false;
    // state, spin-major [Np][Rp]
    float* x[2] = {nullptr, nullptr};
    int cur = 0;
    float* y = nullptr;
    float* p = nullptr;       // individual parameters (GbSB / GdSB)
    int8_t* s8[2] = {nullptr, nullptr};  // sgn x for the CSR sgn coupling
    int csr_grid = 0;                 // CSR: blocks of the fused multi-step kernel (0: one step per launch)
    bool csr_mlp4 = false;            // CSR per-step kernel: four gathers in flight
    uint32_t* csr_bar = nullptr;      // its grid-barrier counter
    float* csr_psched = nullptr;      // p(t_{m+1}), m = 0..M-1 (shared schedule)
    float* A = nullptr;       // [Rp]
    // twin runs (Sec. IV): pair q runs as replicas q and twin_pairs + q
    int twin_pairs = 0;
    double* twin_part = nullptr;  // partial sums of Eq. 8, [chunks][twin_pairs] + [twin_pairs]
    float* sched = nullptr;   // [M+1] or null
    // tcgen05 operands, replica-major [Rp][Np] (K-major B operand)
    uint8_t* v8[2] = {nullptr, nullptr};     // FP8: sgn x [Rp][Np]; FX16: four digit planes [4][Rp][Np]
    __nv_bfloat16* v16[2] = {nullptr, nullptr};  // FX32: four digit planes [4][Rp][Np] each;
                                                 // split bf16: [planes][Rp][Np], V(t_m) in [m & 1]
    // energy bookkeeping
    double* e_acc = nullptr;    // [Rp] sum_i s_i (J s)_i
    double* e_part = nullptr;   // [Np / 128][Rp] partials of the FP32 energy kernel (dense runs)
    double* best_e = nullptr;   // [Rp]
    int32_t* best_step = nullptr;
    int8_t* best_s = nullptr;   // [Np][Rp]
    int8_t* best_out = nullptr; // [R][N]: best spins in the host layout (gsb_best, lazily)
    int32_t* flag = nullptr;    // [Rp]
    int* status = nullptr;      // device status word
    void* tc = nullptr;         // tcgen05 path state (tensor maps, barriers)
    std::vector<float> sched_host;  // caller schedule p(t_m), m = 0..M (bSB / dSB)
    // GSB_RUN_PROFILE: event pairs around step-kernel launches
    std::vector<cudaEvent_t> prof_events;
    size_t prof_used = 0;
    int64_t prof_steps = 0;  // time steps covered by the recorded launches
};

namespace gsb {

// Kernel attributes (the dynamic shared-memory limit) are set per device: a
// call site keeps one bit per device it has set them on, so a process using
// several GPUs sets them on each. True the first time the current device
// reaches the site.
inline bool first_on_device(std::atomic<uint64_t>& seen) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return true;
    const uint64_t bit = 1ull << dev;
    return !(seen.fetch_or(bit) & bit);
}

// Error reporting (thread-local message, set by the API layer).
gsb_status set_error(gsb_status st, const std::string& msg);
gsb_status cuda_error(cudaError_t err, const char* what);
void count_launch(int n = 1);

#define GSB_CUDA_TRY(call)                                     \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return ::gsb::cuda_error(e_, #call); \
    } while (0)

// Programmatic dependent launch: a step kernel launched with launch_pdl may
// start (its prologue, its loads of data no earlier kernel writes) while the
// kernel before it in the stream finishes. It calls griddep_trigger() once its
// own CTAs are all resident, so the next step may be scheduled, and
// griddep_wait() before its first access to anything the earlier kernel
// writes or reads; the wait returns once that kernel has completed and its
// memory operations are visible.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

// Device memory of problems and runs. Blocks freed by a destroyed problem or
// run (after the GPU is done with them) are kept, up to 1 GiB, for the next
// allocation of the same size on the same device, so creating a problem and a
// run of the same shape again allocates nothing. cache_free returns a block
// that did not come from cache_alloc straight to CUDA.
void* cache_alloc(size_t bytes);
void cache_free(void* p);
gsb_status cache_release();

template <typename T>
gsb_status dev_alloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) return GSB_OK;
    *p = (T*)cache_alloc(sizeof(T) * count);
    if (!*p)
        return set_error(GSB_ENOMEM, "device allocation of " + std::to_string(sizeof(T) * count) +
                                         " bytes failed (device memory, or the library's limit)");
    return GSB_OK;
}
inline void dev_free(void* p) { cache_free(p); }

#define GSB_LAUNCH_CHECK(what)                                 \
    do {                                                       \
        ::gsb::count_launch();                                 \
        cudaError_t e_ = cudaGetLastError();                   \
        if (e_ != cudaSuccess) return ::gsb::cuda_error(e_, what); \
    } while (0)

// ---- kernels' host-side launchers (defined in the .cu files) ----
// init / util
gsb_status launch_init_state(gsb_run_state* run, const float* x0_dev_rm, const float* y0_dev_rm);
gsb_status launch_sign_extract(gsb_run_state* run);
gsb_status launch_rm_to_sm(const float* src_rm, float* dst_sm, int ncols, int N, int R, int Np,
                           int Rp, cudaStream_t s);
gsb_status launch_rm_to_sm_i8(const int8_t* src_rm, int8_t* dst_sm, int ncols, int N, int R,
                              int Np, int Rp, int8_t aux, cudaStream_t s);
gsb_status launch_transpose_to_host_layout(const float* src_sm, float* dst_rm, int Np, int Rp,
                                           int N, int R, cudaStream_t s);
gsb_status launch_transpose_i8_to_host_layout(const int8_t* src_sm, int8_t* dst_rm, int Np,
                                              int Rp, int N, int R, cudaStream_t s);
gsb_status launch_spins_to_state(const int8_t* spins_rm, float* x_sm, int N, int R, int Np,
                                 int Rp, cudaStream_t s);
// dense FP32 path
gsb_status launch_dense_f32_step(gsb_run_state* run, const StepScalars& sc);
// e_acc[r] += sum_i s_i (J s)_i; e_part: scratch of Np / 128 x Rp doubles, for
// per-row-block partials added in a fixed order (the same bits every run)
gsb_status launch_dense_f32_energy(const gsb_problem* prob, const float* x_sm, int Rp,
                                   double* e_acc, double* e_part, cudaStream_t s);
// CSR path
gsb_status launch_csr_step(gsb_run_state* run, const StepScalars& sc);
gsb_status launch_csr_energy(const gsb_problem* prob, const float* x_sm, int Rp, double* e_acc,
                             cudaStream_t s, int* status = nullptr);
gsb_status csr_setup(gsb_run_state* run);
// debug build: planted out-of-range inputs for the CSR and FP8 energy kernels
// (status: a device word the kernels report into)
gsb_status csr_debug_selftest(int* status, cudaStream_t s);
gsb_status tc_debug_selftest(int* status, cudaStream_t s);
gsb_status csr_steps(gsb_run_state* run, int m0, int nsteps);
// best keeping
gsb_status launch_best_keep(gsb_run_state* run, int step);
// Lanczos iteration (App. A)
gsb_status compute_lambda(gsb_problem* prob, cudaStream_t s);
// tcgen05 path
bool tc_available();
gsb_status tc_setup(gsb_run_state* run);
gsb_status tc_prepare(gsb_run_state* run);
gsb_status tc_steps(gsb_run_state* run, int m0, int nsteps);
gsb_status tc_energy(gsb_run_state* run, int step);  // energies of sgn x(t_step)
void tc_free(gsb_run_state* run);
const char* tc_kernel_name(const gsb_run_state* run);
// split-bf16 path (k_bf16.cu)
gsb_status bf16_ensure_planes(gsb_problem* P, cudaStream_t s);
// TMA map of a bf16 [outer][inner] array (inner contiguous): boxes of one
// 128-byte K atom (64 elements) x 128 rows, 128-byte swizzle.
gsb_status bf16_tensor_map(CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer);
// K-split partial products Fp[s] = J[:, K_s] V[K_s, :] on the tensor cores
// (split bf16; V and Fp[s] spin-major [Np][Rp] FP32), for the adjoint.
struct SplitGemm;
gsb_status split_gemm_create(gsb_problem* P, int Rp, SplitGemm** out, cudaStream_t s);
gsb_status split_gemm_partials(SplitGemm* g, const float* V, bool sign, int nslices, float* Fp,
                               cudaStream_t s);
// synchronises s; GSB_ETIMEOUT / GSB_ECUDA when a kernel reported a failed wait or check
gsb_status split_gemm_status(SplitGemm* g, cudaStream_t s);
void split_gemm_destroy(SplitGemm* g);
// gsb_lyapunov's tangent-linear steps with J x and J dx on the tensor cores
// (split bf16): R replicas (A_rep[r] each), log-norm sums into log_sum[R].
gsb_status tangent_bf16x3(gsb_problem* P, bool sign, bool control, int R, const float* A_rep,
                          float c, float dt, int M, int nsteps, int renorm_every, uint64_t seed,
                          float x0_range, bool y0_uniform, double* log_sum, cudaStream_t s);
gsb_status bf16_setup(gsb_run_state* run);
gsb_status bf16_prepare(gsb_run_state* run);
gsb_status bf16_steps(gsb_run_state* run, int m0, int nsteps);
void bf16_free(gsb_run_state* run);
gsb_status bf16_batch(gsb_run_state* const* runs, int n, const int* stop, int per_cta,
                      double max_mb, bool graph, int* windows_out, int* grid_out,
                      int* graphed_out, cudaStream_t s);
// GSB_RUN_PROFILE bracketing of a step-kernel launch
gsb_status prof_begin(gsb_run_state* run);
gsb_status prof_end(gsb_run_state* run, int steps);
// gsb_set_call_profiling: CUDA events around the step-kernel launches of the
// calling thread's next gsb_batch_run / gsb_lyapunov / gsb_relaxed_energy_grad.
// call_prof_reset at the call's start, begin/end around each launch (no-ops
// while profiling is off), call_prof_collect once the stream is synchronised.
void call_prof_reset();
gsb_status call_prof_begin(cudaStream_t s);
gsb_status call_prof_end(cudaStream_t s, int steps);
gsb_status call_prof_collect();
// host loop helpers shared with the tcgen05 path
bool run_is_eval_step(const gsb_run_state* run, int step);
float run_p_shared(const gsb_run_state* run, int step);
gsb_status run_evaluate(gsb_run_state* run, int step);

}  // namespace gsb
