/*
 * gsb.h -- C ABI of libgsb: generalized ballistic simulated bifurcation (GbSB)
 * and its relatives bSB / dSB on one NVIDIA GB300 (sm_103a).
 *
 * Method: Goto, Hidaka, Tatsumura, "Edge-of-chaos enhanced quantum-inspired
 * algorithm for combinatorial optimization", arXiv:2508.17655.
 *   - Problem: the Ising energy E = -1/2 sum_ij J_ij s_i s_j with J symmetric
 *     and J_ii = 0 (Sec. II, Eq. 1); Max-Cut with edge weights W = -J (Sec. III).
 *   - Per time step m = 0..M-1, for every replica and spin i (Sec. II; order of
 *     the Fig. 2 caption):
 *       FP (Eq. 7):  p_i <- p_i - (1 - A x_i^2) p_i / (M - m)        [GbSB]
 *                    p   <- 1 - (m+1)/M, or a caller schedule      [bSB, dSB; Eq. 6]
 *       JX:          f_i = sum_j J_ij v_j,  v = x (bSB/GbSB) or sgn x (dSB, Sec. VI)
 *       FX (Eq. 3):  y_i <- y_i - (p_i x_i - c f_i) dt
 *       FY (Eq. 4):  x_i <- x_i + y_i dt
 *       wall (Eq. 5): if |x_i| > 1 then x_i <- sgn x_i, y_i <- 0
 *   - Initial state (App. A): x_i(0) uniform in [-0.1, 0.1), y_i(0) = 0, p_i(0) = 1.
 *   - c = 1/lambda_max and dt = D_t sqrt(2 / (1 - lambda_min/lambda_max)) with
 *     D_t = 1.25 (App. A, Eq. 13) when the caller passes 0 for them.
 *
 * Conventions for every entry point:
 *   - Return a gsb_status; GSB_OK is 0. No C++ exception crosses the ABI.
 *     gsb_last_error() gives a message for the last failure on this thread.
 *   - Pointers documented as "host" are caller-owned host memory, read or
 *     written before the call returns (gsb_best and gsb_get_state block on the
 *     run's stream first). Pointers documented as "device" are caller-owned
 *     device memory on the current device.
 *   - Handles (gsb_problem, gsb_run_state) are library-owned; they own their device
 *     buffers. A handle must not be used from two threads at once.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream). Work is enqueued asynchronously on it.
 *   - Spins are int8 +-1; sgn(0) = +1. Energies are double; for integer J they
 *     are exact integers.
 *   - Layouts: J dense is row-major N x N. Per-replica arrays of length R;
 *     per-replica vectors (spins, x, y, p) are replica-major R x N.
 */
#ifndef GSB_H
#define GSB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gsb_status {
    GSB_OK = 0,
    GSB_EINVAL = 1,       /* bad argument: size, null pointer, asymmetric J, nonzero diagonal */
    GSB_ENOMEM = 2,       /* device allocation failed */
    GSB_ECUDA = 3,        /* a CUDA runtime or driver call failed */
    GSB_ETIMEOUT = 4,     /* a bounded device-side wait gave up (status word set by a kernel) */
    GSB_EUNSUPPORTED = 5, /* valid request the library cannot serve (e.g. FP8 with non-integer J) */
    GSB_ENUMERIC = 6,     /* a NaN or Inf reached the state */
    GSB_ENODEV = 7        /* no usable sm_103 device */
} gsb_status;

/* Variant = (coupling, control). bSB and GbSB couple through x, dSB and GdSB
 * through sgn x (Sec. VI). bSB and dSB share one parameter p (Eq. 6); GbSB and
 * GdSB control individual parameters by Eq. 7. GdSB (Eq. 7 with sgn x
 * coupling) is not in the paper; it is named there as a direction only. */
typedef enum gsb_variant { GSB_BSB = 0, GSB_GBSB = 1, GSB_DSB = 2, GSB_GDSB = 3 } gsb_variant;

/* Coupling arithmetic. */
typedef enum gsb_precision {
    GSB_PREC_AUTO = 0,   /* FP8 for sgn-x coupling with integer |J| <= 16, FX32 for x coupling
                            with integer J (128 max_i sum_j |J_ij| < 2^24), BF16X3 for
                            real-valued J, FP32 otherwise; CSR problems always use CSR,
                            with the exact fixed-point x coupling (int64 sums of
                            J_ij rint(2^30 x_j)) for integer J */
    GSB_PREC_FP32 = 1,   /* FP32 on CUDA cores (the plain form); for CSR problems, FP32 sums
                            in the nonzeros' order for any J (no fixed-point form) */
    GSB_PREC_FP8 = 2,    /* tcgen05 kind::f8f6f4, e4m3 J and sgn x, FP32 accumulate: exact for
                            integer |J| <= 16; sgn-x coupling (dSB, GdSB) only */
    GSB_PREC_FX32 = 3,   /* tcgen05 kind::f16 with integer J in bf16 and x as 32-bit fixed point
                            rint(x 2^30) in four signed base-256 bf16 digits; each digit plane
                            accumulates exactly, the planes are combined in int64 and rounded
                            once: the coupling is the correctly rounded J x (x exact for
                            |x| >= 2^-7, else rounded at 2^-31). Needs integer J with
                            128 max_i sum_j |J_ij| < 2^24 */
    GSB_PREC_BF16X3 = 4, /* tcgen05 kind::f16 with split bf16 operands for any dense J:
                            J = J_hi + J_lo and x = x_hi + x_lo (each term the bf16
                            rounding of the remainder, 16 significant bits a pair), the
                            coupling accumulated in FP32 as J_hi x_hi + J_hi x_lo +
                            J_lo x_hi (J_hi s + J_lo s for sgn x, which is exact in
                            bf16). Each product is exact; the error against FP64 is
                            at most about 3 2^-16 of sum_j |J_ij v_j| (the two
                            splits' residues, 2^-17 each, and the J_lo x_lo term
                            left out, up to 2^-16) plus FP32 accumulation. One
                            persistent launch runs the steps between energy
                            evaluations. Not in the paper, whose machine computes J x
                            in 16-bit fixed point (Sec. VI) */
    GSB_PREC_FX16 = 5    /* the paper's 16-bit fixed-point JX (Sec. VI, Fig. 2 caption):
                            x enters the coupling as q = rint(x 2^15) (half to even),
                            four signed base-16 digits in e4m3 planes on tcgen05
                            kind::f8f6f4, the planes paired into two exact FP32
                            accumulators; f is the correctly rounded J q 2^-15. The
                            state stays FP32. x coupling (bSB, GbSB) with integer
                            |J| <= 16 and 136 max_i sum_j |J_ij| < 2^24; one persistent
                            cooperative launch of (N/128) x (R/128) CTAs, which must
                            fit on the GPU at once (else GSB_EUNSUPPORTED) */
} gsb_precision;

/* J storage passed to gsb_create. */
typedef enum gsb_jformat {
    GSB_J_DENSE_I8 = 0,  /* int8, N x N row-major */
    GSB_J_DENSE_F32 = 1, /* float, N x N row-major */
    GSB_J_CSR_F32 = 2    /* CSR: int32 rowptr[N+1], int32 col[nnz], float val[nnz]; every row's
                            column indices strictly increasing */
} gsb_jformat;

/* gsb_create flags */
#define GSB_CREATE_DEVICE_INPUT 0x1u /* J / rowptr / col / val / h are device pointers */
#define GSB_CREATE_NO_VALIDATE 0x2u  /* skip the symmetry and zero-diagonal check */

typedef struct gsb_problem gsb_problem;
typedef struct gsb_run_state gsb_run_state;

/* Run parameters. Zero-initialise, then set what you need; zero means the
 * documented default. */
typedef struct gsb_params {
    int32_t variant;          /* gsb_variant */
    int32_t M;                /* total steps of the run (t_M = M dt), >= 1 */
    int32_t R;                /* replicas, >= 1 */
    int32_t precision;        /* gsb_precision */
    double c;                 /* > 0, or 0: 1/lambda_max (App. A) */
    double dt;                /* > 0, or 0: Eq. 13 with D_t = 1.25 */
    float A;                  /* control strength of Eq. 7 for every replica (GbSB, GdSB) */
    const float* A_per_replica; /* host, length R, or NULL: per-replica control strengths */
    const float* schedule;    /* host, length M+1, or NULL: p(t_m) for bSB / dSB (default Eq. 6) */
    uint64_t seed;            /* Philox4x32-10 key for the initial conditions */
    float x0_range;           /* 0: 0.1 (App. A) */
    int32_t y0_uniform;       /* 0: y(0) = 0 (App. A); 1: y(0) uniform in [-x0_range, x0_range) */
    int32_t eval_every;       /* 0: evaluate the energy at t_M only (Sec. III); k > 0: also
                                 at every step that is a multiple of k */
    int32_t steps_per_launch; /* 0: as many as possible (up to the next energy evaluation);
                                 1: one step per launch; k: at most k steps per launch, on
                                 the paths that fuse steps (the persistent FP8 kernel) */
    const float* x0;          /* host, R x N, or NULL: explicit x(0) instead of the Philox draw */
    const float* y0;          /* host, R x N, or NULL: explicit y(0) */
    uint32_t flags;           /* GSB_RUN_* */
} gsb_params;

#define GSB_RUN_DEFER 0x1u   /* gsb_run sets up the state but advances no step */
#define GSB_RUN_PROFILE 0x2u /* record CUDA events around every launch of the step kernel */
#define GSB_RUN_FUSED_CSR 0x8u /* CSR runs: one cooperative launch per stretch of steps (a grid
                                  barrier between steps) instead of one launch per step; the
                                  same bits, measured slower on the ER workloads */
#define GSB_RUN_SM_PAIRS 0x4u /* the persistent FP8 kernel's grid form runs on SM pairs (two
                                 CTAs per MMA, cta_group::2) where it fits; the same bits,
                                 measured slower on the N = 2000, R = 1024 workload */

/* Create a problem from a coupling matrix (Eq. 1). The library copies J into
 * the device formats its kernels need (FP32, e4m3, bf16 and/or CSR), padded
 * to its tile sizes. Validation (unless GSB_CREATE_NO_VALIDATE): square,
 * symmetric, zero diagonal, finite -- else GSB_EINVAL. h (host or device,
 * length N, nullable) adds a local field -h_i s_i to Eq. 1 (not in the paper):
 * it is folded in exactly as an extra spin N coupled by J_{i,N} = h_i, and
 * results are reported with that spin gauge-fixed to +1.
 * Arguments not used by `format` must be NULL / 0. */
gsb_status gsb_create(gsb_problem** out, int32_t N, int32_t format, const void* J,
                      const int32_t* rowptr, const int32_t* col, const float* val, int64_t nnz,
                      const float* h, uint32_t flags, void* stream);
gsb_status gsb_destroy(gsb_problem* problem);

/* QUBO input (not in the paper, which notes only that other problems map to
 * the Ising form of Eq. 1): minimise f(b) = sum_ij Q_ij b_i b_j over
 * b in {0,1}^N, with Q (N x N row-major float, any square matrix: asymmetric
 * entries and the diagonal, which acts as a linear term since b_i^2 = b_i,
 * are allowed). With s = 2b - 1 and Qs = (Q + Q^T)/2 this is the Ising problem
 * J_ij = -(Q_ij + Q_ji) for i != j, J_ii = 0, local field
 * h_i = -sum_j (Q_ij + Q_ji), scaled by 4 so that integer Q keeps integer J
 * and h (and the exact tensor-core paths): f(b) = scale * E(s) + offset with
 * scale = 1/4 and offset = (sum_ij Q_ij + sum_i Q_ii)/4, E as gsb_best
 * reports it. The scale does not change the dynamics when c is left to its
 * default 1/lambda_max (App. A) and dt to Eq. 13.
 *
 * gsb_qubo_to_ising: that map on the host, no GPU needed: Q (host, N x N) ->
 * J (host, N x N, written), h (host, length N, written), scale and offset
 * (host, nullable). GSB_EINVAL for N outside 1..65536, a NULL array or a
 * non-finite entry of Q.
 *
 * gsb_create_qubo: gsb_create of that Ising problem (dense FP32 J with the
 * local field h, so one auxiliary spin is added and gauge-fixed to +1 on
 * output: b_i = (1 + s_i)/2 for the spins gsb_best returns). Q is host memory,
 * or device memory with flags = GSB_CREATE_DEVICE_INPUT (no other flag is
 * accepted). scale and offset as above (nullable). */
gsb_status gsb_qubo_to_ising(int32_t N, const float* Q, float* J, float* h, double* scale,
                             double* offset);
gsb_status gsb_create_qubo(gsb_problem** out, int32_t N, const float* Q, uint32_t flags,
                           double* scale, double* offset, void* stream);

/* Device memory: the blocks of destroyed problems and runs are kept (up to
 * 1 GiB in all) and handed to the next problem or run that needs a block of the
 * same size on the same device, so creating one of the same shape again costs
 * no cudaMalloc / cudaFree. gsb_destroy waits for the device to be idle, and
 * gsb_run_destroy for the run's stream, before their blocks are kept. This call
 * returns every kept block to CUDA (for an application that needs the memory).
 * Host side only; not to be called while another thread creates or destroys
 * handles. */
gsb_status gsb_release_cached_memory(void);

/* Cap on the device memory the library's problems and runs hold at once
 * (bytes; 0 = no cap). An allocation that would pass it fails with GSB_ENOMEM,
 * and the call that needed it leaves nothing allocated. gsb_memory_usage
 * reports the bytes held by live handles and the bytes kept for reuse (each
 * output nullable). Host side only. */
gsb_status gsb_set_memory_limit(int64_t bytes);
gsb_status gsb_memory_usage(int64_t* in_use, int64_t* kept);

/* Number of spins (including the auxiliary one when h was given) and the
 * extreme eigenvalues of J used for c and dt (computed on the GPU on first use
 * by the Lanczos method in FP64, to 1e-14 relative stationarity of the Ritz
 * values; App. A). Blocks on `stream` the first time. */
gsb_status gsb_problem_info(gsb_problem* problem, int32_t* n_spins, double* lambda_max,
                            double* lambda_min, void* stream);

/* Start a run: allocate its device state, draw or upload x(0), y(0), set
 * p(0) = 1, and (unless GSB_RUN_DEFER) enqueue all M steps on `stream`. */
gsb_status gsb_run(gsb_problem* problem, const gsb_params* params, gsb_run_state** out, void* stream);

/* Advance a run by nsteps (<= M - steps already done) on its stream. Runs
 * split into several calls follow the same trajectory as one call. */
gsb_status gsb_run_steps(gsb_run_state* run, int32_t nsteps);

/* Start the same run again from step 0 with another seed, reusing its device
 * buffers: x(0), y(0) drawn as in gsb_run (explicit x0/y0 are not kept),
 * p(0) = 1, best states cleared. flags: GSB_RUN_DEFER as in gsb_params.
 * Enqueued on the run's stream; allocates nothing. */
gsb_status gsb_run_restart(gsb_run_state* run, uint64_t seed, uint32_t flags);

/* With GSB_RUN_PROFILE: total device time (ms, from CUDA events on the run's
 * stream) of the run's step-kernel launches since the last gsb_run /
 * gsb_run_restart, how many launches that was, and how many time steps they
 * covered (a persistent launch covers many). Each output is nullable. Blocks
 * on the run's stream. */
gsb_status gsb_kernel_time(gsb_run_state* run, double* ms, int64_t* launches, int64_t* steps);

/* Name of the step kernel the run selected at gsb_run: "k_tc_persist<cluster>"
 * (FP8, many steps per launch, one thread-block cluster per 128 replicas),
 * "k_tc_persist<grid>" (the same, one cooperative launch), "k_tc_step<e4m3>"
 * (FP8, one step per launch), "k_fx32_step" (FX32 digit planes, one step per
 * launch), "k_fx16_persist" (FX16, many steps per launch), "k_bf16_multi"
 * (split bf16, many steps per launch), "k_dense_f32_step" or "k_csr_step". A static string owned by the
 * library; "" for NULL. No GPU work. */
const char* gsb_run_kernel(const gsb_run_state* run);

/* Best state per replica (host outputs, each nullable): spins R x N int8,
 * energies (Eq. 1), cut values (W_tot - E)/2 with W = -J (Sec. III), and the
 * step m at which it was found. Blocks on the run's stream. Replicas that have
 * not been evaluated yet report energy +inf and step -1. Without h the spins are
 * copied from the device straight into `spins` (page-locked host memory makes
 * that copy fastest). */
gsb_status gsb_best(gsb_run_state* run, int8_t* spins, double* energies, double* cuts,
                    int32_t* step_found);

/* Current state, host outputs R x N each (nullable), and the number of steps
 * done so far. For bSB/dSB, p holds the shared parameter in every entry. */
gsb_status gsb_get_state(gsb_run_state* run, float* x, float* y, float* p, int32_t* steps_done);

/* Checkpoint / resume (not in the paper): put a run at step steps_done
 * (0..M) with the state x, y (and p for GbSB / GdSB; ignored otherwise), host
 * R x n_spins each in the layout gsb_get_state returns, and optionally the best
 * records as gsb_best returns them (spins R x N, energies R, step found R; all
 * three or none: none clears them). gsb_run_steps then continues exactly as the
 * run the state was taken from would have: a run stopped after k steps, saved
 * with gsb_get_state and gsb_best, and restored into a fresh deferred run of the
 * same problem and parameters ends bit-identical to one never interrupted.
 * Blocks on the run's stream. */
gsb_status gsb_run_set_state(gsb_run_state* run, const float* x, const float* y, const float* p,
                             int32_t steps_done, const int8_t* best_spins,
                             const double* best_energies, const int32_t* best_step);

/* Ising energies (Eq. 1) of R caller spin vectors (host, R x N int8 +-1) into
 * energies (host, length R). Evaluated on the GPU. */
gsb_status gsb_energy(gsb_problem* problem, int32_t R, const int8_t* spins, double* energies,
                      void* stream);

gsb_status gsb_run_destroy(gsb_run_state* run);

/* Largest Lyapunov exponent per replica by tangent-linear propagation (not in
 * the paper, whose chaos measure is the two-trajectory distance of Eq. 8).
 * Linearisation of one step of Eqs. 3-7 in (x, y, p): dp' = dp - [(1 - A x^2)
 * dp - 2 A x dx p]/(M - m) (individual control; 0 with a shared schedule),
 * dy' = dy - [dp' x + p' dx - c J dx] dt (no J dx term for sgn-x coupling),
 * dx' = dx + dy' dt, and dx' = dy' = 0 where Eq. 5 clamps. nA control strengths
 * A_values (host) times params->R replicas each run together (replica k R + r
 * uses A_values[k] and draws x(0) as gsb_run would for that index); each
 * tangent starts as dx uniform in [-1, 1) (Philox stream 4), dy = dp = 0, unit
 * norm, and is renormalised every renorm_every steps and after the last of the
 * first nsteps steps (0 = all M) of the Eq. 6 schedule. mle_out (host, nA x R)
 * receives sum(log norms) / (nsteps dt), accumulated in FP64. Dense problems.
 * params->precision: GSB_PREC_AUTO or GSB_PREC_FP32, the FP32 coupling on CUDA
 * cores; GSB_PREC_BF16X3, J x and J dx on the tensor cores in the split-bf16
 * form (error against FP64 up to about 3 2^-16 of the coupling's magnitude);
 * any other: GSB_EUNSUPPORTED. Blocks on `stream`. */
gsb_status gsb_lyapunov(gsb_problem* problem, const gsb_params* params, int32_t nA,
                        const float* A_values, int32_t renorm_every, int32_t nsteps,
                        double* mle_out, void* stream);

/* Twin trajectories, the chaos measure of Sec. IV. Starts a run (as gsb_run)
 * of 2 nA R replicas in nA x R pairs: replica a R + r is trajectory (1) of pair
 * (a, r) and replica nA R + a R + r its trajectory (2); both use the control
 * strength A_values[a] (host, length nA; unused by bSB / dSB). Initial state:
 * x^(1)_i = +-0.1 and x^(2)_i = x^(1)_i +- 2e-6 with independent random signs
 * (Philox4x32-10 keyed by params->seed, counter (i, pair index, 2, 0) for the
 * first sign and (i, pair index, 3, 0) for the second, a draw >= 0 meaning +),
 * the FP64 value rounded once to FP32; y = 0, p = 1. params->R is the number of
 * pairs per control strength; x0, y0 and A_per_replica must be NULL; x0_range
 * and y0_uniform are ignored; everything else as in gsb_run (GSB_RUN_DEFER
 * included). gsb_run_restart on the handle redraws twin initial states. Dense or
 * CSR problems without h (GSB_EUNSUPPORTED otherwise). */
gsb_status gsb_twin_run(gsb_problem* problem, const gsb_params* params, int32_t nA,
                        const float* A_values, gsb_run_state** out, void* stream);

/* Normalised distance of Eq. 8 between the twins of every pair at the run's
 * current step: delta = sqrt(sum_i (x^(1)_i - x^(2)_i)^2 / (4N)), summed in FP64
 * in a fixed order. delta_out: host, nA R doubles in pair order. GSB_EINVAL for
 * a run not made by gsb_twin_run. Blocks on the run's stream. */
gsb_status gsb_twin_delta(gsb_run_state* run, double* delta_out);

/* Gradient of the relaxed energy E = -1/2 x(t_W)^T J x(t_W) (Eq. 1 with the
 * continuous positions; not in the paper) after the first `window` steps of an
 * M-step run started from x(0) = x0, y(0) = 0, p(0) = 1, with respect to x0,
 * the control strength A (Eq. 7) and the time step dt. Hand-written reverse
 * sweep of Eqs. 3-7 (the wall of Eq. 5 passes no gradient through clamped
 * components; the sgn coupling of dSB has none), with the forward states
 * recomputed from checkpoints taken every ckpt_every steps. Uses params->
 * variant, M, R, c (> 0), dt (> 0), A / A_per_replica. Device buffers owned by
 * the caller: x0 (R x N float, replica-major), energy (R doubles, written),
 * grad_x0 (R x N float), grad_A and grad_dt (R doubles each; nullable).
 * Dense problems without h, FP32 arithmetic. params->precision: GSB_PREC_AUTO or
 * GSB_PREC_FP32, the products J v as FP32 SGEMMs on CUDA cores; GSB_PREC_BF16X3,
 * as K-split partial products on the tensor cores in the split-bf16 form (J and
 * v split into bf16 hi + lo terms; error up to about 3 2^-16 of the coupling's
 * magnitude); any other: GSB_EUNSUPPORTED. Blocks on `stream`. */
gsb_status gsb_relaxed_energy_grad(gsb_problem* problem, const gsb_params* params,
                                   int32_t window, int32_t ckpt_every, const float* x0,
                                   double* energy, float* grad_x0, double* grad_A,
                                   double* grad_dt, void* stream);

/* Batched runs: n independent instances (each its own dense problem and
 * parameters; uneven N and R) advanced together (the paper solves several
 * instances at once on one machine, N_batch, Sec. VI). Every instance gets an
 * ordinary run handle in runs_out[k] (query it with gsb_best / gsb_get_state,
 * free it with gsb_run_destroy) and follows exactly the trajectory gsb_run
 * would give it with the same precision. Energies are evaluated at t_M
 * (eval_every must be 0). Two forms, chosen by the instances' precision (all
 * the same): AUTO or BF16X3 -- the split-bf16 tensor-core path: the instances
 * are packed, largest first, into windows of at most tiles_per_cta x (number of
 * SMs) tiles of 128 spins x 128 replicas and a working set (J, state, operands)
 * of 80, 120, 160 or 240 MB for 1, 2, 4 or 8 tiles per CTA (the smallest stays
 * resident in the L2), and each window runs all its steps in one
 * persistent cooperative launch over a device work list of (step, tile) items
 * (per-instance step counters order the items; the launches of all windows
 * are captured as one CUDA graph, see graphed below). An autotuner picks tiles_per_cta (1, 2, 4
 * or 8) by timing a few real steps of the whole batch under each. FP32 -- the CUDA-core path: one
 * launch per time step over a work list of tiles, chunks of steps replayed
 * from CUDA graphs; the autotuner picks the tile (128 or 64 spins x
 * replicas) and the graph chunk length on the first steps. info (nullable)
 * reports the choices; info->force_tile = 128 or 64 skips the FP32 tile probe,
 * info->force_tiles_per_cta = 1, 2, 4 or 8 the bf16 one; info->max_steps > 0 stops
 * every instance after that many steps (continue each with gsb_run_steps).
 * Blocks on `stream` until every instance is done. */
typedef struct gsb_batch_info {
    int32_t force_tile;       /* in: FP32 form: 0 = autotune, 128 or 64 */
    int32_t max_steps;        /* in: 0 = run every instance to its M */
    int32_t tile;             /* out: tile used (spins and replicas per tile) */
    int32_t steps_per_graph;  /* out: FP32 form: steps captured per graph launch; bf16 form:
                                 the most steps one launch covered */
    int32_t tiles;            /* out: tiles per step */
    double ms_step_tile128;   /* out: FP32 probe time per step, tile 128 (-1 if not probed) */
    double ms_step_tile64;    /* out: FP32 probe time per step, tile 64 (-1 if not probed) */
    int32_t force_tiles_per_cta; /* in: bf16 form: 0 = autotune, 1, 2, 4 or 8 */
    int32_t tiles_per_cta;    /* out: bf16 form: window size in tiles per CTA */
    int32_t windows;          /* out: bf16 form: persistent launches (windows) */
    int32_t ctas;             /* out: bf16 form: CTAs per launch */
    double ms_step_probe[4];  /* out: bf16 probe time per step with 1, 2, 4 and 8 tiles per
                                 CTA (-1 if not probed) */
    int32_t graphed;          /* out: bf16 form: 1 if the windows' launches ran as one CUDA
                                 graph, 0 if they were launched one by one */
} gsb_batch_info;

gsb_status gsb_batch_run(int32_t n, gsb_problem* const* problems, const gsb_params* params,
                         gsb_run_state** runs_out, gsb_batch_info* info, void* stream);

/* Allocation-free energies, for callers that cannot call cudaMalloc / cudaFree
 * (a steady-state loop that must not block on them, or an application whose own
 * allocator owns the device memory). The paper has no counterpart: it is an
 * interface variant of gsb_energy. J (device, N x N row-major float), spins
 * (device, R x N int8 +-1) and energies (device, length R, written) belong to
 * the caller; the kernels run on `stream`. The per-replica accumulators are a
 * fixed array inside the library (1 <= R <= 65536 and 1 <= N <= 29,000; other
 * sizes give GSB_EINVAL), one per device, held by every device that loads the
 * library until the process exits, and shared by all calls: each call clears it
 * first, and calls whose work overlaps on the GPU race on it. Each call looks
 * up that array's device address with the caller's device current (a host-side
 * lookup, so it stays right after a device reset); the first call on a device
 * may load the library's module there and should come before any stream
 * capture. */
gsb_status gsb_energy_noalloc(const float* J, int32_t N, const int8_t* spins, int32_t R,
                              double* energies, void* stream);

/* Check of the device-side failure detection (not in the paper). Every wait of
 * the library's kernels (on an mbarrier, a counter another CTA advances, a
 * barrier of a thread-block cluster) gives up after a time limit, sets a
 * status word and lets the kernel return, so a lost arrival ends the call with
 * GSB_ETIMEOUT instead of hanging the GPU (the kernels' limit is 8e9 SM clock
 * cycles, about 4 s). This entry runs one such wait, limited to limit_ns
 * (1 us .. 10 s) worth of cycles at the device's rated SM clock, in a one-warp
 * kernel on `stream`:
 * kind 0 waits on an mbarrier nobody arrives on, kind 1 on a counter in global
 * memory nobody advances -- both return GSB_ETIMEOUT after about limit_ns --
 * and kind 2 on a counter that already holds (GSB_OK at once). The CUDA
 * context stays usable afterwards. Blocks on `stream`. */
gsb_status gsb_wait_check(int32_t kind, int64_t limit_ns, void* stream);

/* Debug build (not in the paper: a stand-in for a memory checker, which this
 * library's test machines do not offer). The same sources built with
 * -DGSB_DEBUG (paper_2508_17655_gb300/_build_debug/libgsb.so; the Python
 * binding loads it when GSB_LIBRARY=debug) check on the device the indices
 * that come from the caller's data -- CSR row ranges and column indices, the
 * tile lists of batched runs -- and the launch geometry of the tensor-core and
 * dense step kernels (grid against the padded shape, steps against M). A
 * failed check skips the access it guards (a column out of range is read as
 * row 0 with weight 0; a kernel with a wrong grid returns before its first
 * barrier) and sets a bit in the run's status word, which gsb_best then
 * reports as GSB_ECUDA ("a kernel detected an out-of-range index"). Nothing
 * traps, so the CUDA context stays usable. In the release build the checks
 * compile away. gsb_debug_build: 1 in the debug build, 0 in the release build
 * (host only). */
int32_t gsb_debug_build(void);
/* Debug build only: runs two kernels on inputs planted to fail their checks --
 * the CSR energy kernel on a 4-row matrix one of whose columns is out of range,
 * and the FP8 energy kernel on a grid one spin block taller than its matrix --
 * and returns GSB_OK when both checks fired (the status bit set, the access not
 * made), GSB_ECUDA otherwise. In the release build GSB_EUNSUPPORTED, with
 * nothing launched. Uses the current device and synchronises it. */
gsb_status gsb_debug_selftest(void);

/* Device-time profile of the library's own multi-launch calls (not in the
 * paper). After gsb_set_call_profiling(1) on a thread, each later
 * gsb_batch_run, gsb_lyapunov and gsb_relaxed_energy_grad on that thread
 * records CUDA events on its stream around every launch of its step kernels
 * (graph launches of captured steps included; the events also keep launches
 * from overlapping), and gsb_last_call_profile then gives the summed device
 * time of those launches in ms, their number, and the time steps they covered
 * (each output nullable). Allocation, set-up and copies are outside the
 * bracketed launches. gsb_set_call_profiling(0) turns it off. Host side; no
 * GPU work of its own. */
gsb_status gsb_set_call_profiling(int32_t on);
gsb_status gsb_last_call_profile(double* kernel_ms, int64_t* launches, int64_t* steps);

/* Message for the last non-OK status returned on the calling thread. */
const char* gsb_last_error(void);

/* Library version, and the number of kernels this library has launched in
 * this process (a counter the host increments at every launch). */
int32_t gsb_version(void);
int64_t gsb_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* GSB_H */
