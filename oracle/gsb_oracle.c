/*
 * gsb_oracle.c -- plain FP64 CPU reference for generalized ballistic simulated
 * bifurcation (GbSB) and its relatives bSB and dSB.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the oracle that the CUDA library is
 * checked against. Only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark may load it. It shares no code, header, table or constant with
 * the CUDA library; the two are written independently from the paper
 * (Goto, Hidaka, Tatsumura, "Edge-of-chaos enhanced quantum-inspired algorithm
 * for combinatorial optimization", arXiv:2508.17655).
 *
 * Everything here is deliberately slow and literal: one replica at a time, one
 * spin at a time, in double precision, in the order the paper states the
 * update (Sec. II, Eqs. 3-7; Fig. 2 caption for the FP -> FX/JX -> FY -> wall
 * order). Replicas are independent, so an OpenMP loop over replicas is the only
 * parallelism.
 *
 * Readings of points the paper leaves open:
 *   - Eq. 5 writes t_{k+1}; it is read as t_{m+1}.
 *   - The wall test is strict: |x| > 1. |x| == 1 keeps y.
 *   - sgn(0) = +1, for spins and for the dSB coupling.
 *   - Eq. 7 uses x(t_m) (the old position) and the denominator M - m for the
 *     update that produces p(t_{m+1}); m runs over 0..M-1.
 *   - Eq. 3 uses p(t_{m+1}) (the new bifurcation parameter), x(t_m) and the
 *     coupling of x(t_m); Eq. 4 uses y(t_{m+1}).
 *   - dSB (Sec. VI) replaces J x by J sgn(x) in Eq. 3 only; the p x term keeps x.
 *   - The shared schedule of bSB/dSB is p(t_m) = 1 - m/M (Eq. 6) unless a
 *     schedule array is passed.
 *   - Energy and best-state evaluation: at every step m+1 that is a multiple of
 *     eval_every, and always at m+1 == M; strict improvement, so the earliest
 *     step wins a tie.
 *
 * Parity status per function (what pins each one):
 *   orc_philox4x32_10 .... pinned (published known-answer vectors)
 *   orc_init_uniform ..... pinned (range, symmetry of the integer map)
 *   orc_energy_* / cut ... pinned (cut identity, closed-form graphs, brute force)
 *   orc_bruteforce ....... pinned (closed-form max-cut graphs, exhaustive numpy)
 *   orc_run .............. pinned (Eq. 10 closed form, A=0 -> bSB (Eq. 6),
 *                          Eq. 7 product formula, time reversal, sign and
 *                          gauge symmetry, ground states of small instances;
 *                          the 16-bit JX grid by a hand-computed step on
 *                          grid midpoints and its quantisation bound)
 *   orc_lambda_extremes .. pinned (LAPACK eigvalsh on small matrices)
 *   orc_tangent_run ...... pinned (central finite differences of orc_run, the
 *                          closed-form growth rate about the x = 0 equilibrium)
 *   orc_relaxed_energy_grad pinned (central finite differences of the forward
 *                          energy, the dot-product identity with the tangent)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11. Ten rounds of the 4x32 Philox S-box with the published
 * multipliers and Weyl key increments. */
static void orc_mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
    uint64_t prod = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(prod >> 32);
    *lo = (uint32_t)prod;
}

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    const uint32_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k[2] = {key_in[0], key_in[1]};
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k[0] += weyl0;
            k[1] += weyl1;
        }
        uint32_t hi0, lo0, hi1, lo1;
        orc_mulhilo32(mult0, c[0], &hi0, &lo0);
        orc_mulhilo32(mult1, c[2], &hi1, &lo1);
        uint32_t n0 = hi1 ^ c[1] ^ k[0];
        uint32_t n2 = hi0 ^ c[3] ^ k[1];
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
    out[0] = c[0];
    out[1] = c[1];
    out[2] = c[2];
    out[3] = c[3];
}

/* Uniform draw used for the initial conditions (App. A: x_i(0) uniform in
 * (-0.1, 0.1)). Counter (i, r, stream, 0), key (seed low, seed high); the top
 * 24 bits of the first output word give k in [-2^23, 2^23), and the value is
 * k * (range * 2^-23) rounded once to FP32. The result is returned in double. */
void orc_init_uniform(int32_t R, int32_t N, uint64_t seed, uint32_t stream, float range,
                      double* out /* R*N, replica-major */) {
    const float scale = range * 1.1920928955078125e-07f; /* exact: times 2^-23 */
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int32_t r = 0; r < R; ++r) {
        for (int32_t i = 0; i < N; ++i) {
            uint32_t ctr[4] = {(uint32_t)i, (uint32_t)r, stream, 0u};
            uint32_t w[4];
            orc_philox4x32_10(ctr, key, w);
            int32_t kk = (int32_t)(w[0] >> 8) - 8388608;
            volatile float xf = (float)kk * scale;
            out[(int64_t)r * N + i] = (double)xf;
        }
    }
}

/* ------------------------------------------------------------------------- */
static double orc_sgn(double v) { return v >= 0.0 ? 1.0 : -1.0; }

/* f = J v for a dense row-major N x N matrix (the many-body term of Eq. 3). */
static void orc_coupling_dense(int32_t N, const double* J, const double* v, double* f) {
    for (int32_t i = 0; i < N; ++i) {
        double acc = 0.0;
        const double* row = J + (int64_t)i * N;
        for (int32_t j = 0; j < N; ++j) acc += row[j] * v[j];
        f[i] = acc;
    }
}

/* f = J v for J stored as CSR (row pointers, column indices, values). */
static void orc_coupling_csr(int32_t N, const int32_t* rowptr, const int32_t* col,
                             const double* val, const double* v, double* f) {
    for (int32_t i = 0; i < N; ++i) {
        double acc = 0.0;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) acc += val[k] * v[col[k]];
        f[i] = acc;
    }
}

static void orc_coupling(int32_t N, const double* J, const int32_t* rowptr, const int32_t* col,
                         const double* val, const double* v, double* f) {
    if (J)
        orc_coupling_dense(N, J, v, f);
    else
        orc_coupling_csr(N, rowptr, col, val, v, f);
}

/* Ising energy, Eq. 1: E = -1/2 sum_i sum_j J_ij s_i s_j. */
double orc_energy(int32_t N, const double* J, const int32_t* rowptr, const int32_t* col,
                  const double* val, const int8_t* s) {
    double* v = (double*)calloc((size_t)(N > 0 ? N : 1), sizeof(double));
    double* f = (double*)calloc((size_t)(N > 0 ? N : 1), sizeof(double));
    for (int32_t i = 0; i < N; ++i) v[i] = (double)s[i];
    orc_coupling(N, J, rowptr, col, val, v, f);
    double e = 0.0;
    for (int32_t i = 0; i < N; ++i) e += v[i] * f[i];
    free(v);
    free(f);
    return -0.5 * e;
}

/* Energies of R spin vectors (R x N, replica-major). */
void orc_energy_batch(int32_t N, const double* J, const int32_t* rowptr, const int32_t* col,
                      const double* val, int32_t R, const int8_t* s, double* e_out) {
#pragma omp parallel for schedule(dynamic)
    for (int32_t r = 0; r < R; ++r)
        e_out[r] = orc_energy(N, J, rowptr, col, val, s + (int64_t)r * N);
}

/* Cut value by its definition: with edge weights W = -J (Sec. III), the cut is
 * the total weight of the edges {i, j}, i < j, whose endpoints have different
 * spins. Dense J only. */
double orc_cut_dense(int32_t N, const double* J, const int8_t* s) {
    double cut = 0.0;
    for (int32_t i = 0; i < N; ++i)
        for (int32_t j = i + 1; j < N; ++j)
            if (s[i] != s[j]) cut += -J[(int64_t)i * N + j];
    return cut;
}

/* Exhaustive minimum of Eq. 1 over all 2^N spin vectors (N <= 30), visiting
 * them in Gray-code order with s_0 fixed to +1 (E is invariant under s -> -s).
 * Returns the minimum energy; writes one minimiser to s_best. */
double orc_bruteforce(int32_t N, const double* J, int8_t* s_best) {
    if (N <= 0) return 0.0;
    int8_t* s = (int8_t*)malloc((size_t)N);
    double* h = (double*)malloc(sizeof(double) * (size_t)N);
    for (int32_t i = 0; i < N; ++i) s[i] = 1;
    for (int32_t i = 0; i < N; ++i) {
        double acc = 0.0;
        for (int32_t j = 0; j < N; ++j) acc += J[(int64_t)i * N + j];
        h[i] = acc; /* local field sum_j J_ij s_j */
    }
    double e = 0.0;
    for (int32_t i = 0; i < N; ++i) e += h[i];
    e *= -0.5;
    double best = e;
    memcpy(s_best, s, (size_t)N);
    uint64_t count = (N > 1) ? (1ull << (N - 1)) : 1ull;
    for (uint64_t g = 1; g < count; ++g) {
        /* spin to flip: lowest set bit of g, offset by one (spin 0 is fixed) */
        int32_t k = 1 + __builtin_ctzll(g);
        /* flipping s_k changes E by 2 s_k h_k */
        e += 2.0 * (double)s[k] * h[k];
        double two_sk = 2.0 * (double)s[k];
        s[k] = (int8_t)(-s[k]);
        for (int32_t j = 0; j < N; ++j) h[j] -= two_sk * J[(int64_t)j * N + k];
        if (e < best) {
            best = e;
            memcpy(s_best, s, (size_t)N);
        }
    }
    free(s);
    free(h);
    return best;
}

/* ------------------------------------------------------------------------- */
/* The GbSB iteration for R independent replicas, steps m = m0 .. m0+nsteps-1
 * of a run with M steps in total (Sec. II).
 *
 *   coupling: 0 -> J x   (bSB, GbSB; Eq. 3)
 *             1 -> J sgn(x)   (dSB; Sec. VI)
 *             2 -> J x with x taken on the 16-bit fixed-point grid of the
 *                  paper's JX module (Sec. VI, Fig. 2 caption: the many-body
 *                  term is computed in 16-bit fixed point, the rest in FP32):
 *                  x -> rint(x 2^15) 2^-15, rounding half to even; |x| <= 1
 *                  after the wall, so 16 bits with the sign
 *   control:  0 -> one shared bifurcation parameter: sched[m+1] if sched is
 *                  given, else 1 - (m+1)/M (Eq. 6)
 *             1 -> individual parameters p_i controlled by Eq. 7 with the
 *                  replica's control strength A[r]
 *
 * x, y, p are R x N (replica-major) and updated in place. For control 0 the p
 * array receives the shared value. Each evaluation step writes sgn(x) energy
 * (Eq. 1) and keeps the strictly best one per replica in best_E, best_s,
 * best_step (best_E must be initialised by the caller, e.g. to +inf).
 * margin (nullable, length R) receives, per replica, the smallest distance of
 * any floating-point decision from its threshold over this segment: | |x| - 1 |
 * before the wall test of Eq. 5, |x| where sgn x enters the coupling, and the
 * distance of x from a rounding midpoint of the fixed-point grid (coupling 2).
 * It only observes the iteration; a decision closer than rounding error to its
 * threshold may go either way in another precision. wall_margin (nullable,
 * length R) receives the wall tests' part of it alone.
 * Returns 0, or -1 on bad arguments. */
int orc_run(int32_t N, const double* J, const int32_t* rowptr, const int32_t* col,
            const double* val, int32_t coupling, int32_t control, const double* A,
            const double* sched, double c, double dt, int32_t M, int32_t m0, int32_t nsteps,
            int32_t R, double* x, double* y, double* p, int32_t eval_every, double* best_E,
            int8_t* best_s, int32_t* best_step, int32_t nthreads, double* margin,
            double* wall_margin) {
    if (N <= 0 || R <= 0 || M <= 0 || m0 < 0 || nsteps < 0 || m0 + nsteps > M) return -1;
    if (!J && !(rowptr && col && val)) return -1;
    if (control == 1 && !A) return -1;
    if (coupling < 0 || coupling > 2) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic)
    for (int32_t r = 0; r < R; ++r) {
        double* xr = x + (int64_t)r * N;
        double* yr = y + (int64_t)r * N;
        double* pr = p + (int64_t)r * N;
        double* v = (double*)malloc(sizeof(double) * (size_t)N);
        double* f = (double*)malloc(sizeof(double) * (size_t)N);
        int8_t* s = (int8_t*)malloc((size_t)N);
        double mrg = INFINITY, wmrg = INFINITY;
        for (int32_t m = m0; m < m0 + nsteps; ++m) {
            /* FP: bifurcation parameter(s) at t_{m+1}, from x(t_m) */
            if (control == 1) {
                const double a = A[r];
                for (int32_t i = 0; i < N; ++i)
                    pr[i] = pr[i] - (1.0 - a * xr[i] * xr[i]) * pr[i] / (double)(M - m);
            } else {
                double pnext = sched ? sched[m + 1] : 1.0 - (double)(m + 1) / (double)M;
                for (int32_t i = 0; i < N; ++i) pr[i] = pnext;
            }
            /* JX: many-body term of x(t_m) or of its signs */
            for (int32_t j = 0; j < N; ++j) {
                if (coupling == 1) {
                    v[j] = orc_sgn(xr[j]);
                    if (fabs(xr[j]) < mrg) mrg = fabs(xr[j]);
                } else if (coupling == 2) {
                    const double u = xr[j] * 32768.0; /* exact: a power of two */
                    v[j] = rint(u) / 32768.0;
                    /* distance from the nearest midpoint k + 1/2, in units of x */
                    const double d = fabs(fabs(u - floor(u)) - 0.5) / 32768.0;
                    if (d < mrg) mrg = d;
                } else {
                    v[j] = xr[j];
                }
            }
            orc_coupling(N, J, rowptr, col, val, v, f);
            /* Eq. 3: momentum, with p(t_{m+1}) and x(t_m) */
            for (int32_t i = 0; i < N; ++i) yr[i] = yr[i] - (pr[i] * xr[i] - c * f[i]) * dt;
            /* Eq. 4: position, with y(t_{m+1}) */
            for (int32_t i = 0; i < N; ++i) xr[i] = xr[i] + yr[i] * dt;
            /* Eq. 5: perfectly inelastic walls at |x| = 1 */
            for (int32_t i = 0; i < N; ++i) {
                /* a wall test is a near-tie unless x was not moved (y == 0) */
                if (yr[i] != 0.0 && fabs(fabs(xr[i]) - 1.0) < wmrg) wmrg = fabs(fabs(xr[i]) - 1.0);
                if (wmrg < mrg) mrg = wmrg;
                if (fabs(xr[i]) > 1.0) {
                    xr[i] = orc_sgn(xr[i]);
                    yr[i] = 0.0;
                }
            }
            /* Ising energy of sgn x(t_{m+1}) and best-state keeping */
            int32_t step = m + 1;
            int is_eval = (step == M) || (eval_every > 0 && step % eval_every == 0);
            if (is_eval && best_E) {
                for (int32_t i = 0; i < N; ++i) s[i] = (int8_t)(xr[i] >= 0.0 ? 1 : -1);
                double e = orc_energy(N, J, rowptr, col, val, s);
                if (e < best_E[r]) {
                    best_E[r] = e;
                    if (best_s) memcpy(best_s + (int64_t)r * N, s, (size_t)N);
                    if (best_step) best_step[r] = step;
                }
            }
        }
        if (margin) margin[r] = mrg;
        if (wall_margin) wall_margin[r] = wmrg;
        free(v);
        free(f);
        free(s);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Extreme eigenvalues of a symmetric matrix by shifted power iteration (used
 * for c = 1/lambda_max and Eq. 13, App. A). With sigma = 1.01 rho(J) (a
 * bound just above the spectral radius), J + sigma I and sigma I - J are
 * positive semidefinite and their dominant eigenvalues are lambda_max + sigma
 * and sigma - lambda_min.
 * Iterates until the Rayleigh quotient changes by less than tol (relative) or
 * iters is reached. Dense or CSR. */
static double orc_power_dominant(int32_t N, const double* J, const int32_t* rowptr,
                                 const int32_t* col, const double* val, double sigma, double sign,
                                 int32_t iters, double tol) {
    double* v = (double*)malloc(sizeof(double) * (size_t)N);
    double* f = (double*)malloc(sizeof(double) * (size_t)N);
    double* tmp = (double*)malloc(sizeof(double) * (size_t)N);
    uint32_t key[2] = {12345u, 0u};
    for (int32_t i = 0; i < N; ++i) {
        uint32_t ctr[4] = {(uint32_t)i, 0u, 7u, 0u}, w[4];
        orc_philox4x32_10(ctr, key, w);
        v[i] = ((double)(w[0] >> 8) + 0.5) / 16777216.0 - 0.5;
    }
    double rq = 0.0;
    for (int32_t it = 0; it < iters; ++it) {
        double nrm = 0.0;
        for (int32_t i = 0; i < N; ++i) nrm += v[i] * v[i];
        nrm = sqrt(nrm);
        for (int32_t i = 0; i < N; ++i) v[i] /= nrm;
        orc_coupling(N, J, rowptr, col, val, v, f);
        if (sign == 0.0) {
            /* J^2 v: apply the coupling a second time */
            memcpy(tmp, f, sizeof(double) * (size_t)N);
            orc_coupling(N, J, rowptr, col, val, tmp, f);
        }
        double num = 0.0;
        for (int32_t i = 0; i < N; ++i) {
            f[i] = sigma * v[i] + (sign == 0.0 ? 1.0 : sign) * f[i];
            num += v[i] * f[i];
        }
        double prev = rq;
        rq = num;
        memcpy(v, f, sizeof(double) * (size_t)N);
        if (it > 10 && fabs(rq - prev) <= tol * fabs(rq)) break;
    }
    free(v);
    free(f);
    free(tmp);
    return rq;
}

void orc_lambda_extremes(int32_t N, const double* J, const int32_t* rowptr, const int32_t* col,
                         const double* val, int32_t iters, double tol, double* lmax,
                         double* lmin) {
    /* spectral radius rho(J) from ||J^k v|| growth (power iteration with no
     * shift, Rayleigh quotient of J^2), then shifts by 1.01 rho so that both
     * shifted matrices are positive semidefinite */
    double rho2 = orc_power_dominant(N, J, rowptr, col, val, 0.0, 0.0, iters, tol);
    double sigma = 1.01 * sqrt(rho2 > 0.0 ? rho2 : 0.0) + 1e-300;
    double top = orc_power_dominant(N, J, rowptr, col, val, sigma, 1.0, iters, tol);
    double bot = orc_power_dominant(N, J, rowptr, col, val, sigma, -1.0, iters, tol);
    *lmax = top - sigma;
    *lmin = sigma - bot;
}

/* ------------------------------------------------------------------------- */
/* Tangent-linear propagation of the iteration (not in the paper; the paper
 * measures chaos with the two-trajectory distance of Eq. 8). Differentiating
 * one step of Sec. II with respect to the state (x, y, p):
 *   FP:   dp' = dp - [(1 - A x^2) dp - 2 A x dx p] / (M - m)   (individual control;
 *         dp' = 0 with a shared schedule)
 *   FX:   dy' = dy - [dp' x + p' dx - c J dx] dt               (the sgn x coupling of
 *         dSB is piecewise constant: its derivative is 0)
 *   FY:   dx' = dx + dy' dt
 *   wall: where Eq. 5 clamps, x' and y' are constants: dx' = dy' = 0.
 * The tangent (dx, dy, dp) of every replica is renormalised to unit Euclidean
 * norm every renorm_every steps and at the end; log_sum[r] accumulates the log
 * of the norms in double, so log_sum / (nsteps dt) estimates the largest
 * Lyapunov exponent. The inelastic walls zero the tangent of clamped
 * oscillators; when all of them are clamped the norm is 0 and log_sum is -inf.
 * dx, dy, dp are R x N, in/out (start vectors on input). */
int orc_tangent_run(int32_t N, const double* J, const int32_t* rowptr, const int32_t* col,
                    const double* val, int32_t coupling, int32_t control, const double* A,
                    const double* sched, double c, double dt, int32_t M, int32_t m0,
                    int32_t nsteps, int32_t R, double* x, double* y, double* p, double* dx,
                    double* dy, double* dp, int32_t renorm_every, double* log_sum,
                    int32_t nthreads) {
    if (N <= 0 || R <= 0 || M <= 0 || m0 < 0 || nsteps < 0 || m0 + nsteps > M) return -1;
    if (!J && !(rowptr && col && val)) return -1;
    if (control == 1 && !A) return -1;
    if (renorm_every <= 0) return -1;
    if (coupling != 0 && coupling != 1) return -1;  /* no tangent through the grid rounding */
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic)
    for (int32_t r = 0; r < R; ++r) {
        double* xr = x + (int64_t)r * N;
        double* yr = y + (int64_t)r * N;
        double* pr = p + (int64_t)r * N;
        double* dxr = dx + (int64_t)r * N;
        double* dyr = dy + (int64_t)r * N;
        double* dpr = dp + (int64_t)r * N;
        double* v = (double*)malloc(sizeof(double) * (size_t)N);
        double* f = (double*)malloc(sizeof(double) * (size_t)N);
        double* df = (double*)malloc(sizeof(double) * (size_t)N);
        double acc = 0.0;
        for (int32_t m = m0; m < m0 + nsteps; ++m) {
            const double rem = (double)(M - m);
            /* FP and its tangent, both from x(t_m), p(t_m) */
            for (int32_t i = 0; i < N; ++i) {
                if (control == 1) {
                    const double a = A[r];
                    const double g = 1.0 - a * xr[i] * xr[i];
                    const double dpn = dpr[i] - (g * dpr[i] - 2.0 * a * xr[i] * dxr[i] * pr[i]) / rem;
                    pr[i] = pr[i] - g * pr[i] / rem;
                    dpr[i] = dpn;
                } else {
                    pr[i] = sched ? sched[m + 1] : 1.0 - (double)(m + 1) / (double)M;
                    dpr[i] = 0.0;
                }
            }
            for (int32_t j = 0; j < N; ++j) v[j] = coupling ? orc_sgn(xr[j]) : xr[j];
            orc_coupling(N, J, rowptr, col, val, v, f);
            if (!coupling) orc_coupling(N, J, rowptr, col, val, dxr, df);
            for (int32_t i = 0; i < N; ++i) {
                const double dfi = coupling ? 0.0 : df[i];
                const double dyn = dyr[i] - (dpr[i] * xr[i] + pr[i] * dxr[i] - c * dfi) * dt;
                const double yn = yr[i] - (pr[i] * xr[i] - c * f[i]) * dt;
                const double xn = xr[i] + yn * dt;
                const double dxn = dxr[i] + dyn * dt;
                if (fabs(xn) > 1.0) {
                    xr[i] = orc_sgn(xn);
                    yr[i] = 0.0;
                    dxr[i] = 0.0;
                    dyr[i] = 0.0;
                } else {
                    xr[i] = xn;
                    yr[i] = yn;
                    dxr[i] = dxn;
                    dyr[i] = dyn;
                }
            }
            const int32_t done = m - m0 + 1;
            if (done % renorm_every == 0 || done == nsteps) {
                double s2 = 0.0;
                for (int32_t i = 0; i < N; ++i)
                    s2 += dxr[i] * dxr[i] + dyr[i] * dyr[i] + dpr[i] * dpr[i];
                const double nrm = sqrt(s2);
                acc += log(nrm); /* -inf once every oscillator has been clamped (Eq. 5) */
                if (nrm > 0.0) {
                    for (int32_t i = 0; i < N; ++i) {
                        dxr[i] /= nrm;
                        dyr[i] /= nrm;
                        dpr[i] /= nrm;
                    }
                }
            }
        }
        log_sum[r] = acc;
        free(v);
        free(f);
        free(df);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Relaxed energy and its gradient by reverse-mode differentiation (not in the
 * paper). Starting from x(0) = x0, y(0) = 0, p(0) = 1, the first W steps of an
 * M-step run are taken (Sec. II) and E = -1/2 x(t_W)^T J x(t_W) (Eq. 1 with the
 * continuous x in place of s). Each step is differentiated backwards in the
 * reverse of its forward order (wall, FY, FX, JX, FP):
 *   wall:  where clamped, x' and y' are constants: lx~ = ly~ = 0
 *   FY:    x~ = x + y~ dt          -> lx += lx~, ly~ += lx~ dt, gdt += lx~ y~
 *   FX:    y~ = y - (p' x - c f) dt -> ly = ly~, lp' += -ly~ x dt,
 *                                      lx += -ly~ p' dt, lf = ly~ c dt,
 *                                      gdt += -ly~ (p' x - c f)
 *   JX:    f = J x (J symmetric)   -> lx += J lf   (0 for the sgn coupling)
 *   FP:    p' = p - g p / (M - m), g = 1 - A x^2
 *                                  -> lp = lp' (1 - g / (M - m)),
 *                                     lg = -lp' p / (M - m), gA += -lg x^2,
 *                                     lx += -2 A x lg
 * with lx(t_W) = -J x(t_W). Outputs per replica: E, dE/dx0 (R x N), dE/dA,
 * dE/ddt. All states of the window are stored (plain, memory O(W N)).
 * f32_state != 0 rounds x, y, p to FP32 after every forward step (the paper's
 * machine keeps them in 32-bit floating point, Fig. 2 caption); arithmetic
 * stays FP64. Tests use it to measure how much FP32 state storage alone moves
 * E and its gradient. */
int orc_relaxed_energy_grad(int32_t N, const double* J, int32_t coupling, int32_t control,
                            const double* A, double c, double dt, int32_t M, int32_t W,
                            int32_t R, const double* x0, double* E, double* gx0, double* gA,
                            double* gdt, int32_t nthreads, int32_t f32_state) {
    if (N <= 0 || R <= 0 || M <= 0 || W < 0 || W > M || !J) return -1;
    if (coupling != 0 && coupling != 1) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic)
    for (int32_t r = 0; r < R; ++r) {
        const size_t sz = (size_t)N;
        double* xs = (double*)malloc(sizeof(double) * sz * (size_t)(W + 1));
        double* ys = (double*)malloc(sizeof(double) * sz * (size_t)(W + 1));
        double* ps = (double*)malloc(sizeof(double) * sz * (size_t)(W + 1));
        double* v = (double*)malloc(sizeof(double) * sz);
        double* f = (double*)malloc(sizeof(double) * sz);
        double* lx = (double*)malloc(sizeof(double) * sz);
        double* ly = (double*)malloc(sizeof(double) * sz);
        double* lp = (double*)malloc(sizeof(double) * sz);
        double* lf = (double*)malloc(sizeof(double) * sz);
        double* Jlf = (double*)malloc(sizeof(double) * sz);
        const double a = control == 1 ? A[r] : 0.0;
        for (int32_t i = 0; i < N; ++i) {
            xs[i] = x0[(int64_t)r * N + i];
            ys[i] = 0.0;
            ps[i] = 1.0;
        }
        /* forward, storing every state */
        for (int32_t m = 0; m < W; ++m) {
            const double* x = xs + sz * m;
            const double* y = ys + sz * m;
            const double* p = ps + sz * m;
            double* xn = xs + sz * (m + 1);
            double* yn = ys + sz * (m + 1);
            double* pn = ps + sz * (m + 1);
            for (int32_t i = 0; i < N; ++i)
                pn[i] = control == 1 ? p[i] - (1.0 - a * x[i] * x[i]) * p[i] / (double)(M - m)
                                     : 1.0 - (double)(m + 1) / (double)M;
            for (int32_t j = 0; j < N; ++j) v[j] = coupling ? orc_sgn(x[j]) : x[j];
            orc_coupling_dense(N, J, v, f);
            for (int32_t i = 0; i < N; ++i) {
                const double yt = y[i] - (pn[i] * x[i] - c * f[i]) * dt;
                const double xt = x[i] + yt * dt;
                if (fabs(xt) > 1.0) {
                    xn[i] = orc_sgn(xt);
                    yn[i] = 0.0;
                } else {
                    xn[i] = xt;
                    yn[i] = yt;
                }
                if (f32_state) { /* the state kept in FP32 between steps */
                    xn[i] = (double)(float)xn[i];
                    yn[i] = (double)(float)yn[i];
                    pn[i] = (double)(float)pn[i];
                }
            }
        }
        /* E and its adjoint seed */
        const double* xW = xs + sz * W;
        orc_coupling_dense(N, J, xW, f);
        double e = 0.0;
        for (int32_t i = 0; i < N; ++i) {
            e += xW[i] * f[i];
            lx[i] = -f[i];
            ly[i] = 0.0;
            lp[i] = 0.0;
        }
        E[r] = -0.5 * e;
        double sA = 0.0, sdt = 0.0;
        /* backward */
        for (int32_t m = W - 1; m >= 0; --m) {
            const double* x = xs + sz * m;
            const double* y = ys + sz * m;
            const double* p = ps + sz * m;
            const double* pn = ps + sz * (m + 1);
            const double rem = (double)(M - m);
            for (int32_t j = 0; j < N; ++j) v[j] = coupling ? orc_sgn(x[j]) : x[j];
            orc_coupling_dense(N, J, v, f);
            for (int32_t i = 0; i < N; ++i) {
                const double yt = y[i] - (pn[i] * x[i] - c * f[i]) * dt;
                const double xt = x[i] + yt * dt;
                const int clamped = fabs(xt) > 1.0;
                const double lxt = clamped ? 0.0 : lx[i];
                double lyt = clamped ? 0.0 : ly[i];
                /* FY */
                double lxi = lxt;
                lyt += lxt * dt;
                sdt += lxt * yt;
                /* FX */
                const double lyi = lyt;
                double lpn = lp[i] - lyt * x[i] * dt;
                lxi += -lyt * pn[i] * dt;
                lf[i] = coupling ? 0.0 : lyt * c * dt;
                sdt += -lyt * (pn[i] * x[i] - c * f[i]);
                /* FP */
                double lpi = lpn;
                if (control == 1) {
                    const double g = 1.0 - a * x[i] * x[i];
                    lpi = lpn * (1.0 - g / rem);
                    const double lg = -lpn * p[i] / rem;
                    sA += -lg * x[i] * x[i];
                    lxi += -2.0 * a * x[i] * lg;
                }
                lx[i] = lxi;
                ly[i] = lyi;
                lp[i] = lpi;
            }
            /* JX */
            if (!coupling) {
                orc_coupling_dense(N, J, lf, Jlf);
                for (int32_t i = 0; i < N; ++i) lx[i] += Jlf[i];
            }
        }
        for (int32_t i = 0; i < N; ++i) gx0[(int64_t)r * N + i] = lx[i];
        gA[r] = sA;
        gdt[r] = sdt;
        free(xs); free(ys); free(ps); free(v); free(f);
        free(lx); free(ly); free(lp); free(lf); free(Jlf);
    }
    return 0;
}
