/*
 * debyefit -- batched multi-Debye fitting of dielectric spectra on GB300 (sm_103a).
 *
 * C ABI of libdebyefit.so. The method is the hybrid linear/non-linear fit of
 * Majchrowska et al., "Modelling Arbitrary Complex Dielectric Properties -- an
 * automated implementation for gprMax" (arXiv:2109.01928):
 *   - a target spectrum eps(w) = eps'(w) - j eps''(w)                      (Eq. 1)
 *     given by a relaxation model (Debye, Havriliak-Negami, Cole-Cole,
 *     Cole-Davidson, Jonscher, CRIM: Eqs. 3-6) or by tabulated values (Sec. III-A);
 *   - is approximated by the multi-pole Debye expansion
 *     eps_inf + sum_n d_eps_n / (1 + j w tau_n)                             (Eq. 7);
 *   - a global optimiser (particle swarm, differential evolution or dual
 *     annealing) searches the relaxation times, and for
 *     each candidate the weights (eps_inf, d_eps_n) come from damped least squares
 *     over the real and imaginary parts, with negative weights sign-flipped as a
 *     penalty (Sec. III-A, III-B);
 *   - the result is eps_inf and (d_eps_n, tau_n), n = 1..N (Listing 2).
 *
 * Conventions for every entry point
 *   - Array arguments are caller-owned DEVICE memory unless the name ends in
 *     _host. The library reads and writes them in stream order on `stream` and
 *     keeps no reference after the call returns.
 *   - Candidates are log10(tau) vectors theta. A population is theta[S][P][n_max]
 *     (float64, row-major); entries n >= N_s of spectrum s are ignored.
 *   - Weights are x = (eps_inf, d_eps_1..d_eps_N) laid out [S][P][n_max+1];
 *     entries beyond N_s+1 are written as 0.
 *   - Every call returns a status: DEBYE_OK (0) or a negative DEBYE_E* code. No
 *     exception or exit crosses the ABI. debye_last_error() describes the last
 *     failure of a handle. Errors detected on the device (non-finite input, a
 *     work-list bound violated) are recorded in a device status word and returned
 *     by the next debye_sync().
 *   - A candidate whose damped normal matrix is not positive definite gets cost
 *     +inf, weights and gradient 0, and counts in the optional per-spectrum
 *     n_failed output; that is a result, not a call error. With lam_search > 0 the
 *     damped matrix G + lam diag(G) is positive definite for every finite theta
 *     (diag(G) > 0 for Debye columns), so in practice a candidate fails only for a
 *     non-finite theta or with lam_search = 0.
 *   - Calls on one handle must not overlap in time (one host thread at a time);
 *     different handles are independent.
 */
#ifndef DEBYEFIT_H
#define DEBYEFIT_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
#define DEBYE_OK          0
#define DEBYE_EINVAL     -1   /* bad argument (null pointer, size, bounds, N) */
#define DEBYE_ECUDA      -2   /* a CUDA runtime call failed */
#define DEBYE_ENOMEM     -3   /* device workspace allocation failed */
#define DEBYE_ETIMEOUT   -4   /* a bounded device-side wait gave up */
#define DEBYE_EINTERNAL  -5   /* inconsistent internal state */
#define DEBYE_ENOTFINITE -6   /* non-finite frequency or target value on the device */
#define DEBYE_EBOUNDS    -7   /* a device-side index check failed */

/* ------------------------------------------------------------------ precision */
#define DEBYE_PREC_FP64  0    /* FP64 basis, Gram, solve and residual */
#define DEBYE_PREC_MIXED 1    /* float-float column sums of the Debye basis, exact Gram identity,
                                 FP32 factor refined in float-float */
#define DEBYE_PREC_FP64_SUMS 2 /* FP64 throughout, the Gram from FP64 column sums by the exact
                                 identity (no O(K N^2) Gram pass), then the FP64 solve and
                                 residual passes of DEBYE_PREC_FP64 */
#define DEBYE_PREC_MIXED_TABLE 3 /* DEBYE_PREC_MIXED with the column sums read from per-spectrum
                                 Chebyshev tables: once per call, every spectrum's column sums
                                 S(theta), a^T b(theta) and their theta derivatives are
                                 evaluated (float-float pass) at Chebyshev nodes on segments of
                                 0.2 decades over its box [lo, hi] and interpolated (12
                                 coefficients per segment, ~1e-14 relative); each candidate's
                                 sums then cost O(1) per pole instead of O(K). A theta outside
                                 the box takes a direct FP64 sweep. Same solve and tolerances
                                 as DEBYE_PREC_MIXED; needs finite bounds with lo < hi <=
                                 lo + 200 (DEBYE_EINVAL otherwise). Each call reads lo and hi
                                 back to the host (one stream synchronisation).
                                 debye_eval_population_noalloc takes the direct sums. */

#define DEBYE_MAX_POLES 20    /* largest N accepted */

/* ------------------------------------------------------------------ models (target synthesis) */
#define DEBYE_MODEL_DEBYE        0  /* Eq. 3 */
#define DEBYE_MODEL_HN           1  /* Eq. 4 */
#define DEBYE_MODEL_CC           2  /* Eq. 4, beta = 1 */
#define DEBYE_MODEL_CD           3  /* Eq. 4, alpha = 1 */
#define DEBYE_MODEL_JONSCHER     4  /* eps_inf + a_p (w/w_p)^(n-1) [1 - j cot(n pi/2)] */
#define DEBYE_MODEL_JONSCHER_EQ5 5  /* Eq. 5 as printed: eps_inf + A_p (-j w/w_p)^n */
#define DEBYE_MODEL_CRIM         6  /* Eq. 6 over up to 3 Debye components */
#define DEBYE_MODEL_DEBYE_SUM    7  /* Eq. 7 source poles + Jonscher tail + noise */
#define DEBYE_N_PARAMS          16  /* float64 parameter record per spectrum */

/* ------------------------------------------------------------------ search methods */
#define DEBYE_SEARCH_PSO 0    /* particle swarm (Sec. III-B; Kennedy and Eberhart) */
#define DEBYE_SEARCH_DE  1    /* differential evolution (Sec. III-B; Storn and Price) */
#define DEBYE_SEARCH_DA  2    /* dual annealing (Sec. III-B; Tsallis and Stariolo), iters <= 1000 */
#define DEBYE_DE_RAND1   0    /* mutant x_r1 + F (x_r2 - x_r3), needs P >= 4 */
#define DEBYE_DE_BEST1   1    /* mutant x_best + F (x_r1 - x_r2), needs P >= 3 */

typedef struct debye_ctx* debye_handle;

/* Solver options. debye_default_options() fills the documented defaults. */
typedef struct {
  int32_t precision;      /* DEBYE_PREC_FP64, DEBYE_PREC_MIXED (default), DEBYE_PREC_FP64_SUMS
                             or DEBYE_PREC_MIXED_TABLE */
  int32_t refine_steps;   /* FP64 precision: residual passes with refinement after the first
                             solve, 1..4 (default 1); the mixed path refines on its small
                             float-float system instead and ignores it */
  double  lam_search;     /* Marquardt damping of search and polish (default 1e-3) */
  double  lam_final;      /* damping of the reported weights (default 1e-3 = lam_search) */
  double  pso_omega;      /* swarm inertia (default 0.5) */
  double  pso_phi_p;      /* cognitive coefficient (default 0.5) */
  double  pso_phi_g;      /* social coefficient (default 0.5) */
  int32_t lbfgs_m;        /* L-BFGS history pairs, 1..8 (default 8) */
  int32_t lbfgs_max_trials; /* backtracking halvings per iteration, 1..40 (default 20) */
  double  lbfgs_c1;       /* Armijo constant (default 1e-4) */
  int32_t cands_per_block;/* candidates per thread block of full populations, 1..128 with
                             cands_per_block x lanes (lanes_per_candidate, 1 if 0) a
                             multiple of 32 and at most 128; 0 = autotune / 64 */
  int32_t use_graphs;     /* capture the generation and polish loops in CUDA graphs (default 1) */
  double  de_f_lo;        /* differential evolution: scale factor F ~ U[de_f_lo, de_f_hi) drawn */
  double  de_f_hi;        /*   once per generation; 0 <= lo <= hi <= 2 (default 0.5, 1.0) */
  double  de_cr;          /* binomial crossover rate, 0..1 (default 0.7) */
  int32_t de_strategy;    /* DEBYE_DE_RAND1 (default) or DEBYE_DE_BEST1 */
  double  da_t0;          /* dual annealing: initial visiting temperature, > 0 (default 5230) */
  double  da_qa;          /* dual annealing: acceptance parameter, < 1 (default -5) */
  int32_t solve_lanes;    /* mixed precision: lanes per candidate of the small-system solve
                             after the column-sum pass: 1 = one thread per candidate, 32 =
                             one warp per candidate (lane r: row r), 0 = by size (default: a
                             warp per candidate when an evaluation has at most 256
                             candidates per SM). Results agree to rounding either way.
                             debye_eval_population_noalloc always takes one thread per
                             candidate. */
  int32_t lanes_per_candidate; /* lanes that share one candidate's frequency samples in the
                             pass kernels of full populations (a warp or more of
                             candidates per spectrum): 0 = autotune / 1, else 1..32, a
                             power of two */
} debye_options;

/* A ragged batch of S spectra, CSR over frequency (all device memory unless _host). */
typedef struct {
  int64_t        S;          /* number of spectra, >= 0 */
  const int64_t* offsets;    /* [S+1]; spectrum s owns samples offsets[s] .. offsets[s+1]-1 */
  const double*  omega;      /* [offsets[S]] angular frequency (rad/s), > 0 */
  const double*  eps_re;     /* [offsets[S]] eps'  (Eq. 1) */
  const double*  eps_im;     /* [offsets[S]] eps'' (Eq. 1; a lossy sample has eps'' > 0) */
  const int32_t* n_poles;    /* [S] Debye poles N_s to fit, 1..DEBYE_MAX_POLES */
  const double*  lo;         /* [S] lower bound of log10(tau) */
  const double*  hi;         /* [S] upper bound of log10(tau), > lo */
  const int64_t* offsets_host;  /* optional host copy of offsets (avoids a device read) */
  const int32_t* n_poles_host;  /* optional host copy of n_poles */
} debye_spectra;

/* Search settings of debye_fit_batch. */
typedef struct {
  int32_t  P;             /* particles (population members) per spectrum, 1..32768 */
  int32_t  iters;         /* generations after the initial one, >= 0 */
  uint64_t seed;          /* seed of the counter-based generator */
  int32_t  polish_topk;   /* personal bests polished per spectrum, 0..min(P,64) */
  int32_t  polish_iters;  /* L-BFGS iterations per polished candidate, >= 0 */
  double*  trace;         /* optional [S][iters+1] device: global-best cost per generation */
  double*  evals;         /* optional [1] device: candidate evaluations x K, counted as a
                             sequential search evaluates them (the swarm's populations; per
                             polish iteration the trials of a backtracking line search up to
                             the accepted one, not the speculative step lengths after it) */
  int32_t  method;        /* DEBYE_SEARCH_PSO (0), DEBYE_SEARCH_DE or DEBYE_SEARCH_DA */
  int32_t* n_failed;      /* optional [S] device, caller-initialised: incremented once per
                             evaluated candidate of spectrum s (search, polish and final
                             re-solve) whose damped normal matrix is not positive definite */
} debye_search;

/* Fill *opt with the defaults listed above. */
void debye_default_options(debye_options* opt);

/* Create a handle on the current CUDA device. opt may be NULL (defaults).
 * Returns DEBYE_EINVAL for out-of-range options, DEBYE_ECUDA if no device. */
int debye_fit_init(debye_handle* out, const debye_options* opt);

/* Release a handle and its device workspaces. NULL is accepted. */
int debye_fit_destroy(debye_handle h);

/* Target synthesis (Eqs. 3-7): write eps', eps'' of every spectrum from its model
 * id [S] and parameter record params[S][DEBYE_N_PARAMS] (layout per model id:
 * Debye/HN/CC/CD [eps_inf, d_eps, tau0, alpha, beta]; Jonscher [eps_inf, a_p,
 * omega_p, n_p]; CRIM [a, m, f_1..f_3, (eps_inf_i, d_eps_i, tau_i) x 3];
 * Debye sum [eps_inf, a_p, omega_p, n_p, sigma] with source poles
 * pole_tau/pole_deps over pole_offsets[S+1] and multiplicative noise
 * eps'(1 + sigma z_re), eps''(1 + sigma z_im), z given in noise_re/noise_im
 * [offsets[S]] (NULL = no noise)). offsets and omega as in debye_spectra. */
int debye_synth_targets(debye_handle h, int64_t S, const int64_t* offsets, const double* omega,
                        const int32_t* model, const double* params, const int64_t* pole_offsets,
                        const double* pole_tau, const double* pole_deps, const double* noise_re,
                        const double* noise_im, double* eps_re, double* eps_im,
                        cudaStream_t stream);

/* DLS cost of a fed-in population (Sec. III-B): for every candidate theta[s][p],
 * the damped least-squares weights at damping lam_search, the sign flip of
 * negative d_eps, and cost = ||A x_hat - b||^2 + lam sum_j G_jj x_hat_j^2 over the
 * stacked real/imaginary rows. cost [S][P]; weights [S][P][n_max+1] or NULL.
 * n_max >= max_s N_s. n_failed [S] (device, caller-initialised, or NULL) is
 * incremented once per candidate of spectrum s whose damped normal matrix is not
 * positive definite (its cost is +inf and its weights 0). */
int debye_eval_population(debye_handle h, const debye_spectra* spectra, int32_t P, int32_t n_max,
                          const double* theta, double* cost, double* weights, int32_t* n_failed,
                          cudaStream_t stream);

/* Cost (as debye_eval_population) and its exact gradient d cost / d theta
 * (variable projection, including the flipped case), grad [S][P][n_max];
 * n_failed as for debye_eval_population (the gradient of a failed candidate is 0). */
int debye_cost_grad(debye_handle h, const debye_spectra* spectra, int32_t P, int32_t n_max,
                    const double* theta, double* cost, double* grad, int32_t* n_failed,
                    cudaStream_t stream);

/* Whole fit (Sec. III-B, IV): seeded particle swarm, differential evolution or
 * dual annealing over log10(tau) with DLS weights, projected L-BFGS polish of
 * the best polish_topk personal bests (swarm), population members (evolution)
 * or chain states (annealing; iters = outer iterations of 2N moves each), the
 * best result re-solved in FP64 at damping lam_final with the sign flip, poles
 * sorted by ascending tau. Outputs eps_inf [S], d_eps [S][n_max], tau [S][n_max]
 * (seconds; entries beyond N_s are 0) and final_cost [S] (cost at lam_final). */
int debye_fit_batch(debye_handle h, const debye_spectra* spectra, const debye_search* search,
                    int32_t n_max, double* eps_inf, double* d_eps, double* tau,
                    double* final_cost, cudaStream_t stream);

/* Automatic number of poles (Sec. III-B: the pole count set to -1). For every
 * spectrum, complete fits as debye_fit_batch makes them (same search settings)
 * with N = 1, 2, ... poles; the result is the fit with the first N whose average
 * fractional error is below `threshold` (percent; the paper uses 5), or with
 * N = n_poles[s] if none is (n_poles is the per-spectrum cap here; the paper's
 * is 20). The error is the mean over the spectrum's samples of
 * |eps'_fit - eps'| / |eps'| plus the same mean for eps'' (Sec. IV), times 100.
 * Every fit of spectrum s draws its random numbers with s as the spectrum key,
 * whatever N, so the result equals that of the sequential N = 1, 2, ... loop.
 * The fits run in waves of `wave` (1..20) consecutive pole counts, each wave one
 * ragged batch; spectra that found their N leave before the next wave (the call
 * synchronises its work stream once per wave). Outputs as debye_fit_batch
 * (d_eps, tau [S][n_max], zero beyond the chosen N) plus frac_err [S] (percent)
 * and n_chosen [S]. search->trace and search->n_failed must be NULL. */
int debye_fit_auto(debye_handle h, const debye_spectra* spectra, const debye_search* search,
                   int32_t n_max, double threshold, int32_t wave, double* eps_inf, double* d_eps,
                   double* tau, double* final_cost, double* frac_err, int32_t* n_chosen,
                   cudaStream_t stream);

/* Allocation-free evaluation. The paper has no counterpart to this entry point;
 * it exists for callers that cannot let the library allocate device memory, such
 * as an application embedding the fitter that owns a fixed device-memory budget,
 * or a latency-critical loop where cudaMalloc/cudaFree (which may synchronise the
 * device) are not acceptable.
 *
 * Computes what debye_eval_population computes (costs, and weights if `weights`
 * is not NULL) for the options in `opt` (NULL = defaults), without a handle. The
 * results agree with debye_eval_population's to rounding, within the parity
 * tolerances of the cost (relative 1e-10 with DEBYE_PREC_FP64 and
 * DEBYE_PREC_FP64_SUMS, 1e-5 with DEBYE_PREC_MIXED and DEBYE_PREC_MIXED_TABLE, whose
 * column sums are taken directly here), not bit for bit: the two entry points may split a candidate's
 * samples over different numbers of lanes, and the mixed-precision solve here is
 * always the one-thread-per-candidate kernel. It calls no cudaMalloc, cudaFree
 * or other allocating routine: all temporary data lives in one fixed scratch
 * array of DEBYE_NOALLOC_SCRATCH_BYTES (32 MiB) inside the library's device
 * image, held by every GPU that loads the library until the process exits. A
 * batch whose temporaries do not fit (about 2.3 KB per candidate at n_max = 12,
 * plus 64 B per frequency sample), or that needs more than 4096 work units, is
 * rejected with DEBYE_EINVAL and a message. spectra->offsets_host and
 * spectra->n_poles_host are required.
 *
 * The first call on a device, and the first call after that device's context was
 * reset (cudaDeviceReset), looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current; make that call before any
 * stream capture. Every call on a device shares the one array and leaves its
 * contents behind (the call initialises everything it reads); calls whose work
 * overlaps on the GPU race on the array, so order them (one stream, or events).
 * The call returns after the work on `stream` has finished, with
 * DEBYE_ENOTFINITE / DEBYE_EBOUNDS for input problems found on the device.
 * `err` (may be NULL) receives a message of at most err_len bytes. */
#define DEBYE_NOALLOC_SCRATCH_BYTES (32u << 20)
int debye_eval_population_noalloc(const debye_options* opt, const debye_spectra* spectra, int32_t P,
                                  int32_t n_max, const double* theta, double* cost, double* weights,
                                  char* err, int32_t err_len, cudaStream_t stream);

/* Work-layout autotuner, for two shapes. Full populations: times
 * debye_eval_population on the caller's batch (theta as for that call, cost
 * [S][P] is overwritten) for every (candidates per block, lanes per candidate)
 * in {(32,1), (64,1), (96,1), (128,1), (32,2), (64,2), (32,4)}. The polish's
 * accepted points: times debye_cost_grad on the first min(P, 8) candidates of
 * every spectrum for (cb, lanes) in {(16,4), (8,8), (4,16), (2,32), (32,4),
 * (16,8), (8,16), (4,32)}. Each layout's evaluation is planned and uploaded
 * outside the timed interval, 4 evaluations are captured in a CUDA graph (as a fit
 * replays its generations) and one replay is timed (CUDA events), over a warm-up and
 * 5 rounds that interleave the layouts; the layout with the lowest median time of
 * each shape is kept for this handle and used
 * by later calls whose options leave cands_per_block and lanes_per_candidate at
 * 0. cache_path (may be NULL) is a text file of "key | cb lanes polish_cb
 * polish_lanes" lines keyed by the device's SM count, precision, S, P, n_max and
 * sample count: a cached choice is reused without timing, a new one is appended.
 * chosen (may be NULL) receives the four numbers. Synchronises `stream`. */
int debye_autotune(debye_handle h, const debye_spectra* spectra, int32_t P, int32_t n_max,
                   const double* theta, double* cost, const char* cache_path, int32_t* chosen,
                   cudaStream_t stream);

/* Wait for `stream`, then return and clear the device status word
 * (DEBYE_OK, DEBYE_ENOTFINITE, DEBYE_EBOUNDS or DEBYE_ETIMEOUT). */
int debye_sync(debye_handle h, cudaStream_t stream);

/* ------------------------------------------------------------------ kernel timing
 * For measurement tools. While enabled, CUDA-graph capture is switched off and
 * every pass of the evaluation is bracketed by CUDA events recorded on the
 * launching stream: a column-sum, Gram, residual/refinement or gradient pass is
 * one kernel per pole count, launched concurrently on forked streams, and its
 * interval runs from the fork to the join; the solves and the finish are single
 * launches. Per kind the library accumulates the number of passes, the summed
 * event time (ms) and the algorithmic FLOPs of the work, per candidate and
 * frequency sample (FMA counted as 2): mixed precision, 54N for the float-float
 * column-sum pass (103N with the derivative sums of a gradient evaluation);
 * FP64, 4N + 2(N+2)^2 for the Gram pass (basis build plus the unique
 * Gram/right-hand-side products) and 13N + 5 for the residual pass.
 * Passes restricted by an activity mask (the polish line search and its accepted
 * points) are accumulated under their own *_MASKED kinds, with time but no FLOPs. */
#define DEBYE_KERNEL_GRAM          0
#define DEBYE_KERNEL_REFINE        1
#define DEBYE_KERNEL_GRAD          2
#define DEBYE_KERNEL_SOLVE         3
#define DEBYE_KERNEL_FINISH        4
#define DEBYE_KERNEL_GRAM_MASKED   5
#define DEBYE_KERNEL_REFINE_MASKED 6
#define DEBYE_KERNEL_GRAD_MASKED   7
#define DEBYE_KERNEL_SUMS          8
#define DEBYE_KERNEL_SUMS_MASKED   9
#define DEBYE_KERNEL_TABLE         10  /* DEBYE_PREC_MIXED_TABLE: table build (node pass, coefficients) */
#define DEBYE_KERNEL_TABLE_EVAL    11  /* DEBYE_PREC_MIXED_TABLE: candidates' sums from the tables */
#define DEBYE_KERNEL_KINDS         12

/* Failure-path check of the bounded device-side waits: one block runs the column-sum
 * pass's staging wait (an mbarrier wait bounded by about 1 s of SM clock) on a buffer
 * that no copy will fill. The wait gives up, records DEBYE_ETIMEOUT in the handle's
 * status word (returned by the next debye_sync) and the kernel ends; the context and
 * the handle stay usable. Enqueued on `stream`; returns DEBYE_OK once launched. */
int debye_check_bounded_wait(debye_handle h, cudaStream_t stream);

/* Number of kernel launches the handle has enqueued (a CUDA-graph replay counts
 * each of its kernel nodes); reset != 0 sets the counter to zero afterwards. */
int debye_launch_count(debye_handle h, int64_t* count, int32_t reset);

/* Enable (1) or disable (0) kernel timing; enabling clears the totals. */
int debye_profile_enable(debye_handle h, int32_t enable);

/* Totals of kind `kind` since timing was enabled: passes (or launches), summed
 * milliseconds, FLOPs (waits for the recorded events). Any output may be NULL. */
int debye_profile_read(debye_handle h, int32_t kind, int64_t* launches, double* ms, double* flops);

/* Message of the last failed call on h (never NULL; "" if none). */
const char* debye_last_error(debye_handle h);

/* Library version string. */
const char* debye_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DEBYEFIT_H */
