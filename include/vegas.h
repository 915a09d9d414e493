/*
 * vegas.h -- C ABI of the GB300 (sm_103a) VEGAS iteration library.
 *
 * The method is VEGAS adaptive importance sampling (Lepage 1978, 1980), which
 * the paper takes as the algorithm of VegasFlow (Sec. 1).  The calls follow the
 * paper's statement of an integration (Sec. 3.1): an integrand over the unit
 * hypercube of n_dim dimensions, n_events samples per iteration, an
 * events_limit per device batch, and run_integration(n_iter) = n_iter rounds
 * of iterate -> refine, whose per-iteration results are combined.  Each
 * iteration informs the grid of the next (Sec. 3.2).
 *
 * One iteration t of an integral with d dimensions and N bins per dimension:
 *   for s in [0, n):  r_j = Philox4x32-10(ctr = (s_lo, s_hi, t, j/4),
 *                                         key = (seed, integral_id))[j % 4]
 *                     i_j = (r_j * N) >> 32         (64-bit integer product)
 *                     y_j = low 32 bits of r_j * N, times 2^-32
 *                     x_j = e_j[i_j] + (e_j[i_j+1] - e_j[i_j]) * y_j
 *                     J   = prod_j N (e_j[i_j+1] - e_j[i_j])
 *                     v   = J f(x);  S1 += v; S2 += v^2; h_j[i_j] += v^2
 *   I_t = S1/n,  sigma_t^2 = (S2/n - I_t^2)/(n - 1)
 * Refinement per dimension: 3-point smoothing of h_j, normalisation,
 * compression rho = ((1 - d)/ln(1/d))^alpha, rebinning to N bins of equal
 * rho-weight.  Combination: inverse-variance weighted mean, sigma, chi^2/dof.
 *
 * Conventions for every call:
 *   - Every call returns a vegas_status; nothing throws across the ABI.
 *   - Pointers named dev_* are CUDA device pointers; all others are host.
 *   - A context owns no device memory: the caller allocates the workspace
 *     (vegas_workspace_bytes) and keeps it alive until vegas_destroy.  It
 *     owns a small host-side struct only.
 *   - All device work is enqueued on the caller's stream, in stream order.
 *     Calls that return host values synchronise that stream.
 *   - A context must not be used from two threads at once.
 *   - VEGAS_ECUDA: a CUDA runtime call failed; vegas_last_error_string()
 *     gives the CUDA error text.
 */
#ifndef VEGAS_GB300_H
#define VEGAS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VEGAS_OK = 0,
    VEGAS_EINVAL = 1,     /* invalid argument or configuration               */
    VEGAS_ENOMEM = 2,     /* workspace too small                              */
    VEGAS_ECUDA = 3,      /* a CUDA runtime call failed                       */
    VEGAS_ETIMEOUT = 4,   /* a bounded device wait ran out                    */
    VEGAS_EBUSY = 5,      /* no free slot (batched form)                      */
    VEGAS_ENONFINITE = 6, /* every integrand value of the iteration was non-finite */
    VEGAS_EJIT = 7        /* a user integrand did not compile (vegas_jit_log)   */
} vegas_status;

/* Arithmetic of the sampling path.
 *   VEGAS_FP64       : uniforms, grid map, Jacobian, integrand and all sums in
 *                      FP64; histograms in FP64 shared-memory cells.
 *   VEGAS_FP32_ACC64 : map, Jacobian and integrand in FP32 (the in-bin
 *                      position is the 32-bit low word rounded to FP32, not
 *                      truncated); per-thread FP32 partial sums of v and v^2
 *                      over 16 samples, added into FP64.
 *   VEGAS_FP32_KAHAN : as FP32_ACC64, with the per-thread sums of v and v^2
 *                      Kahan-compensated FP32.
 * Histograms in both FP32 modes: in an iteration after a settled one (its
 * mean v^2 at most 1024 times its squared mean v), 32-bit fixed-point integer
 * cells in shared memory, each v^2 rounded to 2^-19 of the previous
 * iteration's mean v^2 (values below 2^-18 of it to 2^-34 of it, never to 0;
 * values above 32 times it straight to FP64); otherwise FP32 cells.  Either
 * is added into FP64 once per block.  The histograms drive only refinement.
 * Refinement and the combination of iterations are FP64 in every mode. */
typedef enum {
    VEGAS_FP64 = 0,
    VEGAS_FP32_ACC64 = 1,
    VEGAS_FP32_KAHAN = 2
} vegas_precision;

/* Built-in integrand families over [0,1]^d, parameters as FP64 arrays:
 *   CONST        f = 1                                   params: none
 *   SUM          f = sum_i x_i (the toy integrand of Sec. 3.1)   none
 *   GAUSS_SYM    f = (a sqrt(pi))^-d exp(-sum (x_i - 1/2)^2 / a^2)   [a]
 *   GENZ_OSC     f = cos(2 pi u + sum c_i x_i)           [u, c_1..c_d]
 *   GENZ_GAUSS   f = exp(-sum c_i^2 (x_i - w_i)^2)       [c_1..c_d, w_1..w_d]
 *   GENZ_PROD    f = prod (c_i^-2 + (x_i - w_i)^2)^-1    [c_1..c_d, w_1..w_d]
 *   GENZ_CORNER  f = (1 + sum c_i x_i)^-(d+1)            [c_1..c_d]
 *   LO           d = 3 LO-style 2->2 toy: x1, x2 momentum fractions with
 *                density g(x) = (35/32) x^-1/2 (1-x)^3, c = 2 x3 - 1,
 *                shat = x1 x2 sqrtS^2, f = g(x1) g(x2) BW(shat) (1+c^2)/shat * 2 * norm
 *                with BW = 1/((shat - M^2)^2 + M^2 Gamma^2), |c| < cut and
 *                mll_lo <= sqrt(shat) <= mll_hi.
 *                params: [sqrtS, M, Gamma, cut, mll_lo, mll_hi, norm]
 * The paper's integrand is a user function of the sample array (Sec. 3.1);
 * these families stand in for it. */
typedef enum {
    VEGAS_F_CONST = 0,
    VEGAS_F_SUM = 1,
    VEGAS_F_GAUSS_SYM = 2,
    VEGAS_F_GENZ_OSC = 3,
    VEGAS_F_GENZ_GAUSS = 4,
    VEGAS_F_GENZ_PROD = 5,
    VEGAS_F_GENZ_CORNER = 6,
    VEGAS_F_LO = 7,
    VEGAS_F_USER = 8,     /* a user's source, vegas_create_user (not vegas_create) */
    VEGAS_F_LO_PDF = 9    /* LO with its density from a grid (vegas_set_pdf_grid) */
} vegas_family;

#define VEGAS_MAX_DIM 32
#define VEGAS_MAX_BINS 1024
#define VEGAS_MAX_ITERS 4096  /* per-iteration records kept (a ring); iterations are unbounded */
#define VEGAS_MAX_USER_PARAMS 72  /* parameters of a user integrand */

typedef struct {
    int32_t family;         /* vegas_family                                   */
    int32_t n_dim;          /* must equal vegas_config.n_dim                  */
    const double *params;   /* host array, n_params values, copied at create  */
    int32_t n_params;       /* exactly the count the family takes             */
} vegas_integrand;

typedef struct {
    int32_t n_dim;          /* d, 1..VEGAS_MAX_DIM (Sec. 3.1: n_dim)          */
    int32_t n_bins;         /* N, 2..VEGAS_MAX_BINS                           */
    int64_t n_events;       /* n samples per iteration, >= 2 (Sec. 3.1)       */
    int64_t events_limit;   /* max samples per kernel launch; <= 0: no limit
                               (Sec. 3.1: events_limit).  Samples are made on
                               the device, so this only splits launches.     */
    double alpha;           /* grid compression exponent, >= 0                */
    uint32_t seed;          /* Philox key word 0                              */
    uint32_t integral_id;   /* Philox key word 1                              */
    int32_t precision;      /* vegas_precision                                */
    int32_t smooth;         /* 1: 3-point smoothing before compression        */
} vegas_config;

typedef struct {
    double I;               /* iteration estimate                             */
    double sigma;           /* its standard error                             */
    int64_t n;              /* samples with finite weight                     */
    int64_t n_nonfinite;    /* samples skipped: v (FP32: or v^2) NaN or Inf   */
} vegas_iter_result;

typedef struct {
    double I;               /* combined estimate over all iterations so far   */
    double sigma;           /* combined standard error                        */
    double chi2_dof;        /* chi^2 per degree of freedom (0 for one iteration) */
    int32_t n_iter;         /* iterations run, including any left out because
                               they had no finite value                       */
    int32_t reserved;
} vegas_result_t;

typedef struct vegas_ctx vegas_ctx;

/* Bytes of device workspace a context with this configuration needs
 * (0 if the configuration is invalid).  The caller allocates it, 256-byte
 * aligned, and passes it to vegas_create. */
size_t vegas_workspace_bytes(const vegas_config *cfg);

/* Validate cfg and integrand, lay out the workspace, upload the uniform grid
 * e_j[k] = k/N and the parameters, zero the accumulators.  stream: a
 * cudaStream_t (NULL = legacy default stream).  On success *out owns a host
 * struct that vegas_destroy frees.  EINVAL for a bad configuration or
 * parameter count, ENOMEM if ws_bytes is below vegas_workspace_bytes. */
vegas_status vegas_create(const vegas_config *cfg, const vegas_integrand *integrand,
                          void *stream, void *dev_workspace, size_t ws_bytes, vegas_ctx **out);

/* A user integrand, as the paper's integrator takes one (Sec. 3.1: the
 * integrand is a function of the sample array passed to compile()).  source
 * is CUDA C++ that defines, at global scope,
 *     template <class T> __device__ T user_integrand(const T *x, int d, const T *p);
 * returning f at the mapped point x[0..d-1] (each in [0,1]) with parameters
 * p[0..n_params-1] (n_params <= VEGAS_MAX_USER_PARAMS, copied at create).  T is
 * float in the FP32 precisions and double in VEGAS_FP64; the standard math
 * functions of both types may be called (exp, cos, pow, ...).  The library
 * compiles it at run time with NVRTC for sm_103a together with its own
 * sampling, stratified-sampling and trace kernels, so the integrand is inlined
 * into the same fused kernel as the built-in families; each (source,
 * precision, d, layout) is compiled once per process and kept loaded until
 * exit.  The first values of f should lie within the FP32 range in the FP32
 * precisions (v is rescaled from the second iteration on).  Everything else is
 * as vegas_create with family VEGAS_F_USER (vegas_export_state records the
 * parameters but not the source: import into a context made from the same
 * source).  VEGAS_EJIT if the source does not compile or NVRTC cannot be
 * loaded (vegas_jit_log gives the compiler's messages).  The batched form and
 * vegas_iterate_noalloc take built-in families only. */
vegas_status vegas_create_user(const vegas_config *cfg, const char *source, const double *params,
                               int32_t n_params, void *stream, void *dev_workspace, size_t ws_bytes,
                               vegas_ctx **out);
/* The compiler's messages of this thread's last vegas_create_user. */
const char *vegas_jit_log(void);

/* Run one iteration on the current grid: sample, accumulate S1, S2 and the
 * histograms, then form I_t, sigma_t and update the combination on the
 * device.  Asynchronous if out == NULL; otherwise synchronises the stream and
 * fills *out.  NaN or infinite values of J f are counted in n_nonfinite and
 * left out of the sums and of n (stratified iterations: counted as 0, n keeps
 * every sample); in the FP32 modes so is a finite J f whose square exceeds
 * the FP32 range (the sums take (J f)^2).  ENONFINITE (with *out filled) if no sample had a finite
 * weight: that iteration has no estimate and is left out of the combination,
 * and a refinement after it keeps the grid (its histograms are zero).
 * The combination: Ibar = sum w_t I_t / sum w_t, w_t = 1/sigma_t^2,
 * sigma = (sum w_t)^-1/2, chi^2/dof = sum w_t (I_t - Ibar)^2 / (m - 1) over the
 * m combined iterations, kept as running sums about the first iteration's
 * estimate (no cancellation when the iterations agree to many digits); if any
 * iteration has sigma_t = 0 (exact), the mean of those is the result with
 * sigma 0. */
vegas_status vegas_iterate(vegas_ctx *ctx, vegas_iter_result *out);

/* Sharded iteration: one integral's samples split over several devices or
 * processes (the paper's multi-device use of one integration, Sec. 3.1 and
 * Sec. 3.2: each iteration's partial results are combined before the grid is
 * refined).  Every shard holds a context with the same configuration and
 * grid; per iteration:
 *   vegas_sample_shard(ctx, s_begin, count)  samples its range of the
 *       iteration's n_events samples into the context's accumulators;
 *   the caller sums the accumulators of all shards in place on every shard
 *       (vegas_accumulators gives them: 2 + d*N FP64 values in the
 *       context's current scale, identical on every shard, plus one
 *       64-bit non-finite count), e.g. with an all-reduce;
 *   vegas_finalize(ctx, out) forms the iteration result for all n_events
 *       samples and advances the iteration (as vegas_iterate does after its
 *       sampling); then vegas_refine gives every shard the same grid.
 * Sample indices are global, so the union of the shards is exactly the
 * single-context iteration.  Asynchronous unless out != NULL. */
vegas_status vegas_sample_shard(vegas_ctx *ctx, int64_t s_begin, int64_t count);
vegas_status vegas_accumulators(vegas_ctx *ctx, double **dev_sums, int64_t *n_sums,
                                unsigned long long **dev_nonfinite);
vegas_status vegas_finalize(vegas_ctx *ctx, vegas_iter_result *out);

/* vegas_iterate followed by vegas_refine, with the iteration result and the
 * refinement in one launch (what run_integration does for every iteration
 * but the last).  Same results as the two calls. */
vegas_status vegas_step(vegas_ctx *ctx, vegas_iter_result *out);

/* One vegas_step (sampling, iteration result and refinement: the iteration of
 * Sec. 1, whose result informs the next grid, Sec. 3.2) of
 * each of n independent integrals, 1 <= n <= VEGAS_MAX_STEP_MANY: their
 * sampling launches in the given order, then ONE launch for all n iteration
 * results and refinements (d_k + 1 blocks for context k), so that a set of
 * integrals advanced together pays one small launch per iteration, not n.
 * ctxs: n distinct contexts (host array, read during the call) that share one
 * stream.  Asynchronous: read the results with vegas_result / vegas_run's
 * records.  Each context's results are those of vegas_step on it, up to the
 * order of the FP64 atomic additions of its block sums (which no launch fixes).
 * Errors: VEGAS_EINVAL for a NULL array or context, n out of range, a context
 * given twice, contexts on different streams, or a density-grid context
 * without its grid (nothing is launched then); a launch error as vegas_step. */
#define VEGAS_MAX_STEP_MANY 8
vegas_status vegas_step_many(vegas_ctx *const *ctxs, int32_t n);

/* Refine the grid from the last iteration's histograms (asynchronous). */
vegas_status vegas_refine(vegas_ctx *ctx);

/* Synchronise the stream and return the combination of all iterations run. */
vegas_status vegas_result(vegas_ctx *ctx, vegas_result_t *out);

/* run_integration of Sec. 3.1: n_iter rounds of iterate + refine (no refine
 * after the last), then vegas_result.  iters (may be NULL; then n_iter <=
 * VEGAS_MAX_ITERS) receives n_iter per-iteration results. */
vegas_status vegas_run(vegas_ctx *ctx, int32_t n_iter, vegas_iter_result *iters,
                       vegas_result_t *out);

/* Grid access (host arrays of d rows of N+1 FP64 edges).  set_grid checks
 * that each row starts at 0, ends at 1 and does not decrease (EINVAL). */
vegas_status vegas_get_grid(vegas_ctx *ctx, double *edges_host);
vegas_status vegas_set_grid(vegas_ctx *ctx, const double *edges_host);

/* The last iteration's FP64 sums, host array of 2 + d*N values:
 * [S1, S2, h_0[0..N-1], ..., h_{d-1}[0..N-1]].  Synchronises the stream. */
vegas_status vegas_get_sums(vegas_ctx *ctx, double *sums_host);

/* Samples per iteration from the next vegas_iterate on (>= 2).  The sample
 * indices of an iteration are always 0..n_events-1. */
vegas_status vegas_set_events(vegas_ctx *ctx, int64_t n_events);

/* Iteration counter t (the Philox counter word 2 of the next iteration). */
vegas_status vegas_get_iteration(vegas_ctx *ctx, int32_t *t);
vegas_status vegas_set_iteration(vegas_ctx *ctx, int32_t t);

/* Per-sample view of iteration t on the current grid, for samples
 * [s_begin, s_begin + count): dev_bins (int32, count x d, row-major),
 * dev_x (FP64, count x d) and dev_w (FP64, count: v = J f before any
 * scaling).  Any output pointer may be NULL.  Computed by the same device
 * code as vegas_iterate, in the context's precision.  Asynchronous. */
vegas_status vegas_trace(vegas_ctx *ctx, int32_t t, int64_t s_begin, int64_t count,
                         int32_t *dev_bins, double *dev_x, double *dev_w);

/* Observable histogram of iteration t's weights, for the analysis step that
 * follows integration in the paper's generator chain (Fig. 1: histogramming).
 * Every sample iteration t would draw on the context's current grid (the
 * stratified set when vegas_set_strata is on) is computed again, and its
 * weight v = J f (unscaled; left out if not finite) is added to the bin of
 * its observable o, in shared memory per block, with no traffic per sample:
 *   observable >= 0 : o = x_observable (a coordinate, < n_dim);
 *   -1 (LO families): o = sqrt(shat) = sqrt(x1 x2) sqrtS, in GeV;
 *   -2 (LO families): o = cos(theta) = 2 x3 - 1.
 * dev_out (device, FP64, 2 (nbins + 2) values, zeroed by the call): dev_out[b]
 * = sum of v and dev_out[nbins + 2 + b] = sum of v^2 over the samples of bin b,
 * with bin 0 below lo, bin 1 + floor((o - lo)/w) (w = (hi - lo)/nbins, at most
 * nbins) up to hi and bin nbins + 1 at or above hi.  dev_out[b] / n is bin b's
 * part of the iteration's estimate (n = the samples the iteration uses).  Does
 * not change the context's state.  1 <= nbins <= 1024.  Asynchronous. */
vegas_status vegas_histogram(vegas_ctx *ctx, int32_t t, int32_t observable, int32_t nbins, double lo, double hi,
                             double *dev_out);

/* Stratified + importance hybrid: the combined mode of Lepage's VEGAS (Cornell
 * CLNS-80/447, 1980; the method the paper takes as VegasFlow's, Sec. 1), in
 * which y-space is also cut into equal hypercubes that each receive the same
 * number of samples.  With B != 0 every later iteration uses H = 2^B
 * hypercubes of P = floor(n_events / H) samples, H P samples in all.
 * Dimension j is halved b_j = floor(B/d) + (j < B mod d ? 1 : 0) times;
 * hypercube h's stratum in it, k_j, is the integer in bits
 * [b_0 + ... + b_(j-1), b_0 + ... + b_j) of h.  Sample s lies in hypercube
 * s / P, and its Philox word r_j is moved into the stratum,
 *     R_j = k_j 2^(32 - b_j) + (r_j >> b_j)    (y_j = (k_j + r_j 2^-32) / 2^b_j),
 * which then takes r_j's place in the grid map (bin, interpolation, J).  The
 * estimate is the mean of the hypercube means, I = S1 / (H P); its variance
 * the sum of the hypercubes' variances of the mean,
 *     sigma^2 = sum_h m2_h / (H^2 P (P - 1)),  m2_h = sum_(s in h) (v_s - mean_h)^2.
 * The histograms take (J f)^2 per sample as in plain sampling.  A non-finite
 * J f counts as 0 (and in n_nonfinite), so every hypercube keeps P samples.
 *   B = 0  : plain importance sampling (the default);
 *   B = -1 : as many hypercubes as leave P >= 2;
 *   B > 0  : 2^B hypercubes, fewer where P would drop below 2.
 * B never exceeds 16 halvings per dimension nor 31 in all.  EINVAL for B
 * outside [-1, 31] and, in the FP32 modes, when one hypercube's P samples
 * exceed what one block's fixed-point histogram cells hold between flushes
 * (64 N copies-per-cell samples; vegas_set_events checks the same).
 * Stratified iterations are not sharded: vegas_sample_shard returns EINVAL.
 * vegas_trace follows the setting (sample s of the stratified iteration). */
vegas_status vegas_set_strata(vegas_ctx *ctx, int32_t B);
/* The stratification of the next iteration: *B (0: plain), *P (0: plain) and
 * *n_used, the samples it takes (n_events when plain).  Any pointer may be NULL. */
vegas_status vegas_get_strata(vegas_ctx *ctx, int32_t *B, int64_t *P, int64_t *n_used);

/* Density grid of the VEGAS_F_LO_PDF family: the LO toy of VEGAS_F_LO (same
 * parameters, cuts and Breit-Wigner) with the parton density g(x, Q^2) taken
 * at the scale Q^2 = shat from a tabulated grid, as the paper's companion tool
 * (PDFFlow, Sec. 2) evaluates parton densities from grids on the GPU:
 *     f = g(x1, shat) g(x2, shat) BW(shat) (1 + c^2)/shat * 2 * norm.
 * dev_xg (device, FP64, row-major nx x nq, 2 <= nx, nq, (nx + 2)(nq + 2) <= 6144) holds
 * x g(x, Q^2) at ln x = u0 + i (u1 - u0)/(nx - 1), ln Q^2 = v0 + j (v1 - v0)/(nq - 1).
 * Between knots: bicubic Hermite interpolation in (ln x, ln Q^2) with each
 * knot's tangent the central difference of its neighbours (one-sided at the
 * first and last knot); outside the grid the coordinates are clamped to it.
 * The caller owns dev_xg and keeps it alive and unchanged while the context
 * samples; each sampling block copies it into shared memory in the path's
 * precision.  Call before the first iteration (iterating without a grid:
 * EINVAL); may be called again with another grid.  EINVAL for another family,
 * bad sizes or ranges, or a grid that does not fit shared memory with the
 * context's cells. */
vegas_status vegas_set_pdf_grid(vegas_ctx *ctx, const double *dev_xg, int32_t nx, int32_t nq, double u0,
                                double u1, double v0, double v1);

/* Checkpoint: a byte blob holding config, parameters, FP64 grid, iteration
 * counter, per-iteration results and the running combination (format 4).
 * export with buf == NULL sets *size.  import restores them into a context
 * created with the same configuration, family and parameters (EINVAL
 * otherwise, and for a blob of another format). */
vegas_status vegas_export_state(vegas_ctx *ctx, void *buf, size_t *size);
vegas_status vegas_import_state(vegas_ctx *ctx, const void *buf, size_t size);

/* Device Philox4x32-10 (Salmon et al., SC'11) over n counters:
 * dev_ctr (n x 4 u32), dev_key (n x 2 u32) -> dev_out (n x 4 u32).
 * The same device function the sampling kernel uses.  Asynchronous. */
vegas_status vegas_philox(const uint32_t *dev_ctr, const uint32_t *dev_key, uint32_t *dev_out,
                          int64_t n, void *stream);

/* No-allocation form of one iteration's sums.  (The paper has no counterpart:
 * this entry point exists for callers of this library, not for the method.)
 *
 * Some callers cannot allocate device memory when they call us: a runtime
 * that owns the whole device through its own pool or arena and forbids other
 * allocations, a plugin or callback that must not grow the process's memory
 * footprint, or code on a path where cudaMalloc's implicit device
 * synchronisation would stall other work.  vegas_iterate_noalloc needs no
 * workspace and no context: its scratch (accumulators, counters, grid table)
 * lives in a fixed device array inside this library, of 2 + 4096 FP64 sums
 * plus a 4096-entry table (about 100 KB), which every GPU that loads the
 * library holds until the process exits.  It never calls cudaMalloc,
 * cudaFree or an allocating library routine.
 *
 * It computes what vegas_iterate's sampling does for iteration t (the Philox
 * counter word) of the given configuration and integrand on the grid
 * dev_edges (device, d rows of N+1 FP64 edges, read only), and writes
 * dev_sums (device, 3 + d*N FP64: S1, S2, h_0[0..N-1], ..., in the layout of
 * vegas_get_sums, then the number of samples whose J f was NaN or infinite,
 * which S1, S2 and the histograms leave out: I = S1 / (n_events - that
 * count)).  Asynchronous on stream; nothing else is reported back except the
 * status.
 *   - EINVAL for an invalid configuration or integrand, and when
 *     n_dim * n_bins exceeds 4096 (vegas_last_error_string says so).
 *   - The first call on each device looks up the scratch array's device
 *     address (once per device, with that device current); make that first
 *     call before any stream capture.
 *   - Every call uses the same array: each call clears it before use, and
 *     calls that overlap on the GPU (other streams, other host threads)
 *     race and corrupt each other's sums.  Serialise them.
 *   - FP32 modes always use FP32 histogram cells here (as the first
 *     iteration of a context does). */
vegas_status vegas_iterate_noalloc(const vegas_config *cfg, const vegas_integrand *integrand,
                                   int32_t t, const double *dev_edges, double *dev_sums,
                                   void *stream);

/* Tracing: with enable != 0, every vegas_iterate records a CUDA event pair
 * on the context's stream around its sampling-kernel launches.
 * vegas_profile_read synchronises the stream, writes up to cap durations in
 * milliseconds (oldest first) to ms_out, sets *count to the number written
 * and forgets all recorded pairs. */
vegas_status vegas_profile(vegas_ctx *ctx, int32_t enable);
vegas_status vegas_profile_read(vegas_ctx *ctx, float *ms_out, int32_t cap, int32_t *count);

/* ------------------------------------------------------------------------
 * Batched form: many integrals of uneven dimension, family and sample count
 * advance one iteration each per step, in one persistent sampling launch plus
 * a finalize and a refinement launch, replayed as one captured CUDA graph.
 * (The paper distributes one integral's events over devices, Sec. 3.1-3.2;
 * batching many integrals on one device is this library's serving form.)
 *
 * Sample s of a slot in iteration t draws the same Philox words as in a
 * single-integral context with the same seed and integral_id, so each slot's
 * iteration estimates equal its estimates alone up to summation order.  The
 * combination across iterations is vegas_iterate's (running sums about the
 * first estimate; iterations without a finite value left out).
 *
 * The workspace (caller-allocated, 256-byte aligned) holds the step plan,
 * the per-slot state table and a pool from which each added integral takes
 * vegas_batch_slot_bytes(cfg) bytes (grid, table, accumulators) until it is
 * removed: admission is by free slots (EBUSY) and pool bytes (ENOMEM).
 * Only FP32 precisions (VEGAS_FP32_KAHAN, VEGAS_FP32_ACC64).  A step is a
 * captured CUDA graph, which the legacy NULL stream cannot hold: with
 * stream == NULL the batch creates (and destroys) its own stream. */
typedef struct vegas_batch vegas_batch;

typedef struct {
    int32_t slot;              /* slot id                                   */
    int32_t t;                 /* Philox iteration word of the step's iteration */
    vegas_iter_result it;      /* that iteration                            */
    vegas_result_t comb;       /* combination of all its iterations so far;
                                  comb.reserved = 6 if every weight was non-finite */
} vegas_batch_result;

size_t vegas_batch_workspace_bytes(int32_t max_slots, size_t pool_bytes);
size_t vegas_batch_slot_bytes(const vegas_config *cfg);
vegas_status vegas_batch_create(int32_t max_slots, int32_t precision, void *stream, void *dev_workspace,
                                size_t ws_bytes, vegas_batch **out);
/* Add an integral (uniform grid, iteration 0).  cfg->precision must be the
 * batch's; cfg->n_events is its samples per iteration.  Synchronises the
 * stream.  *slot receives its id. */
vegas_status vegas_batch_add(vegas_batch *b, const vegas_config *cfg, const vegas_integrand *integrand,
                             int32_t *slot);
vegas_status vegas_batch_remove(vegas_batch *b, int32_t slot);
/* One iteration of every slot (asynchronous; waits for the previous step). */
vegas_status vegas_batch_step(vegas_batch *b);
/* Wait for the last step and copy out up to cap results (one per slot run,
 * largest sample count first); *count = number written. */
vegas_status vegas_batch_wait(vegas_batch *b, vegas_batch_result *out, int32_t cap, int32_t *count);
vegas_status vegas_batch_get_grid(vegas_batch *b, int32_t slot, double *edges_host);
/* Samples per iteration of a slot from the next step on (>= 2).  Synchronises. */
vegas_status vegas_batch_set_events(vegas_batch *b, int32_t slot, int64_t n_events);
/* Samples per tile (multiple of 512): the unit blocks claim.  Autotune times
 * the sampling kernel for each candidate on the current slots (results are
 * discarded, slot state is unchanged), keeps the fastest and writes the
 * average times (ms) to ms_out (may be NULL). */
vegas_status vegas_batch_set_tile(vegas_batch *b, int32_t tile_samples);

/* Launch shape of the batch's persistent sampling kernel: tile_samples (as
 * above), threads per block (a multiple of 32 in [128, 768]; one block per SM
 * at most 768 threads because the out-of-line samplers keep up to 80
 * registers a thread) and the shared-memory layout (1: lane-private copies of
 * the table and histogram cells, 2: half as many, 0: one copy; -1: the most
 * copies that fit the largest slot, the default).  set_shape synchronises;
 * EINVAL if a value is out of range or the layout does not fit the largest
 * slot (the shape is then unchanged).  A later vegas_batch_add that no longer
 * fits the requested layout falls back to the default rule; get_shape reports
 * the layout in effect. */
typedef struct {
    int32_t tile_samples;
    int32_t threads;
    int32_t layout;
} vegas_batch_shape;
vegas_status vegas_batch_set_shape(vegas_batch *b, const vegas_batch_shape *shape);
vegas_status vegas_batch_get_shape(vegas_batch *b, vegas_batch_shape *out);
/* Autotuner over launch shapes: for each candidate that fits, times reps
 * launches of the sampling kernel on the current slots (their sums are
 * discarded, slot state is unchanged), writes the mean time in ms to ms_out[k]
 * (-1 for a candidate that was skipped; ms_out may be NULL), sets the fastest
 * shape and its index in *best.  EINVAL if no candidate fits. */
vegas_status vegas_batch_autotune_shapes(vegas_batch *b, const vegas_batch_shape *candidates, int32_t n_candidates,
                                         int32_t reps, float *ms_out, int32_t *best);
vegas_status vegas_batch_autotune(vegas_batch *b, const int32_t *candidates, int32_t n_candidates,
                                  int32_t reps, float *ms_out, int32_t *best);
vegas_status vegas_batch_info(vegas_batch *b, int32_t *n_active, size_t *pool_free, size_t *pool_largest,
                              int32_t *tile_samples);
void vegas_batch_destroy(vegas_batch *b);
const char *vegas_batch_last_error(void);

void vegas_destroy(vegas_ctx *ctx);
const char *vegas_strerror(vegas_status st);
const char *vegas_last_error_string(void);

#ifdef __cplusplus
}
#endif
#endif /* VEGAS_GB300_H */
