/*
 * vegas_oracle.h -- plain FP64 CPU oracle for one VEGAS importance-sampling
 * iteration, the method the paper builds on (Sec. 1 names VEGAS, Lepage 1978
 * and 1980; Sec. 3 and Sec. 3.2 describe the iterate -> refine loop).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library; the two are written
 * independently and compared.
 *
 * Everything is double precision, computed in the order the algorithm
 * states, with no blocking or reordering beyond a plain loop over samples.
 */
#ifndef VEGAS_ORACLE_H
#define VEGAS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Integrand families (oracle's own numbering; tests map them by name). */
enum {
    ORACLE_F_CONST = 0,     /* f = 1                                         */
    ORACLE_F_SUM = 1,       /* f = sum_i x_i   (the toy of Sec. 3.1)          */
    ORACLE_F_GAUSS_SYM = 2, /* f = (a sqrt(pi))^-d exp(-sum (x_i-1/2)^2/a^2)  */
    ORACLE_F_GENZ_OSC = 3,  /* f = cos(2 pi u + sum c_i x_i)                  */
    ORACLE_F_GENZ_GAUSS = 4,/* f = exp(-sum c_i^2 (x_i - w_i)^2)              */
    ORACLE_F_GENZ_PROD = 5, /* f = prod (c_i^-2 + (x_i - w_i)^2)^-1           */
    ORACLE_F_GENZ_CORNER = 6,/* f = (1 + sum c_i x_i)^-(d+1)                  */
    ORACLE_F_LO = 7,        /* LO-style 2->2 toy, d = 3 (see the .c file)     */
    ORACLE_F_USER = 8,      /* the function set by oracle_set_user            */
    ORACLE_F_LO_PDF = 9     /* LO toy with g(x, Q^2 = shat) from the grid set by
                               oracle_set_pdf_grid                            */
};

/* Parton-density grid of ORACLE_F_LO_PDF: xg[i * nq + j] = x g(x, Q^2) at
 * ln x = u0 + i (u1 - u0)/(nx - 1), ln Q^2 = v0 + j (v1 - v0)/(nq - 1)
 * (nx, nq >= 2).  The table is referenced, not copied. */
void oracle_set_pdf_grid(int nx, int nq, double u0, double u1, double v0, double v1, const double *xg);

/* x g(x, Q^2) from that grid: bicubic Hermite interpolation in (ln x, ln Q^2),
 * see the .c file. */
double oracle_pdf_xg(double x, double q2);

/* The integrand of ORACLE_F_USER: f(x, d, params), FP64, set by the test
 * from the user's source compiled for the host (one per process). */
typedef double (*oracle_user_fn)(const double *x, int d, const double *params);
void oracle_set_user(oracle_user_fn f);

/* Philox4x32-10 block function (Salmon, Moraes, Dror, Shaw, SC'11). */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* n independent blocks: out[4i..4i+3] = Philox(ctr[4i..4i+3], key[2i..2i+1]). */
void oracle_philox_many(int64_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out);

/* Uniform u32 draw r_j of sample s, dimension j, iteration t:
 * ctr = (s_lo, s_hi, t, j/4), key = (seed, integral_id), word j%4. */
uint32_t oracle_draw(uint64_t s, uint32_t t, int j, uint32_t seed, uint32_t integral_id);

/* FP64 integrand value at point x[d]. Returns 0 for an unknown family. */
double oracle_integrand(int family, int d, const double *params, int n_params, const double *x);

/* Number of parameters a family takes for dimension d (-1: unknown family). */
int oracle_n_params(int family, int d);

/* One sample: bins[d], x[d], Jacobian J, f(x). edges: d rows of N+1. */
void oracle_sample(int d, int N, const double *edges, int family, const double *params,
                   int n_params, uint32_t seed, uint32_t integral_id, uint32_t t,
                   uint64_t s, int32_t *bins, double *x, double *J, double *f);

/* Samples s_begin .. s_begin + count - 1 of iteration t, one oracle_sample
 * each: bins[k*d + j], x[k*d + j] and v[k] = J f. */
void oracle_trace(int d, int N, const double *edges, int family, const double *params,
                  int n_params, uint32_t seed, uint32_t integral_id, uint32_t t,
                  uint64_t s_begin, int64_t count, int32_t *bins, double *x, double *v);

/* Accumulate samples s in [s_begin, s_end) of iteration t into
 * *S1 += v, *S2 += v^2, hist[j*N + i_j] += v^2 (v = J f).  Non-finite v are
 * counted in *n_nonfinite and skipped.  cnt (may be NULL) gets per-bin
 * sample counts, cnt[j*N + i] += 1. */
void oracle_iterate(int d, int N, const double *edges, int family, const double *params,
                    int n_params, uint32_t seed, uint32_t integral_id, uint32_t t,
                    int64_t s_begin, int64_t s_end, double *S1, double *S2, double *hist,
                    int64_t *cnt, int64_t *n_nonfinite);

/* Iteration estimate: I = S1/n, var = (S2/n - I^2)/(n-1) (clamped at 0). */
void oracle_iteration_result(double S1, double S2, int64_t n, double *I, double *var);

/* Grid refinement of every dimension (smooth, normalise, compress with
 * exponent alpha, rebin to N equal-weight bins).  hist: d rows of N;
 * edges_in/edges_out: d rows of N+1.  smooth != 0 enables the 3-point
 * smoothing.  A dimension whose weights sum to zero keeps its old edges. */
void oracle_refine(int d, int N, const double *hist, const double *edges_in, double alpha,
                   int smooth, double *edges_out);

/* Stratified + importance hybrid (Lepage 1980's combined mode): 2^B
 * hypercubes, bits[j] = number of halvings of dimension j
 * (floor(B/d) + (j < B mod d)). */
void oracle_strata_bits(int d, int B, int32_t *bits);

/* One sample s of a stratified iteration with P samples per hypercube
 * (hypercube floor(s/P)); otherwise as oracle_sample. */
void oracle_sample_strat(int d, int N, const double *edges, int family, const double *params,
                         int n_params, uint32_t seed, uint32_t integral_id, uint32_t t, int B,
                         int64_t P, uint64_t s, int32_t *bins, double *x, double *J, double *f);

/* Hypercubes [h_begin, h_end) of a stratified iteration: S1, S2, hist as in
 * oracle_iterate (non-finite v count as 0 and are counted) and
 * *Q += sum_h sum_p (v - mean_h)^2.  vbuf: scratch of P doubles. */
void oracle_iterate_strat(int d, int N, const double *edges, int family, const double *params,
                          int n_params, uint32_t seed, uint32_t integral_id, uint32_t t, int B,
                          int64_t P, int64_t h_begin, int64_t h_end, double *vbuf, double *S1,
                          double *S2, double *Q, double *hist, int64_t *n_nonfinite);

/* Stratified estimate: I = S1/(H P), var = Q/(H^2 P (P-1)). */
void oracle_strat_result(double S1, double Q, int64_t H, int64_t P, double *I, double *var);

/* Observable histogram of samples [s_begin, s_end) of iteration t (P > 0:
 * the stratified iteration of 2^B hypercubes of P samples, else plain):
 * out[b] += v, out[nb + 2 + b] += v^2 for the bin b of the sample's observable
 * (obs >= 0: x_obs; -1: sqrt(shat) = sqrt(x1 x2) params[0]; -2: 2 x3 - 1);
 * bin 0 below lo, bins 1..nb of width (hi - lo)/nb, bin nb + 1 at or above hi.
 * Non-finite v are left out.  out: 2 (nb + 2) values, accumulated into. */
void oracle_histogram(int d, int N, const double *edges, int family, const double *params,
                      int n_params, uint32_t seed, uint32_t integral_id, uint32_t t, int B, int64_t P,
                      int64_t s_begin, int64_t s_end, int obs, int nb, double lo, double hi,
                      double *out);

/* Inverse-variance combination of m iteration results. */
void oracle_combine(int m, const double *I, const double *sigma, double *Ibar, double *sbar,
                    double *chi2_dof);

#ifdef __cplusplus
}
#endif
#endif
