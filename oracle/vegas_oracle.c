/*
 * vegas_oracle.c -- plain FP64 CPU oracle for one VEGAS iteration.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  It shares no
 * code with the CUDA library.
 *
 * The paper (Sec. 1) takes the VEGAS algorithm of Lepage (J. Comput. Phys.
 * 27 (1978) 192; Cornell CLNS-80/447, 1980) as its method and does not
 * restate it; Sec. 3.2 says each iteration's result informs the grid of the
 * next.  The steps below are that published algorithm, restated:
 *
 *   1. uniform grid:   e_j[k] = k/N, Delta_j[k] = 1/N
 *   2. one iteration:  per sample s draw y in [0,1)^d, find the bin
 *      i_j = floor(y_j N), map x_j = e_j[i_j] + Delta_j[i_j] (y_j N - i_j),
 *      weight J = prod_j N Delta_j[i_j], v = J f(x);
 *      S1 += v, S2 += v^2, hist_j[i_j] += v^2
 *      I = S1/n, sigma^2 = (S2/n - I^2)/(n-1)
 *   3. refinement per dimension: smooth, normalise, compress
 *      rho = ((1-d)/ln(1/d))^alpha, rebin to N bins of equal rho-weight
 *   4. combination of iterations by inverse-variance weights, chi^2/dof.
 *
 * Readings where the paper is silent (all stated in the design notes):
 *   - the uniforms are Philox4x32-10 words, ctr = (s_lo, s_hi, t, j/4),
 *     key = (seed, integral_id);
 *   - y_j N is split with integer arithmetic: (uint64) r_j * N gives the
 *     bin in the high word and the in-bin fraction (low word) * 2^-32,
 *     which is exact in FP64;
 *   - the histogram quantity is (J f)^2 (Lepage's), zero-weight bins are
 *     skipped when rebinning, and a new edge that falls exactly on an old
 *     edge takes the lower bin.
 */
#include "vegas_oracle.h"

#include <math.h>
#include <stddef.h>

/* ---------------------------------------------------------------- Philox */
/* Philox4x32 round and key schedule constants as published by Salmon et al.
 * (SC'11, Sec. 5): multipliers M0, M1 and Weyl increments W0, W1. */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { /* key bump between rounds */
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void oracle_philox_many(int64_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
    for (int64_t i = 0; i < n; ++i) oracle_philox4x32_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}

uint32_t oracle_draw(uint64_t s, uint32_t t, int j, uint32_t seed, uint32_t integral_id) {
    uint32_t ctr[4], key[2], out[4];
    ctr[0] = (uint32_t)(s & 0xFFFFFFFFu);
    ctr[1] = (uint32_t)(s >> 32);
    ctr[2] = t;
    ctr[3] = (uint32_t)(j / 4);
    key[0] = seed;
    key[1] = integral_id;
    oracle_philox4x32_10(ctr, key, out);
    return out[j % 4];
}

/* ------------------------------------------------------------ integrands */
static const double ORACLE_PI = 3.14159265358979323846;

int oracle_n_params(int family, int d) {
    switch (family) {
    case ORACLE_F_CONST: return 0;
    case ORACLE_F_SUM: return 0;
    case ORACLE_F_GAUSS_SYM: return 1;          /* a                         */
    case ORACLE_F_GENZ_OSC: return 1 + d;       /* u, c_1..c_d               */
    case ORACLE_F_GENZ_GAUSS: return 2 * d;     /* c_1..c_d, w_1..w_d        */
    case ORACLE_F_GENZ_PROD: return 2 * d;      /* c_1..c_d, w_1..w_d        */
    case ORACLE_F_GENZ_CORNER: return d;        /* c_1..c_d                  */
    case ORACLE_F_LO: return 7;                 /* sqrtS M Gamma cut lo hi norm */
    case ORACLE_F_LO_PDF: return 7;             /* the same; g from the grid   */
    default: return -1;
    }
}

/* Parametric parton density of the LO toy, normalised to unit integral:
 * int_0^1 x^-1/2 (1-x)^3 dx = B(1/2, 4) = 32/35. */
static double lo_density(double x) {
    double omx = 1.0 - x;
    return (35.0 / 32.0) * omx * omx * omx / sqrt(x);
}

/* LO-style 2->2 toy (d = 3): x1, x2 momentum fractions, x3 -> c = cos(theta).
 * f = g(x1) g(x2) BW(shat) (1 + c^2)/shat * 2 * norm, shat = x1 x2 S, with
 * |c| < cut and lo <= sqrt(shat) <= hi; BW = 1/((shat-M^2)^2 + M^2 Gamma^2).
 * The factor 2 is dc/dx3. */
static double lo_integrand(const double *x, const double *p) {
    double sqrtS = p[0], M = p[1], G = p[2], cut = p[3], mlo = p[4], mhi = p[5], norm = p[6];
    double shat = x[0] * x[1] * (sqrtS * sqrtS);
    double mll = sqrt(shat);
    if (!(mll >= mlo && mll <= mhi)) return 0.0;
    double c = 2.0 * x[2] - 1.0;
    if (!(fabs(c) < cut)) return 0.0;
    double M2 = M * M;
    double dm = shat - M2;
    double bw = 1.0 / (dm * dm + M2 * G * G);
    return lo_density(x[0]) * lo_density(x[1]) * bw * (1.0 + c * c) / shat * 2.0 * norm;
}

/* ---------------------------------------------------- parton-density grid */
/* A tabulated density as the paper's companion tool evaluates them (PDFFlow,
 * Sec. 2): values of x g(x, Q^2) on a uniform grid in (u, v) = (ln x, ln Q^2),
 * interpolated by cubic Hermite polynomials in each variable (the tensor
 * product, first along u at four v-knots, then along v), with the tangent at a
 * knot the central difference of its neighbours, and the one-sided difference
 * at the first and last knot.  Outside the grid, u and v are clamped to it. */
static int g_pdf_nx = 0, g_pdf_nq = 0;
static double g_pdf_u0, g_pdf_u1, g_pdf_v0, g_pdf_v1;
static const double *g_pdf_xg = 0;

void oracle_set_pdf_grid(int nx, int nq, double u0, double u1, double v0, double v1, const double *xg) {
    g_pdf_nx = nx;
    g_pdf_nq = nq;
    g_pdf_u0 = u0;
    g_pdf_u1 = u1;
    g_pdf_v0 = v0;
    g_pdf_v1 = v1;
    g_pdf_xg = xg;
}

/* Cubic Hermite basis on [0, 1]: value at t of the cubic with values y0, y1
 * and slopes m0, m1 (per unit t) at t = 0, 1. */
static double hermite(double t, double y0, double y1, double m0, double m1) {
    double t2 = t * t, t3 = t2 * t;
    return (2.0 * t3 - 3.0 * t2 + 1.0) * y0 + (t3 - 2.0 * t2 + t) * m0 + (-2.0 * t3 + 3.0 * t2) * y1 +
           (t3 - t2) * m1;
}

/* Slope per knot spacing at knot k of the samples y[0..n-1] (stride s). */
static double knot_slope(const double *y, int n, int s, int k) {
    if (k == 0) return y[s] - y[0];
    if (k == n - 1) return y[(n - 1) * s] - y[(n - 2) * s];
    return (y[(k + 1) * s] - y[(k - 1) * s]) / 2.0;
}

/* Cell index and position in the cell of coordinate w on n uniform knots
 * from w0 to w1 (w clamped to the grid). */
static void locate(double w, double w0, double w1, int n, int *k, double *t) {
    double h = (w1 - w0) / (double)(n - 1);
    double r = (w - w0) / h;
    if (r < 0.0) r = 0.0;
    if (r > (double)(n - 1)) r = (double)(n - 1);
    int i = (int)floor(r);
    if (i > n - 2) i = n - 2;
    *k = i;
    *t = r - (double)i;
}

/* Interpolation along u of row... the value at (u-cell iu, position tu) of
 * the column j of the table. */
static double along_u(int iu, double tu, int j) {
    const double *col = g_pdf_xg + j;
    int s = g_pdf_nq;
    return hermite(tu, col[iu * s], col[(iu + 1) * s], knot_slope(col, g_pdf_nx, s, iu),
                   knot_slope(col, g_pdf_nx, s, iu + 1));
}

double oracle_pdf_xg(double x, double q2) {
    if (!g_pdf_xg || g_pdf_nx < 2 || g_pdf_nq < 2) return 0.0;
    int iu, iv;
    double tu, tv;
    locate(log(x), g_pdf_u0, g_pdf_u1, g_pdf_nx, &iu, &tu);
    locate(log(q2), g_pdf_v0, g_pdf_v1, g_pdf_nq, &iv, &tv);
    /* the u-interpolants at the v-knots iv-1 .. iv+2 that exist */
    double w[4];
    int jlo = iv - 1 < 0 ? 0 : iv - 1;
    int jhi = iv + 2 > g_pdf_nq - 1 ? g_pdf_nq - 1 : iv + 2;
    for (int j = jlo; j <= jhi; ++j) w[j - (iv - 1)] = along_u(iu, tu, j);
    /* slopes along v at knots iv and iv+1, from those values */
    double m0 = iv == 0 ? w[2] - w[1] : (w[2] - w[0]) / 2.0;
    double m1 = iv + 1 == g_pdf_nq - 1 ? w[2] - w[1] : (w[3] - w[1]) / 2.0;
    return hermite(tv, w[1], w[2], m0, m1);
}

/* LO toy with the density from the grid at the factorisation scale Q^2 = shat:
 * f = g(x1, shat) g(x2, shat) BW(shat) (1 + c^2)/shat * 2 * norm with the same
 * cuts as lo_integrand, g = (x g)/x. */
static double lo_pdf_integrand(const double *x, const double *p) {
    double sqrtS = p[0], M = p[1], G = p[2], cut = p[3], mlo = p[4], mhi = p[5], norm = p[6];
    double shat = x[0] * x[1] * (sqrtS * sqrtS);
    double mll = sqrt(shat);
    if (!(mll >= mlo && mll <= mhi)) return 0.0;
    double c = 2.0 * x[2] - 1.0;
    if (!(fabs(c) < cut)) return 0.0;
    double M2 = M * M;
    double dm = shat - M2;
    double bw = 1.0 / (dm * dm + M2 * G * G);
    double g1 = oracle_pdf_xg(x[0], shat) / x[0];
    double g2 = oracle_pdf_xg(x[1], shat) / x[1];
    return g1 * g2 * bw * (1.0 + c * c) / shat * 2.0 * norm;
}

static oracle_user_fn g_user_fn = 0;

void oracle_set_user(oracle_user_fn f) { g_user_fn = f; }

double oracle_integrand(int family, int d, const double *p, int n_params, const double *x) {
    (void)n_params;
    switch (family) {
    case ORACLE_F_USER:
        return g_user_fn ? g_user_fn(x, d, p) : 0.0;
    case ORACLE_F_LO_PDF:
        return lo_pdf_integrand(x, p);
    case ORACLE_F_CONST:
        return 1.0;
    case ORACLE_F_SUM: {
        double s = 0.0;
        for (int i = 0; i < d; ++i) s += x[i];
        return s;
    }
    case ORACLE_F_GAUSS_SYM: {
        double a = p[0];
        double q = 0.0;
        for (int i = 0; i < d; ++i) q += (x[i] - 0.5) * (x[i] - 0.5);
        return pow(a * sqrt(ORACLE_PI), -(double)d) * exp(-q / (a * a));
    }
    case ORACLE_F_GENZ_OSC: {
        double arg = 2.0 * ORACLE_PI * p[0];
        for (int i = 0; i < d; ++i) arg += p[1 + i] * x[i];
        return cos(arg);
    }
    case ORACLE_F_GENZ_GAUSS: {
        double q = 0.0;
        for (int i = 0; i < d; ++i) {
            double c = p[i], w = p[d + i];
            q += c * c * (x[i] - w) * (x[i] - w);
        }
        return exp(-q);
    }
    case ORACLE_F_GENZ_PROD: {
        double r = 1.0;
        for (int i = 0; i < d; ++i) {
            double c = p[i], w = p[d + i];
            r *= 1.0 / (1.0 / (c * c) + (x[i] - w) * (x[i] - w));
        }
        return r;
    }
    case ORACLE_F_GENZ_CORNER: {
        double s = 1.0;
        for (int i = 0; i < d; ++i) s += p[i] * x[i];
        return pow(s, -(double)(d + 1));
    }
    case ORACLE_F_LO:
        return lo_integrand(x, p);
    default:
        return 0.0;
    }
}

/* ------------------------------------------------------------- sampling */
#define ORACLE_MAXD 64

void oracle_sample(int d, int N, const double *edges, int family, const double *params,
                   int n_params, uint32_t seed, uint32_t integral_id, uint32_t t,
                   uint64_t s, int32_t *bins, double *x, double *J, double *f) {
    double jac = 1.0;
    for (int j = 0; j < d; ++j) {
        uint32_t r = oracle_draw(s, t, j, seed, integral_id);
        /* y N = r N / 2^32: the bin is the integer part, the fraction the rest */
        uint64_t prod = (uint64_t)r * (uint64_t)N;
        int32_t i = (int32_t)(prod >> 32);
        double frac = (double)(uint32_t)(prod & 0xFFFFFFFFu) * (1.0 / 4294967296.0);
        const double *e = edges + (size_t)j * (size_t)(N + 1);
        double delta = e[i + 1] - e[i];
        bins[j] = i;
        x[j] = e[i] + delta * frac;
        jac *= (double)N * delta;
    }
    *J = jac;
    *f = oracle_integrand(family, d, params, n_params, x);
}


void oracle_trace(int d, int N, const double *edges, int family, const double *params,
                  int n_params, uint32_t seed, uint32_t integral_id, uint32_t t,
                  uint64_t s_begin, int64_t count, int32_t *bins, double *x, double *v) {
    for (int64_t k = 0; k < count; ++k) {
        double J, f;
        oracle_sample(d, N, edges, family, params, n_params, seed, integral_id, t, s_begin + (uint64_t)k,
                      bins + (size_t)k * (size_t)d, x + (size_t)k * (size_t)d, &J, &f);
        v[k] = J * f;
    }
}

void oracle_iterate(int d, int N, const double *edges, int family, const double *params,
                    int n_params, uint32_t seed, uint32_t integral_id, uint32_t t,
                    int64_t s_begin, int64_t s_end, double *S1, double *S2, double *hist,
                    int64_t *cnt, int64_t *n_nonfinite) {
    int32_t bins[ORACLE_MAXD];
    double x[ORACLE_MAXD];
    if (d < 1 || d > ORACLE_MAXD) return;
    for (int64_t s = s_begin; s < s_end; ++s) {
        double J, f;
        oracle_sample(d, N, edges, family, params, n_params, seed, integral_id, t, (uint64_t)s,
                      bins, x, &J, &f);
        double v = J * f;
        if (!isfinite(v)) {
            if (n_nonfinite) *n_nonfinite += 1;
            continue;
        }
        double v2 = v * v;
        *S1 += v;
        *S2 += v2;
        for (int j = 0; j < d; ++j) {
            hist[(size_t)j * (size_t)N + (size_t)bins[j]] += v2;
            if (cnt) cnt[(size_t)j * (size_t)N + (size_t)bins[j]] += 1;
        }
    }
}

void oracle_iteration_result(double S1, double S2, int64_t n, double *I, double *var) {
    double mean = S1 / (double)n;
    double v = (S2 / (double)n - mean * mean) / (double)(n - 1);
    *I = mean;
    *var = v > 0.0 ? v : 0.0;
}

/* ----------------------------------------------------------- refinement */
#define ORACLE_MAXN 4096

static void refine_one(int N, const double *h, const double *e, double alpha, int smooth,
                       double *out) {
    double dsm[ORACLE_MAXN], rho[ORACLE_MAXN];
    /* smoothing: 3-point average inside, 2-point average at the ends */
    for (int k = 0; k < N; ++k) {
        if (!smooth || N < 2) {
            dsm[k] = h[k];
        } else if (k == 0) {
            dsm[k] = (h[0] + h[1]) / 2.0;
        } else if (k == N - 1) {
            dsm[k] = (h[N - 2] + h[N - 1]) / 2.0;
        } else {
            dsm[k] = (h[k - 1] + h[k] + h[k + 1]) / 3.0;
        }
    }
    double total = 0.0;
    for (int k = 0; k < N; ++k) total += dsm[k];
    if (!(total > 0.0) || !isfinite(total)) {
        for (int k = 0; k <= N; ++k) out[k] = e[k];
        return;
    }
    /* normalise and compress */
    double rsum = 0.0;
    for (int k = 0; k < N; ++k) {
        double dk = dsm[k] / total;
        double r;
        if (dk <= 0.0) r = 0.0;
        else if (dk >= 1.0) r = 1.0;
        else r = pow((1.0 - dk) / log(1.0 / dk), alpha);
        rho[k] = r;
        rsum += r;
    }
    if (!(rsum > 0.0)) {
        for (int k = 0; k <= N; ++k) out[k] = e[k];
        return;
    }
    /* rebin: the k-th new edge sits where the running rho sum reaches
     * k * delta, interpolated linearly inside the old bin */
    double delta = rsum / (double)N;
    out[0] = 0.0;
    out[N] = 1.0;
    int b = 0;
    double acc = 0.0; /* sum of rho over old bins before b */
    for (int k = 1; k < N; ++k) {
        double target = (double)k * delta;
        while (b < N - 1 && !(acc + rho[b] >= target)) {
            acc += rho[b];
            ++b;
        }
        double width = e[b + 1] - e[b];
        double frac = rho[b] > 0.0 ? (target - acc) / rho[b] : 1.0;
        if (frac < 0.0) frac = 0.0;
        if (frac > 1.0) frac = 1.0;
        out[k] = e[b] + frac * width;
    }
}

void oracle_refine(int d, int N, const double *hist, const double *edges_in, double alpha,
                   int smooth, double *edges_out) {
    if (N < 1 || N > ORACLE_MAXN) return;
    for (int j = 0; j < d; ++j) {
        refine_one(N, hist + (size_t)j * (size_t)N, edges_in + (size_t)j * (size_t)(N + 1),
                   alpha, smooth, edges_out + (size_t)j * (size_t)(N + 1));
    }
}

/* ----------------------------------------------------------- combination */
void oracle_combine(int m, const double *I, const double *sigma, double *Ibar, double *sbar,
                    double *chi2_dof) {
    *Ibar = 0.0;
    *sbar = 0.0;
    *chi2_dof = 0.0;
    if (m <= 0) return;
    /* iterations with zero variance are exact: their plain mean is the result */
    int nzero = 0;
    double zsum = 0.0;
    for (int j = 0; j < m; ++j) {
        if (sigma[j] == 0.0) {
            ++nzero;
            zsum += I[j];
        }
    }
    if (nzero > 0) {
        *Ibar = zsum / (double)nzero;
        *sbar = 0.0;
        *chi2_dof = 0.0;
        return;
    }
    double wsum = 0.0, wisum = 0.0;
    for (int j = 0; j < m; ++j) {
        double w = 1.0 / (sigma[j] * sigma[j]);
        wsum += w;
        wisum += w * I[j];
    }
    double mean = wisum / wsum;
    double chi2 = 0.0;
    for (int j = 0; j < m; ++j) {
        double r = (I[j] - mean) / sigma[j];
        chi2 += r * r;
    }
    *Ibar = mean;
    *sbar = 1.0 / sqrt(wsum);
    *chi2_dof = m > 1 ? chi2 / (double)(m - 1) : 0.0;
}

/* ------------------------------------------- stratified + importance hybrid */
/* Lepage 1980 combines the importance map with stratified sampling: y-space is
 * cut into equal hypercubes and every hypercube receives the same number P of
 * samples; the estimate is the mean of the hypercube means and its variance
 * the sum of the hypercube variances of the mean.  Readings (the paper and
 * Lepage leave the counts to the implementation):
 *   - 2^B hypercubes; dimension j is cut into M_j = 2^b_j strata with
 *     b_j = floor(B/d) + (j < B mod d ? 1 : 0);
 *   - hypercube h's stratum in dimension j is k_j = floor(h / prod_{i<j} M_i) mod M_j;
 *   - sample s belongs to hypercube floor(s / P); its uniform word r_j (the
 *     same Philox counter as in plain sampling) is placed in the stratum as
 *     y_j = (k_j + r_j 2^-32) / M_j, kept on the 2^-32 lattice by flooring:
 *     R_j = floor((k_j 2^32 + r_j) / M_j), y_j = R_j 2^-32;
 *   - the importance map then treats R_j exactly as plain sampling treats r_j;
 *   - the histograms take (J f)^2 per sample, as in plain sampling;
 *   - a non-finite J f counts as 0 (and is counted), so every hypercube keeps
 *     its P samples. */
void oracle_strata_bits(int d, int B, int32_t *bits) {
    for (int j = 0; j < d; ++j) bits[j] = B / d + (j < B % d ? 1 : 0);
}

static uint32_t strat_word(uint32_t r, uint64_t h, int d, int B, int j) {
    /* k_j: digit j of h in the mixed radix (M_0, M_1, ...) */
    uint64_t below = 1;
    for (int i = 0; i < j; ++i) below *= (uint64_t)1 << (B / d + (i < B % d ? 1 : 0));
    uint64_t Mj = (uint64_t)1 << (B / d + (j < B % d ? 1 : 0));
    uint64_t k = (h / below) % Mj;
    return (uint32_t)((k * 4294967296ull + (uint64_t)r) / Mj);
}

void oracle_sample_strat(int d, int N, const double *edges, int family, const double *params,
                         int n_params, uint32_t seed, uint32_t integral_id, uint32_t t, int B,
                         int64_t P, uint64_t s, int32_t *bins, double *x, double *J, double *f) {
    double jac = 1.0;
    uint64_t h = s / (uint64_t)P;
    for (int j = 0; j < d; ++j) {
        uint32_t r = strat_word(oracle_draw(s, t, j, seed, integral_id), h, d, B, j);
        uint64_t prod = (uint64_t)r * (uint64_t)N;
        int32_t i = (int32_t)(prod >> 32);
        double frac = (double)(uint32_t)(prod & 0xFFFFFFFFu) * (1.0 / 4294967296.0);
        const double *e = edges + (size_t)j * (size_t)(N + 1);
        double delta = e[i + 1] - e[i];
        bins[j] = i;
        x[j] = e[i] + delta * frac;
        jac *= (double)N * delta;
    }
    *J = jac;
    *f = oracle_integrand(family, d, params, n_params, x);
}

/* Hypercubes h in [h_begin, h_end) of iteration t, P samples each:
 * *S1 += v, *S2 += v^2, hist as in plain sampling, and
 * *Q += sum over the hypercube of (v - mean_h)^2 (two passes: the mean first).
 * vbuf: scratch of P doubles. */
void oracle_iterate_strat(int d, int N, const double *edges, int family, const double *params,
                          int n_params, uint32_t seed, uint32_t integral_id, uint32_t t, int B,
                          int64_t P, int64_t h_begin, int64_t h_end, double *vbuf, double *S1,
                          double *S2, double *Q, double *hist, int64_t *n_nonfinite) {
    int32_t bins[ORACLE_MAXD];
    double x[ORACLE_MAXD];
    if (d < 1 || d > ORACLE_MAXD || P < 1) return;
    for (int64_t h = h_begin; h < h_end; ++h) {
        double sum = 0.0;
        for (int64_t p = 0; p < P; ++p) {
            double J, f;
            oracle_sample_strat(d, N, edges, family, params, n_params, seed, integral_id, t, B,
                                P, (uint64_t)(h * P + p), bins, x, &J, &f);
            double v = J * f;
            if (!isfinite(v)) {
                if (n_nonfinite) *n_nonfinite += 1;
                v = 0.0;
            }
            double v2 = v * v;
            vbuf[p] = v;
            sum += v;
            *S1 += v;
            *S2 += v2;
            for (int j = 0; j < d; ++j) hist[(size_t)j * (size_t)N + (size_t)bins[j]] += v2;
        }
        double mean = sum / (double)P;
        double m2 = 0.0;
        for (int64_t p = 0; p < P; ++p) m2 += (vbuf[p] - mean) * (vbuf[p] - mean);
        *Q += m2;
    }
}

/* Estimate of a stratified iteration over H hypercubes of P samples:
 * I = S1 / (H P) (the mean of the hypercube means) and
 * var = sum_h s_h^2 / (H^2 P) with s_h^2 = m2_h / (P - 1), i.e. Q / (H^2 P (P - 1)). */
void oracle_strat_result(double S1, double Q, int64_t H, int64_t P, double *I, double *var) {
    double Hd = (double)H, Pd = (double)P;
    *I = S1 / (Hd * Pd);
    *var = P > 1 ? Q / (Hd * Hd * Pd * (Pd - 1.0)) : 0.0;
}

/* ------------------------------------------------ observable histograms */
/* The paper's generator chain ends in histogramming (Fig. 1): the samples'
 * weights v = J f binned in an observable.  Observables: a coordinate x_k
 * (obs = k >= 0), or for the LO toys sqrt(shat) in GeV (obs = -1) and
 * cos(theta) = 2 x_3 - 1 (obs = -2).  Bin b in 1..nb holds the samples with
 * lo + (b-1) w <= o < lo + b w, w = (hi - lo)/nb; bin 0 those below lo and bin
 * nb + 1 those at or above hi.  out[b] += v, out[nb + 2 + b] += v^2; samples
 * with a non-finite v are left out (a stratified iteration counts them as 0,
 * which adds nothing). */
static double observable(int obs, const double *x, const double *params) {
    if (obs >= 0) return x[obs];
    if (obs == -1) return sqrt(x[0] * x[1]) * params[0];
    return 2.0 * x[2] - 1.0;
}

void oracle_histogram(int d, int N, const double *edges, int family, const double *params,
                      int n_params, uint32_t seed, uint32_t integral_id, uint32_t t, int B, int64_t P,
                      int64_t s_begin, int64_t s_end, int obs, int nb, double lo, double hi,
                      double *out) {
    int32_t bins[ORACLE_MAXD];
    double x[ORACLE_MAXD];
    double w = (hi - lo) / (double)nb;
    for (int64_t s = s_begin; s < s_end; ++s) {
        double J, f;
        if (P > 0)
            oracle_sample_strat(d, N, edges, family, params, n_params, seed, integral_id, t, B, P,
                                (uint64_t)s, bins, x, &J, &f);
        else
            oracle_sample(d, N, edges, family, params, n_params, seed, integral_id, t, (uint64_t)s,
                          bins, x, &J, &f);
        double v = J * f;
        if (!isfinite(v)) continue;
        double o = observable(obs, x, params);
        int b;
        if (o < lo) b = 0;
        else if (o >= hi) b = nb + 1;
        else {
            b = 1 + (int)floor((o - lo) / w);
            if (b > nb) b = nb;
        }
        out[b] += v;
        out[nb + 2 + b] += v * v;
    }
}
