// vegas_kernels.cuh -- declarations shared by the kernel translation units and
// the C-ABI host code of the VEGAS library.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "vegas_sample.cuh"
#include "vegas_trace.cuh"

namespace vegas {

// One record per iteration, written on the device by the finalize kernel.
struct IterRec {
    double I;
    double sigma;
    long long n;            // samples with finite weight
    long long n_nonfinite;
};

// Running sums of the combination (finalize kernels), taken about I0, the
// estimate of the first combined iteration with a nonzero variance.
struct CombState {
    double wsum;    // sum of w = 1/sigma^2
    double wdsum;   // sum of w (I - I0)
    double wd2sum;  // sum of w (I - I0)^2
    double zsum;    // sum of the zero-variance iterations' estimates
    double i0;
    int m;          // iterations combined (those with at least one finite value)
    int nzero;      // of which with zero variance
    int n_done;     // all iterations finalized
    int have_i0;
};

// Iteration records are kept in a ring of this many entries.
constexpr int kIterRing = 4096;

// Running combination over all iterations so far (finalize kernel).
struct CombRec {
    double I;
    double sigma;
    double chi2_dof;
    int n_iter;
    int status;             // 0 ok, 6 = every weight of the last iteration non-finite
};

// Inverse-variance combination of the iterations (Lepage; weights 1/sigma^2
// of every iteration with a finite value, no warm-up discard), kept as
// running sums about I0 so that chi^2 does not cancel when the iterations
// agree to many digits (a one-pass sum w I^2 - Ibar sum w I loses all of
// chi^2 once (Ibar/sigma)^2 nears 1/eps):
//   Ibar = I0 + sum w (I - I0) / sum w,  sigma = (sum w)^-1/2,
//   chi^2/dof = (sum w (I - I0)^2 - (sum w (I - I0))^2 / sum w) / (m - 1).
// Iterations with zero variance are exact: if any, their plain mean is the
// result, with sigma 0.  `combined`: false for an iteration without a finite
// value, which has no estimate and is left out.
__host__ __device__ inline void comb_add(CombState &st, double I, double sigma, bool combined) {
    st.n_done += 1;
    if (!combined) return;
    st.m += 1;
    if (sigma == 0.0) {
        st.nzero += 1;
        st.zsum += I;
        return;
    }
    if (!st.have_i0) {
        st.i0 = I;
        st.have_i0 = 1;
    }
    const double w = 1.0 / (sigma * sigma);
    const double dI = I - st.i0;
    st.wsum += w;
    st.wdsum += w * dI;
    st.wd2sum += w * dI * dI;
}

__host__ __device__ inline CombRec comb_result(const CombState &st, bool last_combined) {
    CombRec out;
    out.n_iter = st.n_done;
    out.status = last_combined ? 0 : 6;
    if (st.nzero > 0) {
        out.I = st.zsum / st.nzero;
        out.sigma = 0.0;
        out.chi2_dof = 0.0;
    } else if (st.wsum > 0.0) {
        const double mean_d = st.wdsum / st.wsum;
        out.I = st.i0 + mean_d;
        out.sigma = 1.0 / sqrt(st.wsum);
        const double chi = st.wd2sum - mean_d * st.wdsum;
        out.chi2_dof = st.m > 1 ? fmax(chi, 0.0) / static_cast<double>(st.m - 1) : 0.0;
    } else {
        out.I = 0.0;
        out.sigma = 0.0;
        out.chi2_dof = 0.0;
    }
    return out;
}

// Sampling kernel for (accumulation mode, family, dimension, lane-private
// layout); nullptr if the combination does not exist.
const void *sample_kernel(int mode, int fam, int d, bool priv);
// Stratified sampling kernel for the same arguments (vegas_sample_strat_kernel).
const void *sample_strat_kernel(int mode, int fam, int d, bool priv);
// FP64 sampling kernel with one histogram copy per lane (layout kLayoutWide);
// nullptr where there is none.
const void *sample_kernel_wide(int mode, int fam, int d);

inline int tier_of(int d) { return d <= 4 ? 0 : (d <= 8 ? 1 : (d <= 16 ? 2 : 3)); }

// Shared memory of one sampling block in layout 0 (one copy per cell), 1
// (lane-private copies), 2 (half as many copies) or kLayoutWide (FP64: one
// histogram copy per lane).
size_t sample_smem(int mode, int layout, int d, int N);

// FP32 modes: samples one block may add to its fixed-point histogram cells
// between flushes (layout as above).
long long block_samples_max(int mode, int layout, int N);

// Finalize: move the accumulators (unscaled) to `last`, zero them, form
// I_t and sigma_t, store the record, update the combination and the scales
// of the next iteration (fixed-point histogram scale, v-rescale).
struct FinalizeArgs {
    double *acc, *last;
    unsigned long long *n_nonfinite;
    float *hscale;
    double *jmul2;        // two slots, selected by record parity
    IterRec *iters;
    CombState *cs;
    CombRec *comb;
    int rec;              // record index of this iteration
    int total;            // 2 + d N
    long long n;          // samples of the iteration
    double inv_scale0, jinit0;
    // stratified iterations (strat_P > 0): strat_H hypercubes of strat_P
    // samples; q[0] accumulates sum_h m2_h (scaled like S2), q[1] keeps the
    // last iteration's, unscaled
    long long strat_H, strat_P;
    double *q;
};
cudaError_t launch_finalize(const FinalizeArgs &f, cudaStream_t stream);
// Finalize and refinement of one integral's iteration: its FP64 edges and
// sampling table (of `mode`), d dimensions of N bins, damping alpha.
struct RefineJob {
    FinalizeArgs f;
    double *edges;
    void *table;
    const double *center;   // d table centres (table_center)
    int mode, d, N, smooth;
    double alpha;
};
constexpr int kMaxRefineJobs = 8;
struct RefineJobs {
    RefineJob job[kMaxRefineJobs];
    int n;
};
// Finalize and refinement of n <= kMaxRefineJobs integrals in one launch
// (vegas_step, vegas_step_many).
cudaError_t launch_finalize_refine(const RefineJob *jobs, int n, cudaStream_t stream);
// A launch with programmatic stream serialisation (the kernel calls
// pdl_begin before it reads anything an earlier launch wrote).
cudaError_t launch_programmatic(const void *fn, dim3 grid, dim3 block, void **params, size_t smem,
                                cudaStream_t stream);

// Refine every dimension from the histograms in last[2..] and write the new
// FP64 edges and the sampling table of the given mode (about the d centres).
cudaError_t launch_refine(const double *last, double *edges, void *table, const double *center, int mode,
                          int d, int N, double alpha, int smooth, cudaStream_t stream);

// Build the sampling table of `mode` from FP64 edges, about the d centres
// (device array, table_center).
cudaError_t launch_table_from_edges(const double *edges, void *table, const double *center, int mode, int d,
                                    int N, cudaStream_t stream);

// The d table centres of a family (table_center), by value.
struct TableCenters {
    double c[32];
};
// Write the family's d table centres to the device array dst (no host copy).
cudaError_t launch_set_centers(double *dst, int family, int d, const FamConsts<double> &fc, cudaStream_t stream);

// Per-sample trace on the given table (same device arithmetic as sampling).
cudaError_t launch_trace(const SampleArgs &a, int fam, int mode, double inv_scale, int32_t *bins,
                         double *x, double *w, cudaStream_t stream);

// The same with the trace kernel given (a run-time compiled user integrand's);
// with hist, the samples' weights are also binned in an observable (HistArgs).
cudaError_t launch_trace_fn(const void *fn, const SampleArgs &a, double inv_scale, int32_t *bins,
                            double *x, double *w, const HistArgs *hist, cudaStream_t stream);
// The built-in trace kernel of (family, mode, d); null if none.
const void *trace_kernel_for(int fam, int mode, int d);

// Largest density grid of the F_LO_PDF family, counted with its padding,
// (nx + 2)(nq + 2) values: 48 KB of FP64.
constexpr int kMaxPdfValues = 6144;

// Kernels of a user integrand compiled at run time (vegas_jit.cu): sampling,
// stratified sampling and trace for one (mode, d, layout).
struct JitKernels {
    const void *sample = nullptr;
    const void *strat = nullptr;
    const void *trace = nullptr;
};
// 0: compiled (or found in the cache); 1: the run-time compiler could not be
// loaded; 2: the source did not compile (log holds the compiler's messages);
// 3: a CUDA call failed (log holds its message).
int jit_user_kernels(const char *source, int mode, int d, bool priv, JitKernels *out, const char **log);
// The compiler's messages of this thread's last run-time compilation.
const char *jit_last_log();

cudaError_t launch_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, long long n,
                          cudaStream_t stream);

}  // namespace vegas
