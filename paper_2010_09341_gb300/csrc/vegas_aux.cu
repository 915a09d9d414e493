// vegas_aux.cu -- the small kernels around the sampling kernel: iteration
// result and combination, grid refinement, table building, per-sample trace
// and a bare Philox kernel.
//
// All of them are FP64: the refinement and the combination of iterations need
// it (a rebinned edge is a difference of running sums; chi^2 is a sum of
// squared deviations), and they touch O(d N) values, so their cost is
// launch latency, not arithmetic.
#include <algorithm>
#include <cstring>

#include "vegas_kernels.cuh"
#include "vegas_refine.cuh"
#include "vegas_trace.cuh"

namespace vegas {

// ------------------------------------------------------------- finalize
// Iteration estimate (Lepage 1978): I = S1/n, sigma^2 = (S2/n - I^2)/(n-1).
// Iteration result (Lepage): I = S1/n, sigma^2 = (S2/n - I^2)/(n - 1) over
// the n samples with a finite value (stratified: every sample, a non-finite
// value counted as 0), then the running combination (comb_add).  An
// iteration without a finite value has no estimate: status 6, left out.
//
// The v-rescale is double-buffered by record parity: iteration `rec` was
// sampled with jmul[rec & 1] and the next one uses jmul[(rec + 1) & 1], so
// blocks that still read the current value never race with the update.
__device__ void finalize_stats(const FinalizeArgs &f) {
    // thread 0 only: S1, S2, the counters, the scales and the combination
    const double jm = f.jmul2[f.rec & 1];
    const double inv1 = f.inv_scale0 / jm;
    const long long nf = static_cast<long long>(*f.n_nonfinite);
    *f.n_nonfinite = 0ull;
    // stratified: a non-finite value counts as 0, so every sample stays in n
    const bool strat = f.strat_P > 0;
    const long long ne = strat ? f.n : f.n - nf;
    const double S1 = f.acc[0] * inv1, S2 = f.acc[1] * inv1 * inv1;
    const double m2 = ne > 0 ? f.acc[1] / static_cast<double>(ne) : 0.0;
    const double m1 = ne > 0 ? f.acc[0] / static_cast<double>(ne) : 0.0;
    f.last[0] = S1;
    f.last[1] = S2;
    f.acc[0] = 0.0;
    f.acc[1] = 0.0;
    double ratio;
    float hs;
    next_scales(m2, m1, f.jinit0 * jm, &ratio, &hs);
    *f.hscale = hs;
    f.jmul2[(f.rec + 1) & 1] = jm * ratio;
    IterRec r;
    r.n = ne;
    r.n_nonfinite = nf;
    if (strat) {
        // Lepage 1980's combined mode: the mean of the hypercube means and the
        // sum of their variances of the mean, var = Q / (H^2 P (P - 1))
        const double Q = f.q[0] * inv1 * inv1;
        f.q[1] = Q;
        f.q[0] = 0.0;
        const double H = static_cast<double>(f.strat_H), P = static_cast<double>(f.strat_P);
        r.I = S1 / (H * P);
        const double var = f.strat_P > 1 ? Q / (H * H * P * (P - 1.0)) : 0.0;
        r.sigma = var > 0.0 ? sqrt(var) : 0.0;
    } else if (ne >= 2) {
        const double rn = 1.0 / static_cast<double>(ne);
        const double I = S1 * rn;
        const double var = (S2 * rn - I * I) / static_cast<double>(ne - 1);
        r.I = I;
        r.sigma = var > 0.0 ? sqrt(var) : 0.0;
    } else {
        r.I = ne == 1 ? S1 : 0.0;
        r.sigma = 0.0;
    }
    f.iters[f.rec % kIterRing] = r;
    // no finite value among the f.n samples drawn: no estimate
    const bool combined = nf < f.n;
    CombState st = *f.cs;
    comb_add(st, r.I, r.sigma, combined);
    *f.cs = st;
    *f.comb = comb_result(st, combined);
}

// Histogram rows of one iteration: last = acc * inv^2, acc = 0, for the
// values [begin, end) of the accumulator row (every thread of the block).
__device__ __forceinline__ void move_rows(const FinalizeArgs &f, int begin, int end) {
    const double inv = f.inv_scale0 / f.jmul2[f.rec & 1];
    const double inv2 = inv * inv;
    for (int c = begin + threadIdx.x; c < end; c += blockDim.x) {
        f.last[c] = f.acc[c] * inv2;
        f.acc[c] = 0.0;
    }
}

__global__ void __launch_bounds__(256) finalize_kernel(const FinalizeArgs f) {
    if (threadIdx.x == 0) finalize_stats(f);
    move_rows(f, 2, f.total);
}

cudaError_t launch_finalize(const FinalizeArgs &f, cudaStream_t stream) {
    finalize_kernel<<<1, 256, 0, stream>>>(f);
    return cudaGetLastError();
}

// --------------------------------------------------------------- refine
__global__ void __launch_bounds__(kRefineThreads)
refine_kernel(const double *last, double *edges, void *table, const double *center, int mode, int N,
              double alpha, int smooth) {
    extern __shared__ double rs[];
    const int j = blockIdx.x;
    const size_t entry = mode == ACC_F64 ? sizeof(double2) : sizeof(float2);
    refine_block(last + 2 + static_cast<size_t>(j) * N, edges + static_cast<size_t>(j) * (N + 1),
                 static_cast<char *>(table) + entry * static_cast<size_t>(j) * N, mode, N, alpha,
                 smooth, center[j], rs);
}

// Finalize and refinement of one iteration of each of js.n integrals in one
// launch (d_k + 1 blocks for integral k, in order): block j < d_k refines
// dimension j of integral k from its accumulator row (refinement only
// normalises the histogram, so the row's scale does not matter) and then
// moves the row to `last`; block d_k forms integral k's iteration result.
__global__ void __launch_bounds__(kRefineThreads) finalize_refine_kernel(const RefineJobs js) {
    extern __shared__ double rs[];
    pdl_begin();
    int j = blockIdx.x, k = 0;
    while (k + 1 < js.n && j > js.job[k].d) {
        j -= js.job[k].d + 1;
        ++k;
    }
    const RefineJob &r = js.job[k];
    if (j == r.d) {
        if (threadIdx.x == 0) finalize_stats(r.f);
        return;
    }
    const int N = r.N;
    const size_t entry = r.mode == ACC_F64 ? sizeof(double2) : sizeof(float2);
    refine_block(r.f.acc + 2 + static_cast<size_t>(j) * N, r.edges + static_cast<size_t>(j) * (N + 1),
                 static_cast<char *>(r.table) + entry * static_cast<size_t>(j) * N, r.mode, N, r.alpha,
                 r.smooth, r.center[j], rs);
    __syncthreads();
    move_rows(r.f, 2 + j * N, 2 + (j + 1) * N);
}

cudaError_t launch_finalize_refine(const RefineJob *jobs, int n, cudaStream_t stream) {
    if (n < 1 || n > kMaxRefineJobs) return cudaErrorInvalidValue;
    RefineJobs js;
    js.n = n;
    int blocks = 0, maxN = 0;
    for (int k = 0; k < n; ++k) {
        js.job[k] = jobs[k];
        blocks += jobs[k].d + 1;
        maxN = std::max(maxN, jobs[k].N);
    }
    const size_t smem = static_cast<size_t>(4 * maxN + 2) * sizeof(double);
    // An ordinary launch: its few FP64-bound blocks then start on idle SMs,
    // one per SM.  Launched early (programmatic), they would take the first
    // SMs that the sampling kernel's tail frees, several to an SM, and share
    // its FP64 units.  Its pdl_begin still lets the next sampling launch start
    // early.
    finalize_refine_kernel<<<blocks, kRefineThreads, smem, stream>>>(js);
    return cudaGetLastError();
}

cudaError_t launch_programmatic(const void *fn, dim3 grid, dim3 block, void **params, size_t smem,
                                cudaStream_t stream) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, params);
}

cudaError_t launch_refine(const double *last, double *edges, void *table, const double *center, int mode,
                          int d, int N, double alpha, int smooth, cudaStream_t stream) {
    const size_t smem = static_cast<size_t>(4 * N + 2) * sizeof(double);
    refine_kernel<<<d, kRefineThreads, smem, stream>>>(last, edges, table, center, mode, N, alpha, smooth);
    return cudaGetLastError();
}

__global__ void table_kernel(const double *edges, void *table, const double *center, int mode, int d, int N) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= d * N) return;
    const int j = idx / N, k = idx - j * N;
    const double *e = edges + static_cast<size_t>(j) * (N + 1);
    store_table(table, mode, idx, e[k], e[k + 1] - e[k], center[j]);
}

cudaError_t launch_table_from_edges(const double *edges, void *table, const double *center, int mode, int d,
                                    int N, cudaStream_t stream) {
    const int total = d * N;
    table_kernel<<<(total + 255) / 256, 256, 0, stream>>>(edges, table, center, mode, d, N);
    return cudaGetLastError();
}

__global__ void centers_kernel(double *dst, int d, const TableCenters c) {
    const int j = threadIdx.x;
    if (j < d) dst[j] = c.c[j];
}

cudaError_t launch_set_centers(double *dst, int family, int d, const FamConsts<double> &fc, cudaStream_t stream) {
    TableCenters c;
    for (int j = 0; j < 32; ++j) c.c[j] = j < d ? table_center(family, fc, j) : 0.0;
    centers_kernel<<<1, 32, 0, stream>>>(dst, d, c);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- trace
// trace_kernel: vegas_trace.cuh
template <int MODE, int FAM>
static const void *trace_pick(int tier) {
    switch (tier) {
    case 0: return reinterpret_cast<const void *>(&trace_kernel<FAM, MODE, 4>);
    case 1: return reinterpret_cast<const void *>(&trace_kernel<FAM, MODE, 8>);
    case 2: return reinterpret_cast<const void *>(&trace_kernel<FAM, MODE, 16>);
    default: return reinterpret_cast<const void *>(&trace_kernel<FAM, MODE, 32>);
    }
}

template <int MODE>
static const void *trace_pick_fam(int fam, int tier) {
    switch (fam) {
    case F_CONST: return trace_pick<MODE, F_CONST>(tier);
    case F_SUM: return trace_pick<MODE, F_SUM>(tier);
    case F_GAUSS_SYM: return trace_pick<MODE, F_GAUSS_SYM>(tier);
    case F_GENZ_OSC: return trace_pick<MODE, F_GENZ_OSC>(tier);
    case F_GENZ_GAUSS: return trace_pick<MODE, F_GENZ_GAUSS>(tier);
    case F_GENZ_PROD: return trace_pick<MODE, F_GENZ_PROD>(tier);
    case F_GENZ_CORNER: return trace_pick<MODE, F_GENZ_CORNER>(tier);
    case F_LO: return tier == 0 ? reinterpret_cast<const void *>(&trace_kernel<F_LO, MODE, 4>) : nullptr;
    case F_LO_PDF: return tier == 0 ? reinterpret_cast<const void *>(&trace_kernel<F_LO_PDF, MODE, 4>) : nullptr;
    default: return nullptr;
    }
}

cudaError_t launch_trace(const SampleArgs &a, int fam, int mode, double inv_scale, int32_t *bins,
                         double *x, double *w, cudaStream_t stream) {
    const int tier = tier_of(a.d);
    const void *fn = nullptr;
    // FP32 modes share the map/integrand arithmetic; the accumulation mode
    // only changes how sums are kept, which the trace does not do.
    if (mode == ACC_F64) fn = trace_pick_fam<ACC_F64>(fam, tier);
    else fn = trace_pick_fam<ACC_F32_KAHAN>(fam, tier);
    return launch_trace_fn(fn, a, inv_scale, bins, x, w, nullptr, stream);
}

const void *trace_kernel_for(int fam, int mode, int d) {
    const int tier = tier_of(d);
    return mode == ACC_F64 ? trace_pick_fam<ACC_F64>(fam, tier) : trace_pick_fam<ACC_F32_KAHAN>(fam, tier);
}

cudaError_t launch_trace_fn(const void *fn, const SampleArgs &a, double inv_scale, int32_t *bins,
                            double *x, double *w, const HistArgs *hist, cudaStream_t stream) {
    if (!fn) return cudaErrorInvalidValue;
    if (a.n <= 0) return cudaSuccess;
    const unsigned threads = 256;
    long long blocks = (a.n + threads - 1) / threads;
    HistArgs h;
    memset(&h, 0, sizeof(h));
    if (hist) {
        h = *hist;
        blocks = std::min(blocks, 2048LL);  // grid-stride: one histogram flush per block
    }
    SampleArgs args = a;
    void *params[] = {&args, &inv_scale, &bins, &x, &w, &h};
    // shared memory: a density grid, padded (at most kMaxPdfValues FP64 values: 48 KB), then the
    // block's histogram (at most 2 (1024 + 2) FP64 values)
    size_t smem = a.pdf ? (static_cast<size_t>(a.pdf_nx + 2) * (a.pdf_nq + 2) * sizeof(double) + 15) / 16 * 16 : 0;
    if (hist) smem += static_cast<size_t>(2 * (h.nb + 2)) * sizeof(double);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    return cudaLaunchKernel(fn, dim3(static_cast<unsigned>(blocks)), dim3(threads), params, smem, stream);
}

// --------------------------------------------------------------- Philox
__global__ void philox_kernel(const uint4 *ctr, const uint2 *key, uint4 *out, long long n) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint2 k = key[i];
    out[i] = philox4x32_10(ctr[i], k.x, k.y);
}

cudaError_t launch_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, long long n,
                          cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    const unsigned blocks = static_cast<unsigned>((n + 255) / 256);
    philox_kernel<<<blocks, 256, 0, stream>>>(reinterpret_cast<const uint4 *>(ctr),
                                              reinterpret_cast<const uint2 *>(key),
                                              reinterpret_cast<uint4 *>(out), n);
    return cudaGetLastError();
}

template <int MODE>
static size_t smem_of(int layout, int d, int N) {
    if (layout == kLayoutWide) return sample_smem_bytes<MODE, kLayoutWide>(d, N);
    return layout == 1 ? sample_smem_bytes<MODE, 1>(d, N)
                       : (layout == 2 ? sample_smem_bytes<MODE, 2>(d, N) : sample_smem_bytes<MODE, 0>(d, N));
}

size_t sample_smem(int mode, int layout, int d, int N) {
    switch (mode) {
    case ACC_F64: return smem_of<ACC_F64>(layout, d, N);
    case ACC_F32_SUM64: return smem_of<ACC_F32_SUM64>(layout, d, N);
    default: return smem_of<ACC_F32_KAHAN>(layout, d, N);
    }
}

template <int MODE>
static long long cap_of(int layout, int N) {
    return layout == 1 ? block_sample_cap<MODE, 1>(N)
                       : (layout == 2 ? block_sample_cap<MODE, 2>(N) : block_sample_cap<MODE, 0>(N));
}

long long block_samples_max(int mode, int layout, int N) {
    return mode == ACC_F32_SUM64 ? cap_of<ACC_F32_SUM64>(layout, N) : cap_of<ACC_F32_KAHAN>(layout, N);
}

}  // namespace vegas
