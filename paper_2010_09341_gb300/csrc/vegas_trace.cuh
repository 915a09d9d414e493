// vegas_trace.cuh -- per-sample trace and observable histograms of an
// iteration: bins, points and weights of given samples written to device
// buffers (event weights), or the weights binned in an observable in shared
// memory (no traffic per sample).  The same split, stratum, map, Jacobian and
// integrand arithmetic as the sampling kernels, reading the table from global
// memory.
#pragma once

#include "vegas_sample.cuh"

namespace vegas {

// Observable histogram of an iteration's weights (vegas_histogram, computed by
// the trace kernel): out holds 2 (nb + 2) FP64 sums, sum v then sum v^2, each
// with bin 0 below lo, bin 1 + floor((o - lo)/w) (at most nb) up to hi, bin
// nb + 1 at or above hi.  obs >= 0: the coordinate x_obs; -1: sqrt(shat) =
// sqrt(x1 x2) sqrt_s; -2: cos(theta) = 2 x3 - 1.
struct HistArgs {
    double *out;   // null: no histogram
    int nb;
    int obs;
    double lo, hi, w, sqrt_s;
};

// Grid-stride over samples [a.s_begin, a.s_begin + a.n): bins, xs, ws (any
// may be null) get each sample's bins, points and weight v = J f (unscaled);
// with h.out, v and v^2 of each sample with a finite v are added to its
// observable's bin (HistArgs), per block in shared memory, then once per bin
// to h.out.  Dynamic shared memory: the padded density grid (F_LO_PDF), then
// the block's histogram.
template <int FAM, int MODE, int MAXD>
__global__ void trace_kernel(const SampleArgs a, double inv_scale, int32_t *bins, double *xs,
                             double *ws, const HistArgs h) {
    using T = typename ModeTraits<MODE>::T;
    using T2 = typename Prec<T>::T2;
    extern __shared__ __align__(16) unsigned char trace_smem[];
    unsigned char *raw = trace_smem;
    Integrand<FAM, T, MAXD> fam;
    if (FAM == F_LO_PDF) {
        // the density grid in shared memory, in the path's precision
        T *t = reinterpret_cast<T *>(raw);
        stage_grid(t, a.pdf, a.pdf_nx, a.pdf_nq);
        fam.tbl = t;
        raw += pdf_grid_offset(pdf_grid_bytes(MODE, a.pdf_nx, a.pdf_nq));
    }
    double *hs = h.out ? reinterpret_cast<double *>(raw) : nullptr;
    const int hn = 2 * (h.nb + 2);
    if (hs)
        for (int i = threadIdx.x; i < hn; i += blockDim.x) hs[i] = 0.0;
    __syncthreads();
    const int d = a.d, N = a.N;
    const T2 *tab = static_cast<const T2 *>(a.table);
    const FamConsts<T> &fc = consts<T>(a);
    const double jm = a.jmul ? *a.jmul : 1.0;
    const T n4 = static_cast<T>(a.nblk4);
    const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
    for (long long k = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; k < a.n; k += stride) {
        const unsigned long long s = static_cast<unsigned long long>(a.s_begin + k);
        const uint32_t slo = static_cast<uint32_t>(s), shi = static_cast<uint32_t>(s >> 32);
        T J = static_cast<T>(a.jinit * jm);
        double xo = 0.0, x0 = 0.0, x1 = 0.0, x2 = 0.0;
        fam.begin(fc);
#pragma unroll
        for (int q = 0; q < (MAXD + 3) / 4; ++q) {
            if (4 * q < d) {
                const uint4 r = philox4x32_10(make_uint4(slo, shi, a.iter, static_cast<uint32_t>(q)),
                                              a.key0, a.key1);
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    const int j = 4 * q + w;
                    if (j < MAXD && j < d) {
                        uint32_t rw = word(r, w);
                        if (a.st.P > 0)
                            rw = strat_word(rw, static_cast<uint32_t>(s / a.st.P), a.st.off[j], a.st.bits[j]);
                        const Split sp = split_bin(rw, static_cast<uint32_t>(N));
                        const uint32_t cell = static_cast<uint32_t>(j * N) + sp.bin;
                        const T2 ent = tab[cell];
                        const T x = Prec<T>::coord(ent, sp.lo);
                        J *= ent.y;
                        if (sizeof(T) == 4 && (j & 3) == 3) J *= n4;
                        fam.dim(j, x, fc);
                        // the coordinate itself (FP32 works in 2^32 (x - c), exactly
                        // scaled; the table centre c added back in FP64)
                        const double xd = static_cast<double>(x) * Prec<T>::kInvXS + a.center[j];
                        if (j == h.obs) xo = xd;
                        if (j == 0) x0 = xd;
                        if (j == 1) x1 = xd;
                        if (j == 2) x2 = xd;
                        if (bins) bins[k * d + j] = static_cast<int32_t>(sp.bin);
                        if (xs) xs[k * d + j] = xd;
                    }
                }
            }
        }
        T v = J * fam.finish(fc);
        if (a.st.P > 0 && !isfinite(v)) v = T(0);  // stratified: non-finite counts as 0
        const double vd = static_cast<double>(v) * (inv_scale / jm);
        if (ws) ws[k] = vd;
        if (hs && isfinite(vd)) {
            double o;
            if (h.obs >= 0) o = xo;
            else if (h.obs == -1) o = sqrt(x0 * x1) * h.sqrt_s;
            else o = 2.0 * x2 - 1.0;
            int b;
            if (o < h.lo) b = 0;
            else if (o >= h.hi) b = h.nb + 1;
            else b = min(h.nb, 1 + static_cast<int>(floor((o - h.lo) / h.w)));
            atomicAdd(hs + b, vd);
            atomicAdd(hs + h.nb + 2 + b, vd * vd);
        }
    }
    if (hs) {
        __syncthreads();
        for (int i = threadIdx.x; i < hn; i += blockDim.x)
            if (hs[i] != 0.0) atomicAdd(h.out + i, hs[i]);
    }
}

}  // namespace vegas
