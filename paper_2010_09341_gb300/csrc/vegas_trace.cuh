// vegas_trace.cuh -- per-sample trace: bins, points and weights of given
// samples of an iteration, written to device buffers (event weights for
// histogramming an observable).  The same split, stratum, map, Jacobian and
// integrand arithmetic as the sampling kernels, reading the table from global
// memory.
#pragma once

#include "vegas_sample.cuh"

namespace vegas {

// One thread per sample; the same split, map, Jacobian and integrand code as
// the sampling kernel, reading the table from global memory.
template <int FAM, int MODE, int MAXD>
__global__ void trace_kernel(const SampleArgs a, double inv_scale, int32_t *bins, double *xs,
                             double *ws) {
    using T = typename ModeTraits<MODE>::T;
    using T2 = typename Prec<T>::T2;
    extern __shared__ __align__(16) unsigned char trace_smem[];
    const long long k = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    Integrand<FAM, T, MAXD> fam;
    if (FAM == F_LO_PDF) {
        // the density grid in shared memory, in the path's precision
        T *t = reinterpret_cast<T *>(trace_smem);
        stage_grid(t, a.pdf, a.pdf_nx, a.pdf_nq);
        __syncthreads();
        fam.tbl = t;
    }
    if (k >= a.n) return;
    const int d = a.d, N = a.N;
    const T2 *tab = static_cast<const T2 *>(a.table);
    const FamConsts<T> &fc = consts<T>(a);
    const unsigned long long s = static_cast<unsigned long long>(a.s_begin + k);
    const uint32_t slo = static_cast<uint32_t>(s), shi = static_cast<uint32_t>(s >> 32);
    const double jm = a.jmul ? *a.jmul : 1.0;
    T J = static_cast<T>(a.jinit * jm);
    const T n4 = static_cast<T>(a.nblk4);
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
                    if (a.st.P > 0) rw = strat_word(rw, static_cast<uint32_t>(s / a.st.P), a.st.off[j], a.st.bits[j]);
                    const Split sp = split_bin(rw, static_cast<uint32_t>(N));
                    const uint32_t cell = static_cast<uint32_t>(j * N) + sp.bin;
                    const T2 ent = tab[cell];
                    const T m = Prec<T>::mant(sp.lo);
                    const T x = ffma(ent.y, m, ent.x);
                    J *= ent.y;
                    if (sizeof(T) == 4 && (j & 3) == 3) J *= n4;
                    fam.dim(j, x, fc);
                    if (bins) bins[k * d + j] = static_cast<int32_t>(sp.bin);
                    if (xs) xs[k * d + j] = static_cast<double>(x);
                }
            }
        }
    }
    T v = J * fam.finish(fc);
    if (a.st.P > 0 && !isfinite(v)) v = T(0);  // stratified: non-finite counts as 0
    if (ws) ws[k] = static_cast<double>(v) * (inv_scale / jm);
}

}  // namespace vegas
