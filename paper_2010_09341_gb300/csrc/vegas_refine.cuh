// vegas_refine.cuh -- grid refinement of one dimension by one block.
#pragma once

#include "vegas_kernels.cuh"

namespace vegas {

// Grid refinement of one dimension per block (Lepage 1980):
//   smooth   d_0 = (h_0+h_1)/2, d_k = (h_{k-1}+h_k+h_{k+1})/3, d_{N-1} = (h_{N-2}+h_{N-1})/2
//   normalise d_k /= sum d
//   compress rho_k = ((1 - d_k)/ln(1/d_k))^alpha   (0 at d = 0, 1 at d = 1)
//   rebin    new edge k (1..N-1) where the running rho sum reaches k sum(rho)/N,
//            interpolated linearly inside the old bin; zero-weight bins are
//            skipped and an edge on an old edge takes the lower bin.
// A dimension whose weights sum to zero keeps its grid.
// Sampling-table entry of the bin [e, e + w) of a dimension whose integrand
// takes its coordinate relative to the centre c (Prec<T>::coord gives x - c;
// c = 0 for most families): FP64 (e - w - c, w), x - c = (e - w - c) + w m with
// m in [1, 2); FP32 (2^32 (e - c), w), 2^32 (x - c) = 2^32 (e - c) + w float(lo).
__device__ __forceinline__ void store_table(void *table, int mode, int idx, double e, double w, double c) {
    if (mode == ACC_F64) reinterpret_cast<double2 *>(table)[idx] = double2{(e - c) - w, w};
    else reinterpret_cast<float2 *>(table)[idx] = float2{static_cast<float>((e - c) * 4294967296.0), static_cast<float>(w)};
}

constexpr int kRefineThreads = 128;

// Refines one dimension with the whole block (blockDim.x == kRefineThreads):
// h = its N histogram values, e = its N+1 FP64 edges (updated in place),
// table_row = its N sampling-table entries of `mode` about the centre c
// (store_table); rs = 4N+2 doubles of shared memory.  A dimension whose
// weights sum to zero keeps its grid.
__device__ __forceinline__ void refine_block(const double *h, double *e, void *table_row, int mode, int N,
                             double alpha, int smooth, double c, double *rs) {
    double *eo = rs;            // old edges, N+1
    double *rho = rs + (N + 1); // compressed weights, N
    double *cum = rho + N;      // inclusive running sum, N
    double *en = cum + N;       // new edges, N+1
    __shared__ double red[kRefineThreads / 32];
    __shared__ double total_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __syncthreads();  // rs and red may still be read by a previous call
    for (int k = tid; k <= N; k += blockDim.x) eo[k] = e[k];

    // smoothing, kept in rho[] for now
    double part = 0.0;
    for (int k = tid; k < N; k += blockDim.x) {
        double v;
        if (!smooth) v = h[k];
        else if (k == 0) v = (h[0] + h[1]) / 2.0;
        else if (k == N - 1) v = (h[N - 2] + h[N - 1]) / 2.0;
        else v = (h[k - 1] + h[k] + h[k + 1]) / 3.0;
        rho[k] = v;
        part += v;
    }
    part = warp_sum(part);
    if (lane == 0) red[warp] = part;
    __syncthreads();
    if (tid == 0) {
        double sum = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) sum += red[k];
        total_s = sum;
    }
    __syncthreads();
    const double total = total_s;
    if (!(total > 0.0) || !isfinite(total)) return;  // keep the grid (table unchanged)

    // normalise and compress
    for (int k = tid; k < N; k += blockDim.x) {
        const double dk = rho[k] / total;
        double r;
        if (dk <= 0.0) r = 0.0;
        else if (dk >= 1.0) r = 1.0;
        else {
            const double g = (1.0 - dk) / log(1.0 / dk);
            // g^alpha; the usual exponents without a general power
            if (alpha == 1.5) r = g * sqrt(g);
            else if (alpha == 1.0) r = g;
            else if (alpha == 0.5) r = sqrt(g);
            else if (alpha == 2.0) r = g * g;
            else if (alpha == 0.0) r = 1.0;
            else r = pow(g, alpha);
        }
        rho[k] = r;
    }
    __syncthreads();

    // inclusive scan of rho: each thread a contiguous chunk, then chunk offsets
    const int chunk = (N + blockDim.x - 1) / blockDim.x;
    const int k0 = tid * chunk, k1 = min(N, k0 + chunk);
    double run = 0.0;
    for (int k = k0; k < k1; ++k) {
        run += rho[k];
        cum[k] = run;
    }
    double incl = run;  // warp inclusive scan of chunk totals
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    __syncthreads();  // red[] reuse
    if (lane == 31) red[warp] = incl;
    __syncthreads();
    double off = incl - run;
    for (int w = 0; w < warp; ++w) off += red[w];
    for (int k = k0; k < k1; ++k) cum[k] += off;
    __syncthreads();
    const double rsum = cum[N - 1];
    if (!(rsum > 0.0)) return;
    const double delta = rsum / static_cast<double>(N);

    // rebin: new edge k is in the first old bin whose inclusive sum reaches k delta
    for (int k = tid; k <= N; k += blockDim.x) {
        double ek;
        if (k == 0) ek = 0.0;
        else if (k == N) ek = 1.0;
        else {
            const double target = static_cast<double>(k) * delta;
            int lo = 0, hi = N - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (cum[mid] >= target) hi = mid;
                else lo = mid + 1;
            }
            const int b = lo;
            const double before = b > 0 ? cum[b - 1] : 0.0;
            double frac = rho[b] > 0.0 ? (target - before) / rho[b] : 1.0;
            frac = fmin(fmax(frac, 0.0), 1.0);
            ek = eo[b] + frac * (eo[b + 1] - eo[b]);
        }
        en[k] = ek;
    }
    __syncthreads();
    for (int k = tid; k <= N; k += blockDim.x) e[k] = en[k];
    for (int k = tid; k < N; k += blockDim.x) store_table(table_row, mode, k, en[k], en[k + 1] - en[k], c);
}


}  // namespace vegas
