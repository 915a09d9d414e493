// hist_prereduce.cu -- the sampling loop's histogram update, two ways, on the
// GPU it runs on: lane-private integer cells (what the library's FP32 kernels
// do) against warp pre-reduction of the updates (lanes that hit the same cell
// found with match.any.sync, their values summed with redux.sync, one atomic
// by the group's lowest lane into a single-copy cell).
//
// Each variant runs the same loop over 1e7 samples: two Philox4x32-10 calls
// per sample (d <= 8), the integer bin split, the in-bin position, the table
// map and Jacobian, the symmetric Gaussian (a = 0.1), v^2 as a fixed-point
// integer (1 .. 2^23), and one histogram update per dimension.  The integer
// histograms of the two variants must agree exactly (integer sums do not
// depend on the order); the program fails otherwise.
//
// Build and run (one GPU):
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 -o hist_prereduce hist_prereduce.cu && ./hist_prereduce
// Output: per shape (d, N) and variant, the kernel time (CUDA events, mean of
// 5 launches after 2 warm-up launches) and the samples per second.
//
// A third variant keeps the lane-private cells with half as many copies
// (8 table and 16 histogram copies per cell, two lanes per copy) and asks
// for 4 blocks of 512 threads per SM instead of 2: twice the resident warps
// for some two-way bank conflicts, a test of whether the loop is bound by
// latency that more warps would hide.
#include <cstdint>
#include <cstdio>
#include <vector>
#include <cuda_runtime.h>

#include "../csrc/vegas_device.cuh"

namespace {

constexpr int kThreads = 512;

// Copies per cell: table TP, histogram HP (1 for the pre-reduction), and the
// blocks per SM the launch bounds ask for.
template <int V> struct Var;
template <> struct Var<0> { static constexpr int TP = 16, HP = 32, MINB = 1; static constexpr bool PRE = false; };
template <> struct Var<1> { static constexpr int TP = 16, HP = 1, MINB = 1; static constexpr bool PRE = true; };
template <> struct Var<2> { static constexpr int TP = 8, HP = 16, MINB = 4; static constexpr bool PRE = false; };

template <int D, int N, int V>
__global__ void __launch_bounds__(kThreads, Var<V>::MINB)
sample_hist(const float2 *gtab, unsigned long long *ghist, long long n, uint32_t key0, uint32_t key1, float s0,
            float hscale) {
    constexpr int kTP = Var<V>::TP, HC = Var<V>::HP;
    constexpr bool PRE = Var<V>::PRE;
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *tab = reinterpret_cast<float2 *>(smem);
    uint32_t *hist = reinterpret_cast<uint32_t *>(tab + D * N * kTP);
    for (int k = threadIdx.x; k < D * N * kTP; k += blockDim.x) tab[k] = gtab[k / kTP];
    for (int k = threadIdx.x; k < D * N * HC; k += blockDim.x) hist[k] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const float2 *tab_l = tab + (lane % kTP);
    uint32_t *hist_l = hist + (PRE ? 0 : lane % HC);
    const long long per = (n + gridDim.x - 1) / gridDim.x;
    const long long lo = static_cast<long long>(blockIdx.x) * per;
    const long long hi = lo + per < n ? lo + per : n;
    // every lane of a warp runs the same number of iterations (the
    // pre-reduction's warp-wide instructions need the whole warp)
    for (long long base = lo; base < hi; base += blockDim.x) {
        const long long s = base + threadIdx.x;
        const bool live = s < hi;
        const uint32_t slo = static_cast<uint32_t>(s), shi = static_cast<uint32_t>(s >> 32);
        uint32_t cell[D];
        float J = 1.f, acc = 0.f;
#pragma unroll
        for (int q = 0; q < (D + 3) / 4; ++q) {
            const uint4 r = vegas::philox4x32_10(make_uint4(slo, shi, 0u, static_cast<uint32_t>(q)), key0, key1);
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const int j = 4 * q + w;
                if (j < D) {
                    const vegas::Split sp = vegas::split_bin(vegas::word(r, w), N);
                    cell[j] = static_cast<uint32_t>(j * N) + sp.bin;
                    const float2 e = tab_l[cell[j] * kTP];
                    const float x = vegas::Prec<float>::coord(e, sp.lo);
                    J *= e.y;
                    acc = __fmaf_rn(x, x, acc);
                }
            }
        }
        const float v = J * vegas::fexp2(s0 * acc);
        const float qf = fminf(fmaxf(v * v * hscale, 1.0f), 8388607.0f);
        const uint32_t qv = live ? static_cast<uint32_t>(__float2uint_rn(qf)) : 0u;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            if (PRE) {
                // the lanes that hit this cell (dead lanes carry their cell but add 0)
                const unsigned grp = __match_any_sync(0xFFFFFFFFu, cell[j]);
                const unsigned sum = __reduce_add_sync(grp, qv);
                if (lane == __ffs(grp) - 1 && sum) atomicAdd(hist_l + cell[j], sum);
            } else if (qv) {
                atomicAdd(hist_l + cell[j] * HC, qv);
            }
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < D * N; c += blockDim.x) {
        unsigned long long t = 0;
        for (int k = 0; k < HC; ++k) t += hist[c * HC + k];
        if (t) atomicAdd(ghist + c, t);
    }
}

template <int D, int N, int V>
bool run(const float2 *dtab, unsigned long long *dhist, long long n, int sms, float *ms_out,
         std::vector<unsigned long long> &out, int *blocks_per_sm) {
    const size_t smem = static_cast<size_t>(D) * N * (Var<V>::TP * sizeof(float2) + Var<V>::HP * sizeof(uint32_t));
    auto k = sample_hist<D, N, V>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
        return false;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kThreads, smem) != cudaSuccess || occ < 1) return false;
    *blocks_per_sm = occ;
    const int blocks = occ * sms;
    // f = exp(-sum (x - 1/2)^2 / a^2) from acc = sum X^2, X = 2^32 (x - 1/2) (table about 1/2)
    const float s0 = -1.4426950408889634f / (0.1f * 0.1f) * 5.421010862427522e-20f;  // x 2^-64
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float total = 0.f;
    for (int it = 0; it < 7; ++it) {
        if (cudaMemset(dhist, 0, sizeof(unsigned long long) * D * N) != cudaSuccess) return false;
        cudaEventRecord(a);
        k<<<blocks, kThreads, smem>>>(dtab, dhist, n, 7u, 11u, s0, 262144.0f);  // v^2 <= 1 -> q <= 2^18
        cudaEventRecord(b);
        if (cudaEventSynchronize(b) != cudaSuccess) return false;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (it >= 2) total += ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *ms_out = total / 5.f;
    out.assign(D * N, 0ull);
    return cudaMemcpy(out.data(), dhist, sizeof(unsigned long long) * D * N, cudaMemcpyDeviceToHost) == cudaSuccess;
}

template <int D, int N>
int shape(int sms, long long n) {
    // a non-uniform grid, entries about the centre 1/2 (2^32 (e - 1/2), w)
    std::vector<float2> tab(D * N);
    for (int j = 0; j < D; ++j) {
        std::vector<double> e(N + 1);
        for (int k = 0; k <= N; ++k) {
            const double u = static_cast<double>(k) / N;
            e[k] = u + 0.08 * u * (1.0 - u) * (u - 0.5);  // monotone, pinned at 0 and 1
        }
        for (int k = 0; k < N; ++k)
            tab[j * N + k] = make_float2(static_cast<float>((e[k] - 0.5) * 4294967296.0),
                                         static_cast<float>((e[k + 1] - e[k]) * N));
    }
    float2 *dtab = nullptr;
    unsigned long long *dhist = nullptr;
    if (cudaMalloc(&dtab, sizeof(float2) * D * N) != cudaSuccess ||
        cudaMalloc(&dhist, sizeof(unsigned long long) * D * N) != cudaSuccess) {
        fprintf(stderr, "cudaMalloc failed\n");
        return 1;
    }
    cudaMemcpy(dtab, tab.data(), sizeof(float2) * D * N, cudaMemcpyHostToDevice);
    float ms_priv = 0.f, ms_pre = 0.f, ms_half = 0.f;
    int occ_priv = 0, occ_pre = 0, occ_half = 0;
    std::vector<unsigned long long> h_priv, h_pre, h_half;
    const bool ok = run<D, N, 0>(dtab, dhist, n, sms, &ms_priv, h_priv, &occ_priv) &&
                    run<D, N, 1>(dtab, dhist, n, sms, &ms_pre, h_pre, &occ_pre) &&
                    run<D, N, 2>(dtab, dhist, n, sms, &ms_half, h_half, &occ_half);
    cudaFree(dtab);
    cudaFree(dhist);
    if (!ok) {
        fprintf(stderr, "d=%d N=%d: %s\n", D, N, cudaGetErrorString(cudaGetLastError()));
        return 1;
    }
    if (h_priv != h_pre || h_priv != h_half) {
        fprintf(stderr, "d=%d N=%d: the two variants' histograms differ\n", D, N);
        return 1;
    }
    unsigned long long tot = 0;
    for (auto x : h_priv) tot += x;
    printf("d=%d N=%-4d lane-private cells : %8.3f ms  %7.2f G samples/s  (%d blocks/SM)\n", D, N, ms_priv,
           n / (ms_priv * 1e6), occ_priv);
    printf("d=%d N=%-4d warp pre-reduction : %8.3f ms  %7.2f G samples/s  (%.2fx the time, %d blocks/SM)\n", D, N,
           ms_pre, n / (ms_pre * 1e6), ms_pre / ms_priv, occ_pre);
    printf("d=%d N=%-4d half the copies    : %8.3f ms  %7.2f G samples/s  (%.2fx the time, %d blocks/SM)\n", D, N,
           ms_half, n / (ms_half * 1e6), ms_half / ms_priv, occ_half);
    printf("   histograms identical (sum %llu)\n", tot);
    return 0;
}

}  // namespace

int main() {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess || sms <= 0) {
        fprintf(stderr, "no CUDA device\n");
        return 1;
    }
    const long long n = 10000000;
    int rc = shape<8, 50>(sms, n);
    if (rc == 0) rc = shape<3, 100>(sms, n);
    return rc;
}
