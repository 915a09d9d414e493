// vegas_sample.cuh -- the fused sample + map + integrand + accumulate kernel.
//
// One launch covers samples [s_begin, s_begin + n) of iteration t.  Each block
// takes a contiguous range, each thread every blockDim-th sample of it.
// Per sample (VEGAS, Lepage 1978; the paper's method, Sec. 1):
//   r   = Philox4x32-10 words (ceil(d/4) calls, registers only)
//   i_j = bin of r_j, x_j = (e - w)_j[i_j] + w_j[i_j] m_j,  m_j in [1, 2)
//   J   = C prod_j w_j[i_j]            (C = N^d times constant factors of f)
//   v   = J f(x);  S1 += v, S2 += v^2, h_j[i_j] += v^2
//
// Shared memory holds, per (dimension, bin) cell, TP copies of the table
// entry (e - w, w) and HP copies of the histogram cell, so that the 32 lanes
// of a warp read and update distinct banks whatever bins they draw
// (lane-private copies).  When the copies do not fit, a single-copy layout is
// used (PRIV = false) and bank conflicts are accepted.
#pragma once

#include "vegas_device.cuh"

namespace vegas {

enum AccMode : int { ACC_F64 = 0, ACC_F32_SUM64 = 1, ACC_F32_KAHAN = 2 };

struct SampleArgs {
    const void *table;        // [d][N] entries (e - w, w): double2 or float2
    double *acc;              // [2 + d N] FP64 accumulators: S1, S2, histograms
    unsigned long long *n_nonfinite;
    long long s_begin;        // first sample index of this launch
    long long n;              // samples in this launch
    int d, N;
    uint32_t key0, key1;      // Philox key (seed, integral id)
    uint32_t iter;            // Philox counter word 2
    double jinit;             // initial weight C (includes N^d and scale)
    double nblk4;             // N^4 (FP32 path multiplies it in every 4 dims)
    const float *hscale;      // FP32 modes: fixed-point scale of v^2 (0: float cells)
    FamConsts<double> fc64;   // integrand constants, FP64 path
    FamConsts<float> fc32;    // the same rounded to FP32, FP32 paths
};

template <class T> __device__ __forceinline__ const FamConsts<T> &consts(const SampleArgs &a);
template <> __device__ __forceinline__ const FamConsts<double> &consts<double>(const SampleArgs &a) {
    return a.fc64;
}
template <> __device__ __forceinline__ const FamConsts<float> &consts<float>(const SampleArgs &a) {
    return a.fc32;
}

// FP32 histogram cells (ACC_F32_*).  Shared-memory FP32 atomic add has no
// native instruction on this GPU (it runs as a compare-and-swap loop), while
// 32-bit integer atomic add is native.  When a scale S > 0 is known (from the
// previous iteration's mean v^2, set so that it maps to 2^18), each v^2 with
// q = S v^2 < 2^23 is added as an integer with one native atomic per
// dimension:
//   q >= 1 : rint(q) into the lane-private coarse cell (error <= 1/2 quantum,
//            i.e. <= 2^-19 of the mean per value);
//   q <  1 : max(1, rint(2^16 q)) into a single-copy fine cell (error <= 2^-16
//            quantum; a positive value never adds zero, so no bin that saw a
//            positive weight loses all of it);
//   q >= 2^23 (more than 32x the previous mean): straight to the FP64
//            accumulator in global memory.
// The lane's choice of cell array is a select, not a branch, so a warp whose
// lanes mix coarse and fine values still issues one atomic per dimension.
// Capacity: a coarse cell receives ~64 values on average per block (the
// launch keeps block samples <= 2048 N; 512 values would be needed to reach
// 2^32); a fine cell at most 2048 N values below 2^16.  With S = 0 (first
// iteration) the lane-private cells hold FP32 and take every value.  Zero
// weights touch no cell.
constexpr float kFineScale = 65536.0f;    // 2^16
constexpr float kFineInv = 1.0f / 65536.0f;
constexpr float kFixedMax = 8388608.0f;   // 2^23

template <int MODE> struct ModeTraits;
template <> struct ModeTraits<ACC_F64> {
    using T = double;   // map, Jacobian, integrand
    using H = double;   // shared histogram cell
    static constexpr int TP = 8;    // 16-byte entries: 8 lanes per wavefront
    static constexpr int HP = 16;   // 8-byte cells: 16 lanes per wavefront
};
template <> struct ModeTraits<ACC_F32_SUM64> {
    using T = float;
    using H = float;                // bounded-depth cells, promoted to FP64 per block
    static constexpr int TP = 16;   // 8-byte entries: 16 lanes per wavefront
    static constexpr int HP = 32;   // 4-byte cells: a whole warp per wavefront
};
template <> struct ModeTraits<ACC_F32_KAHAN> {
    using T = float;
    using H = float;
    static constexpr int TP = 16;
    static constexpr int HP = 32;   // 4-byte cells: a whole warp per wavefront
};

template <int MODE, bool PRIV>
__host__ __device__ constexpr size_t sample_smem_bytes(int d, int N) {
    using Tr = ModeTraits<MODE>;
    return static_cast<size_t>(d) * N *
           ((PRIV ? Tr::TP : 1) * 2 * sizeof(typename Tr::T) + (PRIV ? Tr::HP : 1) * sizeof(typename Tr::H) +
            (MODE != ACC_F64 ? sizeof(uint32_t) : 0));  // single-copy fine cells
}

__device__ __forceinline__ void red_add_shared(float *p, float v) { atomicAdd(p, v); }
__device__ __forceinline__ void red_add_shared(double *p, double v) { atomicAdd(p, v); }

// Warp-level FP64 sum.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// EXACT: the dimension equals MAXD (no per-dimension guards); otherwise
// 1 <= a.d <= MAXD at run time.
template <int FAM, int MODE, int MAXD, bool EXACT, bool PRIV>
__global__ void __launch_bounds__(512)
vegas_sample_kernel(const SampleArgs a) {
    using Tr = ModeTraits<MODE>;
    using T = typename Tr::T;
    using T2 = typename Prec<T>::T2;
    using H = typename Tr::H;
    constexpr int TP = PRIV ? Tr::TP : 1;
    constexpr int HP = PRIV ? Tr::HP : 1;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int d = EXACT ? MAXD : a.d;
    const int N = a.N;
    const int cells = d * N;
    T2 *tab = reinterpret_cast<T2 *>(smem_raw);
    H *hist = reinterpret_cast<H *>(smem_raw + static_cast<size_t>(cells) * TP * sizeof(T2));
    uint32_t *fine = reinterpret_cast<uint32_t *>(hist + static_cast<size_t>(cells) * HP);  // FP32 modes

    // stage the grid table (TP copies per cell) and zero the histogram
    const float hs = (MODE != ACC_F64) ? *a.hscale : 0.f;
    const bool fixed = hs > 0.f;
    const T2 *gtab = static_cast<const T2 *>(a.table);
    for (int k = threadIdx.x; k < cells * TP; k += blockDim.x) tab[k] = gtab[k / TP];
    for (int k = threadIdx.x; k < cells * HP; k += blockDim.x) hist[k] = H(0);
    if (MODE != ACC_F64)
        for (int k = threadIdx.x; k < cells; k += blockDim.x) fine[k] = 0u;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const T2 *tab_l = tab + (lane % TP);
    H *hist_l = hist + (lane % HP);

    Integrand<FAM, T, MAXD> fam;
    const FamConsts<T> &fc = consts<T>(a);
    const T jinit = static_cast<T>(a.jinit);
    const T n4 = static_cast<T>(a.nblk4);

    // contiguous sample range of this block
    const long long per = (a.n + gridDim.x - 1) / gridDim.x;
    const long long lo = static_cast<long long>(blockIdx.x) * per;
    const long long hi = min(a.n, lo + per);

    double s1d = 0.0, s2d = 0.0;       // FP64 sums (ACC_F64, ACC_F32_SUM64)
    float s1f = 0.f, c1f = 0.f, s2f = 0.f, c2f = 0.f;  // ACC_F32_KAHAN
    unsigned int nonfinite = 0;

    // Each thread takes every blockDim-th sample of the block's range, in
    // chunks of kChunk; ACC_F32_SUM64 adds a chunk's FP32 partial sums into
    // the FP64 sums once per chunk.
    constexpr int kChunk = 8;
    const int cnt = static_cast<int>(hi - lo);  // samples of this block (< 2^31)
    const int stride = blockDim.x;
    for (int k0 = threadIdx.x; k0 < cnt; k0 += kChunk * stride) {
        float p1 = 0.f, p2 = 0.f;
#pragma unroll 1
        for (int u = 0; u < kChunk; ++u) {
            const int k = k0 + u * stride;
            if (k >= cnt) break;
            const unsigned long long s = static_cast<unsigned long long>(a.s_begin + lo + k);
            const uint32_t slo = static_cast<uint32_t>(s), shi = static_cast<uint32_t>(s >> 32);
            uint32_t cellj[MAXD];
            T J = jinit;
            fam.begin(fc);
#pragma unroll
            for (int q = 0; q < (MAXD + 3) / 4; ++q) {
                if (EXACT || 4 * q < d) {
                    const uint4 r = philox4x32_10(make_uint4(slo, shi, a.iter, static_cast<uint32_t>(q)),
                                                  a.key0, a.key1);
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        const int j = 4 * q + w;
                        if (j < MAXD && (EXACT || j < d)) {
                            const Split sp = split_bin(word(r, w), static_cast<uint32_t>(N));
                            const uint32_t cell = static_cast<uint32_t>(j * N) + sp.bin;
                            const T2 ent = tab_l[cell * TP];
                            const T m = Prec<T>::mant(sp.lo);
                            const T x = ffma(ent.y, m, ent.x);
                            J *= ent.y;
                            if (sizeof(T) == 4 && (j & 3) == 3) J *= n4;
                            cellj[j] = cell;
                            fam.dim(j, x, fc);
                        }
                    }
                }
            }
            T v = J * fam.finish(fc);
            if (!isfinite(v)) {
                v = T(0);
                ++nonfinite;
            }
            const T v2 = v * v;
            if (MODE == ACC_F32_KAHAN) {
                const float y1 = static_cast<float>(v) - c1f;
                const float t1 = s1f + y1;
                c1f = (t1 - s1f) - y1;
                s1f = t1;
                const float y2 = static_cast<float>(v2) - c2f;
                const float t2 = s2f + y2;
                c2f = (t2 - s2f) - y2;
                s2f = t2;
            } else if (MODE == ACC_F32_SUM64) {
                p1 += static_cast<float>(v);
                p2 += static_cast<float>(v2);
            } else {
                const double vd = static_cast<double>(v);
                s1d += vd;
                s2d = __fma_rn(vd, vd, s2d);
            }
            if (MODE == ACC_F64) {
#pragma unroll
                for (int j = 0; j < MAXD; ++j) {
                    if (EXACT || j < d) red_add_shared(hist_l + cellj[j] * HP, static_cast<H>(v2));
                }
            } else if (v2 == T(0)) {
                // nothing to add
            } else if (fixed) {
                const float qf = static_cast<float>(v2) * hs;
                if (qf < kFixedMax) {
                    // rint by adding 2^23 (the integer lands in the mantissa's
                    // low bits; exact for values below 2^23)
                    const bool is_fine = qf < 1.0f;
                    const float t = __fmaf_rn(qf, is_fine ? kFineScale : 1.0f, 8388608.0f);
                    uint32_t q = __float_as_uint(t) - 0x4B000000u;
                    q = max(q, 1u);
                    unsigned int *base = is_fine ? fine : reinterpret_cast<unsigned int *>(hist_l);
                    const uint32_t step = is_fine ? 1u : static_cast<uint32_t>(HP);
#pragma unroll
                    for (int j = 0; j < MAXD; ++j) {
                        if (EXACT || j < d) atomicAdd(base + cellj[j] * step, q);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < MAXD; ++j) {
                        if (EXACT || j < d) atomicAdd(a.acc + 2 + cellj[j], static_cast<double>(v2));
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < MAXD; ++j) {
                    if (EXACT || j < d) red_add_shared(reinterpret_cast<float *>(hist_l) + cellj[j] * HP,
                                                       static_cast<float>(v2));
                }
            }
        }
        if (MODE == ACC_F32_SUM64) {
            s1d += static_cast<double>(p1);
            s2d += static_cast<double>(p2);
        }
    }

    // block reduction of S1, S2 and the non-finite count
    double b1, b2;
    if (MODE == ACC_F32_KAHAN) {
        b1 = static_cast<double>(s1f) - static_cast<double>(c1f);
        b2 = static_cast<double>(s2f) - static_cast<double>(c2f);
    } else {
        b1 = s1d;
        b2 = s2d;
    }
    b1 = warp_sum(b1);
    b2 = warp_sum(b2);
    unsigned int nf = __reduce_add_sync(0xFFFFFFFFu, nonfinite);
    __shared__ double red1[16], red2[16];
    __shared__ unsigned int rednf[16];
    const int warp = threadIdx.x >> 5;
    if (lane == 0) {
        red1[warp] = b1;
        red2[warp] = b2;
        rednf[warp] = nf;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        double x1 = lane < nw ? red1[lane] : 0.0;
        double x2 = lane < nw ? red2[lane] : 0.0;
        unsigned int xn = lane < nw ? rednf[lane] : 0u;
        x1 = warp_sum(x1);
        x2 = warp_sum(x2);
        xn = __reduce_add_sync(0xFFFFFFFFu, xn);
        if (lane == 0) {
            atomicAdd(a.acc + 0, x1);
            atomicAdd(a.acc + 1, x2);
            if (xn) atomicAdd(a.n_nonfinite, static_cast<unsigned long long>(xn));
        }
    }
    // histogram flush: one warp per cell, lanes over the HP copies.  FP32
    // cells are summed as a warp tree in FP32 (5 levels) and promoted once.
    const int nwarps = blockDim.x >> 5;
    const float inv_hs = fixed ? 1.0f / hs : 0.f;
    for (int c = warp; c < cells; c += nwarps) {
        H h = H(0);
        for (int k = lane; k < HP; k += 32) {
            if (MODE != ACC_F64 && fixed)
                h += static_cast<H>(static_cast<float>(reinterpret_cast<const unsigned int *>(hist)[c * HP + k]) * inv_hs);
            else
                h += hist[c * HP + k];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xFFFFFFFFu, h, o);
        if (MODE != ACC_F64 && fixed && lane == 0) h += static_cast<H>(static_cast<float>(fine[c]) * (inv_hs * kFineInv));
        if (lane == 0 && h != H(0)) atomicAdd(a.acc + 2 + c, static_cast<double>(h));
    }
}

}  // namespace vegas
