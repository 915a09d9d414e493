// vegas_sample.cuh -- the fused sample + map + integrand + accumulate kernel.
//
// One launch covers samples [s_begin, s_begin + n) of iteration t.  Each block
// takes a contiguous range, each thread every blockDim-th sample of it.
// Per sample (VEGAS, Lepage 1978; the paper's method, Sec. 1):
//   r   = Philox4x32-10 words (ceil(d/4) calls, registers only)
//   i_j = bin of r_j, x_j = e_j[i_j] + w_j[i_j] lo_j 2^-32  (lo_j: the low word
//         of r_j N; FP32 works in X = 2^32 x, see Prec<T>::coord)
//   J   = C prod_j w_j[i_j]            (C = N^d times constant factors of f)
//   v   = J f(x);  S1 += v, S2 += v^2, h_j[i_j] += v^2
//
// Shared memory holds, per (dimension, bin) cell, TP copies of the table
// entry (Prec<T>::coord) and HP copies of the histogram cell, so that the 32 lanes
// of a warp read and update distinct banks whatever bins they draw
// (lane-private copies).  Layouts (template parameter PRIV): 1 = TP and HP
// copies as above, 2 = half as many (two lanes share a copy: some two-way
// conflicts, half the memory), 0 = one copy (conflicts accepted) for what
// fits neither.
#pragma once

#include "vegas_device.cuh"

namespace vegas {

enum AccMode : int { ACC_F64 = 0, ACC_F32_SUM64 = 1, ACC_F32_KAHAN = 2 };

// Stratified + importance hybrid (Lepage 1980's combined mode).  y-space is cut
// into 2^B equal hypercubes and hypercube h takes samples hP .. hP + P - 1.
// Dimension j is halved bits[j] times; h's stratum in it is k_j = bits
// [off[j], off[j] + bits[j]) of h.  The stratum takes the top bits[j] bits of
// the sample's Philox word r_j:
//   R_j = k_j 2^(32 - bits[j]) + floor(r_j / 2^bits[j]),
// i.e. y_j = (k_j + r_j 2^-32) / 2^bits[j] on the 2^-32 lattice, and the
// importance map then treats R_j as plain sampling treats r_j.
struct StratArgs {
    uint32_t P;          // samples per hypercube; 0: plain sampling
    uint32_t off[32];
    uint32_t bits[32];   // each <= 16
    double *q;           // FP64 accumulator: sum_h sum_p (v - mean_h)^2
};

// R_j from r_j: the 64-bit pair (h >> off : r) shifted right by bits keeps the
// stratum's bits of h on top of the word's top 32 - bits bits.
__device__ __forceinline__ uint32_t strat_word(uint32_t r, uint32_t h, uint32_t off, uint32_t bits) {
    return __funnelshift_r(r, h >> off, bits);
}

struct SampleArgs {
    const void *table;        // [d][N] entries about the centres (store_table): double2 or float2
    const double *center;     // the d table centres (table_center; device)
    double *acc;              // [2 + d N] FP64 accumulators: S1, S2, histograms
    unsigned long long *n_nonfinite;
    long long s_begin;        // first sample index of this launch
    long long n;              // samples in this launch
    int d, N;
    uint32_t key0, key1;      // Philox key (seed, integral id)
    uint32_t iter;            // Philox counter word 2
    double jinit;             // initial weight C (includes N^d and the initial scale of v)
    const double *jmul;       // device: power-of-two rescale of v set by the last finalize (null: 1)
    double nblk4;             // N^4 (FP32 path multiplies it in every 4 dims)
    const float *hscale;      // FP32 modes: fixed-point scale of v^2 (0: float cells)
    FamConsts<double> fc64;   // integrand constants, FP64 path
    FamConsts<float> fc32;    // the same for the FP32 paths' X = 2^32 x, rounded to FP32
    StratArgs st;             // stratified launches: s_begin, n count hypercubes
    const double *pdf;        // F_LO_PDF: the density grid, pdf_nx x pdf_nq FP64 values (device)
    int pdf_nx, pdf_nq;
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
// Capacity: a block adds at most block_sample_cap(N) samples between flushes
// (below), so that no cell can reach 2^32.  With S = 0 (first
// iteration) the lane-private cells hold FP32 and take every value.  Zero
// weights touch no cell.
constexpr int kFineShift = 16;
constexpr float kFineScale = 65536.0f;    // 2^kFineShift
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

// Copies per (dimension, bin) cell of the table entry (TP) and of the
// histogram cell (HP) in layout PRIV: 0 one copy, 1 ModeTraits' copies, 2 half
// as many, 3 (kLayoutWide, the FP64 path) ModeTraits' table copies and one
// histogram copy per lane.
constexpr int kLayoutWide = 3;
template <int MODE, int PRIV> struct Copies {
    static constexpr int TP = PRIV == 0 ? 1 : (PRIV == 2 ? ModeTraits<MODE>::TP / 2 : ModeTraits<MODE>::TP);
    static constexpr int HP = PRIV == 0 ? 1
                                        : (PRIV == 1 ? ModeTraits<MODE>::HP
                                                     : (PRIV == 2 ? ModeTraits<MODE>::HP / 2 : 32));
};

template <int MODE, int PRIV>
__host__ __device__ constexpr size_t sample_smem_bytes(int d, int N) {
    using Tr = ModeTraits<MODE>;
    return static_cast<size_t>(d) * N *
           (Copies<MODE, PRIV>::TP * 2 * sizeof(typename Tr::T) + Copies<MODE, PRIV>::HP * sizeof(typename Tr::H) +
            (MODE != ACC_F64 ? sizeof(uint32_t) : 0));  // single-copy fine cells
}

// F_LO_PDF: the density grid (nx x nq FP64, row-major) padded by one knot on
// every side with the linear ghost values 2 f_edge - f_next (a corner: the
// ghost of the ghost row); knot (r, c) of the padded grid, 0 <= r < nx + 2,
// 0 <= c < nq + 2.
__device__ __forceinline__ double padded_knot(const double *g, int nx, int nq, int r, int c) {
    // the row (and column) of g and its neighbour the ghost extrapolates from
    const int ri = min(max(r - 1, 0), nx - 1), rn = r == 0 ? 1 : nx - 2;
    const int ci = min(max(c - 1, 0), nq - 1), cn = c == 0 ? 1 : nq - 2;
    const bool gr = r == 0 || r == nx + 1, gc = c == 0 || c == nq + 1;
    double v = g[ri * nq + ci];
    if (gr) v = 2.0 * v - g[rn * nq + ci];
    if (gc) {
        double w = g[ri * nq + cn];
        if (gr) w = 2.0 * w - g[rn * nq + cn];
        v = 2.0 * v - w;
    }
    return v;
}

// Bytes of the staged grid in the path's precision (mode): FP64 keeps the
// (nx + 2) x (nq + 2) padded knots; FP32 keeps (nx + 2) x (nq + 1) pairs
// (knot (r, c), knot (r, c + 1)), so that the four knots of a row that a
// bicubic lookup reads are two 8-byte loads (grid_xg), not four.
__host__ __device__ constexpr size_t pdf_grid_bytes(int mode, int nx, int nq) {
    return mode == ACC_F64 ? static_cast<size_t>(nx + 2) * (nq + 2) * sizeof(double)
                           : static_cast<size_t>(nx + 2) * (nq + 1) * 2 * sizeof(float);
}

// Offset of the staged grid after `before` bytes of shared memory (16-byte
// aligned: the FP32 pairs are read as 8-byte vectors).
__host__ __device__ constexpr size_t pdf_grid_offset(size_t before) { return (before + 15) / 16 * 16; }

// Stages the padded grid into t in the layout of pdf_grid_bytes for T; every
// thread of the block calls this, the caller synchronises.
template <class T>
__device__ __forceinline__ void stage_grid(T *t, const double *g, int nx, int nq) {
    if constexpr (sizeof(T) == sizeof(double)) {
        const int P = nq + 2;
        for (int k = threadIdx.x; k < (nx + 2) * P; k += blockDim.x) {
            const int r = k / P, c = k - r * P;
            t[k] = static_cast<T>(padded_knot(g, nx, nq, r, c));
        }
    } else {
        const int P = nq + 1;
        float2 *t2 = reinterpret_cast<float2 *>(t);
        for (int k = threadIdx.x; k < (nx + 2) * P; k += blockDim.x) {
            const int r = k / P, c = k - r * P;
            t2[k] = make_float2(static_cast<float>(padded_knot(g, nx, nq, r, c)),
                                static_cast<float>(padded_knot(g, nx, nq, r, c + 1)));
        }
    }
}

// F_LO_PDF: the padded density grid follows the block's cells in shared
// memory; every thread calls this after carve/stage.
template <int FAM, int MODE, int PRIV>
__device__ __forceinline__ const typename ModeTraits<MODE>::T *stage_pdf(unsigned char *raw, const SampleArgs &a,
                                                                          int d) {
    using T = typename ModeTraits<MODE>::T;
    if (FAM != F_LO_PDF) return nullptr;
    T *t = reinterpret_cast<T *>(raw + pdf_grid_offset(sample_smem_bytes<MODE, PRIV>(d, a.N)));
    stage_grid(t, a.pdf, a.pdf_nx, a.pdf_nq);
    return t;
}

// Samples one block may add to its fixed-point cells between two flushes:
// every bin is drawn with probability 1/N, so a coarse cell copy receives 64
// values on average, far below the 512 values at the largest coarse value
// (2^23) that would reach 2^32; a fine cell (one copy, values below 2^16)
// receives 64 HP on average.
constexpr long long kValuesPerCopy = 64;
template <int MODE, int PRIV> __host__ __device__ constexpr long long block_sample_cap(int N) {
    return kValuesPerCopy * N * Copies<MODE, PRIV>::HP;
}

__device__ __forceinline__ void red_add_shared(float *p, float v) { atomicAdd(p, v); }
__device__ __forceinline__ void red_add_shared(double *p, double v) { atomicAdd(p, v); }

__device__ __forceinline__ int binary_exponent(double x) {  // floor(log2 x) for x > 0 normal
    return static_cast<int>((__double_as_longlong(x) >> 52) & 0x7FF) - 1023;
}

// Scales for the next iteration from m2 and m1, the means of this iteration's
// scaled v^2 and v (0 if none): a power of two `ratio` that brings the mean of
// v^2 near 1 (FP32 keeps its full precision for v and v^2 whatever the size
// of the integral), limited so that the initial weight jinit * jmul * ratio
// stays within 2^-100..2^100, and the fixed-point histogram scale that maps
// the rescaled mean to 2^18.  The scale is used only where this iteration's
// m2 predicts the next one's: when m2 exceeds kSettled m1^2 (a relative
// variance per sample above 1023: the grid is far from adapted, or a few
// samples dominated the iteration), the next mean of v^2 may be orders of
// magnitude lower, and a scale fixed from m2 would leave its values a few
// integer units; the next iteration then keeps FP32 cells (hs = 0).
constexpr double kSettled = 1024.0;
__device__ __forceinline__ void next_scales(double m2, double m1, double jinit_eff, double *ratio, float *hs) {
    // exponents from the bits, not from FP64 log2 (a long chain on this GPU's FP64 pipe)
    double r = 1.0;
    float h = 0.f;
    if (m2 > 0.0 && isfinite(m2)) {
        const int ex = binary_exponent(m2);                  // m2 in [2^ex, 2^(ex+1))
        int e = -(ex >> 1);                                  // m2 r^2 in [1, 4)
        const double aj = fabs(jinit_eff);
        const int ej = (aj > 0.0 && isfinite(aj)) ? binary_exponent(aj) : 0;
        e = max(-100 - ej, min(100 - ej, e));
        e = max(-1000, min(1000, e));
        r = __longlong_as_double(static_cast<long long>(e + 1023) << 52);
        const double y = m2 * r * r;                         // exact (power-of-two factors)
        const long long yb = __double_as_longlong(y);
        const int cl = binary_exponent(y) + ((yb & 0xFFFFFFFFFFFFFLL) != 0 ? 1 : 0);  // ceil(log2 y)
        int eh = 18 - cl;
        eh = max(-100, min(100, eh));
        h = m2 <= kSettled * m1 * m1 ? __int_as_float((eh + 127) << 23) : 0.f;
    }
    *ratio = r;
    *hs = h;
}

// Warp-level FP64 sum.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Shared-memory working set of one block for one integral: the table (TP
// copies per cell), the coarse histogram cells (HP copies per cell) and, in
// the FP32 modes, one fine cell per (dimension, bin).
template <int MODE, int PRIV> struct BlockState {
    using Tr = ModeTraits<MODE>;
    using T = typename Tr::T;
    using T2 = typename Prec<T>::T2;
    using H = typename Tr::H;
    static constexpr int TP = Copies<MODE, PRIV>::TP;
    static constexpr int HP = Copies<MODE, PRIV>::HP;
    T2 *tab;
    H *hist;
    uint32_t *fine;
    int cells;

    __device__ __forceinline__ void carve(unsigned char *raw, int ncells) {
        cells = ncells;
        tab = reinterpret_cast<T2 *>(raw);
        hist = reinterpret_cast<H *>(raw + static_cast<size_t>(cells) * TP * sizeof(T2));
        fine = reinterpret_cast<uint32_t *>(hist + static_cast<size_t>(cells) * HP);
    }
    // Every thread of the block calls this; the caller synchronises after it.
    __device__ __forceinline__ void stage(const void *gtable) {
        const T2 *g = static_cast<const T2 *>(gtable);
        for (int k = threadIdx.x; k < cells * TP; k += blockDim.x) tab[k] = g[k / TP];
        clear();
    }
    // Zeroes the histogram cells (every thread calls; the caller synchronises).
    __device__ __forceinline__ void clear() {
        for (int k = threadIdx.x; k < cells * HP; k += blockDim.x) hist[k] = H(0);
        if (MODE != ACC_F64)
            for (int k = threadIdx.x; k < cells; k += blockDim.x) fine[k] = 0u;
    }
};

// Per-thread running sums of v and v^2 and the non-finite count.
template <int MODE> struct ThreadSums {
    double s1d = 0.0, s2d = 0.0;                     // ACC_F64, ACC_F32_SUM64
    float s1f = 0.f, c1f = 0.f, s2f = 0.f, c2f = 0.f;  // ACC_F32_KAHAN
    double qd = 0.0;                                 // stratified: sum of hypercube m2
    unsigned int nonfinite = 0;
};

// Scalars of one integral's iteration that the sampling loop needs.
template <class T> struct RangeParams {
    int d, N;
    uint32_t key0, key1, iter;
    T jinit, n4;
    float hs;        // fixed-point scale of v^2 (FP32 modes); 0: FP32 cells
    double *acc;     // FP64 accumulators [2 + d N] (values beyond the fixed range)
    const T *aux = nullptr;  // F_LO_PDF: the density grid in shared memory
};

// Cell indices of one sample's dimensions, one per register or, with PACK,
// two 16-bit indices per register (d N <= 32768): half the registers for one
// more operation per dimension.
template <int MAXD, bool PACK> struct SampleCells {
    uint32_t c[PACK ? (MAXD + 1) / 2 : MAXD];
    __device__ __forceinline__ void set(int j, uint32_t cell) {
        if (!PACK) c[j] = cell;
        else if (j & 1) c[j >> 1] = __byte_perm(c[j >> 1], cell, 0x5410);
        else c[j >> 1] = cell;
    }
    __device__ __forceinline__ uint32_t get(int j) const {
        if (!PACK) return c[j];
        return (j & 1) ? (c[j >> 1] >> 16) : (c[j >> 1] & 0xFFFFu);
    }
};

// Grid map and integrand of sample s: its Philox words (placed in hypercube
// h's strata when STRAT), each dimension's cell (recorded in cellj) and
// v = J f.  CHECK: v is set to 0 and counted in nonfinite when it is not
// finite, or, in FP32, when v^2 is not (CHECK false: the caller tests, see
// hist_add_fixed).
template <int FAM, int MODE, int MAXD, bool EXACT, int PRIV, bool PACK, bool STRAT, bool CHECK = true>
__device__ __forceinline__ typename ModeTraits<MODE>::T map_sample(
    const typename BlockState<MODE, PRIV>::T2 *tab_l, const RangeParams<typename ModeTraits<MODE>::T> &rp,
    const FamConsts<typename ModeTraits<MODE>::T> &fc, const StratArgs *st, uint32_t h,
    unsigned long long s, SampleCells<MAXD, PACK> &cellj, unsigned int &nonfinite) {
    using BS = BlockState<MODE, PRIV>;
    using T = typename BS::T;
    using T2 = typename BS::T2;
    constexpr int TP = BS::TP;
    const int d = EXACT ? MAXD : rp.d;
    const int N = rp.N;
    const uint32_t slo = static_cast<uint32_t>(s), shi = static_cast<uint32_t>(s >> 32);
    Integrand<FAM, T, MAXD> fam;
    if (FAM == F_LO_PDF) fam.tbl = rp.aux;
    T J = rp.jinit;
    fam.begin(fc);
#pragma unroll
    for (int q = 0; q < (MAXD + 3) / 4; ++q) {
        if (EXACT || 4 * q < d) {
            const uint4 r = philox4x32_10(make_uint4(slo, shi, rp.iter, static_cast<uint32_t>(q)),
                                          rp.key0, rp.key1);
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const int j = 4 * q + w;
                if (j < MAXD && (EXACT || j < d)) {
                    uint32_t rw = word(r, w);
                    if (STRAT) rw = strat_word(rw, h, st->off[j], st->bits[j]);
                    const Split sp = split_bin(rw, static_cast<uint32_t>(N));
                    const uint32_t cell = static_cast<uint32_t>(j * N) + sp.bin;
                    const T2 ent = tab_l[cell * TP];
                    const T x = Prec<T>::coord(ent, sp.lo);
                    J *= ent.y;
                    if (sizeof(T) == 4 && (j & 3) == 3) J *= rp.n4;
                    cellj.set(j, cell);
                    fam.dim(j, x, fc);
                }
            }
        }
    }
    T v = J * fam.finish(fc);
    if (CHECK && !isfinite(sizeof(T) == 4 ? v * v : v)) {
        v = T(0);
        ++nonfinite;
    }
    return v;
}

// Adds v2 = v^2 to the histogram cell of each of the sample's dimensions (the
// cell arrays and fixed-point rules above).
template <int MODE, int PRIV, int MAXD, bool EXACT, bool PACK>
__device__ __forceinline__ void hist_add(const BlockState<MODE, PRIV> &bs, typename BlockState<MODE, PRIV>::H *hist_l,
                                         const RangeParams<typename ModeTraits<MODE>::T> &rp,
                                         const SampleCells<MAXD, PACK> &cellj, typename ModeTraits<MODE>::T v2,
                                         bool fixed, float hs) {
    using BS = BlockState<MODE, PRIV>;
    using T = typename BS::T;
    using H = typename BS::H;
    constexpr int HP = BS::HP;
    const int d = EXACT ? MAXD : rp.d;
    if (MODE == ACC_F64) {
#pragma unroll
        for (int j = 0; j < MAXD; ++j) {
            if (EXACT || j < d) red_add_shared(hist_l + cellj.get(j) * HP, static_cast<H>(v2));
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
            unsigned int *base = is_fine ? bs.fine : reinterpret_cast<unsigned int *>(hist_l);
            const uint32_t step = is_fine ? 1u : static_cast<uint32_t>(HP);
#pragma unroll
            for (int j = 0; j < MAXD; ++j) {
                if (EXACT || j < d) atomicAdd(base + cellj.get(j) * step, q);
            }
        } else {
#pragma unroll
            for (int j = 0; j < MAXD; ++j) {
                if (EXACT || j < d) atomicAdd(rp.acc + 2 + cellj.get(j), static_cast<double>(v2));
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < MAXD; ++j) {
            if (EXACT || j < d) red_add_shared(reinterpret_cast<float *>(hist_l) + cellj.get(j) * HP,
                                               static_cast<float>(v2));
        }
    }
}

// The fixed-point update of hist_add (FP32 modes, scale hs > 0) for a v that
// map_sample did not test: a NaN or infinite v^2 fails qf < 2^23 as well, so
// the test sits in that rare branch, which counts such a sample in nonfinite
// and zeroes v and v2 (the caller adds them to the sums afterwards).  Saves
// the per-sample test of the common path.
template <int MODE, int PRIV, int MAXD, bool EXACT, bool PACK>
__device__ __forceinline__ void hist_add_fixed(const BlockState<MODE, PRIV> &bs, typename BlockState<MODE, PRIV>::H *hist_l,
                                               const RangeParams<float> &rp, const SampleCells<MAXD, PACK> &cellj,
                                               float &v, float &v2, float hs, unsigned int &nonfinite) {
    constexpr int HP = BlockState<MODE, PRIV>::HP;
    const int d = EXACT ? MAXD : rp.d;
    if (v2 == 0.f) return;
    const float qf = v2 * hs;
    if (qf < kFixedMax) {
        const bool is_fine = qf < 1.0f;
        const float t = __fmaf_rn(qf, is_fine ? kFineScale : 1.0f, 8388608.0f);
        uint32_t q = __float_as_uint(t) - 0x4B000000u;
        q = max(q, 1u);
        unsigned int *base = is_fine ? bs.fine : reinterpret_cast<unsigned int *>(hist_l);
        const uint32_t step = is_fine ? 1u : static_cast<uint32_t>(HP);
#pragma unroll
        for (int j = 0; j < MAXD; ++j) {
            if (EXACT || j < d) atomicAdd(base + cellj.get(j) * step, q);
        }
    } else if (isfinite(v2)) {
#pragma unroll
        for (int j = 0; j < MAXD; ++j) {
            if (EXACT || j < d) atomicAdd(rp.acc + 2 + cellj.get(j), static_cast<double>(v2));
        }
    } else {
        v = 0.f;
        v2 = 0.f;
        ++nonfinite;
    }
}

// Kahan step of the FP32-compensated sums of v and v^2.
template <int MODE>
__device__ __forceinline__ void kahan_add(ThreadSums<MODE> &ts, float v, float v2) {
    const float y1 = v - ts.c1f;
    const float t1 = ts.s1f + y1;
    ts.c1f = (t1 - ts.s1f) - y1;
    ts.s1f = t1;
    const float y2 = v2 - ts.c2f;
    const float t2 = ts.s2f + y2;
    ts.c2f = (t2 - ts.s2f) - y2;
    ts.s2f = t2;
}

// The block samples [s0, s0 + cnt) of one integral: thread t takes
// s0 + t + u * blockDim, in chunks of kChunk samples (ACC_F32_SUM64 adds a
// chunk's FP32 partial sums into the FP64 sums once per chunk: 16 samples,
// a relative error of at most about 1e-6 per partial; half the FP64
// instructions of 8-sample chunks ran the d = 8 headline 1% faster).
// EXACT: the dimension equals MAXD (no per-dimension guards); otherwise
// 1 <= rp.d <= MAXD at run time.  PACK: 16-bit cell indices (SampleCells).
// FOLD (FP32 modes with fixed-point cells): the non-finite test in the
// histogram update's rare branch (hist_add_fixed) and the sums after it;
// otherwise the test in map_sample and hist_add's general form.  WIDE: the
// block's samples may cross a multiple of 2^32, so each sample index is a
// 64-bit sum; otherwise its high word is the block's own.
template <int FAM, int MODE, int MAXD, bool EXACT, int PRIV, bool PACK, bool FOLD, bool WIDE = true>
__device__ __forceinline__ void sample_loop(const BlockState<MODE, PRIV> &bs,
                                            const RangeParams<typename ModeTraits<MODE>::T> &rp,
                                            const FamConsts<typename ModeTraits<MODE>::T> &fc,
                                            ThreadSums<MODE> &ts, unsigned long long s0, int cnt) {
    using BS = BlockState<MODE, PRIV>;
    using T = typename BS::T;
    using T2 = typename BS::T2;
    using H = typename BS::H;
    constexpr int TP = BS::TP;
    constexpr int HP = BS::HP;
    const int lane = threadIdx.x & 31;
    const T2 *tab_l = bs.tab + (lane % TP);
    H *hist_l = bs.hist + (lane % HP);
    const float hs = rp.hs;
    const bool fixed = hs > 0.f;

    constexpr int kChunk = 16;
    const int stride = blockDim.x;
    for (int k0 = threadIdx.x; k0 < cnt; k0 += kChunk * stride) {
        float p1 = 0.f, p2 = 0.f;
        // two samples in flight (their Philox and table-load chains
        // interleave), one above 8 dimensions (register budget: the batched
        // samplers at 80 registers run the 512-integral mix 1.7% faster)
#pragma unroll(MAXD > 8 ? 1 : 2)
        for (int u = 0; u < kChunk; ++u) {
            const int k = k0 + u * stride;
            if (k >= cnt) break;
            const unsigned long long s =
                WIDE ? s0 + static_cast<unsigned long long>(k)
                     : (s0 & 0xFFFFFFFF00000000ull) |
                           static_cast<uint32_t>(static_cast<uint32_t>(s0) + static_cast<uint32_t>(k));
            SampleCells<MAXD, PACK> cellj;
            T v = map_sample<FAM, MODE, MAXD, EXACT, PRIV, PACK, false, !FOLD>(tab_l, rp, fc, nullptr, 0u, s, cellj,
                                                                             ts.nonfinite);
            T v2 = v * v;
            if constexpr (FOLD) hist_add_fixed<MODE, PRIV, MAXD, EXACT, PACK>(bs, hist_l, rp, cellj, v, v2, hs,
                                                                              ts.nonfinite);
            if (MODE == ACC_F32_KAHAN) {
                kahan_add(ts, static_cast<float>(v), static_cast<float>(v2));
            } else if (MODE == ACC_F32_SUM64) {
                p1 += static_cast<float>(v);
                p2 += static_cast<float>(v2);
            } else {
                const double vd = static_cast<double>(v);
                ts.s1d += vd;
                ts.s2d = __fma_rn(vd, vd, ts.s2d);
            }
            if constexpr (!FOLD) hist_add<MODE, PRIV, MAXD, EXACT, PACK>(bs, hist_l, rp, cellj, v2, fixed, hs);
        }
        if (MODE == ACC_F32_SUM64) {
            ts.s1d += static_cast<double>(p1);
            ts.s2d += static_cast<double>(p2);
        }
    }
}

// Families whose single-integral kernel also takes a loop without the
// 64-bit index sum (sample_loop's WIDE = false) when the block's samples stay
// below a multiple of 2^32: measured 1-3% faster for the d = 8 Gaussian,
// oscillatory and product-peak integrals, the LO toy and d = 2..12, but
// 1.5% and 2% slower for the Genz Gaussian and corner-peak integrals.
template <int FAM> constexpr bool kNarrowIndex = FAM != F_GENZ_GAUSS && FAM != F_GENZ_CORNER;

// sample_loop in the form the iteration's cells take: FOLD where the FP32
// cells hold fixed-point integers (every iteration after the first), and
// there, with NARROW, the block-uniform high word of the sample index where
// the family takes it and the block's range allows it.
template <int FAM, int MODE, int MAXD, bool EXACT, int PRIV, bool PACK = false, bool NARROW = kNarrowIndex<FAM>>
__device__ __forceinline__ void sample_range(const BlockState<MODE, PRIV> &bs,
                                             const RangeParams<typename ModeTraits<MODE>::T> &rp,
                                             const FamConsts<typename ModeTraits<MODE>::T> &fc,
                                             ThreadSums<MODE> &ts, unsigned long long s0, int cnt) {
    if constexpr (MODE != ACC_F64) {
        if (rp.hs > 0.f) {
            if constexpr (NARROW) {
                if ((s0 & 0xFFFFFFFFull) + static_cast<unsigned long long>(cnt) <= 0x100000000ull) {
                    sample_loop<FAM, MODE, MAXD, EXACT, PRIV, PACK, true, false>(bs, rp, fc, ts, s0, cnt);
                    return;
                }
            }
            sample_loop<FAM, MODE, MAXD, EXACT, PRIV, PACK, true>(bs, rp, fc, ts, s0, cnt);
            return;
        }
    }
    sample_loop<FAM, MODE, MAXD, EXACT, PRIV, PACK, false>(bs, rp, fc, ts, s0, cnt);
}

// Adds the block's sums to the integral's FP64 accumulators: S1, S2 and the
// non-finite count by a block reduction, each histogram cell by one thread.  Starts
// with a barrier (every thread's samples are in) and ends with one (the
// shared cells may be reused).  Resets ts.
// q (stratified launches, else null): FP64 accumulator of the hypercube m2 sums.
// table_free: the caller reads the staged table no more (the end of a launch,
// or a re-stage next), so its shared memory may hold the block's partial sums.
template <int MODE, int PRIV>
__device__ __forceinline__ void flush_block(const BlockState<MODE, PRIV> &bs, ThreadSums<MODE> &ts,
                                            float hs, double *acc, unsigned long long *n_nonfinite,
                                            double *q = nullptr, bool table_free = false) {
    using BS = BlockState<MODE, PRIV>;
    using H = typename BS::H;
    using T2 = typename BS::T2;
    constexpr int HP = BS::HP;
    constexpr int TP = BS::TP;
    __shared__ double red1[32], red2[32], redq[32];
    __shared__ unsigned int rednf[32];
    __shared__ double inv_s[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthr = blockDim.x, nwarps = nthr >> 5;
    const bool fixed = hs > 0.f;
    double b1, b2;
    if (MODE == ACC_F32_KAHAN) {
        b1 = static_cast<double>(ts.s1f) - static_cast<double>(ts.c1f);
        b2 = static_cast<double>(ts.s2f) - static_cast<double>(ts.c2f);
    } else {
        b1 = ts.s1d;
        b2 = ts.s2d;
    }
    double bq = ts.qd;
    const unsigned int nf = __reduce_add_sync(0xFFFFFFFFu, ts.nonfinite);
    ts = ThreadSums<MODE>();
    // A warp's FP64 instruction holds its scheduler's FP64 unit for about 76
    // cycles on this GPU, and every block flushes at the same moment at the end
    // of a launch.  So the FP64 scalars are formed once per block, and, where the
    // table copies are no longer needed, the block sums take a shared-memory
    // tree (each level half the warps of the one before: 40 FP64 warp
    // instructions for two sums of 512) instead of a shuffle tree in every warp
    // (170).
    const int nsum = q ? 3 : 2;
    const bool tree = table_free && nthr >= 64 && (nthr & (nthr - 1)) == 0 &&
                      static_cast<size_t>(bs.cells) * TP * sizeof(T2) >=
                          static_cast<size_t>(nsum) * nthr * sizeof(double);
    __syncthreads();  // every thread's samples are in
    if (tid == 0) {
        inv_s[0] = fixed ? 1.0 / static_cast<double>(hs) : 0.0;
        inv_s[1] = inv_s[0] * static_cast<double>(kFineInv);
    }
    if (lane == 0) rednf[warp] = nf;
    if (tree) {
        double *part = reinterpret_cast<double *>(bs.tab);
        part[tid] = b1;
        part[nthr + tid] = b2;
        if (q) part[2 * nthr + tid] = bq;
        __syncthreads();
        for (int h = nthr >> 1; h >= 32; h >>= 1) {
            const int lh = __ffs(h) - 1;
            for (int t = tid; t < nsum * h; t += nthr) {
                double *p = part + (t >> lh) * nthr + (t & (h - 1));
                p[0] += p[h];
            }
            __syncthreads();
        }
        if (warp < nsum) {
            const double x = warp_sum(part[warp * nthr + lane]);
            if (lane == 0) atomicAdd(warp == 2 ? q : acc + warp, x);
        }
    } else {
        b1 = warp_sum(b1);
        b2 = warp_sum(b2);
        if (q) bq = warp_sum(bq);
        if (lane == 0) {
            red1[warp] = b1;
            red2[warp] = b2;
            redq[warp] = bq;
        }
        __syncthreads();
        if (warp == 0) {
            const double x1 = warp_sum(lane < nwarps ? red1[lane] : 0.0);
            const double x2 = warp_sum(lane < nwarps ? red2[lane] : 0.0);
            if (q) {
                const double xq = warp_sum(lane < nwarps ? redq[lane] : 0.0);
                if (lane == 0) atomicAdd(q, xq);
            }
            if (lane == 0) {
                atomicAdd(acc + 0, x1);
                atomicAdd(acc + 1, x2);
            }
        }
    }
    if (warp == nwarps - 1) {
        const unsigned int xn = __reduce_add_sync(0xFFFFFFFFu, lane < nwarps ? rednf[lane] : 0u);
        if (lane == 0 && xn) atomicAdd(n_nonfinite, static_cast<unsigned long long>(xn));
    }
    // One thread per cell sums the cell's HP copies, reading them from copy
    // c mod HP on so that the lanes of a warp touch distinct banks.
    // Fixed-point copies and the fine cell are summed exactly as one integer
    // (the coarse cells count units of 1/hs, the fine cell units of 2^-16/hs;
    // below 2^53 + 2^32) and scaled once; floating-point copies pairwise.
    const double inv_fine = inv_s[1];
    for (int c = tid; c < bs.cells; c += nthr) {
        double h;
        if (MODE != ACC_F64 && fixed) {
            const unsigned int *hu = reinterpret_cast<const unsigned int *>(bs.hist) + c * HP;
            unsigned long long qs = 0;
#pragma unroll
            for (int k = 0; k < HP; ++k) qs += hu[(k + c) & (HP - 1)];
            h = static_cast<double>((qs << kFineShift) + bs.fine[c]) * inv_fine;
        } else {
            // pairwise: the rounding of a tree of log2(HP) levels
            const H *hc = bs.hist + c * HP;
            H a[HP];
#pragma unroll
            for (int k = 0; k < HP; ++k) a[k] = hc[(k + c) & (HP - 1)];
#pragma unroll
            for (int w = HP / 2; w >= 1; w >>= 1)
#pragma unroll
                for (int k = 0; k < w; ++k) a[k] += a[k + w];
            h = static_cast<double>(a[0]);
        }
        if (h != 0.0) atomicAdd(acc + 2 + c, h);
    }
    __syncthreads();
}

// The iteration's scalars every thread needs, the v-rescaled Jacobian factor
// and N^4, formed by thread 0 (FP64 arithmetic issues at 1.68 lanes per clock
// per SM here): scal[0..1] after the caller's next barrier.
template <class T> __device__ __forceinline__ void block_scalars(const SampleArgs &a, T *scal) {
    if (threadIdx.x == 0) {
        scal[0] = static_cast<T>(a.jinit * (a.jmul ? *a.jmul : 1.0));
        scal[1] = static_cast<T>(a.nblk4);
    }
}

// Blocks of 512 threads an SM should hold, which sets the registers the
// compiler may give a thread: the LO toy at 2 (64 registers: its short
// integrand chain wants the warps; measured 6-8% faster than at one block),
// every other kernel at 1 (up to 128 registers: fewer instructions per
// sample; the d = 8 families ran 2.4-6.4% faster, d = 12 8%, the FP64 d = 4
// iteration of 1e5 samples 14%).  The density-grid family's paired grid
// (pdf_grid_bytes) leaves room for one block anyway; with 116 registers it ran
// 7% faster than the single-knot grid at two blocks of 64.
template <int FAM> constexpr int kSampleMinBlocks = FAM == F_LO ? 2 : 1;

// One integral, samples [a.s_begin, a.s_begin + a.n): each block takes a
// contiguous range of them.
// WIDEH (FP64 path, layout PRIV = 1 only): one histogram copy per lane
// (kLayoutWide) instead of one per lane pair, so that no two lanes of a warp
// update the same FP64 cell and its compare-and-swap loop never retries
// within a warp (lanes l and l + 16 of a pair hit the same cell with
// probability 1/N per dimension: 38% of the warp instructions retried at d = 8,
// N = 50); the flush then sums twice the copies, so the host takes it for
// iterations of many samples per block only.
template <int FAM, int MODE, int MAXD, bool EXACT, bool PRIV, bool WIDEH = false>
__global__ void __launch_bounds__(512, kSampleMinBlocks<FAM>)
vegas_sample_kernel(const SampleArgs a) {
    pdl_begin();
    constexpr int LAY = WIDEH ? kLayoutWide : (PRIV ? 1 : 0);
    using BS = BlockState<MODE, LAY>;
    using T = typename BS::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int d = EXACT ? MAXD : a.d;
    BS bs;
    bs.carve(smem_raw, d * a.N);
    bs.stage(a.table);
    RangeParams<T> rp;
    rp.aux = stage_pdf<FAM, MODE, LAY>(smem_raw, a, d);
    rp.d = d;
    rp.N = a.N;
    rp.key0 = a.key0;
    rp.key1 = a.key1;
    rp.iter = a.iter;
    __shared__ T scal[2];
    block_scalars(a, scal);
    rp.hs = (MODE != ACC_F64) ? *a.hscale : 0.f;
    rp.acc = a.acc;
    __syncthreads();
    rp.jinit = scal[0];
    rp.n4 = scal[1];

    const long long per = (a.n + gridDim.x - 1) / gridDim.x;
    const long long lo = static_cast<long long>(blockIdx.x) * per;
    const long long hi = min(a.n, lo + per);
    ThreadSums<MODE> ts;
    if (hi > lo)
        sample_range<FAM, MODE, MAXD, EXACT, LAY>(bs, rp, consts<T>(a), ts,
                                                   static_cast<unsigned long long>(a.s_begin + lo),
                                                   static_cast<int>(hi - lo));
    flush_block<MODE, LAY>(bs, ts, rp.hs, a.acc, a.n_nonfinite, nullptr, true);
}

}  // namespace vegas
