// vegas_device.cuh -- device building blocks of one VEGAS iteration on sm_103a.
//
// The iteration (VEGAS, Lepage 1978/1980; the method of the paper, Sec. 1):
// per sample draw d uniforms, find each uniform's bin, interpolate inside the
// bin, multiply the per-dimension Jacobian factors, evaluate the integrand and
// accumulate v = J f, v^2 and the per-bin histograms of v^2.
//
// Everything a sample needs lives in registers: the Philox words are drawn,
// split and consumed without touching memory.  The grid table and the
// histograms live in shared memory.
#pragma once

#ifdef __CUDACC_RTC__
// Run-time compilation (NVRTC, user integrands) has no standard headers: the
// fixed-width integer types the kernels use.
typedef unsigned int uint32_t;
typedef int int32_t;
typedef unsigned long long uint64_t;
typedef long long int64_t;
typedef unsigned long size_t;
#else
#include <cstdint>
#include <cuda_runtime.h>
#endif

// The user integrand of the F_USER family: defined, at global scope, by the
// source passed to vegas_create_user and compiled with these headers at run
// time.  x: the d mapped coordinates, p: the parameters, in the path's
// precision T (float in the FP32 modes, double in the FP64 mode).
template <class T> __device__ T user_integrand(const T *x, int d, const T *p);

namespace vegas {

// ------------------------------------------------- programmatic launch
// The sampling kernels are launched with programmatic stream serialisation:
// such a launch may be scheduled once every block of the kernel before it has
// passed pdl_begin (or exited), and its blocks wait in pdl_begin until that
// grid has completed and its writes are visible.  So the next kernel's launch
// and block dispatch overlap this one's tail.  A kernel that calls pdl_begin
// reads nothing an earlier launch wrote before it; launched without the
// attribute, the wait returns at once.
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies and
// xors, with the key advanced by the Weyl constants between rounds.
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = static_cast<uint64_t>(kPhiloxM0) * c.x;
        const uint64_t p1 = static_cast<uint64_t>(kPhiloxM1) * c.z;
        const uint32_t rk0 = k0 + static_cast<uint32_t>(r) * kPhiloxW0;
        const uint32_t rk1 = k1 + static_cast<uint32_t>(r) * kPhiloxW1;
        c = make_uint4(static_cast<uint32_t>(p1 >> 32) ^ c.y ^ rk0, static_cast<uint32_t>(p1),
                       static_cast<uint32_t>(p0 >> 32) ^ c.w ^ rk1, static_cast<uint32_t>(p0));
    }
    return c;
}

__device__ __forceinline__ uint32_t word(const uint4 &r, int k) {
    return k == 0 ? r.x : (k == 1 ? r.y : (k == 2 ? r.z : r.w));
}

// ------------------------------------------------------------ bin split
// y N with y = r 2^-32 is split with one 32x32->64 integer multiply: the high
// word is the bin, the low word the in-bin position.  Bins are therefore the
// same integers in every precision.  The in-bin position becomes x with a
// single fused multiply-add from the bin's table entry (Prec<T>::coord).
struct Split {
    uint32_t bin;
    uint32_t lo;
};

__device__ __forceinline__ Split split_bin(uint32_t r, uint32_t N) {
    const uint64_t t = static_cast<uint64_t>(r) * N;
    return Split{static_cast<uint32_t>(t >> 32), static_cast<uint32_t>(t)};
}

// FP32: the low word rounded to the nearest float (one conversion, relative
// error at most 2^-24, the same issue cost as a funnel shift on this GPU).
// Truncating it to a 23-bit fraction instead would leave an error of up to
// 2^-23 of the bin width, which is a large relative error for points near a
// bin's lower end at 0 (x << w), where integrands such as x^-1/2 live.
__device__ __forceinline__ float low_word_f32(uint32_t lo) {
    float f;
    asm("cvt.rn.f32.u32 %0, %1;" : "=f"(f) : "r"(lo));
    return f;
}

// FP64: m = 1 + lo 2^-32, exact (all 32 bits fit in the 52-bit mantissa).
__device__ __forceinline__ double unit_mantissa_f64(uint32_t lo) {
    return __hiloint2double(static_cast<int>(0x3FF00000u | (lo >> 12)), static_cast<int>(lo << 20));
}

// Coordinates and table entries per precision.
//   FP64: entry (e - w, w) of a bin [e, e + w); x = (e - w) + w m, m = 1 + lo 2^-32.
//   FP32: the path works in X = 2^32 x (kXS): entry (2^32 e, w);
//         X = 2^32 e + w float(lo).  The power of two is folded into each
//         family's FP32 constants (and, where it remains a constant factor of
//         f, into the initial weight), so the integrands cost what they cost
//         in x.  Every sample's X carries a relative error of a few 2^-24.
template <class T> struct Prec;
template <> struct Prec<float> {
    using T2 = float2;
    static constexpr float kXS = 4294967296.0f;            // 2^32
    static constexpr float kInvXS = 2.3283064365386963e-10f;  // 2^-32
    __device__ static __forceinline__ float coord(float2 ent, uint32_t lo) {
        return __fmaf_rn(ent.y, low_word_f32(lo), ent.x);
    }
};
template <> struct Prec<double> {
    using T2 = double2;
    static constexpr double kXS = 1.0;
    static constexpr double kInvXS = 1.0;
    __device__ static __forceinline__ double coord(double2 ent, uint32_t lo) {
        return __fma_rn(ent.y, unit_mantissa_f64(lo), ent.x);
    }
};

// ----------------------------------------------------------- integrands
// Family ids match vegas_family in vegas.h.
enum Family : int {
    F_CONST = 0,
    F_SUM = 1,
    F_GAUSS_SYM = 2,
    F_GENZ_OSC = 3,
    F_GENZ_GAUSS = 4,
    F_GENZ_PROD = 5,
    F_GENZ_CORNER = 6,
    F_LO = 7,
    F_USER = 8,   // user source, compiled at run time (vegas_create_user)
    F_LO_PDF = 9  // LO toy with its density from a tabulated grid (vegas_set_pdf_grid)
};




// Per-integral constants a family needs, prepared on the host in FP64 and
// passed to the kernels in both precisions:
//   p[j], q[j] per dimension (meaning per family below), s[0..7] scalars.
// The kernels read them straight from the kernel-parameter space with
// compile-time indices (after unrolling), so the FP32 path never converts
// an FP64 constant per sample.
template <class T> struct FamConsts {
    T p[32];
    T q[32];
    T s[8];
};
using FamilyConsts = FamConsts<double>;

// Centre of dimension j's sampling-table coordinate (store_table): 1/2 for
// GAUSS_SYM, the peak position q_j for GENZ_GAUSS and GENZ_PROD, else 0.
__host__ __device__ inline double table_center(int family, const FamConsts<double> &fc, int j) {
    if (family == F_GAUSS_SYM) return 0.5;
    if (family == F_GENZ_GAUSS || family == F_GENZ_PROD) return fc.q[j];
    return 0.0;
}

// Precision-typed helpers: the float versions must never promote to FP64
// (GB300's FP64 pipe issues 2 operations per clock per SM).
__device__ __forceinline__ float ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double ffma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fabs_t(float x) { return fabsf(x); }
__device__ __forceinline__ double fabs_t(double x) { return fabs(x); }
// 2^x for the FP32 path: the hardware approximation (relative error about
// 2^-22), results below the normal range flushed to zero.
__device__ __forceinline__ float fexp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// 2^x for the FP64 path, from the table-driven method of P. T. P. Tang
// ("Table-driven implementation of the exponential function in IEEE
// floating-point arithmetic", ACM Trans. Math. Softw. 15 (1989) 144):
// x = m + j/64 + r with integers m, j (0 <= j < 64) and |r| <= 1/128, so
// 2^x = 2^m 2^(j/64) 2^r; 2^(j/64) comes from a table, 2^r from its Taylor
// series 1 + sum_n (r ln 2)^n / n! to n = 5 (the first term left out is below
// 4e-17 relative), and 2^m goes into the exponent field.  9 FP64 operations
// in the normal range against the library exp2's 17 DFMA-equivalents; within
// 2 ulp of it (tests/cuda/exp2_check.cu compares the two), with the same
// subnormal results, 0, infinity and NaN outside the normal range.
// kExp2Tab[j] = 2^(j/64) and kExp2Taylor[n-1] = (ln 2)^n / n!, each rounded to
// the nearest double (exact decimal arithmetic; tests/test_oracle_pins.py
// recomputes them).
__device__ const double kExp2Tab[64] = {
    0x1.0000000000000p+0, 0x1.02c9a3e778061p+0, 0x1.059b0d3158574p+0, 0x1.0874518759bc8p+0,
    0x1.0b5586cf9890fp+0, 0x1.0e3ec32d3d1a2p+0, 0x1.11301d0125b51p+0, 0x1.1429aaea92de0p+0,
    0x1.172b83c7d517bp+0, 0x1.1a35beb6fcb75p+0, 0x1.1d4873168b9aap+0, 0x1.2063b88628cd6p+0,
    0x1.2387a6e756238p+0, 0x1.26b4565e27cddp+0, 0x1.29e9df51fdee1p+0, 0x1.2d285a6e4030bp+0,
    0x1.306fe0a31b715p+0, 0x1.33c08b26416ffp+0, 0x1.371a7373aa9cbp+0, 0x1.3a7db34e59ff7p+0,
    0x1.3dea64c123422p+0, 0x1.4160a21f72e2ap+0, 0x1.44e086061892dp+0, 0x1.486a2b5c13cd0p+0,
    0x1.4bfdad5362a27p+0, 0x1.4f9b2769d2ca7p+0, 0x1.5342b569d4f82p+0, 0x1.56f4736b527dap+0,
    0x1.5ab07dd485429p+0, 0x1.5e76f15ad2148p+0, 0x1.6247eb03a5585p+0, 0x1.6623882552225p+0,
    0x1.6a09e667f3bcdp+0, 0x1.6dfb23c651a2fp+0, 0x1.71f75e8ec5f74p+0, 0x1.75feb564267c9p+0,
    0x1.7a11473eb0187p+0, 0x1.7e2f336cf4e62p+0, 0x1.82589994cce13p+0, 0x1.868d99b4492edp+0,
    0x1.8ace5422aa0dbp+0, 0x1.8f1ae99157736p+0, 0x1.93737b0cdc5e5p+0, 0x1.97d829fde4e50p+0,
    0x1.9c49182a3f090p+0, 0x1.a0c667b5de565p+0, 0x1.a5503b23e255dp+0, 0x1.a9e6b5579fdbfp+0,
    0x1.ae89f995ad3adp+0, 0x1.b33a2b84f15fbp+0, 0x1.b7f76f2fb5e47p+0, 0x1.bcc1e904bc1d2p+0,
    0x1.c199bdd85529cp+0, 0x1.c67f12e57d14bp+0, 0x1.cb720dcef9069p+0, 0x1.d072d4a07897cp+0,
    0x1.d5818dcfba487p+0, 0x1.da9e603db3285p+0, 0x1.dfc97337b9b5fp+0, 0x1.e502ee78b3ff6p+0,
    0x1.ea4afa2a490dap+0, 0x1.efa1bee615a27p+0, 0x1.f50765b6e4540p+0, 0x1.fa7c1819e90d8p+0,
};
__device__ const double kExp2Taylor[5] = {0x1.62e42fefa39efp-1, 0x1.ebfbdff82c58fp-3, 0x1.c6b08d704a0c0p-5, 0x1.3b2ab6fba4e77p-7, 0x1.5d87fe78a6731p-10};

// 2^(j/64) 2^r for k = rint(64 x) = 64 m + j (the steps above); *m = floor(k / 64).
__device__ __forceinline__ double exp2_core(double x, int *m) {
    const double kShift = 6755399441055744.0;           // 1.5 * 2^52: rounds 64 x to an integer
    const double t = __fma_rn(x, 64.0, kShift);
    const int k = __double2loint(t);                    // rint(64 x)
    const double r = __fma_rn(t - kShift, -0.015625, x);  // x - k/64, exact
    double p = kExp2Taylor[4];
    p = __fma_rn(p, r, kExp2Taylor[3]);
    p = __fma_rn(p, r, kExp2Taylor[2]);
    p = __fma_rn(p, r, kExp2Taylor[1]);
    p = __fma_rn(p, r, kExp2Taylor[0]);                  // (2^r - 1) / r
    const double tj = __ldg(&kExp2Tab[k & 63]);
    *m = k >> 6;
    return __fma_rn(tj * r, p, tj);                      // in [0.99, 1.99)
}

__device__ __forceinline__ double fexp2(double x) {
    // results in the normal range for -1021 <= x <= 1023, tested on the high
    // word with integer operations (the FP64 pipe bounds this path); 2^m then
    // goes straight into the exponent field
    const int hx = __double2hiint(x);
    const bool normal = hx >= 0 ? hx <= 0x408FF800 : (hx & 0x7FFFFFFF) <= 0x408FE800;  // 1023, 1021
    int m;
    if (normal) {
        const double y = exp2_core(x, &m);
        return __hiloint2double(__double2hiint(y) + (m << 20), __double2loint(y));
    }
    // NaN; otherwise scale in two steps, the second rounding to a subnormal
    // result, to 0 (below 2^-1080) or to infinity (from 2^1024 up)
    if (x != x) return x;
    const double y = exp2_core(fmin(fmax(x, -1080.0), 1025.0), &m);
    const bool up = m > 0;
    return __hiloint2double(__double2hiint(y) + ((up ? m - 64 : m + 64) << 20), __double2loint(y)) *
           (up ? 18446744073709551616.0 : 5.421010862427522e-20);  // 2^64, 2^-64
}
// log2 x for the FP32 path: the hardware approximation (absolute error about
// 2^-22), subnormal arguments flushed to zero.
__device__ __forceinline__ float flog2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double flog2(double x) { return log2(x); }
// FP32 cosine for moderate arguments: reduce by 2 pi with a two-part constant
// (Cody & Waite, "Software Manual for the Elementary Functions", 1980):
// 2 pi = C1 + C2, C1 = the float nearest 2 pi, C2 = 2 pi - C1; the nearest
// multiple k comes from adding and subtracting 1.5 * 2^23 (valid for
// |x| < 2^22 * 2 pi).  The reduced argument lies in [-pi, pi], where the
// hardware approximation __cosf has an absolute error below 2^-21.
__device__ __forceinline__ float fcos(float x) {
    const float kInv2Pi = 0.159154943091895336f;
    const float kC1 = 6.28318548202514648f;
    const float kC2 = -1.74845553146951720e-7f;
    const float kShift = 12582912.0f;  // 1.5 * 2^23
    const float k = __fadd_rn(__fmaf_rn(x, kInv2Pi, kShift), -kShift);
    float r = __fmaf_rn(-k, kC1, x);
    r = __fmaf_rn(-k, kC2, r);
    return __cosf(r);
}
__device__ __forceinline__ double fcos(double x) { return cos(x); }
__device__ __forceinline__ float frsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double frsqrt(double x) { return rsqrt(x); }
// 1/x for the FP32 path: the hardware approximation (at most 1 ulp), results
// below the normal range flushed to zero; an IEEE division would take a
// multi-instruction sequence with a slow-path branch per sample.
__device__ __forceinline__ float frcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double frcp(double x) { return 1.0 / x; }

// Weights of the cubic through four equally spaced values f0..f3 at t in
// [0, 1] from f1: the Hermite cubic whose tangents are the central
// differences (f2 - f0)/2 and (f3 - f1)/2 (the Catmull-Rom form),
// value = w0 f0 + w1 f1 + w2 f2 + w3 f3.
template <class T> struct CubicWeights {
    T w0, w1, w2, w3;
    __device__ __forceinline__ explicit CubicWeights(T t) {
        const T t2 = t * t, t3 = t2 * t;
        w0 = T(0.5) * (T(2) * t2 - t - t3);
        w1 = T(0.5) * (T(3) * t3 - T(5) * t2 + T(2));
        w2 = T(0.5) * (T(4) * t2 + t - T(3) * t3);
        w3 = T(0.5) * (t3 - t2);
    }
};

// Cell index and weights of one coordinate of a density grid: r = knots from
// the first (clamped to the grid), cell i in [0, n-2], weights at r - i.
template <class T> __device__ __forceinline__ int grid_cell(T r, int n, T *t) {
    r = fmin(fmax(r, T(0)), T(n - 1));
    const int i = min(static_cast<int>(r), n - 2);
    *t = r - T(i);
    return i;
}

// x g(x, Q^2) from a density grid (F_LO_PDF): bicubic Hermite in
// (log2 x, log2 Q^2) with central-difference tangents.  tbl is the grid padded
// by one knot on every side, the padding the linear ghost value
// 2 f_edge - f_next (which makes the tangent at the first and last knot
// one-sided); so the 4 x 4 knots around any cell are in the table.  FP64:
// (nx + 2) x (nq + 2) knots row-major; FP32: (nx + 2) x (nq + 1) pairs of
// neighbouring knots (knot (r, c), knot (r, c + 1)), a row's four knots read
// as two pairs.  iu / wu: the cell and weights along x, jv / wv along Q^2.
template <class T>
__device__ __forceinline__ T grid_xg(const T *tbl, int nq, int iu, const CubicWeights<T> &wu, int jv,
                                     const CubicWeights<T> &wv) {
    T acc[4];
    if constexpr (sizeof(T) == sizeof(double)) {
        const int pitch = nq + 2;
        const T *r = tbl + iu * pitch + jv;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const T *row = r + a * pitch;
            acc[a] = ffma(wv.w3, row[3], ffma(wv.w2, row[2], ffma(wv.w1, row[1], wv.w0 * row[0])));
        }
    } else {
        const int pitch = nq + 1;
        const float2 *r = reinterpret_cast<const float2 *>(tbl) + iu * pitch + jv;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const float2 p = r[a * pitch], q = r[a * pitch + 2];
            acc[a] = ffma(wv.w3, q.y, ffma(wv.w2, q.x, ffma(wv.w1, p.y, wv.w0 * p.x)));
        }
    }
    return ffma(wu.w3, acc[3], ffma(wu.w2, acc[2], ffma(wu.w1, acc[1], wu.w0 * acc[0])));
}

// The integrand is split into a per-dimension update (called as each
// coordinate is produced) and a final step.  Normalisation constants that do
// not depend on x (the Gaussian's (a sqrt(pi))^-d, the product-peak's scale)
// are folded into the initial weight on the host, so the kernels return f up
// to that factor.  The coordinate passed in is X = S (x - c) with S = Prec<T>::kXS
// (2^32 in FP32, 1 in FP64); the FP32 constants are prepared for it on the
// host (p_j / S, q_j S, s0 / S^2 where the formula below has them), and a
// power of S left over as a factor of f (SUM: S; LO: 1/S; LO_PDF: 1/S^2) is
// divided out of the initial weight.
//
// GAUSS_SYM, GENZ_GAUSS and GENZ_PROD take their coordinate relative to a
// centre (1/2; the peak positions w_j = q_j) that the sampling table already
// holds (table_center), so the subtraction costs nothing per sample; the
// formulas below show it.
//
//   CONST        acc unused                        f = 1
//   SUM          acc += x                          f = acc
//   GAUSS_SYM    acc += (x - 1/2)^2                f = 2^(s0 acc), s0 = -log2(e)/a^2
//   GENZ_OSC     acc += p_j x  (acc0 = 2 pi u)     f = cos(acc)
//   GENZ_GAUSS   acc += (p_j (x - q_j))^2          f = 2^(-log2(e) acc), p_j = c_j
//   GENZ_PROD    prod *= q_j^2... see below        f = 1/prod
//   GENZ_CORNER  acc += p_j x  (acc0 = 1)          f = 2^(-(d+1) log2 acc)
//   LO           x kept in registers               f from s0..s6
//   USER         x kept in registers               f = user_integrand(x, d, p), p = the
//                                                  parameters in p[], q[], s[] in order
//                                                  (x unscaled: x = X / S)
template <int FAM, class T, int MAXD> struct Integrand {
    using C = FamConsts<T>;
    T acc;
    T x0, x1, x2;
    T xs[FAM == F_USER ? MAXD : 1];
    int nd;
    const T *tbl;   // F_LO_PDF: the density grid (shared memory)

    __device__ __forceinline__ void begin(const C &fc) {
        if (FAM == F_GENZ_OSC) acc = fc.s[1];     // 2 pi u
        else if (FAM == F_GENZ_CORNER) acc = T(1);
        else if (FAM == F_GENZ_PROD) acc = T(1);
        else acc = T(0);
    }

    __device__ __forceinline__ void dim(int j, T x, const C &fc) {
        if (FAM == F_SUM) {
            acc += x;
        } else if (FAM == F_GAUSS_SYM) {
            acc = ffma(x, x, acc);  // x - 1/2 (table centre)
        } else if (FAM == F_GENZ_OSC || FAM == F_GENZ_CORNER) {
            acc = ffma(fc.p[j], x, acc);
        } else if (FAM == F_GENZ_GAUSS) {
            const T t = fc.p[j] * x;  // x - q_j (table centre)
            acc = ffma(t, t, acc);
        } else if (FAM == F_GENZ_PROD) {
            // (c^-2 + (x-w)^2) c^2 = 1 + (c (x-w))^2; the c^2 factors are in
            // the initial weight.  Multiply the denominators, invert once.
            const T t = fc.p[j] * x;  // x - q_j (table centre)
            acc *= ffma(t, t, T(1));
        } else if (FAM == F_LO || FAM == F_LO_PDF) {
            if (j == 0) x0 = x;
            else if (j == 1) x1 = x;
            else if (j == 2) x2 = x;
        } else if (FAM == F_USER) {
            xs[FAM == F_USER ? j : 0] = x * Prec<T>::kInvXS;
            nd = j + 1;
        }
    }

    __device__ __forceinline__ T finish(const C &fc) {
        const T s0 = fc.s[0];
        if (FAM == F_CONST) return T(1);
        if (FAM == F_SUM) return acc;
        if (FAM == F_GAUSS_SYM) return fexp2(s0 * acc);
        if (FAM == F_GENZ_OSC) return fcos(acc);
        if (FAM == F_GENZ_GAUSS) return fexp2(s0 * acc);
        if (FAM == F_GENZ_PROD) return frcp(acc);
        if (FAM == F_GENZ_CORNER) return fexp2(s0 * flog2(acc));
        if (FAM == F_USER) return ::user_integrand<T>(xs, nd, reinterpret_cast<const T *>(&fc));
        if (FAM == F_LO_PDF) {
            // the LO toy with g(x, Q^2 = shat) = grid_xg / x; s0..s5 as for LO,
            // p[0..5] the grid (grid_xg), the constant 2 norm in the initial weight
            const T s1 = fc.s[1], s2 = fc.s[2], s3 = fc.s[3], s4 = fc.s[4], s5 = fc.s[5];
            const T shat = x0 * x1 * s0;
            const T c = ffma(T(2) * Prec<T>::kInvXS, x2, T(-1));
            const bool in = (shat >= s4) && (shat <= s5) && (fabs_t(c) < s3);
            // p[0..5]: log2 X of the first knot, knots per unit of log2 x, the
            // same for log2 Q^2, nx, nq; the scale's weights serve both densities
            const int nx = static_cast<int>(fc.p[4]), nq = static_cast<int>(fc.p[5]);
            T tv, t1, t2;
            const int jv = grid_cell((flog2(shat) - fc.p[2]) * fc.p[3], nq, &tv);
            const int i1 = grid_cell((flog2(x0) - fc.p[0]) * fc.p[1], nx, &t1);
            const int i2 = grid_cell((flog2(x1) - fc.p[0]) * fc.p[1], nx, &t2);
            const CubicWeights<T> wv(tv), w1(t1), w2(t2);
            const T g1 = grid_xg(tbl, nq, i1, w1, jv, wv);
            const T g2 = grid_xg(tbl, nq, i2, w2, jv, wv);
            const T dm = shat - s1;
            const T den = ffma(dm, dm, s2) * shat * x0 * x1;
            const T val = g1 * g2 * ffma(c, c, T(1)) * frcp(den);
            return in ? val : T(0);
        }
        if (FAM == F_LO) {
            // s0 = sqrtS^2, s1 = M^2, s2 = (M Gamma)^2, s3 = cut,
            // s4 = mll_lo^2, s5 = mll_hi^2; the constant 2 (35/32)^2 norm is
            // in the initial weight.
            const T s1 = fc.s[1], s2 = fc.s[2], s3 = fc.s[3], s4 = fc.s[4], s5 = fc.s[5];
            const T shat = x0 * x1 * s0;
            const T c = ffma(T(2) * Prec<T>::kInvXS, x2, T(-1));
            const bool in = (shat >= s4) && (shat <= s5) && (fabs_t(c) < s3);
            const T om0 = ffma(-Prec<T>::kInvXS, x0, T(1)), om1 = ffma(-Prec<T>::kInvXS, x1, T(1));
            const T g = om0 * om0 * om0 * om1 * om1 * om1 * frsqrt(x0 * x1);
            const T dm = shat - s1;
            const T den = ffma(dm, dm, s2) * shat;
            const T val = g * ffma(c, c, T(1)) * frcp(den);
            return in ? val : T(0);
        }
        return T(0);
    }
};

}  // namespace vegas
