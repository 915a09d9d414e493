// vegas_strat.cuh -- the stratified + importance hybrid sampling kernel.
//
// Lepage's combined mode (VEGAS, Cornell CLNS-80/447, 1980): y-space is also
// cut into 2^B equal hypercubes that each take the same number P of samples;
// the iteration's estimate is the mean of the hypercube means and its variance
// the sum of the hypercubes' variances of the mean.  The grid map, integrand,
// sums and histograms are the plain kernel's (map_sample, hist_add); only the
// Philox words are moved into the sample's strata (StratArgs, strat_word) and
// each thread takes whole hypercubes, so that their spread about their own
// mean stays in registers.
#pragma once

#include "vegas_sample.cuh"

namespace vegas {

// Stratified form: the block samples hypercubes [h0, h0 + cnt) of one
// integral, P samples each; thread t takes hypercubes h0 + t + u * blockDim
// and all of their samples, so each hypercube's spread about its own mean,
//   m2_h = sum_p (v_p - mean_h)^2 = B - A^2 / P,
// comes from A = sum (v - c) and B = sum (v - c)^2 with c = the hypercube's
// first value (shifted sums: no cancellation of the mean).  Samples go two at
// a time (independent Philox and table-load chains).  In the FP32 modes the
// partial sums of v, v^2 (FP32_SUM64) and m2 are kept in FP32 and added in
// FP64 once a thread has taken kChunk samples since the last addition.
template <int FAM, int MODE, int MAXD, bool EXACT, int PRIV>
__device__ __forceinline__ void sample_range_strat_any(const BlockState<MODE, PRIV> &bs,
                                                       const RangeParams<typename ModeTraits<MODE>::T> &rp,
                                                       const FamConsts<typename ModeTraits<MODE>::T> &fc,
                                                       const StratArgs &st, ThreadSums<MODE> &ts, uint32_t h0,
                                                       int cnt) {
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
    const uint32_t P = st.P;
    const T invP = T(1) / static_cast<T>(P);
    constexpr uint32_t kChunk = 8;
    // generic tiers: two samples' cells in 16-bit halves (d N <= 32768), which
    // keeps them in registers; the exact-dimension kernels have room for both
    constexpr bool kPack = !EXACT;
    float p1 = 0.f, p2 = 0.f;   // FP32_SUM64 partial sums of v, v^2
    T qt = T(0);                // partial sum of m2 (FP32 modes)
    uint32_t since = 0;         // samples since the partials were last added in FP64
    auto flush_partials = [&]() {
        if (MODE == ACC_F32_SUM64) {
            ts.s1d += static_cast<double>(p1);
            ts.s2d += static_cast<double>(p2);
            p1 = 0.f;
            p2 = 0.f;
        }
        ts.qd += static_cast<double>(qt);
        qt = T(0);
        since = 0;
    };
    auto add_sums = [&](T v, T v2) {
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
    };
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
        const uint32_t h = h0 + static_cast<uint32_t>(k);
        const unsigned long long sb = static_cast<unsigned long long>(h) * P;
        T c = T(0), a = T(0), b = T(0);
        uint32_t p = 0;
        for (; p + 1 < P; p += 2) {
            SampleCells<MAXD, kPack> ca, cb;
            const T va = map_sample<FAM, MODE, MAXD, EXACT, PRIV, kPack, true>(tab_l, rp, fc, &st, h, sb + p, ca,
                                                                               ts.nonfinite);
            const T vb = map_sample<FAM, MODE, MAXD, EXACT, PRIV, kPack, true>(tab_l, rp, fc, &st, h, sb + p + 1,
                                                                               cb, ts.nonfinite);
            const T va2 = va * va, vb2 = vb * vb;
            add_sums(va, va2);
            add_sums(vb, vb2);
            if (p == 0) c = va;
            const T da = va - c, db = vb - c;
            a += da + db;
            b = ffma(da, da, ffma(db, db, b));
            hist_add<MODE, PRIV, MAXD, EXACT, kPack>(bs, hist_l, rp, ca, va2, fixed, hs);
            hist_add<MODE, PRIV, MAXD, EXACT, kPack>(bs, hist_l, rp, cb, vb2, fixed, hs);
            if (MODE == ACC_F32_SUM64 && P > kChunk && ((p + 2) & (kChunk - 1)) == 0) {
                // long hypercubes: the FP32 partials of v, v^2 stay short
                ts.s1d += static_cast<double>(p1);
                ts.s2d += static_cast<double>(p2);
                p1 = 0.f;
                p2 = 0.f;
            }
        }
        if (p < P) {
            SampleCells<MAXD, kPack> ca;
            const T va = map_sample<FAM, MODE, MAXD, EXACT, PRIV, kPack, true>(tab_l, rp, fc, &st, h, sb + p, ca,
                                                                               ts.nonfinite);
            const T va2 = va * va;
            add_sums(va, va2);
            if (p == 0) c = va;
            const T da = va - c;
            a += da;
            b = ffma(da, da, b);
            hist_add<MODE, PRIV, MAXD, EXACT, kPack>(bs, hist_l, rp, ca, va2, fixed, hs);
        }
        const T m2 = b - a * a * invP;
        qt += m2 > T(0) ? m2 : T(0);
        since += P;
        if (MODE == ACC_F64 || since >= kChunk) flush_partials();
    }
    flush_partials();
}

// The same for P <= kChunk in the exact-dimension kernels, with the FP64
// additions of the FP32 partials at the end of each group of ceil(kChunk / P)
// hypercubes (the same points as above), not behind a test inside the loop:
// the compiler predicates a short conditional block, and a predicated-off FP64
// instruction still holds the FP64 unit for its ~76 cycles on GB300.
template <int FAM, int MODE, int MAXD, bool EXACT, int PRIV, bool FOLD>
__device__ __forceinline__ void sample_range_strat_grouped(const BlockState<MODE, PRIV> &bs,
                                                     const RangeParams<typename ModeTraits<MODE>::T> &rp,
                                                     const FamConsts<typename ModeTraits<MODE>::T> &fc,
                                                     const StratArgs &st, ThreadSums<MODE> &ts, uint32_t h0,
                                                     int cnt) {
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
    const uint32_t P = st.P;
    const T invP = T(1) / static_cast<T>(P);
    constexpr uint32_t kChunk = 8;
    // generic tiers: two samples' cells in 16-bit halves (d N <= 32768), which
    // keeps them in registers; the exact-dimension kernels have room for both
    constexpr bool kPack = !EXACT;
    float p1 = 0.f, p2 = 0.f;   // FP32_SUM64 partial sums of v, v^2
    T qt = T(0);                // partial sum of m2 (FP32 modes)
    auto add_vv = [&]() {       // the FP32 partials of v, v^2 into FP64
        if (MODE == ACC_F32_SUM64) {
            ts.s1d += static_cast<double>(p1);
            ts.s2d += static_cast<double>(p2);
            p1 = 0.f;
            p2 = 0.f;
        }
    };
    auto add_q = [&]() {
        ts.qd += static_cast<double>(qt);
        qt = T(0);
    };
    auto add_sums = [&](T v, T v2) {
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
    };
    // one sample's update: with FOLD (FP32 fixed-point cells) the histogram
    // first, whose rare branch zeroes a non-finite v (hist_add_fixed), then
    // the sums and the hypercube's spread
    auto update = [&](T v, T v2, const SampleCells<MAXD, kPack> &cj, bool first, T &c, T &a, T &b) {
        if constexpr (FOLD) hist_add_fixed<MODE, PRIV, MAXD, EXACT, kPack>(bs, hist_l, rp, cj, v, v2, hs, ts.nonfinite);
        add_sums(v, v2);
        if (first) c = v;
        const T dv = v - c;
        a += dv;
        b = ffma(dv, dv, b);
        if constexpr (!FOLD) hist_add<MODE, PRIV, MAXD, EXACT, kPack>(bs, hist_l, rp, cj, v2, fixed, hs);
    };
    // samples [pb, pe) of hypercube h (first sample index sb), into A, B
    auto run = [&](uint32_t h, unsigned long long sb, uint32_t pb, uint32_t pe, T &c, T &a, T &b) {
        uint32_t p = pb;
        for (; p + 1 < pe; p += 2) {
            SampleCells<MAXD, kPack> ca, cb;
            const T va = map_sample<FAM, MODE, MAXD, EXACT, PRIV, kPack, true, !FOLD>(tab_l, rp, fc, &st, h, sb + p,
                                                                                      ca, ts.nonfinite);
            const T vb = map_sample<FAM, MODE, MAXD, EXACT, PRIV, kPack, true, !FOLD>(tab_l, rp, fc, &st, h,
                                                                                      sb + p + 1, cb, ts.nonfinite);
            update(va, va * va, ca, p == 0, c, a, b);
            update(vb, vb * vb, cb, false, c, a, b);
        }
        if (p < pe) {
            SampleCells<MAXD, kPack> ca;
            const T va = map_sample<FAM, MODE, MAXD, EXACT, PRIV, kPack, true, !FOLD>(tab_l, rp, fc, &st, h, sb + p,
                                                                                      ca, ts.nonfinite);
            update(va, va * va, ca, p == 0, c, a, b);
        }
    };
    auto finish = [&](T a, T b) {
        const T m2 = b - a * a * invP;
        qt += m2 > T(0) ? m2 : T(0);
    };
    // P <= kChunk: the FP32 partials go into FP64 after each group of
    // ceil(kChunk / P) hypercubes (one hypercube in the FP64 mode)
    const int G = MODE == ACC_F64 ? 1 : static_cast<int>((kChunk + P - 1) / P);
    const int step = blockDim.x;
    for (int k0 = threadIdx.x; k0 < cnt; k0 += G * step) {
        const int kend = min(cnt, k0 + G * step);
        for (int k = k0; k < kend; k += step) {
            const uint32_t h = h0 + static_cast<uint32_t>(k);
            const unsigned long long sb = static_cast<unsigned long long>(h) * P;
            T c = T(0), a = T(0), b = T(0);
            run(h, sb, 0u, P, c, a, b);
            finish(a, b);
        }
        add_vv();
        add_q();
    }
}

template <int FAM, int MODE, int MAXD, bool EXACT, int PRIV>
__device__ __forceinline__ void sample_range_strat(const BlockState<MODE, PRIV> &bs,
                                                   const RangeParams<typename ModeTraits<MODE>::T> &rp,
                                                   const FamConsts<typename ModeTraits<MODE>::T> &fc,
                                                   const StratArgs &st, ThreadSums<MODE> &ts, uint32_t h0,
                                                   int cnt) {
    // the generic tiers keep one copy of the sample loop (a second one would
    // push the 32-dimension tier past its 128 registers)
    if constexpr (EXACT) {
        if (st.P <= 8u) {
            if (MODE != ACC_F64 && rp.hs > 0.f)
                sample_range_strat_grouped<FAM, MODE, MAXD, EXACT, PRIV, MODE != ACC_F64>(bs, rp, fc, st, ts, h0, cnt);
            else
                sample_range_strat_grouped<FAM, MODE, MAXD, EXACT, PRIV, false>(bs, rp, fc, st, ts, h0, cnt);
            return;
        }
    }
    sample_range_strat_any<FAM, MODE, MAXD, EXACT, PRIV>(bs, rp, fc, st, ts, h0, cnt);
}

// Stratified form: hypercubes [a.s_begin, a.s_begin + a.n) of P = a.st.P
// samples each; each block takes a contiguous range of hypercubes.
// Blocks per SM as for the plain kernel (kSampleMinBlocks: one, whose threads
// may use up to 128 registers, except for the LO toy); above 8
// dimensions a block's lane-private cells take most of an SM's shared memory
// anyway.  At d = 8 one block ran the stratified Gaussian 3.5% faster than
// two, the oscillatory integral 1% slower.
template <int FAM, int MODE, int MAXD, bool EXACT, bool PRIV>
__global__ void __launch_bounds__(512, kSampleMinBlocks<FAM>)
vegas_sample_strat_kernel(const SampleArgs a) {
    pdl_begin();
    using BS = BlockState<MODE, PRIV>;
    using T = typename BS::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int d = EXACT ? MAXD : a.d;
    BS bs;
    bs.carve(smem_raw, d * a.N);
    bs.stage(a.table);
    RangeParams<T> rp;
    rp.aux = stage_pdf<FAM, MODE, PRIV>(smem_raw, a, d);
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
        sample_range_strat<FAM, MODE, MAXD, EXACT, PRIV>(bs, rp, consts<T>(a), a.st, ts,
                                                         static_cast<uint32_t>(a.s_begin + lo),
                                                         static_cast<int>(hi - lo));
    flush_block<MODE, PRIV>(bs, ts, rp.hs, a.acc, a.n_nonfinite, a.st.q, true);
}

}  // namespace vegas
