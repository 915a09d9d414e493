// vegas_batch_sample.cuh -- the persistent sampling kernel of the batched form.
//
// Each block loops: claim the next tile (atomic counter), find its slot by a
// binary search of the tile prefix, and sample the tile's range of that
// slot's samples into the block's shared-memory cells.  Tiles of one slot are
// consecutive, so a block usually claims several tiles of the same slot in a
// row; when the slot changes, the block adds its sums to the old slot's FP64
// accumulators and stages the new slot's table.  The fixed-point cells are
// also flushed whenever the block has added block_sample_cap samples to them.
#pragma once

#include "vegas_batch.cuh"

namespace vegas {

// The current slot's integrand constants, staged per slot switch.  File-scope
// shared variables (one per precision) so that the out-of-line tile samplers
// address them as shared memory rather than through a generic pointer.
__shared__ FamConsts<float> g_batch_fc32;
__shared__ FamConsts<double> g_batch_fc64;
template <class T> __device__ __forceinline__ FamConsts<T> &batch_fc();
template <> __device__ __forceinline__ FamConsts<float> &batch_fc<float>() { return g_batch_fc32; }
template <> __device__ __forceinline__ FamConsts<double> &batch_fc<double>() { return g_batch_fc64; }

// One range of one slot.  Kept out of line: each (family, dimension)
// variant gets its own register allocation instead of the union of all of
// them.  Arguments are scalars (passed in registers; a structure argument
// would live in memory and be re-read in the loop); the running sums are
// read and written once per call.
template <int MODE, int PRIV, int FAM, int MAXD, bool EXACT>
__device__ __noinline__ void batch_range(typename BlockState<MODE, PRIV>::T2 *tab,
                                         typename BlockState<MODE, PRIV>::H *hist, uint32_t *fine, int d, int N,
                                         uint32_t key0, uint32_t key1, uint32_t iter,
                                         typename ModeTraits<MODE>::T jinit, typename ModeTraits<MODE>::T n4,
                                         float hs, double *acc, unsigned long long s0, int cnt,
                                         ThreadSums<MODE> *tsp) {
    BlockState<MODE, PRIV> bs;
    bs.tab = tab;
    bs.hist = hist;
    bs.fine = fine;
    bs.cells = d * N;
    RangeParams<typename ModeTraits<MODE>::T> rp;
    rp.d = d;
    rp.N = N;
    rp.key0 = key0;
    rp.key1 = key1;
    rp.iter = iter;
    rp.jinit = jinit;
    rp.n4 = n4;
    rp.hs = hs;
    rp.acc = acc;
    ThreadSums<MODE> ts = *tsp;
    sample_range<FAM, MODE, MAXD, EXACT, PRIV, (MAXD > 16), false>(bs, rp, batch_fc<typename ModeTraits<MODE>::T>(), ts, s0, cnt);
    *tsp = ts;
}

template <int MODE, int PRIV, int FAM, int MAXD, bool EXACT>
__device__ __forceinline__ void batch_call(const BlockState<MODE, PRIV> &bs,
                                           const RangeParams<typename ModeTraits<MODE>::T> &rp,
                                           ThreadSums<MODE> &ts, unsigned long long s0, int cnt) {
    batch_range<MODE, PRIV, FAM, MAXD, EXACT>(bs.tab, bs.hist, bs.fine, rp.d, rp.N, rp.key0, rp.key1, rp.iter,
                                              rp.jinit, rp.n4, rp.hs, rp.acc, s0, cnt, &ts);
}

// Dimensions 1..16 get a sampler each (no per-dimension guards or branches:
// 12.5 -> 10.6 ms per step of the 512-integral mix against four dimension
// tiers); 17..32 share the generic one.
template <int MODE, int PRIV, int FAM>
__device__ __forceinline__ void batch_dispatch_dim(const BlockState<MODE, PRIV> &bs,
                                                    const RangeParams<typename ModeTraits<MODE>::T> &rp,
                                                    ThreadSums<MODE> &ts, unsigned long long s0, int cnt) {
    if (FAM == F_LO) {
        batch_call<MODE, PRIV, FAM, 3, true>(bs, rp, ts, s0, cnt);
        return;
    }
    switch (rp.d) {
    case 1: batch_call<MODE, PRIV, FAM, 1, true>(bs, rp, ts, s0, cnt); break;
    case 2: batch_call<MODE, PRIV, FAM, 2, true>(bs, rp, ts, s0, cnt); break;
    case 3: batch_call<MODE, PRIV, FAM, 3, true>(bs, rp, ts, s0, cnt); break;
    case 4: batch_call<MODE, PRIV, FAM, 4, true>(bs, rp, ts, s0, cnt); break;
    case 5: batch_call<MODE, PRIV, FAM, 5, true>(bs, rp, ts, s0, cnt); break;
    case 6: batch_call<MODE, PRIV, FAM, 6, true>(bs, rp, ts, s0, cnt); break;
    case 7: batch_call<MODE, PRIV, FAM, 7, true>(bs, rp, ts, s0, cnt); break;
    case 8: batch_call<MODE, PRIV, FAM, 8, true>(bs, rp, ts, s0, cnt); break;
    case 9: batch_call<MODE, PRIV, FAM, 9, true>(bs, rp, ts, s0, cnt); break;
    case 10: batch_call<MODE, PRIV, FAM, 10, true>(bs, rp, ts, s0, cnt); break;
    case 11: batch_call<MODE, PRIV, FAM, 11, true>(bs, rp, ts, s0, cnt); break;
    case 12: batch_call<MODE, PRIV, FAM, 12, true>(bs, rp, ts, s0, cnt); break;
    case 13: batch_call<MODE, PRIV, FAM, 13, true>(bs, rp, ts, s0, cnt); break;
    case 14: batch_call<MODE, PRIV, FAM, 14, true>(bs, rp, ts, s0, cnt); break;
    case 15: batch_call<MODE, PRIV, FAM, 15, true>(bs, rp, ts, s0, cnt); break;
    case 16: batch_call<MODE, PRIV, FAM, 16, true>(bs, rp, ts, s0, cnt); break;
    default: batch_call<MODE, PRIV, FAM, 32, false>(bs, rp, ts, s0, cnt); break;
    }
}

template <int MODE, int PRIV>
__device__ __forceinline__ void batch_dispatch(int fam, const BlockState<MODE, PRIV> &bs,
                                               const RangeParams<typename ModeTraits<MODE>::T> &rp,
                                               ThreadSums<MODE> &ts, unsigned long long s0, int cnt) {
    switch (fam) {
    case F_CONST: batch_dispatch_dim<MODE, PRIV, F_CONST>(bs, rp, ts, s0, cnt); break;
    case F_SUM: batch_dispatch_dim<MODE, PRIV, F_SUM>(bs, rp, ts, s0, cnt); break;
    case F_GAUSS_SYM: batch_dispatch_dim<MODE, PRIV, F_GAUSS_SYM>(bs, rp, ts, s0, cnt); break;
    case F_GENZ_OSC: batch_dispatch_dim<MODE, PRIV, F_GENZ_OSC>(bs, rp, ts, s0, cnt); break;
    case F_GENZ_GAUSS: batch_dispatch_dim<MODE, PRIV, F_GENZ_GAUSS>(bs, rp, ts, s0, cnt); break;
    case F_GENZ_PROD: batch_dispatch_dim<MODE, PRIV, F_GENZ_PROD>(bs, rp, ts, s0, cnt); break;
    case F_GENZ_CORNER: batch_dispatch_dim<MODE, PRIV, F_GENZ_CORNER>(bs, rp, ts, s0, cnt); break;
    case F_LO: batch_dispatch_dim<MODE, PRIV, F_LO>(bs, rp, ts, s0, cnt); break;
    default: break;
    }
}

template <int MODE, int PRIV>
__global__ void __launch_bounds__(kBatchThreads, 1)
batch_sample_kernel_t(const BatchArgs ba) {
    using BS = BlockState<MODE, PRIV>;
    using T = typename BS::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FamConsts<T> &fc_s = batch_fc<T>();
    __shared__ long long s_tile;
    __shared__ int s_item;
    __shared__ T s_scal[2];
    const PlanHeader hdr = *ba.hdr;
    BS bs;
    ThreadSums<MODE> ts;
    RangeParams<T> rp;
    rp.d = 1;
    rp.N = 2;
    rp.hs = 0.f;
    rp.acc = nullptr;
    int cur = -1;
    int fam = 0;
    long long n_cur = 0;
    long long cap = 0;     // samples between flushes of the fixed-point cells
    long long since = 0;   // samples added since the last flush
    SlotDev *sd = nullptr;
    for (;;) {
        if (threadIdx.x == 0) {
            const long long tile = static_cast<long long>(atomicAdd(ba.counter, 1ull));
            int item = -1;
            if (tile < hdr.total_tiles) {
                int lo = 0, hi = hdr.n_items - 1;  // last k with tile_prefix[k] <= tile
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (ba.tile_prefix[mid] <= tile) lo = mid;
                    else hi = mid - 1;
                }
                item = lo;
            }
            s_tile = tile;
            s_item = item;
        }
        __syncthreads();
        const long long tile = s_tile;
        const int item = s_item;
        if (item < 0) break;
        if (item != cur) {
            if (cur >= 0) flush_block<MODE, PRIV>(bs, ts, rp.hs, sd->acc, &sd->nonfinite, nullptr, true);
            sd = &ba.slots[ba.items[item]];
            fam = sd->family;
            rp.d = sd->d;
            rp.N = sd->N;
            rp.key0 = sd->key0;
            rp.key1 = sd->key1;
            rp.iter = static_cast<uint32_t>(sd->t);
            if (threadIdx.x == 0) {  // FP64 scalars once per block (read after the barrier below)
                s_scal[0] = MODE == ACC_F64 ? static_cast<T>(sd->jinit64 * sd->jmul)
                                            : static_cast<T>(static_cast<double>(sd->jinit32) * sd->jmul);
                s_scal[1] = static_cast<T>(sd->n4);
            }
            rp.hs = MODE != ACC_F64 ? sd->hscale : 0.f;
            rp.acc = sd->acc;
            n_cur = sd->n;
            cap = block_sample_cap<MODE, PRIV>(rp.N);
            since = 0;
            const FamConsts<T> *src;
            if (MODE == ACC_F64) src = reinterpret_cast<const FamConsts<T> *>(&sd->fc64);
            else src = reinterpret_cast<const FamConsts<T> *>(&sd->fc32);
            const uint32_t *s32 = reinterpret_cast<const uint32_t *>(src);
            uint32_t *d32 = reinterpret_cast<uint32_t *>(&fc_s);
            for (int k = threadIdx.x; k < static_cast<int>(sizeof(FamConsts<T>) / 4); k += blockDim.x)
                d32[k] = s32[k];
            bs.carve(smem_raw, rp.d * rp.N);
            bs.stage(sd->table);
            __syncthreads();
            rp.jinit = s_scal[0];
            rp.n4 = s_scal[1];
            cur = item;
        }
        long long s0 = (tile - ba.tile_prefix[item]) * static_cast<long long>(hdr.tile_samples);
        long long cnt = min(static_cast<long long>(hdr.tile_samples), n_cur - s0);
        while (cnt > 0) {
            if (MODE != ACC_F64 && since >= cap) {
                // the cells are full: add them to the slot's sums and restart
                flush_block<MODE, PRIV>(bs, ts, rp.hs, sd->acc, &sd->nonfinite);
                bs.clear();
                __syncthreads();
                since = 0;
            }
            const long long part = MODE != ACC_F64 ? min(cnt, cap - since) : cnt;
            batch_dispatch<MODE, PRIV>(fam, bs, rp, ts, static_cast<unsigned long long>(s0), static_cast<int>(part));
            s0 += part;
            cnt -= part;
            since += part;
        }
        __syncthreads();  // s_tile / s_item are rewritten by the next claim
    }
    if (cur >= 0) flush_block<MODE, PRIV>(bs, ts, rp.hs, sd->acc, &sd->nonfinite, nullptr, true);
}

}  // namespace vegas
