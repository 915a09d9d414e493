// vegas_batch_sample.cuh -- the persistent sampling kernel of the batched form.
//
// Each block loops: claim the next tile (atomic counter), find its slot by a
// binary search of the tile prefix, and sample the tile's range of that
// slot's samples into the block's shared-memory cells.  Tiles of one slot are
// consecutive, so a block usually claims several tiles of the same slot in a
// row; when the slot changes, the block adds its sums to the old slot's FP64
// accumulators and stages the new slot's table.
#pragma once

#include "vegas_batch.cuh"

namespace vegas {

// One tile of one slot.  Kept out of line: each (family, dimension tier)
// variant gets its own register allocation instead of sharing the persistent
// loop's; the call happens once per tile of thousands of samples.
template <int MODE, bool PRIV, int FAM, int MAXD, bool EXACT>
__device__ __noinline__ ThreadSums<MODE> batch_tile(BlockState<MODE, PRIV> bs,
                                                    RangeParams<typename ModeTraits<MODE>::T> rp,
                                                    const FamConsts<typename ModeTraits<MODE>::T> *fc,
                                                    ThreadSums<MODE> ts, unsigned long long s0, int cnt) {
    sample_range<FAM, MODE, MAXD, EXACT, PRIV>(bs, rp, *fc, ts, s0, cnt);
    return ts;
}

template <int MODE, bool PRIV, int FAM>
__device__ __forceinline__ void batch_dispatch_tier(const BlockState<MODE, PRIV> &bs,
                                                    const RangeParams<typename ModeTraits<MODE>::T> &rp,
                                                    const FamConsts<typename ModeTraits<MODE>::T> *fc,
                                                    ThreadSums<MODE> &ts, unsigned long long s0, int cnt) {
    if (FAM == F_LO) {
        ts = batch_tile<MODE, PRIV, FAM, 3, true>(bs, rp, fc, ts, s0, cnt);
    } else if (rp.d <= 4) {
        ts = batch_tile<MODE, PRIV, FAM, 4, false>(bs, rp, fc, ts, s0, cnt);
    } else if (rp.d <= 8) {
        ts = batch_tile<MODE, PRIV, FAM, 8, false>(bs, rp, fc, ts, s0, cnt);
    } else if (rp.d <= 16) {
        ts = batch_tile<MODE, PRIV, FAM, 16, false>(bs, rp, fc, ts, s0, cnt);
    } else {
        ts = batch_tile<MODE, PRIV, FAM, 32, false>(bs, rp, fc, ts, s0, cnt);
    }
}

template <int MODE, bool PRIV>
__global__ void __launch_bounds__(512, 1)
batch_sample_kernel_t(const BatchArgs ba) {
    using BS = BlockState<MODE, PRIV>;
    using T = typename BS::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ FamConsts<T> fc_s;
    __shared__ long long s_tile;
    __shared__ int s_item;
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
            if (cur >= 0) flush_block<MODE, PRIV>(bs, ts, rp.hs, sd->acc, &sd->nonfinite);
            sd = &ba.slots[ba.items[item]];
            fam = sd->family;
            rp.d = sd->d;
            rp.N = sd->N;
            rp.key0 = sd->key0;
            rp.key1 = sd->key1;
            rp.iter = static_cast<uint32_t>(sd->t);
            rp.jinit = MODE == ACC_F64 ? static_cast<T>(sd->jinit64 * sd->jmul)
                                       : static_cast<T>(static_cast<double>(sd->jinit32) * sd->jmul);
            rp.n4 = static_cast<T>(sd->n4);
            rp.hs = MODE != ACC_F64 ? sd->hscale : 0.f;
            rp.acc = sd->acc;
            n_cur = sd->n;
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
            cur = item;
        }
        const long long s0 = (tile - ba.tile_prefix[item]) * static_cast<long long>(hdr.tile_samples);
        const int cnt = static_cast<int>(min(static_cast<long long>(hdr.tile_samples), n_cur - s0));
        if (cnt > 0) {
            const unsigned long long u0 = static_cast<unsigned long long>(s0);
            switch (fam) {
            case F_CONST: batch_dispatch_tier<MODE, PRIV, F_CONST>(bs, rp, &fc_s, ts, u0, cnt); break;
            case F_SUM: batch_dispatch_tier<MODE, PRIV, F_SUM>(bs, rp, &fc_s, ts, u0, cnt); break;
            case F_GAUSS_SYM: batch_dispatch_tier<MODE, PRIV, F_GAUSS_SYM>(bs, rp, &fc_s, ts, u0, cnt); break;
            case F_GENZ_OSC: batch_dispatch_tier<MODE, PRIV, F_GENZ_OSC>(bs, rp, &fc_s, ts, u0, cnt); break;
            case F_GENZ_GAUSS: batch_dispatch_tier<MODE, PRIV, F_GENZ_GAUSS>(bs, rp, &fc_s, ts, u0, cnt); break;
            case F_GENZ_PROD: batch_dispatch_tier<MODE, PRIV, F_GENZ_PROD>(bs, rp, &fc_s, ts, u0, cnt); break;
            case F_GENZ_CORNER: batch_dispatch_tier<MODE, PRIV, F_GENZ_CORNER>(bs, rp, &fc_s, ts, u0, cnt); break;
            case F_LO: batch_dispatch_tier<MODE, PRIV, F_LO>(bs, rp, &fc_s, ts, u0, cnt); break;
            default: break;
            }
        }
        __syncthreads();  // s_tile / s_item are rewritten by the next claim
    }
    if (cur >= 0) flush_block<MODE, PRIV>(bs, ts, rp.hs, sd->acc, &sd->nonfinite);
}

}  // namespace vegas
