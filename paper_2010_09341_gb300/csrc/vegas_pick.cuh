// vegas_pick.cuh -- table of sampling-kernel instantiations for one mode.
// Included by the translation units of one accumulation mode; each unit
// instantiates a subset of the families so that they compile in parallel.
#pragma once

#include "vegas_kernels.cuh"
#include "vegas_strat.cuh"

namespace vegas {

template <int MODE, int FAM, int MAXD, bool EXACT>
static const void *pick_priv(bool priv) {
    if constexpr (EXACT) {
        return reinterpret_cast<const void *>(&vegas_sample_kernel<FAM, MODE, MAXD, true, true>);
    } else {
        return priv ? reinterpret_cast<const void *>(&vegas_sample_kernel<FAM, MODE, MAXD, false, true>)
                    : reinterpret_cast<const void *>(&vegas_sample_kernel<FAM, MODE, MAXD, false, false>);
    }
}

// Exact-dimension kernels (no per-dimension guards) for d <= 8 with the
// lane-private layout; generic kernels with a run-time d otherwise.  Only the
// kernels a branch can return are instantiated (constexpr branches).
template <int MODE, int FAM>
static const void *pick_family(int d, bool priv) {
    constexpr bool kExact = MODE != ACC_F64;  // the FP64 path is FP64-pipe bound either way
    if constexpr (FAM == F_LO || FAM == F_LO_PDF) {
        if (d != 3) return nullptr;
        if constexpr (kExact) {
            if (priv) return pick_priv<MODE, FAM, 3, true>(true);
        }
        return pick_priv<MODE, FAM, 4, false>(priv);
    } else {
        if constexpr (kExact) {
            if (priv) switch (d) {
            case 1: return pick_priv<MODE, FAM, 1, true>(true);
            case 2: return pick_priv<MODE, FAM, 2, true>(true);
            case 3: return pick_priv<MODE, FAM, 3, true>(true);
            case 4: return pick_priv<MODE, FAM, 4, true>(true);
            case 5: return pick_priv<MODE, FAM, 5, true>(true);
            case 6: return pick_priv<MODE, FAM, 6, true>(true);
            case 7: return pick_priv<MODE, FAM, 7, true>(true);
            case 8: return pick_priv<MODE, FAM, 8, true>(true);
            default: break;
            }
        }
        if (d <= 8) return pick_priv<MODE, FAM, 8, false>(priv);
        if (d <= 16) return pick_priv<MODE, FAM, 16, false>(priv);
        return pick_priv<MODE, FAM, 32, false>(priv);
    }
}

// FP64 kernels with one histogram copy per lane (kLayoutWide; the host takes
// them where the layout fits and an iteration has many samples per block):
// the generic tiers of 8 and 16 dimensions, the LO toy's tier of 4; none above
// 16 dimensions, whose cells would not fit.
template <int MODE, int FAM>
static const void *pick_family_wide(int d) {
    static_assert(MODE == ACC_F64, "the wide histogram layout is the FP64 path's");
    if constexpr (FAM == F_LO) {
        if (d != 3) return nullptr;
        return reinterpret_cast<const void *>(&vegas_sample_kernel<FAM, MODE, 4, false, true, true>);
    } else {
        if (d <= 8) return reinterpret_cast<const void *>(&vegas_sample_kernel<FAM, MODE, 8, false, true, true>);
        if (d <= 16) return reinterpret_cast<const void *>(&vegas_sample_kernel<FAM, MODE, 16, false, true, true>);
        return nullptr;
    }
}

// Stratified kernels: as above, exact-dimension kernels for d <= 8 in the
// FP32 modes with the lane-private layout, generic tiers otherwise.
template <int MODE, int FAM, int MAXD, bool EXACT>
static const void *pick_strat_priv(bool priv) {
    if constexpr (EXACT) {
        return reinterpret_cast<const void *>(&vegas_sample_strat_kernel<FAM, MODE, MAXD, true, true>);
    } else {
        return priv ? reinterpret_cast<const void *>(&vegas_sample_strat_kernel<FAM, MODE, MAXD, false, true>)
                    : reinterpret_cast<const void *>(&vegas_sample_strat_kernel<FAM, MODE, MAXD, false, false>);
    }
}

template <int MODE, int FAM>
static const void *pick_strat(int d, bool priv) {
    constexpr bool kExact = MODE != ACC_F64;
    if constexpr (FAM == F_LO || FAM == F_LO_PDF) {
        if (d != 3) return nullptr;
        if constexpr (kExact) {
            if (priv) return pick_strat_priv<MODE, FAM, 3, true>(true);
        }
        return pick_strat_priv<MODE, FAM, 4, false>(priv);
    } else {
        if constexpr (kExact) {
            if (priv) switch (d) {
            case 1: return pick_strat_priv<MODE, FAM, 1, true>(true);
            case 2: return pick_strat_priv<MODE, FAM, 2, true>(true);
            case 3: return pick_strat_priv<MODE, FAM, 3, true>(true);
            case 4: return pick_strat_priv<MODE, FAM, 4, true>(true);
            case 5: return pick_strat_priv<MODE, FAM, 5, true>(true);
            case 6: return pick_strat_priv<MODE, FAM, 6, true>(true);
            case 7: return pick_strat_priv<MODE, FAM, 7, true>(true);
            case 8: return pick_strat_priv<MODE, FAM, 8, true>(true);
            default: break;
            }
        }
        if (d <= 8) return pick_strat_priv<MODE, FAM, 8, false>(priv);
        if (d <= 16) return pick_strat_priv<MODE, FAM, 16, false>(priv);
        return pick_strat_priv<MODE, FAM, 32, false>(priv);
    }
}

}  // namespace vegas
