// vegas_pick.cuh -- table of sampling-kernel instantiations for one mode.
// Included by exactly one translation unit per accumulation mode so that the
// three modes compile in parallel.
#pragma once

#include "vegas_kernels.cuh"

namespace vegas {

template <int MODE, int FAM, int MAXD>
static const void *pick_priv(bool priv) {
    return priv ? reinterpret_cast<const void *>(&vegas_sample_kernel<FAM, MODE, MAXD, true>)
                : reinterpret_cast<const void *>(&vegas_sample_kernel<FAM, MODE, MAXD, false>);
}

template <int MODE, int FAM>
static const void *pick_tier(int tier, bool priv) {
    switch (tier) {
    case 0: return pick_priv<MODE, FAM, 4>(priv);
    case 1: return pick_priv<MODE, FAM, 8>(priv);
    case 2: return pick_priv<MODE, FAM, 16>(priv);
    default: return pick_priv<MODE, FAM, 32>(priv);
    }
}

template <int MODE>
static const void *pick_kernel(int fam, int tier, bool priv) {
    switch (fam) {
    case F_CONST: return pick_tier<MODE, F_CONST>(tier, priv);
    case F_SUM: return pick_tier<MODE, F_SUM>(tier, priv);
    case F_GAUSS_SYM: return pick_tier<MODE, F_GAUSS_SYM>(tier, priv);
    case F_GENZ_OSC: return pick_tier<MODE, F_GENZ_OSC>(tier, priv);
    case F_GENZ_GAUSS: return pick_tier<MODE, F_GENZ_GAUSS>(tier, priv);
    case F_GENZ_PROD: return pick_tier<MODE, F_GENZ_PROD>(tier, priv);
    case F_GENZ_CORNER: return pick_tier<MODE, F_GENZ_CORNER>(tier, priv);
    case F_LO: return tier == 0 ? pick_priv<MODE, F_LO, 4>(priv) : nullptr;  // d = 3 only
    default: return nullptr;
    }
}

}  // namespace vegas
