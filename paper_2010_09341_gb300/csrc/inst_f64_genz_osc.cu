// Sampling kernels: mode ACC_F64, family F_GENZ_OSC (generated instantiation unit).
#include "vegas_pick.cuh"

namespace vegas {
const void *sample_kernel_f64_genz_osc(int d, bool priv) { return pick_family<ACC_F64, F_GENZ_OSC>(d, priv); }
const void *sample_strat_kernel_f64_genz_osc(int d, bool priv) { return pick_strat<ACC_F64, F_GENZ_OSC>(d, priv); }
const void *sample_kernel_f64_genz_osc_wide(int d) { return pick_family_wide<ACC_F64, F_GENZ_OSC>(d); }
}  // namespace vegas
