// Sampling kernels: mode ACC_F64, family F_LO (generated instantiation unit).
#include "vegas_pick.cuh"

namespace vegas {
const void *sample_kernel_f64_lo(int d, bool priv) { return pick_family<ACC_F64, F_LO>(d, priv); }
const void *sample_strat_kernel_f64_lo(int d, bool priv) { return pick_strat<ACC_F64, F_LO>(d, priv); }
const void *sample_kernel_f64_lo_wide(int d) { return pick_family_wide<ACC_F64, F_LO>(d); }
}  // namespace vegas
