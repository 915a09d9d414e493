// Sampling kernels: mode ACC_F32_SUM64, family F_GENZ_GAUSS (generated instantiation unit).
#include "vegas_pick.cuh"

namespace vegas {
const void *sample_kernel_f32sum64_genz_gauss(int d, bool priv) { return pick_family<ACC_F32_SUM64, F_GENZ_GAUSS>(d, priv); }
const void *sample_strat_kernel_f32sum64_genz_gauss(int d, bool priv) { return pick_strat<ACC_F32_SUM64, F_GENZ_GAUSS>(d, priv); }
}  // namespace vegas
