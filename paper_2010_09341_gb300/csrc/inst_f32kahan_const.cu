// Sampling kernels: mode ACC_F32_KAHAN, family F_CONST (generated instantiation unit).
#include "vegas_pick.cuh"

namespace vegas {
const void *sample_kernel_f32kahan_const(int d, bool priv) { return pick_family<ACC_F32_KAHAN, F_CONST>(d, priv); }
const void *sample_strat_kernel_f32kahan_const(int d, bool priv) { return pick_strat<ACC_F32_KAHAN, F_CONST>(d, priv); }
}  // namespace vegas
