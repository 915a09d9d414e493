// Sampling kernels of mode ACC_F32_SUM64 (see vegas_sample.cuh).
#include "vegas_pick.cuh"

namespace vegas {
const void *sample_kernel_f32sum64(int fam, int tier, bool priv) { return pick_kernel<ACC_F32_SUM64>(fam, tier, priv); }
}  // namespace vegas
