// Sampling kernels of mode ACC_F32_KAHAN (see vegas_sample.cuh).
#include "vegas_pick.cuh"

namespace vegas {
const void *sample_kernel_f32kahan(int fam, int tier, bool priv) { return pick_kernel<ACC_F32_KAHAN>(fam, tier, priv); }
}  // namespace vegas
