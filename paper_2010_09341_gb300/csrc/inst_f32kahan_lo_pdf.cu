// Sampling kernels: mode ACC_F32_KAHAN, family F_LO_PDF (generated instantiation unit).
#include "vegas_pick.cuh"

namespace vegas {
const void *sample_kernel_f32kahan_lo_pdf(int d, bool priv) { return pick_family<ACC_F32_KAHAN, F_LO_PDF>(d, priv); }
const void *sample_strat_kernel_f32kahan_lo_pdf(int d, bool priv) { return pick_strat<ACC_F32_KAHAN, F_LO_PDF>(d, priv); }
}  // namespace vegas
