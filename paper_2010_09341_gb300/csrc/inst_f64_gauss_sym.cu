// Sampling kernels: mode ACC_F64, family F_GAUSS_SYM (generated instantiation unit).
#include "vegas_pick.cuh"

namespace vegas {
const void *sample_kernel_f64_gauss_sym(int d, bool priv) { return pick_family<ACC_F64, F_GAUSS_SYM>(d, priv); }
const void *sample_strat_kernel_f64_gauss_sym(int d, bool priv) { return pick_strat<ACC_F64, F_GAUSS_SYM>(d, priv); }
const void *sample_kernel_f64_gauss_sym_wide(int d) { return pick_family_wide<ACC_F64, F_GAUSS_SYM>(d); }
}  // namespace vegas
