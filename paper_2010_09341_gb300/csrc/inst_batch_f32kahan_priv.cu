// Batched sampling kernel: mode ACC_F32_KAHAN, layout 1 (lane-private copies) (instantiation unit).
#include "vegas_batch_sample.cuh"

namespace vegas {
const void *batch_sample_kernel_f32kahan_priv() {
    return reinterpret_cast<const void *>(&batch_sample_kernel_t<ACC_F32_KAHAN, 1>);
}
}  // namespace vegas
