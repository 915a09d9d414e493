// Batched sampling kernel: mode ACC_F32_SUM64, layout 0 (one copy per cell) (instantiation unit).
#include "vegas_batch_sample.cuh"

namespace vegas {
const void *batch_sample_kernel_f32sum64_shared() {
    return reinterpret_cast<const void *>(&batch_sample_kernel_t<ACC_F32_SUM64, 0>);
}
}  // namespace vegas
