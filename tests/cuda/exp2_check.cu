// exp2_check.cu -- the library's FP64 2^x (vegas::fexp2, Tang's table-driven
// method) beside CUDA's exp2 on the same inputs, for the test that compares
// them in ulp.  Built by the test with nvcc into a shared library.
#include <cuda_runtime.h>

#include "../../paper_2010_09341_gb300/csrc/vegas_device.cuh"

__global__ void exp2_pair(const double *x, double *mine, double *ref, long long n) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) {
        mine[i] = vegas::fexp2(x[i]);
        ref[i] = exp2(x[i]);
    }
}

extern "C" int exp2_check(const double *x, double *mine, double *ref, long long n) {
    if (n <= 0) return 0;
    exp2_pair<<<static_cast<unsigned>((n + 255) / 256), 256>>>(x, mine, ref, n);
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : 1;
}
