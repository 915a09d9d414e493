// Test-only reference: runs cuRAND's own Philox4x32-10 device function over
// n counters so the library's independent implementation can be compared to
// it on the GPU.
#include <cstdint>
#include <curand_kernel.h>

__global__ void curand_ref_kernel(const uint4 *ctr, const uint2 *key, uint4 *out, long long n) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

extern "C" int curand_ref_philox(const void *ctr, const void *key, void *out, long long n) {
    if (n <= 0) return 0;
    const unsigned blocks = static_cast<unsigned>((n + 255) / 256);
    curand_ref_kernel<<<blocks, 256>>>(static_cast<const uint4 *>(ctr), static_cast<const uint2 *>(key),
                                       static_cast<uint4 *>(out), n);
    return static_cast<int>(cudaDeviceSynchronize());
}
