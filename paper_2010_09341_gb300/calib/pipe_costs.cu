// pipe_costs.cu -- issue cost of the instruction kinds the VEGAS sampling
// kernel is made of, measured on the GPU it runs on.
//
// One block of 1024 threads (32 warps) per SM; every thread runs 8
// independent chains of one instruction kind for IT iterations between two
// clock64() reads, so latency is hidden and the per-SM-sub-partition cost of
// one warp instruction is  cycles / (8 warps * 8 chains * IT).  The loop
// itself adds three instructions per 8 chain steps (reported as "loop").
// Shared-memory atomics go to lane-private addresses (no bank conflicts).
//
// Build and run (one GPU):
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o pipe_costs pipe_costs.cu && ./pipe_costs
// Output: one line per kind, cycles per warp instruction per sub-partition
// (1.0 = one warp instruction per clock per scheduler, 32 lanes per clock).
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

#include "../csrc/vegas_device.cuh"

constexpr int kIt = 2048;
constexpr int kThreads = 1024;

enum Kind : int {
    K_FFMA, K_IADD, K_LOP3, K_IMAD, K_MULHI, K_MULWIDE_XOR, K_MULWIDE_XOR_2FFMA, K_FFMA_LOP3,
    K_ATOMS_U32, K_ATOMS_F32, K_ATOMS_F64, K_DFMA, K_EX2, K_EXP64, K_I2F, K_I2F_2FFMA, K_SHF,
    K_ATOMS_U64, K_MATCH_ANY, K_COS64, K_LOG2_64, K_EXP2_64, K_RCP64, K_FEXP2_64, K_COUNT
};

template <int V>
__global__ void __launch_bounds__(kThreads) chains(unsigned long long *cycles, unsigned *sink, unsigned seed) {
    __shared__ unsigned cells_u[32 * 8];
    __shared__ float cells_f[32 * 8];
    __shared__ double cells_d[32 * 8];
    __shared__ unsigned long long cells_q[32 * 8];
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned lane = threadIdx.x & 31;
    if (threadIdx.x < 32 * 8) {
        cells_u[threadIdx.x] = 0u;
        cells_f[threadIdx.x] = 0.f;
        cells_d[threadIdx.x] = 0.0;
        cells_q[threadIdx.x] = 0ull;
    }
    unsigned x[8];
    float f[8];
    double g[8];
    float g2f[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        g2f[c] = 1.0f + c * 1e-4f;
        x[c] = t * 2654435761u + c * 977u + seed;
        f[c] = 1.0f + (t & 7) * 1e-3f + c * 1e-4f;
        g[c] = 1.0 + c * 1e-4;
    }
    __syncthreads();
    const unsigned long long c0 = clock64();
#pragma unroll 1
    for (int it = 0; it < kIt; ++it) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            if (V == K_FFMA) {
                asm volatile("fma.rn.f32 %0, %0, 0f3F7FFFEF, 0f33D6BF95;" : "+f"(f[c]));
            } else if (V == K_IADD) {
                asm volatile("add.u32 %0, %0, 0x9E3779B9;" : "+r"(x[c]));
            } else if (V == K_LOP3) {
                asm volatile("lop3.b32 %0, %0, 0x9E3779B9, 0x7F4A7C15, 0x96;" : "+r"(x[c]));
            } else if (V == K_IMAD) {
                asm volatile("mad.lo.u32 %0, %0, 0x2545F491, 0x9E3779B9;" : "+r"(x[c]));
            } else if (V == K_MULHI) {
                asm volatile("mul.hi.u32 %0, %0, 0xD2511F53;" : "+r"(x[c]));
            } else if (V == K_MULWIDE_XOR || V == K_MULWIDE_XOR_2FFMA) {
                unsigned lo, hi;
                asm volatile("{ .reg .u64 p; mul.wide.u32 p, %2, 0xD2511F53; mov.b64 {%0, %1}, p; }"
                             : "=r"(lo), "=r"(hi) : "r"(x[c]));
                asm volatile("xor.b32 %0, %1, %2;" : "=r"(x[c]) : "r"(lo), "r"(hi));
                if (V == K_MULWIDE_XOR_2FFMA) {
                    asm volatile("fma.rn.f32 %0, %0, 0f3F7FFFEF, 0f33D6BF95;" : "+f"(f[c]));
                    asm volatile("fma.rn.f32 %0, %0, 0f3F7FFFEF, 0f33D6BF95;" : "+f"(f[c]));
                }
            } else if (V == K_FFMA_LOP3) {
                asm volatile("fma.rn.f32 %0, %0, 0f3F7FFFEF, 0f33D6BF95;" : "+f"(f[c]));
                asm volatile("lop3.b32 %0, %0, 0x9E3779B9, 0x7F4A7C15, 0x96;" : "+r"(x[c]));
            } else if (V == K_ATOMS_U32) {
                atomicAdd(&cells_u[c * 32 + lane], x[c]);  // lane-private: bank = lane
            } else if (V == K_ATOMS_F32) {
                atomicAdd(&cells_f[c * 32 + lane], f[c]);
            } else if (V == K_ATOMS_F64) {
                atomicAdd(&cells_d[c * 32 + lane], g[c]);
            } else if (V == K_EXP64) {
                g[c] = exp(-g[c]);  // stays in (0.3, 1]: converges to 0.567
            } else if (V == K_EXP2_64) {
                g[c] = exp2(-g[c]);  // stays in (0.5, 1]: converges to 0.64
            } else if (V == K_FEXP2_64) {
                g[c] = vegas::fexp2(-g[c]);  // the library's table-driven 2^x
            } else if (V == K_COS64) {
                g[c] = cos(g[c]);   // stays in [cos 1, 1]: converges to 0.739
            } else if (V == K_RCP64) {
                g[c] = 1.0 / (g[c] + 1.0);  // converges to 0.618
            } else if (V == K_LOG2_64) {
                g[c] = 1.0 + log2(g[c] + 1.0);  // stays in [1, 2]: converges to 2
            } else if (V == K_DFMA) {
                asm volatile("fma.rn.f64 %0, %0, 0d3FEFFFFFDE7210BE, 0d3E7AD7F29ABCAF48;" : "+d"(g[c]));
            } else if (V == K_EX2) {
                asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(f[c]));
            } else if (V == K_I2F || V == K_I2F_2FFMA) {
                // the float's own bits converted as an unsigned integer: a chain of conversions
                asm volatile("{ .reg .u32 b; mov.b32 b, %0; cvt.rn.f32.u32 %0, b; }" : "+f"(f[c]));
                if (V == K_I2F_2FFMA) {
                    asm volatile("fma.rn.f32 %0, %0, 0f3F7FFFEF, 0f33D6BF95;" : "+f"(g2f[c]));
                    asm volatile("fma.rn.f32 %0, %0, 0f3F7FFFEF, 0f33D6BF95;" : "+f"(g2f[c]));
                }
            } else if (V == K_SHF) {
                asm volatile("shf.r.clamp.b32 %0, %0, 0x7F, 9;" : "+r"(x[c]));
            } else if (V == K_ATOMS_U64) {
                atomicAdd(&cells_q[c * 32 + lane], static_cast<unsigned long long>(x[c]));
            } else if (V == K_MATCH_ANY) {
                unsigned m;
                asm volatile("match.any.sync.b32 %0, %1, 0xFFFFFFFF;" : "=r"(m) : "r"(x[c]));
                x[c] ^= m;
            }
        }
    }
    const unsigned long long c1 = clock64();
    __syncthreads();
    unsigned r = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        r += x[c] + __float_as_uint(f[c]) + __float_as_uint(g2f[c]) + static_cast<unsigned>(g[c] * 1e3);
    if (threadIdx.x < 32 * 8)
        r += cells_u[threadIdx.x] + __float_as_uint(cells_f[threadIdx.x]) + static_cast<unsigned>(cells_d[threadIdx.x]) +
             static_cast<unsigned>(cells_q[threadIdx.x]);
    sink[t] = r;
    if (threadIdx.x == 0) cycles[blockIdx.x] = c1 - c0;
}

int main() {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess || sms <= 0) {
        fprintf(stderr, "no CUDA device\n");
        return 1;
    }
    const int blocks = sms;  // one block of 32 warps per SM
    unsigned *sink = nullptr;
    unsigned long long *cyc = nullptr;
    if (cudaMalloc(&sink, sizeof(unsigned) * blocks * kThreads) != cudaSuccess ||
        cudaMalloc(&cyc, sizeof(unsigned long long) * blocks) != cudaSuccess) {
        fprintf(stderr, "cudaMalloc failed\n");
        return 1;
    }
    struct Case {
        const char *name;
        double instr;  // instructions per chain step
        void (*k)(unsigned long long *, unsigned *, unsigned);
    } cases[] = {
        {"ffma", 1, chains<K_FFMA>},
        {"iadd", 1, chains<K_IADD>},
        {"lop3", 1, chains<K_LOP3>},
        {"imad (32-bit)", 1, chains<K_IMAD>},
        {"mul.hi.u32", 1, chains<K_MULHI>},
        {"mul.wide.u32 + xor", 2, chains<K_MULWIDE_XOR>},
        {"mul.wide.u32 + xor + 2 ffma", 4, chains<K_MULWIDE_XOR_2FFMA>},
        {"ffma + lop3", 2, chains<K_FFMA_LOP3>},
        {"shared atomic add u32", 1, chains<K_ATOMS_U32>},
        {"shared atomic add f32", 1, chains<K_ATOMS_F32>},
        {"shared atomic add f64", 1, chains<K_ATOMS_F64>},
        {"dfma", 1, chains<K_DFMA>},
        {"ex2.approx", 1, chains<K_EX2>},
        {"exp (double, one call)", 1, chains<K_EXP64>},
        {"cvt.rn.f32.u32", 1, chains<K_I2F>},
        {"cvt.rn.f32.u32 + 2 ffma", 3, chains<K_I2F_2FFMA>},
        {"shf.r (funnel shift)", 1, chains<K_SHF>},
        {"shared atomic add u64", 1, chains<K_ATOMS_U64>},
        {"match.any.sync.b32", 2, chains<K_MATCH_ANY>},
        {"exp2 (double, one call)", 1, chains<K_EXP2_64>},
        {"cos (double, one call)", 1, chains<K_COS64>},
        {"log2 (double, one call + 2 dadd)", 1, chains<K_LOG2_64>},
        {"1/x (double, one division + dadd)", 1, chains<K_RCP64>},
        {"vegas::fexp2 (double, table-driven)", 1, chains<K_FEXP2_64>},
    };
    unsigned long long *h = new unsigned long long[blocks];
    int rc = 0;
    printf("# cycles per chain step per SM sub-partition (8 warps x 8 chains x %d steps each)\n", kIt);
    for (const Case &cs : cases) {
        cs.k<<<blocks, kThreads>>>(cyc, sink, 1u);  // warm-up
        cs.k<<<blocks, kThreads>>>(cyc, sink, 2u);
        const cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess || cudaMemcpy(h, cyc, sizeof(unsigned long long) * blocks, cudaMemcpyDeviceToHost) != cudaSuccess) {
            fprintf(stderr, "%s: %s\n", cs.name, cudaGetErrorString(e));
            rc = 1;
            break;
        }
        double mean = 0.0;
        for (int b = 0; b < blocks; ++b) mean += static_cast<double>(h[b]);
        mean /= blocks;
        const double steps = 8.0 * 8.0 * kIt;  // per sub-partition: 8 warps x 8 chains x kIt
        const double per_step = mean / steps;
        printf("%-30s %7.3f cycles/step  %7.3f cycles/instruction\n", cs.name, per_step, per_step / cs.instr);
    }
    printf("# loop overhead included: 3 instructions per 8 chain steps\n");
    delete[] h;
    cudaFree(sink);
    cudaFree(cyc);
    return rc;
}
