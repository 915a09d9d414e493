// vegas_batch.cuh -- many integrals of uneven size in one persistent launch.
//
// The batched form of one VEGAS iteration: every active integral (slot) runs
// one iteration -- sampling, finalize, refinement -- per step.  Sampling work
// is split into tiles of (slot, sample range); the blocks of a persistent
// kernel claim tiles from a global counter, so large and small integrals mix
// without idle SMs.  Sample s of slot k in iteration t draws the same Philox
// words as in a single-integral context with the same seed and integral id,
// so a slot's result equals its result alone up to summation order.
#pragma once

#include "vegas_kernels.cuh"

namespace vegas {

// Per-slot state, resident in the batch pool on the device.
struct SlotDev {
    // set when the slot is added
    int family, d, N, smooth;
    long long n;              // samples per iteration
    uint32_t key0, key1;
    double jinit64;           // initial weight, FP64 path
    float jinit32, n4;        // initial weight and N^4, FP32 paths
    double alpha;
    double inv_scale;         // 1 / (initial power-of-two scale of v)
    double jmul;              // power-of-two rescale of v set by the last finalize
    FamConsts<float> fc32;
    FamConsts<double> fc64;
    double *edges;            // d x (N+1)
    void *table;              // d x N entries of the batch's mode
    double *acc;              // 2 + d N (scaled), zeroed after each finalize
    double *last;             // 2 + d N (unscaled) of the last iteration
    double *center;           // d sampling-table centres (table_center)
    // updated by the kernels
    unsigned long long nonfinite;
    float hscale;
    int t;                    // Philox iteration word of the next iteration
    CombState cs;             // running combination (comb_add)
    IterRec last_it;
    CombRec comb;
};

// What one step runs: the active slots in order, the first tile of each
// (tile_prefix[k], with tile_prefix[n_items] = total) and the first
// (slot, dimension) pair of each for the refinement.
struct PlanHeader {
    int n_items;
    int total_dims;
    int tile_samples;
    int pad;
    long long total_tiles;
};

struct BatchResult {
    int slot;
    int t;                    // Philox iteration word of the iteration just run
    IterRec it;
    CombRec comb;
};

struct BatchArgs {
    const PlanHeader *hdr;
    const int *items;             // slot index per item
    const long long *tile_prefix; // n_items + 1
    const int *dim_prefix;        // n_items + 1
    SlotDev *slots;               // slot table (indexed by slot id)
    unsigned long long *counter;  // tile claim counter (reset by finalize)
    BatchResult *results;         // n_items
    int mode;
};

// Threads per block of the persistent sampling kernel: one block per SM, 24
// warps, up to 80 registers a thread.  (Measured on the 512-integral mix:
// 640 threads 10.78 ms per step, 768 10.64, 896 10.73, 1024 11.11 -- with
// fewer registers the out-of-line samplers spill.)
constexpr int kBatchThreads = 768;

// The batched sampling kernel of one mode and shared-memory layout (1 =
// lane-private copies, 2 = half as many, 0 = one copy per cell; instantiated
// in inst_batch_*.cu) and its dynamic shared memory for max_cells cells.
const void *batch_sample_kernel(int mode, int layout);
size_t batch_sample_smem(int mode, int layout, int max_cells);

}  // namespace vegas
