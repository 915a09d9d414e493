// vegas_batch.cu -- the batched form: a slot pool on the device, one step =
// one VEGAS iteration of every active slot in three kernels captured as a
// CUDA graph (plan upload, persistent sampling, finalize, refinement, result
// download).  Host code: slot admission over a first-fit pool, the step plan,
// graph capture and the tile-size autotuner.
#include "../../include/vegas.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <vector>

#include "vegas_batch.cuh"
#include "vegas_nvtx.h"
#include "vegas_refine.cuh"

namespace vegas {

const void *batch_sample_kernel_f32kahan_priv();
const void *batch_sample_kernel_f32kahan_half();
const void *batch_sample_kernel_f32kahan_shared();
const void *batch_sample_kernel_f32sum64_priv();
const void *batch_sample_kernel_f32sum64_half();
const void *batch_sample_kernel_f32sum64_shared();

const void *batch_sample_kernel(int mode, int layout) {
    if (mode == ACC_F32_KAHAN)
        return layout == 1 ? batch_sample_kernel_f32kahan_priv()
                           : (layout == 2 ? batch_sample_kernel_f32kahan_half() : batch_sample_kernel_f32kahan_shared());
    if (mode == ACC_F32_SUM64)
        return layout == 1 ? batch_sample_kernel_f32sum64_priv()
                           : (layout == 2 ? batch_sample_kernel_f32sum64_half() : batch_sample_kernel_f32sum64_shared());
    return nullptr;
}

size_t batch_sample_smem(int mode, int layout, int max_cells) { return sample_smem(mode, layout, max_cells, 1); }

// ------------------------------------------------------------- kernels
// Iteration result and running combination of every item's slot (one block
// per item, grid-stride), then the accumulators move to `last` and clear.
// The running combination is comb_add's (shifted sums; iterations without a
// finite value left out).  Also writes the next iteration's fixed-point
// histogram scale and resets the tile counter for the next step.
__global__ void __launch_bounds__(128)
batch_finalize_kernel(const BatchArgs ba) {
    const int n_items = ba.hdr->n_items;
    if (blockIdx.x == 0 && threadIdx.x == 0) *ba.counter = 0ull;
    for (int k = blockIdx.x; k < n_items; k += gridDim.x) {
        const int slot = ba.items[k];
        SlotDev &sd = ba.slots[slot];
        const int total = 2 + sd.d * sd.N;
        __shared__ double inv_s;
        if (threadIdx.x == 0) {
            const long long nf = static_cast<long long>(sd.nonfinite);
            const long long ne = sd.n - nf;
            const double m2 = ne > 0 ? sd.acc[1] / static_cast<double>(ne) : 0.0;
            const double jm = sd.jmul;
            double ratio;
            float hs;
            const double m1 = ne > 0 ? sd.acc[0] / static_cast<double>(ne) : 0.0;
            next_scales(m2, m1, static_cast<double>(sd.jinit32) * jm, &ratio, &hs);
            const double inv1 = sd.inv_scale / jm, inv2 = inv1 * inv1;
            inv_s = inv1;
            sd.jmul = jm * ratio;
            IterRec r;
            r.n = ne;
            r.n_nonfinite = nf;
            if (ne >= 2) {
                const double I = sd.acc[0] * inv1 / static_cast<double>(ne);
                const double var = (sd.acc[1] * inv2 / static_cast<double>(ne) - I * I) /
                                   static_cast<double>(ne - 1);
                r.I = I;
                r.sigma = var > 0.0 ? sqrt(var) : 0.0;
            } else {
                r.I = ne == 1 ? sd.acc[0] * inv1 : 0.0;
                r.sigma = 0.0;
            }
            const bool combined = ne > 0;
            comb_add(sd.cs, r.I, r.sigma, combined);
            const CombRec c = comb_result(sd.cs, combined);
            sd.last_it = r;
            sd.comb = c;
            BatchResult br;
            br.slot = slot;
            br.t = sd.t;
            br.it = r;
            br.comb = c;
            ba.results[k] = br;
            sd.t += 1;
            sd.nonfinite = 0ull;
            sd.hscale = hs;
        }
        __syncthreads();
        const double inv1 = inv_s, inv2 = inv_s * inv_s;
        for (int c = threadIdx.x; c < total; c += blockDim.x) {
            sd.last[c] = sd.acc[c] * (c == 0 ? inv1 : inv2);
            sd.acc[c] = 0.0;
        }
        __syncthreads();
    }
}

// Refinement of every (item, dimension) pair: one block per pair, grid-stride.
__global__ void __launch_bounds__(kRefineThreads)
batch_refine_kernel(const BatchArgs ba) {
    extern __shared__ double rs[];
    const int n_items = ba.hdr->n_items;
    const int total = ba.hdr->total_dims;
    for (int p = blockIdx.x; p < total; p += gridDim.x) {
        int lo = 0, hi = n_items - 1;  // last item with dim_prefix <= p
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (ba.dim_prefix[mid] <= p) lo = mid;
            else hi = mid - 1;
        }
        SlotDev &sd = ba.slots[ba.items[lo]];
        const int j = p - ba.dim_prefix[lo];
        const int N = sd.N;
        const size_t entry = ba.mode == ACC_F64 ? sizeof(double2) : sizeof(float2);
        refine_block(sd.last + 2 + static_cast<size_t>(j) * N, sd.edges + static_cast<size_t>(j) * (N + 1),
                     static_cast<char *>(sd.table) + entry * static_cast<size_t>(j) * N, ba.mode, N,
                     sd.alpha, sd.smooth, sd.center[j], rs);
    }
}

// Undo a sampling pass without a finalize (autotuning): clear every item's
// accumulators and non-finite count, and the tile counter.
__global__ void batch_reset_kernel(const BatchArgs ba) {
    const int n_items = ba.hdr->n_items;
    if (blockIdx.x == 0 && threadIdx.x == 0) *ba.counter = 0ull;
    for (int k = blockIdx.x; k < n_items; k += gridDim.x) {
        SlotDev &sd = ba.slots[ba.items[k]];
        const int total = 2 + sd.d * sd.N;
        for (int c = threadIdx.x; c < total; c += blockDim.x) sd.acc[c] = 0.0;
        if (threadIdx.x == 0) sd.nonfinite = 0ull;
    }
}

}  // namespace vegas

using namespace vegas;

namespace {

thread_local char g_batch_error[256] = "";

#define VB_CK(call)                                                                       \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            snprintf(g_batch_error, sizeof(g_batch_error), "%s: %s", #call, cudaGetErrorString(e_)); \
            return VEGAS_ECUDA;                                                           \
        }                                                                                 \
    } while (0)

constexpr size_t kA = 256;
inline size_t up(size_t x) { return (x + kA - 1) / kA * kA; }

// Fixed part of the batch workspace for max_slots slots.
struct BatchLayout {
    size_t plan, items, tile_prefix, dim_prefix, results, counter, slots, pool, fixed;
};

BatchLayout batch_layout(int max_slots) {
    BatchLayout L;
    size_t o = 0;
    L.plan = o;
    o = up(o + sizeof(PlanHeader));
    L.items = o;
    o = up(o + sizeof(int) * max_slots);
    L.tile_prefix = o;
    o = up(o + sizeof(long long) * (max_slots + 1));
    L.dim_prefix = o;
    o = up(o + sizeof(int) * (max_slots + 1));
    L.results = o;
    o = up(o + sizeof(BatchResult) * max_slots);
    L.counter = o;
    o = up(o + sizeof(unsigned long long));
    L.slots = o;
    o = up(o + sizeof(SlotDev) * max_slots);
    L.pool = o;
    L.fixed = o;
    return L;
}

size_t slot_pool_bytes(int d, int N) {
    const size_t cells = static_cast<size_t>(d) * N;
    return up(sizeof(double) * d * (N + 1)) + up(16 * cells) + 2 * up(sizeof(double) * (2 + cells)) +
           up(sizeof(double) * d);  // the table centres
}

// First-fit allocator over byte ranges of the device pool (host bookkeeping).
class PoolAllocator {
  public:
    void reset(size_t bytes) {
        free_.clear();
        if (bytes) free_[0] = bytes;
        total_ = bytes;
    }
    bool alloc(size_t n, size_t *off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n;
                const size_t roff = it->first + n;
                free_.erase(it);
                if (rest) free_[roff] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n) {
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {  // merge right
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {  // merge left
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t free_bytes() const {
        size_t s = 0;
        for (auto &kv : free_) s += kv.second;
        return s;
    }
    size_t largest() const {
        size_t s = 0;
        for (auto &kv : free_) s = std::max(s, kv.second);
        return s;
    }

  private:
    std::map<size_t, size_t> free_;
    size_t total_ = 0;
};

// Host copy of the step plan (pinned; the graph's upload reads it).
struct HostPlan {
    PlanHeader hdr;
    std::vector<int> items;
};

}  // namespace

struct SlotHost {
    bool used = false;
    size_t off = 0, bytes = 0;
    long long n = 0;
    int d = 0, N = 0;
};

struct vegas_batch {
    int max_slots, mode, precision;
    cudaStream_t stream;
    bool own_stream = false;
    char *ws;
    size_t ws_bytes;
    BatchLayout L;
    PoolAllocator pool;
    std::vector<SlotHost> slots;
    int max_cells = 0;     // largest d N the kernels were configured for
    int max_N = 2;
    int tile_samples = 8192;
    int threads = kBatchThreads;
    // pinned host buffers
    char *h_plan = nullptr;      // image of the device plan region [L.plan, L.results)
    BatchResult *h_results = nullptr;
    // graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool graph_ok = false;
    int graph_cells = 0, graph_N = 0, graph_tile = 0;
    bool in_flight = false;
    int last_items = 0;
    BatchArgs args;
    int sm_count = 0;
    size_t smem_optin = 0;
    int layout = 1;        // shared-memory layout of the sampling kernel
    int layout_req = -1;   // requested layout (vegas_batch_set_shape); -1: the most copies that fit
    const void *kfn = nullptr;
    size_t smem = 0;
    int sample_blocks = 0;
};

namespace {

vegas_status batch_invalidate_graph(vegas_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_ok = false;
    return VEGAS_OK;
}

// Choose the sampling kernel and its launch for the current largest slot:
// the requested layout if it fits, else the most lane-private copies that fit.
vegas_status batch_configure(vegas_batch *b, int cells) {
    const size_t budget = b->smem_optin > 2048 ? b->smem_optin - 2048 : 0;
    int layout = 1;
    if (batch_sample_smem(b->mode, layout, cells) > budget) layout = 2;
    if (batch_sample_smem(b->mode, layout, cells) > budget) layout = 0;
    if (b->layout_req >= 0 && batch_sample_smem(b->mode, b->layout_req, cells) <= budget) layout = b->layout_req;
    size_t smem = batch_sample_smem(b->mode, layout, cells);
    if (smem > budget) return VEGAS_EINVAL;
    const void *fn = batch_sample_kernel(b->mode, layout);
    if (!fn) return VEGAS_EINVAL;
    VB_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    int occ = 0;
    VB_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, b->threads, smem));
    if (occ < 1) return VEGAS_EINVAL;
    b->layout = layout;
    b->kfn = fn;
    b->smem = smem;
    b->sample_blocks = occ * b->sm_count;
    b->max_cells = cells;
    return VEGAS_OK;
}

void batch_fill_args(vegas_batch *b) {
    BatchArgs &a = b->args;
    a.hdr = reinterpret_cast<const PlanHeader *>(b->ws + b->L.plan);
    a.items = reinterpret_cast<const int *>(b->ws + b->L.items);
    a.tile_prefix = reinterpret_cast<const long long *>(b->ws + b->L.tile_prefix);
    a.dim_prefix = reinterpret_cast<const int *>(b->ws + b->L.dim_prefix);
    a.slots = reinterpret_cast<SlotDev *>(b->ws + b->L.slots);
    a.counter = reinterpret_cast<unsigned long long *>(b->ws + b->L.counter);
    a.results = reinterpret_cast<BatchResult *>(b->ws + b->L.results);
    a.mode = b->mode;
}

// Build the host plan: active slots, largest sample count first (its tiles
// are claimed first, small slots fill the tail of the step).
int batch_build_plan(vegas_batch *b) {
    std::vector<int> act;
    for (int s = 0; s < b->max_slots; ++s)
        if (b->slots[s].used) act.push_back(s);
    std::stable_sort(act.begin(), act.end(),
                     [&](int x, int y) { return b->slots[x].n > b->slots[y].n; });
    const BatchLayout &L = b->L;
    PlanHeader *hdr = reinterpret_cast<PlanHeader *>(b->h_plan + (L.plan - L.plan));
    int *items = reinterpret_cast<int *>(b->h_plan + (L.items - L.plan));
    long long *tp = reinterpret_cast<long long *>(b->h_plan + (L.tile_prefix - L.plan));
    int *dp = reinterpret_cast<int *>(b->h_plan + (L.dim_prefix - L.plan));
    long long tiles = 0;
    int dims = 0;
    for (size_t k = 0; k < act.size(); ++k) {
        const SlotHost &sh = b->slots[act[k]];
        items[k] = act[k];
        tp[k] = tiles;
        dp[k] = dims;
        tiles += (sh.n + b->tile_samples - 1) / b->tile_samples;
        dims += sh.d;
    }
    tp[act.size()] = tiles;
    dp[act.size()] = dims;
    hdr->n_items = static_cast<int>(act.size());
    hdr->total_dims = dims;
    hdr->tile_samples = b->tile_samples;
    hdr->pad = 0;
    hdr->total_tiles = tiles;
    return static_cast<int>(act.size());
}

vegas_status batch_enqueue_kernels(vegas_batch *b, bool finalize) {
    void *params[] = {&b->args};
    VB_CK(cudaLaunchKernel(b->kfn, dim3(b->sample_blocks), dim3(b->threads), params, b->smem, b->stream));
    if (finalize) {
        const int fblocks = std::min(b->max_slots, 4 * b->sm_count);
        VB_CK(cudaLaunchKernel(reinterpret_cast<const void *>(&batch_finalize_kernel), dim3(fblocks), dim3(128),
                               params, 0, b->stream));
        const size_t rsm = static_cast<size_t>(4 * b->max_N + 2) * sizeof(double);
        VB_CK(cudaLaunchKernel(reinterpret_cast<const void *>(&batch_refine_kernel), dim3(4 * b->sm_count),
                               dim3(kRefineThreads), params, rsm, b->stream));
    }
    return VEGAS_OK;
}

vegas_status batch_capture(vegas_batch *b) {
    batch_invalidate_graph(b);
    const size_t plan_bytes = b->L.results - b->L.plan;
    VB_CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemcpyAsync(b->ws + b->L.plan, b->h_plan, plan_bytes, cudaMemcpyHostToDevice, b->stream);
    vegas_status st = VEGAS_OK;
    if (e == cudaSuccess) st = batch_enqueue_kernels(b, true);
    if (e == cudaSuccess && st == VEGAS_OK)
        e = cudaMemcpyAsync(b->h_results, b->ws + b->L.results, sizeof(BatchResult) * b->max_slots,
                            cudaMemcpyDeviceToHost, b->stream);
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->stream, &g);
    if (st != VEGAS_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess || ee != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        snprintf(g_batch_error, sizeof(g_batch_error), "graph capture: %s",
                 cudaGetErrorString(e != cudaSuccess ? e : ee));
        return VEGAS_ECUDA;
    }
    b->graph = g;
    VB_CK(cudaGraphInstantiate(&b->exec, g, 0));
    b->graph_ok = true;
    b->graph_cells = b->max_cells;
    b->graph_N = b->max_N;
    b->graph_tile = b->tile_samples;
    return VEGAS_OK;
}

vegas_status batch_sync(vegas_batch *b) {
    if (b->in_flight) {
        VB_CK(cudaStreamSynchronize(b->stream));
        b->in_flight = false;
    }
    return VEGAS_OK;
}

int prec_mode(int precision) {
    if (precision == VEGAS_FP32_KAHAN) return ACC_F32_KAHAN;
    if (precision == VEGAS_FP32_ACC64) return ACC_F32_SUM64;
    return -1;
}

}  // namespace

// Host-side helpers of vegas_api.cu (family constants, parameter counts).
namespace vegas {
bool host_prepare_family(int family, int d, const double *p, FamilyConsts &fc, double &norm, double &fmax);
void host_fp32_consts(int family, int d, const FamilyConsts &fc, FamConsts<float> &out, double &kappa);
int host_n_params(int family, int d);
}

extern "C" {

const char *vegas_batch_last_error(void) { return g_batch_error; }

size_t vegas_batch_workspace_bytes(int32_t max_slots, size_t pool_bytes) {
    if (max_slots < 1 || max_slots > (1 << 20)) return 0;
    return batch_layout(max_slots).fixed + up(pool_bytes);
}

size_t vegas_batch_slot_bytes(const vegas_config *cfg) {
    if (!cfg || cfg->n_dim < 1 || cfg->n_dim > VEGAS_MAX_DIM || cfg->n_bins < 2 || cfg->n_bins > VEGAS_MAX_BINS)
        return 0;
    return slot_pool_bytes(cfg->n_dim, cfg->n_bins);
}

vegas_status vegas_batch_create(int32_t max_slots, int32_t precision, void *stream, void *dev_ws,
                                size_t ws_bytes, vegas_batch **out) {
    VEGAS_NVTX_RANGE();
    if (!out) return VEGAS_EINVAL;
    *out = nullptr;
    const int mode = prec_mode(precision);
    if (mode < 0 || max_slots < 1 || max_slots > (1 << 20) || !dev_ws) return VEGAS_EINVAL;
    if (reinterpret_cast<uintptr_t>(dev_ws) % kA) return VEGAS_EINVAL;
    const BatchLayout L = batch_layout(max_slots);
    if (ws_bytes < L.fixed) return VEGAS_ENOMEM;
    vegas_batch *b = new vegas_batch();
    b->max_slots = max_slots;
    b->mode = mode;
    b->precision = precision;
    b->stream = static_cast<cudaStream_t>(stream);
    if (!b->stream) {  // the legacy NULL stream cannot be captured into a graph
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return VEGAS_ECUDA;
        }
        b->own_stream = true;
    }
    b->ws = static_cast<char *>(dev_ws);
    b->ws_bytes = ws_bytes;
    b->L = L;
    b->pool.reset(ws_bytes - L.fixed);
    b->slots.resize(max_slots);
    int dev = 0, v = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    b->smem_optin = static_cast<size_t>(v);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_plan, L.results - L.plan);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_results, sizeof(BatchResult) * max_slots);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->ws, 0, L.fixed, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        snprintf(g_batch_error, sizeof(g_batch_error), "vegas_batch_create: %s", cudaGetErrorString(e));
        if (b->h_plan) cudaFreeHost(b->h_plan);
        if (b->h_results) cudaFreeHost(b->h_results);
        if (b->own_stream) cudaStreamDestroy(b->stream);
        delete b;
        return VEGAS_ECUDA;
    }
    memset(b->h_plan, 0, L.results - L.plan);
    batch_fill_args(b);
    const vegas_status st = batch_configure(b, 64);
    if (st != VEGAS_OK) {
        cudaFreeHost(b->h_plan);
        cudaFreeHost(b->h_results);
        if (b->own_stream) cudaStreamDestroy(b->stream);
        delete b;
        return st;
    }
    *out = b;
    return VEGAS_OK;
}

vegas_status vegas_batch_add(vegas_batch *b, const vegas_config *cfg, const vegas_integrand *itg,
                             int32_t *slot_out) {
    VEGAS_NVTX_RANGE();
    if (!b || !cfg || !itg || !slot_out) return VEGAS_EINVAL;
    const int d = cfg->n_dim, N = cfg->n_bins;
    if (d < 1 || d > VEGAS_MAX_DIM || N < 2 || N > VEGAS_MAX_BINS || cfg->n_events < 2 ||
        !(cfg->alpha >= 0.0) || !std::isfinite(cfg->alpha) || cfg->precision != b->precision)
        return VEGAS_EINVAL;
    if (itg->n_dim != d) return VEGAS_EINVAL;
    const int np = host_n_params(itg->family, d);
    if (np < 0 || itg->n_params != np || (np > 0 && !itg->params)) return VEGAS_EINVAL;
    if (itg->family == VEGAS_F_LO && d != 3) return VEGAS_EINVAL;
    if (itg->family == VEGAS_F_LO_PDF) return VEGAS_EINVAL;  // its density grid is per context
    FamilyConsts fc;
    double norm = 1.0, fmax = 1.0;
    if (!host_prepare_family(itg->family, d, itg->params, fc, norm, fmax)) return VEGAS_EINVAL;
    // the shared-memory working set must fit for the largest slot
    if (d * N > b->max_cells) {
        const size_t budget = b->smem_optin > 2048 ? b->smem_optin - 2048 : 0;
        if (batch_sample_smem(b->mode, 0, d * N) > budget) return VEGAS_EINVAL;
    }
    int s = -1;
    for (int k = 0; k < b->max_slots; ++k)
        if (!b->slots[k].used) {
            s = k;
            break;
        }
    if (s < 0) return VEGAS_EBUSY;
    const size_t need = slot_pool_bytes(d, N);
    size_t off = 0;
    if (!b->pool.alloc(need, &off)) return VEGAS_ENOMEM;
    vegas_status st = batch_sync(b);
    if (st != VEGAS_OK) {
        b->pool.release(off, need);
        return st;
    }
    if (d * N > b->max_cells || N > b->max_N) {
        if (d * N > b->max_cells) {
            st = batch_configure(b, d * N);
            if (st != VEGAS_OK) {
                b->pool.release(off, need);
                return st;
            }
        }
        b->max_N = std::max(b->max_N, N);
        batch_invalidate_graph(b);
    }
    char *base = b->ws + b->L.pool + off;
    const size_t cells = static_cast<size_t>(d) * N;
    SlotDev sd;
    memset(&sd, 0, sizeof(sd));
    sd.family = itg->family;
    sd.d = d;
    sd.N = N;
    sd.smooth = cfg->smooth;
    sd.n = cfg->n_events;
    sd.key0 = cfg->seed;
    sd.key1 = cfg->integral_id;
    const double scale = std::ldexp(1.0, -static_cast<int>(std::lround(std::log2(fmax))));
    const double Nd = static_cast<double>(N);
    double kappa = 1.0;
    host_fp32_consts(itg->family, d, fc, sd.fc32, kappa);
    sd.jinit64 = norm * scale * std::pow(Nd, d);
    sd.jinit32 = static_cast<float>(norm * scale * std::pow(Nd, d % 4) / kappa);
    sd.n4 = static_cast<float>(Nd * Nd * Nd * Nd);
    sd.alpha = cfg->alpha;
    sd.inv_scale = 1.0 / scale;
    sd.jmul = 1.0;
    sd.fc64 = fc;
    sd.edges = reinterpret_cast<double *>(base);
    sd.table = base + up(sizeof(double) * d * (N + 1));
    sd.acc = reinterpret_cast<double *>(static_cast<char *>(sd.table) + up(16 * cells));
    sd.last = reinterpret_cast<double *>(reinterpret_cast<char *>(sd.acc) + up(sizeof(double) * (2 + cells)));
    sd.center = reinterpret_cast<double *>(reinterpret_cast<char *>(sd.last) + up(sizeof(double) * (2 + cells)));
    std::vector<double> e(static_cast<size_t>(d) * (N + 1));
    for (int j = 0; j < d; ++j)
        for (int k = 0; k <= N; ++k) e[static_cast<size_t>(j) * (N + 1) + k] = static_cast<double>(k) / N;
    SlotDev *dsd = reinterpret_cast<SlotDev *>(b->ws + b->L.slots) + s;
    cudaError_t ce = cudaMemcpyAsync(dsd, &sd, sizeof(sd), cudaMemcpyHostToDevice, b->stream);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(sd.edges, e.data(), e.size() * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(sd.acc, 0, 2 * up(sizeof(double) * (2 + cells)), b->stream);
    if (ce == cudaSuccess) ce = launch_set_centers(sd.center, itg->family, d, fc, b->stream);
    if (ce == cudaSuccess) ce = launch_table_from_edges(sd.edges, sd.table, sd.center, b->mode, d, N, b->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(b->stream);  // host buffers go out of scope
    if (ce != cudaSuccess) {
        b->pool.release(off, need);
        snprintf(g_batch_error, sizeof(g_batch_error), "vegas_batch_add: %s", cudaGetErrorString(ce));
        return VEGAS_ECUDA;
    }
    SlotHost &h = b->slots[s];
    h.used = true;
    h.off = off;
    h.bytes = need;
    h.n = cfg->n_events;
    h.d = d;
    h.N = N;
    *slot_out = s;
    return VEGAS_OK;
}

vegas_status vegas_batch_remove(vegas_batch *b, int32_t slot) {
    VEGAS_NVTX_RANGE();
    if (!b || slot < 0 || slot >= b->max_slots || !b->slots[slot].used) return VEGAS_EINVAL;
    const vegas_status st = batch_sync(b);
    if (st != VEGAS_OK) return st;
    b->pool.release(b->slots[slot].off, b->slots[slot].bytes);
    b->slots[slot] = SlotHost();
    return VEGAS_OK;
}

vegas_status vegas_batch_step(vegas_batch *b) {
    VEGAS_NVTX_RANGE();
    if (!b) return VEGAS_EINVAL;
    vegas_status st = batch_sync(b);
    if (st != VEGAS_OK) return st;
    const int n = batch_build_plan(b);
    b->last_items = n;
    if (n == 0) return VEGAS_OK;
    if (!b->graph_ok || b->graph_cells != b->max_cells || b->graph_N != b->max_N ||
        b->graph_tile != b->tile_samples) {
        st = batch_capture(b);
        if (st != VEGAS_OK) return st;
    }
    VB_CK(cudaGraphLaunch(b->exec, b->stream));
    b->in_flight = true;
    return VEGAS_OK;
}

vegas_status vegas_batch_wait(vegas_batch *b, vegas_batch_result *out, int32_t cap, int32_t *count) {
    VEGAS_NVTX_RANGE();
    if (!b || !count || cap < 0 || (cap > 0 && !out)) return VEGAS_EINVAL;
    const vegas_status st = batch_sync(b);
    if (st != VEGAS_OK) return st;
    const int n = std::min(cap, b->last_items);
    for (int k = 0; k < n; ++k) {
        const BatchResult &r = b->h_results[k];
        out[k].slot = r.slot;
        out[k].t = r.t;
        out[k].it.I = r.it.I;
        out[k].it.sigma = r.it.sigma;
        out[k].it.n = r.it.n;
        out[k].it.n_nonfinite = r.it.n_nonfinite;
        out[k].comb.I = r.comb.I;
        out[k].comb.sigma = r.comb.sigma;
        out[k].comb.chi2_dof = r.comb.chi2_dof;
        out[k].comb.n_iter = r.comb.n_iter;
        out[k].comb.reserved = r.comb.status;
    }
    *count = n;
    return VEGAS_OK;
}

vegas_status vegas_batch_get_grid(vegas_batch *b, int32_t slot, double *edges_host) {
    if (!b || slot < 0 || slot >= b->max_slots || !b->slots[slot].used || !edges_host) return VEGAS_EINVAL;
    vegas_status st = batch_sync(b);
    if (st != VEGAS_OK) return st;
    SlotDev sd;
    const SlotDev *dsd = reinterpret_cast<const SlotDev *>(b->ws + b->L.slots) + slot;
    VB_CK(cudaMemcpyAsync(&sd, dsd, sizeof(sd), cudaMemcpyDeviceToHost, b->stream));
    VB_CK(cudaStreamSynchronize(b->stream));
    VB_CK(cudaMemcpyAsync(edges_host, sd.edges, sizeof(double) * sd.d * (sd.N + 1), cudaMemcpyDeviceToHost,
                          b->stream));
    VB_CK(cudaStreamSynchronize(b->stream));
    return VEGAS_OK;
}

vegas_status vegas_batch_set_events(vegas_batch *b, int32_t slot, int64_t n_events) {
    VEGAS_NVTX_RANGE();
    if (!b || slot < 0 || slot >= b->max_slots || !b->slots[slot].used || n_events < 2) return VEGAS_EINVAL;
    if (n_events == b->slots[slot].n) return VEGAS_OK;
    vegas_status st = batch_sync(b);
    if (st != VEGAS_OK) return st;
    SlotDev *dsd = reinterpret_cast<SlotDev *>(b->ws + b->L.slots) + slot;
    // the host value must outlive the asynchronous copy: keep it in the slot
    b->slots[slot].n = n_events;
    VB_CK(cudaMemcpyAsync(&dsd->n, &b->slots[slot].n, sizeof(long long), cudaMemcpyHostToDevice, b->stream));
    VB_CK(cudaStreamSynchronize(b->stream));
    return VEGAS_OK;
}

vegas_status vegas_batch_set_tile(vegas_batch *b, int32_t tile_samples) {
    if (!b || tile_samples < 512 || tile_samples > (1 << 26) || tile_samples % 512) return VEGAS_EINVAL;
    b->tile_samples = tile_samples;
    return VEGAS_OK;
}

vegas_status vegas_batch_autotune(vegas_batch *b, const int32_t *cand, int32_t n_cand, int32_t reps,
                                  float *ms_out, int32_t *best) {
    VEGAS_NVTX_RANGE();
    if (!b || !cand || n_cand < 1 || reps < 1 || !best) return VEGAS_EINVAL;
    vegas_status st = batch_sync(b);
    if (st != VEGAS_OK) return st;
    const int saved = b->tile_samples;
    cudaEvent_t e0, e1;
    VB_CK(cudaEventCreate(&e0));
    VB_CK(cudaEventCreate(&e1));
    float best_ms = 0.f;
    int best_tile = saved;
    const size_t plan_bytes = b->L.results - b->L.plan;
    for (int c = 0; c < n_cand; ++c) {
        if (cand[c] < 512 || cand[c] % 512) {
            if (ms_out) ms_out[c] = -1.f;
            continue;
        }
        b->tile_samples = cand[c];
        if (batch_build_plan(b) == 0) break;
        cudaError_t e = cudaMemcpyAsync(b->ws + b->L.plan, b->h_plan, plan_bytes, cudaMemcpyHostToDevice, b->stream);
        float total = 0.f;
        void *params[] = {&b->args};
        for (int r = 0; r < reps && e == cudaSuccess; ++r) {
            e = cudaEventRecord(e0, b->stream);
            if (e == cudaSuccess)
                e = cudaLaunchKernel(b->kfn, dim3(b->sample_blocks), dim3(b->threads), params, b->smem, b->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess)
                e = cudaLaunchKernel(reinterpret_cast<const void *>(&batch_reset_kernel), dim3(4 * b->sm_count),
                                     dim3(128), params, 0, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            total += ms;
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            b->tile_samples = saved;
            snprintf(g_batch_error, sizeof(g_batch_error), "autotune: %s", cudaGetErrorString(e));
            return VEGAS_ECUDA;
        }
        const float avg = total / reps;
        if (ms_out) ms_out[c] = avg;
        if (c == 0 || avg < best_ms) {
            best_ms = avg;
            best_tile = cand[c];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tile_samples = best_tile;
    *best = best_tile;
    return VEGAS_OK;
}

vegas_status vegas_batch_get_shape(vegas_batch *b, vegas_batch_shape *out) {
    if (!b || !out) return VEGAS_EINVAL;
    out->tile_samples = b->tile_samples;
    out->threads = b->threads;
    out->layout = b->layout;
    return VEGAS_OK;
}

vegas_status vegas_batch_set_shape(vegas_batch *b, const vegas_batch_shape *shape) {
    VEGAS_NVTX_RANGE();
    if (!b || !shape) return VEGAS_EINVAL;
    const vegas_batch_shape s = *shape;
    if (s.tile_samples < 512 || s.tile_samples > (1 << 26) || s.tile_samples % 512 || s.threads < 128 ||
        s.threads > kBatchThreads || s.threads % 32 || s.layout < -1 || s.layout > 2)
        return VEGAS_EINVAL;
    vegas_status st = batch_sync(b);
    if (st != VEGAS_OK) return st;
    const int keep_threads = b->threads, keep_req = b->layout_req;
    b->threads = s.threads;
    b->layout_req = s.layout;
    st = batch_configure(b, b->max_cells);
    if (st == VEGAS_OK && s.layout >= 0 && b->layout != s.layout) st = VEGAS_EINVAL;  // does not fit
    if (st != VEGAS_OK) {
        b->threads = keep_threads;
        b->layout_req = keep_req;
        batch_configure(b, b->max_cells);
        return st;
    }
    b->tile_samples = s.tile_samples;
    batch_invalidate_graph(b);
    return VEGAS_OK;
}

vegas_status vegas_batch_autotune_shapes(vegas_batch *b, const vegas_batch_shape *cand, int32_t n_cand, int32_t reps,
                                         float *ms_out, int32_t *best) {
    VEGAS_NVTX_RANGE();
    if (!b || !cand || n_cand < 1 || reps < 1 || !best) return VEGAS_EINVAL;
    vegas_batch_shape saved;
    vegas_batch_get_shape(b, &saved);
    saved.layout = b->layout_req;
    const size_t plan_bytes = b->L.results - b->L.plan;
    cudaEvent_t e0, e1;
    VB_CK(cudaEventCreate(&e0));
    VB_CK(cudaEventCreate(&e1));
    float best_ms = -1.f;
    int best_k = -1;
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < n_cand && e == cudaSuccess; ++c) {
        if (ms_out) ms_out[c] = -1.f;
        if (vegas_batch_set_shape(b, &cand[c]) != VEGAS_OK) continue;  // out of range or does not fit
        if (batch_build_plan(b) == 0) break;
        e = cudaMemcpyAsync(b->ws + b->L.plan, b->h_plan, plan_bytes, cudaMemcpyHostToDevice, b->stream);
        float total = 0.f;
        void *params[] = {&b->args};
        for (int r = 0; r < reps && e == cudaSuccess; ++r) {
            e = cudaEventRecord(e0, b->stream);
            if (e == cudaSuccess)
                e = cudaLaunchKernel(b->kfn, dim3(b->sample_blocks), dim3(b->threads), params, b->smem, b->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
            // the trial's sums are discarded
            if (e == cudaSuccess)
                e = cudaLaunchKernel(reinterpret_cast<const void *>(&batch_reset_kernel), dim3(4 * b->sm_count),
                                     dim3(128), params, 0, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            total += ms;
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) break;
        const float avg = total / reps;
        if (ms_out) ms_out[c] = avg;
        if (best_k < 0 || avg < best_ms) {
            best_ms = avg;
            best_k = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        vegas_batch_set_shape(b, &saved);
        snprintf(g_batch_error, sizeof(g_batch_error), "autotune: %s", cudaGetErrorString(e));
        return VEGAS_ECUDA;
    }
    if (best_k < 0) {
        vegas_batch_set_shape(b, &saved);
        return VEGAS_EINVAL;  // no candidate fits
    }
    *best = best_k;
    return vegas_batch_set_shape(b, &cand[best_k]);
}

vegas_status vegas_batch_info(vegas_batch *b, int32_t *n_active, size_t *pool_free, size_t *pool_largest,
                              int32_t *tile_samples) {
    if (!b) return VEGAS_EINVAL;
    int n = 0;
    for (auto &s : b->slots) n += s.used ? 1 : 0;
    if (n_active) *n_active = n;
    if (pool_free) *pool_free = b->pool.free_bytes();
    if (pool_largest) *pool_largest = b->pool.largest();
    if (tile_samples) *tile_samples = b->tile_samples;
    return VEGAS_OK;
}

void vegas_batch_destroy(vegas_batch *b) {
    if (!b) return;
    if (b->in_flight) cudaStreamSynchronize(b->stream);
    batch_invalidate_graph(b);
    if (b->h_plan) cudaFreeHost(b->h_plan);
    if (b->h_results) cudaFreeHost(b->h_results);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"
