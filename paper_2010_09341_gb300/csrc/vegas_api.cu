// vegas_api.cu -- the C ABI of include/vegas.h.
//
// Host code only: validation, workspace layout, per-integral constants and
// kernel launches.  Every arithmetic step of an iteration (sampling, sums,
// iteration result, combination, refinement) runs in the device kernels.
#include "../../include/vegas.h"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "vegas_kernels.cuh"
#include "vegas_nvtx.h"

using namespace vegas;

namespace {

thread_local char g_last_error[256] = "";

void set_error(const char *what, cudaError_t e) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, cudaGetErrorString(e));
}

#define VEGAS_CK(call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) {                         \
            set_error(#call, e_);                        \
            return VEGAS_ECUDA;                          \
        }                                                \
    } while (0)

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
    size_t edges, table, acc, last, nonfinite, hscale, jmul, iters, comb, cstate, q, center, total;
};

Layout layout_for(int d, int N) {
    Layout L;
    size_t off = 0;
    L.edges = off;
    off = align_up(off + sizeof(double) * d * (N + 1));
    L.table = off;
    off = align_up(off + 16 * static_cast<size_t>(d) * N);
    L.acc = off;
    off = align_up(off + sizeof(double) * (2 + static_cast<size_t>(d) * N));
    L.last = off;
    off = align_up(off + sizeof(double) * (2 + static_cast<size_t>(d) * N));
    L.nonfinite = off;
    off = align_up(off + sizeof(unsigned long long));
    L.hscale = off;
    off = align_up(off + sizeof(float));
    L.jmul = off;
    off = align_up(off + 2 * sizeof(double));  // double-buffered by record parity
    L.iters = off;
    off = align_up(off + sizeof(IterRec) * kIterRing);
    L.comb = off;
    off = align_up(off + sizeof(CombRec));
    L.cstate = off;
    off = align_up(off + sizeof(CombState));
    L.q = off;                                 // stratified: running and last sum of m2
    off = align_up(off + 2 * sizeof(double));
    L.center = off;                            // the table's d centres (table_center)
    off = align_up(off + sizeof(double) * d);
    L.total = off;
    return L;
}

int n_params_for(int family, int d) {
    switch (family) {
    case VEGAS_F_CONST: return 0;
    case VEGAS_F_SUM: return 0;
    case VEGAS_F_GAUSS_SYM: return 1;
    case VEGAS_F_GENZ_OSC: return 1 + d;
    case VEGAS_F_GENZ_GAUSS: return 2 * d;
    case VEGAS_F_GENZ_PROD: return 2 * d;
    case VEGAS_F_GENZ_CORNER: return d;
    case VEGAS_F_LO: return 7;
    case VEGAS_F_LO_PDF: return 7;
    default: return -1;
    }
}

int mode_of(int precision) {
    switch (precision) {
    case VEGAS_FP64: return ACC_F64;
    case VEGAS_FP32_ACC64: return ACC_F32_SUM64;
    case VEGAS_FP32_KAHAN: return ACC_F32_KAHAN;
    default: return -1;
    }
}


struct DeviceInfo {
    int sms = 0;
    size_t smem_optin = 0;
};

DeviceInfo device_info(cudaError_t *err) {
    int dev = 0;
    DeviceInfo di;
    *err = cudaGetDevice(&dev);
    if (*err != cudaSuccess) return di;
    *err = cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, dev);
    if (*err != cudaSuccess) return di;
    int v = 0;
    *err = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    di.smem_optin = static_cast<size_t>(v);
    return di;
}

// f's constant factors and the per-dimension constants of each family.
// Returns false if a parameter is out of its domain.
bool prepare_family(int family, int d, const double *p, FamilyConsts &fc, double &norm,
                    double &fmax) {
    memset(&fc, 0, sizeof(fc));
    const double log2e = 1.4426950408889634;
    norm = 1.0;
    fmax = 1.0;
    switch (family) {
    case VEGAS_F_CONST: break;
    case VEGAS_F_SUM: fmax = d; break;
    case VEGAS_F_GAUSS_SYM: {
        const double a = p[0];
        if (!(a > 0.0) || !std::isfinite(a)) return false;
        fc.s[0] = -log2e / (a * a);
        norm = std::pow(a * std::sqrt(M_PI), -static_cast<double>(d));
        fmax = norm;
        break;
    }
    case VEGAS_F_GENZ_OSC:
        fc.s[1] = 2.0 * M_PI * p[0];
        for (int j = 0; j < d; ++j) fc.p[j] = p[1 + j];
        break;
    case VEGAS_F_GENZ_GAUSS:
        fc.s[0] = -log2e;
        for (int j = 0; j < d; ++j) {
            fc.p[j] = p[j];
            fc.q[j] = p[d + j];
        }
        break;
    case VEGAS_F_GENZ_PROD:
        for (int j = 0; j < d; ++j) {
            if (!(p[j] != 0.0) || !std::isfinite(p[j])) return false;
            fc.p[j] = p[j];
            fc.q[j] = p[d + j];
            norm *= p[j] * p[j];
        }
        fmax = norm;
        break;
    case VEGAS_F_GENZ_CORNER:
        for (int j = 0; j < d; ++j) {
            if (!(p[j] >= 0.0)) return false;
            fc.p[j] = p[j];
        }
        fc.s[0] = -static_cast<double>(d + 1);
        break;
    case VEGAS_F_LO:
    case VEGAS_F_LO_PDF: {
        const double sqrtS = p[0], M = p[1], G = p[2], cut = p[3], mlo = p[4], mhi = p[5], nrm = p[6];
        if (!(sqrtS > 0 && M > 0 && G > 0 && cut > 0 && mlo >= 0 && mhi > mlo)) return false;
        fc.s[0] = sqrtS * sqrtS;
        fc.s[1] = M * M;
        fc.s[2] = M * M * G * G;
        fc.s[3] = cut;
        fc.s[4] = mlo * mlo;
        fc.s[5] = mhi * mhi;
        // LO: the parametric density's normalisation (35/32)^2 is a constant
        // factor; LO_PDF takes g from the grid (vegas_set_pdf_grid)
        const double gn = family == VEGAS_F_LO ? 35.0 / 32.0 : 1.0;
        norm = 2.0 * gn * gn * nrm;
        // size of f near the resonance: g(x)^2 ~ 1/sqrt(tau0), BW/shat ~ 1/(M^2 G)^2
        fmax = std::fabs(norm) * (sqrtS / M) / (M * M * M * M * G * G);
        break;
    }
    default: return false;
    }
    if (!std::isfinite(norm) || !(fmax > 0.0) || !std::isfinite(fmax)) return false;
    return true;
}

// The FP32 paths work in the coordinate X = 2^32 x (the sampling table holds
// (2^32 e, w); Prec<float>::coord in the kernels).  Their constants are the
// family's FP64 constants with that power of two folded in where the formula
// meets x (p_j / 2^32 beside x, q_j 2^32 subtracted from it, s0 / 2^64 for a
// product or square of two coordinates, log2 offsets + 32), rounded to FP32.
// kappa: the constant factor by which the FP32 kernel's value of the integrand
// differs from f (SUM adds X: 2^32; the LO toy's rsqrt(x1 x2) becomes
// rsqrt(X1 X2): 2^-32; the density-grid toy divides by x1 x2 as well: 2^-64);
// the FP32 initial weight is divided by it.  User integrands see x itself.
void fp32_consts(int family, int d, const FamilyConsts &fc, FamConsts<float> &out, double &kappa) {
    const double S = 4294967296.0, iS = 1.0 / S;
    FamilyConsts t = fc;
    kappa = 1.0;
    switch (family) {
    case VEGAS_F_SUM: kappa = S; break;
    case VEGAS_F_GAUSS_SYM: t.s[0] = fc.s[0] * iS * iS; break;
    case VEGAS_F_GENZ_OSC:
    case VEGAS_F_GENZ_CORNER:
        for (int j = 0; j < d; ++j) t.p[j] = fc.p[j] * iS;
        break;
    case VEGAS_F_GENZ_GAUSS:
    case VEGAS_F_GENZ_PROD:
        for (int j = 0; j < d; ++j) {
            t.p[j] = fc.p[j] * iS;
            t.q[j] = fc.q[j] * S;
        }
        break;
    case VEGAS_F_LO:
        t.s[0] = fc.s[0] * iS * iS;
        kappa = iS;
        break;
    case VEGAS_F_LO_PDF:
        t.s[0] = fc.s[0] * iS * iS;
        t.p[0] = fc.p[0] + 32.0;  // log2 X of the first knot
        kappa = iS * iS;
        break;
    default: break;  // CONST; USER (x unscaled in the kernel)
    }
    for (int k = 0; k < 32; ++k) {
        out.p[k] = static_cast<float>(t.p[k]);
        out.q[k] = static_cast<float>(t.q[k]);
    }
    for (int k = 0; k < 8; ++k) out.s[k] = static_cast<float>(t.s[k]);
}

}  // namespace

struct vegas_ctx {
    vegas_config cfg;
    int family;
    int mode;
    std::vector<double> params;
    cudaStream_t stream;
    char *ws;
    size_t ws_bytes;
    Layout L;
    double *edges;
    void *table;
    double *acc;
    double *last;
    unsigned long long *nonfinite;
    float *hscale;
    double *jmul;
    IterRec *iters;
    CombRec *comb;
    CombState *cstate;
    double *center;   // d sampling-table centres (table_center)
    int sms = 0;      // the device's SM count (launch sizing)
    int t;          // Philox iteration word of the next iteration
    int n_done;     // iterations recorded in iters[]
    FamilyConsts fc;
    double jinit;
    double scale;   // v is accumulated as v * scale (a power of two)
    double nblk4;
    const void *kfn;
    size_t smem;
    bool priv;          // lane-private shared-memory layout
    int threads;
    int max_blocks;
    bool profiling = false;
    double *q;          // stratified: sum of hypercube m2 (running, last)
    int strat_req = 0;  // requested 2^B hypercubes: 0 off, -1 automatic, else B
    const void *kfn_strat = nullptr;
    int max_blocks_strat = 0;
    JitKernels jit;     // user integrand's run-time compiled kernels (family VEGAS_F_USER)
    const double *pdf = nullptr;  // VEGAS_F_LO_PDF: the caller's density grid (device)
    int pdf_nx = 0, pdf_nq = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;  // event pool
    size_t ev_used = 0;

    ~vegas_ctx() {
        for (auto &p : ev) {
            cudaEventDestroy(p.first);
            cudaEventDestroy(p.second);
        }
    }
};

extern "C" {

const char *vegas_strerror(vegas_status st) {
    switch (st) {
    case VEGAS_OK: return "ok";
    case VEGAS_EINVAL: return "invalid argument";
    case VEGAS_ENOMEM: return "workspace too small";
    case VEGAS_ECUDA: return "CUDA error";
    case VEGAS_ETIMEOUT: return "device wait timed out";
    case VEGAS_EBUSY: return "no free slot";
    case VEGAS_ENONFINITE: return "every integrand value was non-finite";
    case VEGAS_EJIT: return "the user integrand could not be compiled";
    default: return "unknown status";
    }
}

const char *vegas_last_error_string(void) { return g_last_error; }

static bool config_ok(const vegas_config *c) {
    if (!c) return false;
    if (c->n_dim < 1 || c->n_dim > VEGAS_MAX_DIM) return false;
    if (c->n_bins < 2 || c->n_bins > VEGAS_MAX_BINS) return false;
    if (c->n_events < 2) return false;
    if (!(c->alpha >= 0.0) || !std::isfinite(c->alpha)) return false;
    if (mode_of(c->precision) < 0) return false;
    return true;
}

size_t vegas_workspace_bytes(const vegas_config *cfg) {
    if (!config_ok(cfg)) return 0;
    return layout_for(cfg->n_dim, cfg->n_bins).total;
}

// vegas_create and vegas_create_user: source == nullptr for a built-in family.
static vegas_status create_impl(const vegas_config *cfg, const vegas_integrand *itg, const char *source,
                                void *stream, void *dev_workspace, size_t ws_bytes, vegas_ctx **out) {
    if (!out) return VEGAS_EINVAL;
    *out = nullptr;
    if (!config_ok(cfg) || !itg) return VEGAS_EINVAL;
    const int d = cfg->n_dim, N = cfg->n_bins;
    if (itg->n_dim != d) return VEGAS_EINVAL;
    const bool user = source != nullptr;
    if (user != (itg->family == VEGAS_F_USER)) return VEGAS_EINVAL;
    const int np = user ? itg->n_params : n_params_for(itg->family, d);
    if (np < 0 || np > VEGAS_MAX_USER_PARAMS || itg->n_params != np || (np > 0 && !itg->params))
        return VEGAS_EINVAL;
    if ((itg->family == VEGAS_F_LO || itg->family == VEGAS_F_LO_PDF) && d != 3) return VEGAS_EINVAL;
    const Layout L = layout_for(d, N);
    if (!dev_workspace || (reinterpret_cast<uintptr_t>(dev_workspace) % kAlign) != 0)
        return VEGAS_EINVAL;
    if (ws_bytes < L.total) return VEGAS_ENOMEM;

    FamilyConsts fc;
    double norm = 1.0, fmax = 1.0;
    if (user) {
        // the parameters in order through p[], q[], s[] (one FP64 array of 72)
        memset(&fc, 0, sizeof(fc));
        double *flat = reinterpret_cast<double *>(&fc);
        for (int k = 0; k < np; ++k) {
            if (!std::isfinite(itg->params[k])) return VEGAS_EINVAL;
            flat[k] = itg->params[k];
        }
    } else if (!prepare_family(itg->family, d, itg->params, fc, norm, fmax)) {
        return VEGAS_EINVAL;
    }

    cudaError_t err;
    const DeviceInfo di = device_info(&err);
    if (err != cudaSuccess) {
        set_error("device query", err);
        return VEGAS_ECUDA;
    }
    const int mode = mode_of(cfg->precision);
    // 1 KB margin for the kernel's static shared memory (block reduction)
    const size_t budget = di.smem_optin > 1024 ? di.smem_optin - 1024 : 0;
    bool priv = sample_smem(mode, true, d, N) <= budget;
    size_t smem = sample_smem(mode, priv, d, N);
    if (smem > budget) return VEGAS_EINVAL;  // d N too large for shared memory
    JitKernels jit;
    if (user) {
        const int rc = jit_user_kernels(source, mode, d, priv, &jit, nullptr);
        if (rc != 0) {
            snprintf(g_last_error, sizeof(g_last_error), "vegas_create_user: %s",
                     rc == 1 ? "the run-time compiler could not be loaded"
                             : (rc == 2 ? "the source did not compile (vegas_jit_log)" : "loading the module failed"));
            return rc == 3 ? VEGAS_ECUDA : VEGAS_EJIT;
        }
    }
    const void *fn = user ? jit.sample : sample_kernel(mode, itg->family, d, priv);
    if (!fn) return VEGAS_EINVAL;
    // FP64: one histogram copy per lane (no compare-and-swap retries within a
    // warp) where the cells fit and a launch has enough samples per block for
    // the retries it saves to outweigh the flush's second set of copies
    // (measured at d = 4..12, N = 50: 4.6-6% faster at 1e7 samples, 4.5%
    // slower at 1e5; the two balance near 3e5).  Every launch flushes, so the
    // samples per launch count (events_limit splits an iteration).  Not for the
    // density-grid family, whose grid sits after the cells in the stratified
    // kernel's layout.
    constexpr long long kWideMinEvents = 1000000;
    const long long per_launch =
        cfg->events_limit > 0 ? std::min<long long>(cfg->events_limit, cfg->n_events) : cfg->n_events;
    if (!user && priv && mode == ACC_F64 && itg->family != VEGAS_F_LO_PDF && per_launch >= kWideMinEvents) {
        const void *fw = sample_kernel_wide(mode, itg->family, d);
        const size_t smem_w = sample_smem(mode, kLayoutWide, d, N);
        if (fw && smem_w <= budget) {
            fn = fw;
            smem = smem_w;
        }
    }
    VEGAS_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(smem)));
    const int threads = 512;
    int occ = 0;
    VEGAS_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem));
    if (occ < 1) return VEGAS_EINVAL;

    vegas_ctx *c = new vegas_ctx();
    c->cfg = *cfg;
    c->family = itg->family;
    c->jit = jit;
    c->mode = mode;
    c->params.assign(itg->params, itg->params + np);
    c->stream = static_cast<cudaStream_t>(stream);
    c->ws = static_cast<char *>(dev_workspace);
    c->ws_bytes = ws_bytes;
    c->L = L;
    c->edges = reinterpret_cast<double *>(c->ws + L.edges);
    c->table = c->ws + L.table;
    c->acc = reinterpret_cast<double *>(c->ws + L.acc);
    c->last = reinterpret_cast<double *>(c->ws + L.last);
    c->nonfinite = reinterpret_cast<unsigned long long *>(c->ws + L.nonfinite);
    c->hscale = reinterpret_cast<float *>(c->ws + L.hscale);
    c->jmul = reinterpret_cast<double *>(c->ws + L.jmul);
    c->iters = reinterpret_cast<IterRec *>(c->ws + L.iters);
    c->comb = reinterpret_cast<CombRec *>(c->ws + L.comb);
    c->cstate = reinterpret_cast<CombState *>(c->ws + L.cstate);
    c->q = reinterpret_cast<double *>(c->ws + L.q);
    c->center = reinterpret_cast<double *>(c->ws + L.center);
    c->t = 0;
    c->n_done = 0;
    c->fc = fc;
    // v is accumulated scaled by a power of two near 1/max f so that v^2 and
    // the histograms stay far from the FP32 range limits; the finalize kernel
    // divides it out exactly.
    c->scale = std::ldexp(1.0, -static_cast<int>(std::lround(std::log2(fmax))));
    const double Nd = static_cast<double>(N);
    if (mode == ACC_F64) {
        c->jinit = norm * c->scale * std::pow(Nd, d);
    } else {
        FamConsts<float> unused;
        double kappa = 1.0;
        fp32_consts(itg->family, d, fc, unused, kappa);
        c->jinit = norm * c->scale * std::pow(Nd, d % 4) / kappa;
    }
    c->nblk4 = Nd * Nd * Nd * Nd;
    c->kfn = fn;
    c->smem = smem;
    c->priv = priv;
    c->threads = threads;
    c->max_blocks = occ * di.sms;
    c->sms = di.sms;

    // uniform grid, zeroed accumulators
    std::vector<double> e(static_cast<size_t>(d) * (N + 1));
    for (int j = 0; j < d; ++j)
        for (int k = 0; k <= N; ++k) e[static_cast<size_t>(j) * (N + 1) + k] = static_cast<double>(k) / N;
    cudaError_t ce = cudaMemcpyAsync(c->edges, e.data(), e.size() * sizeof(double),
                                     cudaMemcpyHostToDevice, c->stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(c->acc, 0, (L.hscale + sizeof(float)) - L.acc, c->stream);
    static const double kOnes[2] = {1.0, 1.0};
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(c->jmul, kOnes, sizeof(kOnes), cudaMemcpyHostToDevice, c->stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(c->comb, 0, (L.cstate + sizeof(CombState)) - L.comb, c->stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(c->q, 0, 2 * sizeof(double), c->stream);
    if (ce == cudaSuccess) ce = launch_set_centers(c->center, itg->family, d, fc, c->stream);
    if (ce == cudaSuccess) ce = launch_table_from_edges(c->edges, c->table, c->center, mode, d, N, c->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
    if (ce != cudaSuccess) {
        set_error("vegas_create", ce);
        delete c;
        return VEGAS_ECUDA;
    }
    *out = c;
    return VEGAS_OK;
}

vegas_status vegas_create(const vegas_config *cfg, const vegas_integrand *itg, void *stream,
                          void *dev_workspace, size_t ws_bytes, vegas_ctx **out) {
    VEGAS_NVTX_RANGE();
    return create_impl(cfg, itg, nullptr, stream, dev_workspace, ws_bytes, out);
}

vegas_status vegas_create_user(const vegas_config *cfg, const char *source, const double *params,
                               int32_t n_params, void *stream, void *dev_workspace, size_t ws_bytes,
                               vegas_ctx **out) {
    VEGAS_NVTX_RANGE();
    if (!source || !cfg) return VEGAS_EINVAL;
    vegas_integrand itg;
    itg.family = VEGAS_F_USER;
    itg.n_dim = cfg->n_dim;
    itg.params = params;
    itg.n_params = n_params;
    return create_impl(cfg, &itg, source, stream, dev_workspace, ws_bytes, out);
}

const char *vegas_jit_log(void) { return jit_last_log(); }

// More blocks than fit the GPU at once run in waves: round their number up to
// whole waves (each block then takes fewer samples), so that the last wave
// does not leave most SMs idle.  Between one and two blocks per SM's worth, round
// up to a whole number of blocks per SM: otherwise some SMs run two blocks,
// sharing their pipes, while others run one, and the two-block SMs set the
// time (1e5 FP64 samples in 196 blocks: 44 SMs with two blocks).
static long long whole_waves(long long blocks, long long resident, long long sms) {
    if (resident <= 0) return blocks;
    if (blocks <= resident) {
        if (sms > 0 && blocks > sms) blocks = std::min(resident, (blocks + sms - 1) / sms * sms);
        return blocks;
    }
    return (blocks + resident - 1) / resident * resident;
}

// Stratification in effect for n samples: 2^B hypercubes of P samples, with
// B = the requested B (or, automatically, as many as leave P >= 2), never more
// than leave P >= 2, 16 halvings per dimension or 2^31 hypercubes.
struct Strata {
    int B = 0;
    long long H = 0, P = 0;   // P = 0: plain sampling
};

static Strata strata_for(int req, int d, long long n) {
    Strata st;
    if (req == 0 || n < 2) return st;
    int bmax = 0;
    while (bmax < 62 && (n >> (bmax + 1)) >= 2) ++bmax;   // largest B with n / 2^B >= 2
    int B = req < 0 ? bmax : std::min(req, bmax);
    B = std::min(B, std::min(16 * d, 31));
    st.B = B;
    st.H = 1LL << B;
    st.P = n / st.H;
    return st;
}

static void fill_strata(SampleArgs &a, const Strata &st, int d, double *q) {
    memset(&a.st, 0, sizeof(a.st));
    a.st.P = static_cast<uint32_t>(st.P);
    a.st.q = q;
    uint32_t off = 0;
    for (int j = 0; j < d; ++j) {
        const uint32_t b = static_cast<uint32_t>(st.B / d + (j < st.B % d ? 1 : 0));
        a.st.off[j] = off;
        a.st.bits[j] = b;
        off += b;
    }
}

static SampleArgs make_args(const vegas_ctx *c, long long s_begin, long long n, int t) {
    SampleArgs a{};
    a.table = c->table;
    a.center = c->center;
    a.acc = c->acc;
    a.n_nonfinite = c->nonfinite;
    a.s_begin = s_begin;
    a.n = n;
    a.d = c->cfg.n_dim;
    a.N = c->cfg.n_bins;
    a.key0 = c->cfg.seed;
    a.key1 = c->cfg.integral_id;
    a.iter = static_cast<uint32_t>(t);
    a.jinit = c->jinit;
    a.nblk4 = c->nblk4;
    a.jmul = c->jmul + (c->n_done & 1);
    a.hscale = c->hscale;
    a.fc64 = c->fc;
    double kappa;
    fp32_consts(c->family, c->cfg.n_dim, c->fc, a.fc32, kappa);
    memset(&a.st, 0, sizeof(a.st));
    a.pdf = c->pdf;
    a.pdf_nx = c->pdf_nx;
    a.pdf_nq = c->pdf_nq;
    return a;
}

// Hypercubes [h_begin, h_begin + count) of a stratified iteration.
static vegas_status launch_sampling_strat(vegas_ctx *c, const Strata &st, long long h_begin, long long count) {
    SampleArgs a = make_args(c, h_begin, count, c->t);
    fill_strata(a, st, c->cfg.n_dim, c->q);
    // whole hypercubes per thread, a few samples per thread at least
    const long long per_thread = std::max(1LL, (c->mode == ACC_F64 ? 1 : 4) / st.P);
    const long long want = (count + static_cast<long long>(c->threads) * per_thread - 1) /
                           (static_cast<long long>(c->threads) * per_thread);
    long long blocks = std::max(1LL, std::min<long long>(c->max_blocks_strat, want));
    if (c->mode != ACC_F64) {
        // fixed-point histogram cells: a bounded number of samples per block
        const long long cap = block_samples_max(c->mode, c->priv ? 1 : 0, c->cfg.n_bins) / st.P;
        blocks = std::max(blocks, (count + cap - 1) / cap);
    }
    blocks = whole_waves(blocks, c->max_blocks_strat, c->sms);
    void *params[] = {&a};
    VEGAS_CK(launch_programmatic(c->kfn_strat, dim3(static_cast<unsigned>(blocks)), dim3(c->threads), params,
                                 c->smem, c->stream));
    return VEGAS_OK;
}

static vegas_status launch_sampling(vegas_ctx *c, long long s_begin, long long n) {
    SampleArgs a = make_args(c, s_begin, n, c->t);
    // a few samples per thread at least (FP32 modes: 4; FP64: 1, a sample
    // costs tens of cycles of the narrow FP64 pipe, which every SM should
    // contribute); otherwise fill every SM
    const long long per_thread = c->mode == ACC_F64 ? 1 : 4;
    const long long want = (n + static_cast<long long>(c->threads) * per_thread - 1) /
                           (static_cast<long long>(c->threads) * per_thread);
    long long blocks = std::max(1LL, std::min<long long>(c->max_blocks, want));
    if (c->mode != ACC_F64) {
        // fixed-point histogram cells: a bounded number of samples per block
        const long long cap = block_samples_max(c->mode, c->priv ? 1 : 0, c->cfg.n_bins);
        blocks = std::max(blocks, (n + cap - 1) / cap);
    }
    blocks = whole_waves(blocks, c->max_blocks, c->sms);
    void *params[] = {&a};
    VEGAS_CK(launch_programmatic(c->kfn, dim3(static_cast<unsigned>(blocks)), dim3(c->threads), params,
                                 c->smem, c->stream));
    return VEGAS_OK;
}

// Sampling of samples [s_begin, s_begin + count) of the next iteration into
// the accumulators (split into launches of at most events_limit samples).
static vegas_status sample_samples(vegas_ctx *c, long long s_begin, long long count) {
    if (c->family == VEGAS_F_LO_PDF && !c->pdf) return VEGAS_EINVAL;  // vegas_set_pdf_grid first
    const long long lim = c->cfg.events_limit > 0 ? c->cfg.events_limit : count;
    std::pair<cudaEvent_t, cudaEvent_t> *pe = nullptr;
    if (c->profiling) {
        if (c->ev_used == c->ev.size()) {
            std::pair<cudaEvent_t, cudaEvent_t> p;
            VEGAS_CK(cudaEventCreate(&p.first));
            VEGAS_CK(cudaEventCreate(&p.second));
            c->ev.push_back(p);
        }
        pe = &c->ev[c->ev_used++];
        VEGAS_CK(cudaEventRecord(pe->first, c->stream));
    }
    const Strata sg = strata_for(c->strat_req, c->cfg.n_dim, c->cfg.n_events);
    if (sg.P > 0) {
        // whole hypercubes per launch (samples [s_begin, s_begin + count) are
        // the whole iteration here: stratified iterations are not sharded)
        const long long limh = std::max(1LL, lim / sg.P);
        for (long long h0 = 0; h0 < sg.H; h0 += limh) {
            const vegas_status st = launch_sampling_strat(c, sg, h0, std::min(limh, sg.H - h0));
            if (st != VEGAS_OK) return st;
        }
    } else {
        for (long long s0 = 0; s0 < count; s0 += lim) {
            const vegas_status st = launch_sampling(c, s_begin + s0, std::min(lim, count - s0));
            if (st != VEGAS_OK) return st;
        }
    }
    if (pe) VEGAS_CK(cudaEventRecord(pe->second, c->stream));
    return VEGAS_OK;
}

// Iteration result from the accumulators (n_events samples in all) and the
// step to the next iteration.
static FinalizeArgs finalize_args(vegas_ctx *c) {
    FinalizeArgs f;
    f.acc = c->acc;
    f.last = c->last;
    f.n_nonfinite = c->nonfinite;
    f.hscale = c->hscale;
    f.jmul2 = c->jmul;
    f.iters = c->iters;
    f.cs = c->cstate;
    f.comb = c->comb;
    f.rec = c->n_done;
    f.total = 2 + c->cfg.n_dim * c->cfg.n_bins;
    f.n = c->cfg.n_events;
    f.inv_scale0 = 1.0 / c->scale;
    f.jinit0 = c->jinit;
    const Strata sg = strata_for(c->strat_req, c->cfg.n_dim, c->cfg.n_events);
    f.strat_H = sg.H;
    f.strat_P = sg.P;
    f.q = c->q;
    if (sg.P > 0) f.n = sg.H * sg.P;
    return f;
}

// Advance the counters after a finalize; copy the record out if asked.
static vegas_status after_finalize(vegas_ctx *c, vegas_iter_result *out) {
    const int rec = c->n_done;
    c->n_done += 1;
    c->t += 1;
    if (!out) return VEGAS_OK;
    IterRec r;
    VEGAS_CK(cudaMemcpyAsync(&r, c->iters + rec % kIterRing, sizeof(r), cudaMemcpyDeviceToHost, c->stream));
    VEGAS_CK(cudaStreamSynchronize(c->stream));
    out->I = r.I;
    out->sigma = r.sigma;
    out->n = r.n;
    out->n_nonfinite = r.n_nonfinite;
    // no finite value: plain iterations count only finite samples in n,
    // stratified ones count every sample (a non-finite value as 0)
    const bool strat = strata_for(c->strat_req, c->cfg.n_dim, c->cfg.n_events).P > 0;
    const bool none = strat ? r.n_nonfinite >= r.n : r.n <= 0;
    return none ? VEGAS_ENONFINITE : VEGAS_OK;
}

// Iteration result from the accumulators (n_events samples in all) and the
// step to the next iteration.
static vegas_status finalize_iteration(vegas_ctx *c, vegas_iter_result *out) {
    VEGAS_CK(launch_finalize(finalize_args(c), c->stream));
    return after_finalize(c, out);
}

vegas_status vegas_iterate(vegas_ctx *c, vegas_iter_result *out) {
    VEGAS_NVTX_RANGE();
    if (!c) return VEGAS_EINVAL;
    const vegas_status st = sample_samples(c, 0, c->cfg.n_events);
    if (st != VEGAS_OK) return st;
    return finalize_iteration(c, out);
}

static RefineJob refine_job(vegas_ctx *c) {
    RefineJob r;
    r.f = finalize_args(c);
    r.edges = c->edges;
    r.table = c->table;
    r.center = c->center;
    r.mode = c->mode;
    r.d = c->cfg.n_dim;
    r.N = c->cfg.n_bins;
    r.smooth = c->cfg.smooth;
    r.alpha = c->cfg.alpha;
    return r;
}

vegas_status vegas_step(vegas_ctx *c, vegas_iter_result *out) {
    VEGAS_NVTX_RANGE();
    if (!c) return VEGAS_EINVAL;
    const vegas_status st = sample_samples(c, 0, c->cfg.n_events);
    if (st != VEGAS_OK) return st;
    const RefineJob r = refine_job(c);
    VEGAS_CK(launch_finalize_refine(&r, 1, c->stream));
    return after_finalize(c, out);
}

vegas_status vegas_step_many(vegas_ctx *const *ctxs, int32_t n) {
    VEGAS_NVTX_RANGE();
    if (!ctxs || n < 1 || n > VEGAS_MAX_STEP_MANY) return VEGAS_EINVAL;
    for (int k = 0; k < n; ++k) {
        if (!ctxs[k] || ctxs[k]->stream != ctxs[0]->stream) return VEGAS_EINVAL;
        for (int i = 0; i < k; ++i)
            if (ctxs[i] == ctxs[k]) return VEGAS_EINVAL;
        if (ctxs[k]->family == VEGAS_F_LO_PDF && !ctxs[k]->pdf) return VEGAS_EINVAL;
    }
    RefineJob jobs[VEGAS_MAX_STEP_MANY];
    for (int k = 0; k < n; ++k) {
        const vegas_status st = sample_samples(ctxs[k], 0, ctxs[k]->cfg.n_events);
        if (st != VEGAS_OK) return st;
        jobs[k] = refine_job(ctxs[k]);
    }
    VEGAS_CK(launch_finalize_refine(jobs, n, ctxs[0]->stream));
    for (int k = 0; k < n; ++k) after_finalize(ctxs[k], nullptr);
    return VEGAS_OK;
}

vegas_status vegas_sample_shard(vegas_ctx *c, int64_t s_begin, int64_t count) {
    VEGAS_NVTX_RANGE();
    if (!c || s_begin < 0 || count < 0 || s_begin + count > c->cfg.n_events) return VEGAS_EINVAL;
    if (c->strat_req != 0) return VEGAS_EINVAL;  // stratified iterations are not sharded
    if (count == 0) return VEGAS_OK;
    return sample_samples(c, s_begin, count);
}

vegas_status vegas_accumulators(vegas_ctx *c, double **dev_sums, int64_t *n_sums,
                                unsigned long long **dev_nonfinite) {
    if (!c) return VEGAS_EINVAL;
    if (dev_sums) *dev_sums = c->acc;
    if (n_sums) *n_sums = 2 + static_cast<int64_t>(c->cfg.n_dim) * c->cfg.n_bins;
    if (dev_nonfinite) *dev_nonfinite = c->nonfinite;
    return VEGAS_OK;
}

vegas_status vegas_finalize(vegas_ctx *c, vegas_iter_result *out) {
    VEGAS_NVTX_RANGE();
    if (!c) return VEGAS_EINVAL;
    return finalize_iteration(c, out);
}

vegas_status vegas_refine(vegas_ctx *c) {
    VEGAS_NVTX_RANGE();
    if (!c) return VEGAS_EINVAL;
    if (c->n_done == 0) return VEGAS_OK;  // nothing sampled yet: keep the grid
    VEGAS_CK(launch_refine(c->last, c->edges, c->table, c->center, c->mode, c->cfg.n_dim, c->cfg.n_bins,
                           c->cfg.alpha, c->cfg.smooth, c->stream));
    return VEGAS_OK;
}

vegas_status vegas_result(vegas_ctx *c, vegas_result_t *out) {
    VEGAS_NVTX_RANGE();
    if (!c || !out) return VEGAS_EINVAL;
    CombRec r;
    VEGAS_CK(cudaMemcpyAsync(&r, c->comb, sizeof(r), cudaMemcpyDeviceToHost, c->stream));
    VEGAS_CK(cudaStreamSynchronize(c->stream));
    out->I = r.I;
    out->sigma = r.sigma;
    out->chi2_dof = r.chi2_dof;
    out->n_iter = r.n_iter;
    out->reserved = 0;
    return VEGAS_OK;
}

// Copy count iteration records, starting at record index first, out of the ring.
static vegas_status read_records(vegas_ctx *c, int first, int count, IterRec *dst) {
    int done = 0;
    while (done < count) {
        const int pos = (first + done) % kIterRing;
        const int len = std::min(count - done, kIterRing - pos);
        VEGAS_CK(cudaMemcpyAsync(dst + done, c->iters + pos, sizeof(IterRec) * len, cudaMemcpyDeviceToHost,
                                 c->stream));
        done += len;
    }
    VEGAS_CK(cudaStreamSynchronize(c->stream));
    return VEGAS_OK;
}

vegas_status vegas_run(vegas_ctx *c, int32_t n_iter, vegas_iter_result *iters, vegas_result_t *out) {
    VEGAS_NVTX_RANGE();
    if (!c || n_iter < 1 || !out) return VEGAS_EINVAL;
    if (iters && n_iter > kIterRing) return VEGAS_EINVAL;
    const int first = c->n_done;
    for (int k = 0; k < n_iter; ++k) {
        const vegas_status st = k + 1 < n_iter ? vegas_step(c, nullptr) : vegas_iterate(c, nullptr);
        if (st != VEGAS_OK) return st;
    }
    if (iters) {
        std::vector<IterRec> rs(n_iter);
        const vegas_status st = read_records(c, first, n_iter, rs.data());
        if (st != VEGAS_OK) return st;
        for (int k = 0; k < n_iter; ++k) {
            iters[k].I = rs[k].I;
            iters[k].sigma = rs[k].sigma;
            iters[k].n = rs[k].n;
            iters[k].n_nonfinite = rs[k].n_nonfinite;
        }
    }
    return vegas_result(c, out);
}

vegas_status vegas_get_grid(vegas_ctx *c, double *edges_host) {
    VEGAS_NVTX_RANGE();
    if (!c || !edges_host) return VEGAS_EINVAL;
    const size_t bytes = sizeof(double) * c->cfg.n_dim * (c->cfg.n_bins + 1);
    VEGAS_CK(cudaMemcpyAsync(edges_host, c->edges, bytes, cudaMemcpyDeviceToHost, c->stream));
    VEGAS_CK(cudaStreamSynchronize(c->stream));
    return VEGAS_OK;
}

vegas_status vegas_set_grid(vegas_ctx *c, const double *e) {
    VEGAS_NVTX_RANGE();
    if (!c || !e) return VEGAS_EINVAL;
    const int d = c->cfg.n_dim, N = c->cfg.n_bins;
    for (int j = 0; j < d; ++j) {
        const double *row = e + static_cast<size_t>(j) * (N + 1);
        if (row[0] != 0.0 || row[N] != 1.0) return VEGAS_EINVAL;
        for (int k = 0; k < N; ++k)
            if (!(row[k + 1] >= row[k])) return VEGAS_EINVAL;
    }
    VEGAS_CK(cudaMemcpyAsync(c->edges, e, sizeof(double) * d * (N + 1), cudaMemcpyHostToDevice,
                             c->stream));
    VEGAS_CK(launch_table_from_edges(c->edges, c->table, c->center, c->mode, d, N, c->stream));
    VEGAS_CK(cudaStreamSynchronize(c->stream));
    return VEGAS_OK;
}

vegas_status vegas_get_sums(vegas_ctx *c, double *sums_host) {
    if (!c || !sums_host) return VEGAS_EINVAL;
    const size_t cnt = 2 + static_cast<size_t>(c->cfg.n_dim) * c->cfg.n_bins;
    VEGAS_CK(cudaMemcpyAsync(sums_host, c->last, cnt * sizeof(double), cudaMemcpyDeviceToHost,
                             c->stream));
    VEGAS_CK(cudaStreamSynchronize(c->stream));
    return VEGAS_OK;
}

vegas_status vegas_set_events(vegas_ctx *c, int64_t n_events) {
    if (!c || n_events < 2) return VEGAS_EINVAL;
    if (c->strat_req != 0 && c->mode != ACC_F64 &&
        strata_for(c->strat_req, c->cfg.n_dim, n_events).P >
            block_samples_max(c->mode, c->priv ? 1 : 0, c->cfg.n_bins))
        return VEGAS_EINVAL;
    c->cfg.n_events = n_events;
    return VEGAS_OK;
}

vegas_status vegas_get_iteration(vegas_ctx *c, int32_t *t) {
    if (!c || !t) return VEGAS_EINVAL;
    *t = c->t;
    return VEGAS_OK;
}

vegas_status vegas_set_iteration(vegas_ctx *c, int32_t t) {
    if (!c || t < 0) return VEGAS_EINVAL;
    c->t = t;
    return VEGAS_OK;
}

vegas_status vegas_trace(vegas_ctx *c, int32_t t, int64_t s_begin, int64_t count, int32_t *bins,
                         double *x, double *w) {
    VEGAS_NVTX_RANGE();
    if (!c || t < 0 || s_begin < 0 || count < 0) return VEGAS_EINVAL;
    if (c->family == VEGAS_F_LO_PDF && !c->pdf) return VEGAS_EINVAL;
    if (count == 0) return VEGAS_OK;
    SampleArgs a = make_args(c, s_begin, count, t);
    const Strata sg = strata_for(c->strat_req, c->cfg.n_dim, c->cfg.n_events);
    if (sg.P > 0) {
        if (s_begin + count > sg.H * sg.P) return VEGAS_EINVAL;
        fill_strata(a, sg, c->cfg.n_dim, nullptr);
    }
    if (c->family == VEGAS_F_USER)
        VEGAS_CK(launch_trace_fn(c->jit.trace, a, 1.0 / c->scale, bins, x, w, nullptr, c->stream));
    else
        VEGAS_CK(launch_trace(a, c->family, c->mode, 1.0 / c->scale, bins, x, w, c->stream));
    return VEGAS_OK;
}

vegas_status vegas_histogram(vegas_ctx *c, int32_t t, int32_t observable, int32_t nbins, double lo, double hi,
                             double *dev_out) {
    VEGAS_NVTX_RANGE();
    if (!c || t < 0 || nbins < 1 || nbins > 1024 || !(hi > lo) || !std::isfinite(lo) || !std::isfinite(hi) ||
        !dev_out || (reinterpret_cast<uintptr_t>(dev_out) % alignof(double)) != 0)
        return VEGAS_EINVAL;
    const bool lo_family = c->family == VEGAS_F_LO || c->family == VEGAS_F_LO_PDF;
    if (observable >= c->cfg.n_dim || observable < -2 || (observable < 0 && !lo_family)) return VEGAS_EINVAL;
    if (c->family == VEGAS_F_LO_PDF && !c->pdf) return VEGAS_EINVAL;
    const Strata sg = strata_for(c->strat_req, c->cfg.n_dim, c->cfg.n_events);
    const long long n = sg.P > 0 ? sg.H * sg.P : c->cfg.n_events;
    SampleArgs a = make_args(c, 0, n, t);
    if (sg.P > 0) fill_strata(a, sg, c->cfg.n_dim, nullptr);
    HistArgs h;
    h.out = dev_out;
    h.nb = nbins;
    h.obs = observable;
    h.lo = lo;
    h.hi = hi;
    h.w = (hi - lo) / static_cast<double>(nbins);
    h.sqrt_s = lo_family ? c->params[0] : 0.0;
    VEGAS_CK(cudaMemsetAsync(dev_out, 0, sizeof(double) * 2 * (nbins + 2), c->stream));
    const void *fn = c->family == VEGAS_F_USER ? c->jit.trace : trace_kernel_for(c->family, c->mode, c->cfg.n_dim);
    VEGAS_CK(launch_trace_fn(fn, a, 1.0 / c->scale, nullptr, nullptr, nullptr, &h, c->stream));
    return VEGAS_OK;
}

vegas_status vegas_set_strata(vegas_ctx *c, int32_t B) {
    VEGAS_NVTX_RANGE();
    if (!c || B < -1 || B > 31) return VEGAS_EINVAL;
    if (B != 0 && !c->kfn_strat) {
        const void *fn = c->family == VEGAS_F_USER ? c->jit.strat
                                                   : sample_strat_kernel(c->mode, c->family, c->cfg.n_dim, c->priv);
        if (!fn) return VEGAS_EINVAL;
        VEGAS_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(c->smem)));
        int occ = 0;
        VEGAS_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, c->threads, c->smem));
        if (occ < 1) return VEGAS_EINVAL;
        cudaError_t err;
        const DeviceInfo di = device_info(&err);
        if (err != cudaSuccess) {
            set_error("device query", err);
            return VEGAS_ECUDA;
        }
        c->kfn_strat = fn;
        c->max_blocks_strat = occ * di.sms;
    }
    if (B != 0) {
        // a hypercube must fit one block's fixed-point histogram capacity
        const Strata sg = strata_for(B, c->cfg.n_dim, c->cfg.n_events);
        if (c->mode != ACC_F64 && sg.P > block_samples_max(c->mode, c->priv ? 1 : 0, c->cfg.n_bins))
            return VEGAS_EINVAL;
    }
    c->strat_req = B;
    return VEGAS_OK;
}

vegas_status vegas_set_pdf_grid(vegas_ctx *c, const double *dev_xg, int32_t nx, int32_t nq, double u0,
                                double u1, double v0, double v1) {
    VEGAS_NVTX_RANGE();
    if (!c || c->family != VEGAS_F_LO_PDF || !dev_xg || nx < 2 || nq < 2 ||
        static_cast<long long>(nx + 2) * (nq + 2) > kMaxPdfValues || !(u1 > u0) || !(v1 > v0) || !std::isfinite(u0) ||
        !std::isfinite(u1) || !std::isfinite(v0) || !std::isfinite(v1) ||
        (reinterpret_cast<uintptr_t>(dev_xg) % alignof(double)) != 0)
        return VEGAS_EINVAL;
    // shared memory: the block's cells and the grid in the path's precision
    const size_t smem = pdf_grid_offset(sample_smem(c->mode, c->priv ? 1 : 0, c->cfg.n_dim, c->cfg.n_bins)) +
                        pdf_grid_bytes(c->mode, nx, nq);
    cudaError_t err;
    const DeviceInfo di = device_info(&err);
    if (err != cudaSuccess) {
        set_error("device query", err);
        return VEGAS_ECUDA;
    }
    if (smem + 1024 > di.smem_optin) return VEGAS_EINVAL;
    int occ = 0;
    VEGAS_CK(cudaFuncSetAttribute(c->kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    VEGAS_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, c->kfn, c->threads, smem));
    if (occ < 1) return VEGAS_EINVAL;
    c->max_blocks = occ * di.sms;
    if (c->kfn_strat) {
        int occ_s = 0;
        VEGAS_CK(cudaFuncSetAttribute(c->kfn_strat, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(smem)));
        VEGAS_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_s, c->kfn_strat, c->threads, smem));
        if (occ_s < 1) return VEGAS_EINVAL;
        c->max_blocks_strat = occ_s * di.sms;
    }
    c->smem = smem;
    // grid_xg works in log2 units: first knot and knots per unit of log2 x, log2 Q^2
    const double log2e = 1.4426950408889634;
    c->fc.p[0] = u0 * log2e;
    c->fc.p[1] = static_cast<double>(nx - 1) / ((u1 - u0) * log2e);
    c->fc.p[2] = v0 * log2e;
    c->fc.p[3] = static_cast<double>(nq - 1) / ((v1 - v0) * log2e);
    c->fc.p[4] = nx;
    c->fc.p[5] = nq;
    c->pdf = dev_xg;
    c->pdf_nx = nx;
    c->pdf_nq = nq;
    return VEGAS_OK;
}

vegas_status vegas_get_strata(vegas_ctx *c, int32_t *B, int64_t *P, int64_t *n_used) {
    if (!c) return VEGAS_EINVAL;
    const Strata sg = strata_for(c->strat_req, c->cfg.n_dim, c->cfg.n_events);
    if (B) *B = sg.P > 0 ? sg.B : 0;
    if (P) *P = sg.P;
    if (n_used) *n_used = sg.P > 0 ? sg.H * sg.P : c->cfg.n_events;
    return VEGAS_OK;
}

// ------------------------------------------------------------ checkpoint
namespace {
struct BlobHeader {
    uint32_t magic;
    uint32_t version;
    vegas_config cfg;
    int32_t family;
    int32_t n_params;
    int32_t t;
    int32_t n_done;
    float hscale;       // fixed-point histogram scale of the next iteration
    int32_t strat_req;  // vegas_set_strata's B (0: plain sampling)
    double jmul;        // rescale of v of the next iteration
};
constexpr uint32_t kMagic = 0x56454741u;  // "VEGA"
}  // namespace

vegas_status vegas_export_state(vegas_ctx *c, void *buf, size_t *size) {
    VEGAS_NVTX_RANGE();
    if (!c || !size) return VEGAS_EINVAL;
    const int d = c->cfg.n_dim, N = c->cfg.n_bins;
    const size_t ne = static_cast<size_t>(d) * (N + 1);
    const int nrec = std::min(c->n_done, kIterRing);
    const size_t need = sizeof(BlobHeader) + sizeof(double) * c->params.size() +
                        sizeof(double) * ne + sizeof(IterRec) * nrec + sizeof(CombRec) + sizeof(CombState);
    if (!buf) {
        *size = need;
        return VEGAS_OK;
    }
    if (*size < need) return VEGAS_ENOMEM;
    char *p = static_cast<char *>(buf);
    BlobHeader h;
    memset(&h, 0, sizeof(h));
    VEGAS_CK(cudaMemcpyAsync(&h.hscale, c->hscale, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    VEGAS_CK(cudaMemcpyAsync(&h.jmul, c->jmul + (c->n_done & 1), sizeof(double), cudaMemcpyDeviceToHost,
                             c->stream));
    VEGAS_CK(cudaStreamSynchronize(c->stream));
    h.magic = kMagic;
    h.version = 4;
    h.cfg = c->cfg;
    h.family = c->family;
    h.n_params = static_cast<int32_t>(c->params.size());
    h.t = c->t;
    h.n_done = c->n_done;
    h.strat_req = c->strat_req;
    memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    memcpy(p, c->params.data(), sizeof(double) * c->params.size());
    p += sizeof(double) * c->params.size();
    VEGAS_CK(cudaMemcpyAsync(p, c->edges, sizeof(double) * ne, cudaMemcpyDeviceToHost, c->stream));
    p += sizeof(double) * ne;
    if (nrec > 0) {
        const vegas_status st = read_records(c, c->n_done - nrec, nrec, reinterpret_cast<IterRec *>(p));
        if (st != VEGAS_OK) return st;
    }
    p += sizeof(IterRec) * nrec;
    VEGAS_CK(cudaMemcpyAsync(p, c->comb, sizeof(CombRec), cudaMemcpyDeviceToHost, c->stream));
    p += sizeof(CombRec);
    VEGAS_CK(cudaMemcpyAsync(p, c->cstate, sizeof(CombState), cudaMemcpyDeviceToHost, c->stream));
    VEGAS_CK(cudaStreamSynchronize(c->stream));
    *size = need;
    return VEGAS_OK;
}

vegas_status vegas_import_state(vegas_ctx *c, const void *buf, size_t size) {
    VEGAS_NVTX_RANGE();
    if (!c || !buf || size < sizeof(BlobHeader)) return VEGAS_EINVAL;
    const char *p = static_cast<const char *>(buf);
    BlobHeader h;
    memcpy(&h, p, sizeof(h));
    p += sizeof(h);
    if (h.magic != kMagic || h.version != 4) return VEGAS_EINVAL;
    const vegas_config &a = h.cfg, &b = c->cfg;
    if (a.n_dim != b.n_dim || a.n_bins != b.n_bins || a.n_events != b.n_events ||
        a.seed != b.seed || a.integral_id != b.integral_id || a.precision != b.precision ||
        a.alpha != b.alpha || a.smooth != b.smooth || h.family != c->family ||
        h.n_params != static_cast<int32_t>(c->params.size()))
        return VEGAS_EINVAL;
    if (h.n_done < 0 || h.t < 0) return VEGAS_EINVAL;
    const int nrec = std::min(h.n_done, kIterRing);
    const int d = b.n_dim, N = b.n_bins;
    const size_t ne = static_cast<size_t>(d) * (N + 1);
    const size_t need = sizeof(BlobHeader) + sizeof(double) * h.n_params + sizeof(double) * ne +
                        sizeof(IterRec) * nrec + sizeof(CombRec) + sizeof(CombState);
    if (size < need) return VEGAS_EINVAL;
    if (memcmp(p, c->params.data(), sizeof(double) * h.n_params) != 0) return VEGAS_EINVAL;
    p += sizeof(double) * h.n_params;
    VEGAS_CK(cudaMemcpyAsync(c->edges, p, sizeof(double) * ne, cudaMemcpyHostToDevice, c->stream));
    p += sizeof(double) * ne;
    for (int k = 0; k < nrec; ++k) {
        const int pos = (h.n_done - nrec + k) % kIterRing;
        VEGAS_CK(cudaMemcpyAsync(c->iters + pos, p + sizeof(IterRec) * k, sizeof(IterRec),
                                 cudaMemcpyHostToDevice, c->stream));
    }
    p += sizeof(IterRec) * nrec;
    VEGAS_CK(cudaMemcpyAsync(c->comb, p, sizeof(CombRec), cudaMemcpyHostToDevice, c->stream));
    p += sizeof(CombRec);
    VEGAS_CK(cudaMemcpyAsync(c->cstate, p, sizeof(CombState), cudaMemcpyHostToDevice, c->stream));
    VEGAS_CK(cudaMemcpyAsync(c->hscale, &h.hscale, sizeof(float), cudaMemcpyHostToDevice, c->stream));
    VEGAS_CK(cudaMemcpyAsync(c->jmul + (h.n_done & 1), &h.jmul, sizeof(double), cudaMemcpyHostToDevice,
                             c->stream));
    VEGAS_CK(launch_table_from_edges(c->edges, c->table, c->center, c->mode, d, N, c->stream));
    VEGAS_CK(cudaStreamSynchronize(c->stream));
    c->t = h.t;
    c->n_done = h.n_done;
    return vegas_set_strata(c, h.strat_req);
}

vegas_status vegas_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t n,
                          void *stream) {
    VEGAS_NVTX_RANGE();
    if (n < 0 || (n > 0 && (!ctr || !key || !out))) return VEGAS_EINVAL;
    VEGAS_CK(launch_philox(ctr, key, out, n, static_cast<cudaStream_t>(stream)));
    return VEGAS_OK;
}

vegas_status vegas_profile(vegas_ctx *c, int32_t enable) {
    if (!c) return VEGAS_EINVAL;
    c->profiling = enable != 0;
    return VEGAS_OK;
}

vegas_status vegas_profile_read(vegas_ctx *c, float *ms_out, int32_t cap, int32_t *count) {
    if (!c || !count || cap < 0 || (cap > 0 && !ms_out)) return VEGAS_EINVAL;
    VEGAS_CK(cudaStreamSynchronize(c->stream));
    int32_t k = 0;
    for (size_t i = 0; i < c->ev_used && k < cap; ++i) {
        float ms = 0.f;
        VEGAS_CK(cudaEventElapsedTime(&ms, c->ev[i].first, c->ev[i].second));
        ms_out[k++] = ms;
    }
    *count = k;
    c->ev_used = 0;
    return VEGAS_OK;
}

void vegas_destroy(vegas_ctx *c) { delete c; }

}  // extern "C"

// Family constants and parameter counts for the batched form (vegas_batch.cu).
namespace vegas {
bool host_prepare_family(int family, int d, const double *p, FamilyConsts &fc, double &norm, double &fmax) {
    return prepare_family(family, d, p, fc, norm, fmax);
}
void host_fp32_consts(int family, int d, const FamilyConsts &fc, FamConsts<float> &out, double &kappa) {
    fp32_consts(family, d, fc, out, kappa);
}
int host_n_params(int family, int d) { return n_params_for(family, d); }
}  // namespace vegas

// ------------------------------------------------------- no-allocation form
// One iteration's sums with every piece of scratch in a file-scope device
// array instead of a caller workspace.  For callers that cannot allocate
// device memory (see vegas_iterate_noalloc in vegas.h).
namespace {

constexpr int kNoallocMaxCells = 4096;  // d * N
constexpr size_t kNaAcc = 0;                                                    // 2 + cells doubles
constexpr size_t kNaNonfinite = (sizeof(double) * (2 + kNoallocMaxCells) + 255) / 256 * 256;
constexpr size_t kNaHscale = kNaNonfinite + kAlign;                             // float, kept 0
constexpr size_t kNaTable = kNaHscale + kAlign;                                 // cells x 16 bytes
constexpr size_t kNaCenter = kNaTable + 16 * static_cast<size_t>(kNoallocMaxCells);  // 32 doubles
constexpr size_t kNaBytes = kNaCenter + sizeof(double) * VEGAS_MAX_DIM;

// Shared by every call in the process, on every device that loads the library.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
char *g_noalloc_ptr[kMaxDevices] = {};

// out[0 .. total-1]: the sums unscaled; out[total]: the non-finite count.
__global__ void noalloc_unscale_kernel(const double *acc, const unsigned long long *nonfinite, double *out,
                                       int total, double inv1, double inv2) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < total) out[c] = acc[c] * (c == 0 ? inv1 : inv2);
    else if (c == total) out[c] = static_cast<double>(*nonfinite);
}

// Device address of the scratch array on the current device, looked up once
// per device (host code may not use the symbol itself as a pointer).
vegas_status noalloc_scratch(char **out) {
    int dev = 0;
    VEGAS_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return VEGAS_EINVAL;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        VEGAS_CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = static_cast<char *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return VEGAS_OK;
}

}  // namespace

extern "C" vegas_status vegas_iterate_noalloc(const vegas_config *cfg, const vegas_integrand *itg,
                                              int32_t t, const double *dev_edges, double *dev_sums,
                                              void *stream) {
    if (!config_ok(cfg) || !itg || t < 0 || !dev_edges || !dev_sums) return VEGAS_EINVAL;
    const int d = cfg->n_dim, N = cfg->n_bins;
    if (d * N > kNoallocMaxCells) {
        snprintf(g_last_error, sizeof(g_last_error),
                 "vegas_iterate_noalloc: n_dim * n_bins = %d exceeds the static scratch limit %d",
                 d * N, kNoallocMaxCells);
        return VEGAS_EINVAL;
    }
    if (itg->n_dim != d) return VEGAS_EINVAL;
    const int np = n_params_for(itg->family, d);
    if (np < 0 || itg->n_params != np || (np > 0 && !itg->params)) return VEGAS_EINVAL;
    if (itg->family == VEGAS_F_LO && d != 3) return VEGAS_EINVAL;
    if (itg->family == VEGAS_F_LO_PDF) return VEGAS_EINVAL;  // needs a context's density grid
    FamilyConsts fc;
    double norm = 1.0, fmax = 1.0;
    if (!prepare_family(itg->family, d, itg->params, fc, norm, fmax)) return VEGAS_EINVAL;

    char *scratch = nullptr;
    const vegas_status st = noalloc_scratch(&scratch);
    if (st != VEGAS_OK) return st;
    cudaError_t err;
    const DeviceInfo di = device_info(&err);
    if (err != cudaSuccess) {
        set_error("device query", err);
        return VEGAS_ECUDA;
    }
    const int mode = mode_of(cfg->precision);
    const size_t budget = di.smem_optin > 1024 ? di.smem_optin - 1024 : 0;
    const bool priv = sample_smem(mode, true, d, N) <= budget;
    const size_t smem = sample_smem(mode, priv, d, N);
    if (smem > budget) return VEGAS_EINVAL;
    const void *fn = sample_kernel(mode, itg->family, d, priv);
    if (!fn) return VEGAS_EINVAL;
    VEGAS_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(smem)));
    const int threads = 512;
    int occ = 0;
    VEGAS_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem));
    if (occ < 1) return VEGAS_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    double *acc = reinterpret_cast<double *>(scratch + kNaAcc);
    auto *nonfinite = reinterpret_cast<unsigned long long *>(scratch + kNaNonfinite);
    float *hscale = reinterpret_cast<float *>(scratch + kNaHscale);
    void *table = scratch + kNaTable;
    double *center = reinterpret_cast<double *>(scratch + kNaCenter);
    // the array keeps the previous call's contents: clear the accumulators,
    // the non-finite counter and the histogram scale (0: FP32 cells)
    VEGAS_CK(cudaMemsetAsync(scratch, 0, kNaTable, s));
    VEGAS_CK(launch_set_centers(center, itg->family, d, fc, s));
    VEGAS_CK(launch_table_from_edges(dev_edges, table, center, mode, d, N, s));

    const double scale = std::ldexp(1.0, -static_cast<int>(std::lround(std::log2(fmax))));
    const double Nd = static_cast<double>(N);
    SampleArgs a{};
    a.table = table;
    a.center = center;
    a.acc = acc;
    a.n_nonfinite = nonfinite;
    a.d = d;
    a.N = N;
    a.key0 = cfg->seed;
    a.key1 = cfg->integral_id;
    a.iter = static_cast<uint32_t>(t);
    double kappa = 1.0;
    fp32_consts(itg->family, d, fc, a.fc32, kappa);
    a.jinit = mode == ACC_F64 ? norm * scale * std::pow(Nd, d) : norm * scale * std::pow(Nd, d % 4) / kappa;
    a.nblk4 = Nd * Nd * Nd * Nd;
    a.jmul = nullptr;
    a.hscale = hscale;
    a.fc64 = fc;
    const long long n = cfg->n_events;
    const long long lim = cfg->events_limit > 0 ? cfg->events_limit : n;
    for (long long s0 = 0; s0 < n; s0 += lim) {
        a.s_begin = s0;
        a.n = std::min(lim, n - s0);
        // the grid of launch_sampling: 4 samples per thread at least in the
        // FP32 modes, 1 in FP64 (every SM's FP64 pipe should contribute), the
        // fixed-point cells' capacity, whole waves
        const long long per_thread = mode == ACC_F64 ? 1 : 4;
        const long long resident = static_cast<long long>(occ) * di.sms;
        const long long want = (a.n + threads * per_thread - 1) / (threads * per_thread);
        long long blocks = std::max(1LL, std::min<long long>(resident, want));
        if (mode != ACC_F64) {
            const long long cap = block_samples_max(mode, priv ? 1 : 0, N);
            blocks = std::max(blocks, (a.n + cap - 1) / cap);
        }
        blocks = whole_waves(blocks, resident, di.sms);
        void *params[] = {&a};
        VEGAS_CK(cudaLaunchKernel(fn, dim3(static_cast<unsigned>(blocks)), dim3(threads), params, smem, s));
    }
    const int total = 2 + d * N;
    noalloc_unscale_kernel<<<(total + 256) / 256, 256, 0, s>>>(acc, nonfinite, dev_sums, total, 1.0 / scale,
                                                               1.0 / (scale * scale));
    VEGAS_CK(cudaGetLastError());
    return VEGAS_OK;
}
