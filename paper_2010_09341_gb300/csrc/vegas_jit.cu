// vegas_jit.cu -- run-time compilation of user integrands.
//
// The paper's integrator takes the integrand as a function of the sample array
// (Sec. 3.1: compile(integrand)).  Here the user passes CUDA C++ source that
// defines, at global scope,
//     template <class T> __device__ T user_integrand(const T *x, int d, const T *p);
// and the library compiles it at run time (NVRTC, sm_103a) together with its
// own kernel headers (embedded in the library by the build), so the integrand
// is inlined into the same fused sampling kernel as the built-in families.
// Three kernels are compiled per (mode, d, layout): sampling, stratified
// sampling and the per-sample trace.  NVRTC is opened with dlopen on first
// use, so the library loads without it; the compiled modules are cached per
// (source, mode, d, layout) and stay loaded until the process exits.
#include <dlfcn.h>
#include <nvrtc.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "vegas_kernels.cuh"
#include "_jit_sources.h"

namespace vegas {
namespace {

// The NVRTC entry points used here, resolved from the shared library.
struct Nvrtc {
    bool ok = false;
    std::string why;
    nvrtcResult (*create)(nvrtcProgram *, const char *, const char *, int, const char *const *,
                          const char *const *) = nullptr;
    nvrtcResult (*destroy)(nvrtcProgram *) = nullptr;
    nvrtcResult (*add_name)(nvrtcProgram, const char *) = nullptr;
    nvrtcResult (*compile)(nvrtcProgram, int, const char *const *) = nullptr;
    nvrtcResult (*log_size)(nvrtcProgram, size_t *) = nullptr;
    nvrtcResult (*log)(nvrtcProgram, char *) = nullptr;
    nvrtcResult (*lowered)(nvrtcProgram, const char *, const char **) = nullptr;
    nvrtcResult (*cubin_size)(nvrtcProgram, size_t *) = nullptr;
    nvrtcResult (*cubin)(nvrtcProgram, char *) = nullptr;
};

template <class F> bool resolve(void *h, const char *name, F *fp) {
    *fp = reinterpret_cast<F>(dlsym(h, name));
    return *fp != nullptr;
}

Nvrtc load_nvrtc() {
    Nvrtc n;
    static const char *kNames[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                                   "/usr/local/cuda/lib64/libnvrtc.so"};
    void *h = nullptr;
    for (const char *nm : kNames)
        if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
    if (!h) {
        n.why = "the run-time compiler (libnvrtc) could not be loaded";
        return n;
    }
    n.ok = resolve(h, "nvrtcCreateProgram", &n.create) && resolve(h, "nvrtcDestroyProgram", &n.destroy) &&
           resolve(h, "nvrtcAddNameExpression", &n.add_name) && resolve(h, "nvrtcCompileProgram", &n.compile) &&
           resolve(h, "nvrtcGetProgramLogSize", &n.log_size) && resolve(h, "nvrtcGetProgramLog", &n.log) &&
           resolve(h, "nvrtcGetLoweredName", &n.lowered) && resolve(h, "nvrtcGetCUBINSize", &n.cubin_size) &&
           resolve(h, "nvrtcGetCUBIN", &n.cubin);
    if (!n.ok) n.why = "libnvrtc lacks an entry point this library needs";
    return n;
}

Nvrtc &nvrtc() {
    static Nvrtc n = load_nvrtc();
    return n;
}

std::mutex g_mu;
std::map<std::string, JitKernels> g_cache;
thread_local std::string g_log;

// Template arguments of the three kernels, chosen as for the built-in
// families: exact-dimension kernels for d <= 8 in the FP32 modes with the
// lane-private layout, tiers of 8, 16 and 32 dimensions otherwise.
std::string sample_args(int mode, int d, bool priv, bool *exact_out) {
    const bool exact = mode != ACC_F64 && priv && d <= 8;
    *exact_out = exact;
    const int maxd = exact ? d : (d <= 8 ? 8 : (d <= 16 ? 16 : 32));
    return std::to_string(F_USER) + ", " + std::to_string(mode) + ", " + std::to_string(maxd) + ", " +
           (exact ? "true" : "false") + ", " + ((exact || priv) ? "true" : "false");
}

std::string trace_args(int mode, int d) {
    const int tier = tier_of(d);
    const int maxd = tier == 0 ? 4 : (tier == 1 ? 8 : (tier == 2 ? 16 : 32));
    // FP32 modes share the trace's arithmetic (it keeps no sums)
    const int tmode = mode == ACC_F64 ? ACC_F64 : ACC_F32_KAHAN;
    return std::to_string(F_USER) + ", " + std::to_string(tmode) + ", " + std::to_string(maxd);
}

int compile_and_load(const std::string &source, int mode, int d, bool priv, JitKernels *out) {
    Nvrtc &nv = nvrtc();
    if (!nv.ok) {
        g_log = nv.why;
        return 1;
    }
    bool exact = false;
    const std::string sargs = sample_args(mode, d, priv, &exact);
    const std::string names[3] = {"vegas::vegas_sample_kernel<" + sargs + ">",
                                  "vegas::vegas_sample_strat_kernel<" + sargs + ">",
                                  "vegas::trace_kernel<" + trace_args(mode, d) + ">"};
    std::string prog_src = "#include \"vegas_sample.cuh\"\n#include \"vegas_strat.cuh\"\n"
                           "#include \"vegas_trace.cuh\"\n#line 1 \"user_source\"\n" +
                           source + "\n";
    const char *hdr_text[kJitHeaderCount];
    const char *hdr_name[kJitHeaderCount];
    for (int k = 0; k < kJitHeaderCount; ++k) {
        hdr_text[k] = kJitHeaders[k].text;
        hdr_name[k] = kJitHeaders[k].name;
    }
    nvrtcProgram prog = nullptr;
    if (nv.create(&prog, prog_src.c_str(), "vegas_user.cu", kJitHeaderCount, hdr_text, hdr_name) !=
        NVRTC_SUCCESS) {
        g_log = "nvrtcCreateProgram failed";
        return 2;
    }
    for (const std::string &nm : names) nv.add_name(prog, nm.c_str());
    const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo"};
    const nvrtcResult cr = nv.compile(prog, 3, opts);
    size_t lsz = 0;
    nv.log_size(prog, &lsz);
    std::string log(lsz, '\0');
    if (lsz) nv.log(prog, &log[0]);
    if (cr != NVRTC_SUCCESS) {
        g_log = log;
        nv.destroy(&prog);
        return 2;
    }
    std::string lowered[3];
    for (int k = 0; k < 3; ++k) {
        const char *ln = nullptr;
        if (nv.lowered(prog, names[k].c_str(), &ln) != NVRTC_SUCCESS || !ln) {
            g_log = "no lowered name for " + names[k];
            nv.destroy(&prog);
            return 2;
        }
        lowered[k] = ln;
    }
    size_t csz = 0;
    nv.cubin_size(prog, &csz);
    std::vector<char> cubin(csz);
    nv.cubin(prog, cubin.data());
    nv.destroy(&prog);

    cudaLibrary_t lib;
    cudaError_t ce = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (ce != cudaSuccess) {
        g_log = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(ce);
        return 3;
    }
    cudaKernel_t k[3];
    for (int i = 0; i < 3; ++i) {
        ce = cudaLibraryGetKernel(&k[i], lib, lowered[i].c_str());
        if (ce != cudaSuccess) {
            g_log = std::string("cudaLibraryGetKernel: ") + cudaGetErrorString(ce);
            return 3;
        }
    }
    out->sample = reinterpret_cast<const void *>(k[0]);
    out->strat = reinterpret_cast<const void *>(k[1]);
    out->trace = reinterpret_cast<const void *>(k[2]);
    g_log = log;
    return 0;
}

}  // namespace

int jit_user_kernels(const char *source, int mode, int d, bool priv, JitKernels *out, const char **log) {
    const std::string key = std::to_string(mode) + "/" + std::to_string(d) + "/" + (priv ? "1" : "0") + "/" +
                            source;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    int rc = 0;
    if (it != g_cache.end()) {
        *out = it->second;
        g_log.clear();
    } else {
        rc = compile_and_load(source, mode, d, priv, out);
        if (rc == 0) g_cache[key] = *out;
    }
    if (log) *log = g_log.c_str();
    return rc;
}

const char *jit_last_log() { return g_log.c_str(); }

}  // namespace vegas
