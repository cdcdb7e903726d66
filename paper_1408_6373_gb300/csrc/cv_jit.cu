// cv_jit.cu -- runtime specialisation of the FP32 sampling kernel.
//
// The generic sampling kernel reads each component's family and parameters
// from its launch parameters, so every point pays for a per-component
// family dispatch and for parameter loads.  For one integral run many times
// (a device-resident integral, a Vegas run of many iterations) the library
// can instead compile, at run time with NVRTC, the same kernel body with an
// integrand policy whose families and parameters are compile-time constants
// (hexadecimal float literals, so the values are bit-identical): the
// dispatch folds away and the parameters become instruction immediates.
// The kernel source is the library's own device header, embedded at build
// time.  NVRTC is loaded with dlopen; when it is missing or a compile
// fails, callers fall back to the generic kernel.  Compiled kernels are
// cached per device and source for the life of the process.
#include <dlfcn.h>
#include <nvrtc.h>

#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "cv_internal.cuh"
#include "cv_jit_sources.inc"  // generated: kJitHeaderNames[], kJitHeaderTexts[], kJitHeaderCount

namespace cv {

namespace {

struct Nvrtc {
    bool tried = false, ok = false;
    nvrtcResult (*create)(nvrtcProgram *, const char *, const char *, int, const char *const *,
                          const char *const *) = nullptr;
    nvrtcResult (*compile)(nvrtcProgram, int, const char *const *) = nullptr;
    nvrtcResult (*log_size)(nvrtcProgram, size_t *) = nullptr;
    nvrtcResult (*log)(nvrtcProgram, char *) = nullptr;
    nvrtcResult (*cubin_size)(nvrtcProgram, size_t *) = nullptr;
    nvrtcResult (*cubin)(nvrtcProgram, char *) = nullptr;
    nvrtcResult (*destroy)(nvrtcProgram *) = nullptr;
};

std::mutex g_mu;
Nvrtc g_nvrtc;
std::map<std::string, JitKernel> g_cache;  // key: device + source

bool load_nvrtc(std::string *err)
{
    if (g_nvrtc.tried) return g_nvrtc.ok;
    g_nvrtc.tried = true;
    const char *names[] = {"libnvrtc.so.13", "libnvrtc.so"};
    void *h = nullptr;
    for (const char *n : names)
        if ((h = dlopen(n, RTLD_NOW | RTLD_LOCAL))) break;
    if (!h) {
        *err = "libnvrtc not found";
        return false;
    }
#define CV_SYM(field, name)                                                          \
    g_nvrtc.field = reinterpret_cast<decltype(g_nvrtc.field)>(dlsym(h, name));        \
    if (!g_nvrtc.field) {                                                             \
        *err = "libnvrtc lacks " name;                                                \
        return false;                                                                 \
    }
    CV_SYM(create, "nvrtcCreateProgram")
    CV_SYM(compile, "nvrtcCompileProgram")
    CV_SYM(log_size, "nvrtcGetProgramLogSize")
    CV_SYM(log, "nvrtcGetProgramLog")
    CV_SYM(cubin_size, "nvrtcGetCUBINSize")
    CV_SYM(cubin, "nvrtcGetCUBIN")
    CV_SYM(destroy, "nvrtcDestroyProgram")
#undef CV_SYM
    g_nvrtc.ok = true;
    return true;
}

void hexf(std::string &s, float v)
{
    char buf[64];
    snprintf(buf, sizeof(buf), "%af", (double)v);
    s += buf;
}

// The integrand policy of the specialised kernels: families, parameters
// and (for the sampling kernel) map choices as compile-time constants.
std::string policy_source(const SampleArgs<float> &a, int ndim, bool pow2)
{
    const GenzParams<float> &g = a.g;
    std::string s = "#include \"cv_device.cuh\"\nnamespace cv {\nstruct JitIntegrand {\n";
    s += "  static constexpr int kMode = 0;\n";
    s += std::string("  static constexpr int kGen = ") + (a.gen == kGenPseudo ? "2" : "0") + ";\n";
    s += "  template <int C> __device__ __forceinline__ static constexpr int family(const GenzParams<float>&) { constexpr int f[4] = {";
    for (int c = 0; c < 4; ++c) s += std::to_string(c < g.ncomp ? g.family[c] : CV_CONST) + (c < 3 ? "," : "");
    s += "}; return f[C]; }\n";
    s += "  __device__ __forceinline__ static constexpr int ncomp(const GenzParams<float>&) { return " +
         std::to_string(g.ncomp) + "; }\n";
    const float(*tabs[2])[CV_MAX_DIM] = {g.p0, g.p1};
    const char *names[2] = {"p0", "p1"};
    for (int t = 0; t < 2; ++t) {
        s += "  template <int C> __device__ __forceinline__ static float ";
        s += names[t];
        s += "(const GenzParams<float>&, int d) { constexpr float v[4][" + std::to_string(ndim) + "] = {";
        for (int c = 0; c < 4; ++c) {
            s += "{";
            for (int d = 0; d < ndim; ++d) {
                hexf(s, c < g.ncomp ? tabs[t][c][d] : 0.0f);
                if (d + 1 < ndim) s += ",";
            }
            s += c < 3 ? "}," : "}";
        }
        s += "}; return v[C][d]; }\n";
    }
    const float *qs[2] = {g.q0, g.q1};
    const char *qnames[2] = {"q0", "q1"};
    for (int t = 0; t < 2; ++t) {
        s += "  template <int C> __device__ __forceinline__ static float ";
        s += qnames[t];
        s += "(const GenzParams<float>&) { constexpr float v[4] = {";
        for (int c = 0; c < 4; ++c) {
            hexf(s, c < g.ncomp ? qs[t][c] : 0.0f);
            if (c < 3) s += ",";
        }
        s += "}; return v[C]; }\n";
    }
    s += "  __device__ __forceinline__ static constexpr int delay(const GenzParams<float>&) { return " +
         std::to_string(g.delay) + "; }\n";
    s += "  __device__ __forceinline__ static constexpr int table(const MapParams&) { return " +
         std::to_string(pow2 ? a.map.li : 0) + "; }\n";
    s += "  __device__ __forceinline__ static constexpr bool priv(const MapParams&) { return " +
         std::string(pow2 && a.map.priv ? "true" : "false") + "; }\n";
    s += "  __device__ __forceinline__ static constexpr int nbins(int) { return " + std::to_string(a.nbins) +
         "; }\n";
    s += "};\n}\n";
    return s;
}

// Source of the specialised sampling kernel for these parameters.
std::string specialised_source(const SampleArgs<float> &a, int ndim, bool pow2, int min_blocks)
{
    std::string s = policy_source(a, ndim, pow2);
    s += "extern \"C\" __global__ void __launch_bounds__(" + std::to_string(kBlock) + ", " +
         std::to_string(min_blocks) + ") cv_jit_sample(const __grid_constant__ cv::SampleArgs<float> A)\n{\n";
    s += "    cv::sample_pass<" + std::to_string(ndim) + ", float, " + (pow2 ? "true" : "false") +
         ", cv::JitIntegrand>(A);\n}\n";
    return s;
}

// Source of the specialised built-in integrand on materialised points
// (dimension-major FP32): the policy's families and parameters only.
std::string points_source(const GenzParams<float> &g, int ndim)
{
    SampleArgs<float> a;
    memset(&a, 0, sizeof(a));
    a.g = g;
    std::string s = policy_source(a, ndim, false);
    s += "extern \"C\" __global__ void __launch_bounds__(" + std::to_string(kBlock) +
         ") cv_jit_points(const __grid_constant__ cv::GenzParams<float> g, const float *x, float *f, "
         "long long n, long long ld)\n{\n";
    s += "    cv::genz_points_f32<" + std::to_string(ndim) + ", cv::JitIntegrand>(g, x, f, n, ld);\n}\n";
    return s;
}


}  // namespace

// Compile a specialised source to a cubin (NVRTC; no device needed).
int compile_source(const std::string &src, std::vector<char> *cubin, std::string *err)
{
    if (!load_nvrtc(err)) return -1;
    nvrtcProgram prog;
    if (g_nvrtc.create(&prog, src.c_str(), "cv_jit_sample.cu", kJitHeaderCount, kJitHeaderTexts,
                       kJitHeaderNames) != NVRTC_SUCCESS) {
        *err = "nvrtcCreateProgram failed";
        return -1;
    }
    // (-default-device: the C ABI prototypes in the embedded header are then
    // unused device declarations instead of host functions NVRTC rejects)
    const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-default-device"};
    const nvrtcResult rc = g_nvrtc.compile(prog, 3, opts);
    if (rc != NVRTC_SUCCESS) {
        size_t n = 0;
        g_nvrtc.log_size(prog, &n);
        std::string log(n, '\0');
        if (n) g_nvrtc.log(prog, &log[0]);
        *err = "NVRTC compile failed: " + log.substr(0, 400);
        g_nvrtc.destroy(&prog);
        return -1;
    }
    size_t n = 0;
    g_nvrtc.cubin_size(prog, &n);
    cubin->resize(n);
    g_nvrtc.cubin(prog, cubin->data());
    g_nvrtc.destroy(&prog);
    return 0;
}

int jit_compile_check(const SampleArgs<float> &a, int ndim, bool pow2, int min_blocks, std::string *err)
{
    std::vector<char> cubin;
    std::lock_guard<std::mutex> lk(g_mu);
    if (compile_source(specialised_source(a, ndim, pow2, min_blocks), &cubin, err)) return -1;
    // (and the built-in integrand's kernel for the same problem)
    return compile_source(points_source(a.g, ndim), &cubin, err);
}

// Compile (once per device and source) and load a kernel named `name`.
static int jit_load(int device, const std::string &src, const char *name, size_t smem, JitKernel *out,
                    std::string *err);

namespace {
// Loaded kernels by the raw values their source is generated from, so that
// a launch finds its kernel without generating the source text again.
std::map<std::string, JitKernel> g_fast;

void key_add(std::string &k, const void *p, size_t n) { k.append(static_cast<const char *>(p), n); }
}  // namespace

int jit_sample_kernel(int device, const SampleArgs<float> &a, int ndim, bool pow2, int min_blocks,
                      JitKernel *out, std::string *err)
{
    std::string key("S");
    const int v[8] = {device, ndim, pow2 ? 1 : 0, min_blocks, a.nbins, a.gen == kGenPseudo ? 1 : 0,
                      pow2 ? a.map.li : 0, pow2 && a.map.priv ? 1 : 0};
    key_add(key, v, sizeof(v));
    key_add(key, &a.g, sizeof(a.g));  // (GenzParams is zeroed before it is filled)
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_fast.find(key);
        if (it != g_fast.end()) {
            *out = it->second;
            return 0;
        }
    }
    const int rc = jit_load(device, specialised_source(a, ndim, pow2, min_blocks), "cv_jit_sample",
                            sample_smem_bytes(ndim, a.nbins, false, pow2 && a.map.priv), out, err);
    if (rc == 0) {
        std::lock_guard<std::mutex> lk(g_mu);
        g_fast[key] = *out;
    }
    return rc;
}

int jit_points_kernel(int device, const GenzParams<float> &g, int ndim, JitKernel *out, std::string *err)
{
    std::string key("P");
    const int v[2] = {device, ndim};
    key_add(key, v, sizeof(v));
    key_add(key, &g, sizeof(g));
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_fast.find(key);
        if (it != g_fast.end()) {
            *out = it->second;
            return 0;
        }
    }
    const int rc = jit_load(device, points_source(g, ndim), "cv_jit_points", 0, out, err);
    if (rc == 0) {
        std::lock_guard<std::mutex> lk(g_mu);
        g_fast[key] = *out;
    }
    return rc;
}

static int jit_load(int device, const std::string &src, const char *name, size_t smem, JitKernel *out,
                    std::string *err)
{
    const std::string key = std::to_string(device) + "\n" + src;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
        *out = it->second;
        return 0;
    }
    std::vector<char> cubin;
    if (compile_source(src, &cubin, err)) return -1;
    JitKernel k;
    if (cudaLibraryLoadData(&k.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess ||
        cudaLibraryGetKernel(&k.kernel, k.lib, name) != cudaSuccess) {
        cudaGetLastError();
        *err = "loading the specialised kernel failed";
        return -1;
    }
    k.smem = smem;
    if (cudaFuncSetAttribute((const void *)k.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)k.smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k.occ, (const void *)k.kernel, kBlock, k.smem) !=
            cudaSuccess) {
        cudaGetLastError();
        *err = "configuring the specialised kernel failed";
        return -1;
    }
    if (k.occ < 1) k.occ = 1;
    g_cache[key] = k;
    *out = k;
    return 0;
}

int jit_info(int *compiled)
{
    std::lock_guard<std::mutex> lk(g_mu);
    std::string err;
    const bool ok = load_nvrtc(&err);
    *compiled = (int)g_cache.size();
    return ok ? 1 : 0;
}

cudaError_t launch_jit_points(const JitKernel &k, const GenzParams<float> &g, const float *x, float *f, long long n,
                              long long ld, int grid, cudaStream_t s)
{
    void *args[5] = {const_cast<GenzParams<float> *>(&g), &x, &f, &n, &ld};
    return cudaLaunchKernel((const void *)k.kernel, dim3(grid), dim3(kBlock), args, 0, s);
}

cudaError_t launch_jit_sample(const JitKernel &k, const SampleArgs<float> &a, int grid, cudaStream_t s)
{
    void *args[1] = {const_cast<SampleArgs<float> *>(&a)};
    return cudaLaunchKernel((const void *)k.kernel, dim3(grid), dim3(kBlock), args, k.smem, s);
}

}  // namespace cv
