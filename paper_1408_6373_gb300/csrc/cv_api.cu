// cv_api.cu -- the C ABI (include/cubagpu.h): contexts, argument checks,
// launch configuration, and the Vegas iteration driver.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <set>
#include <vector>

#include "cv_internal.cuh"

#define CV_FOR_EACH_NDIM(X)                                                                  \
    X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) \
    X(17) X(18) X(19) X(20) X(21) X(22) X(23) X(24) X(25) X(26) X(27) X(28) X(29) X(30)    \
    X(31) X(32)

namespace cv {
// explicit instantiations live in cv_sample_*.cu
#define CV_EXTERN(D)                                                                        \
    extern template cudaError_t launch_sample<D, float>(const SampleArgs<float> &, int,     \
                                                        cudaStream_t);                      \
    extern template cudaError_t launch_sample<D, double>(const SampleArgs<double> &, int,   \
                                                         cudaStream_t);                     \
    extern template cudaError_t sample_occupancy<D, float>(int, int *);                     \
    extern template cudaError_t sample_occupancy<D, double>(int, int *);                    \
    extern template cudaError_t launch_sobol<D, unsigned int>(                              \
        unsigned long long, long long, int, const PointArgs &, unsigned long long *, int,   \
        cudaStream_t);                                                                      \
    extern template cudaError_t launch_sobol<D, unsigned long long>(                        \
        unsigned long long, long long, int, const PointArgs &, unsigned long long *, int,   \
        cudaStream_t);
CV_FOR_EACH_NDIM(CV_EXTERN)
#undef CV_EXTERN

template <typename Real>
static cudaError_t dispatch_sample(int ndim, const SampleArgs<Real> &a, int grid, cudaStream_t s)
{
    switch (ndim) {
#define CV_CASE(D) case D: return launch_sample<D, Real>(a, grid, s);
        CV_FOR_EACH_NDIM(CV_CASE)
#undef CV_CASE
    }
    return cudaErrorInvalidValue;
}

template <typename Real>
static cudaError_t dispatch_occupancy(int ndim, int nbins, int *occ)
{
    switch (ndim) {
#define CV_CASE(D) case D: return sample_occupancy<D, Real>(nbins, occ);
        CV_FOR_EACH_NDIM(CV_CASE)
#undef CV_CASE
    }
    return cudaErrorInvalidValue;
}

template <typename W>
static cudaError_t dispatch_sobol(int ndim, unsigned long long start, long long n, int bits,
                                  const PointArgs &pa, unsigned long long *Y, int grid, cudaStream_t s)
{
    switch (ndim) {
#define CV_CASE(D) case D: return launch_sobol<D, W>(start, n, bits, pa, Y, grid, s);
        CV_FOR_EACH_NDIM(CV_CASE)
#undef CV_CASE
    }
    return cudaErrorInvalidValue;
}
}  // namespace cv

using namespace cv;

constexpr int kSideStreams = 8;  // concurrent per-class launches of a batched iteration

struct cv_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;  // graph capture happens here
    cudaStream_t side[kSideStreams] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kSideStreams] = {};
    bool own_stream = false;
    int sms = 0;
    char msg[512] = {0};
    // cached occupancy, [precision][ndim][nbins]; 0 = unknown
    std::vector<int> occ;
    // integrals created on this context (released by cv_destroy if the
    // caller has not destroyed them)
    std::set<struct cv_integral *> integrals;
    std::set<struct cv_batch *> batches;
    std::set<struct cv_server *> servers;
    // materialised-sample scratch (state, grid, histogram, x, f), grown on
    // demand and kept until cv_destroy; pinned words for the per-iteration
    // stop check of that mode
    void *mat_mem = nullptr;
    size_t mat_cap = 0;
    // the state of cv_vegas's one-shot integral, grown on demand and kept
    // (no allocation, and no free with its device synchronisation, per call)
    void *vegas_mem = nullptr;
    size_t vegas_cap = 0;
    // cv_vegas's integral of the last call, kept for a call with the same
    // problem (its iterations then replayed from a captured graph)
    struct cv_integral *vegas_last = nullptr;
    // per-block partials of standalone deterministic passes (cv_sample),
    // grown on demand: room for parts_G blocks of the largest problem
    void *parts_mem = nullptr;
    size_t parts_cap = 0;
    int parts_G = 0;
    int *pinned = nullptr;  // [0] = 1 (pass_active), [1] = stopped read back
    // cv_kernel_timer: event pairs around the sampling launches
    cudaEvent_t tev[2 * CV_TIMER_CAP] = {};
    int timer_on = 0, timer_n = 0;
};

static void integral_free(struct cv_integral *I);
static void batch_release(struct cv_batch *B);
static void server_release(struct cv_server *S);

static int fail_msg(cv_ctx *ctx, int code, const char *fmt, ...)
{
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->msg, sizeof(ctx->msg), fmt, ap);
        va_end(ap);
    }
    return code;
}

static int cuda_fail(cv_ctx *ctx, cudaError_t e, const char *where)
{
    return fail_msg(ctx, CV_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CV_CUDA(ctx, call)                                                  \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);          \
    } while (0)

extern "C" const char *cv_strerror(int code)
{
    switch (code) {
    case CV_OK: return "ok";
    case CV_EINVAL: return "invalid argument";
    case CV_ENOMEM: return "out of memory";
    case CV_ECUDA: return "CUDA error";
    case CV_EABORT: return "integrand aborted (-999)";
    case CV_ETIMEOUT: return "timed out";
    case CV_EADMIT: return "admission refused";
    case CV_EBUSY: return "busy";
    case CV_ENOTFOUND: return "not found";
    case CV_ESCRATCH: return "problem too large for the static scratch area";
    case CV_ENONFINITE: return "an iteration result was not finite";
    }
    return "unknown error";
}

extern "C" const char *cv_last_error(const cv_ctx *ctx) { return ctx ? ctx->msg : "no context"; }

extern "C" int cv_create(cv_ctx **out, int device, void *stream)
{
    if (!out) return CV_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return CV_ECUDA;
    cv_ctx *ctx = new cv_ctx();
    ctx->device = device;
    if (cudaSetDevice(device) != cudaSuccess) {
        delete ctx;
        return CV_ECUDA;
    }
    cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device);
    if (stream) {
        ctx->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return CV_ECUDA;
        }
        ctx->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        delete ctx;
        return CV_ECUDA;
    }
    ctx->occ.assign(2 * (CV_MAX_DIM + 1) * (CV_MAX_BINS + 1), 0);
    bool ok = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; k < kSideStreams && ok; ++k)
        ok = cudaStreamCreateWithFlags(&ctx->side[k], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&ctx->ev_join[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        cv_destroy(ctx);
        return CV_ECUDA;
    }
    *out = ctx;
    return CV_OK;
}

extern "C" void cv_destroy(cv_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (struct cv_integral *I : ctx->integrals) integral_free(I);
    ctx->integrals.clear();
    for (struct cv_batch *B : ctx->batches) batch_release(B);
    ctx->batches.clear();
    for (struct cv_server *S : ctx->servers) server_release(S);
    ctx->servers.clear();
    cudaStreamDestroy(ctx->cap_stream);
    for (int k = 0; k < kSideStreams; ++k) {
        if (ctx->side[k]) cudaStreamDestroy(ctx->side[k]);
        if (ctx->ev_join[k]) cudaEventDestroy(ctx->ev_join[k]);
    }
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    for (cudaEvent_t ev : ctx->tev)
        if (ev) cudaEventDestroy(ev);
    if (ctx->mat_mem) cudaFree(ctx->mat_mem);
    if (ctx->vegas_mem) cudaFree(ctx->vegas_mem);
    if (ctx->parts_mem) cudaFree(ctx->parts_mem);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

extern "C" int cv_kernel_timer(cv_ctx *ctx, int enable)
{
    if (!ctx) return CV_EINVAL;
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    if (enable && !ctx->tev[0]) {
        for (cudaEvent_t &ev : ctx->tev) CV_CUDA(ctx, cudaEventCreate(&ev));
    }
    ctx->timer_on = enable ? 1 : 0;
    if (enable) ctx->timer_n = 0;
    return CV_OK;
}

extern "C" int cv_kernel_times(cv_ctx *ctx, float *ms, int cap, int *count)
{
    if (!ctx || !count || cap < 0 || (cap > 0 && !ms)) return CV_EINVAL;
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    const int n = ctx->timer_n < cap ? ctx->timer_n : cap;
    for (int k = 0; k < n; ++k) {
        CV_CUDA(ctx, cudaEventSynchronize(ctx->tev[2 * k + 1]));
        CV_CUDA(ctx, cudaEventElapsedTime(&ms[k], ctx->tev[2 * k], ctx->tev[2 * k + 1]));
    }
    *count = ctx->timer_n;
    return CV_OK;
}

// The event pair for the next sampling launch on ctx->stream: -1 when the
// timer is off or full, or the stream is being captured into a graph.
static int timer_begin(cv_ctx *ctx)
{
    if (!ctx->timer_on || ctx->timer_n >= CV_TIMER_CAP) return -1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return -1;
    }
    if (cudaEventRecord(ctx->tev[2 * ctx->timer_n], ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return ctx->timer_n;
}

static void timer_end(cv_ctx *ctx, int k)
{
    if (k < 0) return;
    if (cudaEventRecord(ctx->tev[2 * k + 1], ctx->stream) == cudaSuccess) ctx->timer_n = k + 1;
    else cudaGetLastError();
}

extern "C" int cv_synchronize(cv_ctx *ctx)
{
    if (!ctx) return CV_EINVAL;
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    CV_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return CV_OK;
}

// ------------------------------------------------------------ helpers
static int check_genz(cv_ctx *ctx, const cv_genz *g)
{
    if (!g) return fail_msg(ctx, CV_EINVAL, "null integrand description");
    if (g->ndim < 1 || g->ndim > CV_MAX_DIM)
        return fail_msg(ctx, CV_EINVAL, "ndim %d outside 1..%d", g->ndim, CV_MAX_DIM);
    if (g->ncomp < 1 || g->ncomp > CV_MAX_COMP)
        return fail_msg(ctx, CV_EINVAL, "ncomp %d outside 1..%d", g->ncomp, CV_MAX_COMP);
    for (int c = 0; c < g->ncomp; ++c) {
        if (g->family[c] < 0 || g->family[c] >= CV_NUM_FAMILIES)
            return fail_msg(ctx, CV_EINVAL, "family %d of component %d unknown", g->family[c], c);
        for (int d = 0; d < g->ndim; ++d)
            if (!std::isfinite(g->a[c][d]) || !std::isfinite(g->u[c][d]))
                return fail_msg(ctx, CV_EINVAL, "non-finite parameter a/u[%d][%d]", c, d);
    }
    if (g->delay < 0 || g->delay > CV_MAX_DELAY)
        return fail_msg(ctx, CV_EINVAL, "delay %d outside 0..%d", g->delay, CV_MAX_DELAY);
    return CV_OK;
}

static const double kTwoPi = 6.283185307179586476925286766559;

namespace cv {
// The FP32 path's range precondition for a built-in integrand.  Its sums
// hold J f and (J f)^2 in binary32, whose normal range ends at 2^-126 and
// 2^128, so a component is accepted only when its largest value over the
// cube and its value at the centre (1/2, ..., 1/2) -- where a grid starts
// sampling, and a proxy for where its mass lies -- have squares within
// [2^-120, 2^120]: |f| within [2^-60, 2^60] there (log2 bounds from the
// closed formulas of each family).  The oscillatory family (|f| <= 1, zeros
// anywhere) and the constant pass; the discontinuous family's centre is
// checked only where it lies inside both cuts.  A component that fails
// needs CV_FP64.  Returns the first failing component (and a message), or -1.
int fp32_range_check(const cv_genz *g, char *msg, size_t len)
{
    const double log2e = 1.4426950408889634;
    for (int c = 0; c < g->ncomp; ++c) {
        const int D = g->ndim;
        const double *a = g->a[c], *u = g->u[c];
        double lmax = 0.0, lcen = 0.0;
        bool has_centre = true;
        switch (g->family[c]) {
        case CV_PRODUCT_PEAK:
            for (int d = 0; d < D; ++d) {
                lmax += 2.0 * std::log2(a[d]);
                lcen -= std::log2(1.0 / (a[d] * a[d]) + (0.5 - u[d]) * (0.5 - u[d]));
            }
            break;
        case CV_CORNER_PEAK: {
            double s = 0.0;
            for (int d = 0; d < D; ++d) s += a[d];
            lcen = -(D + 1) * std::log2(1.0 + 0.5 * s);
            break;
        }
        case CV_GAUSSIAN:
            for (int d = 0; d < D; ++d) lcen -= a[d] * a[d] * (0.5 - u[d]) * (0.5 - u[d]) * log2e;
            break;
        case CV_C0:
            for (int d = 0; d < D; ++d) lcen -= a[d] * std::fabs(0.5 - u[d]) * log2e;
            break;
        case CV_DISCONTINUOUS: {
            double smax = 0.0, scen = 0.0;
            for (int d = 0; d < D; ++d) {
                smax += a[d] * (d < 2 ? std::min(std::max(u[d], 0.0), 1.0) : 1.0);
                scen += 0.5 * a[d];
                if (d < 2 && u[d] < 0.5) has_centre = false;
            }
            lmax = smax * log2e;
            lcen = scen * log2e;
            break;
        }
        default:
            has_centre = false;
            break;
        }
        if (lmax > 60.0 || (has_centre && lcen < -60.0)) {
            if (msg)
                snprintf(msg, len, "component %d: values up to 2^%.0f, 2^%.0f at the centre: outside the "
                         "FP32 path's range (squares must stay in binary32); use CV_FP64", c, lmax, lcen);
            return c;
        }
    }
    return -1;
}
}  // namespace cv

static int check_fp32_range(cv_ctx *ctx, const cv_genz *g)
{
    char msg[256];
    if (fp32_range_check(g, msg, sizeof(msg)) >= 0) return fail_msg(ctx, CV_EINVAL, "%s", msg);
    return CV_OK;
}

namespace cv {
// The per-component parameters of GenzParams (their forms are listed with
// the struct): FP64 for x in [0, 1]; FP32 for the centred coordinate
// z = x - 1/2 with base-2 exponents, constants that the evaluation adds to
// a small sum split into a binary32 pair q0 + q1, rounded once each.
template <typename Real>
void fill_genz_params(const cv_genz *g, GenzParams<Real> *p)
{
    memset(p, 0, sizeof(*p));
    p->ndim = g->ndim;
    p->ncomp = g->ncomp;
    p->delay = g->delay;
    const bool f32 = sizeof(Real) == 4;
    const double l2e = 1.4426950408889634, sl2e = std::sqrt(1.4426950408889634);
    for (int c = 0; c < g->ncomp; ++c) {
        const int fam = g->family[c];
        const double *a = g->a[c], *u = g->u[c];
        p->family[c] = fam;
        double sa = 0.0;
        for (int d = 0; d < g->ndim; ++d) sa += a[d];
        for (int d = 0; d < g->ndim; ++d) {
            double p0 = 0.0, p1 = 0.0;
            switch (fam) {
            case CV_OSCILLATORY: p0 = f32 ? a[d] / kTwoPi : a[d]; break;
            case CV_PRODUCT_PEAK: p0 = 1.0 / (a[d] * a[d]); p1 = f32 ? 0.5 - u[d] : u[d]; break;
            case CV_CORNER_PEAK:
                p0 = a[d];
                if (f32) p1 = a[d] - (double)(float)a[d];  // the low half of a
                break;
            case CV_GAUSSIAN:
                if (f32) { p0 = a[d] * sl2e; p1 = a[d] * sl2e * (0.5 - u[d]); }
                else { p0 = a[d] * a[d]; p1 = u[d]; }
                break;
            case CV_C0:
                if (f32) { p0 = a[d] * l2e; p1 = 0.5 - u[d]; }
                else { p0 = a[d]; p1 = u[d]; }
                break;
            case CV_DISCONTINUOUS:
                if (f32) { p0 = a[d] * l2e; p1 = u[d] - 0.5; }
                else { p0 = a[d]; p1 = u[d]; }
                break;
            default: break;
            }
            p->p0[c][d] = (Real)p0;
            p->p1[c][d] = (Real)p1;
        }
        double q = 0.0;
        bool split = false;
        if (fam == CV_OSCILLATORY) {
            if (f32) {
                // phase in turns at z = 0, reduced to [-1/2, 1/2]
                q = u[0] + sa / (2.0 * kTwoPi);
                q -= std::nearbyint(q);
                split = true;
            } else {
                q = kTwoPi * u[0];
            }
        } else if (fam == CV_DISCONTINUOUS && f32) {
            q = std::exp(0.5 * sa);
        }
        p->q0[c] = (Real)q;
        if (split) p->q1[c] = (Real)(q - (double)p->q0[c]);
    }
}
template void fill_genz_params<float>(const cv_genz *, GenzParams<float> *);
template void fill_genz_params<double>(const cv_genz *, GenzParams<double> *);
}  // namespace cv

template <typename Real>
static void fill_params(const cv_genz *g, GenzParams<Real> *p)
{
    fill_genz_params<Real>(g, p);
}

static int occupancy(cv_ctx *ctx, int ndim, int nbins, bool fp64, int *occ)
{
    int &slot = ctx->occ[((fp64 ? 1 : 0) * (CV_MAX_DIM + 1) + ndim) * (CV_MAX_BINS + 1) + nbins];
    if (slot == 0) {
        int o = 0;
        cudaError_t e = fp64 ? dispatch_occupancy<double>(ndim, nbins, &o)
                             : dispatch_occupancy<float>(ndim, nbins, &o);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "occupancy query");
        slot = o > 0 ? o : 1;
    }
    *occ = slot;
    return CV_OK;
}

// Blocks for a pass over n points: about 16 32-point blocks per warp, at
// most one full wave of resident CTAs.  A pass too small to fill that wave
// spreads over more warps instead (down to 2 blocks each): its time is the
// dependent arithmetic of one warp's blocks (FP64 especially), not issue.
static int sample_grid(cv_ctx *ctx, int occ, long long n)
{
    const long long nblk = (n + 63) / 32;
    const long long cap = (long long)ctx->sms * occ;
    long long want = (nblk + (long long)kWarpsPerBlock * 16 - 1) / ((long long)kWarpsPerBlock * 16);
    if (want < cap) {
        want = (nblk + (long long)kWarpsPerBlock * 2 - 1) / ((long long)kWarpsPerBlock * 2);
        if (want > cap) want = cap;
    }
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    return (int)want;
}



// Per-block partials of a deterministic pass, in one device block laid out
// as [ticket (256 bytes)][S: G_cap x 2 CV_MAX_COMP doubles][H: G_cap x ndim
// x nbins values] (zeroed once; the ticket is reset by each launch's last
// block).
struct PassParts {
    void *mem = nullptr;
    int G_cap = 0;
    bool consumer_sums = false;  // the combination adds the sum partials (no ticket)
};

static void parts_args(const PassParts *pp, int grid, double **S, void **H, unsigned **ticket)
{
    char *base = static_cast<char *>(pp->mem);
    *ticket = reinterpret_cast<unsigned *>(base);
    *S = reinterpret_cast<double *>(base + 256);
    *H = base + 256 + (size_t)pp->G_cap * 2 * CV_MAX_COMP * sizeof(double);
    (void)grid;
}

// The grid of a sampling pass over n_grid points as launch_pass chooses it
// (the run-time specialised kernel's occupancy when CV_JIT compiles, else
// the generic kernel's).
template <typename Real>
static int pass_grid(cv_ctx *ctx, const cv_genz *g, int nbins, int flags, long long n_grid, int *grid)
{
    if constexpr (sizeof(Real) == 4) {
        if (flags & CV_JIT) {
            SampleArgs<float> a;
            memset(&a, 0, sizeof(a));
            fill_params<float>(g, &a.g);
            a.nbins = nbins;
            a.map = make_map(nbins, g->ndim, false);
            set_generator(&a, g->ndim, flags, 0);
            JitKernel k;
            std::string err;
            if (jit_sample_kernel(ctx->device, a, g->ndim, a.map.pow2 != 0, min_blocks_f32(g->ndim), &k, &err) == 0) {
                *grid = sample_grid(ctx, k.occ, n_grid);
                return CV_OK;
            }
        }
    }
    int occ = 0, rc = occupancy(ctx, g->ndim, nbins, sizeof(Real) == 8, &occ);
    if (rc) return rc;
    *grid = sample_grid(ctx, occ, n_grid);
    return CV_OK;
}

// One sampling pass.  pp: per-block partials for a deterministic reduction
// (else FP64 atomics); *grid_out receives the grid used.
template <typename Real>
static int launch_pass(cv_ctx *ctx, const cv_genz *g, int nbins, const double *edges,
                       unsigned long long start, long long n, long long n_grid,
                       double *S1, double *S2, double *H, DevState *st, int flags, uint64_t seed,
                       const float2 *ew32 = nullptr, const PassParts *pp = nullptr, int *grid_out = nullptr)
{
    SampleArgs<Real> a;
    memset(&a, 0, sizeof(a));
    fill_params<Real>(g, &a.g);
    a.nbins = nbins;
    a.chunk_min = 2;
    a.map = make_map(nbins, g->ndim, sizeof(Real) == 8);
    set_generator(&a, g->ndim, flags, seed);
    const bool jit = (flags & CV_JIT) != 0;
    a.edges = edges;
    if constexpr (sizeof(Real) == 4) a.ew32 = ew32;
    a.S1 = S1;
    a.S2 = S2;
    a.H = H;
    a.start = start;
    a.n = n;
    a.st = st;
    auto use_parts = [&](int grid) {
        if (grid_out) *grid_out = grid;
        if (pp && pp->mem && grid <= pp->G_cap) {
            parts_args(pp, grid, &a.part_S, &a.part_H, &a.part_ticket);
            if (pp->consumer_sums) a.part_ticket = nullptr;
            a.part_G = grid;
        }
    };
    if constexpr (sizeof(Real) == 4) {
        if (jit) {
            JitKernel k;
            std::string err;
            if (jit_sample_kernel(ctx->device, a, g->ndim, a.map.pow2 != 0, min_blocks_f32(g->ndim), &k, &err) == 0) {
                const int grid = sample_grid(ctx, k.occ, n_grid);
                use_parts(grid);
                const int tk = timer_begin(ctx);
                cudaError_t e = launch_jit_sample(k, a, grid, ctx->stream);
                if (e != cudaSuccess) return cuda_fail(ctx, e, "specialised sampling kernel launch");
                timer_end(ctx, tk);
                return CV_OK;
            }
            snprintf(ctx->msg, sizeof(ctx->msg), "run-time specialisation unavailable (%s); generic kernel used",
                     err.c_str());
        }
    }
    int occ = 0, rc = occupancy(ctx, g->ndim, nbins, sizeof(Real) == 8, &occ);
    if (rc) return rc;
    const int grid = sample_grid(ctx, occ, n_grid);
    use_parts(grid);
    const int tk = timer_begin(ctx);
    cudaError_t e = dispatch_sample<Real>(g->ndim, a, grid, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sampling kernel launch");
    timer_end(ctx, tk);
    return CV_OK;
}

// A standalone pass adds its histogram partials to H (its sums were added
// by its last block).
static int finish_parts(cv_ctx *ctx, const PassParts *pp, int grid, int nh, bool fp64, double *H)
{
    if (!pp || !pp->mem || grid > pp->G_cap) return CV_OK;
    double *S;
    void *Hp;
    unsigned *t;
    parts_args(pp, grid, &S, &Hp, &t);
    CV_CUDA(ctx, launch_add_parts(Hp, grid, fp64 ? 0 : 1, nh, H, ctx->stream));
    return CV_OK;
}

// The context's partial buffer for standalone passes: room for `grid`
// blocks of the largest problem (32 dimensions x 256 bins, FP64), grown
// when a pass needs more blocks.
static int ctx_parts(cv_ctx *ctx, int grid, PassParts *out)
{
    if (grid > ctx->parts_G) {
        if (ctx->parts_mem) cudaFree(ctx->parts_mem);
        ctx->parts_mem = nullptr;
        ctx->parts_cap = 0;
        ctx->parts_G = 0;
        const int G = grid;
        const size_t bytes = pass_parts_bytes(G, CV_MAX_DIM, CV_MAX_BINS, true) + 256;
        if (cudaMalloc(&ctx->parts_mem, bytes) != cudaSuccess) {
            cudaGetLastError();
            ctx->parts_mem = nullptr;
            return fail_msg(ctx, CV_ENOMEM, "device allocation of the pass partials failed");
        }
        CV_CUDA(ctx, cudaMemsetAsync(ctx->parts_mem, 0, bytes, ctx->stream));
        ctx->parts_cap = bytes;
        ctx->parts_G = G;
    }
    out->mem = ctx->parts_mem;
    out->G_cap = ctx->parts_G;
    return CV_OK;
}

extern "C" int cv_jit_check(const cv_genz *g, int nbins, int flags, char *log, int log_len)
{
    if (log && log_len > 0) log[0] = '\0';
    if (check_genz(nullptr, g) || nbins < CV_MIN_BINS || nbins > CV_MAX_BINS) return CV_EINVAL;
    SampleArgs<float> a;
    memset(&a, 0, sizeof(a));
    fill_params<float>(g, &a.g);
    a.nbins = nbins;
    a.map = make_map(nbins, g->ndim, false);
    set_generator(&a, g->ndim, flags, 1);
    std::string err;
    const int rc = jit_compile_check(a, g->ndim, a.map.pow2 != 0, min_blocks_f32(g->ndim), &err);
    if (rc && log && log_len > 0) snprintf(log, (size_t)log_len, "%s", err.c_str());
    return rc ? CV_ENOTFOUND : CV_OK;
}

extern "C" int cv_jit_info(int *available, int *compiled)
{
    int c = 0;
    const int a = jit_info(&c);
    if (available) *available = a;
    if (compiled) *compiled = c;
    return CV_OK;
}

// ------------------------------------------------------------ building blocks
extern "C" int cv_sobol(cv_ctx *ctx, int ndim, uint64_t start, int64_t n, int bits,
                        uint64_t *Y_dev)
{
    return cv_points(ctx, ndim, start, n, bits, 0, 0, Y_dev);
}

extern "C" int cv_points(cv_ctx *ctx, int ndim, uint64_t start, int64_t n, int bits, int flags,
                         uint64_t seed, uint64_t *Y_dev)
{
    if (!ctx) return CV_EINVAL;
    if ((flags & CV_SCRAMBLE) && (flags & CV_PSEUDO))
        return fail_msg(ctx, CV_EINVAL, "CV_SCRAMBLE and CV_PSEUDO exclude each other");
    if (ndim < 1 || ndim > CV_MAX_DIM) return fail_msg(ctx, CV_EINVAL, "ndim %d outside 1..%d", ndim, CV_MAX_DIM);
    if (bits != 23 && bits != 52) return fail_msg(ctx, CV_EINVAL, "bits must be 23 or 52");
    if (n < 0 || start > CV_INDEX_LIMIT || (uint64_t)n > CV_INDEX_LIMIT - start)
        return fail_msg(ctx, CV_EINVAL, "index range beyond 2^52");
    if (n == 0) return CV_OK;
    if (!Y_dev) return fail_msg(ctx, CV_EINVAL, "null output");
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    long long nblk = (n + 63) / 32;
    long long grid = (nblk + kWarpsPerBlock * 4 - 1) / (kWarpsPerBlock * 4);
    if (grid > (long long)ctx->sms * 8) grid = (long long)ctx->sms * 8;
    // the generator, with unpermuted shift words (the plain Sobol table)
    PointArgs pa;
    memset(&pa, 0, sizeof(pa));
    {
        SampleArgs<double> a;
        memset(&a, 0, sizeof(a));
        set_generator(&a, ndim, flags, seed);
        pa.gen = a.gen;
        pa.seed = a.seed;
        for (int d = 0; d < ndim; ++d) pa.shift[d] = bits == 23 ? (a.shift[d] >> 32) : a.shift[d];
    }
    cudaError_t e = bits == 23
        ? dispatch_sobol<unsigned int>(ndim, start, n, bits, pa, (unsigned long long *)Y_dev, (int)grid, ctx->stream)
        : dispatch_sobol<unsigned long long>(ndim, start, n, bits, pa, (unsigned long long *)Y_dev, (int)grid,
                                             ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sobol kernel launch");
    return CV_OK;
}

extern "C" int cv_sample(cv_ctx *ctx, const cv_genz *g, int nbins, const double *edges_dev,
                         uint64_t start, int64_t n, int flags, uint64_t seed, double *S1_dev,
                         double *S2_dev, double *hist_dev)
{
    if (!ctx) return CV_EINVAL;
    int rc = check_genz(ctx, g);
    if (rc) return rc;
    if (nbins < CV_MIN_BINS || nbins > CV_MAX_BINS)
        return fail_msg(ctx, CV_EINVAL, "nbins %d outside %d..%d", nbins, CV_MIN_BINS, CV_MAX_BINS);
    if (n < 0 || start > CV_INDEX_LIMIT || (uint64_t)n > CV_INDEX_LIMIT - start)
        return fail_msg(ctx, CV_EINVAL, "index range beyond 2^52");
    if (n == 0) return CV_OK;
    if (!edges_dev || !S1_dev || !S2_dev || !hist_dev) return fail_msg(ctx, CV_EINVAL, "null buffer");
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    if ((flags & CV_SCRAMBLE) && (flags & CV_PSEUDO))
        return fail_msg(ctx, CV_EINVAL, "CV_SCRAMBLE and CV_PSEUDO exclude each other");
    const bool fp64 = (flags & CV_FP64) != 0;
    if (!fp64 && (rc = check_fp32_range(ctx, g))) return rc;
    // (deterministic sums: per-block partials added in block order)
    int grid = 0;
    rc = fp64 ? pass_grid<double>(ctx, g, nbins, flags, n, &grid) : pass_grid<float>(ctx, g, nbins, flags, n, &grid);
    if (rc) return rc;
    PassParts pp;
    if ((rc = ctx_parts(ctx, grid, &pp))) return rc;
    int used = 0;
    rc = fp64 ? launch_pass<double>(ctx, g, nbins, edges_dev, start, n, n, S1_dev, S2_dev, hist_dev, nullptr,
                                    flags, seed, nullptr, &pp, &used)
              : launch_pass<float>(ctx, g, nbins, edges_dev, start, n, n, S1_dev, S2_dev, hist_dev, nullptr,
                                   flags, seed, nullptr, &pp, &used);
    if (rc) return rc;
    return finish_parts(ctx, &pp, used, g->ndim * nbins, fp64, hist_dev);
}

// The sampling map an FP32 pass takes for nbins bins and these flags (the
// pseudo-random generator takes the general map).
static MapParams sampling_map(int nbins, int ndim, int flags)
{
    SampleArgs<float> a;
    memset(&a, 0, sizeof(a));
    a.map = make_map(nbins, ndim, false);
    set_generator(&a, ndim, flags, 0);
    return a.map;
}

extern "C" int cv_stage_grid(cv_ctx *ctx, int ndim, int nbins, int flags, const double *edges_dev,
                             void *table_dev)
{
    if (!ctx) return CV_EINVAL;
    if (ndim < 1 || ndim > CV_MAX_DIM) return fail_msg(ctx, CV_EINVAL, "ndim %d outside 1..%d", ndim, CV_MAX_DIM);
    if (nbins < CV_MIN_BINS || nbins > CV_MAX_BINS) return fail_msg(ctx, CV_EINVAL, "nbins out of range");
    if (!edges_dev || !table_dev || ((uintptr_t)table_dev & 7u)) return fail_msg(ctx, CV_EINVAL, "null or unaligned buffer");
    if (flags & CV_FP64) return fail_msg(ctx, CV_EINVAL, "the staged grid is the FP32 path's");
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaError_t e = launch_stage_grid(ndim, nbins, edges_dev, static_cast<float2 *>(table_dev),
                                      sampling_map(nbins, ndim, flags), ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "grid staging kernel launch");
    return CV_OK;
}

extern "C" int cv_sample_staged(cv_ctx *ctx, const cv_genz *g, int nbins, const void *table_dev,
                                uint64_t start, int64_t n, int flags, uint64_t seed, double *S1_dev,
                                double *S2_dev, double *hist_dev)
{
    if (!ctx) return CV_EINVAL;
    int rc = check_genz(ctx, g);
    if (rc) return rc;
    if (nbins < CV_MIN_BINS || nbins > CV_MAX_BINS)
        return fail_msg(ctx, CV_EINVAL, "nbins %d outside %d..%d", nbins, CV_MIN_BINS, CV_MAX_BINS);
    if (n < 0 || start > CV_INDEX_LIMIT || (uint64_t)n > CV_INDEX_LIMIT - start)
        return fail_msg(ctx, CV_EINVAL, "index range beyond 2^52");
    if (flags & CV_FP64) return fail_msg(ctx, CV_EINVAL, "the staged grid is the FP32 path's");
    if ((flags & CV_SCRAMBLE) && (flags & CV_PSEUDO))
        return fail_msg(ctx, CV_EINVAL, "CV_SCRAMBLE and CV_PSEUDO exclude each other");
    if ((rc = check_fp32_range(ctx, g))) return rc;
    if (n == 0) return CV_OK;
    if (!table_dev || ((uintptr_t)table_dev & 7u) || !S1_dev || !S2_dev || !hist_dev)
        return fail_msg(ctx, CV_EINVAL, "null or unaligned buffer");
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    int grid = 0;
    if ((rc = pass_grid<float>(ctx, g, nbins, flags, n, &grid))) return rc;
    PassParts pp;
    if ((rc = ctx_parts(ctx, grid, &pp))) return rc;
    int used = 0;
    rc = launch_pass<float>(ctx, g, nbins, nullptr, start, n, n, S1_dev, S2_dev, hist_dev, nullptr, flags, seed,
                            static_cast<const float2 *>(table_dev), &pp, &used);
    if (rc) return rc;
    return finish_parts(ctx, &pp, used, g->ndim * nbins, false, hist_dev);
}

extern "C" int cv_refine(cv_ctx *ctx, int ndim, int nbins, const double *hist_dev, double *edges_dev)
{
    if (!ctx) return CV_EINVAL;
    if (ndim < 1 || ndim > CV_MAX_DIM) return fail_msg(ctx, CV_EINVAL, "ndim %d outside 1..%d", ndim, CV_MAX_DIM);
    if (nbins < CV_MIN_BINS || nbins > CV_MAX_BINS) return fail_msg(ctx, CV_EINVAL, "nbins out of range");
    if (!hist_dev || !edges_dev) return fail_msg(ctx, CV_EINVAL, "null buffer");
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaError_t e = launch_refine(ndim, nbins, const_cast<double *>(hist_dev), edges_dev, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "refine kernel launch");
    return CV_OK;
}

// ------------------------------------------------------------ Vegas driver

// One integral's device-resident run: parameters, state, grid, histogram
// and the captured iteration graph.
struct cv_integral {
    cv_ctx *ctx = nullptr;
    cv_spec spec;
    void *mem = nullptr;
    DevState *st = nullptr;
    double *edges = nullptr, *H = nullptr, *log_I = nullptr, *log_var = nullptr;
    float2 *ew32 = nullptr;    // FP32 runs: the grid staged for the sampling kernel
    MapParams map;             // its slot order
    int jmax = 0;              // iterations the sample budget allows
    long long nmax = 0;        // largest iteration
    int K = 0;                 // iterations per graph replay
    cudaGraphExec_t exec = nullptr;
    PassParts parts;           // per-block partials of the passes (deterministic sums)
    int launched_kernels = 0;  // kernels in one run (reset + iterations)
    bool oneshot = false;      // cv_vegas's: state in ctx->vegas_mem, kernels enqueued directly ...
    bool replay = false;       // ... unless the same problem came again: then a captured graph
};

static int check_spec(cv_ctx *ctx, const cv_spec *sp)
{
    if (!sp) return fail_msg(ctx, CV_EINVAL, "null spec");
    int rc = check_genz(ctx, &sp->g);
    if (rc) return rc;
    if (sp->nbins < CV_MIN_BINS || sp->nbins > CV_MAX_BINS)
        return fail_msg(ctx, CV_EINVAL, "nbins %d outside %d..%d", sp->nbins, CV_MIN_BINS, CV_MAX_BINS);
    if (sp->nstart < 2 || sp->nincrease < 0 || sp->maxeval < sp->nstart || sp->mineval < 0)
        return fail_msg(ctx, CV_EINVAL, "need 2 <= nstart <= maxeval, nincrease >= 0, mineval >= 0");
    if ((uint64_t)sp->maxeval >= CV_INDEX_LIMIT)
        return fail_msg(ctx, CV_EINVAL, "maxeval beyond the 2^52 Sobol index range");
    if (!(sp->epsrel >= 0) || !(sp->epsabs >= 0)) return fail_msg(ctx, CV_EINVAL, "negative tolerance");
    if ((sp->flags & CV_SCRAMBLE) && (sp->flags & CV_PSEUDO))
        return fail_msg(ctx, CV_EINVAL, "CV_SCRAMBLE and CV_PSEUDO exclude each other");
    if (!(sp->flags & CV_FP64)) return check_fp32_range(ctx, &sp->g);
    return CV_OK;
}

// Number of iterations the sample budget allows, and the largest one.
static void plan(long long nstart, long long nincrease, long long maxeval, int *jmax, long long *nmax)
{
    long long sum = 0, nj = nstart;
    int j = 0;
    while (j < (1 << 20) && nj <= maxeval - sum) {
        sum += nj;
        *nmax = nj;
        ++j;
        nj += nincrease;
    }
    *jmax = j;
}

// Enqueue one iteration (sample -> refine -> combine) on `s`.
static int enqueue_iteration(cv_integral *I, cudaStream_t s)
{
    cv_ctx *ctx = I->ctx;
    const cv_spec &sp = I->spec;
    cudaStream_t keep = ctx->stream;
    ctx->stream = s;
    int grid = 0;
    int rc = (sp.flags & CV_FP64)
        ? launch_pass<double>(ctx, &sp.g, sp.nbins, I->edges, 0, 0, I->nmax, I->st->S1, I->st->S2, I->H, I->st,
                              sp.flags, sp.seed, nullptr, &I->parts, &grid)
        : launch_pass<float>(ctx, &sp.g, sp.nbins, I->edges, 0, 0, I->nmax, I->st->S1, I->st->S2, I->H, I->st,
                             sp.flags, sp.seed, I->ew32, &I->parts, &grid);
    ctx->stream = keep;
    if (rc) return rc;
    CombineArgs ca = {};
    ca.st = I->st;
    ca.ncomp = sp.g.ncomp;
    ca.epsrel = sp.epsrel;
    ca.epsabs = sp.epsabs;
    ca.mineval = sp.mineval;
    ca.maxeval = sp.maxeval;
    ca.nstart = sp.nstart;
    ca.nincrease = sp.nincrease;
    ca.log_I = I->log_I;
    ca.log_var = I->log_var;
    ca.log_cap = kLogCap;
    if (grid <= I->parts.G_cap) {
        // the refinement sums the pass's histogram partials in block order
        double *S;
        void *Hp;
        unsigned *t;
        parts_args(&I->parts, grid, &S, &Hp, &t);
        ca.part_H = Hp;
        ca.part_S = S;
        ca.part_G = grid;
        ca.part_nh = sp.g.ndim * sp.nbins;
        ca.part_f32 = (sp.flags & CV_FP64) ? 0 : 1;
    }
    cudaError_t e = launch_refine_combine(sp.g.ndim, sp.nbins, I->H, I->edges, ca, I->ew32, I->map, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "refine/combine kernel launch");
    return CV_OK;
}

static int read_stopped(cv_integral *I, int *stopped)
{
    cv_ctx *ctx = I->ctx;
    CV_CUDA(ctx, cudaMemcpyAsync(stopped, &I->st->stopped, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CV_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return CV_OK;
}

static int capture_graph(cv_integral *I)
{
    cv_ctx *ctx = I->ctx;
    // the occupancy query sets kernel attributes, and a run-time
    // specialisation compiles and loads a module: both before capturing
    int occ = 0;
    int rc = occupancy(ctx, I->spec.g.ndim, I->spec.nbins, (I->spec.flags & CV_FP64) != 0, &occ);
    if (rc) return rc;
    if ((I->spec.flags & CV_JIT) && !(I->spec.flags & CV_FP64)) {
        SampleArgs<float> a;
        memset(&a, 0, sizeof(a));
        fill_params<float>(&I->spec.g, &a.g);
        a.nbins = I->spec.nbins;
        a.map = make_map(I->spec.nbins, I->spec.g.ndim, false);
        set_generator(&a, I->spec.g.ndim, I->spec.flags, I->spec.seed);
        JitKernel k;
        std::string err;
        jit_sample_kernel(ctx->device, a, I->spec.g.ndim, a.map.pow2 != 0, min_blocks_f32(I->spec.g.ndim), &k, &err);
    }
    I->K = I->jmax < 32 ? I->jmax : 32;
    cudaGraph_t graph = nullptr;
    CV_CUDA(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    for (int j = 0; j < I->K && rc == CV_OK; ++j) rc = enqueue_iteration(I, ctx->cap_stream);
    cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "graph capture");
    e = cudaGraphInstantiate(&I->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "graph instantiate");
    return CV_OK;
}

static int integral_create(cv_ctx *ctx, const cv_spec *spec, cv_integral **out, bool oneshot)
{
    if (!ctx || !out) return CV_EINVAL;
    *out = nullptr;
    int rc = check_spec(ctx, spec);
    if (rc) return rc;
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    cv_integral *I = new cv_integral();
    I->ctx = ctx;
    I->spec = *spec;
    I->oneshot = oneshot;
    plan(spec->nstart, spec->nincrease, spec->maxeval, &I->jmax, &I->nmax);
    const int ndim = spec->g.ndim, N = spec->nbins;
    const size_t sz_state = (sizeof(DevState) + 255) & ~(size_t)255;
    const size_t sz_edges = (((size_t)ndim * (N + 1) * sizeof(double)) + 255) & ~(size_t)255;
    const size_t sz_H = (((size_t)ndim * N * sizeof(double)) + 255) & ~(size_t)255;
    const size_t sz_log = (size_t)kLogCap * CV_MAX_COMP * sizeof(double);
    const bool fp32 = !(spec->flags & CV_FP64);
    const size_t sz_ew = fp32 ? (size_t)ndim * N * sizeof(float2) : 0;
    // the passes' per-block partials, for the grid every pass of this run uses
    int G = 0;
    rc = fp32 ? pass_grid<float>(ctx, &spec->g, N, spec->flags, I->nmax, &G)
              : pass_grid<double>(ctx, &spec->g, N, spec->flags, I->nmax, &G);
    if (rc) {
        delete I;
        return rc;
    }
    const size_t sz_parts = ((pass_parts_bytes(G, ndim, N, !fp32) + 256) + 255) & ~(size_t)255;
    const size_t bytes = sz_state + sz_edges + sz_H + 2 * sz_log + ((sz_ew + 255) & ~(size_t)255) + sz_parts;
    char *p = nullptr;
    if (oneshot) {
        if (bytes > ctx->vegas_cap) {
            if (ctx->vegas_mem) cudaFree(ctx->vegas_mem);
            ctx->vegas_mem = nullptr;
            ctx->vegas_cap = 0;
            if (cudaMalloc(&ctx->vegas_mem, bytes) != cudaSuccess) {
                cudaGetLastError();
                ctx->vegas_mem = nullptr;
                delete I;
                return fail_msg(ctx, CV_ENOMEM, "device allocation of the Vegas state failed");
            }
            ctx->vegas_cap = bytes;
        }
        p = (char *)ctx->vegas_mem;
    } else {
        if (cudaMalloc(&I->mem, bytes) != cudaSuccess) {
            cudaGetLastError();
            delete I;
            return fail_msg(ctx, CV_ENOMEM, "device allocation of the Vegas state failed");
        }
        p = (char *)I->mem;
    }
    I->st = (DevState *)p;
    I->edges = (double *)(p + sz_state);
    I->H = (double *)(p + sz_state + sz_edges);
    I->log_I = (double *)(p + sz_state + sz_edges + sz_H);
    I->log_var = (double *)(p + sz_state + sz_edges + sz_H + sz_log);
    if (fp32) I->ew32 = (float2 *)(p + sz_state + sz_edges + sz_H + 2 * sz_log);
    I->parts.mem = p + sz_state + sz_edges + sz_H + 2 * sz_log + ((sz_ew + 255) & ~(size_t)255);
    I->parts.G_cap = G;
    I->parts.consumer_sums = true;  // (the iteration's combination adds the sums)
    // (the ticket starts at zero; every pass's last block leaves it so)
    CV_CUDA(ctx, cudaMemsetAsync(I->parts.mem, 0, 256, ctx->stream));
    {
        // the map the sampling kernel takes (the point generator can change it)
        I->map = sampling_map(N, ndim, spec->flags);
    }
    I->launched_kernels = 1 + 2 * I->jmax;
    ctx->integrals.insert(I);
    *out = I;
    return CV_OK;
}

extern "C" int cv_integral_create(cv_ctx *ctx, const cv_spec *spec, cv_integral **out)
{
    return integral_create(ctx, spec, out, false);
}

static void integral_free(cv_integral *I)
{
    if (I->exec) cudaGraphExecDestroy(I->exec);
    if (I->mem) cudaFree(I->mem);  // (a one-shot integral's state is the context's)
    delete I;
}

extern "C" void cv_integral_destroy(cv_integral *I)
{
    if (!I) return;
    cv_ctx *ctx = I->ctx;
    if (!ctx->integrals.erase(I)) return;  // not (or no longer) a live handle
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    integral_free(I);
}

extern "C" int cv_integral_reset(cv_integral *I)
{
    if (!I) return CV_EINVAL;
    cv_ctx *ctx = I->ctx;
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaError_t e = launch_reset(I->st, I->edges, I->H, I->spec.g.ndim, I->spec.nbins,
                                 I->spec.nstart, I->ew32, I->map, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reset kernel launch");
    return CV_OK;
}

extern "C" int cv_integral_run(cv_integral *I)
{
    if (!I) return CV_EINVAL;
    cv_ctx *ctx = I->ctx;
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    int stopped = 0, rc = CV_OK;
    if (I->spec.flags & CV_PLAIN) {
        for (int j = 0; j < I->jmax && !stopped; ++j) {
            rc = enqueue_iteration(I, ctx->stream);
            if (rc) return rc;
            rc = read_stopped(I, &stopped);
            if (rc) return rc;
        }
        return CV_OK;
    }
    const bool fixed = I->spec.epsrel == 0.0 && I->spec.epsabs == 0.0;
    if (I->oneshot && !I->replay) {
        // a single run: capturing and instantiating a graph would cost more
        // than the launches it saves, so the iterations are enqueued directly
        // (32 at a time, the device's stop decision read in between unless
        // the iteration count is fixed)
        for (int done = 0; done < I->jmax && !stopped;) {
            const int K = I->jmax - done < 32 ? I->jmax - done : 32;
            for (int j = 0; j < K; ++j) {
                rc = enqueue_iteration(I, ctx->stream);
                if (rc) return rc;
            }
            done += K;
            if (!fixed && done < I->jmax) {
                rc = read_stopped(I, &stopped);
                if (rc) return rc;
            }
        }
        return CV_OK;
    }
    if (!I->exec) {
        rc = capture_graph(I);
        if (rc) return rc;
    }
    // Without an accuracy goal the iteration count is fixed and every replay
    // is enqueued at once; otherwise poll the device between replays.
    for (int done = 0; done < I->jmax && !stopped; done += I->K) {
        cudaError_t e = cudaGraphLaunch(I->exec, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "graph launch");
        if (!fixed && done + I->K < I->jmax) {
            rc = read_stopped(I, &stopped);
            if (rc) return rc;
        }
    }
    return CV_OK;
}

extern "C" int cv_integral_result(cv_integral *I, cv_result *out)
{
    if (!I || !out) return CV_EINVAL;
    cv_ctx *ctx = I->ctx;
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    DevState h;
    CV_CUDA(ctx, cudaMemcpyAsync(&h, I->st, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    CV_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    memset(out, 0, sizeof(*out));
    out->neval = h.neval;
    out->fail = h.stopped ? h.fail : 1;  // iteration cap reached without a decision
    out->iterations = h.iter;
    out->status = h.status;
    for (int c = 0; c < I->spec.g.ncomp; ++c) {
        out->integral[c] = h.integral[c];
        out->error[c] = h.error[c];
        out->prob[c] = h.prob[c];
        out->chi2[c] = h.chi2[c];
    }
    return CV_OK;
}

extern "C" int cv_integral_grid(cv_integral *I, double *edges)
{
    if (!I || !edges) return CV_EINVAL;
    cv_ctx *ctx = I->ctx;
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    const size_t bytes = (size_t)I->spec.g.ndim * (I->spec.nbins + 1) * sizeof(double);
    CV_CUDA(ctx, cudaMemcpyAsync(edges, I->edges, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CV_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return CV_OK;
}

extern "C" int cv_integral_log(cv_integral *I, int max_iter, double *iter_I, double *iter_var)
{
    if (!I || max_iter < 0 || (max_iter > 0 && (!iter_I || !iter_var))) return CV_EINVAL;
    cv_ctx *ctx = I->ctx;
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    std::vector<double> lI(kLogCap * CV_MAX_COMP), lV(kLogCap * CV_MAX_COMP);
    CV_CUDA(ctx, cudaMemcpyAsync(lI.data(), I->log_I, lI.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CV_CUDA(ctx, cudaMemcpyAsync(lV.data(), I->log_var, lV.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CV_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const int nc = I->spec.g.ncomp;
    const int m = max_iter < kLogCap ? max_iter : kLogCap;
    for (int j = 0; j < m; ++j)
        for (int c = 0; c < nc; ++c) {
            iter_I[(size_t)j * nc + c] = lI[(size_t)j * CV_MAX_COMP + c];
            iter_var[(size_t)j * nc + c] = lV[(size_t)j * CV_MAX_COMP + c];
        }
    return CV_OK;
}

// ---- checkpoint / resume and grid reuse
extern "C" int cv_integral_step(cv_integral *I, int max_iter)
{
    if (!I || max_iter < 0) return CV_EINVAL;
    cv_ctx *ctx = I->ctx;
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    if ((I->spec.flags & CV_JIT) && !(I->spec.flags & CV_FP64)) {
        // compile (if needed) before the first launch
        SampleArgs<float> a;
        memset(&a, 0, sizeof(a));
        fill_params<float>(&I->spec.g, &a.g);
        a.nbins = I->spec.nbins;
        a.map = make_map(I->spec.nbins, I->spec.g.ndim, false);
        set_generator(&a, I->spec.g.ndim, I->spec.flags, I->spec.seed);
        JitKernel k;
        std::string err;
        jit_sample_kernel(ctx->device, a, I->spec.g.ndim, a.map.pow2 != 0, min_blocks_f32(I->spec.g.ndim), &k, &err);
    }
    // iterations past the device's stop decision return at once
    for (int j = 0; j < max_iter; ++j) {
        int rc = enqueue_iteration(I, ctx->stream);
        if (rc) return rc;
    }
    return CV_OK;
}

namespace {
struct StateFileHeader {
    char magic[8];                 // "CUBAGPU\0"
    unsigned version;              // 1
    unsigned state_bytes;          // sizeof(DevState)
    int ndim, ncomp, nbins, flags;
    int family[CV_MAX_COMP];
    double a[CV_MAX_COMP][CV_MAX_DIM], u[CV_MAX_COMP][CV_MAX_DIM];
    double epsrel, epsabs;
    long long mineval, maxeval, nstart, nincrease;
    unsigned long long seed;
};

void fill_header(const cv_spec &sp, StateFileHeader *h)
{
    memset(h, 0, sizeof(*h));
    memcpy(h->magic, "CUBAGPU", 8);
    h->version = 2;
    h->state_bytes = (unsigned)sizeof(DevState);
    h->ndim = sp.g.ndim;
    h->ncomp = sp.g.ncomp;
    h->nbins = sp.nbins;
    h->flags = sp.flags & (CV_FP64 | CV_JIT | CV_SCRAMBLE | CV_PSEUDO);
    for (int c = 0; c < sp.g.ncomp; ++c) {
        h->family[c] = sp.g.family[c];
        for (int d = 0; d < sp.g.ndim; ++d) {
            h->a[c][d] = sp.g.a[c][d];
            h->u[c][d] = sp.g.u[c][d];
        }
    }
    h->epsrel = sp.epsrel;
    h->epsabs = sp.epsabs;
    h->mineval = sp.mineval;
    h->maxeval = sp.maxeval;
    h->nstart = sp.nstart;
    h->nincrease = sp.nincrease;
    h->seed = sp.seed;
}
}  // namespace

extern "C" int cv_integral_save(cv_integral *I, const char *path)
{
    if (!I || !path) return CV_EINVAL;
    cv_ctx *ctx = I->ctx;
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    const int ndim = I->spec.g.ndim, N = I->spec.nbins;
    std::vector<char> st(sizeof(DevState));
    std::vector<double> e((size_t)ndim * (N + 1)), H((size_t)ndim * N);
    std::vector<double> lI((size_t)kLogCap * CV_MAX_COMP), lV((size_t)kLogCap * CV_MAX_COMP);
    CV_CUDA(ctx, cudaMemcpyAsync(st.data(), I->st, st.size(), cudaMemcpyDeviceToHost, ctx->stream));
    CV_CUDA(ctx, cudaMemcpyAsync(e.data(), I->edges, e.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CV_CUDA(ctx, cudaMemcpyAsync(H.data(), I->H, H.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CV_CUDA(ctx, cudaMemcpyAsync(lI.data(), I->log_I, lI.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CV_CUDA(ctx, cudaMemcpyAsync(lV.data(), I->log_var, lV.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CV_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    StateFileHeader h;
    fill_header(I->spec, &h);
    FILE *f = fopen(path, "wb");
    if (!f) return fail_msg(ctx, CV_EINVAL, "cannot open %s for writing", path);
    bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(st.data(), st.size(), 1, f) == 1 &&
              fwrite(e.data(), sizeof(double), e.size(), f) == e.size() &&
              fwrite(H.data(), sizeof(double), H.size(), f) == H.size() &&
              fwrite(lI.data(), sizeof(double), lI.size(), f) == lI.size() &&
              fwrite(lV.data(), sizeof(double), lV.size(), f) == lV.size();
    ok = (fclose(f) == 0) && ok;
    if (!ok) return fail_msg(ctx, CV_EINVAL, "writing %s failed", path);
    return CV_OK;
}

namespace {
// A state file read into host memory.
struct StateImage {
    std::vector<char> st;
    std::vector<double> e, H, lI, lV;
};

// Read a file written by cv_integral_save for the problem sp and check it
// before anything reaches a device: the problem description, the grid (each
// axis from 0 to 1, strictly increasing), the histogram (finite, >= 0) and
// the counters of the saved run against the schedule sp implies -- iteration
// j has nstart + j nincrease points, so after `iter` iterations neval is
// their sum (at most maxeval), the next iteration's size follows, and the
// next Sobol index is 1 + the points before it (the last iteration's own
// points not yet counted once the run has stopped).  The reason for a
// refusal goes to msg.
int read_state_file(const cv_spec &sp, const char *path, StateImage *img, char *msg, size_t len)
{
    auto refuse = [&](const char *why) {
        if (msg && len) snprintf(msg, len, "%s: %s", path, why);
        return CV_EINVAL;
    };
    FILE *f = fopen(path, "rb");
    if (!f) return refuse("cannot open");
    StateFileHeader h, want;
    fill_header(sp, &want);
    const int ndim = sp.g.ndim, N = sp.nbins;
    img->st.assign(sizeof(DevState), 0);
    img->e.assign((size_t)ndim * (N + 1), 0.0);
    img->H.assign((size_t)ndim * N, 0.0);
    img->lI.assign((size_t)kLogCap * CV_MAX_COMP, 0.0);
    img->lV.assign((size_t)kLogCap * CV_MAX_COMP, 0.0);
    bool ok = fread(&h, sizeof(h), 1, f) == 1;
    if (ok && memcmp(&h, &want, sizeof(h)) != 0) {
        fclose(f);
        return refuse("holds the state of another problem or format");
    }
    ok = ok && fread(img->st.data(), img->st.size(), 1, f) == 1 &&
         fread(img->e.data(), sizeof(double), img->e.size(), f) == img->e.size() &&
         fread(img->H.data(), sizeof(double), img->H.size(), f) == img->H.size() &&
         fread(img->lI.data(), sizeof(double), img->lI.size(), f) == img->lI.size() &&
         fread(img->lV.data(), sizeof(double), img->lV.size(), f) == img->lV.size();
    const bool extra = ok && fgetc(f) != EOF;
    fclose(f);
    if (!ok) return refuse("is truncated");
    if (extra) return refuse("has bytes after the saved state");
    for (int d = 0; d < ndim; ++d) {
        const double *e = img->e.data() + (size_t)d * (N + 1);
        if (e[0] != 0.0 || e[N] != 1.0) return refuse("a grid axis does not run from 0 to 1");
        for (int k = 0; k < N; ++k)
            if (!(e[k + 1] > e[k])) return refuse("a grid axis is not increasing");
    }
    for (double v : img->H)
        if (!(v >= 0.0) || !std::isfinite(v)) return refuse("the histogram holds a negative or non-finite value");
    DevState S;
    memcpy(&S, img->st.data(), sizeof(S));
    int jmax = 0;
    long long nmax = 0;
    plan(sp.nstart, sp.nincrease, sp.maxeval, &jmax, &nmax);
    if (S.iter < 0 || S.iter > jmax) return refuse("the iteration count is outside the schedule");
    if ((S.stopped != 0 && S.stopped != 1) || (S.fail != 0 && S.fail != 1) || (S.status & ~1) != 0)
        return refuse("the run's flags are not 0 or 1");
    if (S.stopped && S.iter == 0) return refuse("a run stopped before its first iteration");
    long long neval = 0;
    for (int j = 0; j < S.iter; ++j) neval += sp.nstart + (long long)j * sp.nincrease;
    if (S.neval != neval || S.neval > sp.maxeval)
        return refuse("the sample count disagrees with the iterations done");
    const long long n_next = sp.nstart + (long long)S.iter * sp.nincrease;
    const long long n_last = S.iter > 0 ? n_next - sp.nincrease : 0;
    const long long n_cur = S.stopped ? n_last : n_next;
    const unsigned long long next = 1ull + (unsigned long long)(S.stopped ? neval - n_last : neval);
    if (S.n_cur != n_cur) return refuse("the next iteration's size disagrees with the schedule");
    if (S.next_index != next || S.next_index + (unsigned long long)S.n_cur > CV_INDEX_LIMIT)
        return refuse("the next Sobol index disagrees with the samples taken");
    return CV_OK;
}
}  // namespace

extern "C" int cv_integral_check_file(const cv_spec *spec, const char *path, char *msg, int len)
{
    if (msg && len > 0) msg[0] = '\0';
    if (!spec || !path || len < 0 || (len > 0 && !msg)) return CV_EINVAL;
    cv_ctx tmp;  // (host-side messages only: no device is touched)
    if (check_spec(&tmp, spec)) {
        if (msg && len > 0) snprintf(msg, (size_t)len, "%s", tmp.msg);
        return CV_EINVAL;
    }
    StateImage img;
    return read_state_file(*spec, path, &img, msg, (size_t)len);
}

extern "C" int cv_integral_load(cv_integral *I, const char *path)
{
    if (!I || !path) return CV_EINVAL;
    cv_ctx *ctx = I->ctx;
    StateImage img;
    int rc = read_state_file(I->spec, path, &img, ctx->msg, sizeof(ctx->msg));
    if (rc) return rc;
    const int ndim = I->spec.g.ndim, N = I->spec.nbins;
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    CV_CUDA(ctx, cudaMemcpyAsync(I->st, img.st.data(), img.st.size(), cudaMemcpyHostToDevice, ctx->stream));
    CV_CUDA(ctx, cudaMemcpyAsync(I->edges, img.e.data(), img.e.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CV_CUDA(ctx, cudaMemcpyAsync(I->H, img.H.data(), img.H.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CV_CUDA(ctx, cudaMemcpyAsync(I->log_I, img.lI.data(), img.lI.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CV_CUDA(ctx, cudaMemcpyAsync(I->log_var, img.lV.data(), img.lV.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    if (I->ew32) CV_CUDA(ctx, launch_stage_grid(ndim, N, I->edges, I->ew32, I->map, ctx->stream));
    CV_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return CV_OK;
}

extern "C" int cv_integral_set_grid(cv_integral *I, const double *edges)
{
    if (!I || !edges) return CV_EINVAL;
    cv_ctx *ctx = I->ctx;
    const int ndim = I->spec.g.ndim, N = I->spec.nbins;
    for (int d = 0; d < ndim; ++d) {
        const double *e = edges + (size_t)d * (N + 1);
        if (e[0] != 0.0 || e[N] != 1.0) return fail_msg(ctx, CV_EINVAL, "grid axis %d must run from 0 to 1", d);
        for (int k = 0; k < N; ++k)
            if (!(e[k + 1] > e[k])) return fail_msg(ctx, CV_EINVAL, "grid axis %d is not increasing", d);
    }
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    CV_CUDA(ctx, cudaMemcpyAsync(I->edges, edges, (size_t)ndim * (N + 1) * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    if (I->ew32) CV_CUDA(ctx, launch_stage_grid(ndim, N, I->edges, I->ew32, I->map, ctx->stream));
    CV_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return CV_OK;
}

extern "C" int cv_integral_kernels_per_run(const cv_integral *I)
{
    return I ? I->launched_kernels : 0;
}

extern "C" int cv_vegas(cv_ctx *ctx, int ndim, int ncomp, const cv_genz *g, double epsrel,
                        double epsabs, int flags, int seed, int64_t mineval, int64_t maxeval,
                        int64_t nstart, int64_t nincrease, int64_t nbatch, int nbins,
                        int64_t *neval, int *fail, double integral[], double error[],
                        double prob[])
{
    if (!ctx) return CV_EINVAL;
    if (!g) return fail_msg(ctx, CV_EINVAL, "null integrand description");
    if (g->ndim != ndim || g->ncomp != ncomp)
        return fail_msg(ctx, CV_EINVAL, "ndim/ncomp disagree with the integrand description");
    if (!neval || !fail || !integral || !error || !prob) return fail_msg(ctx, CV_EINVAL, "null output");
    cv_spec sp;
    memset(&sp, 0, sizeof(sp));
    sp.g = *g;
    sp.nbins = nbins;
    sp.flags = flags;
    sp.epsrel = epsrel;
    sp.epsabs = epsabs;
    sp.mineval = mineval;
    sp.maxeval = maxeval;
    sp.nstart = nstart;
    sp.nincrease = nincrease;
    sp.nbatch = nbatch;
    sp.seed = (uint64_t)(int64_t)seed;
    // The same problem as the previous call (every field of the spec): its
    // integral again, its iterations from the second repeat on replayed from
    // a graph captured once (the kernel timer needs direct launches).  Any
    // other problem: a fresh one-shot integral with enqueued launches.
    cv_integral *I = ctx->vegas_last;
    int rc = CV_OK;
    if (I && ctx->integrals.count(I) && memcmp(&I->spec, &sp, sizeof(sp)) == 0) {
        I->replay = !ctx->timer_on;
    } else {
        if (I && ctx->integrals.erase(I)) {
            CV_CUDA(ctx, cudaSetDevice(ctx->device));
            cudaStreamSynchronize(ctx->stream);
            integral_free(I);
        }
        ctx->vegas_last = nullptr;
        rc = integral_create(ctx, &sp, &I, true);
        if (rc) return rc;
        ctx->vegas_last = I;
    }
    cv_result res;
    rc = cv_integral_reset(I);
    if (!rc) rc = cv_integral_run(I);
    if (!rc) rc = cv_integral_result(I, &res);
    if (!rc && (flags & CV_VERBOSE_MASK)) {
        std::vector<double> lI((size_t)kLogCap * ncomp), lV((size_t)kLogCap * ncomp);
        if (cv_integral_log(I, kLogCap, lI.data(), lV.data()) == CV_OK)
            for (int j = 0; j < res.iterations && j < kLogCap; ++j)
                for (int c = 0; c < ncomp; ++c)
                    fprintf(stderr, "cv_vegas iteration %d comp %d: %.15g +- %.6g\n", j + 1, c,
                            lI[(size_t)j * ncomp + c], std::sqrt(std::fabs(lV[(size_t)j * ncomp + c])));
    }
    if (rc) return rc;
    *neval = res.neval;
    *fail = res.fail;
    for (int c = 0; c < ncomp; ++c) {
        integral[c] = res.integral[c];
        error[c] = res.error[c];
        prob[c] = res.prob[c];
    }
    if (res.status & 1) return fail_msg(ctx, CV_ENONFINITE, "iteration %d gave a non-finite result", res.iterations);
    return CV_OK;
}

// ------------------------------------------------------------ FP32 peak
// The FP32 pipe's measured rate: every thread runs 8 independent chains
// x <- x b + c (b and c are launch arguments, so nothing folds), 16 steps
// per loop trip; an FMA counts 2 flops.  Four 256-thread blocks per SM keep
// 8 warps per scheduler, far more independent FMAs than the pipe's latency.
namespace {
constexpr int kFmaChains = 8, kFmaUnroll = 16;

__global__ void __launch_bounds__(256) k_fma_chains(float b, float c, int trips, float *sink)
{
    float x[kFmaChains];
#pragma unroll
    for (int j = 0; j < kFmaChains; ++j) x[j] = 1e-3f * (float)threadIdx.x + (float)j;
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < kFmaUnroll; ++u) {
#pragma unroll
            for (int j = 0; j < kFmaChains; ++j) x[j] = __fmaf_rn(x[j], b, c);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < kFmaChains; ++j) s += x[j];
    if (s == -1.0f) *sink = s;  // (never true: keeps the chains live)
}
}  // namespace

extern "C" int cv_fp32_fma_rate(cv_ctx *ctx, double *tflops, double *ms)
{
    if (!ctx || !tflops) return CV_EINVAL;
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    float *sink = nullptr;
    CV_CUDA(ctx, cudaMalloc(&sink, sizeof(float)));
    const int grid = 4 * ctx->sms, trips = 40000;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        k_fma_chains<<<grid, 256, 0, ctx->stream>>>(0.999f, 1e-3f, trips / 10, sink);  // warm-up
        e = cudaEventRecord(e0, ctx->stream);
    }
    if (e == cudaSuccess) {
        k_fma_chains<<<grid, 256, 0, ctx->stream>>>(0.999f, 1e-3f, trips, sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "FP32 FMA rate kernel");
    const double flops = 2.0 * kFmaChains * kFmaUnroll * (double)trips * grid * 256.0;
    *tflops = flops / (t * 1e-3) / 1e12;
    if (ms) *ms = t;
    return CV_OK;
}

extern "C" int cv_vegas_io_bytes(int ndim, int nbins, int64_t *h2d, int64_t *d2h)
{
    if (!h2d || !d2h || ndim < 1 || nbins < 1) return CV_EINVAL;
    // kernel parameters of one iteration (integrand + launch arguments) and
    // the final state read back; the grid and state start on the device.
    *h2d = (int64_t)sizeof(SampleArgs<double>) + (int64_t)sizeof(CombineArgs);
    *d2h = (int64_t)sizeof(DevState);
    return CV_OK;
}

// ------------------------------------------------------------ batched runs
namespace cv {
#define CV_EXTERN_B(D)                                                                       \
    extern template cudaError_t launch_batch_sample<D, true>(const BatchSampleArgs &, int,   \
                                                             cudaStream_t);                  \
    extern template cudaError_t launch_batch_sample<D, false>(const BatchSampleArgs &, int,  \
                                                              cudaStream_t);                 \
    extern template cudaError_t batch_occupancy<D>(bool, int, int *);
CV_FOR_EACH_NDIM(CV_EXTERN_B)
#undef CV_EXTERN_B

static cudaError_t dispatch_batch_sample(int ndim, bool pow2, const BatchSampleArgs &b, int grid,
                                         cudaStream_t s)
{
    switch (ndim) {
#define CV_CASE(D) \
    case D: return pow2 ? launch_batch_sample<D, true>(b, grid, s) : launch_batch_sample<D, false>(b, grid, s);
        CV_FOR_EACH_NDIM(CV_CASE)
#undef CV_CASE
    }
    return cudaErrorInvalidValue;
}

static cudaError_t dispatch_batch_occupancy(int ndim, bool pow2, int stride, int *occ)
{
    switch (ndim) {
#define CV_CASE(D) case D: return batch_occupancy<D>(pow2, stride, occ);
        CV_FOR_EACH_NDIM(CV_CASE)
#undef CV_CASE
    }
    return cudaErrorInvalidValue;
}
}  // namespace cv

// Tile size, in 32-point blocks, of one integral's iteration of n points:
// about 16 tiles per iteration, a power of two between 64 and cap.  It
// depends on the integral alone, so a batch or a serving round never
// changes how an integral's points are grouped and summed.
// Tile of an iteration of n points: the smallest power of two >= 64
// blocks that cuts the iteration into at most `split` tiles, capped at
// `cap` blocks.  A tile is shared evenly by a CTA's eight warps, so the
// points each thread takes from a tile are tile / 8: split and cap set the
// points per thread (the autotuner picks both).
static int tile_blocks_for(long long n, int cap, int split = 16)
{
    const long long blocks = (n + 31) / 32 + 1;
    long long t = 64;
    while (t < cap && t * split < blocks) t <<= 1;
    return (int)t;
}

// A set of integrals run together: per iteration one persistent sampling
// launch per dimension class (ndim, power-of-two bins) over a queue of
// tiles, then one batched refinement and one batched combination.
struct cv_batch {
    cv_ctx *ctx = nullptr;
    int count = 0;
    std::vector<cv_spec> specs;
    std::vector<int> jmax;                       // iterations of each integral
    std::vector<long long> n0;                   // first iteration size
    void *mem = nullptr;                         // states, grids, histograms, logs
    std::vector<double *> edges, log_I, log_var; // per integral (device)
    std::vector<int> log_cap;                    // iterations each log holds
    BatchItem *d_items = nullptr;
    CombineArgs *d_cargs = nullptr;
    int2 *d_axes = nullptr;
    int naxes = 0;
    Tile *d_tiles = nullptr;
    int *d_counters = nullptr;
    size_t tiles_cap = 0, counters_cap = 0;
    int J = 0;                                   // iterations of the longest run
    // dimension classes: slots per axis, persistent grid
    struct Class { int ndim; bool pow2; int stride; int grid; };
    std::vector<Class> classes;
    int tile_cap = 2048;                         // largest tile, in 32-point blocks
    int tile_split = 16;                         // an iteration's tiles (at most), below the cap
    int tile_fixed = 0;                          // CUBAGPU_TILE: every tile this size
    std::vector<int> item_class;
    // launch plan: per iteration, per class: tile offset and count, counter index
    struct Launch { int j, cls, tile_off, ntiles, counter; };
    std::vector<Launch> plan;
    // the tiles' partial rows (one iteration's at a time) and, per
    // iteration and integral, where its rows are
    double *d_part_S = nullptr;
    float *d_part_H = nullptr;
    TileParts *d_tparts = nullptr;
    size_t part_rows_cap = 0, part_floats_cap = 0, tparts_cap = 0;
    cudaGraphExec_t exec = nullptr;
    int kernels_per_run = 0;
};

static void batch_free_device(cv_batch *B)
{
    if (B->exec) cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
    if (B->mem) cudaFree(B->mem);
    if (B->d_tiles) cudaFree(B->d_tiles);
    if (B->d_counters) cudaFree(B->d_counters);
    if (B->d_part_S) cudaFree(B->d_part_S);
    if (B->d_part_H) cudaFree(B->d_part_H);
    if (B->d_tparts) cudaFree(B->d_tparts);
    B->mem = nullptr;
    B->d_tiles = nullptr;
    B->d_counters = nullptr;
    B->d_part_S = nullptr;
    B->d_part_H = nullptr;
    B->d_tparts = nullptr;
    B->part_rows_cap = B->part_floats_cap = B->tparts_cap = 0;
}

// A device buffer of at least `need` elements of T, grown (never shrunk)
// when it is smaller; *cap counts elements.
template <typename T>
static int grow_device(cv_ctx *ctx, T **p, size_t *cap, size_t need, const char *what)
{
    if (need <= *cap && *p) return CV_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (cudaMalloc((void **)p, std::max<size_t>(need, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail_msg(ctx, CV_ENOMEM, "device allocation of %s failed", what);
    }
    *cap = need;
    return CV_OK;
}

// Histogram row stride of a tile partial: ndim nbins floats rounded up to
// a multiple of 4 (16-byte aligned rows).
static unsigned tile_row_floats(int ndim, int nbins) { return ((unsigned)(ndim * nbins) + 3u) & ~3u; }

// Generate every tile of every iteration for the current tile sizes.
static int batch_build_tiles(cv_batch *B, int only_first_iteration)
{
    cv_ctx *ctx = B->ctx;
    std::vector<Tile> tiles;
    B->plan.clear();
    const int J = only_first_iteration ? 1 : B->J;
    int counter = 0;
    // partial rows: numbered from 0 in every iteration (an iteration's
    // launches finish before the next iteration's start)
    std::vector<TileParts> tparts((size_t)J * B->count, TileParts{0, 0, 0u, 0});
    size_t rows_max = 0, floats_max = 0;
    for (int j = 0; j < J; ++j) {
        const size_t it0 = tiles.size();
        size_t hf = 0;
        for (size_t c = 0; c < B->classes.size(); ++c) {
            const int off = (int)tiles.size();
            for (int i = 0; i < B->count; ++i) {
                if (B->item_class[i] != (int)c || j >= B->jmax[i]) continue;
                TileParts &tp = tparts[(size_t)j * B->count + i];
                tp.row0 = (int)(tiles.size() - it0);
                tp.hoff0 = (unsigned)hf;
                tp.stride = (int)tile_row_floats(B->specs[i].g.ndim, B->specs[i].nbins);
                const cv_spec &sp = B->specs[i];
                // start index and size of iteration j (the device follows the same plan)
                unsigned long long s = 1;
                for (int jj = 0; jj < j; ++jj) s += (unsigned long long)(sp.nstart + (long long)jj * sp.nincrease);
                const unsigned long long n = (unsigned long long)(sp.nstart + (long long)j * sp.nincrease);
                const int TB = B->tile_fixed ? B->tile_fixed : tile_blocks_for((long long)n, B->tile_cap, B->tile_split);
                // (tiles start on even 32-point blocks: see run_steps)
                const unsigned long long qa = (s >> 5) & ~1ull, qb = (s + n + 31) >> 5;
                for (unsigned long long q = qa; q < qb; q += (unsigned long long)TB) {
                    Tile t;
                    t.item = i;
                    t.nblk = (int)(qb - q < (unsigned long long)TB ? qb - q : (unsigned long long)TB);
                    t.q0 = q;
                    t.row = (int)(tiles.size() - it0);
                    t.hoff = (unsigned)hf;
                    hf += (size_t)tp.stride;
                    tiles.push_back(t);
                    ++tp.count;
                }
            }
            const int nt = (int)tiles.size() - off;
            if (nt > 0) B->plan.push_back({j, (int)c, off, nt, counter++});
        }
        rows_max = std::max(rows_max, tiles.size() - it0);
        floats_max = std::max(floats_max, hf);
    }
    if (floats_max > 0xffffffffull) return fail_msg(ctx, CV_ENOMEM, "tile partials beyond 2^32 floats per iteration");
    {
        int rc = grow_device(ctx, &B->d_part_S, &B->part_rows_cap, rows_max * 2 * CV_MAX_COMP, "tile sum partials");
        if (!rc) rc = grow_device(ctx, &B->d_part_H, &B->part_floats_cap, floats_max, "tile histogram partials");
        if (!rc) rc = grow_device(ctx, &B->d_tparts, &B->tparts_cap, tparts.size(), "tile partial maps");
        if (rc) return rc;
    }
    if (tiles.size() > B->tiles_cap) {
        if (B->d_tiles) cudaFree(B->d_tiles);
        B->d_tiles = nullptr;
        if (cudaMalloc(&B->d_tiles, tiles.size() * sizeof(Tile)) != cudaSuccess) {
            cudaGetLastError();
            return fail_msg(ctx, CV_ENOMEM, "tile queue allocation failed");
        }
        B->tiles_cap = tiles.size();
    }
    if ((size_t)counter > B->counters_cap) {
        if (B->d_counters) cudaFree(B->d_counters);
        B->d_counters = nullptr;
        if (cudaMalloc(&B->d_counters, (size_t)counter * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            return fail_msg(ctx, CV_ENOMEM, "tile counter allocation failed");
        }
        B->counters_cap = counter;
    }
    if (!tiles.empty()) {
        CV_CUDA(ctx, cudaMemcpyAsync(B->d_tiles, tiles.data(), tiles.size() * sizeof(Tile),
                                     cudaMemcpyHostToDevice, ctx->stream));
        CV_CUDA(ctx, cudaMemcpyAsync(B->d_tparts, tparts.data(), tparts.size() * sizeof(TileParts),
                                     cudaMemcpyHostToDevice, ctx->stream));
        CV_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return CV_OK;
}

// Enqueue the whole run (reset + every iteration) on stream s.
static int batch_enqueue(cv_batch *B, cudaStream_t s, int first_iteration_sampling_only)
{
    cv_ctx *ctx = B->ctx;
    int kernels = 0;
    if (B->counters_cap)
        CV_CUDA(ctx, cudaMemsetAsync(B->d_counters, 0, B->counters_cap * sizeof(int), s));
    CV_CUDA(ctx, launch_batch_reset(B->d_items, B->d_cargs, B->count, s));
    ++kernels;
    size_t p = 0;
    const int J = first_iteration_sampling_only ? 1 : B->J;
    for (int j = 0; j < J; ++j) {
        // the classes of an iteration run concurrently on side streams
        CV_CUDA(ctx, cudaEventRecord(ctx->ev_fork, s));
        for (int k = 0; k < kSideStreams; ++k) CV_CUDA(ctx, cudaStreamWaitEvent(ctx->side[k], ctx->ev_fork, 0));
        int used = 0;
        for (; p < B->plan.size() && B->plan[p].j == j; ++p) {
            const cv_batch::Launch &L = B->plan[p];
            const cv_batch::Class &C = B->classes[L.cls];
            BatchSampleArgs a;
            a.items = B->d_items;
            a.tiles = B->d_tiles + L.tile_off;
            a.ntiles = L.ntiles;
            a.stride = C.stride;
            a.counter = B->d_counters + L.counter;
            a.part_S = B->d_part_S;
            a.part_H = B->d_part_H;
            const int grid = C.grid < L.ntiles ? C.grid : L.ntiles;
            CV_CUDA(ctx, dispatch_batch_sample(C.ndim, C.pow2, a, grid, ctx->side[used % kSideStreams]));
            ++used;
            ++kernels;
        }
        for (int k = 0; k < kSideStreams; ++k) {
            CV_CUDA(ctx, cudaEventRecord(ctx->ev_join[k], ctx->side[k]));
            CV_CUDA(ctx, cudaStreamWaitEvent(s, ctx->ev_join[k], 0));
        }
        if (first_iteration_sampling_only) break;
        const TileParts *tp = B->d_tparts + (size_t)j * B->count;
        CV_CUDA(ctx, launch_batch_refine(B->d_items, B->d_axes, B->naxes, s, tp, B->d_part_H));
        CV_CUDA(ctx, launch_batch_combine(B->d_cargs, B->count, s, nullptr, tp, B->d_part_S));
        kernels += 2;
    }
    B->kernels_per_run = kernels;
    return CV_OK;
}

static int batch_capture(cv_batch *B)
{
    cv_ctx *ctx = B->ctx;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
    cudaGraph_t graph = nullptr;
    CV_CUDA(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = batch_enqueue(B, ctx->cap_stream, 0);
    cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch graph capture");
    e = cudaGraphInstantiate(&B->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch graph instantiate");
    return CV_OK;
}

// Tile cap from the environment (CUBAGPU_TILE, points per tile: every tile
// that size) or the default.
static void batch_default_tiles(cv_batch *B)
{
    const char *env = getenv("CUBAGPU_TILE");
    const long long forced = env ? atoll(env) : 0;
    B->tile_fixed = forced > 0 ? (int)(forced / 32 > 0 ? forced / 32 : 1) : 0;
}

extern "C" int cv_batch_create(cv_ctx *ctx, int count, const cv_spec *specs, cv_batch **out)
{
    if (!ctx || !out) return CV_EINVAL;
    *out = nullptr;
    if (count < 1 || !specs) return fail_msg(ctx, CV_EINVAL, "empty batch");
    for (int i = 0; i < count; ++i) {
        int rc = check_spec(ctx, &specs[i]);
        if (rc) return rc;
        if (specs[i].flags & (CV_FP64 | CV_PLAIN))
            return fail_msg(ctx, CV_EINVAL, "batched runs use the FP32 path (item %d asks for CV_FP64/CV_PLAIN)", i);
        if (specs[i].flags & CV_PSEUDO)
            return fail_msg(ctx, CV_EINVAL, "batched runs take Sobol or scrambled Sobol points (item %d)", i);
    }
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    cv_batch *B = new cv_batch();
    B->ctx = ctx;
    B->count = count;
    B->specs.assign(specs, specs + count);
    B->jmax.resize(count);
    B->n0.resize(count);
    B->item_class.resize(count);
    // per-integral device memory: state, grid, histogram
    const size_t sz_state = (sizeof(DevState) + 255) & ~(size_t)255;
    std::vector<size_t> off(count);
    size_t total = 0;
    for (int i = 0; i < count; ++i) {
        const int ndim = specs[i].g.ndim, N = specs[i].nbins;
        long long nmax = 0;
        plan(specs[i].nstart, specs[i].nincrease, specs[i].maxeval, &B->jmax[i], &nmax);
        B->n0[i] = specs[i].nstart;
        B->J = B->J > B->jmax[i] ? B->J : B->jmax[i];
        off[i] = total;
        const size_t lcap = (size_t)(B->jmax[i] < kLogCap ? B->jmax[i] : kLogCap);
        total += sz_state + ((((size_t)ndim * (N + 1) * sizeof(double)) + 255) & ~(size_t)255) +
                 ((((size_t)ndim * N * sizeof(double)) + 255) & ~(size_t)255) +
                 ((2 * lcap * CV_MAX_COMP * sizeof(double) + 255) & ~(size_t)255);
        // (the map's form decides the kernel: powers of two from 32 bins)
        const bool p2 = make_map(N, ndim, false).pow2 != 0;
        int c = -1;
        for (size_t k = 0; k < B->classes.size(); ++k)
            if (B->classes[k].ndim == ndim && B->classes[k].pow2 == p2) c = (int)k;
        if (c < 0) {
            B->classes.push_back({ndim, p2, N, 0});
            c = (int)B->classes.size() - 1;
        }
        if (N > B->classes[c].stride) B->classes[c].stride = N;
        B->item_class[i] = c;
    }
    for (cv_batch::Class &C : B->classes) {
        int occ = 0;
        cudaError_t e = dispatch_batch_occupancy(C.ndim, C.pow2, C.stride, &occ);
        if (e != cudaSuccess || occ < 1) {
            cudaGetLastError();
            const int nd = C.ndim, st = C.stride;
            delete B;
            return fail_msg(ctx, CV_EINVAL, "%d dimensions x %d bins exceed the batched path's shared "
                            "memory (per-warp histograms); run such integrals with cv_vegas",
                            nd, st);
        }
        C.grid = ctx->sms * occ;
    }
    size_t sz_items = (((size_t)count * sizeof(BatchItem)) + 255) & ~(size_t)255;
    size_t sz_cargs = (((size_t)count * sizeof(CombineArgs)) + 255) & ~(size_t)255;
    B->naxes = 0;
    for (int i = 0; i < count; ++i) B->naxes += specs[i].g.ndim;
    size_t sz_axes = (size_t)B->naxes * sizeof(int2);
    if (cudaMalloc(&B->mem, total + sz_items + sz_cargs + sz_axes) != cudaSuccess) {
        cudaGetLastError();
        delete B;
        return fail_msg(ctx, CV_ENOMEM, "device allocation of %zu bytes for the batch failed", total);
    }
    char *base = (char *)B->mem;
    B->d_items = (BatchItem *)(base + total);
    B->d_cargs = (CombineArgs *)(base + total + sz_items);
    B->d_axes = (int2 *)(base + total + sz_items + sz_cargs);
    std::vector<BatchItem> items(count);
    std::vector<CombineArgs> cargs(count);
    std::vector<int2> axes;
    axes.reserve(B->naxes);
    for (int i = 0; i < count; ++i) {
        const cv_spec &sp = specs[i];
        const int ndim = sp.g.ndim, N = sp.nbins;
        char *p = base + off[i];
        BatchItem &it = items[i];
        memset(&it, 0, sizeof(it));
        fill_params<float>(&sp.g, &it.a.g);
        it.a.nbins = N;
        it.a.chunk_min = 4;
        it.a.map = make_map(N, ndim, false);
        it.a.map.priv = it.a.map.pow2;  // every warp has its own histogram
        set_generator(&it.a, ndim, sp.flags, sp.seed);
        it.st = (DevState *)p;
        it.edges = (double *)(p + sz_state);
        it.H = (double *)(p + sz_state + ((((size_t)ndim * (N + 1) * sizeof(double)) + 255) & ~(size_t)255));
        const int lcap = B->jmax[i] < kLogCap ? B->jmax[i] : kLogCap;
        double *logs = it.H + (((((size_t)ndim * N * sizeof(double)) + 255) & ~(size_t)255) / sizeof(double));
        B->edges.push_back(it.edges);
        B->log_I.push_back(logs);
        B->log_var.push_back(logs + (size_t)lcap * CV_MAX_COMP);
        B->log_cap.push_back(lcap);
        CombineArgs &ca = cargs[i];
        ca.st = it.st;
        ca.ncomp = sp.g.ncomp;
        ca.epsrel = sp.epsrel;
        ca.epsabs = sp.epsabs;
        ca.mineval = sp.mineval;
        ca.maxeval = sp.maxeval;
        ca.nstart = sp.nstart;
        ca.nincrease = sp.nincrease;
        ca.log_I = B->log_I[i];
        ca.log_var = B->log_var[i];
        ca.log_cap = lcap;
        for (int d = 0; d < ndim; ++d) axes.push_back(make_int2(i, d));
    }
    int rc = CV_OK;
    cudaError_t e = cudaMemcpyAsync(B->d_items, items.data(), count * sizeof(BatchItem), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(B->d_cargs, cargs.data(), count * sizeof(CombineArgs), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(B->d_axes, axes.data(), axes.size() * sizeof(int2), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "batch upload");
    if (!rc) {
        batch_default_tiles(B);
        rc = batch_build_tiles(B, 0);
    }
    if (rc) {
        batch_free_device(B);
        delete B;
        return rc;
    }
    ctx->batches.insert(B);
    *out = B;
    return CV_OK;
}

static void batch_release(cv_batch *B)
{
    batch_free_device(B);
    delete B;
}

extern "C" void cv_batch_destroy(cv_batch *B)
{
    if (!B) return;
    cv_ctx *ctx = B->ctx;
    if (!ctx->batches.erase(B)) return;  // not (or no longer) a live handle
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    batch_release(B);
}

extern "C" int cv_batch_run(cv_batch *B)
{
    if (!B) return CV_EINVAL;
    cv_ctx *ctx = B->ctx;
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    if (!B->exec) {
        int rc = batch_capture(B);
        if (rc) return rc;
    }
    CV_CUDA(ctx, cudaGraphLaunch(B->exec, ctx->stream));
    return CV_OK;
}

extern "C" int cv_batch_results(cv_batch *B, cv_result *out)
{
    if (!B || !out) return CV_EINVAL;
    cv_ctx *ctx = B->ctx;
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    std::vector<BatchItem> items(B->count);
    CV_CUDA(ctx, cudaMemcpyAsync(items.data(), B->d_items, B->count * sizeof(BatchItem), cudaMemcpyDeviceToHost, ctx->stream));
    CV_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < B->count; ++i) {
        DevState h;
        CV_CUDA(ctx, cudaMemcpyAsync(&h, items[i].st, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
        CV_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        cv_result &r = out[i];
        memset(&r, 0, sizeof(r));
        r.neval = h.neval;
        r.fail = h.stopped ? h.fail : 1;
        r.iterations = h.iter;
        r.status = h.status;
        for (int c = 0; c < B->specs[i].g.ncomp; ++c) {
            r.integral[c] = h.integral[c];
            r.error[c] = h.error[c];
            r.prob[c] = h.prob[c];
            r.chi2[c] = h.chi2[c];
        }
    }
    return CV_OK;
}

extern "C" int cv_batch_log(cv_batch *B, int item, int max_iter, double *iter_I, double *iter_var)
{
    if (!B || !iter_I || !iter_var || item < 0 || item >= B->count || max_iter < 0) return CV_EINVAL;
    cv_ctx *ctx = B->ctx;
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    const int lc = B->log_cap[item], nc = B->specs[item].g.ncomp;
    std::vector<double> lI((size_t)lc * CV_MAX_COMP), lV((size_t)lc * CV_MAX_COMP);
    if (lc > 0) {
        CV_CUDA(ctx, cudaMemcpyAsync(lI.data(), B->log_I[item], lI.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CV_CUDA(ctx, cudaMemcpyAsync(lV.data(), B->log_var[item], lV.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    }
    CV_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const int m = max_iter < lc ? max_iter : lc;
    for (int j = 0; j < m; ++j)
        for (int c = 0; c < nc; ++c) {
            iter_I[j * nc + c] = lI[(size_t)j * CV_MAX_COMP + c];
            iter_var[j * nc + c] = lV[(size_t)j * CV_MAX_COMP + c];
        }
    return CV_OK;
}

extern "C" int cv_batch_grid(cv_batch *B, int item, double *edges)
{
    if (!B || !edges || item < 0 || item >= B->count) return CV_EINVAL;
    cv_ctx *ctx = B->ctx;
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    const size_t n = (size_t)B->specs[item].g.ndim * (B->specs[item].nbins + 1);
    CV_CUDA(ctx, cudaMemcpyAsync(edges, B->edges[item], n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CV_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return CV_OK;
}

extern "C" int cv_batch_kernels_per_run(const cv_batch *B) { return B ? B->kernels_per_run : 0; }

extern "C" int cv_batch_tile_points(const cv_batch *B, long long n)
{
    if (!B) return 0;
    return 32 * (B->tile_fixed ? B->tile_fixed : tile_blocks_for(n, B->tile_cap, B->tile_split));
}

// Measured tuning of the tiles: time the first iteration's sampling
// launches of every class for tile caps of 256, 1024 and 4096 blocks and
// iterations cut into at most 8, 16 or 32 tiles below the cap (the points
// per thread), a reset before each trial so no result is affected, and
// keep the fastest total.  The tiles still depend on each integral alone.
extern "C" int cv_batch_autotune(cv_batch *B)
{
    if (!B) return CV_EINVAL;
    if (B->tile_fixed) return CV_OK;
    cv_ctx *ctx = B->ctx;
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    static const int caps[] = {256, 1024, 4096};
    static const int splits[] = {8, 16, 32};
    float best = 1e30f;
    int best_cap = B->tile_cap, best_split = B->tile_split;
    cudaEvent_t e0, e1;
    CV_CUDA(ctx, cudaEventCreate(&e0));
    CV_CUDA(ctx, cudaEventCreate(&e1));
    int rc = CV_OK;
    for (int ci = 0; ci < 3 && !rc; ++ci) {
        for (int si = 0; si < 3 && !rc; ++si) {
            B->tile_cap = caps[ci];
            B->tile_split = splits[si];
            rc = batch_build_tiles(B, 1);
            if (rc) break;
            if (B->counters_cap) cudaMemsetAsync(B->d_counters, 0, B->counters_cap * sizeof(int), ctx->stream);
            launch_batch_reset(B->d_items, B->d_cargs, B->count, ctx->stream);
            cudaEventRecord(e0, ctx->stream);
            for (const cv_batch::Launch &L : B->plan) {
                const cv_batch::Class &C = B->classes[L.cls];
                BatchSampleArgs a;
                a.items = B->d_items;
                a.tiles = B->d_tiles + L.tile_off;
                a.ntiles = L.ntiles;
                a.stride = C.stride;
                a.counter = B->d_counters + L.counter;
                a.part_S = B->d_part_S;
                a.part_H = B->d_part_H;
                cudaError_t e = dispatch_batch_sample(C.ndim, C.pow2, a, C.grid < L.ntiles ? C.grid : L.ntiles, ctx->stream);
                if (e != cudaSuccess) {
                    rc = cuda_fail(ctx, e, "autotune launch");
                    break;
                }
            }
            cudaEventRecord(e1, ctx->stream);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_cap = caps[ci];
                best_split = splits[si];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    B->tile_cap = best_cap;
    B->tile_split = best_split;
    if (!rc) rc = batch_build_tiles(B, 0);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
    return rc;
}

extern "C" int cv_batch_vegas(cv_ctx *ctx, int count, const cv_spec *specs, cv_result *out)
{
    if (!out) return fail_msg(ctx, CV_EINVAL, "null output");
    cv_batch *B = nullptr;
    int rc = cv_batch_create(ctx, count, specs, &B);
    if (rc) return rc;
    rc = cv_batch_run(B);
    if (!rc) rc = cv_batch_results(B, out);
    cv_batch_destroy(B);
    return rc;
}

// ------------------------------------------------------------ serving loop
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator of device offsets inside the server's arena (the HBM
// budget), 256-byte granules, neighbours coalesced on free.
class Arena {
public:
    explicit Arena(size_t bytes) { free_[0] = bytes; }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = (bytes + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = (bytes + 255) & ~(size_t)255;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }

private:
    std::map<size_t, size_t> free_;
};

size_t request_bytes(const cv_spec &sp)
{
    const size_t st = (sizeof(DevState) + 255) & ~(size_t)255;
    const size_t e = (((size_t)sp.g.ndim * (sp.nbins + 1) * sizeof(double)) + 255) & ~(size_t)255;
    const size_t h = (((size_t)sp.g.ndim * sp.nbins * sizeof(double)) + 255) & ~(size_t)255;
    return st + e + h;
}

struct Request {
    uint64_t id;
    cv_spec spec;
    Clock::time_point arrival;
    // while live
    int slot = -1;
    size_t off = 0, bytes = 0;
    int j = 0;                          // iterations done (host mirror of the device plan)
    unsigned long long next_index = 1;
    int jmax = 0;
};

}  // namespace

struct cv_server {
    cv_ctx *ctx = nullptr;
    cv_server_opts opts;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_new, cv_done;
    bool stopping = false;
    int error = CV_OK;
    uint64_t next_id = 1;
    std::deque<Request> pending;
    std::map<uint64_t, cv_result> done;
    std::map<uint64_t, double> latency_ms;
    // statistics
    int64_t submitted = 0, completed = 0, rounds = 0, samples = 0;
    int max_live_seen = 0;
    double busy_s = 0, gpu_s = 0;
    Clock::time_point t_start;
    // device resources (worker thread only)
    cudaStream_t stream = nullptr;
    cudaStream_t side[kSideStreams] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kSideStreams] = {};
    cudaEvent_t ev_t0 = nullptr, ev_t1 = nullptr;  // device time of a round
    void *arena_mem = nullptr;
    BatchItem *d_items = nullptr;
    CombineArgs *d_cargs = nullptr;
    int *d_lists = nullptr;              // reset list | combine/gather list
    int2 *d_axes = nullptr;
    Tile *d_tiles = nullptr;
    size_t tiles_cap = 0;
    int *d_counters = nullptr;
    DevState *d_gather = nullptr;
    DevState *h_gather = nullptr;        // pinned
    std::vector<int> class_grid;         // persistent grid per (ndim, pow2) class, 0 = unknown
    // the round's tile partial rows, and per slot where its request's are
    double *d_part_S = nullptr;
    float *d_part_H = nullptr;
    size_t part_rows_cap = 0, part_floats_cap = 0;
    TileParts *d_tparts = nullptr;       // [max_live]
    std::vector<TileParts> h_tparts;     // [max_live]
    std::vector<unsigned> slot_stride;   // [max_live]: histogram row floats of the slot's request
};

namespace {

int server_round(cv_server *S, std::vector<Request> &live, Arena &arena,
                 std::vector<int> &free_slots)
{
    cv_ctx *ctx = S->ctx;
    const int max_live = S->opts.max_live;
    // ---- admission: FIFO, while a slot and the budget allow
    std::vector<int> fresh;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        while (!S->pending.empty() && !free_slots.empty()) {
            Request &r = S->pending.front();
            size_t off;
            if (!arena.alloc(r.bytes, &off)) break;
            r.off = off;
            r.slot = free_slots.back();
            free_slots.pop_back();
            long long nmax = 0;
            plan(r.spec.nstart, r.spec.nincrease, r.spec.maxeval, &r.jmax, &nmax);
            live.push_back(r);
            fresh.push_back(r.slot);
            S->pending.pop_front();
        }
    }
    (void)max_live;
    if (live.empty()) return CV_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if ((int)live.size() > S->max_live_seen) S->max_live_seen = (int)live.size();
    }
    const auto t0 = Clock::now();
    CV_CUDA(ctx, cudaEventRecord(S->ev_t0, S->stream));
    // descriptors of newly admitted requests
    const size_t sz_state = (sizeof(DevState) + 255) & ~(size_t)255;
    for (const Request &r : live) {
        if (std::find(fresh.begin(), fresh.end(), r.slot) == fresh.end()) continue;
        const cv_spec &sp = r.spec;
        const int ndim = sp.g.ndim, N = sp.nbins;
        char *p = (char *)S->arena_mem + r.off;
        BatchItem it;
        memset(&it, 0, sizeof(it));
        fill_params<float>(&sp.g, &it.a.g);
        it.a.nbins = N;
        it.a.chunk_min = 4;
        it.a.map = make_map(N, ndim, false);
        it.a.map.priv = it.a.map.pow2;  // every warp has its own histogram
        set_generator(&it.a, ndim, sp.flags, sp.seed);
        it.st = (DevState *)p;
        it.edges = (double *)(p + sz_state);
        it.H = (double *)(p + sz_state + ((((size_t)ndim * (N + 1) * sizeof(double)) + 255) & ~(size_t)255));
        CombineArgs ca = {};
        ca.st = it.st;
        ca.ncomp = sp.g.ncomp;
        ca.epsrel = sp.epsrel;
        ca.epsabs = sp.epsabs;
        ca.mineval = sp.mineval;
        ca.maxeval = sp.maxeval;
        ca.nstart = sp.nstart;
        ca.nincrease = sp.nincrease;
        ca.log_I = nullptr;
        ca.log_var = nullptr;
        ca.log_cap = 0;
        CV_CUDA(ctx, cudaMemcpyAsync(S->d_items + r.slot, &it, sizeof(it), cudaMemcpyHostToDevice, S->stream));
        CV_CUDA(ctx, cudaMemcpyAsync(S->d_cargs + r.slot, &ca, sizeof(ca), cudaMemcpyHostToDevice, S->stream));
    }
    // ---- this round's work: one iteration of every live request
    std::vector<int> lists(fresh);
    const int nfresh = (int)fresh.size();
    std::vector<int2> axes;
    for (const Request &r : live) {
        lists.push_back(r.slot);
        for (int d = 0; d < r.spec.g.ndim; ++d) axes.push_back(make_int2(r.slot, d));
    }
    const int nlive = (int)live.size();
    // tiles grouped by dimension class
    struct Cls { int ndim; bool pow2; int stride; std::vector<Tile> tiles; };
    std::vector<Cls> cls;
    int64_t round_samples = 0;
    for (const Request &r : live) {
        const int ndim = r.spec.g.ndim;
        S->slot_stride[r.slot] = tile_row_floats(ndim, r.spec.nbins);
        const bool p2 = make_map(r.spec.nbins, ndim, false).pow2 != 0;  // (powers of two from 32 bins)
        Cls *c = nullptr;
        for (Cls &k : cls)
            if (k.ndim == ndim && k.pow2 == p2) c = &k;
        if (!c) {
            cls.push_back({ndim, p2, r.spec.nbins, {}});
            c = &cls.back();
        }
        c->stride = std::max(c->stride, r.spec.nbins);
        const unsigned long long s = r.next_index;
        const unsigned long long n = (unsigned long long)(r.spec.nstart + (long long)r.j * r.spec.nincrease);
        const long long tb = S->opts.tile_points > 0 ? std::max(1, S->opts.tile_points / 32)
                                                     : tile_blocks_for((long long)n, 2048);
        const unsigned long long qa = (s >> 5) & ~1ull, qb = (s + n + 31) >> 5;
        for (unsigned long long q = qa; q < qb; q += (unsigned long long)tb) {
            Tile t;
            t.item = r.slot;
            t.nblk = (int)std::min<unsigned long long>(qb - q, (unsigned long long)tb);
            t.q0 = q;
            c->tiles.push_back(t);
        }
        round_samples += (int64_t)n;
    }
    size_t ntiles = 0;
    for (const Cls &c : cls) ntiles += c.tiles.size();
    if (ntiles > S->tiles_cap) {
        if (S->d_tiles) cudaFree(S->d_tiles);
        S->d_tiles = nullptr;
        const size_t cap = std::max(ntiles, 2 * S->tiles_cap);
        CV_CUDA(ctx, cudaMalloc(&S->d_tiles, cap * sizeof(Tile)));
        S->tiles_cap = cap;
    }
    std::vector<Tile> all;
    all.reserve(ntiles);
    for (const Cls &c : cls) all.insert(all.end(), c.tiles.begin(), c.tiles.end());
    // the round's partial rows: tile k of the queue at row k, its histogram
    // after the previous tiles'; a request's tiles are consecutive
    size_t hf = 0;
    for (size_t k = 0; k < all.size(); ++k) {
        Tile &t = all[k];
        TileParts &tp = S->h_tparts[t.item];
        const unsigned stride = S->slot_stride[t.item];
        if (k == 0 || all[k - 1].item != t.item) tp = TileParts{(int)k, 0, (unsigned)hf, (int)stride};
        t.row = (int)k;
        t.hoff = (unsigned)hf;
        hf += stride;
        ++tp.count;
    }
    if (hf > 0xffffffffull) return fail_msg(ctx, CV_ENOMEM, "tile partials beyond 2^32 floats per round");
    {
        int rc = grow_device(ctx, &S->d_part_S, &S->part_rows_cap, all.size() * 2 * CV_MAX_COMP, "tile sum partials");
        if (!rc) rc = grow_device(ctx, &S->d_part_H, &S->part_floats_cap, hf, "tile histogram partials");
        if (rc) return rc;
    }
    CV_CUDA(ctx, cudaMemcpyAsync(S->d_tiles, all.data(), all.size() * sizeof(Tile), cudaMemcpyHostToDevice, S->stream));
    CV_CUDA(ctx, cudaMemcpyAsync(S->d_tparts, S->h_tparts.data(), S->h_tparts.size() * sizeof(TileParts),
                                 cudaMemcpyHostToDevice, S->stream));
    CV_CUDA(ctx, cudaMemcpyAsync(S->d_lists, lists.data(), lists.size() * sizeof(int), cudaMemcpyHostToDevice, S->stream));
    CV_CUDA(ctx, cudaMemcpyAsync(S->d_axes, axes.data(), axes.size() * sizeof(int2), cudaMemcpyHostToDevice, S->stream));
    CV_CUDA(ctx, cudaMemsetAsync(S->d_counters, 0, 2 * (CV_MAX_DIM + 1) * sizeof(int), S->stream));
    CV_CUDA(ctx, launch_batch_reset(S->d_items, S->d_cargs, nfresh, S->stream, S->d_lists));
    // classes run concurrently on side streams, the largest first
    std::vector<int> order(cls.size());
    for (size_t i = 0; i < cls.size(); ++i) order[i] = (int)i;
    std::vector<size_t> offs(cls.size());
    {
        size_t o = 0;
        for (size_t i = 0; i < cls.size(); ++i) {
            offs[i] = o;
            o += cls[i].tiles.size();
        }
    }
    std::sort(order.begin(), order.end(), [&](int x, int y) { return cls[x].tiles.size() > cls[y].tiles.size(); });
    CV_CUDA(ctx, cudaEventRecord(S->ev_fork, S->stream));
    for (int k = 0; k < kSideStreams; ++k) CV_CUDA(ctx, cudaStreamWaitEvent(S->side[k], S->ev_fork, 0));
    int used = 0;
    for (int ci : order) {
        const Cls &c = cls[ci];
        const size_t off = offs[ci];
        int &g = S->class_grid[((c.pow2 ? 1 : 0) * (CV_MAX_DIM + 1) + c.ndim) * (CV_MAX_BINS + 1) + c.stride];
        if (!g) {
            int occ = 0;
            CV_CUDA(ctx, dispatch_batch_occupancy(c.ndim, c.pow2, c.stride, &occ));
            g = ctx->sms * std::max(occ, 1);
        }
        BatchSampleArgs a;
        a.items = S->d_items;
        a.tiles = S->d_tiles + off;
        a.ntiles = (int)c.tiles.size();
        a.stride = c.stride;
        a.counter = S->d_counters + (c.pow2 ? 1 : 0) * (CV_MAX_DIM + 1) + c.ndim;
        a.part_S = S->d_part_S;
        a.part_H = S->d_part_H;
        CV_CUDA(ctx, dispatch_batch_sample(c.ndim, c.pow2, a, std::min<int>(g, a.ntiles),
                                           S->side[used % kSideStreams]));
        ++used;
    }
    for (int k = 0; k < kSideStreams; ++k) {
        CV_CUDA(ctx, cudaEventRecord(S->ev_join[k], S->side[k]));
        CV_CUDA(ctx, cudaStreamWaitEvent(S->stream, S->ev_join[k], 0));
    }
    CV_CUDA(ctx, launch_batch_refine(S->d_items, S->d_axes, (int)axes.size(), S->stream, S->d_tparts, S->d_part_H));
    CV_CUDA(ctx, launch_batch_combine(S->d_cargs, nlive, S->stream, S->d_lists + nfresh, S->d_tparts,
                                      S->d_part_S));
    CV_CUDA(ctx, launch_gather_states(S->d_items, S->d_lists + nfresh, nlive, S->d_gather, S->stream));
    CV_CUDA(ctx, cudaMemcpyAsync(S->h_gather, S->d_gather, nlive * sizeof(DevState), cudaMemcpyDeviceToHost, S->stream));
    CV_CUDA(ctx, cudaEventRecord(S->ev_t1, S->stream));
    CV_CUDA(ctx, cudaStreamSynchronize(S->stream));
    const auto t1 = Clock::now();
    float gpu_ms = 0.0f;
    CV_CUDA(ctx, cudaEventElapsedTime(&gpu_ms, S->ev_t0, S->ev_t1));
    // ---- retire finished requests, advance the rest
    std::vector<Request> keep;
    keep.reserve(live.size());
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->busy_s += std::chrono::duration<double>(t1 - t0).count();
        S->gpu_s += 1e-3 * gpu_ms;
        ++S->rounds;
        S->samples += round_samples;
        for (int k = 0; k < nlive; ++k) {
            Request &r = live[k];
            const DevState &h = S->h_gather[k];
            if (h.stopped || r.j + 1 >= r.jmax) {
                cv_result res;
                memset(&res, 0, sizeof(res));
                res.neval = h.neval;
                res.fail = h.stopped ? h.fail : 1;
                res.iterations = h.iter;
                res.status = h.status;
                for (int c = 0; c < r.spec.g.ncomp; ++c) {
                    res.integral[c] = h.integral[c];
                    res.error[c] = h.error[c];
                    res.prob[c] = h.prob[c];
                    res.chi2[c] = h.chi2[c];
                }
                S->done[r.id] = res;
                S->latency_ms[r.id] = std::chrono::duration<double, std::milli>(t1 - r.arrival).count();
                ++S->completed;
                arena.release(r.off, r.bytes);
                free_slots.push_back(r.slot);
            } else {
                r.next_index += (unsigned long long)(r.spec.nstart + (long long)r.j * r.spec.nincrease);
                r.j += 1;
                keep.push_back(r);
            }
        }
    }
    live.swap(keep);
    S->cv_done.notify_all();
    return CV_OK;
}

void server_main(cv_server *S)
{
    cv_ctx *ctx = S->ctx;
    cudaSetDevice(ctx->device);
    Arena arena((size_t)S->opts.hbm_budget_bytes);
    std::vector<int> free_slots;
    for (int i = S->opts.max_live - 1; i >= 0; --i) free_slots.push_back(i);
    std::vector<Request> live;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (live.empty()) {
                S->cv_new.wait(lk, [&] { return S->stopping || !S->pending.empty(); });
                if (S->stopping && S->pending.empty()) break;
            }
        }
        int rc = server_round(S, live, arena, free_slots);
        if (rc) {
            std::lock_guard<std::mutex> lk(S->mu);
            S->error = rc;
            S->stopping = true;
            S->cv_done.notify_all();
            break;
        }
    }
}

}  // namespace

extern "C" int cv_server_start(cv_ctx *ctx, const cv_server_opts *opts, cv_server **out)
{
    if (!ctx || !out) return CV_EINVAL;
    *out = nullptr;
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    cv_server *S = new cv_server();
    S->ctx = ctx;
    memset(&S->opts, 0, sizeof(S->opts));
    if (opts) S->opts = *opts;
    if (S->opts.hbm_budget_bytes <= 0) S->opts.hbm_budget_bytes = (int64_t)1 << 30;
    if (S->opts.max_live <= 0) S->opts.max_live = 4096;
    const int L = S->opts.max_live;
    S->class_grid.assign(2 * (CV_MAX_DIM + 1) * (CV_MAX_BINS + 1), 0);
    cudaError_t e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&S->ev_t0);
    if (e == cudaSuccess) e = cudaEventCreate(&S->ev_t1);
    for (int k = 0; k < kSideStreams && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&S->side[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev_join[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaMalloc(&S->arena_mem, (size_t)S->opts.hbm_budget_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&S->d_items, (size_t)L * sizeof(BatchItem));
    if (e == cudaSuccess) e = cudaMalloc(&S->d_cargs, (size_t)L * sizeof(CombineArgs));
    if (e == cudaSuccess) e = cudaMalloc(&S->d_lists, (size_t)2 * L * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&S->d_axes, (size_t)L * CV_MAX_DIM * sizeof(int2));
    if (e == cudaSuccess) e = cudaMalloc(&S->d_counters, 2 * (CV_MAX_DIM + 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&S->d_gather, (size_t)L * sizeof(DevState));
    if (e == cudaSuccess) e = cudaMallocHost(&S->h_gather, (size_t)L * sizeof(DevState));
    if (e == cudaSuccess) e = cudaMalloc(&S->d_tparts, (size_t)L * sizeof(TileParts));
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(S->arena_mem);
        cudaFree(S->d_items);
        cudaFree(S->d_cargs);
        cudaFree(S->d_lists);
        cudaFree(S->d_axes);
        cudaFree(S->d_counters);
        cudaFree(S->d_gather);
        cudaFree(S->d_tparts);
        if (S->h_gather) cudaFreeHost(S->h_gather);
        if (S->stream) cudaStreamDestroy(S->stream);
        delete S;
        return fail_msg(ctx, CV_ENOMEM, "server allocation failed: %s", cudaGetErrorString(e));
    }
    S->h_tparts.assign((size_t)L, TileParts{0, 0, 0u, 0});
    S->slot_stride.assign((size_t)L, 0u);
    S->t_start = Clock::now();
    S->worker = std::thread(server_main, S);
    ctx->servers.insert(S);
    *out = S;
    return CV_OK;
}

extern "C" int cv_submit(cv_server *S, const cv_spec *spec, uint64_t *id)
{
    if (!S || !id) return CV_EINVAL;
    int rc = check_spec(S->ctx, spec);
    if (rc) return rc;
    if (spec->flags & (CV_FP64 | CV_PLAIN))
        return fail_msg(S->ctx, CV_EINVAL, "served requests use the FP32 path");
    if (spec->flags & CV_PSEUDO)
        return fail_msg(S->ctx, CV_EINVAL, "served requests take Sobol or scrambled Sobol points");
    if (batch_smem_bytes(spec->g.ndim, spec->nbins) > 223 * 1024)
        return fail_msg(S->ctx, CV_EINVAL, "%d dimensions x %d bins exceed the batched path's shared memory",
                        spec->g.ndim, spec->nbins);
    Request r;
    r.spec = *spec;
    r.bytes = request_bytes(*spec);
    if ((int64_t)r.bytes > S->opts.hbm_budget_bytes)
        return fail_msg(S->ctx, CV_EADMIT, "request needs %zu bytes, the budget is %lld", r.bytes,
                        (long long)S->opts.hbm_budget_bytes);
    r.arrival = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stopping) return fail_msg(S->ctx, CV_EBUSY, "server is stopping");
        if (S->error) return S->error;
        r.id = S->next_id++;
        *id = r.id;
        S->pending.push_back(r);
        ++S->submitted;
    }
    S->cv_new.notify_one();
    return CV_OK;
}

extern "C" int cv_poll(cv_server *S, uint64_t id, cv_result *out)
{
    if (!S || !out) return CV_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->done.find(id);
    if (it != S->done.end()) {
        *out = it->second;
        return CV_OK;
    }
    if (id == 0 || id >= S->next_id) return CV_ENOTFOUND;
    return S->error ? S->error : CV_EBUSY;
}

extern "C" int cv_wait(cv_server *S, uint64_t id, int timeout_ms, cv_result *out)
{
    if (!S || !out) return CV_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    if (id == 0 || id >= S->next_id) return CV_ENOTFOUND;
    const bool ok = S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                        [&] { return S->done.count(id) || S->error; });
    if (S->done.count(id)) {
        *out = S->done[id];
        return CV_OK;
    }
    if (S->error) return S->error;
    return ok ? CV_EBUSY : CV_ETIMEOUT;
}

extern "C" int cv_server_stats(cv_server *S, cv_serve_stats *out)
{
    if (!S || !out) return CV_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    memset(out, 0, sizeof(*out));
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->rounds = S->rounds;
    out->samples = S->samples;
    out->max_live = S->max_live_seen;
    out->pending = (int)S->pending.size();
    out->busy_s = S->busy_s;
    out->gpu_s = S->gpu_s;
    out->wall_s = std::chrono::duration<double>(Clock::now() - S->t_start).count();
    std::vector<double> lat;
    lat.reserve(S->latency_ms.size());
    for (auto &kv : S->latency_ms) lat.push_back(kv.second);
    if (!lat.empty()) {
        std::sort(lat.begin(), lat.end());
        auto q = [&](double p) { return lat[std::min(lat.size() - 1, (size_t)(p * (lat.size() - 1) + 0.5))]; };
        out->p50_ms = q(0.50);
        out->p99_ms = q(0.99);
        out->max_ms = lat.back();
    }
    return CV_OK;
}

static void server_release(cv_server *S)
{
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
    }
    S->cv_new.notify_all();
    if (S->worker.joinable()) S->worker.join();
    cudaSetDevice(S->ctx->device);
    cudaFree(S->arena_mem);
    cudaFree(S->d_items);
    cudaFree(S->d_cargs);
    cudaFree(S->d_lists);
    cudaFree(S->d_axes);
    cudaFree(S->d_counters);
    cudaFree(S->d_gather);
    if (S->d_tiles) cudaFree(S->d_tiles);
    cudaFree(S->d_tparts);
    if (S->d_part_S) cudaFree(S->d_part_S);
    if (S->d_part_H) cudaFree(S->d_part_H);
    if (S->h_gather) cudaFreeHost(S->h_gather);
    if (S->stream) cudaStreamDestroy(S->stream);
    for (int k = 0; k < kSideStreams; ++k) {
        if (S->side[k]) cudaStreamDestroy(S->side[k]);
        if (S->ev_join[k]) cudaEventDestroy(S->ev_join[k]);
    }
    if (S->ev_fork) cudaEventDestroy(S->ev_fork);
    if (S->ev_t0) cudaEventDestroy(S->ev_t0);
    if (S->ev_t1) cudaEventDestroy(S->ev_t1);
    delete S;
}

extern "C" int cv_server_stop(cv_server *S)
{
    if (!S) return CV_EINVAL;
    cv_ctx *ctx = S->ctx;
    if (!ctx->servers.erase(S)) return CV_EINVAL;
    const int err = S->error;
    server_release(S);
    return err;
}

// ------------------------------------------------------------ user integrands
namespace cv {
#define CV_EXTERN_M(D)                                                                          \
    extern template cudaError_t launch_matpass<D, float, 1>(const SampleArgs<float> &, int, cudaStream_t, int *);   \
    extern template cudaError_t launch_matpass<D, float, 2>(const SampleArgs<float> &, int, cudaStream_t, int *);   \
    extern template cudaError_t launch_matpass<D, double, 1>(const SampleArgs<double> &, int, cudaStream_t, int *); \
    extern template cudaError_t launch_matpass<D, double, 2>(const SampleArgs<double> &, int, cudaStream_t, int *);
CV_FOR_EACH_NDIM(CV_EXTERN_M)
#undef CV_EXTERN_M

// acc = false: store the points; acc = true: accumulate the caller's values.
// *grid_used: the launch's grid (the accumulate pass keeps to one wave of
// its own residency)
template <typename Real>
static cudaError_t dispatch_matpass(int ndim, bool acc, const SampleArgs<Real> &a, int grid, cudaStream_t s,
                                   int *grid_used)
{
    switch (ndim) {
#define CV_CASE(D)                                                                 \
    case D:                                                                        \
        return acc ? launch_matpass<D, Real, 2>(a, grid, s, grid_used)             \
                   : launch_matpass<D, Real, 1>(a, grid, s, grid_used);
        CV_FOR_EACH_NDIM(CV_CASE)
#undef CV_CASE
    }
    return cudaErrorInvalidValue;
}

template <typename Real>
static cudaError_t dispatch_genz_points(int ndim, bool aos, const GenzParams<Real> &g, const Real *x,
                                        Real *f, long long n, long long ld, int grid, cudaStream_t s)
{
    switch (ndim) {
#define CV_CASE(D)                                                                                  \
    case D: return aos ? launch_genz_points<D, Real, true>(g, x, f, n, ld, grid, s)               \
                       : launch_genz_points<D, Real, false>(g, x, f, n, ld, grid, s);
        CV_FOR_EACH_NDIM(CV_CASE)
#undef CV_CASE
    }
    return cudaErrorInvalidValue;
}
}  // namespace cv

extern "C" int cv_genz_callback(const int *ndim, const void *x_dev, const int *ncomp, void *f_dev,
                                void *userdata, const int64_t *nvec, const int64_t *ld, void *stream)
{
    const cv_genz_cb_data *u = (const cv_genz_cb_data *)userdata;
    if (!u || !ndim || !ncomp || !nvec || !ld || *ndim != u->g.ndim || *ncomp != u->g.ncomp) return -999;
    const long long n = *nvec;
    if (n <= 0) return 0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return -999;
    }
    long long grid = (n + kBlock - 1) / kBlock;
    if (grid > (long long)sms * 16) grid = (long long)sms * 16;
    const bool aos = (u->flags & CV_AOS) != 0;
    cudaError_t e;
    if ((u->flags & CV_JIT) && !(u->flags & CV_FP64) && !aos) {
        // families and parameters compiled in (NVRTC, cached per problem);
        // without NVRTC the generic kernel below runs
        GenzParams<float> g;
        fill_params<float>(&u->g, &g);
        JitKernel k;
        std::string err;
        if (jit_points_kernel(dev, g, *ndim, &k, &err) == 0) {
            const long long cap = (long long)sms * k.occ;
            e = launch_jit_points(k, g, (const float *)x_dev, (float *)f_dev, n, *ld,
                                  (int)(grid < cap ? grid : cap), (cudaStream_t)stream);
            return e == cudaSuccess ? 0 : -999;
        }
    }
    if (u->flags & CV_FP64) {
        GenzParams<double> g;
        fill_params<double>(&u->g, &g);
        e = dispatch_genz_points<double>(*ndim, aos, g, (const double *)x_dev, (double *)f_dev, n, *ld,
                                         (int)grid, (cudaStream_t)stream);
    } else {
        GenzParams<float> g;
        fill_params<float>(&u->g, &g);
        e = dispatch_genz_points<float>(*ndim, aos, g, (const float *)x_dev, (float *)f_dev, n, *ld,
                                        (int)grid, (cudaStream_t)stream);
    }
    return e == cudaSuccess ? 0 : -999;
}

template <typename Real>
static int vegas_cb_run(cv_ctx *ctx, int ndim, int ncomp, cv_integrand_dev cb, void *userdata,
                        long long nvec, const cv_spec &sp, cv_result *res)
{
    const bool aos = (sp.flags & CV_AOS) != 0;
    const int N = sp.nbins;
    int jmax = 0;
    long long nmax = 0;
    plan(sp.nstart, sp.nincrease, sp.maxeval, &jmax, &nmax);
    const long long tile = nvec < nmax ? nvec : nmax;
    // row stride of the dimension-major layout: a multiple of 32 values, so
    // that with 256-byte aligned arrays every aligned 32-point group of a
    // row is whole 128-byte lines
    const long long ldx = aos ? tile : (tile + 31) / 32 * 32;
    const bool fp32 = sizeof(Real) == 4;
    // device memory: state, grid, histogram, staged FP32 grid, x, f
    const size_t sz_state = (sizeof(DevState) + 255) & ~(size_t)255;
    const size_t sz_edges = (((size_t)ndim * (N + 1) * sizeof(double)) + 255) & ~(size_t)255;
    const size_t sz_H = (((size_t)ndim * N * sizeof(double)) + 255) & ~(size_t)255;
    const size_t sz_ew = fp32 ? (((size_t)ndim * N * sizeof(float2)) + 255) & ~(size_t)255 : 0;
    const size_t sz_x = (((size_t)ndim * ldx * sizeof(Real)) + 255) & ~(size_t)255;
    const size_t sz_f = (size_t)ncomp * ldx * sizeof(Real);
    const size_t need = sz_state + sz_edges + sz_H + sz_ew + sz_x + sz_f;
    if (!ctx->pinned) {
        if (cudaHostAlloc((void **)&ctx->pinned, 2 * sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            ctx->pinned = nullptr;
            return fail_msg(ctx, CV_ENOMEM, "pinned host allocation failed");
        }
    }
    if (need > ctx->mat_cap) {
        // the previous scratch may still be in use by work on the stream
        CV_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (ctx->mat_mem) cudaFree(ctx->mat_mem);
        ctx->mat_mem = nullptr;
        ctx->mat_cap = 0;
        if (cudaMalloc(&ctx->mat_mem, need) != cudaSuccess) {
            cudaGetLastError();
            ctx->mat_mem = nullptr;
            return fail_msg(ctx, CV_ENOMEM, "device allocation for %lld materialised points failed", tile);
        }
        ctx->mat_cap = need;
    }
    int *const pin = ctx->pinned;
    char *p = (char *)ctx->mat_mem;
    DevState *st = (DevState *)p;
    double *edges = (double *)(p + sz_state);
    double *H = (double *)(p + sz_state + sz_edges);
    float2 *ew32 = fp32 ? (float2 *)(p + sz_state + sz_edges + sz_H) : nullptr;
    Real *x = (Real *)(p + sz_state + sz_edges + sz_H + sz_ew);
    Real *f = (Real *)(p + sz_state + sz_edges + sz_H + sz_ew + sz_x);
    int rc = CV_OK;
    cudaStream_t s = ctx->stream;
    CombineArgs ca = {};
    memset(&ca, 0, sizeof(ca));
    ca.st = st;
    ca.ncomp = ncomp;
    ca.epsrel = sp.epsrel;
    ca.epsabs = sp.epsabs;
    ca.mineval = sp.mineval;
    ca.maxeval = sp.maxeval;
    ca.nstart = sp.nstart;
    ca.nincrease = sp.nincrease;
    SampleArgs<Real> a;
    memset(&a, 0, sizeof(a));
    a.g.ndim = ndim;
    a.g.ncomp = ncomp;
    a.nbins = N;
    a.chunk_min = 4;
    a.map = make_map(N, ndim, sizeof(Real) == 8);
    set_generator(&a, ndim, sp.flags, sp.seed);
    a.edges = edges;
    if constexpr (sizeof(Real) == 4) a.ew32 = ew32;  // (staged by reset and by each refinement)
    a.ld = ldx;
    a.aos = aos ? 1 : 0;
    a.x = x;
    a.f = f;
    a.S1 = st->S1;
    a.S2 = st->S2;
    a.H = H;
    int occ = 0;
    rc = occupancy(ctx, ndim, N, sizeof(Real) == 8, &occ);
    if (rc) return rc;
    pin[0] = 1;
    int aborted = 0;
    // (the dimension-major FP32 kernels for N = 2^L flag the refinement
    // themselves: their accumulate pass sets pass_active from the stop flag)
    const bool lean = fp32 && a.map.pow2 && !aos && a.gen != kGenPseudo && a.map.priv;
    if (lean) a.st = st;
    // the stop flag through host-mapped memory (no copy per iteration),
    // where the pinned buffer has a device address
    int *host_stop = nullptr;
    if (cudaHostGetDevicePointer((void **)&host_stop, &pin[1], 0) != cudaSuccess) {
        cudaGetLastError();
        host_stop = nullptr;
    }
    pin[1] = 0;
    ca.host_stop = host_stop;
    cudaEvent_t ev_stop = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev_stop, cudaEventDisableTiming);
    if (e == cudaSuccess) e = launch_reset(st, edges, H, ndim, N, sp.nstart, ew32, a.map, s);
    // Per iteration: for each tile the store pass, the integrand, the
    // accumulate pass; then refinement and combination, and the device's
    // stop flag copied back.  The next iteration's first store pass is
    // enqueued before the host waits for that flag, so the GPU writes the
    // next points while the host decides whether to call the integrand
    // again (if the run stopped, those points are never used).
    unsigned long long start = 1;
    // The accumulate passes' sums and histograms go through per-block
    // partials, added in a fixed order: an iteration of one tile hands them
    // to the refinement and combination (as a fused pass does); with more
    // tiles each pass adds its own (its last block the sums, then the
    // histogram rows) before the next.
    PassParts pp;
    if (e == cudaSuccess) {
        const int rc_p = ctx_parts(ctx, sample_grid(ctx, occ, tile), &pp);
        if (rc_p) {
            cudaEventDestroy(ev_stop);
            return rc_p;
        }
    }
    const int nh = ndim * N;
    int grid_used = 0;
    auto store = [&](unsigned long long s0, long long m) {
        SampleArgs<Real> b = a;
        b.start = s0;
        b.n = m;
        // (the same grid as a fused pass: the kernels share its occupancy)
        return dispatch_matpass<Real>(ndim, false, b, sample_grid(ctx, occ, m), s, &grid_used);
    };
    if (e == cudaSuccess && jmax > 0) e = store(start, sp.nstart < tile ? sp.nstart : tile);
    double *pp_S = nullptr;
    void *pp_H = nullptr;
    unsigned *pp_ticket = nullptr;
    if (e == cudaSuccess) parts_args(&pp, 0, &pp_S, &pp_H, &pp_ticket);
    for (int j = 0; j < jmax && e == cudaSuccess && !aborted; ++j) {
        const long long nj = sp.nstart + (long long)j * sp.nincrease;
        const bool one_tile = nj <= tile;
        for (long long off = 0; off < nj && e == cudaSuccess; off += tile) {
            const long long m = nj - off < tile ? nj - off : tile;
            if (off > 0) e = store(start + (unsigned long long)off, m);
            if (e != cudaSuccess) break;
            const int64_t nv = m, ld = ldx;
            const int r = cb(&ndim, x, &ncomp, f, userdata, &nv, &ld, (void *)s);
            if (r == -999) {
                aborted = 1;
                break;
            }
            SampleArgs<Real> b = a;
            b.start = start + (unsigned long long)off;
            b.n = m;
            parts_args(&pp, 0, &b.part_S, &b.part_H, &b.part_ticket);
            b.part_G = pp.G_cap;
            if (one_tile) b.part_ticket = nullptr;  // (the combination adds the sums)
            e = dispatch_matpass<Real>(ndim, true, b, sample_grid(ctx, occ, m), s, &grid_used);
            if (e == cudaSuccess && !one_tile)
                e = launch_add_parts(b.part_H, grid_used, fp32 ? 1 : 0, nh, H, s);
        }
        if (aborted || e != cudaSuccess) break;
        if (one_tile) {
            ca.part_S = reinterpret_cast<const double *>(pp_S);
            ca.part_H = pp_H;
            ca.part_G = grid_used;
            ca.part_nh = nh;
            ca.part_f32 = fp32 ? 1 : 0;
        } else {
            ca.part_S = nullptr;
            ca.part_H = nullptr;
            ca.part_G = 0;
        }
        if (!lean) e = cudaMemcpyAsync(&st->pass_active, &pin[0], sizeof(int), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = launch_refine_combine(ndim, N, H, edges, ca, ew32, a.map, s);
        if (e == cudaSuccess && !host_stop)
            e = cudaMemcpyAsync(&pin[1], &st->stopped, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaEventRecord(ev_stop, s);
        start += (unsigned long long)nj;
        if (e == cudaSuccess && j + 1 < jmax) {
            const long long nn = nj + sp.nincrease;
            e = store(start, nn < tile ? nn : tile);
        }
        if (e == cudaSuccess) e = cudaEventSynchronize(ev_stop);
        if (pin[1]) break;
    }
    if (ev_stop) cudaEventDestroy(ev_stop);
    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "materialised pass");
    DevState h;
    memset(&h, 0, sizeof(h));
    if (!rc) {
        e = cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "result copy");
    }
    cudaStreamSynchronize(s);
    if (rc) return rc;
    memset(res, 0, sizeof(*res));
    res->neval = h.neval;
    res->iterations = h.iter;
    res->status = h.status;
    res->fail = aborted ? -999 : (h.stopped ? h.fail : 1);
    for (int c = 0; c < ncomp; ++c) {
        res->integral[c] = h.integral[c];
        res->error[c] = h.error[c];
        res->prob[c] = h.prob[c];
    }
    if (aborted) return fail_msg(ctx, CV_EABORT, "the integrand returned -999");
    return CV_OK;
}

extern "C" int cv_vegas_cb(cv_ctx *ctx, int ndim, int ncomp, cv_integrand_dev integrand,
                           void *userdata, int64_t nvec, double epsrel, double epsabs, int flags,
                           int seed, int64_t mineval, int64_t maxeval, int64_t nstart,
                           int64_t nincrease, int64_t nbatch, int nbins, int64_t *neval, int *fail,
                           double integral[], double error[], double prob[])
{
    (void)nbatch;
    if (!ctx) return CV_EINVAL;
    if (!integrand) return fail_msg(ctx, CV_EINVAL, "null integrand");
    if (flags & CV_PSEUDO)
        return fail_msg(ctx, CV_EINVAL, "materialised samples take Sobol or scrambled Sobol points");
    if (ndim < 1 || ndim > CV_MAX_DIM || ncomp < 1 || ncomp > CV_MAX_COMP)
        return fail_msg(ctx, CV_EINVAL, "ndim/ncomp out of range");
    if (nvec < 1) return fail_msg(ctx, CV_EINVAL, "nvec must be >= 1");
    cv_spec sp;
    memset(&sp, 0, sizeof(sp));
    sp.g.ndim = ndim;
    sp.g.ncomp = ncomp;
    sp.nbins = nbins;
    sp.flags = flags;
    sp.epsrel = epsrel;
    sp.epsabs = epsabs;
    sp.mineval = mineval;
    sp.maxeval = maxeval;
    sp.nstart = nstart;
    sp.nincrease = nincrease;
    sp.seed = (uint64_t)(int64_t)seed;
    int rc = check_spec(ctx, &sp);
    if (rc) return rc;
    if (!neval || !fail || !integral || !error || !prob) return fail_msg(ctx, CV_EINVAL, "null output");
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    cv_result res;
    rc = (flags & CV_FP64) ? vegas_cb_run<double>(ctx, ndim, ncomp, integrand, userdata, nvec, sp, &res)
                           : vegas_cb_run<float>(ctx, ndim, ncomp, integrand, userdata, nvec, sp, &res);
    if (rc && rc != CV_EABORT) return rc;
    *neval = res.neval;
    *fail = res.fail;
    for (int c = 0; c < ncomp; ++c) {
        integral[c] = res.integral[c];
        error[c] = res.error[c];
        prob[c] = res.prob[c];
    }
    if (!rc && (res.status & 1))
        return fail_msg(ctx, CV_ENONFINITE, "iteration %d gave a non-finite result", res.iterations);
    return rc;
}

// ------------------------------------------------------------ Suave
// Subregion-adaptive Vegas as declared in cubagpu.h: the host takes every
// decision from FP64 values read back from the device; the device samples
// and refines the regions of a pass together (each region has its own grid,
// histogram and sums).  In FP32 with Sobol or scrambled points a pass is one
// launch of the batched sampling kernel over a queue of tiles of all its
// regions (regions are batch items), one batched refinement and two small
// kernels that stage the regions in and their results out through mapped
// pinned memory; otherwise every region is one sampling launch (FP64 and
// pseudo-random points), spread over the side streams.
namespace {

struct SuaveRegion {
    double I[CV_MAX_COMP], var[CV_MAX_COMP];
    double fluct[CV_MAX_DIM];
};

// One region of a batched pass: its Sobol indices start at `start`; its
// grid is taken from the host mirror first if `upload`.
struct SuaveEntry {
    int region;
    int upload;
    unsigned long long start;
};

struct SuaveMem {
    double *edges = nullptr;  // [max_regions][ndim][N+1]
    double *H = nullptr;      // [max_regions][ndim][N]
    double *S = nullptr;      // [max_regions][2][CV_MAX_COMP]: S1 then S2
    double *h_edges = nullptr;  // pinned host mirrors of edges, S and (batched) fluct
    double *h_S = nullptr;
    double *h_fluct = nullptr;  // [max_regions][CV_MAX_DIM]
    // batched form
    bool batched = false;
    bool pow2 = false;
    int grid = 0;               // persistent sampling grid
    int tile_cap = 0;           // tiles one pass may queue
    BatchItem *d_items = nullptr;  // [max_regions]: region k is item k
    int *d_counter = nullptr;
    char *d_stage = nullptr, *h_stage = nullptr;  // entries, tiles, axes of a pass
    double *dh_edges = nullptr, *dh_S = nullptr, *dh_fluct = nullptr;  // device addresses of the mirrors
};

__global__ void k_suave_prep(const SuaveEntry *E, const BatchItem *items, const double *dh_edges, int ndim,
                             int N, long long nnew, int *counter)
{
    const SuaveEntry e = E[blockIdx.x];
    const BatchItem &it = items[e.region];
    const int ge = ndim * (N + 1);
    if (e.upload)
        for (int i = threadIdx.x; i < ge; i += blockDim.x) it.edges[i] = dh_edges[(size_t)ge * e.region + i];
    for (int i = threadIdx.x; i < ndim * N; i += blockDim.x) it.H[i] = 0.0;
    if (threadIdx.x < CV_MAX_COMP) {
        it.st->S1[threadIdx.x] = 0.0;
        it.st->S2[threadIdx.x] = 0.0;
    }
    if (threadIdx.x == 0) {
        it.st->next_index = e.start;
        it.st->n_cur = nnew;
        it.st->stopped = 0;
        if (blockIdx.x == 0) *counter = 0;
    }
}

// The listed regions' sums, and after a refinement their grids and the
// fluctuation of each axis, (mean_k |ln(w_k / mean w)|^flatness)^(1/flatness)
// (one warp per axis), into the host mirrors.
__global__ void k_suave_gather(const SuaveEntry *E, const BatchItem *items, double *dh_S, double *dh_edges,
                               double *dh_fluct, int ndim, int N, int refined, double flatness)
{
    const int r = E[blockIdx.x].region;
    const BatchItem &it = items[r];
    const int ge = ndim * (N + 1);
    if (threadIdx.x < CV_MAX_COMP) {
        dh_S[(size_t)2 * CV_MAX_COMP * r + threadIdx.x] = it.st->S1[threadIdx.x];
        dh_S[(size_t)2 * CV_MAX_COMP * r + CV_MAX_COMP + threadIdx.x] = it.st->S2[threadIdx.x];
    }
    if (!refined) return;
    for (int i = threadIdx.x; i < ge; i += blockDim.x) dh_edges[(size_t)ge * r + i] = it.edges[i];
    const int lane = threadIdx.x & 31;
    for (int d = threadIdx.x >> 5; d < ndim; d += blockDim.x >> 5) {
        const double *e = it.edges + (size_t)d * (N + 1);
        const double mean = (e[N] - e[0]) / N;
        double acc = 0.0;
        for (int k = lane; k < N; k += 32) acc += pow(fabs(log((e[k + 1] - e[k]) / mean)), flatness);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) dh_fluct[(size_t)CV_MAX_DIM * r + d] = pow(acc / N, 1.0 / flatness);
    }
}

// The estimates of the listed regions from their sums in the host mirror,
// and (refined grids) the fluctuation of each axis of their grids.
void suave_read(const cv_genz *g, int N, long long nnew, const std::vector<int> &list, bool refined,
                double flatness, const SuaveMem &m, std::vector<SuaveRegion> &R)
{
    const int ndim = g->ndim, nc = g->ncomp;
    const size_t ge = (size_t)ndim * (N + 1), gs = 2 * CV_MAX_COMP;
    for (size_t i = 0; i < list.size(); ++i) {
        SuaveRegion &q = R[list[i]];
        const double dn = (double)nnew;
        const double *S = m.h_S + gs * list[i];
        for (int c = 0; c < nc; ++c) {
            q.I[c] = S[c] / dn;
            q.var[c] = (S[CV_MAX_COMP + c] / dn - q.I[c] * q.I[c]) / (dn - 1.0);
            if (!(q.var[c] > 0.0)) q.var[c] = 0.0;
        }
        if (refined && m.batched) {
            for (int d = 0; d < ndim; ++d) q.fluct[d] = m.h_fluct[(size_t)CV_MAX_DIM * list[i] + d];
        } else if (refined) {
            for (int d = 0; d < ndim; ++d) {
                const double *e = &m.h_edges[ge * list[i] + (size_t)d * (N + 1)];
                const double mean = (e[N] - e[0]) / N;
                double acc = 0.0;
                for (int k = 0; k < N; ++k) acc += pow(fabs(log((e[k + 1] - e[k]) / mean)), flatness);
                q.fluct[d] = pow(acc / N, 1.0 / flatness);
            }
        }
    }
}

static size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// A batched pass: the listed regions' tiles in one queue.  Tiles are powers
// of two of 32-point blocks, at least 64, large enough to keep the queue
// within tile_cap and no larger than needed for four tiles per resident CTA.
int suave_pass_batched(cv_ctx *ctx, const cv_genz *g, int N, long long nnew, const std::vector<int> &list,
                       unsigned long long start, bool refine, bool upload, double flatness, const SuaveMem &m,
                       std::vector<SuaveRegion> &R)
{
    const int ndim = g->ndim;
    const long long nl = (long long)list.size();
    const long long span = (nnew + 31) / 32 + 2;  // 32-point blocks of one region, with the even alignment
    long long TB = 64;
    while (TB < 1024 && nl * ((span + TB - 1) / TB) > 4LL * m.grid) TB <<= 1;
    while (nl * ((span + TB - 1) / TB + 1) > m.tile_cap) TB <<= 1;
    SuaveEntry *E = reinterpret_cast<SuaveEntry *>(m.h_stage);
    const size_t off_t = align16((size_t)nl * sizeof(SuaveEntry));
    Tile *T = reinterpret_cast<Tile *>(m.h_stage + off_t);
    int nt = 0;
    for (long long i = 0; i < nl; ++i) {
        const unsigned long long s = start + (unsigned long long)i * (unsigned long long)nnew;
        E[i].region = list[(size_t)i];
        E[i].upload = upload ? 1 : 0;
        E[i].start = s;
        // (tiles start on even 32-point blocks: see run_steps)
        const unsigned long long qa = (s >> 5) & ~1ull, qb = (s + (unsigned long long)nnew + 31) >> 5;
        for (unsigned long long q = qa; q < qb; q += (unsigned long long)TB) {
            T[nt].item = list[(size_t)i];
            T[nt].nblk = (int)(qb - q < (unsigned long long)TB ? qb - q : (unsigned long long)TB);
            T[nt].q0 = q;
            ++nt;
        }
    }
    const size_t off_a = off_t + align16((size_t)nt * sizeof(Tile));
    int2 *A = reinterpret_cast<int2 *>(m.h_stage + off_a);
    const int naxes = refine ? (int)nl * ndim : 0;
    for (int i = 0; i < naxes; ++i) A[i] = make_int2(list[(size_t)(i / ndim)], i % ndim);
    const size_t bytes = off_a + (size_t)naxes * sizeof(int2);
    const cudaStream_t s = ctx->stream;
    CV_CUDA(ctx, cudaMemcpyAsync(m.d_stage, m.h_stage, bytes, cudaMemcpyHostToDevice, s));
    const SuaveEntry *dE = reinterpret_cast<const SuaveEntry *>(m.d_stage);
    k_suave_prep<<<(unsigned)nl, 256, 0, s>>>(dE, m.d_items, m.dh_edges, ndim, N, nnew, m.d_counter);
    CV_CUDA(ctx, cudaGetLastError());
    BatchSampleArgs a;
    a.items = m.d_items;
    a.tiles = reinterpret_cast<const Tile *>(m.d_stage + off_t);
    a.ntiles = nt;
    a.stride = N;
    a.counter = m.d_counter;
    a.part_S = nullptr;  // (FP64 atomics: the regions' sums are read from their states)
    a.part_H = nullptr;
    CV_CUDA(ctx, dispatch_batch_sample(ndim, m.pow2, a, m.grid < nt ? m.grid : nt, s));
    if (refine)
        CV_CUDA(ctx, launch_batch_refine(m.d_items, reinterpret_cast<const int2 *>(m.d_stage + off_a), naxes, s));
    k_suave_gather<<<(unsigned)nl, 256, 0, s>>>(dE, m.d_items, m.dh_S, m.dh_edges, m.dh_fluct, ndim, N,
                                                 refine ? 1 : 0, flatness);
    CV_CUDA(ctx, cudaGetLastError());
    CV_CUDA(ctx, cudaStreamSynchronize(s));
    suave_read(g, N, nnew, list, refine, flatness, m, R);
    return CV_OK;
}

// Sample the regions of `list` (region list[i] with the nnew Sobol indices
// from start + i nnew), refine their grids if `refine`, and read back their
// estimates (and refined grids, with their fluctuation per axis).
template <typename Real>
int suave_pass(cv_ctx *ctx, const cv_genz *g, int N, int flags, uint64_t seed, long long nnew,
               const std::vector<int> &list, unsigned long long start, bool refine, bool upload, double flatness,
               const SuaveMem &m, std::vector<SuaveRegion> &R)
{
    if (m.batched) return suave_pass_batched(ctx, g, N, nnew, list, start, refine, upload, flatness, m, R);
    double *const h_edges = m.h_edges;
    const int ndim = g->ndim;
    const size_t ge = (size_t)ndim * (N + 1), gh = (size_t)ndim * N, gs = 2 * CV_MAX_COMP;
    const cudaStream_t main = ctx->stream;
    for (int r : list) {
        if (upload)
            CV_CUDA(ctx, cudaMemcpyAsync(m.edges + ge * r, h_edges + ge * r, ge * sizeof(double),
                                         cudaMemcpyHostToDevice, main));
        CV_CUDA(ctx, cudaMemsetAsync(m.H + gh * r, 0, gh * sizeof(double), main));
        CV_CUDA(ctx, cudaMemsetAsync(m.S + gs * r, 0, gs * sizeof(double), main));
    }
    CV_CUDA(ctx, cudaEventRecord(ctx->ev_fork, main));
    for (int k = 0; k < kSideStreams; ++k) CV_CUDA(ctx, cudaStreamWaitEvent(ctx->side[k], ctx->ev_fork, 0));
    int rc = CV_OK;
    for (size_t i = 0; i < list.size() && rc == CV_OK; ++i) {
        const int r = list[i];
        ctx->stream = ctx->side[i % kSideStreams];
        rc = launch_pass<Real>(ctx, g, N, m.edges + ge * r, start + (unsigned long long)i * nnew, nnew, nnew,
                               m.S + gs * r, m.S + gs * r + CV_MAX_COMP, m.H + gh * r, nullptr, flags, seed);
        if (rc == CV_OK && refine) {
            cudaError_t e = launch_refine(ndim, N, m.H + gh * r, m.edges + ge * r, ctx->stream);
            if (e != cudaSuccess) rc = cuda_fail(ctx, e, "refine kernel launch");
        }
    }
    ctx->stream = main;
    for (int k = 0; k < kSideStreams; ++k) {
        CV_CUDA(ctx, cudaEventRecord(ctx->ev_join[k], ctx->side[k]));
        CV_CUDA(ctx, cudaStreamWaitEvent(main, ctx->ev_join[k], 0));
    }
    if (rc) return rc;
    // (pinned mirrors: the copies queue without host round trips)
    for (size_t i = 0; i < list.size(); ++i) {
        CV_CUDA(ctx, cudaMemcpyAsync(m.h_S + gs * list[i], m.S + gs * list[i], gs * sizeof(double),
                                     cudaMemcpyDeviceToHost, main));
        if (refine)
            CV_CUDA(ctx, cudaMemcpyAsync(&h_edges[ge * list[i]], m.edges + ge * list[i], ge * sizeof(double),
                                         cudaMemcpyDeviceToHost, main));
    }
    CV_CUDA(ctx, cudaStreamSynchronize(main));
    suave_read(g, N, nnew, list, refine, flatness, m, R);
    return CV_OK;
}

// The children of a split of grid pe along axis a at edge N/2.
void suave_children(int ndim, int N, int a, const double *pe, double *le, double *re)
{
    for (int d = 0; d < ndim; ++d) {
        const double *e = pe + (size_t)d * (N + 1);
        double *l = le + (size_t)d * (N + 1), *r = re + (size_t)d * (N + 1);
        if (d != a) {
            memcpy(l, e, sizeof(double) * (N + 1));
            memcpy(r, e, sizeof(double) * (N + 1));
            continue;
        }
        for (int j = 0; j < N / 2; ++j) {
            l[2 * j] = e[j];
            l[2 * j + 1] = 0.5 * (e[j] + e[j + 1]);
            r[2 * j] = e[N / 2 + j];
            r[2 * j + 1] = 0.5 * (e[N / 2 + j] + e[N / 2 + j + 1]);
        }
        l[N] = e[N / 2];
        r[N] = e[N];
    }
}

template <typename Real>
int suave_run(cv_ctx *ctx, const cv_genz *g, int N, int flags, uint64_t seed, double epsrel, double epsabs,
              long long mineval, long long maxeval, long long nnew, double flatness, int width, int max_regions,
              const SuaveMem &m, int *nregions, int64_t *neval, int *fail, double *integral, double *error,
              double *boxes)
{
    const int ndim = g->ndim, nc = g->ncomp;
    const size_t ge = (size_t)ndim * (N + 1);
    double *const h_edges = m.h_edges;
    std::vector<SuaveRegion> R((size_t)max_regions);
    for (int d = 0; d < ndim; ++d)
        for (int k = 0; k <= N; ++k) h_edges[(size_t)d * (N + 1) + k] = (double)k / (double)N;
    unsigned long long next = 1;
    int nr = 1;
    int rc = suave_pass<Real>(ctx, g, N, flags, seed, nnew, {0}, next, true, true, flatness, m, R);
    if (rc) return rc;
    next += (unsigned long long)nnew;
    long long done = nnew;
    std::vector<int> order;
    for (;;) {
        bool ok = done >= mineval;
        for (int c = 0; c < nc; ++c) {
            double I = 0.0, v = 0.0;
            for (int k = 0; k < nr; ++k) {
                I += R[k].I[c];
                v += R[k].var[c];
            }
            if (!(sqrt(v) <= std::max(epsabs, epsrel * fabs(I)))) ok = false;
        }
        if (ok) break;
        order.clear();
        for (int k = 0; k < nr; ++k)
            if (R[k].var[0] > 0.0) order.push_back(k);
        long long K = std::min<long long>((long long)order.size(), width);
        // the K largest var[0], ties in region order (as a stable sort would)
        std::partial_sort(order.begin(), order.begin() + K, order.end(), [&](int x, int y) {
            return R[x].var[0] > R[y].var[0] || (R[x].var[0] == R[y].var[0] && x < y);
        });
        if (K == 0) break;
        const long long room = maxeval - done - (long long)nr * nnew;
        K = std::min(K, room / (3 * nnew));
        K = std::min<long long>(K, max_regions - nr);
        if (K <= 0) break;
        std::vector<int> list;
        std::vector<double> child((size_t)ge);
        for (long long i = 0; i < K; ++i) {
            const int k = order[(size_t)i];
            int a = 0;
            for (int d = 1; d < ndim; ++d)
                if (R[k].fluct[d] > R[k].fluct[a]) a = d;
            double *pe = &h_edges[ge * k];
            double *re = &h_edges[ge * nr];
            suave_children(ndim, N, a, pe, child.data(), re);
            memcpy(pe, child.data(), sizeof(double) * ge);
            list.push_back(k);
            list.push_back(nr);
            ++nr;
        }
        rc = suave_pass<Real>(ctx, g, N, flags, seed, nnew, list, next, true, true, flatness, m, R);
        if (rc) return rc;
        next += (unsigned long long)list.size() * nnew;
        done += (long long)list.size() * nnew;
    }
    // the final pass: every region sampled afresh, its grid kept
    if (done + (long long)nr * nnew <= maxeval || nr == 1) {
        std::vector<int> all((size_t)nr);
        for (int k = 0; k < nr; ++k) all[(size_t)k] = k;
        rc = suave_pass<Real>(ctx, g, N, flags, seed, nnew, all, next, false, false, flatness, m, R);
        if (rc) return rc;
        done += (long long)nr * nnew;
    }
    int status = 0;
    for (int c = 0; c < nc; ++c) {
        double I = 0.0, v = 0.0;
        for (int k = 0; k < nr; ++k) {
            I += R[k].I[c];
            v += R[k].var[c];
        }
        integral[c] = I;
        error[c] = sqrt(v);
        if (!(error[c] <= std::max(epsabs, epsrel * fabs(I)))) status = 1;
    }
    if (done < mineval) status = 1;
    *nregions = nr;
    *neval = done;
    *fail = status;
    if (boxes)
        for (int k = 0; k < nr; ++k)
            for (int d = 0; d < ndim; ++d) {
                boxes[((size_t)k * ndim + d) * 2] = h_edges[ge * k + (size_t)d * (N + 1)];
                boxes[((size_t)k * ndim + d) * 2 + 1] = h_edges[ge * k + (size_t)d * (N + 1) + N];
            }
    return CV_OK;
}

// The batched form's descriptors (one batch item per region, states, tile
// queue and staging), when the pass can take it: FP32, Sobol or scrambled
// points, a region's pass within the tiles' int range and a grid that fits
// the batched kernel's shared memory.  Otherwise m stays per-region.
int suave_batched_setup(cv_ctx *ctx, const cv_genz *g, int N, int flags, uint64_t seed, long long nnew,
                        int max_regions, SuaveMem &m, void **bmem, void **hstage)
{
    const int ndim = g->ndim;
    if ((flags & (CV_FP64 | CV_PSEUDO)) || nnew > (1LL << 31)) return CV_OK;
    const bool pow2 = make_map(N, ndim, false).pow2 != 0;  // (powers of two from 32 bins)
    int occ = 0;
    if (dispatch_batch_occupancy(ndim, pow2, N, &occ) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        return CV_OK;
    }
    const int tile_cap = std::max(1 << 16, 4 * max_regions);
    const size_t sz_items = align16((size_t)max_regions * sizeof(BatchItem));
    const size_t sz_state = align16((size_t)max_regions * sizeof(DevState));
    const size_t sz_stage = align16((size_t)max_regions * sizeof(SuaveEntry)) + (size_t)tile_cap * sizeof(Tile) +
                            (size_t)max_regions * ndim * sizeof(int2) + 64;
    char *d = nullptr;
    if (cudaMalloc((void **)&d, sz_items + sz_state + sz_stage + 16) != cudaSuccess) {
        cudaGetLastError();
        return fail_msg(ctx, CV_ENOMEM, "device allocation of the batched regions failed");
    }
    *bmem = d;
    if (cudaMallocHost(hstage, sz_stage) != cudaSuccess) {
        cudaGetLastError();
        *hstage = nullptr;
        return fail_msg(ctx, CV_ENOMEM, "pinned staging allocation failed");
    }
    // (the mirrors are one mapped pinned allocation starting at h_edges)
    CV_CUDA(ctx, cudaHostGetDevicePointer((void **)&m.dh_edges, m.h_edges, 0));
    m.dh_S = m.dh_edges + (m.h_S - m.h_edges);
    m.dh_fluct = m.dh_edges + (m.h_fluct - m.h_edges);
    m.d_items = reinterpret_cast<BatchItem *>(d);
    DevState *st = reinterpret_cast<DevState *>(d + sz_items);
    m.d_stage = d + sz_items + sz_state;
    m.d_counter = reinterpret_cast<int *>(m.d_stage + sz_stage);
    m.h_stage = static_cast<char *>(*hstage);
    m.tile_cap = tile_cap;
    m.grid = ctx->sms * occ;
    m.pow2 = pow2;
    const size_t ge = (size_t)ndim * (N + 1), gh = (size_t)ndim * N;
    std::vector<BatchItem> items((size_t)max_regions);
    BatchItem proto;
    memset(&proto, 0, sizeof(proto));
    fill_params<float>(g, &proto.a.g);
    proto.a.nbins = N;
    proto.a.chunk_min = 4;
    proto.a.map = make_map(N, ndim, false);
    proto.a.map.priv = proto.a.map.pow2;  // every warp has its own histogram
    set_generator(&proto.a, ndim, flags, seed);
    for (int k = 0; k < max_regions; ++k) {
        items[(size_t)k] = proto;
        items[(size_t)k].st = st + k;
        items[(size_t)k].edges = m.edges + ge * k;
        items[(size_t)k].H = m.H + gh * k;
    }
    CV_CUDA(ctx, cudaMemsetAsync(st, 0, sz_state, ctx->stream));
    CV_CUDA(ctx, cudaMemcpyAsync(m.d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice,
                                 ctx->stream));
    CV_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    m.batched = true;
    return CV_OK;
}

}  // namespace

extern "C" int cv_suave(cv_ctx *ctx, const cv_genz *g, int nbins, int flags, uint64_t seed, double epsrel,
                        double epsabs, int64_t mineval, int64_t maxeval, int64_t nnew, double flatness, int width,
                        int max_regions, int *nregions, int64_t *neval, int *fail, double integral[],
                        double error[], double *boxes)
{
    if (!ctx) return CV_EINVAL;
    int rc = check_genz(ctx, g);
    if (rc) return rc;
    if (nbins < CV_MIN_BINS || nbins > CV_MAX_BINS || (nbins & 1))
        return fail_msg(ctx, CV_EINVAL, "nbins must be even, %d..%d", CV_MIN_BINS, CV_MAX_BINS);
    if (nnew < 2 || maxeval < nnew || mineval < 0 || width < 1 || max_regions < 1 || !(flatness > 0.0) ||
        !(epsrel >= 0) || !(epsabs >= 0))
        return fail_msg(ctx, CV_EINVAL, "need nnew >= 2, maxeval >= nnew, width, max_regions >= 1, flatness > 0");
    if ((uint64_t)maxeval >= CV_INDEX_LIMIT) return fail_msg(ctx, CV_EINVAL, "maxeval beyond the 2^52 index range");
    if ((flags & CV_SCRAMBLE) && (flags & CV_PSEUDO))
        return fail_msg(ctx, CV_EINVAL, "CV_SCRAMBLE and CV_PSEUDO exclude each other");
    if (!nregions || !neval || !fail || !integral || !error) return fail_msg(ctx, CV_EINVAL, "null output");
    if (!(flags & CV_FP64) && (rc = check_fp32_range(ctx, g))) return rc;
    CV_CUDA(ctx, cudaSetDevice(ctx->device));
    const int ndim = g->ndim;
    const size_t ge = (size_t)ndim * (nbins + 1), gh = (size_t)ndim * nbins, gs = 2 * CV_MAX_COMP;
    SuaveMem m;
    const size_t bytes = sizeof(double) * (ge + gh + gs) * (size_t)max_regions;
    void *mem = nullptr;
    if (cudaMalloc(&mem, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail_msg(ctx, CV_ENOMEM, "device allocation for %d regions failed", max_regions);
    }
    m.edges = (double *)mem;
    m.H = m.edges + ge * (size_t)max_regions;
    m.S = m.H + gh * (size_t)max_regions;
    void *hmem = nullptr;
    if (cudaMallocHost(&hmem, sizeof(double) * (ge + gs + CV_MAX_DIM) * (size_t)max_regions) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(mem);
        return fail_msg(ctx, CV_ENOMEM, "pinned host allocation for %d regions failed", max_regions);
    }
    m.h_edges = (double *)hmem;
    m.h_S = m.h_edges + ge * (size_t)max_regions;
    m.h_fluct = m.h_S + gs * (size_t)max_regions;
    void *bmem = nullptr, *hstage = nullptr;
    rc = suave_batched_setup(ctx, g, nbins, flags, seed, nnew, max_regions, m, &bmem, &hstage);
    if (rc == CV_OK) rc = (flags & CV_FP64)
        ? suave_run<double>(ctx, g, nbins, flags, seed, epsrel, epsabs, mineval, maxeval, nnew, flatness, width,
                            max_regions, m, nregions, neval, fail, integral, error, boxes)
        : suave_run<float>(ctx, g, nbins, flags, seed, epsrel, epsabs, mineval, maxeval, nnew, flatness, width,
                           max_regions, m, nregions, neval, fail, integral, error, boxes);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(mem);
    cudaFreeHost(hmem);
    if (bmem) cudaFree(bmem);
    if (hstage) cudaFreeHost(hstage);
    return rc;
}
