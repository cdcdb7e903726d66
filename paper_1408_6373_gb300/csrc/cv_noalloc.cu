// cv_noalloc.cu -- cv_vegas_noalloc: the Vegas call for callers that cannot
// allocate device memory.
//
// Some callers of this library run where a cudaMalloc is not available or
// not allowed: code inside a process whose allocator is owned by another
// framework, a region that must not touch the device heap (for example
// while another component holds every byte of a memory pool), or a caller
// that only ever receives a device and a stream.  For them this file keeps
// the scratch memory of one Vegas run -- the device state, the grid and
// the histogram -- in one file-scope static device array, so the call
// allocates nothing: it launches the same sampling, refinement and
// combination kernels as cv_vegas, on pointers into that array.
//
// Limits and sharing: the array holds CV_STATIC_SCRATCH_BYTES per GPU and
// lives until the process exits.  Every call on a device uses the same
// array and overwrites what the previous call left there (each run starts
// by clearing its state and histogram and writing a uniform grid), so
// calls whose GPU work overlaps -- on two streams, or from two host
// threads -- race and give wrong results; serialise them.
//
// The caller's thread state is left as it was: the call makes `device`
// current only for its own work and restores the previous current device
// on every return, and it refuses a stream that belongs to another device.
#include <cmath>
#include <cstring>
#include <mutex>

#include "cv_internal.cuh"

namespace {

// One Vegas run's scratch: DevState, edges[ndim][nbins+1], hist[ndim][nbins].
static __device__ __align__(256) unsigned char g_scratch[CV_STATIC_SCRATCH_BYTES];

constexpr size_t kStateBytes = (sizeof(cv::DevState) + 255) & ~(size_t)255;
static_assert(kStateBytes == 512, "the size rule documented in cubagpu.h counts 512 bytes of state");
constexpr int kMaxDevices = 64;

std::mutex g_setup_mutex;
void *g_scratch_dev[kMaxDevices];  // device address of g_scratch per device

size_t scratch_need(int ndim, int nbins)
{
    const size_t edges = (((size_t)ndim * (nbins + 1) * sizeof(double)) + 255) & ~(size_t)255;
    return kStateBytes + edges + (size_t)ndim * nbins * sizeof(double);
}

// Device address of the static array on `device` (the current device).  The
// host-side name g_scratch is only a stand-in, so the address is looked up
// once per device with cudaGetSymbolAddress.
cudaError_t scratch_address(int device, char **out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_dev[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_dev[device] = p;
    }
    *out = static_cast<char *>(g_scratch_dev[device]);
    return cudaSuccess;
}

// Makes a device current for the life of the guard, then restores the
// device that was current before.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int device)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            prev = -1;
            return;
        }
        ok = prev == device || cudaSetDevice(device) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

#define CV_NA_FOR_EACH_NDIM(X)                                                               \
    X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) \
    X(17) X(18) X(19) X(20) X(21) X(22) X(23) X(24) X(25) X(26) X(27) X(28) X(29) X(30)    \
    X(31) X(32)

template <typename Real>
cudaError_t occupancy_of(int ndim, int nbins, int *occ)
{
    switch (ndim) {
#define CV_NA_CASE(D) case D: return cv::sample_occupancy<D, Real>(nbins, occ);
        CV_NA_FOR_EACH_NDIM(CV_NA_CASE)
#undef CV_NA_CASE
    }
    return cudaErrorInvalidValue;
}

template <typename Real>
cudaError_t launch_of(int ndim, const cv::SampleArgs<Real> &a, int grid, cudaStream_t s)
{
    switch (ndim) {
#define CV_NA_CASE(D) case D: return cv::launch_sample<D, Real>(a, grid, s);
        CV_NA_FOR_EACH_NDIM(CV_NA_CASE)
#undef CV_NA_CASE
    }
    return cudaErrorInvalidValue;
}

template <typename Real>
cudaError_t run(const cv_genz *g, int nbins, int flags, unsigned long long seed, int sms, long long nmax,
                int jmax, bool poll, const cv::CombineArgs &ca, double *edges, double *H, cv::DevState *st,
                cudaStream_t s)
{
    cv::SampleArgs<Real> a;
    memset(&a, 0, sizeof(a));
    cv::fill_genz_params<Real>(g, &a.g);
    a.nbins = nbins;
    a.chunk_min = 4;
    a.map = cv::make_map(nbins, g->ndim, sizeof(Real) == 8);
    cv::set_generator(&a, g->ndim, flags, seed);
    a.edges = edges;
    a.S1 = st->S1;
    a.S2 = st->S2;
    a.H = H;
    a.st = st;
    int occ = 0;
    cudaError_t e = occupancy_of<Real>(g->ndim, nbins, &occ);
    if (e != cudaSuccess) return e;
    const long long nblk = (nmax + 63) / 32;
    long long grid = (nblk + (long long)cv::kWarpsPerBlock * 16 - 1) / ((long long)cv::kWarpsPerBlock * 16);
    if (grid > (long long)sms * (occ > 0 ? occ : 1)) grid = (long long)sms * (occ > 0 ? occ : 1);
    if (grid < 1) grid = 1;
    e = cv::launch_reset(st, edges, H, g->ndim, nbins, ca.nstart, nullptr, a.map, s);
    if (e != cudaSuccess) return e;
    for (int j = 0; j < jmax; ++j) {
        e = launch_of<Real>(g->ndim, a, (int)grid, s);
        if (e != cudaSuccess) return e;
        e = cv::launch_refine_combine(g->ndim, nbins, H, edges, ca, nullptr, a.map, s);
        if (e != cudaSuccess) return e;
        if (poll && (j & 31) == 31 && j + 1 < jmax) {
            int stopped = 0;
            e = cudaMemcpyAsync(&stopped, &st->stopped, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return e;
            if (stopped) break;
        }
    }
    return cudaSuccess;
}

}  // namespace

extern "C" int cv_vegas_noalloc(int device, void *stream, int ndim, int ncomp, const cv_genz *g,
                                double epsrel, double epsabs, int flags, int seed,
                                int64_t mineval, int64_t maxeval, int64_t nstart,
                                int64_t nincrease, int64_t nbatch, int nbins, int64_t *neval,
                                int *fail, double integral[], double error[], double prob[])
{
    (void)nbatch;
    if (!g || g->ndim != ndim || g->ncomp != ncomp) return CV_EINVAL;
    if ((flags & CV_SCRAMBLE) && (flags & CV_PSEUDO)) return CV_EINVAL;
    if (ndim < 1 || ndim > CV_MAX_DIM || ncomp < 1 || ncomp > CV_MAX_COMP) return CV_EINVAL;
    for (int c = 0; c < ncomp; ++c) {
        if (g->family[c] < 0 || g->family[c] >= CV_NUM_FAMILIES) return CV_EINVAL;
        for (int d = 0; d < ndim; ++d)
            if (!std::isfinite(g->a[c][d]) || !std::isfinite(g->u[c][d])) return CV_EINVAL;
    }
    if (nbins < CV_MIN_BINS || nbins > CV_MAX_BINS) return CV_EINVAL;
    if (nstart < 2 || nincrease < 0 || maxeval < nstart || mineval < 0) return CV_EINVAL;
    if ((uint64_t)maxeval >= CV_INDEX_LIMIT || !(epsrel >= 0) || !(epsabs >= 0)) return CV_EINVAL;
    if (!neval || !fail || !integral || !error || !prob) return CV_EINVAL;
    if (!(flags & CV_FP64) && cv::fp32_range_check(g, nullptr, 0) >= 0) return CV_EINVAL;
    // the run's scratch must fit the static area
    if (scratch_need(ndim, nbins) > CV_STATIC_SCRATCH_BYTES) return CV_ESCRATCH;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev ||
        device >= kMaxDevices)
        return CV_EINVAL;
    DeviceGuard guard(device);
    if (!guard.ok) return CV_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    // a stream of another device would run this device's kernels there (the
    // legacy and per-thread default handles mean the current device)
    if (s && s != cudaStreamLegacy && s != cudaStreamPerThread) {
        int sdev = -1;
        if (cudaStreamGetDevice(s, &sdev) != cudaSuccess) {
            cudaGetLastError();
            return CV_EINVAL;
        }
        if (sdev != device) return CV_EINVAL;
    }
    char *base = nullptr;
    if (scratch_address(device, &base) != cudaSuccess) return CV_ECUDA;
    cv::DevState *st = reinterpret_cast<cv::DevState *>(base);
    double *edges = reinterpret_cast<double *>(base + kStateBytes);
    const size_t sz_edges = (((size_t)ndim * (nbins + 1) * sizeof(double)) + 255) & ~(size_t)255;
    double *H = reinterpret_cast<double *>(base + kStateBytes + sz_edges);

    // iterations the sample budget allows
    long long sum = 0, nj = nstart, nmax = nstart;
    int jmax = 0;
    while (jmax < (1 << 20) && nj <= maxeval - sum) {
        sum += nj;
        nmax = nj;
        ++jmax;
        nj += nincrease;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return CV_ECUDA;

    cv::CombineArgs ca = {};
    ca.st = st;
    ca.ncomp = ncomp;
    ca.epsrel = epsrel;
    ca.epsabs = epsabs;
    ca.mineval = mineval;
    ca.maxeval = maxeval;
    ca.nstart = nstart;
    ca.nincrease = nincrease;
    ca.log_I = nullptr;
    ca.log_var = nullptr;
    ca.log_cap = 0;
    const bool poll = !(epsrel == 0.0 && epsabs == 0.0);
    cudaError_t e = (flags & CV_FP64)
        ? run<double>(g, nbins, flags, (unsigned long long)(long long)seed, sms, nmax, jmax, poll, ca, edges, H, st, s)
        : run<float>(g, nbins, flags, (unsigned long long)(long long)seed, sms, nmax, jmax, poll, ca, edges, H, st, s);
    if (e != cudaSuccess) return CV_ECUDA;
    cv::DevState h;
    if (cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CV_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CV_ECUDA;
    *neval = h.neval;
    *fail = h.stopped ? h.fail : 1;
    for (int c = 0; c < ncomp; ++c) {
        integral[c] = h.integral[c];
        error[c] = h.error[c];
        prob[c] = h.prob[c];
    }
    return (h.status & 1) ? CV_ENONFINITE : CV_OK;
}
