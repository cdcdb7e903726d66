/*
 * cubagpu.h -- C ABI of the GB300 (sm_103a) Vegas sampling library.
 *
 * The library implements the sampling hot path of Cuba's integrators as
 * described in "Concurrent Cuba" (T. Hahn): the routine that samples n
 * points for an integrator (DoSample, Sect. 2.1), driven by Vegas, whose
 * argument list (ndim, ncomp, integrand, userdata, nvec, epsrel, epsabs,
 * flags, seed, mineval, maxeval, nstart, nincrease, nbatch, ..., neval,
 * fail, integral, error, prob) is given in Sect. 3.2.2.  The paper leaves
 * the Vegas algorithm itself to the Cuba manual; this library follows
 * Lepage (1978) for the importance grid, Sobol (1967) with the Gray-code
 * order of Antonov and Saleev (1979) for the points, and Genz (1984) for
 * the built-in test integrands.
 *
 * Conventions for every call:
 *   - Return value: CV_OK (0) or a negative CV_E* code; cv_strerror() names
 *     it and cv_last_error() gives the context's last message.
 *   - "_dev" pointers are device memory the caller owns (for example from
 *     torch); every other pointer is host memory.  Device work is enqueued
 *     on the context's stream; calls that return host results synchronise
 *     that stream first.
 *   - Arrays are C order.  A grid is edges[ndim][nbins+1] (double), a
 *     histogram hist[ndim][nbins] (double), coordinates Y[ndim][n].
 *   - A context is not thread-safe; use one per host thread.
 */
#ifndef CUBAGPU_H
#define CUBAGPU_H

#if defined(__CUDACC_RTC__)
typedef long long int64_t;
typedef unsigned long long uint64_t;
#else
#include <stdint.h>
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- limits */
#define CV_MAX_DIM 32          /* dimensions of the Sobol table            */
#define CV_MAX_COMP 4          /* integrand components                     */
#define CV_MIN_BINS 2
#define CV_MAX_BINS 256        /* grid bins per axis                       */
#define CV_INDEX_LIMIT (1ull << 52) /* Sobol indices must stay below this  */

/* ---------------------------------------------------------------- errors */
#define CV_OK 0
#define CV_EINVAL (-1)         /* an argument is out of range              */
#define CV_ENOMEM (-2)         /* device or host allocation failed         */
#define CV_ECUDA (-3)          /* a CUDA call failed                       */
#define CV_EABORT (-4)         /* the integrand returned -999              */
#define CV_ETIMEOUT (-5)       /* a bounded wait gave up                   */
#define CV_EADMIT (-6)         /* admission refused (memory budget)        */
#define CV_EBUSY (-7)          /* no free slot                             */
#define CV_ENOTFOUND (-8)      /* unknown request id                       */
#define CV_ESCRATCH (-9)       /* the problem does not fit the static scratch
                                  area of cv_vegas_noalloc                 */
#define CV_ENONFINITE (-10)    /* an iteration result was NaN or infinite:
                                  the run stopped there with fail = 1      */

/* ------------------------------------------------- built-in integrands */
/* Genz (1984) test families over [0,1]^ndim with parameters a_i > 0 and
 * u_i in [0,1]:
 *   CV_OSCILLATORY    cos(2 pi u_1 + sum a_i x_i)
 *   CV_PRODUCT_PEAK   prod (a_i^-2 + (x_i - u_i)^2)^-1
 *   CV_CORNER_PEAK    (1 + sum a_i x_i)^-(ndim+1)
 *   CV_GAUSSIAN       exp(-sum a_i^2 (x_i - u_i)^2)
 *   CV_C0             exp(-sum a_i |x_i - u_i|)
 *   CV_DISCONTINUOUS  0 if x_1 > u_1 or x_2 > u_2, else exp(sum a_i x_i)
 *   CV_CONST          1 (for exact checks)                                */
#define CV_OSCILLATORY 0
#define CV_PRODUCT_PEAK 1
#define CV_CORNER_PEAK 2
#define CV_GAUSSIAN 3
#define CV_C0 4
#define CV_DISCONTINUOUS 5
#define CV_CONST 6
#define CV_NUM_FAMILIES 7

/* ------------------------------------------------------------------ flags */
/* bits 0-1: verbosity (as Cuba's flags word).  CV_FP64 selects the plain
 * FP64 path (Sobol coordinate with 52 fraction bits, FP64 map, integrand and
 * sums); without it the point, map and integrand run in FP32 (23 fraction
 * bits) with Kahan-compensated per-thread sums and FP64 block/global
 * reduction, refinement and combination.  CV_PLAIN launches each kernel of
 * each iteration separately and synchronises the host after every
 * iteration (the one-launch-per-iteration comparator); without it the
 * iterations are replayed from a captured CUDA graph and stop on the
 * device. */
#define CV_VERBOSE_MASK 0x3
#define CV_FP64 0x100
#define CV_PLAIN 0x200
#define CV_AOS 0x400           /* cv_vegas_cb: x[nvec][ndim], f[nvec][ncomp] */
/* CV_JIT: FP32 path only -- sample with a kernel compiled at run time
 * (NVRTC) for this integrand: its component families and parameters become
 * compile-time constants (bit-identical values), which removes the
 * per-point family dispatch and parameter loads.  The first use of a given
 * integrand compiles (about a second) and caches the kernel for the
 * process; without NVRTC, or if a compile fails, the generic kernel runs.
 * Results equal those of the generic kernel. */
#define CV_JIT 0x800
/* Point generators other than the plain Sobol sequence (the seed argument
 * of Sect. 3.2.2), both keyed by a 64-bit seed through the counter-based generator
 * Philox4x64-10 (Salmon et al., SC 2011):
 *   CV_SCRAMBLE  randomized QMC: every coordinate of every Sobol point is
 *                XORed with a random digital shift of its dimension, the
 *                Philox word (0, d/4, 1, 0)[d mod 4] under key (seed, 0).
 *                All net properties of the sequence are kept; runs with
 *                independent seeds are independent unbiased replicates.
 *   CV_PSEUDO    pseudo-random sampling: the word of point i in dimension d
 *                is the Philox word (i, d/4, 0, 0)[d mod 4] under key
 *                (seed, 0).  Single integrals only (cv_sample, cv_points,
 *                cv_vegas, cv_integral_*); the batched, served and
 *                materialised paths return CV_EINVAL.
 * The y-coordinate takes the top 23 (FP32 path) or 52 (CV_FP64) bits of
 * the 64-bit word, as for Sobol points.  At most one of the two. */
#define CV_SCRAMBLE 0x1000
#define CV_PSEUDO 0x2000

/* One integral: ncomp components of one ndim-dimensional Genz problem.
 * a[c][i], u[c][i] are the parameters of component c (unused entries
 * ignored).  Component 0 drives the grid refinement.
 * delay (0 <= delay <= CV_MAX_DELAY): an integrand-cost knob, the GPU
 * counterpart of the calibrated delay the paper adds to its integrands
 * (Sect. 4.1).  Every evaluation of every component also pays about delay
 * dependent multiply-adds over the point's coordinates (the fused kernels
 * run delay * ncomp of them as one chain per point, in rounds of ndim)
 * whose bounded result enters as 0 * z: values are unchanged bit for bit,
 * only the cost grows. */
#define CV_MAX_DELAY (1 << 20)
typedef struct {
    int ndim;
    int ncomp;
    int family[CV_MAX_COMP];
    double a[CV_MAX_COMP][CV_MAX_DIM];
    double u[CV_MAX_COMP][CV_MAX_DIM];
    int delay;
} cv_genz;

typedef struct cv_ctx cv_ctx;

/* Create a context on CUDA device `device`, enqueueing on `stream` (a
 * cudaStream_t; NULL = the context creates its own non-blocking stream;
 * pass cudaStreamLegacy, (void *)1, for the legacy default stream).
 * The context owns the library's device memory; cv_destroy releases it,
 * including every cv_integral, cv_batch and cv_server still attached to
 * it, whose handles then become invalid (the analogue of cubawait for the spinning workers,
 * Sect. 3.2.3). */
int cv_create(cv_ctx **ctx, int device, void *stream);
void cv_destroy(cv_ctx *ctx);
const char *cv_strerror(int code);
const char *cv_last_error(const cv_ctx *ctx);
/* Wait for all work enqueued by the context. */
int cv_synchronize(cv_ctx *ctx);

/* Device time of individual sampling-kernel launches (the kernel of the
 * sampling pass, Sect. 2.1's DoSample, without the launches around it).
 * cv_kernel_timer(ctx, 1) clears the record and starts timing: every
 * sampling launch the context then makes on its stream outside stream
 * capture (cv_sample, cv_sample_staged, the iterations of cv_vegas and of
 * a CV_PLAIN integral) gets a CUDA event recorded on that stream immediately
 * before and after it, for the first CV_TIMER_CAP launches; later launches
 * and launches inside a graph (an integral's captured iterations) are not
 * timed.  cv_kernel_timer(ctx, 0) stops timing and keeps the record.  The
 * first enable creates 2 * CV_TIMER_CAP events (released by cv_destroy).
 * cv_kernel_times waits for the recorded launches and writes the first
 * min(cap, count) durations, in milliseconds, to the host array ms[cap];
 * *count receives the number recorded.  The events add one event record
 * before and after each timed launch on the stream. */
#define CV_TIMER_CAP 256
int cv_kernel_timer(cv_ctx *ctx, int enable);
int cv_kernel_times(cv_ctx *ctx, float *ms, int cap, int *count);

/* ------------------------------------------------ DoSample building blocks */

/* Sobol coordinates (Sect. 2: the master alone generates samples, each
 * index used once): Y_dev[d*n + j] = X_d(start + j) >> (64 - bits), where
 * X_d(i) is the 64-bit Sobol word of index i in Gray-code order.  bits is
 * 23 (the FP32 path's coordinate) or 52 (the FP64 path's).  Requires
 * 1 <= ndim <= CV_MAX_DIM, n >= 0, start + n <= CV_INDEX_LIMIT. */
int cv_sobol(cv_ctx *ctx, int ndim, uint64_t start, int64_t n, int bits,
             uint64_t *Y_dev);
/* The same for any point generator: flags 0 (Sobol), CV_SCRAMBLE or
 * CV_PSEUDO, keyed by seed (see the flags). */
int cv_points(cv_ctx *ctx, int ndim, uint64_t start, int64_t n, int bits, int flags,
              uint64_t seed, uint64_t *Y_dev);

/* One sampling pass (DoSample, Sect. 2.1): the n points with Sobol indices
 * start..start+n-1 mapped through the grid edges_dev, evaluated by the
 * built-in integrand, ADDED to the accumulators:
 *   S1_dev[c] += sum J f_c,  S2_dev[c] += sum (J f_c)^2,
 *   hist_dev[d*nbins + k] += sum over points in bin k of axis d of (J f_0)^2
 * with J = prod_d nbins (e_(k_d+1) - e_(k_d)).  flags: CV_FP64 or 0, plus
 * CV_JIT and CV_SCRAMBLE or CV_PSEUDO with their seed (see above).
 * 2 <= nbins <= CV_MAX_BINS, edges increasing from 0 to 1. */
int cv_sample(cv_ctx *ctx, const cv_genz *g, int nbins,
              const double *edges_dev, uint64_t start, int64_t n, int flags,
              uint64_t seed, double *S1_dev, double *S2_dev, double *hist_dev);

/* The FP32 pass as an integral's iterations run it: its refinement stages
 * the grid once into a table the sampling kernel copies as it is, instead
 * of every CTA converting the FP64 edges (FP64 arithmetic is slow on this
 * GPU).  cv_stage_grid writes that table for edges_dev:
 *   table_dev[d*nbins + s] = {e_k - c w_k - 1/2, m w_k}, float2 (8 bytes),
 *   w_k = e_(k+1) - e_k computed in FP64 and each entry rounded once to
 *   FP32; when nbins = 2^L >= 32 and flags has no CV_PSEUDO, m = nbins and
 *   c = 2^max(0, L-6), and s is the kernel's slot of bin k (a bit
 *   permutation of k); otherwise m = c = 1 and s = k (the FP32 kernels
 *   map to the centred coordinate x - 1/2);
 * table_dev holds ndim*nbins float2, 8-byte aligned, caller-owned; flags
 * are the sampling flags the table is for (the generator decides the
 * layout).  cv_sample_staged is cv_sample (FP32 only: CV_FP64 is refused)
 * reading such a table in place of the edges: the same sums as cv_sample
 * over the edges the table came from, up to the order of FP64 additions.
 * Both enqueue on the context's stream and return CV_OK, CV_EINVAL (bad
 * sizes, null buffers, CV_FP64) or CV_ECUDA. */
int cv_stage_grid(cv_ctx *ctx, int ndim, int nbins, int flags, const double *edges_dev,
                  void *table_dev);
int cv_sample_staged(cv_ctx *ctx, const cv_genz *g, int nbins, const void *table_dev,
                     uint64_t start, int64_t n, int flags, uint64_t seed, double *S1_dev,
                     double *S2_dev, double *hist_dev);

/* Grid refinement (Lepage 1978) in FP64, in place, per axis: smooth the
 * histogram, compress with exponent 1.5, and rebin so that every new bin
 * holds an equal share.  An axis whose histogram is all zero or not finite
 * keeps its grid. */
int cv_refine(cv_ctx *ctx, int ndim, int nbins, const double *hist_dev,
              double *edges_dev);

/* ------------------------------------------------------------ Vegas */

/* The Vegas call with the paper's argument list (Sect. 3.2.2) for a
 * built-in integrand.  ndim/ncomp must equal g->ndim/g->ncomp.  Iteration
 * j = 1, 2, ... samples n_j = nstart + (j-1) nincrease points, Sobol
 * indices continuing from 1; the run stops with fail = 0 once
 * neval >= mineval and every component has error <= max(epsabs,
 * epsrel |integral|), or with fail = 1 when the next iteration would exceed
 * maxeval.  nbatch is a performance hint only (it never changes results);
 * seed keys the CV_SCRAMBLE / CV_PSEUDO generators (the plain Sobol stream
 * does not depend on it).  integral/error/prob receive ncomp values each;
 * prob is the chi-square probability that the iteration results are not
 * consistent (P((m-1)/2, chi2/2) over m iterations).  An iteration whose
 * result is NaN or infinite stops the run there: the call fills the
 * outputs with *fail = 1 and returns CV_ENONFINITE (cv_result.status bit 0
 * in the integral, batch and server calls).  The context keeps the call's
 * device state (and with it the iterations of a problem met twice in a
 * row, as a captured CUDA graph, unless cv_kernel_timer is on): a call
 * with the same arguments replays them, with the same results bit for
 * bit. */
int cv_vegas(cv_ctx *ctx, int ndim, int ncomp, const cv_genz *g,
             double epsrel, double epsabs, int flags, int seed,
             int64_t mineval, int64_t maxeval, int64_t nstart,
             int64_t nincrease, int64_t nbatch, int nbins, int64_t *neval,
             int *fail, double integral[], double error[], double prob[]);

/* ------------------------------------------- user integrands (materialised) */
/* The integrand contract of Sect. 3.2.1-3.2.2 on the device: the library
 * writes up to nvec points to device memory and calls the integrand, which
 * fills f and returns 0, or -999 to abort the integration at once.  *nvec
 * is the actual number of points of this call (<= the requested nvec).
 * x_dev / f_dev hold float (FP32 path) or double (CV_FP64) values: by
 * default dimension-major x[d*nvec_cap + j], f[c*nvec_cap + j] (coalesced;
 * *nvec_cap, passed as userdata-independent argument `ld`, is the row
 * stride), with CV_AOS the paper's point-major x[j*ndim + d],
 * f[j*ncomp + c].  `stream` is the cudaStream_t the points were written on;
 * the integrand must enqueue its device work on it (or finish it before
 * returning).  The buffers are valid only during the call. */
typedef int (*cv_integrand_dev)(const int *ndim, const void *x_dev, const int *ncomp,
                                void *f_dev, void *userdata, const int64_t *nvec,
                                const int64_t *ld, void *stream);

/* Vegas with a user integrand (materialised-sample mode).  Per iteration
 * the points are written in tiles of at most nvec, the integrand is called
 * per tile, and the values are accumulated, with bins and Jacobians
 * recomputed from the Sobol index.  Arguments and results as cv_vegas;
 * flags may add CV_AOS.  Returns CV_EABORT (and *fail = -999) when the
 * integrand returns -999, and CV_ENONFINITE (*fail = 1, outputs filled)
 * when an iteration's result is NaN or infinite -- e.g. the integrand wrote
 * a NaN.  The accumulate passes leave per-block partial rows that are
 * added in block order (no floating-point atomics), so the same call gives
 * the same bits on every run (with nbins other than 2^L >= 32 in FP32 the
 * histogram takes shared-memory atomics within a block, in hardware order).
 * The points, values and state live in a device
 * scratch area of the context (about (ndim + ncomp) * nvec values), grown
 * on demand and kept until cv_destroy, so calls on one context must not
 * overlap. */
int cv_vegas_cb(cv_ctx *ctx, int ndim, int ncomp, cv_integrand_dev integrand,
                void *userdata, int64_t nvec, double epsrel, double epsabs,
                int flags, int seed, int64_t mineval, int64_t maxeval,
                int64_t nstart, int64_t nincrease, int64_t nbatch, int nbins,
                int64_t *neval, int *fail, double integral[], double error[],
                double prob[]);

/* A ready-made device integrand: the Genz components of `g` evaluated on
 * the materialised points (userdata = cv_genz_cb_data*; its flags carry
 * CV_FP64 / CV_AOS to match the call).  CV_JIT in those flags (FP32,
 * dimension-major): the kernel is compiled at run time with the families
 * and parameters as constants (NVRTC, cached per problem for the process;
 * without NVRTC the generic kernel runs, with the same values).  Returns 0,
 * or -999 when a launch fails. */
typedef struct {
    cv_genz g;
    int flags;
} cv_genz_cb_data;
int cv_genz_callback(const int *ndim, const void *x_dev, const int *ncomp, void *f_dev,
                     void *userdata, const int64_t *nvec, const int64_t *ld, void *stream);

/* Number of specialised kernels compiled so far in this process (CV_JIT);
 * *available is 1 if run-time compilation can be used at all. */
int cv_jit_info(int *available, int *compiled);
/* Compile (without loading) the specialised sampling kernel CV_JIT would
 * build for integrand g with nbins bins and the point generator of flags
 * (0, CV_SCRAMBLE or CV_PSEUDO), and the specialised built-in integrand
 * (cv_genz_callback with CV_JIT) for g: a check that run-time
 * compilation works here and accepts this problem.  Needs no device.
 * Returns CV_OK, CV_EINVAL for an invalid g or nbins, or CV_ENOTFOUND when
 * NVRTC is missing or rejects the source; then `log` (log_len bytes,
 * may be null) receives the reason. */
int cv_jit_check(const cv_genz *g, int nbins, int flags, char *log, int log_len);

/* The FP32 pipe's measured rate on this device, the denominator beside
 * the nominal one (SMs x 128 lanes x 2 flops x clock) for the fused
 * sampling kernel, which is bound by FP32 arithmetic and instruction issue:
 * one ~20 ms launch, four 256-thread blocks per SM, every thread 8
 * independent FMA chains (2 flops per FMA), timed with CUDA events on the
 * context's stream after a shorter warm-up launch.  *tflops receives
 * TFLOP/s, *ms (may be null) the timed launch's milliseconds.  Returns
 * CV_OK, CV_EINVAL for null ctx/tflops, or CV_ECUDA. */
int cv_fp32_fma_rate(cv_ctx *ctx, double *tflops, double *ms);

/* Bytes cv_vegas moves between host and device per call for an integral of
 * this shape: kernel parameters in (h2d), the final state out (d2h). */
int cv_vegas_io_bytes(int ndim, int nbins, int64_t *h2d, int64_t *d2h);

/* ------------------------------------------------------------- Suave */
/* Suave, the subregion-adaptive Vegas of the paper's argument list
 * (Sect. 3.2.2: nnew, flatness, nregions; the paper gives no algorithm,
 * so this is a stated reading).  Regions are axis-aligned boxes, each with
 * its own Vegas grid of nbins bins per axis (nbins even) spanning the box.
 *   Start: [0,1]^ndim sampled with nnew points, its grid refined.
 *   Round: stop once neval >= mineval and every component's
 *     sqrt(sum var) <= max(epsabs, epsrel |sum I|); else take the `width`
 *     regions of largest variance of component 0 (ties by position, only
 *     var > 0) and split each along the axis whose refined grid is least
 *     even -- the flatness-norm of |ln(w_k / mean w)| over its bins, ties
 *     by the lower axis -- at its middle edge; the children inherit the
 *     grid with the split axis's half subdivided into nbins bins, and are
 *     sampled (left first) with nnew fresh points each and refined.  The
 *     left child replaces the parent, the right one is appended.
 *   Stop adapting when a round plus the final pass would exceed maxeval or
 *     max_regions.
 *   Final pass: every region is sampled once more with nnew fresh points,
 *     and the result comes from that pass alone (the samples that chose the
 *     partition are biased by the choice): integral = sum of the regions'
 *     I, error = sqrt(sum var); *fail = 0 if the goal is met, else 1.
 * Points: one stream of indices from 1, never reused, mapped through each
 * region's grid; flags as cv_vegas (CV_FP64, CV_JIT, CV_SCRAMBLE or
 * CV_PSEUDO with seed).  With Sobol or scrambled points the final pass is
 * correlated with the partition, so on discontinuous integrands the error
 * can be underestimated; CV_PSEUDO gives independent points.
 * Execution: in FP32 with Sobol or scrambled points every pass is one
 * batched sampling launch over all its regions (CV_JIT has no effect), the
 * flatness measure computed on the device; FP64 and CV_PSEUDO passes launch
 * once per region and take every decision value on the host.  Memory,
 * allocated per call for max_regions regions: per region ndim (2 nbins + 1)
 * doubles of grid and histogram and ~2 KB of descriptors and state on the
 * device, its grid and sums in pinned host memory, and a staging area for
 * up to max(65536, 4 max_regions) tiles.
 * boxes (host, may be null): [max_regions][ndim][2], the final regions'
 * (lo, hi).  *nregions, *neval, *fail, integral[ncomp], error[ncomp] are
 * host outputs.  Errors: CV_EINVAL (arguments), CV_ENOMEM, CV_ECUDA. */
int cv_suave(cv_ctx *ctx, const cv_genz *g, int nbins, int flags, uint64_t seed,
             double epsrel, double epsabs, int64_t mineval, int64_t maxeval,
             int64_t nnew, double flatness, int width, int max_regions,
             int *nregions, int64_t *neval, int *fail, double integral[],
             double error[], double *boxes);

/* ------------------------------------------- no-allocation Vegas call */
/* cv_vegas for callers that cannot allocate device memory.  The paper has
 * no counterpart; this entry point exists because some callers of a GPU
 * library may not call cudaMalloc: a process whose device memory belongs to
 * another framework's caching allocator, a component running while a pool
 * holds every byte of the device, or code that is handed only a device and
 * a stream.  It computes what cv_vegas computes (same arguments, same
 * kernels, same results) without allocating anything: the device state,
 * grid and histogram of the run live in one static device array of
 * CV_STATIC_SCRATCH_BYTES that every GPU loading this library holds until
 * the process exits.  No context is needed: `device` is the CUDA device and
 * `stream` the cudaStream_t to run on (NULL = the legacy default stream);
 * a stream that belongs to another device is refused with CV_EINVAL.  The
 * call makes `device` current for its own work and restores the caller's
 * current device before it returns, on every path.  It waits for its work
 * on `stream` (it synchronises the stream) before returning the results.
 * Limits: the run needs 512 + R(ndim * (nbins + 1) * 8) + ndim * nbins * 8
 * bytes of the array, R() rounding up to a multiple of 256, and must fit
 * CV_STATIC_SCRATCH_BYTES, else the call returns CV_ESCRATCH (16
 * dimensions x 256 bins fit, and 32 x 254; 32 x 255 do not); otherwise
 * the arguments and return codes are those of cv_vegas.
 * The first call on a device looks up the array's device address, so make
 * it before any stream capture.  Every call on a device
 * shares the one array and leaves its last contents there (each run clears
 * what must start at zero itself); calls whose GPU work overlaps -- two
 * streams, two host threads -- race and corrupt each other: serialise
 * them. */
#define CV_STATIC_SCRATCH_BYTES (128 * 1024)
int cv_vegas_noalloc(int device, void *stream, int ndim, int ncomp,
                     const cv_genz *g, double epsrel, double epsabs, int flags,
                     int seed, int64_t mineval, int64_t maxeval,
                     int64_t nstart, int64_t nincrease, int64_t nbatch,
                     int nbins, int64_t *neval, int *fail, double integral[],
                     double error[], double prob[]);

/* ------------------------------------------- device-resident integrals */
/* A Vegas problem whose grid, sums and combination state stay in device
 * memory between iterations and between runs -- the GPU analogue of the
 * paper's spinning cores (Sect. 3.2.3), which keep workers alive across
 * integrations.  cv_vegas is create + reset + run + result + destroy. */
typedef struct {
    cv_genz g;
    int nbins;
    int flags;                 /* CV_FP64, CV_PLAIN, CV_JIT, CV_SCRAMBLE, CV_PSEUDO */
    double epsrel, epsabs;
    int64_t mineval, maxeval, nstart, nincrease, nbatch;
    uint64_t seed;             /* key of CV_SCRAMBLE / CV_PSEUDO          */
} cv_spec;

typedef struct {
    int64_t neval;
    int fail;                  /* 0 accuracy reached, 1 maxeval           */
    int iterations;
    int status;                /* bit 0: a non-finite iteration result    */
    double integral[CV_MAX_COMP];
    double error[CV_MAX_COMP];
    double prob[CV_MAX_COMP];
    double chi2[CV_MAX_COMP];
} cv_result;

typedef struct cv_integral cv_integral;

/* Allocate the device state of one problem (validated as for cv_vegas). */
int cv_integral_create(cv_ctx *ctx, const cv_spec *spec, cv_integral **out);
/* Enqueue a fresh start: uniform grid, empty sums, Sobol index 1. */
int cv_integral_reset(cv_integral *I);
/* Enqueue the iterations until the run stops.  Without an accuracy goal
 * (epsrel = epsabs = 0) this is fully asynchronous: the captured iteration
 * graph is replayed and later iterations return at once once the device has
 * stopped the run.  With a goal, the host polls the stop flag every 32
 * iterations.  CV_PLAIN: one launch per kernel and a host sync per
 * iteration. */
int cv_integral_run(cv_integral *I);
/* Synchronise and copy the results of the last run. */
int cv_integral_result(cv_integral *I, cv_result *out);
/* Synchronise and copy the current grid edges[ndim][nbins+1]. */
int cv_integral_grid(cv_integral *I, double *edges);
/* Synchronise and copy up to max_iter logged iteration results
 * I[j][c] = S1/n, var[j][c] (j < 256), ncomp values per iteration. */
int cv_integral_log(cv_integral *I, int max_iter, double *iter_I, double *iter_var);
/* Kernels one reset + run enqueues when it runs to the sample budget. */
int cv_integral_kernels_per_run(const cv_integral *I);
/* Enqueue at most max_iter more iterations (fewer if the run stops). */
int cv_integral_step(cv_integral *I, int max_iter);
/* Checkpoint and resume -- the statefile of the Vegas prototype
 * (Sect. 3.2.2): save writes the device state, grid, histogram and
 * iteration log of I to `path` (synchronising first); load restores such
 * a file into an integral of the same problem (same dimensions, bins,
 * integrand, goals, schedule and precision flags; otherwise CV_EINVAL), after
 * which cv_integral_step / cv_integral_run continue exactly where the saved
 * run stopped, Sobol index included. */
int cv_integral_save(cv_integral *I, const char *path);
int cv_integral_load(cv_integral *I, const char *path);
/* The checks cv_integral_load makes before it copies anything to the
 * device, on the host alone (no device, no context): the file must hold
 * exactly one saved state of the problem `spec` (as above); each grid axis
 * must run from 0 to 1 and increase strictly; the histogram must be finite
 * and non-negative; and the saved counters must follow the schedule the
 * spec implies -- iteration j of nstart + j nincrease points, neval the sum
 * over the iterations done (at most maxeval), the next iteration's size and
 * its first Sobol index 1 + the points sampled before it (the last
 * iteration's points not yet counted once the run has stopped).  Returns
 * CV_OK, or CV_EINVAL with the reason written to msg[len] (NUL-terminated;
 * msg may be NULL when len is 0). */
int cv_integral_check_file(const cv_spec *spec, const char *path, char *msg, int len);
/* Grid reuse (the role of Vegas's gridno): replace the grid of I, after a
 * reset, with edges[ndim][nbins+1] (increasing from 0 to 1), e.g. the
 * refined grid of an earlier integral from cv_integral_grid. */
int cv_integral_set_grid(cv_integral *I, const double *edges);
/* Release an integral; a no-op on a handle its context already released. */
void cv_integral_destroy(cv_integral *I);

/* ------------------------------------------------- batched persistent runs */
/* Many independent Vegas integrals run together (the paper's "n/N points
 * per core" of Sect. 2.1 applied across integrals as well as within one):
 * every iteration, one persistent sampling launch per dimension class walks
 * a queue of (integral, iteration, 32-point-block range) tiles of uneven
 * size, then one launch refines every axis of every integral and one
 * combines every integral; all iterations are one captured CUDA graph and
 * each integral stops on the device when its own goal or budget is reached.
 * FP32 path only (CV_FP64 / CV_PLAIN are rejected); ndim * nbins must fit
 * the per-warp histograms in shared memory (10 * ndim * nbins * 4 bytes
 * <= 227 KiB, e.g. 32 x 128 or 20 x 256).  An integral's points are cut
 * into tiles by a rule that depends on that integral alone (about 16
 * tiles per iteration, 2^11 .. cap points each; CUBAGPU_TILE, points,
 * forces one size), and each tile leaves its sums and histogram as
 * partial rows that the refinement and combination add in tile order (no
 * floating-point atomics), so an integral's result is the same alone, in
 * any batch and on every run, bit for bit, for the same tile cap and split
 * (with nbins other than 2^L >= 32 a warp's histogram copy takes shared-
 * memory atomics, whose order within a tile the hardware picks).  It
 * agrees with cv_vegas within the FP32 tolerance (the single-integral
 * kernel groups points differently). */
typedef struct cv_batch cv_batch;
int cv_batch_create(cv_ctx *ctx, int count, const cv_spec *specs, cv_batch **out);
/* Enqueue one complete run of every integral (asynchronous). */
int cv_batch_run(cv_batch *B);
/* Synchronise and copy count results. */
int cv_batch_results(cv_batch *B, cv_result *out);
/* Time the first iteration's sampling with tile caps of 2^13, 2^15 and
 * 2^17 points and, below the cap, iterations cut into at most 8, 16 or 32
 * tiles (a tile is shared by the eight warps of a CTA, so these set the
 * points per thread), and keep the fastest pair (resets the integrals;
 * call before run). */
int cv_batch_autotune(cv_batch *B);
/* The per-iteration results of integral `item` of the batch's last run,
 * as cv_integral_log: iter_I[j*ncomp + c] = S1/n_j, iter_var[j*ncomp + c] =
 * (S2/n_j - (S1/n_j)^2)/(n_j - 1) for j < min(max_iter, the iterations its
 * budget allows), ncomp its component count; host arrays of that size.
 * cv_batch_grid copies its current grid edges[ndim][nbins+1] (after a run:
 * refined once per iteration run).  Both synchronise the context's stream
 * and return CV_OK, CV_EINVAL (bad handle, item or pointer) or CV_ECUDA. */
int cv_batch_log(cv_batch *B, int item, int max_iter, double *iter_I, double *iter_var);
int cv_batch_grid(cv_batch *B, int item, double *edges);
/* Points per tile the batch uses for an iteration of n points. */
int cv_batch_tile_points(const cv_batch *B, long long n);
/* Kernels one cv_batch_run enqueues. */
int cv_batch_kernels_per_run(const cv_batch *B);
/* Release a batch; a no-op on a handle its context already released. */
void cv_batch_destroy(cv_batch *B);
/* create + run + results + destroy. */
int cv_batch_vegas(cv_ctx *ctx, int count, const cv_spec *specs, cv_result *out);

/* --------------------------------------------------------------- serving */
/* A request loop with continuous batching: requests of any ndim, ncomp and
 * accuracy goal are submitted from any host thread; a worker thread admits
 * them in arrival order while a slot and the device-memory budget allow,
 * keeps each admitted request's grid and sums resident on the device, and
 * runs rounds in which every admitted request advances by one iteration
 * through the batched kernels (requests that arrive meanwhile join at the
 * next round boundary).  A request whose goal or budget is reached leaves
 * at once and frees its slot and memory.  Each request's result is the
 * same alone and in any mix of requests, bit for bit (see cv_batch_create
 * for the tiling rule, the partial rows, the ndim * nbins limit and the
 * bin counts this holds for).
 * The analogue of the paper's spinning cores (Sect. 3.2.3): the worker and
 * its device state persist between integrations until cv_server_stop. */
typedef struct {
    int64_t hbm_budget_bytes;  /* device memory for request state (0: 1 GiB) */
    int max_live;              /* requests on the device at once (0: 4096)    */
    int tile_points;           /* points per tile (0: automatic)              */
} cv_server_opts;

typedef struct {
    int64_t submitted, completed, rounds, samples;
    int max_live;              /* most requests on the device in one round    */
    int pending;               /* requests waiting for admission now          */
    double p50_ms, p99_ms, max_ms;  /* submit-to-result latency               */
    double busy_s, wall_s;     /* time in rounds, time since start            */
    double gpu_s;              /* device time of the rounds (CUDA events)     */
} cv_serve_stats;

typedef struct cv_server cv_server;
int cv_server_start(cv_ctx *ctx, const cv_server_opts *opts, cv_server **out);
/* Queue a request (FP32 path); CV_EADMIT if it can never fit the budget. */
int cv_submit(cv_server *S, const cv_spec *spec, uint64_t *id);
/* CV_OK with the result, CV_EBUSY while it runs, CV_ENOTFOUND. */
int cv_poll(cv_server *S, uint64_t id, cv_result *out);
/* Wait up to timeout_ms; CV_ETIMEOUT if it has not finished. */
int cv_wait(cv_server *S, uint64_t id, int timeout_ms, cv_result *out);
int cv_server_stats(cv_server *S, cv_serve_stats *out);
/* Finish every submitted request, stop the worker, release the server. */
int cv_server_stop(cv_server *S);

#ifdef __cplusplus
}
#endif

#endif /* CUBAGPU_H */
