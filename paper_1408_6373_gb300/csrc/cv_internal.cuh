// cv_internal.cuh -- internal types shared by the CUDA translation units of
// the Vegas sampling library (not part of the public C ABI).
#pragma once

#if !defined(__CUDACC_RTC__)
#include <cuda_runtime.h>
#include <cmath>
#include <cstdint>
#include <cstring>
#endif

#include "../../include/cubagpu.h"

namespace cv {

constexpr int kWarp = 32;
constexpr int kBlock = 256;                 // threads per sampling block
constexpr int kWarpsPerBlock = kBlock / kWarp;
constexpr int kLogCap = 256;                // iterations logged per integral

// Device-resident state of one integral between iterations: the analogue of
// Cuba's spinning workers keeping their state (Sect. 3.2.3), here kept in
// HBM so iterations chain on the device without host round trips.
struct DevState {
    unsigned long long next_index;  // Sobol index of the next iteration's first point
    long long n_cur;                // points of the next iteration
    long long neval;                // points sampled so far
    int iter;                       // iterations completed
    int stopped;                    // 1 once the run has terminated
    int fail;                       // Cuba's fail: 0 accuracy reached, 1 maxeval
    int status;                     // bit 0: a non-finite iteration result
    int pass_active;                // the last sampling launch ran (set by that launch)
    double S1[CV_MAX_COMP];         // sum J f_c of the running iteration
    double S2[CV_MAX_COMP];         // sum (J f_c)^2
    // inverse-variance combination (West's weighted incremental update)
    double W[CV_MAX_COMP];          // sum 1/var_j
    double mean[CV_MAX_COMP];       // weighted mean
    double M2[CV_MAX_COMP];         // sum (I_j - mean)^2 / var_j
    double sumI[CV_MAX_COMP];       // plain sum of I_j (zero-variance fallback)
    int zero[CV_MAX_COMP];          // a var_j <= 0 was seen
    double integral[CV_MAX_COMP];
    double error[CV_MAX_COMP];
    double chi2[CV_MAX_COMP];
    double prob[CV_MAX_COMP];
};

// Per-component integrand parameters in the precision of the evaluation,
// pre-transformed on the host so the inner loop is FMA-shaped.  FP64 takes
// x in [0, 1]:
//   oscillatory   p0 = a, q0 = 2 pi u_1;  product peak p0 = 1/a^2, p1 = u
//   corner peak   p0 = a;  gaussian p0 = a^2, p1 = u
//   c0, discontinuous p0 = a, p1 = u
// FP32 takes the centred coordinate z = x - 1/2 and base-2 exponents
// (l = log2 e; pairs q0 + q1 carry a constant to twice binary32 precision):
//   oscillatory   p0 = a/(2 pi) (turns); q0 + q1 = u_1 + sum a/(4 pi), mod 1
//   product peak  p0 = 1/a^2, p1 = 1/2 - u
//   corner peak   p0 + p1 = a (high and low halves), taken on x = z + 1/2
//   gaussian      p0 = a sqrt(l), p1 = a sqrt(l) (1/2 - u)
//   c0            p0 = a l, p1 = 1/2 - u
//   discontinuous p0 = a l, p1 = u - 1/2, q0 = exp(sum a / 2)
template <typename Real>
struct GenzParams {
    int ndim;
    int ncomp;
    int family[CV_MAX_COMP];
    // (16-byte aligned: runs of four parameters can be read with one
    // vector load when they sit in shared memory)
    alignas(16) Real p0[CV_MAX_COMP][CV_MAX_DIM];
    alignas(16) Real p1[CV_MAX_COMP][CV_MAX_DIM];
    Real q0[CV_MAX_COMP];
    Real q1[CV_MAX_COMP];           // FP32: the low half of a constant held as q0 + q1
    int delay;                      // extra dependent FMAs per evaluation (cost knob)
};

// ---- point generators ----
enum { kGenSobol = 0, kGenScrambled = 1, kGenPseudo = 2 };

// The generator of a point-only launch (cv_points): shift[d] in the
// launch's word layout (64-bit words, or their unpermuted top halves).
struct PointArgs {
    int gen;
    unsigned long long seed;
    unsigned long long shift[CV_MAX_DIM];
};

// Philox4x64-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC 2011): ten rounds on a 256-bit counter block c under
// a 128-bit key k; a round takes the 128-bit products of c0 and c2 with two
// odd constants and forms (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0), and the
// key advances by two Weyl constants (golden ratio, sqrt(3) - 1) between
// rounds.  c is replaced by the output block.
__host__ __device__ inline void mulhilo64(unsigned long long a, unsigned long long b,
                                          unsigned long long &hi, unsigned long long &lo)
{
#if defined(__CUDA_ARCH__)
    lo = a * b;
    hi = __umul64hi(a, b);
#else
    const unsigned __int128 p = (unsigned __int128)a * b;
    hi = (unsigned long long)(p >> 64);
    lo = (unsigned long long)p;
#endif
}

__host__ __device__ inline void philox4x64_10(unsigned long long (&c)[4], unsigned long long k0,
                                              unsigned long long k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        unsigned long long hi0, lo0, hi1, lo1;
        mulhilo64(0xD2E7470EE14C6C93ull, c[0], hi0, lo0);
        mulhilo64(0xCA5A826395121157ull, c[2], hi1, lo1);
        const unsigned long long c1 = c[1], c3 = c[3];
        c[0] = hi1 ^ c1 ^ k0;
        c[1] = lo1;
        c[2] = hi0 ^ c3 ^ k1;
        c[3] = lo0;
        k0 += 0x9E3779B97F4A7C15ull;
        k1 += 0xBB67AE8584CAA73Bull;
    }
}

// Uniform constants of the FP32 map for N = 2^L (see cv_device.cuh).
struct MapParams {
    int pow2;                       // N = 2^L with L >= 5: the bit-level map below
    int L;                          // log2 N
    unsigned mF;                    // the fraction's mantissa bits in the permuted word
    unsigned expE;                  // exponent field of 2^(G - L)
    int li;                         // direction table: L - 4 (permuted words), else 0
    unsigned sA;                    // byte offset of the bin's grid entry = word >> sA, sA = 29 - L
    int G;                          // the fraction sits 2^-G below the mantissa's top (G = max(0, L - 6))
    int priv;                       // per-warp f^2 histograms updated without atomics
};

// The FP32 sampling kernels' table entry of a bin with left edge e and
// width w (both FP64), each half rounded once to binary32.  The kernels map
// to the centred coordinate x - 1/2 (binary32 keeps absolute precision
// near 0, so the integrands' sums over coordinates round far less than over
// [0, 1] values): x - 1/2 = fma(s w, f1, e - c w - 1/2), f1 the mantissa
// construction of the fraction, c = 2^G and s = N for the power-of-two map,
// c = s = 1 for the general one (where the kernel multiplies J by N).
__host__ __device__ __forceinline__ float2 grid_entry_f32(double e, double w, int N, const MapParams &m)
{
    const double c = m.pow2 ? (double)(1 << m.G) : 1.0;
    const double s = m.pow2 ? (double)N : 1.0;
#if defined(__CUDA_ARCH__)
    return make_float2(__double2float_rn(e - c * w - 0.5), __double2float_rn(s * w));
#else
    return make_float2((float)(e - c * w - 0.5), (float)(s * w));
#endif
}

// Grid slot of bin k of an axis (and back).  Power-of-two N >= 32: the bit
// permutation of the direction words puts bin bits (y_6..y_L) above y_5 above
// (y_1..y_4), so the 32 points of an aligned block occupy 32 distinct slots
// modulo 32 (distinct shared-memory banks); other N: the identity.
__host__ __device__ __forceinline__ int slot_of_bin(int k, const MapParams &m)
{
    if (m.pow2) {
        const int L = m.L;
        return ((k & ((1 << (L - 5)) - 1)) << 5) | (((k >> (L - 5)) & 1) << 4) | (k >> (L - 4));
    }
    return k;
}
__host__ __device__ __forceinline__ int bin_of_slot(int p, const MapParams &m)
{
    if (m.pow2) {
        const int L = m.L;
        return ((p & 15) << (L - 4)) | (((p >> 4) & 1) << (L - 5)) | (p >> 5);
    }
    return p;
}

// Arguments of one sampling launch.  When `st` is non-null the launch reads
// its index range from the device state (and returns at once if the run has
// stopped), which is what lets a captured graph replay iterations whose
// sizes are decided on the device.
template <typename Real>
struct SampleArgs {
    GenzParams<Real> g;
    int nbins;
    int chunk_min;                  // minimum warp-steps per chunk
    MapParams map;
    const double *edges;            // [ndim][nbins+1]
    // FP32 path: the grid already staged for the kernel, {e_k - w_k, w_k}
    // (w_k scaled by N for power-of-two N) in slot order, [ndim][nbins],
    // written by the refinement that produced `edges`; null: the kernel
    // converts `edges` itself (the same FP64 operations, so the same values)
    const float2 *ew32;
    double *S1;                     // [ncomp]
    double *S2;                     // [ncomp]
    double *H;                      // [ndim][nbins]
    unsigned long long start;
    long long n;
    DevState *st;
    // materialised samples (the caller's integrand): the points written to
    // x, the values read from f, point j = index - start of the launch at
    // x[d ld + j], f[c ld + j] (aos = 0) or x[j ndim + d], f[j ncomp + c]
    Real *x;
    const Real *f;
    long long ld;
    int aos;
    // point generator: kGenSobol, kGenScrambled (Sobol words XOR shift[d],
    // in the kernel's word layout) or kGenPseudo (Philox words keyed by seed)
    int gen;
    unsigned long long seed;
    unsigned long long shift[CV_MAX_DIM];
    // Deterministic reduction (part_S non-null; the launch's grid must be
    // part_G blocks): block b writes its sums to part_S[b][2 c + {0, 1}] and
    // its histogram to part_H[b][ndim][nbins] (Real), no atomics.  With a
    // ticket (zero before the launch and reset by that block) the last
    // block to finish adds the blocks' sums to S1, S2 in block order;
    // without one the sums are left to the kernel that consumes the pass
    // (the combination of an integral's iteration).  The histogram partials
    // are summed per bin in block order by that kernel too (refinement, or
    // a reduction after a standalone pass).  Null: FP64 atomics, whose
    // order varies from run to run.
    double *part_S;                 // [part_G][2 CV_MAX_COMP]
    void *part_H;                   // [part_G][ndim][nbins]
    unsigned *part_ticket;
    int part_G;
};

// Bytes of the per-block partials of a deterministic pass.
inline size_t pass_parts_bytes(int G, int ndim, int nbins, bool fp64)
{
    return (size_t)G * 2 * CV_MAX_COMP * sizeof(double) +
           (size_t)G * ndim * nbins * (fp64 ? sizeof(double) : sizeof(float)) + 256;
}

struct CombineArgs {
    DevState *st;
    int ncomp;
    double epsrel, epsabs;
    long long mineval, maxeval, nstart, nincrease;
    double *log_I;                  // [log_cap][CV_MAX_COMP] or null
    double *log_var;
    int log_cap;                    // iterations the log holds (<= kLogCap)
    // the sampling pass's histogram partials (SampleArgs::part_H), summed by
    // the refinement in block order; null: the pass added them to H itself
    const void *part_H;
    int part_G;
    int part_nh;                    // ndim * nbins: values per block
    int part_f32;                   // partials are floats (FP32 pass)
    // the pass's sum partials (SampleArgs::part_S of a launch without a
    // ticket), summed by the combination in block order; null: the pass
    // added them to S1, S2 itself
    const double *part_S;
    // a host-mapped word that receives the run's stop flag after every
    // combination (the host reads it once the launch has completed); null:
    // none
    int *host_stop;
};

// ---- batched persistent launch (many integrals) ----
// One integral of a batch as the device sees it.
struct BatchItem {
    SampleArgs<float> a;            // parameters, map, nbins (pointers unused)
    DevState *st;
    double *edges;                  // [ndim][nbins+1]
    double *H;                      // [ndim][nbins]
};

// A tile: nblk consecutive 32-point Sobol blocks of one integral's
// iteration, starting at absolute block q0.  row, hoff: where the tile
// leaves its sums and histogram when the launch reduces through partials.
struct Tile {
    int item;
    int nblk;
    unsigned long long q0;
    int row;                        // row of BatchSampleArgs::part_S
    unsigned hoff;                  // first float of its [ndim][nbins] rows in part_H
};

// The partial rows of one integral's tiles in one iteration: count
// consecutive sum rows from row0, and histogram rows of `stride` floats
// (ndim nbins rounded up to a multiple of 4) from float hoff0.
struct TileParts {
    int row0;
    int count;
    unsigned hoff0;
    int stride;
};

struct BatchSampleArgs {
    const BatchItem *items;
    const Tile *tiles;
    int ntiles;
    int stride;                     // slots per axis: the class's largest nbins
    int *counter;                   // next tile to take (zero before the launch)
    // Deterministic reduction (part_S non-null): tile t writes its sums to
    // part_S[t.row][2 c + {0, 1}] and its histogram, by bin, to part_H +
    // t.hoff, no atomics; the batched refinement and combination add an
    // integral's rows in tile order.  Null: FP64 atomics into the
    // integral's state and histogram.
    double *part_S;
    float *part_H;
};

// Shared memory of a batched sampling block: grid e, w and one f^2
// histogram per warp, `stride` slots per axis each, and 8 stride bytes to
// align the grid for the kernels' funnel-shift addressing.
inline size_t batch_smem_bytes(int ndim, int stride) {
    return (size_t)(2 + kWarpsPerBlock) * ndim * stride * sizeof(float) + 8 * (size_t)stride;
}

#if !defined(__CUDACC_RTC__)
// ---- launchers (template definitions in cv_device.cuh, instantiated per
// ---- dimension range in cv_sample_*.cu) ----
template <int NDIM, typename Real>
cudaError_t launch_sample(const SampleArgs<Real> &a, int grid, cudaStream_t s);
template <int NDIM, typename Real>
cudaError_t sample_occupancy(int nbins, int *blocks_per_sm);
template <int NDIM, bool POW2>
cudaError_t launch_batch_sample(const BatchSampleArgs &b, int grid, cudaStream_t s);
template <int NDIM>
cudaError_t batch_occupancy(bool pow2, int stride, int *blocks_per_sm);
template <int NDIM, typename Word>
cudaError_t launch_sobol(unsigned long long start, long long n, int bits, const PointArgs &pa,
                         unsigned long long *Y, int grid, cudaStream_t s);

// materialised samples: store the points (mode 1) or accumulate the
// caller's values (mode 2) over [a.start, a.start + a.n)
template <int NDIM, typename Real, int MODE>
cudaError_t launch_matpass(const SampleArgs<Real> &a, int grid, cudaStream_t s, int *grid_used);

template <int NDIM, typename Real, bool AOS>
cudaError_t launch_genz_points(const GenzParams<Real> &g, const Real *x, Real *f, long long n,
                               long long ld, int grid, cudaStream_t s);

// cv_refine.cu
cudaError_t launch_refine(int ndim, int nbins, double *H, double *edges, cudaStream_t s);
// H[i] += the G blocks' partials of bin i (nh bins), in block order
cudaError_t launch_add_parts(const void *part_H, int G, int f32, int nh, double *H, cudaStream_t s);
// (ew32, map: when ew32 is non-null the kernels also write the FP32 grid
// table of SampleArgs::ew32 for the grid they leave, in map's slot order)
cudaError_t launch_refine_combine(int ndim, int nbins, double *H, double *edges,
                                  const CombineArgs &a, float2 *ew32, const MapParams &map,
                                  cudaStream_t s);
cudaError_t launch_reset(DevState *st, double *edges, double *H, int ndim, int nbins,
                         long long nstart, float2 *ew32, const MapParams &map, cudaStream_t s);
cudaError_t launch_stage_grid(int ndim, int nbins, const double *edges, float2 *ew32,
                              const MapParams &map, cudaStream_t s);
// (list: optional indices of the integrals to act on, else 0..count-1)
cudaError_t launch_batch_reset(const BatchItem *items, const CombineArgs *cargs, int count,
                               cudaStream_t s, const int *list = nullptr);
// (parts, part_S, part_H: the tiles' partial rows of this iteration, parts
// indexed by integral; null parts: the sums and histograms are in the
// integrals' states)
cudaError_t launch_batch_refine(const BatchItem *items, const int2 *axes, int naxes,
                                cudaStream_t s, const TileParts *parts = nullptr,
                                const float *part_H = nullptr);
cudaError_t launch_batch_combine(const CombineArgs *cargs, int count, cudaStream_t s,
                                 const int *list = nullptr, const TileParts *parts = nullptr,
                                 const double *part_S = nullptr);
cudaError_t launch_gather_states(const BatchItem *items, const int *list, int count,
                                 DevState *out, cudaStream_t s);

// cv_jit.cu: the sampling kernel specialised at run time for one integrand
struct JitKernel {
    cudaLibrary_t lib;
    cudaKernel_t kernel;
    int occ;                        // resident blocks per SM
    size_t smem;
};
}  // namespace cv
#include <string>
namespace cv {
int jit_sample_kernel(int device, const SampleArgs<float> &a, int ndim, bool pow2, int min_blocks,
                      JitKernel *out, std::string *err);
// compile the specialised source without loading it (checks NVRTC and the source)
int jit_compile_check(const SampleArgs<float> &a, int ndim, bool pow2, int min_blocks, std::string *err);
cudaError_t launch_jit_sample(const JitKernel &k, const SampleArgs<float> &a, int grid, cudaStream_t s);
// the built-in integrand on dimension-major FP32 points, specialised for g
int jit_points_kernel(int device, const GenzParams<float> &g, int ndim, JitKernel *out, std::string *err);
cudaError_t launch_jit_points(const JitKernel &k, const GenzParams<float> &g, const float *x, float *f, long long n,
                              long long ld, int grid, cudaStream_t s);
int jit_info(int *compiled);
// cv_api.cu: the parameters of a built-in integrand in the kernels' forms
template <typename Real>
void fill_genz_params(const cv_genz *g, GenzParams<Real> *p);
// cv_api.cu: the FP32 path's range precondition for built-in integrands
// (first failing component and a message, or -1)
int fp32_range_check(const cv_genz *g, char *msg, size_t len);
#endif  // !__CUDACC_RTC__

// Shared memory of a sampling block.  FP64: grid {e, w} with CV_MAX_BINS
// slots per axis, then the block's histogram with CV_MAX_BINS slots per
// axis or, with private histograms, one [ndim][nbins] copy per warp.  FP32: the grid table [ndim][nbins] (8-byte
// entries, aligned to 8 nbins bytes), then either one block histogram
// [ndim][nbins] of floats or, with private histograms, one such copy per
// warp.
inline size_t sample_smem_bytes(int ndim, int nbins, bool fp64, bool priv) {
    if (fp64)
        return (size_t)ndim * CV_MAX_BINS * 2 * sizeof(double) +
               (priv ? (size_t)kWarpsPerBlock * ndim * nbins : (size_t)ndim * CV_MAX_BINS) * sizeof(double);
    return (size_t)ndim * nbins * 2 * sizeof(float) +
           (priv ? (size_t)kWarpsPerBlock * ndim * nbins : (size_t)ndim * nbins) * sizeof(float) +
           8 * (size_t)nbins;  // (to align the grid to 8 nbins bytes)
}

// Resident 256-thread blocks per SM the FP32 sampling kernels are compiled
// for (their __launch_bounds__): three up to 8 dimensions, else two.
inline int min_blocks_f32(int ndim) { return ndim <= 8 ? 3 : 2; }

constexpr size_t kSmemPerSM = 228 * 1024;     // shared memory of one SM
constexpr size_t kSmemBlockReserve = 2048;    // per block: runtime reserve + static arrays

#if !defined(__CUDACC_RTC__)
// Map constants of an axis with N bins for the sampling kernels.
//   N = 2^L >= 32: frac/N and the bin's slot come straight from the bits of
//   the Sobol word (table li = L - 4 holds the words bit-permuted so that
//   the slot is word >> (32 - L) and the fraction's bits sit at mantissa
//   position: word & mF).  Other N take the generic map.
//   priv: for N >= 32 the 32 points of an aligned block fall into 32
//   distinct 1/32-strata of every axis, hence into 32 distinct bins, so a
//   warp can keep its own f^2 histogram and update it with plain loads and
//   stores.  Used on the FP32 path when every warp's copy fits beside the
//   grid at the occupancy the kernel is compiled for.
inline MapParams make_map(int N, int ndim, bool fp64)
{
    MapParams m;
    memset(&m, 0, sizeof(m));
    m.pow2 = (N & (N - 1)) == 0 && N >= 32;
    if (m.pow2) {
        int L = 0;
        while ((1 << L) < N) ++L;
        m.L = L;
        // (the layout slot_perm writes: slot, three zero bits, the 23 - L
        // fraction bits from mantissa bit `top` down)
        const int top = 28 - L < 22 ? 28 - L : 22;
        const int F = 23 - L;
        m.G = 22 - top;
        m.mF = ((1u << F) - 1u) << (top - F + 1);
        m.expE = (unsigned)(127 + m.G - L) << 23;
        m.li = L - 4;
        m.sA = 29 - L;
        const int blocks = min_blocks_f32(ndim);
        // (FP64: the kernel is compiled for one block per SM; its copies must
        // still leave room for a second)
        m.priv = fp64 ? 2 * (sample_smem_bytes(ndim, N, true, true) + kSmemBlockReserve) <= kSmemPerSM
                      : (size_t)blocks * (sample_smem_bytes(ndim, N, false, true) + kSmemBlockReserve) <= kSmemPerSM;
    }
    return m;
}

// The bit layout of the FP32 direction words for N = 2^L (5 <= L <= 8),
// a linear map of the word's bits (it commutes with XOR, so a point's word
// is the map of its unmapped word).  With y_t the bit of weight 2^-t of
// w / 2^32:
//   bits 31..32-L   the bin's slot (y_6..y_L, y_5, y_1..y_4),
//   bits 31-L..29-L zero, so that word >> (29 - L) is the slot times 8, the
//                   byte offset of the bin's 8-byte grid entry,
//   y_(L+1)..y_23   the fraction within the bin, at mantissa bits
//                   top .. top - 22 + L with top = min(22, 28 - L),
//   y_24..y_29      the remaining bits; y_30..y_32 are dropped
// (the FP32 path's coordinate keeps 23 bits).  A digital shift of the
// scrambled generator is mapped the same way.
inline unsigned slot_perm(unsigned w, int L)
{
    const int top = 28 - L < 22 ? 28 - L : 22;
    unsigned used = 0;
    unsigned out = 0;
    int pos[33];
    for (int t = 1; t <= 32; ++t) pos[t] = -1;
    for (int t = 1; t <= 4; ++t) pos[t] = 32 - L + (4 - t);
    pos[5] = 32 - L + 4;
    for (int t = 6; t <= L; ++t) pos[t] = 37 - t;
    for (int t = L + 1; t <= 23; ++t) pos[t] = top - (t - L - 1);
    for (int t = 1; t <= 23; ++t) used |= 1u << pos[t];
    used |= 7u << (29 - L);
    int t = 24;
    for (int b = 31; b >= 0 && t <= 29; --b)
        if (!((used >> b) & 1u)) pos[t++] = b;
    for (int u = 1; u <= 29; ++u) out |= ((w >> (32 - u)) & 1u) << pos[u];
    return out;
}

// The point generator of a launch from the flags: the digital shifts of
// CV_SCRAMBLE in the kernel's word layout (64-bit words on the FP64 path,
// top halves -- permuted on the power-of-two FP32 map -- on the FP32 path);
// CV_PSEUDO takes the generic map with block histograms, since its points
// have no net structure.
template <typename Real>
inline void set_generator(SampleArgs<Real> *a, int ndim, int flags, unsigned long long seed)
{
    a->gen = (flags & CV_PSEUDO) ? kGenPseudo : ((flags & CV_SCRAMBLE) ? kGenScrambled : kGenSobol);
    a->seed = seed;
    memset(a->shift, 0, sizeof(a->shift));
    if (a->gen == kGenPseudo) {
        a->map.pow2 = 0;
        a->map.priv = 0;
        a->map.li = 0;
    } else if (a->gen == kGenScrambled) {
        for (int d = 0; d < ndim; ++d) {
            unsigned long long c[4] = {0ull, (unsigned long long)(d / 4), 1ull, 0ull};
            philox4x64_10(c, seed, 0ull);
            const unsigned long long S = c[d % 4];
            if (sizeof(Real) == 8) a->shift[d] = S;
            else a->shift[d] = a->map.pow2 ? slot_perm((unsigned)(S >> 32), a->map.L) : (unsigned)(S >> 32);
        }
    }
}
#endif

}  // namespace cv
