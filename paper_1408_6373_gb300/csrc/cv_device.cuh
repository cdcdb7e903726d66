// cv_device.cuh -- device code of the fused sampling path (one pass of
// DoSample, "Concurrent Cuba" Sect. 2.1, as Vegas drives it):
//
//   Sobol word X_d(i) (Gray-code order, skip-ahead + recurrence)
//     -> y-coordinate with b fraction bits (b = 23 FP32 path, 52 FP64 path)
//     -> Vegas grid map x_d = e_k + w_k frac, J = prod_d N w_k (Lepage 1978)
//     -> Genz integrand f_c(x) (Genz 1984)
//     -> per-thread sums of J f_c and (J f_c)^2 (Kahan in FP32)
//     -> f^2 histogram H[d][k_d] += (J f_0)^2 in shared memory
//     -> FP64 block/global reduction.
//
// Work decomposition.  The n indices of one pass are cut into aligned
// blocks of 32 (one index per lane), and every warp owns a contiguous run of
// such blocks (a "chunk").  Lane l of a warp handles index 32 q + l of block
// q, so the 32 points a warp evaluates together form an aligned Gray-code
// block: by the (0,1)-property of each Sobol coordinate they fall into 32
// distinct 1/32-strata of every axis, which keeps the shared-memory
// histogram nearly free of same-address conflicts.  Stepping from block q
// to q+1 changes the Gray code of every lane's index by the same two bits,
// 4 and 5 + ctz(q+1), so each coordinate advances with one warp-uniform
// table lookup and one XOR.
#pragma once

#include "cv_internal.cuh"
#include "sobol_dirs.h"

namespace cv {

// Direction words in constant memory (every access below is warp-uniform),
// in step form: entry k is V_k for k < 5 and V_4 ^ V_k for k >= 5, so the
// step between aligned 32-point blocks (Gray-code bits 4 and 5 + c flip
// together) is one word.
static __constant__ unsigned long long c_W64[CV_SOBOL_DIMS][CV_SOBOL_BITS] = CV_SOBOL_W64_INIT;
// Top 32 bits of the words: table 0 as they are; table li = L - 4 for
// N = 2^L bins (L = 5..8) with the bits permuted so that the bin's slot is
// the word's top L bits and the fraction's bits sit at mantissa position
// (layout at the maps below).  A bit permutation commutes with XOR, so a point's
// permuted word is the permutation of its word.
static __constant__ unsigned int c_W32P[5][CV_SOBOL_DIMS][CV_SOBOL_BITS] = CV_SOBOL_W32P_INIT;

template <typename W> struct Dir;
template <> struct Dir<unsigned long long> {
    static __device__ __forceinline__ unsigned long long w(int, int d, int k) { return c_W64[d][k]; }
};
template <> struct Dir<unsigned int> {
    static __device__ __forceinline__ unsigned int w(int li, int d, int k) { return c_W32P[li][d][k]; }
};

// Sobol words of index i = 32 q + lane for every dimension (skip-ahead):
// X_d(i) = XOR over the set bits k of g(i) = i ^ (i >> 1) of V_d[k].  The
// bits of g above bit 4 are g(q) and the same for the whole warp; bits 0-4
// depend on the lane.
template <int NDIM, typename W>
__device__ __forceinline__ void sobol_skip(W (&X)[NDIM], unsigned long long q, int lane, int li = 0)
{
    const unsigned long long i = q * 32ull + (unsigned long long)lane;
    const unsigned long long g = i ^ (i >> 1);
    const unsigned glo = (unsigned)g & 31u;
    unsigned long long ghi = g >> 5;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
        W x = 0;
#pragma unroll
        for (int k = 0; k < 5; ++k)
            x ^= ((glo >> k) & 1u) ? Dir<W>::w(li, d, k) : W(0);
        // V_k = W_k ^ W_4 for k >= 5: W_4 once per set bit of ghi
        if (__popcll(ghi) & 1) x ^= Dir<W>::w(li, d, 4);
        X[d] = x;
    }
    while (ghi) {  // warp-uniform
        const int k = __ffsll((long long)ghi) - 1 + 5;
#pragma unroll
        for (int d = 0; d < NDIM; ++d)
            X[d] ^= Dir<W>::w(li, d, k);
        ghi &= ghi - 1;
    }
}

// Advance every lane from block q to block q+1:
// g(32(q+1)+l) ^ g(32q+l) = 2^4 ^ 2^(5 + ctz(q+1)).
template <int NDIM, typename W>
__device__ __forceinline__ void sobol_step(W (&X)[NDIM], unsigned long long q, int li = 0)
{
    // (c <= 46 for every q + 1 < 2^47; clamped so that a step past the last
    // block of the index range stays inside the table)
    const int c = min(__ffsll((long long)(q + 1ull)) - 1, CV_SOBOL_BITS - 6);
#pragma unroll
    for (int d = 0; d < NDIM; ++d)
        X[d] ^= Dir<W>::w(li, d, 5 + c);
}

// Pseudo-random words of point i (CV_PSEUDO): word d is Philox4x64-10 block
// (i, d/4, 0, 0)[d mod 4] under key (seed, 0); the FP32 path keeps the top
// 32 bits (its y takes the top 23 of them).
template <int NDIM, typename W>
__device__ __forceinline__ void pseudo_words(W (&X)[NDIM], unsigned long long seed, unsigned long long i)
{
#pragma unroll
    for (int d0 = 0; d0 < NDIM; d0 += 4) {
        unsigned long long c[4] = {i, (unsigned long long)(d0 / 4), 0ull, 0ull};
        philox4x64_10(c, seed, 0ull);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (d0 + j < NDIM) X[d0 + j] = (W)(sizeof(W) == 8 ? c[j] : (c[j] >> 32));
    }
}

// The step from an even block q (q + 1 is odd, c = 0): a fixed word.
template <int NDIM, typename W>
__device__ __forceinline__ void sobol_step_even(W (&X)[NDIM], int li = 0)
{
#pragma unroll
    for (int d = 0; d < NDIM; ++d)
        X[d] ^= Dir<W>::w(li, d, 5);
}

// ------------------------------------------------------------ maps
// FP32 path: the 32-bit word is the top half of the 64-bit Sobol word and
// the coordinate keeps its top 23 bits; the kernels map to the centred
// coordinate z = x - 1/2 through the grid table of grid_entry_f32.
// FP64 path: 64-bit word, y keeps 52 bits, x in [0, 1].
//
// Shared-memory layout (FP32) for N = 2^L >= 32.  Writing the bin index
// k = y_1 .. y_L (the top L bits of y), bin k sits at slot
//   s = (y_6 .. y_L) * 32 + y_5 * 16 + (y_1 .. y_4),
// the top L bits of the point's mapped word (slot_perm), followed there by
// three zero bits, so the word shifted right by 29 - L is the byte offset
// 8 s of the bin's grid entry.  The 32 lanes of a warp always hold 32
// distinct 1/32-strata (y_1 .. y_5), so their slots are distinct mod 32 and
// each half-warp (Gray-code bit 4 fixed) holds 16 distinct y_1 .. y_4: the
// 8-byte grid gathers and the histogram updates are free of bank
// conflicts.  Every warp's own f^2 histogram sits at the grid's stride (a
// pair of warps shares 8-byte entries, one float each), so the same offset
// plus a per-warp constant addresses it.  Other N use slot = k.

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// 1/x: the special-function unit's reciprocal refined by one Newton step,
// r + r (1 - x r), which brings it to about half an ulp; the corner and
// product peaks raise or use it directly, so its error must not be biased.
__device__ __forceinline__ float rcp_refined(float x)
{
    const float r = rcp_approx(x);
    return __fmaf_rn(r, __fmaf_rn(-x, r, 1.0f), r);
}

// 2^x on the special-function unit (the FP32 exponential families take
// their arguments already scaled by log2 e).
__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// Packed FP32 pairs: one FFMA2 / FADD2 / FMUL2 instruction performs the
// operation on both halves of a register pair.  The FP32 pipe's rate is the
// same as for two scalar instructions, but the pair takes one issue slot, and
// the sampling pass is bound by instruction issue: the integrands' sums over
// axes go two axes per instruction, the accumulations two components.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// ------------------------------------------------------------ integrands
template <int E>
__device__ __forceinline__ float ipow(float r)
{
    // r^E by repeated squaring (E is a compile-time constant)
    float acc = 1.0f, b = r;
    int e = E;
    bool first = true;
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        if (e & 1) {
            acc = first ? b : acc * b;
            first = false;
        }
        e >>= 1;
        if (e) b *= b;
    }
    return acc;
}

// (h + l)^E for h + l carried to about twice binary32 precision: each
// product of pairs keeps its rounding error (FMA) and the cross terms,
// (ah + al)(bh + bl) = ah bh + [err(ah bh) + al bh + ah bl] + al bl, the
// last term below the pair's precision.  Returns the high part, the low
// part in lo.
__device__ __forceinline__ void mul_df(float ah, float al, float bh, float bl, float &h, float &l)
{
    h = ah * bh;
    l = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, __fmaf_rn(ah, bh, -h)));
}
template <int E>
__device__ __forceinline__ float ipow_df(float h, float l, float &lo)
{
    float ah = 1.0f, al = 0.0f, bh = h, bl = l;
    int e = E;
    bool first = true;
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        if (e & 1) {
            if (first) {
                ah = bh;
                al = bl;
            } else {
                mul_df(ah, al, bh, bl, ah, al);
            }
            first = false;
        }
        e >>= 1;
        if (e) mul_df(bh, bl, bh, bl, bh, bl);
    }
    lo = al;
    return ah;
}

// Integrand policies: where component C's family and parameters come from.
// RuntimeIntegrand reads them from the launch's parameter block (constant
// bank operands).  A policy generated for one problem returns compile-time
// constants instead, so the family dispatch folds away.
template <typename Real>
struct RuntimeIntegrand {
    static constexpr int kMode = 0;  // the integrand is evaluated in the pass
    static constexpr int kGen = 0;   // Sobol points (optionally digitally shifted)
    template <int C> __device__ __forceinline__ static int family(const GenzParams<Real> &g) { return g.family[C]; }
    __device__ __forceinline__ static int ncomp(const GenzParams<Real> &g) { return g.ncomp; }
    template <int C> __device__ __forceinline__ static Real p0(const GenzParams<Real> &g, int d) { return g.p0[C][d]; }
    template <int C> __device__ __forceinline__ static Real p1(const GenzParams<Real> &g, int d) { return g.p1[C][d]; }
    template <int C> __device__ __forceinline__ static Real q0(const GenzParams<Real> &g) { return g.q0[C]; }
    template <int C> __device__ __forceinline__ static Real q1(const GenzParams<Real> &g) { return g.q1[C]; }
    __device__ __forceinline__ static int delay(const GenzParams<Real> &g) { return g.delay; }
    __device__ __forceinline__ static int table(const MapParams &m) { return m.li; }
    __device__ __forceinline__ static bool priv(const MapParams &m) { return m.priv != 0; }
    __device__ __forceinline__ static int nbins(int n) { return n; }
};

// Pseudo-random points (Philox words per point instead of the Sobol
// recurrence) with the integrand evaluated in the pass.
template <typename Real>
struct PseudoIntegrand : RuntimeIntegrand<Real> {
    static constexpr int kGen = 2;
};

// Materialised samples (the caller's integrand): the same pass either
// stores the mapped points (MODE 1) or accumulates the caller's values
// read back from HBM (MODE 2) instead of evaluating a Genz integrand.
template <typename Real, int MODE>
struct MatIntegrand : RuntimeIntegrand<Real> {
    static constexpr int kMode = MODE;
};

// The integrand-cost knob (cv_genz.delay): a chain of dependent
// multiply-adds over the coordinates, in rounds of NDIM, z <- z/2 + x_d.
// |z| stays below 2 max |x_d|, so 0 * z is an exact zero and the value it
// is added to is unchanged; the compiler cannot drop the chain (0 * z would
// not be zero for an infinite or NaN z).
template <int NDIM, typename Real>
__device__ __forceinline__ Real delay_chain(const Real (&x)[NDIM], int n)
{
    Real z = Real(0);
    for (int j = 0; j < n; j += NDIM) {
#pragma unroll
        for (int d = 0; d < NDIM; ++d) z = fma_rn(z, Real(0.5), x[d]);
    }
    return z;
}

// s0 + sum_d w[d] z[d] for component C with w = p0 (P = 0) or p1 (P = 1):
// scalar FMAs, whose parameter operands are immediates or constant-bank
// operands (a packed instruction would need its parameter pair in
// registers), in two interleaved chains.
template <int NDIM, int C, int P, class I, class G>
__device__ __forceinline__ float axis_dot(const G &g, const float (&z)[NDIM], float s0)
{
    float a0 = s0, a1 = 0.0f;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
        const float w = P == 0 ? I::template p0<C>(g, d) : I::template p1<C>(g, d);
        if (d & 1) a1 = __fmaf_rn(w, z[d], a1);
        else a0 = __fmaf_rn(w, z[d], a0);
    }
    return a0 + a1;
}

// FP32 Genz evaluation of component C at the centred point z = x - 1/2,
// with the parameter forms of GenzParams (base-2 exponents, q0 + q1 pairs).
// Steps whose operands are all computed values (squares, the product over
// axes) go two axes per packed instruction.
template <int NDIM, int C, class I, class G>
__device__ __forceinline__ float genz_f32(const G &g, const float (&z)[NDIM])
{
    switch (I::template family<C>(g)) {
    case CV_OSCILLATORY: {
        // phase in turns: (q0 + q1) + sum p0 z, reduced to [-1/2, 1/2]
        float t = I::template q0<C>(g) + axis_dot<NDIM, C, 0, I>(g, z, I::template q1<C>(g));
        t -= rintf(t);
        return __cosf(6.28318530717958647692f * t);
    }
    case CV_PRODUCT_PEAK: {
        // prod (1/a^2 + (z - (u - 1/2))^2), then one refined reciprocal
        float q[NDIM];
#pragma unroll
        for (int d = 0; d < NDIM; ++d) {
            const float dz = z[d] + I::template p1<C>(g, d);
            q[d] = __fmaf_rn(dz, dz, I::template p0<C>(g, d));
        }
        float2 P = make_float2(q[0], NDIM > 1 ? q[NDIM > 1 ? 1 : 0] : 1.0f);
#pragma unroll
        for (int d = 2; d + 1 < NDIM; d += 2) P = mul2(P, make_float2(q[d], q[d + 1]));
        float Pr = P.x * P.y;
        if ((NDIM & 1) && NDIM > 1) Pr *= q[NDIM - 1];
        return rcp_refined(Pr);
    }
    case CV_CORNER_PEAK: {
        // s^-(NDIM+1) with s = 1 + sum a x over the uncentred x = z + 1/2.
        // Every term is non-negative, so near the corner, where f is
        // largest, the sum is small beside the 1 and its roundings are small
        // against s (the centred form 1 + sum a/2 + sum a z cancels there:
        // partial sums of size sum a/2 for an s near 1).  Every relative
        // error of s or of 1/s comes back NDIM + 1 times larger, so s is
        // carried as sh + sl to about twice binary32 precision: a = p0 + p1
        // as high and low halves, the exact products (FMA), TwoSum for the
        // additions -- each one from 9 axes on, the final 1 + t below that.
        // 1/s is r (1 + w) to first order; below 9 axes the power takes w to
        // first order, r^k (1 + k w), from 9 axes on it is a product of
        // pairs, whose roundings would otherwise add up to about k units.
        float sh, sl;
        if (NDIM >= 9) {
            sh = 1.0f;
            sl = 0.0f;
#pragma unroll
            for (int d = 0; d < NDIM; ++d) {
                const float x = z[d] + 0.5f;
                const float a = I::template p0<C>(g, d);
                const float p = a * x;
                const float pe = __fmaf_rn(a, x, -p);
                const float t1 = sh + p;
                const float bb = t1 - sh;
                sl += ((sh - (t1 - bb)) + (p - bb)) + pe;
                sl = __fmaf_rn(I::template p1<C>(g, d), x, sl);
                sh = t1;
            }
        } else {
            // the high sum in two chains
            float t0 = 0.0f, t1 = 0.0f, te = 0.0f;
#pragma unroll
            for (int d = 0; d < NDIM; ++d) {
                const float x = z[d] + 0.5f;
                if (d & 1) t1 = __fmaf_rn(I::template p0<C>(g, d), x, t1);
                else t0 = __fmaf_rn(I::template p0<C>(g, d), x, t0);
                te = __fmaf_rn(I::template p1<C>(g, d), x, te);
            }
            const float t = t0 + t1;
            sh = 1.0f + t;
            const float bb = sh - 1.0f;
            sl = ((1.0f - (sh - bb)) + (t - bb)) + te;
        }
        // 1/(sh + sl) = r (1 + w) to first order, w = (1 - sh r) - sl r
        // (the first term exact by FMA: the reciprocal's own error)
        const float r = rcp_refined(sh);
        const float w = __fmaf_rn(-sl, r, __fmaf_rn(-sh, r, 1.0f));
        if (NDIM >= 9) {
            float fl;
            const float fh = ipow_df<NDIM + 1>(r, r * w, fl);
            return fh + fl;
        }
        const float f = ipow<NDIM + 1>(r);
        return __fmaf_rn(f, (float)(NDIM + 1) * w, f);
    }
    case CV_GAUSSIAN: {
        // 2^-(sum (p0 z + p1)^2)
        float t[NDIM];
#pragma unroll
        for (int d = 0; d < NDIM; ++d) t[d] = __fmaf_rn(I::template p0<C>(g, d), z[d], I::template p1<C>(g, d));
        float2 s2 = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int d = 0; d + 1 < NDIM; d += 2) {
            const float2 tt = make_float2(t[d], t[d + 1]);
            s2 = fma2(tt, tt, s2);
        }
        if (NDIM & 1) s2.x = __fmaf_rn(t[NDIM - 1], t[NDIM - 1], s2.x);
        return ex2_approx(-(s2.x + s2.y));
    }
    case CV_C0: {
        // 2^-(sum p0 |z + p1|)
        float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
        for (int d = 0; d < NDIM; ++d) {
            const float v = __fmaf_rn(I::template p0<C>(g, d), fabsf(z[d] + I::template p1<C>(g, d)), d & 1 ? a1 : a0);
            if (d & 1) a1 = v;
            else a0 = v;
        }
        return ex2_approx(-(a0 + a1));
    }
    case CV_DISCONTINUOUS: {
        bool out = z[0] > I::template p1<C>(g, 0);
        if (NDIM > 1) out = out || (z[NDIM > 1 ? 1 : 0] > I::template p1<C>(g, NDIM > 1 ? 1 : 0));
        const float s = axis_dot<NDIM, C, 0, I>(g, z, 0.0f);
        return out ? 0.0f : I::template q0<C>(g) * ex2_approx(s);
    }
    default:
        return 1.0f;
    }
}

// FP64 Genz evaluation of component C (x in [0, 1]).
template <int NDIM, int C, class I>
__device__ __forceinline__ double genz_f64(const GenzParams<double> &g, const double (&x)[NDIM])
{
    double s = 0.0, P = 1.0;
    switch (I::template family<C>(g)) {
    case CV_OSCILLATORY:
#pragma unroll
        for (int d = 0; d < NDIM; ++d) s = __fma_rn(I::template p0<C>(g, d), x[d], s);
        return cos(I::template q0<C>(g) + s);
    case CV_PRODUCT_PEAK:
#pragma unroll
        for (int d = 0; d < NDIM; ++d) {
            const double dx = x[d] - I::template p1<C>(g, d);
            P *= 1.0 / __fma_rn(dx, dx, I::template p0<C>(g, d));
        }
        return P;
    case CV_CORNER_PEAK:
#pragma unroll
        for (int d = 0; d < NDIM; ++d) s = __fma_rn(I::template p0<C>(g, d), x[d], s);
        return pow(1.0 + s, -(double)(NDIM + 1));
    case CV_GAUSSIAN:
#pragma unroll
        for (int d = 0; d < NDIM; ++d) {
            const double dx = x[d] - I::template p1<C>(g, d);
            s = __fma_rn(I::template p0<C>(g, d) * dx, dx, s);
        }
        return exp(-s);
    case CV_C0:
#pragma unroll
        for (int d = 0; d < NDIM; ++d)
            s = __fma_rn(I::template p0<C>(g, d), fabs(x[d] - I::template p1<C>(g, d)), s);
        return exp(-s);
    case CV_DISCONTINUOUS: {
        bool out = x[0] > I::template p1<C>(g, 0);
        if (NDIM > 1) out = out || (x[NDIM > 1 ? 1 : 0] > I::template p1<C>(g, NDIM > 1 ? 1 : 0));
#pragma unroll
        for (int d = 0; d < NDIM; ++d) s = __fma_rn(I::template p0<C>(g, d), x[d], s);
        return out ? 0.0 : exp(s);
    }
    default:
        return 1.0;
    }
}

template <int NDIM, int C, class I = RuntimeIntegrand<float>>
__device__ __forceinline__ float genz_eval(const GenzParams<float> &g, const float (&x)[NDIM])
{
    return genz_f32<NDIM, C, I>(g, x);
}
template <int NDIM, int C, class I = RuntimeIntegrand<double>>
__device__ __forceinline__ double genz_eval(const GenzParams<double> &g, const double (&x)[NDIM])
{
    return genz_f64<NDIM, C, I>(g, x);
}

// ------------------------------------------------------------ sums
// FP32 path: per-thread Kahan-compensated sums, fed with plain FP32 partial
// sums over short runs of steps (blocked Kahan summation); value = s - c.
// FP64 path: plain per-thread sums.
template <typename Real> struct Acc;
template <> struct Acc<float> {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float v)
    {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};
template <> struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
};

// Warp sum of per-lane values, returned on every lane in FP64.  The FP32
// path reduces the Kahan pairs as float-float numbers (Knuth's TwoSum) so
// that FP64 arithmetic, slow on this GPU, runs once per warp.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ double warp_total(const Acc<float> &a)
{
    float hi = a.s, lo = -a.c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
        const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
        float s, e;
        two_sum(hi, ohi, s, e);
        e += lo + olo;
        hi = s + e;
        lo = e - (hi - s);
    }
    return (double)hi + (double)lo;
}

__device__ __forceinline__ double warp_total(const Acc<double> &a)
{
    double v = a.s;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------------ sampling steps
// Shared-memory views of one block.  FP64: every axis owns a stride of
// CV_MAX_BINS slots.  FP32: `stride` entries per axis (nbins, or the batch
// class's largest nbins), a compile-time constant in the specialised kernel.
constexpr int kStride = CV_MAX_BINS;

template <typename Real> struct Smem;
template <> struct Smem<float> {
    float2 *ew;        // [NDIM][stride]: grid_entry_f32 of each slot (8N-aligned)
    float *h;          // the histogram copy this warp updates: its own [NDIM][stride], or the block's
    int stride;
    // 32-bit shared-window addresses; for the power-of-two map the grid's
    // and this warp's histogram's, shifted down by 3 + L and 2 + L (both
    // bases are multiples of 8N and 4N), so one funnel shift of a point's
    // word gives the absolute address of its bin's entry
    unsigned g_sa, h_sa, g_hi, h_hi;
};
template <> struct Smem<double> {
    double2 *ew;       // [NDIM][stride] {e_k, w_k}
    double *h;         // [NDIM][hs]
    int stride, hs;
};

// How a block accumulates its FP32 f^2 histogram: one copy per warp,
// updated with plain loads and stores when the 32 lanes' bins are distinct
// (N = 2^L >= 32) or with shared atomics otherwise; or one block copy with
// shared atomics.
enum { kHistWarpPlain = 0, kHistWarpAtomic = 1, kHistBlock = 2 };

// The shared-window addresses of a block's FP32 grid and histogram copy
// (L = log2 N of the power-of-two map, else 0).
__device__ __forceinline__ void set_addresses(Smem<float> &sm, int L)
{
    sm.g_sa = (unsigned)__cvta_generic_to_shared(sm.ew);
    sm.h_sa = (unsigned)__cvta_generic_to_shared(sm.h);
    sm.g_hi = L ? sm.g_sa >> (3 + L) : 0u;
    sm.h_hi = L ? sm.h_sa >> (2 + L) : 0u;
}

// The FP32 grid table in a block's dynamic shared memory: the first
// multiple of 8N bytes (the funnel-shift addressing needs the alignment;
// the allocation has 8N bytes to spare for it).
__device__ __forceinline__ float2 *align_table(unsigned char *raw, int N)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(raw);
    const unsigned al = 8u * (unsigned)N;
    return reinterpret_cast<float2 *>(raw + ((al - a % al) % al));
}

// Shared-memory accesses through 32-bit shared-window addresses.
__device__ __forceinline__ float2 lds_f2(unsigned a)
{
    float2 v;
    asm("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ unsigned lds_u(unsigned a)
{
    unsigned v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ float lds_f(unsigned a)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
    return v;
}
// A read of a table that does not change while it is read (staged before
// a barrier): free to move and combine like any load.
__device__ __forceinline__ float lds_f_ro(unsigned a)
{
    float v;
    asm("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts_f(unsigned a, float v)
{
    asm volatile("st.shared.f32 [%0], %1;" :: "r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void reds_add_f(unsigned a, float v)
{
    asm volatile("red.shared.add.f32 [%0], %1;" :: "r"(a), "f"(v) : "memory");
}

// Map one FP32 coordinate: returns z = x - 1/2 and multiplies the
// Jacobian; `slot` receives the bin's slot (general map only: the
// power-of-two map takes it from the word again when it updates the
// histogram).
template <bool POW2>
__device__ __forceinline__ float map_f32(unsigned X, int d, int N, const MapParams &m,
                                         const Smem<float> &sm, float &J, unsigned &slot)
{
    if (POW2) {
        // X is the mapped word (table m.li): the grid entry's address from
        // one funnel shift, 2^(G-L) (1 + frac 2^-G) from the fraction's bits
        const float f1 = __uint_as_float((X & m.mF) | m.expE);
        const float2 ew = lds_f2(__funnelshift_r(X, sm.g_hi, m.sA) + (unsigned)(d * sm.stride * 8));
        J *= ew.y;
        slot = 0u;
        return __fmaf_rn(ew.y, f1, ew.x);
    } else {
        const unsigned t = (X >> 9) * (unsigned)N;
        const float f1 = __uint_as_float(0x3f800000u | (t & 0x7fffffu));  // 1 + frac
        slot = t >> 23;
        const float2 ew = lds_f2(sm.g_sa + (unsigned)((d * sm.stride + (int)slot) * 8));
        J = J * ((float)N * ew.y);
        return __fmaf_rn(ew.y, f1, ew.x);
    }
}

__device__ __forceinline__ double map_f64(unsigned long long X, int d, int N,
                                          const Smem<double> &sm, double &J, int &slot)
{
    const unsigned long long t = (X >> 12) * (unsigned long long)N;  // < 2^60
    const double frac = __longlong_as_double((long long)(0x3ff0000000000000ull |
                                                         (t & 0xfffffffffffffull))) - 1.0;
    const int p = (int)(t >> 52);
    const double2 ew = sm.ew[d * sm.stride + p];
    J = J * ((double)N * ew.y);
    slot = p;
    return __fma_rn(ew.y, frac, ew.x);
}

template <typename Real> struct Word;
template <> struct Word<float> { using type = unsigned int; };
template <> struct Word<double> { using type = unsigned long long; };

// Per-lane partial sums of a run of blocks: FP32 pairs of components
// (0, 1) and (2, 3); FP64 one value per component.
template <typename Real> struct Partial;
template <> struct Partial<float> {
    float2 s1[2], s2[2];
    __device__ __forceinline__ void zero()
    {
        s1[0] = s1[1] = s2[0] = s2[1] = make_float2(0.0f, 0.0f);
    }
    __device__ __forceinline__ float v1(int c) const { return (c & 1) ? s1[c >> 1].y : s1[c >> 1].x; }
    __device__ __forceinline__ float v2(int c) const { return (c & 1) ? s2[c >> 1].y : s2[c >> 1].x; }
};
template <> struct Partial<double> {
    double s1[CV_MAX_COMP], s2[CV_MAX_COMP];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int c = 0; c < CV_MAX_COMP; ++c) s1[c] = s2[c] = 0.0;
    }
    __device__ __forceinline__ double v1(int c) const { return s1[c]; }
    __device__ __forceinline__ double v2(int c) const { return s2[c]; }
};

// The caller's values of this lane's point in block q (materialised
// samples, accumulate mode), 0 outside [start, end).
template <int NDIM, typename Real, bool EDGE>
__device__ __forceinline__ void load_values(const SampleArgs<Real> &A, unsigned long long q,
                                            unsigned long long start, unsigned long long end, int lane,
                                            Real (&fv)[CV_MAX_COMP])
{
    const unsigned long long i = q * 32ull + (unsigned long long)lane;
    const bool valid = !EDGE || (i >= start && i < end);
    const long long j = (long long)(i - start);
    // both layouts as strides: value c of point j at f[j sj + c sc]
    const long long sj = A.aos ? A.g.ncomp : 1, sc = A.aos ? 1 : A.ld;
    const Real *fp = A.f + j * sj;
#pragma unroll
    for (int c = 0; c < CV_MAX_COMP; ++c) {
        fv[c] = Real(0);
        if (c < A.g.ncomp && valid) fv[c] = fp[c * sc];
    }
}

// Store one point for the caller's integrand (materialised samples, store
// mode): coordinate d of point j = index - start at x[j sj + d sd].
template <int NDIM, typename Real>
__device__ __forceinline__ void store_point(const SampleArgs<Real> &A, long long j, const Real (&x)[NDIM])
{
    const long long sj = A.aos ? NDIM : 1, sd = A.aos ? 1 : A.ld;
    Real *xp = A.x + j * sj;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) xp[d * sd] = x[d];
}

// Axes whose histogram bins a lane reads before it writes them back.
constexpr int kHistBatch = 4;

// One aligned 32-point block q, FP32: map, integrand, partial sums,
// histogram.  EDGE: the block may hold indices outside [start, end), which
// add nothing.  fv: the caller's values of the block (accumulate mode only).
template <int NDIM, bool POW2, bool EDGE, class I, class G>
__device__ __forceinline__ void sample_block(const SampleArgs<float> &A, const Smem<float> &sm,
                                             const unsigned (&X)[NDIM], unsigned long long q,
                                             unsigned long long start, unsigned long long end, int lane,
                                             int hmode, Partial<float> &P, const float (&fv)[CV_MAX_COMP],
                                             int delay, const G &gp)
{
    const int N = I::nbins(A.nbins);
    bool valid = true;
    if (EDGE) {
        const unsigned long long i = q * 32ull + (unsigned long long)lane;
        valid = (i >= start) && (i < end);
    }
    float z[NDIM];
    unsigned slot[NDIM];
    float J = 1.0f;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) z[d] = map_f32<POW2>(X[d], d, N, A.map, sm, J, slot[d]);
    if constexpr (I::kMode == 1) {
        // store the point (x = z + 1/2) for the caller's integrand
        if (!EDGE || valid) {
            float x[NDIM];
#pragma unroll
            for (int d = 0; d < NDIM; ++d) x[d] = z[d] + 0.5f;
            store_point<NDIM, float>(A, (long long)(q * 32ull + (unsigned long long)lane - start), x);
        }
        return;
    }
    const int ncomp = I::ncomp(gp);
    float f[CV_MAX_COMP];
    if constexpr (I::kMode == 2) {
#pragma unroll
        for (int c = 0; c < CV_MAX_COMP; ++c) f[c] = fv[c];
    } else {
        // the integrand-cost knob: delay multiply-adds per component, run
        // once per point and folded into J as J + 0 * t (exact: J is finite)
        if (delay) J += 0.0f * delay_chain<NDIM>(z, delay * ncomp);
        f[0] = genz_f32<NDIM, 0, I>(gp, z);
    }
    if (EDGE && !valid) J = 0.0f;  // (f is finite at every point of the block)
    // the f^2 histogram needs component 0 only: updated before the other
    // components are evaluated, so the bins' offsets are dead by then
    const float v0 = J * f[0];
    if (!EDGE || valid) {
        const float h = v0 * v0;
        // the bin's float in the histogram copy: one funnel shift of the
        // word (power-of-two map), or slot * 4 (general map)
        auto haddr = [&](int d) {
            return (POW2 ? __funnelshift_r(X[d], sm.h_hi, A.map.sA + 1u) : sm.h_sa + slot[d] * 4u) +
                   (unsigned)(d * sm.stride * 4);
        };
        if (hmode == kHistWarpPlain) {
            // a few axes' bins read first, then written (the axes' rows are
            // disjoint, so the reads need not wait for the writes)
#pragma unroll
            for (int d0 = 0; d0 < NDIM; d0 += kHistBatch) {
                float hv[kHistBatch];
#pragma unroll
                for (int d = d0; d < d0 + kHistBatch && d < NDIM; ++d) hv[d - d0] = lds_f(haddr(d));
#pragma unroll
                for (int d = d0; d < d0 + kHistBatch && d < NDIM; ++d) sts_f(haddr(d), hv[d - d0] + h);
            }
        } else {
#pragma unroll
            for (int d = 0; d < NDIM; ++d) reds_add_f(haddr(d), h);
        }
    }
    if constexpr (I::kMode != 2) {
        f[1] = ncomp > 1 ? genz_f32<NDIM, 1, I>(gp, z) : 0.0f;
        f[2] = ncomp > 2 ? genz_f32<NDIM, 2, I>(gp, z) : 0.0f;
        f[3] = ncomp > 3 ? genz_f32<NDIM, 3, I>(gp, z) : 0.0f;
    }
    // the partial sums of J f and (J f)^2, two components per packed
    // instruction
    const float2 v01 = make_float2(v0, J * f[1]);
    P.s1[0] = add2(P.s1[0], v01);
    P.s2[0] = fma2(v01, v01, P.s2[0]);
    if (ncomp > 2) {
        const float2 v23 = make_float2(J * f[2], J * f[3]);
        P.s1[1] = add2(P.s1[1], v23);
        P.s2[1] = fma2(v23, v23, P.s2[1]);
    }
    // the next block's reads of the warp's own copy see this block's writes
    if (hmode == kHistWarpPlain) __syncwarp();
}

// One aligned 32-point block q, FP64.
template <int NDIM, bool EDGE, class I>
__device__ __forceinline__ void sample_block(const SampleArgs<double> &A, const Smem<double> &sm,
                                             const unsigned long long (&X)[NDIM], unsigned long long q,
                                             unsigned long long start, unsigned long long end, int lane,
                                             int hmode, Partial<double> &P, const double (&fv)[CV_MAX_COMP],
                                             int delay)
{
    const int N = A.nbins;
    bool valid = true;
    if (EDGE) {
        const unsigned long long i = q * 32ull + (unsigned long long)lane;
        valid = (i >= start) && (i < end);
    }
    double x[NDIM];
    int slot[NDIM];
    double J = 1.0;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) x[d] = map_f64(X[d], d, N, sm, J, slot[d]);
    if constexpr (I::kMode == 1) {
        if (!EDGE || valid) store_point<NDIM, double>(A, (long long)(q * 32ull + (unsigned long long)lane - start), x);
        return;
    }
    const int ncomp = A.g.ncomp;
    double f0 = 0.0;
#pragma unroll
    for (int c = 0; c < CV_MAX_COMP; ++c) {
        if (c < ncomp) {
            double f;
            if constexpr (I::kMode == 2) {
                f = fv[c];
            } else {
                if (c == 0 && delay) J += 0.0 * delay_chain<NDIM>(x, delay * ncomp);
                f = c == 0 ? genz_f64<NDIM, 0, I>(A.g, x)
                  : c == 1 ? genz_f64<NDIM, 1, I>(A.g, x)
                  : c == 2 ? genz_f64<NDIM, 2, I>(A.g, x) : genz_f64<NDIM, 3, I>(A.g, x);
            }
            double v = J * f;
            if (EDGE && !valid) v = 0.0;
            P.s1[c] += v;
            P.s2[c] += v * v;
            if (c == 0) f0 = v;
        }
    }
    if (!EDGE || valid) {
        const double h = f0 * f0;
        if (hmode == kHistWarpPlain) {
            // the warp's own copy: its 32 points are in 32 distinct bins
#pragma unroll
            for (int d = 0; d < NDIM; ++d) sm.h[d * sm.hs + slot[d]] += h;
        } else {
#pragma unroll
            for (int d = 0; d < NDIM; ++d) atomicAdd(&sm.h[d * sm.hs + slot[d]], h);
        }
    }
    if (hmode == kHistWarpPlain) __syncwarp();
}

// nsteps consecutive 32-point blocks starting at block q0, every lane's
// words advanced past them.  The values are summed in FP32 (FP64) over
// runs of kRun blocks, and each run's sum is added to the per-thread
// accumulators.
//   EDGE = false: every index of the range is inside [start, end), q0 and
//   nsteps are even; the blocks go in (even, odd) pairs, and the step out
//   of an even block is the fixed word W_5.
//   EDGE = true: any range (the first and last chunks of a pass), one block
//   at a time.
constexpr unsigned kRun = 16;

// gp: where the integrand policy reads its parameters (the launch's
// GenzParams, or a register copy of one integral's).
template <int NDIM, typename Real, bool POW2, bool EDGE, class I = RuntimeIntegrand<Real>, class G = GenzParams<Real>>
__device__ __forceinline__ void run_steps(const SampleArgs<Real> &A, const Smem<Real> &sm,
                                          typename Word<Real>::type (&X)[NDIM],
                                          unsigned long long q0, unsigned nsteps,
                                          unsigned long long start, unsigned long long end,
                                          int lane, int hmode, Acc<Real> (&s1)[CV_MAX_COMP],
                                          Acc<Real> (&s2)[CV_MAX_COMP], const G &gp)
{
    using W = typename Word<Real>::type;
    const int li = (sizeof(Real) == 4 && POW2) ? I::table(A.map) : 0;  // direction table
    const unsigned per = EDGE ? 1u : 2u;  // blocks per loop trip
    const int delay = I::delay(gp);       // (read once: the integrand-cost knob)
    for (unsigned r0 = 0; r0 < nsteps; r0 += kRun) {
        const unsigned r1 = min(r0 + kRun, nsteps);
        Partial<Real> P;
        P.zero();
        for (unsigned st = r0; st < r1; st += per) {
            const unsigned long long q = q0 + st;
            // accumulate mode: both blocks' values are requested before any
            // arithmetic, so their latency overlaps the map
            Real fa[CV_MAX_COMP], fb[CV_MAX_COMP];
            if constexpr (I::kMode == 2) {
                load_values<NDIM, Real, EDGE>(A, q, start, end, lane, fa);
                if (!EDGE) load_values<NDIM, Real, EDGE>(A, q + 1, start, end, lane, fb);
            }
            auto block = [&](unsigned long long qq, const Real (&fv)[CV_MAX_COMP]) {
                if constexpr (sizeof(Real) == 4)
                    sample_block<NDIM, POW2, EDGE, I>(A, sm, X, qq, start, end, lane, hmode, P, fv, delay, gp);
                else
                    sample_block<NDIM, EDGE, I>(A, sm, X, qq, start, end, lane, hmode, P, fv, delay);
            };
            if constexpr (I::kGen == 2) {
                // pseudo-random points: fresh words for every block
                pseudo_words<NDIM, W>(X, A.seed, q * 32ull + (unsigned long long)lane);
                block(q, fa);
                if (!EDGE) {
                    pseudo_words<NDIM, W>(X, A.seed, (q + 1) * 32ull + (unsigned long long)lane);
                    block(q + 1, fb);
                }
                continue;
            }
            block(q, fa);
            if (EDGE) {
                sobol_step<NDIM, W>(X, q, li);
            } else {
                sobol_step_even<NDIM, W>(X, li);
                block(q + 1, fb);
                sobol_step<NDIM, W>(X, q + 1, li);
            }
        }
#pragma unroll
        for (int c = 0; c < CV_MAX_COMP; ++c) {
            if (c < I::ncomp(gp)) {
                s1[c].add(P.v1(c));
                s2[c].add(P.v2(c));
            }
        }
    }
}

// ------------------------------------------------------------ the kernel
// Register budget: three resident blocks of 256 threads per SM for up to 8
// FP32 dimensions (80 registers), two for 9..32 (128 registers: the batched
// kernel spills a little from 24 dimensions on, and is still 30-40% faster
// than at one block of up to 255 registers, which hides too little
// latency with 8 warps); FP64 kernels get what they need.
template <int NDIM, typename Real>
constexpr int kMinBlocks = sizeof(Real) != 4 ? 1 : (NDIM <= 8 ? 3 : 2);

// Stage an FP32 block's grid table from the FP64 edges (slot order).
__device__ __forceinline__ void stage_grid_f32(float2 *ew, int ndim, int N, int stride, const double *edges,
                                               const MapParams &map)
{
    // (by bin: coalesced reads of the FP64 grid)
    for (int idx = threadIdx.x; idx < ndim * N; idx += blockDim.x) {
        const int d = idx / N, k = idx - d * N;
        const double *e = edges + (size_t)d * (N + 1);
        ew[d * stride + slot_of_bin(k, map)] = grid_entry_f32(e[k], e[k + 1] - e[k], N, map);
    }
}

// The last block of a deterministic pass to finish adds every block's sums
// to S1, S2 in a fixed order: warp v sums value v (S1 and S2 of each
// component) over the blocks, lane l taking blocks l, l + 32, ..., then a
// fixed shuffle tree.  The ticket counts finished blocks (no block waits
// for another) and is reset for the next launch.
__device__ __forceinline__ void last_block_sums(const double *part_S, unsigned *ticket, double *S1, double *S2,
                                                int ncomp)
{
    __shared__ int s_last;
    __threadfence();  // this block's partials, before its ticket
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int lane = threadIdx.x & 31;
    for (int v = threadIdx.x >> 5; v < 2 * ncomp; v += kWarpsPerBlock) {
        double acc = 0.0;
        for (unsigned b = lane; b < gridDim.x; b += 32) acc += __ldcg(&part_S[b * (2 * CV_MAX_COMP) + v]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            double *dst = (v & 1) ? &S2[v >> 1] : &S1[v >> 1];
            *dst += acc;
        }
    }
    if (threadIdx.x == 0) *ticket = 0u;
}

// One fused sampling pass (the kernel body, shared by every specialisation).
template <int NDIM, typename Real, bool POW2, class I>
__device__ __forceinline__ void sample_pass(const SampleArgs<Real> &A)
{
    using W = typename Word<Real>::type;
    unsigned long long start;
    long long n;
    if (A.st) {
        const int stopped = *(volatile const int *)&A.st->stopped;
        if (blockIdx.x == 0 && threadIdx.x == 0) A.st->pass_active = stopped ? 0 : 1;
        if (stopped) return;
        start = A.st->next_index;
        n = A.st->n_cur;
    } else {
        start = A.start;
        n = A.n;
    }
    const int N = I::nbins(A.nbins);
    const int ncomp = A.g.ncomp;
    const bool priv = sizeof(Real) == 4 && POW2 && I::priv(A.map);
    // FP64: warp copies for Sobol points and N = 2^L >= 32 when they fit
    const bool priv64 = sizeof(Real) == 8 && I::kGen != 2 && A.map.priv != 0;
    const int hmode = (priv || priv64) ? kHistWarpPlain : kHistBlock;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<Real> sm;
    if constexpr (sizeof(Real) == 4) {
        sm.stride = N;
        sm.ew = align_table(smem_raw, N);
        float *hist = reinterpret_cast<float *>(sm.ew + NDIM * N);
        if (I::kMode != 1) {
            // the histogram copies: every warp's [NDIM][N], or the block's
            const int nh = priv ? kWarpsPerBlock * NDIM * N : NDIM * N;
            for (int i = threadIdx.x; i < nh; i += blockDim.x) hist[i] = 0.0f;
        }
        const int warp = threadIdx.x >> 5;
        sm.h = priv ? hist + warp * NDIM * N : hist;
        set_addresses(sm, POW2 ? A.map.L : 0);
        if (A.ew32) {
            // the table the refinement staged (FP64 arithmetic is slow here:
            // done once per pass there instead of once per CTA)
            for (int idx = threadIdx.x; idx < NDIM * N; idx += blockDim.x) sm.ew[idx] = A.ew32[idx];
        } else {
            stage_grid_f32(sm.ew, NDIM, N, N, A.edges, A.map);
        }
    } else {
        sm.stride = kStride;
        sm.ew = reinterpret_cast<double2 *>(smem_raw);
        double *hist = reinterpret_cast<double *>(sm.ew + NDIM * kStride);
        // the block's histogram (kStride slots per axis), or every warp's [NDIM][N]
        sm.hs = priv64 ? N : kStride;
        sm.h = priv64 ? hist + (threadIdx.x >> 5) * NDIM * N : hist;
        for (int i = threadIdx.x; i < (priv64 ? kWarpsPerBlock * NDIM * N : NDIM * kStride); i += blockDim.x)
            hist[i] = 0.0;
        for (int idx = threadIdx.x; idx < NDIM * N; idx += blockDim.x) {
            const int d = idx / N, k = idx - d * N;
            const double *e = A.edges + (size_t)d * (N + 1);
            sm.ew[d * kStride + k] = make_double2(e[k], e[k + 1] - e[k]);
        }
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    // blocks [qa, qb) cover the pass; qa and the chunk length are even, so
    // every chunk starts on an even block
    const unsigned long long qa = (start >> 5) & ~1ull;
    const unsigned long long end = start + (unsigned long long)n;
    const unsigned long long qb = (end + 31ull) >> 5;
    const unsigned long long nblk = n > 0 ? qb - qa : 0ull;
    const unsigned long long gwarp = (unsigned long long)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const unsigned long long twarps = (unsigned long long)gridDim.x * kWarpsPerBlock;
    unsigned long long plen = (nblk + twarps - 1) / twarps;
    if (plen < (unsigned long long)A.chunk_min) plen = A.chunk_min;
    // materialised samples: short chunks taken in rounds, so that at any
    // time all warps read or write within one window of the point arrays
    // (DRAM locality) instead of one long stretch each
    if (I::kMode != 0 && plen > kRun) plen = kRun;
    plen = (plen + 1ull) & ~1ull;
    const unsigned long long nchunk = (nblk + plen - 1) / plen;

    Acc<Real> s1[CV_MAX_COMP], s2[CV_MAX_COMP];

    for (unsigned long long ch = gwarp; ch < nchunk; ch += twarps) {
        const unsigned long long q0 = qa + ch * plen;
        const unsigned long long q1 = min(q0 + plen, qb);
        W X[NDIM];
        if constexpr (I::kGen != 2) {
            sobol_skip<NDIM, W>(X, q0, lane, (sizeof(Real) == 4 && POW2) ? I::table(A.map) : 0);
            if (A.gen == kGenScrambled) {
#pragma unroll
                for (int d = 0; d < NDIM; ++d) X[d] ^= (W)A.shift[d];
            }
        }
        const bool interior = (q0 * 32ull >= start) && (q1 * 32ull <= end) && !((q0 | q1) & 1ull);
        if (interior)
            run_steps<NDIM, Real, POW2, false, I>(A, sm, X, q0, (unsigned)(q1 - q0), start, end, lane, hmode, s1, s2, A.g);
        else
            run_steps<NDIM, Real, POW2, true, I>(A, sm, X, q0, (unsigned)(q1 - q0), start, end, lane, hmode, s1, s2, A.g);
    }

    if constexpr (I::kMode == 1) return;  // points stored: nothing to reduce

    // Reduction: warp, then across the block's warps in FP64.
    __shared__ double red[kWarpsPerBlock][2 * CV_MAX_COMP];
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < CV_MAX_COMP; ++c) {
        if (c < ncomp) {
            const double a = warp_total(s1[c]);
            const double b = warp_total(s2[c]);
            if (lane == 0) {
                red[warp][2 * c] = a;
                red[warp][2 * c + 1] = b;
            }
        }
    }
    __syncthreads();
    const bool parts = A.part_S != nullptr;
    if (threadIdx.x < 2 * ncomp) {
        double t = 0.0;
        for (int w = 0; w < kWarpsPerBlock; ++w) t += red[w][threadIdx.x];
        const int c = threadIdx.x >> 1;
        if (parts) A.part_S[blockIdx.x * (2 * CV_MAX_COMP) + threadIdx.x] = t;
        else atomicAdd((threadIdx.x & 1) ? &A.S2[c] : &A.S1[c], t);
    }
    // (by bin: the FP64 atomics of a warp go to consecutive addresses,
    // which the L2 merges; every block flushes at about the same time)
    Real *ph = parts ? reinterpret_cast<Real *>(A.part_H) + (size_t)blockIdx.x * NDIM * N : nullptr;
    for (int idx = threadIdx.x; idx < NDIM * N; idx += blockDim.x) {
        const int d = idx / N;
        const int k = idx - d * N;
        Real v;
        if constexpr (sizeof(Real) == 4) {
            const int p = slot_of_bin(k, A.map);
            const float *hist = reinterpret_cast<const float *>(sm.ew + NDIM * N);
            if (priv) {
                // the warps' copies, summed in warp order
                v = 0.0f;
#pragma unroll
                for (int w = 0; w < kWarpsPerBlock; ++w) v += hist[(w * NDIM + d) * N + p];
            } else {
                v = hist[d * N + p];
            }
        } else if (priv64) {
            // the warps' copies, summed in warp order
            const double *hist = reinterpret_cast<const double *>(sm.ew + NDIM * kStride);
            v = 0.0;
#pragma unroll
            for (int w = 0; w < kWarpsPerBlock; ++w) v += hist[(w * NDIM + d) * N + k];
        } else {
            v = sm.h[d * kStride + k];
        }
        if (parts) ph[d * N + k] = v;
        else if (v != Real(0)) atomicAdd(&A.H[d * N + k], (double)v);
    }
    if (parts && A.part_ticket) last_block_sums(A.part_S, A.part_ticket, A.S1, A.S2, ncomp);
}

template <int NDIM, typename Real, bool POW2>
__global__ void __launch_bounds__(kBlock, (kMinBlocks<NDIM, Real>))
k_sample(const __grid_constant__ SampleArgs<Real> A)
{
    sample_pass<NDIM, Real, POW2, RuntimeIntegrand<Real>>(A);
}

// The pass with pseudo-random points (CV_PSEUDO), on the generic map.
template <int NDIM, typename Real>
__global__ void __launch_bounds__(kBlock, (kMinBlocks<NDIM, Real>))
k_sample_pseudo(const __grid_constant__ SampleArgs<Real> A)
{
    sample_pass<NDIM, Real, false, PseudoIntegrand<Real>>(A);
}

// ------------------------------------------------------------ batched kernel
// A batched tile's single-component integral: its parameters held in
// registers for the tile's loop (read once from the staged description).
template <int NDIM>
struct TileRegs {
    float p0[NDIM], p1[NDIM];
    float q0, q1;
    int delay;
};

// The policy of one single-component integral of family F (a batched
// tile's integral): family, component count and the loop over components
// are compile-time; the parameters come from a TileRegs.
template <int F>
struct TileIntegrand {
    static constexpr int kMode = 0;
    static constexpr int kGen = 0;
    template <int C, class G> __device__ __forceinline__ static constexpr int family(const G &)
    {
        return C == 0 ? F : CV_CONST;
    }
    template <class G> __device__ __forceinline__ static constexpr int ncomp(const G &) { return 1; }
    template <int C, class G> __device__ __forceinline__ static float p0(const G &g, int d) { return g.p0[d]; }
    template <int C, class G> __device__ __forceinline__ static float p1(const G &g, int d) { return g.p1[d]; }
    template <int C, class G> __device__ __forceinline__ static float q0(const G &g) { return g.q0; }
    template <int C, class G> __device__ __forceinline__ static float q1(const G &g) { return g.q1; }
    template <class G> __device__ __forceinline__ static int delay(const G &g) { return g.delay; }
    __device__ __forceinline__ static int table(const MapParams &m) { return m.li; }
    __device__ __forceinline__ static bool priv(const MapParams &m) { return m.priv != 0; }
    __device__ __forceinline__ static int nbins(int n) { return n; }
};

// Dimension counts up to which the batched kernel evaluates single-component
// integrals through TileIntegrand (the build compiles six more loops per
// dimension count; the 17-32 dimension classes keep the general policy).
constexpr int kTileSpecMaxDim = 16;

// A warp's share of a batched tile: single-component integrals of the six
// Genz families through their own policy, anything else through the
// run-time one (parameters read from the staged description).  Both give
// the same values: the same operations on the same parameters.
template <int NDIM, bool POW2, bool EDGE>
__device__ __forceinline__ void batch_steps(const SampleArgs<float> &A, const Smem<float> &sm, unsigned (&X)[NDIM],
                                            unsigned long long w0, unsigned nsteps, unsigned long long start,
                                            unsigned long long end, int lane, int hmode,
                                            Acc<float> (&s1)[CV_MAX_COMP], Acc<float> (&s2)[CV_MAX_COMP])
{
    if constexpr (NDIM <= kTileSpecMaxDim) {
        const int fam = A.g.family[0];
        if (A.g.ncomp == 1 && fam >= 0 && fam < CV_CONST) {
            TileRegs<NDIM> tr;
#pragma unroll
            for (int d = 0; d < NDIM; ++d) {
                tr.p0[d] = A.g.p0[0][d];
                tr.p1[d] = A.g.p1[0][d];
            }
            tr.q0 = A.g.q0[0];
            tr.q1 = A.g.q1[0];
            tr.delay = A.g.delay;
            switch (fam) {
#define CV_TILE_FAMILY(F)                                                                                   \
    case F:                                                                                                 \
        run_steps<NDIM, float, POW2, EDGE, TileIntegrand<F>>(A, sm, X, w0, nsteps, start, end, lane, hmode, \
                                                             s1, s2, tr);                                  \
        return;
                CV_TILE_FAMILY(CV_OSCILLATORY)
                CV_TILE_FAMILY(CV_PRODUCT_PEAK)
                CV_TILE_FAMILY(CV_CORNER_PEAK)
                CV_TILE_FAMILY(CV_GAUSSIAN)
                CV_TILE_FAMILY(CV_C0)
                CV_TILE_FAMILY(CV_DISCONTINUOUS)
#undef CV_TILE_FAMILY
            default: break;
            }
        }
    }
    run_steps<NDIM, float, POW2, EDGE>(A, sm, X, w0, nsteps, start, end, lane, hmode, s1, s2, A.g);
}

// Persistent sampling over a queue of tiles of many integrals (one
// dimension class per launch).  A CTA takes the next tile from a device
// counter, stages the tile's integral (grid and parameters) when it differs
// from the last one, and splits the tile's 32-point blocks over its warps.
// Every warp accumulates its own copy of the f^2 histogram, and after each
// tile the copies are summed in warp order and written as the tile's
// partial row (or, without partial rows, added to the integral's FP64
// histogram): the sums of a tile never depend on which CTA ran it or on
// what else was in the queue, and the rows are added in tile order, so an
// integral gives the same result alone and in any mix, bit for bit.
template <int NDIM, bool POW2>
__global__ void __launch_bounds__(kBlock, (kMinBlocks<NDIM, float>))
k_batch_sample(const BatchSampleArgs B)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int stride = B.stride;
    Smem<float> sm;
    sm.stride = stride;
    sm.ew = align_table(smem_raw, stride);
    float *hist = reinterpret_cast<float *>(sm.ew + NDIM * stride);  // [kWarpsPerBlock][NDIM][stride]
    __shared__ __align__(16) SampleArgs<float> A;
    __shared__ int s_tile;
    __shared__ double red[kWarpsPerBlock][2 * CV_MAX_COMP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int hsize = NDIM * stride;  // floats per warp copy
    sm.h = hist + warp * hsize;
    for (int i = threadIdx.x; i < kWarpsPerBlock * hsize; i += blockDim.x) hist[i] = 0.0f;
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(B.counter, 1);
        __syncthreads();
        const int t = s_tile;
        if (t >= B.ntiles) break;
        const Tile tile = B.tiles[t];
        const BatchItem &it = B.items[tile.item];
        if (*(volatile const int *)&it.st->stopped) {
            __syncthreads();
            continue;
        }
        if (tile.item != cur) {
            // stage the integral's parameters and grid
            const int *src = reinterpret_cast<const int *>(&it.a);
            int *dst = reinterpret_cast<int *>(&A);
            for (int i = threadIdx.x; i < (int)(sizeof(SampleArgs<float>) / sizeof(int)); i += blockDim.x)
                dst[i] = src[i];
            __syncthreads();
            stage_grid_f32(sm.ew, NDIM, A.nbins, stride, it.edges, A.map);
            // (the grid and histogram bases are multiples of 8 stride and
            // 4 stride, stride a multiple of this integral's N)
            set_addresses(sm, POW2 ? A.map.L : 0);
            cur = tile.item;
            __syncthreads();
        }
        const unsigned long long start = it.st->next_index;
        const unsigned long long end = start + (unsigned long long)it.st->n_cur;
        Acc<float> s1[CV_MAX_COMP], s2[CV_MAX_COMP];
        // (an even share, so that warps start on even blocks of an even tile)
        const unsigned per = ((((unsigned)tile.nblk + kWarpsPerBlock - 1) / kWarpsPerBlock) + 1u) & ~1u;
        const unsigned long long w0 = tile.q0 + (unsigned long long)warp * per;
        const unsigned long long w1 = min(w0 + per, tile.q0 + (unsigned long long)tile.nblk);
        const int hmode = A.map.priv ? kHistWarpPlain : kHistWarpAtomic;
        if (w0 < w1) {
            unsigned X[NDIM];
            sobol_skip<NDIM, unsigned>(X, w0, lane, POW2 ? A.map.li : 0);
            if (A.gen == kGenScrambled) {
#pragma unroll
                for (int d = 0; d < NDIM; ++d) X[d] ^= (unsigned)A.shift[d];
            }
            const bool interior = (w0 * 32ull >= start) && (w1 * 32ull <= end) && !((w0 | w1) & 1ull);
            if (interior)
                batch_steps<NDIM, POW2, false>(A, sm, X, w0, (unsigned)(w1 - w0), start, end, lane, hmode, s1, s2);
            else
                batch_steps<NDIM, POW2, true>(A, sm, X, w0, (unsigned)(w1 - w0), start, end, lane, hmode, s1, s2);
        }
        const int ncomp = A.g.ncomp;
#pragma unroll
        for (int c = 0; c < CV_MAX_COMP; ++c) {
            if (c < ncomp) {
                const double a = warp_total(s1[c]);
                const double b = warp_total(s2[c]);
                if (lane == 0) {
                    red[warp][2 * c] = a;
                    red[warp][2 * c + 1] = b;
                }
            }
        }
        __syncthreads();
        // the tile's sums and histogram: its partial rows (part_S), else
        // FP64 atomics into the integral's state
        if (threadIdx.x < 2 * ncomp) {
            double v = 0.0;
            for (int w = 0; w < kWarpsPerBlock; ++w) v += red[w][threadIdx.x];
            const int c = threadIdx.x >> 1;
            if (B.part_S) B.part_S[(size_t)tile.row * (2 * CV_MAX_COMP) + threadIdx.x] = v;
            else atomicAdd((threadIdx.x & 1) ? &it.st->S2[c] : &it.st->S1[c], v);
        }
        // (warp copies summed in warp order, then cleared)
        const int N = A.nbins;
        float *ph = B.part_S ? B.part_H + tile.hoff : nullptr;
        for (int idx = threadIdx.x; idx < NDIM * N; idx += blockDim.x) {
            const int d = idx / N, sl = idx - d * N;  // (by slot: conflict-free)
            const int p = d * stride + sl;
            float v = 0.0f;
#pragma unroll
            for (int w = 0; w < kWarpsPerBlock; ++w) {
                float &e = hist[w * hsize + p];
                v += e;
                e = 0.0f;
            }
            if (ph) ph[d * N + bin_of_slot(sl, A.map)] = v;
            else if (v != 0.0f) atomicAdd(&it.H[d * N + bin_of_slot(sl, A.map)], (double)v);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ materialised samples
// The two halves of a pass whose integrand is the caller's, both the fused
// pass with a different integrand policy: MODE 1 writes the mapped points
// (dimension-major: each warp store covers 32 consecutive points, fully
// coalesced; or the paper's point-major layout), MODE 2 reads the caller's
// values back and accumulates them, recomputing each point's bins and
// Jacobian from its Sobol index -- nothing but x and f goes through HBM.
template <int NDIM, typename Real, bool POW2, int MODE>
__global__ void __launch_bounds__(kBlock, (kMinBlocks<NDIM, Real>))
k_matpass(const __grid_constant__ SampleArgs<Real> A)
{
    sample_pass<NDIM, Real, POW2, MatIntegrand<Real, MODE>>(A);
}

// ---- materialised samples, FP32, dimension-major, N = 2^L >= 32
// The two passes of the common case as kernels of their own: the store
// pass is bound by HBM writes and the accumulate pass by its reads, so both
// keep to the instructions the point needs (no integrand, no runtime
// layout or component loops).

// Asynchronous 4-byte copies global -> shared (cp.async; bytes = 0 copies
// nothing and writes a zero), grouped, and the wait for all but the newest
// N groups of this thread.
__device__ __forceinline__ void cp_async4(unsigned dst, const void *src, unsigned bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async4_full(unsigned dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// Funnel shift right by a compile-time amount: the low word of (hi:lo) >>
// SH, one instruction (the compiler would split a constant-amount funnel
// shift into several).
template <unsigned SH>
__device__ __forceinline__ unsigned funnel_r(unsigned lo, unsigned hi)
{
    unsigned r;
    asm("shf.r.wrap.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(lo), "r"(hi), "n"(SH));
    return r;
}
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Blocks of values the accumulate pass has requested ahead of the one it
// works on (each a warp's 32 points x CV_MAX_COMP values), and its resident
// CTAs per SM (two: 128 registers, so a block's bins can all be read before
// they are written; the ring keeps 16 warps x 8 blocks of values in flight).
constexpr int kMatAhead = 8;
constexpr int kMatAccumBlocks = 2;
// Blocks per unrolled group of the accumulate pass (its chunks start on
// multiples of it, so the Gray-code steps inside a group are known in
// advance).
constexpr int kMatGroup = 8;

// The grid table of a materialised pass in a block's shared memory: the
// staged table when there is one, else converted from the FP64 edges.
template <int NDIM>
__device__ __forceinline__ void mat_table(const SampleArgs<float> &A, Smem<float> &sm, unsigned char *raw, int N)
{
    sm.stride = N;
    sm.ew = align_table(raw, N);
    if (A.ew32) {
        for (int idx = threadIdx.x; idx < NDIM * N; idx += blockDim.x) sm.ew[idx] = A.ew32[idx];
    } else {
        stage_grid_f32(sm.ew, NDIM, N, N, A.edges, A.map);
    }
}

// Trailing zero bits of a nonzero constant (a loop, not a recursion, so
// that a call with an unrolled loop's counter is inlined and folded).
__host__ __device__ constexpr int ctz_const(unsigned v)
{
    int c = 0;
    while (!(v & 1u)) {
        v >>= 1;
        ++c;
    }
    return c;
}

// The bit-level map's constants for N = 2^L as compile-time values (the
// same formulas as the host's make_map).
template <int L>
struct Pow2Map {
    static constexpr int N = 1 << L;
    static constexpr int top = 28 - L < 22 ? 28 - L : 22;
    static constexpr int F = 23 - L;
    static constexpr int G = 22 - top;
    static constexpr unsigned mF = ((1u << F) - 1u) << (top - F + 1);
    static constexpr unsigned expE = (unsigned)(127 + G - L) << 23;
    static constexpr int li = L - 4;
    static constexpr unsigned sA = 29 - L;
};

// Store pass: the points of indices [start, start + n) at x[d ld + j],
// j = index - start.  A warp writes 32 consecutive j of a tile aligned in
// j (one full 128-byte line per coordinate when x and ld are aligned), so
// its lanes' indices straddle two aligned Sobol blocks whenever start is
// not a multiple of 32: every lane steps its words by the Gray-code rule
// for its own block, g(32(q+1)+k) ^ g(32q+k) = 2^4 ^ 2^(5 + ctz(q+1)).  Of
// the two blocks a step leaves, one is even (step word W_5 of the axis, held
// in a register) and one odd (its word index the same for the whole warp:
// one constant-bank load), so no lane reads a table in shared memory.
// Tiles go to warps in rounds of kRun so that all warps
// write within one window of x at a time.  N = 2^L at compile time: table
// offsets and map constants are immediates.
template <int NDIM, int L>
__global__ void __launch_bounds__(kBlock, (kMinBlocks<NDIM, float>))
k_mat_store(const __grid_constant__ SampleArgs<float> A)
{
    using P = Pow2Map<L>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned sx0[kWarpsPerBlock][NDIM][32];
    Smem<float> sm;
    mat_table<NDIM>(A, sm, smem_raw, P::N);
    sm.h = nullptr;
    set_addresses(sm, L);
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const long long n = A.n;
    const long long ntile = (n + 31) / 32;
    const long long gwarp = (long long)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const long long twarps = (long long)gridDim.x * kWarpsPerBlock;
    constexpr int kSub = (int)kRun;  // tiles per sub-chunk (the unrolled loop)
    // one chunk of consecutive tiles per warp (one skip-ahead each, an even
    // share), walked in sub-chunks
    const long long per = max(1ll, (ntile + twarps - 1) / twarps);
    const long long nchunk = (ntile + per - 1) / per;
    const long long ld = A.ld;
    const unsigned g_hi = sm.g_hi;
    unsigned *x0s = &sx0[threadIdx.x >> 5][0][lane];  // this lane's running words, stride 32
    // this lane's index lies one block past lane 0's (start is not a multiple of 32)
    const bool inB = (unsigned)(A.start & 31ull) + (unsigned)lane >= 32u;
    for (long long ch = gwarp; ch < nchunk; ch += twarps) {
        // the chunk's first words: lane 0's block qw holds this lane's index
        // at offset k (carry 0) or the next block does (carry 1); the high
        // part of the skip-ahead is the same for the whole warp
        const unsigned long long iw = A.start + (unsigned long long)(ch * per * 32);
        const unsigned long long qw = iw >> 5;
        const unsigned kofs = (unsigned)(iw & 31ull) + (unsigned)lane;
        {
            unsigned X[NDIM];
            sobol_skip<NDIM, unsigned>(X, qw, (int)(kofs & 31u), P::li);
            const int cw = min(__ffsll((long long)(qw + 1ull)) - 1, CV_SOBOL_BITS - 6);
#pragma unroll
            for (int d = 0; d < NDIM; ++d) {
                unsigned x = X[d];
                if (kofs >= 32u) x ^= Dir<unsigned>::w(P::li, d, 5 + cw);
                if (A.gen == kGenScrambled) x ^= (unsigned)A.shift[d];
                x0s[d * 32] = x;
            }
        }
        const long long tend = min(ntile, (ch + 1) * per);
        for (long long t0 = ch * per; t0 < tend; t0 += kSub) {
            const long long j0 = t0 * 32 + lane;
            const int nt = (int)min((long long)kSub, tend - t0);
            // this lane's point of tile tt exists while tt < nv
            const long long r = n - j0;
            const int nv = r <= 0 ? 0 : (int)min((long long)nt, (r + 31) / 32);
            const bool full = nt == kSub && (t0 + kSub) * 32 <= n;  // (every lane's point of every tile)
            // the step after tile tt: lane 0's block is qa + tt, this lane's
            // qa + tt + inB; the odd one of the two steps with word index
            // kk[tt] = 5 + ctz(odd block + 1), the even one with 5
            const unsigned long long qa = (A.start + (unsigned long long)(t0 * 32)) >> 5;
            int kk[kSub];
#pragma unroll
            for (int tt = 0; tt < kSub; ++tt) {
                const unsigned long long b = (qa + (unsigned long long)tt) | 1ull;
                kk[tt] = 5 + min(__ffsll((long long)(b + 1ull)) - 1, CV_SOBOL_BITS - 6);
            }
            // this lane's block at tile 0 is odd (then at tile tt iff tt is even)
            const bool odd0 = ((qa + (inB ? 1ull : 0ull)) & 1ull) != 0ull;
            // one axis at a time: its row of x, kSub tiles of 32 points; the
            // words after the last tile start the next sub-chunk
            if (full) {
#pragma unroll 1
                for (int d = 0; d < NDIM; ++d) {
                    unsigned X = x0s[d * 32];
                    float *px = A.x + d * ld + j0;
                    const unsigned gd = g_hi + (unsigned)d;  // (table base of axis d >> (3 + L))
                    const unsigned w5 = Dir<unsigned>::w(P::li, d, 5);
#pragma unroll
                    for (int tt = 0; tt < kSub; ++tt) {
                        const float f1 = __uint_as_float((X & P::mF) | P::expE);
                        const float2 ew = lds_f2(funnel_r<P::sA>(X, gd));
                        const float z = __fmaf_rn(ew.y, f1, ew.x);
                        px[32 * tt] = z + 0.5f;
                        const unsigned wo = Dir<unsigned>::w(P::li, d, kk[tt]);
                        X ^= (odd0 == ((tt & 1) == 0)) ? wo : w5;
                    }
                    x0s[d * 32] = X;
                }
            } else {
#pragma unroll 1
                for (int d = 0; d < NDIM; ++d) {
                    unsigned X = x0s[d * 32];
                    float *px = A.x + d * ld + j0;
                    const unsigned gd = g_hi + (unsigned)d;
                    const unsigned w5 = Dir<unsigned>::w(P::li, d, 5);
#pragma unroll
                    for (int tt = 0; tt < kSub; ++tt) {
                        if (tt < nt) {
                            const float f1 = __uint_as_float((X & P::mF) | P::expE);
                            const float2 ew = lds_f2(funnel_r<P::sA>(X, gd));
                            const float z = __fmaf_rn(ew.y, f1, ew.x);
                            if (tt < nv) px[32 * tt] = z + 0.5f;
                            const unsigned wo = Dir<unsigned>::w(P::li, d, kk[tt]);
                            X ^= (odd0 == ((tt & 1) == 0)) ? wo : w5;
                        }
                    }
                    x0s[d * 32] = X;
                }
            }
        }
    }
}

// One block of the accumulate pass on its values f (stage of the ring):
// the Jacobian from the bins' widths (sm.g_hi: the float table of the
// widths N w_k, its base >> (2 + L)), the warp's histogram, the partial
// sums.  valid = 0 makes the block's points add nothing.
template <int NDIM, int L>
__device__ __forceinline__ void mat_accum_block(const Smem<float> &sm, const unsigned (&X)[NDIM], unsigned stage,
                                                int ncomp, float valid, Partial<float> &Pt)
{
    using P = Pow2Map<L>;
    float f[CV_MAX_COMP];
#pragma unroll
    for (int c = 0; c < CV_MAX_COMP; ++c) f[c] = c < ncomp ? lds_f(stage + (unsigned)(c * 128)) : 0.0f;
    // J = valid prod_d N w_d as a pairwise product (a dependent chain of
    // log2 NDIM multiplies instead of NDIM)
    float w[NDIM];
#pragma unroll
    for (int d = 0; d < NDIM; ++d) w[d] = lds_f_ro(funnel_r<P::sA + 1u>(X[d], sm.g_hi + (unsigned)d));
#pragma unroll
    for (int h = 1; h < NDIM; h <<= 1) {
#pragma unroll
        for (int d = 0; d + h < NDIM; d += 2 * h) w[d] *= w[d + h];
    }
    const float J = valid * w[0];
    const float v0 = J * f[0];
    const float h = v0 * v0;
    // the bins of up to eight axes read first, then written (the axes'
    // rows are disjoint, so the reads need not wait for the writes)
#pragma unroll
    for (int d0 = 0; d0 < NDIM; d0 += 8) {
        float hv[8];
#pragma unroll
        for (int d = d0; d < d0 + 8 && d < NDIM; ++d)
            hv[d - d0] = lds_f(funnel_r<P::sA + 1u>(X[d], sm.h_hi + (unsigned)d));
#pragma unroll
        for (int d = d0; d < d0 + 8 && d < NDIM; ++d)
            sts_f(funnel_r<P::sA + 1u>(X[d], sm.h_hi + (unsigned)d), hv[d - d0] + h);
    }
    const float2 v01 = make_float2(v0, J * f[1]);
    Pt.s1[0] = add2(Pt.s1[0], v01);
    Pt.s2[0] = fma2(v01, v01, Pt.s2[0]);
    if (ncomp > 2) {
        const float2 v23 = make_float2(J * f[2], J * f[3]);
        Pt.s1[1] = add2(Pt.s1[1], v23);
        Pt.s2[1] = fma2(v23, v23, Pt.s2[1]);
    }
    __syncwarp();
}

__device__ __forceinline__ void mat_fold(Partial<float> &Pt, int ncomp, Acc<float> (&s1)[CV_MAX_COMP],
                                         Acc<float> (&s2)[CV_MAX_COMP])
{
#pragma unroll
    for (int c = 0; c < CV_MAX_COMP; ++c) {
        if (c < ncomp) {
            s1[c].add(Pt.v1(c));
            s2[c].add(Pt.v2(c));
        }
    }
    Pt.zero();
}

// Trailing zero bits of v != 0, as a call (a boundary the compiler does not
// schedule across).
static __device__ __noinline__ int ctz_call(unsigned v) { return __ffs((int)v) - 1; }

// The Gray-code word of the step out of block kk (< kMatGroup - 1) of a
// group: 5 + ctz(kk + 1).  Up to 16 dimensions a compile-time constant (the
// words are constant-bank operands); beyond, from a call, so that the
// compiler does not interleave the group's blocks and keep every axis's
// words in registers (measured: 24 to 32 dimensions spill more without it).
template <int NDIM>
__device__ __forceinline__ int group_step_word(int kk)
{
    if constexpr (NDIM <= 16) return 5 + ctz_const((unsigned)(kk + 1));
    else return 5 + ctz_call((unsigned)(kk + 1));
}

// One chunk of the accumulate pass: blocks q0 .. q0 + nk - 1 (q0 a multiple
// of kMatGroup).  EDGE = false: every lane's point of every block is in
// [start, start + n) and nk is a multiple of kMatGroup; EDGE = true: any
// chunk, points outside add nothing.  The values of block k + kMatAhead are
// requested while block k is worked on: asynchronous copies into the warp's
// ring (each lane copies and later reads only its own words; points outside
// copy zeros).  Plain FP32 partial sums over runs of kRun blocks are folded
// into the per-thread Kahan sums after each run (as in the fused pass).
template <int NDIM, int L, bool EDGE>
__device__ __forceinline__ void mat_accum_chunk(const SampleArgs<float> &A, const Smem<float> &sm,
                                                unsigned long long q0, int nk, int lane, unsigned ring,
                                                int ncomp, Acc<float> (&s1)[CV_MAX_COMP],
                                                Acc<float> (&s2)[CV_MAX_COMP])
{
    using P = Pow2Map<L>;
    constexpr unsigned kStage = CV_MAX_COMP * 32 * 4;  // bytes of one block's values in the ring
    Partial<float> Pt;
    Pt.zero();
    const long long ld = A.ld;
    const long long j0 = (long long)(q0 * 32ull + (unsigned long long)lane) - (long long)A.start;
    unsigned X[NDIM];
    sobol_skip<NDIM, unsigned>(X, q0, lane, P::li);
    if (A.gen == kGenScrambled) {
#pragma unroll
        for (int d = 0; d < NDIM; ++d) X[d] ^= (unsigned)A.shift[d];
    }
    if constexpr (!EDGE) {
        static_assert(kMatAhead == kMatGroup, "one ring stage per block of a group");
        // this lane's values of the group's blocks: component c of block
        // k0 + kk at pv[c] + 32 kk (the pointers advance by a group)
        const float *pv[CV_MAX_COMP];
#pragma unroll
        for (int c = 0; c < CV_MAX_COMP; ++c) pv[c] = A.f + j0 + c * ld;
#pragma unroll
        for (int kk = 0; kk < kMatGroup; ++kk) {
#pragma unroll
            for (int c = 0; c < CV_MAX_COMP; ++c)
                if (c < ncomp) cp_async4_full(ring + kk * kStage + (unsigned)(c * 128), pv[c] + 32 * kk);
            cp_async_commit();
        }
        // groups of kMatGroup blocks from multiples of kMatGroup: the step
        // out of block q0 + 8 m + kk flips Gray-code bits 4 and 5 +
        // ctz(kk + 1), a word known at compile time (a constant-bank
        // operand), except the step out of a group's last block (ctz >= 3:
        // read at run time); block kk of the next group is requested into
        // the stage block kk has just left
        for (int k0 = 0; k0 < nk; k0 += kMatGroup) {
            const bool more = k0 + kMatGroup < nk;
#pragma unroll
            for (int c = 0; c < CV_MAX_COMP; ++c) pv[c] += 32 * kMatGroup;
#pragma unroll
            for (int kk = 0; kk < kMatGroup; ++kk) {
                cp_async_wait<kMatAhead - 1>();  // (block k0 + kk's copies have landed)
                mat_accum_block<NDIM, L>(sm, X, ring + kk * kStage, ncomp, 1.0f, Pt);
                if (kk + 1 < kMatGroup) {
#pragma unroll
                    {
                        const int k = group_step_word<NDIM>(kk);
#pragma unroll
                        for (int d = 0; d < NDIM; ++d) X[d] ^= Dir<unsigned>::w(P::li, d, k);
                    }
                } else if (more) {
                    sobol_step<NDIM, unsigned>(X, q0 + (unsigned long long)(k0 + kk), P::li);
                }
                if (more) {
#pragma unroll
                    for (int c = 0; c < CV_MAX_COMP; ++c)
                        if (c < ncomp) cp_async4_full(ring + kk * kStage + (unsigned)(c * 128), pv[c] + 32 * kk);
                }
                cp_async_commit();
            }
            if (((k0 + kMatGroup) % (int)kRun) == 0) mat_fold(Pt, ncomp, s1, s2);
        }
    } else {
        // this lane's point of block k is j0 + 32 k, valid for k in [klo, khi)
        const int klo = j0 >= 0 ? 0 : (int)((31 - j0) / 32);
        const long long r = A.n - j0;
        const int khi = r <= 0 ? 0 : (int)min((long long)nk, (r + 31) / 32);
        const float *pf = A.f + j0;  // (dereferenced at valid k only)
        auto request = [&](int k) {
            const unsigned stage = ring + (unsigned)((k & (kMatAhead - 1)) * kStage);
            const bool v = k >= klo && k < khi;
            const float *src = v ? pf + 32 * k : A.f;
#pragma unroll
            for (int c = 0; c < CV_MAX_COMP; ++c)
                if (c < ncomp) cp_async4(stage + (unsigned)(c * 128), src + c * ld, v ? 4u : 0u);
            cp_async_commit();
        };
        auto block = [&](int k) {
            cp_async_wait<kMatAhead - 1>();
            mat_accum_block<NDIM, L>(sm, X, ring + (unsigned)((k & (kMatAhead - 1)) * kStage), ncomp,
                                     (k >= klo && k < khi) ? 1.0f : 0.0f, Pt);
        };
#pragma unroll
        for (int k = 0; k < kMatAhead; ++k) request(k);
        for (int k = 0; k < nk; k += 2) {
            block(k);
            sobol_step_even<NDIM, unsigned>(X, P::li);
            request(k + kMatAhead);
            if (k + 1 >= nk) break;
            block(k + 1);
            sobol_step<NDIM, unsigned>(X, q0 + (unsigned long long)(k + 1), P::li);
            request(k + 1 + kMatAhead);
            if (((k + 2) % (int)kRun) == 0) mat_fold(Pt, ncomp, s1, s2);
        }
    }
    mat_fold(Pt, ncomp, s1, s2);
    cp_async_wait<0>();  // (the ring is reused by the next chunk)
}

// Accumulate pass: the caller's values f[c ld + j] of the points of
// [start, start + n), with every point's bins and Jacobian recomputed from
// its Sobol words in aligned 32-index blocks (lane = the index's low five
// bits), so each warp's f^2 histogram copy takes plain updates (the 32
// lanes' bins are distinct); sums and histogram as the fused pass.  N = 2^L
// at compile time.
template <int NDIM, int L>
__global__ void __launch_bounds__(kBlock, kMatAccumBlocks)
k_mat_accum(const __grid_constant__ SampleArgs<float> A)
{
    using P = Pow2Map<L>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ncomp = A.g.ncomp;
    // The pass needs only the bins' widths: a float table of N w_k per axis
    // (the lanes of a block read 32 distinct slots, so a read is one
    // wavefront, against two for the {e, w} pairs), then the warps' copies.
    float *wt = reinterpret_cast<float *>(align_table(smem_raw, P::N));
    float *hist = wt + NDIM * P::N;
    if (A.ew32) {
        for (int i = threadIdx.x; i < NDIM * P::N; i += blockDim.x) wt[i] = A.ew32[i].y;
    } else {
        // (converted from the FP64 edges in the histograms' space first)
        float2 *tmp = reinterpret_cast<float2 *>(hist);
        stage_grid_f32(tmp, NDIM, P::N, P::N, A.edges, A.map);
        __syncthreads();
        for (int i = threadIdx.x; i < NDIM * P::N; i += blockDim.x) wt[i] = tmp[i].y;
        __syncthreads();
    }
    for (int i = threadIdx.x; i < kWarpsPerBlock * NDIM * P::N; i += blockDim.x) hist[i] = 0.0f;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Smem<float> sm;
    sm.ew = reinterpret_cast<float2 *>(wt);
    sm.stride = P::N;
    sm.h = hist + warp * NDIM * P::N;
    set_addresses(sm, L);
    // (the width table's base >> (2 + L), as the histogram's: a multiple of 4N bytes)
    sm.g_sa = (unsigned)__cvta_generic_to_shared(wt);
    sm.g_hi = sm.g_sa >> (2 + L);
    // this lane's words in its warp's ring of value stages, after the
    // histogram copies: stage k at + k CV_MAX_COMP 128, value c at + c 128
    const unsigned ring = (unsigned)__cvta_generic_to_shared(hist + kWarpsPerBlock * NDIM * P::N) +
                          (unsigned)(warp * kMatAhead * CV_MAX_COMP * 32 * 4 + lane * 4);
    __syncthreads();

    // (st, when given, only carries the run's stop flag to the refinement
    // that follows: start and n are the launch's)
    if (A.st && blockIdx.x == 0 && threadIdx.x == 0)
        A.st->pass_active = *(volatile const int *)&A.st->stopped ? 0 : 1;
    const unsigned long long start = A.start;
    const long long n = A.n;
    // blocks [qa, qb) cover the pass; qa a multiple of kMatGroup, so every
    // chunk starts on one (its steps' words are known in advance)
    const unsigned long long qa = (start >> 5) & ~(unsigned long long)(kMatGroup - 1);
    const unsigned long long qb = (start + (unsigned long long)n + 31ull) >> 5;
    const unsigned long long nblk = n > 0 ? qb - qa : 0ull;
    const unsigned long long gwarp = (unsigned long long)blockIdx.x * kWarpsPerBlock + warp;
    const unsigned long long twarps = (unsigned long long)gridDim.x * kWarpsPerBlock;
    // one chunk per warp (an even share, a multiple of kMatGroup blocks)
    const unsigned long long per =
        max((unsigned long long)kMatGroup, (nblk + twarps * kMatGroup - 1) / (twarps * kMatGroup) * kMatGroup);
    const unsigned long long nchunk = (nblk + per - 1) / per;
    Acc<float> s1[CV_MAX_COMP], s2[CV_MAX_COMP];
    for (unsigned long long ch = gwarp; ch < nchunk; ch += twarps) {
        const unsigned long long q0 = qa + ch * per;
        const int nk = (int)min(per, qb - q0);
        if ((unsigned long long)nk == per && q0 * 32ull >= start && (q0 + per) * 32ull <= start + (unsigned long long)n)
            mat_accum_chunk<NDIM, L, false>(A, sm, q0, nk, lane, ring, ncomp, s1, s2);
        else
            mat_accum_chunk<NDIM, L, true>(A, sm, q0, nk, lane, ring, ncomp, s1, s2);
    }
    const int N = P::N;

    __shared__ double red[kWarpsPerBlock][2 * CV_MAX_COMP];
#pragma unroll
    for (int c = 0; c < CV_MAX_COMP; ++c) {
        if (c < ncomp) {
            const double a = warp_total(s1[c]);
            const double b = warp_total(s2[c]);
            if (lane == 0) {
                red[warp][2 * c] = a;
                red[warp][2 * c + 1] = b;
            }
        }
    }
    __syncthreads();
    // the block's sums and histogram as its partial rows (with part_S), else
    // added with FP64 atomics
    const bool parts = A.part_S != nullptr;
    if (threadIdx.x < 2 * ncomp) {
        double t = 0.0;
        for (int w = 0; w < kWarpsPerBlock; ++w) t += red[w][threadIdx.x];
        const int c = threadIdx.x >> 1;
        if (parts) A.part_S[blockIdx.x * (2 * CV_MAX_COMP) + threadIdx.x] = t;
        else atomicAdd((threadIdx.x & 1) ? &A.S2[c] : &A.S1[c], t);
    }
    // the warps' copies, summed in warp order
    float *ph = parts ? reinterpret_cast<float *>(A.part_H) + (size_t)blockIdx.x * NDIM * N : nullptr;
    for (int idx = threadIdx.x; idx < NDIM * N; idx += blockDim.x) {
        const int d = idx / N;
        const int k = idx - d * N;
        const int p = slot_of_bin(k, A.map);
        float v = 0.0f;
#pragma unroll
        for (int w = 0; w < kWarpsPerBlock; ++w) v += hist[(w * NDIM + d) * N + p];
        if (parts) ph[d * N + k] = v;
        else if (v != 0.0f) atomicAdd(&A.H[d * N + k], (double)v);
    }
    if (parts && A.part_ticket) last_block_sums(A.part_S, A.part_ticket, A.S1, A.S2, ncomp);
}

// Built-in integrand on materialised points (the library's own callback):
// f_c(x_j) for the Genz components of g, same formulas as the fused pass.
// FP32, dimension-major, with any integrand policy (the run-time
// specialised one makes families and parameters constants).
template <int NDIM, class I>
__device__ __forceinline__ void genz_points_f32(const GenzParams<float> &g, const float *x, float *f, long long n,
                                                long long ld)
{
    const int ncomp = I::ncomp(g);
    const int delay = I::delay(g);
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x) {
        float z[NDIM];
#pragma unroll
        for (int d = 0; d < NDIM; ++d) z[d] = x[(long long)d * ld + j] - 0.5f;
        float v[CV_MAX_COMP];
        v[0] = genz_f32<NDIM, 0, I>(g, z);
        v[1] = ncomp > 1 ? genz_f32<NDIM, 1, I>(g, z) : 0.0f;
        v[2] = ncomp > 2 ? genz_f32<NDIM, 2, I>(g, z) : 0.0f;
        v[3] = ncomp > 3 ? genz_f32<NDIM, 3, I>(g, z) : 0.0f;
        if (delay) {
#pragma unroll
            for (int c = 0; c < CV_MAX_COMP; ++c)
                if (c < ncomp) v[c] += 0.0f * delay_chain<NDIM>(z, delay);
        }
#pragma unroll
        for (int c = 0; c < CV_MAX_COMP; ++c)
            if (c < ncomp) f[(long long)c * ld + j] = v[c];
    }
}

template <int NDIM, typename Real, bool AOS>
__global__ void __launch_bounds__(kBlock)
k_genz_points(const __grid_constant__ GenzParams<Real> g, const Real *x, Real *f, long long n, long long ld)
{
    if constexpr (sizeof(Real) == 4 && !AOS) {
        genz_points_f32<NDIM, RuntimeIntegrand<float>>(g, x, f, n, ld);
        return;
    }
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x) {
        // (FP32 evaluates at the centred coordinate x - 1/2, FP64 at x)
        const Real c = sizeof(Real) == 4 ? Real(0.5) : Real(0);
        Real xx[NDIM];
#pragma unroll
        for (int d = 0; d < NDIM; ++d) xx[d] = (AOS ? x[j * NDIM + d] : x[(long long)d * ld + j]) - c;
        Real v[CV_MAX_COMP];
        v[0] = genz_eval<NDIM, 0>(g, xx);
        if (g.ncomp > 1) v[1] = genz_eval<NDIM, 1>(g, xx);
        if (g.ncomp > 2) v[2] = genz_eval<NDIM, 2>(g, xx);
        if (g.ncomp > 3) v[3] = genz_eval<NDIM, 3>(g, xx);
        if (g.delay) {
#pragma unroll
            for (int c = 0; c < CV_MAX_COMP; ++c)
                if (c < g.ncomp) v[c] += Real(0) * delay_chain<NDIM>(xx, g.delay);
        }
#pragma unroll
        for (int c = 0; c < CV_MAX_COMP; ++c)
            if (c < g.ncomp) {
                if (AOS) f[j * g.ncomp + c] = v[c];
                else f[(long long)c * ld + j] = v[c];
            }
    }
}

// Sobol coordinates only (the point generator of the sampling kernels,
// written out for bit-exact checks): Y[d*n + j] = X_d(start + j) >> shift,
// for the Sobol, digitally shifted (P.shift) or pseudo-random generator.
template <int NDIM, typename W>
__global__ void __launch_bounds__(kBlock)
k_sobol(unsigned long long start, long long n, int shift, const __grid_constant__ PointArgs P,
        unsigned long long *Y)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long qa = start >> 5;
    const unsigned long long end = start + (unsigned long long)n;
    const unsigned long long qb = (end + 31ull) >> 5;
    const unsigned long long nblk = n > 0 ? qb - qa : 0ull;
    const unsigned long long gwarp = (unsigned long long)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const unsigned long long twarps = (unsigned long long)gridDim.x * kWarpsPerBlock;
    unsigned long long plen = (nblk + twarps - 1) / twarps;
    if (plen < 4) plen = 4;
    const unsigned long long nchunk = (nblk + plen - 1) / plen;
    for (unsigned long long ch = gwarp; ch < nchunk; ch += twarps) {
        const unsigned long long q0 = qa + ch * plen;
        const unsigned long long q1 = min(q0 + plen, qb);
        W X[NDIM];
        sobol_skip<NDIM, W>(X, q0, lane);
        if (P.gen == kGenScrambled) {
#pragma unroll
            for (int d = 0; d < NDIM; ++d) X[d] ^= (W)P.shift[d];
        }
        for (unsigned long long q = q0; q < q1; ++q) {
            const unsigned long long i = q * 32ull + (unsigned long long)lane;
            if (P.gen == kGenPseudo) pseudo_words<NDIM, W>(X, P.seed, i);
            if (i >= start && i < end) {
                const unsigned long long j = i - start;
#pragma unroll
                for (int d = 0; d < NDIM; ++d)
                    Y[(size_t)d * n + j] = (unsigned long long)(X[d] >> shift);
            }
            if (q + 1 < q1) sobol_step<NDIM, W>(X, q);
        }
    }
}

// ------------------------------------------------------------ launchers
#if !defined(__CUDACC_RTC__)
template <int NDIM, typename Real>
static void *sample_fn(bool pow2)
{
    if constexpr (sizeof(Real) == 4)
        return pow2 ? (void *)k_sample<NDIM, float, true> : (void *)k_sample<NDIM, float, false>;
    else
        return (void *)k_sample<NDIM, double, false>;
}

template <int NDIM, typename Real>
cudaError_t launch_sample(const SampleArgs<Real> &a, int grid, cudaStream_t s)
{
    // (sample_occupancy, always called first, sets the shared-memory limit)
    const size_t smem = sample_smem_bytes(NDIM, a.nbins, sizeof(Real) == 8, a.map.priv != 0);
    if (a.gen == kGenPseudo) {
        k_sample_pseudo<NDIM, Real><<<grid, kBlock, smem, s>>>(a);
    } else if constexpr (sizeof(Real) == 4) {
        if (a.map.pow2) k_sample<NDIM, float, true><<<grid, kBlock, smem, s>>>(a);
        else k_sample<NDIM, float, false><<<grid, kBlock, smem, s>>>(a);
    } else {
        k_sample<NDIM, double, false><<<grid, kBlock, smem, s>>>(a);
    }
    return cudaGetLastError();
}

template <int NDIM, typename Real>
cudaError_t sample_occupancy(int nbins, int *blocks_per_sm)
{
    const MapParams m = make_map(nbins, NDIM, sizeof(Real) == 8);
    const size_t smem = sample_smem_bytes(NDIM, nbins, sizeof(Real) == 8, m.priv != 0);
    int optin = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    for (int v = 0; v < 2; ++v) {
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, sample_fn<NDIM, Real>(v == 1));
        if (e != cudaSuccess) return e;
        // (the limit, not the launch size: static shared memory counts too)
        e = cudaFuncSetAttribute(sample_fn<NDIM, Real>(v == 1), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return e;
    }
    {
        void *f = (void *)k_sample_pseudo<NDIM, Real>;
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, f);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return e;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, sample_fn<NDIM, Real>(m.pow2 != 0),
                                                         kBlock, smem);
}

template <int NDIM, bool POW2>
cudaError_t launch_batch_sample(const BatchSampleArgs &b, int grid, cudaStream_t s)
{
    // (batch_occupancy, always called first, sets the shared-memory limit)
    k_batch_sample<NDIM, POW2><<<grid, kBlock, batch_smem_bytes(NDIM, b.stride), s>>>(b);
    return cudaGetLastError();
}

template <int NDIM>
cudaError_t batch_occupancy(bool pow2, int stride, int *blocks_per_sm)
{
    void *f = pow2 ? (void *)k_batch_sample<NDIM, true> : (void *)k_batch_sample<NDIM, false>;
    int optin = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
    const int dyn_max = optin - (int)fa.sharedSizeBytes;  // static shared memory counts too
    const size_t want = batch_smem_bytes(NDIM, stride);
    if ((int)want > dyn_max) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, kBlock, want);
}

template <int NDIM, int L, int MODE>
static cudaError_t launch_mat_lean(const SampleArgs<float> &a, int grid, cudaStream_t s, int *grid_used)
{
    using P = Pow2Map<L>;
    // (the compile-time map must be the one the host chose)
    if (a.nbins != P::N || a.map.mF != P::mF || a.map.expE != P::expE || a.map.sA != P::sA || a.map.li != P::li)
        return cudaErrorInvalidValue;
    if (MODE == 1) {
        const size_t smem = (size_t)NDIM * P::N * 8 + 8 * (size_t)P::N;
        cudaError_t e = cudaFuncSetAttribute(k_mat_store<NDIM, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        *grid_used = grid;
        k_mat_store<NDIM, L><<<grid, kBlock, smem, s>>>(a);
        return cudaGetLastError();
    }
    // (the width table, the warps' histogram copies, 8N bytes to align the
    // table, the warps' value rings)
    const size_t smem = (size_t)(1 + kWarpsPerBlock) * NDIM * P::N * 4 + 8 * (size_t)P::N +
                        (size_t)kWarpsPerBlock * kMatAhead * CV_MAX_COMP * 32 * 4;
    cudaError_t e = cudaFuncSetAttribute(k_mat_accum<NDIM, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // (at most one wave of this kernel's own residency)
    static int occ = 0;
    int dev = 0, sms = 0;
    if (!occ) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mat_accum<NDIM, L>, kBlock, smem);
        if (e != cudaSuccess) return e;
        if (occ < 1) occ = 1;
    }
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (grid > sms * occ) grid = sms * occ;
    if (a.part_S && grid > a.part_G) return cudaErrorInvalidValue;  // (partial rows for every block)
    *grid_used = grid;
    k_mat_accum<NDIM, L><<<grid, kBlock, smem, s>>>(a);
    return cudaGetLastError();
}

template <int NDIM, typename Real, bool POW2, int MODE>
static cudaError_t launch_matpass_v(const SampleArgs<Real> &a, int grid, cudaStream_t s, int *grid_used)
{
    if constexpr (sizeof(Real) == 4 && POW2) {
        // the common case's own kernels (dimension-major, Sobol points; the
        // accumulate pass needs the warps' histogram copies to fit)
        if (!a.aos && a.gen != kGenPseudo && (MODE == 1 || a.map.priv)) {
            switch (a.map.L) {
            case 5: return launch_mat_lean<NDIM, 5, MODE>(a, grid, s, grid_used);
            case 6: return launch_mat_lean<NDIM, 6, MODE>(a, grid, s, grid_used);
            case 7: return launch_mat_lean<NDIM, 7, MODE>(a, grid, s, grid_used);
            case 8: return launch_mat_lean<NDIM, 8, MODE>(a, grid, s, grid_used);
            default: break;
            }
        }
    }
    const size_t smem = sample_smem_bytes(NDIM, a.nbins, sizeof(Real) == 8, a.map.priv != 0);
    cudaError_t e = cudaFuncSetAttribute(k_matpass<NDIM, Real, POW2, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (a.part_S && grid > a.part_G) return cudaErrorInvalidValue;
    *grid_used = grid;
    k_matpass<NDIM, Real, POW2, MODE><<<grid, kBlock, smem, s>>>(a);
    return cudaGetLastError();
}

template <int NDIM, typename Real, int MODE>
cudaError_t launch_matpass(const SampleArgs<Real> &a, int grid, cudaStream_t s, int *grid_used)
{
    if constexpr (sizeof(Real) == 4) {
        if (a.map.pow2) return launch_matpass_v<NDIM, float, true, MODE>(a, grid, s, grid_used);
    }
    return launch_matpass_v<NDIM, Real, false, MODE>(a, grid, s, grid_used);
}

template <int NDIM, typename Real, bool AOS>
cudaError_t launch_genz_points(const GenzParams<Real> &g, const Real *x, Real *f, long long n,
                               long long ld, int grid, cudaStream_t s)
{
    k_genz_points<NDIM, Real, AOS><<<grid, kBlock, 0, s>>>(g, x, f, n, ld);
    return cudaGetLastError();
}

template <int NDIM, typename W>
cudaError_t launch_sobol(unsigned long long start, long long n, int bits, const PointArgs &pa,
                         unsigned long long *Y, int grid, cudaStream_t s)
{
    const int shift = (int)(8 * sizeof(W)) - bits;
    k_sobol<NDIM, W><<<grid, kBlock, 0, s>>>(start, n, shift, pa, Y);
    return cudaGetLastError();
}

#endif  // !__CUDACC_RTC__

}  // namespace cv

#define CV_INSTANTIATE_NDIM(D)                                                              \
    template cudaError_t cv::launch_sample<D, float>(const cv::SampleArgs<float> &, int,    \
                                                     cudaStream_t);                         \
    template cudaError_t cv::launch_sample<D, double>(const cv::SampleArgs<double> &, int,  \
                                                      cudaStream_t);                        \
    template cudaError_t cv::sample_occupancy<D, float>(int, int *);                        \
    template cudaError_t cv::sample_occupancy<D, double>(int, int *);                       \
    template cudaError_t cv::launch_batch_sample<D, true>(const cv::BatchSampleArgs &, int,  \
                                                          cudaStream_t);                    \
    template cudaError_t cv::launch_batch_sample<D, false>(const cv::BatchSampleArgs &, int, \
                                                           cudaStream_t);                   \
    template cudaError_t cv::batch_occupancy<D>(bool, int, int *);                          \
    template cudaError_t cv::launch_matpass<D, float, 1>(const cv::SampleArgs<float> &, int, cudaStream_t, int *); \
    template cudaError_t cv::launch_matpass<D, float, 2>(const cv::SampleArgs<float> &, int, cudaStream_t, int *); \
    template cudaError_t cv::launch_matpass<D, double, 1>(const cv::SampleArgs<double> &, int, cudaStream_t, int *); \
    template cudaError_t cv::launch_matpass<D, double, 2>(const cv::SampleArgs<double> &, int, cudaStream_t, int *); \
    template cudaError_t cv::launch_genz_points<D, float, false>(const cv::GenzParams<float> &, const float *, float *, long long, long long, int, cudaStream_t); \
    template cudaError_t cv::launch_genz_points<D, float, true>(const cv::GenzParams<float> &, const float *, float *, long long, long long, int, cudaStream_t); \
    template cudaError_t cv::launch_genz_points<D, double, false>(const cv::GenzParams<double> &, const double *, double *, long long, long long, int, cudaStream_t); \
    template cudaError_t cv::launch_genz_points<D, double, true>(const cv::GenzParams<double> &, const double *, double *, long long, long long, int, cudaStream_t); \
    template cudaError_t cv::launch_sobol<D, unsigned int>(unsigned long long, long long,   \
                                                           int, const cv::PointArgs &,      \
                                                           unsigned long long *, int,       \
                                                           cudaStream_t);                   \
    template cudaError_t cv::launch_sobol<D, unsigned long long>(                           \
        unsigned long long, long long, int, const cv::PointArgs &, unsigned long long *, int, \
        cudaStream_t);
