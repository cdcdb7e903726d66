/*
 * cuba_oracle.c -- plain, slow, FP64 CPU oracle for the Vegas sampling path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header, table or helper with the CUDA path: it derives its own Sobol
 * direction numbers (Bratley-Fox recurrence on the Joe-Kuo primitive
 * polynomials and initial numbers that scipy ships), evaluates every sample
 * point directly from its index, and sums with Neumaier compensation.
 *
 * What it computes, step by step (the method is "DoSample as driven by
 * Vegas", "Concurrent Cuba" Sect. 2.1 for the sampling unit and Sect. 3.2.2
 * for the Vegas argument list; the paper does not spell out the Vegas
 * algorithm, so the steps follow Lepage 1978, Sobol 1967, Antonov-Saleev
 * 1979, Bratley-Fox 1988 and Genz 1984):
 *
 *   1. Sobol word  X_d(i) = XOR over set bits k of g(i) = i ^ (i >> 1) of
 *      V_d[k], with V_d[k] = m_{d,k+1} << (63 - k)        (Antonov-Saleev)
 *   2. y-coordinate  Y_d = X_d >> (64 - b),  b = 52 (FP64) or 23 (FP32 path)
 *   3. grid map  t = Y_d * N,  k = t >> b,  frac = (t mod 2^b) 2^-b,
 *      x_d = fma(w_k, frac, e_k),  w_k = e_{k+1} - e_k,  J = prod_d N w_k
 *   4. integrand  f_c(x), Genz families
 *   5. sums  S1_c = sum J f_c,  S2_c = sum (J f_c)^2,
 *      histogram  H[d][k_d] += (J f_0)^2
 *   6. iteration result  I = S1/n,  var = (S2/n - I^2)/(n - 1)
 *   7. combination over iterations by inverse variance, chi^2 and its
 *      probability P((m-1)/2, chi^2/2)
 *   8. grid refinement (smooth, compress with alpha = 1.5, rebin)
 *
 * Parity status: every function here is pinned by a test against something
 * other than itself (scipy's Sobol points, the digital-net property, Genz
 * closed forms checked by independent quadrature, exact special cases); see
 * the oracle tests.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define OR_MAX_DIM 64
#define OR_MAX_COMP 8
#define OR_MAX_BINS 256
#define OR_WORD_BITS 64

/* Genz 1984 test families (Genz, "Testing multidimensional integration
 * routines", 1984) plus the constant function used for exact pins. */
enum {
    OR_OSCILLATORY = 0,
    OR_PRODUCT_PEAK = 1,
    OR_CORNER_PEAK = 2,
    OR_GAUSSIAN = 3,
    OR_C0 = 4,
    OR_DISCONTINUOUS = 5,
    OR_CONST = 6
};

typedef struct {
    int ndim;
    int ncomp;
    int nbins;
    int bits;          /* fraction bits b of the y-coordinate */
    int band_bits;     /* significand bits p of the evaluation a pass is
                        * compared with (24: binary32), 0: none; sets the
                        * discontinuity band of or_sample_bounds */
    int family[OR_MAX_COMP];
    double a[OR_MAX_COMP][OR_MAX_DIM];
    double u[OR_MAX_COMP][OR_MAX_DIM];
    int gen;           /* point generator: OR_GEN_SOBOL, _SCRAMBLED, _PSEUDO */
    uint64_t seed;     /* key of the counter-based generator */
    int delay;         /* integrand-cost knob: extra multiply-adds per evaluation */
} or_problem;

/* ------------------------------------------------------------------ */
/* Neumaier (improved Kahan) compensated summation.                    */
/* ------------------------------------------------------------------ */
typedef struct {
    double s;
    double c;
} or_sum;

static void sum_add(or_sum *acc, double x)
{
    double t = acc->s + x;
    if (fabs(acc->s) >= fabs(x))
        acc->c += (acc->s - t) + x;
    else
        acc->c += (x - t) + acc->s;
    acc->s = t;
}

static double sum_value(const or_sum *acc) { return acc->s + acc->c; }

/* ------------------------------------------------------------------ */
/* 1. Sobol direction numbers (Bratley & Fox 1988, Algorithm 659).      */
/* ------------------------------------------------------------------ */

/*
 * Dimension 0 is the van der Corput sequence: m_k = 1 for every k.
 * Dimension d >= 1 uses the primitive polynomial
 *     p(x) = x^s + a_1 x^(s-1) + ... + a_(s-1) x + 1
 * given as the integer poly[d] (bit j holds the coefficient of x^j), the
 * s initial odd numbers m_1..m_s (vinit[d][0..s-1]), and for k > s
 *     m_k = 2 a_1 m_(k-1) ^ 4 a_2 m_(k-2) ^ ... ^ 2^(s-1) a_(s-1) m_(k-s+1)
 *           ^ 2^s m_(k-s) ^ m_(k-s).
 * The direction word for bit k of the Gray-code index (0-based) is
 *     V[d][k] = m_(k+1) << (63 - k),
 * i.e. the binary fraction m_(k+1) / 2^(k+1) held in 64 bits.
 * Returns 0, or -1 if an input is out of range.
 */
int or_sobol_directions(int ndim, const int64_t *poly, const int64_t *vinit,
                        int vinit_stride, uint64_t *V)
{
    if (ndim < 1 || ndim > OR_MAX_DIM)
        return -1;
    for (int d = 0; d < ndim; ++d) {
        uint64_t m[OR_WORD_BITS + 1]; /* 1-based: m[1..64] */
        if (d == 0) {
            for (int k = 1; k <= OR_WORD_BITS; ++k)
                m[k] = 1;
        } else {
            int64_t p = poly[d];
            int s = 0;
            while ((p >> (s + 1)) != 0)
                ++s; /* degree of p */
            if (s < 1 || s > 18)
                return -1;
            for (int k = 1; k <= s; ++k) {
                int64_t mk = vinit[(size_t)d * vinit_stride + (k - 1)];
                if (mk <= 0 || (mk & 1) == 0 || mk >= ((int64_t)1 << k))
                    return -1;
                m[k] = (uint64_t)mk;
            }
            for (int k = s + 1; k <= OR_WORD_BITS; ++k) {
                uint64_t mk = m[k - s] ^ (m[k - s] << s);
                for (int j = 1; j <= s - 1; ++j) {
                    int a_j = (int)((p >> (s - j)) & 1);
                    if (a_j)
                        mk ^= m[k - j] << j;
                }
                m[k] = mk;
            }
        }
        for (int k = 0; k < OR_WORD_BITS; ++k)
            V[(size_t)d * OR_WORD_BITS + k] = m[k + 1] << (63 - k);
    }
    return 0;
}

/* Sobol word of index i in Gray-code order, computed directly from i
 * (Antonov & Saleev 1979): X_d(i) = XOR_{k : bit k of i^(i>>1)} V[d][k]. */
void or_sobol_word(int ndim, const uint64_t *V, uint64_t i, uint64_t *X)
{
    uint64_t g = i ^ (i >> 1);
    for (int d = 0; d < ndim; ++d) {
        uint64_t x = 0;
        for (int k = 0; k < OR_WORD_BITS; ++k)
            if ((g >> k) & 1)
                x ^= V[(size_t)d * OR_WORD_BITS + k];
        X[d] = x;
    }
}

/* y-coordinates with b fraction bits for indices start..start+n-1, written
 * dimension-major: Y[d*n + j] = X_d(start + j) >> (64 - b). */
int or_sobol_coords(int ndim, const uint64_t *V, uint64_t start, int64_t n,
                    int bits, uint64_t *Y)
{
    if (bits < 1 || bits > 63 || n < 0)
        return -1;
    uint64_t X[OR_MAX_DIM];
    for (int64_t j = 0; j < n; ++j) {
        or_sobol_word(ndim, V, start + (uint64_t)j, X);
        for (int d = 0; d < ndim; ++d)
            Y[(size_t)d * n + j] = X[d] >> (64 - bits);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* 1b. Counter-based random words and the other point generators.      */
/* ------------------------------------------------------------------ */

/*
 * Philox4x64-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC 2011): a 256-bit counter c and a 128-bit key k go
 * through ten rounds; each round multiplies c0 and c2 by fixed odd
 * constants into 128-bit products (hi, lo) and forms
 *     c' = (hi(M1 c2) ^ c1 ^ k0,  lo(M1 c2),  hi(M0 c0) ^ c3 ^ k1,  lo(M0 c0)),
 * and the key advances by the Weyl constants (golden ratio, sqrt(3) - 1)
 * between rounds.  The output is the final counter block.
 */
void or_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        const unsigned __int128 p0 = (unsigned __int128)M0 * c0;
        const unsigned __int128 p1 = (unsigned __int128)M1 * c2;
        const uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        const uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

enum { OR_GEN_SOBOL = 0, OR_GEN_SCRAMBLED = 1, OR_GEN_PSEUDO = 2 };

/* Word d of the Philox block (a, d / 4, b, 0) under key (seed, 0). */
static uint64_t philox_word(uint64_t seed, uint64_t a, int d, uint64_t b)
{
    const uint64_t ctr[4] = {a, (uint64_t)(d / 4), b, 0};
    const uint64_t key[2] = {seed, 0};
    uint64_t out[4];
    or_philox4x64(ctr, key, out);
    return out[d % 4];
}

/*
 * Word of point i in dimension d for each generator:
 *   Sobol      X_d(i) as above;
 *   scrambled  X_d(i) ^ S_d, a random digital shift per dimension,
 *              S_d = Philox word (0, d/4, 1, 0)[d mod 4]: every point moves
 *              by the same XOR, so every net property of the sequence is
 *              kept, and independent seeds give independent replicates
 *              (randomized QMC);
 *   pseudo     Philox word (i, d/4, 0, 0)[d mod 4]: independent uniform
 *              64-bit words, no net structure.
 * The y-coordinate takes the top b bits of the word in every case.
 */
void or_point_words(int gen, uint64_t seed, int ndim, const uint64_t *V, uint64_t i,
                    uint64_t *X)
{
    if (gen == OR_GEN_PSEUDO) {
        for (int d = 0; d < ndim; ++d)
            X[d] = philox_word(seed, i, d, 0);
        return;
    }
    or_sobol_word(ndim, V, i, X);
    if (gen == OR_GEN_SCRAMBLED)
        for (int d = 0; d < ndim; ++d)
            X[d] ^= philox_word(seed, 0, d, 1);
}

/* y-coordinates of any generator, dimension-major as or_sobol_coords. */
int or_point_coords(int gen, uint64_t seed, int ndim, const uint64_t *V, uint64_t start,
                    int64_t n, int bits, uint64_t *Y)
{
    if (bits < 1 || bits > 63 || n < 0 || gen < 0 || gen > 2)
        return -1;
    uint64_t X[OR_MAX_DIM];
    for (int64_t j = 0; j < n; ++j) {
        or_point_words(gen, seed, ndim, V, start + (uint64_t)j, X);
        for (int d = 0; d < ndim; ++d)
            Y[(size_t)d * n + j] = X[d] >> (64 - bits);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* 3. Vegas grid map (Lepage 1978).                                     */
/* ------------------------------------------------------------------ */

/* Initial grid: e_k = k / N on every axis; edges[d*(N+1) + k]. */
void or_grid_uniform(int ndim, int nbins, double *edges)
{
    for (int d = 0; d < ndim; ++d)
        for (int k = 0; k <= nbins; ++k)
            edges[(size_t)d * (nbins + 1) + k] = (double)k / (double)nbins;
}

/* Map one point: y-coordinates Y (b fraction bits) to x, returning the
 * Jacobian J = prod_d N w_(k_d) and the bin indices k_d. */
static double map_point(int ndim, int nbins, const double *edges,
                        const uint64_t *Y, int bits, double *x, int *kbin)
{
    double J = 1.0;
    const uint64_t mask = (((uint64_t)1) << bits) - 1;
    for (int d = 0; d < ndim; ++d) {
        uint64_t t = Y[d] * (uint64_t)nbins;
        int k = (int)(t >> bits);
        double frac = ldexp((double)(t & mask), -bits);
        const double *e = edges + (size_t)d * (nbins + 1);
        double w = e[k + 1] - e[k];
        x[d] = fma(w, frac, e[k]);
        J *= (double)nbins * w;
        kbin[d] = k;
    }
    return J;
}

/* Exported form of map_point for the brute-force pins. */
double or_map(int ndim, int nbins, const double *edges, const uint64_t *Y,
              int bits, double *x, int *kbin)
{
    return map_point(ndim, nbins, edges, Y, bits, x, kbin);
}

/* ------------------------------------------------------------------ */
/* 4. Genz 1984 test integrands and their exact integrals over [0,1]^d. */
/* ------------------------------------------------------------------ */

static const double OR_PI = 3.14159265358979323846264338327950288;

/* f for one component at the FP64 point x. */
static double genz_eval(int family, int ndim, const double *a, const double *u,
                        const double *x)
{
    double s = 0.0, p = 1.0;
    switch (family) {
    case OR_OSCILLATORY:
        for (int i = 0; i < ndim; ++i)
            s += a[i] * x[i];
        return cos(2.0 * OR_PI * u[0] + s);
    case OR_PRODUCT_PEAK:
        for (int i = 0; i < ndim; ++i) {
            double dx = x[i] - u[i];
            p *= 1.0 / (1.0 / (a[i] * a[i]) + dx * dx);
        }
        return p;
    case OR_CORNER_PEAK:
        for (int i = 0; i < ndim; ++i)
            s += a[i] * x[i];
        return pow(1.0 + s, -(double)(ndim + 1));
    case OR_GAUSSIAN:
        for (int i = 0; i < ndim; ++i) {
            double dx = x[i] - u[i];
            s += a[i] * a[i] * dx * dx;
        }
        return exp(-s);
    case OR_C0:
        for (int i = 0; i < ndim; ++i)
            s += a[i] * fabs(x[i] - u[i]);
        return exp(-s);
    case OR_DISCONTINUOUS: {
        int ncut = ndim < 2 ? ndim : 2;
        for (int i = 0; i < ncut; ++i)
            if (x[i] > u[i])
                return 0.0;
        for (int i = 0; i < ndim; ++i)
            s += a[i] * x[i];
        return exp(s);
    }
    case OR_CONST:
        return 1.0;
    }
    return NAN;
}

double or_genz(int family, int ndim, const double *a, const double *u,
               const double *x)
{
    return genz_eval(family, ndim, a, u, x);
}

/* Gauss-Legendre nodes/weights on [-1,1] by Newton's method on P_n. */
static void gauss_legendre(int n, double *t, double *wt)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(OR_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= n; ++j) {
                double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16)
                break;
        }
        t[i] = z;
        wt[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/*
 * Corner peak:  int (1 + a.x)^-(d+1) dx
 *   = (1/d!) int_0^inf t^d e^-t prod_i (1 - e^(-a_i t)) / (a_i t) dt,
 * from (1+s)^-(d+1) = (1/d!) int_0^inf t^d e^(-t(1+s)) dt and the product
 * form of the exponential over the cube; integrated with 20-point
 * Gauss-Legendre panels of width 1/2 out to where the gamma-like weight
 * is negligible.
 */
static double corner_peak_exact(int ndim, const double *a)
{
    double t20[20], w20[20];
    gauss_legendre(20, t20, w20);
    double lgd = lgamma((double)ndim + 1.0);
    double T = ndim + 1.0 + 40.0 * sqrt(ndim + 1.0) + 80.0;
    or_sum acc = {0.0, 0.0};
    for (double lo = 0.0; lo < T; lo += 0.5) {
        for (int q = 0; q < 20; ++q) {
            double t = lo + 0.25 * (t20[q] + 1.0);
            double g = 1.0;
            for (int i = 0; i < ndim; ++i) {
                double z = a[i] * t;
                g *= (z == 0.0) ? 1.0 : -expm1(-z) / z;
            }
            double val = exp(ndim * log(t) - t - lgd) * g;
            sum_add(&acc, 0.25 * w20[q] * val);
        }
    }
    return sum_value(&acc);
}

/* Inclusion-exclusion form of the corner-peak integral (for ndim <= 20):
 *   (1 / (d! prod a_i)) sum_{S subset} (-1)^|S| / (1 + sum_{i in S} a_i).
 * Loses digits to cancellation as d grows; used as an independent check. */
double or_corner_peak_incl_excl(int ndim, const double *a)
{
    if (ndim < 1 || ndim > 20)
        return NAN;
    or_sum acc = {0.0, 0.0};
    for (uint32_t S = 0; S < (1u << ndim); ++S) {
        double s = 1.0;
        int cnt = 0;
        for (int i = 0; i < ndim; ++i)
            if ((S >> i) & 1) {
                s += a[i];
                ++cnt;
            }
        sum_add(&acc, ((cnt & 1) ? -1.0 : 1.0) / s);
    }
    double pa = 1.0;
    for (int i = 0; i < ndim; ++i)
        pa *= a[i];
    return sum_value(&acc) / (exp(lgamma(ndim + 1.0)) * pa);
}

double or_genz_exact(int family, int ndim, const double *a, const double *u)
{
    double p = 1.0;
    switch (family) {
    case OR_OSCILLATORY: {
        /* Re[ e^{i 2 pi u_1} prod_k (e^{i a_k} - 1)/(i a_k) ], where
         * (e^{ia}-1)/(ia) = sin(a)/a + i (1 - cos a)/a. */
        double re = cos(2.0 * OR_PI * u[0]), im = sin(2.0 * OR_PI * u[0]);
        for (int k = 0; k < ndim; ++k) {
            double h = 0.5 * a[k];
            double fr = sin(a[k]) / a[k];
            double fi = 2.0 * sin(h) * sin(h) / a[k];
            double nre = re * fr - im * fi;
            double nim = re * fi + im * fr;
            re = nre;
            im = nim;
        }
        return re;
    }
    case OR_PRODUCT_PEAK:
        for (int i = 0; i < ndim; ++i)
            p *= a[i] * (atan(a[i] * (1.0 - u[i])) + atan(a[i] * u[i]));
        return p;
    case OR_CORNER_PEAK:
        return corner_peak_exact(ndim, a);
    case OR_GAUSSIAN:
        for (int i = 0; i < ndim; ++i)
            p *= sqrt(OR_PI) / (2.0 * a[i]) *
                 (erf(a[i] * (1.0 - u[i])) + erf(a[i] * u[i]));
        return p;
    case OR_C0:
        for (int i = 0; i < ndim; ++i)
            p *= (2.0 - exp(-a[i] * u[i]) - exp(-a[i] * (1.0 - u[i]))) / a[i];
        return p;
    case OR_DISCONTINUOUS:
        for (int i = 0; i < ndim; ++i) {
            double c = (i < 2) ? u[i] : 1.0;
            p *= expm1(a[i] * c) / a[i];
        }
        return p;
    case OR_CONST:
        return 1.0;
    }
    return NAN;
}

/* ------------------------------------------------------------------ */
/* 5. One sampling pass ("DoSample", Sect. 2.1): n points from index     */
/*    start on the given grid -> S1[c], S2[c], H[d][k].                  */
/* ------------------------------------------------------------------ */

typedef struct {
    const or_problem *p;
    const uint64_t *V;
    const double *edges;
    uint64_t start;
    int64_t n;
    or_sum S1[OR_MAX_COMP], S2[OR_MAX_COMP];
    or_sum A1[OR_MAX_COMP];            /* sum |J f_c| */
    or_sum B1[OR_MAX_COMP], B2[OR_MAX_COMP]; /* boundary mass, see below */
    or_sum *H; /* [ndim][nbins] */
} sample_job;

/*
 * The discontinuity band.  The discontinuous family switches between 0 and
 * exp(sum a_i x_i) where x_1 or x_2 crosses u_1 or u_2.  The oracle takes
 * that decision on its FP64 point.  An evaluation in a precision of p
 * significand bits (binary32: p = 24) forms the point from the FP64 edge
 * e_k and width w_k of its bin with a few roundings of quantities no larger
 * than a small multiple of the unit interval -- e_k shifted by a few widths
 * or by a constant origin (1/2 to centre the coordinate) and w_k rounded
 * once each, one fused multiply-add for the point, the comparison value
 * rounded once -- which moves x - u by at most about 2^-p (2 + 9 w_k) <=
 * 11 * 2^-p.  So a point whose FP64 coordinate lies within 2^(4-p) of u_i
 * may be decided either way there, and nowhere else.  Such a point is
 * "ambiguous" when no other cut already puts it outside; its alternative
 * value is g = exp(sum a_i x_i).  The boundary mass of a pass is
 * B1_c = sum |J g| and B2_c = sum (J g)^2 over its ambiguous points: a
 * binary32 pass may differ from the oracle's by at most that much in S1_c
 * and S2_c (and in any histogram bin, by B2_0).
 * Returns g for an ambiguous point, else 0.
 */
static double disc_ambiguous(int ndim, const double *a, const double *u, const double *x,
                             int band_bits)
{
    if (band_bits <= 0)
        return 0.0;
    const double band = ldexp(1.0, 4 - band_bits);
    int ncut = ndim < 2 ? ndim : 2, amb = 0;
    for (int i = 0; i < ncut; ++i) {
        if (fabs(x[i] - u[i]) <= band)
            amb = 1;
        else if (x[i] > u[i])
            return 0.0;  /* outside whichever way the other cut goes */
    }
    if (!amb)
        return 0.0;
    double s = 0.0;
    for (int i = 0; i < ndim; ++i)
        s += a[i] * x[i];
    return exp(s);
}

static void *sample_range(void *arg)
{
    sample_job *job = (sample_job *)arg;
    const or_problem *p = job->p;
    const int ndim = p->ndim, N = p->nbins;
    uint64_t X[OR_MAX_DIM], Y[OR_MAX_DIM];
    double x[OR_MAX_DIM];
    int kbin[OR_MAX_DIM];
    for (int64_t j = 0; j < job->n; ++j) {
        or_point_words(p->gen, p->seed, ndim, job->V, job->start + (uint64_t)j, X);
        for (int d = 0; d < ndim; ++d)
            Y[d] = X[d] >> (64 - p->bits);
        double J = map_point(ndim, N, job->edges, Y, p->bits, x, kbin);
        double Jf0 = 0.0;
        for (int c = 0; c < p->ncomp; ++c) {
            double f = genz_eval(p->family[c], ndim, p->a[c], p->u[c], x);
            if (p->delay > 0) {
                /* the cost knob (the paper's calibrated delay, Sect. 4.1):
                 * rounds of ndim dependent multiply-adds z <- z/2 + x_d,
                 * whose bounded result enters as 0 * z (value unchanged) */
                double z = 0.0;
                for (int j = 0; j < p->delay; j += ndim)
                    for (int d = 0; d < ndim; ++d)
                        z = fma(z, 0.5, x[d]);
                f += 0.0 * z;
            }
            double Jf = J * f;
            sum_add(&job->S1[c], Jf);
            sum_add(&job->S2[c], Jf * Jf);
            sum_add(&job->A1[c], fabs(Jf));
            if (p->family[c] == OR_DISCONTINUOUS) {
                double g = disc_ambiguous(ndim, p->a[c], p->u[c], x, p->band_bits);
                if (g != 0.0) {
                    sum_add(&job->B1[c], fabs(J * g));
                    sum_add(&job->B2[c], (J * g) * (J * g));
                }
            }
            if (c == 0)
                Jf0 = Jf;
        }
        double h = Jf0 * Jf0;
        for (int d = 0; d < ndim; ++d)
            sum_add(&job->H[(size_t)d * N + kbin[d]], h);
    }
    return NULL;
}

/*
 * Sample n points with indices start..start+n-1 on the grid `edges`
 * ([ndim][nbins+1]).  Outputs: S1[c] = sum J f_c, S2[c] = sum (J f_c)^2,
 * H[d*nbins + k] = sum over points in bin k of axis d of (J f_0)^2; and,
 * when A1 is not NULL, A1[c] = sum |J f_c| and the boundary mass B1[c],
 * B2[c] of the discontinuity band (above; zero unless p->band_bits > 0).
 * nthreads > 1 splits the index range into contiguous chunks (the CPU
 * analogue of the paper's n/N points per core); the partial sums are
 * combined in chunk order.
 */
int or_sample_bounds(const or_problem *p, const uint64_t *V, const double *edges,
                     uint64_t start, int64_t n, int nthreads, double *S1, double *S2,
                     double *H, double *A1, double *B1, double *B2)
{
    if (p->ndim < 1 || p->ndim > OR_MAX_DIM || p->ncomp < 1 ||
        p->ncomp > OR_MAX_COMP || p->nbins < 2 || p->nbins > OR_MAX_BINS ||
        p->bits < 1 || p->bits > 55 || n < 0 || p->band_bits < 0 || p->band_bits > 53)
        return -1;
    if (nthreads < 1)
        nthreads = 1;
    if (nthreads > 256)
        nthreads = 256;
    if ((int64_t)nthreads > n)
        nthreads = n > 0 ? (int)n : 1;
    const size_t nh = (size_t)p->ndim * p->nbins;
    sample_job *jobs = (sample_job *)calloc((size_t)nthreads, sizeof(sample_job));
    or_sum *hbuf = (or_sum *)calloc(nh * nthreads, sizeof(or_sum));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !hbuf || !th) {
        free(jobs);
        free(hbuf);
        free(th);
        return -2;
    }
    int64_t base = n / nthreads, rem = n % nthreads;
    uint64_t s = start;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].p = p;
        jobs[t].V = V;
        jobs[t].edges = edges;
        jobs[t].start = s;
        jobs[t].n = base + (t < rem ? 1 : 0);
        jobs[t].H = hbuf + nh * t;
        s += (uint64_t)jobs[t].n;
    }
    if (nthreads == 1) {
        sample_range(&jobs[0]);
    } else {
        for (int t = 0; t < nthreads; ++t)
            pthread_create(&th[t], NULL, sample_range, &jobs[t]);
        for (int t = 0; t < nthreads; ++t)
            pthread_join(th[t], NULL);
    }
    for (int c = 0; c < p->ncomp; ++c) {
        or_sum a1 = {0, 0}, a2 = {0, 0}, aa = {0, 0}, b1 = {0, 0}, b2 = {0, 0};
        for (int t = 0; t < nthreads; ++t) {
            sum_add(&a1, sum_value(&jobs[t].S1[c]));
            sum_add(&a2, sum_value(&jobs[t].S2[c]));
            sum_add(&aa, sum_value(&jobs[t].A1[c]));
            sum_add(&b1, sum_value(&jobs[t].B1[c]));
            sum_add(&b2, sum_value(&jobs[t].B2[c]));
        }
        S1[c] = sum_value(&a1);
        S2[c] = sum_value(&a2);
        if (A1) {
            A1[c] = sum_value(&aa);
            B1[c] = sum_value(&b1);
            B2[c] = sum_value(&b2);
        }
    }
    for (size_t b = 0; b < nh; ++b) {
        or_sum a = {0, 0};
        for (int t = 0; t < nthreads; ++t)
            sum_add(&a, sum_value(&hbuf[nh * t + b]));
        H[b] = sum_value(&a);
    }
    free(jobs);
    free(hbuf);
    free(th);
    return 0;
}

/* The pass without the error bounds. */
int or_sample(const or_problem *p, const uint64_t *V, const double *edges,
              uint64_t start, int64_t n, int nthreads, double *S1, double *S2,
              double *H)
{
    return or_sample_bounds(p, V, edges, start, n, nthreads, S1, S2, H, NULL, NULL, NULL);
}

/* ------------------------------------------------------------------ */
/* 8. Grid refinement (Lepage 1978).                                    */
/* ------------------------------------------------------------------ */

/*
 * Per axis, from the f^2 histogram H[k] (k < N):
 *   smooth   h_0 = (H_0+H_1)/2,  h_k = (H_(k-1)+H_k+H_(k+1))/3,
 *            h_(N-1) = (H_(N-2)+H_(N-1))/2
 *   compress r_k = ((1 - h_k/s) / ln(s/h_k))^1.5 with s = sum_k h_k
 *            (r_k = 0 where h_k = 0, r_k = 1 where h_k = s),
 *            then r_k /= max_k r_k (a common scale; the rebinning is
 *            invariant under it, and equal r_k become exactly 1)
 *   rebin    with C_0 = 0, C_(k+1) = C_k + r_k and R = C_N, new edge m
 *            (0 < m < N) sits where the cumulative r reaches m R / N:
 *            the k with C_k <= m R / N < C_(k+1), and
 *            e'_m = fma(e_(k+1) - e_k, (m R / N - C_k) / r_k, e_k).
 *            e'_0 = 0 and e'_N = 1 stay.
 * An axis whose histogram is all zero, or holds a non-finite value, keeps
 * its grid.
 */
/* Rebin one axis: e (N+1 edges) -> e_new so that every new bin holds an
 * equal share R/N of the piecewise-constant weight r_k of the old bins. */
static void rebin_axis(int N, const double *r, const double *e, double *e_new)
{
    double C[OR_MAX_BINS + 1];
    C[0] = 0.0;
    for (int k = 0; k < N; ++k)
        C[k + 1] = C[k] + r[k];
    double R = C[N];
    /* only the interior edges move: the outer ones bound the domain (the
     * unit interval for Vegas, a box side for a Suave region) */
    e_new[0] = e[0];
    e_new[N] = e[N];
    int k = 0;
    for (int m = 1; m < N; ++m) {
        double t = ((double)m * R) / (double)N;
        while (k < N - 1 && !(t < C[k + 1]))
            ++k;
        e_new[m] = fma(e[k + 1] - e[k], (t - C[k]) / r[k], e[k]);
    }
}

/* Exported rebin for the pins: r is [ndim][nbins] (non-negative, at least
 * one positive per axis), edges [ndim][nbins+1] is replaced in place. */
void or_rebin(int ndim, int nbins, const double *r, double *edges)
{
    double e_new[OR_MAX_BINS + 1];
    for (int d = 0; d < ndim; ++d) {
        double *e = edges + (size_t)d * (nbins + 1);
        rebin_axis(nbins, r + (size_t)d * nbins, e, e_new);
        for (int m = 0; m <= nbins; ++m)
            e[m] = e_new[m];
    }
}

void or_refine(int ndim, int nbins, const double *H, double *edges)
{
    const int N = nbins;
    double h[OR_MAX_BINS], r[OR_MAX_BINS], e_new[OR_MAX_BINS + 1];
    for (int d = 0; d < ndim; ++d) {
        const double *Hd = H + (size_t)d * N;
        double *e = edges + (size_t)d * (N + 1);
        int usable = 0, finite = 1;
        for (int k = 0; k < N; ++k) {
            if (!isfinite(Hd[k]))
                finite = 0;
            if (Hd[k] != 0.0)
                usable = 1;
        }
        if (!usable || !finite)
            continue;
        h[0] = (Hd[0] + Hd[1]) / 2.0;
        for (int k = 1; k < N - 1; ++k)
            h[k] = (Hd[k - 1] + Hd[k] + Hd[k + 1]) / 3.0;
        h[N - 1] = (Hd[N - 2] + Hd[N - 1]) / 2.0;
        double s = 0.0;
        for (int k = 0; k < N; ++k)
            s += h[k];
        double rmax = 0.0;
        for (int k = 0; k < N; ++k) {
            if (h[k] == 0.0) {
                r[k] = 0.0;
            } else if (h[k] == s) {
                r[k] = 1.0;
            } else {
                double q = (1.0 - h[k] / s) / log(s / h[k]);
                r[k] = q * sqrt(q); /* q^1.5 */
            }
            if (r[k] > rmax)
                rmax = r[k];
        }
        if (!(rmax > 0.0))
            continue;
        for (int k = 0; k < N; ++k)
            r[k] = r[k] / rmax;
        rebin_axis(N, r, e, e_new);
        for (int m = 0; m <= N; ++m)
            e[m] = e_new[m];
    }
}

/* ------------------------------------------------------------------ */
/* 7. Combination of iterations.                                        */
/* ------------------------------------------------------------------ */

/*
 * P(chi^2 <= x) for k degrees of freedom, from the finite sums of the
 * chi-square distribution function (Abramowitz & Stegun 26.4.4, 26.4.5):
 *   k even: Q = e^{-x/2} sum_{j=0}^{k/2-1} (x/2)^j / j!
 *   k odd : Q = erfc(sqrt(x/2)) + e^{-x/2} sum_{j=1}^{(k-1)/2}
 *               (x/2)^{j-1/2} / Gamma(j+1/2)
 * and P = 1 - Q.
 */
double or_chi2_cdf(double x, int k)
{
    if (k < 1 || !(x > 0.0))
        return 0.0;
    double z = 0.5 * x, Q;
    if ((k & 1) == 0) {
        double term = 1.0, acc = 1.0;
        for (int j = 1; j < k / 2; ++j) {
            term *= z / j;
            acc += term;
        }
        Q = exp(-z) * acc;
    } else {
        double term = sqrt(z) / (0.5 * sqrt(OR_PI)); /* z^{1/2}/Gamma(3/2) */
        double acc = 0.0;
        for (int j = 1; j <= (k - 1) / 2; ++j) {
            acc += term;
            term *= z / (j + 0.5);
        }
        Q = erfc(sqrt(z)) + exp(-z) * acc;
    }
    double P = 1.0 - Q;
    return P < 0.0 ? 0.0 : P;
}

/*
 * Inverse-variance combination of m iteration results I_j, var_j:
 *   mean = sum(I_j/var_j) / sum(1/var_j),  err = (sum 1/var_j)^(-1/2),
 *   chi2 = sum (I_j - mean)^2 / var_j,     prob = P(chi2; m-1 dof)
 * (prob = 0 for m = 1).  If any var_j <= 0, the plain mean of the I_j is
 * returned with err = chi2 = prob = 0.
 */
void or_combine(int m, const double *I, const double *var, double *mean,
                double *err, double *chi2, double *prob)
{
    *mean = *err = *chi2 = *prob = 0.0;
    if (m < 1)
        return;
    int zero = 0;
    for (int j = 0; j < m; ++j)
        if (!(var[j] > 0.0))
            zero = 1;
    if (zero) {
        or_sum a = {0, 0};
        for (int j = 0; j < m; ++j)
            sum_add(&a, I[j]);
        *mean = sum_value(&a) / m;
        return;
    }
    or_sum W = {0, 0}, WI = {0, 0};
    for (int j = 0; j < m; ++j) {
        sum_add(&W, 1.0 / var[j]);
        sum_add(&WI, I[j] / var[j]);
    }
    double w = sum_value(&W);
    *mean = sum_value(&WI) / w;
    *err = sqrt(1.0 / w);
    or_sum X = {0, 0};
    for (int j = 0; j < m; ++j) {
        double dI = I[j] - *mean;
        sum_add(&X, dI * dI / var[j]);
    }
    *chi2 = sum_value(&X);
    *prob = (m > 1) ? or_chi2_cdf(*chi2, m - 1) : 0.0;
}

/* ------------------------------------------------------------------ */
/* The Vegas driver (argument list of Vegas, Sect. 3.2.2).              */
/* ------------------------------------------------------------------ */

/*
 * Iteration j = 1, 2, ... samples n_j = nstart + (j-1) nincrease points
 * with Sobol indices continuing from 1 (index 0, the all-zero point, is
 * skipped), accumulates the iteration result of every component, refines
 * the grid from component 0's histogram, and stops
 *   - with fail = 0 once neval >= mineval and every component has
 *     err_c <= max(epsabs, epsrel |I_c|), or
 *   - with fail = 1 when the next iteration would take neval past maxeval.
 * `edges` holds the starting grid on entry and the refined grid on return
 * (NULL: start from the uniform grid and drop it).  iter_I / iter_var, if
 * non-NULL, receive up to max_log iteration results [j][c].
 * Returns 0, -1 on bad arguments, -2 on allocation failure.
 */
int or_vegas(const or_problem *p, const uint64_t *V, double epsrel,
             double epsabs, int64_t mineval, int64_t maxeval, int64_t nstart,
             int64_t nincrease, int nthreads, double *edges, int64_t *neval,
             int *fail, int *niter, double *integral, double *error,
             double *chi2, double *prob, int max_log, double *iter_I,
             double *iter_var)
{
    const int ndim = p->ndim, ncomp = p->ncomp, N = p->nbins;
    if (ndim < 1 || ndim > OR_MAX_DIM || ncomp < 1 || ncomp > OR_MAX_COMP ||
        N < 2 || N > OR_MAX_BINS || nstart < 2 || nincrease < 0 ||
        nstart > maxeval)
        return -1;
    double *grid = edges;
    double *own = NULL;
    if (!grid) {
        own = grid = (double *)malloc(sizeof(double) * ndim * (N + 1));
        if (!own)
            return -2;
        or_grid_uniform(ndim, N, grid);
    }
    int cap = 64;
    double *Ij = (double *)malloc(sizeof(double) * cap * ncomp);
    double *Vj = (double *)malloc(sizeof(double) * cap * ncomp);
    double *H = (double *)malloc(sizeof(double) * ndim * N);
    double Icol[4096], Vcol[4096];
    if (!Ij || !Vj || !H) {
        free(own);
        free(Ij);
        free(Vj);
        free(H);
        return -2;
    }
    uint64_t next_index = 1;
    int64_t done = 0;
    int m = 0, ok = 0;
    double S1[OR_MAX_COMP], S2[OR_MAX_COMP];
    for (;;) {
        int64_t nj = nstart + (int64_t)m * nincrease;
        if (done + nj > maxeval || m >= 4096)
            break;
        if (or_sample(p, V, grid, next_index, nj, nthreads, S1, S2, H) != 0) {
            free(own);
            free(Ij);
            free(Vj);
            free(H);
            return -2;
        }
        next_index += (uint64_t)nj;
        done += nj;
        if (m == cap) {
            cap *= 2;
            Ij = (double *)realloc(Ij, sizeof(double) * cap * ncomp);
            Vj = (double *)realloc(Vj, sizeof(double) * cap * ncomp);
        }
        for (int c = 0; c < ncomp; ++c) {
            double I = S1[c] / (double)nj;
            double var = (S2[c] / (double)nj - I * I) / (double)(nj - 1);
            Ij[(size_t)m * ncomp + c] = I;
            Vj[(size_t)m * ncomp + c] = var;
            if (iter_I && m < max_log) {
                iter_I[(size_t)m * ncomp + c] = I;
                iter_var[(size_t)m * ncomp + c] = var;
            }
        }
        ++m;
        or_refine(ndim, N, H, grid);
        ok = 1;
        for (int c = 0; c < ncomp; ++c) {
            for (int j = 0; j < m; ++j) {
                Icol[j] = Ij[(size_t)j * ncomp + c];
                Vcol[j] = Vj[(size_t)j * ncomp + c];
            }
            or_combine(m, Icol, Vcol, &integral[c], &error[c], &chi2[c],
                       &prob[c]);
            double tol = fmax(epsabs, epsrel * fabs(integral[c]));
            if (!(error[c] <= tol))
                ok = 0;
        }
        if (done >= mineval && ok)
            break;
        ok = 0;
    }
    if (m == 0)
        for (int c = 0; c < ncomp; ++c)
            integral[c] = error[c] = chi2[c] = prob[c] = 0.0;
    *neval = done;
    *fail = ok ? 0 : 1;
    *niter = m;
    free(own);
    free(Ij);
    free(Vj);
    free(H);
    return 0;
}

/* ------------------------------------------------------------------ */
/* 9. Suave: subregion-adaptive Vegas (the paper gives only its        */
/*    argument list, Sect. 3.2.2; this is the reading stated below).   */
/* ------------------------------------------------------------------ */

/*
 * Every region is an axis-aligned box carrying its own Vegas grid, whose
 * outer edges are the box (e_0 = lo, e_N = hi per axis), so the Vegas map
 * of the box's grid puts points into the box and J includes its volume.
 * Sampling a region: nnew fresh Sobol points (indices continuing one
 * global stream from 1), estimate I = S1/n, var = (S2/n - I^2)/(n - 1),
 * then the region's grid is refined from its histogram.  The refined grid
 * shows where the integrand has structure: along an axis it does not
 * depend on, the bins stay even.  So the fluctuation of axis d is the
 * p-norm (p = flatness) of |ln(w_k / mean w)| over its bins,
 *     fl_d = ((1/N) sum_k |ln(w_k / mean w)|^p)^(1/p).
 * A round: stop with fail = 0 once neval >= mineval and every component
 * has sqrt(sum var) <= max(epsabs, epsrel |sum I|); otherwise take the
 * `width` regions of largest var (component 0; ties by position, only
 * var > 0), split each along the axis of largest fluctuation (ties by the
 * lower axis) at its middle edge e_(N/2) (equal shares of the grid), the children
 * inheriting the grid with the split axis's half subdivided into N bins
 * (each parent bin halved), and sample the children in order (left child
 * first); the left child takes the parent's place, the right one is
 * appended.  Adaptation also stops when a round, plus the final pass,
 * would exceed maxeval, or max_regions.
 * The samples that chose the partition are biased by that choice (a region
 * is kept because its own sample looked flat), so they only steer: the
 * result comes from a final pass that samples every region once more with
 * nnew fresh points (in region order): integral = sum of the final I,
 * error = sqrt(sum of the final var), fail = 0 if that error meets the
 * goal, else 1.
 */
typedef struct {
    double I[OR_MAX_COMP], var[OR_MAX_COMP];
    double fluct[OR_MAX_DIM];
} suave_region;

static void suave_sample(const or_problem *p, const uint64_t *V, double *edges,
                         uint64_t start, int64_t n, int nthreads, double flatness,
                         suave_region *r)
{
    const int ndim = p->ndim, N = p->nbins;
    double S1[OR_MAX_COMP], S2[OR_MAX_COMP];
    double *H = calloc((size_t)ndim * N, sizeof(double));
    or_sample(p, V, edges, start, n, nthreads, S1, S2, H);
    for (int c = 0; c < p->ncomp; ++c) {
        r->I[c] = S1[c] / (double)n;
        r->var[c] = (S2[c] / (double)n - r->I[c] * r->I[c]) / (double)(n - 1);
        if (!(r->var[c] > 0.0))
            r->var[c] = 0.0;
    }
    or_refine(ndim, N, H, edges);
    for (int d = 0; d < ndim; ++d) {
        const double *e = edges + (size_t)d * (N + 1);
        const double mean = (e[N] - e[0]) / N;
        or_sum acc = {0, 0};
        for (int k = 0; k < N; ++k)
            sum_add(&acc, pow(fabs(log((e[k + 1] - e[k]) / mean)), flatness));
        r->fluct[d] = pow(sum_value(&acc) / N, 1.0 / flatness);
    }
    free(H);
}

/* Children grids of a split of `pe` along axis a at edge N/2. */
static void suave_children(int ndim, int N, int a, const double *pe, double *le, double *re)
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

/* Suave as read above.  box_out (optional, [max_regions][ndim][2]) gets the
 * final regions' boxes.  Returns 0, or -1 on bad arguments. */
int or_suave(const or_problem *p, const uint64_t *V, double epsrel, double epsabs,
             int64_t mineval, int64_t maxeval, int64_t nnew, double flatness, int width,
             int max_regions, int nthreads, int *nregions, int64_t *neval, int *fail,
             double *integral, double *error, double *box_out)
{
    const int ndim = p->ndim, N = p->nbins, nc = p->ncomp;
    if (nnew < 2 || maxeval < nnew || width < 1 || max_regions < 1 || !(flatness > 0.0) ||
        (N & 1) || N < 2)
        return -1;
    const size_t ge = (size_t)ndim * (N + 1);
    double *grids = malloc(sizeof(double) * ge * (size_t)max_regions);
    suave_region *R = malloc(sizeof(suave_region) * (size_t)max_regions);
    int *order = malloc(sizeof(int) * (size_t)max_regions);
    or_grid_uniform(ndim, N, grids);
    uint64_t next = 1;
    int nr = 1;
    suave_sample(p, V, grids, next, nnew, nthreads, flatness, &R[0]);
    next += (uint64_t)nnew;
    int64_t done = nnew;
    int status = 1;
    for (;;) {
        int ok = done >= mineval;
        for (int c = 0; c < nc; ++c) {
            or_sum I = {0, 0}, v = {0, 0};
            for (int k = 0; k < nr; ++k) {
                sum_add(&I, R[k].I[c]);
                sum_add(&v, R[k].var[c]);
            }
            integral[c] = sum_value(&I);
            error[c] = sqrt(sum_value(&v));
            if (!(error[c] <= fmax(epsabs, epsrel * fabs(integral[c]))))
                ok = 0;
        }
        if (ok) {
            status = 0;
            break;
        }
        /* the regions to split: largest var of component 0 first */
        int K = 0;
        for (int k = 0; k < nr; ++k)
            if (R[k].var[0] > 0.0)
                order[K++] = k;
        for (int i = 1; i < K; ++i) { /* stable insertion sort, descending */
            int x = order[i], j = i - 1;
            while (j >= 0 && R[order[j]].var[0] < R[x].var[0]) {
                order[j + 1] = order[j];
                --j;
            }
            order[j + 1] = x;
        }
        if (K > width)
            K = width;
        if (K == 0) {
            status = 0; /* every region exact */
            break;
        }
        /* (room for this round and for the final pass over every region) */
        const int64_t room = maxeval - done - (int64_t)nr * nnew;
        if ((int64_t)K > room / (3 * nnew))
            K = (int)(room / (3 * nnew));
        if (K > (max_regions - nr))
            K = max_regions - nr;
        if (K <= 0)
            break; /* fail = 1 */
        for (int i = 0; i < K; ++i) {
            const int k = order[i];
            int a = 0;
            for (int d = 1; d < ndim; ++d)
                if (R[k].fluct[d] > R[k].fluct[a])
                    a = d;
            double *pe = grids + ge * (size_t)k;
            double *le = malloc(sizeof(double) * ge), *re = grids + ge * (size_t)nr;
            suave_children(ndim, N, a, pe, le, re);
            memcpy(pe, le, sizeof(double) * ge);
            free(le);
            suave_sample(p, V, pe, next, nnew, nthreads, flatness, &R[k]);
            next += (uint64_t)nnew;
            suave_sample(p, V, re, next, nnew, nthreads, flatness, &R[nr]);
            next += (uint64_t)nnew;
            ++nr;
            done += 2 * nnew;
        }
    }
    /* the final pass: every region sampled afresh, the result from it alone */
    if (done + (int64_t)nr * nnew <= maxeval || nr == 1) {
        double *tmp = malloc(sizeof(double) * ge);
        for (int k = 0; k < nr; ++k) {
            memcpy(tmp, grids + ge * (size_t)k, sizeof(double) * ge);
            suave_sample(p, V, tmp, next, nnew, nthreads, flatness, &R[k]);
            next += (uint64_t)nnew;
            done += nnew;
        }
        free(tmp);
    }
    status = 0;
    for (int c = 0; c < nc; ++c) {
        or_sum I = {0, 0}, v = {0, 0};
        for (int k = 0; k < nr; ++k) {
            sum_add(&I, R[k].I[c]);
            sum_add(&v, R[k].var[c]);
        }
        integral[c] = sum_value(&I);
        error[c] = sqrt(sum_value(&v));
        if (!(error[c] <= fmax(epsabs, epsrel * fabs(integral[c]))))
            status = 1;
    }
    if (done < mineval)
        status = 1;
    *nregions = nr;
    *neval = done;
    *fail = status;
    if (box_out)
        for (int k = 0; k < nr; ++k)
            for (int d = 0; d < ndim; ++d) {
                box_out[((size_t)k * ndim + d) * 2] = grids[ge * (size_t)k + (size_t)d * (N + 1)];
                box_out[((size_t)k * ndim + d) * 2 + 1] = grids[ge * (size_t)k + (size_t)d * (N + 1) + N];
            }
    free(grids);
    free(R);
    free(order);
    return 0;
}
