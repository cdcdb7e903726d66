// cv_refine.cu -- FP64 grid refinement and iteration combination kernels.
//
// Refinement (Lepage 1978; the paper gives only the Vegas arguments,
// Sect. 3.2.2): per axis, smooth the f^2 histogram over neighbouring bins,
// compress it with exponent 1.5, and move the N-1 interior edges so every
// new bin holds an equal share of the compressed weight.  One CTA per axis;
// the order of every FP64 operation is fixed so the result is reproducible.
//
// Combination: per component, the iteration result I_j = S1/n and
// var_j = (S2/n - I_j^2)/(n-1) are folded into the inverse-variance weighted
// mean with West's (1979) incremental update, which also yields
// chi^2 = sum_j (I_j - mean)^2 / var_j without cancellation; the chi-square
// probability P((m-1)/2, chi^2/2) uses the regularized incomplete gamma
// function (series for x < a+1, Legendre continued fraction otherwise).
#include <cfloat>

#include "cv_internal.cuh"

namespace cv {

// Regularized lower incomplete gamma P(a, x), a > 0, x >= 0.
__device__ double gamma_p(double a, double x)
{
    if (!(x > 0.0)) return 0.0;
    const double lg = lgamma(a);
    if (x < a + 1.0) {
        // P = e^{-x} x^a / Gamma(a) * sum_n x^n / (a (a+1) ... (a+n))
        double ap = a, term = 1.0 / a, sum = term;
        for (int n = 0; n < 1000; ++n) {
            ap += 1.0;
            term *= x / ap;
            sum += term;
            if (fabs(term) < fabs(sum) * 1e-17) break;
        }
        return sum * exp(-x + a * log(x) - lg);
    }
    // Q by the continued fraction 1/(x+1-a- 1(1-a)/(x+3-a- 2(2-a)/(x+5-a- ...)))
    // evaluated with the modified Lentz method.
    const double tiny = 1e-300;
    double b = x + 1.0 - a, c = 1.0 / tiny, d = 1.0 / b, h = d;
    for (int i = 1; i < 1000; ++i) {
        const double an = -i * (i - a);
        b += 2.0;
        d = an * d + b;
        if (fabs(d) < tiny) d = tiny;
        c = b + an / c;
        if (fabs(c) < tiny) c = tiny;
        d = 1.0 / d;
        const double del = d * c;
        h *= del;
        if (fabs(del - 1.0) < 1e-17) break;
    }
    const double Q = exp(-x + a * log(x) - lg) * h;
    return 1.0 - Q;
}

// The FP32 sampling kernel's table of bins [k0, N) of axis d (step dk),
// from the FP64 edges: grid_entry_f32 of each bin at its slot.  The same
// FP64 operations the sampling kernel applies when it converts the grid
// itself, so either way it samples with the same values.
__device__ __forceinline__ void stage_axis(int d, int N, const double *edges, float2 *ew32, const MapParams &map,
                                           int k0, int dk)
{
    const double *e = edges + (size_t)d * (N + 1);
    for (int k = k0; k < N; k += dk)
        ew32[(size_t)d * N + slot_of_bin(k, map)] = grid_entry_f32(e[k], e[k + 1] - e[k], N, map);
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// Maximum of non-negative doubles through their bit patterns: for x, y >= 0
// the IEEE order is the order of the 64-bit integers, and integer compares
// avoid the long FP64 latency of this part.
__device__ __forceinline__ long long warp_max_bits(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Refine axis `d` of the grid in place (one CTA of at least N threads, at
// most 256).  Every reduction has a fixed order, so the result is
// reproducible.  GB300 issues FP64 at a small fraction of the FP32 rate, so
// the CTA is sized to the bins (idle warps would still spend FP64 issue
// slots on the reductions), the per-axis scalars (1/s, 1/max r, R/N) are
// computed once, and the per-bin divisions other than the smoothing's are
// multiplications by correctly rounded reciprocals (each result within
// 1.5 ulp of the quotient).  FP64 results take ~200 cycles here, so the
// refinement is bound by its chain of dependent FP64 operations: maxima
// and searches over non-negative doubles compare bit patterns instead.
// The G blocks' partial histograms of axis d, summed into sH[0, N) by all
// the CTA's threads: thread t takes the V-wide column q = t mod (N/V) of
// the rows r, r + R, r + 2R, ... (r = t div (N/V), R row groups), so a
// warp's loads are contiguous vectors and each thread keeps four in flight;
// the R group sums of a bin are then added in group order.  FP32 partials
// are summed with Kahan's compensation in FP32 throughout (FP64 throughput,
// conversions included, is a small fraction of FP32 here) and converted
// once per bin; FP64 partials are summed in FP64.  The assignment of rows
// to threads is fixed, so the same partials give the same bits.  Called by
// every thread of the CTA (it synchronises).
template <typename T, int V>
__device__ __forceinline__ void load_vec(const T *p, T (&v)[V])
{
    if constexpr (V == 4) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else if constexpr (V == 2 && sizeof(T) == 4) {
        const float2 q = *reinterpret_cast<const float2 *>(p);
        v[0] = q.x; v[1] = q.y;
    } else if constexpr (V == 2) {
        const double2 q = *reinterpret_cast<const double2 *>(p);
        v[0] = q.x; v[1] = q.y;
    } else {
        v[0] = *p;
    }
}

// s + y with the running compensation c (Kahan), FP32
__device__ __forceinline__ void kahan_add(float &s, float &c, float y)
{
    const float t = y - c;
    const float u = s + t;
    c = (u - s) - t;
    s = u;
}

// Group sums: FP32 as (sum, compensation) pairs, FP64 as (sum, 0).
template <typename T>
struct GroupSum { using type = float2; };
template <>
struct GroupSum<double> { using type = double2; };

template <typename T, int V>
__device__ __forceinline__ void sum_rows(const T *P, int G, size_t nh, int N,
                                         typename GroupSum<T>::type *grp)
{
    const int cols = N / V, R = (int)blockDim.x / cols;
    const int t = threadIdx.x, q = t % cols, r = t / cols;
    if (r >= R) return;
    T s[V], c[V];
#pragma unroll
    for (int i = 0; i < V; ++i) s[i] = c[i] = T(0);
    auto add = [&](const T (&v)[V]) {
#pragma unroll
        for (int i = 0; i < V; ++i) {
            if constexpr (sizeof(T) == 4) kahan_add(s[i], c[i], v[i]);
            else s[i] += v[i];
        }
    };
    const T *p = P + (size_t)q * V;
    int b = r;
    // (eight rows in flight, then four: the loads' latency, not their
    // bandwidth, bounds this loop)
    for (; b + 7 * R < G; b += 8 * R) {
        T v[8][V];
#pragma unroll
        for (int i = 0; i < 8; ++i) load_vec<T, V>(p + (size_t)(b + i * R) * nh, v[i]);
#pragma unroll
        for (int i = 0; i < 8; ++i) add(v[i]);
    }
    for (; b + 3 * R < G; b += 4 * R) {
        T v0[V], v1[V], v2[V], v3[V];
        load_vec<T, V>(p + (size_t)b * nh, v0);
        load_vec<T, V>(p + (size_t)(b + R) * nh, v1);
        load_vec<T, V>(p + (size_t)(b + 2 * R) * nh, v2);
        load_vec<T, V>(p + (size_t)(b + 3 * R) * nh, v3);
        add(v0);
        add(v1);
        add(v2);
        add(v3);
    }
    for (; b < G; b += R) {
        T v[V];
        load_vec<T, V>(p + (size_t)b * nh, v);
        add(v);
    }
#pragma unroll
    for (int i = 0; i < V; ++i) grp[r * N + q * V + i] = {s[i], c[i]};
}

__device__ void sum_parts_axis(const CombineArgs *pa, int d, int N, double *sH)
{
    // R x N group sums, R N <= 4 blockDim (FP32), 2 blockDim (FP64)
    __shared__ __align__(16) unsigned char grp_raw[4096 * sizeof(float2)];
    const size_t nh = (size_t)pa->part_nh;
    const int G = pa->part_G;
    const int k = threadIdx.x;
    if (pa->part_f32) {
        float2 *grp = reinterpret_cast<float2 *>(grp_raw);
        const float *P = static_cast<const float *>(pa->part_H) + (size_t)d * N;
        const int V = N % 4 == 0 ? 4 : N % 2 == 0 ? 2 : 1;
        if (V == 4) sum_rows<float, 4>(P, G, nh, N, grp);
        else if (V == 2) sum_rows<float, 2>(P, G, nh, N, grp);
        else sum_rows<float, 1>(P, G, nh, N, grp);
        __syncthreads();
        if (k < N) {
            const int R = (int)blockDim.x / (N / V);
            float s = 0.0f, c = 0.0f;
            for (int r = 0; r < R; ++r) {
                const float2 g = grp[r * N + k];
                kahan_add(s, c, g.x);
                kahan_add(s, c, -g.y);
            }
            sH[k] = (double)s - (double)c;
        }
    } else {
        double2 *grp = reinterpret_cast<double2 *>(grp_raw);
        const double *P = static_cast<const double *>(pa->part_H) + (size_t)d * N;
        const int V = N % 2 == 0 ? 2 : 1;
        if (V == 2) sum_rows<double, 2>(P, G, nh, N, grp);
        else sum_rows<double, 1>(P, G, nh, N, grp);
        __syncthreads();
        if (k < N) {
            const int R = (int)blockDim.x / (N / V);
            double a[4] = {0.0, 0.0, 0.0, 0.0};
            for (int r = 0; r < R; ++r) a[r & 3] += grp[r * N + k].x;
            sH[k] = (a[0] + a[1]) + (a[2] + a[3]);
        }
    }
}

__device__ void refine_axis(int d, int N, double *H, double *edges, int zero_hist, float2 *ew32 = nullptr,
                            const MapParams *map = nullptr, const CombineArgs *pa = nullptr)
{
    double *Hd = H + (size_t)d * N;
    double *e = edges + (size_t)d * (N + 1);
    __shared__ double sH[CV_MAX_BINS], sq[CV_MAX_BINS];
    __shared__ double sC[CV_MAX_BINS + 1], se[CV_MAX_BINS + 1];
    __shared__ double wred[32];
    __shared__ double s_sum, s_inv, s_rmax, s_RN;
    const int k = threadIdx.x;            // bin of this thread
    const int lane = k & 31, warp = k >> 5;
    // the warps holding bins; the others (a CTA sized for the partial sums)
    // only meet the barriers: the FP64 pipe is a small fraction of FP32 here
    const int nw = (N + 31) >> 5;
    const bool act = warp < nw;
    const double invN = __drcp_rn((double)N);  // (off the dependent chain)

    if (pa && pa->part_H) sum_parts_axis(pa, d, N, sH);
    else if (k < N) sH[k] = Hd[k];
    for (int i = k; i <= N; i += blockDim.x) se[i] = e[i];
    __syncthreads();
    const bool bad = k < N && !isfinite(sH[k]);
    const bool nz = k < N && sH[k] != 0.0;
    const int any_bad = __syncthreads_or(bad);
    const int any_nz = __syncthreads_or(nz);
    if (!any_bad && any_nz) {
        // smoothing over the neighbours (correctly rounded: an even
        // histogram stays exactly even)
        double h = 0.0;
        if (k < N) {
            if (k == 0) h = __dmul_rn(__dadd_rn(sH[0], sH[1]), 0.5);
            else if (k == N - 1) h = __dmul_rn(__dadd_rn(sH[N - 2], sH[N - 1]), 0.5);
            else h = __ddiv_rn(__dadd_rn(__dadd_rn(sH[k - 1], sH[k]), sH[k + 1]), 3.0);
        }
        // s = sum_k h_k (warp sums, then the warps in order by one thread;
        // the per-axis scalars are computed once and shared)
        if (act) {
            const double ws = warp_sum_d(h);
            if (lane == 0) wred[warp] = ws;
        }
        __syncthreads();
        if (k == 0) {
            double t = 0.0;
            for (int w = 0; w < nw; ++w) t = __dadd_rn(t, wred[w]);
            s_sum = t;
            s_inv = __drcp_rn(t);
        }
        __syncthreads();
        const double s = s_sum;
        // compression r = ((1 - h/s) / ln(s/h))^1.5 = ((x - 1) / ln x)^1.5,
        // x = h/s in (0, 1]
        double r = 0.0;
        if (k < N && h != 0.0) {
            const double x = __dmul_rn(h, s_inv);
            if (h == s || !(x < 1.0)) {
                r = 1.0;
            } else {
                const double q = __dmul_rn(__dadd_rn(x, -1.0), __drcp_rn(log(x)));
                r = __dmul_rn(q, sqrt(q));
            }
        }
        if (act) {
            const long long wm = warp_max_bits(__double_as_longlong(r));
            if (lane == 0) wred[warp] = __longlong_as_double(wm);
        }
        __syncthreads();
        if (k == 0) {
            long long t = 0;
            for (int w = 0; w < nw; ++w) t = max(t, __double_as_longlong(wred[w]));
            s_rmax = __longlong_as_double(t);
            s_inv = t > 0 ? __drcp_rn(__longlong_as_double(t)) : 0.0;
        }
        __syncthreads();
        const long long rmax_bits = __double_as_longlong(s_rmax);
        if (rmax_bits > 0) {
            // scale to max 1 (the largest bins exactly 1)
            double c = 0.0;
            if (act) {
                r = (__double_as_longlong(r) == rmax_bits) ? 1.0 : __dmul_rn(r, s_inv);
                if (k < N) sq[k] = r > 0.0 ? __drcp_rn(r) : 0.0;
                // inclusive prefix sum C_(k+1) = r_0 + ... + r_k
                c = r;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const double t = __shfl_up_sync(0xffffffffu, c, o);
                    if (lane >= o) c = __dadd_rn(t, c);
                }
                if (lane == 31) wred[warp] = c;
            }
            __syncthreads();
            if (act) {
                double off = 0.0;
                for (int w = 0; w < warp; ++w) off = __dadd_rn(off, wred[w]);
                c = __dadd_rn(off, c);
                if (k < N) sC[k + 1] = c;
                if (k == 0) sC[0] = 0.0;
                if (k == N - 1) s_RN = __dmul_rn(c, invN);  // R / N, R = C_N
            }
            __syncthreads();
            const int m = k;
            if (m >= 1 && m < N) {
                // new edge m at compressed weight t = m R / N
                const double t = __dmul_rn((double)m, s_RN);
                // largest j in [0, N-1] with C_j <= t (C, t >= 0: bit-pattern compares)
                const long long tb = __double_as_longlong(t);
                int lo = 0, hi = N - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (__double_as_longlong(sC[mid]) <= tb) lo = mid;
                    else hi = mid - 1;
                }
                e[m] = __fma_rn(__dadd_rn(se[lo + 1], -se[lo]),
                                __dmul_rn(__dadd_rn(t, -sC[lo]), sq[lo]), se[lo]);
            }
        }
    }
    if (zero_hist && k < N) Hd[k] = 0.0;
    if (ew32) {
        __syncthreads();  // (the new edges of this axis, written by every thread)
        stage_axis(d, N, edges, ew32, *map, k, blockDim.x);
    }
}

// After a deterministic standalone pass: H[i] += the G blocks' partials of
// bin i.  32 bins per CTA, 8 threads per bin: thread j sums the blocks
// b = j (mod 8) in order (Kahan in FP32 for FP32 partials, FP64 else), and
// the 8 results are added in j order -- a fixed order, so deterministic.
__global__ void __launch_bounds__(256) k_add_parts(const void *part_H, int G, int f32, int nh, double *H)
{
    __shared__ double part[8][32];
    const int bin = threadIdx.x & 31, j = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + bin;
    double v = 0.0;
    if (i < nh) {
        if (f32) {
            const float *p = static_cast<const float *>(part_H) + i;
            float s = 0.0f, c = 0.0f;
            for (int b = j; b < G; b += 8) {
                const float y = p[(size_t)b * nh] - c;
                const float t = s + y;
                c = (t - s) - y;
                s = t;
            }
            v = (double)s - (double)c;
        } else {
            const double *p = static_cast<const double *>(part_H) + i;
            for (int b = j; b < G; b += 8) v += p[(size_t)b * nh];
        }
    }
    part[j][bin] = v;
    __syncthreads();
    if (j == 0 && i < nh) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += part[q][bin];
        H[i] += t;
    }
}

__global__ void __launch_bounds__(256) k_refine(int N, double *H, double *edges)
{
    refine_axis(blockIdx.x, N, H, edges, 0);
}

// Per component: fold the iteration result into the combination; thread 0
// then updates the iteration control.  The chi-square probability is only
// needed for the final answer and is evaluated when the run stops.
__device__ void combine_iteration(const CombineArgs &A)
{
    DevState *st = A.st;
    const int c = threadIdx.x;
    const long long n = st->n_cur;
    const int j = st->iter;
    __shared__ int s_ok[CV_MAX_COMP];
    __shared__ int s_bad[CV_MAX_COMP];
    __shared__ int s_stop;
    __shared__ double s_sum[2 * CV_MAX_COMP];
    if (A.part_S) {
        // the pass's sums, block partials added in block order: warp w takes
        // values w, w + warps, ...; lane l the blocks l, l + 32, ..., then a
        // fixed shuffle tree (as a pass's last block would)
        const int lane = c & 31, nwarp = (int)(blockDim.x >> 5);
        for (int v = c >> 5; v < 2 * A.ncomp; v += nwarp) {
            double acc = 0.0;
            for (int b = lane; b < A.part_G; b += 32) acc += __ldcg(&A.part_S[b * (2 * CV_MAX_COMP) + v]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) s_sum[v] = acc;
        }
        __syncthreads();
    }
    if (c < A.ncomp) {
        // every input first (independent loads), then the arithmetic: FP64
        // latency is high, so divisions are reciprocal multiplications
        // except where a reciprocal itself is the result
        const double S1 = A.part_S ? s_sum[2 * c] : st->S1[c];
        const double S2 = A.part_S ? s_sum[2 * c + 1] : st->S2[c];
        const double sumI0 = st->sumI[c], W0 = st->W[c], mean0 = st->mean[c], M20 = st->M2[c];
        int zero = st->zero[c];
        const double dn = (double)n;
        const double inv_n = __drcp_rn(dn);
        const double inv_n1 = __drcp_rn((double)(n - 1));
        const double I = __dmul_rn(S1, inv_n);
        const double var = __dmul_rn(__fma_rn(-I, I, __dmul_rn(S2, inv_n)), inv_n1);
        if (A.log_I && j < A.log_cap) {
            A.log_I[j * CV_MAX_COMP + c] = I;
            A.log_var[j * CV_MAX_COMP + c] = var;
        }
        const bool bad = !isfinite(I) || !isfinite(var);
        if (bad) atomicOr(&st->status, 1);
        s_bad[c] = bad;
        const int m = j + 1;
        const double sumI = sumI0 + I;
        st->sumI[c] = sumI;
        if (!(var > 0.0)) zero = 1;
        double W = W0, mean = mean0, M2 = M20;
        if (!zero) {
            const double w = __drcp_rn(var);
            W = W0 + w;
            const double dI = I - mean0;
            mean = __fma_rn(dI, __dmul_rn(w, __drcp_rn(W)), mean0);
            M2 = __fma_rn(__dmul_rn(w, dI), I - mean, M20);
            st->mean[c] = mean;
            st->W[c] = W;
            st->M2[c] = M2;
        } else {
            st->zero[c] = 1;
        }
        double integral, error, chi2;
        if (zero) {
            integral = sumI / (double)m;
            error = chi2 = 0.0;
        } else {
            integral = mean;
            error = rsqrt(W);
            chi2 = M2 > 0.0 ? M2 : 0.0;
        }
        st->integral[c] = integral;
        st->error[c] = error;
        st->chi2[c] = chi2;
        const double tol = fmax(A.epsabs, A.epsrel * fabs(integral));
        s_ok[c] = !bad && error <= tol;
        st->S1[c] = 0.0;
        st->S2[c] = 0.0;
    }
    __syncthreads();
    if (c == 0) {
        int ok = 1, bad = 0;
        for (int i = 0; i < A.ncomp; ++i) {
            ok &= s_ok[i];
            bad |= s_bad[i];
        }
        const long long neval = st->neval + n;
        st->neval = neval;
        st->iter = j + 1;
        const long long next = A.nstart + (long long)(j + 1) * A.nincrease;
        int stop = 0;
        if (bad) {
            // a non-finite iteration result (the integrand returned NaN or
            // Inf, or its squares overflowed): the run stops unconverged
            st->fail = 1;
            stop = 1;
        } else if (neval >= A.mineval && ok) {
            st->fail = 0;
            stop = 1;
        } else if (neval + next > A.maxeval) {
            st->fail = 1;
            stop = 1;
        } else {
            st->next_index += (unsigned long long)n;
            st->n_cur = next;
        }
        s_stop = stop;
    }
    __syncthreads();
    if (c < A.ncomp) {
        const int m = j + 1;
        st->prob[c] = (s_stop && !st->zero[c] && m > 1) ? gamma_p(0.5 * (m - 1), 0.5 * st->chi2[c]) : 0.0;
    }
    __syncthreads();
    // read by the next sampling launch only, so no block of this launch
    // sees the change
    if (c == 0 && s_stop) st->stopped = 1;
    if (c == 0 && A.host_stop) *(volatile int *)A.host_stop = s_stop;
}

// One Vegas iteration after its sampling pass: blocks 0..ndim-1 refine one
// axis each from the histogram (and clear it), block ndim combines the
// iteration.  Runs only if the sampling launch before it ran.
__global__ void __launch_bounds__(1024)
k_refine_combine(int ndim, int N, double *H, double *edges, const CombineArgs A, float2 *ew32, MapParams map)
{
    if (!*(volatile const int *)&A.st->pass_active) return;
    if ((int)blockIdx.x < ndim) refine_axis(blockIdx.x, N, H, edges, 1, ew32, &map, &A);
    else combine_iteration(A);
}

// Start of a run: uniform grid e_k = k/N, empty histogram and sums, Sobol
// index 1 (index 0, the all-zero point, is skipped).
__global__ void k_reset(DevState *st, double *edges, double *H, int ndim, int N, long long nstart, float2 *ew32,
                        MapParams map)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    for (int i = tid; i < ndim * (N + 1); i += stride) {
        const int k = i % (N + 1);
        edges[i] = (double)k / (double)N;
    }
    for (int i = tid; i < ndim * N; i += stride) H[i] = 0.0;
    int *w = reinterpret_cast<int *>(st);
    for (int i = tid; i < (int)(sizeof(DevState) / sizeof(int)); i += stride) w[i] = 0;
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->next_index = 1ull;
        st->n_cur = nstart;
    }
    if (ew32)  // (one block: the edges above are this block's own writes)
        for (int d = 0; d < ndim; ++d) stage_axis(d, N, edges, ew32, map, tid, stride);
}

__global__ void k_stage_grid(int ndim, int N, const double *edges, float2 *ew32, MapParams map)
{
    stage_axis(blockIdx.x, N, edges, ew32, map, threadIdx.x, blockDim.x);
}

// ---- batched forms: one CTA per integral (reset, combine) or per
// (integral, axis) (refine).  An integral whose run has stopped is skipped;
// its stop flag is only ever set by a later combine launch.
__global__ void k_batch_reset(const BatchItem *items, const CombineArgs *cargs, const int *list)
{
    const int i = list ? list[blockIdx.x] : (int)blockIdx.x;
    const BatchItem &it = items[i];
    const int N = it.a.nbins, ndim = it.a.g.ndim;
    for (int i = threadIdx.x; i < ndim * (N + 1); i += blockDim.x) {
        const int k = i % (N + 1);
        it.edges[i] = (double)k / (double)N;
    }
    for (int i = threadIdx.x; i < ndim * N; i += blockDim.x) it.H[i] = 0.0;
    int *w = reinterpret_cast<int *>(it.st);
    for (int i = threadIdx.x; i < (int)(sizeof(DevState) / sizeof(int)); i += blockDim.x) w[i] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        it.st->next_index = 1ull;
        it.st->n_cur = cargs[i].nstart;
    }
}

__global__ void __launch_bounds__(256) k_batch_refine(const BatchItem *items, const int2 *axes,
                                                      const TileParts *parts, const float *part_H)
{
    const int2 ax = axes[blockIdx.x];
    const BatchItem &it = items[ax.x];
    if (*(volatile const int *)&it.st->stopped) return;
    if (parts) {
        // the histogram of the integral's tiles, rows added in tile order
        const TileParts tp = parts[ax.x];
        CombineArgs pa;
        pa.part_H = part_H + tp.hoff0;
        pa.part_G = tp.count;
        pa.part_nh = tp.stride;
        pa.part_f32 = 1;
        refine_axis(ax.y, it.a.nbins, it.H, it.edges, 1, nullptr, nullptr, &pa);
    } else {
        refine_axis(ax.y, it.a.nbins, it.H, it.edges, 1);
    }
}

__global__ void k_batch_combine(const CombineArgs *cargs, const int *list, const TileParts *parts,
                                const double *part_S)
{
    const int i = list ? list[blockIdx.x] : (int)blockIdx.x;
    const CombineArgs &A = cargs[i];
    if (*(volatile const int *)&A.st->stopped) return;
    if (parts) {
        // the sums of the integral's tiles, rows added in tile order
        CombineArgs B = A;
        B.part_S = part_S + (size_t)parts[i].row0 * (2 * CV_MAX_COMP);
        B.part_G = parts[i].count;
        combine_iteration(B);
    } else {
        combine_iteration(A);
    }
}

cudaError_t launch_batch_reset(const BatchItem *items, const CombineArgs *cargs, int count,
                               cudaStream_t s, const int *list)
{
    if (count <= 0) return cudaSuccess;
    k_batch_reset<<<count, 256, 0, s>>>(items, cargs, list);
    return cudaGetLastError();
}

// Copy the states of the listed integrals into one contiguous array.
__global__ void k_gather_states(const BatchItem *items, const int *list, DevState *out)
{
    const int *src = reinterpret_cast<const int *>(items[list[blockIdx.x]].st);
    int *dst = reinterpret_cast<int *>(out + blockIdx.x);
    for (int i = threadIdx.x; i < (int)(sizeof(DevState) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
}

cudaError_t launch_gather_states(const BatchItem *items, const int *list, int count, DevState *out,
                                 cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    k_gather_states<<<count, 32, 0, s>>>(items, list, out);
    return cudaGetLastError();
}

cudaError_t launch_batch_refine(const BatchItem *items, const int2 *axes, int naxes, cudaStream_t s,
                                const TileParts *parts, const float *part_H)
{
    if (naxes <= 0) return cudaSuccess;
    k_batch_refine<<<naxes, 256, 0, s>>>(items, axes, parts, part_H);
    return cudaGetLastError();
}

cudaError_t launch_batch_combine(const CombineArgs *cargs, int count, cudaStream_t s, const int *list,
                                 const TileParts *parts, const double *part_S)
{
    if (count <= 0) return cudaSuccess;
    k_batch_combine<<<count, 32, 0, s>>>(cargs, list, parts, part_S);
    return cudaGetLastError();
}

cudaError_t launch_reset(DevState *st, double *edges, double *H, int ndim, int nbins,
                         long long nstart, float2 *ew32, const MapParams &map, cudaStream_t s)
{
    k_reset<<<1, 256, 0, s>>>(st, edges, H, ndim, nbins, nstart, ew32, map);
    return cudaGetLastError();
}

cudaError_t launch_stage_grid(int ndim, int nbins, const double *edges, float2 *ew32,
                              const MapParams &map, cudaStream_t s)
{
    k_stage_grid<<<ndim, 256, 0, s>>>(ndim, nbins, edges, ew32, map);
    return cudaGetLastError();
}

// Threads of a refinement CTA: the bins rounded up to whole warps, at least
// two warps (the combination CTA of k_refine_combine needs one).
static int refine_threads(int nbins) { return nbins <= 64 ? 64 : (nbins + 31) / 32 * 32; }

cudaError_t launch_add_parts(const void *part_H, int G, int f32, int nh, double *H, cudaStream_t s)
{
    k_add_parts<<<(nh + 31) / 32, 256, 0, s>>>(part_H, G, f32, nh, H);
    return cudaGetLastError();
}

cudaError_t launch_refine(int ndim, int nbins, double *H, double *edges, cudaStream_t s)
{
    k_refine<<<ndim, refine_threads(nbins), 0, s>>>(nbins, H, edges);
    return cudaGetLastError();
}

cudaError_t launch_refine_combine(int ndim, int nbins, double *H, double *edges,
                                  const CombineArgs &a, float2 *ew32, const MapParams &map,
                                  cudaStream_t s)
{
    // (with many block partials to add, a full CTA per axis: see
    // sum_parts_axis; a few are summed by the threads of the bins)
    const int threads = a.part_H && a.part_G >= 64 ? 1024 : refine_threads(nbins);
    k_refine_combine<<<ndim + 1, threads, 0, s>>>(ndim, nbins, H, edges, a, ew32, map);
    return cudaGetLastError();
}

}  // namespace cv
