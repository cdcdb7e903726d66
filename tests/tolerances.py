"""Tolerances of the CUDA path against the FP64 oracle (shared by the GPU tests).

FP64 path (same operations, FP64 sums in another order): S1, S2 and the
iteration variance within 1e-12 relative.

FP32 path (point, map and integrand in binary32, Kahan per thread, FP64
between blocks), per sampling pass on the same grid -- 1e-6 relative, the
mixed-precision bound, measured against the sum of magnitudes so that it
does not vanish for an oscillatory integrand whose sum cancels:

  |S1 - S1o| <= 1e-6 * A1 + B1            A1 = sum |J f_c| (= S1o when f > 0)
  |S2 - S2o| <= 1e-6 * S2o + B2
  |H - Ho|   <= 1e-5 * max_k Ho[d, k] + B2[0]   per bin

B1, B2 are the oracle's boundary mass: the discontinuous family's points
whose FP64 coordinate lies within 2^-20 (sixteen binary32 units at 1) of a
cut, which a binary32 evaluation of the point may put on either side (zero
for every other family).  The histogram bound is looser than the sums' because each bin is a
short FP32 running sum in shared memory before it reaches FP64.

The iteration variance var = (S2/n - (S1/n)^2)/(n-1) follows from the two
sum bounds b1 = 1e-6 A1 + B1 and b2 = 1e-6 S2o + B2:

  |var - var_o| <= (b2/n + (2 |S1o| b1 + b1^2)/n^2)/(n-1) + 1e-15 (S2o/n)/(n-1)

(the last term is the FP64 rounding of the formula itself).
"""
import numpy as np

FP32_REL = 1e-6
FP32_HIST = 1e-5


def fp32_sum_bounds(ob, c):
    """(b1, b2): bounds on |dS1|, |dS2| of component c for oracle pass ob."""
    b1 = FP32_REL * ob.A1[c] + ob.B1[c]
    b2 = FP32_REL * ob.S2[c] + ob.B2[c]
    return b1, b2


def fp32_var_bound(ob, c, n):
    b1, b2 = fp32_sum_bounds(ob, c)
    S1, S2 = ob.S1[c], ob.S2[c]
    return (b2 / n + (2 * abs(S1) * b1 + b1 * b1) / (n * n)) / (n - 1) + 1e-15 * (S2 / n) / (n - 1)


def variance(S1, S2, n):
    I = S1 / n
    return (S2 / n - I * I) / (n - 1)


def check_fp32_pass(S1, S2, H, ob, n, ncomp=None, what=""):
    """Assert a GPU FP32 pass (S1, S2, H) against oracle pass bounds ob."""
    ncomp = len(ob.S1) if ncomp is None else ncomp
    for c in range(ncomp):
        b1, b2 = fp32_sum_bounds(ob, c)
        assert abs(S1[c] - ob.S1[c]) <= b1, (what, c, "S1", S1[c], ob.S1[c], b1)
        assert abs(S2[c] - ob.S2[c]) <= b2, (what, c, "S2", S2[c], ob.S2[c], b2)
        if n > 1:
            vb = fp32_var_bound(ob, c, n)
            vg, vo = variance(S1[c], S2[c], n), variance(ob.S1[c], ob.S2[c], n)
            assert abs(vg - vo) <= vb, (what, c, "var", vg, vo, vb)
    if H is not None:
        scale = ob.H.max(axis=1, keepdims=True)
        assert np.all(np.abs(H - ob.H) <= FP32_HIST * scale + ob.B2[0]), (what, "H")


def check_fp32_iteration(I, var, ob, n, ncomp=None, what=""):
    """Assert one logged FP32 iteration (I_j = S1/n, var_j) against ob."""
    ncomp = len(ob.S1) if ncomp is None else ncomp
    for c in range(ncomp):
        b1, _ = fp32_sum_bounds(ob, c)
        assert abs(I[c] - ob.S1[c] / n) <= b1 / n + 1e-15 * abs(ob.S1[c] / n), (what, c, "I", I[c], ob.S1[c] / n)
        vo = variance(ob.S1[c], ob.S2[c], n)
        assert abs(var[c] - vo) <= fp32_var_bound(ob, c, n), (what, c, "var", var[c], vo)
