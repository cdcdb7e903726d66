"""Writes sobol_dirs.h, the Sobol direction words of the CUDA path.

Build step, run by hand when the table has to change (the header is
committed, so the library build needs no scipy).  The primitive polynomials
and initial direction numbers are the Joe-Kuo set (new-joe-kuo-6.21201)
as scipy ships it; the words are expanded here with the Sobol (1967)
recurrence over GF(2) written as a shift-register update on whole words,
and the first 2^17 points they generate are checked against scipy's own
unscrambled Sobol engine before the header is written.

Word layout: V[d][k] is the direction number for bit k of the Gray-code
index, the binary fraction m_{k+1} / 2^{k+1} stored in the top k+1 bits of
a 64-bit word (V = m_{k+1} << (63 - k)).  For k < 52 the low 12 bits are
zero, so every point of an index below 2^52 is a multiple of 2^-52.

The tables are written in step form W: W[d][k] = V[d][k] for k < 5 and
W[d][k] = V[d][4] ^ V[d][k] for k >= 5.  The kernels advance a warp's 32
lanes from one aligned block of 32 indices to the next by flipping Gray-code
bits 4 and 5 + c together, so one step is a single XOR with W[d][5 + c];
skip-ahead recovers V[d][k] = W[d][k] ^ W[d][4].

usage: python gen_sobol_dirs.py [out_path]
"""
import os
import sys

import numpy as np

MAX_DIM = 32
NBITS = 52  # index bits supported: indices 0 .. 2^52 - 1


def joe_kuo():
    import scipy.stats._sobol as s
    z = np.load(os.path.join(os.path.dirname(s.__file__), "_sobol_direction_numbers.npz"))
    return z["poly"], z["vinit"]


def direction_words(ndim: int) -> list:
    poly, vinit = joe_kuo()
    table = []
    for d in range(ndim):
        if d == 0:
            words = [1 << (63 - k) for k in range(NBITS)]
        else:
            p = int(poly[d])
            deg = p.bit_length() - 1
            # coefficient list c_1..c_{deg-1} of x^{deg-1}..x^1
            inner = [(p >> (deg - j)) & 1 for j in range(1, deg)]
            words = [int(vinit[d, k]) << (63 - k) for k in range(deg)]
            for k in range(deg, NBITS):
                # v_k = v_{k-deg} ^ (v_{k-deg} >> deg) ^ XOR_j c_j v_{k-j}
                w = words[k - deg] ^ (words[k - deg] >> deg)
                for j, c in enumerate(inner, start=1):
                    if c:
                        w ^= words[k - j]
                words.append(w)
        table.append(words)
    return table


def slot_positions(L: int) -> dict:
    """Bit position of y_t (t = 1..29) in the mapped 32-bit word for
    N = 2^L bins, 5 <= L <= 8.

    With y_t the bit of weight 2^-t of y = w / 2^32 (y_1 = bit 31):
      bits 31..32-L     the bin's shared-memory slot
                        s = (y_6 .. y_L) * 32 + y_5 * 16 + (y_1 .. y_4)
      bits 31-L..29-L   zero, so word >> (29 - L) = 8 s, the byte offset of
                        the bin's 8-byte grid entry
      y_(L+1) .. y_23   the fraction within the bin, at mantissa bits
                        top .. top - 22 + L, top = min(22, 28 - L)
      y_24 .. y_29      the free positions from the top down
    y_30 .. y_32 are dropped (the FP32 coordinate keeps 23 bits); the map is
    linear over GF(2), so it commutes with the XOR recurrence.
    """
    top = min(22, 28 - L)
    pos = {}
    for t in range(1, 5):
        pos[t] = 32 - L + (4 - t)
    pos[5] = 32 - L + 4
    for t in range(6, L + 1):
        pos[t] = 37 - t
    for t in range(L + 1, 24):
        pos[t] = top - (t - L - 1)
    used = set(pos.values()) | {31 - L, 30 - L, 29 - L}
    free = [b for b in range(31, -1, -1) if b not in used]
    for t, b in zip(range(24, 30), free):
        pos[t] = b
    return pos


def slot_perm(w32: int, L: int) -> int:
    """The mapped word of slot_positions(L)."""
    out = 0
    for t, b in slot_positions(L).items():
        out |= ((w32 >> (32 - t)) & 1) << b
    return out


def step_form(words: list) -> list:
    """W[k] = V[k] for k < 5, V[4] ^ V[k] for k >= 5."""
    return [w if k < 5 else (words[4] ^ w) for k, w in enumerate(words)]


def check_against_scipy(table, npts=1 << 17):
    from scipy.stats import qmc
    ndim = len(table)
    ref = qmc.Sobol(ndim, scramble=False, bits=52).random(npts)
    X = np.zeros(ndim, dtype=np.uint64)
    V = np.array(table, dtype=np.uint64)
    for i in range(1, npts):
        # Gray code: g(i) ^ g(i-1) = 2^ctz(i)
        k = (i & -i).bit_length() - 1
        X ^= V[:, k]
        got = (X >> np.uint64(12)).astype(np.float64) / 2.0 ** 52
        if not np.array_equal(got, ref[i]):
            raise SystemExit(f"direction words disagree with scipy at index {i}")


def main():
    out = sys.argv[1] if len(sys.argv) > 1 else os.path.join(
        os.path.dirname(os.path.abspath(__file__)), "sobol_dirs.h")
    table = direction_words(MAX_DIM)
    check_against_scipy(table)
    steps = [step_form(words) for words in table]
    for L in (5, 6, 7, 8):
        pos = slot_positions(L)
        # 29 source bits to 29 distinct positions, the three gap bits never set
        assert len(set(pos.values())) == 29 and not {31 - L, 30 - L, 29 - L} & set(pos.values())
        assert all(slot_perm(1 << (32 - t), L) == 1 << b for t, b in pos.items())
    for words, w in zip(table, steps):
        assert [x if k < 5 else x ^ w[4] for k, x in enumerate(w)] == words
    lines = [
        "/* Generated by gen_sobol_dirs.py -- do not edit.",
        " * Sobol direction words, Joe-Kuo primitive polynomials and initial",
        " * numbers (new-joe-kuo-6.21201), in step form: with",
        " * V[d][k] = m_{d,k+1} << (63-k), the direction number of Gray-code index",
        " * bit k in dimension d as a 64-bit fraction, entry [d][k] is V[d][k] for",
        " * k < 5 and V[d][4] ^ V[d][k] for k >= 5; as 64-bit words (W64) and as",
        " * their top 32 bits (W32P[0]), also bit-mapped for N = 2^L bins,",
        " * L = 5..8 (W32P[L - 4]; see slot_positions in the generator). */",
        "#pragma once",
        f"#define CV_SOBOL_DIMS {MAX_DIM}",
        f"#define CV_SOBOL_BITS {NBITS}",
        "#define CV_SOBOL_W64_INIT { \\",
    ]
    for d, words in enumerate(steps):
        body = ", ".join(f"0x{w:016x}ull" for w in words)
        lines.append(f"  {{{body}}}, \\")
    lines.append("}")
    # top-32-bit words: table 0 as they are, tables 1..4 permuted for
    # N = 2^L, L = 5, 6, 7, 8 (slot_perm)
    lines.append("#define CV_SOBOL_W32P_INIT { \\")
    for L in (0, 5, 6, 7, 8):
        lines.append("  { \\")
        for d, words in enumerate(steps):
            body = ", ".join(f"0x{(slot_perm(w >> 32, L) if L else w >> 32):08x}u" for w in words)
            lines.append(f"    {{{body}}}, \\")
        lines.append("  }, \\")
    lines.append("}")
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(f"wrote {out}")


if __name__ == "__main__":
    main()
