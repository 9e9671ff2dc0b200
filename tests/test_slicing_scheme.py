"""The exact-slicing scheme of the FP64-accurate tensor-core GEMM, checked on the CPU.

The GPU kernel (tc_zgemm_oz_kernel) relies on three facts, restated here in NumPy and checked
against exact arithmetic (Python integers and fractions), with no GPU and no library code:
  1. five round-to-nearest slices of 8 bits under the row's power of two reconstruct x to
     2^(e - 41), with |s0| <= 256 and |s1..s4| <= 128, and every plane value (s_i scaled by
     2^-8i) has at most 9 significant bits, so it is exact in TF32 (11 bits);
  2. over a chunk of 128 real K the integer sums T0, T1, T2 stay at or below 2^24 in magnitude,
     so the FP32 accumulator holds them exactly (the kernel's chunk length is read from its source);
  3. the dot product assembled as the kernel does (exact T0, T1, T2; T accumulated in FP32;
     terms with i + j > 4 dropped) is within 2^-40 n max|a| max|b| of the exact one (each term's
     error is set by the row's and the column's largest magnitude, not by the term itself).
"""
import os
import re
from fractions import Fraction

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def exponent(amax):
    return int(np.frexp(amax)[1]) if amax > 0 else 0


def slices(x, e):
    t = np.ldexp(x, 8 - e)
    out = []
    for i in range(5):
        s = np.rint(t)
        out.append(s)
        t = (t - s) * 256.0
    return np.array(out)


def significant_bits(v):
    """Bits between the leading one and the lowest set bit of a float64 (0 for 0)."""
    if v == 0:
        return 0
    m, _ = np.frexp(abs(v))
    f = Fraction(float(m))                  # m in [1/2, 1) = odd / 2^k: k significant bits
    return f.denominator.bit_length() - 1


def test_slices_reconstruct_and_fit_tf32():
    rng = np.random.default_rng(3)
    for scale in (1e-6, 1.0, 3e4):
        row = rng.normal(size=400) * scale * np.exp(rng.normal(size=400))
        e = exponent(np.abs(row).max())
        S = slices(row, e)
        assert np.abs(S[0]).max() <= 256 and np.abs(S[1:]).max() <= 128
        recon = sum(S[i] * 2.0 ** (e - 8 * (i + 1)) for i in range(5))
        assert np.abs(recon - row).max() <= 2.0 ** (e - 41)
        planes = [S[0], S[1], S[2], S[1] * 2.0 ** -8, S[2] * 2.0 ** -16, S[3] * 2.0 ** -24, S[4] * 2.0 ** -32]
        for p in planes:
            assert max(significant_bits(v) for v in p) <= 9


def test_chunk_sums_stay_exact_in_fp32():
    src = open(os.path.join(ROOT, "paper_2208_07478_gb300", "csrc", "tc_gemm.cu")).read()
    stages = int(re.search(r"constexpr int OZ_CHUNK_STAGES = (\d+);", src).group(1))
    kc = stages * 16   # 16 real K per stage
    # worst case per real K: |s0| <= 256, |s1|, |s2| <= 128 (same for t)
    t0 = 256 * 256
    t1 = 256 * 128 + 128 * 256
    t2 = 256 * 128 + 128 * 128 + 128 * 256
    assert kc * max(t0, t1, t2) <= 2 ** 24, (kc, max(t0, t1, t2))


def sliced_dot(a, b):
    """The kernel's assembly for one real dot product: exact integer T0, T1, T2, FP32 T."""
    ea, eb = exponent(np.abs(a).max()), exponent(np.abs(b).max())
    S, T = slices(a, ea), slices(b, eb)
    Si, Ti = S.astype(np.int64), T.astype(np.int64)
    T0 = int((Si[0] * Ti[0]).sum())
    T1 = int((Si[0] * Ti[1] + Si[1] * Ti[0]).sum())
    T2 = int((Si[0] * Ti[2] + Si[1] * Ti[1] + Si[2] * Ti[0]).sum())
    rest = np.float32(0.0)
    for i in range(5):
        for j in range(5):
            if 3 <= i + j <= 4:
                pa = (S[i] * 2.0 ** (-8 * i)).astype(np.float32)
                pb = (T[j] * 2.0 ** (-8 * j)).astype(np.float32)
                for k in range(len(a)):
                    rest = np.float32(rest + pa[k] * pb[k])
    exact_part = Fraction(T0) * Fraction(2) ** -16 + Fraction(T1) * Fraction(2) ** -24 + Fraction(T2) * Fraction(2) ** -32
    return (exact_part + Fraction(float(rest)) * Fraction(2) ** -16) * Fraction(2) ** (ea + eb)


def test_sliced_dot_error_bound():
    rng = np.random.default_rng(11)
    for n in (16, 128):
        for trial in range(4):
            a = rng.normal(size=n) * np.exp(rng.normal(size=n))
            b = rng.normal(size=n) * np.exp(rng.normal(size=n))
            exact = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))
            got = sliced_dot(a, b)
            scale = Fraction(float(np.abs(a).max())) * Fraction(float(np.abs(b).max())) * n
            assert abs(got - exact) <= Fraction(2) ** -40 * scale, (n, trial, float(abs(got - exact) / scale))
