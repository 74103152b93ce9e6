"""The arithmetic of the block coarse solve's tensor-core products, restated on the CPU.

With more than two right-hand sides the block products W_i X of the coarse sweeps are
formed from digit slices: each row of A = [Re W | Im W] and each column of B is scaled
by a power of two 2^e bounding it, |v| 2^(56 - e) is truncated to an integer and cut into
8 signed 7-bit digits; the 36 slice pairs (s, t) with s + t <= 9 are multiplied (bf16
digits, FP32 accumulation on the tensor cores) and summed with the weights 2^-7(s+t).
This file restates those steps with exact integers and checks what the design relies on:

* digits reconstruct the truncated value exactly, and the truncation loses less than
  2^(e - 56);
* every slice-pair sum of K <= 1040 terms stays below 2^24 (so FP32 accumulation is
  exact), including the worst case of all digits 127;
* the kept pairs give the product to within 2^-50.5 K max|A_r| max|B_c| (the documented
  bound), checked against the exact rational product on random and adversarial inputs.
"""
from fractions import Fraction

import numpy as np
import pytest

S, BETA = 8, 7


def exponent(m):
    """e with |v| < 2^e for the largest |v| = m (0 for m = 0)."""
    if m == 0:
        return 0
    return int(np.frexp(m)[1])          # m = f 2^E, 0.5 <= f < 1  ->  m < 2^E


def digits(v, e):
    """Sign and the 8 digits of trunc(|v| 2^(56 - e))."""
    if v == 0:
        return 0, [0] * S
    a = int(Fraction(abs(v)) * Fraction(2) ** (56 - e))    # truncation toward zero
    assert a < 2 ** 56
    return (-1 if v < 0 else 1), [(a >> (56 - BETA * s)) & 127 for s in range(1, S + 1)]


def sliced_product(A, B):
    """The kept-pair product of the design, exactly: rows of A and columns of B sliced."""
    M, K = A.shape
    N = B.shape[1]
    er = [exponent(np.max(np.abs(A[r]))) for r in range(M)]
    fc = [exponent(np.max(np.abs(B[:, c]))) for c in range(N)]
    Ad = np.zeros((S, M, K), dtype=np.int64)
    Bd = np.zeros((S, K, N), dtype=np.int64)
    for r in range(M):
        for k in range(K):
            sg, d = digits(A[r, k], er[r])
            Ad[:, r, k] = [sg * x for x in d]
    for c in range(N):
        for k in range(K):
            sg, d = digits(B[k, c], fc[c])
            Bd[:, k, c] = [sg * x for x in d]
    out = [[Fraction(0)] * N for _ in range(M)]
    for s in range(1, S + 1):
        for t in range(1, S + 1):
            if s + t > 9:
                continue
            P = Ad[s - 1] @ Bd[t - 1]                      # exact in int64
            assert np.max(np.abs(P)) < 2 ** 24             # exact in FP32 as well
            for r in range(M):
                for c in range(N):
                    out[r][c] += Fraction(int(P[r, c])) * Fraction(2) ** (er[r] + fc[c] - BETA * (s + t))
    return out


def exact_product(A, B):
    M, K = A.shape
    N = B.shape[1]
    return [[sum(Fraction(A[r, k]) * Fraction(B[k, c]) for k in range(K)) for c in range(N)] for r in range(M)]


def test_digits_reconstruct_the_truncated_value():
    rng = np.random.default_rng(1)
    for v in list(rng.standard_normal(200) * 10.0 ** rng.integers(-30, 30, 200)) + [1.0, -0.5, 2.0 ** -40]:
        e = exponent(abs(v)) + int(rng.integers(0, 20))          # row scales at or above |v|
        sg, d = digits(v, e)
        rec = sg * sum(Fraction(x) * Fraction(2) ** (e - BETA * s) for s, x in zip(range(1, S + 1), d))
        assert all(0 <= x <= 127 for x in d)
        assert abs(Fraction(v) - rec) < Fraction(2) ** (e - 56)
        assert abs(rec) <= abs(Fraction(v))                       # truncation toward zero


def test_pair_sums_fit_fp32_at_the_largest_k():
    """K terms of the largest digit product stay below 2^24 up to K = 1040 and not beyond:
    the limit 2b <= 1040 on the block width (b <= 520)."""
    assert 1040 * 127 * 127 < 2 ** 24 <= 1041 * 127 * 127


@pytest.mark.parametrize("case", ["gaussian", "scaled_rows", "cancelling", "widest"])
def test_kept_pairs_meet_the_bound(case):
    rng = np.random.default_rng({"gaussian": 2, "scaled_rows": 3, "cancelling": 4, "widest": 5}[case])
    M, N, K = 3, 2, 64
    if case == "widest":
        K = 1028                                      # 2b at the widest blocks (b = 514)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    if case == "scaled_rows":
        A *= 10.0 ** rng.integers(-12, 12, (M, K))   # entries far below their row's maximum
    if case == "cancelling":
        B[:, 1] = -B[:, 0] + 1e-9 * rng.standard_normal(K)
        A[:, K // 2:] = A[:, :K // 2]                # sums that nearly cancel
    Y = sliced_product(A, B)
    X = exact_product(A, B)
    for r in range(M):
        for c in range(N):
            lim = K * float(np.max(np.abs(A[r]))) * float(np.max(np.abs(B[:, c]))) * 2.0 ** -50.5
            assert abs(float(Y[r][c] - X[r][c])) <= lim, (case, r, c)


def test_worst_case_digits_stay_exact():
    """Values just below the row and column scales (their first seven digits 127) at K = 1028."""
    K = 1028
    v = 1.0 - 2.0 ** -53
    A = np.full((1, K), v)
    B = np.full((K, 1), -v)
    Y = sliced_product(A, B)                           # asserts every pair sum < 2^24
    X = exact_product(A, B)
    assert abs(float(Y[0][0] - X[0][0])) <= K * 2.0 ** -50.5
