"""The arithmetic facts the tensor-core FP64 product (exact bf16 slices) rests
on, checked on the CPU with an independent restatement of the slicing in exact
integer arithmetic: 8 slices of 7 bits on the grid of each row's largest
exponent (Y = |x| 2^(56 - e) rounded half up, balanced base-128 digits),
integers that bf16 holds exactly, a remainder below 2^(e - 57), and level
sums over chunks of 256 products that stay below 2^24 (every integer up to
2^24 is an FP32 value, so FP32 accumulation of them is exact).
The slice-level sum reconstructs the FP64 product to a few units of the last
place."""
from fractions import Fraction

import numpy as np
import pytest


def digits_of(x, e, s=8):
    """Balanced base-128 digits q_1..q_s of x on the grid 2^e (|x| < 2^e):
    Y = round(|x| 2^(56 - e)) (half up), then digits in [-64, 63] from the
    bottom, the top one in [0, 128]; signed like x."""
    mag = abs(Fraction(float(x))) * Fraction(2) ** (56 - int(e))
    Y = int(mag + Fraction(1, 2))  # floor(mag + 1/2): round half up
    d = []
    for _ in range(s - 1):
        g = Y % 128
        if g >= 64:
            g -= 128
        d.append(g)
        Y = (Y - g) // 128
    d.append(Y)
    sign = -1 if x < 0 else 1
    return [sign * v for v in reversed(d)]


def slices(x, e, s=8):
    """Rows of x on the grid 2^(e_r - 7 i): integer slices q_i and the remainder."""
    R, K = x.shape
    q = np.zeros((s, R, K))
    rem = np.zeros((R, K))
    for r in range(R):
        for k in range(K):
            dig = digits_of(x[r, k], e[r], s)
            q[:, r, k] = dig
            exact = sum(Fraction(v) * Fraction(2) ** (int(e[r]) - 7 * (i + 1)) for i, v in enumerate(dig))
            rem[r, k] = float(Fraction(float(x[r, k])) - exact)
    return q, rem


def row_exponents(x):
    mx = np.abs(x).max(axis=1)
    _, ex = np.frexp(mx)
    return np.where(mx > 0, ex, 0)


def bf16_exact(q):
    """True where q is exactly representable in bf16 (8 significant bits)."""
    f = q.astype(np.float32)
    bits = f.view(np.uint32)
    return np.all((bits & 0xFFFF) == 0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_slices_are_exact_bf16_integers_with_small_remainder(seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((12, 40)) * np.exp(rng.uniform(-20, 20, size=(12, 1)))
    # edge values in the last rows: the row maximum itself, values just below a
    # power of two, ties of the rounding, subnormals, zeros, both signs
    x[-1, :8] = [np.nextafter(1.0, 0.0), -np.nextafter(1.0, 0.0), 0.5, -0.25, 2.0 ** -56, 3 * 2.0 ** -57,
                 -(2.0 ** -57), 0.0]
    x[-2, :6] = [5e-324, -5e-324, 2.2e-308, -1e-310, 4e-320, 0.0]
    e = row_exponents(x)
    q, rem = slices(x, e)
    assert np.all(q == np.rint(q))
    assert np.abs(q[0]).max() <= 128 and np.abs(q[1:]).max() <= 64
    assert bf16_exact(q)
    # x = sum_i q_i 2^(e - 7 i) + remainder, remainder at most 2^(e - 57)
    assert np.all(np.abs(rem) <= np.ldexp(1.0, e[:, None] - 57))


def test_digit_carry_constant_and_worst_cases():
    """64 (1 + 128 + ... + 128^6) is the constant the slicing adds; the top
    digit reaches 128 just below 2^e (1 - 2^-53 = 128 2^-7 - 8 2^-56), the
    others stay in [-64, 63]."""
    assert sum(64 * 128 ** j for j in range(7)) == 0x0001020408102040
    top = digits_of(np.nextafter(1.0, 0.0), 0)
    assert top == [128, 0, 0, 0, 0, 0, 0, -8]
    low = digits_of(-(1.0 - 2.0 ** -50), 0)
    assert abs(low[0]) <= 128 and all(-64 <= -v <= 63 for v in low[1:])
    for x in (0.3, -0.7, 2.0 ** -30, 1 - 2.0 ** -8):
        d = digits_of(x, 0)
        assert all(-64 <= (v if x > 0 else -v) <= 63 for v in d[1:]) and 0 <= abs(d[0]) <= 128


def test_level_sums_over_a_chunk_stay_below_2_24():
    """Worst case: every slice at its bound, 256 products per chunk (the top
    levels reach 2^23.3)."""
    for L in range(2, 10):
        pairs = [(i, L - i) for i in range(1, L) if 1 <= L - i <= 8 and i <= 8]
        bound = sum((128 if i == 1 else 64) * (128 if j == 1 else 64) for i, j in pairs) * 256
        assert bound < 2 ** 24, (L, bound)


@pytest.mark.parametrize("m,n,k", [(16, 12, 300), (8, 8, 1000)])
def test_level_sum_product_matches_fp64(m, n, k):
    """sum_L 2^(e_r + f_c - 7L) sum_{i+j=L} Q_i P_j reproduces A B to a few ulps
    of |A||B| (exact integer level sums, FP64 combination)."""
    rng = np.random.default_rng(m + n + k)
    A = rng.standard_normal((m, k))
    B = rng.standard_normal((k, n))
    ea, fb = row_exponents(A), row_exponents(B.T)
    qa, _ = slices(A, ea)
    qb, _ = slices(B.T, fb)
    C = np.zeros((m, n))
    for L in range(2, 10):
        acc = np.zeros((m, n))
        for i in range(1, 9):
            j = L - i
            if 1 <= j <= 8:
                acc += qa[i - 1] @ qb[j - 1].T  # integers below 2^53: exact in FP64 here
        C += np.ldexp(acc, (ea[:, None] + fb[None, :]) - 7 * L)
    ref = A @ B
    scale = np.abs(A) @ np.abs(B)
    assert np.abs(C - ref).max() <= 2 * k * 2.0 ** -53 * scale.max()
