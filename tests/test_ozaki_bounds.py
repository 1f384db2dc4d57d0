"""The arithmetic facts the tensor-core FP64 product (exact bf16 slices) rests
on, checked on the CPU with an independent numpy restatement of the slicing:
8 slices of 7 bits on the grid of each row's largest exponent, integers that
bf16 holds exactly, a remainder below 2^(e - 57), and level sums over chunks
of 256 products that stay below 2^24 (every integer up to 2^24 is an FP32
value, so FP32 accumulation of them is exact).
The slice-level sum reconstructs the FP64 product to a few units of the last
place."""
import numpy as np
import pytest


def slices(x, e, s=8):
    """Rows of x on the grid 2^(e_r - 7 i): integer slices q_i and the remainder."""
    y = np.ldexp(x, -e[:, None])
    out = []
    for _ in range(s):
        y = y * 128.0
        q = np.rint(y)
        y = y - q
        out.append(q)
    return np.stack(out), y


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
    x = rng.standard_normal((40, 300)) * np.exp(rng.uniform(-20, 20, size=(40, 1)))
    e = row_exponents(x)
    q, rem = slices(x, e)
    assert np.all(q == np.rint(q))
    assert np.abs(q[0]).max() <= 128 and np.abs(q[1:]).max() <= 64
    assert bf16_exact(q)
    # x = sum_i q_i 2^(e - 7 i) + remainder, remainder below 2^(e - 57)
    recon = sum(np.ldexp(q[i], e[:, None] - 7 * (i + 1)) for i in range(8))
    assert np.all(np.abs(x - recon) <= np.ldexp(1.0, e[:, None] - 57))


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
