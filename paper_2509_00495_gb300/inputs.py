"""Seeded synthetic test matrices (input generation only).

Both the CUDA path's tests/benchmark and the CPU oracle draw their inputs from
here; the module holds none of the eigensolver's arithmetic.  The recipe
follows the paper's test-matrix construction (Appendix B, ``my_randsvd``: a
random orthogonal matrix times a prescribed spectrum times its transpose,
then symmetrized), with a Haar-random orthogonal factor and genuinely random
eigenvalue signs:

* Haar Q = QR(G) with G ~ N(0,1)^{n x n}, columns sign-fixed by diag(R);
* A = Q diag(lam) Q^T, then A = (A + A^T)/2;
* draw order: G first, then the signs.

All arrays are float64 in Fortran (column-major) order.
"""
from __future__ import annotations

import numpy as np


def haar_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    g = rng.standard_normal((n, n))
    q, r = np.linalg.qr(g)
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return np.asfortranarray(q * d)


def from_spectrum(lam: np.ndarray, q: np.ndarray) -> np.ndarray:
    a = (q * lam) @ q.T
    return np.asfortranarray((a + a.T) / 2.0)


def geometric_spectrum(n: int, lo: float, hi: float = 1.0) -> np.ndarray:
    if n == 1:
        return np.array([hi])
    return np.geomspace(lo, hi, n)


def random_signs(n: int, rng: np.random.Generator) -> np.ndarray:
    return rng.choice(np.array([-1.0, 1.0]), size=n)


def geo_matrix(n: int, kappa: float, seed: int = 0, signs: bool = True):
    """A with |lam| geometric in [1/kappa, 1] and random signs.  Returns (A, lam)."""
    rng = np.random.default_rng(seed)
    q = haar_orthogonal(n, rng)
    lam = geometric_spectrum(n, 1.0 / kappa)
    if signs:
        lam = lam * random_signs(n, rng)
    return from_spectrum(lam, q), lam


def ari_matrix(n: int, kappa: float, seed: int = 0, signs: bool = True):
    """A with |lam| arithmetic in [1/kappa, 1] (the paper's 'ari' mode) and random signs."""
    rng = np.random.default_rng(seed)
    q = haar_orthogonal(n, rng)
    lam = 1.0 - np.arange(n) / max(n - 1, 1) * (1.0 - 1.0 / kappa)
    if signs:
        lam = lam * random_signs(n, rng)
    return from_spectrum(lam, q), lam


def small_geo(seed: int = 0):
    """n = 96, |lam| geometric in [1e-3, 1], random signs (the small single-matrix case)."""
    return geo_matrix(96, 1e3, seed)


def clustered_1024(seed: int = 0, n: int = 1024):
    """n = 1024: 992 eigenvalues linear in [-1, 1] plus 32 within 1e-8 of 0.5."""
    rng = np.random.default_rng(seed)
    q = haar_orthogonal(n, rng)
    k = 32
    lam = np.concatenate([np.linspace(-1.0, 1.0, n - k), 0.5 + 1e-8 * np.linspace(-1.0, 1.0, k)])
    return from_spectrum(lam, q), lam


def geo_4096(seed: int = 0, n: int = 4096):
    """n = 4096: |lam| geometric in [1e-6, 1] (condition 1e6), random signs."""
    return geo_matrix(n, 1e6, seed)


def batch_sizes(count: int = 2048, lo: int = 8, hi: int = 256, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=count)


def batch_goe(count: int = 2048, lo: int = 8, hi: int = 256, seed: int = 0):
    """The batched workload: sizes uniform in [lo, hi], each A_i = (G + G^T)/2 with
    G ~ N(0, 1/n_i), drawn in batch order from the same generator."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(lo, hi + 1, size=count)
    mats = []
    for n in sizes:
        g = rng.standard_normal((int(n), int(n))) / np.sqrt(n)
        mats.append(np.asfortranarray((g + g.T) / 2.0))
    return sizes, mats


def gapped_spectrum(n: int, rng: np.random.Generator, gap: float = 1e-3) -> np.ndarray:
    """lam uniform in [-1, 1] with min gap >= `gap` by spacing:
    s = sort(U[0,1]^n), lam_i = -1 + (2 - (n-1) gap) s_i + i gap."""
    s = np.sort(rng.random(n))
    i = np.arange(n)
    return -1.0 + (2.0 - (n - 1) * gap) * s + i * gap


def backward_batch(count: int = 64, n: int = 512, seed: int = 0, grad_seed: int = 1):
    """The differentiation workload: `count` matrices with gapped spectra, Haar
    eigenvectors, plus upstream gradients dW, dQ ~ N(0,1) from `grad_seed`."""
    rng = np.random.default_rng(seed)
    mats, lams = [], []
    for _ in range(count):
        q = haar_orthogonal(n, rng)
        lam = gapped_spectrum(n, rng)
        mats.append(from_spectrum(lam, q))
        lams.append(lam)
    grng = np.random.default_rng(grad_seed)
    dW = [grng.standard_normal(n) for _ in range(count)]
    dQ = [np.asfortranarray(grng.standard_normal((n, n))) for _ in range(count)]
    return mats, lams, dW, dQ


def randn_sym(n: int, seed: int = 0) -> np.ndarray:
    """A = R + R^T with R ~ N(0,1) (the paper's Jacobi test matrix, Sec. 2.4/2.5)."""
    rng = np.random.default_rng(seed)
    r = rng.standard_normal((n, n))
    return np.asfortranarray(r + r.T)


def near_diagonal(n: int, lam: np.ndarray, eps: float, seed: int = 0) -> np.ndarray:
    """A = Q diag(lam) Q^T with Q the Cayley transform (I - eps S)^-1 (I + eps S)
    of a random skew-symmetric S (entries N(0, 1/n)): an orthogonal Q within
    about 2 eps of the identity, so A is nearly diagonal, like the matrix the
    FP64 sweeps receive after preconditioning."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, n)) / np.sqrt(n)
    s = eps * (g - g.T) / 2.0
    eye = np.eye(n)
    q = np.linalg.solve(eye - s, eye + s)
    return from_spectrum(lam, q)
