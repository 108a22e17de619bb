"""Seeded synthetic inputs for the mixed-precision Jacobi SVD workloads.

This module only draws random test matrices; it contains none of the SVD method's
arithmetic, and both the GPU path and the CPU oracle take its outputs as inputs.
Every matrix is float64, column-major (numpy Fortran order), so the same bytes can be
handed to the C oracle and copied to the GPU.

Recipes (test matrices of Section 7.1, Tables 1-2, and the five named workloads):
  * ``known_sigma``: A = U diag(sigma) V^T, U and V from the QR of Gaussian matrices.
  * ``graded``: A = B D with B = W1 diag(sigma_B) W2^T and D diagonal (column grading).
  * ``xlatm1``: the five distribution modes of Table 2 for a diagonal with condition kappa.
"""
import numpy as np


def orthonormal(rng, m, n):
    """m x n with orthonormal columns: Q of the QR of an m x n standard Gaussian, with the
    column signs fixed by sign(diag R) so the distribution is Haar."""
    G = rng.standard_normal((m, n))
    Q, R = np.linalg.qr(G)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return np.asfortranarray(Q * d)


def known_sigma(rng, m, n, sigma):
    """A = U diag(sigma) V^T (m x n) with Haar U (m x n) and V (n x n)."""
    sigma = np.asarray(sigma, dtype=np.float64)
    U = orthonormal(rng, m, n)
    V = orthonormal(rng, n, n)
    return np.asfortranarray((U * sigma) @ V.T)


def xlatm1(rng, mode, n, kappa):
    """Diagonal entries d(1..n) of Table 2 (modes 1-5) with condition number kappa."""
    i = np.arange(n, dtype=np.float64)
    if mode == 1:
        d = np.full(n, 1.0 / kappa)
        d[0] = 1.0
    elif mode == 2:
        d = np.ones(n)
        d[-1] = 1.0 / kappa
    elif mode == 3:
        d = kappa ** (-i / max(n - 1, 1))
    elif mode == 4:
        # 1 - t (1 - 1/kappa) with t = (i-1)/(n-1), evaluated as (1 - t) + t / kappa: the same
        # numbers without the cancellation that turns d(n) = 1/kappa into 0 for kappa > 1e16
        t = i / max(n - 1, 1)
        d = (1.0 - t) + t / kappa
    elif mode == 5:
        d = np.exp(rng.uniform(np.log(1.0 / kappa), 0.0, n))
    else:
        raise ValueError("mode must be 1..5")
    return d


def graded(rng, m, n, sigma_b, d):
    """A = B D with B = W1 diag(sigma_b) W2^T (W1 m x n, W2 n x n Haar) and D = diag(d)."""
    B = known_sigma(rng, m, n, sigma_b)
    return np.asfortranarray(B * np.asarray(d, dtype=np.float64)[None, :])


# ------------------------------------------------------------------------------------
# The five named workloads.
# ------------------------------------------------------------------------------------

def plain_256x128(seed=0, m=256, n=128):
    """Single 256 x 128 matrix, sigma log-spaced 1 .. 1e-6 (known singular values)."""
    rng = np.random.default_rng(seed)
    sigma = np.logspace(0.0, -6.0, n)
    return known_sigma(rng, m, n, sigma), sigma


def precision_2048x1024(seed=1, m=2048, n=1024):
    """Single A = B D, 2048 x 1024: B with singular values log-spaced 1 .. 1e-3,
    D = diag(10^U(-8, 0)) (log-random grading, Table 2 mode 5 with kappa = 1e8)."""
    rng = np.random.default_rng(seed)
    sigma_b = np.logspace(0.0, -3.0, n)
    B = known_sigma(rng, m, n, sigma_b)
    d = 10.0 ** rng.uniform(-8.0, 0.0, n)
    return np.asfortranarray(B * d[None, :])


def batch_sizes(seed=2, count=4096, nmin=16, nmax=256):
    """(m, n, kappa) per matrix: n ~ U{nmin..nmax}, m = n + U{0..n}, kappa = 10^U(1, 8)."""
    rng = np.random.default_rng(seed)
    n = rng.integers(nmin, nmax + 1, size=count)
    m = n + np.array([rng.integers(0, k + 1) for k in n])
    kappa = 10.0 ** rng.uniform(1.0, 8.0, count)
    return m.astype(np.int64), n.astype(np.int64), kappa


def batch_matrices(seed=2, count=4096, nmin=16, nmax=256):
    """The uneven batch: A_i = U diag(sigma_i) V^T, sigma_i log-spaced 1 .. 1/kappa_i.
    Returns (list of matrices, list of sigma, m, n, kappa)."""
    m, n, kappa = batch_sizes(seed, count, nmin, nmax)
    rng = np.random.default_rng(seed + 1000003)
    mats, sigmas = [], []
    for mi, ni, ki in zip(m, n, kappa):
        s = np.logspace(0.0, -np.log10(ki), int(ni))
        mats.append(known_sigma(rng, int(mi), int(ni), s))
        sigmas.append(s)
    return mats, sigmas, m, n, kappa


def differentiation(seed=3, batch=512, small=(64, 32), large=(1024, 512)):
    """Differentiation workload: ``batch`` matrices of shape ``small`` plus one of shape
    ``large``; sigma log-spaced 1 .. 1e-2 (adjacent ratio <= 1 - 1e-3 for n <= 4605);
    loss weights w ~ N(0,1)^n and cotangents G_U ~ N^{m x n}, G_V ~ N^{n x n}."""
    rng = np.random.default_rng(seed)
    out = []
    shapes = [small] * batch + [large]
    for (m, n) in shapes:
        s = np.logspace(0.0, -2.0, n)
        A = known_sigma(rng, m, n, s)
        w = rng.standard_normal(n)
        GU = np.asfortranarray(rng.standard_normal((m, n)))
        GV = np.asfortranarray(rng.standard_normal((n, n)))
        out.append((A, s, w, GU, GV))
    return out


def large_8192(seed=4, n=8192, m=None):
    """Single A = B D, n x n: B with singular values log-spaced 1 .. 1e-2,
    D = diag(10^U(-10, 0))."""
    m = n if m is None else m
    rng = np.random.default_rng(seed)
    sigma_b = np.logspace(0.0, -2.0, n)
    B = known_sigma(rng, m, n, sigma_b)
    d = 10.0 ** rng.uniform(-10.0, 0.0, n)
    return np.asfortranarray(B * d[None, :])


def table1_pair(rng, n, mode_d, mode_s, kappa_d, kappa_b, m=None):
    """One Table 1 test matrix A = B D (without the unit-column W3 step): D from mode_d
    with kappa_d, B = W1 diag(Sigma) W2^T with Sigma from mode_s and kappa_b."""
    m = n if m is None else m
    d = xlatm1(rng, mode_d, n, kappa_d)
    s = xlatm1(rng, mode_s, n, kappa_b)
    return graded(rng, m, n, s, d)


TABLE1 = [(1, 2), (1, 3), (1, 4), (1, 5), (2, 3), (2, 4), (2, 5), (3, 2), (3, 4), (3, 5),
          (4, 2), (4, 3), (4, 5), (5, 2), (5, 3), (5, 4)]
