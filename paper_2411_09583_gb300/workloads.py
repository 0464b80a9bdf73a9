"""Seeded synthetic inputs for the NUHT (shared by tests, smoke and bench).

Holds no arithmetic of the transform itself: only the random draws that
stand in for the paper's synthetic experiments (Sec. 5.1: uniform,
clustered, exponential and Fourier-Bessel point sets, sparse coefficients).  Draw order is r, omega, c (for a
complex c: real part, then imaginary part), from numpy's PCG64.
"""
import numpy as np


def uniform_problem(n, m, r_max=1.0, omega_max=None, seed=0, nvec=1,
                    complex_c=False):
    """r ~ U[0, r_max], omega ~ U[0, omega_max], c ~ N(0, 1); unsorted."""
    if omega_max is None:
        omega_max = float(m)
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.0, r_max, n)
    omega = rng.uniform(0.0, omega_max, m)
    shape = (n,) if nvec == 1 else (n, nvec)
    c = rng.standard_normal(shape)
    if complex_c:
        c = c + 1j * rng.standard_normal(shape)
    return r, omega, c


def loguniform_problem(n, m, r_lo=1e-3, r_hi=1.0, omega_max=4e4, seed=0,
                       complex_c=True):
    """r = 10^U[log10 r_lo, log10 r_hi] (clustered near 0), omega ~ U[0, omega_max]."""
    rng = np.random.default_rng(seed)
    r = 10.0 ** rng.uniform(np.log10(r_lo), np.log10(r_hi), n)
    omega = rng.uniform(0.0, omega_max, m)
    c = rng.standard_normal(n)
    if complex_c:
        c = c + 1j * rng.standard_normal(n)
    return r, omega, c


def large_grid_problem(n=4_000_000, m=4_000_000, seed=11):
    """One asymptotic block whose type-3 grids are larger than the L2 cache:
    r ~ U[1, 2], omega ~ U[1e7, 2e7] (every omega r far above z), c ~ N(0, 1).
    The half-widths X = 0.5 and S = 5e6 give about 2 X S / pi = 1.6e6 cells on
    each side of the spreading grid and an FFT of 2^23 points per Hankel term."""
    rng = np.random.default_rng(seed)
    r = rng.uniform(1.0, 2.0, n)
    omega = rng.uniform(1e7, 2e7, m)
    c = rng.standard_normal(n)
    return r, omega, c


def exponential_grid(n):
    """omega_j = r_j = 10^(log10 j - log10(n)/2), j = 1..n (Sec. 5.1.1, the
    worst case for the subdivision)."""
    j = np.arange(1, n + 1, dtype=np.float64)
    v = 10.0 ** (np.log10(j) - 0.5 * np.log10(n))
    return v.copy(), v.copy()


def fourier_bessel_grid(nu, n):
    """The Fourier-Bessel case of Sec. 5.1.1 (n = m): omega_k = j_{nu,k},
    r_j = j_{nu,j} / j_{nu,n+1} for j, k = 1..n, where j_{nu,k} is the k-th
    positive root of J_nu (from scipy.special.jn_zeros, a library routine).
    A fixed grid (no random draws), in ascending order."""
    from scipy.special import jn_zeros
    roots = jn_zeros(int(abs(nu)), n + 1)
    return roots[:n] / roots[n], roots[:n].copy()


def sparse_coefficients(n, nnz=1000, seed=0):
    """Sec. 5.1.3's input: nnz entries at random distinct indices with
    standard Gaussian values, zero elsewhere.  Returns (c, indices)."""
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(n, size=min(nnz, n), replace=False))
    c = np.zeros(n)
    c[idx] = rng.standard_normal(idx.size)
    return c, idx


def batch_problems(count=256, lo=1e3, hi=1e5, nu_max=20, seed=5):
    """Uneven batch: n, m = floor(10^U[log10 lo, log10 hi]) independently,
    nu ~ U{0..nu_max}, r ~ U[0, 1], omega ~ U[0, m], c ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    probs = []
    for _ in range(count):
        n = int(10.0 ** rng.uniform(np.log10(lo), np.log10(hi)))
        m = int(10.0 ** rng.uniform(np.log10(lo), np.log10(hi)))
        nu = int(rng.integers(0, nu_max + 1))
        r = rng.uniform(0.0, 1.0, n)
        omega = rng.uniform(0.0, float(m), m)
        c = rng.standard_normal(n)
        probs.append((nu, r, omega, c))
    return probs


def sample_rows(m, count=1000, seed=12345):
    """Seeded random output indices for sampled parity checks."""
    rng = np.random.default_rng(seed)
    count = min(count, m)
    return np.sort(rng.choice(m, size=count, replace=False))
