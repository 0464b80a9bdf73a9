"""Pins for the oracle's direct sum g_k = sum_j c_j J_nu(omega_k r_j)."""
import math

import mpmath as mp
import numpy as np
import pytest

import oracle


def _gauss_legendre(a, b, n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


@pytest.mark.parametrize("nu", [0, 1, 4])
def test_gaussian_hankel_pair(nu):
    # int_0^inf exp(-r^2/2) J_nu(w r) r^(nu+1) dr = w^nu exp(-w^2/2)
    r, wq = _gauss_legendre(0.0, 12.0, 240)
    c = wq * r ** (nu + 1) * np.exp(-0.5 * r * r)
    omega = np.linspace(0.0, 6.0, 61)
    g = oracle.direct(nu, r, omega, c)
    ref = omega ** nu * np.exp(-0.5 * omega ** 2)
    assert np.max(np.abs(g - ref)) < 1e-13


@pytest.mark.parametrize("nu", [0, 2, 5])
def test_unit_disk_transform(nu):
    # int_0^1 J_nu(w r) r^(nu+1) dr = J_{nu+1}(w) / w  (Sec. 5.2 for nu = 0)
    r, wq = _gauss_legendre(0.0, 1.0, 400)
    c = wq * r ** (nu + 1)
    omega = np.array([0.5, 3.0, 17.0, 64.0, 150.0, 200.0])
    g = oracle.direct(nu, r, omega, c)
    ref = np.array([float(mp.besselj(nu + 1, mp.mpf(w)) / w) for w in omega])
    assert np.max(np.abs(g - ref)) < 1e-14


def test_all_points_at_origin():
    c = np.random.default_rng(0).standard_normal(50)
    omega = np.linspace(0, 100, 9)
    r = np.zeros(50)
    assert np.allclose(oracle.direct(0, r, omega, c), c.sum(), rtol=0, atol=1e-13)
    assert np.all(oracle.direct(3, r, omega, c) == 0.0)


def test_brute_force_mpmath_tiny():
    rng = np.random.default_rng(3)
    for nu in [0, 1, 6]:
        r = rng.uniform(0, 1, 5)
        omega = np.concatenate([rng.uniform(0, 50, 3), [0.0, 2000.0]])
        c = rng.standard_normal(5)
        g = oracle.direct(nu, r, omega, c)
        for k, w in enumerate(omega):
            ref = mp.fsum(mp.mpf(c[j]) * mp.besselj(nu, mp.mpf(w) * mp.mpf(r[j]))
                          for j in range(5))
            # each term carries at most ~5e-16 evaluator error
            assert abs(g[k] - float(ref)) < 5e-16 * np.abs(c).sum() + 1e-16


def test_linearity_permutation_rows_complex():
    rng = np.random.default_rng(4)
    n, m = 300, 200
    r = rng.uniform(0, 1, n)
    omega = rng.uniform(0, 500, m)
    a, b = rng.standard_normal(n), rng.standard_normal(n)
    ga, gb = oracle.direct(2, r, omega, a), oracle.direct(2, r, omega, b)
    gab = oracle.direct(2, r, omega, 2.0 * a - 3.0 * b)
    assert np.max(np.abs(gab - (2 * ga - 3 * gb))) < 1e-12
    p = rng.permutation(n)
    assert np.max(np.abs(oracle.direct(2, r[p], omega, a[p]) - ga)) < 1e-12
    rows = np.array([5, 0, 199, 77])
    assert np.array_equal(oracle.direct_rows(2, r, omega, a, rows), ga[rows])
    gc = oracle.direct(2, r, omega, a + 1j * b)
    assert np.array_equal(gc.real, ga) and np.array_equal(gc.imag, gb)
    gm = oracle.direct(2, r, omega, np.stack([a, b], axis=1))
    assert np.array_equal(gm[:, 0], ga) and np.array_equal(gm[:, 1], gb)


def test_empty_inputs():
    assert oracle.direct(0, np.zeros(0), np.ones(4), np.zeros(0)).shape == (4,)
    assert np.all(oracle.direct(0, np.zeros(0), np.ones(4), np.zeros(0)) == 0)
    assert oracle.direct(0, np.ones(3), np.zeros(0), np.ones(3)).shape == (0,)
