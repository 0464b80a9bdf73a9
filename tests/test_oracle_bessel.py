"""Pins for the oracle's Bessel evaluator (each path against facts that do
not come from the oracle itself: closed forms, mpmath, identities)."""
import math

import mpmath as mp
import numpy as np
import pytest

import oracle

mp.mp.dps = 40


def _mp_j(n, x):
    return float(mp.besselj(n, mp.mpf(x)))


@pytest.mark.parametrize("x", [1e-3, 0.1, 0.7, 1.3, 2.0, 3.1, 4.0])
def test_series_half_integer_closed_form(x):
    # J_{1/2}(x) = sqrt(2/(pi x)) sin x ; J_{3/2}(x) = sqrt(2/(pi x)) (sin x / x - cos x)
    j12 = math.sqrt(2 / (math.pi * x)) * math.sin(x)
    j32 = math.sqrt(2 / (math.pi * x)) * (math.sin(x) / x - math.cos(x))
    assert abs(oracle.jv_series(0.5, x) - j12) <= 2e-16 * max(1, abs(j12)) + 1e-17
    assert abs(oracle.jv_series(1.5, x) - j32) <= 1e-15 * max(1, abs(j32)) + 1e-17


@pytest.mark.parametrize("x", [1.0, 3.7, 25.0, 1234.5, 98765.4321])
def test_hankel_half_integer_is_exact(x):
    # for nu = 1/2 all a_k(nu), k >= 1, vanish; for nu = 3/2 the series stops after a_1
    v, ok = oracle.jv_hankel(0.5, x)
    assert ok
    ref = math.sqrt(2 / (math.pi * x)) * math.sin(x)
    assert abs(v - ref) <= 4e-16
    v, ok = oracle.jv_hankel(1.5, x)
    assert ok
    ref = math.sqrt(2 / (math.pi * x)) * (math.sin(x) / x - math.cos(x))
    assert abs(v - ref) <= 4e-16


@pytest.mark.parametrize("nu", [0.0, 1.0, 2.5, 7.0])
def test_series_three_term_recurrence(nu):
    for x in [0.3, 1.1, 1.9]:
        lhs = oracle.jv_series(nu, x) + oracle.jv_series(nu + 2, x)
        rhs = 2 * (nu + 1) / x * oracle.jv_series(nu + 1, x)
        assert abs(lhs - rhs) <= 1e-15


@pytest.mark.parametrize("nu", [1, 2, 5, 10])
def test_hankel_three_term_recurrence(nu):
    for x in [400.0, 1e3 + 0.37, 5e4 + 0.123]:
        a, ok1 = oracle.jv_hankel(nu - 1, x)
        b, ok2 = oracle.jv_hankel(nu + 1, x)
        c, ok3 = oracle.jv_hankel(nu, x)
        assert ok1 and ok2 and ok3
        assert abs(a + b - 2 * nu / x * c) <= 1e-16


def test_miller_known_zeros_and_values():
    # first zeros of J_0 and J_1 (A&S Table 9.5)
    assert abs(oracle.jn_miller(0, 2.404825557695773)) < 1e-15
    assert abs(oracle.jn_miller(1, 3.8317059702075123)) < 1e-15
    for n, x in [(0, 3.0), (0, 17.3), (1, 9.9), (4, 30.0), (12, 5.5), (20, 150.0), (3, 0.9)]:
        assert abs(oracle.jn_miller(n, x) - _mp_j(n, x)) <= 4e-16


def test_dispatcher_against_mpmath():
    rng = np.random.default_rng(11)
    for n in [0, 1, 2, 5, 10, 11, 20, 21]:
        xs = np.concatenate([rng.uniform(0, 3, 20), rng.uniform(3, 60, 40),
                             rng.uniform(60, 400, 20), 10 ** rng.uniform(2.6, 5.3, 20)])
        for x in xs:
            ref = _mp_j(n, x)
            assert abs(oracle.jn(n, x) - ref) <= 5e-16, (n, x)


def test_dispatcher_against_scipy():
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.uniform(0, 50, 20000), 10 ** rng.uniform(1.5, 5, 20000)])
    for n in [0, 1, 3, 8]:
        assert np.max(np.abs(oracle.jn(n, x) - sp.jv(n, x))) < 2e-14


def test_negative_order_symmetry():
    for n in [1, 2, 3, 7]:
        for x in [0.5, 9.0, 300.0]:
            assert oracle.jn(-n, x) == (-1) ** n * oracle.jn(n, x)


def test_neumann_addition_theorem_across_branches():
    # J_n(a+b) = sum_k J_k(a) J_{n-k}(b)  (DLMF 10.23.2 with integer orders)
    for (a, b, n) in [(1.0, 1.5, 0), (4.0, 30.0, 1), (60.0, 45.0, 3), (0.5, 300.0, 2)]:
        kmax = int(a + b) + 60
        s = math.fsum(oracle.jn(k, a) * oracle.jn(n - k, b) for k in range(-kmax, kmax + 1))
        assert abs(s - oracle.jn(n, a + b)) < 2e-14


def test_exact_product_argument():
    # J_n at the exact product of two doubles (the oracle refines the argument)
    for n, a, b in [(0, 98765.4321, 0.987654321), (3, 12345.678, 0.777)]:
        x = mp.mpf(a) * mp.mpf(b)
        ref = float(mp.besselj(n, x))
        assert abs(oracle.jn_prod(n, a, b) - ref) <= 4e-16


def test_zero_argument():
    assert oracle.jn(0, 0.0) == 1.0
    assert oracle.jn(3, 0.0) == 0.0
