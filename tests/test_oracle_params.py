"""Pins for the oracle's error bounds and parameter choice (Sec. 3)."""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import expansions as E
from oracle import params as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig1_expansion_orders.txt")


def _golden_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                nu, eps, M, L = line.split()
                rows.append((int(nu), float(eps), int(M), int(L)))
    return rows


@pytest.mark.parametrize("nu,eps,M,L", _golden_rows())
def test_fig1_worked_example(nu, eps, M, L):
    Mo, z, Lo = P.choose_params(nu, eps)
    assert (Mo, Lo) == (M, L)


def test_m_heuristic_by_hand():
    # Sec. 3.3, eq. num-asy-terms, evaluated by hand
    assert P.choose_m(0, 1e-8) == 3      # floor(1 + 0 + 2)
    assert P.choose_m(10, 1e-12) == 6    # floor(1 + 2 + 3)
    assert P.choose_m(1, 1e-5) == 2      # floor(1 + 0.2 + 1.25)
    assert P.choose_m(100, 1e-15) == 20  # capped


def test_hankel_coefficients_closed_forms():
    for nu in [0.0, 1.0, 3.0, 10.0]:
        mu = 4 * nu * nu
        assert P.hankel_a(0, nu) == 1.0
        assert math.isclose(P.hankel_a(1, nu), (mu - 1) / 8, rel_tol=1e-15)
        assert math.isclose(P.hankel_a(2, nu), (mu - 1) * (mu - 9) / 128, rel_tol=1e-15)
        assert math.isclose(P.hankel_a(3, nu), (mu - 1) * (mu - 9) * (mu - 25) / 3072,
                            rel_tol=1e-15)
    assert all(P.hankel_a(k, 0.5) == 0.0 for k in range(1, 8))


CASES = [(0, 1e-12), (1, 1e-8), (2, 1e-10), (3, 1e-12), (10, 1e-12), (20, 1e-8),
         (19, 1e-8), (7, 1e-5), (0, 1e-8), (1, 1e-10), (1, 1e-5)]


@pytest.mark.parametrize("nu,eps", CASES)
def test_crossover_root_and_local_order_minimal(nu, eps):
    M, z, L = P.choose_params(nu, eps)
    assert abs(P.b_asy(nu, M, z) / eps - 1) < 1e-10
    assert P.b_loc(nu, L, z) < eps
    if L > 0:
        assert P.b_loc(nu, L - 1, z) >= eps


@pytest.mark.parametrize("nu,eps", CASES)
def test_hankel_truncation_within_bound(nu, eps):
    # Sec. 3.2, eq. asy-error: |J - Hankel_M| <= B^asy(x) <= eps for x >= z, and the bound is tight
    M, z, L = P.choose_params(nu, eps)
    xs = np.concatenate([np.linspace(z, 1.05 * z, 120), np.linspace(z, 30 * z, 600)])
    errs = np.array([abs(E.hankel_sum(nu, M, x) - oracle.jn(nu, x)) for x in xs])
    bnd = np.array([P.b_asy(nu, M, x) for x in xs])
    assert np.all(errs <= bnd * (1 + 1e-6) + 5e-16)   # + FP64 evaluation noise
    assert errs[:120].max() > 0.3 * eps


@pytest.mark.parametrize("nu,eps", CASES)
def test_wimp_truncation_within_bound(nu, eps):
    # Lemma 3.1 on the rectangle [0, Omega] x [0, R] with Omega R = z (R = 1 and R = 0.37)
    M, z, L = P.choose_params(nu, eps)
    bound = P.b_loc(nu, L, z)
    for R in [1.0, 0.37]:
        Om = z / R
        for w in np.linspace(0, Om, 13):
            for r in np.linspace(0, R, 13):
                approx = E.wimp_sum(nu, L, w * R, r / R)
                assert abs(approx - oracle.jn(nu, w * r)) <= bound + 1e-15


@pytest.mark.parametrize("nu", [0, 1, 2, 3, 4, 9, 10])
def test_wimp_series_converges_to_bessel(nu):
    # reading of the Wimp coefficient (argument x/2) and of the odd-order form
    for x, y in [(3.0, 0.4), (20.0, 1.0), (31.5, 0.77), (45.0, 0.1)]:
        assert abs(E.wimp_sum(nu, 80, x, y) - oracle.jn(nu, x * y)) < 2e-15


def test_wimp_literal_printed_argument_would_fail():
    # the printed C_l(x) (argument x rather than x/2) is not an expansion of J_0(xy)
    x, y = 10.0, 0.6
    literal = sum((1 if l == 0 else 2) * oracle.jn(l, x) * oracle.jn(-l, x)
                  * math.cos(2 * l * math.acos(y)) for l in range(60))
    assert abs(literal - oracle.jn(0, x * y)) > 1e-2


def test_bounds_monotone():
    zs = [P.choose_params(0, e)[1] for e in [1e-4, 1e-6, 1e-8, 1e-10, 1e-12, 1e-14]]
    Ls = [P.choose_params(0, e)[2] for e in [1e-4, 1e-6, 1e-8, 1e-10, 1e-12, 1e-14]]
    assert Ls == sorted(Ls)
    assert P.b_loc(0, 10, 5.0) < P.b_loc(0, 10, 6.0)
    assert P.b_asy(0, 3, 20.0) > P.b_asy(0, 3, 21.0)
    assert math.isinf(P.b_loc(0, 3, 100.0))
    assert zs  # defined for every eps
