"""GPU parity at the exact configurations the benchmark times, and at the
tightest tolerance the library accepts.

Bar: per problem and vector, max_k |g_k - g_k^oracle| <= 10 eps ||c||_1 (the
accuracy contract), on sampled output rows (columns for the adjoint) that the
oracle's direct sum computes one by one.
"""
import numpy as np
import pytest

import oracle
from paper_2411_09583_gb300.workloads import batch_problems, large_grid_problem, sample_rows, uniform_problem

pytestmark = pytest.mark.gpu

from gpu_helpers import to_dev, tol  # noqa: E402


def _sample(size, count, rng):
    return np.sort(rng.choice(size, size=min(count, size), replace=False))


def test_uneven_batch_of_256_forward_and_adjoint():
    # The batched benchmark's workload exactly: 256 problems, n and m
    # log-uniform in [1e3, 1e5], nu uniform in 0..20, omega ~ U[0, m], seed 5,
    # eps = 1e-8, one plan.  Forward and adjoint, 50 sampled rows (columns) of
    # every problem against the oracle.
    from paper_2411_09583_gb300 import Plan
    eps = 1e-8
    probs = batch_problems(count=256, lo=1e3, hi=1e5, nu_max=20, seed=5)
    nus = [p[0] for p in probs]
    n = [p[1].size for p in probs]
    m = [p[2].size for p in probs]
    r = np.concatenate([p[1] for p in probs])
    omega = np.concatenate([p[2] for p in probs])
    c = np.concatenate([p[3] for p in probs])
    e = np.random.default_rng(55).standard_normal(omega.size)
    with Plan.many(nus, to_dev(r), n, to_dev(omega), m, eps) as bp:
        g = bp.execute(to_dev(c)).cpu().numpy()
        ca = bp.adjoint(to_dev(e)).cpu().numpy()
    ro = np.concatenate([[0], np.cumsum(n)])
    wo = np.concatenate([[0], np.cumsum(m)])
    rng = np.random.default_rng(56)
    worst_f = worst_a = 0.0
    for i, (nu, rr, ww, cc) in enumerate(probs):
        rows = _sample(ww.size, 50, rng)
        err = np.max(np.abs(g[wo[i]:wo[i + 1]][rows] - oracle.direct_rows(nu, rr, ww, cc, rows)))
        worst_f = max(worst_f, err / tol(eps, cc))
        ei = e[wo[i]:wo[i + 1]]
        cols = _sample(rr.size, 50, rng)
        err = np.max(np.abs(ca[ro[i]:ro[i + 1]][cols] - oracle.direct_rows(nu, ww, rr, ei, cols)))
        worst_a = max(worst_a, err / tol(eps, ei))
    assert worst_f <= 1.0, worst_f
    assert worst_a <= 1.0, worst_a


@pytest.mark.parametrize("nu", [0, 1, 10])
def test_tightest_tolerance_both_directions(nu):
    # eps = 1e-15, the smallest the library accepts: the whole path (the
    # double-float loops included) must still meet 10 eps ||c||_1
    from paper_2411_09583_gb300 import Plan
    eps = 1e-15
    r, omega, c = uniform_problem(2000, 1800, omega_max=3000.0, seed=600 + nu)
    e = np.random.default_rng(601 + nu).standard_normal(omega.size)
    with Plan(nu, to_dev(r), to_dev(omega), eps) as p:
        info = p.info()
        assert info["n_local"] > 0 and info["n_asy"] > 0 and info["n_direct"] > 0
        g = p.execute(to_dev(c)).cpu().numpy()
        ca = p.adjoint(to_dev(e)).cpu().numpy()
    err = np.max(np.abs(g - oracle.direct(nu, r, omega, c)))
    assert err <= tol(eps, c), (err, tol(eps, c))
    err = np.max(np.abs(ca - oracle.direct(nu, omega, r, e)))
    assert err <= tol(eps, e), (err, tol(eps, e))


@pytest.mark.parametrize("precision,eps", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_large_grid_single_block(precision, eps):
    # one asymptotic block whose spreading grid (~3.2e6 cells x 2M terms) and
    # FFT (2^23 points x 2M terms) are far larger than the L2 cache: n = m =
    # 4e6, r ~ U[1,2], omega ~ U[1e7,2e7]; sampled rows and columns against
    # the oracle, both directions
    from paper_2411_09583_gb300 import Plan
    r, omega, c = large_grid_problem()
    e = np.random.default_rng(12).standard_normal(omega.size)
    with Plan(0, to_dev(r), to_dev(omega), eps, precision=precision) as p:
        info = p.info()
        assert info["n_asy"] == 1 and info["n_local"] == 0 and info["n_direct"] == 0
        assert info["fft_points"] >= 1 << 23
        g = p.execute(to_dev(c)).cpu().numpy()
        ca = p.adjoint(to_dev(e)).cpu().numpy()
    rows = sample_rows(omega.size, 60, seed=13)
    cols = sample_rows(r.size, 60, seed=14)
    assert np.max(np.abs(g[rows] - oracle.direct_rows(0, r, omega, c, rows))) <= tol(eps, c)
    assert np.max(np.abs(ca[cols] - oracle.direct_rows(0, omega, r, e, cols))) <= tol(eps, e)


def test_sixteen_vectors_both_directions():
    # nvec = 16 real vectors in one call (pairs of components share the local
    # and direct blocks' Bessel values), forward and adjoint, each vector
    # against the oracle on sampled rows
    from paper_2411_09583_gb300 import Plan
    eps = 1e-10
    r, omega, _ = uniform_problem(6000, 5000, omega_max=8000.0, seed=640)
    rng = np.random.default_rng(641)
    C, E = rng.standard_normal((r.size, 16)), rng.standard_normal((omega.size, 16))
    with Plan(2, to_dev(r), to_dev(omega), eps) as p:
        G = p.execute(to_dev(C)).cpu().numpy()
        A = p.adjoint(to_dev(E)).cpu().numpy()
    rows, cols = sample_rows(omega.size, 80, seed=642), sample_rows(r.size, 80, seed=643)
    ref_g = oracle.direct_rows(2, r, omega, C, rows)
    ref_a = oracle.direct_rows(2, omega, r, E, cols)
    assert np.all(np.max(np.abs(G[rows] - ref_g), axis=0) <= tol(eps, C))
    assert np.all(np.max(np.abs(A[cols] - ref_a), axis=0) <= tol(eps, E))
