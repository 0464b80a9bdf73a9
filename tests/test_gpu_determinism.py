"""Deterministic mode (nuht_opts.deterministic = 1): the same inputs give the
same bits on every run, in both directions, and the results still meet the
accuracy contract against the oracle.

The default mode adds the blocks' contributions with FP64 atomics, whose
order (and so the last bits) varies between runs; the deterministic mode adds
them as exact fixed-point integers, so repeated calls, and separately built
plans of the same inputs, must agree bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2411_09583_gb300.workloads import loguniform_problem, sample_rows, uniform_problem

pytestmark = pytest.mark.gpu

from gpu_helpers import to_dev, tol  # noqa: E402


def _bits(x):
    return np.ascontiguousarray(x).view(np.uint64)


@pytest.mark.parametrize("nu,eps,precision", [(0, 1e-10, "fp64"), (3, 1e-12, "fp64"), (1, 1e-6, "mixed")])
def test_repeated_calls_are_bitwise_equal(nu, eps, precision):
    from paper_2411_09583_gb300 import Plan
    r, omega, c = uniform_problem(20000, 18000, omega_max=2e4, seed=700 + nu)
    e = np.random.default_rng(701).standard_normal(omega.size)
    with Plan(nu, to_dev(r), to_dev(omega), eps, precision=precision, deterministic=True) as p:
        info = p.info()
        assert info["n_local"] > 0 and info["n_asy"] > 0 and info["n_direct"] > 0
        g1 = p.execute(to_dev(c)).cpu().numpy()
        a1 = p.adjoint(to_dev(e)).cpu().numpy()
        g2 = p.execute(to_dev(c)).cpu().numpy()
        a2 = p.adjoint(to_dev(e)).cpu().numpy()
    # a second plan of the same inputs
    with Plan(nu, to_dev(r), to_dev(omega), eps, precision=precision, deterministic=True) as p:
        g3 = p.execute(to_dev(c)).cpu().numpy()
        a3 = p.adjoint(to_dev(e)).cpu().numpy()
    assert np.array_equal(_bits(g1), _bits(g2)) and np.array_equal(_bits(g1), _bits(g3))
    assert np.array_equal(_bits(a1), _bits(a2)) and np.array_equal(_bits(a1), _bits(a3))
    rows = sample_rows(omega.size, 300, seed=702)
    cols = sample_rows(r.size, 300, seed=703)
    assert np.max(np.abs(g1[rows] - oracle.direct_rows(nu, r, omega, c, rows))) <= tol(eps, c)
    assert np.max(np.abs(a1[cols] - oracle.direct_rows(nu, omega, r, e, cols))) <= tol(eps, e)
    # and the default (FP64 atomics) mode agrees with it within the contract
    with Plan(nu, to_dev(r), to_dev(omega), eps, precision=precision) as p:
        g0 = p.execute(to_dev(c)).cpu().numpy()
    assert np.max(np.abs(g0 - g1)) <= tol(eps, c)


def test_component_pairs_and_complex_vectors():
    # complex c (a component pair) and three real vectors (a pair and a single
    # one), both directions; pairs share the local and direct blocks' Bessel
    # values and accumulate into the second component's own sums
    from paper_2411_09583_gb300 import Plan
    r, omega, c = loguniform_problem(6000, 5000, omega_max=4e3, seed=710, complex_c=True)
    rng = np.random.default_rng(711)
    c3 = rng.standard_normal((r.size, 3))
    e3 = rng.standard_normal((omega.size, 3))
    eps = 1e-9
    with Plan(1, to_dev(r), to_dev(omega), eps, deterministic=True) as p:
        outs = [(p.execute(to_dev(c)).cpu().numpy(), p.execute(to_dev(c3)).cpu().numpy(),
                 p.adjoint(to_dev(e3)).cpu().numpy()) for _ in range(2)]
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(_bits(a.view(np.float64)), _bits(b.view(np.float64)))
    g, g3, a3 = outs[0]
    rows = sample_rows(omega.size, 100, seed=712)
    assert np.max(np.abs(g[rows] - oracle.direct_rows(1, r, omega, c, rows))) <= tol(eps, c)
    for v in range(3):
        cv, ev = np.ascontiguousarray(c3[:, v]), np.ascontiguousarray(e3[:, v])
        assert np.max(np.abs(g3[rows, v] - oracle.direct_rows(1, r, omega, cv, rows))) <= tol(eps, cv)
        cols = sample_rows(r.size, 100, seed=713 + v)
        assert np.max(np.abs(a3[cols, v] - oracle.direct_rows(1, omega, r, ev, cols))) <= tol(eps, ev)


def test_batched_plan():
    from paper_2411_09583_gb300 import Plan
    from paper_2411_09583_gb300.workloads import batch_problems
    probs = batch_problems(count=12, lo=300, hi=8000, nu_max=20, seed=720)
    nus = [p[0] for p in probs]
    n = [p[1].size for p in probs]
    m = [p[2].size for p in probs]
    r = np.concatenate([p[1] for p in probs])
    omega = np.concatenate([p[2] for p in probs])
    c = np.concatenate([p[3] for p in probs])
    eps = 1e-8
    with Plan.many(nus, to_dev(r), n, to_dev(omega), m, eps, deterministic=True) as bp:
        g1 = bp.execute(to_dev(c)).cpu().numpy()
        g2 = bp.execute(to_dev(c)).cpu().numpy()
    assert np.array_equal(_bits(g1), _bits(g2))
    off = 0
    for nu, rr, ww, cc in probs:
        assert np.max(np.abs(g1[off:off + ww.size] - oracle.direct(nu, rr, ww, cc))) <= tol(eps, cc)
        off += ww.size


def test_full_size_sampled_and_repeatable():
    # n = m = 1e6, r ~ U[0,1], omega ~ U[0,1e5], eps = 1e-12 (the benchmark's workload)
    from paper_2411_09583_gb300 import Plan
    eps = 1e-12
    r, omega, c = uniform_problem(1_000_000, 1_000_000, omega_max=1e5, seed=2)
    with Plan(0, to_dev(r), to_dev(omega), eps, deterministic=True) as p:
        g1 = p.execute(to_dev(c)).cpu().numpy()
        g2 = p.execute(to_dev(c)).cpu().numpy()
    assert np.array_equal(_bits(g1), _bits(g2))
    rows = sample_rows(omega.size, 200, seed=99)
    assert np.max(np.abs(g1[rows] - oracle.direct_rows(0, r, omega, c, rows))) <= tol(eps, c)


@pytest.mark.parametrize("det", [False, True])
def test_zero_and_extreme_magnitudes(det):
    # all-zero inputs give exact zeros; inputs far outside the FP32 exponent
    # range of the double-float kernels keep the accuracy contract, in both
    # directions: every call scales its input by a power of two from its
    # largest magnitude (and, deterministically, its fixed-point sums)
    from paper_2411_09583_gb300 import Plan
    r, omega, c = uniform_problem(3000, 2500, omega_max=3000.0, seed=730)
    e = np.random.default_rng(731).standard_normal(omega.size)
    eps = 1e-10
    ref_g, ref_a = oracle.direct(2, r, omega, c), oracle.direct(2, omega, r, e)
    with Plan(2, to_dev(r), to_dev(omega), eps, deterministic=det) as p:
        z = p.execute(to_dev(np.zeros_like(c))).cpu().numpy()
        assert np.array_equal(z, np.zeros_like(z))
        za = p.adjoint(to_dev(np.zeros_like(e))).cpu().numpy()
        assert np.array_equal(za, np.zeros_like(za))
        for scale in (2.0 ** -1000, 1e-300, 1e-45, 1e40, 1e250):
            g = p.execute(to_dev(c * scale)).cpu().numpy() / scale
            assert np.max(np.abs(g - ref_g)) <= tol(eps, c), scale
            a = p.adjoint(to_dev(e * scale)).cpu().numpy() / scale
            assert np.max(np.abs(a - ref_a)) <= tol(eps, e), scale
