"""GPU parity of vector groups (opts.vec_group): the local and direct blocks
of up to 16 real components applied together, with one Bessel evaluation
(moment basis, Miller sweep, direct entry) shared by all of them.

Bar: per vector, max_k |g_k - g_k^oracle| <= 10 eps ||c||_1 against the
oracle's direct sum, and the grouped result equal within that bar to the
same call with groups of one.
"""
import numpy as np
import pytest

import oracle
from paper_2411_09583_gb300.workloads import batch_problems, sample_rows, uniform_problem

pytestmark = pytest.mark.gpu

from gpu_helpers import to_dev, tol  # noqa: E402


@pytest.mark.parametrize("nu,nvec,group", [(0, 3, 0), (0, 5, 4), (1, 16, 16), (3, 7, 3), (2, 9, 8), (0, 2, 1),
                                            (100, 6, 6)])
def test_groups_forward_match_oracle(nu, nvec, group):
    # every row of a problem with all three block classes, each vector
    # against the oracle; groups of `group` with a ragged last group
    from paper_2411_09583_gb300 import Plan
    eps = 1e-10
    r, omega, _ = uniform_problem(2500, 2200, omega_max=3000.0, seed=700 + nu)
    C = np.random.default_rng(701 + nvec).standard_normal((r.size, nvec))
    with Plan(nu, to_dev(r), to_dev(omega), eps, vec_group=group) as p:
        info = p.info()
        assert info["n_local"] > 0 and (nu == 100 or (info["n_asy"] > 0 and info["n_direct"] > 0))
        G = p.execute(to_dev(C)).cpu().numpy()
    ref = oracle.direct(nu, r, omega, C)
    assert np.all(np.max(np.abs(G - ref), axis=0) <= tol(eps, C))


def test_group_equals_single_components():
    # groups of 16, of 2 and of 1 give the same sums within the contract
    from paper_2411_09583_gb300 import Plan
    eps = 1e-12
    r, omega, _ = uniform_problem(20000, 18000, omega_max=20000.0, seed=710)
    C = np.random.default_rng(711).standard_normal((r.size, 16))
    out = {}
    for group in (16, 0, 1):
        with Plan(0, to_dev(r), to_dev(omega), eps, vec_group=group) as p:
            out[group] = p.execute(to_dev(C)).cpu().numpy()
    bar = tol(eps, C)
    assert np.all(np.max(np.abs(out[16] - out[1]), axis=0) <= bar)
    assert np.all(np.max(np.abs(out[0] - out[1]), axis=0) <= bar)
    rows = sample_rows(omega.size, 60, seed=712)
    ref = oracle.direct_rows(0, r, omega, C, rows)
    assert np.all(np.max(np.abs(out[16][rows] - ref), axis=0) <= bar)


def test_group_complex_and_mixed_precision():
    # complex c: 2 nvec real components in groups of 6 (the parts of one
    # column may fall in different groups); mixed precision at eps = 1e-6
    from paper_2411_09583_gb300 import Plan
    r, omega, _ = uniform_problem(3000, 2800, omega_max=4000.0, seed=720)
    rng = np.random.default_rng(721)
    C = rng.standard_normal((r.size, 5)) + 1j * rng.standard_normal((r.size, 5))
    for precision, eps in (("fp64", 1e-9), ("mixed", 1e-6)):
        with Plan(1, to_dev(r), to_dev(omega), eps, precision=precision, vec_group=6) as p:
            G = p.execute(to_dev(C)).cpu().numpy()
        ref = oracle.direct(1, r, omega, C)
        bar = 10.0 * eps * (np.abs(C.real).sum(axis=0) + np.abs(C.imag).sum(axis=0))
        assert np.all(np.max(np.abs(G - ref), axis=0) <= bar), precision


def test_group_batched_plan():
    # a batch of problems with different orders (different L per problem in
    # one group launch), eight vectors in one group
    from paper_2411_09583_gb300 import Plan
    eps = 1e-9
    probs = batch_problems(count=12, lo=300, hi=3000, nu_max=12, seed=730)
    nus = [p[0] for p in probs]
    n = [p[1].size for p in probs]
    m = [p[2].size for p in probs]
    r = np.concatenate([p[1] for p in probs])
    omega = np.concatenate([p[2] for p in probs])
    C = np.random.default_rng(731).standard_normal((r.size, 8))
    with Plan.many(nus, to_dev(r), n, to_dev(omega), m, eps, vec_group=8) as bp:
        G = bp.execute(to_dev(C)).cpu().numpy()
    ro = np.concatenate([[0], np.cumsum(n)])
    wo = np.concatenate([[0], np.cumsum(m)])
    for i, (nu, rr, ww, _) in enumerate(probs):
        Ci = C[ro[i]:ro[i + 1]]
        ref = oracle.direct(nu, rr, ww, Ci)
        assert np.all(np.max(np.abs(G[wo[i]:wo[i + 1]] - ref), axis=0) <= tol(eps, Ci)), i


@pytest.mark.parametrize("nu,nvec,group,precision", [(0, 5, 4, "fp64"), (1, 16, 16, "fp64"), (3, 3, 0, "fp64"),
                                                     (0, 6, 8, "mixed"), (2, 3, 1, "fp64")])
def test_groups_adjoint_match_oracle(nu, nvec, group, precision):
    # the adjoint with the same groups: asymptotic members share each
    # frequency's and point's cell, basis and factors, the local blocks run
    # in pairs; every column of every vector against the oracle's transposed sum
    from paper_2411_09583_gb300 import Plan
    eps = 1e-10 if precision == "fp64" else 1e-6
    r, omega, _ = uniform_problem(2400, 2600, omega_max=3000.0, seed=740 + nu)
    E = np.random.default_rng(741 + nvec).standard_normal((omega.size, nvec))
    with Plan(nu, to_dev(r), to_dev(omega), eps, vec_group=group, precision=precision) as p:
        info = p.info()
        assert info["asy_members"] >= 1
        A = p.adjoint(to_dev(E)).cpu().numpy()
    ref = oracle.direct(nu, omega, r, E)
    assert np.all(np.max(np.abs(A - ref), axis=0) <= tol(eps, E))


def test_asy_members_from_group_size():
    # a plan takes as many members per asymptotic launch as its group (grids
    # permitting), one with groups of one or in the deterministic mode
    from paper_2411_09583_gb300 import Plan
    r, omega, _ = uniform_problem(3000, 3000, omega_max=4000.0, seed=750)
    for opts, want in (({"vec_group": 8}, 8), ({}, 2), ({"vec_group": 1}, 1), ({"deterministic": True}, 1)):
        with Plan(0, to_dev(r), to_dev(omega), 1e-9, **opts) as p:
            assert p.info()["asy_members"] == want, opts
