"""The persistent local stage (nuht_opts.persistent = 1) and its bounded waits.

One launch of resident CTAs takes the local blocks' moment tiles and then
their evaluation tiles from a device queue; an evaluation tile polls a
per-block counter until its block's moments are complete.  The polls are
bounded: a wait that gives up records NUHT_ERR_TIMEOUT (read by nuht_status)
and the launch still finishes, so the GPU context stays usable.  The timeout
test makes one block's wait impossible (NUHT_QUEUE_STALL asks for one moment
tile more than the block has) with a short poll limit.
"""
import numpy as np
import pytest

import oracle
from paper_2411_09583_gb300.workloads import batch_problems, loguniform_problem, sample_rows, uniform_problem

pytestmark = pytest.mark.gpu

from gpu_helpers import to_dev, tol  # noqa: E402


@pytest.mark.parametrize("nu,eps,precision", [(0, 1e-12, "fp64"), (5, 1e-9, "fp64"), (1, 1e-6, "mixed")])
def test_persistent_local_stage_matches_oracle(nu, eps, precision):
    from paper_2411_09583_gb300 import Plan
    from paper_2411_09583_gb300 import _native as N
    r, omega, c = uniform_problem(30000, 25000, omega_max=3e4, seed=900 + nu)
    with Plan(nu, to_dev(r), to_dev(omega), eps, precision=precision, persistent=True) as p:
        assert p.info()["n_local"] > 0
        g = p.execute(to_dev(c)).cpu().numpy()
        assert p.status() == N.NUHT_OK
    with Plan(nu, to_dev(r), to_dev(omega), eps, precision=precision) as p:
        g0 = p.execute(to_dev(c)).cpu().numpy()
    rows = sample_rows(omega.size, 300, seed=901)
    assert np.max(np.abs(g[rows] - oracle.direct_rows(nu, r, omega, c, rows))) <= tol(eps, c)
    assert np.max(np.abs(g - g0)) <= 1e-2 * tol(eps, c)


def test_persistent_pairs_and_batch():
    from paper_2411_09583_gb300 import Plan
    from paper_2411_09583_gb300 import _native as N
    eps = 1e-9
    # complex c: the two components' moments in one queue
    r, omega, c = loguniform_problem(8000, 7000, omega_max=5e3, seed=910, complex_c=True)
    with Plan(1, to_dev(r), to_dev(omega), eps, persistent=True) as p:
        g = p.execute(to_dev(c)).cpu().numpy()
        assert p.status() == N.NUHT_OK
    rows = sample_rows(omega.size, 150, seed=911)
    assert np.max(np.abs(g[rows] - oracle.direct_rows(1, r, omega, c, rows))) <= tol(eps, c)
    # a batch of uneven problems in one plan
    probs = batch_problems(count=20, lo=200, hi=6000, nu_max=20, seed=912)
    nus = [q[0] for q in probs]
    n = [q[1].size for q in probs]
    m = [q[2].size for q in probs]
    cc = np.concatenate([q[3] for q in probs])
    with Plan.many(nus, to_dev(np.concatenate([q[1] for q in probs])), n,
                   to_dev(np.concatenate([q[2] for q in probs])), m, 1e-8, persistent=True) as bp:
        gb = bp.execute(to_dev(cc)).cpu().numpy()
        assert bp.status() == N.NUHT_OK
    off = 0
    for nu, rr, ww, ci in probs:
        assert np.max(np.abs(gb[off:off + ww.size] - oracle.direct(nu, rr, ww, ci))) <= tol(1e-8, ci)
        off += ww.size


def test_bounded_wait_gives_up_and_context_recovers(monkeypatch):
    from paper_2411_09583_gb300 import Plan
    from paper_2411_09583_gb300 import _native as N
    eps = 1e-10
    r, omega, c = uniform_problem(6000, 5000, omega_max=6e3, seed=920)
    with Plan(0, to_dev(r), to_dev(omega), eps, persistent=True) as p:
        assert p.info()["n_local"] > 0
        monkeypatch.setenv("NUHT_QUEUE_STALL", "1")
        p.execute(to_dev(c))
        assert p.status() == N.NUHT_ERR_TIMEOUT
        assert p.status() == N.NUHT_OK          # cleared by the read
        monkeypatch.delenv("NUHT_QUEUE_STALL")
        g = p.execute(to_dev(c)).cpu().numpy()
        assert p.status() == N.NUHT_OK
    assert np.max(np.abs(g - oracle.direct(0, r, omega, c))) <= tol(eps, c)
