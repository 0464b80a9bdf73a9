"""Pins for the oracle's subdivision (Algorithm 1): the block sets tile the
matrix exactly once and every block satisfies its class condition."""
import numpy as np
import pytest

from oracle import subdivide as S


def _check(r, omega, z, min_size, n_cand=16):
    Lb, Ab, Db = S.subdivide(list(r), list(omega), z, min_size, n_cand)
    m, n = len(omega), len(r)
    cover = np.zeros((m, n), dtype=np.int32)
    prod = np.outer(omega, r)
    for blk in Lb + Ab + Db:
        k0, k1, j0, j1 = blk
        assert 0 <= k0 <= k1 < m and 0 <= j0 <= j1 < n
        cover[k0:k1 + 1, j0:j1 + 1] += 1
    assert np.all(cover == 1)
    for k0, k1, j0, j1 in Lb:
        assert np.all(prod[k0:k1 + 1, j0:j1 + 1] <= z)
    for k0, k1, j0, j1 in Ab:
        assert np.all(prod[k0:k1 + 1, j0:j1 + 1] > z)
    for k0, k1, j0, j1 in Db:
        assert (k1 - k0 + 1) * (j1 - j0 + 1) <= min_size
        sub = prod[k0:k1 + 1, j0:j1 + 1]
        assert np.any(sub <= z) and np.any(sub > z)
    return Lb, Ab, Db


@pytest.mark.parametrize("seed", range(6))
def test_tiling_random(seed):
    rng = np.random.default_rng(seed)
    n, m = rng.integers(1, 90, 2)
    r = np.sort(rng.uniform(0, 1, n))
    omega = np.sort(rng.uniform(0, 300, m))
    for z in [0.5, 15.5, 80.0]:
        for ms in [1, 16, 64]:
            for nc in [2, 4, 16]:
                _check(r, omega, z, ms, nc)


def test_ties_and_duplicates():
    r = np.sort(np.array([0.0, 0.0, 0.25, 0.25, 0.5, 1.0, 1.0]))
    omega = np.sort(np.array([0.0, 10.0, 20.0, 20.0, 40.0, 62.0]))
    for z in [5.0, 10.0, 20.0]:      # includes products exactly equal to z
        _check(r, omega, z, 2, 3)


def test_pure_matrices():
    r = np.linspace(0, 1, 50)
    omega = np.linspace(0, 10, 40)
    Lb, Ab, Db = S.subdivide(list(r), list(omega), 100.0)
    assert Lb == [(0, 39, 0, 49)] and not Ab and not Db
    Lb, Ab, Db = S.subdivide(list(r + 1), list(omega + 200), 100.0)
    assert Ab == [(0, 39, 0, 49)] and not Lb and not Db


def test_split_minimises_mixed_area_among_candidates():
    rng = np.random.default_rng(9)
    r = np.sort(rng.uniform(0, 1, 200))
    omega = np.sort(rng.uniform(0, 1000, 150))
    z = 30.0
    blk = (0, 149, 0, 199)
    k, j = S.split_indices(r, omega, z, blk, n_cand=150)   # every row is a candidate
    def area(kk):
        jj = int(np.searchsorted(omega[kk] * r, z, side="right")) - 1
        return kk * 0 + (kk + 1) * (199 - jj) + (149 - kk) * (jj + 1), jj
    best = min(area(kk)[0] for kk in range(150))
    assert area(k) == (best, j)
    assert omega[k] * r[j] <= z and (j == 199 or omega[k] * r[j + 1] > z)


def test_levels_logarithmic():
    # the number of mixed-block generations grows like log min(n, m) (Thm. 4.1)
    rng = np.random.default_rng(2)
    for n in [1000, 8000]:
        r = np.sort(rng.uniform(0, 1, n))
        omega = np.sort(rng.uniform(0, n, n))
        Lb, Ab, Db = S.subdivide(list(r), list(omega), 15.5)
        assert len(Lb) + len(Ab) + len(Db) < 40 * n / 100
