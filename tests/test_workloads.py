"""The seeded input generators checked against facts they must satisfy."""
import numpy as np
import pytest

import oracle
from paper_2411_09583_gb300.workloads import exponential_grid, fourier_bessel_grid, sparse_coefficients


@pytest.mark.parametrize("nu", [0, 1, 7])
def test_fourier_bessel_grid_are_roots(nu):
    # omega_k = j_{nu,k}: the oracle's J_nu vanishes there (to rounding of a
    # root of size ~ k pi, with |J_nu'| ~ sqrt(2 / (pi x))), the roots are
    # increasing with gaps tending to pi (McMahon), and r = omega / j_{nu,n+1}
    # lies in (0, 1)
    r, omega = fourier_bessel_grid(nu, 400)
    assert omega.size == r.size == 400
    assert np.all(np.abs(oracle.jn(nu, omega)) <= 1e-13 * np.maximum(omega, 1.0))
    # the root after the last one scales r: J_nu(omega_last / r_last) = 0 too
    assert abs(oracle.jn(nu, omega[-1] / r[-1])) <= 1e-12
    assert np.all(np.diff(omega) > 0) and np.all((r > 0) & (r < 1))
    assert abs((omega[-1] - omega[-2]) - np.pi) < 1e-3
    # J_nu has no positive root below nu
    assert omega[0] > nu


def test_exponential_grid_endpoints():
    # omega_j = r_j = 10^(log10 j - log10(n)/2): geometric, r_1 r_n = 1
    v, w = exponential_grid(1000)
    assert np.allclose(v, w) and np.isclose(v[0] * v[-1], 1.0)
    assert np.allclose(v[1:] / v[:-1], np.arange(2, 1001) / np.arange(1, 1000))


def test_sparse_coefficients():
    c, idx = sparse_coefficients(5000, nnz=1000, seed=3)
    assert np.count_nonzero(c) == 1000 and np.unique(idx).size == 1000
    assert np.all(c[idx] != 0) and np.isclose(c[idx].std(), 1.0, atol=0.1)
