"""Pins for the oracle's direct type-3 DFT (the matrix F of Sec. 3.2)."""
import numpy as np

from oracle.nudft import nudft3


def test_single_point_is_a_pure_exponential():
    omega = np.linspace(0, 500, 37)
    out = nudft3(np.array([0.3]), omega, np.array([2.0 - 1.0j]))
    assert np.max(np.abs(out - (2.0 - 1.0j) * np.exp(0.3j * omega))) < 1e-13


def test_equispaced_points_geometric_sum():
    # sum_{j<n} e^{i w j h} = (1 - e^{i w n h}) / (1 - e^{i w h})
    n, h = 50, 0.013
    r = h * np.arange(n)
    omega = np.array([0.7, 3.3, 101.0, 2000.5])
    ref = (1 - np.exp(1j * omega * n * h)) / (1 - np.exp(1j * omega * h))
    assert np.max(np.abs(nudft3(r, omega, np.ones(n)) - ref)) < 1e-11


def test_conjugate_symmetry_and_linearity():
    rng = np.random.default_rng(1)
    r = rng.uniform(0, 1, 40)
    omega = rng.uniform(0, 300, 30)
    x = rng.standard_normal(40)
    assert np.max(np.abs(nudft3(r, -omega, x) - np.conj(nudft3(r, omega, x)))) < 1e-12
    y = rng.standard_normal(40)
    assert np.max(np.abs(nudft3(r, omega, x + 2j * y) - nudft3(r, omega, x) - 2j * nudft3(r, omega, y))) < 1e-12
