"""Pins for the oracle gradients: central finite differences of the oracle loss
(second order in the step) and the closed form J_0' = -J_1."""
import numpy as np

import oracle
from oracle import gradient as G


def _setup(nu, seed=0, n=40, m=35):
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.05, 1, n)
    omega = rng.uniform(0, 60, m)
    c = rng.standard_normal(n)
    gstar = oracle.direct(nu, r, omega, c + 0.01 * rng.standard_normal(n))
    return r, omega, c, gstar


def test_derivative_identity():
    x = np.linspace(0.1, 40, 50)
    # J_0' = -J_1 and (J_{-1} - J_1)/2 = -J_1
    assert np.max(np.abs(0.5 * (oracle.jn(-1, x) - oracle.jn(1, x)) + oracle.jn(1, x))) < 1e-15


def test_gradients_match_finite_differences():
    for nu in (0, 1, 3):
        r, omega, c, gstar = _setup(nu, seed=nu)
        L0, dc, dr, dw = G.gradients(nu, r, omega, c, gstar)
        h = 2e-6   # central differences: O(h^2) truncation, O(1e-16 L / h) rounding
        for j in (0, 7, 21):
            for arr, grad in ((c, dc), (r, dr)):
                xp, xm = arr.copy(), arr.copy()
                xp[j] += h
                xm[j] -= h
                args_p = (xp, omega) if arr is r else (r, omega)
                args_m = (xm, omega) if arr is r else (r, omega)
                cp = c if arr is r else xp
                cm = c if arr is r else xm
                fd = (G.loss(nu, *args_p, cp, gstar) - G.loss(nu, *args_m, cm, gstar)) / (2 * h)
                assert abs(fd - grad[j]) <= 1e-6 * max(1.0, abs(grad[j])), (nu, j)
        for k in (0, 11):
            wp, wm = omega.copy(), omega.copy()
            wp[k] += h
            wm[k] -= h
            fd = (G.loss(nu, r, wp, c, gstar) - G.loss(nu, r, wm, c, gstar)) / (2 * h)
            assert abs(fd - dw[k]) <= 1e-6 * max(1.0, abs(dw[k]))
