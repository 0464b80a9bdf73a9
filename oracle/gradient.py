"""Oracle: gradients of L = 1/2 ||A(r, omega) c - g*||^2 (test infrastructure only).

A(k, j) = J_nu(omega_k r_j) (Sec. 1, eq. DHT).  With e = A c - g*:
  dL/dc_j     = sum_k e_k J_nu(omega_k r_j)                       (the transpose)
  dL/dr_j     = c_j sum_k e_k omega_k J_nu'(omega_k r_j)
  dL/domega_k = e_k sum_j c_j r_j J_nu'(omega_k r_j)
with J_nu' = (J_{nu-1} - J_{nu+1}) / 2 (DLMF 10.6.1) and J_{-1} = -J_1.
Every sum is the oracle's direct sum; real c only.
"""
import numpy as np

from . import _lib


def loss(nu, r, omega, c, gstar):
    e = _lib.direct(nu, r, omega, c) - gstar
    return 0.5 * float(np.dot(e, e))


def gradients(nu, r, omega, c, gstar):
    """(loss, dL/dc, dL/dr, dL/domega) by direct sums."""
    r = np.asarray(r, dtype=np.float64)
    omega = np.asarray(omega, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    e = _lib.direct(nu, r, omega, c) - gstar
    # the transpose A^T e: J(omega r) is symmetric in its two arguments
    dc = _lib.direct(nu, omega, r, e)
    we = omega * e
    dr = c * 0.5 * (_lib.direct(nu - 1, omega, r, we) - _lib.direct(nu + 1, omega, r, we))
    rc = r * c
    dw = e * 0.5 * (_lib.direct(nu - 1, r, omega, rc) - _lib.direct(nu + 1, r, omega, rc))
    return 0.5 * float(np.dot(e, e)), dc, dr, dw
