"""Oracle: direct type-3 nonuniform DFT (test infrastructure only).

F(omega_k) = sum_j x_j exp(+i omega_k r_j), the matrix F of Sec. 3.2 evaluated by its definition, O(nm), in FP64.
"""
import numpy as np


def nudft3(r, omega, x, chunk=512):
    r = np.asarray(r, dtype=np.float64)
    omega = np.asarray(omega, dtype=np.float64)
    x = np.asarray(x, dtype=np.complex128)
    out = np.empty(omega.size, dtype=np.complex128)
    for s in range(0, omega.size, chunk):
        ph = np.outer(omega[s:s + chunk], r)
        out[s:s + chunk] = np.exp(1j * ph) @ x
    return out
