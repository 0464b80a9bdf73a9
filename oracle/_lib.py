"""ctypes loader for the oracle's C code (test infrastructure only).

The shared library is compiled with plain gcc from ``direct.c`` into
``oracle/_build/`` on first use (or by ``__graft_entry__.build()``).
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "direct.c")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the oracle's C code (gcc, -O2, no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            d, i, i64 = ctypes.c_double, ctypes.c_int, ctypes.c_int64
            p = ctypes.c_void_p
            lib.oracle_jn.restype = d
            lib.oracle_jn.argtypes = [i, d]
            lib.oracle_jn_prod.restype = d
            lib.oracle_jn_prod.argtypes = [i, d, d]
            lib.oracle_jv_series.restype = d
            lib.oracle_jv_series.argtypes = [d, d]
            lib.oracle_jv_hankel.restype = d
            lib.oracle_jv_hankel.argtypes = [d, d, ctypes.POINTER(i)]
            lib.oracle_jn_miller.restype = d
            lib.oracle_jn_miller.argtypes = [i, d]
            lib.oracle_direct.restype = i
            lib.oracle_direct.argtypes = [i, p, i64, p, p, i64, p, i, p, i]
            lib.oracle_jn_array.restype = None
            lib.oracle_jn_array.argtypes = [i, p, p, i64]
            _lib = lib
    return _lib


def jn(n, x):
    """J_n(x) for integer n, x >= 0 (scalar or array)."""
    lib = _load()
    x = np.asarray(x, dtype=np.float64)
    if x.ndim == 0:
        return lib.oracle_jn(int(n), float(x))
    xs = np.ascontiguousarray(x.ravel())
    out = np.empty_like(xs)
    lib.oracle_jn_array(int(n), xs.ctypes.data, out.ctypes.data, xs.size)
    return out.reshape(x.shape)


def jn_prod(n, a, b):
    """J_n(a*b) at the exact product of the doubles a and b."""
    return _load().oracle_jn_prod(int(n), float(a), float(b))


def jv_series(nu, x):
    """Power-series path only (DLMF 10.2.2), any real nu >= 0."""
    return _load().oracle_jv_series(float(nu), float(x))


def jv_hankel(nu, x):
    """Hankel-expansion path only; returns (value, converged)."""
    ok = ctypes.c_int(0)
    v = _load().oracle_jv_hankel(float(nu), float(x), ctypes.byref(ok))
    return v, bool(ok.value)


def jn_miller(n, x):
    """Miller backward-recurrence path only (integer n >= 0)."""
    return _load().oracle_jn_miller(int(n), float(x))


def _prep(r, omega, c):
    r = np.ascontiguousarray(r, dtype=np.float64)
    omega = np.ascontiguousarray(omega, dtype=np.float64)
    c = np.asarray(c)
    cplx = np.iscomplexobj(c)
    if cplx:
        cv = np.ascontiguousarray(
            np.stack([c.real, c.imag], axis=-1).reshape(c.shape[0], -1)
            if c.size else np.zeros((c.shape[0], 2)), dtype=np.float64)
    else:
        cv = np.ascontiguousarray(c.reshape(c.shape[0], -1) if c.ndim > 1
                                  else c.reshape(-1, 1), dtype=np.float64)
    if cv.shape[0] != r.shape[0]:
        raise ValueError("c must have one row per point r_j")
    return r, omega, c, cv, cplx


def _finish(g, c, cplx, nrows):
    if cplx:
        g = g.reshape(nrows, -1, 2)
        g = g[..., 0] + 1j * g[..., 1]
    if c.ndim == 1:
        return g.reshape(nrows)
    return g.reshape((nrows,) + c.shape[1:])


def direct_rows(nu, r, omega, c, rows, nthreads=0):
    """g_i = sum_j c_j J_nu(omega[rows_i] r_j) for the selected rows only.

    c may be real or complex, shape (n,) or (n, nvec).  The operator is
    real, so a complex c is transformed as its real and imaginary parts.
    """
    lib = _load()
    r, omega, c, cv, cplx = _prep(r, omega, c)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    if rows.size and (rows.min() < 0 or rows.max() >= omega.size):
        raise IndexError("row index out of range")
    nvec = cv.shape[1]
    g = np.zeros((rows.size, nvec), dtype=np.float64)
    if rows.size and r.size:
        lib.oracle_direct(int(nu), r.ctypes.data, r.size, omega.ctypes.data,
                          rows.ctypes.data, rows.size, cv.ctypes.data, nvec,
                          g.ctypes.data, int(nthreads))
    return _finish(g, c, cplx, rows.size)


def direct(nu, r, omega, c, nthreads=0):
    """Full O(nm) direct sum g_k = sum_j c_j J_nu(omega_k r_j) (Sec. 1, eq. DHT)."""
    return direct_rows(nu, r, omega, c, np.arange(np.asarray(omega).size),
                       nthreads)
