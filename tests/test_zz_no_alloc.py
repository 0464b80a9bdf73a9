"""The no-allocation entry point nuht_local_apply_noalloc.

Callers that cannot let a library allocate device memory (frameworks that
reserve nearly all of it up front, loops that must not stall on the implicit
synchronisation of cudaMalloc / cudaFree) use this call for transforms whose
whole matrix is local.  Its scratch is a fixed device array shared by all
calls, so the test runs it twice in a row (second call with other sizes and
data) and compares each result with the planned path (nuht_plan +
nuht_execute) on the same inputs, and with the oracle's direct sum, within the
accuracy contract.  Frequencies down to 1e-90 (and exactly 0) check the small
argument path of the Bessel values.  This file is collected last so that a run
stopping at the first failure has run the others.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402


def _lib():
    from paper_2411_09583_gb300 import _native, build_native
    build_native.build()
    return _native.lib()


def _noalloc(L, nu, eps, r, rmax, w, wmax, c, nvec):
    dev = torch.device("cuda:0")
    dr, dw, dc = (torch.tensor(x, device=dev) for x in (r, w, c))
    g = torch.full((w.size * nvec,), np.nan, dtype=torch.float64, device=dev)
    s = torch.cuda.current_stream(dev)
    rc = L.nuht_local_apply_noalloc(nu, eps, ctypes.c_void_p(dr.data_ptr()), r.size, rmax,
                                    ctypes.c_void_p(dw.data_ptr()), w.size, wmax,
                                    ctypes.c_void_p(dc.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                    nvec, ctypes.c_void_p(s.cuda_stream))
    torch.cuda.synchronize(dev)
    return rc, g.cpu().numpy().reshape((w.size,) + ((nvec,) if nvec > 1 else ()))


def _planned(nu, eps, r, w, c):
    from paper_2411_09583_gb300 import Plan
    dev = torch.device("cuda:0")
    with Plan(nu, torch.tensor(r, device=dev), torch.tensor(w, device=dev), eps) as p:
        assert p.info()["n_asy"] == 0 and p.info()["n_direct"] == 0   # one local block
        return p.execute(torch.tensor(c, device=dev)).cpu().numpy()


def test_no_alloc_matches_planned_path_twice():
    from paper_2411_09583_gb300 import _native as N
    from paper_2411_09583_gb300 import choose_params
    L = _lib()
    rng = np.random.default_rng(2024)
    # the last case reaches Bessel index 375 (order 100 at 1e-12)
    cases = [(0, 1e-12, 6000, 5000, 1), (3, 1e-9, 1700, 2300, 3), (100, 1e-12, 900, 800, 2)]
    for nu, eps, n, m, nvec in cases:
        M, z, Lw = choose_params(nu, eps)
        r = rng.uniform(0.0, 1.0, n)
        r[0] = 1.0
        w = rng.uniform(0.0, z, m)                 # omega_max * r_max = z: all local
        c = rng.standard_normal((n, nvec)) if nvec > 1 else rng.standard_normal(n)
        w[:5] = [0.0, 1e-90, 1e-60, 1e-20, 1e-3]   # small arguments of the Bessel values
        rc, g = _noalloc(L, nu, eps, r, 1.0, w, z, c, nvec)
        assert rc == N.NUHT_OK, N.lib().nuht_strerror(rc)
        assert np.all(np.isfinite(g))
        ref = _planned(nu, eps, r, w, c)
        tol = 10 * eps * np.abs(c).sum(axis=0)
        assert np.all(np.max(np.abs(g - ref), axis=0) <= tol)
        # against the exact sum on a sample of rows (and every small-argument row)
        rows = np.concatenate([np.arange(5), rng.choice(np.arange(5, m), 60, replace=False)])
        cm = c.reshape(n, -1)
        exact = np.stack([oracle.direct_rows(nu, r, w, cm[:, v], rows) for v in range(cm.shape[1])], axis=1)
        assert np.all(np.max(np.abs(g.reshape(m, -1)[rows] - exact), axis=0) <= tol)


def test_no_alloc_rejects_requests_beyond_its_scratch():
    from paper_2411_09583_gb300 import _native as N
    from paper_2411_09583_gb300 import choose_params
    L = _lib()
    M, z, Lw = choose_params(0, 1e-8)
    r = np.linspace(0, 1, 10)
    w = np.linspace(0, z, 10)
    nvec = N.NOALLOC_MAX_MOMENTS // (Lw + 1) + 1
    c = np.zeros((10, nvec))
    rc, _ = _noalloc(L, 0, 1e-8, r, 1.0, w, z, c, nvec)
    assert rc == N.NUHT_ERR_SCRATCH
    rc, _ = _noalloc(L, 0, 1e-8, r, 1.0, w, 2 * z, np.zeros(10), 1)
    assert rc == N.NUHT_ERR_DOMAIN
