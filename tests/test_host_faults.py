"""Host-side fault injection and work-list checks (no GPU needed).

* A forced device-allocation failure (NUHT_FAULT_ALLOC=k fails the k-th
  allocation of the library) makes the entry points return NUHT_ERR_NOMEM,
  with no plan handed out; it acts before any CUDA call, so it runs here.
* nuht_check_blocks accepts the oracle's subdivision (Algorithm 1) of a
  sorted problem and rejects lists with a gap, an overlap, a block of the
  wrong class, a direct block above min_size, indices outside the matrix or
  unsorted inputs.
"""
import ctypes

import numpy as np
import pytest

from oracle import params as OP
from oracle import subdivide as OS


@pytest.fixture(scope="module")
def lib():
    from paper_2411_09583_gb300 import _native, build_native
    build_native.build()
    return _native.lib()


def test_forced_allocation_failure_returns_nomem(lib, monkeypatch):
    from paper_2411_09583_gb300 import _native as N
    r = (ctypes.c_double * 4)(0.1, 0.2, 0.3, 0.4)
    w = (ctypes.c_double * 4)(1.0, 2.0, 3.0, 4.0)
    monkeypatch.setenv("NUHT_FAULT_ALLOC", "1")
    h = ctypes.c_void_p(12345)
    assert lib.nuht_plan(ctypes.byref(h), 0, r, 4, w, 4, 1e-8, None, None) == N.NUHT_ERR_NOMEM
    assert h.value is None
    assert lib.nuht_strerror(N.NUHT_ERR_NOMEM).decode() == "out of memory"
    assert "cudaErrorMemoryAllocation" in lib.nuht_last_cuda_error().decode() or \
        "out of memory" in lib.nuht_last_cuda_error().decode()
    nus = (ctypes.c_int * 1)(0)
    ns = (ctypes.c_int64 * 1)(4)
    monkeypatch.setenv("NUHT_FAULT_ALLOC", "01")   # a new value restarts the count
    assert lib.nuht_plan_many(ctypes.byref(h), 1, nus, r, ns, w, ns, 1e-8, None, None) == N.NUHT_ERR_NOMEM
    assert h.value is None
    c = (ctypes.c_double * 4)(1.0, -1.0, 0.5, 2.0)
    g = (ctypes.c_double * 4)()
    monkeypatch.setenv("NUHT_FAULT_ALLOC", "1")
    assert lib.nuht_transform_host(0, r, 4, w, 4, 1e-8, c, g, 1, None, None) == N.NUHT_ERR_NOMEM
    ms, ops = ctypes.c_double(), ctypes.c_double()
    monkeypatch.setenv("NUHT_FAULT_ALLOC", "001")
    rc = lib.nuht_probe_alu(0, 16, ctypes.byref(ms), ctypes.byref(ops), None)
    # without a GPU the probe may fail at the device query before it allocates
    assert rc in (N.NUHT_ERR_NOMEM, N.NUHT_ERR_CUDA)


def _problem(seed, n=300, m=260, omega_max=900.0, nu=0, eps=1e-8):
    rng = np.random.default_rng(seed)
    r = np.sort(rng.uniform(0, 1, n))
    w = np.sort(rng.uniform(0, omega_max, m))
    M, z, L = OP.choose_params(nu, eps)
    Lb, Ab, Db = OS.subdivide(list(r), list(w), z, min_size=256, n_cand=16)
    ranges = np.array(Lb + Ab + Db, dtype=np.int64).reshape(-1, 4)
    cls = np.array([0] * len(Lb) + [1] * len(Ab) + [2] * len(Db), dtype=np.int32)
    return r, w, ranges, cls


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_valid_subdivision_accepted(lib, seed):
    from paper_2411_09583_gb300 import _native as N
    from paper_2411_09583_gb300.nuht import check_blocks
    r, w, ranges, cls = _problem(seed)
    assert len(set(cls.tolist())) == 3
    assert check_blocks(0, 1e-8, r, w, ranges, cls, min_size=256) == N.NUHT_OK


def test_invalid_work_lists_rejected(lib):
    from paper_2411_09583_gb300 import _native as N
    from paper_2411_09583_gb300.nuht import check_blocks
    r, w, ranges, cls = _problem(7)
    bad = N.NUHT_ERR_BAD_BLOCKS

    def chk(rg, cl, **kw):
        return check_blocks(0, 1e-8, kw.get("r", r), kw.get("w", w), rg, cl, min_size=kw.get("min_size", 256))

    # a gap: one block dropped
    for i in (0, len(cls) // 2, len(cls) - 1):
        assert chk(np.delete(ranges, i, 0), np.delete(cls, i)) == bad
    # an overlap: one block listed twice
    assert chk(np.vstack([ranges, ranges[:1]]), np.append(cls, cls[0])) == bad
    # a block widened by one column (overlaps its neighbour or leaves the matrix)
    rg = ranges.copy()
    rg[3, 3] += 1
    assert chk(rg, cls) == bad
    # a row index outside the matrix
    rg = ranges.copy()
    rg[np.argmax(rg[:, 1]), 1] = w.size
    assert chk(rg, cls) == bad
    # local / asymptotic blocks relabelled
    iloc, iasy = int(np.flatnonzero(cls == 0)[0]), int(np.flatnonzero(cls == 1)[0])
    for i, c in ((iloc, 1), (iasy, 0), (iloc, 7)):
        cl = cls.copy()
        cl[i] = c
        assert chk(ranges, cl) == bad
    # a direct block above min_size
    idir = int(np.flatnonzero(cls == 2)[0])
    area = (ranges[idir, 1] - ranges[idir, 0] + 1) * (ranges[idir, 3] - ranges[idir, 2] + 1)
    assert chk(ranges, cls, min_size=int(area) - 1) == bad
    # unsorted inputs
    r2 = r.copy()
    r2[[5, 6]] = r2[[6, 5]] if r2[5] != r2[6] else (r2[5] + 1, r2[6])
    assert chk(ranges, cls, r=r2) == bad
    # empty matrix: only the empty list is valid
    assert chk(np.zeros((0, 4), np.int64), np.zeros(0, np.int32), r=r[:0]) == N.NUHT_OK
    assert chk(ranges[:1], cls[:1], r=r[:0]) == bad
    # arguments
    assert check_blocks(0, 2.0, r, w, ranges, cls) == N.NUHT_ERR_INVALID_ARG
    assert check_blocks(101, 1e-8, r, w, ranges, cls) == N.NUHT_ERR_UNSUPPORTED
