"""CPU-side checks of the C ABI: the library loads, exports every symbol the
header declares, and its host-only parameter choice matches the oracle."""
import ctypes
import os
import re

import pytest

from oracle import params as OP

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2411_09583_gb300 import _native, build_native
    build_native.build()
    return _native.lib()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "nuht.h")).read()
    declared = set(re.findall(r"\b(nuht_[a-z_]+)\s*\(", hdr))
    from paper_2411_09583_gb300 import _native
    assert declared == set(_native.EXPORTED)
    for name in declared:
        assert hasattr(lib, name), name


@pytest.mark.parametrize("nu,eps", [(0, 1e-12), (0, 1e-8), (1, 1e-5), (1, 1e-10), (2, 1e-12),
                                    (3, 1e-12), (10, 1e-12), (19, 1e-8), (20, 1e-8), (7, 1e-4),
                                    (5, 1e-15), (50, 1e-10)])
def test_params_match_oracle(lib, nu, eps):
    from paper_2411_09583_gb300 import choose_params
    M, z, L = choose_params(nu, eps)
    Mo, zo, Lo = OP.choose_params(nu, eps)
    assert (M, L) == (Mo, Lo)
    assert abs(z - zo) <= 1e-12 * zo


def test_params_cached_and_concurrent_calls_agree(lib):
    # the parameter choice is remembered per (order, tolerance, forced M): a
    # repeated call (answered from memory) and calls from several host threads
    # return the first call's values, which are the oracle's
    import concurrent.futures as cf
    from paper_2411_09583_gb300 import choose_params
    cases = [(nu, eps, mt) for nu in (0, 1, 4, 13) for eps in (1e-6, 1e-9, 1e-13) for mt in (0, 6)]
    first = {c: choose_params(c[0], c[1], m_terms=c[2]) for c in cases}
    with cf.ThreadPoolExecutor(8) as ex:
        again = list(ex.map(lambda c: (c, choose_params(c[0], c[1], m_terms=c[2])), cases * 4))
    for c, v in again:
        assert v == first[c], c
    for (nu, eps, mt), (M, z, L) in first.items():
        if mt == 0:
            Mo, zo, Lo = OP.choose_params(nu, eps)
            assert (M, L) == (Mo, Lo)
            assert abs(z - zo) <= 1e-12 * zo
        else:
            assert M == mt
            assert abs(z - OP.crossover_z(nu, mt, eps)) <= 1e-12 * z
            assert L == OP.choose_l(nu, z, eps)


def test_params_negative_order_and_forced_m(lib):
    from paper_2411_09583_gb300 import choose_params
    assert choose_params(-3, 1e-8) == choose_params(3, 1e-8)
    M, z, L = choose_params(0, 1e-10, m_terms=5)
    assert M == 5
    assert abs(z - OP.crossover_z(0, 5, 1e-10)) <= 1e-12 * z
    assert L == OP.choose_l(0, z, 1e-10)


def test_invalid_arguments(lib):
    from paper_2411_09583_gb300 import _native as N
    M, z, L = ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
    assert lib.nuht_choose_params(0, 1.0, 0, ctypes.byref(M), ctypes.byref(z), ctypes.byref(L)) == N.NUHT_ERR_INVALID_ARG
    assert lib.nuht_choose_params(0, 1e-20, 0, ctypes.byref(M), ctypes.byref(z), ctypes.byref(L)) == N.NUHT_ERR_INVALID_ARG
    assert lib.nuht_choose_params(0, 1e-8, 21, ctypes.byref(M), ctypes.byref(z), ctypes.byref(L)) == N.NUHT_ERR_INVALID_ARG
    assert lib.nuht_choose_params(101, 1e-8, 0, ctypes.byref(M), ctypes.byref(z), ctypes.byref(L)) == N.NUHT_ERR_UNSUPPORTED
    h = ctypes.c_void_p()
    assert lib.nuht_plan(ctypes.byref(h), 0, None, -1, None, 0, 1e-8, None, None) == N.NUHT_ERR_INVALID_ARG
    assert lib.nuht_plan(ctypes.byref(h), 0, None, 0, None, 0, 2.0, None, None) == N.NUHT_ERR_INVALID_ARG
    assert lib.nuht_plan(None, 0, None, 0, None, 0, 1e-8, None, None) == N.NUHT_ERR_INVALID_ARG
    assert lib.nuht_execute(None, None, None, 1, 0, None) == N.NUHT_ERR_INVALID_ARG
    assert lib.nuht_strerror(N.NUHT_ERR_DOMAIN).decode().startswith("r and omega")
    o = N.NuhtOpts()
    lib.nuht_default_opts(ctypes.byref(o))
    assert (o.precision, o.min_size, o.n_split_cand, o.m_terms, o.class_mask) == (0, 1024, 16, 0, 7)
    # option checks run before any device work
    one = (ctypes.c_double * 1)(0.5)
    for field, bad in (("min_size", 0), ("min_size", 16385), ("n_split_cand", 1), ("spread_tile", 96 + 1),
                       ("precision", 2), ("m_terms", 21), ("deterministic", 2), ("persistent", 3),
                       ("interp_tile", 64), ("interp_tile", 512), ("vec_group", -1), ("vec_group", 17),
                       ("reserved", 1)):
        b = N.NuhtOpts()
        lib.nuht_default_opts(ctypes.byref(b))
        setattr(b, field, bad)
        assert lib.nuht_plan(ctypes.byref(h), 0, one, 1, one, 1, 1e-8, ctypes.byref(b), None) == \
            N.NUHT_ERR_INVALID_ARG, field
    # vector groups above a pair exclude the deterministic and persistent modes
    for field in ("deterministic", "persistent"):
        b = N.NuhtOpts()
        lib.nuht_default_opts(ctypes.byref(b))
        b.vec_group = 3
        setattr(b, field, 1)
        assert lib.nuht_plan(ctypes.byref(h), 0, one, 1, one, 1, 1e-8, ctypes.byref(b), None) == \
            N.NUHT_ERR_INVALID_ARG, field
