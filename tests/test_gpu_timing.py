"""Stage timing of the execute (opts.timing): live events on each stage's own
stream (the block classes run concurrently, as without timing) and serial
events (every stage in order on the caller's stream)."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2411_09583_gb300.workloads import uniform_problem

pytestmark = pytest.mark.gpu

from gpu_helpers import to_dev, tol  # noqa: E402

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("mode", [True, "serial"])
def test_stage_times_and_results(mode):
    from paper_2411_09583_gb300 import Plan
    r, omega, c = uniform_problem(3000, 2800, omega_max=4000.0, seed=41)
    eps = 1e-10
    e = np.random.default_rng(42).standard_normal(omega.size)
    with Plan(0, to_dev(r), to_dev(omega), eps, timing=mode) as p:
        info = p.info()
        assert min(info["n_local"], info["n_asy"], info["n_direct"]) > 0
        dc = to_dev(c)
        p.execute(dc)
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        g = p.execute(dc)
        s1.record()
        torch.cuda.synchronize()
        st = p.stage_times()
        wall = s0.elapsed_time(s1)
        ca = p.adjoint(to_dev(e)).cpu().numpy()
        sta = p.stage_times()
    rows = np.arange(0, omega.size, 7)
    assert np.max(np.abs(g.cpu().numpy()[rows] - oracle.direct_rows(0, r, omega, c, rows))) <= tol(eps, c)
    cols = np.arange(0, r.size, 7)
    assert np.max(np.abs(ca[cols] - oracle.direct_rows(0, omega, r, e, cols))) <= tol(eps, e)
    for times in (st, sta):
        for k in ("local_moments", "local_eval", "direct", "asy_spread", "asy_fft", "asy_interp"):
            assert times[k] > 0.0, (k, times)
    if mode == "serial":
        # one stream, stages in order: their times add up to at most the wall time
        assert sum(st.values()) <= 1.05 * wall + 0.02, (st, wall)


def test_invalid_timing_mode_rejected():
    from paper_2411_09583_gb300 import _native as N
    from paper_2411_09583_gb300.nuht import _stream_ptr, make_opts
    r, omega, _ = uniform_problem(100, 100, omega_max=100.0, seed=43)
    dr, dw = to_dev(r), to_dev(omega)
    o = make_opts()
    o.timing = 3
    h = ctypes.c_void_p()
    rc = N.lib().nuht_plan(ctypes.byref(h), 0, ctypes.c_void_p(dr.data_ptr()), r.size,
                           ctypes.c_void_p(dw.data_ptr()), omega.size, 1e-8, ctypes.byref(o),
                           _stream_ptr(None))
    assert rc == N.NUHT_ERR_INVALID_ARG
    assert not h.value
