"""GPU parity of the adjoint (transposed) NUHT and of the differentiable transform."""
import numpy as np
import pytest

import oracle
from oracle import gradient as OG
from paper_2411_09583_gb300.workloads import loguniform_problem, sample_rows, uniform_problem

pytestmark = pytest.mark.gpu

from gpu_helpers import class_reference, dev, to_dev, tol  # noqa: E402

torch = pytest.importorskip("torch")


def _adjoint(nu, r, omega, e, eps, **opts):
    from paper_2411_09583_gb300 import Plan
    with Plan(nu, to_dev(r), to_dev(omega), eps, **opts) as p:
        return p.adjoint(to_dev(e)).cpu().numpy(), [p.blocks(k) for k in range(3)]


@pytest.mark.parametrize("nu", [0, 1, 5, 12])
def test_adjoint_matches_oracle_transpose(nu):
    r, omega, _ = uniform_problem(1500, 1300, omega_max=2500.0, seed=60 + nu)
    e = np.random.default_rng(61 + nu).standard_normal(omega.size)
    eps = 1e-10
    ca, _ = _adjoint(nu, r, omega, e, eps)
    ref = oracle.direct(nu, omega, r, e)       # (A^T e)_j = sum_k e_k J(omega_k r_j)
    assert np.max(np.abs(ca - ref)) <= tol(eps, e)


@pytest.mark.parametrize("nu,eps", [(50, 1e-8), (100, 1e-6), (100, 1e-12), (20, 1e-14)])
def test_adjoint_extreme_orders(nu, eps):
    """High orders (Hankel coefficients beyond the FP32 range unless scaled,
    Bessel indices above 256) through the transposed block kernels."""
    r, omega, _ = uniform_problem(1100, 1000, omega_max=3000.0 + 30 * nu, seed=90 + nu)
    e = np.random.default_rng(91 + nu).standard_normal(omega.size)
    ca, _ = _adjoint(nu, r, omega, e, eps)
    ref = oracle.direct(nu, omega, r, e)
    assert np.max(np.abs(ca - ref)) <= tol(eps, e)


def test_adjoint_scaled_inputs():
    # the fixed-point frames of the transposed kernels far from unit scale
    r, omega, _ = uniform_problem(1200, 1100, omega_max=3000.0, seed=92)
    e = np.random.default_rng(93).standard_normal(omega.size)
    for sr, sw in ((1e5, 1e-5), (1e-6, 1e6)):
        ca, _ = _adjoint(2, r * sr, omega * sw, e, 1e-10)
        ref = oracle.direct(2, omega * sw, r * sr, e)
        assert np.max(np.abs(ca - ref)) <= tol(1e-10, e)


@pytest.mark.parametrize("nu", [0, 3])
def test_dot_product_identity(nu):
    # <A c, e> = <c, A^T e> for the approximate operator itself (exact transpose)
    from paper_2411_09583_gb300 import Plan
    r, omega, c = uniform_problem(3000, 2800, omega_max=4000.0, seed=70 + nu)
    e = np.random.default_rng(71).standard_normal(omega.size)
    with Plan(nu, to_dev(r), to_dev(omega), 1e-8) as p:
        g = p.execute(to_dev(c)).cpu().numpy()
        ca = p.adjoint(to_dev(e)).cpu().numpy()
    lhs, rhs = float(np.dot(g, e)), float(np.dot(c, ca))
    scale = float(np.abs(g).dot(np.abs(e)) + np.abs(c).dot(np.abs(ca)))
    assert abs(lhs - rhs) <= 1e-13 * scale, (lhs, rhs)


@pytest.mark.parametrize("cls", [0, 1, 2])
def test_adjoint_each_block_class(cls):
    r, omega, _ = uniform_problem(1400, 1600, omega_max=3000.0, seed=72)
    e = np.random.default_rng(73).standard_normal(omega.size)
    eps = 1e-10
    ca, blocks = _adjoint(0, r, omega, e, eps, class_mask=1 << cls)
    # transposed blocks: swap the roles of rows and columns
    swapped = [(j0, j1, k0, k1) for k0, k1, j0, j1 in blocks[cls]]
    ref = class_reference(0, omega, r, e, swapped)
    assert np.max(np.abs(ca - ref)) <= tol(eps, e)


def test_adjoint_complex_multi_and_clustered():
    r, omega, _ = loguniform_problem(1200, 1000, omega_max=4e4, seed=74, complex_c=False)
    rng = np.random.default_rng(75)
    e = rng.standard_normal((omega.size, 2))
    ca, _ = _adjoint(1, r, omega, e, 1e-9)
    ref = oracle.direct(1, omega, r, e)
    assert np.all(np.max(np.abs(ca - ref), axis=0) <= tol(1e-9, e))
    ez = e[:, 0] + 1j * e[:, 1]
    cz, _ = _adjoint(1, r, omega, ez, 1e-9)
    assert np.max(np.abs(cz - oracle.direct(1, omega, r, ez))) <= 10 * 1e-9 * np.abs(ez).sum()


def test_batched_adjoint():
    from paper_2411_09583_gb300 import Plan
    from paper_2411_09583_gb300.workloads import batch_problems
    probs = batch_problems(count=10, lo=100, hi=2000, nu_max=20, seed=76)
    nus = [p[0] for p in probs]
    n = [p[1].size for p in probs]
    m = [p[2].size for p in probs]
    es = [np.random.default_rng(77 + i).standard_normal(mi) for i, mi in enumerate(m)]
    with Plan.many(nus, to_dev(np.concatenate([p[1] for p in probs])), n,
                   to_dev(np.concatenate([p[2] for p in probs])), m, 1e-8) as bp:
        ca = bp.adjoint(to_dev(np.concatenate(es))).cpu().numpy()
    off = 0
    for (nu, rr, ww, _), e in zip(probs, es):
        ref = oracle.direct(nu, ww, rr, e)
        assert np.max(np.abs(ca[off:off + rr.size] - ref)) <= tol(1e-8, e)
        off += rr.size


def test_full_size_adjoint_sampled():
    eps = 1e-12
    r, omega, _ = uniform_problem(1_000_000, 1_000_000, omega_max=1e5, seed=6)
    e = np.random.default_rng(78).standard_normal(omega.size)
    ca, _ = _adjoint(0, r, omega, e, eps)
    rows = sample_rows(r.size, 100, seed=79)
    ref = oracle.direct_rows(0, omega, r, e, rows)
    assert np.max(np.abs(ca[rows] - ref)) <= tol(eps, e)


@pytest.mark.parametrize("nu", [0, 2])
def test_autograd_gradients_match_oracle(nu):
    # loss 1/2 ||g - g*||^2 with g* from a perturbed c (n = m = 2000), eps = 1e-10
    from paper_2411_09583_gb300 import nuht_autograd
    eps = 1e-10
    r, omega, c = uniform_problem(2000, 2000, omega_max=3000.0, seed=7 + nu)
    rng = np.random.default_rng(80)
    gstar = oracle.direct(nu, r, omega, c + 0.01 * rng.standard_normal(c.size))
    L, dc, dr, dw = OG.gradients(nu, r, omega, c, gstar)
    tc = to_dev(c).requires_grad_(True)
    tr = to_dev(r).requires_grad_(True)
    tw = to_dev(omega).requires_grad_(True)
    g = nuht_autograd(tc, tr, tw, nu, eps)
    loss = 0.5 * ((g - to_dev(gstar)) ** 2).sum()
    loss.backward()
    e = oracle.direct(nu, r, omega, c) - gstar
    assert abs(loss.item() - L) <= 1e-6 * L
    # first-order error bounds: the transforms in the gradient are accurate to
    # 10 eps ||input||_1, and e itself carries the forward error 10 eps ||c||_1
    de = 10 * eps * np.abs(c).sum()
    assert np.max(np.abs(tc.grad.cpu().numpy() - dc)) <= 10 * eps * np.abs(e).sum() + de * omega.size
    bound_r = np.abs(c) * (10 * eps * np.abs(omega * e).sum() + de * np.abs(omega).sum())
    assert np.all(np.abs(tr.grad.cpu().numpy() - dr) <= bound_r + 1e-12)
    bound_w = np.abs(r * c).sum() * (10 * eps * np.abs(e) + de)
    assert np.all(np.abs(tw.grad.cpu().numpy() - dw) <= bound_w + 1e-12)


def test_autograd_finite_differences():
    # central differences of the GPU loss itself in a few coordinates of c and r
    from paper_2411_09583_gb300 import nuht_autograd
    eps = 1e-12
    r, omega, c = uniform_problem(400, 300, omega_max=800.0, seed=81)
    gstar = to_dev(np.random.default_rng(82).standard_normal(omega.size))

    def loss_of(cc, rr):
        g = nuht_autograd(cc, rr, to_dev(omega), 0, eps)
        return 0.5 * ((g - gstar) ** 2).sum()

    tc = to_dev(c).requires_grad_(True)
    tr = to_dev(r).requires_grad_(True)
    loss_of(tc, tr).backward()
    h = 1e-6
    for j in (3, 150, 399):
        for which in ("c", "r"):
            base_c, base_r = to_dev(c), to_dev(r)
            dp = torch.zeros_like(base_c)
            dp[j] = h
            if which == "c":
                lp, lm = loss_of(base_c + dp, base_r).item(), loss_of(base_c - dp, base_r).item()
                grad = tc.grad[j].item()
            else:
                lp, lm = loss_of(base_c, base_r + dp).item(), loss_of(base_c, base_r - dp).item()
                grad = tr.grad[j].item()
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grad) <= 1e-5 * max(1.0, abs(grad)), (which, j, fd, grad)


@pytest.mark.parametrize("layout", ["frequencies", "narrow", "points"])
@pytest.mark.parametrize("nu", [0, 3])
def test_dense_bins_both_directions(layout, nu):
    # One asymptotic region (omega r >= 1000 > z) with a small product of the
    # r and omega ranges, so its FFT grid is short: 20000 frequencies (or
    # points) fall in a few dozen cells, and the tiles take the per-bin moment
    # paths (adjoint spreading of frequencies, adjoint interpolation at points,
    # and their forward counterparts).  "narrow" (r range 1e-3) puts all
    # frequencies in one or two FFT cells wider than the omega range.
    rng = np.random.default_rng(95 + nu)
    if layout == "frequencies":
        r, omega = rng.uniform(1.0, 2.0, 2000), rng.uniform(1000.0, 1010.0, 20000)
    elif layout == "narrow":
        r, omega = rng.uniform(1.0, 1.001, 2000), rng.uniform(1000.0, 1010.0, 20000)
    else:
        r, omega = rng.uniform(1.0, 1.01, 20000), rng.uniform(1000.0, 2000.0, 2000)
    c = rng.standard_normal(r.size)
    e = rng.standard_normal(omega.size)
    eps = 1e-10
    from paper_2411_09583_gb300 import Plan
    with Plan(nu, to_dev(r), to_dev(omega), eps) as p:
        info = p.info()
        assert info["n_asy"] > 0
        # at least 20 packed targets per FFT point: the moment paths' tiles
        # need 16 per cell
        assert max(r.size, omega.size) >= 20 * info["fft_points"]
        g = p.execute(to_dev(c)).cpu().numpy()
        ca = p.adjoint(to_dev(e)).cpu().numpy()
    assert np.max(np.abs(g - oracle.direct(nu, r, omega, c))) <= tol(eps, c)
    assert np.max(np.abs(ca - oracle.direct(nu, omega, r, e))) <= tol(eps, e)


@pytest.mark.parametrize("nu", [0, 3, 100])
@pytest.mark.parametrize("precision,eps", [("fp64", 1e-10), ("mixed", 1e-6)])
def test_three_vectors_pair_and_single(precision, eps, nu):
    # three real vectors: the first two share the local and direct blocks'
    # Bessel values, the third runs alone; both directions against the oracle.
    # Orders 3 and 100 take the general C_l products (odd order, and the
    # largest Bessel index and shared-memory columns).
    from paper_2411_09583_gb300 import Plan
    r, omega, _ = uniform_problem(2500, 2300, omega_max=3000.0, seed=78)
    rng = np.random.default_rng(79)
    c = rng.standard_normal((r.size, 3))
    e = rng.standard_normal((omega.size, 3))
    with Plan(nu, to_dev(r), to_dev(omega), eps, precision=precision) as p:
        assert p.info()["n_local"] > 0
        g = p.execute(to_dev(c)).cpu().numpy()
        ca = p.adjoint(to_dev(e)).cpu().numpy()
    rows = np.arange(0, omega.size, 5)
    cols = np.arange(0, r.size, 5)
    for v in range(3):
        cv, ev = np.ascontiguousarray(c[:, v]), np.ascontiguousarray(e[:, v])
        assert np.max(np.abs(g[rows, v] - oracle.direct_rows(nu, r, omega, cv, rows))) <= tol(eps, cv)
        assert np.max(np.abs(ca[cols, v] - oracle.direct_rows(nu, omega, r, ev, cols))) <= tol(eps, ev)


def _deriv_oracle(nu, r, omega, c, e):
    """(grad_r, grad_omega) of sum_k e_k g_k by the oracle's direct sums of
    orders nu - 1 and nu + 1 (J_nu' = (J_{nu-1} - J_{nu+1}) / 2); c, e (n, v), (m, v)."""
    c2, e2 = c.reshape(r.size, -1), e.reshape(omega.size, -1)
    gr = np.zeros(r.size)
    gw = np.zeros(omega.size)
    for v in range(c2.shape[1]):
        we, rc = omega * e2[:, v], r * c2[:, v]
        gr += c2[:, v] * 0.5 * (oracle.direct(nu - 1, omega, r, we) - oracle.direct(nu + 1, omega, r, we))
        gw += e2[:, v] * 0.5 * (oracle.direct(nu - 1, r, omega, rc) - oracle.direct(nu + 1, r, omega, rc))
    return gr, gw


@pytest.mark.parametrize("nu,nvec,det", [(0, 1, False), (1, 1, False), (-3, 1, False), (7, 3, False),
                                         (20, 1, False), (2, 2, True)])
def test_derivative_plan_gradients(nu, nvec, det):
    # nuht_plan_deriv + nuht_grad_r / nuht_grad_omega against the oracle, per
    # entry within 10 eps |c_j| ||omega e||_1 (r) and 10 eps |e_k| ||r c||_1
    # (omega), summed over the vectors
    from paper_2411_09583_gb300 import Plan
    eps = 1e-10
    r, omega, _ = uniform_problem(1800, 1600, omega_max=2500.0, seed=820 + abs(nu))
    rng = np.random.default_rng(821)
    shape_c = (r.size,) if nvec == 1 else (r.size, nvec)
    shape_e = (omega.size,) if nvec == 1 else (omega.size, nvec)
    c, e = rng.standard_normal(shape_c), rng.standard_normal(shape_e)
    with Plan(nu, to_dev(r), to_dev(omega), eps, deterministic=det) as p:
        with p.deriv() as d:
            assert d.n == r.size and d.m == omega.size
            gr = d.grad_r(to_dev(c), to_dev(e)).cpu().numpy()
            gw = d.grad_omega(to_dev(c), to_dev(e)).cpu().numpy()
            if det:
                assert np.array_equal(gr, d.grad_r(to_dev(c), to_dev(e)).cpu().numpy())
    ref_r, ref_w = _deriv_oracle(nu, r, omega, c, e)
    c2, e2 = c.reshape(r.size, -1), e.reshape(omega.size, -1)
    bound_r = sum(10 * eps * np.abs(c2[:, v]) * np.abs(omega * e2[:, v]).sum() for v in range(nvec))
    bound_w = sum(10 * eps * np.abs(e2[:, v]) * np.abs(r * c2[:, v]).sum() for v in range(nvec))
    assert np.all(np.abs(gr - ref_r) <= bound_r + 1e-300)
    assert np.all(np.abs(gw - ref_w) <= bound_w + 1e-300)


def test_derivative_plan_outlives_base_and_rejects_misuse():
    import ctypes
    from paper_2411_09583_gb300 import Plan
    from paper_2411_09583_gb300 import _native as N
    eps = 1e-9
    r, omega, c = uniform_problem(700, 900, omega_max=1500.0, seed=830)
    e = np.random.default_rng(831).standard_normal(omega.size)
    p = Plan(4, to_dev(r), to_dev(omega), eps)
    d = p.deriv()
    lib = N.lib()
    # a derivative plan is not an ordinary plan
    out = to_dev(np.zeros(omega.size))
    assert lib.nuht_execute(d._h, ctypes.c_void_p(to_dev(c).data_ptr()), ctypes.c_void_p(out.data_ptr()),
                            1, 0, None) == N.NUHT_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert lib.nuht_plan_deriv(ctypes.byref(h), d._h, None) == N.NUHT_ERR_INVALID_ARG
    assert lib.nuht_grad_r(p._h, None, None, None, 1, None) == N.NUHT_ERR_INVALID_ARG
    p.close()                          # the derivative plan keeps its own copies
    gr = d.grad_r(to_dev(c), to_dev(e)).cpu().numpy()
    d.close()
    ref_r, _ = _deriv_oracle(4, r, omega, c, e)
    assert np.all(np.abs(gr - ref_r) <= 10 * eps * np.abs(c) * np.abs(omega * e).sum() + 1e-300)
    with Plan(100, to_dev(r), to_dev(omega), 1e-8) as p100:
        assert lib.nuht_plan_deriv(ctypes.byref(h), p100._h, None) == N.NUHT_ERR_UNSUPPORTED
    with Plan.many([0, 1], to_dev(np.concatenate([r, r])), [r.size, r.size],
                   to_dev(np.concatenate([omega, omega])), [omega.size, omega.size], 1e-8) as bp:
        assert lib.nuht_plan_deriv(ctypes.byref(h), bp._h, None) == N.NUHT_ERR_INVALID_ARG


def test_full_size_gradients_sampled():
    # n = m = 1e6, nu = 0, eps = 1e-10 (the differentiation workload): both
    # gradients on 100 sampled entries against the oracle
    from paper_2411_09583_gb300 import Plan
    eps = 1e-10
    r, omega, c = uniform_problem(1_000_000, 1_000_000, omega_max=1e5, seed=6)
    e = np.random.default_rng(7).standard_normal(omega.size)
    with Plan(0, to_dev(r), to_dev(omega), eps) as p, p.deriv() as d:
        gr = d.grad_r(to_dev(c), to_dev(e)).cpu().numpy()
        gw = d.grad_omega(to_dev(c), to_dev(e)).cpu().numpy()
    cols = sample_rows(r.size, 100, seed=832)
    rows = sample_rows(omega.size, 100, seed=833)
    we, rc = omega * e, r * c
    ref_r = c[cols] * 0.5 * (oracle.direct_rows(-1, omega, r, we, cols) - oracle.direct_rows(1, omega, r, we, cols))
    ref_w = e[rows] * 0.5 * (oracle.direct_rows(-1, r, omega, rc, rows) - oracle.direct_rows(1, r, omega, rc, rows))
    assert np.all(np.abs(gr[cols] - ref_r) <= 10 * eps * np.abs(c[cols]) * np.abs(we).sum())
    assert np.all(np.abs(gw[rows] - ref_w) <= 10 * eps * np.abs(e[rows]) * np.abs(rc).sum())
