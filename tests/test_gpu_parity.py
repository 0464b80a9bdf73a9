"""GPU parity: the CUDA NUHT against the oracle's direct sum.

Bar: max_k |g_k - g_k^oracle| <= 10 eps ||c||_1 (the accuracy contract), on
seeded synthetic inputs shaped like the paper's experiments.
"""
import numpy as np
import pytest

import oracle
from oracle import subdivide as OS
from paper_2411_09583_gb300.workloads import (exponential_grid, fourier_bessel_grid, loguniform_problem,
                                              sample_rows, sparse_coefficients,
                                              uniform_problem)

pytestmark = pytest.mark.gpu

from gpu_helpers import class_reference, dev, run_forward, to_dev, tol  # noqa: E402


def _check(nu, r, omega, c, eps, **opts):
    g, info, blocks = run_forward(nu, r, omega, c, eps, **opts)
    ref = oracle.direct(nu, r, omega, c)
    err = np.max(np.abs(g - ref), axis=0) if g.size else 0.0
    assert np.all(err <= tol(eps, c)), (err, tol(eps, c), info)
    return g, info, blocks, err


def test_small_uniform_config():
    # n = m = 2000, nu = 0, eps = 1e-8, r ~ U[0,1], omega ~ U[0,2000] (seed 1)
    r, omega, c = uniform_problem(2000, 2000, omega_max=2000.0, seed=1)
    g, info, blocks, err = _check(0, r, omega, c, 1e-8)
    assert info["n_local"] > 0 and info["n_asy"] > 0 and info["n_direct"] > 0
    # far inside the contract in practice
    assert err <= 1e-2 * tol(1e-8, c)


@pytest.mark.parametrize("cls", [0, 1, 2])
def test_each_block_class_alone(cls):
    r, omega, c = uniform_problem(1500, 1700, omega_max=3000.0, seed=21)
    eps = 1e-10
    g, info, blocks = run_forward(0, r, omega, c, eps, class_mask=1 << cls)
    ref = class_reference(0, r, omega, c, blocks[cls])
    assert np.max(np.abs(g - ref)) <= tol(eps, c)


@pytest.mark.parametrize("nu", [0, 1, 2, 3, 4, 7, 10, 15, 20])
def test_orders(nu):
    r, omega, c = uniform_problem(1300, 1100, omega_max=1500.0 + 40 * nu, seed=100 + nu)
    _check(nu, r, omega, c, 1e-10)


@pytest.mark.parametrize("nu,eps,opts", [(50, 1e-8, {}), (100, 1e-6, {}), (100, 1e-12, {}), (0, 1e-10, {"m_terms": 20}),
                                         (3, 1e-2, {}), (0, 1e-3, {}), (20, 1e-14, {})])
def test_extreme_orders_terms_and_tolerances(nu, eps, opts):
    """Orders up to the supported 100, the largest number of Hankel terms
    (2M = 40), and the loosest / tightest tolerances."""
    r, omega, c = uniform_problem(1100, 1000, omega_max=3000.0 + 30 * nu, seed=300 + nu)
    _check(nu, r, omega, c, eps, **opts)


@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-9, 1e-12, 1e-14])
def test_tolerances(eps):
    r, omega, c = uniform_problem(1200, 1250, omega_max=2500.0, seed=7)
    for nu in (0, 5):
        _check(nu, r, omega, c, eps)


def test_negative_order():
    r, omega, c = uniform_problem(700, 600, omega_max=900.0, seed=8)
    g3, _, _ = run_forward(3, r, omega, c, 1e-10)
    gm3, _, _ = run_forward(-3, r, omega, c, 1e-10)
    assert np.max(np.abs(gm3 + g3)) <= 1e-13 * np.abs(c).sum()


def test_clustered_and_exponential_points():
    r, omega, c = loguniform_problem(1500, 1400, omega_max=4e4, seed=4, complex_c=False)
    _check(1, r, omega, c, 1e-10)
    v, _ = exponential_grid(1500)
    c = np.random.default_rng(3).standard_normal(1500)
    _check(0, v, v * 40.0, c, 1e-8)


@pytest.mark.parametrize("ties", [False, True])
def test_block_lists_match_oracle_subdivision(ties):
    # m = 2300 rows: the staircase's per-CTA ranges (1024 rows) with a ragged
    # tail; "ties" repeats frequencies and points and puts zeros among them
    r, omega, c = uniform_problem(2500, 2300, omega_max=3000.0, seed=11)
    if ties:
        r, omega = np.round(r, 3), np.round(omega, -1)
        omega[::7] = 0.0
    g, info, blocks = run_forward(2, r, omega, c, 1e-9)
    rs, ws = np.sort(r), np.sort(omega)
    Lb, Ab, Db = OS.subdivide(list(rs), list(ws), info["z"], 1024, 16)
    for mine, ref in zip(blocks, (Lb, Ab, Db)):
        assert [tuple(b) for b in mine.tolist()] == [tuple(b) for b in ref]


def test_permutations_are_stable_sorts():
    from paper_2411_09583_gb300 import Plan
    rng = np.random.default_rng(12)
    r = np.round(rng.uniform(0, 1, 3000), 2)          # many ties
    omega = rng.uniform(0, 500, 2000)
    omega[::7] = 0.0
    with Plan(0, to_dev(r), to_dev(omega), 1e-8) as p:
        pr, pw = p.permutations()
    assert np.array_equal(pr, np.argsort(r, kind="stable"))
    assert np.array_equal(pw, np.argsort(omega, kind="stable"))


def test_complex_and_multiple_vectors():
    r, omega, c = uniform_problem(900, 800, omega_max=1200.0, seed=13, nvec=3)
    g, info, _ = run_forward(1, r, omega, c, 1e-9)
    ref = oracle.direct(1, r, omega, c)
    assert np.all(np.max(np.abs(g - ref), axis=0) <= tol(1e-9, c))
    cz = c[:, 0] + 1j * c[:, 1]
    gz, _, _ = run_forward(1, r, omega, cz, 1e-9)
    refz = oracle.direct(1, r, omega, cz)
    assert np.max(np.abs(gz - refz)) <= 10 * 1e-9 * np.abs(cz).sum()


@pytest.mark.parametrize("nvec", [1, 2])
def test_host_buffer_entry_point(nvec):
    # nuht_transform_host: host arrays in and out
    from paper_2411_09583_gb300.nuht import transform_host
    r, omega, c = uniform_problem(2000, 1800, omega_max=2500.0, seed=44, nvec=nvec)
    eps = 1e-10
    g = transform_host(0, r, omega, c, eps)
    ref = oracle.direct(0, r, omega, c)
    assert g.shape == ref.shape
    assert np.all(np.max(np.abs(g - ref), axis=0) <= tol(eps, c))
    # pinned output buffer, repeated calls
    import torch
    out = torch.empty(g.shape, dtype=torch.float64).pin_memory().numpy()
    for _ in range(2):
        g2 = transform_host(0, r, omega, c, eps, out=out)
        assert np.max(np.abs(g2 - g)) <= 1e-12 * np.abs(c).sum()


def test_edge_cases():
    rng = np.random.default_rng(14)
    # empty sides
    g, _, _ = run_forward(0, np.zeros(0), rng.uniform(0, 10, 5), np.zeros(0), 1e-8)
    assert g.shape == (5,) and np.all(g == 0)
    g, _, _ = run_forward(0, rng.uniform(0, 1, 5), np.zeros(0), rng.standard_normal(5), 1e-8)
    assert g.shape == (0,)
    # single point / frequency, zeros, duplicates
    for (n, m) in [(1, 1), (1, 300), (300, 1), (33, 47)]:
        r = rng.uniform(0, 1, n)
        omega = rng.uniform(0, 3000, m)
        c = rng.standard_normal(n)
        _check(2, r, omega, c, 1e-9)
    r = np.zeros(50)
    c = rng.standard_normal(50)
    g, _, _ = run_forward(0, r, rng.uniform(0, 100, 40), c, 1e-10)
    assert np.max(np.abs(g - c.sum())) <= 1e-12 * np.abs(c).sum()
    g, _, _ = run_forward(4, r, rng.uniform(0, 100, 40), c, 1e-10)
    assert np.max(np.abs(g)) <= 1e-12 * np.abs(c).sum()
    r = np.repeat(rng.uniform(0, 1, 20), 30)
    omega = np.concatenate([np.zeros(10), np.repeat(rng.uniform(0, 5000, 25), 20)])
    c = rng.standard_normal(r.size)
    _check(1, r, omega, c, 1e-9)


def test_invalid_inputs_rejected():
    from paper_2411_09583_gb300 import Plan
    from paper_2411_09583_gb300._native import NUHT_ERR_DOMAIN, NuhtError
    r = np.array([0.1, -0.2, 0.3])
    with pytest.raises(NuhtError) as e:
        Plan(0, to_dev(r), to_dev(np.ones(3)), 1e-8)
    assert e.value.code == NUHT_ERR_DOMAIN
    with pytest.raises(NuhtError):
        Plan(0, to_dev(np.ones(3)), to_dev(np.array([1.0, np.nan])), 1e-8)
    with pytest.raises(NuhtError):
        Plan(0, to_dev(np.ones(3)), to_dev(np.array([1.0, np.inf])), 1e-8)


@pytest.mark.parametrize("nu", [0, 2, 5])
def test_gaussian_pair_end_to_end(nu):
    # int_0^inf exp(-r^2/2) J_nu(w r) r^(nu+1) dr = w^nu exp(-w^2/2), Gauss-Legendre on [0, 12]
    x, wq = np.polynomial.legendre.leggauss(400)
    r = 6.0 * (x + 1.0)
    c = 6.0 * wq * r ** (nu + 1) * np.exp(-0.5 * r * r)
    omega = np.linspace(0.0, 6.0, 301)
    g, _, _ = run_forward(nu, r, omega, c, 1e-12)
    assert np.max(np.abs(g - omega ** nu * np.exp(-0.5 * omega ** 2))) < 1e-11


def test_unit_disk_end_to_end():
    # Sec. 5.2: int_0^1 J_0(w r) r dr = J_1(w)/w
    x, wq = np.polynomial.legendre.leggauss(2000)
    r = 0.5 * (x + 1.0)
    c = 0.5 * wq * r
    omega = np.linspace(1.0, 1500.0, 700)
    g, _, _ = run_forward(0, r, omega, c, 1e-12)
    ref = oracle.jn(1, omega) / omega
    assert np.max(np.abs(g - ref)) < 1e-11


def test_linearity_and_input_permutation():
    r, omega, c = uniform_problem(1000, 900, omega_max=2000.0, seed=15)
    d = np.random.default_rng(16).standard_normal(1000)
    g1, _, _ = run_forward(0, r, omega, c, 1e-10)
    g2, _, _ = run_forward(0, r, omega, d, 1e-10)
    g3, _, _ = run_forward(0, r, omega, 2 * c - 3 * d, 1e-10)
    assert np.max(np.abs(g3 - (2 * g1 - 3 * g2))) <= 1e-12 * np.abs(c).sum() * 5
    p = np.random.default_rng(17).permutation(1000)
    g4, _, _ = run_forward(0, r[p], omega, c[p], 1e-10)
    assert np.max(np.abs(g4 - g1)) <= 1e-12 * np.abs(c).sum()


@pytest.mark.parametrize("nu", [0, 10])
def test_full_size_sampled_rows(nu):
    # n = m = 1e6, r ~ U[0,1], omega ~ U[0,1e5], eps = 1e-12: sampled outputs vs the oracle
    eps = 1e-12
    r, omega, c = uniform_problem(1_000_000, 1_000_000, omega_max=1e5, seed=2 if nu == 0 else 3)
    g, info, _ = run_forward(nu, r, omega, c, eps)
    rows = sample_rows(omega.size, 200, seed=99)
    ref = oracle.direct_rows(nu, r, omega, c, rows)
    err = np.max(np.abs(g[rows] - ref))
    assert err <= tol(eps, c), (err, tol(eps, c))


@pytest.mark.parametrize("nu", [0, 3])
def test_relative_l2_error_tracks_eps(nu):
    # Sec. 5.1.3 measures the relative 2-norm error against eps; it follows eps
    # down to 1e-12 here.  The double-float (~48-bit) loops put a floor near
    # 1e-13 under it, so at eps = 1e-14 the bound is that floor (the accuracy
    # contract 10 eps ||c||_1 still holds there, see test_tolerances).
    r, omega, c = uniform_problem(1000, 1000, omega_max=3000.0, seed=31 + nu)
    ref = oracle.direct(nu, r, omega, c)
    for eps in (1e-6, 1e-9, 1e-12, 1e-14):
        g, _, _ = run_forward(nu, r, omega, c, eps)
        rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
        assert rel <= max(10 * eps, 3e-13), (eps, rel)


@pytest.mark.parametrize("scale_r,scale_w", [(1e4, 1e-4), (1e-5, 1e5), (3e7, 3e-7), (1e-9, 1e9)])
def test_scaled_inputs(scale_r, scale_w):
    # J_nu(omega r) depends on omega r only: the same matrix with r scaled up
    # and omega down (or the reverse) exercises the fixed-point frames of the
    # blocks (bit positions set by each block's largest r and omega) far from
    # unit scale; the oracle sees the same scaled inputs
    r, omega, c = uniform_problem(1500, 1400, omega_max=3000.0, seed=80)
    _check(0, r * scale_r, omega * scale_w, c, 1e-10)


def test_wide_dynamic_range():
    # r log-uniform over 11 decades, omega over 8: blocks whose points (or
    # frequencies) span many binary orders of magnitude
    rng = np.random.default_rng(81)
    r = 10.0 ** rng.uniform(-8, 3, 1600)
    omega = 10.0 ** rng.uniform(-3, 5, 1500)
    c = rng.standard_normal(1600)
    for nu, eps in ((0, 1e-9), (5, 1e-12)):
        _check(nu, r, omega, c, eps)


@pytest.mark.parametrize("nu,eps", [(0, 1e-8), (3, 1e-12), (10, 1e-10)])
def test_fourier_bessel_grid(nu, eps):
    # Sec. 5.1.1's Fourier-Bessel case (n = m): frequencies at the roots of
    # J_nu, points at the roots scaled by the (n+1)-th
    r, omega = fourier_bessel_grid(nu, 2000)
    c = np.random.default_rng(40 + nu).standard_normal(r.size)
    _check(nu, r, omega, c, eps)


@pytest.mark.parametrize("n", [1000, 100000])
def test_sparse_input_relative_error(n):
    # Sec. 5.1.3's accuracy experiment: nu = 0 on the Fourier-Bessel grid with
    # 1000 nonzero Gaussian coefficients; the NUHT of the full c against the
    # direct sum over the nonzeros only, as relative 2-norm error.  It follows
    # eps down to a floor: that of the double-float loops (~1e-13) at n = 1e3,
    # and at larger n the saturation the paper reports, error ~ n times the
    # FP64 rounding unit (the arguments omega_k r_j reach ~ n pi, rounded
    # differently by the oracle and the transform); measured 4.8e-12 at n = 1e5
    r, omega = fourier_bessel_grid(0, n)
    c, idx = sparse_coefficients(n, 1000, seed=41)
    ref = oracle.direct(0, r[idx], omega, c[idx])
    floor = max(3e-13, n * 2.0 ** -53)
    rels = {}
    for eps in (1e-4, 1e-6, 1e-8, 1e-10, 1e-12, 1e-14):
        g, _, _ = run_forward(0, r, omega, c, eps)
        rels[eps] = float(np.linalg.norm(g - ref) / np.linalg.norm(ref))
    bad = {eps: rel for eps, rel in rels.items() if not rel <= max(10 * eps, floor)}
    assert not bad, ("failing", bad, "all", sorted(rels.items()))


def _batch(count, lo, hi, nu_max, seed):
    from paper_2411_09583_gb300.workloads import batch_problems
    return batch_problems(count=count, lo=lo, hi=hi, nu_max=nu_max, seed=seed)


def test_batched_plan_matches_oracle_and_single_plans():
    # uneven problems (sizes log-uniform, orders 0..20) in one plan, one launch per stage
    from paper_2411_09583_gb300 import Plan
    eps = 1e-8
    probs = _batch(24, 50, 3000, 20, 41)
    nus = [p[0] for p in probs]
    r = np.concatenate([p[1] for p in probs])
    omega = np.concatenate([p[2] for p in probs])
    c = np.concatenate([p[3] for p in probs])
    n = [p[1].size for p in probs]
    m = [p[2].size for p in probs]
    with Plan.many(nus, to_dev(r), n, to_dev(omega), m, eps) as bp:
        g = bp.execute(to_dev(c)).cpu().numpy()
        nblk = sum(len(bp.blocks(k)) for k in range(3))
    ro = np.concatenate([[0], np.cumsum(n)])
    wo = np.concatenate([[0], np.cumsum(m)])
    total_blocks = 0
    for i, (nu, rr, ww, cc) in enumerate(probs):
        gi = g[wo[i]:wo[i + 1]]
        ref = oracle.direct(nu, rr, ww, cc)
        assert np.max(np.abs(gi - ref)) <= tol(eps, cc), i
        gs, info, blocks = run_forward(nu, rr, ww, cc, eps)
        assert np.max(np.abs(gi - gs)) <= 1e-3 * tol(eps, cc)
        total_blocks += sum(len(b) for b in blocks)
    assert nblk == total_blocks


def test_batched_edge_problems():
    from paper_2411_09583_gb300 import Plan
    rng = np.random.default_rng(43)
    sizes = [(0, 5), (7, 0), (1, 1), (300, 200), (0, 0), (50, 60)]
    nus = [0, 3, 1, 2, 0, 20]
    rs = [rng.uniform(0, 1, a) for a, _ in sizes]
    ws = [rng.uniform(0, 500, b) for _, b in sizes]
    cs = [rng.standard_normal(a) for a, _ in sizes]
    with Plan.many(nus, to_dev(np.concatenate(rs)), [a for a, _ in sizes],
                   to_dev(np.concatenate(ws)), [b for _, b in sizes], 1e-9) as bp:
        g = bp.execute(to_dev(np.concatenate(cs))).cpu().numpy()
    off = 0
    for nu, rr, ww, cc in zip(nus, rs, ws, cs):
        gi = g[off:off + ww.size]
        off += ww.size
        ref = oracle.direct(nu, rr, ww, cc) if rr.size else np.zeros(ww.size)
        assert np.max(np.abs(gi - ref), initial=0.0) <= 10 * 1e-9 * max(np.abs(cc).sum(), 1e-300)


@pytest.mark.parametrize("nu", [0, 1, 4, 20])
def test_mixed_precision_small(nu):
    # FP32 spreading / interpolation at eps = 1e-5 (and 1e-6) against the FP64 oracle
    r, omega, c = loguniform_problem(3000, 2500, omega_max=4e4, seed=50 + nu, complex_c=True)
    ref = oracle.direct(nu, r, omega, c)
    for eps in (1e-5, 1e-6):
        g, info, _ = run_forward(nu, r, omega, c, eps, precision="mixed")
        err = np.max(np.abs(g - ref))
        assert err <= 10 * eps * np.abs(c).sum(), (eps, err)
        rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
        assert rel <= 10 * eps, (eps, rel)


@pytest.mark.parametrize("cls", [0, 1, 2])
@pytest.mark.parametrize("eps,min_size", [(1e-6, 1024), (1e-5, 4096)])
def test_mixed_precision_each_class_alone(cls, eps, min_size):
    # one block class at a time in mixed precision: FP32 local evaluation,
    # FP32 direct entries and (where the rounding bound allows) FP32 row sums,
    # FP32 spreading, FFT butterflies and interpolation
    r, omega, c = loguniform_problem(3000, 2500, omega_max=4e4, seed=58, complex_c=False)
    g, info, blocks = run_forward(1, r, omega, c, eps, precision="mixed", class_mask=1 << cls,
                                  min_size=min_size)
    assert len(blocks[cls]) > 0
    ref = class_reference(1, r, omega, c, blocks[cls])
    assert np.max(np.abs(g - ref)) <= tol(eps, c)


def test_mixed_precision_rejects_tight_eps():
    from paper_2411_09583_gb300 import Plan
    from paper_2411_09583_gb300._native import NUHT_ERR_UNSUPPORTED, NuhtError
    with pytest.raises(NuhtError) as e:
        Plan(0, to_dev(np.ones(4)), to_dev(np.ones(4)), 1e-9, precision="mixed")
    assert e.value.code == NUHT_ERR_UNSUPPORTED


def test_mixed_precision_full_size_sampled():
    # n = m = 4e6, nu = 1, r log-uniform on [1e-3, 1], omega ~ U[0, 4e4], complex c, eps = 1e-5
    eps = 1e-5
    r, omega, c = loguniform_problem(4_000_000, 4_000_000, omega_max=4e4, seed=4, complex_c=True)
    g, info, _ = run_forward(1, r, omega, c, eps, precision="mixed")
    rows = sample_rows(omega.size, 100, seed=98)
    ref = oracle.direct_rows(1, r, omega, c, rows)
    err = np.max(np.abs(g[rows] - ref))
    assert err <= 10 * eps * np.abs(c).sum(), err


def test_autotuner_picks_valid_fast_options():
    from paper_2411_09583_gb300.autotune import autotune, candidates
    r, omega, c = uniform_problem(20000, 20000, omega_max=5000.0, seed=90)
    grid = candidates([0], 1e-10, min_sizes=(512, 2048), spread_tiles=(0, 128), m_offsets=(0, 1))
    best, table = autotune(0, to_dev(r), to_dev(omega), to_dev(c), 1e-10, grid=grid, reps=2)
    assert len(table) == len(grid) and table[0][0] <= table[-1][0]
    g, _, _ = run_forward(0, r, omega, c, 1e-10, **best)
    rows = np.arange(0, omega.size, 97)
    ref = oracle.direct_rows(0, r, omega, c, rows)
    assert np.max(np.abs(g[rows] - ref)) <= tol(1e-10, c)


@pytest.mark.parametrize("opts", [{"min_size": 64}, {"min_size": 5000}, {"m_terms": 2},
                                  {"m_terms": 7}, {"spread_tile": 64}, {"n_split_cand": 3},
                                  {"interp_tile": 128}, {"interp_tile": 256}])
def test_option_variants_keep_accuracy(opts):
    r, omega, c = uniform_problem(1500, 1400, omega_max=2500.0, seed=91)
    _check(1, r, omega, c, 1e-10, **opts)


@pytest.mark.parametrize("interp_tile", [128, 256])
def test_interp_tile_both_directions_dense_and_mixed(interp_tile):
    # both interpolation tile sizes on dense bins (the per-bin sums, up to 16
    # bins of a 256-frequency tile) and in mixed precision, forward and adjoint
    from paper_2411_09583_gb300 import Plan
    rng = np.random.default_rng(96)
    r, omega = rng.uniform(1.0, 1.05, 3000), rng.uniform(1000.0, 1200.0, 30000)
    c, e = rng.standard_normal(r.size), rng.standard_normal(omega.size)
    for precision, eps in (("fp64", 1e-11), ("mixed", 1e-6)):
        with Plan(2, to_dev(r), to_dev(omega), eps, precision=precision, interp_tile=interp_tile) as p:
            g = p.execute(to_dev(c)).cpu().numpy()
            a = p.adjoint(to_dev(e)).cpu().numpy() if precision == "fp64" else None
        rows = np.arange(0, omega.size, 37)
        assert np.max(np.abs(g[rows] - oracle.direct_rows(2, r, omega, c, rows))) <= tol(eps, c)
        if a is not None:
            assert np.max(np.abs(a - oracle.direct(2, omega, r, e))) <= tol(eps, e)


def test_host_subdivision_fallback_matches(monkeypatch):
    """Device block lists over capacity: the plan falls back to the host walk
    of Algorithm 1 and builds the same transform."""
    r, omega, c = uniform_problem(2500, 2300, omega_max=3000.0, seed=11)
    g0, info0, b0 = run_forward(2, r, omega, c, 1e-9)
    monkeypatch.setenv("NUHT_SUBDIVIDE_CAPACITY", "16")
    g1, info1, b1 = run_forward(2, r, omega, c, 1e-9)
    for x, y in zip(b0, b1):
        assert sorted(map(tuple, x.tolist())) == sorted(map(tuple, y.tolist()))
    assert max(len(x) for x in b1) > 16          # the fallback was needed
    assert np.max(np.abs(g0 - g1)) <= 1e-12 * np.abs(c).sum()


def test_batched_host_subdivision_fallback_matches(monkeypatch):
    from paper_2411_09583_gb300 import Plan
    from paper_2411_09583_gb300.workloads import batch_problems
    probs = batch_problems(count=5, lo=300, hi=1500, nu_max=4, seed=21)
    nus = [q[0] for q in probs]
    n = [q[1].size for q in probs]
    m = [q[2].size for q in probs]
    dr = to_dev(np.concatenate([q[1] for q in probs]))
    dw = to_dev(np.concatenate([q[2] for q in probs]))
    cc = np.concatenate([q[3] for q in probs])
    with Plan.many(nus, dr, n, dw, m, 1e-8) as p:
        g0 = p.execute(to_dev(cc)).cpu().numpy()
    monkeypatch.setenv("NUHT_SUBDIVIDE_CAPACITY", "8")
    with Plan.many(nus, dr, n, dw, m, 1e-8) as p:
        g1 = p.execute(to_dev(cc)).cpu().numpy()
    assert np.max(np.abs(g0 - g1)) <= 1e-12 * np.abs(cc).sum()


def test_checked_mode_and_plan_lists_pass_the_work_list_check(monkeypatch):
    # NUHT_CHECKED: the plan checks its device-built lists on the host before
    # returning (exact cover, classes, direct areas); a plan's lists, read
    # back with nuht_get_blocks, also pass nuht_check_blocks directly
    from paper_2411_09583_gb300 import Plan
    from paper_2411_09583_gb300 import _native as N
    from paper_2411_09583_gb300.nuht import check_blocks
    r, omega, c = uniform_problem(20000, 15000, omega_max=2e4, seed=92)
    monkeypatch.setenv("NUHT_CHECKED", "1")
    with Plan(3, to_dev(r), to_dev(omega), 1e-9, min_size=512) as p:
        g = p.execute(to_dev(c)).cpu().numpy()
        blocks = [p.blocks(k) for k in range(3)]
    monkeypatch.delenv("NUHT_CHECKED")
    rows = sample_rows(omega.size, 100, seed=93)
    assert np.max(np.abs(g[rows] - oracle.direct_rows(3, r, omega, c, rows))) <= tol(1e-9, c)
    ranges = np.concatenate(blocks)
    cls = np.concatenate([np.full(len(b), k, np.int32) for k, b in enumerate(blocks)])
    rs, ws = np.sort(r), np.sort(omega)
    assert check_blocks(3, 1e-9, rs, ws, ranges, cls, min_size=512) == N.NUHT_OK
    bad = ranges.copy()
    bad[0, 3] += 1
    assert check_blocks(3, 1e-9, rs, ws, bad, cls, min_size=512) == N.NUHT_ERR_BAD_BLOCKS


@pytest.mark.parametrize("nu,min_size", [(0, 256), (7, 1024)])
def test_multi_cta_subdivision_matches_host_walk(monkeypatch, nu, min_size):
    # n = m = 1e6: levels of the subdivision with thousands of mixed blocks,
    # which the device splits over all SMs (cooperative launch); its lists must
    # equal, entry for entry, the host walk's (forced by a tiny device list
    # capacity), and pass the host check
    from paper_2411_09583_gb300 import Plan
    from paper_2411_09583_gb300 import _native as N
    from paper_2411_09583_gb300.nuht import check_blocks
    r, omega, _ = uniform_problem(1_000_000, 1_000_000, omega_max=1e5, seed=94 + nu)
    dr, dw = to_dev(r), to_dev(omega)
    with Plan(nu, dr, dw, 1e-10, min_size=min_size) as p:
        dev_blocks = [p.blocks(k) for k in range(3)]
    monkeypatch.setenv("NUHT_SUBDIVIDE_CAPACITY", "64")
    with Plan(nu, dr, dw, 1e-10, min_size=min_size) as p:
        host_blocks = [p.blocks(k) for k in range(3)]
    monkeypatch.delenv("NUHT_SUBDIVIDE_CAPACITY")
    assert sum(len(b) for b in dev_blocks) > 8000
    for a, b in zip(dev_blocks, host_blocks):
        assert np.array_equal(a, b)
    ranges = np.concatenate(dev_blocks)
    cls = np.concatenate([np.full(len(b), k, np.int32) for k, b in enumerate(dev_blocks)])
    assert check_blocks(nu, 1e-10, np.sort(r), np.sort(omega), ranges, cls, min_size=min_size) == N.NUHT_OK
