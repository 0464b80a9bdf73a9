"""Shared helpers of the GPU parity tests (call the library through the binding)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402


def dev():
    return torch.device("cuda:0")


def to_dev(x):
    return torch.tensor(np.asarray(x), device=dev())


def run_forward(nu, r, omega, c, eps, **opts):
    from paper_2411_09583_gb300 import Plan
    with Plan(nu, to_dev(r), to_dev(omega), eps, **opts) as p:
        g = p.execute(to_dev(c)).cpu().numpy()
        info = p.info()
        blocks = [p.blocks(k) for k in range(3)]
    return g, info, blocks


def tol(eps, c):
    """Accuracy contract: max_k |g_k - g_k^exact| <= 10 eps ||c||_1 (per vector)."""
    return 10.0 * eps * np.abs(np.asarray(c)).sum(axis=0)


def class_reference(nu, r, omega, c, blocks):
    """Oracle sum restricted to the entries of the given blocks (sorted indices)."""
    ir = np.argsort(r, kind="stable")
    iw = np.argsort(omega, kind="stable")
    rs, ws, cs = r[ir], omega[iw], np.asarray(c)[ir]
    gs = np.zeros(len(omega), dtype=np.result_type(cs, np.float64))
    for k0, k1, j0, j1 in blocks:
        gs[k0:k1 + 1] += oracle.direct(nu, rs[j0:j1 + 1], ws[k0:k1 + 1], cs[j0:j1 + 1])
    g = np.zeros_like(gs)
    g[iw] = gs
    return g
