"""Autotuner for the plan options of a workload (single problem or batch).

It times plan + execute (or execute alone, for a plan reused many times) over
a small grid of options and keeps the fastest:
  * min_size      -- largest mixed block summed directly (Sec. 4.1): moves work
                     between the direct kernel and deeper subdivision levels;
  * m_terms       -- Hankel terms M around the heuristic of Sec. 3.3: moves the
                     crossover z (and with it L), i.e. work between the local
                     and the asymptotic expansions; z and L are re-derived from
                     the error bounds, so every candidate keeps the accuracy;
  * spread_tile   -- points per spreading CTA;
  * interp_tile   -- frequencies per interpolation CTA.
Every candidate runs the same kernels through the C ABI; nothing is skipped.
"""
import itertools
import statistics

import torch

from .nuht import Plan, choose_params


def _time(fn, stream, reps):
    ms = []
    for _ in range(reps):
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        fn()
        s1.record(stream)
        torch.cuda.synchronize()
        ms.append(s0.elapsed_time(s1))
    return statistics.median(ms)


def candidates(nus, eps, min_sizes=(256, 512, 1024, 2048, 4096), spread_tiles=(0, 128),
               m_offsets=(-1, 0, 1), interp_tiles=(0, 128)):
    """Option grid; m_terms offsets apply to the heuristic M of the first order."""
    M0 = choose_params(int(nus[0]), eps)[0]
    ms = sorted({max(1, min(20, M0 + d)) for d in m_offsets})
    out = []
    for mn, st, M, it in itertools.product(min_sizes, spread_tiles, ms, interp_tiles):
        out.append({"min_size": mn, "spread_tile": st, "m_terms": 0 if M == M0 else M, "interp_tile": it})
    return out


def autotune(nus, r, omega, c, eps, sizes=None, objective="plan+execute", reps=3, grid=None,
             precision="fp64"):
    """Fastest options for the workload.  nus: order (int) or per-problem orders
    (with sizes = (n_list, m_list) for a batch).  Returns (best_opts, table)."""
    batch = sizes is not None
    nus_l = list(nus) if batch else [int(nus)]
    grid = grid if grid is not None else candidates(nus_l, eps)
    stream = torch.cuda.current_stream()
    table = []

    def make(opts):
        if batch:
            return Plan.many(nus_l, r, sizes[0], omega, sizes[1], eps, precision=precision, **opts)
        return Plan(nus_l[0], r, omega, eps, precision=precision, **opts)

    for opts in grid:
        make(opts).close()                      # warm up (tables, pools)
        if objective == "execute":
            with make(opts) as p:
                p.execute(c)
                t = _time(lambda: p.execute(c), stream, reps)
        else:
            def step():
                with make(opts) as p:
                    p.execute(c)
            t = _time(step, stream, reps)
        table.append((t, opts))
    table.sort(key=lambda x: x[0])
    return dict(table[0][1]), table
