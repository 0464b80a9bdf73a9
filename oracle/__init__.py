"""Oracle for the nonuniform Hankel transform — TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, FP64 CPU restatement of what the paper's
method computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product path (``paper_2411_09583_gb300``) never imports, links or runs
anything here, and nothing here imports the product.

Contents
--------
direct.c       J_nu evaluator (series / Miller / Hankel) and the O(nm) direct
               sum g_k = sum_j c_j J_nu(omega_k r_j)  (Eq. 1.5, Sec. 2).
params.py      error bounds B^loc (Lemma 3.1), B^asy (Eq. 3.5), the M
               heuristic (Eq. 3.7) and the crossover z / local order L
               (Sec. 3.3).
subdivide.py   SplitIndices (Eq. 4.1) and Subdivide (Algorithm 1).
expansions.py  pointwise Wimp (Eq. 3.1) and Hankel (Eq. 3.4/3.5) sums.
nudft.py       direct type-3 nonuniform DFT sum (the operator F of Eq. 3.6).
"""
from ._lib import (build, jn, jn_prod, jv_series, jv_hankel, jn_miller,
                   direct, direct_rows)

__all__ = ["build", "jn", "jn_prod", "jv_series", "jv_hankel", "jn_miller",
           "direct", "direct_rows"]
