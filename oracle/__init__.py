"""Oracle for the nonuniform Hankel transform — TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, FP64 CPU restatement of what the paper's
method computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product path (``paper_2411_09583_gb300``) never imports, links or runs
anything here, and nothing here imports the product.

Contents
--------
direct.c       J_nu evaluator (series / Miller / Hankel) and the O(nm) direct
               sum g_k = sum_j c_j J_nu(omega_k r_j)  (Sec. 1, eq. DHT).
params.py      error bounds B^loc (Lemma 3.1), B^asy (Sec. 3.2, eq. asy-error),
               the M heuristic (Sec. 3.3, eq. num-asy-terms) and the crossover z / local order L
               (Sec. 3.3).
subdivide.py   SplitIndices (Sec. 4.1, eq. subdiv-optim) and Subdivide
               (Algorithm 1).
expansions.py  pointwise Wimp (Sec. 3.1) and Hankel (Sec. 3.2) sums.
nudft.py       direct type-3 nonuniform DFT sum (the matrix F of Sec. 3.2).
"""
from ._lib import (build, jn, jn_prod, jv_series, jv_hankel, jn_miller,
                   direct, direct_rows)

__all__ = ["build", "jn", "jn_prod", "jv_series", "jv_hankel", "jn_miller",
           "direct", "direct_rows"]
