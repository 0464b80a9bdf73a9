"""Oracle: block subdivision of the Hankel matrix (test infrastructure only).

Plain restatement of Sec. 4.1: SplitIndices (eq. subdiv-optim, with the quasi-optimal
candidate search the paper recommends) and Algorithm 1 (Subdivide).

Indexing: rows are frequencies omega (sorted ascending, 0-based k), columns
are points r (sorted ascending, 0-based j).  A block is (k0, k1, j0, j1),
inclusive.  An entry is local when omega_k * r_j <= z (products in FP64),
asymptotic otherwise.

Readings of the printed algorithm (see the design notes):
* eq. subdiv-optim writes argmax of the mixed area; the text says the chosen pair
  minimises it, which is what makes the fast blocks large.  The mixed area
  (k-k0+1)(j1-j) + (k1-k)(j-j0+1) is minimised.
* For a candidate row k the column is j(k) = max{ j in [j0, j1] :
  omega_k r_j <= z } (j0-1 when there is none), so that the lower-right
  block is purely asymptotic.
* Candidates: all rows when the block has at most n_cand rows, else
  k0 + floor(c (k1-k0) / (n_cand-1)), c = 0..n_cand-1; ties go to the
  first candidate.
* Algorithm 1 swaps the index names of r and omega in its size tests; the
  areas used are (rows)x(cols) of each off-diagonal block.  A mixed
  off-diagonal block with area <= min_size goes to the direct set (the
  paper's text says "<", its algorithm ">"; ties go to direct).
* Blocks that are entirely local or entirely asymptotic are appended to the
  local / asymptotic sets whatever their size (the proof of the complexity
  theorem treats such blocks this way); empty blocks are dropped.
* The work list is processed first-in first-out.
"""
from bisect import bisect_right
from collections import deque


def _last_local_col(r, w, z, j0, j1):
    """max{j in [j0, j1] : w * r[j] <= z}, or j0 - 1."""
    return bisect_right(r, z, j0, j1 + 1, key=lambda v: w * v) - 1


def split_indices(r, omega, z, blk, n_cand=16):
    """Quasi-optimal (k, j) for a mixed block (Sec. 4.1, eq. subdiv-optim)."""
    k0, k1, j0, j1 = blk
    nrows = k1 - k0 + 1
    if nrows <= n_cand:
        cands = range(k0, k1 + 1)
    else:
        cands = [k0 + (c * (k1 - k0)) // (n_cand - 1) for c in range(n_cand)]
    best = None
    for k in cands:
        j = _last_local_col(r, omega[k], z, j0, j1)
        area = (k - k0 + 1) * (j1 - j) + (k1 - k) * (j - j0 + 1)
        if best is None or area < best[0]:
            best = (area, k, j)
    return best[1], best[2]


def classify(r, omega, z, blk):
    """'local', 'asy' or 'mixed' for a non-empty block."""
    k0, k1, j0, j1 = blk
    if omega[k1] * r[j1] <= z:
        return "local"
    if omega[k0] * r[j0] > z:
        return "asy"
    return "mixed"


def subdivide(r, omega, z, min_size=1024, n_cand=16):
    """Algorithm 1.  r, omega sorted ascending.  Returns (L, A, D) lists of
    (k0, k1, j0, j1) blocks, local / asymptotic / direct."""
    n, m = len(r), len(omega)
    Lb, Ab, Db = [], [], []
    if n == 0 or m == 0:
        return Lb, Ab, Db
    work = deque()

    def place(blk, is_root=False):
        k0, k1, j0, j1 = blk
        if k1 < k0 or j1 < j0:
            return
        cls = classify(r, omega, z, blk)
        if cls == "local":
            Lb.append(blk)
        elif cls == "asy":
            Ab.append(blk)
        elif (k1 - k0 + 1) * (j1 - j0 + 1) <= min_size:
            Db.append(blk)
        else:
            work.append(blk)

    place((0, m - 1, 0, n - 1), True)
    while work:
        k0, k1, j0, j1 = work.popleft()
        k, j = split_indices(r, omega, z, (k0, k1, j0, j1), n_cand)
        place((k0, k, j0, j))           # upper left: local
        place((k + 1, k1, j + 1, j1))   # lower right: asymptotic
        place((k0, k, j + 1, j1))       # upper right: mixed
        place((k + 1, k1, j0, j))       # lower left: mixed
    return Lb, Ab, Db
