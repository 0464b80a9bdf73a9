"""Oracle: pointwise local (Wimp) and asymptotic (Hankel) sums.

Test infrastructure only.  These evaluate, term by term with the oracle's own
J_n, the two truncated expansions whose errors Lemma 3.1 and the remainder bound of Sec. 3.2 (eq. asy-error) bound:

* Wimp expansion (Sec. 3.1).  The printed coefficient
  C_l(x) = delta_l J_{nu/2+l}(x) J_{nu/2-l}(x) contradicts the proof of
  Lemma 3.1, which evaluates the factors at x/2; the reading used is
      even nu:  J_nu(x y) = sum_l delta_l J_{nu/2+l}(x/2) J_{nu/2-l}(x/2) T_{2l}(y),
      odd nu:   J_nu(x y) = sum_l 2 J_{(nu+1)/2+l}(x/2) J_{(nu-1)/2-l}(x/2) T_{2l+1}(y),
  delta_0 = 1, delta_l = 2 otherwise, |y| <= 1 (the odd form follows from
  Graf's addition theorem, DLMF 10.23.7, with both arguments x/2).
* Hankel expansion (Sec. 3.2, eq. asymptotic-expansion / the bracket of
  eq. asy-error), M pairs of
  terms, phi = -(2nu+1)pi/4.
"""
import math

import numpy as np

from . import _lib
from .params import hankel_a


def _cheb_t(k, y):
    """T_k(y) = cos(k arccos y) for |y| <= 1 (textbook definition)."""
    return math.cos(k * math.acos(max(-1.0, min(1.0, y))))


def wimp_coeff(nu, l, x):
    """C_l(x) of the (reading of the) Wimp expansion."""
    nu = int(nu)
    if nu % 2 == 0:
        h = nu // 2
        d = 1.0 if l == 0 else 2.0
        return d * _lib.jn(h + l, 0.5 * x) * _lib.jn(h - l, 0.5 * x) if h - l >= 0 else \
            d * _lib.jn(h + l, 0.5 * x) * ((-1) ** (l - h)) * _lib.jn(l - h, 0.5 * x)
    hp = (nu + 1) // 2
    hm = (nu - 1) // 2 - l
    jm = _lib.jn(hm, 0.5 * x) if hm >= 0 else ((-1) ** (-hm)) * _lib.jn(-hm, 0.5 * x)
    return 2.0 * _lib.jn(hp + l, 0.5 * x) * jm


def wimp_sum(nu, L, x, y):
    """sum_{l=0..L} C_l(x) T_{2l (+1)}(y), the Wimp expansion truncated after l = L."""
    nu = int(nu)
    odd = nu % 2
    s = 0.0
    for l in range(L + 1):
        s += wimp_coeff(nu, l, x) * _cheb_t(2 * l + odd, y)
    return s


def hankel_sum(nu, M, x):
    """sqrt(2/pi) sum_{l<M} [(-1)^l a_2l x^(-2l-1/2) cos(x+phi)
                             - (-1)^l a_2l+1 x^(-2l-3/2) sin(x+phi)], Sec. 3.2."""
    phi = -(2.0 * nu + 1.0) * math.pi / 4.0
    # cos/sin(x + phi) by angle addition, so that x + phi is never rounded
    cx, sx, cp, sp = math.cos(x), math.sin(x), math.cos(phi), math.sin(phi)
    c, s = cx * cp - sx * sp, sx * cp + cx * sp
    acc = 0.0
    for l in range(M):
        sg = -1.0 if l % 2 else 1.0
        acc += sg * hankel_a(2 * l, nu) * x ** (-2 * l - 0.5) * c
        acc -= sg * hankel_a(2 * l + 1, nu) * x ** (-2 * l - 1.5) * s
    return math.sqrt(2.0 / math.pi) * acc


def wimp_sum_vec(nu, L, x, y):
    """Vectorised wimp_sum over arrays x, y (same shape)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    out = np.empty(np.broadcast(x, y).shape)
    for idx in np.ndindex(out.shape):
        out[idx] = wimp_sum(nu, L, float(np.broadcast_to(x, out.shape)[idx]),
                            float(np.broadcast_to(y, out.shape)[idx]))
    return out
