"""Oracle: expansion orders and crossover point (test infrastructure only).

Plain-Python restatement of Sec. 3.1-3.3 of the paper:

* B^loc_{nu,L}(Omega R): Lemma 3.1, the truncation bound of the Wimp
  expansion after the terms l = 0..L.  For odd nu the paper only states that
  "a similar calculation" applies; the reading used here repeats the proof of
  Lemma 3.1 for the odd-order Wimp expansion
      J_nu(x y) = sum_{l>=0} 2 J_{(nu+1)/2+l}(x/2) J_{(nu-1)/2-l}(x/2) T_{2l+1}(y),
  giving beta = psi(x/(2L+3+nu)), gamma = psi(x/(2L+3-nu)) (when
  L+1 > (nu-1)/2, else 0) and
      B = 2 exp(((nu+1)/2) beta - ((nu-1)/2) gamma + (L+1)(beta+gamma))
          / (1 - exp(beta+gamma)).
  The gamma case of the even bound is taken with strict inequality
  L+1 > nu/2 (equality would divide by zero).  Arguments outside Siegel's
  range (p >= 1) or beta+gamma >= 0 give an infinite bound.
* B^asy_{nu,M}(z): Sec. 3.2, eq. asy-error, the first-neglected-terms remainder of the
  M-term Hankel expansion, with a_k(nu) = prod_{i=1..k}(4nu^2-(2i-1)^2)/(k! 8^k)
  (DLMF 10.17.1; the printed product is garbled).
* M: the heuristic of Sec. 3.3 (eq. num-asy-terms).
* z: the root of B^asy(z) = eps (Sec. 3.3; any accurate root finder gives the
  same value, Newton with a bisection safeguard is used here).
* L: the smallest L with B^loc(z) < eps (Sec. 3.3).
"""
import math


def hankel_a(k, nu):
    """a_k(nu) = prod_{i=1..k} (4 nu^2 - (2i-1)^2) / (k! 8^k)."""
    mu = 4.0 * nu * nu
    v = 1.0
    for i in range(1, k + 1):
        v *= (mu - (2 * i - 1) ** 2) / (i * 8.0)
    return v


def psi(p):
    """psi(p) = log p + sqrt(1-p^2) - log(1 + sqrt(1-p^2)), Lemma 3.1."""
    s = math.sqrt(1.0 - p * p)
    return math.log(p) + s - math.log1p(s)


def b_loc(nu, L, x):
    """Lemma 3.1 bound for the Wimp expansion truncated after l = L, at Omega*R = x."""
    if x <= 0.0:
        return 0.0
    nu = abs(int(nu))
    if nu % 2 == 0:
        d_beta = 2 * L + 2 + nu
        d_gamma = 2 * L + 2 - nu
        use_gamma = (L + 1) > nu / 2.0
        a_beta, a_gamma = nu / 2.0, nu / 2.0
    else:
        d_beta = 2 * L + 3 + nu
        d_gamma = 2 * L + 3 - nu
        use_gamma = (L + 1) > (nu - 1) / 2.0
        a_beta, a_gamma = (nu + 1) / 2.0, (nu - 1) / 2.0
    p = x / d_beta
    if p >= 1.0:
        return math.inf
    beta = psi(p)
    gamma = 0.0
    if use_gamma:
        pg = x / d_gamma
        if pg >= 1.0:
            return math.inf
        gamma = psi(pg)
    if beta + gamma >= 0.0:
        return math.inf
    return (2.0 * math.exp(a_beta * beta - a_gamma * gamma + (L + 1) * (beta + gamma))
            / (1.0 - math.exp(beta + gamma)))


def b_asy(nu, M, z):
    """Sec. 3.2, eq. asy-error: sqrt(2/pi) (|a_2M|/z^(2M+1/2) + |a_2M+1|/z^(2M+3/2))."""
    return math.sqrt(2.0 / math.pi) * (
        abs(hankel_a(2 * M, nu)) / z ** (2 * M + 0.5)
        + abs(hankel_a(2 * M + 1, nu)) / z ** (2 * M + 1.5))


def choose_m(nu, eps):
    """Sec. 3.3, eq. num-asy-terms: M = min(floor(1 + nu/5 - log10(eps)/4), 20)."""
    return min(int(math.floor(1.0 + abs(nu) / 5.0 - math.log10(eps) / 4.0)), 20)


def crossover_z(nu, M, eps):
    """z with B^asy_{nu,M}(z) = eps (B^asy is decreasing in z)."""
    lo, hi = 1e-3, 1.0
    while b_asy(nu, M, hi) > eps:
        hi *= 2.0
    while b_asy(nu, M, lo) < eps:
        lo *= 0.5
    z = hi
    for _ in range(200):
        # Newton step on log B - log eps, kept inside the bracket
        f = math.log(b_asy(nu, M, z)) - math.log(eps)
        if f > 0:
            lo = z
        else:
            hi = z
        h = z * 1e-6
        df = (math.log(b_asy(nu, M, z + h)) - math.log(b_asy(nu, M, z - h))) / (2 * h)
        zn = z - f / df if df != 0 else 0.5 * (lo + hi)
        if not (lo < zn < hi):
            zn = 0.5 * (lo + hi)
        if abs(zn - z) <= 1e-15 * z:
            z = zn
            break
        z = zn
    return z


def choose_l(nu, z, eps, lmax=1000):
    """Smallest L >= 0 with B^loc_{nu,L}(z) < eps."""
    for L in range(lmax + 1):
        if b_loc(nu, L, z) < eps:
            return L
    raise ValueError("no L <= %d meets eps" % lmax)


def choose_params(nu, eps, M=None):
    """(M, z, L) for order nu and tolerance eps, Sec. 3.3."""
    if M is None:
        M = choose_m(nu, eps)
    z = crossover_z(nu, M, eps)
    L = choose_l(nu, z, eps)
    return M, z, L
