"""Exact and closed-form results for the 2D square Ising model (J = 1, K = 1,
h = 0, periodic).  TEST INFRASTRUCTURE ONLY, used to pin the oracle chain to
something other than itself.

- ``enumerate_torus``: brute force over all 2^(L*L) states of a small torus,
  with the energy of Eq. 1 written independently of oracle.c (numpy rolls).
- ``kaufman_logz``: Kaufman's closed-form partition function of a finite
  m x n torus (Phys. Rev. 76, 1232 (1949)), a second, independent route to the
  same finite-lattice averages.
- ``onsager_energy`` / ``yang_magnetization``: the infinite-lattice energy per
  spin (Onsager 1944) and spontaneous magnetisation (Yang 1952).
"""
from __future__ import annotations

import math

import numpy as np


def enumerate_torus(L: int):
    """All 2^(L*L) configurations of an L x L torus.  Returns (E, M) as int64
    arrays with E = -sum_<mn> s_m s_n (each bond once) and M = sum s."""
    n = L * L
    assert n <= 20, "brute force is only for tiny lattices"
    idx = np.arange(1 << n, dtype=np.int64)
    bits = ((idx[:, None] >> np.arange(n, dtype=np.int64)[None, :]) & 1).astype(np.int64)
    s = (2 * bits - 1).reshape(-1, L, L)
    E = -(s * np.roll(s, -1, axis=1)).sum(axis=(1, 2)) - (s * np.roll(s, -1, axis=2)).sum(axis=(1, 2))
    M = s.sum(axis=(1, 2))
    return E.astype(np.int64), M.astype(np.int64)


def exact_means(L: int, beta: float):
    """Boltzmann averages <E>/N and <|M|>/N, and the probability of each energy
    level, for an L x L torus by enumeration."""
    E, M = enumerate_torus(L)
    e0 = E.min()
    w = np.exp(-beta * (E - e0).astype(np.float64))
    Z = w.sum()
    n = L * L
    mean_e = float((w * E).sum() / Z) / n
    mean_absm = float((w * np.abs(M)).sum() / Z) / n
    levels = np.unique(E)
    probs = np.array([w[E == lv].sum() / Z for lv in levels])
    return mean_e, mean_absm, levels, probs


def kaufman_logz(m: int, n: int, beta: float) -> float:
    """ln Z of an m x n periodic square lattice (m rows, n columns), J = 1.
    Kaufman (1949):  Z = 1/2 (2 sinh 2K)^{mn/2} [Z1 + Z2 + Z3 + Z4] with
    Z1 = prod_{r=0}^{n-1} 2 cosh(m g_{2r+1}/2), Z2 = prod 2 sinh(m g_{2r+1}/2),
    Z3 = prod 2 cosh(m g_{2r}/2),  Z4 = prod 2 sinh(m g_{2r}/2), and
    cosh g_k = cosh 2K* cosh 2K - sinh 2K* sinh 2K cos(pi k / n), where
    tanh K* = exp(-2K) and g_0 = 2(K - K*) carries its sign."""
    K = beta
    Ks = math.atanh(math.exp(-2.0 * K))

    def gamma(k):
        if k == 0:
            return 2.0 * (K - Ks)
        c = math.cosh(2 * Ks) * math.cosh(2 * K) - math.sinh(2 * Ks) * math.sinh(2 * K) * math.cos(math.pi * k / n)
        return math.acosh(c)

    odd = [gamma(2 * r + 1) for r in range(n)]
    even = [gamma(2 * r) for r in range(n)]

    def log_prod_cosh(gs):
        return sum(math.log(2 * math.cosh(m * g / 2)) for g in gs)

    def log_prod_sinh(gs):
        # returns (sign, log|prod|)
        sign = 1.0
        tot = 0.0
        for g in gs:
            v = 2 * math.sinh(m * g / 2)
            if v == 0.0:
                return 0.0, -math.inf
            sign *= math.copysign(1.0, v)
            tot += math.log(abs(v))
        return sign, tot

    terms = []
    signs = []
    terms.append(log_prod_cosh(odd)); signs.append(1.0)
    s2, l2 = log_prod_sinh(odd); terms.append(l2); signs.append(s2)
    terms.append(log_prod_cosh(even)); signs.append(1.0)
    s4, l4 = log_prod_sinh(even); terms.append(l4); signs.append(s4)
    mx = max(t for t in terms if t != -math.inf)
    tot = sum(sg * math.exp(t - mx) for sg, t in zip(signs, terms) if t != -math.inf)
    return math.log(0.5) + 0.5 * m * n * math.log(2 * math.sinh(2 * K)) + mx + math.log(tot)


def kaufman_energy(L: int, beta: float, h: float = 1e-5) -> float:
    """<E>/N = -(1/N) d ln Z / d beta for the L x L torus, by a central
    difference of Kaufman's ln Z (step h)."""
    lp = kaufman_logz(L, L, beta + h)
    lm = kaufman_logz(L, L, beta - h)
    return -(lp - lm) / (2 * h) / (L * L)


def onsager_energy(beta: float) -> float:
    """Infinite-lattice energy per spin (Onsager 1944):
    u = -coth 2b [1 + (2/pi)(2 tanh^2 2b - 1) K(k)], k = 2 sinh 2b / cosh^2 2b,
    K the complete elliptic integral of the first kind (modulus k)."""
    from scipy.special import ellipk
    b2 = 2.0 * beta
    k = 2.0 * math.sinh(b2) / math.cosh(b2) ** 2
    return float(-(1.0 / math.tanh(b2)) * (1.0 + (2.0 / math.pi) * (2.0 * math.tanh(b2) ** 2 - 1.0) * ellipk(k * k)))


BETA_C = 0.5 * math.log(1.0 + math.sqrt(2.0))


def yang_magnetization(beta: float) -> float:
    """Spontaneous magnetisation per spin (Yang 1952): (1 - sinh^-4 2b)^(1/8)
    below T_c, zero above."""
    if beta <= BETA_C:
        return 0.0
    return (1.0 - math.sinh(2.0 * beta) ** -4) ** 0.125


def binned_error(x: np.ndarray, nbins: int = 32) -> tuple[float, float]:
    """Mean and standard error of a correlated series from nbins block means."""
    x = np.asarray(x, dtype=np.float64)
    n = (len(x) // nbins) * nbins
    blocks = x[:n].reshape(nbins, -1).mean(axis=1)
    return float(x.mean()), float(blocks.std(ddof=1) / math.sqrt(nbins))
