"""Exact results the oracle is pinned to (test helper, no method arithmetic).

* Kaufman's closed form for the partition function of the L x L periodic
  Ising model (B. Kaufman, Phys. Rev. 76, 1232 (1949); the four-product form
  of A. E. Ferdinand and M. E. Fisher, Phys. Rev. 185, 832 (1969)),
  evaluated in 60-digit arithmetic with mpmath.
* Brute-force enumeration of every state of a tiny lattice, given an energy
  function, and the Boltzmann averages that follow from it.
"""
from __future__ import annotations

import mpmath as mp
import numpy as np

mp.mp.dps = 60


def kaufman_lnZ(L: int, K) -> mp.mpf:
    """ln Z of the L x L torus with H = -sum_<ij> s_i s_j at coupling K = beta.

    Z = 1/2 (2 sinh 2K)^{L^2/2} (Z1 + Z2 + Z3 + Z4) with
    Z1 = prod_r 2 cosh(L g_{2r+1}/2), Z2 = prod_r 2 sinh(L g_{2r+1}/2),
    Z3 = prod_r 2 cosh(L g_{2r}/2),   Z4 = prod_r 2 sinh(L g_{2r}/2),
    r = 0..L-1, cosh g_l = cosh 2K coth 2K - cos(pi l / L) for l != 0 and
    g_0 = 2K + ln tanh K (negative above T_c, which flips the sign of Z4).
    """
    K = mp.mpf(K)
    if K == 0:
        return (L * L) * mp.log(2)

    def gam(l):
        if l % (2 * L) == 0:
            return 2 * K + mp.log(mp.tanh(K))
        return mp.acosh(mp.cosh(2 * K) * mp.coth(2 * K) - mp.cos(mp.pi * l / L))

    Z1 = mp.fprod(2 * mp.cosh(L * gam(2 * r + 1) / 2) for r in range(L))
    Z2 = mp.fprod(2 * mp.sinh(L * gam(2 * r + 1) / 2) for r in range(L))
    Z3 = mp.fprod(2 * mp.cosh(L * gam(2 * r) / 2) for r in range(L))
    Z4 = mp.fprod(2 * mp.sinh(L * gam(2 * r) / 2) for r in range(L))
    return mp.log(mp.mpf(1) / 2) + (L * L / mp.mpf(2)) * mp.log(2 * mp.sinh(2 * K)) + mp.log(
        Z1 + Z2 + Z3 + Z4)


def kaufman_energy_per_site(L: int, K) -> float:
    """<E>/N = -(1/N) d ln Z / d beta."""
    return float(-mp.diff(lambda k: kaufman_lnZ(L, k), mp.mpf(K)) / (L * L))


def all_states(N: int) -> np.ndarray:
    """Every +-1 configuration of N sites as an int8 array [2^N, N]."""
    idx = np.arange(1 << N, dtype=np.int64)[:, None]
    bits = (idx >> np.arange(N, dtype=np.int64)[None, :]) & 1
    return np.where(bits == 1, -1, 1).astype(np.int8)


def density_of_states(energies) -> dict:
    g: dict[int, int] = {}
    for E in energies:
        g[int(E)] = g.get(int(E), 0) + 1
    return g


def lnZ_from_dos(g: dict, beta) -> mp.mpf:
    b = mp.mpf(beta)
    return mp.log(mp.fsum(c * mp.exp(-b * E) for E, c in g.items()))


def mean_energy_from_dos(g: dict, beta) -> float:
    b = mp.mpf(beta)
    Z = mp.fsum(c * mp.exp(-b * E) for E, c in g.items())
    return float(mp.fsum(c * E * mp.exp(-b * E) for E, c in g.items()) / Z)


def boltzmann_from_dos(g: dict, beta) -> dict:
    b = mp.mpf(beta)
    Z = mp.fsum(c * mp.exp(-b * E) for E, c in g.items())
    return {E: float(c * mp.exp(-b * E) / Z) for E, c in g.items()}
