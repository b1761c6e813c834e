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


def kaufman_cv_per_site(L: int, K) -> float:
    """Specific heat per site of the L x L torus from the thermodynamic
    definition C = beta^2 d^2 ln Z / d beta^2, differentiated numerically
    (60-digit arithmetic) through Kaufman's closed form."""
    K = mp.mpf(K)
    return float(K * K * mp.diff(lambda k: kaufman_lnZ(L, k), K, 2) / (L * L))


def joint_dos_2d_torus(L: int) -> dict:
    """g(E, M) of the L x L ferromagnetic torus by enumeration of all 2^(L^2)
    states: E = -sum over the 2 L^2 bonds of s_i s_j (one term per bond,
    periodic), M = sum of the spins.  Written with array shifts, independently
    of any energy routine under test."""
    S = all_states(L * L).reshape(-1, L, L).astype(np.int64)  # [state, y, x]
    E = -(S * np.roll(S, -1, axis=2)).sum(axis=(1, 2)) - (S * np.roll(S, -1, axis=1)).sum(
        axis=(1, 2))
    M = S.sum(axis=(1, 2))
    pairs, counts = np.unique(np.stack([E, M], axis=1), axis=0, return_counts=True)
    return {(int(e), int(m)): int(c) for (e, m), c in zip(pairs, counts)}


def exact_observables(g: dict, N: int, beta) -> dict:
    """Boltzmann averages at inverse temperature beta > 0 from a joint density
    of states g(E, M):
      C_v per site   = beta^2 d^2 ln Z / d beta^2 / N (thermodynamic definition),
      <|m|>          = sum |M| g e^{-beta E} / (N Z),
      <M^2>          = d^2 ln Z(h) / d(beta h)^2 at h = 0, with
                       Z(h) = sum g e^{-beta E + beta h M} (the field derivative;
                       <M> = 0 by symmetry),
      chi per site   = beta (<M^2> - <|M|>^2) / N, the finite-lattice
                       susceptibility with |M| in place of M."""
    b = mp.mpf(beta)
    items = [(mp.mpf(E), mp.mpf(M), c) for (E, M), c in g.items()]

    def lnZ_beta(bb):
        return mp.log(mp.fsum(c * mp.exp(-bb * E) for E, M, c in items))

    def lnZ_field(x):  # x = beta h
        return mp.log(mp.fsum(c * mp.exp(-b * E + x * M) for E, M, c in items))

    Z = mp.fsum(c * mp.exp(-b * E) for E, M, c in items)
    mabs = mp.fsum(c * abs(M) * mp.exp(-b * E) for E, M, c in items) / Z
    m2 = mp.diff(lnZ_field, mp.mpf(0), 2)
    e = mp.fsum(c * E * mp.exp(-b * E) for E, M, c in items) / Z
    return {
        "e": float(e / N),
        "cv": float(b * b * mp.diff(lnZ_beta, b, 2) / N),
        "m_abs": float(mabs / N),
        "m2": float(m2),
        "chi": float(b * (m2 - mabs * mabs) / N),
    }
