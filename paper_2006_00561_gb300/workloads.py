"""Seeded synthetic workloads (run descriptions only, no method arithmetic).

The paper's workload is the 2D Ising model at L = 64 with 20 480 replicas per
GPU (Sec. 3) and 2 129 920 replicas in its largest run (Sec. 4); it uses no
dataset.  These generators describe runs of that shape and the two
multi-run forms (a +-J disorder ensemble, a stream of requests) from a numpy
PCG64 stream, so every description is reproducible from its seed.
"""
from __future__ import annotations

import numpy as np

# (dim, L) classes of the serving mix
SERVING_CLASSES = [(2, 16), (2, 32), (2, 64), (2, 128), (3, 6), (3, 8), (3, 10)]


def ea_ensemble(n: int = 256, seed: int = 4, K: int = 150, theta: int = 10,
                beta_max: float = 3.0, Ls=(6, 8, 10), R0s=(1 << 14, 1 << 15, 1 << 16)) -> list:
    """n independent 3D +-J Edwards-Anderson instances: L and R0 uniform over
    the given sets, one coupling seed and one Metropolis seed per instance."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        out.append(dict(dim=3, L=int(rng.choice(Ls)), model=1, R0=int(rng.choice(R0s)), K=K,
                        theta=theta, beta0=0.0, beta_max=beta_max,
                        seed=int(rng.integers(1, 2 ** 63)),
                        coupling_seed=int(rng.integers(1, 2 ** 63)), instance_id=i))
    return out


def serving_trace(n: int = 256, rate: float = 50.0, seed: int = 5, theta: int = 10,
                  R0_exp=(12, 18), K_range=(100, 300), beta_maxes=(1.0, 3.0)) -> list:
    """n requests with Poisson arrivals at `rate` per second: (dim, L) uniform
    over SERVING_CLASSES (2D ferromagnet, 3D +-J), R0 = 2^U with U uniform in
    R0_exp, K uniform in K_range, beta_max uniform over beta_maxes."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += float(rng.exponential(1.0 / rate))
        dim, L = SERVING_CLASSES[int(rng.integers(len(SERVING_CLASSES)))]
        out.append(dict(arrival=t, dim=dim, L=L, model=0 if dim == 2 else 1,
                        R0=1 << int(rng.integers(R0_exp[0], R0_exp[1] + 1)),
                        K=int(rng.integers(K_range[0], K_range[1] + 1)), theta=theta,
                        beta0=0.0, beta_max=float(rng.choice(beta_maxes)),
                        seed=int(rng.integers(1, 2 ** 63)),
                        coupling_seed=int(rng.integers(1, 2 ** 63)), instance_id=i))
    return out
