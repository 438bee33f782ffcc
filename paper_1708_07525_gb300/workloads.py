"""Synthetic cavity workloads (seeded).  Holds parameter sets and seeded draws
only -- none of the method's arithmetic -- so that the GPU path, the oracle
and the benchmark are fed identical inputs.

Physics of every cavity: left wall T = C = 1, right wall T = C = 0, top and
bottom adiabatic and impermeable, no-slip walls; u = 0 and T = C = 1/2 plus
uniform noise at t = 0; Pr, J, sigma as given; F_eps from the Ergun relation.
"""
from __future__ import annotations

from dataclasses import dataclass, asdict

import numpy as np


@dataclass(frozen=True)
class CavitySpec:
    nx: int
    ny: int
    Ra: float
    Da: float
    eps: float
    Pr: float = 1.0
    Le: float = 1.0
    N: float = 1.0
    J: float = 1.0
    sigma: float = 1.0
    seed: int = 1
    noise: float = 1e-3
    varpi: float = 0.4

    def args(self):
        return (self.nx, self.ny, self.Ra, self.Da, self.eps, self.Pr, self.Le, self.N, self.J,
                self.sigma)

    def as_dict(self):
        return asdict(self)


# 64 x 64 porous cavity, aiding buoyancy, FP64 reference case (10,000 steps).
SMALL_AIDING = CavitySpec(64, 64, Ra=1e4, Da=1e-2, eps=0.6, Pr=1.0, Le=2.0, N=1.0, seed=1)


def throughput_cavity(n: int) -> CavitySpec:
    """Square n x n cavity with opposing buoyancy (N = -1), Ra = 1e5, Da = 1e-3,
    eps = 0.4, Le = 5: the throughput workload (256^2, 1024^2, 4096^2; FP32)."""
    return CavitySpec(n, n, Ra=1e5, Da=1e-3, eps=0.4, Pr=1.0, Le=5.0, N=-1.0, seed=2)


# 1024^2 precision-study cavity: Ra = 1e5, Da = 1e-2, eps = 0.6, Le = 10, N = 2.
PRECISION_STUDY = CavitySpec(1024, 1024, Ra=1e5, Da=1e-2, eps=0.6, Pr=1.0, Le=10.0, N=2.0, seed=3)

# Non-porous double-diffusive cavity, aspect ratio 2 (100 x 200), Ra = 1e5, Pr = 1,
# Le = 2, N = -0.8, eps = 1, Da = 1e8 (the paper's Sec. 4.1 case).
NONPOROUS_A2 = CavitySpec(100, 200, Ra=1e5, Da=1e8, eps=1.0, Pr=1.0, Le=2.0, N=-0.8, seed=7)


def stable_varpi(eps: float, sigma: float) -> float:
    """The D2Q5 parameter varpi (Sec. 3.2, free in (0, 1); 2/5 in the paper's runs),
    lowered where eps or sigma is small: the rest equilibria (sigma - varpi) T and
    (eps - varpi) C of Eq. 28 must stay positive for a stable scheme."""
    return min(0.4, 0.8 * min(eps, sigma))


def draw_batch(count: int, seed: int, sizes=(32, 64, 128, 256)) -> list[CavitySpec]:
    """Mixed cavities: grid from `sizes` uniformly, log-uniform Ra in [1e3, 1e5] and
    Da in [1e-4, 1e-1], uniform eps in [0.3, 0.9], Le in [0.5, 10], N in [-5, 5],
    sigma in [0.5, 2], Pr = J = 1; varpi from stable_varpi()."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(rng.choice(sizes))
        Ra = float(10 ** rng.uniform(3, 5))
        Da = float(10 ** rng.uniform(-4, -1))
        eps = float(rng.uniform(0.3, 0.9))
        Le = float(rng.uniform(0.5, 10))
        N = float(rng.uniform(-5, 5))
        sigma = float(rng.uniform(0.5, 2.0))
        out.append(CavitySpec(n, n, Ra=Ra, Da=Da, eps=eps, Pr=1.0, Le=Le, N=N, J=1.0, sigma=sigma,
                              seed=int(rng.integers(1, 2 ** 31)), varpi=stable_varpi(eps, sigma)))
    return out


def arrivals(count: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Poisson arrival times (s) of `count` requests at the given mean rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


def random_fields(nx: int, ny: int, seed: int, amp: float = 1e-3):
    """Seeded initial T and C fields (1/2 plus uniform noise) as [ny][nx] arrays."""
    rng = np.random.default_rng(seed)
    T = 0.5 + amp * rng.uniform(-1, 1, (ny, nx))
    C = 0.5 + amp * rng.uniform(-1, 1, (ny, nx))
    return T, C
