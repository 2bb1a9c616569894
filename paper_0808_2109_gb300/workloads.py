"""Seeded synthetic workloads (inputs only: no Swendsen-Wang arithmetic here).

The paper measures on lattices it generates itself (Sec. II.C: L = 7920 at
T_c on the Dawning 4000A, several L and T on the SGI Onyx 3900); there is no
dataset.  These generators give the shapes the benchmark and the tests use:
plain SW at the critical temperature, the three temperature regimes, a PCC
lattice, an uneven batch of replicas and a Poisson stream of served jobs.
Lattice spins themselves come from each side's own hot start (the INIT
Philox stream), so nothing here draws spins.
"""
from __future__ import annotations

from dataclasses import asdict, dataclass

import numpy as np

T_CRITICAL_ROUNDED = 2.269185   # the critical configuration's temperature as written
J = 1.0


@dataclass(frozen=True)
class Plain:
    L: int
    T: float
    sweeps: int
    seed: int = 1


# L=64 at T_c, 1000 sweeps: the small case the oracle finishes in seconds.
SMALL = Plain(64, T_CRITICAL_ROUNDED, 1000)
# L=4096 in the giant-cluster, critical and small-cluster regimes.
REGIMES = tuple(Plain(4096, T, 200) for T in (2.0, T_CRITICAL_ROUNDED, 3.0))
# The benchmark lattice: 268M sites at T_c, 50 sweeps.
LARGE = Plain(16384, T_CRITICAL_ROUNDED, 50)


@dataclass(frozen=True)
class PCC:
    L: int = 2048
    sweeps: int = 10000
    seed: int = 1


PCC_RUN = PCC()


@dataclass(frozen=True)
class Job:
    """One replica or served job: plain SW at (J, T) or a PCC lattice."""
    L: int
    T: float
    seed: int
    sweeps: int
    pcc: bool = False
    arrival_s: float = 0.0

    def as_dict(self):
        return asdict(self)


def batch_manifest(n: int = 512, sweeps: int = 500, rng_seed: int = 20260) -> list[Job]:
    """Uneven replica mix: L from {64,...,1024} with weights {.4,.25,.2,.1,.05},
    T on a 32-point ladder 2.0 .. 2.6 (endpoints included), seed 1000 + r."""
    rng = np.random.default_rng(rng_seed)
    sizes = rng.choice([64, 128, 256, 512, 1024], size=n, p=[0.4, 0.25, 0.2, 0.1, 0.05])
    return [Job(int(sizes[r]), 2.0 + 0.6 * (r % 32) / 31.0, 1000 + r, sweeps) for r in range(n)]


def serve_trace(rate_hz: float = 200.0, duration_s: float = 60.0, rng_seed: int = 20261,
                L_min: int = 32, L_max: int = 4096, sweeps_lo: int = 10, sweeps_hi: int = 1000,
                pcc_fraction: float = 0.2) -> list[Job]:
    """Poisson arrivals; L log-uniform in [L_min, L_max]; sweeps uniform in
    [sweeps_lo, sweeps_hi]; 80% plain SW with T uniform in [1.8, 3.2], 20% PCC."""
    rng = np.random.default_rng(rng_seed)
    jobs, t, k = [], 0.0, 0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        L = int(round(np.exp(rng.uniform(np.log(L_min), np.log(L_max)))))
        sweeps = int(rng.integers(sweeps_lo, sweeps_hi + 1))
        pcc = bool(rng.random() < pcc_fraction)
        T = float(rng.uniform(1.8, 3.2))
        jobs.append(Job(L, T, 5000 + k, sweeps, pcc, float(t)))
        k += 1
    return jobs
