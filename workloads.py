"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module generates lattice shapes, auxiliary fields sigma, right-hand sides
and request streams.  It holds none of the method's arithmetic (no fermion
matrix, no solver, no HMC step), so the CUDA path and the CPU oracle can both be
fed from it without sharing any computation.  Every generator is NumPy's
Philox bit generator keyed by an explicit seed.

The workloads follow the shapes of the paper's benchmarks (Sec. 5: 3+1
dimensional lattices with N_x of 8-20+, and 1+1 dimensional lattices), with the
common physical parameters t = 1, dtau = 0.05, A = 0.5; sigma is i.i.d.
uniform on [-pi, pi) (a hot start) and sources are i.i.d. N(0, 1).
"""
from dataclasses import dataclass, field

import numpy as np

T_HOP = 1.0
DTAU = 0.05
A_HS = 0.5


@dataclass(frozen=True)
class Workload:
    name: str
    d: int
    nx: int
    ntau: int
    seed: int
    n_md: int = 10
    dt: float = 0.0     # MD step; 0: 1 / n_md (trajectory length 1)
    notes: str = ""

    @property
    def nsites(self) -> int:
        return self.nx ** self.d * self.ntau


# The single-lattice workloads.  C0 is small enough for the oracle to run whole
# trajectories in seconds; C1 and C2 are the at-scale d=1 and d=3 lattices.
C0 = Workload("d1_nx32_nt64", 1, 32, 64, 1007, n_md=10,
              notes="d=1, Nx=32, Ntau=64: one 10-step trajectory, FP64")
C1 = Workload("d1_nx1024_nt512", 1, 1024, 512, 1008, n_md=20, dt=0.002,
              notes="d=1, Nx=1024, Ntau=512: HMC trajectories of 20 leapfrog steps, FP64; from the "
                    "uniform (hot) field the forces reach 1.5e6 and dH is 5e20 at dt = 0.05, 9e7 at "
                    "0.01 and 1.2 at 0.002 (measured), hence dt = 0.002")
C2 = Workload("d3_nx32_nt128", 3, 32, 128, 1009, n_md=10,
              notes="d=3, Nx=32^3, Ntau=128: FP64 CG vs FP32-inner CG")
BATCH_SEED = 1010
SERVE_SEED = 1011
BATCH_NX = (8, 10, 12, 16, 20)
BATCH_NTAU = (40, 64, 96, 160)


def _gen(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed), int(stream)]))


def sigma_field(nsites: int, seed: int, chain: int = 0) -> np.ndarray:
    """Hot-start auxiliary field: i.i.d. uniform on [-pi, pi)."""
    return _gen(seed, 1 + 2 * chain).uniform(-np.pi, np.pi, nsites)


def source(nsites: int, seed: int, chain: int = 0, rhs: int = 0) -> np.ndarray:
    """A right-hand side b with i.i.d. N(0, 1) entries."""
    return _gen(seed, 1000 + 64 * chain + rhs).standard_normal(nsites)


def unit_normal(nsites: int, seed: int, stream: int) -> np.ndarray:
    return _gen(seed, 100000 + stream).standard_normal(nsites)


@dataclass
class ChainShape:
    chain: int
    d: int
    nx: int
    ntau: int

    @property
    def nsites(self) -> int:
        return self.nx ** self.d * self.ntau


def batch_chains(n_chains: int = 64, seed: int = BATCH_SEED,
                 nx_choices=BATCH_NX, ntau_choices=BATCH_NTAU) -> list:
    """Independent d=3 chains of uneven volume: N_x and N_tau drawn uniformly."""
    g = _gen(seed, 4)
    out = []
    for c in range(n_chains):
        nx = int(nx_choices[g.integers(len(nx_choices))])
        nt = int(ntau_choices[g.integers(len(ntau_choices))])
        out.append(ChainShape(c, 3, nx, nt))
    return out


@dataclass
class Request:
    rid: int
    arrival_s: float
    kind: str          # "solve" or "trajectory"
    d: int
    nx: int
    ntau: int
    seed: int

    @property
    def nsites(self) -> int:
        return self.nx ** self.d * self.ntau


def poisson_requests(rate_hz: float, n: int, seed: int = SERVE_SEED,
                     d1_nx=(64, 2048), d1_ntau=(64, 512),
                     d3_nx=(8, 24), d3_ntau=(40, 256)) -> list:
    """A Poisson stream of solve and trajectory requests.

    Gaps are exponential with mean 1/rate; d is 1 or 3 with equal probability,
    sizes are uniform within the ranges (N_tau rounded to a multiple of 8), and
    half the requests are solves, half trajectories."""
    g = _gen(seed, 5)
    t = 0.0
    out = []
    for k in range(n):
        t += g.exponential(1.0 / rate_hz)
        d = 1 if g.random() < 0.5 else 3
        if d == 1:
            nx = int(g.integers(d1_nx[0], d1_nx[1] + 1))
            nt = int(g.integers(d1_ntau[0] // 8, d1_ntau[1] // 8 + 1)) * 8
        else:
            nx = int(g.integers(d3_nx[0], d3_nx[1] + 1))
            nt = int(g.integers(d3_ntau[0] // 8, d3_ntau[1] // 8 + 1)) * 8
        kind = "solve" if g.random() < 0.5 else "trajectory"
        out.append(Request(k, t, kind, d, nx, nt, int(seed * 100003 + k)))
    return out
