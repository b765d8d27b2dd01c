"""Seeded synthetic workloads shared by the oracle tests, the CUDA path and bench.py.

This module holds no arithmetic of the method itself: it only draws the random
numbers a workload needs (interface jitter, point-source locations, Gaussian bump
centres) from a counter-free SplitMix64 stream and packages the problem
parameters.  Both sides receive these numbers as plain inputs.

Workloads (all on the unit square, P1 elements, §2–§3; Dirichlet boundary unless bc = 1, the
first-order absorbing condition du/dn - i k u = 0 on all four sides):

  tiny      k=20,  N=32,   2x2 subdomains, overlap 2, point source at the centre
  k100      k=100, N=320,  4x4 subdomains, overlap 2, centre point source + Gaussian bump
  k200      k=200, N=640,  8x8 subdomains, overlap 2, centre point source + Gaussian bump
  k400x32   k=400, N=1280, 16x16 subdomains with jittered interfaces, 32 point sources
  k200ws    k200 geometry, used for the learned warm start
  k200s     k200 geometry and load with the impedance (Sommerfeld) boundary on all four sides

N is the number of mesh intervals per side (h = 1/N), chosen so that
h ≈ 2π/(k·ppwl) with ppwl ≈ 10 (tiny) or ≈ 20 (the rest), §2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) with 53-bit uniform doubles."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / 9007199254740992.0))


@dataclass
class PointSource:
    x: float
    y: float
    amp: float = 1.0


@dataclass
class Bump:
    """Gaussian g(x) = amp * exp(-|x - c|^2 / (2 sigma^2))."""
    cx: float
    cy: float
    sigma: float = 0.05
    amp: float = 1.0


@dataclass
class RHSSpec:
    points: list = field(default_factory=list)
    bumps: list = field(default_factory=list)


@dataclass
class Workload:
    name: str
    k: float
    N: int
    Sx: int
    Sy: int
    overlap: int
    ifx: list          # interface node indices a_0=0 < ... < a_Sx = N
    ify: list
    rhs: list          # one RHSSpec per right-hand side
    inner_tol: float = 1e-2
    outer_tol: float = 1e-6
    bc: int = 0        # 0: u = 0 on the boundary; 1: impedance (Sommerfeld) on all four sides

    @property
    def h(self) -> float:
        return 1.0 / self.N

    @property
    def n_global(self) -> int:
        return (self.N + 1) ** 2 if self.bc else (self.N - 1) ** 2

    @property
    def ppwl(self) -> float:
        return 2.0 * math.pi * self.N / self.k

    @property
    def nrhs(self) -> int:
        return len(self.rhs)


def uniform_interfaces(N: int, S: int) -> list:
    """a_p = round(p N / S): uniform Cartesian partition (§3)."""
    return [int(math.floor(p * N / S + 0.5)) for p in range(S + 1)]


def jittered_interfaces(N: int, S: int, rng: SplitMix64, frac: float = 0.25) -> list:
    """Interior interfaces moved by U(-frac, frac) of a subdomain width, then rounded."""
    a = [0]
    w = N / S
    for p in range(1, S):
        a.append(int(math.floor(p * w + rng.uniform(-frac, frac) * w + 0.5)))
    a.append(N)
    for p in range(S):
        if a[p + 1] - a[p] < 2:
            raise ValueError("jittered partition produced a degenerate subdomain")
    return a


def point_sources(n: int, rng: SplitMix64, lo: float, hi: float) -> list:
    return [PointSource(rng.uniform(lo, hi), rng.uniform(lo, hi)) for _ in range(n)]


def make(name: str, seed: int = 0) -> Workload:
    """Build one of the named workloads with its seeded random draws."""
    if name == "tiny":
        N, S = 32, 2
        return Workload(name, 20.0, N, S, S, 2, uniform_interfaces(N, S), uniform_interfaces(N, S),
                        [RHSSpec([PointSource(0.5, 0.5)])])
    if name in ("k100", "k200", "k200ws", "k200s"):
        k, N, S = {"k100": (100.0, 320, 4), "k200": (200.0, 640, 8), "k200ws": (200.0, 640, 8),
                   "k200s": (200.0, 640, 8)}[name]
        rng = SplitMix64(seed)
        bump = Bump(rng.uniform(0.2, 0.8), rng.uniform(0.2, 0.8))
        return Workload(name, k, N, S, S, 2, uniform_interfaces(N, S), uniform_interfaces(N, S),
                        [RHSSpec([PointSource(0.5, 0.5)], [bump])], bc=1 if name == "k200s" else 0)
    if name in ("k400x32", "k400x4"):
        # k400x4: the same geometry with the first 4 of the 32 right-hand sides (a batched case
        # small enough for multi-pass profiling)
        N, S = 1280, 16
        rj = SplitMix64(seed)
        ifx = jittered_interfaces(N, S, rj)
        ify = jittered_interfaces(N, S, rj)
        rs = SplitMix64(seed + 1)
        rhs = [RHSSpec([p]) for p in point_sources(32, rs, 0.1, 0.9)]
        return Workload(name, 400.0, N, S, S, 2, ifx, ify, rhs if name == "k400x32" else rhs[:4])
    raise KeyError(name)


def custom(k: float, N: int, S: int, overlap: int = 2, rhs=None, Sy: int | None = None,
           ifx=None, ify=None, name: str = "custom", bc: int = 0) -> Workload:
    Sy = S if Sy is None else Sy
    return Workload(name, k, N, S, Sy, overlap,
                    list(ifx) if ifx is not None else uniform_interfaces(N, S),
                    list(ify) if ify is not None else uniform_interfaces(N, Sy),
                    rhs if rhs is not None else [RHSSpec([PointSource(0.5, 0.5)])], bc=bc)


def random_complex(n: int, seed: int):
    """Seeded complex test vector with entries uniform in [-1,1] + i[-1,1] (numpy complex128)."""
    import numpy as np
    rng = SplitMix64(seed)
    out = np.empty(n, dtype=np.complex128)
    for t in range(n):
        out[t] = complex(rng.uniform(-1.0, 1.0), rng.uniform(-1.0, 1.0))
    return out


def random_complex_fast(n: int, seed: int):
    """Seeded complex vector for large n (numpy PCG64; not shared with any C generator)."""
    import numpy as np
    g = np.random.default_rng(seed)
    return (g.uniform(-1, 1, n) + 1j * g.uniform(-1, 1, n)).astype(np.complex128)
