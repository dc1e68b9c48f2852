"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the method: only the workload shapes
(grid sizes, the non-dimensional groups T, C, M, Fe, the magic parameter,
step budgets), seeded random draws (splitmix64, Steele, Lea & Flood 2014) and
random population arrays for state-level parity tests.  Both the CUDA path
and the oracle receive exactly these numbers as inputs.

The paper's workloads are synthetic channels (Sec. IV.4 and V.2 of
arXiv:1812.05711): Lx/H ~ 1.22, C = 10, M = 10, Fe = 4000; the grids below
keep that aspect ratio with power-of-two Nx (Ny = 8 round(0.82 Nx / 8)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64(state: int):
    """One step of splitmix64: returns (new_state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


def uniforms(seed: int, n: int):
    """n doubles in [0, 1) from splitmix64 (top 53 bits)."""
    s = seed & MASK64
    out = []
    for _ in range(n):
        s, z = splitmix64(s)
        out.append((z >> 11) * (1.0 / (1 << 53)))
    return out


def ny_for(nx: int) -> int:
    """Ny = 8 round(0.82 Nx / 8): 64->56, 128->104, 256->208, 512->416, 1024->840, 2048->1680."""
    return 8 * int(round(0.82 * nx / 8))


@dataclass
class Workload:
    name: str
    Nx: int
    Ny: int
    T: float
    C: float = 10.0
    M: float = 10.0
    Fe: float = 4000.0
    Lambda: float = 0.25
    steps: int = 1000
    amp: list = field(default_factory=list)     # Eq. 29 mode amplitudes (units of u_ion)
    phase: list = field(default_factory=list)   # Eq. 29 mode x-phases (radians)

    def args(self):
        return (self.Nx, self.Ny, self.T, self.C, self.M, self.Fe, self.Lambda)


def roll(seed: int, amplitude: float):
    """A single Eq. 29 roll with a seeded x-phase."""
    (u,) = uniforms(seed, 1)
    return [amplitude], [2 * math.pi * u]


def random_modes(seed: int, amplitude: float, n_modes: int = 16):
    """Modes 1..n with amplitudes U[-1,1]*amplitude and seeded phases."""
    u = uniforms(seed, 2 * n_modes)
    amp = [(2 * u[2 * k] - 1) * amplitude for k in range(n_modes)]
    phase = [2 * math.pi * u[2 * k + 1] for k in range(n_modes)]
    return amp, phase


def plain_fp64_channel() -> Workload:
    """128 x 104 plain FP64 single run, T = 200, Eq. 29 roll 1e-3, seed 1."""
    a, p = roll(1, 1e-3)
    return Workload("channel-128x104-T200", 128, 104, 200.0, steps=10000, amp=a, phase=p)


def large_channel() -> Workload:
    """2048 x 1680 channel, T ~ U[150, 250] (seed 2), random modes 1e-4 (seed 2)."""
    (u,) = uniforms(2, 1)
    a, p = random_modes(2, 1e-4)
    return Workload("channel-2048x1680", 2048, 1680, 150.0 + 100.0 * u, steps=2000, amp=a, phase=p)


def precision_channel() -> Workload:
    """1024 x 840 channel, T = 170, Eq. 29 roll 1e-3, seed 3."""
    a, p = roll(3, 1e-3)
    return Workload("channel-1024x840-T170", 1024, 840, 170.0, steps=5000, amp=a, phase=p)


def small_channel(Nx=32, seed=7, T=200.0) -> Workload:
    a, p = roll(seed, 1e-3)
    return Workload(f"channel-{Nx}x{ny_for(Nx)}", Nx, ny_for(Nx), T, amp=a, phase=p)


def random_populations(Nx: int, Ny: int, seed: int, centre: float, spread: float):
    """Random [9][Ny][Nx] arrays centre * (1 + spread * U[-1, 1]) (numpy PCG64)."""
    rng = np.random.default_rng(seed)
    return centre * (1.0 + spread * rng.uniform(-1.0, 1.0, size=(9, Ny, Nx)))


def batch_workloads(seed: int = 4, n: int = 64):
    """64 runs: Nx from {64,128,256,512}, T a seeded shuffle of linspace(140,260),
    C from {5,10,20}, Fe from {2000,4000}, M = 10."""
    rng = np.random.default_rng(seed)
    nxs = rng.choice([64, 128, 256, 512], size=n)
    Ts = rng.permutation(np.linspace(140.0, 260.0, n))
    Cs = rng.choice([5.0, 10.0, 20.0], size=n)
    Fes = rng.choice([2000.0, 4000.0], size=n)
    out = []
    for k in range(n):
        a, p = roll(1000 + k, 1e-3)
        out.append(Workload(f"batch-{k}", int(nxs[k]), ny_for(int(nxs[k])), float(Ts[k]), C=float(Cs[k]),
                            Fe=float(Fes[k]), steps=3000, amp=a, phase=p))
    return out


def serving_stream(seed: int = 5, n: int = 600, rate: float = 20.0):
    """Poisson arrivals (mean `rate` per second) of stability-sweep requests."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    reqs = []
    for k in range(n):
        nx = int(rng.choice([128, 256, 512, 1024]))
        a, p = roll(2000 + k, 1e-3)
        w = Workload(f"req-{k}", nx, ny_for(nx), float(rng.uniform(100.0, 300.0)),
                     C=float(rng.choice([1.0, 10.0, 100.0])), steps=int(rng.integers(1000, 20001)),
                     amp=a, phase=p)
        reqs.append((float(t[k]), w))
    return reqs
