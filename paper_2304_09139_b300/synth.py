"""Seeded synthetic inputs shaped like the paper's workloads (random initial conditions).

This module holds no arithmetic of the method: it only draws numbers.  Both the CUDA path and the
oracle's tests take their inputs from here, so it imports neither.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014): state += 0x9E3779B97F4A7C15, then two xor-shift-multiply rounds.  The i-th output
(i = 0, 1, ...) of a stream seeded with s is mix(s + (i + 1) * gamma), so a whole stream is one
vectorised numpy expression.

Positions: i.i.d. uniform fractional coordinates s = (u >> 11) * 2**-53 in [0, 1), drawn in
row-major [N][d] order, low word 0.  The paper starts from "random initial conditions ... a Poisson
point process" (Simulations); at fixed N that is the binomial process drawn here.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """First `count` outputs of a SplitMix64 stream seeded with `seed` (uint64 array)."""
    with np.errstate(over="ignore"):
        i = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits: (u >> 11) * 2**-53."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def positions(seed: int, N: int, d: int) -> np.ndarray:
    """Fractional positions s (float64 [N, d], low word zero) of N uniform points in the unit cell."""
    return uniform01(seed, N * d).reshape(N, d)


def box_length_unit_density(N: int, d: int) -> float:
    """Side L of the periodic box that holds N points at number density 1."""
    return float(N) ** (1.0 / d)


@dataclasses.dataclass(frozen=True)
class Config:
    """One configuration: dimension, particle count, box side, and chi or K, plus the position seed."""
    d: int
    N: int
    L: float
    chi: float
    seed: int
    K: float = 0.0


# The three single-configuration workloads.  The first is small enough for the oracle to minimise in
# seconds; the second and third are the throughput and staging workloads.
SMALL_D2 = Config(d=2, N=100, L=1.0, chi=0.30, seed=1)
MEDIUM_D2 = Config(d=2, N=10_000, L=100.0, chi=0.45, seed=2)
LARGE_D3 = Config(d=3, N=32_768, L=32.0, chi=0.40, seed=3)
# four axes at unit density: N = 4096 in a box of side 8, M = 4914
MEDIUM_D4 = Config(d=4, N=4096, L=8.0, chi=0.30, seed=44)
# The paper's own size (d = 2, N = 2 x 10^6, unit density) at its smallest and largest chi: M = 400000 and
# 1600000 wavevectors.
PAPER_D2 = Config(d=2, N=2_000_000, L=math.sqrt(2_000_000.0), chi=0.10, seed=6)
# a tenth of the paper's N at chi = 0.10 (M = 40000): the largest quench that fits a benchmark run
PAPER_D2_TENTH = Config(d=2, N=200_000, L=math.sqrt(200_000.0), chi=0.10, seed=61)
PAPER_D2_CHI40 = Config(d=2, N=2_000_000, L=math.sqrt(2_000_000.0), chi=0.40, seed=7)


def _loguniform_int(u: float, lo: int, hi: int) -> int:
    return int(round(math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))))


def mixed_batch(master_seed: int = 4, count: int = 256, n_lo: int = 64, n_hi: int = 8192,
                chi_lo: float = 0.10, chi_hi: float = 0.49, dims=(2, 3)) -> list[Config]:
    """Independent configurations: d uniform over `dims`, N log-uniform in [n_lo, n_hi], chi uniform in
    [chi_lo, chi_hi], unit density, one position sub-seed each (the batched workload)."""
    u = uniform01(master_seed, 4 * count).reshape(count, 4)
    out = []
    for i in range(count):
        d = dims[min(int(u[i, 0] * len(dims)), len(dims) - 1)]
        N = _loguniform_int(u[i, 1], n_lo, n_hi)
        chi = chi_lo + (chi_hi - chi_lo) * u[i, 2]
        seed = int(splitmix64(master_seed * 1_000_003 + i, 1)[0])
        out.append(Config(d=d, N=N, L=box_length_unit_density(N, d), chi=float(chi), seed=seed))
    return out


def poisson_arrivals(master_seed: int, count: int, mean_interval_s: float) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: cumulative sums of exponential gaps with the given mean."""
    u = uniform01(master_seed ^ 0x5DEECE66D, count)
    return np.cumsum(-mean_interval_s * np.log1p(-u))


def serving_requests(master_seed: int = 5, count: int = 2000, mean_interval_s: float = 0.020):
    """Ensemble requests: d in {1,2,3}, N log-uniform in [64, 32768], chi in [0.10, 0.49], Poisson arrivals."""
    cfgs = mixed_batch(master_seed, count, n_lo=64, n_hi=32768, dims=(1, 2, 3))
    return cfgs, poisson_arrivals(master_seed, count, mean_interval_s)
