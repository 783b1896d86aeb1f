"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

This module holds no arithmetic of the lattice Boltzmann method: it draws
random numbers and states the workload shapes.  Equilibria, weights and rates
always come from the side under test (the oracle or the CUDA library).
"""
from __future__ import annotations

import numpy as np

SEEDS = (1, 2, 3, 4, 5)


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def perturb(r: np.random.Generator, base: np.ndarray, spread: float = 0.2) -> np.ndarray:
    """base * (1 + U(-spread, spread)), element-wise."""
    return base * (1.0 + r.uniform(-spread, spread, size=base.shape))


def force(r: np.random.Generator, scale: float = 1e-3) -> tuple[float, float]:
    fx, fy = r.uniform(-scale, scale, size=2)
    return float(fx), float(fy)


def velocity(r: np.random.Generator, scale: float = 0.1) -> tuple[float, float]:
    ux, uy = r.uniform(-scale, scale, size=2)
    return float(ux), float(uy)


def rates(r: np.random.Generator, lo: float = 0.2, hi: float = 1.8, tied: bool = True) -> np.ndarray:
    """Relaxation rates s_0..s_8; with ``tied`` s4 = s5 and s6 = s7 as in the paper."""
    s = np.zeros(9)
    s[3:] = r.uniform(lo, hi, size=6)
    if tied:
        s[5] = s[4]
        s[7] = s[6]
    return s


# Workload shapes (sizes, Knudsen numbers, drives), shaped after the paper's
# Sec. 3.1 periodic channel and Sec. 3.2 L/H = 100 pressure-driven channel.
PERIODIC_4x32 = dict(nx=4, ny=32, kn=0.1, a=2.0, sigma=1.0, gx=1e-6)
PRESSURE_1601x16 = dict(nx=1601, ny=16, ratio=2.0, kn_out=(0.0194, 0.05, 0.1, 0.2))
PRESSURE_25601x256 = dict(nx=25601, ny=256, ratio=2.47, kn_out=0.1)
BATCH_48 = dict(n=48, nx=4, ny_cycle=(16, 32, 64, 128), kn_lo=0.01, kn_hi=10.0, gx=1e-6)
