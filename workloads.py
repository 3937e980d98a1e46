"""Seeded synthetic workloads shared by the oracle checks, the GPU tests and the benchmark.

This module holds the run parameters and the initial conditions only: nodal samples of
seeded 1D functions.  It contains none of the method's arithmetic (no shape functions,
operators, contractions or solves) and imports neither ``oracle`` nor the CUDA package.

The paper's own initial fields are random and not published; these stand in for them.
Parametrisation: runs are specified as ``u_t = eps^2 Lap u - (u^3 - u)`` with stabiliser
``S``; in the paper's symbols (Eq. AC, Eq. energyfunction, Eq.
AC-discrete-semi-stable) this is ``L = 1, kappa = eps^2, a0 = 1/4, alpha = S``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64Stream:
    """Sequential SplitMix64 stream (state += golden gamma; output = finaliser(state))."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))


@dataclasses.dataclass
class Workload:
    """One Allen-Cahn run: grid, C-FEM parameters, PDE coefficients, stopping rules."""
    name: str
    dim: int
    n: Sequence[int]
    length: Sequence[float]
    s: int
    p: int
    a: float
    eps: float
    S: float
    dt: float
    steps: int
    M_max: int
    I_max: int
    tol_als: float
    tol_enrich: float
    seed: int
    ic_rank: int
    ic_k: int
    ic_tanh: bool = False

    # paper symbols (Table coef): mobility, gradient coefficient, energy coefficient, stabiliser
    @property
    def L(self) -> float:
        return 1.0

    @property
    def kappa(self) -> float:
        return self.eps ** 2

    @property
    def a0(self) -> float:
        return 0.25

    @property
    def alpha(self) -> float:
        return self.S

    @property
    def grid_points(self) -> int:
        return int(np.prod(self.n))


def cosine_modes(n: Sequence[int], length: Sequence[float], rank: int, kmax: int, seed: int,
                 amp: float = 0.1) -> List[np.ndarray]:
    """Rank-``rank`` separated initial condition; factor ``(r, d)`` is the nodal sample of
    ``amp * sum_{k=1..kmax} a_k cos(k pi x / length_d)``, ``a_k ~ U(-1, 1)`` drawn from
    one SplitMix64 stream in the order mode -> dimension -> k."""
    rng = SplitMix64Stream(seed)
    D = len(n)
    out = [np.zeros((n[d], rank)) for d in range(D)]
    for r in range(rank):
        for d in range(D):
            x = np.linspace(0.0, length[d], n[d])
            f = np.zeros(n[d])
            for k in range(1, kmax + 1):
                ak = rng.uniform(-1.0, 1.0)
                f += ak * np.cos(k * math.pi * x / length[d])
            out[d][:, r] = amp * f
    return out


def tanh_mode(n: Sequence[int], length: Sequence[float], eps: float) -> List[np.ndarray]:
    """``tanh((x - length/2) / (sqrt(2) eps)) (x) 1 (x) 1`` as one separated mode."""
    D = len(n)
    x = np.linspace(0.0, length[0], n[0])
    out = [np.tanh((x - 0.5 * length[0]) / (math.sqrt(2.0) * eps))[:, None]]
    for d in range(1, D):
        out.append(np.ones((n[d], 1)))
    return out


def initial_modes(w: Workload) -> List[np.ndarray]:
    modes = cosine_modes(w.n, w.length, w.ic_rank, w.ic_k, w.seed)
    if w.ic_tanh:
        t = tanh_mode(w.n, w.length, w.eps)
        modes = [np.concatenate([modes[d], t[d]], axis=1) for d in range(w.dim)]
    return modes


def preset(name: str, **overrides) -> Workload:
    """Named runs.  ``c0``..``c3``: the single-instance configurations (2D 64^2, 2D 4096^2,
    3D 512^3, 3D 1024^3); the ALS tolerance 1e-8 and enrichment tolerance 1e-4 apply to all
    (the paper suggests eps2 = O(1e-4))."""
    base = dict(length=None, a=12.0, S=2.0, I_max=50, tol_als=1e-8, tol_enrich=1e-4)
    table = {
        "c0": dict(dim=2, n=(64, 64), s=1, p=1, eps=0.05, dt=0.01, steps=100, M_max=20,
                   seed=0, ic_rank=4, ic_k=4),
        "c1": dict(dim=2, n=(4096, 4096), s=2, p=2, eps=0.01, dt=1e-3, steps=1000, M_max=50,
                   seed=1, ic_rank=8, ic_k=4),
        # c1 from a phase-separated state: one straight interface (tanh profile) across x
        "c1i": dict(dim=2, n=(4096, 4096), s=2, p=2, eps=0.01, dt=1e-3, steps=1000, M_max=50,
                    seed=1, ic_rank=0, ic_k=4, ic_tanh=True),
        "c2": dict(dim=3, n=(512, 512, 512), s=2, p=2, eps=0.02, dt=5e-3, steps=500,
                   M_max=60, seed=2, ic_rank=6, ic_k=6, ic_tanh=True),
        "c3": dict(dim=3, n=(1024, 1024, 1024), s=3, p=3, eps=0.01, dt=2e-3, steps=200,
                   M_max=80, seed=3, ic_rank=10, ic_k=4),
    }
    cfg = dict(base)
    cfg.update(table[name])
    cfg.update(overrides)
    if cfg["length"] is None:
        cfg["length"] = tuple(1.0 for _ in range(cfg["dim"]))
    return Workload(name=name, **cfg)


def batch_instances(count: int, seed: int, n_choices=(256, 512, 1024, 2048),
                    eps_range=(0.01, 0.05), cap_range=(8, 40)) -> List[Workload]:
    """The batched 2D workload: per instance n, eps, mode cap and IC seed drawn from one
    SplitMix64 stream."""
    rng = SplitMix64Stream(seed)
    out = []
    for i in range(count):
        n = n_choices[int(rng.next_u64() % len(n_choices))]
        eps = rng.uniform(*eps_range)
        cap = cap_range[0] + int(rng.next_u64() % (cap_range[1] - cap_range[0] + 1))
        out.append(Workload(name=f"batch{i}", dim=2, n=(n, n), length=(1.0, 1.0), s=2, p=2,
                            a=12.0, eps=eps, S=2.0, dt=1e-3, steps=300, M_max=cap, I_max=50,
                            tol_als=1e-8, tol_enrich=1e-4, seed=int(rng.next_u64() & 0x7fffffff),
                            ic_rank=4, ic_k=4))
    return out
