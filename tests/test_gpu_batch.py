"""Batched time steps (ctd_step_batch, one CTA per instance) against the FP64 oracle:
instances of different sizes, C-FEM orders and arithmetic in one launch per step.  The FP64
instances must match the oracle within 1e-12 (u and energy) with the same mode and sweep
counts; the split-BF16 instance within 1e-5, the mixed-precision bar."""
import numpy as np
import pytest

import workloads
from oracle import ctd as octd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_15519_gb300 import build, ctd
    build.build()
    return ctd


def oracle_problem(w):
    return octd.Problem(dim=w.dim, n=w.n, length=w.length, s=w.s, p=w.p, a=w.a, L=w.L, kappa=w.kappa,
                        a0=w.a0, alpha=w.alpha, dt=w.dt, M_max=w.M_max, I_max=w.I_max, tol_als=w.tol_als,
                        tol_enrich=w.tol_enrich, seed=w.seed)


CASES = [
    (dict(), "fp64", 1e-12),
    (dict(n=(77, 130), s=2, p=2, eps=0.04, M_max=12, seed=3), "fp64", 1e-12),
    (dict(n=(100, 100), s=3, p=3, eps=0.05, M_max=10, seed=5), "fp64", 1e-12),
    (dict(n=(96, 64), seed=7), "mixed", 1e-5),
]


def test_batch_matches_oracle(lib):
    nsteps = 3
    ws = [workloads.preset("c0", **over) for over, _, _ in CASES]
    solvers = []
    for w, (_, prec, _) in zip(ws, CASES):
        cfg = lib.config_from_workload(w, precision=lib.PREC_FP64 if prec == "fp64" else lib.PREC_SPLIT_BF16)
        s = lib.Solver(cfg)
        s.set_initial_modes(workloads.initial_modes(w))
        solvers.append(s)
    stats = lib.step_batch(solvers, nsteps)
    for w, s, st, (_, prec, tol) in zip(ws, solvers, stats, CASES):
        prob = oracle_problem(w)
        ops = octd.build_operators(prob)
        A = workloads.initial_modes(w)
        for k in range(nsteps):
            A, so = octd.step(prob, ops, A, k)
            if prec == "fp64":
                assert st[k]["modes"] == so["modes"], (w.n, k, st[k], so["modes"])
                assert st[k]["als_sweeps"] == sum(so["als_iters"]), (w.n, k, st[k])
        G = s.get_modes()
        assert octd.rel_l2_between(G, A) < tol, (w.n, prec, octd.rel_l2_between(G, A))
        eo = octd.energy(prob, ops, A)
        assert abs(s.energy() - eo) / abs(eo) < tol, (w.n, prec)
        s.close()


def test_batch_then_single_steps_continue(lib):
    # an instance stepped in a batch continues with ctd_step from the new state
    w = workloads.preset("c0")
    a = lib.Solver(lib.config_from_workload(w))
    b = lib.Solver(lib.config_from_workload(w))
    for s in (a, b):
        s.set_initial_modes(workloads.initial_modes(w))
    lib.step_batch([a], 2)
    a.step(1)
    b.step(3)
    Ga, Gb = a.get_modes(), b.get_modes()
    assert octd.rel_l2_between(Ga, Gb) < 1e-12
    a.close()
    b.close()
