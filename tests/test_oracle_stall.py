"""Oracle pins of the optional stall rule of the fixed-point sweeps (``als_stall_tol``).

The rule reads Section 3.3's fixed point "until the mode stops changing" with the paper's
absolute example test (the change of the rank-1 term in the units of the field): a mode
whose change, relative to the step's leading mode, is below ``als_stall_tol`` and no longer
shrinking ends its sweeps.  It exists for arithmetic with a rounding floor (the tensor-core
contraction's FP32 sums).  The pins:

* without a floor (plain FP64) the rule never fires on these runs: the result is bitwise that
  of the run without it;
* with a floor planted in the oracle (every nonlinear projection perturbed by 2^-24 relative,
  the unit roundoff of FP32), the run without the rule spends its trailing mode's sweeps up to
  I_max against that floor, the run with it stops those modes (counted as stalled, and the
  step flagged as not converged), and both fields are equally close to the floor-free field.
"""
import numpy as np
import pytest

import workloads
from oracle import ctd as octd


def problem(w, **over):
    p = octd.Problem(dim=w.dim, n=w.n, length=w.length, s=w.s, p=w.p, a=w.a, L=w.L, kappa=w.kappa,
                     a0=w.a0, alpha=w.alpha, dt=w.dt, M_max=w.M_max, I_max=w.I_max, tol_als=w.tol_als,
                     tol_enrich=w.tol_enrich, seed=w.seed)
    for k, v in over.items():
        setattr(p, k, v)
    return p


def run(w, nsteps, **over):
    prob = problem(w, **over)
    ops = octd.build_operators(prob)
    A = workloads.initial_modes(w)
    hist = []
    for k in range(nsteps):
        A, st = octd.step(prob, ops, A, k)
        hist.append(st)
    return A, hist


def planted_floor(monkeypatch, level, seed=0):
    """Every nonlinear projection of the oracle comes back perturbed by `level` relative."""
    rng = np.random.default_rng(seed)
    orig = octd.nonlinear_projection

    def noisy(prob, ops, nl, v, x):
        r = orig(prob, ops, nl, v, x)
        return r * (1.0 + level * rng.uniform(-1.0, 1.0, size=r.shape))

    monkeypatch.setattr(octd, "nonlinear_projection", noisy)


CASES = [dict(), dict(n=(96, 80), s=2, p=2, eps=0.03)]


@pytest.mark.parametrize("over", CASES)
def test_rule_is_inert_in_exact_fp64(over):
    w = workloads.preset("c0", **over)
    A0, h0 = run(w, 3)
    A1, h1 = run(w, 3, als_stall_tol=1e-6)
    for a, b in zip(A0, A1):
        assert np.array_equal(a, b)
    assert [h["als_iters"] for h in h0] == [h["als_iters"] for h in h1]
    assert all(h["als_stalled"] == 0 for h in h0 + h1)


@pytest.mark.parametrize("over", CASES)
def test_rule_ends_sweeps_at_a_rounding_floor(monkeypatch, over):
    w = workloads.preset("c0", **over)
    A_ref, h_ref = run(w, 3)
    planted_floor(monkeypatch, 2.0 ** -24, seed=1)
    A_off, h_off = run(w, 3)
    planted_floor(monkeypatch, 2.0 ** -24, seed=1)
    A_on, h_on = run(w, 3, als_stall_tol=1e-6)
    sweeps = lambda h: [sum(s["als_iters"]) for s in h]
    # the floor costs sweeps without the rule (a mode runs to I_max against it) ...
    assert sum(sweeps(h_off)) > sum(sweeps(h_ref)) + 20, (sweeps(h_off), sweeps(h_ref))
    assert any(w.I_max in s["als_iters"] for s in h_off[1:])
    assert all(s["als_stalled"] == 0 for s in h_off)
    # ... the rule stops the stalled modes, counts them and flags the step
    assert sum(s["als_stalled"] for s in h_on) >= 2
    assert all(s["als_not_converged"] for s in h_on if s["als_stalled"])
    assert sum(sweeps(h_on)) <= sum(sweeps(h_ref)) + 6, (sweeps(h_on), sweeps(h_ref))
    assert [s["modes"] for s in h_on] == [s["modes"] for s in h_ref]
    # and the field stays as close to the floor-free one as the run without the rule
    e_off = octd.rel_l2_between(A_off, A_ref)
    e_on = octd.rel_l2_between(A_on, A_ref)
    assert e_on < 1e-8 and e_off < 1e-8, (e_on, e_off)
    assert e_on < 2.0 * e_off + 1e-9, (e_on, e_off)
