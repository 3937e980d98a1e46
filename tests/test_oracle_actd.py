"""Pins for the oracle's adaptive CTD (Section 3.3 "Adaptivity": switch to a full-grid C-FEM
step when the mode count exceeds M_c) against the brute-force dense full-grid solve, the
factor form of the same right-hand side, and the scheme's invariants."""
import numpy as np
import pytest

import workloads
from oracle import actd, cfem, ctd, fullgrid


def make_problem(dim=2, n=9, s=2, p=2, eps=0.05, S=2.0, dt=0.01, **kw):
    args = dict(dim=dim, n=(n,) * dim, length=(1.0,) * dim, s=s, p=p, a=12.0, L=1.0,
                kappa=eps ** 2, a0=0.25, alpha=S, dt=dt, M_max=30, I_max=200, tol_als=1e-10,
                tol_enrich=1e-8, seed=0)
    args.update(kw)
    return ctd.Problem(**args)


@pytest.mark.parametrize("dim,n,rule", [(2, 9, "nodal"), (2, 8, "gauss"), (3, 5, "nodal"),
                                        (3, 4, "gauss")])
def test_fast_diagonalisation_equals_dense_full_grid_solve(dim, n, rule):
    prob = make_problem(dim=dim, n=n, quad_rule=rule, quad_q=3)
    ops = ctd.build_operators(prob)
    U = ctd.reconstruct(workloads.cosine_modes(prob.n, prob.length, 3, 4, 7, amp=0.9))
    got = actd.cfe_step(prob, ops, U)
    ref = fullgrid.step(prob, ops, U)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_eigenpairs_are_mass_orthonormal_and_start_at_zero():
    # K is singular with the constants as null space (Neumann), so lambda_0 = 0
    prob = make_problem(n=10)
    ops = ctd.build_operators(prob)
    lam, V = actd.eigenpairs(ops, 0)
    M, K = ops.M[0].toarray(), ops.K[0].toarray()
    assert np.max(np.abs(V.T @ M @ V - np.eye(10))) < 1e-12
    assert np.max(np.abs(K @ V - M @ V * lam)) < 1e-10 * np.max(np.abs(lam))
    assert abs(lam[0]) < 1e-10 * lam[-1] and np.all(lam[1:] > 0)


@pytest.mark.parametrize("rule", ["nodal", "gauss"])
def test_grid_source_gives_the_factor_right_hand_side(rule):
    # a half-sweep from u^k on the full grid (no factors) equals the one from its factors
    prob = make_problem(n=9, quad_rule=rule, quad_q=3)
    ops = ctd.build_operators(prob)
    A = workloads.cosine_modes(prob.n, prob.length, 3, 3, 4, amp=0.8)
    rng = np.random.default_rng(1)
    v = [rng.standard_normal(9) for _ in range(2)]
    B = [0.3 * rng.standard_normal((9, 2)) for _ in range(2)]
    empty = [np.zeros((9, 0)) for _ in range(2)]
    G = ("grid", actd.grid_source(prob, ops, ctd.reconstruct(A)))
    for x in range(2):
        ref, ab_ref = ctd.half_sweep(prob, ops, x, list(v), A, B, ctd.nonlinear_operator(prob, ops, A))
        got, ab = ctd.half_sweep(prob, ops, x, list(v), empty, B, G)
        assert ab == ab_ref
        assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_no_switch_below_the_critical_mode_count_is_plain_ctd():
    prob = make_problem(n=10)
    ops = ctd.build_operators(prob)
    A = workloads.cosine_modes(prob.n, prob.length, 2, 2, 3, amp=0.8)
    state, st = actd.step(prob, ops, ("modes", A), M_c=50, step_index=0)
    B, st_ref = ctd.step(prob, ops, A, 0)
    assert state[0] == "modes" and not st["switched"]
    assert st["modes"] == st_ref["modes"]
    for d in range(2):
        assert np.array_equal(state[1][d], B[d])


def test_switch_above_the_critical_mode_count_gives_the_full_grid_step():
    prob = make_problem(n=10)
    ops = ctd.build_operators(prob)
    A = workloads.cosine_modes(prob.n, prob.length, 4, 4, 3, amp=0.9)
    _, st_ctd = ctd.step(prob, ops, A, 0)
    M_c = 2
    assert st_ctd["modes"] > M_c
    state, st = actd.step(prob, ops, ("modes", A), M_c=M_c, step_index=0)
    assert state[0] == "grid" and st["switched"] and st["ctd_modes_tried"] == M_c + 1
    ref = fullgrid.step(prob, ops, ctd.reconstruct(A))
    assert np.max(np.abs(state[1] - ref)) < 1e-12 * np.max(np.abs(ref))


def test_ctd_step_from_a_grid_state_converges_to_the_full_grid_solution():
    # after a switch the next step runs CTD from u^k on the full grid; with enough modes it
    # reaches that step's full-grid solution (Section 3.2)
    prob = make_problem(n=8, M_max=20, I_max=300, tol_als=1e-12, tol_enrich=1e-15)
    ops = ctd.build_operators(prob)
    U0 = ctd.reconstruct(workloads.cosine_modes(prob.n, prob.length, 3, 4, 11, amp=0.8))
    state, st = actd.step(prob, ops, ("grid", U0), M_c=40, step_index=1)
    assert state[0] == "modes" and not st["switched"]
    U1 = fullgrid.step(prob, ops, U0)
    err = np.linalg.norm(ctd.reconstruct(state[1]) - U1) / np.linalg.norm(U1)
    assert err < 1e-12


def test_actd_run_alternates_and_keeps_the_energy_law():
    # a rich start (|u| <= 0.9, where the stabiliser bound holds) switches on the first steps;
    # diffusion then simplifies the field and CTD takes over.  Every step's energy is
    # non-increasing (exact on CFE steps, up to the CTD tolerances otherwise).
    prob = make_problem(n=16, s=1, p=1, eps=0.2, dt=1.0, tol_als=1e-10, tol_enrich=1e-3)
    ops = ctd.build_operators(prob)
    A0 = workloads.cosine_modes(prob.n, prob.length, 5, 5, 9, amp=0.9)
    A0[0] = A0[0] * (0.9 / np.max(np.abs(ctd.reconstruct(A0))))
    state = ("modes", A0)
    E = actd.energy(prob, ops, state)
    kinds = []
    for k in range(5):
        U = actd.field(state)
        state, st = actd.step(prob, ops, state, M_c=4, step_index=k)
        kinds.append(state[0])
        if st["switched"]:
            ref = fullgrid.step(prob, ops, U)
            assert np.max(np.abs(state[1] - ref)) < 1e-12 * np.max(np.abs(ref))
        else:
            assert st["modes"] <= 4
        E1 = actd.energy(prob, ops, state)
        assert E1 <= E + 1e-10 * abs(E)
        E = E1
    assert kinds == ["grid", "grid", "modes", "modes", "modes"]
