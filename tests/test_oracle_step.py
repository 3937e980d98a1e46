"""Pins for the oracle's CTD step (Section 3.3, Eq. KxQx, App. D) and energy (Eq.
energylaw, App. A) against a brute-force full-grid solve, closed forms and invariants."""
import json
import math
import os

import numpy as np
import pytest

import workloads
from oracle import cfem, ctd, fullgrid, splitmix

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def make_problem(dim=2, n=10, s=1, p=1, eps=0.05, S=2.0, dt=0.01, **kw):
    args = dict(dim=dim, n=(n,) * dim, length=(1.0,) * dim, s=s, p=p, a=12.0, L=1.0,
                kappa=eps ** 2, a0=0.25, alpha=S, dt=dt, M_max=20, I_max=50, tol_als=1e-8,
                tol_enrich=1e-4, seed=0)
    args.update(kw)
    return ctd.Problem(**args)


def test_splitmix_published_vectors():
    # Reference outputs of the SplitMix64 generator for seeds 0 and 1234567.
    r = workloads.SplitMix64Stream(1234567)
    assert [r.next_u64() for _ in range(3)] == [6457827717110365317, 3203168211198807973,
                                                9817491932198370423]
    assert workloads.SplitMix64Stream(0).next_u64() == 0xE220A8397B1DCDAF
    # the oracle's counter form uses the same finaliser
    assert splitmix.mix64(0) == 0xE220A8397B1DCDAF
    v = splitmix.mode_init_vector(7, 3, 2, 1, 50)
    assert np.all((v >= 0.5) & (v < 1.5))


def test_rel_change_equals_brute_force_tensor_norm():
    rng = np.random.default_rng(0)
    for D in (2, 3):
        new = [rng.standard_normal(5 + d) for d in range(D)]
        old = [x + 1e-3 * rng.standard_normal(x.shape) for x in new]

        def full(f):
            T = f[0]
            for y in f[1:]:
                T = np.multiply.outer(T, y)
            return T
        ref = np.linalg.norm(full(new) - full(old)) / np.linalg.norm(full(new))
        assert ctd.rel_change(new, old) == pytest.approx(ref, rel=1e-10)


@pytest.mark.parametrize("dim,n,s,p,tol,bound", [(2, 8, 1, 1, 1e-12, 1e-10), (2, 7, 2, 2, 1e-12, 1e-10),
                                                  (3, 4, 1, 1, 1e-10, 1e-6)])
def test_ctd_converges_to_full_grid_solution(dim, n, s, p, tol, bound):
    prob = make_problem(dim=dim, n=n, s=s, p=p, M_max=n ** (dim - 1) * 4, I_max=3000,
                        tol_als=tol, tol_enrich=1e-15)
    ops = ctd.build_operators(prob)
    A = workloads.cosine_modes(prob.n, prob.length, 3, 4, 11, amp=0.8)
    B, st = ctd.step(prob, ops, A, 0)
    U1 = fullgrid.step(prob, ops, ctd.reconstruct(A))
    err = np.linalg.norm(ctd.reconstruct(B) - U1) / np.linalg.norm(U1)
    assert err < bound


def test_more_modes_approach_full_grid_monotonically():
    # Section 4.1 / Fig. ctd_m: the CTD solution approaches CFE as modes are added.
    prob = make_problem(n=12, I_max=400, tol_als=1e-12, tol_enrich=0.0)
    ops = ctd.build_operators(prob)
    A = workloads.cosine_modes(prob.n, prob.length, 4, 4, 3, amp=0.8)
    U1 = fullgrid.step(prob, ops, ctd.reconstruct(A))
    errs = []
    for M in (1, 2, 4, 8):
        prob.fixed_modes = M
        prob.fixed_als_iters = 0
        prob.M_max = M
        B, _ = ctd.step(prob, ops, A, 0)
        errs.append(np.linalg.norm(ctd.reconstruct(B) - U1) / np.linalg.norm(U1))
    assert all(b < a for a, b in zip(errs, errs[1:]))


def test_linear_separable_eigenpair_is_reproduced_exactly():
    # a0 = 0 removes w; an initial condition phi_x (x) phi_y made of generalised
    # eigenvectors (K phi = lambda M phi) decays by c_t / (c_t + c_k (lx + ly)) in one mode.
    prob = make_problem(n=14, s=2, p=2, a0=0.0, kappa=0.01, tol_als=1e-12)
    ops = ctd.build_operators(prob)
    import scipy.linalg as sla
    lam, vecs = [], []
    for d, idx in ((0, 2), (1, 3)):
        ev, V = sla.eigh(ops.K[d].toarray(), np.diag(ops.omega[d]))
        lam.append(ev[idx])
        vecs.append(V[:, idx])
    A = [vecs[0][:, None], vecs[1][:, None]]
    B, st = ctd.step(prob, ops, A, 0)
    factor = prob.c_t / (prob.c_t + prob.c_k * (lam[0] + lam[1]))
    assert st["modes"] == 1
    ref = factor * np.outer(vecs[0], vecs[1])
    assert np.max(np.abs(ctd.reconstruct(B) - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("c", [0.3, -0.7, 1.0])
def test_constant_state_follows_scalar_recursion(c):
    # K 1 = 0 and partition of unity: a constant stays constant with
    # u^{k+1} = u^k - L w(u^k) / c_t  (Eq. AC-discrete-semi-stable-K on constants).
    prob = make_problem(dim=2, n=11, s=2, p=2)
    ops = ctd.build_operators(prob)
    A = [np.full((11, 1), abs(c) ** 0.5), np.full((11, 1), math.copysign(abs(c) ** 0.5, c))]
    u = c
    for k in range(5):
        A, st = ctd.step(prob, ops, A, k)
        u = u - prob.L * 4 * prob.a0 * (u ** 3 - u) / prob.c_t
        assert st["modes"] == 1
        assert np.max(np.abs(ctd.reconstruct(A) - u)) < 1e-12


def test_stationary_tanh_profile_stays_put():
    # u = tanh((x - 1/2) / (sqrt(2) eps)) solves eps^2 u'' = u^3 - u; one mode, small drift.
    eps, n = 0.05, 81
    prob = make_problem(n=n, s=2, p=2, eps=eps, dt=0.01)
    ops = ctd.build_operators(prob)
    A = workloads.tanh_mode(prob.n, prob.length, eps)
    U0 = ctd.reconstruct(A)
    for k in range(30):
        A, st = ctd.step(prob, ops, A, k)
        assert st["modes"] == 1
    h = 1.0 / (n - 1)
    assert np.max(np.abs(ctd.reconstruct(A) - U0)) < 2.0 * (h / eps) ** 2


def test_energy_routes_agree_and_constant_energy():
    prob = make_problem(n=9, s=2, p=2)
    ops = ctd.build_operators(prob)
    A = workloads.cosine_modes(prob.n, prob.length, 2, 3, 5, amp=0.9)
    assert ctd.energy(prob, ops, A) == pytest.approx(
        fullgrid.energy(prob, ops, ctd.reconstruct(A)), rel=1e-13)
    A = [np.full((9, 1), 0.5), np.full((9, 1), 0.5)]
    assert ctd.energy(prob, ops, A) == pytest.approx(prob.a0 * (0.25 ** 2 - 1) ** 2, rel=1e-13)


def test_paper_stabiliser_satisfies_bound():
    # Section 2.5 / App. A: alpha >= max(w')/2 with w' = 4 a0 (3u^2 - 1), u in [-1, 1].
    g = json.load(open(GOLDEN))["stabiliser_case_2d"]
    u = np.linspace(-1, 1, 2001)
    wprime = 4 * g["a0"] * (3 * u ** 2 - 1)
    assert g["alpha"] >= wprime.max() / 2
    assert wprime.max() / 2 == pytest.approx(40.0)


def test_full_grid_energy_law_holds_for_any_dt():
    # Theorem of App. A on the full-grid scheme with the nodal rule: E non-increasing for
    # S >= max(w')/2 = 1 (eps form), even for a large dt.
    for dt in (0.01, 1.0):
        prob = make_problem(n=10, s=1, p=1, S=1.0, dt=dt, eps=0.08)
        ops = ctd.build_operators(prob)
        U = ctd.reconstruct(workloads.cosine_modes(prob.n, prob.length, 3, 4, 2, amp=0.9))
        E = fullgrid.energy(prob, ops, U)
        for k in range(15):
            U = fullgrid.step(prob, ops, U)
            E1 = fullgrid.energy(prob, ops, U)
            assert E1 <= E + 1e-14 * abs(E)
            E = E1


def test_ctd_energy_non_increasing_on_small_run():
    prob = make_problem(n=32, s=1, p=1, eps=0.05, dt=0.01)
    ops = ctd.build_operators(prob)
    A = workloads.cosine_modes(prob.n, prob.length, 4, 4, 0)
    E = ctd.energy(prob, ops, A)
    for k in range(10):
        A, st = ctd.step(prob, ops, A, k)
        E1 = ctd.energy(prob, ops, A)
        assert E1 <= E + 1e-10 * abs(E)
        E = E1


def test_half_sweeps_never_increase_the_galerkin_functional():
    # Each half-sweep minimises J(u) = 1/2 u^T K u - u^T Q exactly over one factor.
    prob = make_problem(n=10, s=1, p=1, M_max=3)
    ops = ctd.build_operators(prob)
    A = workloads.cosine_modes(prob.n, prob.length, 3, 4, 9, amp=0.8)
    Uk = ctd.reconstruct(A)
    tr = []
    B, st = ctd.step(prob, ops, A, 0, trace=tr)
    # rebuild u after each half-sweep: committed modes so far + current trial mode
    committed = [np.zeros((10, 0)), np.zeros((10, 0))]
    last_J = None
    count = 0
    for (m, it, x, v) in tr:
        if m > count:   # modes < m are committed (same values as B's columns)
            committed = [B[d][:, :m] for d in range(2)]
            count = m
            last_J = None
        u = ctd.reconstruct(committed) + np.outer(v[0], v[1])
        if x == 0:      # after the x-solve v is a full iterate
            J = fullgrid.galerkin_functional(prob, ops, Uk, u)
            if last_J is not None:
                assert J <= last_J + 1e-13 * abs(last_J)
            last_J = J


def test_zero_initial_condition_gives_zero_solution():
    prob = make_problem(n=8)
    ops = ctd.build_operators(prob)
    A = [np.zeros((8, 2)), np.zeros((8, 2))]
    B, st = ctd.step(prob, ops, A, 0)
    assert st["modes"] == 0 and not st["capped"]


def test_mode_cap_sets_capped_flag():
    prob = make_problem(n=12, M_max=1, tol_enrich=0.0)
    ops = ctd.build_operators(prob)
    A = workloads.cosine_modes(prob.n, prob.length, 3, 4, 1)
    B, st = ctd.step(prob, ops, A, 0)
    assert st["modes"] == 1 and st["capped"]


# ---------------------------------------------------------------- reduced integration domain
def _reduced_case(tol, block=8):
    w = workloads.preset("c0", n=(40, 36), eps=0.05, ic_rank=0, ic_tanh=True)
    prob = ctd.Problem(dim=2, n=w.n, length=w.length, s=w.s, p=w.p, a=w.a, L=w.L, kappa=w.kappa, a0=w.a0,
                        alpha=w.alpha, dt=w.dt, M_max=w.M_max, I_max=w.I_max, tol_als=w.tol_als,
                        tol_enrich=w.tol_enrich, seed=w.seed, reduced_tol=tol, reduced_block=block)
    return w, prob, ctd.build_operators(prob), workloads.initial_modes(w)


def test_reduced_domain_zero_tolerance_is_the_full_integral():
    w, prob, ops, A = _reduced_case(0.0)
    full = ctd.nonlinear_tensor(prob, ops, A)
    prob.reduced_tol = 0.0
    U = ctd.reconstruct(A)
    assert np.array_equal(full, prob.L * ctd.grid_weights(ops) * ctd.w_of_u(U, prob.a0))


def test_reduced_domain_mask_brute_force_blocks():
    # every block is kept iff some node in it has |w| > tol (plain loops over the nodes)
    w, prob, ops, A = _reduced_case(1e-3, block=8)
    W = ctd.w_of_u(ctd.reconstruct(A), prob.a0)
    mask = ctd.reduced_domain_mask(prob, W)
    n0, n1 = W.shape
    for i in range(n0):
        for j in range(n1):
            bi, bj = i // 8, j // 8
            big = False
            for ii in range(bi * 8, min(bi * 8 + 8, n0)):
                for jj in range(bj * 8, min(bj * 8 + 8, n1)):
                    big = big or abs(W[ii, jj]) > 1e-3
            assert mask[i, j] == big
    # the tanh interface sits at x = 1/2: blocks far from it drop out, blocks on it stay
    assert not mask[0, 0] and not mask[-1, -1] and mask[n0 // 2, 0]


def test_reduced_domain_error_bound_and_limits():
    w, prob, ops, A = _reduced_case(1e-3, block=8)
    red = ctd.nonlinear_tensor(prob, ops, A)
    prob.reduced_tol = 0.0
    full = ctd.nonlinear_tensor(prob, ops, A)
    v = [np.random.default_rng(2).uniform(0.5, 1.5, size=w.n[d]) for d in range(2)]
    W = ctd.w_of_u(ctd.reconstruct(A), prob.a0)
    prob.reduced_tol = 1e-3
    drop = ~ctd.reduced_domain_mask(prob, W)
    for x in range(2):
        diff = np.abs(ctd.contract_except(full - red, v, x))
        bound = 1e-3 * ctd.contract_except(prob.L * ctd.grid_weights(ops) * drop, v, x)
        assert np.all(diff <= bound * (1 + 1e-12) + 1e-300)
    # a tolerance above every |w| removes the whole nonlinear term
    prob.reduced_tol = 10.0 * float(np.max(np.abs(W)))
    assert not np.any(ctd.nonlinear_tensor(prob, ops, A))


# ---- separated nonlinearity (Eq. MxySep)

def _separated_case(dim, rank, seed=3):
    n = (11, 9) if dim == 2 else (7, 6, 5)
    prob = ctd.Problem(dim=dim, n=n, length=(1.0,) * dim, s=1, p=1, a=12.0, L=1.3, kappa=1e-3, a0=0.25,
                       alpha=2.0, dt=0.01, M_max=20, I_max=50, tol_als=1e-8, tol_enrich=1e-4, seed=0)
    ops = ctd.build_operators(prob)
    rng = np.random.default_rng(seed)
    A = [rng.uniform(-1.0, 1.0, size=(n[d], rank)) for d in range(dim)]
    return prob, ops, A


@pytest.mark.parametrize("dim,rank", [(2, 1), (2, 4), (3, 3)])
def test_separated_terms_reproduce_w_on_the_grid(dim, rank):
    # sum_q c_q prod_d f_q,d evaluated node by node against w(u) of the reconstructed field
    prob, ops, A = _separated_case(dim, rank)
    terms = ctd.separated_nonlinear_terms(prob, A)
    assert len(terms) == math.comb(rank + 2, 3) + rank
    W = ctd.w_of_u(ctd.reconstruct(A), prob.a0)
    S = np.zeros_like(W)
    for idx in np.ndindex(*W.shape):
        S[idx] = sum(c * np.prod([f[d][idx[d]] for d in range(dim)]) for c, f in terms)
    assert np.max(np.abs(S - W)) <= 1e-13 * max(1.0, np.max(np.abs(W)))


@pytest.mark.parametrize("dim,rank", [(2, 4), (3, 3)])
def test_separated_contraction_equals_full_integral(dim, rank):
    # Eq. MxySep against Eq. KxxMxx (the full nodal integral over the grid)
    prob, ops, A = _separated_case(dim, rank)
    terms = ctd.separated_nonlinear_terms(prob, A)
    Mxy = ctd.nonlinear_tensor(prob, ops, A)
    v = [np.random.default_rng(9).uniform(-1.0, 1.0, size=prob.n[d]) for d in range(dim)]
    for x in range(dim):
        ref = ctd.contract_except(Mxy, v, x)
        got = ctd.separated_contraction(prob, ops, terms, v, x)
        assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref), x


def test_separated_step_equals_grid_step():
    # same step with either form of the nonlinear term: same decisions, same field
    w = workloads.preset("c0", n=(20, 17), M_max=8)
    kw = dict(dim=2, n=w.n, length=w.length, s=w.s, p=w.p, a=w.a, L=w.L, kappa=w.kappa, a0=w.a0,
              alpha=w.alpha, dt=w.dt, M_max=w.M_max, I_max=w.I_max, tol_als=w.tol_als,
              tol_enrich=w.tol_enrich, seed=w.seed)
    pg = ctd.Problem(**kw)
    ps = ctd.Problem(**kw, nonlinear_form="separated")
    ops = ctd.build_operators(pg)
    Ag = As = workloads.initial_modes(w)
    for k in range(3):
        Ag, sg = ctd.step(pg, ops, Ag, k)
        As, ss = ctd.step(ps, ops, As, k)
        assert sg["modes"] == ss["modes"] and sg["als_iters"] == ss["als_iters"], (k, sg, ss)
        assert ctd.rel_l2_between(As, Ag) < 1e-12, k


def test_separated_form_falls_back_above_the_mode_limit():
    prob, ops, A = _separated_case(2, 4)
    prob.nonlinear_form = "separated"
    prob.separated_max_modes = 3
    assert ctd.nonlinear_operator(prob, ops, A)[0] == "grid"
    prob.separated_max_modes = 4
    assert ctd.nonlinear_operator(prob, ops, A)[0] == "separated"
    assert ctd.nonlinear_operator(prob, ops, [a[:, :0] for a in A])[0] == "grid"   # u^k = 0


def test_stalled_3d_case_amplifies_last_bit_perturbations():
    # Conditioning of the 3D case whose modes stall at I_max (the GPU parity test of the same
    # case): perturbing every banded solve of the oracle by one unit in the last place moves its
    # own field after three steps by far more than one unit -- the near-neutral sweep map carries
    # the perturbation over 50 sweeps -- yet stays below 1e-12, the FP64 parity bar.
    w = workloads.preset("c0", dim=3, n=(14, 11, 17), length=(1.0, 1.0, 1.0), eps=0.08, M_max=10, ic_rank=3)
    prob = ctd.Problem(dim=w.dim, n=w.n, length=w.length, s=w.s, p=w.p, a=w.a, L=w.L, kappa=w.kappa,
                       a0=w.a0, alpha=w.alpha, dt=w.dt, M_max=w.M_max, I_max=w.I_max, tol_als=w.tol_als,
                       tol_enrich=w.tol_enrich, seed=w.seed)
    ops = ctd.build_operators(prob)
    orig = ctd.banded_spd_solve

    def run(seed):
        rng = np.random.default_rng(seed) if seed is not None else None

        def solve(A, rhs):
            x = orig(A, rhs)
            return x if rng is None else x * (1.0 + 2.0 ** -52 * rng.uniform(-1.0, 1.0, size=x.shape))

        ctd.banded_spd_solve = solve
        try:
            A = workloads.initial_modes(w)
            hist = []
            for k in range(3):
                A, st = ctd.step(prob, ops, A, k)
                hist.append(st["als_iters"])
            return A, hist
        finally:
            ctd.banded_spd_solve = orig

    A0, h0 = run(None)
    errs = []
    for seed in range(3):
        A1, h1 = run(seed)
        assert h1 == h0
        errs.append(ctd.rel_l2_between(A1, A0))
    assert max(errs) > 1e-14 and max(errs) < 1e-12, errs


def test_interface_workload_conditioning():
    # The 3D workload with a tanh interface mode (eps = 0.02, s = p = 2), on a 40^3 grid: a
    # 1e-7 relative perturbation of the oracle's own nonlinear term (the size of a tensor-core
    # contraction's rounding) leaves a step with a fixed mode count and converged sweeps within
    # 1e-8, but six fixed sweeps per mode move it by more than 1e-5, and free running it flips
    # the greedy mode count, moving the field by more than 1e-5 (the enrichment truncation,
    # tol_enrich = 1e-4, sets that level).  Comparisons of two arithmetics on this workload are
    # therefore made on a fixed mode count with converged sweeps.
    w = workloads.preset("c2", n=(40, 40, 40))
    orig = ctd.nonlinear_projection

    def step(level, **over):
        rng = np.random.default_rng(1)

        def noisy(prob, ops, nl, v, x):
            r = orig(prob, ops, nl, v, x)
            return r * (1.0 + level * rng.uniform(-1.0, 1.0, size=r.shape)) if level else r

        prob = ctd.Problem(dim=w.dim, n=w.n, length=w.length, s=w.s, p=w.p, a=w.a, L=w.L, kappa=w.kappa,
                           a0=w.a0, alpha=w.alpha, dt=w.dt, M_max=w.M_max, I_max=w.I_max, tol_als=w.tol_als,
                           tol_enrich=w.tol_enrich, seed=w.seed)
        for k, v in over.items():
            setattr(prob, k, v)
        ctd.nonlinear_projection = noisy
        try:
            return ctd.step(prob, ctd.build_operators(prob), workloads.initial_modes(w), 0)
        finally:
            ctd.nonlinear_projection = orig

    for over, lo, hi in ((dict(fixed_modes=12), 0.0, 1e-8), (dict(fixed_modes=12, fixed_als_iters=6), 1e-5, 1.0)):
        A0, _ = step(0.0, **over)
        A1, _ = step(1e-7, **over)
        assert lo <= ctd.rel_l2_between(A1, A0) < hi, over
    A0, s0 = step(0.0, als_stall_tol=1e-6)
    A1, s1 = step(1e-7, als_stall_tol=1e-6)
    assert s0["modes"] != s1["modes"]
    assert 1e-5 < ctd.rel_l2_between(A1, A0) < w.tol_enrich
