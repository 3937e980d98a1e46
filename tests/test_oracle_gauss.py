"""Pins for the oracle's Gauss-point quadrature (the consistent-mass variant of Eq. KxxMxx;
Section 3.3 evaluates w(u^k) at the Gauss points of each element) against closed forms,
polynomial exactness, the brute-force full-grid solve and the scheme's invariants."""
import math

import numpy as np
import pytest

import workloads
from oracle import cfem, ctd, fullgrid


def make_problem(dim=2, n=9, s=2, p=2, q=5, eps=0.05, S=2.0, dt=0.01, **kw):
    args = dict(dim=dim, n=(n,) * dim, length=(1.0,) * dim, s=s, p=p, a=12.0, L=1.0,
                kappa=eps ** 2, a0=0.25, alpha=S, dt=dt, M_max=20, I_max=50, tol_als=1e-8,
                tol_enrich=1e-4, seed=0, quad_rule="gauss", quad_q=q)
    args.update(kw)
    return ctd.Problem(**args)


@pytest.mark.parametrize("q", [2, 3, 5])
def test_composite_gauss_rule_moments(q):
    # a q-point Gauss rule integrates x^k exactly for k <= 2q - 1 on every element
    n, X = 7, 1.7
    x, w = cfem.gauss_quadrature(n, X, q)
    assert x.shape == w.shape == (q * (n - 1),)
    assert np.all(np.diff(x) > 0) and x[0] > 0 and x[-1] < X
    for k in range(2 * q):
        assert float(w @ x ** k) == pytest.approx(X ** (k + 1) / (k + 1), rel=1e-13)
    # the first moment beyond exactness is not integrated exactly
    k = 2 * q
    assert abs(float(w @ x ** k) - X ** (k + 1) / (k + 1)) > 1e-14


@pytest.mark.parametrize("s,p", [(1, 1), (2, 2), (3, 3)])
def test_basis_at_gauss_points_reproduces_polynomials(s, p):
    # C-FEM shape functions form a partition of unity and reproduce degree <= p (Section 3.2)
    n, X = 12, 2.0
    xq, _ = cfem.gauss_quadrature(n, X, 4)
    Phi = cfem.quadrature_basis(n, X, s, p, 12.0, 4)
    assert Phi.shape == (4 * (n - 1), n)
    xn = cfem.nodes(n, X)
    for k in range(p + 1):
        assert np.max(np.abs(Phi @ xn ** k - xq ** k)) < 1e-11 * max(1.0, X ** k)
    # each point sees only the support of its element: nodes e - s .. e + 1 + s
    e = np.repeat(np.arange(n - 1), 4)
    rows, cols = Phi.nonzero()
    assert np.all(cols >= e[rows] - s) and np.all(cols <= e[rows] + 1 + s)


def test_gauss_mass_is_the_exact_consistent_mass():
    # q >= 5 integrates N~_i N~_j (piecewise degree <= 8) exactly; closed-form moments
    n, X, s, p = 10, 1.5, 2, 2
    prob = make_problem(n=n, s=s, p=p, q=5, length=(X, X))
    ops = ctd.build_operators(prob)
    M = ops.M[0].toarray()
    M8 = cfem.consistent_mass_matrix(n, X, s, p, 12.0, gauss_points=8)
    assert np.max(np.abs(M - M8)) < 1e-14 * np.max(np.abs(M8))
    assert np.max(np.abs(M - M.T)) < 1e-15 * np.max(np.abs(M))
    assert np.min(np.linalg.eigvalsh(M)) > 0
    xn, one = cfem.nodes(n, X), np.ones(n)
    assert one @ M @ one == pytest.approx(X, rel=1e-13)                 # int 1
    assert xn @ M @ one == pytest.approx(X ** 2 / 2, rel=1e-13)         # int x
    assert xn @ M @ xn == pytest.approx(X ** 3 / 3, rel=1e-13)          # int x^2
    assert (xn ** 2) @ M @ (xn ** 2) == pytest.approx(X ** 5 / 5, rel=1e-12)   # int x^4
    # the nodal rule's mass is diagonal and differs from it
    nodal = ctd.build_operators(make_problem(n=n, s=s, p=p, length=(X, X), quad_rule="nodal"))
    assert np.max(np.abs(nodal.M[0].toarray() - M)) > 1e-3 * np.max(np.abs(M))


def test_phi_transpose_weights_equals_mass_times_one():
    # partition of unity: Phi 1 = 1 (up to the rounding of the App. B solves), so
    # Phi^T omega = M 1 for any rule
    prob = make_problem(n=11, q=3)
    ops = ctd.build_operators(prob)
    assert np.max(np.abs(ops.Phi[0] @ np.ones(11) - 1.0)) < 1e-13
    lhs = ops.Phi[0].T @ ops.omega[0]
    assert np.max(np.abs(lhs - ops.M[0] @ np.ones(11))) < 1e-13 * np.max(lhs)


@pytest.mark.parametrize("dim", [2, 3])
def test_contraction_of_a_linear_field_has_closed_form_moments(dim):
    # u^k = x (exactly reproduced for p >= 1), v_d = 1: the nonlinear integral against N~_i
    # sums to L Y (Z) int_0^X w(x) dx, and its first moment to L Y (Z) int_0^X x w(x) dx
    # (integrands of degree <= 8 per element, exact for q = 5).
    X, Y, Z = 1.3, 0.7, 1.1
    lengths = (X, Y, Z)[:dim]
    n = 8 if dim == 2 else 6
    prob = make_problem(dim=dim, n=n, q=5, length=lengths, a0=0.6, L=1.7)
    ops = ctd.build_operators(prob)
    xn = cfem.nodes(n, X)
    A = [xn[:, None]] + [np.ones((n, 1))] * (dim - 1)
    nl = ctd.nonlinear_operator(prob, ops, A)
    v = [np.ones(n)] * dim
    R = ctd.nonlinear_projection(prob, ops, nl, v, 0)
    other = float(np.prod(lengths[1:]))
    c = 4 * prob.a0 * prob.L * other
    assert R.sum() == pytest.approx(c * (X ** 4 / 4 - X ** 2 / 2), rel=1e-12)
    assert xn @ R == pytest.approx(c * (X ** 5 / 5 - X ** 3 / 3), rel=1e-12)
    # along another axis: int w(x) dx over X times int N~_j over that axis (= M 1)
    R1 = ctd.nonlinear_projection(prob, ops, nl, v, 1)
    ref = prob.L * 4 * prob.a0 * (X ** 4 / 4 - X ** 2 / 2) * (ops.M[1] @ np.ones(n))
    if dim == 3:
        ref = ref * Z
    assert np.max(np.abs(R1 - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("dim,rank", [(2, 3), (3, 2)])
def test_separated_contraction_equals_gauss_grid_integral(dim, rank):
    # the decomposition of the cubic is exact at every quadrature point (Eq. MxySep)
    n = 9 if dim == 2 else 6
    prob = make_problem(dim=dim, n=n, q=3)
    ops = ctd.build_operators(prob)
    rng = np.random.default_rng(5)
    A = [0.6 * rng.standard_normal((n, rank)) for _ in range(dim)]
    v = [rng.standard_normal(n) for _ in range(dim)]
    grid = ("grid", ctd.nonlinear_tensor(prob, ops, A))
    terms = ctd.separated_nonlinear_terms(prob, A, ops)
    for x in range(dim):
        ref = ctd.nonlinear_projection(prob, ops, grid, v, x)
        got = ctd.separated_contraction(prob, ops, terms, v, x)
        assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("dim,n,q,s,modes,sweeps,bound", [(2, 8, 5, 2, 20, 300, 1e-12),
                                                            (2, 7, 2, 2, 14, 400, 1e-12),
                                                            (3, 4, 5, 1, 48, 200, 1e-6)])
def test_gauss_ctd_converges_to_full_grid_solution(dim, n, q, s, modes, sweeps, bound):
    # Section 3.2: the separated solution approaches the full-grid C-FEM solution of the same
    # discrete equations (consistent mass, Gauss-point nonlinearity) as modes are added
    prob = make_problem(dim=dim, n=n, q=q, s=s, p=s, M_max=modes, I_max=sweeps,
                        tol_als=1e-12 if dim == 2 else 1e-10, tol_enrich=1e-15)
    ops = ctd.build_operators(prob)
    A = workloads.cosine_modes(prob.n, prob.length, 3, 4, 11, amp=0.8)
    B, st = ctd.step(prob, ops, A, 0)
    U1 = fullgrid.step(prob, ops, ctd.reconstruct(A))
    err = np.linalg.norm(ctd.reconstruct(B) - U1) / np.linalg.norm(U1)
    assert err < bound


@pytest.mark.parametrize("c", [0.4, -0.8])
def test_gauss_constant_state_follows_scalar_recursion(c):
    # K 1 = 0 and Phi^T omega = M 1: a constant stays constant, u <- u - L w(u) / c_t
    prob = make_problem(n=10, q=5)
    ops = ctd.build_operators(prob)
    A = [np.full((10, 1), abs(c) ** 0.5), np.full((10, 1), math.copysign(abs(c) ** 0.5, c))]
    u = c
    for k in range(3):
        A, st = ctd.step(prob, ops, A, k)
        u = u - prob.L * 4 * prob.a0 * (u ** 3 - u) / prob.c_t
        assert st["modes"] == 1
        assert np.max(np.abs(ctd.reconstruct(A) - u)) < 1e-12


def test_gauss_energy_routes_and_closed_forms():
    prob = make_problem(n=9, q=5)
    ops = ctd.build_operators(prob)
    A = workloads.cosine_modes(prob.n, prob.length, 2, 3, 5, amp=0.9)
    assert ctd.energy(prob, ops, A) == pytest.approx(
        fullgrid.energy(prob, ops, ctd.reconstruct(A)), rel=1e-13)
    # u = x: bulk a0 int (x^2 - 1)^2 over the unit square, gradient 1/2 kappa |grad u|^2 = kappa / 2
    xn = cfem.nodes(9, 1.0)
    A = [xn[:, None], np.ones((9, 1))]
    ref = prob.a0 * (1 / 5 - 2 / 3 + 1) + 0.5 * prob.kappa
    assert ctd.energy(prob, ops, A) == pytest.approx(ref, rel=1e-12)


def test_gauss_full_grid_energy_law():
    # App. A's Taylor step holds at every quadrature point when F, w and M share the rule:
    # E is non-increasing for S >= max(w')/2 = 1, even for a large dt.
    for dt in (0.01, 1.0):
        prob = make_problem(n=8, s=1, p=1, q=5, S=1.0, dt=dt, eps=0.08)
        ops = ctd.build_operators(prob)
        U = ctd.reconstruct(workloads.cosine_modes(prob.n, prob.length, 3, 4, 2, amp=0.9))
        E = fullgrid.energy(prob, ops, U)
        for k in range(10):
            U = fullgrid.step(prob, ops, U)
            E1 = fullgrid.energy(prob, ops, U)
            assert E1 <= E + 1e-14 * abs(E)
            E = E1


def test_gauss_rule_refuses_the_reduced_domain():
    prob = make_problem(n=8, q=3, reduced_tol=1e-3)
    ops = ctd.build_operators(prob)
    A = workloads.cosine_modes(prob.n, prob.length, 2, 2, 1, amp=0.8)
    with pytest.raises(ValueError):
        ctd.nonlinear_tensor(prob, ops, A)
    with pytest.raises(ValueError):
        ctd.build_operators(make_problem(quad_rule="simpson"))


def test_gauss_separated_step_equals_gauss_grid_step():
    # the decomposition of the cubic is exact at the Gauss points too: same decisions, same field
    w = workloads.preset("c0", n=(14, 12), M_max=6)
    kw = dict(dim=2, n=w.n, length=w.length, s=w.s, p=w.p, a=w.a, L=w.L, kappa=w.kappa, a0=w.a0,
              alpha=w.alpha, dt=w.dt, M_max=w.M_max, I_max=w.I_max, tol_als=w.tol_als,
              tol_enrich=w.tol_enrich, seed=w.seed, quad_rule="gauss", quad_q=3)
    pg = ctd.Problem(**kw)
    ps = ctd.Problem(**kw, nonlinear_form="separated")
    ops = ctd.build_operators(pg)
    Ag = As = workloads.initial_modes(w)
    for k in range(2):
        Ag, sg = ctd.step(pg, ops, Ag, k)
        As, ss = ctd.step(ps, ops, As, k)
        assert sg["modes"] == ss["modes"] and sg["als_iters"] == ss["als_iters"], (k, sg, ss)
        assert ctd.rel_l2_between(As, Ag) < 1e-12, k


def test_gauss_ctd_energy_non_increasing_on_small_run():
    # the energy law carried to the separated solution (tolerances 1e-8 / 1e-4)
    prob = make_problem(n=24, s=1, p=1, q=3, eps=0.05, dt=0.01, M_max=12)
    ops = ctd.build_operators(prob)
    A = workloads.cosine_modes(prob.n, prob.length, 4, 4, 0)
    E = ctd.energy(prob, ops, A)
    for k in range(6):
        A, st = ctd.step(prob, ops, A, k)
        E1 = ctd.energy(prob, ops, A)
        assert E1 <= E + 1e-10 * abs(E)
        E = E1
