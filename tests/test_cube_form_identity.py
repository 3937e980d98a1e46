"""The algebra the cube form of the tensor-core contraction relies on, checked in FP64 against
the oracle's nonlinear integral (Eq. KxxMxx, no GPU).

With c_j the column weight (the quadrature weight times the fixed factors of the other
dimensions), the row sum sum_j c_j w(u_ij) with w(u) = 4 a0 (u^3 - u) is computed as
4 a0 (sum_j v_ij^3 - lin_i): v_ij = cbrt(c_j) u_ij from a column operand scaled row by row,
and the linear part lin_i = sum_m a_m,x(i) H_m, H_m = prod_{d != x} h_d,m with h_d,m the
weighted Gram sum of the fixed factor and factor m (omega_d v_d . a_m,d at the nodes,
v_d . M_d a_m,d under the Gauss rule, M_d = Phi_d^T diag(omega_q) Phi_d).  Under the Gauss
rule the point sums go through Phi_x^T diag(omega_q) and the linear part becomes
sum_m (M_x a_m,x)_i H_m.  A dropped term, a wrong Gram weight or a 4 a0 applied twice fails
these checks.
"""
import numpy as np
import pytest

import workloads
from oracle import ctd as octd


def problem(w, **over):
    kw = dict(dim=w.dim, n=w.n, length=w.length, s=w.s, p=w.p, a=w.a, L=w.L, kappa=w.kappa, a0=w.a0,
              alpha=w.alpha, dt=w.dt, M_max=w.M_max, I_max=w.I_max, tol_als=w.tol_als, tol_enrich=w.tol_enrich,
              seed=w.seed)
    kw.update(over)
    return octd.Problem(**kw)


def grid_of(A):
    if len(A) == 2:
        return A[0] @ A[1].T
    return np.einsum("im,jm,km->ijk", A[0], A[1], A[2])


def cube_form_rows(prob, ops, A, v, x, drop_linear=False):
    """The cube form's row sums for direction x, as the kernels compose them (FP64 here)."""
    D = len(A)
    gauss = ops.Phi is not None
    Aq = [ops.Phi[d] @ A[d] if gauss else A[d] for d in range(D)]      # factors at the points
    vq = [ops.Phi[d] @ v[d] if gauss else v[d] for d in range(D)]
    # column weights and their cube roots, one vector per other dimension
    c = [ops.omega[d] * vq[d] for d in range(D)]
    s = [np.cbrt(cd) for cd in c]
    # the scaled operand: u at the points times cbrt(c_j) over the other dimensions
    scaled = [Aq[d] * s[d][:, None] if d != x else Aq[d] for d in range(D)]
    V = np.moveaxis(grid_of(scaled), x, 0).reshape(Aq[x].shape[0], -1)
    S3 = np.sum(V ** 3, axis=1)
    if gauss:
        S3 = ops.Phi[x].T @ (ops.omega[x] * S3)
        ax = ops.M[x] @ A[x]
        h = [v[d] @ (ops.M[d] @ A[d]) for d in range(D)]
    else:
        ax = A[x]
        h = [(ops.omega[d] * v[d]) @ A[d] for d in range(D)]
    H = np.ones(A[0].shape[1])
    for d in range(D):
        if d != x:
            H = H * h[d]
    return 4.0 * prob.a0 * (S3 - (0.0 if drop_linear else ax @ H))


@pytest.mark.parametrize("dim,n,rank,amp,a0,L", [(2, (40, 31), 4, 0.3, 0.25, 1.0), (2, (40, 31), 6, 0.8, 0.6, 1.7),
                                                 (3, (12, 9, 14), 3, 0.5, 0.45, 1.3)])
def test_cube_form_equals_the_nodal_integral(dim, n, rank, amp, a0, L):
    w = workloads.preset("c0", dim=dim, n=n, length=(1.0,) * dim)
    prob = problem(w, a0=a0, L=L)
    ops = octd.build_operators(prob)
    A = workloads.cosine_modes(n, (1.0,) * dim, rank, 4, 3, amp=amp)
    rng = np.random.default_rng(7)
    v = [rng.uniform(-1.5, 1.5, size=n[d]) for d in range(dim)]   # signed weights: the real cube root
    Mxy = octd.nonlinear_tensor(prob, ops, A)
    for x in range(dim):
        ref = octd.contract_except(Mxy, v, x) / (prob.L * ops.omega[x])
        got = cube_form_rows(prob, ops, A, v, x)
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref)), x


@pytest.mark.parametrize("dim,n,q", [(2, (24, 19), 3), (2, (24, 19), 5), (3, (10, 8, 9), 2)])
def test_cube_form_equals_the_gauss_integral(dim, n, q):
    w = workloads.preset("c0", dim=dim, n=n, length=(1.0,) * dim)
    prob = problem(w, a0=0.4, L=1.2, quad_rule="gauss", quad_q=q)
    ops = octd.build_operators(prob)
    A = workloads.cosine_modes(n, (1.0,) * dim, 4, 4, 3, amp=0.6)
    rng = np.random.default_rng(8)
    v = [rng.uniform(0.5, 1.5, size=n[d]) for d in range(dim)]
    nl = octd.nonlinear_operator(prob, ops, A)
    for x in range(dim):
        ref = octd.nonlinear_projection(prob, ops, nl, v, x) / prob.L
        got = cube_form_rows(prob, ops, A, v, x)
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref)), x


def test_dropping_the_linear_part_or_doubling_4a0_fails():
    # the identity is sharp: each plausible slip moves the result far outside 1e-12
    w = workloads.preset("c0", n=(40, 31))
    prob = problem(w, a0=0.6)
    ops = octd.build_operators(prob)
    A = workloads.cosine_modes(w.n, w.length, 4, 4, 3, amp=0.3)
    v = [np.linspace(0.5, 1.5, w.n[d]) for d in range(2)]
    ref = octd.contract_except(octd.nonlinear_tensor(prob, ops, A), v, 0) / (prob.L * ops.omega[0])
    good = cube_form_rows(prob, ops, A, v, 0)
    assert np.max(np.abs(good - ref)) <= 1e-12 * np.max(np.abs(ref))
    doubled = 4.0 * prob.a0 * good
    assert np.max(np.abs(doubled - ref)) > 1e-3 * np.max(np.abs(ref))
    no_linear = cube_form_rows(prob, ops, A, v, 0, drop_linear=True)
    assert np.max(np.abs(no_linear - ref)) > 1e-3 * np.max(np.abs(ref))
