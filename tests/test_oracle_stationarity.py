"""Pin of the half-sweep assembly (Eq. ux with K_x, Q_x of Eq. KxQx / KyQy, App. D): a
half-sweep minimises the step's Galerkin functional J(u) = 1/2 u^T K u - u^T Q exactly over
one factor, so the full-grid gradient K u - Q, built independently from Kronecker-assembled
operators, must vanish when contracted with the other (fixed) factors.  A dropped, mis-signed
or mis-indexed term of the separated assembly fails this at any size."""
import numpy as np
import pytest

import workloads
from oracle import ctd, fullgrid


def make_problem(dim, n, rule, form="grid", **kw):
    args = dict(dim=dim, n=n, length=(1.0, 0.8, 1.2)[:dim], s=2, p=2, a=12.0, L=1.3, kappa=0.02,
                a0=0.25, alpha=2.0, dt=0.05, M_max=6, I_max=20, tol_als=1e-10, tol_enrich=1e-8,
                seed=0, quad_rule=rule, quad_q=3, nonlinear_form=form)
    args.update(kw)
    return ctd.Problem(**args)


def kron_vec(vs):
    out = vs[0]
    for v in vs[1:]:
        out = np.kron(out, v)
    return out


@pytest.mark.parametrize("dim,n,rule,form", [(2, (9, 7), "nodal", "grid"), (2, (8, 9), "gauss", "grid"),
                                             (3, (6, 5, 7), "nodal", "grid"), (3, (5, 6, 5), "gauss", "grid"),
                                             (2, (9, 7), "nodal", "separated"), (3, (6, 5, 7), "gauss", "separated")])
def test_half_sweep_is_a_stationary_point_of_the_galerkin_functional(dim, n, rule, form):
    prob = make_problem(dim, n, rule, form)
    ops = ctd.build_operators(prob)
    rng = np.random.default_rng(3)
    A = workloads.cosine_modes(n, prob.length, 3, 3, 5, amp=0.7)
    B = [0.2 * rng.standard_normal((n[d], 2)) for d in range(dim)]
    v = [rng.uniform(0.5, 1.5, n[d]) for d in range(dim)]
    nl = ctd.nonlinear_operator(prob, ops, A)
    Mfull, Kfull = fullgrid.operators_full(prob, ops)
    Ksys = prob.c_t * Mfull + prob.c_k * Kfull
    uk = ctd.reconstruct(A).reshape(-1)
    Q = prob.c_t * (Mfull @ uk) - fullgrid.nonlinear_full(prob, ops, uk)
    for x in range(dim):
        vx, _ = ctd.half_sweep(prob, ops, x, list(v), A, B, nl)
        w = list(v)
        w[x] = vx
        u = ctd.reconstruct(B).reshape(-1) + kron_vec(w)
        g = (Ksys @ u - Q).reshape(n)
        # contract the gradient with every fixed factor: d J / d v_x
        others = [w[d] if d != x else None for d in range(dim)]
        dJ = g
        for d in reversed(range(dim)):
            if d != x:
                dJ = np.tensordot(dJ, others[d], axes=([d], [0]))
        scale = np.linalg.norm(ctd.contract_except(np.abs(Q.reshape(n)), [np.abs(y) for y in w], x))
        assert np.linalg.norm(dJ) < 1e-12 * scale, (x, np.linalg.norm(dJ) / scale)
        # and a perturbation of vx raises J: the stationary point is the minimum
        J0 = 0.5 * u @ (Ksys @ u) - u @ Q
        d = rng.standard_normal(n[x]) * 1e-3 * np.linalg.norm(vx)
        w[x] = vx + d
        u1 = ctd.reconstruct(B).reshape(-1) + kron_vec(w)
        assert 0.5 * u1 @ (Ksys @ u1) - u1 @ Q > J0
        v[x] = vx / np.linalg.norm(vx)
