"""Brute-force full-grid solution of the stabilized semi-implicit step -- oracle pin.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Eq. AC-discrete-semi-stable-K solved directly on the tensor-product C-FEM space, with no
separation of variables: the D-dimensional mass and stiffness are assembled as Kronecker
products of the 1D matrices (``N~(x, y) = N~_x(x) N~_y(y)``), ``K = c_t M + c_k K_grad`` and
``Q = c_t M u^k - L M w(u^k)`` (nonlinear term under the nodal rule, so its integral is
``M`` times the nodal values of ``w``; under the Gauss rule it is ``Phi^T diag(omega)
w(Phi u^k)`` with the Kronecker products of the 1D ``Phi_d`` and weights), then one dense
solve.  Used only on tiny grids to
check ``oracle.ctd``, whose greedy separated solution must approach this one as the mode
budget and tolerances tighten (Section 3.2: CTD converges to the CFE solution).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .ctd import Operators, Problem, w_of_u


def kron_all(mats):
    out = mats[0]
    for m in mats[1:]:
        out = sp.kron(out, m, format="csr")
    return out


def operators_full(prob: Problem, ops: Operators):
    """Full-grid mass ``M = (x)_d M_d`` and gradient operator
    ``K_grad = sum_d M_0 (x) .. K_d .. (x) M_{D-1}`` (row-major node ordering)."""
    D = prob.dim
    Mfull = kron_all([ops.M[d] for d in range(D)])
    Kfull = None
    for d in range(D):
        mats = [ops.K[e] if e == d else ops.M[e] for e in range(D)]
        term = kron_all(mats)
        Kfull = term if Kfull is None else Kfull + term
    return Mfull, Kfull


def weights_full(ops: Operators) -> np.ndarray:
    """Weights of the tensor-product quadrature points (row-major ordering)."""
    W = ops.omega[0]
    for w in ops.omega[1:]:
        W = np.kron(W, w)
    return W


def nonlinear_full(prob: Problem, ops: Operators, uk: np.ndarray) -> np.ndarray:
    """``int N~^T L w(u^k)``: ``L M w`` at the nodes under the nodal rule, else
    ``L Phi^T (omega w(Phi u^k))`` over the tensor-product Gauss points."""
    if ops.Phi is None:
        Mfull, _ = operators_full(prob, ops)
        return prob.L * (Mfull @ w_of_u(uk, prob.a0))
    Phif = kron_all(ops.Phi)
    return prob.L * (Phif.T @ (weights_full(ops) * w_of_u(Phif @ uk, prob.a0)))


def step(prob: Problem, ops: Operators, u_k: np.ndarray) -> np.ndarray:
    """``u^{k+1}`` on the full grid from nodal values ``u_k`` (D-way array)."""
    Mfull, Kfull = operators_full(prob, ops)
    uk = u_k.reshape(-1)
    Ksys = (prob.c_t * Mfull + prob.c_k * Kfull).toarray()
    Q = prob.c_t * (Mfull @ uk) - nonlinear_full(prob, ops, uk)
    return np.linalg.solve(Ksys, Q).reshape(u_k.shape)


def energy(prob: Problem, ops: Operators, u: np.ndarray) -> float:
    """Same discrete energy as ``ctd.energy`` but from full-grid values."""
    Mfull, Kfull = operators_full(prob, ops)
    uv = u.reshape(-1)
    if ops.Phi is None:
        bulk = float(Mfull.diagonal() @ (prob.a0 * (uv ** 2 - 1.0) ** 2))
    else:
        uq = kron_all(ops.Phi) @ uv
        bulk = float(weights_full(ops) @ (prob.a0 * (uq ** 2 - 1.0) ** 2))
    return bulk + 0.5 * prob.kappa * float(uv @ (Kfull @ uv))


def galerkin_functional(prob: Problem, ops: Operators, u_k: np.ndarray, u: np.ndarray) -> float:
    """``J(u) = 1/2 u^T K u - u^T Q`` of the step from ``u_k``; each ALS half-sweep is an
    exact minimisation of ``J`` over one factor, so ``J`` cannot increase."""
    Mfull, Kfull = operators_full(prob, ops)
    uk = u_k.reshape(-1)
    uv = u.reshape(-1)
    Q = prob.c_t * (Mfull @ uk) - nonlinear_full(prob, ops, uk)
    Kv = prob.c_t * (Mfull @ uv) + prob.c_k * (Kfull @ uv)
    return 0.5 * float(uv @ Kv) - float(uv @ Q)
