"""Adaptive CTD (ACTD): the hybrid CTD / full-grid C-FEM step of Section 3.3 ("Adaptivity")
-- oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

What is computed: each time step starts the greedy CTD solve (``ctd.step``); if the number
of modes M would exceed the critical value M_c, that step is solved on the full
tensor-product C-FEM space instead (the CFE step of Eq. AC-discrete-semi-stable-K), and the
next step starts CTD again.

Readings of points the paper leaves open (each also listed in the design notes):
  * Switch rule: the greedy loop is run with the mode budget ``min(M_max, M_c + 1)``; when it
    commits an (M_c + 1)-th mode (the enrichment test still asks for one after M_c), M > M_c
    and the separated result is discarded.
  * CFE step: solved exactly by fast diagonalisation.  With the generalised eigenpairs
    ``K_d V_d = M_d V_d diag(lambda_d)``, ``V_d^T M_d V_d = I`` of every dimension, the
    full-grid operator ``c_t (x)M_d + c_k sum_d M..K_d..M`` becomes diagonal in the
    product basis ``(x)V_d`` with entries ``c_t + c_k sum_d lambda_d,i_d``.
  * State after a CFE step: the full-grid field ``u^{k+1}`` itself, with no re-decomposition.
    The next step needs ``u^k`` only through ``c_t M u^k - int N~ L w(u^k)``.  Both are
    full-grid terms, so they are folded into one array at the quadrature points
    (``grid_source``), and that step's modes start from the SplitMix64 vectors.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np
import scipy.linalg as sla

from . import ctd, fullgrid


def eigenpairs(ops: ctd.Operators, d: int):
    """``(lambda, V)`` with ``K_d V = M_d V diag(lambda)`` and ``V^T M_d V = I`` (LAPACK)."""
    return sla.eigh(ops.K[d].toarray(), ops.M[d].toarray())


def cfe_step(prob: ctd.Problem, ops: ctd.Operators, U: np.ndarray) -> np.ndarray:
    """Full-grid ``u^{k+1}`` from the full-grid nodal coefficients ``U`` of ``u^k`` by fast
    diagonalisation (Eq. AC-discrete-semi-stable-K on the tensor-product C-FEM space)."""
    D = prob.dim
    pairs = [eigenpairs(ops, d) for d in range(D)]
    # right-hand side c_t M u^k - int N~ L w(u^k) at the nodes (its own quadrature rule)
    Q = -ctd.from_quadrature_grid(ops, grid_source(prob, ops, U))
    # y = (x)V^T Q; divide by the diagonal; u = (x)V y
    Y = Q
    for d in range(D):
        Y = ctd.apply_along(pairs[d][1].T, Y, d)
    diag = np.full(Y.shape, prob.c_t)
    for d in range(D):
        sh = [1] * D
        sh[d] = -1
        diag = diag + prob.c_k * pairs[d][0].reshape(sh)
    Y = Y / diag
    for d in range(D):
        Y = ctd.apply_along(pairs[d][1], Y, d)
    return Y


def grid_source(prob: ctd.Problem, ops: ctd.Operators, U: np.ndarray) -> np.ndarray:
    """``G = prod_d omega_d (L w(u^k) - c_t u^k)`` at the quadrature points, from the
    full-grid nodal coefficients ``U``.  Its projection onto the shape functions is
    ``int N~ L w(u^k) - c_t M u^k``, so as the nonlinear operator of ``ctd.step`` (with no
    factors of u^k) it gives the right-hand side of Eq. KxQx with u^k on the full grid."""
    Uq = U
    for d in range(prob.dim):
        Uq = ctd.apply_along(ops.Phi[d], Uq, d) if ops.Phi is not None else Uq
    return ctd.grid_weights(ops) * (prob.L * ctd.w_of_u(Uq, prob.a0) - prob.c_t * Uq)


def step(prob: ctd.Problem, ops: ctd.Operators, state, M_c: int, step_index: int = 0):
    """One ACTD time step.  ``state`` is ``("modes", A)`` (factors of u^k) or ``("grid", U)``
    (full-grid nodal coefficients).  Returns ``(new_state, stats)``; ``stats["switched"]``
    says whether the step was solved on the full grid."""
    kind, data = state
    budget = min(prob.M_max, M_c + 1)
    sub = ctd.Problem(**{**prob.__dict__, "M_max": budget})
    if kind == "modes":
        B, st = ctd.step(sub, ops, data, step_index)
    else:
        empty = [np.zeros((prob.n[d], 0)) for d in range(prob.dim)]
        B, st = ctd.step(sub, ops, empty, step_index, nl=("grid", grid_source(prob, ops, data)))
    if st["modes"] <= M_c:       # (a capped step here has M_max <= M_c modes)
        st["switched"] = False
        return ("modes", B), st
    U = data if kind == "grid" else ctd.reconstruct(data)
    return ("grid", cfe_step(prob, ops, U)), {"switched": True, "ctd_modes_tried": st["modes"]}


def field(state) -> np.ndarray:
    """Full-grid nodal coefficients of a state."""
    kind, data = state
    return data if kind == "grid" else ctd.reconstruct(data)


def energy(prob: ctd.Problem, ops: ctd.Operators, state) -> float:
    """Discrete energy of a state (``ctd.energy`` on factors, ``fullgrid.energy`` on a grid)."""
    kind, data = state
    if kind == "modes":
        return ctd.energy(prob, ops, data)
    return fullgrid.energy(prob, ops, data)


def run(prob: ctd.Problem, ops: ctd.Operators, A0: Sequence[np.ndarray], nsteps: int, M_c: int):
    """Advance ``nsteps`` ACTD steps from factors ``A0``; returns (state, list of stats)."""
    state = ("modes", [np.asarray(a, dtype=np.float64) for a in A0])
    hist = []
    for k in range(nsteps):
        state, st = step(prob, ops, state, M_c, k)
        hist.append(st)
    return state, hist
