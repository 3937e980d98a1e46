"""CTD solution of the stabilized semi-implicit Allen-Cahn step -- oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

What is computed (paper passages):
  * Eq. AC (Section 2.1): ``u_t + L (w(u) - kappa Lap u) = 0``, ``w = dF/du``, with
    ``F(u) = a0 (u^2 - 1)^2`` (Eq. energyfunction), so ``w(u) = 4 a0 (u^3 - u)``.
  * Eq. AC-discrete-semi-stable-K (Section 2.5): each time step solves ``K u = Q`` with
    ``K = c_t M + c_k K_stiff`` and ``Q = c_t M u^k - int N^T L w(u^k)``, where
    ``c_t = 1/dt + alpha L`` and ``c_k = L kappa``.
  * Eq. CTD (Section 3.1): ``u = sum_m prod_d u_d^(m)``.
  * Section 3.3 and App. D: greedy enrichment; each new mode is found by the alternating
    fixed point (fix every factor but one, solve Eq. ux ``K_x u_x = Q_x`` with ``K_x`` and
    ``Q_x`` from Eq. KxQx / Eq. KyQy), sweeping x -> y (-> z) until the mode stops
    changing; stop adding modes once a mode's size is negligible.
  * Eq. KxxMxx: ``M_xy = int N~_x^T N~_y L w(u^k) dx dy``, the nonlinear term.
  * Eq. MxySep (Section 3.3): the same term from a separated form ``w = sum_q prod_d w_d^(q)``
    of the nonlinearity, integrated as products of 1D integrals.

Readings of silent or ambiguous points (each also listed in the design notes):
  * Quadrature (the paper only mentions "Gauss points" for the reduced domain): all
    mass-type integrals -- ``M_dd``, ``M_xy`` and ``int F`` in the energy -- share one rule;
    the stiffness is integrated exactly (see ``cfem``).  The default (``quad_rule =
    "nodal"``) is the nodal trapezoid rule, so ``M_dd = diag(omega_d)`` and ``[M_xy]_ij = L
    omega_x[i] omega_y[j] w(u^k(x_i, y_j))``.  ``quad_rule = "gauss"`` takes ``quad_q``
    Gauss points per element (weights ``omega_d``, shape function values ``Phi_d``):
    ``M_dd = Phi_d^T diag(omega_d) Phi_d`` (the exact consistent mass of Eq. KxxMxx for
    ``quad_q >= 5``), ``w(u^k)`` is evaluated at the tensor-product Gauss points and its
    integral against ``N~_x N~_y`` is ``Phi_x^T`` of the weighted sums there.
  * The 3D equations follow from the same derivation as App. D with one more factor.
  * Start of a mode: the previous step's mode of the same index if it exists and is not
    identically zero, else the SplitMix64 vector of ``splitmix``.
  * Scaling: after each solve the factor is normalised to unit 2-norm unless it is the
    last dimension; a committed mode gets equal 2-norms in every factor.
  * Mode convergence (paper: ``max|(u_x u_y^T)^(i) - (u_x u_y^T)^(i-1)| <= eps1``): the
    relative Frobenius change ``||(x)v - (x)v_old||_F / ||(x)v||_F <= tol_als``, evaluated
    exactly from 1D inner products (``rel_change``); at most ``I_max`` sweeps.
  * Enrichment stop (paper: ``max|u_x u_y^T| <= eps2``): ``prod_d max|v_d| <= tol_enrich``
    (exactly the max of the rank-1 tensor); the failing mode is discarded.  Reaching
    ``M_max`` committed modes ends the step with the "capped" flag.
  * Stall rule (optional, ``als_stall_tol > 0``; off by default): the paper's own example
    test is an absolute one, ``max|Delta(u_x u_y^T)| <= eps1``, i.e. a change measured in
    the units of the field.  Read that way, a mode whose change, in units of the step's
    leading mode (``delta * amp <= als_stall_tol * amp_lead``, ``amp = prod_d max|v_d|``,
    ``amp_lead`` the leading mode's amplitude, the mode's own for mode 0), is small and no
    longer shrinking (``delta >= delta_prev / 2``) after at least 3 sweeps ends its sweeps.
    Such a mode has not met ``tol_als``: it is counted as stalled and the step reports
    ``als_not_converged``.
  * If a solve returns an all-zero factor the mode is zero: its sweep stops at once and the
    enrichment test discards it.
  * Separated nonlinearity (the paper names SVD or HOPGD for the decomposition of w(u^k)):
    for the cubic w and a separated u^k the decomposition is exact and needs neither --
    ``u^3`` expands into one separated term per multiset {m1, m2, m3} of mode indices
    (weight = its number of orderings) and ``-u`` into one per mode, so
    Q = C(M_k + 2, 3) + M_k terms reproduce w(u^k) on the grid up to rounding.  It is used
    for steps with M_k <= ``separated_max_modes`` and the full integral otherwise.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import cfem
from .splitmix import mode_init_vector


@dataclasses.dataclass
class Problem:
    """Parameters of one Allen-Cahn CTD run (Table coef symbols: L, kappa, a0, alpha)."""
    dim: int
    n: Sequence[int]
    length: Sequence[float]
    s: int
    p: int
    a: float
    L: float
    kappa: float
    a0: float
    alpha: float
    dt: float
    M_max: int
    I_max: int
    tol_als: float
    tol_enrich: float
    seed: int = 0
    fixed_als_iters: int = 0   # >0: exactly this many sweeps per mode (strict-parity mode)
    fixed_modes: int = 0       # >0: exactly this many modes per step (strict-parity mode)
    als_stall_tol: float = 0.0  # >0: stall rule of the fixed-point sweeps (see the readings)
    reduced_tol: float = 0.0   # >0: reduced integration domain (Section 3.3), see below
    reduced_block: int = 128   # nodes per dimension of the element blocks it keeps or drops
    nonlinear_form: str = "grid"   # "grid" (Eq. KxxMxx) or "separated" (Eq. MxySep)
    separated_max_modes: int = 16  # separated form only for steps with M_k up to this
    quad_rule: str = "nodal"       # "nodal" (trapezoid at the nodes) or "gauss" (see above)
    quad_q: int = 5                # Gauss points per element for quad_rule == "gauss"

    @property
    def c_t(self) -> float:
        return 1.0 / self.dt + self.alpha * self.L

    @property
    def c_k(self) -> float:
        return self.L * self.kappa


@dataclasses.dataclass
class Operators:
    omega: List[np.ndarray]       # quadrature weights per dimension (the nodes' for "nodal")
    M: List[sp.csr_matrix]        # M_dd = Phi_d^T diag(omega_d) Phi_d (diag(omega_d) for "nodal")
    K: List[sp.csr_matrix]        # K_dd = int B~^T B~
    Phi: Optional[List[sp.csr_matrix]] = None   # shape functions at the Gauss points, or None


def build_operators(prob: Problem) -> Operators:
    omega, M, K, Phi = [], [], [], []
    for d in range(prob.dim):
        n, length = prob.n[d], prob.length[d]
        if prob.quad_rule == "nodal":
            w = cfem.nodal_weights(n, length)
            M.append(sp.diags(w).tocsr())
        elif prob.quad_rule == "gauss":
            _, w = cfem.gauss_quadrature(n, length, prob.quad_q)
            ph = cfem.quadrature_basis(n, length, prob.s, prob.p, prob.a, prob.quad_q)
            Phi.append(ph)
            M.append((ph.T @ sp.diags(w) @ ph).tocsr())
        else:
            raise ValueError(f"unknown quadrature rule {prob.quad_rule!r}")
        omega.append(w)
        K.append(cfem.stiffness_matrix(n, length, prob.s, prob.p, prob.a))
    return Operators(omega, M, K, Phi if Phi else None)


def at_quadrature(ops: Operators, d: int, f: np.ndarray) -> np.ndarray:
    """Values at the quadrature points of dimension ``d`` of 1D functions with nodal
    coefficients ``f`` (a vector or an n_d x m matrix): ``Phi_d f``, or ``f`` itself under
    the nodal rule (Kronecker delta property)."""
    return f if ops.Phi is None else ops.Phi[d] @ f


def from_quadrature(ops: Operators, d: int, r: np.ndarray) -> np.ndarray:
    """``Phi_d^T r``: from weighted values at the quadrature points to the integrals against
    each shape function of dimension ``d`` (identity under the nodal rule)."""
    return r if ops.Phi is None else ops.Phi[d].T @ r


def w_of_u(u, a0):
    """``w(u) = dF/du = 4 a0 (u^3 - u)`` for ``F = a0 (u^2 - 1)^2`` (Eq. energyfunction)."""
    return 4.0 * a0 * (u ** 3 - u)


def reconstruct(modes: Sequence[np.ndarray]) -> np.ndarray:
    """Full-grid nodal values of ``sum_m prod_d u_d^(m)`` (Eq. CTD).  Kronecker delta
    property: nodal coefficients are nodal values."""
    D = len(modes)
    shape = tuple(m.shape[0] for m in modes)
    if modes[0].shape[1] == 0:
        return np.zeros(shape)
    if D == 2:
        return modes[0] @ modes[1].T
    return np.einsum("im,jm,lm->ijl", modes[0], modes[1], modes[2])


def grid_weights(ops: Operators) -> np.ndarray:
    """Tensor product of the 1D nodal weights."""
    W = ops.omega[0]
    for w in ops.omega[1:]:
        W = np.multiply.outer(W, w)
    return W


def reduced_domain_mask(prob: Problem, W: np.ndarray) -> np.ndarray:
    """Reduced integration domain (Section 3.3: keep only where ``w(u^k)`` is not close to
    zero).  Reading: the grid is cut into blocks of ``reduced_block`` nodes per dimension
    (the last block of a dimension may be shorter); a block stays in the domain when the
    largest ``|w(u^k)|`` at its nodes exceeds ``reduced_tol``, else its nodes drop out of the
    nonlinear integral.  ``reduced_tol <= 0`` keeps every node."""
    keep = np.ones(W.shape, dtype=bool)
    if prob.reduced_tol <= 0.0:
        return keep
    B = prob.reduced_block
    nb = [(n + B - 1) // B for n in W.shape]
    for blk in np.ndindex(*nb):
        sl = tuple(slice(b * B, min((b + 1) * B, n)) for b, n in zip(blk, W.shape))
        if not np.max(np.abs(W[sl])) > prob.reduced_tol:
            keep[sl] = False
    return keep


def from_quadrature_grid(ops: Operators, G: np.ndarray) -> np.ndarray:
    """``(x)_d Phi_d^T G``: integrals against every product shape function of a D-way array
    of weighted values at the quadrature points (``G`` itself under the nodal rule)."""
    if ops.Phi is None:
        return G
    for d in range(G.ndim):
        G = apply_along(ops.Phi[d].T, G, d)
    return G


def nonlinear_tensor(prob: Problem, ops: Operators, A: Sequence[np.ndarray]) -> np.ndarray:
    """The nonlinear operator of Eq. KxxMxx at the quadrature points, as a D-way array:
    ``Mxy[i, j(, l)] = L prod_d omega_d w(u^k(x_i, y_j(, z_l)))``, zero outside the reduced
    domain when one is set (nodal rule only: its blocks are blocks of nodes)."""
    if ops.Phi is not None and prob.reduced_tol > 0.0:
        raise ValueError("the reduced integration domain is defined for the nodal rule only")
    U = reconstruct([at_quadrature(ops, d, A[d]) for d in range(prob.dim)])
    W = w_of_u(U, prob.a0)
    return prob.L * grid_weights(ops) * W * reduced_domain_mask(prob, W)


def separated_nonlinear_terms(prob: Problem, A: Sequence[np.ndarray], ops: Optional[Operators] = None):
    """Exact separated form of ``w(u^k) = 4 a0 (u^3 - u)`` for ``u^k = sum_m prod_d A[d][:, m]``
    (Eq. energyfunction for w; used by Eq. MxySep): a list of ``(c_q, [f_q,d for d])`` with
    ``w = sum_q c_q prod_d f_q,d``.  The cubic gives one term per multiset m1 <= m2 <= m3
    (``f = A[:, m1] A[:, m2] A[:, m3]``, ``c = 4 a0`` times the multiset's orderings); the
    linear part gives ``c = -4 a0``, ``f = A[:, m]``.  The ``f`` are values at the
    quadrature points of ``ops`` (at the nodes when ``ops`` is None or nodal)."""
    D = prob.dim
    if ops is not None:
        A = [at_quadrature(ops, d, A[d]) for d in range(D)]
    Mk = A[0].shape[1]
    terms = []
    for m1 in range(Mk):
        for m2 in range(m1, Mk):
            for m3 in range(m2, Mk):
                orderings = 6 if (m1 != m2 and m2 != m3) else (1 if m1 == m3 else 3)
                f = [A[d][:, m1] * A[d][:, m2] * A[d][:, m3] for d in range(D)]
                terms.append((4.0 * prob.a0 * orderings, f))
    for m in range(Mk):
        terms.append((-4.0 * prob.a0, [A[d][:, m].copy() for d in range(D)]))
    return terms


def separated_contraction(prob: Problem, ops: Operators, terms, v: Sequence[np.ndarray], x: int) -> np.ndarray:
    """``M_xy`` of Eq. MxySep applied to the fixed factors: ``sum_q L c_q Phi_x^T (omega_x
    f_q,x) prod_{d != x} (f_q,d . omega_d Phi_d v_d)`` (the shared rule for every 1D integral;
    ``Phi = I`` under the nodal rule)."""
    out = np.zeros(len(ops.omega[x]))
    for c, f in terms:
        s = prob.L * c
        for d in range(prob.dim):
            if d != x:
                s = s * float(f[d] @ (ops.omega[d] * at_quadrature(ops, d, v[d])))
        out = out + s * (ops.omega[x] * f[x])
    return from_quadrature(ops, x, out)


def nonlinear_projection(prob: Problem, ops: Operators, nl, v: Sequence[np.ndarray], x: int) -> np.ndarray:
    """``M_xy u_y`` (and its D-way analogue): ``nl`` is ``("grid", Mxy)`` or
    ``("separated", terms)``."""
    kind, data = nl
    if kind == "grid":
        vq = [at_quadrature(ops, d, v[d]) for d in range(prob.dim)]
        return from_quadrature(ops, x, contract_except(data, vq, x))
    return separated_contraction(prob, ops, data, v, x)


def nonlinear_operator(prob: Problem, ops: Operators, A: Sequence[np.ndarray]):
    """The nonlinear term of a step in the form the problem asks for (see the readings)."""
    Mk = A[0].shape[1]
    if prob.nonlinear_form == "separated" and 0 < Mk <= prob.separated_max_modes:
        return ("separated", separated_nonlinear_terms(prob, A, ops))
    return ("grid", nonlinear_tensor(prob, ops, A))


def contract_except(T: np.ndarray, vecs: Sequence[np.ndarray], keep: int) -> np.ndarray:
    """Contract the D-way array ``T`` with ``vecs[d]`` on every axis except ``keep``."""
    out = T
    for d in reversed(range(T.ndim)):
        if d != keep:
            out = np.tensordot(out, vecs[d], axes=([d], [0]))
    return out


def to_upper_band(A: sp.spmatrix):
    """Upper banded storage (LAPACK ``pbsv`` layout) of a symmetric sparse matrix."""
    A = A.tocoo()
    b = int(np.max(np.abs(A.row - A.col))) if A.nnz else 0
    n = A.shape[0]
    ab = np.zeros((b + 1, n))
    Ad = A.tocsr()
    for k in range(b + 1):
        ab[b - k, k:] = Ad.diagonal(k)
    return ab


def banded_spd_solve(A: sp.spmatrix, rhs: np.ndarray) -> np.ndarray:
    """Solve ``A x = rhs`` for a symmetric positive definite banded ``A`` (LAPACK)."""
    return sla.solveh_banded(to_upper_band(A), rhs)


def rel_change(new: Sequence[np.ndarray], old: Sequence[np.ndarray]) -> float:
    """``||(x)new - (x)old||_F / ||(x)new||_F`` for rank-1 tensors, from 1D products.

    Telescoping: ``(x)new - (x)old = sum_d T_d`` with ``T_d = old_0 (x) .. old_{d-1} (x)
    (new_d - old_d) (x) new_{d+1} (x) ..``; ``||sum T_d||^2 = sum_{d,e} prod_c
    <T_d(c), T_e(c)>``.  Every factor is a difference or an iterate, so no cancellation of
    two nearly equal squared norms occurs.
    """
    D = len(new)
    delta = [new[c] - old[c] for c in range(D)]

    def factor(d, c):
        if c < d:
            return old[c]
        if c == d:
            return delta[c]
        return new[c]

    num = 0.0
    for d in range(D):
        for e in range(D):
            prod = 1.0
            for c in range(D):
                prod *= float(factor(d, c) @ factor(e, c))
            num += prod
    den = 1.0
    for c in range(D):
        den *= float(new[c] @ new[c])
    if den == 0.0:
        return 0.0
    return float(np.sqrt(max(num, 0.0) / den))


def half_sweep(prob: Problem, ops: Operators, x: int, v: List[np.ndarray],
               A: Sequence[np.ndarray], B: Sequence[np.ndarray], Mxy):
    """Fix every factor but ``v[x]`` and solve Eq. ux for it (Eq. KxQx, generalised to D).

    Returns the new ``v[x]`` (not normalised) and ``(alpha1, alpha2)``.
    """
    D = prob.dim
    c_t, c_k = prob.c_t, prob.c_k
    others = [d for d in range(D) if d != x]
    Mx, Kx = ops.M[x], ops.K[x]

    # Gram products of the fixed factors (App. D: u_y^T M_yy u_y, u_y^T K_yy u_y, ...)
    m = {d: float(v[d] @ (ops.M[d] @ v[d])) for d in others}
    k = {d: float(v[d] @ (ops.K[d] @ v[d])) for d in others}
    hA = {d: A[d].T @ (ops.M[d] @ v[d]) for d in others}     # u_d^T M u_d^(m,k)
    gM = {d: B[d].T @ (ops.M[d] @ v[d]) for d in others}     # u_d^T M u_d^(m)
    gK = {d: B[d].T @ (ops.K[d] @ v[d]) for d in others}     # u_d^T K u_d^(m)

    prod_m = np.prod([m[d] for d in others])
    stiff = 0.0
    for dp in others:
        stiff += k[dp] * np.prod([m[d] for d in others if d != dp])
    alpha1 = c_t * prod_m + c_k * stiff     # coefficient of M_xx in K_x
    alpha2 = c_k * prod_m                   # coefficient of K_xx in K_x

    Mk = A[x].shape[1]
    Mc = B[x].shape[1]
    H = np.ones(Mk)
    for d in others:
        H = H * hA[d]
    GM = np.ones(Mc)
    for d in others:
        GM = GM * gM[d]
    GK = np.zeros(Mc)
    for dp in others:
        term = gK[dp].copy()
        for d in others:
            if d != dp:
                term = term * gM[d]
        GK = GK + term

    # right-hand side, in the term order of Eq. KxQx
    Q = c_t * (Mx @ (A[x] @ H))                 # + sum_m c_t M_xx u_x^(m,k) (...)
    Q = Q - c_t * (Mx @ (B[x] @ GM))            # - sum_m c_t M_xx u_x^(m) (...)
    if not isinstance(Mxy, tuple):
        Mxy = ("grid", Mxy)
    Q = Q - nonlinear_projection(prob, ops, Mxy, v, x)   # - M_xy u_y
    Q = Q - c_k * (Kx @ (B[x] @ GM))            # - sum_m L kappa K_xx u_x^(m) (...)
    Q = Q - c_k * (Mx @ (B[x] @ GK))            # - sum_m L kappa M_xx u_x^(m) (u^T K u^(m))

    Ksys = alpha1 * Mx + alpha2 * Kx
    vx = banded_spd_solve(Ksys, Q)
    return vx, (alpha1, alpha2)


def init_mode(prob: Problem, A: Sequence[np.ndarray], step_index: int, m: int):
    v = []
    for d in range(prob.dim):
        if m < A[d].shape[1] and np.any(A[d][:, m] != 0.0):
            v.append(A[d][:, m].astype(np.float64).copy())
        else:
            v.append(mode_init_vector(prob.seed, step_index, m, d, prob.n[d]))
    return v


def step(prob: Problem, ops: Operators, A: Sequence[np.ndarray], step_index: int = 0,
         trace=None, nl=None):
    """One time step u^k -> u^{k+1}; ``A[d]`` holds u^k's factors (n_d x M_k).

    Returns ``(B, stats)`` with ``B[d]`` the n_d x M factors of u^{k+1}.  ``trace``, if a
    list, receives ``(mode, sweep, x, v_copy)`` after every half-sweep (for tests).  ``nl``,
    if given, replaces the nonlinear operator built from ``A`` (the adaptive scheme passes
    a full-grid one, with ``A`` empty).
    """
    D = prob.dim
    A = [np.asarray(a, dtype=np.float64) for a in A]
    Mxy = nonlinear_operator(prob, ops, A) if nl is None else nl
    B = [np.zeros((prob.n[d], 0)) for d in range(D)]
    stats = {"modes": 0, "als_iters": [], "als_delta": [], "amplitude": [],
             "capped": False, "als_not_converged": False, "als_stalled": 0}
    n_modes = prob.fixed_modes if prob.fixed_modes > 0 else prob.M_max
    stopped = False
    amp_lead = 0.0
    for m in range(n_modes):
        v = init_mode(prob, A, step_index, m)
        zero_mode = False
        delta = np.inf
        delta_prev = np.inf
        it = 0
        n_it = prob.fixed_als_iters if prob.fixed_als_iters > 0 else prob.I_max
        for it in range(1, n_it + 1):
            v_old = [x.copy() for x in v]
            for x in range(D):
                vx, _ = half_sweep(prob, ops, x, v, A, B, Mxy)
                if not np.any(vx != 0.0):
                    zero_mode = True
                    v[x] = vx
                    break
                if x != D - 1:
                    vx = vx / np.linalg.norm(vx)
                v[x] = vx
                if trace is not None:
                    trace.append((m, it, x, [y.copy() for y in v]))
            if zero_mode:
                break
            delta = rel_change(v, v_old)
            if prob.fixed_als_iters == 0 and delta <= prob.tol_als:
                break
            if prob.als_stall_tol > 0.0 and prob.fixed_als_iters == 0 and it >= 3:
                # stall rule (readings): the change in units of the leading mode, no longer shrinking
                amp = float(np.prod([np.max(np.abs(y)) for y in v]))
                lead = amp if m == 0 else amp_lead
                if delta * amp <= prob.als_stall_tol * lead and delta >= 0.5 * delta_prev:
                    stats["als_stalled"] += 1
                    break
            delta_prev = delta
        converged = zero_mode or prob.fixed_als_iters > 0 or delta <= prob.tol_als
        if not converged:
            stats["als_not_converged"] = True
        amp = 0.0 if zero_mode else float(np.prod([np.max(np.abs(x)) for x in v]))
        if m == 0:
            amp_lead = amp
        stats["als_iters"].append(it)
        stats["als_delta"].append(0.0 if zero_mode else float(delta))
        stats["amplitude"].append(amp)
        if prob.fixed_modes == 0 and amp <= prob.tol_enrich:
            stopped = True
            break
        # commit with equal 2-norms in every factor
        norms = [np.linalg.norm(x) for x in v]
        target = np.prod(norms) ** (1.0 / D)
        for d in range(D):
            B[d] = np.column_stack([B[d], v[d] * (target / norms[d])])
    stats["modes"] = B[0].shape[1]
    stats["capped"] = (prob.fixed_modes == 0) and (not stopped)
    return B, stats


def energy(prob: Problem, ops: Operators, modes: Sequence[np.ndarray]) -> float:
    """Discrete energy ``E_h(u) = sum_grid omega F(u) + 1/2 kappa u^T K_grad u``.

    ``F`` is integrated with the step's rule (at the nodes or the Gauss points); the
    gradient term uses the exact 1D stiffness along one axis and the mass along the others
    (same operators as the step).
    """
    U = reconstruct(modes)
    Wg = grid_weights(ops)
    if ops.Phi is not None:
        Uq = reconstruct([at_quadrature(ops, d, modes[d]) for d in range(prob.dim)])
        bulk = float(np.sum(Wg * prob.a0 * (Uq ** 2 - 1.0) ** 2))
        grad = 0.0
        for d in range(prob.dim):
            T = U
            for e in range(prob.dim):
                T = apply_along(ops.K[e] if e == d else ops.M[e], T, e)
            grad += float(np.sum(U * T))
        return bulk + 0.5 * prob.kappa * grad
    bulk = float(np.sum(Wg * prob.a0 * (U ** 2 - 1.0) ** 2))
    grad = 0.0
    for d in range(prob.dim):
        T = np.moveaxis(U, d, 0)
        shape = T.shape
        KT = (ops.K[d] @ T.reshape(shape[0], -1)).reshape(shape)
        KT = np.moveaxis(KT, 0, d)
        other_w = np.ones_like(U)
        for e in range(prob.dim):
            if e != d:
                sh = [1] * prob.dim
                sh[e] = -1
                other_w = other_w * ops.omega[e].reshape(sh)
        grad += float(np.sum(U * KT * other_w))
    return bulk + 0.5 * prob.kappa * grad


def apply_along(mat, T: np.ndarray, axis: int) -> np.ndarray:
    """Multiply the D-way array ``T`` by the matrix ``mat`` along ``axis``."""
    Tm = np.moveaxis(T, axis, 0)
    shape = Tm.shape
    out = (mat @ Tm.reshape(shape[0], -1)).reshape((mat.shape[0],) + shape[1:])
    return np.moveaxis(out, 0, axis)


def run(prob: Problem, ops: Operators, A0: Sequence[np.ndarray], nsteps: int,
        first_step: int = 0, energies: bool = False):
    """Advance ``nsteps`` steps from factors ``A0``; returns (factors, list of stats)."""
    A = [np.asarray(a, dtype=np.float64) for a in A0]
    hist = []
    for k in range(nsteps):
        A, st = step(prob, ops, A, first_step + k)
        if energies:
            st["energy"] = energy(prob, ops, A)
        hist.append(st)
    return A, hist


def rel_l2_between(modes_a: Sequence[np.ndarray], modes_b: Sequence[np.ndarray]) -> float:
    """Relative Euclidean distance ``||a - b|| / ||b||`` of two separated fields, on the
    nodes (both reconstructed on the full grid, so tiny differences are not lost)."""
    Ua = reconstruct(modes_a)
    Ub = reconstruct(modes_b)
    nb = float(np.linalg.norm(Ub))
    diff = float(np.linalg.norm(Ua - Ub))
    return diff / nb if nb > 0 else diff
