"""1D convolution finite element (C-FEM) shape functions and matrices -- oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed:
  * Eq. CFEM / Eq. CFEM-1D (Section 3.2, App. C): the C-FEM approximation on element
    ``e`` is ``sum_{i in A^e} N_i(xi) sum_{j in A^i_s} W^{xi_i}_{a,j}(xi) u_j``.
  * App. B: the patch function ``W = Psi_a(xi) K + p(xi) L`` with
    ``L = (P^T R0^-1 P)^-1 P^T R0^-1`` and ``K = R0^-1 (I - P L)``, cubic spline kernel
    ``Psi_a(z)``, ``z = |xi - xi_I| / a``, monomial basis ``p = [1, xi, ..., xi^p]``.
  * Eq. KxxMxx: ``K_xx = int B~^T B~ dx``, ``M_xx = int N~^T N~ dx``.

Readings (the paper is silent or defers to another paper that is not available):
  * Natural coordinate of element ``e = [x_e, x_{e+1}]`` is ``xi in [-1, 1]``; node ``j``
    sits at ``xi_j = -1 + 2 (j - e)`` (the App. B example places the patch of node 2 at
    ``{-3, -1, 1}``).  The dilation ``a`` is measured in these natural units.
  * Nodal patch ``A^i_s = {max(0, i-s) .. min(n-1, i+s)}``: near the boundary the patch is
    truncated ("reduced by ignoring the part outside the domain", Section 3.2).
  * Mass-type integrals use the nodal (trapezoid) rule, so by the Kronecker delta property
    ``M_dd = diag(omega)``; the stiffness integral is exact (Gauss-Legendre, 5 points per
    element, exact because ``N~`` is a polynomial of degree <= 4 on each element when the
    kernel's break points fall on element ends, which holds for a = 12, s <= 3).
  * The Gauss variant (``gauss_quadrature``, ``quadrature_basis``) evaluates the shape
    functions at ``q`` Gauss points per element instead; with ``q >= 5`` the mass
    ``Phi^T diag(omega) Phi`` is the exact consistent mass of Eq. KxxMxx.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def psi(z):
    """Cubic spline kernel Psi_a(z) of App. B for z >= 0 (piecewise cubic, zero beyond 1)."""
    z = np.abs(np.asarray(z, dtype=np.float64))
    out = np.zeros_like(z)
    m1 = z <= 0.5
    m2 = (z > 0.5) & (z <= 1.0)
    z1 = z[m1]
    z2 = z[m2]
    out[m1] = 2.0 / 3.0 - 4.0 * z1 ** 2 + 4.0 * z1 ** 3
    out[m2] = 4.0 / 3.0 - 4.0 * z2 + 4.0 * z2 ** 2 - (4.0 / 3.0) * z2 ** 3
    return out


def dpsi_dz(z):
    """Derivative of ``psi`` with respect to z, for z >= 0."""
    z = np.abs(np.asarray(z, dtype=np.float64))
    out = np.zeros_like(z)
    m1 = z <= 0.5
    m2 = (z > 0.5) & (z <= 1.0)
    z1 = z[m1]
    z2 = z[m2]
    out[m1] = -8.0 * z1 + 12.0 * z1 ** 2
    out[m2] = -4.0 + 8.0 * z2 - 4.0 * z2 ** 2
    return out


def monomials(xi, p):
    """Rows ``p(xi) = [1, xi, ..., xi^p]`` (App. B polynomial basis)."""
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    return np.stack([xi ** q for q in range(p + 1)], axis=1)


def dmonomials(xi, p):
    """d/dxi of ``monomials``."""
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    cols = [np.zeros_like(xi)] + [q * xi ** (q - 1) for q in range(1, p + 1)]
    return np.stack(cols, axis=1)


def rbf_coefficients(xi_nodes, a, p):
    """Matrices ``K`` (n_p x n_p) and ``L`` ((p+1) x n_p) of the App. B interpolation.

    ``R0[j, l] = Psi_a(|xi_j - xi_l| / a)`` and ``P[j, :] = p(xi_j)`` (App. B, Eq. moment);
    ``L = (P^T R0^-1 P)^-1 P^T R0^-1`` and ``K = R0^-1 (I - P L)``.
    """
    xi_nodes = np.asarray(xi_nodes, dtype=np.float64)
    R0 = psi(np.abs(xi_nodes[:, None] - xi_nodes[None, :]) / a)
    P = monomials(xi_nodes, p)
    R0inv = np.linalg.inv(R0)
    L = np.linalg.solve(P.T @ R0inv @ P, P.T @ R0inv)
    K = R0inv @ (np.eye(len(xi_nodes)) - P @ L)
    return K, L


def rbf_eval(xi, xi_nodes, K, L, a, p):
    """Patch functions ``W(xi) = Psi_a(xi) K + p(xi) L`` and ``dW/dxi`` at points ``xi``.

    Returns two arrays of shape (len(xi), n_p); column j is ``W^{xi_i}_{a,j}``.
    """
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    d = xi[:, None] - np.asarray(xi_nodes, dtype=np.float64)[None, :]
    Psi = psi(np.abs(d) / a)
    dPsi = dpsi_dz(np.abs(d) / a) * np.sign(d) / a
    W = Psi @ K + monomials(xi, p) @ L
    dW = dPsi @ K + dmonomials(xi, p) @ L
    return W, dW


def nodal_patch(i, n, s):
    """``A^i_s``: nodes within ``s`` of node ``i``, truncated at the domain ends."""
    return np.arange(max(0, i - s), min(n - 1, i + s) + 1)


def element_shape(e, n, s, p, a, xi):
    """C-FEM shape functions of element ``e`` at natural points ``xi`` (Eq. CFEM-1D).

    Returns ``(support, N, dN_dxi)``: ``support`` is ``A^e_s`` (global node ids, the union
    of the two end nodes' patches), ``N[q, k]`` is ``N~_{support[k]}(xi_q)``.
    """
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    support = np.arange(max(0, e - s), min(n - 1, e + 1 + s) + 1)
    N = np.zeros((len(xi), len(support)))
    dN = np.zeros((len(xi), len(support)))
    # linear FE shape functions of the two end nodes and their xi-derivatives
    ends = ((e, (1.0 - xi) / 2.0, -0.5), (e + 1, (1.0 + xi) / 2.0, 0.5))
    for i, Ni, dNi in ends:
        patch = nodal_patch(i, n, s)
        xi_nodes = -1.0 + 2.0 * (patch - e)
        K, L = rbf_coefficients(xi_nodes, a, p)
        W, dW = rbf_eval(xi, xi_nodes, K, L, a, p)
        cols = patch - support[0]
        N[:, cols] += Ni[:, None] * W
        dN[:, cols] += dNi * W + Ni[:, None] * dW
    return support, N, dN


def gauss_legendre(q):
    """q-point Gauss-Legendre rule on [-1, 1] (numpy's leggauss)."""
    return np.polynomial.legendre.leggauss(q)


def stiffness_matrix(n, length, s, p, a, gauss_points=5):
    """``K_dd = int B~^T B~ dx`` over ``[0, length]`` with ``n`` nodes (Eq. KxxMxx).

    Element by element: ``dx = (h/2) dxi`` and ``d/dx = (2/h) d/dxi``.  Returned as a
    scipy CSR matrix of shape (n, n).
    """
    h = length / (n - 1)
    xg, wg = gauss_legendre(gauss_points)
    rows, cols, vals = [], [], []
    for e in range(n - 1):
        support, _, dN = element_shape(e, n, s, p, a, xg)
        Ke = (2.0 / h) * (dN.T * wg) @ dN
        rr, cc = np.meshgrid(support, support, indexing="ij")
        rows.append(rr.ravel())
        cols.append(cc.ravel())
        vals.append(Ke.ravel())
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()
    K.sum_duplicates()
    return K


def consistent_mass_matrix(n, length, s, p, a, gauss_points=5):
    """``M_dd = int N~^T N~ dx`` integrated exactly (Eq. KxxMxx), for reference tests."""
    h = length / (n - 1)
    xg, wg = gauss_legendre(gauss_points)
    M = np.zeros((n, n))
    for e in range(n - 1):
        support, N, _ = element_shape(e, n, s, p, a, xg)
        M[np.ix_(support, support)] += (h / 2.0) * (N.T * wg) @ N
    return M


def gauss_quadrature(n, length, q):
    """Composite ``q``-point Gauss-Legendre rule over the ``n - 1`` elements of ``[0, length]``.

    Returns ``(x, omega)`` of length ``q (n - 1)``, ordered element by element: on element
    ``e`` the points are ``x_e + (1 + xi_g) h / 2`` with weights ``w_g h / 2`` (the Gauss
    points of each element of Section 3.3).
    """
    h = length / (n - 1)
    xg, wg = gauss_legendre(q)
    e = np.arange(n - 1)[:, None]
    x = (e * h + (1.0 + xg[None, :]) * (h / 2.0)).reshape(-1)
    omega = np.tile(wg * (h / 2.0), n - 1)
    return x, omega


def quadrature_basis(n, length, s, p, a, q):
    """``Phi[r, j] = N~_j(x_r)`` at the composite Gauss points of ``gauss_quadrature``
    (Eq. CFEM-1D evaluated element by element), as a scipy CSR matrix of shape
    ``(q (n - 1), n)``.  A field with nodal coefficients ``c`` has values ``Phi c`` there."""
    xg, _ = gauss_legendre(q)
    rows, cols, vals = [], [], []
    for e in range(n - 1):
        support, N, _ = element_shape(e, n, s, p, a, xg)
        rr, cc = np.meshgrid(e * q + np.arange(q), support, indexing="ij")
        rows.append(rr.ravel())
        cols.append(cc.ravel())
        vals.append(N.ravel())
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(q * (n - 1), n)).tocsr()


def nodal_weights(n, length):
    """Trapezoid weights of the nodal rule: ``h`` inside, ``h/2`` at the two ends."""
    h = length / (n - 1)
    w = np.full(n, h)
    w[0] = w[-1] = h / 2.0
    return w


def nodes(n, length):
    """Uniform 1D mesh ``x_i = i h``, ``h = length / (n - 1)``."""
    return np.linspace(0.0, length, n)


def evaluate_field(coef, n, length, s, p, a, x):
    """Evaluate ``sum_k N~_k(x) coef_k`` at physical points ``x`` (for tests)."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    h = length / (n - 1)
    e = np.clip(np.floor(x / h).astype(int), 0, n - 2)
    out = np.zeros_like(x)
    for q in range(len(x)):
        xi = 2.0 * (x[q] - e[q] * h) / h - 1.0
        support, N, _ = element_shape(e[q], n, s, p, a, [xi])
        out[q] = N[0] @ coef[support]
    return out
