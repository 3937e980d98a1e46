"""Pins for the oracle's 1D C-FEM (App. B, App. C, Eq. KxxMxx) against closed forms,
library routines and values the paper prints."""
import json
import os

import numpy as np
import pytest
from scipy.interpolate import BarycentricInterpolator, BSpline

from oracle import cfem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def test_psi_is_the_cubic_b_spline():
    # Psi(z) of App. B equals the textbook uniform cubic B-spline B3(t), t = 2z, on knots
    # -2..2; scipy's BSpline.basis_element is an independent evaluation.
    b3 = BSpline.basis_element([-2, -1, 0, 1, 2], extrapolate=False)
    z = np.linspace(0.0, 1.3, 2601)
    ref = np.nan_to_num(b3(2 * z), nan=0.0)
    assert np.max(np.abs(cfem.psi(z) - ref)) < 1e-14
    # printed break-point values
    assert cfem.psi(0.0) == pytest.approx(2 / 3, abs=1e-15)
    assert cfem.psi(0.5) == pytest.approx(1 / 6, abs=1e-15)
    assert cfem.psi(1.0) == pytest.approx(0.0, abs=1e-15)


def test_psi_derivative_matches_finite_differences_and_is_continuous():
    z = np.linspace(0.01, 1.2, 500)
    h = 1e-6
    fd = (cfem.psi(z + h) - cfem.psi(z - h)) / (2 * h)
    assert np.max(np.abs(fd - cfem.dpsi_dz(z))) < 1e-8
    for zb in (0.5, 1.0):
        assert cfem.dpsi_dz(zb - 1e-12) == pytest.approx(cfem.dpsi_dz(zb + 1e-12), abs=1e-9)


@pytest.mark.parametrize("nodes,p", [([-3.0, -1.0, 1.0], 1), ([-5.0, -3.0, -1.0, 1.0, 3.0], 2),
                                      ([-7, -5, -3, -1, 1, 3, 5], 3), ([-1.0, 1.0, 3.0], 1)])
def test_rbf_interpolates_and_reproduces_polynomials(nodes, p):
    nodes = np.asarray(nodes, float)
    K, L = cfem.rbf_coefficients(nodes, 12.0, p)
    W, _ = cfem.rbf_eval(nodes, nodes, K, L, 12.0, p)
    assert np.max(np.abs(W - np.eye(len(nodes)))) < 1e-10      # Kronecker delta, Eq. reproducecondition
    P = cfem.monomials(nodes, p)
    assert np.max(np.abs(P.T @ K)) < 1e-10                      # moment conditions on k
    xi = np.linspace(-1, 1, 41)
    Wx, dWx = cfem.rbf_eval(xi, nodes, K, L, 12.0, p)
    for q in range(p + 1):
        assert np.max(np.abs(Wx @ nodes ** q - xi ** q)) < 1e-9
        dref = q * xi ** (q - 1) if q > 0 else 0 * xi
        assert np.max(np.abs(dWx @ nodes ** q - dref)) < 1e-8


def test_p2_s1_patch_is_quadratic_lagrange():
    # App. B example: patch {-3, -1, 1} with a second-order basis -> P is square, K = 0,
    # W is the quadratic Lagrange basis (scipy.interpolate.lagrange, independent).
    nodes = np.array([-3.0, -1.0, 1.0])
    K, L = cfem.rbf_coefficients(nodes, 12.0, 2)
    assert np.max(np.abs(K)) < 1e-9
    xi = np.linspace(-1, 1, 9)
    W, _ = cfem.rbf_eval(xi, nodes, K, L, 12.0, 2)
    for j in range(3):
        e = np.zeros(3)
        e[j] = 1.0
        assert np.max(np.abs(W[:, j] - BarycentricInterpolator(nodes, e)(xi))) < 1e-10


def test_paper_patch_coordinates_and_shape_function_count():
    g = json.load(open(GOLDEN))
    pc = g["app_b_patch_coordinates"]
    patch = cfem.nodal_patch(pc["node"], 20, pc["s"])
    xi = -1.0 + 2.0 * (patch - pc["element_left_node"])
    assert list(xi) == pc["xi"]
    sf = g["cfe_shape_functions_per_element"]
    for s, count in zip(sf["s"], sf["count"]):
        support, N, _ = cfem.element_shape(10, 30, s, 1, 12.0, np.array([0.0]))
        assert len(support) == count
        assert np.count_nonzero(np.abs(N[0]) > 1e-14) == count


@pytest.mark.parametrize("s,p", [(1, 1), (2, 2), (3, 3), (2, 1)])
def test_shape_functions_kronecker_partition_reproduction(s, p):
    n, length = 13, 1.0
    x = cfem.nodes(n, length)
    pts = np.linspace(0, length, 97)
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        assert np.max(np.abs(cfem.evaluate_field(e, n, length, s, p, 12.0, x) - e)) < 1e-10
    assert np.max(np.abs(cfem.evaluate_field(np.ones(n), n, length, s, p, 12.0, pts) - 1)) < 1e-10
    assert np.max(np.abs(cfem.evaluate_field(x, n, length, s, p, 12.0, pts) - pts)) < 1e-10
    if p >= 2:
        assert np.max(np.abs(cfem.evaluate_field(x ** 2, n, length, s, p, 12.0, pts) - pts ** 2)) < 1e-10


@pytest.mark.parametrize("s,p", [(1, 1), (2, 2), (3, 3)])
def test_stiffness_closed_forms(s, p):
    n, length = 17, 1.3
    K = cfem.stiffness_matrix(n, length, s, p, 12.0).toarray()
    x = cfem.nodes(n, length)
    assert np.max(np.abs(K - K.T)) < 1e-12
    assert np.max(np.abs(K @ np.ones(n))) < 1e-10                 # Neumann null space
    assert x @ K @ x == pytest.approx(length, rel=1e-12)          # int (d x/dx)^2 = length
    if p >= 2:
        assert (x ** 2) @ K @ (x ** 2) == pytest.approx(4 * length ** 3 / 3, rel=1e-11)
    ev = np.linalg.eigvalsh(K)
    assert ev[0] > -1e-10 and ev[1] > 1e-6                        # PSD, one-dimensional kernel
    r, c = np.nonzero(np.abs(K) > 1e-14)
    assert np.max(np.abs(r - c)) == 2 * s + 1                     # half-bandwidth 2s+1
    K8 = cfem.stiffness_matrix(n, length, s, p, 12.0, gauss_points=8).toarray()
    assert np.max(np.abs(K8 - K)) < 1e-12 * np.max(np.abs(K))     # 5-point Gauss is exact


def test_nodal_weights_and_consistent_mass():
    n, length = 11, 2.0
    w = cfem.nodal_weights(n, length)
    assert w.sum() == pytest.approx(length)
    Mc = cfem.consistent_mass_matrix(n, length, 2, 2, 12.0)
    assert np.ones(n) @ Mc @ np.ones(n) == pytest.approx(length, rel=1e-12)
    x = cfem.nodes(n, length)
    assert x @ Mc @ x == pytest.approx(length ** 3 / 3, rel=1e-12)  # int x^2


def test_paper_mesh_dof_counts():
    g = json.load(open(GOLDEN))
    for ne, elems, dofs in g["mesh_dofs_2d"]["rows"]:
        assert ne * ne == elems and (ne + 1) ** 2 == dofs
    for ne, dofs in zip(g["mesh_dofs_3d"]["elements_per_side"], g["mesh_dofs_3d"]["dofs"]):
        assert (ne + 1) ** 3 == dofs
