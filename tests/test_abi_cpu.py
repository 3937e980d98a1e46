"""CPU checks of the C ABI: the library loads without a GPU, exports every entry point the
public header declares, validates configurations, and its host-side C-FEM builder agrees
with the oracle (App. B / App. C shape functions, Eq. KxxMxx stiffness)."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads
from oracle import cfem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ctd.h")


@pytest.fixture(scope="module")
def ctd():
    from paper_2410_15519_gb300 import build, ctd as mod
    build.build()
    return mod


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ctd_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(ctd):
    lib = ctd.load()
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings(ctd):
    lib = ctd.load()
    for code in (0, 1, 2, -1, -2, -3, -4, -5, -6, -7):
        assert len(lib.ctd_status_string(code)) >= 2


@pytest.mark.parametrize("field,value", [("dim", 4), ("s", 0), ("p", 3), ("M_max", 0), ("M_max", 129),
                                          ("dt", -1.0), ("precision", 7), ("I_max", 0)])
def test_invalid_configurations_are_rejected(ctd, field, value):
    w = workloads.preset("c0")
    cfg = ctd.config_from_workload(w)
    if field == "p":
        cfg.s = 2
    setattr(cfg, field, value)
    lib = ctd.load()
    n = ctypes.c_size_t(0)
    assert lib.ctd_workspace_size(ctypes.byref(cfg), ctypes.byref(n)) == -1


def test_node_count_limits(ctd):
    lib = ctd.load()
    for nn in (3, 4097):
        cfg = ctd.config_from_workload(workloads.preset("c0", n=(nn, 64)))
        n = ctypes.c_size_t(0)
        assert lib.ctd_workspace_size(ctypes.byref(cfg), ctypes.byref(n)) == -1


def test_workspace_size_grows_with_the_problem(ctd):
    small = ctd.workspace_size(ctd.config_from_workload(workloads.preset("c0")))
    big = ctd.workspace_size(ctd.config_from_workload(workloads.preset("c0", n=(1024, 1024))))
    mixed = ctd.workspace_size(ctd.config_from_workload(workloads.preset("c0"), precision=ctd.PREC_SPLIT_BF16))
    assert 0 < small < big and mixed > 0


@pytest.mark.parametrize("n,s,p", [(64, 1, 1), (101, 2, 2), (57, 3, 3), (33, 2, 1)])
def test_host_cfem_matches_oracle(ctd, n, s, p):
    cfg = ctd.config_from_workload(workloads.preset("c0", n=(n, n), s=s, p=p))
    om, kb, b = ctd.probe_cfem(cfg, 0)
    assert b == 2 * s + 1
    K = cfem.stiffness_matrix(n, 1.0, s, p, 12.0).toarray()
    Kd = np.zeros((n, n))
    for i in range(n):
        for k in range(-b, b + 1):
            if 0 <= i + k < n:
                Kd[i, i + k] = kb[i, k + b]
            else:
                assert kb[i, k + b] == 0.0
    assert np.max(np.abs(Kd - K)) <= 1e-12 * np.max(np.abs(K))
    assert np.array_equal(om, cfem.nodal_weights(n, 1.0))


@pytest.mark.parametrize("n,s,p,q", [(33, 1, 1, 2), (40, 2, 2, 5), (29, 3, 3, 3), (17, 2, 1, 7), (12, 2, 2, 16)])
def test_host_gauss_rule_matches_oracle(ctd, n, s, p, q):
    # the Gauss-point operators of the consistent-mass variant against the oracle's own
    # (numpy's Gauss-Legendre rule, the App. B / App. C shape functions, Phi^T diag(omega) Phi)
    from scipy import sparse
    cfg = ctd.config_from_workload(workloads.preset("c0", n=(n, n), s=s, p=p))
    xq, om, Phi, mb, bounds = ctd.probe_cfem_gauss(cfg, 0, q)
    x_ref, om_ref = cfem.gauss_quadrature(n, 1.0, q)
    # points to 1e-15; weights to 2e-14 (the three-term recurrence rounds a few ulps at q = 16)
    assert np.max(np.abs(xq - x_ref)) <= 1e-15 and np.max(np.abs(om - om_ref)) <= 2e-14 * np.max(om_ref)
    Phi_ref = cfem.quadrature_basis(n, 1.0, s, p, 12.0, q).toarray()
    assert np.max(np.abs(Phi - Phi_ref)) <= 1e-12
    M_ref = (sparse.csr_matrix(Phi_ref).T @ sparse.diags(om_ref) @ sparse.csr_matrix(Phi_ref)).toarray()
    b = 2 * s + 1
    M = np.zeros((n, n))
    for i in range(n):
        for k in range(-b, b + 1):
            if 0 <= i + k < n:
                M[i, i + k] = mb[i, k + b]
            else:
                assert mb[i, k + b] == 0.0
    assert np.max(np.abs(M - M_ref)) <= 1e-13 * np.max(np.abs(M_ref))
    # spectrum bounds of diag(M)^-1 M: enclose the exact extreme eigenvalues, tightly
    from scipy import linalg
    lam = linalg.eigh(M_ref, np.diag(np.diag(M_ref)), eigvals_only=True)
    lo, hi = bounds
    assert lo <= lam[0] <= lo * (1 + 1e-4) and hi * (1 - 1e-4) <= lam[-1] <= hi, (bounds, lam[0], lam[-1])


def test_host_gauss_legendre_rule_for_every_point_count(ctd):
    # 8 nodes on [0, 7] (h = 1): element e holds the points e + (1 + xi_g) / 2 with weights w_g / 2
    cfg = ctd.config_from_workload(workloads.preset("c0", n=(8, 8), length=(7.0, 7.0), s=1, p=1))
    for q in range(1, 17):
        xq, om, Phi, mb, _ = ctd.probe_cfem_gauss(cfg, 0, q, bounds=False)
        xg, wg = np.polynomial.legendre.leggauss(q)
        for e in range(7):
            assert np.max(np.abs(xq[e * q:(e + 1) * q] - (e + 0.5 * (1.0 + xg)))) <= 1e-14, (q, e)
            assert np.max(np.abs(om[e * q:(e + 1) * q] - 0.5 * wg)) <= 2e-14 * np.max(wg), (q, e)
        assert np.max(np.abs(Phi.sum(axis=1) - 1.0)) <= 1e-13, q      # partition of unity


def test_host_gauss_rule_refuses_bad_point_counts(ctd):
    cfg = ctd.config_from_workload(workloads.preset("c0"))
    lib = ctd.load()
    err_arg = -1   # CTD_ERR_ARG
    # one point per element: 7 points for 8 nodes leave the mass singular, so no bounds
    c8 = ctd.config_from_workload(workloads.preset("c0", n=(8, 8), length=(7.0, 7.0), s=1, p=1))
    bd = np.zeros(2)
    assert lib.ctd_probe_cfem_gauss(ctypes.byref(c8), 0, 1, None, None, None, None, None, bd.ctypes.data) == err_arg
    assert lib.ctd_probe_cfem_gauss(ctypes.byref(c8), 0, 2, None, None, None, None, None, bd.ctypes.data) == 0
    for q in (0, 17):
        assert lib.ctd_probe_cfem_gauss(ctypes.byref(cfg), 0, q, None, None, None, None, None, None) == err_arg
    assert lib.ctd_probe_cfem_gauss(ctypes.byref(cfg), 2, 5, None, None, None, None, None, None) == err_arg


def test_calls_without_a_handle_fail_cleanly(ctd):
    lib = ctd.load()
    st = ctd.StepStats()
    assert lib.ctd_step(None, 1, ctypes.byref(st)) == -1
    e = ctypes.c_double()
    assert lib.ctd_energy(None, ctypes.byref(e)) == -1
    lib.ctd_destroy(None)


@pytest.mark.parametrize("over,status", [
    (dict(quad_rule=2, quad_q=5), -1),                                 # unknown rule: CTD_ERR_ARG
    (dict(quad_rule=1, quad_q=0), -1), (dict(quad_rule=1, quad_q=17), -1),
    (dict(quad_rule=1, quad_q=5, nonlinear_form=1, M_max=8), -7),      # separated form: CTD_ERR_UNSUPPORTED
    (dict(quad_rule=1, quad_q=5, reduced_tol=1e-3), -7),               # reduced domain (nodal rule only)
    (dict(quad_rule=1, quad_q=5, n=(4096, 64)), -7),                   # 20475 points beside direction 1
    (dict(quad_rule=1, quad_q=2, n=(4096, 4096)), 0), (dict(quad_rule=1, quad_q=5), 0),
    (dict(als_stall_tol=-1.0), -1), (dict(als_stall_tol=1e-6), 0),
    (dict(actd_Mc=-1), -1), (dict(actd_Mc=3), 0), (dict(actd_Mc=3, precision=1), -7),
    (dict(actd_Mc=3, quad_rule=1, quad_q=5), -7),
    (dict(contraction_form=-1), -1), (dict(contraction_form=3), -1),   # unknown form: CTD_ERR_ARG
    (dict(contraction_form=2, precision=1), 0), (dict(contraction_form=1, precision=3), 0),
    (dict(contraction_form=2), 0)])                                    # ignored by the FP64 path
def test_gauss_and_stall_configurations(ctd, over, status):
    w = workloads.preset("c0", **({"n": over.pop("n")} if "n" in over else {}))
    cfg = ctd.config_from_workload(w, **over)
    n = ctypes.c_size_t(0)
    assert ctd.load().ctd_workspace_size(ctypes.byref(cfg), ctypes.byref(n)) == status
    if status == 0:
        assert n.value > 0


def test_gauss_workspace_holds_the_point_grid(ctd):
    w = workloads.preset("c0", n=(200, 180))
    nodal = ctd.workspace_size(ctd.config_from_workload(w))
    gauss = ctd.workspace_size(ctd.config_from_workload(w, quad_rule=1, quad_q=5))
    # the FP64 grid of w(u^k) grows from 200 x 180 nodes to 995 x 895 Gauss points
    assert gauss - nodal >= 8 * (995 * 895 - 200 * 180)
