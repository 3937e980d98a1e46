"""GPU parity of the Gauss-point rule (consistent mass; the quadrature of Eq. KxxMxx at Section
3.3's Gauss points of each element) against the oracle with ``quad_rule = "gauss"``: the
banded solve with the consistent mass, the nonlinear contraction at the Gauss points (FP64 and
tensor cores), whole steps at C0 size (FP64 1e-12, mixed 1e-5) and the first step at the
4096^2 size with two points per element."""
import numpy as np
import pytest

import workloads
from oracle import ctd as octd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_15519_gb300 import build, ctd
    build.build()
    return ctd


def oracle_problem(w, q, **over):
    p = octd.Problem(dim=w.dim, n=w.n, length=w.length, s=w.s, p=w.p, a=w.a, L=w.L, kappa=w.kappa,
                     a0=w.a0, alpha=w.alpha, dt=w.dt, M_max=w.M_max, I_max=w.I_max, tol_als=w.tol_als,
                     tol_enrich=w.tol_enrich, seed=w.seed, quad_rule="gauss", quad_q=q)
    for k, v in over.items():
        setattr(p, k, v)
    return p


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gauss_cfg(lib, w, q, prec="fp64", **over):
    p = lib.PREC_FP64 if prec == "fp64" else lib.PREC_SPLIT_BF16
    return lib.config_from_workload(w, precision=p, quad_rule=lib.QUAD_GAUSS, quad_q=q, **over)


@pytest.mark.parametrize("n,s,q", [(64, 1, 5), (333, 2, 5), (1000, 3, 2)])
def test_banded_solve_with_consistent_mass(lib, n, s, q):
    w = workloads.preset("c0", n=(n, 8), s=s, p=s)
    solver = lib.Solver(gauss_cfg(lib, w, q))
    prob = oracle_problem(w, q)
    ops = octd.build_operators(prob)
    rng = np.random.default_rng(n)
    rhs = rng.standard_normal(n)
    beta0 = prob.c_t / prob.c_k
    for a1, a2 in [(beta0 * 2.5e-3, 2.5e-3), (1.7 * beta0 * 0.3, 0.3)]:
        A = a1 * ops.M[0] + a2 * ops.K[0]
        ref = octd.banded_spd_solve(A, rhs)
        y = solver.probe_solve(0, a1, a2, rhs)
        ev = np.linalg.eigvalsh(A.toarray())
        tol = 1e-13 + 64 * 2.0 ** -48 * ev[-1] / ev[0]
        assert rel(y, ref) < tol, (a1, a2, rel(y, ref), tol)
    solver.close()


@pytest.mark.parametrize("dim,n,q,prec,tol", [(2, (64, 64), 5, "fp64", 1e-13), (2, (130, 77), 2, "fp64", 1e-13),
                                              (3, (20, 17, 13), 3, "fp64", 1e-13), (2, (64, 64), 5, "mixed", 1e-4),
                                              (2, (130, 77), 2, "mixed", 1e-4), (3, (20, 17, 13), 3, "mixed", 1e-4)])
def test_gauss_contraction_matches_oracle(lib, dim, n, q, prec, tol):
    w = workloads.preset("c0", dim=dim, n=n, length=(1.0,) * dim)
    solver = lib.Solver(gauss_cfg(lib, w, q, prec))
    A = workloads.cosine_modes(n, (1.0,) * dim, 5, 4, 3, amp=0.7)
    solver.set_initial_modes(A)
    prob = oracle_problem(w, q)
    ops = octd.build_operators(prob)
    nl = octd.nonlinear_operator(prob, ops, A)
    rng = np.random.default_rng(1)
    v = [rng.uniform(0.5, 1.5, size=n[d]) for d in range(dim)]
    for x in range(dim):
        ref = octd.nonlinear_projection(prob, ops, nl, v, x) / prob.L
        got = solver.probe_contract(x, v)
        assert rel(got, ref) < tol, (x, rel(got, ref))
    solver.close()


def run_pair(lib, w, q, nsteps, prec="fp64", **over):
    solver = lib.Solver(gauss_cfg(lib, w, q, prec, **over))
    A0 = workloads.initial_modes(w)
    solver.set_initial_modes(A0)
    prob = oracle_problem(w, q, **over)
    ops = octd.build_operators(prob)
    A = A0
    out = []
    for k in range(nsteps):
        A, st_o = octd.step(prob, ops, A, k)
        st_g = solver.step(1)[0]
        G = solver.get_modes()
        eo, eg = octd.energy(prob, ops, A), solver.energy()
        out.append(dict(k=k, modes=(st_g["modes"], st_o["modes"]), its=(st_g["als_sweeps"], sum(st_o["als_iters"])),
                        itc=(st_g["als_sweeps_committed"], sum(st_o["als_iters"][:st_o["modes"]])),
                        err_u=octd.rel_l2_between(G, A), err_E=abs(eg - eo) / abs(eo)))
    solver.close()
    return out


@pytest.mark.parametrize("q", [5, 2])
def test_c0_gauss_steps_match_oracle(lib, q):
    w = workloads.preset("c0")
    for r in run_pair(lib, w, q, 8):
        assert r["modes"][0] == r["modes"][1] and r["itc"][0] == r["itc"][1], r
        assert abs(r["its"][0] - r["its"][1]) <= 1, r
        assert r["err_u"] < 1e-12 and r["err_E"] < 1e-12, r


def test_ragged_3d_gauss_steps_match_oracle(lib):
    w = workloads.preset("c0", dim=3, n=(14, 11, 17), length=(1.0, 1.0, 1.0), eps=0.1, M_max=8, ic_rank=2,
                         tol_als=1e-6, s=2, p=2)
    for r in run_pair(lib, w, 3, 3):
        assert r["modes"][0] == r["modes"][1] and r["itc"][0] == r["itc"][1], r
        assert abs(r["its"][0] - r["its"][1]) <= 1, r
        assert r["err_u"] < 1e-12 and r["err_E"] < 1e-12, r


def test_c0_gauss_mixed_within_1e5(lib):
    w = workloads.preset("c0")
    for r in run_pair(lib, w, 5, 6, prec="mixed", als_stall_tol=1e-6):
        assert r["err_u"] < 1e-5 and r["err_E"] < 1e-5, r


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_c1_size_gauss_first_step(lib, prec, tol):
    # 4096^2 nodes, s = p = 2, two Gauss points per element (8190^2 points)
    w = workloads.preset("c1")
    r = run_pair(lib, w, 2, 1, prec=prec, als_stall_tol=1e-6)[0]
    assert r["err_u"] < tol and r["err_E"] < tol, r
    if prec == "fp64":
        assert r["modes"][0] == r["modes"][1], r
