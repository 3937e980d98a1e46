"""GPU parity of the two forms of the tensor-core contraction epilogue against the oracle.

The direct form sums c_j u (u^2 - 1) from the reconstructed u; the cube form scales the column
operand's rows by cbrt(c_j), sums v^3 = c_j u^3 and adds the linear part -sum_j c_j u_ij =
-sum_m a_m,i H_m exactly from the Gram products.  Both are exact algebra for the same integral
(Eq. KxxMxx), so both meet the contraction bounds of the split (1e-4 relative), the whole-step
bar (1e-5) and, with a0 != 1/4 and L != 1, place the factor 4 a0 of w once.  Where |u| is
small the cube form's error is far below the direct form's: the split's rounding of u enters
through 3 u^2 instead of |3 u^2 - 1|, and the dominant linear part carries none of it.
"""
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


def problem(w, **over):
    kw = dict(dim=w.dim, n=w.n, length=w.length, s=w.s, p=w.p, a=w.a, L=w.L, kappa=w.kappa, a0=w.a0,
              alpha=w.alpha, dt=w.dt, M_max=w.M_max, I_max=w.I_max, tol_als=w.tol_als, tol_enrich=w.tol_enrich,
              seed=w.seed)
    kw.update(over)
    return octd.Problem(**kw)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


FORMS = ("direct", "cube")


def form_of(lib, name):
    return {"direct": lib.CONTRACT_DIRECT, "cube": lib.CONTRACT_CUBE, "auto": lib.CONTRACT_AUTO}[name]


def grid_of(A):
    """Full-grid values of a separated field (factors n_d x M)."""
    if len(A) == 2:
        return A[0] @ A[1].T
    return np.einsum("im,jm,km->ijk", A[0], A[1], A[2])


def model_bound(prob, ops, A, v, x, form):
    """Per-row bound on the probe's error from the split's error model: a reconstructed value
    is off by at most about 2^-15 S_ij (S = sum_m |prod_d a_m,d|; 5e-5 with margin), which moves
    the direct form's u (u^2 - 1) by |3u^2 - 1| times that and the cube form's u^3 (its linear
    part is exact) by 3u^2 times that; plus 1e-6 of |u^3| + |u| for the FP32 sums.  Scaled as
    the probe's output (4 a0 sum_j c_j ...)."""
    dim = len(A)
    U = np.moveaxis(grid_of(A), x, 0).reshape(A[x].shape[0], -1)
    S = np.moveaxis(grid_of([np.abs(a) for a in A]), x, 0).reshape(A[x].shape[0], -1)
    c = np.ones(1)
    for d in range(dim):
        if d != x:
            c = np.outer(c, ops.omega[d] * v[d]).reshape(-1)
    g = 3 * U * U if form == "cube" else np.abs(3 * U * U - 1)
    return 4 * prob.a0 * ((5e-5 * g * S + 1e-6 * (np.abs(U) ** 3 + np.abs(U))) @ np.abs(c))


def contraction_errors(lib, w, rank, amp, form, quad=None, a0=None, L=None, model=False, prec=None):
    """Relative error of the probe contraction against the oracle for every direction (with
    model, the largest ratio of a row's error to its model_bound instead)."""
    over = {}
    if a0 is not None:
        over["a0"] = a0
    if L is not None:
        over["L"] = L
    cfg_over = dict(over)
    if quad:
        cfg_over.update(quad_rule=lib.QUAD_GAUSS, quad_q=quad)
    s = lib.Solver(lib.config_from_workload(w, precision=lib.PREC_SPLIT_BF16 if prec is None else prec,
                                            contraction_form=form_of(lib, form), **cfg_over))
    A = workloads.cosine_modes(w.n, w.length, rank, 4, 3, amp=amp)
    s.set_initial_modes(A)
    if quad:
        over.update(quad_rule="gauss", quad_q=quad)
    prob = problem(w, **over)
    ops = octd.build_operators(prob)
    rng = np.random.default_rng(1)
    v = [rng.uniform(0.5, 1.5, size=w.n[d]) for d in range(w.dim)]
    errs = []
    if quad:
        nl = octd.nonlinear_operator(prob, ops, A)
        for x in range(w.dim):
            errs.append(rel(s.probe_contract(x, v), octd.nonlinear_projection(prob, ops, nl, v, x) / prob.L))
    else:
        Mxy = octd.nonlinear_tensor(prob, ops, A)
        for x in range(w.dim):
            got = s.probe_contract(x, v)
            ref = octd.contract_except(Mxy, v, x) / (prob.L * ops.omega[x])
            if model:
                errs.append(float(np.max(np.abs(got - ref) / model_bound(prob, ops, A, v, x, form))))
            else:
                errs.append(rel(got, ref))
    s.close()
    return errs


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("dim,n,rank,amp", [(2, (300, 130), 5, 0.7), (2, (160, 140), 24, 0.2),
                                            (3, (20, 33, 17), 5, 0.7), (3, (40, 33, 130), 12, 0.2)])
def test_contraction_forms_match_oracle(lib, form, dim, n, rank, amp):
    # every row within the error model of its form (at amplitude 0.2 the weighted sums cancel:
    # the direct form is there at about 7e-4 of the result's norm, as a CPU emulation of the
    # split reproduces, the cube form at 1e-5)
    w = workloads.preset("c0", dim=dim, n=n, length=(1.0,) * dim, M_max=max(rank, 20))
    for x, e in enumerate(contraction_errors(lib, w, rank, amp, form, model=True)):
        assert e <= 1.0, (form, x, e)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("prec", ["split", "split3"])
def test_contraction_forms_full_k(lib, form, prec):
    # 128 modes fill the padded K range: the most K steps per tile and the fewest ring stages
    w = workloads.preset("c0", n=(160, 140), M_max=128)
    p = lib.PREC_SPLIT_BF16 if prec == "split" else lib.PREC_SPLIT3_BF16
    for x, e in enumerate(contraction_errors(lib, w, 128, 0.2, form, model=True, prec=p)):
        assert e <= 1.0, (form, prec, x, e)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("dim,n", [(2, (130, 77)), (3, (20, 17, 13))])
def test_contraction_forms_a0_and_L(lib, form, dim, n):
    # a0 != 1/4 and L != 1: the factor 4 a0 of w enters once, in both dimension counts
    w = workloads.preset("c0", dim=dim, n=n, length=(1.0,) * dim)
    for x, e in enumerate(contraction_errors(lib, w, 5, 0.5, form, a0=0.6, L=1.7, model=True)):
        assert e <= 1.0, (form, x, e)
    for x, e in enumerate(contraction_errors(lib, w, 5, 0.7, form, a0=0.6, L=1.7)):
        assert e < 1e-4, (form, x, e)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("dim,n,q", [(2, (64, 64), 5), (2, (130, 77), 2), (3, (20, 17, 13), 3)])
def test_gauss_contraction_forms(lib, form, dim, n, q):
    w = workloads.preset("c0", dim=dim, n=n, length=(1.0,) * dim)
    for x, e in enumerate(contraction_errors(lib, w, 5, 0.7, form, quad=q, a0=0.45)):
        assert e < 1e-4, (form, x, e)


@pytest.mark.parametrize("dim,n", [(2, (300, 130)), (3, (40, 33, 130))])
def test_cube_form_more_accurate_at_small_amplitude(lib, dim, n):
    # at |u| ~ 0.05 the linear part dominates w and is exact in the cube form
    w = workloads.preset("c0", dim=dim, n=n, length=(1.0,) * dim, M_max=20)
    ed = contraction_errors(lib, w, 4, 0.05, "direct")
    ec = contraction_errors(lib, w, 4, 0.05, "cube")
    for x in range(dim):
        assert ec[x] < 0.1 * ed[x], (x, ec[x], ed[x])


def test_automatic_choice(lib):
    # the bound sum_m prod_d max|a_m,d| <= 0.6 selects the cube form; forced forms, the reduced
    # domain and the FP64 path override it
    w = workloads.preset("c0", n=(130, 90), M_max=12)

    def used(amp, prec=None, **over):
        s = lib.Solver(lib.config_from_workload(w, precision=lib.PREC_SPLIT_BF16 if prec is None else prec, **over))
        s.set_initial_modes(workloads.cosine_modes(w.n, w.length, 2, 4, 3, amp=amp))
        st = s.step(1)[0]
        s.close()
        return st["cube_form"]

    A = workloads.cosine_modes(w.n, w.length, 2, 4, 3, amp=0.1)
    bound = sum(np.prod([np.max(np.abs(A[d][:, m])) for d in range(2)]) for m in range(2))
    assert bound <= 0.6
    assert used(0.1) is True
    A = workloads.cosine_modes(w.n, w.length, 2, 4, 3, amp=0.9)
    assert sum(np.prod([np.max(np.abs(A[d][:, m])) for d in range(2)]) for m in range(2)) > 0.6
    assert used(0.9) is False
    assert used(0.1, contraction_form=lib.CONTRACT_DIRECT) is False
    assert used(0.9, contraction_form=lib.CONTRACT_CUBE) is True
    assert used(0.1, reduced_tol=1e-3) is False
    assert used(0.1, prec=lib.PREC_FP64) is False


def run_steps(lib, w, nsteps, form, quad=None, **over):
    cfg_over = dict(over)
    p_over = dict(over)
    if quad:
        cfg_over.update(quad_rule=lib.QUAD_GAUSS, quad_q=quad)
        p_over.update(quad_rule="gauss", quad_q=quad)
    s = lib.Solver(lib.config_from_workload(w, precision=lib.PREC_SPLIT_BF16, contraction_form=form_of(lib, form),
                                            **cfg_over))
    A0 = workloads.initial_modes(w)
    s.set_initial_modes(A0)
    prob = problem(w, **p_over)
    ops = octd.build_operators(prob)
    A = A0
    out = []
    for k in range(nsteps):
        A, st = octd.step(prob, ops, A, k)
        sg = s.step(1)[0]
        eo = octd.energy(prob, ops, A)
        out.append(dict(k=k, cube=sg["cube_form"], modes=(sg["modes"], st["modes"]),
                        err_u=octd.rel_l2_between(s.get_modes(), A), err_E=abs(s.energy() - eo) / abs(eo)))
    s.close()
    return out


@pytest.mark.parametrize("form", FORMS + ("auto",))
def test_steps_c0_forms_within_1e5(lib, form):
    w = workloads.preset("c0")
    res = run_steps(lib, w, 6, form)
    for r in res:
        assert r["err_u"] < 1e-5 and r["err_E"] < 1e-5, r
        if form != "auto":
            assert r["cube"] == (form == "cube"), r


@pytest.mark.parametrize("form", FORMS)
def test_steps_3d_forms_a0_within_1e5(lib, form):
    w = workloads.preset("c0", dim=3, n=(14, 11, 17), length=(1.0, 1.0, 1.0), eps=0.1, M_max=8, ic_rank=2,
                         tol_als=1e-6)
    for r in run_steps(lib, w, 3, form, a0=0.6, L=1.3):
        assert r["err_u"] < 1e-5 and r["err_E"] < 1e-5, r


@pytest.mark.parametrize("form", FORMS)
def test_steps_gauss_forms_within_1e5(lib, form):
    w = workloads.preset("c0", n=(48, 40))
    for r in run_steps(lib, w, 3, form, quad=3, a0=0.4):
        assert r["err_u"] < 1e-5 and r["err_E"] < 1e-5, r
