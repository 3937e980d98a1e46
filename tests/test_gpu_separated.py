"""Separated nonlinearity (Eq. MxySep) on the GPU against the oracle with the same form: the
nonlinear term from the exact decomposition of w(u^k) into C(M_k + 2, 3) + M_k separated
terms, integrated as 1D sums (M_max <= 16).  Same tolerances as the grid form: FP64 path
1e-12, split-BF16 path 1e-5 (u and energy)."""
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


def run_pair(lib, w, nsteps, prec, **over):
    cfg = lib.config_from_workload(w, precision=prec, nonlinear_form=lib.NONLINEAR_SEPARATED, **over)
    s = lib.Solver(cfg)
    A = workloads.initial_modes(w)
    s.set_initial_modes(A)
    prob = octd.Problem(dim=w.dim, n=w.n, length=w.length, s=w.s, p=w.p, a=w.a, L=w.L, kappa=w.kappa,
                        a0=w.a0, alpha=w.alpha, dt=w.dt, M_max=w.M_max, I_max=w.I_max, tol_als=w.tol_als,
                        tol_enrich=w.tol_enrich, seed=w.seed, nonlinear_form="separated",
                        fixed_als_iters=over.get("fixed_als_iters", 0), fixed_modes=over.get("fixed_modes", 0))
    ops = octd.build_operators(prob)
    out = []
    for k in range(nsteps):
        mk = A[0].shape[1]
        A, so = octd.step(prob, ops, A, k)
        sg = s.step(1)[0]
        G = s.get_modes()
        eo = octd.energy(prob, ops, A)
        out.append(dict(k=k, mk=mk, modes=(sg["modes"], so["modes"]), its=(sg["als_sweeps"], sum(so["als_iters"])),
                        err_u=octd.rel_l2_between(G, A), err_E=abs(s.energy() - eo) / abs(eo)))
    s.close()
    return out


def test_separated_fp64_matches_oracle(lib):
    w = workloads.preset("c0", M_max=16)
    for r in run_pair(lib, w, 10, lib.PREC_FP64):
        assert r["modes"][0] == r["modes"][1] and r["its"][0] == r["its"][1], r
        assert r["err_u"] < 1e-12 and r["err_E"] < 1e-12, r


def test_separated_ragged_3d_fp64_matches_oracle(lib):
    w = workloads.preset("c0", dim=3, n=(14, 11, 17), length=(1.0, 1.0, 1.0), eps=0.1, M_max=8, ic_rank=2,
                         tol_als=1e-6)
    for r in run_pair(lib, w, 3, lib.PREC_FP64):
        assert r["modes"][0] == r["modes"][1] and r["its"][0] == r["its"][1], r
        assert r["err_u"] < 1e-12 and r["err_E"] < 1e-12, r


def test_separated_mixed_within_1e5(lib):
    w = workloads.preset("c0", n=(200, 130), M_max=16)
    for r in run_pair(lib, w, 5, lib.PREC_SPLIT_BF16):
        assert r["modes"][0] == r["modes"][1], r
        assert r["err_u"] < 1e-5 and r["err_E"] < 1e-5, r


def test_separated_fixed_schedule_at_16_modes(lib):
    # the largest multiset table: 16 modes from the second step on (816 cubic terms)
    w = workloads.preset("c0", n=(40, 52), M_max=16)
    res = run_pair(lib, w, 3, lib.PREC_FP64, fixed_als_iters=3, fixed_modes=16)
    assert res[1]["mk"] == 16 and res[2]["mk"] == 16
    for r in res:
        assert r["err_u"] < 1e-12, r


def test_separated_refusals(lib):
    w = workloads.preset("c0", M_max=16)
    for over in (dict(reduced_tol=1e-4), dict(M_max=17)):
        with pytest.raises(lib.CTDError) as ei:
            lib.Solver(lib.config_from_workload(w, nonlinear_form=lib.NONLINEAR_SEPARATED, **over))
        assert ei.value.status == -1, over
    # batched steps integrate over the grid only
    s = lib.Solver(lib.config_from_workload(w, nonlinear_form=lib.NONLINEAR_SEPARATED))
    s.set_initial_modes(workloads.initial_modes(w))
    with pytest.raises(lib.CTDError) as ei:
        lib.step_batch([s], 1)
    assert ei.value.status == -7
    s.close()
