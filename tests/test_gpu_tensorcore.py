"""GPU parity of the tensor-core (split-BF16, tcgen05) path against the FP64 oracle.

Error model: each factor entry a is carried as hi + lo in BF16 with |a - hi - lo| <= 2^-17
|a| (two round-to-nearest 8-bit significands), and the dropped lo*lo product is below 2^-16
of |a b|; the FP32 accumulator adds about 2^-24 per term.  A reconstructed value therefore
differs from the FP64 one by at most about 2^-15 sum_m |a_m b_m| (3e-5 relative to that
sum); the tests use 5e-5 of max_ij sum_m |a_im b_jm|.
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


def pad128(n):
    return (n + 127) // 128 * 128


# ranks cover every K box width of the tiles: 16 (rank <= 16), 32 (17..32), 64 (33..64) and
# two 64-wide boxes per half (65..128)
@pytest.mark.parametrize("n,rank", [((128, 128), 4), ((200, 77), 5), ((256, 384), 20), ((130, 90), 33),
                                    ((64, 64), 50), ((200, 150), 70)])
def test_tensor_core_reconstruction_2d(lib, n, rank):
    w = workloads.preset("c0", n=n, M_max=max(rank, 8))
    cfg = lib.config_from_workload(w, precision=lib.PREC_SPLIT_BF16)
    s = lib.Solver(cfg)
    A = workloads.cosine_modes(n, (1.0, 1.0), rank, 4, 7, amp=0.9)
    s.set_initial_modes(A)
    U = A[0] @ A[1].T
    S = np.abs(A[0]) @ np.abs(A[1]).T
    for x in range(2):
        got = s.probe_reconstruct(x, pad128(n[x]), pad128(n[1 - x]))
        ref = U if x == 0 else U.T
        sc = S if x == 0 else S.T
        g = got[:n[x], :n[1 - x]].astype(np.float64)
        assert np.max(np.abs(g - ref)) <= 5e-5 * np.max(sc), (x, np.max(np.abs(g - ref)) / np.max(sc))
        assert np.all(got[n[x]:, :] == 0) and np.all(got[:, n[1 - x]:] == 0)   # padding stays zero
    s.close()


@pytest.mark.parametrize("dim,n,rank", [(2, (64, 64), 5), (2, (300, 130), 5), (2, (300, 130), 24),
                                        (2, (160, 140), 40), (3, (20, 33, 17), 5), (3, (20, 33, 17), 20)])
def test_tensor_core_contraction(lib, dim, n, rank):
    w = workloads.preset("c0", dim=dim, n=n, length=(1.0,) * dim, M_max=max(rank, 20))
    cfg = lib.config_from_workload(w, precision=lib.PREC_SPLIT_BF16)
    s = lib.Solver(cfg)
    A = workloads.cosine_modes(n, (1.0,) * dim, rank, 4, 3, amp=0.7)
    s.set_initial_modes(A)
    prob = octd.Problem(dim=dim, n=n, length=(1.0,) * dim, s=w.s, p=w.p, a=w.a, L=w.L, kappa=w.kappa, a0=w.a0,
                        alpha=w.alpha, dt=w.dt, M_max=w.M_max, I_max=w.I_max, tol_als=w.tol_als,
                        tol_enrich=w.tol_enrich)
    ops = octd.build_operators(prob)
    Mxy = octd.nonlinear_tensor(prob, ops, A)
    rng = np.random.default_rng(1)
    v = [rng.uniform(0.5, 1.5, size=n[d]) for d in range(dim)]
    for x in range(dim):
        ref = octd.contract_except(Mxy, v, x) / (prob.L * ops.omega[x])
        got = s.probe_contract(x, v)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < 1e-4, (x, err)
    s.close()


def run_mixed_vs_oracle(lib, w, nsteps):
    cfg = lib.config_from_workload(w, precision=lib.PREC_SPLIT_BF16)
    s = lib.Solver(cfg)
    A0 = workloads.initial_modes(w)
    s.set_initial_modes(A0)
    prob = octd.Problem(dim=w.dim, n=w.n, length=w.length, s=w.s, p=w.p, a=w.a, L=w.L, kappa=w.kappa, a0=w.a0,
                        alpha=w.alpha, dt=w.dt, M_max=w.M_max, I_max=w.I_max, tol_als=w.tol_als,
                        tol_enrich=w.tol_enrich, seed=w.seed)
    ops = octd.build_operators(prob)
    A = A0
    out = []
    for k in range(nsteps):
        A, st = octd.step(prob, ops, A, k)
        sg = s.step(1)[0]
        G = s.get_modes()
        out.append(dict(k=k, err_u=octd.rel_l2_between(G, A), modes=(sg["modes"], st["modes"]),
                        err_E=abs(s.energy() - octd.energy(prob, ops, A)) / abs(octd.energy(prob, ops, A))))
    s.close()
    return out


def test_mixed_step_c0_within_1e5(lib):
    # the mixed form's target: relative L2 of u and of the energy within 1e-5 of the FP64 oracle
    w = workloads.preset("c0")
    res = run_mixed_vs_oracle(lib, w, 10)
    for r in res:
        assert r["err_u"] < 1e-5 and r["err_E"] < 1e-5, r


def test_mixed_step_3d_within_1e5(lib):
    w = workloads.preset("c0", dim=3, n=(14, 11, 17), length=(1.0, 1.0, 1.0), eps=0.1, M_max=8, ic_rank=2,
                         tol_als=1e-6)
    for r in run_mixed_vs_oracle(lib, w, 3):
        assert r["err_u"] < 1e-5 and r["err_E"] < 1e-5, r


# The precision ladder of the tensor-core contraction: a factor value a carried as one BF16
# term (unit roundoff u = 2^-8: a product of two rounded terms is within 2u of |a b|), as
# hi + lo (3 products; about 2^-15) or as hi + mid + lo (6 products; the dropped products
# mid*lo, lo*mid, lo*lo and the representation error are below 3 u^3 of |a b|, the six FP32
# additions in TMEM add 6 * 2^-24): bounds on a reconstructed value against
# max_ij sum_m |a_im b_jm|, and on the contraction relative to its result (in 3D the
# Khatri-Rao operand b_j c_l is first rounded to FP32, 2^-24 more).
LADDER = [("bf16", 1e-2, 2e-2), ("split", 5e-5, 1e-4), ("split3", 1e-6, 5e-6)]


def prec_of(lib, name):
    return {"bf16": lib.PREC_BF16, "split": lib.PREC_SPLIT_BF16, "split3": lib.PREC_SPLIT3_BF16}[name]


@pytest.mark.parametrize("name,rbound,cbound", LADDER)
@pytest.mark.parametrize("n,rank", [((200, 77), 5), ((130, 90), 33), ((300, 140), 128)])
def test_precision_ladder_reconstruction(lib, name, rbound, cbound, n, rank):
    # rank 128 fills the padded K range (the smallest ring of column stages)
    w = workloads.preset("c0", n=n, M_max=max(rank, 8))
    s = lib.Solver(lib.config_from_workload(w, precision=prec_of(lib, name)))
    A = workloads.cosine_modes(n, (1.0, 1.0), rank, 4, 7, amp=0.9)
    s.set_initial_modes(A)
    U = A[0] @ A[1].T
    S = np.abs(A[0]) @ np.abs(A[1]).T
    for x in range(2):
        got = s.probe_reconstruct(x, pad128(n[x]), pad128(n[1 - x]))
        ref = U if x == 0 else U.T
        g = got[:n[x], :n[1 - x]].astype(np.float64)
        assert np.max(np.abs(g - ref)) <= rbound * np.max(S), (name, x, np.max(np.abs(g - ref)) / np.max(S))
        assert np.all(got[n[x]:, :] == 0) and np.all(got[:, n[1 - x]:] == 0)
    s.close()


@pytest.mark.parametrize("name,rbound,cbound", LADDER)
@pytest.mark.parametrize("dim,n,rank", [(2, (300, 130), 24), (3, (20, 33, 17), 20)])
def test_precision_ladder_contraction(lib, name, rbound, cbound, dim, n, rank):
    w = workloads.preset("c0", dim=dim, n=n, length=(1.0,) * dim, M_max=max(rank, 20))
    s = lib.Solver(lib.config_from_workload(w, precision=prec_of(lib, name)))
    A = workloads.cosine_modes(n, (1.0,) * dim, rank, 4, 3, amp=0.7)
    s.set_initial_modes(A)
    prob = octd.Problem(dim=dim, n=n, length=(1.0,) * dim, s=w.s, p=w.p, a=w.a, L=w.L, kappa=w.kappa, a0=w.a0,
                        alpha=w.alpha, dt=w.dt, M_max=w.M_max, I_max=w.I_max, tol_als=w.tol_als,
                        tol_enrich=w.tol_enrich)
    ops = octd.build_operators(prob)
    Mxy = octd.nonlinear_tensor(prob, ops, A)
    rng = np.random.default_rng(1)
    v = [rng.uniform(0.5, 1.5, size=n[d]) for d in range(dim)]
    for x in range(dim):
        ref = octd.contract_except(Mxy, v, x) / (prob.L * ops.omega[x])
        got = s.probe_contract(x, v)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < cbound, (name, x, err)
    s.close()


def test_split3_step_c0_within_1e7(lib):
    # the three-term split carries the factors to FP32 level: the whole step tracks the FP64
    # oracle two orders below the mixed-precision bar
    w = workloads.preset("c0")
    cfg = lib.config_from_workload(w, precision=lib.PREC_SPLIT3_BF16)
    s = lib.Solver(cfg)
    A0 = workloads.initial_modes(w)
    s.set_initial_modes(A0)
    prob = octd.Problem(dim=w.dim, n=w.n, length=w.length, s=w.s, p=w.p, a=w.a, L=w.L, kappa=w.kappa, a0=w.a0,
                        alpha=w.alpha, dt=w.dt, M_max=w.M_max, I_max=w.I_max, tol_als=w.tol_als,
                        tol_enrich=w.tol_enrich, seed=w.seed)
    ops = octd.build_operators(prob)
    A = A0
    for k in range(5):
        A, _ = octd.step(prob, ops, A, k)
        s.step(1)
        assert octd.rel_l2_between(s.get_modes(), A) < 1e-7, k
    s.close()
