"""GPU parity at the full workload sizes, in the launch configuration the benchmark times (one
CTA per SM): a whole 2D 4096 x 4096 step against the oracle's step, and the 3D tensor-core
contraction at 512^3 and 1024^3 nodes on sampled rows that the oracle computes one at a time
(the full 3D grids do not fit the oracle)."""
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


def oracle_problem(w):
    return octd.Problem(dim=w.dim, n=w.n, length=w.length, s=w.s, p=w.p, a=w.a, L=w.L, kappa=w.kappa,
                        a0=w.a0, alpha=w.alpha, dt=w.dt, M_max=w.M_max, I_max=w.I_max, tol_als=w.tol_als,
                        tol_enrich=w.tol_enrich, seed=w.seed)


@pytest.fixture(scope="module")
def c1_oracle():
    w = workloads.preset("c1")
    prob = oracle_problem(w)
    ops = octd.build_operators(prob)
    A0 = workloads.initial_modes(w)
    A, st = octd.step(prob, ops, A0, 0)
    return w, A0, A, st, octd.energy(prob, ops, A)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_c1_first_step_matches_oracle(lib, c1_oracle, prec, tol):
    w, A0, A, st_o, E_o = c1_oracle
    p = lib.PREC_FP64 if prec == "fp64" else lib.PREC_SPLIT_BF16
    s = lib.Solver(lib.config_from_workload(w, precision=p))
    s.set_initial_modes(A0)
    st_g = s.step(1)[0]
    G = s.get_modes()
    E_g = s.energy()
    s.close()
    assert octd.rel_l2_between(G, A) < tol
    assert abs(E_g - E_o) / abs(E_o) < tol
    if prec == "fp64":
        # Same modes.  The sweep total may differ by one: at this size a mode's stop test
        # (relative change <= 1e-8) is met by the oracle at 0.83-0.93 of the tolerance, and
        # the discarded trailing mode (amplitude 2.4e-8 of u) is solved from a right-hand
        # side that has cancelled to that level, which magnifies the last-bit difference of
        # FP64 and the 48-bit double-float solves.  The field above is unaffected (1e-12).
        assert st_g["modes"] == st_o["modes"]
        assert st_g["als_sweeps_committed"] == sum(st_o["als_iters"][:st_o["modes"]])
        assert abs(st_g["als_sweeps"] - sum(st_o["als_iters"])) <= 1


def row_integral(prob, ops, A, v, x, i):
    """Row i along x of the contraction divided by L omega_x[i] (the sum over the other two
    axes of w(u^k) omega v omega v), and its error bound for the split-BF16 path: each
    reconstructed value is within 5e-5 of sum_m |a b c| (the tensor-core tests' model), which
    moves w by |w'(u)| times that, and the FP32 sums within a tile add 2^-20 of sum |w| omega v
    omega v."""
    p, q = [d for d in range(3) if d != x]
    U = octd.reconstruct([A[x][[i]], A[p], A[q]])[0]
    S = octd.reconstruct([np.abs(A[x][[i]]), np.abs(A[p]), np.abs(A[q])])[0]
    W = octd.w_of_u(U, prob.a0)
    a, b = ops.omega[p] * v[p], ops.omega[q] * v[q]
    dw = 4.0 * prob.a0 * np.abs(3.0 * U ** 2 - 1.0) * S
    return float(a @ W @ b), 5e-5 * float(a @ dw @ b) + 2.0 ** -20 * float(a @ np.abs(W) @ b)


@pytest.mark.parametrize("name", ["c2", "c3"])
def test_3d_tensor_core_contraction_sampled_rows(lib, name):
    # Bound per sampled row from the arithmetic (row_integral).  A relative bound on the result
    # does not fit: in c2 most of the domain sits at u = +-1 (the tanh mode), where w(u)
    # cancels to near zero while the reconstruction error still moves it by |w'(u)| = 8 a0.
    w = workloads.preset(name)
    s = lib.Solver(lib.config_from_workload(w, precision=lib.PREC_SPLIT_BF16))
    A = workloads.initial_modes(w)
    s.set_initial_modes(A)
    prob = oracle_problem(w)
    ops = octd.build_operators(prob)
    rng = np.random.default_rng(2)
    v = [rng.uniform(0.5, 1.5, size=w.n[d]) for d in range(3)]
    for x in range(3):
        got = s.probe_contract(x, v)
        n = w.n[x]
        rows = sorted(set([0, 1, 127, 128, n // 2, n - 1] + [int(r) for r in rng.choice(n, 10, replace=False)]))
        rb = np.array([row_integral(prob, ops, A, v, x, i) for i in rows])
        err = np.abs(got[rows] - rb[:, 0])
        assert np.all(err <= rb[:, 1]), (x, np.max(err / rb[:, 1]))
        assert np.linalg.norm(got[rows] - rb[:, 0]) <= 2e-4 * np.linalg.norm(rb[:, 0]), x
        assert np.all(np.isfinite(got))
    s.close()


def field_rel_l2(A, B):
    """||u_A - u_B|| / ||u_B|| on the nodes of two separated fields, rebuilt in FP64 on the GPU
    slab by slab (a Gram-matrix form would cancel at the differences measured here)."""
    import torch
    ta = [torch.as_tensor(a, dtype=torch.float64, device="cuda") for a in A]
    tb = [torch.as_tensor(b, dtype=torch.float64, device="cuda") for b in B]
    n0 = ta[0].shape[0]
    num = den = 0.0
    step = 64 if len(ta) == 3 else n0
    for i0 in range(0, n0, step):
        i1 = min(n0, i0 + step)
        if len(ta) == 2:
            ua, ub = ta[0][i0:i1] @ ta[1].T, tb[0][i0:i1] @ tb[1].T
        else:
            ua = torch.einsum("im,jm,km->ijk", ta[0][i0:i1], ta[1], ta[2])
            ub = torch.einsum("im,jm,km->ijk", tb[0][i0:i1], tb[1], tb[2])
        num += float(torch.sum((ua - ub) ** 2))
        den += float(torch.sum(ub ** 2))
    return (num / den) ** 0.5


@pytest.mark.parametrize("name", ["c2", "c3"])
def test_3d_whole_steps_mixed_vs_fp64(lib, name):
    # The full 3D configurations: the split-BF16 tensor-core form against the plain FP64 form
    # on the GPU (the oracle cannot hold these grids).
    # (1) The same mode count (fixed_modes = 6), every mode swept to its stop rules: the fields
    #     differ by the arithmetic alone, within the mixed-precision bar 1e-5, for the hi + lo
    #     and the hi + mid + lo splits.  (A fixed, unconverged sweep count is no measure of the
    #     arithmetic: with 6 sweeps per mode the oracle's own c2 step moves by 1e-4 under a 1e-7
    #     perturbation of its nonlinear term, tests/test_oracle_step.py.)
    # (2) Free running under the same stop rules: the greedy decisions may differ where a mode's
    #     amplitude sits at the enrichment threshold tol_enrich = 1e-4 (the oracle's own c2 step
    #     changes its mode count under a 1e-7 perturbation), so the fields agree to that
    #     truncation level; the energy decreases in both.
    w = workloads.preset(name)
    A0 = workloads.initial_modes(w)

    def run(prec, nsteps, **over):
        p = {"fp64": lib.PREC_FP64, "mixed": lib.PREC_SPLIT_BF16, "split3": lib.PREC_SPLIT3_BF16}[prec]
        s = lib.Solver(lib.config_from_workload(w, precision=p, **over))
        s.set_initial_modes(A0)
        E = [s.energy()]
        st = []
        for _ in range(nsteps):
            st.append(s.step(1)[0])
            E.append(s.energy())
        G = s.get_modes()
        s.close()
        return G, E, st

    # Six modes: forcing more than the workload's leading modes commits trailing modes of
    # amplitude ~1e-5 whose direction is ill-determined (on c2 a twelfth mode moves the field by
    # 5e-5 between arithmetics whatever the contraction's precision).
    fixed = dict(fixed_modes=6, als_stall_tol=1e-6)
    G64, E64, _ = run("fp64", 1, **fixed)
    for prec in ("mixed", "split3"):
        Gmx, Emx, _ = run(prec, 1, **fixed)
        assert G64[0].shape[1] == Gmx[0].shape[1] == 6
        assert field_rel_l2(Gmx, G64) < 1e-5, prec
        assert abs(Emx[-1] - E64[-1]) < 1e-5 * abs(E64[-1]), prec
    G64, E64, s64 = run("fp64", 2, als_stall_tol=1e-6)
    Gmx, Emx, smx = run("mixed", 2, als_stall_tol=1e-6)
    assert all(r["status"] >= 0 for r in s64 + smx)
    assert field_rel_l2(Gmx, G64) < w.tol_enrich
    assert abs(Emx[-1] - E64[-1]) < 1e-5 * abs(E64[-1])
    for E in (E64, Emx):
        assert E[-1] < E[0], E


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-7), ("mixed", 1e-6), ("split3", 1e-6)])
def test_interface_workload_steps_match_oracle(lib, prec, tol):
    # The tanh interface workload's parameters (eps = 0.02, s = p = 2, rank 6 + tanh mode) on a
    # 128^3 grid, where the oracle holds the grid: one step with 6 modes, each swept to the same
    # stop rules, against the oracle's step.  The stall rule makes the mode stops, hence the
    # field, depend on the arithmetic's rounding floor (the bars sit above it); the mixed forms
    # stay an order under the mixed-precision bar 1e-5.
    w = workloads.preset("c2", n=(128, 128, 128))
    A0 = workloads.initial_modes(w)
    prob = oracle_problem(w)
    prob.fixed_modes, prob.als_stall_tol = 6, 1e-6
    ops = octd.build_operators(prob)
    A, _ = octd.step(prob, ops, A0, 0)
    p = {"fp64": lib.PREC_FP64, "mixed": lib.PREC_SPLIT_BF16, "split3": lib.PREC_SPLIT3_BF16}[prec]
    s = lib.Solver(lib.config_from_workload(w, precision=p, fixed_modes=6, als_stall_tol=1e-6))
    s.set_initial_modes(A0)
    s.step(1)
    G = s.get_modes()
    E = s.energy()
    s.close()
    assert octd.rel_l2_between(G, A) < tol
    Eo = octd.energy(prob, ops, A)
    assert abs(E - Eo) < tol * abs(Eo)
