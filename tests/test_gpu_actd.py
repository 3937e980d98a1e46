"""GPU parity of adaptive CTD (Section 3.3 "Adaptivity": a step that would need more than
M_c modes is solved on the full tensor-product C-FEM space, and the next step runs CTD from
the full-grid field) against the oracle's ``actd``: the switch decisions, the full-grid step
by fast diagonalisation (1e-12), the CTD step from a grid state and the energy law."""
import numpy as np
import pytest

import workloads
from oracle import actd, ctd as octd, fullgrid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_15519_gb300 import build, ctd
    build.build()
    return ctd


def problem(w):
    return octd.Problem(dim=w.dim, n=w.n, length=w.length, s=w.s, p=w.p, a=w.a, L=w.L, kappa=w.kappa,
                        a0=w.a0, alpha=w.alpha, dt=w.dt, M_max=w.M_max, I_max=w.I_max, tol_als=w.tol_als,
                        tol_enrich=w.tol_enrich, seed=w.seed)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_both(lib, w, A0, M_c, nsteps):
    prob = problem(w)
    ops = octd.build_operators(prob)
    s = lib.Solver(lib.config_from_workload(w, actd_Mc=M_c))
    s.set_initial_modes(A0)
    state = ("modes", [np.asarray(a, dtype=np.float64) for a in A0])
    out = []
    for k in range(nsteps):
        U_in = actd.field(state)
        state, st_o = actd.step(prob, ops, state, M_c, k)
        st_g = s.step(1)[0]
        out.append(dict(k=k, switched=(st_g["actd_switched"], st_o["switched"]),
                        modes=(st_g["modes"], st_o.get("modes", st_o.get("ctd_modes_tried"))),
                        err_u=rel(s.get_field(), actd.field(state)),
                        err_E=abs(s.energy() - actd.energy(prob, ops, state)) / abs(actd.energy(prob, ops, state)),
                        kind=state[0], U_in=U_in, U_out=actd.field(state), E=s.energy()))
    s.close()
    return prob, ops, out


@pytest.mark.parametrize("dim,n", [(2, (10, 10)), (2, (23, 17)), (3, (9, 7, 8))])
def test_switch_gives_the_full_grid_step(lib, dim, n):
    w = workloads.preset("c0", dim=dim, n=n, length=(1.0,) * dim, s=2, p=2, M_max=30, I_max=200, tol_als=1e-10,
                         tol_enrich=1e-8)
    A0 = workloads.cosine_modes(n, (1.0,) * dim, 4, 4, 3, amp=0.9)
    prob, ops, res = run_both(lib, w, A0, 2, 1)
    r = res[0]
    assert r["switched"] == (True, True) and r["modes"][0] == 3, r["modes"]
    assert r["err_u"] < 1e-12 and r["err_E"] < 1e-12, (r["err_u"], r["err_E"])
    # and the oracle's own dense full-grid solve
    ref = fullgrid.step(prob, ops, r["U_in"])
    assert rel(r["U_out"], ref) < 1e-12


def test_actd_run_alternates_like_the_oracle(lib):
    # a rich start switches on the first steps, then CTD takes over from the grid state
    w = workloads.preset("c0", n=(16, 16), s=1, p=1, eps=0.2, dt=1.0, M_max=30, I_max=200, tol_als=1e-10,
                         tol_enrich=1e-3)
    A0 = workloads.cosine_modes(w.n, w.length, 5, 5, 9, amp=0.9)
    A0[0] = A0[0] * (0.9 / np.max(np.abs(octd.reconstruct(A0))))
    _, _, res = run_both(lib, w, A0, 4, 5)
    assert [r["kind"] for r in res] == ["grid", "grid", "modes", "modes", "modes"]
    E = None
    for r in res:
        assert r["switched"][0] == r["switched"][1], r["k"]
        if not r["switched"][1]:
            assert r["modes"][0] == r["modes"][1], r["k"]
        assert r["err_u"] < 1e-12 and r["err_E"] < 1e-12, (r["k"], r["err_u"], r["err_E"])
        if E is not None:
            assert r["E"] <= E + 1e-10 * abs(E)
        E = r["E"]


def test_c0_size_actd_run(lib):
    # the 64^2 workload with a small critical mode count: switches and CTD steps from grid
    # states, every field within 1e-12 of the oracle's
    w = workloads.preset("c0")
    _, _, res = run_both(lib, w, workloads.initial_modes(w), 2, 4)
    assert any(r["switched"][1] for r in res)
    for r in res:
        assert r["switched"][0] == r["switched"][1], r["k"]
        assert r["err_u"] < 1e-12 and r["err_E"] < 1e-12, (r["k"], r["err_u"], r["err_E"])


def test_grid_state_has_no_factors(lib):
    w = workloads.preset("c0", n=(10, 10), s=2, p=2, M_max=30, I_max=200, tol_als=1e-10, tol_enrich=1e-8)
    s = lib.Solver(lib.config_from_workload(w, actd_Mc=2))
    s.set_initial_modes(workloads.cosine_modes(w.n, w.length, 4, 4, 3, amp=0.9))
    assert s.step(1)[0]["actd_switched"]
    with pytest.raises(lib.CTDError) as e:
        s.get_modes()
    assert e.value.status == -6          # CTD_ERR_STATE
    s.close()
