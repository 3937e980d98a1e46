"""Reduced integration domain (Section 3.3) on the GPU against the oracle with the same
reading (blocks of 128 nodes per dimension dropped while max |w(u^k)| <= reduced_tol): a
straight interface across a 640 x 300 grid leaves one block row of five in the domain, and in
3D an interface normal to each axis leaves one block of three.  FP64 path within 1e-12,
split-BF16 path within 1e-5 (u and energy).

The energy of a sharp interface is a sum of terms much larger than itself (the stiffness
products of the nearly constant regions cancel), so its FP64 evaluation, in either program,
carries a relative error up to cond_E 2^-53 with cond_E = sum |terms| / |E| (about 1.2e4
here, i.e. 1.4e-12); the energy tolerance adds four times that bound."""
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


def energy_condition(prob, ops, A):
    """sum of |terms| of the discrete energy over |E| (nodal bulk term + stiffness term)."""
    U = octd.reconstruct(A)
    Wg = octd.grid_weights(ops)
    absum = float(np.sum(np.abs(Wg * prob.a0 * (U ** 2 - 1.0) ** 2)))
    for d in range(prob.dim):
        T = np.moveaxis(np.abs(U), d, 0)
        KT = np.moveaxis((abs(ops.K[d]) @ T.reshape(T.shape[0], -1)).reshape(T.shape), 0, d)
        ow = np.ones_like(U)
        for e in range(prob.dim):
            if e != d:
                sh = [1] * prob.dim
                sh[e] = -1
                ow = ow * ops.omega[e].reshape(sh)
        absum += 0.5 * prob.kappa * float(np.sum(np.abs(U) * KT * ow))
    return absum / abs(octd.energy(prob, ops, A))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_reduced_domain_matches_oracle(lib, prec, tol):
    w = workloads.preset("c0", n=(640, 300), s=2, p=2, eps=0.01, dt=1e-3, M_max=10, ic_rank=0, ic_tanh=True)
    red = 1e-4
    cfg = lib.config_from_workload(w, precision=lib.PREC_FP64 if prec == "fp64" else lib.PREC_SPLIT_BF16,
                                   reduced_tol=red)
    s = lib.Solver(cfg)
    A = workloads.initial_modes(w)
    s.set_initial_modes(A)
    prob = octd.Problem(dim=2, n=w.n, length=w.length, s=w.s, p=w.p, a=w.a, L=w.L, kappa=w.kappa, a0=w.a0,
                        alpha=w.alpha, dt=w.dt, M_max=w.M_max, I_max=w.I_max, tol_als=w.tol_als,
                        tol_enrich=w.tol_enrich, seed=w.seed, reduced_tol=red)
    ops = octd.build_operators(prob)
    W = octd.w_of_u(octd.reconstruct(A), prob.a0)
    kept = octd.reduced_domain_mask(prob, W)
    assert 0.1 < kept.mean() < 0.3     # the interface's block row only
    for k in range(3):
        A, so = octd.step(prob, ops, A, k)
        sg = s.step(1)[0]
        # the field is rank 1 (tanh (x) 1): after the first mode only round-off is left, whose
        # sweep count is not meaningful; the mode count and the field are
        assert sg["modes"] == so["modes"], (k, sg, so)
        G = s.get_modes()
        assert octd.rel_l2_between(G, A) < tol, (k, octd.rel_l2_between(G, A))
        eo = octd.energy(prob, ops, A)
        tol_e = tol + 4.0 * energy_condition(prob, ops, A) * 2.0 ** -53
        assert abs(s.energy() - eo) / abs(eo) < tol_e, (k, abs(s.energy() - eo) / abs(eo), tol_e)
    s.close()


def interface_modes(n, axis, eps):
    """u = tanh((x_axis - 1/2) / (sqrt(2) eps)): one separated mode, the interface normal to `axis`."""
    out = []
    for d in range(3):
        x = np.linspace(0.0, 1.0, n[d])
        f = np.tanh((x - 0.5) / (np.sqrt(2.0) * eps)) if d == axis else np.ones(n[d])
        out.append(f[:, None])
    return out


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
@pytest.mark.parametrize("axis,n", [(0, (384, 24, 20)), (1, (20, 384, 24)), (2, (20, 24, 384))])
def test_reduced_domain_3d_matches_oracle(lib, prec, tol, axis, n):
    # an interface normal to each axis in turn: of the three 128-node blocks along that axis
    # only the middle one stays in the domain; the others (u = +-1, w ~ 1e-10) drop out
    w = workloads.preset("c0", dim=3, n=n, length=(1.0, 1.0, 1.0), s=2, p=2, eps=0.01, dt=1e-3, M_max=10)
    red = 1e-4
    cfg = lib.config_from_workload(w, precision=lib.PREC_FP64 if prec == "fp64" else lib.PREC_SPLIT_BF16,
                                   reduced_tol=red)
    s = lib.Solver(cfg)
    A = interface_modes(n, axis, w.eps)
    s.set_initial_modes(A)
    prob = octd.Problem(dim=3, n=w.n, length=w.length, s=w.s, p=w.p, a=w.a, L=w.L, kappa=w.kappa, a0=w.a0,
                        alpha=w.alpha, dt=w.dt, M_max=w.M_max, I_max=w.I_max, tol_als=w.tol_als,
                        tol_enrich=w.tol_enrich, seed=w.seed, reduced_tol=red)
    ops = octd.build_operators(prob)
    kept = octd.reduced_domain_mask(prob, octd.w_of_u(octd.reconstruct(A), prob.a0))
    assert abs(kept.mean() - 1.0 / 3.0) < 1e-12
    for k in range(3):
        A, so = octd.step(prob, ops, A, k)
        sg = s.step(1)[0]
        assert sg["modes"] == so["modes"], (k, sg, so)
        assert octd.rel_l2_between(s.get_modes(), A) < tol, (k, octd.rel_l2_between(s.get_modes(), A))
        eo = octd.energy(prob, ops, A)
        tol_e = tol + 4.0 * energy_condition(prob, ops, A) * 2.0 ** -53
        assert abs(s.energy() - eo) / abs(eo) < tol_e, (k, abs(s.energy() - eo) / abs(eo), tol_e)
    s.close()
