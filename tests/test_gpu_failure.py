"""Failure paths of the step through the C ABI, driven from the host with valid launches:
non-finite initial data, the mode cap, the sweep cap, and a grid-wide wait that runs out of
its time limit (FP64 path: no bulk copies or tensor-core work are in flight when a wait gives
up).  None of these faults, traps or hangs the GPU: each ends in a status the host reads, and
a fresh handle works afterwards."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_15519_gb300 import build, ctd
    build.build()
    return ctd


def fresh_step_ok(lib, w):
    s = lib.Solver(lib.config_from_workload(w))
    s.set_initial_modes(workloads.initial_modes(w))
    st = s.step(1)[0]
    G = s.get_modes()
    s.close()
    assert st["status"] >= 0 and st["modes"] > 0
    assert all(np.all(np.isfinite(g)) for g in G)


def test_nonfinite_host_modes_are_refused(lib):
    w = workloads.preset("c0", n=(40, 36))
    A = workloads.initial_modes(w)
    A[1][7, 2] = np.nan
    s = lib.Solver(lib.config_from_workload(w))
    with pytest.raises(lib.CTDError) as e:
        s.set_initial_modes(A)
    assert e.value.status == -4          # CTD_ERR_NONFINITE
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_nonfinite_device_modes_fail_the_step(lib, prec):
    import torch
    w = workloads.preset("c0", n=(40, 36))
    A = [torch.as_tensor(a, device="cuda") for a in workloads.initial_modes(w)]
    A[0][5, 1] = float("nan")
    p = lib.PREC_FP64 if prec == "fp64" else lib.PREC_SPLIT_BF16
    s = lib.Solver(lib.config_from_workload(w, precision=p))
    s.set_initial_modes(A)                 # device data is not inspected here ...
    with pytest.raises(lib.CTDError) as e:
        s.step(1)                          # ... the step's solve reports it
    assert e.value.status == -4
    s.close()
    fresh_step_ok(lib, w)


def test_mode_cap_reports_capped(lib):
    w = workloads.preset("c0", n=(40, 36), M_max=1, ic_rank=1)
    s = lib.Solver(lib.config_from_workload(w))
    s.set_initial_modes(workloads.initial_modes(w))
    st = s.step(2)
    s.close()
    for r in st:
        assert r["modes"] == 1 and r["capped"] and r["status"] == 1   # CTD_STATUS_CAPPED


def test_sweep_cap_reports_not_converged(lib):
    w = workloads.preset("c0", n=(40, 36), I_max=1)
    s = lib.Solver(lib.config_from_workload(w))
    s.set_initial_modes(workloads.initial_modes(w))
    st = s.step(2)
    s.close()
    for r in st:
        assert r["not_converged"] and r["als_sweeps_max"] == 1
        assert r["status"] == 2                                       # CTD_STATUS_ALS_NOT_CONVERGED
        assert r["als_stalled"] == 0


def test_grid_wait_time_limit_gives_timeout(lib):
    # A 1024^2 FP64 step: the other CTAs wait through CTA 0's banded solve (tens of
    # microseconds), far beyond a 100 ns limit, so a grid-wide wait gives up and every CTA
    # leaves the kernel.
    w = workloads.preset("c1", n=(1024, 1024))
    s = lib.Solver(lib.config_from_workload(w, wait_limit_s=1e-7))
    s.set_initial_modes(workloads.initial_modes(w))
    with pytest.raises(lib.CTDError) as e:
        s.step(1)
    assert e.value.status == -5            # CTD_ERR_TIMEOUT
    assert "wait" in str(e.value)
    # the handle keeps its error state; a fresh handle on the same device works
    with pytest.raises(lib.CTDError):
        s.energy()
    s.close()
    fresh_step_ok(lib, workloads.preset("c1", n=(1024, 1024)))
