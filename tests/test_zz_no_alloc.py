"""ctd_probe_reconstruct_noalloc (dump through the library's static device array) against
ctd_probe_reconstruct (dump through a caller buffer), through the C ABI.

Both run the same tensor-core reconstruction kernel on the same field, so two calls in a row
of the static variant must agree with the caller-buffer entry point within the split-BF16
reconstruction tolerance (5e-5 of max_ij sum_m |a_im b_jm|, derived in
test_gpu_tensorcore.py) and, the kernel being deterministic, bit for bit.  This file runs
last so that it also covers the static array after every other GPU test has used the
library in the same process.
"""
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


def pad128(n):
    return (n + 127) // 128 * 128


def _cols(n, x):
    others = [n[d] for d in range(len(n)) if d != x]
    if len(others) == 1:
        return pad128(others[0])
    return others[0] * pad128(others[1])


@pytest.mark.parametrize("n,rank", [((200, 77), 5), ((20, 33, 17), 4)])
def test_noalloc_matches_caller_scratch(lib, n, rank):
    dim = len(n)
    w = workloads.preset("c0", dim=dim, n=n, length=(1.0,) * dim, M_max=8)
    cfg = lib.config_from_workload(w, precision=lib.PREC_SPLIT_BF16)
    s = lib.Solver(cfg)
    A = workloads.cosine_modes(n, (1.0,) * dim, rank, 4, 11, amp=0.8)
    s.set_initial_modes(A)
    for x in range(dim):
        rows, cols = pad128(n[x]), _cols(n, x)
        ref = s.probe_reconstruct(x, rows, cols)
        # magnitude scale of the reconstruction: max over the grid of sum_m prod_d |a_dm|
        absA = [np.abs(a) for a in A]
        if dim == 2:
            scale = np.max(absA[0] @ absA[1].T)
        else:
            scale = np.max(np.einsum("im,jm,km->ijk", *absA))
        tol = 5e-5 * scale
        for _ in range(2):
            got = s.probe_reconstruct_noalloc(x, rows, cols)
            assert np.max(np.abs(got.astype(np.float64) - ref.astype(np.float64))) <= tol
            assert np.array_equal(got, ref)
    s.close()


def test_noalloc_rejects_grid_beyond_static_array(lib):
    # 2048 x 1024 tile grid of FP32 = 8 MiB > 4 MiB
    n = (2048, 1024)
    w = workloads.preset("c0", n=n, M_max=4)
    cfg = lib.config_from_workload(w, precision=lib.PREC_SPLIT_BF16)
    s = lib.Solver(cfg)
    s.set_initial_modes(workloads.cosine_modes(n, (1.0, 1.0), 2, 4, 3, amp=0.5))
    with pytest.raises(lib.CTDError) as ei:
        s.probe_reconstruct_noalloc(0, 2048, 1024)
    assert ei.value.status == -2 and "static dump array" in str(ei.value)
    s.close()
