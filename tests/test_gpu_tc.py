"""Self-check of the tensor-core (tcgen05.mma, kind::tf32) path through the
C-ABI diagnostic fmm_tc_selftest: D = A B^T for random FP32 operands against
an FP64 product.  One TF32 product is good to ~1e-3; the three-product split
must reach FP32-level accuracy, which also proves both halves of the split
land where the descriptors say."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1602_02244_gb300 import binding

pytestmark = pytest.mark.gpu


def run(cuda, n, k, mode, seed=0):
    L = binding.library()
    f = L.fmm_tc_selftest
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_int, ctypes.c_void_p]
    f.restype = ctypes.c_int
    g = np.random.default_rng(seed)
    A = g.normal(size=(128, k)).astype(np.float32)
    B = g.normal(size=(n, k)).astype(np.float32)
    dA, dB = torch.tensor(A, device=cuda), torch.tensor(B, device=cuda)
    dD = torch.zeros(128, n, dtype=torch.float32, device=cuda)
    st = f(n, k, dA.data_ptr(), dB.data_ptr(), dD.data_ptr(), mode,
           torch.cuda.current_stream().cuda_stream)
    assert st == 0, L.fmm_last_error_message()
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    D = dD.cpu().numpy().astype(np.float64)
    return np.abs(D - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("n,k", [(96, 88), (16, 8), (128, 64), (32, 24)])
def test_tc_three_product_is_fp32_accurate(cuda, n, k):
    e1 = run(cuda, n, k, 1)
    e3 = run(cuda, n, k, 3)
    print("n=%d k=%d: 1-product %.2e, 3-product %.2e" % (n, k, e1, e3))
    assert e1 < 5e-3
    assert e3 < 5e-6
    assert e3 < e1 / 50


def test_bounded_wait_gives_up_and_the_device_stays_usable(cuda):
    """Failure detection without a GPU fault: a wait on an mbarrier that
    nothing arrives at gives up after its limit (about a millisecond here),
    the kernel returns, the host reads FMM_ERR_TIMEOUT, and the device then
    runs an FMM that matches the oracle."""
    import oracle
    from paper_1602_02244_gb300 import workloads
    L = binding.library()
    s = torch.cuda.current_stream().cuda_stream
    assert L.fmm_wait_selftest(1, 2_000_000, s) == 0  # the arrival completes the wait
    assert L.fmm_wait_selftest(0, 2_000_000, s) == 4  # FMM_ERR_TIMEOUT
    assert b"gave up" in L.fmm_last_error_message()
    assert L.fmm_wait_selftest(0, 0, s) == 1  # limit out of range: FMM_ERR_INVALID_ARG
    xyz, q = workloads.uniform_cube_problem(3000, 4)
    plan = binding.Plan(torch.tensor(xyz, device=cuda), leaf_size=32, order=6, precision="mixed")
    phi, _ = plan.eval(torch.tensor(q, device=cuda))
    plan.close()
    po = oracle.Tree(xyz, 32).eval(6, q, grad=False)
    err = np.linalg.norm(phi.cpu().numpy() - po) / np.linalg.norm(po)
    assert err < 1e-5
