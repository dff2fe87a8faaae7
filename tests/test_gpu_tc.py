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
