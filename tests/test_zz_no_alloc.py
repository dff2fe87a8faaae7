"""fmm_morton_sort_noalloc: the Morton-key sort for callers that cannot let a
library allocate device memory (their memory manager owns all free device
memory, or their loop forbids cudaMalloc/cudaFree for latency reasons).

It must give exactly what the allocating path gives (sorting is integer work,
so the comparison is bit for bit) on two calls in a row, and reject inputs
larger than its fixed scratch array.  This file sorts last so that a failure
here stops a `-x` run only after every other test has run."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1602_02244_gb300 import binding, workloads

pytestmark = pytest.mark.gpu

MAX_POINTS = 1048576


def noalloc_fn():
    L = binding.library()
    f = L.fmm_morton_sort_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def test_noalloc_sort_matches_plan_on_two_calls(cuda):
    f = noalloc_fn()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [workloads.plummer(300001, 4), workloads.uniform_cube(MAX_POINTS, 5)]
    for xyz in cases:
        n = len(xyz)
        X = torch.tensor(xyz, device=cuda)
        keys = torch.full((n,), -1, dtype=torch.int64, device=cuda)
        perm = torch.full((n,), -1, dtype=torch.int32, device=cuda)
        root = (ctypes.c_double * 4)()
        st = f(X.data_ptr(), n, keys.data_ptr(), perm.data_ptr(), root, stream)
        assert st == 0, binding.library().fmm_last_error_message()
        torch.cuda.synchronize()
        plan = binding.Plan(X, leaf_size=64, order=2)
        ref = plan.export()
        plan.close()
        assert np.array_equal(keys.cpu().numpy().view(np.uint64), ref["keys"])
        assert np.array_equal(perm.cpu().numpy(), ref["perm"])
        assert list(root) == list(ref["root"])


def test_noalloc_sort_rejects_oversized_input(cuda):
    f = noalloc_fn()
    st = f(None, MAX_POINTS + 1, None, None, None, None)
    assert st == 1
    msg = binding.library().fmm_last_error_message().decode()
    assert "FMM_NOALLOC_MAX_POINTS" in msg


def test_noalloc_sort_refuses_a_capturing_stream(cuda):
    # every call reads the root cube back and synchronises its stream, which a
    # CUDA graph capture cannot hold: the call is refused and the capture stays valid
    f = noalloc_fn()
    n = 1000
    X = torch.tensor(workloads.uniform_cube(n, 6), device=cuda)
    keys = torch.empty(n, dtype=torch.int64, device=cuda)
    perm = torch.empty(n, dtype=torch.int32, device=cuda)
    y = torch.zeros(4, device=cuda)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        st = f(X.data_ptr(), n, keys.data_ptr(), perm.data_ptr(), None, stream)
        y.add_(1.0)
    assert st == 1
    assert "capturing" in binding.library().fmm_last_error_message().decode()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(y.cpu(), torch.ones(4))
