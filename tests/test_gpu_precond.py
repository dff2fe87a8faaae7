"""The FMM as a preconditioner (§4.2), Laplace part: the 7-point operator
against a sparse matrix built with scipy, and the FMM-preconditioned CG
against a sparse direct solve of the same discrete problem."""
import math

import numpy as np
import pytest
import torch

from paper_1602_02244_gb300 import binding, precond

pytestmark = pytest.mark.gpu


def laplacian_csr(m, h):
    import scipy.sparse as sp
    t = sp.diags([-np.ones(m - 1), 2 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1])
    e = sp.identity(m)
    # index (k m + j) m + i: i (x) is the fastest, i.e. the rightmost Kronecker factor
    return ((sp.kron(sp.kron(e, e), t) + sp.kron(sp.kron(e, t), e) + sp.kron(sp.kron(t, e), e))
            / (h * h)).tocsr()


@pytest.mark.parametrize("m", [1, 2, 7, 15])
def test_laplace7_matches_sparse_operator(cuda, m):
    h = 2.0 / (m + 1)
    u = np.random.default_rng(m).normal(size=m ** 3)
    out = binding.laplace7(torch.tensor(u, device=cuda), h).cpu().numpy()
    ref = laplacian_csr(m, h) @ u
    assert np.linalg.norm(out - ref) <= 1e-14 * np.linalg.norm(ref)


def test_fmm_preconditioned_cg_matches_direct_solve(cuda):
    from scipy.sparse.linalg import spsolve
    h = 2.0 ** -4
    pre = precond.GreenPreconditioner(h, order=3, leaf_size=32, device=cuda)
    m = pre.m
    f = np.ones(m ** 3)
    b = torch.tensor(f, device=cuda)
    A = lambda v: binding.laplace7(v, h)
    x, it, hist = precond.fpcg(A, b, pre, tol=1e-10, maxiter=500)
    x0, it0, _ = precond.fpcg(A, b, None, tol=1e-10, maxiter=500)
    pre.close()
    ref = spsolve(laplacian_csr(m, h), f)
    err = np.linalg.norm(x.cpu().numpy() - ref) / np.linalg.norm(ref)
    print("h=2^-4: FMM-preconditioned CG %d iterations, plain CG %d, rel err %.2e" % (it, it0, err))
    assert hist[-1] <= 1e-10 and err <= 1e-8
    assert np.linalg.norm(x0.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)
    assert it < it0
