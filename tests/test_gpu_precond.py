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


KAPPA = 7.0  # §4.2, Fig. 6


@pytest.mark.parametrize("m", [1, 7, 15])
def test_helmholtz7_matches_sparse_operator(cuda, m):
    import scipy.sparse as sp
    h = 2.0 / (m + 1)
    u = np.random.default_rng(m + 1).normal(size=m ** 3)
    out = binding.helmholtz7(torch.tensor(u, device=cuda), h, KAPPA).cpu().numpy()
    ref = (laplacian_csr(m, h) - KAPPA ** 2 * sp.identity(m ** 3)) @ u
    assert np.linalg.norm(out - ref) <= 1e-14 * np.linalg.norm(ref)


def test_helmholtz_fmm_preconditioned_gmres_matches_direct_solve(cuda):
    """-Laplace u - 49 u = 1 on [-1, 1]^3 (indefinite), h = 2^-3 against a
    sparse direct solve, and at h = 2^-4 in fewer iterations than plain GMRES
    (on the 15^3 grid the two take a similar number: 50-80 against 59)."""
    import scipy.sparse as sp
    from scipy.sparse.linalg import spsolve
    for h in (2.0 ** -3, 2.0 ** -4):
        pre = precond.HelmholtzGreenPreconditioner(h, KAPPA, order=4, leaf_size=32, device=cuda)
        m = pre.m
        b = torch.ones(m ** 3, dtype=torch.float64, device=cuda)
        A = lambda v: binding.helmholtz7(v, h, KAPPA)
        x, it, hist = precond.fgmres(A, b, pre, tol=1e-10, restart=50, maxiter=3000)
        x0, it0, hist0 = precond.fgmres(A, b, None, tol=1e-10, restart=50, maxiter=3000)
        pre.close()
        print("h=%g: FMM-preconditioned GMRES %d iterations, plain GMRES(50) %d (residual %.1e)"
              % (h, it, it0, hist0[-1]))
        assert hist[-1] <= 1e-10
        if h == 2.0 ** -4:
            assert it < it0 / 4
        if h == 2.0 ** -3:
            K = (laplacian_csr(m, h) - KAPPA ** 2 * sp.identity(m ** 3)).tocsc()
            ref = spsolve(K, np.ones(m ** 3))
            assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)
