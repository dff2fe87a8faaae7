"""Host-side pins of the preconditioning experiment (§4.2): the cell
self-term constant against numerical quadrature, the flexible PCG against a
dense solve, and the grid ordering the stencil assumes."""
import math

import numpy as np
import pytest
import torch

from paper_1602_02244_gb300 import precond


def test_cell_self_term_matches_quadrature():
    from scipy import integrate
    # 8 corner cubes [0, 1/2]^3 of 1 / (4 pi |x|); the integrand is singular only at a corner
    val, err = integrate.tplquad(lambda z, y, x: 1.0 / math.sqrt(x * x + y * y + z * z),
                                 0, 0.5, 0, 0.5, 0, 0.5, epsabs=1e-11, epsrel=1e-11)
    assert abs(8.0 * val / (4.0 * math.pi) - precond.CELL_SELF) < 1e-8
    assert abs(precond.CELL_SELF - 0.18940) < 1e-5


def test_fpcg_solves_spd_system_on_cpu():
    g = np.random.default_rng(0)
    n = 60
    B = g.normal(size=(n, n))
    A = B @ B.T + n * np.eye(n)
    b = g.normal(size=n)
    At = torch.tensor(A)
    d = torch.tensor(np.diag(A))
    x, it, hist = precond.fpcg(lambda v: At @ v, torch.tensor(b), lambda r: r / d, tol=1e-12)
    assert np.linalg.norm(x.numpy() - np.linalg.solve(A, b)) <= 1e-9 * np.linalg.norm(np.linalg.solve(A, b))
    assert it < n and hist[-1] <= 1e-12
    x0, it0, _ = precond.fpcg(lambda v: At @ v, torch.zeros(n), tol=1e-10)
    assert it0 == 0 and float(x0.abs().max()) == 0.0


def test_grid_points_order_and_spacing():
    pts, m = precond.grid_points(0.25)
    assert m == 7 and pts.shape == (343, 3)
    # index (k m + j) m + i: x varies fastest, then y, then z
    assert torch.allclose(pts[1] - pts[0], torch.tensor([0.25, 0.0, 0.0], dtype=torch.float64))
    assert torch.allclose(pts[m] - pts[0], torch.tensor([0.0, 0.25, 0.0], dtype=torch.float64))
    assert torch.allclose(pts[m * m] - pts[0], torch.tensor([0.0, 0.0, 0.25], dtype=torch.float64))
    assert float(pts.min()) == -0.75 and float(pts.max()) == 0.75


def test_fgmres_solves_nonsymmetric_and_indefinite_systems():
    import numpy as np
    import torch
    rng = np.random.default_rng(0)
    n = 120
    A = 3.0 * np.eye(n) + rng.normal(size=(n, n)) / np.sqrt(n)          # nonsymmetric
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    B = Q @ np.diag(np.linspace(-2.0, 5.0, n) + 0.013) @ Q.T            # symmetric indefinite
    b = rng.normal(size=n)
    for M, restart in ((A, 20), (B, n)):
        Mt = torch.tensor(M)
        x, it, hist = precond.fgmres(lambda v: Mt @ v, torch.tensor(b), None, tol=1e-10,
                                     restart=restart, maxiter=5 * n)
        ref = np.linalg.solve(M, b)
        assert hist[-1] <= 1e-10
        assert np.linalg.norm(x.numpy() - ref) <= 1e-8 * np.linalg.norm(ref)
    # an exact preconditioner converges in one step; a good one in a few
    Bi = torch.tensor(np.linalg.inv(B))
    Bt = torch.tensor(B)
    x, it, hist = precond.fgmres(lambda v: Bt @ v, torch.tensor(b), lambda v: Bi @ v, tol=1e-10)
    assert it <= 2 and hist[-1] <= 1e-10
