"""The FMM as a preconditioner (§4.2): the free-space Green's function of the
Laplacian, applied with the FMM, approximates the inverse of the discrete
Laplacian of a grid problem.

For -Laplace(u) = f on [-1, 1]^3 with u = 0 on the boundary, discretised by
the 7-point stencil on the m^3 interior points of spacing h (m = 2/h - 1):

  A = 7-point Laplacian (``fmm_laplace7_apply``),
  M^{-1} r ~ int G(x - y) r(y) dy,  G(r) = 1 / (4 pi r),

evaluated as the FMM mat-vec with charges r_j h^3 / (4 pi) over the grid
points, plus the cell's own contribution c h^2 r_i.  Here c is the integral
of 1/(4 pi |x|) over the unit cube around its centre.  The corner-cube closed
form gives c = (3 ln((1 + sqrt 3) / sqrt 2) - pi/4) * 2 / (4 pi).

The Krylov solver is the flexible preconditioned conjugate gradient (the
Polak-Ribiere form of beta), which tolerates a preconditioner that is
symmetric only up to rounding, as a low-order mixed-precision FMM is.  The
vector updates are plain tensor operations; the operator and the
preconditioner run in this library's kernels.
"""
import math

import torch

from . import binding

# (1 / 4 pi) * integral over [-1/2, 1/2]^3 of 1 / |x|
CELL_SELF = (3.0 * math.log((1.0 + math.sqrt(3.0)) / math.sqrt(2.0)) - math.pi / 4.0) * 2.0 / (
    4.0 * math.pi)


def grid_points(h, device=None, dtype=torch.float64):
    """Interior points of [-1, 1]^3 at spacing h, index (k m + j) m + i."""
    m = int(round(2.0 / h)) - 1
    g = -1.0 + h * torch.arange(1, m + 1, dtype=dtype, device=device)
    z, y, x = torch.meshgrid(g, g, g, indexing="ij")
    return torch.stack([x.reshape(-1), y.reshape(-1), z.reshape(-1)], dim=1).contiguous(), m


class GreenPreconditioner:
    """z = h^3 / (4 pi) sum_j r_j / |x_i - x_j| + CELL_SELF h^2 r_i, with the
    sum evaluated by the FMM (plan built once over the grid)."""

    def __init__(self, h, order=3, leaf_size=64, precision="mixed", device=None):
        self.h = h
        self.points, self.m = grid_points(h, device=device)
        self.plan = binding.Plan(self.points, leaf_size=leaf_size, order=order,
                                 precision=precision)
        self.scale = h ** 3 / (4.0 * math.pi)
        self.self_coef = CELL_SELF * h * h

    def __call__(self, r):
        phi, _ = self.plan.eval(r, grad=False)
        return self.scale * phi + self.self_coef * r

    def close(self):
        self.plan.close()


def fpcg(apply_a, b, apply_m=None, tol=1e-8, maxiter=1000):
    """Flexible preconditioned conjugate gradient for A x = b (A symmetric
    positive definite).  Returns (x, iterations, relative residual history)."""
    x = torch.zeros_like(b)
    r = b.clone()
    bnorm = float(torch.linalg.vector_norm(b))
    if bnorm == 0.0:
        return x, 0, [0.0]
    z = apply_m(r) if apply_m else r.clone()
    p = z.clone()
    rz = float(torch.dot(r, z))
    hist = [1.0]
    for it in range(1, maxiter + 1):
        ap = apply_a(p)
        alpha = rz / float(torch.dot(p, ap))
        x.add_(p, alpha=alpha)
        r_old_z = z
        r.add_(ap, alpha=-alpha)
        rel = float(torch.linalg.vector_norm(r)) / bnorm
        hist.append(rel)
        if rel <= tol:
            return x, it, hist
        z = apply_m(r) if apply_m else r.clone()
        rz_new = float(torch.dot(r, z))
        beta = (rz_new - float(torch.dot(r, r_old_z))) / rz  # Polak-Ribiere (flexible)
        rz = rz_new
        p.mul_(beta).add_(z)
    return x, maxiter, hist
