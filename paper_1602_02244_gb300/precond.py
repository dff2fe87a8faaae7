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

The Helmholtz half: -Laplace(u) - kappa^2 u = f with the same boundary
condition and stencil (``fmm_helmholtz7_apply``).  Its free-space Green's
function is cos(kappa r) / (4 pi r), the real part of e^{i kappa r} / (4 pi r),
so the preconditioner is the real part of the Helmholtz FMM mat-vec with
charges r_j h^3 / (4 pi), plus the same cell term (the cell integral of
cos(kappa r)/(4 pi r) differs from the Laplace one by O((kappa h)^2)).  The
operator is symmetric but indefinite once kappa^2 exceeds its smallest
eigenvalues (3 pi^2 / 4 on this cube), so the solver is restarted flexible
GMRES (right preconditioning) instead of CG.
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


class HelmholtzGreenPreconditioner:
    """z = Re[h^3 / (4 pi) sum_j r_j e^{i kappa |x_i - x_j|} / |x_i - x_j|] + CELL_SELF h^2 r_i,
    the sum evaluated by the Helmholtz FMM of ``order`` (plan built once;
    "mixed" runs its near field in FP32)."""

    def __init__(self, h, kappa, order=4, leaf_size=64, precision="mixed", device=None):
        self.h = h
        self.kappa = float(kappa)
        self.order = order
        self.points, self.m = grid_points(h, device=device)
        self.plan = binding.Plan(self.points, leaf_size=leaf_size, order=min(order, 8),
                                 precision=precision)
        self.scale = h ** 3 / (4.0 * math.pi)
        self.self_coef = CELL_SELF * h * h

    def __call__(self, r):
        q = (self.scale * r).to(torch.complex128)
        phi = self.plan.helmholtz(q, self.kappa, self.order)
        return phi.real + self.self_coef * r

    def close(self):
        self.plan.close()


def fgmres(apply_a, b, apply_m=None, tol=1e-8, restart=50, maxiter=1000):
    """Restarted flexible GMRES with right preconditioning for A x = b (A need
    not be symmetric or definite).  Arnoldi by classical Gram-Schmidt applied
    twice (CGS2: two matrix-vector products against the basis per step, as
    accurate as modified Gram-Schmidt and one host read-back per step), the
    small least-squares problem by Givens rotations.  Returns (x, iterations,
    relative residual history)."""
    import numpy as np
    x = torch.zeros_like(b)
    bnorm = float(torch.linalg.vector_norm(b))
    if bnorm == 0.0:
        return x, 0, [0.0]
    n = b.numel()
    V = torch.empty(restart + 1, n, dtype=b.dtype, device=b.device)
    Z = torch.empty(restart, n, dtype=b.dtype, device=b.device)
    r = b.clone()
    beta = bnorm
    hist = [1.0]
    it = 0
    while True:
        V[0] = r / beta
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        j_end = 0
        done = False
        for j in range(restart):
            Z[j] = apply_m(V[j]) if apply_m else V[j]
            w = apply_a(Z[j])
            Vj = V[:j + 1]
            h = Vj @ w
            w.sub_(h @ Vj)
            h2 = Vj @ w
            w.sub_(h2 @ Vj)
            h.add_(h2)
            hv = torch.cat([h, torch.linalg.vector_norm(w).view(1)]).cpu().numpy()
            H[:j + 2, j] = hv
            breakdown = not H[j + 1, j] > 0.0
            if not breakdown:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):  # earlier rotations on the new column
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            d = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = (1.0, 0.0) if d == 0.0 else (H[j, j] / d, H[j + 1, j] / d)
            H[j, j] = d
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_end = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if hist[-1] <= tol or it >= maxiter or breakdown:
                done = True
                break
        y = np.zeros(j_end)
        for i in range(j_end - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:j_end] @ y[i + 1:j_end]) / H[i, i]
        x.add_(torch.tensor(y, dtype=b.dtype, device=b.device) @ Z[:j_end])
        r = b - apply_a(x)
        beta = float(torch.linalg.vector_norm(r))
        if done:
            hist[-1] = beta / bnorm  # the true residual, for the record
            if hist[-1] <= tol or it >= maxiter:
                return x, it, hist
        if beta / bnorm <= tol:
            return x, it, hist
