"""Seeded synthetic inputs for the 3D Laplace FMM mat-vec.

Holds none of the method's arithmetic: only point clouds and charges.  Both
the GPU path's tests/benchmark and the CPU oracle's tests draw from here.
All generators use numpy ``Generator(PCG64(seed))`` in float64.

The paper benchmarks uniform lattices (§4) whose sizes it does not print;
these distributions stand in for them:
  - uniform in the unit cube, charges U[-1, 1];
  - Plummer sphere (scale 1, radii truncated at 10), charges 1/N;
  - uniform on the unit sphere surface, charges N(0, 1);
  - batches of uniform problems with log-uniform sizes.
"""
import numpy as np


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def uniform_cube(n, seed=0):
    """n points uniform in [0, 1)^3."""
    return rng(seed).random((n, 3))


def uniform_cube_problem(n, seed=0):
    """Points uniform in [0,1)^3, then charges U[-1,1] from the same stream."""
    g = rng(seed)
    xyz = g.random((n, 3))
    q = g.uniform(-1.0, 1.0, n)
    return xyz, q


def plummer(n, seed=0, scale=1.0, rmax=10.0):
    """Plummer-sphere radii r = a (X^(-2/3) - 1)^(-1/2), X ~ U(0,1), redrawn
    while r > rmax; isotropic directions from normalised N(0, I_3)."""
    g = rng(seed)
    r = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        X = g.random(todo.size)
        with np.errstate(divide="ignore", invalid="ignore"):
            rr = scale / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
        ok = np.isfinite(rr) & (rr <= rmax)
        r[todo[ok]] = rr[ok]
        todo = todo[~ok]
    d = g.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d * r[:, None]


def plummer_problem(n, seed=0):
    """Plummer points and equal positive charges 1/N."""
    return plummer(n, seed), np.full(n, 1.0 / n)


def sphere_surface(n, seed=0):
    """n points uniform on the unit sphere surface (normalised Gaussians)."""
    d = rng(seed).normal(size=(n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def sphere_problem(n, seed=0, weight_seed=2):
    """Sphere-surface points, charges N(0,1) (same stream), loss weights
    w ~ N(0,1) from ``weight_seed``."""
    g = rng(seed)
    d = g.normal(size=(n, 3))
    xyz = d / np.linalg.norm(d, axis=1, keepdims=True)
    q = g.normal(size=n)
    w = rng(weight_seed).normal(size=n)
    return xyz, q, w


def batch_sizes(count=256, lo=2048, hi=65536, seed=0):
    """Problem sizes round(exp(U[ln lo, ln hi]))."""
    return np.rint(np.exp(rng(seed).uniform(np.log(lo), np.log(hi), count))).astype(np.int64)


def batch_problem(count=256, seed=0, lo=2048, hi=65536):
    """``count`` uniform-cube problems; problem b uses seed 1000 + b."""
    sizes = batch_sizes(count, lo, hi, seed)
    pts, qs = [], []
    for b, nb in enumerate(sizes):
        x, q = uniform_cube_problem(int(nb), 1000 + b)
        pts.append(x)
        qs.append(q)
    return sizes, pts, qs


def lattice(side):
    """side^3 points at the cell centres of a uniform lattice on [0, 1)^3
    (the paper's benchmark inputs, §4.1): (i + 1/2) / side per axis.  Relative
    to the root cube's corner they sit exactly on dyadic box boundaries when
    side is a power of two."""
    g = (np.arange(side) + 0.5) / side
    return np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)


def sample_targets(n, k=4096, seed=1):
    """k distinct target indices (all of them when n <= k)."""
    if n <= k:
        return np.arange(n)
    return np.sort(rng(seed).choice(n, k, replace=False))
