"""Batched plans: many independent problems of uneven size in one plan (a
forest of octrees); every pass runs once over all problems.  Each member's
results must equal its own single-problem plan bit for bit, and the single
runs match the oracle (tested elsewhere)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1602_02244_gb300 import binding, workloads

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def concat(count, lo, hi, seed=0):
    sizes, pts, qs = workloads.batch_problem(count, seed, lo, hi)
    off = np.concatenate([[0], np.cumsum(sizes)])
    return sizes, off, np.vstack(pts), np.concatenate(qs), pts, qs


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_members_equal_single_plans(cuda, precision):
    sizes, off, xyz, q, pts, qs = concat(12, 100, 6000, seed=4)
    S, p = 24, 6
    plan = binding.Plan(torch.tensor(xyz, device=cuda), leaf_size=S, order=p,
                        precision=precision, offsets=off)
    phi, g = plan.eval(torch.tensor(q, device=cuda))
    phi, g = phi.cpu().numpy(), g.cpu().numpy()
    roots = plan.export()["root"].reshape(-1, 4)
    plan.close()
    for b in range(len(sizes)):
        single = binding.Plan(torch.tensor(pts[b], device=cuda), leaf_size=S, order=p,
                              precision=precision)
        ps, gs = single.eval(torch.tensor(qs[b], device=cuda))
        assert np.array_equal(phi[off[b]:off[b + 1]], ps.cpu().numpy()), b
        assert np.array_equal(g[off[b]:off[b + 1]], gs.cpu().numpy()), b
        assert np.array_equal(roots[b], single.export()["root"])
        single.close()


def test_batch_fp64_matches_oracle_per_problem(cuda):
    sizes, off, xyz, q, pts, qs = concat(6, 300, 4000, seed=7)
    plan = binding.Plan(torch.tensor(xyz, device=cuda), leaf_size=20, order=5, offsets=off)
    phi, g = plan.eval(torch.tensor(q, device=cuda))
    phi, g = phi.cpu().numpy(), g.cpu().numpy()
    for b in range(len(sizes)):
        po, go = oracle.Tree(pts[b], 20).eval(5, qs[b])
        assert rel(phi[off[b]:off[b + 1]], po) <= 1e-12
        assert rel(g[off[b]:off[b + 1]], go) <= 1e-12
    plan.close()


def test_batch_with_empty_and_tiny_problems(cuda):
    rng = workloads.rng(3)
    pts = [rng.random((n, 3)) for n in (0, 1, 5, 0, 300)]
    qs = [rng.uniform(-1, 1, len(x)) for x in pts]
    off = np.concatenate([[0], np.cumsum([len(x) for x in pts])])
    plan = binding.Plan(torch.tensor(np.vstack(pts), device=cuda), leaf_size=4, order=4, offsets=off)
    phi, _ = plan.eval(torch.tensor(np.concatenate(qs), device=cuda))
    phi = phi.cpu().numpy()
    for b, x in enumerate(pts):
        if len(x) == 0:
            continue
        po = oracle.Tree(x, 4).eval(4, qs[b], grad=False)
        np.testing.assert_allclose(phi[off[b]:off[b + 1]], po, rtol=1e-12, atol=1e-14)
    plan.close()


def test_config5_256_problems(cuda):
    """256 problems, N log-uniform in [2048, 65536] (seed 0, problem b seed
    1000+b), p = 6, mixed precision; spot-check members against their own
    single plans (bitwise) and the oracle."""
    sizes, off, xyz, q, pts, qs = concat(256, 2048, 65536, seed=0)
    plan = binding.Plan(torch.tensor(xyz, device=cuda), leaf_size=64, order=6, precision="mixed",
                        offsets=off)
    phi, g = plan.eval(torch.tensor(q, device=cuda))
    phi = phi.cpu().numpy()
    for b in (0, 17, 128, 255):
        single = binding.Plan(torch.tensor(pts[b], device=cuda), leaf_size=64, order=6,
                              precision="mixed")
        ps, _ = single.eval(torch.tensor(qs[b], device=cuda))
        assert np.array_equal(phi[off[b]:off[b + 1]], ps.cpu().numpy())
        single.close()
        pd = oracle.direct(pts[b], qs[b], grad=False)
        assert rel(phi[off[b]:off[b + 1]], pd) <= 1e-3
    plan.close()


def test_graph_replay_equals_eager(cuda):
    """Forward + adjoint captured once and replayed: identical to eager calls."""
    sizes, off, xyz, q, pts, qs = concat(16, 500, 8000, seed=9)
    w = workloads.rng(5).normal(size=len(q))
    X, Q, W = (torch.tensor(a, device=cuda) for a in (xyz, q, w))
    plan = binding.Plan(X, leaf_size=32, order=6, precision="mixed", offsets=off)
    phi_e, g_e = plan.eval(Q)
    dq_e, dx_e = plan.adjoint(W, Q, grad_q=g_e)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        phi, g = torch.empty_like(phi_e), torch.empty_like(g_e)
        dq, dx = torch.empty_like(dq_e), torch.empty_like(dx_e)
        for _ in range(3):
            phi.zero_(), g.zero_(), dq.zero_(), dx.zero_()
            plan.eval_graph(Q, phi, g, W, dq, dx)
            s.synchronize()
            assert torch.equal(phi, phi_e) and torch.equal(g, g_e)
            assert torch.equal(dq, dq_e) and torch.equal(dx, dx_e)
    plan.close()
