"""Dual-tree walk on the GPU vs the oracle (§2.1: Dehnen's dual tree walk
with a multipole acceptance criterion as the alternative to fixed lists).

Lists and cell radii byte for byte (the acceptance decisions are IEEE
operations in a fixed order on both sides); the FP64 mat-vec within 1e-12
of the oracle's FMM on the same lists; mixed precision against the FP64
oracle; theta = 0 is the direct sum; the adjoint; batches; graph replay."""
import numpy as np
import pytest
import torch

import oracle
from paper_1602_02244_gb300 import binding, workloads

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def problem(kind, n, seed=0):
    if kind == "uniform":
        return workloads.uniform_cube_problem(n, seed)
    if kind == "plummer":
        x, _ = workloads.plummer_problem(n, seed)
        return x, workloads.rng(seed + 50).uniform(-1, 1, n)
    x, q, _ = workloads.sphere_problem(n, seed)
    return x, q


def dual_plan(cuda, xyz, S, p, theta, precision="fp64", **kw):
    return binding.Plan(torch.tensor(xyz, device=cuda), leaf_size=S, order=p, precision=precision,
                        interaction="dual", theta=theta, **kw)


def compare_lists(plan, tree, dual):
    g = plan.export()
    t = tree.arrays()
    for f in ("keys", "perm", "level_offset", "box_key", "box_level", "box_first", "box_count",
              "box_parent", "box_child", "box_nchild"):
        assert np.array_equal(g[f], t[f]), f
    assert np.array_equal(g["u_off"], dual.p2p_off)
    assert np.array_equal(g["u_idx"], dual.p2p_idx)
    assert np.array_equal(g["v_off"], dual.m2l_off)
    assert np.array_equal(g["v_idx"], dual.m2l_idx)
    assert len(g["w_idx"]) == 0 and len(g["x_idx"]) == 0
    assert np.array_equal(g["radius"], dual.radius)


LIST_CASES = [("plummer", 20000, 16, 0.5), ("plummer", 50000, 64, 0.7), ("uniform", 30000, 32, 0.5),
              ("sphere", 20000, 24, 0.6), ("plummer", 3000, 2, 0.3), ("uniform", 900, 1, 0.9)]


@pytest.mark.parametrize("kind,n,S,theta", LIST_CASES)
def test_lists_and_radii_bit_exact(cuda, kind, n, S, theta):
    xyz, _ = problem(kind, n)
    plan = dual_plan(cuda, xyz, S, 4, theta)
    t = oracle.Tree(xyz, S)
    compare_lists(plan, t, oracle.Dual(t, theta))
    plan.close()


FP64_CASES = [("plummer", 20000, 24, 6, 0.5), ("uniform", 10000, 32, 8, 0.6),
              ("sphere", 8000, 16, 4, 0.4), ("plummer", 4000, 8, 10, 0.7), ("plummer", 3000, 20, 0, 0.5),
              ("uniform", 2000, 30, 14, 0.5)]


@pytest.mark.parametrize("kind,n,S,p,theta", FP64_CASES)
def test_fp64_matches_oracle_dual_fmm(cuda, kind, n, S, p, theta):
    xyz, q = problem(kind, n)
    plan = dual_plan(cuda, xyz, S, p, theta)
    phi, g = plan.eval(torch.tensor(q, device=cuda))
    phi, g = phi.cpu().numpy(), g.cpu().numpy()
    plan.close()
    t = oracle.Tree(xyz, S)
    po, go = oracle.Dual(t, theta).eval(p, q)
    assert rel(phi, po) <= 1e-12
    for a in range(3):
        assert rel(g[:, a], go[:, a]) <= 1e-12


@pytest.mark.parametrize("kind,n,S,p,theta", [("plummer", 40000, 32, 8, 0.5), ("uniform", 20000, 32, 6, 0.6),
                                              ("plummer", 20000, 64, 4, 0.7)])
def test_mixed_vs_fp64_oracle(cuda, kind, n, S, p, theta):
    xyz, q = problem(kind, n)
    plan = dual_plan(cuda, xyz, S, p, theta, precision="mixed")
    phi, g = plan.eval(torch.tensor(q, device=cuda))
    phi, g = phi.cpu().numpy(), g.cpu().numpy()
    plan.close()
    po, go = oracle.Dual(oracle.Tree(xyz, S), theta).eval(p, q)
    # FP32 arithmetic; the pairs inside the fixed-offset tiles run on the
    # tensor cores (three-product TF32 split), the rest on the CUDA cores
    assert rel(phi, po) <= 5e-6
    assert rel(g, go) <= 5e-5


def test_tiny_theta_is_the_direct_sum(cuda):
    """8^3 clusters of 8 points: every leaf holds one cluster (radius > 0), so
    a tiny theta accepts nothing and the mat-vec is P2P over all leaf pairs."""
    g = (np.arange(8) + 0.5) / 8
    c = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    o = 0.01 * np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], float)
    xyz = (c[:, None, :] + o[None, :, :]).reshape(-1, 3)
    q = workloads.rng(3).uniform(-1, 1, len(xyz))
    X, Q = torch.tensor(xyz, device=cuda), torch.tensor(q, device=cuda)
    plan = dual_plan(cuda, xyz, 8, 4, 1e-300)
    assert plan.sizes()["nv"] == 0 and plan.sizes()["nu"] == 512 * 512
    phi, gr = plan.eval(Q)
    pd, gd = binding.direct(X, Q, X)
    assert rel(phi.cpu().numpy(), pd.cpu().numpy()) <= 1e-14
    assert rel(gr.cpu().numpy(), gd.cpu().numpy()) <= 1e-14
    plan.close()


def test_adjoint_is_the_forward_with_the_weights(cuda):
    xyz, q = problem("plummer", 12000, 4)
    w = workloads.rng(9).normal(size=len(q))
    plan = dual_plan(cuda, xyz, 16, 6, 0.5)
    Q, W = torch.tensor(q, device=cuda), torch.tensor(w, device=cuda)
    dq, dx = plan.adjoint(W, Q)
    dq, dx = dq.cpu().numpy(), dx.cpu().numpy()
    plan.close()
    d = oracle.Dual(oracle.Tree(xyz, 16), 0.5)
    pq, gq = d.eval(6, q)
    pw, gw = d.eval(6, w)
    assert rel(dq, pw) <= 1e-12
    assert rel(dx, w[:, None] * gq + q[:, None] * gw) <= 1e-12


def test_batch_members_equal_their_single_runs(cuda):
    parts = [problem("plummer", 3000, 20)[0], problem("uniform", 5000, 21)[0], problem("sphere", 2000, 22)[0]]
    xyz = np.vstack(parts)
    q = workloads.rng(23).uniform(-1, 1, len(xyz))
    off = np.cumsum([0] + [len(p) for p in parts]).tolist()
    plan = binding.Plan(torch.tensor(xyz, device=cuda), leaf_size=16, order=6, precision="mixed",
                        offsets=off, interaction="dual", theta=0.5)
    phi, g = plan.eval(torch.tensor(q, device=cuda))
    phi, g = phi.cpu().numpy(), g.cpu().numpy()
    plan.close()
    for b, xp in enumerate(parts):
        sl = slice(off[b], off[b + 1])
        one = dual_plan(cuda, xp, 16, 6, 0.5, precision="mixed")
        p1, g1 = one.eval(torch.tensor(q[sl], device=cuda))
        one.close()
        assert np.array_equal(phi[sl], p1.cpu().numpy())
        assert np.array_equal(g[sl], g1.cpu().numpy())


def test_graph_replay_equals_eager(cuda):
    xyz, q = problem("plummer", 30000, 5)
    plan = dual_plan(cuda, xyz, 32, 8, 0.5, precision="mixed")
    Q = torch.tensor(q, device=cuda)
    phi, g = plan.eval(Q)
    s = torch.cuda.Stream()
    phi2 = torch.empty_like(phi)
    g2 = torch.empty_like(g)
    s.wait_stream(torch.cuda.current_stream())  # the plan's workspace is shared
    with torch.cuda.stream(s):
        plan.eval_graph(Q, phi2, g2, stream=s)
        plan.eval_graph(Q, phi2, g2, stream=s)
    s.synchronize()
    assert torch.equal(phi, phi2) and torch.equal(g, g2)
    plan.close()


def test_edge_cases(cuda):
    # one point, two coincident points, all coincident (a leaf at max depth)
    for xyz in (np.array([[0.3, 0.2, 0.1]]), np.array([[0.5, 0.5, 0.5], [0.5, 0.5, 0.5]]),
                np.tile([[0.1, 0.2, 0.3]], (40, 1))):
        q = np.arange(1.0, len(xyz) + 1.0)
        plan = dual_plan(cuda, xyz, 4, 4, 0.5)
        phi, g = plan.eval(torch.tensor(q, device=cuda))
        assert np.all(phi.cpu().numpy() == 0.0) and np.all(g.cpu().numpy() == 0.0)
        t = oracle.Tree(xyz, 4)
        compare_lists(plan, t, oracle.Dual(t, 0.5))
        plan.close()
    plan = dual_plan(cuda, np.zeros((0, 3)), 4, 4, 0.5)
    plan.close()
    for bad in (1.0, -0.5, float("nan")):
        with pytest.raises(binding.FMMError):
            dual_plan(cuda, workloads.uniform_cube(100, 0), 8, 4, bad)


def test_plummer_1m_mixed_vs_direct(cuda):
    """A larger adaptive case, charges of both signs: sampled targets against
    the direct sum, and the error ordered by theta (truncation well above the
    FP32 floor at the larger theta)."""
    xyz, _ = workloads.plummer_problem(1 << 20, 0)
    q = workloads.rng(8).uniform(-1, 1, len(xyz))
    X, Q = torch.tensor(xyz, device=cuda), torch.tensor(q, device=cuda)
    sel = workloads.sample_targets(len(xyz), 4096, 1)
    pd, gd = oracle.direct(xyz, q, xyz[sel])
    errs = []
    for theta in (0.4, 0.75):
        plan = binding.Plan(X, leaf_size=64, order=8, precision="mixed", interaction="dual", theta=theta)
        phi, g = plan.eval(Q)
        errs.append((rel(phi.cpu().numpy()[sel], pd), rel(g.cpu().numpy()[sel], gd)))
        plan.close()
    print("dual-tree 1M Plummer p=8 mixed: theta 0.4 / 0.75 errors", errs)
    assert errs[0][0] < 1e-5 and errs[0][1] < 1e-4
    assert errs[1][0] < 1e-3 and errs[1][1] < 1e-2
    assert errs[0][0] < errs[1][0] and errs[0][1] < errs[1][1]
