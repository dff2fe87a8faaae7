"""GPU FMM mat-vec vs the oracle.

FP64 mode: potentials and each gradient component within 1e-12 relative L2 of
the oracle FMM with the same tree and order.  Both precisions: error against
the direct sum within the stated bars.  Mixed mode: error against the FP64
oracle is stated per case (FP32 arithmetic, floor ~1e-6)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1602_02244_gb300 import binding, workloads

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_gpu(cuda, xyz, q, S, p, precision="fp64", **kw):
    plan = binding.Plan(torch.tensor(xyz, device=cuda), leaf_size=S, order=p,
                        precision=precision, **kw)
    phi, g = plan.eval(torch.tensor(q, device=cuda))
    out = phi.cpu().numpy(), g.cpu().numpy()
    plan.close()
    return out


def problem(kind, n, seed=0):
    if kind == "uniform":
        return workloads.uniform_cube_problem(n, seed)
    if kind == "plummer":
        x, _ = workloads.plummer_problem(n, seed)
        return x, workloads.rng(seed + 50).uniform(-1, 1, n)
    x, q, _ = workloads.sphere_problem(n, seed)
    return x, q


FP64_CASES = [("uniform", 4096, 64, 4), ("uniform", 20000, 32, 8), ("plummer", 30000, 24, 6),
              ("sphere", 20000, 16, 5), ("plummer", 8000, 5, 3), ("uniform", 3000, 40, 10),
              ("plummer", 6000, 30, 12), ("uniform", 500, 16, 0), ("uniform", 700, 20, 1),
              ("plummer", 2000, 10, 16)]


@pytest.mark.parametrize("kind,n,S,p", FP64_CASES)
def test_fp64_matches_oracle_fmm(cuda, kind, n, S, p):
    xyz, q = problem(kind, n)
    phi, g = run_gpu(cuda, xyz, q, S, p)
    t = oracle.Tree(xyz, S)
    po, go = t.eval(p, q)
    assert rel(phi, po) <= 1e-12
    for a in range(3):
        assert rel(g[:, a], go[:, a]) <= 1e-12


def test_fp64_config1_meets_direct_bar(cuda):
    """N = 4096 uniform, p = 4, leaf <= 64: potential and gradient vs the
    full direct sum."""
    xyz, q = workloads.uniform_cube_problem(4096, 0)
    phi, g = run_gpu(cuda, xyz, q, 64, 4)
    pd, gd = oracle.direct(xyz, q)
    assert rel(phi, pd) <= 1e-3
    assert rel(g, gd) <= 1e-2


def test_fp64_config2_1m_p10_vs_direct(cuda):
    """N = 1,048,576 uniform, p = 10, on 4096 sampled targets.  The
    one-box-separation list gives ~2.5e-6 at p = 10 (1e-6 is reached at
    p = 12, pinned on the oracle), so the bar here is 5e-6."""
    xyz, q = workloads.uniform_cube_problem(1048576, 0)
    phi, g = run_gpu(cuda, xyz, q, 64, 10)
    sel = workloads.sample_targets(len(xyz), 4096, 1)
    pd, gd = oracle.direct(xyz, q, xyz[sel])
    assert rel(phi[sel], pd) <= 5e-6
    assert rel(g[sel], gd) <= 5e-5


MIXED_CASES = [("uniform", 20000, 32, 8), ("plummer", 40000, 32, 8), ("sphere", 20000, 24, 6),
               ("plummer", 5000, 6, 4)]


@pytest.mark.parametrize("kind,n,S,p", MIXED_CASES)
def test_mixed_vs_oracle_and_direct(cuda, kind, n, S, p):
    xyz, q = problem(kind, n)
    phi, g = run_gpu(cuda, xyz, q, S, p, precision="mixed")
    t = oracle.Tree(xyz, S)
    po, go = t.eval(p, q)
    pd, gd = oracle.direct(xyz, q)
    e_or, e_dir, e_fmm = rel(phi, po), rel(phi, pd), rel(po, pd)
    print(kind, n, S, p, "mixed vs oracle %.2e, vs direct %.2e (fp64 fmm %.2e)" % (e_or, e_dir, e_fmm))
    assert e_or <= 1e-5
    assert rel(g, go) <= 1e-4
    assert e_dir <= e_fmm + 1e-5


def test_mixed_config3_plummer_4m(cuda):
    """Headline workload: N = 4,194,304 Plummer, charges 1/N, p = 8, mixed;
    error vs the direct sum on 4096 sampled targets."""
    xyz, q = workloads.plummer_problem(4194304, 0)
    phi, g = run_gpu(cuda, xyz, q, 64, 8, precision="mixed")
    sel = workloads.sample_targets(len(xyz), 4096, 1)
    pd, gd = oracle.direct(xyz, q, xyz[sel])
    print("config3 mixed: phi rel %.2e grad rel %.2e" % (rel(phi[sel], pd), rel(g[sel], gd)))
    assert rel(phi[sel], pd) <= 1e-5
    assert rel(g[sel], gd) <= 1e-4


@pytest.mark.parametrize("wx_direct", [False, True])
def test_full_size_in_the_benchmarked_configuration_vs_oracle_fmm(cuda, wx_direct):
    """4,194,304 Plummer points, p = 8, with the leaf size the autotuner picks
    (the configuration the benchmark times, with and without the direct W/X
    leaf pairs): the FP64 mat-vec within 1e-12 of the oracle's FMM on the same
    tree on every target, and the mixed-precision mat-vec within the mixed
    bars of it."""
    xyz, q = workloads.plummer_problem(4194304, 0)
    X, Q = torch.tensor(xyz, device=cuda), torch.tensor(q, device=cuda)
    mixed = binding.Plan(X, leaf_size=0, order=8, precision="mixed", wx_direct=wx_direct)
    S = mixed.sizes()["leaf_size"]
    phi_m, g_m = (a.cpu().numpy() for a in mixed.eval(Q))
    mixed.close()
    f64 = binding.Plan(X, leaf_size=S, order=8, precision="fp64", wx_direct=wx_direct)
    phi_d, g_d = (a.cpu().numpy() for a in f64.eval(Q))
    f64.close()
    po, go = oracle.Tree(xyz, S, direct_wx=81 if wx_direct else 0).eval(8, q)
    print("4M Plummer, leaf %d: fp64 vs oracle %.2e; mixed vs oracle phi %.2e grad %.2e"
          % (S, rel(phi_d, po), rel(phi_m, po), rel(g_m, go)))
    assert rel(phi_d, po) <= 1e-12
    for a in range(3):
        assert rel(g_d[:, a], go[:, a]) <= 1e-12
    assert rel(phi_m, po) <= 1e-5 and rel(g_m, go) <= 1e-4


@pytest.mark.parametrize("tile", [1, 2, 3, 4])
@pytest.mark.parametrize("c", [2, 5, 16, 17, 31, 32, 33, 63, 64, 65, 127, 128, 129, 300, 449, 1000])
def test_mixed_near_field_of_one_leaf_is_the_direct_sum(cuda, c, tile):
    """A root that is a leaf: the mat-vec is the FP32 near-field kernel alone,
    in each of its staging shapes (192-448 points per buffer).  The counts
    straddle the lane-group thresholds (a leaf of <= 16, 32, 64 targets splits
    its sources over 8, 4, 2 groups of lanes), several target tiles (> 128)
    and a leaf larger than one staged batch (it is staged in parts).  Four
    coincident points contribute nothing to one another."""
    xyz = workloads.rng(c).uniform(0.0, 1.0, (c, 3))
    xyz[-3:] = xyz[0] if c >= 4 else xyz[-3:]
    q = workloads.rng(c + 1).uniform(-1, 1, c)
    plan = binding.Plan(torch.tensor(xyz, device=cuda), leaf_size=c, order=4, precision="mixed",
                        p2p_tile=tile)
    assert plan.sizes()["nboxes"] == 1
    phi, g = plan.eval(torch.tensor(q, device=cuda))
    phi, g = phi.cpu().numpy(), g.cpu().numpy()
    plan.close()
    pd, gd = oracle.direct(xyz, q)
    assert rel(phi, pd) <= 1e-5 and rel(g, gd) <= 1e-4


@pytest.mark.parametrize("tile", [1, 2, 3, 4])
def test_p2p_staging_shapes_match_oracle(cuda, tile):
    """Every staging shape of the FP32 near field on an adaptive Plummer
    tree (leaves of 1..48 points, U lists of every length): the mat-vec
    within the mixed bars of the FP64 oracle FMM, and the shapes within FP32
    rounding of one another (they differ only in where batch sums start)."""
    xyz, q = problem("plummer", 40000)
    phi, g = run_gpu(cuda, xyz, q, 48, 6, precision="mixed", p2p_tile=tile)
    ref_phi, ref_g = run_gpu(cuda, xyz, q, 48, 6, precision="mixed", p2p_tile=1)
    po, go = oracle.Tree(xyz, 48).eval(6, q)
    assert rel(phi, po) <= 1e-5 and rel(g, go) <= 1e-4
    assert rel(phi, ref_phi) <= 1e-6 and rel(g, ref_g) <= 1e-5


def test_coincident_points_and_single_point(cuda):
    xyz = np.vstack([np.tile([[0.5, 0.5, 0.5]], (40, 1)), workloads.uniform_cube(200, 4)])
    q = workloads.rng(9).uniform(-1, 1, len(xyz))
    phi, g = run_gpu(cuda, xyz, q, 8, 6)
    po, go = oracle.Tree(xyz, 8).eval(6, q)
    assert rel(phi, po) <= 1e-12 and rel(g, go) <= 1e-12
    phi1, g1 = run_gpu(cuda, np.array([[1.0, 2.0, 3.0]]), np.array([5.0]), 8, 4)
    assert phi1[0] == 0.0 and np.all(g1 == 0.0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_host_entry_point_matches_device_path(cuda, precision):
    """fmm_solve_host equals the device path, call after call on new points."""
    plan = None
    for seed, (n, gen) in enumerate([(30000, workloads.uniform_cube_problem), (50000, workloads.uniform_cube_problem),
                                     (20000, lambda n, s: (workloads.plummer_problem(n, s)[0],
                                                           workloads.rng(s).uniform(-1, 1, n)))]):
        xyz, q = gen(n, seed + 5)
        dev = binding.Plan(torch.tensor(xyz, device=cuda), leaf_size=32, order=6, precision=precision)
        phi_d, g_d = dev.eval(torch.tensor(q, device=cuda))
        dev.close()
        if plan is None:
            plan = binding.Plan(torch.tensor(xyz, device=cuda), leaf_size=32, order=6, precision=precision)
        phi_h, g_h = plan.solve_host(xyz, q)
        assert np.array_equal(phi_h, phi_d.cpu().numpy())
        assert np.array_equal(g_h, g_d.cpu().numpy())
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_host_forward_adjoint_entry_point_matches_device_path(cuda, precision):
    """fmm_solve_adjoint_host (copies in, rebuild, forward, adjoint with the
    stored forward gradient, copies out) equals the device calls bit for bit."""
    xyz, q = problem("plummer", 30000, 3)
    w = workloads.rng(4).normal(size=len(q))
    X, Q, W = (torch.tensor(a, device=cuda) for a in (xyz, q, w))
    dev = binding.Plan(X, leaf_size=32, order=6, precision=precision)
    phi_d, g_d = dev.eval(Q)
    dq_d, dx_d = dev.adjoint(W, Q, grad_q=g_d)
    dev.close()
    plan = binding.Plan(torch.tensor(workloads.uniform_cube(1000, 1), device=cuda), leaf_size=32,
                        order=6, precision=precision)
    n = len(q)
    out = [np.empty(n), np.empty((n, 3)), np.empty(n), np.empty((n, 3))]
    xyz_c, q_c, w_c = (np.ascontiguousarray(a) for a in (xyz, q, w))
    plan.solve_adjoint_host_ptr(xyz_c.ctypes.data, q_c.ctypes.data, w_c.ctypes.data, n,
                                *(a.ctypes.data for a in out))
    plan.close()
    for a, b in zip(out, (phi_d, g_d, dq_d, dx_d)):
        assert np.array_equal(a, b.cpu().numpy())


@pytest.mark.parametrize("side", [16, 64])
def test_lattice_fp64_matches_oracle_fmm(cuda, side):
    """The paper's uniform-lattice workload (§4.1), leaf 64, p = 8, unit
    charges as in the benchmark's lattice leg: FP64 within 1e-12 of the oracle
    FMM on the same tree, and the mixed path within its bars."""
    xyz = workloads.lattice(side)
    q = np.ones(len(xyz))
    po, go = oracle.Tree(xyz, 64).eval(8, q)
    phi, g = run_gpu(cuda, xyz, q, 64, 8)
    assert rel(phi, po) <= 1e-12
    for a in range(3):
        assert rel(g[:, a], go[:, a]) <= 1e-12
    phi_m, g_m = run_gpu(cuda, xyz, q, 64, 8, precision="mixed")
    assert rel(phi_m, po) <= 1e-5 and rel(g_m, go) <= 1e-4


def test_fp32_peak_probe(cuda):
    """fmm_fp32_peak measures a rate between half and 1.05x the nominal FP32
    peak of the device (SMs x 128 lanes x 2 flop x the highest SM clock)."""
    v = binding.fp32_peak()
    props = torch.cuda.get_device_properties(cuda)
    nominal = props.multi_processor_count * 128 * 2 * 2.1e9 / 1e12
    print("measured FP32 peak %.1f TFLOP/s (nominal at 2.1 GHz %.1f)" % (v, nominal))
    assert 0.5 * nominal <= v <= 1.05 * nominal


def test_rebuild_reuses_plan(cuda):
    xyz1, q1 = workloads.uniform_cube_problem(10000, 1)
    xyz2, q2 = workloads.plummer_problem(15000, 2)
    plan = binding.Plan(torch.tensor(xyz1, device=cuda), leaf_size=16, order=5)
    plan.rebuild(torch.tensor(xyz2, device=cuda))
    phi, g = plan.eval(torch.tensor(q2, device=cuda))
    po, go = oracle.Tree(xyz2, 16).eval(5, q2)
    assert rel(phi.cpu().numpy(), po) <= 1e-12
    plan.close()


@pytest.mark.parametrize("kind,n,S,p", [("plummer", 40000, 32, 8), ("uniform", 30000, 24, 10),
                                       ("sphere", 20000, 16, 6), ("plummer", 8000, 8, 5),
                                       ("uniform", 6000, 12, 9), ("plummer", 5000, 6, 3),
                                       ("uniform", 3000, 20, 4)])
@pytest.mark.parametrize("form", [1, 2])
def test_tensor_core_m2l_matches_cuda_core_path(cuda, kind, n, S, p, form):
    """Mixed precision with M2L on the tensor cores (tcgen05; form 1: the
    three-product TF32 split, form 2: the FP16 split with power-of-two
    scalings) against the same plan with M2L on FP32 CUDA cores, and against
    the FP64 oracle."""
    xyz, q = problem(kind, n)
    X, Q = torch.tensor(xyz, device=cuda), torch.tensor(q, device=cuda)
    out = {}
    for path in ("simt", "tensor"):
        plan = binding.Plan(X, leaf_size=S, order=p, precision="mixed", m2l_path=path,
                            m2l_tile=form)
        phi, g = plan.eval(Q)
        plan.sync()
        out[path] = phi.cpu().numpy(), g.cpu().numpy()
        plan.close()
    po, go = oracle.Tree(xyz, S).eval(p, q)
    e_paths = rel(out["tensor"][0], out["simt"][0])
    e_or = rel(out["tensor"][0], po)
    print(kind, n, S, p, form, "tensor vs cuda-core %.2e, tensor vs oracle %.2e (cuda-core %.2e)"
          % (e_paths, e_or, rel(out["simt"][0], po)))
    assert e_paths <= 3e-6
    assert rel(out["tensor"][1], out["simt"][1]) <= 3e-5
    assert e_or <= 1e-5


ROT_CASES = [("uniform", 20000, 32, 8), ("plummer", 30000, 24, 6), ("plummer", 6000, 30, 12),
             ("uniform", 3000, 40, 10), ("sphere", 8000, 16, 4), ("uniform", 500, 16, 0),
             ("plummer", 2000, 10, 1)]


@pytest.mark.parametrize("kind,n,S,p", ROT_CASES)
def test_rotated_m2l_fp64_matches_oracle(cuda, kind, n, S, p):
    """The rotated operators (rotate onto the offset axis, translate along z,
    rotate back) are an exact factorisation of the dense M2L: FP64 parity
    with the oracle's dense translation at the same bar."""
    xyz, q = problem(kind, n)
    phi, g = run_gpu(cuda, xyz, q, S, p, m2l_path="rotation")
    po, go = oracle.Tree(xyz, S).eval(p, q)
    assert rel(phi, po) <= 1e-12
    for a in range(3):
        assert rel(g[:, a], go[:, a]) <= 1e-12


@pytest.mark.parametrize("kind,n,S,p", [("plummer", 30000, 32, 12), ("uniform", 20000, 32, 8)])
def test_rotated_m2l_mixed_vs_oracle(cuda, kind, n, S, p):
    xyz, q = problem(kind, n)
    phi, g = run_gpu(cuda, xyz, q, S, p, precision="mixed", m2l_path="rotation")
    po, go = oracle.Tree(xyz, S).eval(p, q)
    assert rel(phi, po) <= 1e-5
    assert rel(g, go) <= 1e-4


def test_autotuner_picks_kernel_shapes(cuda):
    """leaf_size 0 on a mixed plan: the autotuner also chooses the FP32
    near-field staging shape and the tensor-core M2L operand form (reported
    by fmm_plan_tiles and kept by a rebuild); explicit options stand."""
    xyz, q = problem("plummer", 60000, 7)
    X, Q = torch.tensor(xyz, device=cuda), torch.tensor(q, device=cuda)
    plan = binding.Plan(X, leaf_size=0, order=6, precision="mixed")
    t = plan.tiles()
    assert 1 <= t["p2p_tile"] <= 4 and t["m2l_tile"] in (1, 2)
    S = plan.sizes()["leaf_size"]
    phi, g = plan.eval(Q)
    plan.rebuild(X)
    assert plan.tiles() == t and plan.sizes()["leaf_size"] == S
    plan.close()
    po, go = oracle.Tree(xyz, S).eval(6, q)
    assert rel(phi.cpu().numpy(), po) <= 1e-5 and rel(g.cpu().numpy(), go) <= 1e-4
    fixed = binding.Plan(X, leaf_size=0, order=6, precision="mixed", p2p_tile=3, m2l_tile=1)
    assert fixed.tiles() == {"p2p_tile": 3, "m2l_tile": 1}
    fixed.close()


@pytest.mark.parametrize("kind,n,S,p", [("plummer", 30000, 24, 6), ("sphere", 20000, 16, 8),
                                         ("plummer", 8000, 5, 3)])
def test_direct_wx_matches_oracle_fmm(cuda, kind, n, S, p):
    """W/X pairs of small leaves by the direct sum (fmm_opts.wx_direct):
    FP64 within 1e-12 of the oracle FMM with the same lists, mixed within the
    mixed bars; the mat-vec stays symmetric (the adjoint's dL/dq is the
    forward with the weights)."""
    xyz, q = problem(kind, n)
    t = oracle.Tree(xyz, S, direct_wx=(p + 1) ** 2)
    assert len(t.w_idx) < len(oracle.Tree(xyz, S).w_idx)
    po, go = t.eval(p, q)
    phi, g = run_gpu(cuda, xyz, q, S, p, wx_direct=True)
    assert rel(phi, po) <= 1e-12
    for a in range(3):
        assert rel(g[:, a], go[:, a]) <= 1e-12
    phi_m, g_m = run_gpu(cuda, xyz, q, S, p, precision="mixed", wx_direct=True)
    assert rel(phi_m, po) <= 1e-5 and rel(g_m, go) <= 1e-4
    w = workloads.rng(9).uniform(-1, 1, n)
    plan = binding.Plan(torch.tensor(xyz, device=cuda), leaf_size=S, order=p, wx_direct=True)
    dq, _ = plan.adjoint(torch.tensor(w, device=cuda), torch.tensor(q, device=cuda))
    fw, _ = plan.eval(torch.tensor(w, device=cuda))
    plan.close()
    assert rel(dq.cpu().numpy(), fw.cpu().numpy()) <= 1e-13
