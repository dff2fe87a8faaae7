"""GPU Helmholtz FMM (kernel e^{i kappa r}/r, FP64 complex) vs the oracle.

The GPU tree and lists equal the oracle's byte for byte, so the GPU mat-vec
must equal the oracle FMM of the same order on the same tree to rounding:
1e-12 relative L2 (the FP64 bar of the Laplace path).  Against the direct sum
the error is the method's truncation error, falling with the order."""
import numpy as np
import pytest
import torch

import oracle
from paper_1602_02244_gb300 import binding, workloads

pytestmark = pytest.mark.gpu

KAPPA = 7.0  # §4.2: Helmholtz with kappa = 7 on [-1, 1]^3


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def charges(n, seed):
    g = workloads.rng(seed)
    return g.uniform(-1, 1, n) + 1j * g.uniform(-1, 1, n)


def points(kind, n, seed=0):
    if kind == "cube":  # [-1, 1]^3
        return workloads.uniform_cube(n, seed) * 2.0 - 1.0
    if kind == "plummer":  # adaptive: W and X lists; scaled to a cube of side ~2
        return workloads.plummer(n, seed) / 10.0
    side = round(n ** (1.0 / 3.0))
    return workloads.lattice(side) * 2.0 - 1.0


def gpu_helmholtz(cuda, xyz, q, S, p, kappa=KAPPA, precision="fp64"):
    plan = binding.Plan(torch.tensor(xyz, device=cuda), leaf_size=S, order=4, precision=precision)
    phi = plan.helmholtz(torch.tensor(q, device=cuda), kappa, p)
    out = phi.cpu().numpy()
    plan.close()
    return out


CASES = [("cube", 2000, 32, 0), ("cube", 2000, 32, 3), ("cube", 3000, 24, 8),
         ("cube", 1500, 40, 12), ("plummer", 2500, 16, 6), ("plummer", 4000, 12, 9),
         ("lattice", 4096, 64, 5), ("lattice", 4096, 8, 7)]


@pytest.mark.parametrize("kind,n,S,p", CASES)
def test_matches_oracle_fmm(cuda, kind, n, S, p):
    xyz = points(kind, n)
    q = charges(n, 3)
    phi = gpu_helmholtz(cuda, xyz, q, S, p)
    t = oracle.Tree(xyz, S)
    if kind == "plummer":
        assert len(t.w_idx) > 0 and len(t.x_idx) > 0
    ref = t.helmholtz_eval(p, KAPPA, q)
    assert rel(phi, ref) <= 1e-12


@pytest.mark.parametrize("kind,n,S,p", [("cube", 3000, 24, 8), ("plummer", 4000, 12, 6),
                                         ("lattice", 4096, 64, 4), ("plummer", 6000, 8, 10),
                                         ("cube", 2000, 32, 12)])
def test_mixed_matches_oracle_fmm(cuda, kind, n, S, p):
    """Mixed plans: M2L (scaled per level) and the near field in FP32, the
    other passes in FP64: within 1e-5 of the oracle (measured 0.5-2.4e-6)."""
    xyz = points(kind, n)
    q = charges(n, 4)
    phi = gpu_helmholtz(cuda, xyz, q, S, p, precision="mixed")
    assert rel(phi, oracle.Tree(xyz, S).helmholtz_eval(p, KAPPA, q)) <= 1e-5


@pytest.mark.parametrize("kappa", [0.5, 7.0])
def test_mixed_on_a_deep_tree_stays_finite_and_close_to_fp64(cuda, kappa):
    """A 20,000-point Plummer sphere at leaf 4 (10 levels): at kappa = 0.5 the
    unscaled h_12(kappa |t|) of its finest level (~6e42) is beyond the FP32
    range; the scaled FP32 M2L stays finite and close to FP64."""
    xyz = workloads.plummer(20000, 3) / 10.0
    q = charges(20000, 5)
    mix = gpu_helmholtz(cuda, xyz, q, 4, 6, kappa, precision="mixed")
    f64 = gpu_helmholtz(cuda, xyz, q, 4, 6, kappa)
    assert np.isfinite(mix).all() and rel(mix, f64) <= 1e-5


def test_converges_to_the_direct_sum(cuda):
    xyz = points("cube", 3000, seed=4)
    q = charges(3000, 5)
    ref = oracle.h_direct(xyz, q, KAPPA)
    errs = [rel(gpu_helmholtz(cuda, xyz, q, 24, p), ref) for p in (4, 8, 12)]
    assert errs[2] < 1e-6 and errs[0] > errs[1] > errs[2], errs


@pytest.mark.parametrize("kappa", [0.5, 3.0, 12.0])
def test_other_wave_numbers_match_oracle(cuda, kappa):
    xyz = points("cube", 2000, seed=6)
    q = charges(2000, 7)
    phi = gpu_helmholtz(cuda, xyz, q, 32, 6, kappa)
    assert rel(phi, oracle.Tree(xyz, 32).helmholtz_eval(6, kappa, q)) <= 1e-12


def test_single_leaf_is_the_direct_sum_and_coincident_points_are_skipped(cuda):
    rng = np.random.default_rng(8)
    xyz = rng.uniform(-1, 1, size=(50, 3))
    xyz[7] = xyz[3]  # a coincident pair: excluded like the self term
    q = charges(50, 9)
    phi = gpu_helmholtz(cuda, xyz, q, 64, 6)
    ref = oracle.h_direct(xyz, q, KAPPA)
    assert rel(phi, ref) <= 1e-14
    one = gpu_helmholtz(cuda, xyz[:1], q[:1], 8, 4)
    assert one[0] == 0


def test_preconditioner_grid_sampled_against_the_direct_sum(cuda):
    """The h = 2^-5 interior grid of [-1, 1]^3 (63^3 = 250,047 points) at
    order 8: sampled targets against the oracle's direct sum."""
    m = 63
    g = -1.0 + (np.arange(m) + 1) / 32.0
    xyz = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    q = charges(len(xyz), 10)
    phi = gpu_helmholtz(cuda, xyz, q, 64, 8)
    idx = workloads.sample_targets(len(xyz), 256, seed=2)
    ref = oracle.h_direct(xyz, q, KAPPA, xyz[idx])
    assert rel(phi[idx], ref) <= 1e-4  # order 8: the truncation error is ~3e-5


def test_direct_wx_plan_matches_oracle_with_the_same_lists(cuda):
    """A plan whose small W/X leaf pairs sit in the U lists (fmm_opts.wx_direct):
    the Helmholtz mat-vec follows its lists, like the oracle with the same rule."""
    xyz = points("plummer", 4000)
    q = charges(4000, 6)
    plan = binding.Plan(torch.tensor(xyz, device=cuda), leaf_size=12, order=5, wx_direct=True)
    phi = plan.helmholtz(torch.tensor(q, device=cuda), KAPPA, 6).cpu().numpy()
    plan.close()
    t = oracle.Tree(xyz, 12, direct_wx=36)
    assert len(t.w_idx) < len(oracle.Tree(xyz, 12).w_idx)
    assert rel(phi, t.helmholtz_eval(6, KAPPA, q)) <= 1e-12


def test_invalid_arguments(cuda):
    xyz = points("cube", 500)
    plan = binding.Plan(torch.tensor(xyz, device=cuda), leaf_size=32, order=4)
    q = torch.tensor(charges(500, 1), device=cuda)
    for kappa, p in ((KAPPA, 13), (KAPPA, -1), (0.0, 4), (-1.0, 4), (float("nan"), 4)):
        with pytest.raises(binding.FMMError) as e:
            plan.helmholtz(q, kappa, p)
        assert e.value.status == 1
    plan.close()
    dual = binding.Plan(torch.tensor(xyz, device=cuda), leaf_size=32, order=4,
                        interaction="dual")
    with pytest.raises(binding.FMMError) as e:
        dual.helmholtz(q, KAPPA, 4)
    assert e.value.status == 1
    dual.close()
    batch = binding.Plan(torch.tensor(xyz, device=cuda), leaf_size=32, order=4,
                         offsets=[0, 200, 500])
    with pytest.raises(binding.FMMError) as e:
        batch.helmholtz(q, KAPPA, 4)
    assert e.value.status == 1
    batch.close()
