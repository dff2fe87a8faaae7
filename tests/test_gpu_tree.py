"""GPU hierarchy vs the oracle, byte for byte: root cube, Morton keys, stable
permutation, boxes numbered by (level, key), and the U/V/W/X lists (§2.2
interaction list, adaptive lists), on every input distribution, edge cases,
and the full 4M-point Plummer problem."""
import numpy as np
import pytest
import torch

import oracle
from paper_1602_02244_gb300 import binding, workloads

pytestmark = pytest.mark.gpu


def gpu_plan(cuda, xyz, S, max_depth=0, order=4):
    return binding.Plan(torch.tensor(xyz, device=cuda), leaf_size=S, order=order,
                        max_depth=max_depth)


def compare(plan, tree):
    g = plan.export()
    o = tree.arrays()
    for f in oracle.Tree.FIELDS:
        a, b = g[f], o[f]
        assert a.dtype == b.dtype and a.shape == b.shape, (f, a.shape, b.shape)
        assert np.array_equal(a, b), (f, np.nonzero(a != b)[0][:10])
    assert tuple(g["root"][:3]) == tuple(tree.lo) and g["root"][3] == tree.D


CASES = [
    ("uniform", 4096, 64), ("uniform", 65536, 32), ("plummer", 20000, 16), ("plummer", 50000, 64),
    ("sphere", 30000, 24), ("uniform", 777, 1), ("plummer", 5000, 3),
]


def points(kind, n, seed=0):
    return {"uniform": workloads.uniform_cube, "plummer": workloads.plummer,
            "sphere": workloads.sphere_surface}[kind](n, seed)


@pytest.mark.parametrize("kind,n,S", CASES)
def test_tree_and_lists_bit_exact(cuda, kind, n, S):
    xyz = points(kind, n)
    plan = gpu_plan(cuda, xyz, S)
    compare(plan, oracle.Tree(xyz, S))
    plan.close()


def test_edge_cases_bit_exact(cuda):
    # single point, N == S, all-coincident points (leaf at max depth),
    # clustered duplicates, reduced max depth
    one = np.array([[0.25, -1.0, 3.0]])
    same = np.tile([[0.1, 0.2, 0.3]], (50, 1))
    dup = np.vstack([same, workloads.uniform_cube(300, 3)])
    for xyz, S, md in ((one, 8, 0), (workloads.uniform_cube(64, 1), 64, 0), (same, 4, 0),
                       (dup, 4, 0), (workloads.plummer(3000, 2), 4, 6)):
        plan = gpu_plan(cuda, xyz, S, md)
        compare(plan, oracle.Tree(xyz, S, md if md else 21))
        plan.close()


def test_empty_plan(cuda):
    plan = binding.Plan(torch.zeros(0, 3, dtype=torch.float64, device=cuda), leaf_size=8, order=4)
    assert plan.sizes()["nboxes"] == 0
    phi, g = plan.eval(torch.zeros(0, dtype=torch.float64, device=cuda))
    assert phi.numel() == 0
    plan.close()


def test_nonfinite_rejected(cuda):
    xyz = workloads.uniform_cube(100, 0)
    xyz[17, 1] = np.nan
    with pytest.raises(binding.FMMError) as e:
        gpu_plan(cuda, xyz, 8)
    assert e.value.status == 5


def test_full_size_plummer_4m_bit_exact(cuda):
    """The benchmark's hierarchy: N = 4,194,304 Plummer points, leaf size 64."""
    xyz = workloads.plummer(4194304, 0)
    plan = gpu_plan(cuda, xyz, 64, order=8)
    compare(plan, oracle.Tree(xyz, 64))
    plan.close()


def test_lists_of_a_mixed_plan_built_on_request(cuda):
    """A mixed-precision plan of order <= 10 builds its M2L source table from
    the colleagues and its V lists only when asked; both must equal the
    oracle's."""
    xyz = points("plummer", 30000)
    plan = binding.Plan(torch.tensor(xyz, device=cuda), leaf_size=24, order=8, precision="mixed")
    compare(plan, oracle.Tree(xyz, 24))
    plan.close()


@pytest.mark.parametrize("side", [16, 64])
def test_lattice_bit_exact(cuda, side):
    """The paper's own workload (§4.1): a uniform lattice, leaf size 64.  Its
    points sit exactly on dyadic box boundaries relative to the root cube's
    corner, the edge case of the quantisation."""
    xyz = workloads.lattice(side)
    plan = gpu_plan(cuda, xyz, 64, order=8)
    compare(plan, oracle.Tree(xyz, 64))
    plan.close()


@pytest.mark.parametrize("kind,n,S,p,precision", [("plummer", 20000, 16, 8, "fp64"),
                                                  ("sphere", 30000, 24, 4, "mixed"),
                                                  ("plummer", 5000, 3, 6, "mixed"),
                                                  ("uniform", 4096, 64, 2, "fp64")])
def test_direct_wx_lists_bit_exact(cuda, kind, n, S, p, precision):
    """fmm_opts.wx_direct: W/X pairs of two leaves whose W leaf holds at most
    (p+1)^2 points move to both leaves' U lists -- equal to the oracle's lists
    with the same rule."""
    xyz = points(kind, n)
    plan = binding.Plan(torch.tensor(xyz, device=cuda), leaf_size=S, order=p,
                        precision=precision, wx_direct=True)
    compare(plan, oracle.Tree(xyz, S, direct_wx=(p + 1) ** 2))
    plan.close()


def test_direct_wx_full_size_plummer_4m_bit_exact(cuda):
    xyz = workloads.plummer(4194304, 0)
    plan = binding.Plan(torch.tensor(xyz, device=cuda), leaf_size=128, order=8,
                        precision="mixed", wx_direct=True)
    compare(plan, oracle.Tree(xyz, 128, direct_wx=81))
    plan.close()
