"""fmm_direct (GPU brute force, FP64) against the oracle's direct sum: the same
plain definition (Eq. 1, kernel 1/r, zero-distance pairs skipped), so the two
agree to rounding."""
import numpy as np
import pytest
import torch

import oracle
from paper_1602_02244_gb300 import binding, workloads

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n,m", [(3000, 500), (20000, 4096), (1, 7), (257, 1)])
def test_direct_matches_oracle(cuda, n, m):
    xyz, q = workloads.uniform_cube_problem(n, 0)
    g = workloads.rng(5)
    # targets: half of them at source positions (coincident pairs are skipped)
    tgt = np.vstack([xyz[g.choice(n, (m + 1) // 2)], g.random((m // 2, 3))])[:m]
    X, Q, T = (torch.tensor(a, device=cuda) for a in (xyz, q, tgt))
    phi, grad = binding.direct(X, Q, T)
    po, go = oracle.direct(xyz, q, tgt)
    assert rel(phi.cpu().numpy(), po) <= 1e-13
    assert rel(grad.cpu().numpy(), go) <= 1e-13
    phi2, none = binding.direct(X, Q, T, grad=False)
    assert none is None and torch.equal(phi2, phi)  # deterministic


def test_direct_edge_cases(cuda):
    X = torch.zeros(0, 3, dtype=torch.float64, device=cuda)
    Q = torch.zeros(0, dtype=torch.float64, device=cuda)
    T = torch.rand(5, 3, dtype=torch.float64, device=cuda)
    phi, grad = binding.direct(X, Q, T)
    assert torch.count_nonzero(phi) == 0 and torch.count_nonzero(grad) == 0
    phi, grad = binding.direct(T, torch.ones(5, dtype=torch.float64, device=cuda), T[:0])
    assert phi.shape == (0,)
    # two charges: closed form q/r and -q r_hat / r^2
    X = torch.tensor([[0.0, 0, 0], [2.0, 0, 0]], dtype=torch.float64, device=cuda)
    Q = torch.tensor([3.0, 5.0], dtype=torch.float64, device=cuda)
    phi, grad = binding.direct(X, Q, X)
    assert phi.tolist() == [2.5, 1.5]
    assert grad.tolist() == [[1.25, 0.0, 0.0], [-0.75, 0.0, 0.0]]


def test_direct_at_full_size_matches_oracle(cuda):
    """The reference of the benchmark's error statement: the GPU brute-force
    sum on the 4,194,304-point Plummer problem at its 4096 sampled targets,
    against the oracle's FP64 direct sum at the same targets."""
    n = 4194304
    xyz, q = workloads.plummer_problem(n, 0)
    sel = workloads.sample_targets(n, 4096, 1)
    X, Q = torch.tensor(xyz, device=cuda), torch.tensor(q, device=cuda)
    phi, grad = binding.direct(X, Q, X[torch.tensor(sel, device=cuda)])
    po, go = oracle.direct(xyz, q, xyz[sel])
    phi, grad = phi.cpu().numpy(), grad.cpu().numpy()
    assert rel(phi, po) <= 1e-13
    assert rel(grad, go) <= 1e-12
    assert np.max(np.abs(phi - po) / np.abs(po)) <= 1e-12
