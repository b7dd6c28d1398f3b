"""GPU parity of the soft-assignment PQ loss and its gradients against the FP64 oracle.

Bars: the loss within 1e-5 relative; dL/dC and dL/dX in FP32 within 1e-4
relative (norm-wise) of the oracle's, and element-wise within 1e-4 of the
largest oracle entry.  Sizes span several 256-row tiles with a ragged tail; the
1M x 256 workload is checked on sampled rows of dL/dX (each row's gradient
depends only on that row and the codebooks) and on the row-additivity of L and
dL/dC, which holds at any size.
"""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_2604_21645_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_21645_gb300 import pqgb
    return pqgb


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def codebooks_from_rows(X, M, Ks, seed, noise=0.02):
    """Codewords = seeded random rows of X (per subspace) plus small noise: a plausible refinement start."""
    rng = np.random.default_rng(seed)
    N, D = X.shape
    ds = D // M
    C = np.empty((M, Ks, ds), dtype=np.float32)
    for m in range(M):
        idx = rng.integers(0, N, size=Ks)
        C[m] = X[idx, m * ds:(m + 1) * ds] + noise * rng.standard_normal((Ks, ds))
    return C


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def check_grad(g, ref, elem=1e-4):
    assert rel(g, ref) < 1e-4, rel(g, ref)
    assert np.max(np.abs(g - ref)) <= elem * np.max(np.abs(ref))


CASES = [(1537, 64, 8, 256, 0.1), (1000, 256, 32, 256, 0.1), (700, 32, 8, 64, 0.05), (900, 64, 4, 100, 0.2),
         (513, 48, 12, 256, 0.1)]


@pytest.mark.parametrize("N,D,M,Ks,tau", CASES)
def test_softpq_matches_oracle(pq, N, D, M, Ks, tau):
    X = datagen.mixture(N, D, 64, "cont", 6100 + N)
    C = codebooks_from_rows(X, M, Ks, 6200 + N)
    L = pq.softpq_forward(dev(X), dev(C), tau).item()
    L_ref = orc.softpq_forward(X, C, tau)
    assert abs(L - L_ref) <= 1e-5 * L_ref
    dC, dX = pq.softpq_backward(dev(X), dev(C), tau)
    dC_ref, dX_ref = orc.softpq_backward(X, C, tau)
    check_grad(dC.cpu().numpy().astype(np.float64), dC_ref)
    check_grad(dX.cpu().numpy().astype(np.float64), dX_ref)


def test_autograd_function(pq):
    from paper_2604_21645_gb300.softpq import softpq_loss
    N, D, M, Ks, tau = 800, 64, 8, 256, 0.1
    X = datagen.mixture(N, D, 32, "cont", 6301)
    C = codebooks_from_rows(X, M, Ks, 6302)
    Xt = dev(X).requires_grad_(True)
    Ct = dev(C).requires_grad_(True)
    loss = softpq_loss(Xt, Ct, tau)
    (3.0 * loss).backward()
    dC_ref, dX_ref = orc.softpq_backward(X, C, tau)
    check_grad(Ct.grad.cpu().numpy().astype(np.float64) / 3.0, dC_ref)
    check_grad(Xt.grad.cpu().numpy().astype(np.float64) / 3.0, dX_ref)
    # only the codebooks need a gradient: dX is not computed
    Ct2 = dev(C).requires_grad_(True)
    (g,) = torch.autograd.grad(softpq_loss(dev(X), Ct2, tau), Ct2)
    check_grad(g.cpu().numpy().astype(np.float64), dC_ref)


def test_far_rows_use_the_shifted_softmax(pq):
    """Rows so far from every codeword that 2^(-d/tau log2 e) underflows take the max-shifted path."""
    N, D, M, Ks, tau = 300, 32, 4, 64, 0.01
    X = datagen.mixture(N, D, 16, "cont", 6401)
    C = codebooks_from_rows(X, M, Ks, 6402)
    X[::3] += 4.0  # d >= 16 per subspace => d/tau >= 1600
    L = pq.softpq_forward(dev(X), dev(C), tau).item()
    L_ref = orc.softpq_forward(X, C, tau)
    assert abs(L - L_ref) <= 1e-5 * L_ref
    dC, dX = pq.softpq_backward(dev(X), dev(C), tau)
    dC_ref, dX_ref = orc.softpq_backward(X, C, tau)
    # The far rows are ill-conditioned in FP32: their logits are near -2^11 and carry an
    # absolute error of about 2^-24 * 2 log2(e)/tau * |x'||c'| (~3e-4), so their entries are
    # held to 5e-4 of the largest one; the norm-wise bar stays 1e-4.
    check_grad(dC.cpu().numpy().astype(np.float64), dC_ref, elem=5e-4)
    check_grad(dX.cpu().numpy().astype(np.float64), dX_ref, elem=5e-4)


def test_empty_input(pq):
    C = torch.randn(8, 256, 8, device="cuda")
    X = torch.empty((0, 64), dtype=torch.float32, device="cuda")
    assert pq.softpq_forward(X, C, 0.1).item() == 0.0
    dC, dX = pq.softpq_backward(X, C, 0.1)
    assert torch.count_nonzero(dC).item() == 0


def test_rejects_bad_arguments(pq):
    X = torch.zeros((10, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(pq.PqError) as e:
        pq.softpq_forward(X, torch.zeros((8, 256, 8), device="cuda"), 0.0)
    assert e.value.status == pq.PQ_EINVAL
    with pytest.raises(pq.PqError) as e:
        pq.softpq_forward(torch.zeros((10, 96), device="cuda"), torch.zeros((8, 256, 12), device="cuda"), 0.1)
    assert e.value.status == pq.PQ_ENOTSUP


def test_refinement_lowers_the_loss(pq):
    from paper_2604_21645_gb300.softpq import refine, softpq_loss
    N, D, M, Ks, tau = 20_000, 64, 8, 256, 0.1
    X = dev(datagen.mixture(N, D, 64, "cont", 6501))
    C0 = dev(codebooks_from_rows(X.cpu().numpy(), M, Ks, 6502, noise=0.1))
    l0 = softpq_loss(X, C0, tau).item()
    C1 = refine(X, C0, tau, steps=20, lr=0.5)
    l1 = softpq_loss(X, C1, tau).item()
    assert l1 < 0.9 * l0


def test_full_size_sampled_rows_and_additivity(pq):
    """1M x 256, M=32, Ks=256, tau=0.1: sampled dX rows against the oracle; L and dC additive over row blocks."""
    w = datagen.SOFTPQ
    X = w.data()
    C = codebooks_from_rows(X[:100_000], w.m, w.ks, w.seed + 11)
    Xd, Cd = dev(X), dev(C)
    L = pq.softpq_forward(Xd, Cd, w.tau).item()
    dC, dX = pq.softpq_backward(Xd, Cd, w.tau)
    rng = np.random.default_rng(w.seed + 12)
    rows = np.sort(rng.choice(w.n, size=48, replace=False))
    _, dX_s = orc.softpq_backward(X[rows], C, w.tau)
    dX_s *= len(rows) / w.n  # the oracle normalises by its own row count
    check_grad(dX[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64), dX_s)
    h = 400_003
    L1 = pq.softpq_forward(Xd[:h].contiguous(), Cd, w.tau).item()
    L2 = pq.softpq_forward(Xd[h:].contiguous(), Cd, w.tau).item()
    assert abs(L - (h * L1 + (w.n - h) * L2) / w.n) <= 1e-5 * L
    dC1, _ = pq.softpq_backward(Xd[:h].contiguous(), Cd, w.tau, need_dx=False)
    dC2, _ = pq.softpq_backward(Xd[h:].contiguous(), Cd, w.tau, need_dx=False)
    comb = (h * dC1.double() + (w.n - h) * dC2.double()) / w.n
    assert rel(dC.double().cpu().numpy(), comb.cpu().numpy()) < 1e-5
