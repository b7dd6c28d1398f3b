"""GPU parity of optimized PQ (OPQ) against the oracle: the rotation X R and the Procrustes
step lock-step (same inputs on both sides), and the whole alternating fit.

Bars: rotated rows within 4e-6 of their norm (FP32 sums of D products against FP64 rounded
once); Procrustes rotations within 1e-5 per entry (the device's X^T Y in float-float against
FP64); the whole fit, whose iterations carry the rotated rows' last-bit differences into the
PQ decisions, within 1e-3 relative in RMSE, and below plain PQ's RMSE on correlated rows.
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
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rotation(d, seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).standard_normal((d, d)))
    return (q * np.sign(np.diag(r))).astype(np.float32)


def correlated(n, d, seed):
    base = datagen.mixture(n, d, 40, "cont", seed).astype(np.float64)
    return np.ascontiguousarray((base @ rotation(d, seed + 1) * np.linspace(2.0, 0.2, d)).astype(np.float32))


@pytest.mark.parametrize("n,d", [(5000, 32), (70_001, 128), (3, 64)])
def test_rotate_matches_oracle(pq, n, d):
    X = datagen.mixture(n, d, 10, "cont", 90 + d)
    R = rotation(d, 91)
    got = pq.opq_rotate(dev(X), dev(R)).cpu().numpy()
    ref = orc.opq_rotate(X, R)
    norm = np.linalg.norm(X.astype(np.float64), axis=1, keepdims=True)
    assert np.all(np.abs(got - ref) <= 4e-6 * norm + 1e-30)


@pytest.mark.parametrize("n,d", [(20_000, 32), (300_000, 128)])
def test_procrustes_matches_oracle(pq, n, d):
    X = correlated(n, d, 92)
    Y = (X.astype(np.float64) @ rotation(d, 93) + 0.05 * np.random.default_rng(94).standard_normal(X.shape))
    Y = Y.astype(np.float32)
    got = pq.opq_procrustes(dev(X), dev(Y)).cpu().numpy().astype(np.float64)
    ref = orc.opq_procrustes(X, Y)
    assert np.abs(got - ref).max() <= 1e-5
    np.testing.assert_allclose(got @ got.T, np.eye(d), atol=1e-5)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_opq_fit_matches_oracle(pq, prec):
    X = correlated(30_000, 32, 95)
    M, Ks = 4, 64
    R, cb = pq.opq_fit(dev(X), M, Ks, outer=4, pq_iters=4, seed=96, prec=prec)
    R_ref, cb_ref, _ = orc.opq_fit(X, M, Ks, 4, 4, 96)
    R = R.cpu().numpy()
    cb = cb.cpu().numpy()
    Y = orc.opq_rotate(X, R)
    r = orc.pq_rmse(Y, orc.pq_encode(Y, cb), cb)
    Yr = orc.opq_rotate(X, R_ref)
    r_ref = orc.pq_rmse(Yr, orc.pq_encode(Yr, cb_ref), cb_ref)
    print(f"OPQ RMSE gpu {r:.6f} oracle {r_ref:.6f}; max |R - R_ref| {np.abs(R - R_ref).max():.2e}")
    assert abs(r - r_ref) <= 1e-3 * r_ref
    np.testing.assert_allclose(R.astype(np.float64) @ R.T, np.eye(32), atol=1e-5)
    plain, _ = orc.pq_fit(X, M, Ks, 4, 96)
    assert r < orc.pq_rmse(X, orc.pq_encode(X, plain), plain)


def test_opq_zero_rounds_is_plain_fit(pq):
    X = correlated(8000, 32, 97)
    R, cb = pq.opq_fit(dev(X), 4, 32, outer=0, pq_iters=3, seed=98)
    assert np.array_equal(R.cpu().numpy(), np.eye(32, dtype=np.float32))
    ref, _ = orc.pq_fit(X, 4, 32, 3, 98)
    np.testing.assert_allclose(cb.cpu().numpy(), ref, rtol=0, atol=1e-5 * np.abs(ref).max())
