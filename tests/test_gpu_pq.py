"""GPU parity for PQ fit / encode / decode-RMSE (Sec. 2.1, Sec. 3) against the FP64 oracle.

Inputs come from the seeded generators; any codebook fed to both sides is made
by the oracle.  Bars: codes bit-exact (the GPU re-decides every uncertain
argmin in FP64), seeding bit-exact, codewords within 1e-5 relative, RMSE within
1e-4 relative.
"""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_2604_21645_gb300 import datagen
from tests.parity import RMSE_RTOL, assert_codebooks_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_21645_gb300 import pqgb
    return pqgb


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


W1 = datagen.PQ_SMALL


@pytest.fixture(scope="module")
def small():
    return W1.data()


# -- seeding -------------------------------------------------------------------------

def test_kmeanspp_bit_exact_all_rows(pq, small):
    ref = orc.kmeanspp(small, W1.m, W1.ks, W1.init_seed)
    got = pq.init_kmeanspp(dev(small), W1.m, W1.ks, W1.init_seed).cpu().numpy()
    assert np.array_equal(got, ref)


def test_kmeanspp_bit_exact_subsample(pq):
    X = datagen.mixture(60_000, 32, 50, "int255", 77)   # 100*Ks = 6,400 < N
    ref = orc.kmeanspp(X, 4, 64, 5)
    got = pq.init_kmeanspp(dev(X), 4, 64, 5).cpu().numpy()
    assert np.array_equal(got, ref)


def test_kmeanspp_duplicates_fall_back_to_uniform(pq):
    rng = np.random.default_rng(0)
    base = rng.normal(size=(40, 8)).astype(np.float32)
    X = base[rng.integers(0, 40, size=512)]              # fewer distinct rows than Ks
    ref = orc.kmeanspp(X, 2, 64, 9)
    got = pq.init_kmeanspp(dev(X), 2, 64, 9).cpu().numpy()
    assert np.array_equal(got, ref)


# -- encode -------------------------------------------------------------------------

@pytest.fixture(scope="module")
def oracle_cb(small):
    cb, _ = orc.pq_fit(small, W1.m, W1.ks, 4, W1.init_seed)
    return cb


@pytest.mark.parametrize("n", [1, 255, 10_000, 10_037])
def test_encode_bit_exact(pq, small, oracle_cb, n):
    X = small[:n] if n <= small.shape[0] else np.concatenate([small, small[:n - small.shape[0]] * 1.5])
    ref = orc.pq_encode(X, oracle_cb)
    got, st = pq.encode(dev(X), dev(oracle_cb), stats=True)
    assert np.array_equal(got.cpu().numpy(), ref)


def test_encode_exact_ties_go_to_lowest_index(pq):
    cb = np.zeros((2, 8, 4), dtype=np.float32)
    cb[:, 3] = 1.0
    cb[:, 5] = 1.0                                      # duplicate codeword: equal distances
    cb[:, 6] = -1.0
    X = np.ones((64, 8), dtype=np.float32)
    X[32:] = 0.0                                        # equidistant from codewords 0,1,2,4,7 (all zero)
    got = pq.encode(dev(X), dev(cb)).cpu().numpy()
    assert np.array_equal(got, orc.pq_encode(X, cb))
    assert np.all(got[:32] == 3) and np.all(got[32:] == 0)


def test_encode_empty_and_sse(pq, small, oracle_cb):
    sse = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = pq.encode(dev(small[:0]), dev(oracle_cb), sse=sse)
    assert out.shape == (0, W1.m) and sse.item() == 0.0
    codes = orc.pq_encode(small, oracle_cb)
    pq.encode(dev(small), dev(oracle_cb), sse=sse)
    ref = orc.pq_rmse(small, codes, oracle_cb)
    got = np.sqrt(sse.item() / small.size)
    assert abs(got - ref) <= RMSE_RTOL * ref


# -- decode + RMSE ---------------------------------------------------------------------

def test_decode_rmse(pq, small, oracle_cb):
    codes = orc.pq_encode(small, oracle_cb)
    xhat, r = pq.decode_rmse(dev(codes), dev(oracle_cb), dev(small), want_xhat=True)
    assert np.array_equal(xhat.cpu().numpy(), orc.pq_decode(codes, oracle_cb))
    ref = orc.pq_rmse(small, codes, oracle_cb)
    assert abs(r - ref) <= RMSE_RTOL * ref


def test_rmse_zero_when_rows_are_codewords(pq):
    rng = np.random.default_rng(1)
    X = rng.normal(size=(256, 16)).astype(np.float32)
    cb = np.stack([X[:, 4 * m:4 * m + 4] for m in range(4)])
    codes = pq.encode(dev(X), dev(cb))
    _, r = pq.decode_rmse(codes, dev(cb), dev(X))
    assert r == 0.0


# -- Lloyd ------------------------------------------------------------------------------

def test_lloyd_lockstep_one_iteration(pq, small):
    init = orc.kmeanspp(small, W1.m, W1.ks, W1.init_seed)
    ref, sse_ref = orc.pq_fit(small, W1.m, W1.ks, 1, 0, init=init)
    got, st = pq.fit(dev(small), W1.m, W1.ks, iters=1, init=dev(init), stats=True)
    got = got.cpu().numpy()
    assert_codebooks_close(got, ref)
    assert abs(st["sse"][0] - sse_ref[0]) <= 1e-5 * sse_ref[0]


def test_fit_free_running_small(pq, small):
    ref, sse_ref = orc.pq_fit(small, W1.m, W1.ks, W1.iters, W1.init_seed)
    got, st = pq.fit(dev(small), W1.m, W1.ks, iters=W1.iters, seed=W1.init_seed, stats=True)
    got = got.cpu().numpy()
    assert_codebooks_close(got, ref)
    r_ref = orc.pq_rmse(small, orc.pq_encode(small, ref), ref)
    codes = pq.encode(dev(small), dev(got))
    _, r = pq.decode_rmse(codes, dev(got), dev(small))
    assert abs(r - r_ref) <= RMSE_RTOL * r_ref
    np.testing.assert_allclose(st["sse"], sse_ref, rtol=1e-5)
    assert all(b <= a * (1 + 1e-6) for a, b in zip(st["sse"], st["sse"][1:]))


@pytest.mark.parametrize("D,M,Ks", [(16, 16, 8), (32, 16, 16), (64, 16, 32), (64, 4, 100), (96, 3, 64), (64, 2, 256)])
def test_fit_shapes(pq, D, M, Ks):
    X = datagen.mixture(3_001, D, 20, "cont", 100 + D + M)
    init = orc.kmeanspp(X, M, Ks, 3)
    assert np.array_equal(pq.init_kmeanspp(dev(X), M, Ks, 3).cpu().numpy(), init)
    ref, _ = orc.pq_fit(X, M, Ks, 3, 0, init=init)
    got = pq.fit(dev(X), M, Ks, iters=3, init=dev(init)).cpu().numpy()
    assert_codebooks_close(got, ref)
    assert np.array_equal(pq.encode(dev(X), dev(ref)).cpu().numpy(), orc.pq_encode(X, ref))


def test_fit_n_equals_ks(pq):
    rng = np.random.default_rng(2)
    X = rng.normal(size=(64, 16)).astype(np.float32)
    got = pq.fit(dev(X), 4, 64, iters=3, seed=11)
    codes = pq.encode(dev(X), got)
    _, r = pq.decode_rmse(codes, got, dev(X))
    assert r == 0.0


def test_fit_int255_lockstep_medium(pq):
    X = datagen.mixture(200_000, 128, 1000, "int255", datagen.IVF_MEDIUM.seed)
    init = orc.kmeanspp(X, 16, 256, 21)
    assert np.array_equal(pq.init_kmeanspp(dev(X), 16, 256, 21).cpu().numpy(), init)
    ref, sse_ref = orc.pq_fit(X, 16, 256, 2, 0, init=init)
    got, st = pq.fit(dev(X), 16, 256, iters=2, init=dev(init), stats=True)
    assert_codebooks_close(got.cpu().numpy(), ref)
    np.testing.assert_allclose(st["sse"], sse_ref, rtol=1e-5)
    assert np.array_equal(pq.encode(dev(X), dev(ref)).cpu().numpy(), orc.pq_encode(X, ref))


@pytest.mark.slow
def test_full_size_medium_config(pq):
    """1M x 128 integer-valued mixture, M=16, Ks=256: seeding bit-exact, one lock-step
    Lloyd iteration over all rows, and codes bit-exact on 50k sampled rows."""
    w = datagen.IVF_MEDIUM
    X = w.data()
    Xd = dev(X)
    init = orc.kmeanspp(X, w.m, w.ks, w.init_seed)
    assert np.array_equal(pq.init_kmeanspp(Xd, w.m, w.ks, w.init_seed).cpu().numpy(), init)
    ref, sse_ref = orc.pq_fit(X, w.m, w.ks, 1, 0, init=init)
    got, st = pq.fit(Xd, w.m, w.ks, iters=1, init=dev(init), stats=True)
    assert_codebooks_close(got.cpu().numpy(), ref)
    assert abs(st["sse"][0] - sse_ref[0]) <= 1e-5 * sse_ref[0]
    rows = np.random.default_rng(3).choice(w.n, 50_000, replace=False)
    codes = pq.encode(Xd, dev(ref)).cpu().numpy()
    assert np.array_equal(codes[rows], orc.pq_encode(X[rows], ref))
    # the full fit in the configuration the benchmark times: SSE never rises
    _, st = pq.fit(Xd, w.m, w.ks, iters=w.iters, seed=w.init_seed, stats=True)
    s = st["sse"]
    assert all(b <= a * (1 + 1e-6) for a, b in zip(s, s[1:]))
