"""GPU parity of the BF16 tcgen05 form of PQ encode / fit against the FP64 oracle.

The BF16 contraction only proposes the nearest codeword; every decision it
cannot certify with its error bound is re-taken exactly, so the bars are the
FP32 form's: codes bit-exact, codewords within 1e-5 relative, RMSE within 1e-4.
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


@pytest.fixture(scope="module")
def small():
    w = datagen.PQ_SMALL
    X = w.data()
    cb, _ = orc.pq_fit(X, w.m, w.ks, 4, w.init_seed)
    return X, cb


@pytest.mark.parametrize("n", [1, 127, 128, 129, 10_000, 10_037])
def test_encode_bf16_bit_exact(pq, small, n):
    X, cb = small
    X = X[:n] if n <= X.shape[0] else np.concatenate([X, X[:n - X.shape[0]] * 1.25])
    got, st = pq.encode(dev(X), dev(cb), prec="bf16", stats=True)
    assert np.array_equal(got.cpu().numpy(), orc.pq_encode(X, cb))


@pytest.mark.parametrize("D,M,Ks,kind", [(128, 16, 256, "int255"), (96, 12, 256, "cont"), (256, 32, 256, "cont"),
                                        (32, 4, 100, "cont"), (64, 8, 7, "int255"),
                                        (48, 6, 256, "cont"), (16, 2, 64, "int255")])
def test_encode_bf16_shapes(pq, D, M, Ks, kind):
    X = datagen.mixture(20_000, D, 300, kind, 300 + D)
    cb, _ = orc.pq_fit(X[:5000], M, Ks, 3, 1)
    got, st = pq.encode(dev(X), dev(cb), prec="bf16", stats=True)
    assert np.array_equal(got.cpu().numpy(), orc.pq_encode(X, cb))
    # the bf16 bound should settle almost every decision without the exact fallback
    assert st["fp64_rechecks"] <= 0.2 * X.shape[0] * M


def test_encode_bf16_ties(pq):
    cb = np.zeros((4, 256, 8), dtype=np.float32)
    rng = np.random.default_rng(7)
    cb[:] = rng.normal(size=cb.shape).astype(np.float32)
    cb[:, 200] = cb[:, 3]                                 # duplicate codeword: exact ties
    X = np.repeat(cb[:, 3].reshape(1, -1), 256, axis=0)   # rows sitting on codeword 3
    got = pq.encode(dev(X), dev(cb), prec="bf16").cpu().numpy()
    assert np.array_equal(got, orc.pq_encode(X, cb))
    assert np.all(got == 3)


def test_encode_bf16_sse(pq, small):
    X, cb = small
    sse = torch.zeros(1, dtype=torch.float64, device="cuda")
    pq.encode(dev(X), dev(cb), prec="bf16", sse=sse)
    ref = orc.pq_rmse(X, orc.pq_encode(X, cb), cb)
    assert abs(np.sqrt(sse.item() / X.size) - ref) <= RMSE_RTOL * ref


def test_lloyd_bf16_lockstep(pq, small):
    X, _ = small
    w = datagen.PQ_SMALL
    init = orc.kmeanspp(X, w.m, w.ks, w.init_seed)
    ref, sse_ref = orc.pq_fit(X, w.m, w.ks, 1, 0, init=init)
    got, st = pq.fit(dev(X), w.m, w.ks, iters=1, init=dev(init), prec="bf16", stats=True)
    assert_codebooks_close(got.cpu().numpy(), ref)
    assert abs(st["sse"][0] - sse_ref[0]) <= 1e-5 * sse_ref[0]


def test_fit_bf16_free_running(pq, small):
    X, _ = small
    w = datagen.PQ_SMALL
    ref, sse_ref = orc.pq_fit(X, w.m, w.ks, w.iters, w.init_seed)
    got, st = pq.fit(dev(X), w.m, w.ks, iters=w.iters, seed=w.init_seed, prec="bf16", stats=True)
    got = got.cpu().numpy()
    assert_codebooks_close(got, ref)
    r_ref = orc.pq_rmse(X, orc.pq_encode(X, ref), ref)
    codes = pq.encode(dev(X), dev(got), prec="bf16")
    _, r = pq.decode_rmse(codes, dev(got), dev(X))
    assert abs(r - r_ref) <= RMSE_RTOL * r_ref


def test_fit_bf16_int255_lockstep_medium(pq):
    X = datagen.mixture(200_000, 128, 1000, "int255", datagen.IVF_MEDIUM.seed)
    init = orc.kmeanspp(X, 16, 256, 21)
    ref, sse_ref = orc.pq_fit(X, 16, 256, 2, 0, init=init)
    got, st = pq.fit(dev(X), 16, 256, iters=2, init=dev(init), prec="bf16", stats=True)
    assert_codebooks_close(got.cpu().numpy(), ref)
    np.testing.assert_allclose(st["sse"], sse_ref, rtol=1e-5)
    assert np.array_equal(pq.encode(dev(X), dev(ref), prec="bf16").cpu().numpy(), orc.pq_encode(X, ref))


def test_bf16_unsupported_shape(pq):
    X = torch.zeros((1000, 64), dtype=torch.float32, device="cuda")
    cb = torch.zeros((16, 256, 4), dtype=torch.float32, device="cuda")  # Ds = 4
    with pytest.raises(pq.PqError) as e:
        pq.encode(X, cb, prec="bf16")
    assert e.value.status == pq.PQ_ENOTSUP


@pytest.mark.slow
def test_full_size_bf16_benchmarked_config(pq):
    """1M x 128, M=16, Ks=256, BF16 -- the configuration the benchmark times: one lock-step BF16
    Lloyd iteration over all rows against the oracle, codes bit-exact on 50k sampled rows, and the
    BF16 coarse index after its 25 iterations: every sampled row sits in the list of its exact
    (FP64, ties to the lower list) nearest coarse centroid."""
    w = datagen.IVF_MEDIUM
    X = w.data()
    Xd = dev(X)
    init = orc.kmeanspp(X, w.m, w.ks, w.init_seed)
    ref, sse_ref = orc.pq_fit(X, w.m, w.ks, 1, 0, init=init)
    got, st = pq.fit(Xd, w.m, w.ks, iters=1, init=dev(init), prec="bf16", stats=True)
    assert_codebooks_close(got.cpu().numpy(), ref)
    assert abs(st["sse"][0] - sse_ref[0]) <= 1e-5 * sse_ref[0]
    rng = np.random.default_rng(11)
    rows = rng.choice(w.n, 50_000, replace=False)
    codes = pq.encode(Xd, dev(ref), prec="bf16")
    assert np.array_equal(codes.cpu().numpy()[rows], orc.pq_encode(X[rows], ref))
    idx = pq.IVFIndex.build(Xd, codes, w.nlist, iters=w.ivf_iters, seed=w.coarse_seed, prec="bf16")
    coarse = idx.coarse().cpu().numpy()
    off, ids, _ = (t.cpu().numpy() for t in idx.lists())
    idx.close()
    assert off[0] == 0 and off[-1] == w.n and np.array_equal(np.sort(ids), np.arange(w.n))
    list_of = np.empty(w.n, dtype=np.int64)
    for l in range(w.nlist):
        list_of[ids[off[l]:off[l + 1]]] = l
    sample = rng.choice(w.n, 2_000, replace=False)
    nearest, _ = orc.exact_knn(coarse, X[sample], 1)
    assert np.array_equal(list_of[sample], nearest[:, 0])


@pytest.mark.slow
def test_full_size_precision_form(pq):
    """10M x 128, M=16, Ks=256, 20 iterations -- the precision form as the benchmark runs it: the BF16
    and FP32 forms reach the same RMSE (within 1e-4), each form's RMSE equals the FP64 oracle's over
    all 10M rows (within 1e-4), and both forms' codes are exact on 50k sampled rows against the
    oracle's encode under their codebooks."""
    w = datagen.PQ_10M
    X = w.data()
    Xd = dev(X)
    cb16 = pq.fit(Xd, w.m, w.ks, iters=w.iters, seed=w.init_seed, prec="bf16")
    codes16 = pq.encode(Xd, cb16, prec="bf16")
    _, r16 = pq.decode_rmse(codes16, cb16, Xd)
    cb32 = pq.fit(Xd, w.m, w.ks, iters=w.iters, seed=w.init_seed, prec="fp32")
    codes32 = pq.encode(Xd, cb32)
    _, r32 = pq.decode_rmse(codes32, cb32, Xd)
    assert abs(r16 - r32) <= RMSE_RTOL * r32
    # each form's RMSE against the FP64 oracle's, over all 10M rows, with that form's codes and codebooks
    o16 = orc.pq_rmse(X, codes16.cpu().numpy(), cb16.cpu().numpy())
    o32 = orc.pq_rmse(X, codes32.cpu().numpy(), cb32.cpu().numpy())
    print(f"RMSE relative error against the oracle: bf16 {abs(r16 - o16) / o16:.3e}, fp32 {abs(r32 - o32) / o32:.3e}")
    assert abs(r16 - o16) <= RMSE_RTOL * o16
    assert abs(r32 - o32) <= RMSE_RTOL * o32
    rows = np.random.default_rng(13).choice(w.n, 50_000, replace=False)
    assert np.array_equal(codes16.cpu().numpy()[rows], orc.pq_encode(X[rows], cb16.cpu().numpy()))
    assert np.array_equal(codes32.cpu().numpy()[rows], orc.pq_encode(X[rows], cb32.cpu().numpy()))
