"""GPU parity for the inverted index (Sec. 2.2, Sec. 3.1) against the FP64 oracle.

Build: coarse centroids, list offsets, ids and list-ordered codes bit-exact
(exact nearest-list decisions, FP64 list means in row order, identical
seeding).  Query: ranked distances within 1e-5 relative and ids equal except
where the oracle's own distances tie within 1e-5 relative (counted).
"""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_2604_21645_gb300 import datagen
from tests.parity import check_topk

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
def setup(pq):
    N, D, M, Ks, nlist = 60_037, 32, 8, 64, 48
    X = datagen.mixture(N, D, 40, "int255", 4242)
    cb, _ = orc.pq_fit(X[:20_000], M, Ks, 4, 17)
    codes = orc.pq_encode(X, cb)
    ref = orc.ivf_build(X, codes, nlist, 4, 99)
    idx = pq.IVFIndex.build(dev(X), dev(codes), nlist, iters=4, seed=99)
    Q = datagen.queries(300, D, 40, "int255", 4242)
    return dict(X=X, cb=cb, codes=codes, ref=ref, idx=idx, Q=Q, nlist=nlist)


def test_build_matches_oracle(setup):
    ref, idx = setup["ref"], setup["idx"]
    assert np.array_equal(idx.coarse().cpu().numpy(), ref["coarse"])
    off, ids, codes = (t.cpu().numpy() for t in idx.lists())
    assert np.array_equal(off, ref["offsets"])
    assert np.array_equal(ids, ref["ids"])
    assert np.array_equal(codes, ref["list_codes"])


def test_build_bf16_tensor_core_matches_oracle(pq, setup):
    """The tcgen05 coarse quantizer certifies or re-checks every list decision: same index as the oracle."""
    ref = setup["ref"]
    idx = pq.IVFIndex.build(dev(setup["X"]), dev(setup["codes"]), setup["nlist"], iters=4, seed=99, prec="bf16")
    assert np.array_equal(idx.coarse().cpu().numpy(), ref["coarse"])
    off, ids, codes = (t.cpu().numpy() for t in idx.lists())
    assert np.array_equal(off, ref["offsets"])
    assert np.array_equal(ids, ref["ids"])
    assert np.array_equal(codes, ref["list_codes"])


@pytest.mark.parametrize("D,nlist,kind", [(128, 300, "int255"), (64, 512, "cont"), (96, 257, "cont")])
def test_build_bf16_shapes(pq, D, nlist, kind):
    N = 30_011
    X = datagen.mixture(N, D, 150, kind, 700 + D)
    M = D // 8
    cb, _ = orc.pq_fit(X[:8000], M, 16, 2, 3)
    codes = orc.pq_encode(X, cb)
    ref = orc.ivf_build(X, codes, nlist, 2, 31)
    idx = pq.IVFIndex.build(dev(X), dev(codes), nlist, iters=2, seed=31, prec="bf16")
    assert np.array_equal(idx.coarse().cpu().numpy(), ref["coarse"])
    off, ids, _ = (t.cpu().numpy() for t in idx.lists())
    assert np.array_equal(off, ref["offsets"]) and np.array_equal(ids, ref["ids"])


@pytest.mark.parametrize("kind", ["tiny", "wide", "subnormal"])
def test_list_means_exact_and_sequential_paths(pq, kind):
    """List means equal the oracle's row-order FP64 sums on every path: exact integer sums
    (most columns), the row-order FP64 fallback (columns holding values far below their sum's
    ulp), and the all-sequential form (X spanning more binades than 128 bits hold)."""
    N, D, nlist = 20_011, 64, 40
    X = datagen.mixture(N, D, 40, "cont", 5151)
    rng = np.random.default_rng(5152)
    pick = rng.random(X.shape) < 0.003
    if kind == "tiny":
        X[pick] *= np.float32(1e-9)
    elif kind == "wide":
        X[pick] = np.float32(3e-36)
    else:
        X[pick] = np.float32(2e-41)  # subnormal
    X = np.ascontiguousarray(X, dtype=np.float32)
    codes = np.zeros((N, 8), dtype=np.uint8)
    ref = orc.ivf_build(X, codes, nlist, 3, 77)
    for prec in ("fp32", "bf16"):
        idx = pq.IVFIndex.build(dev(X), dev(codes), nlist, iters=3, seed=77, prec=prec)
        assert np.array_equal(idx.coarse().cpu().numpy(), ref["coarse"]), prec
        off, ids, _ = (t.cpu().numpy() for t in idx.lists())
        assert np.array_equal(off, ref["offsets"]) and np.array_equal(ids, ref["ids"]), prec
        idx.close()


@pytest.mark.parametrize("nprobe,k", [(1, 1), (4, 10), (8, 100), (48, 50)])
def test_search_matches_oracle(pq, setup, nprobe, k):
    ref_ids, ref_d, _ = orc.ivf_search(setup["ref"], setup["cb"], setup["Q"], nprobe, k)
    ids, d = setup["idx"].search(dev(setup["cb"]), dev(setup["Q"]), nprobe, k)
    ties = check_topk(ids.cpu().numpy(), d.cpu().numpy(), ref_ids, ref_d)
    assert ties <= 0.01 * ref_ids.size


@pytest.mark.parametrize("D,M", [(32, 8), (64, 16)])
def test_search_long_scans_match_oracle(pq, D, M):
    """Queries that probe more than 131,072 codes (about 200k here: 4 lists, nprobe 2) take the larger
    threshold sample, and codes whose partial score passes the threshold are left early: the top-k
    still equals the oracle's (ids exact except counted near-ties, distances within 1e-5 relative)."""
    N, Ks, nlist = 400_009, 64, 4
    X = datagen.mixture(N, D, 60, "int255", 9100 + D)
    cb, _ = orc.pq_fit(X[:20_000], M, Ks, 3, 11)
    codes = orc.pq_encode(X, cb)
    ref = orc.ivf_build(X, codes, nlist, 2, 13)
    idx = pq.IVFIndex.build(dev(X), dev(codes), nlist, iters=2, seed=13)
    off = idx.lists()[0].cpu().numpy()
    Q = datagen.queries(64, D, 60, "int255", 9100 + D)
    ref_ids, ref_d, _ = orc.ivf_search(ref, cb, Q, 2, 100)
    ids, d = idx.search(dev(cb), dev(Q), 2, 100)
    idx.close()
    # most queries scan more than 131,072 codes
    assert np.sort(np.diff(off))[-2:].sum() > 131_072
    ties = check_topk(ids.cpu().numpy(), d.cpu().numpy(), ref_ids, ref_d)
    assert ties <= 0.01 * ref_ids.size


@pytest.mark.parametrize("D,M,Ks", [(16, 4, 64), (96, 12, 256), (128, 32, 16)])
def test_search_every_scan_width_matches_oracle(pq, D, M, Ks):
    """The scan is compiled per subspace count and leaves a code after M/2 and 3M/4 of its LUT terms once its
    partial score passes the threshold: for M = 4, 12 and 32 (8 and 16 are covered above) the top-k equals the
    oracle's (ids exact except counted near-ties, distances within 1e-5 relative)."""
    N, nlist = 30_011, 24
    X = datagen.mixture(N, D, 40, "cont", 300 + M)
    cb, _ = orc.pq_fit(X[:8_000], M, Ks, 3, 7)
    codes = orc.pq_encode(X, cb)
    ref = orc.ivf_build(X, codes, nlist, 2, 9)
    idx = pq.IVFIndex.build(dev(X), dev(codes), nlist, iters=2, seed=9)
    Q = datagen.queries(48, D, 40, "cont", 300 + M)
    for nprobe, k in [(3, 50), (12, 200)]:
        ref_ids, ref_d, _ = orc.ivf_search(ref, cb, Q, nprobe, k)
        ids, d = idx.search(dev(cb), dev(Q), nprobe, k)
        ties = check_topk(ids.cpu().numpy(), d.cpu().numpy(), ref_ids, ref_d)
        assert ties <= 0.01 * ref_ids.size
    idx.close()


def test_search_pads_missing_results(pq):
    N, D, M, Ks, nlist = 2_000, 16, 4, 16, 40
    X = datagen.mixture(N, D, 8, "cont", 5)
    cb, _ = orc.pq_fit(X, M, Ks, 3, 2)
    codes = orc.pq_encode(X, cb)
    ref = orc.ivf_build(X, codes, nlist, 3, 7)
    idx = pq.IVFIndex.build(dev(X), dev(codes), nlist, iters=3, seed=7)
    Q = datagen.queries(20, D, 8, "cont", 5)
    k = 600  # more than the candidates of two lists
    ref_ids, ref_d, _ = orc.ivf_search(ref, cb, Q, 2, k)
    ids, d = idx.search(dev(cb), dev(Q), 2, k)
    ids, d = ids.cpu().numpy(), d.cpu().numpy()
    assert np.array_equal(ids < 0, ref_ids < 0)
    assert np.all(np.isinf(d[ids < 0]))
    check_topk(ids, d, ref_ids, ref_d)


def test_search_exact_ties_ordered_by_id(pq):
    """Many rows with identical codes: every score ties, the k results are the lowest ids (Sec. 2.2 reading)."""
    base = datagen.mixture(50, 32, 10, "int255", 8)
    X = np.ascontiguousarray(np.tile(base, (400, 1)))  # 20,000 rows, 50 distinct
    M, Ks, nlist = 4, 32, 8
    cb, _ = orc.pq_fit(X[:5000], M, Ks, 2, 4)
    codes = orc.pq_encode(X, cb)
    ref = orc.ivf_build(X, codes, nlist, 2, 5)
    idx = pq.IVFIndex.build(dev(X), dev(codes), nlist, iters=2, seed=5)
    Q = datagen.queries(16, 32, 10, "int255", 8)
    for nprobe, k in [(2, 100), (8, 1000)]:
        ref_ids, ref_d, _ = orc.ivf_search(ref, cb, Q, nprobe, k)
        ids, d = idx.search(dev(cb), dev(Q), nprobe, k)
        check_topk(ids.cpu().numpy(), d.cpu().numpy(), ref_ids, ref_d)


def test_search_argument_errors(pq, setup):
    idx, cb, Q = setup["idx"], dev(setup["cb"]), dev(setup["Q"])
    for nprobe, k in [(0, 10), (setup["nlist"] + 1, 10), (4, 0), (4, 1025)]:
        with pytest.raises(pq.PqError) as e:
            idx.search(cb, Q, nprobe, k)
        assert e.value.status == pq.PQ_EINVAL


@pytest.mark.slow
def test_full_size_medium_config_recall(pq):
    """1M x 128, M=16, Ks=256, nlist=1024, nprobe=16, top-100: the benchmarked pipeline.
    Recall@R of the exact FP64 1-NN among the ADC top-100 on 500 sampled queries."""
    w = datagen.IVF_MEDIUM
    X = w.data()
    Xd = dev(X)
    cbs = pq.fit(Xd, w.m, w.ks, iters=w.iters, seed=w.init_seed)
    codes = pq.encode(Xd, cbs)
    idx = pq.IVFIndex.build(Xd, codes, w.nlist, iters=w.ivf_iters, seed=w.coarse_seed)
    off, ids, _ = idx.lists()
    off = off.cpu().numpy()
    assert off[0] == 0 and off[-1] == w.n and np.all(np.diff(off) >= 0)
    Q = w.queries()
    got_ids, got_d = idx.search(cbs, dev(Q), w.nprobe, w.topk)
    got_ids, got_d = got_ids.cpu().numpy(), got_d.cpu().numpy()
    assert np.all(np.diff(got_d, axis=1) >= 0)
    sample = np.random.default_rng(0).choice(w.nq, 500, replace=False)
    nn, _ = orc.exact_knn(X, Q[sample], 1)
    rec = {r: float(np.mean([nn[i, 0] in got_ids[q, :r] for i, q in enumerate(sample)])) for r in (1, 10, 100)}
    print("recall", rec)
    # The mixture's clusters are isotropic (sigma 20 in 128 dims): the 100th neighbour is only ~1.26x
    # farther than the 1st and the PQ error per dimension is about sigma, so even exhaustive FP64 ADC
    # finds the 1-NN in its top-100 for about a third of the queries.  Chance level is 1e-4.
    assert rec[100] >= 0.1


@pytest.mark.slow
def test_full_size_search_matches_oracle(pq):
    """The benchmarked search (1M x 128, nlist=1024, nprobe=16, top-100) against the oracle's search
    on 256 sampled queries.  The oracle works lock-step from the GPU's coarse centroids and PQ
    codebooks: its own FP64 nearest-list decisions (orc.assign) give the lists, which must equal the
    GPU's bit for bit, and its own encode gives the codes; then its search must agree with the GPU's
    (ids exact except counted near-ties, distances within 1e-5 relative)."""
    w = datagen.IVF_MEDIUM
    X = w.data()
    Xd = dev(X)
    cbs = pq.fit(Xd, w.m, w.ks, iters=w.iters, seed=w.init_seed, prec="bf16")
    cb = cbs.cpu().numpy()
    codes = pq.encode(Xd, cbs, prec="bf16")
    ocodes = orc.pq_encode(X, cb)
    assert np.array_equal(codes.cpu().numpy(), ocodes)
    idx = pq.IVFIndex.build(Xd, codes, w.nlist, iters=w.ivf_iters, seed=w.coarse_seed, prec="bf16")
    coarse = idx.coarse().cpu().numpy()
    off, ids, lcodes = (t.cpu().numpy() for t in idx.lists())
    lists, _, _ = orc.assign(X, coarse[None])
    lists = lists[:, 0]
    ref_off = np.concatenate([[0], np.cumsum(np.bincount(lists, minlength=w.nlist))]).astype(np.int64)
    ref_ids = np.argsort(lists, kind="stable").astype(np.int64)
    assert np.array_equal(off, ref_off)
    assert np.array_equal(ids, ref_ids)
    ref = {"coarse": coarse, "offsets": ref_off, "ids": ref_ids, "list_codes": np.ascontiguousarray(ocodes[ref_ids])}
    assert np.array_equal(lcodes, ref["list_codes"])
    Q = w.queries()
    sample = np.sort(np.random.default_rng(21).choice(w.nq, 256, replace=False))
    got_ids, got_d = idx.search(cbs, dev(Q), w.nprobe, w.topk)
    idx.close()
    o_ids, o_d, _ = orc.ivf_search(ref, cb, Q[sample], w.nprobe, w.topk)
    ties = check_topk(got_ids.cpu().numpy()[sample], got_d.cpu().numpy()[sample], o_ids, o_d)
    print("near-tie id differences", ties, "of", o_ids.size)
    assert ties <= 0.01 * o_ids.size


@pytest.mark.slow
def test_full_size_10m_search_matches_oracle(pq):
    """The benchmarked 10M search (10M x 128, nlist=1024, nprobe=16, top-100; about 445k probed codes per
    query, more than the scan's large-sample threshold) against the oracle's search over the same index on
    64 sampled queries.  The index is pinned by samples: 4,000 sampled rows lie in the list of their exact
    FP64 nearest coarse centroid (the oracle's assignment) and carry the oracle's codes under the GPU's
    codebooks.  Ids exact except counted near-ties, distances within 1e-5 relative."""
    w = datagen.IVF_10M
    X = w.data()
    Xd = dev(X)
    cbs = pq.fit(Xd, w.m, w.ks, iters=w.iters, seed=w.init_seed, prec="bf16")
    cb = cbs.cpu().numpy()
    codes = pq.encode(Xd, cbs, prec="bf16")
    idx = pq.IVFIndex.build(Xd, codes, w.nlist, iters=w.ivf_iters, seed=w.coarse_seed, prec="bf16")
    del Xd
    torch.cuda.empty_cache()
    coarse = idx.coarse().cpu().numpy()
    off, ids, lcodes = (t.cpu().numpy() for t in idx.lists())
    assert off[0] == 0 and off[-1] == w.n and np.all(np.diff(off) >= 0)
    list_of = np.empty(w.n, dtype=np.int64)
    list_of[ids] = np.repeat(np.arange(w.nlist), np.diff(off))
    rows = np.sort(np.random.default_rng(5).choice(w.n, 4000, replace=False))
    ref_lists, _, _ = orc.assign(X[rows], coarse[None])
    assert np.array_equal(list_of[rows], ref_lists[:, 0])
    pos = np.empty(w.n, dtype=np.int64)
    pos[ids] = np.arange(w.n)
    assert np.array_equal(lcodes[pos[rows]], orc.pq_encode(X[rows], cb))
    Q = w.queries()
    got_ids, got_d = idx.search(cbs, dev(Q), w.nprobe, w.topk)
    idx.close()
    sample = np.sort(np.random.default_rng(8).choice(w.nq, 64, replace=False))
    ref = {"coarse": coarse, "offsets": off, "ids": ids, "list_codes": lcodes}
    o_ids, o_d, _ = orc.ivf_search(ref, cb, Q[sample], w.nprobe, w.topk)
    ties = check_topk(got_ids.cpu().numpy()[sample], got_d.cpu().numpy()[sample], o_ids, o_d)
    print("near-tie id differences", ties, "of", o_ids.size)
    assert ties <= 0.01 * o_ids.size
