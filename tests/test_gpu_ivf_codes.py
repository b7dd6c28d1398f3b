"""GPU parity of the code-space inverted index (Rii, Sec. 3.1) and of growing an index by
add and merge, against the FP64 oracle.

Build: centre codes, list offsets, ids and list-ordered codes bit-exact (exact symmetric-
distance decisions, exact sparse-voting updates, the same centre draw).  Query: ranked
distances within 1e-5 relative, ids equal except where the oracle's own distances tie within
1e-5 relative.  Add and merge: the lists equal those of one assignment of all rows to the same
coarse quantizer, bit for bit.
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


def lists_of(labels, codes, nlist):
    """CSR lists with ids ascending inside a list, from each row's list."""
    off = np.concatenate([[0], np.cumsum(np.bincount(labels, minlength=nlist))]).astype(np.int64)
    ids = np.argsort(labels, kind="stable").astype(np.int64)
    return off, ids, np.ascontiguousarray(codes[ids])


def assert_lists(idx, off, ids, lcodes):
    o, i, c = (t.cpu().numpy() for t in idx.lists())
    assert np.array_equal(o, off)
    assert np.array_equal(i, ids)
    assert np.array_equal(c, lcodes)


CASES = [  # N, D, M, Ks, nlist, iters, kind
    (20_011, 32, 4, 64, 40, 4, "cont"),
    (30_007, 128, 16, 256, 64, 3, "int255"),
    (12_000, 48, 4, 100, 33, 5, "cont"),
]


@pytest.fixture(scope="module", params=range(len(CASES)))
def case(request):
    N, D, M, Ks, nlist, iters, kind = CASES[request.param]
    X = datagen.mixture(N, D, 60, kind, 800 + request.param)
    cb, _ = orc.pq_fit(X[:6000], M, Ks, 3, 11)
    codes = orc.pq_encode(X, cb)
    ref = orc.ivf_build_codes(codes, cb, nlist, iters, 77)
    return dict(X=X, cb=cb, codes=codes, ref=ref, nlist=nlist, iters=iters, kind=kind)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_build_codes_matches_oracle(pq, case, prec):
    ref = case["ref"]
    idx = pq.IVFIndex.build_codes(dev(case["codes"]), dev(case["cb"]), case["nlist"], iters=case["iters"], seed=77,
                                  prec=prec)
    assert np.array_equal(idx.centers().cpu().numpy(), ref["centers"])
    assert_lists(idx, ref["offsets"], ref["ids"], ref["list_codes"])
    idx.close()


@pytest.mark.parametrize("nprobe,k", [(1, 10), (4, 100), (12, 50)])
def test_search_codes_matches_oracle(pq, case, nprobe, k):
    idx = pq.IVFIndex.build_codes(dev(case["codes"]), dev(case["cb"]), case["nlist"], iters=case["iters"], seed=77)
    X = case["X"]
    Q = datagen.queries(200, X.shape[1], 60, case["kind"], 900)
    ref_ids, ref_d, _ = orc.ivf_search_codes(case["ref"], case["cb"], Q, nprobe, k)
    ids, d = idx.search(dev(case["cb"]), dev(Q), nprobe, k)
    ties = check_topk(ids.cpu().numpy(), d.cpu().numpy(), ref_ids, ref_d)
    assert ties <= 0.01 * ref_ids.size
    idx.close()


def test_build_codes_rejects_bad_arguments(pq):
    codes = torch.zeros((100, 4), dtype=torch.uint8, device="cuda")
    cb = torch.zeros((4, 16, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(pq.PqError) as e:
        pq.IVFIndex.build_codes(codes, cb, 101)
    assert e.value.status == pq.PQ_EINVAL


def _raw_case():
    N, D, M, Ks, nlist = 30_011, 64, 8, 32, 48
    X = datagen.mixture(N, D, 50, "cont", 321)
    cb, _ = orc.pq_fit(X[:5000], M, Ks, 3, 7)
    return X, cb, orc.pq_encode(X, cb), nlist


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_add_equals_one_assignment_of_all_rows(pq, prec):
    X, cb, codes, nlist = _raw_case()
    a = 11_000
    idx = pq.IVFIndex.build(dev(X[:a]), dev(codes[:a]), nlist, iters=4, seed=3, prec=prec)
    idx.add(dev(codes[a:]), dev(X[a:]), prec=prec)
    assert idx.N == len(X)
    coarse = idx.coarse().cpu().numpy()
    lab, _, _ = orc.assign(X, coarse[None])
    assert_lists(idx, *lists_of(lab[:, 0], codes, nlist))
    idx.close()


def test_merge_of_chunks_equals_one_assignment(pq):
    X, cb, codes, nlist = _raw_case()
    bounds = [0, 7_000, 7_001, 19_500, len(X)]
    base = pq.IVFIndex.build(dev(X[:5000]), dev(codes[:5000]), nlist, iters=4, seed=3)
    merged = base.clone_empty()
    for c in range(len(bounds) - 1):
        part = base.clone_empty()
        r0, r1 = bounds[c], bounds[c + 1]
        part.add(dev(codes[r0:r1]), dev(X[r0:r1]))
        merged.merge(part)
        part.close()
    assert merged.N == len(X)
    lab, _, _ = orc.assign(X, base.coarse().cpu().numpy()[None])
    assert_lists(merged, *lists_of(lab[:, 0], codes, nlist))
    # a search over the merged index equals the oracle's over the same lists
    ref = dict(zip(("offsets", "ids", "list_codes"), lists_of(lab[:, 0], codes, nlist)))
    ref["coarse"] = base.coarse().cpu().numpy()
    Q = datagen.queries(100, X.shape[1], 50, "cont", 322)
    r_ids, r_d, _ = orc.ivf_search(ref, cb, Q, 6, 40)
    ids, d = merged.search(dev(cb), dev(Q), 6, 40)
    check_topk(ids.cpu().numpy(), d.cpu().numpy(), r_ids, r_d)
    base.close()
    merged.close()


def test_code_space_add_and_merge(pq):
    X, cb, codes, nlist = _raw_case()
    base = pq.IVFIndex.build_codes(dev(codes[:8000]), dev(cb), nlist, iters=3, seed=9)
    centers = base.centers().cpu().numpy()
    DT = orc.sdc_table(cb)
    lab, _ = orc.assign_codes(codes, DT, centers)
    grown = base.clone_empty()
    grown.add(dev(codes[:15_000]))
    part = base.clone_empty()
    part.add(dev(codes[15_000:]))
    grown.merge(part)
    assert_lists(grown, *lists_of(lab, codes, nlist))
    for i in (base, grown, part):
        i.close()


def test_merge_rejects_other_quantizers(pq):
    X, cb, codes, nlist = _raw_case()
    a = pq.IVFIndex.build(dev(X[:4000]), dev(codes[:4000]), nlist, iters=2, seed=3)
    b = pq.IVFIndex.build(dev(X[:4000]), dev(codes[:4000]), nlist, iters=2, seed=4)
    with pytest.raises(pq.PqError) as e:
        a.merge(b)
    assert e.value.status == pq.PQ_EINVAL
    a.close()
    b.close()
