"""Pins of the oracle's code-space inverted index (Rii's index over the PQ codes, Sec. 3.1).

Each function is checked against something other than itself: scipy's distance routine,
the squared distance of the two reconstructions, brute-force enumeration over members and
centres on small inputs, the monotone objective of the alternating minimisation, the
uniformity of the centre draw, and exhaustive ADC for a full probe.
"""
import numpy as np
import pytest
from scipy.spatial.distance import cdist
from scipy.stats import chisquare

import oracle as orc
from paper_2604_21645_gb300 import datagen


def _small(n=1500, d=16, m=4, ks=16, seed=40):
    X = datagen.mixture(n, d, 12, "cont", seed)
    cb, _ = orc.pq_fit(X, m, ks, 4, seed + 1)
    codes = orc.pq_encode(X, cb)
    return X, cb, codes


def test_sdc_table_matches_cdist():
    _, cb, _ = _small()
    DT = orc.sdc_table(cb)
    for m in range(cb.shape[0]):
        ref = cdist(cb[m].astype(np.float64), cb[m].astype(np.float64), "sqeuclidean")
        np.testing.assert_allclose(DT[m], ref, rtol=1e-12, atol=1e-15)
        assert np.all(np.diag(DT[m]) == 0.0)


def test_sdc_is_the_distance_of_the_reconstructions():
    _, cb, codes = _small()
    DT = orc.sdc_table(cb)
    rng = np.random.default_rng(0)
    a = codes[rng.integers(0, len(codes), 50)]
    b = codes[rng.integers(0, len(codes), 50)]
    sdc = np.array([sum(DT[m, a[i, m], b[i, m]] for m in range(cb.shape[0])) for i in range(50)])
    xa = orc.pq_decode(a, cb).astype(np.float64)
    xb = orc.pq_decode(b, cb).astype(np.float64)
    np.testing.assert_allclose(sdc, ((xa - xb) ** 2).sum(axis=1), rtol=1e-12)


def test_assign_codes_brute_force_and_ties():
    _, cb, codes = _small()
    DT = orc.sdc_table(cb)
    rng = np.random.default_rng(1)
    centers = codes[rng.choice(len(codes), 20, replace=False)].copy()
    centers[7] = centers[3]  # duplicate centre: ties must go to the lower index
    lst, dist = orc.assign_codes(codes, DT, centers)
    M = cb.shape[0]
    full = np.zeros((len(codes), len(centers)))
    for m in range(M):
        full += DT[m][codes[:, m][:, None], centers[:, m][None, :]]
    np.testing.assert_array_equal(lst, np.argmin(full, axis=1))  # argmin returns the first minimum
    np.testing.assert_allclose(dist, full.min(axis=1), rtol=1e-12)
    assert not np.any(lst == 7)


def test_update_centers_brute_force_over_members():
    _, cb, codes = _small(n=600)
    DT = orc.sdc_table(cb)
    M, Ks = cb.shape[0], cb.shape[1]
    rng = np.random.default_rng(2)
    nlist = 9
    centers = codes[rng.choice(len(codes), nlist, replace=False)].copy()
    lists = rng.integers(0, nlist - 1, len(codes)).astype(np.int32)  # list nlist-1 stays empty
    got = orc.update_centers(codes, DT, lists, centers)
    for l in range(nlist):
        members = np.nonzero(lists == l)[0]
        for m in range(M):
            if members.size == 0:
                assert got[l, m] == centers[l, m]
                continue
            cost = np.array([sum(DT[m, k, codes[n, m]] for n in members) for k in range(Ks)])
            assert got[l, m] == int(np.argmin(cost)), (l, m)


def test_pick_distinct_is_a_uniform_sample():
    for seed in range(20):
        p = orc.pick_distinct(1000, 50, seed)
        assert len(set(p.tolist())) == 50 and p.min() >= 0 and p.max() < 1000
    assert sorted(orc.pick_distinct(7, 7, 3).tolist()) == list(range(7))
    counts = np.zeros(10)
    for seed in range(4000):
        counts[orc.pick_distinct(10, 3, seed)] += 1
    assert chisquare(counts).pvalue > 1e-3  # every element drawn with probability 3/10


def test_build_codes_objective_and_lists():
    X, cb, codes = _small(n=3000)
    idx = orc.ivf_build_codes(codes, cb, 24, 8, 5)
    obj = idx["obj"]
    assert np.all(np.diff(obj) <= 1e-9 * obj[0])  # each round never raises the total SDC
    DT = orc.sdc_table(cb)
    lst, _ = orc.assign_codes(codes, DT, idx["centers"])
    np.testing.assert_array_equal(idx["list_of_row"], lst)
    off, ids = idx["offsets"], idx["ids"]
    assert off[0] == 0 and off[-1] == len(codes)
    for l in range(24):
        seg = ids[off[l]:off[l + 1]]
        assert np.all(np.diff(seg) > 0) and np.all(lst[seg] == l)
        np.testing.assert_array_equal(idx["list_codes"][off[l]:off[l + 1]], codes[seg])
    # starting centres: rows drawn by pick_distinct; zero rounds keep them
    idx0 = orc.ivf_build_codes(codes, cb, 24, 0, 5)
    np.testing.assert_array_equal(idx0["centers"], codes[orc.pick_distinct(len(codes), 24, 5)])


def test_search_codes_full_probe_is_exhaustive_adc():
    X, cb, codes = _small(n=2000)
    idx = orc.ivf_build_codes(codes, cb, 16, 4, 6)
    Q = datagen.queries(25, X.shape[1], 12, "cont", 40)
    M, Ks, ds = cb.shape
    ids, dist, probes = orc.ivf_search_codes(idx, cb, Q, 16, 30)
    ids3, dist3, probes3 = orc.ivf_search_codes(idx, cb, Q, 3, 2000)
    for q in range(len(Q)):
        lut = np.stack([cdist(Q[q:q + 1, m * ds:(m + 1) * ds].astype(np.float64), cb[m].astype(np.float64),
                              "sqeuclidean")[0] for m in range(M)])
        adc = lut[np.arange(M)[None, :], codes].sum(axis=1)
        order = np.lexsort((np.arange(len(codes)), adc))[:30]
        np.testing.assert_array_equal(ids[q], order)
        np.testing.assert_allclose(dist[q], adc[order], rtol=1e-12)
        # probe order: ADC of the query to the centre codes, ties to the lower list
        cadc = lut[np.arange(M)[None, :], idx["centers"]].sum(axis=1)
        np.testing.assert_array_equal(probes3[q], np.lexsort((np.arange(16), cadc))[:3])
        n_cand = sum(idx["offsets"][l + 1] - idx["offsets"][l] for l in probes3[q])
        assert np.all(ids3[q, n_cand:] == -1) and np.all(ids3[q, :n_cand] >= 0)
