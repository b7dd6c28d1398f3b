"""Pins for the FP64 oracle (CPU only).

Each test checks the oracle against something other than itself: a published
generator output, a library routine (scipy's vq/kmeans2/cdist, numpy sorts),
a hand-worked example, a closed form or an invariant of the method.  The
method is PQ as described in Sec. 2.1 (per-subspace k-means, encode, decode),
RMSE (Sec. 2.1/Sec. 3), the inverted index (Sec. 2.2) and the chunked fit
(Sec. 3).
"""
import os

import numpy as np
import pytest
from scipy.cluster.vq import kmeans2, vq
from scipy.spatial.distance import cdist

import oracle as orc
from paper_2604_21645_gb300 import datagen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sections(path):
    sec, out = None, {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.isalpha() and line.isupper():
            sec = line
            out[sec] = []
            continue
        out[sec].append([float(v) for v in line.split()])
    return out


# -- generator -------------------------------------------------------------------

def test_splitmix64_published_outputs():
    vals = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if not l.startswith("#")]
    assert [orc.sm64(0, i) for i in range(4)] == vals


def test_scale53_is_uniform_index():
    n = 1000
    assert orc.scale53(0, n) == 0
    assert orc.scale53((1 << 53) - 1, n) == n - 1
    idx = [orc.scale53(orc.draw(7, 3, i) >> 11, 10) for i in range(20000)]
    counts = np.bincount(idx, minlength=10)
    # chi-square with 9 dof: 99.9th percentile is 27.9
    chi2 = ((counts - 2000.0) ** 2 / 2000.0).sum()
    assert chi2 < 27.9


def test_streams_differ():
    a = [orc.draw(1, 0, i) for i in range(8)]
    b = [orc.draw(1, 1, i) for i in range(8)]
    assert len(set(a) & set(b)) == 0


# -- assignment and update (Sec. 2.1) ---------------------------------------------

def test_assign_matches_scipy_vq():
    rng = np.random.default_rng(0)
    X = rng.normal(size=(300, 12)).astype(np.float32)
    cb = rng.normal(size=(3, 20, 4)).astype(np.float32)
    codes, mind, gap = orc.assign(X, cb)
    for m in range(3):
        ref, dist = vq(X[:, 4 * m:4 * m + 4].astype(np.float64), cb[m].astype(np.float64))
        assert np.array_equal(codes[:, m], ref)
        np.testing.assert_allclose(mind[:, m], dist ** 2, rtol=1e-12)
        full = cdist(X[:, 4 * m:4 * m + 4].astype(np.float64), cb[m].astype(np.float64), "sqeuclidean")
        full.sort(axis=1)
        np.testing.assert_allclose(gap[:, m], full[:, 1] - full[:, 0], rtol=1e-9, atol=1e-12)


def test_assign_ties_go_to_lowest_index():
    X = np.array([[0.0, 0.0], [1.0, 1.0]], dtype=np.float32)
    cb = np.array([[[5.0, 5.0], [1.0, 1.0], [1.0, 1.0], [0.0, 0.0], [0.0, 0.0]]], dtype=np.float32)
    codes, _, gap = orc.assign(X, cb)
    assert codes[:, 0].tolist() == [3, 1]
    assert gap[:, 0].tolist() == [0.0, 0.0]
    # equal distance on both sides of a point
    X2 = np.array([[1.0]], dtype=np.float32)
    cb2 = np.array([[[2.0], [0.0]]], dtype=np.float32)
    assert orc.assign(X2, cb2)[0][0, 0] == 0


def test_update_is_the_mean_and_keeps_empty():
    rng = np.random.default_rng(1)
    X = rng.normal(size=(500, 6)).astype(np.float32)
    cb = rng.normal(size=(2, 9, 3)).astype(np.float32)
    codes = rng.integers(0, 8, size=(500, 2)).astype(np.int32)  # centroid 8 stays empty
    new, counts = orc.update(X, codes, cb)
    for m in range(2):
        sub = X[:, 3 * m:3 * m + 3].astype(np.float64)
        for k in range(9):
            sel = codes[:, m] == k
            assert counts[m, k] == sel.sum()
            if sel.any():
                assert np.array_equal(new[m, k], sub[sel].mean(axis=0).astype(np.float32)) or \
                    np.allclose(new[m, k], sub[sel].mean(axis=0), rtol=1e-7, atol=0)
            else:
                assert np.array_equal(new[m, k], cb[m, k])


def test_lloyd_single_subspace_is_plain_kmeans():
    """M = 1 reduces PQ fit to plain k-means; scipy's kmeans2 with a given init is the same Lloyd loop."""
    X = datagen.mixture(3000, 4, 6, "cont", 11).astype(np.float64)
    init = X[[5, 700, 1400, 2100, 2800, 2999]].copy()
    ours, _ = orc.pq_fit(X.astype(np.float32), 1, 6, 15, 0, init=init[None].astype(np.float32))
    ref, lab = kmeans2(X, init.copy(), iter=15, minit="matrix", missing="raise")
    np.testing.assert_allclose(ours[0], ref, rtol=2e-6, atol=2e-7)


def test_lloyd_subspaces_are_independent_kmeans():
    X = datagen.mixture(2000, 8, 5, "cont", 12)
    M, Ks = 2, 5
    init = np.stack([X[[1, 400, 800, 1200, 1600], 4 * m:4 * m + 4] for m in range(M)])
    ours, _ = orc.pq_fit(X, M, Ks, 10, 0, init=init)
    for m in range(M):
        ref, _ = kmeans2(X[:, 4 * m:4 * m + 4].astype(np.float64), init[m].astype(np.float64), iter=10,
                         minit="matrix", missing="raise")
        np.testing.assert_allclose(ours[m], ref, rtol=2e-6, atol=2e-7)


def test_lloyd_sse_never_increases():
    X = datagen.mixture(4000, 16, 12, "cont", 13)
    _, sse = orc.pq_fit(X, 4, 32, 20, 99)
    assert np.all(np.diff(sse) <= 1e-9 * sse[:-1])
    assert sse[-1] < sse[0]


def test_sse_matches_rmse_after_fit():
    X = datagen.mixture(1500, 8, 4, "cont", 14)
    cb, sse = orc.pq_fit(X, 2, 8, 5, 3)
    # an extra zero-iteration fit from the result: its assignment SSE equals N*D*RMSE^2
    codes = orc.pq_encode(X, cb)
    r = orc.pq_rmse(X, codes, cb)
    _, sse2 = orc.pq_fit(X, 2, 8, 1, 0, init=cb)
    np.testing.assert_allclose(sse2[0], r * r * X.size, rtol=1e-12)


# -- k-means++ seeding --------------------------------------------------------------

def test_kmeanspp_distinct_points_all_picked():
    """Ks equal to the number of distinct points: every point becomes a seed, so the error is 0."""
    rng = np.random.default_rng(2)
    X = rng.normal(size=(32, 6)).astype(np.float32)
    cb = orc.kmeanspp(X, 3, 32, 5)
    for m in range(3):
        got = {tuple(r) for r in cb[m]}
        want = {tuple(r) for r in X[:, 2 * m:2 * m + 2]}
        assert got == want
    codes = orc.pq_encode(X, cb)
    assert orc.pq_rmse(X, codes, cb) == 0.0


def test_kmeanspp_d2_sampling_frequencies():
    """Second seed drawn with probability proportional to the squared distance to the first."""
    X = np.array([[0.0], [1.0], [3.0], [6.0]], dtype=np.float32)
    trials = 12000
    first = np.zeros(4)
    second = np.zeros((4, 4))
    for s in range(trials):
        cb = orc.kmeanspp(X, 1, 2, s)
        i0 = int(np.where(X[:, 0] == cb[0, 0, 0])[0][0])
        i1 = int(np.where(X[:, 0] == cb[0, 1, 0])[0][0])
        first[i0] += 1
        second[i0, i1] += 1
    chi2 = ((first - trials / 4) ** 2 / (trials / 4)).sum()
    assert chi2 < 16.3  # 3 dof, 99.9th percentile
    for i0 in range(4):
        d2 = (X[:, 0] - X[i0, 0]) ** 2
        p = d2 / d2.sum()
        exp = p * first[i0]
        mask = exp > 0
        assert second[i0, ~mask].sum() == 0  # zero-weight points never drawn
        chi2 = ((second[i0, mask] - exp[mask]) ** 2 / exp[mask]).sum()
        assert chi2 < 16.3


def test_kmeanspp_single_positive_weight():
    X = np.array([[1.0], [1.0], [1.0], [9.0], [1.0]], dtype=np.float32)
    for s in range(50):
        cb = orc.kmeanspp(X, 1, 2, s)
        assert set(cb[0, :, 0].tolist()) == {1.0, 9.0}


def test_kmeanspp_subsample_rows_are_data_rows():
    X = datagen.mixture(30000, 4, 3, "cont", 15)  # N > 100*Ks for Ks = 8
    cb = orc.kmeanspp(X, 2, 8, 1)
    for m in range(2):
        sub = X[:, 2 * m:2 * m + 2]
        for r in cb[m]:
            assert np.any(np.all(sub == r, axis=1))


# -- encode / decode / RMSE (Sec. 2.1, Sec. 3) ---------------------------------------

def test_rmse_hand_worked_example():
    g = _sections(os.path.join(GOLDEN, "rmse_4x4.txt"))
    X = np.array(g["X"], dtype=np.float32)
    cb = np.zeros((2, 2, 2), dtype=np.float32)
    for m, k, a, b in g["CODEBOOK"]:
        cb[int(m), int(k)] = (a, b)
    codes = orc.pq_encode(X, cb)
    assert codes.tolist() == np.array(g["CODES"], dtype=np.uint8).tolist()
    np.testing.assert_allclose(orc.pq_rmse(X, codes, cb), g["RMSE"][0][0], rtol=1e-15)


def test_decode_reconstruction_and_zero_rmse():
    rng = np.random.default_rng(3)
    X = rng.normal(size=(16, 8)).astype(np.float32)
    cb = np.stack([X[:, 2 * m:2 * m + 2] for m in range(4)])  # every row is a codeword
    codes = orc.pq_encode(X, cb)
    assert np.array_equal(orc.pq_decode(codes, cb), X)
    assert orc.pq_rmse(X, codes, cb) == 0.0


def test_more_subspaces_or_codewords_lower_rmse():
    """Sec. 2.1: a larger M or Ks gives a lower reconstruction error (trend on mixture data)."""
    X = datagen.mixture(6000, 16, 64, "cont", 16)
    def rmse(M, Ks):
        cb, _ = orc.pq_fit(X, M, Ks, 8, 4)
        return orc.pq_rmse(X, orc.pq_encode(X, cb), cb)
    assert rmse(8, 16) < rmse(4, 16) < rmse(2, 16)
    assert rmse(4, 64) < rmse(4, 16) < rmse(4, 4)


# -- inverted index (Sec. 2.2, Sec. 3.1) ----------------------------------------------

def _small_index(seed=17, N=3000, D=16, M=4, Ks=16, nlist=12):
    X = datagen.mixture(N, D, 20, "int255", seed)
    cb, _ = orc.pq_fit(X, M, Ks, 6, seed)
    codes = orc.pq_encode(X, cb)
    idx = orc.ivf_build(X, codes, nlist, 6, seed + 1)
    return X, cb, codes, idx


def test_ivf_lists_partition_rows():
    X, cb, codes, idx = _small_index()
    off, ids = idx["offsets"], idx["ids"]
    assert off[0] == 0 and off[-1] == X.shape[0]
    assert np.array_equal(np.sort(ids), np.arange(X.shape[0]))
    lab = cdist(X.astype(np.float64), idx["coarse"].astype(np.float64), "sqeuclidean").argmin(axis=1)
    assert np.array_equal(idx["list_of_row"], lab)
    for l in range(len(off) - 1):
        seg = ids[off[l]:off[l + 1]]
        assert np.all(np.diff(seg) > 0)
        assert np.all(lab[seg] == l)
        assert np.array_equal(idx["list_codes"][off[l]:off[l + 1]], codes[seg])


def test_ivf_full_probe_equals_exhaustive_adc():
    X, cb, codes, idx = _small_index()
    Q = datagen.queries(40, X.shape[1], 20, "int255", 17)
    M, Ks, ds = cb.shape
    ids, dist, _ = orc.ivf_search(idx, cb, Q, nprobe=12, k=25)
    for q in range(Q.shape[0]):
        lut = np.stack([cdist(Q[q:q + 1, m * ds:(m + 1) * ds].astype(np.float64), cb[m].astype(np.float64),
                              "sqeuclidean")[0] for m in range(M)])
        adc = lut[np.arange(M)[None, :], codes].sum(axis=1)
        order = np.lexsort((np.arange(X.shape[0]), adc))[:25]
        assert np.array_equal(ids[q], order)
        np.testing.assert_allclose(dist[q], adc[order], rtol=1e-12)


def test_ivf_probe_order_and_padding():
    X, cb, codes, idx = _small_index()
    Q = datagen.queries(10, X.shape[1], 20, "int255", 18)
    ids, dist, probes = orc.ivf_search(idx, cb, Q, nprobe=3, k=X.shape[0])
    dc = cdist(Q.astype(np.float64), idx["coarse"].astype(np.float64), "sqeuclidean")
    for q in range(10):
        want = np.lexsort((np.arange(dc.shape[1]), dc[q]))[:3]
        assert np.array_equal(probes[q], want)
        n_cand = sum(idx["offsets"][l + 1] - idx["offsets"][l] for l in want)
        assert np.all(ids[q, n_cand:] == -1) and np.all(np.isinf(dist[q, n_cand:]))
        assert np.all(ids[q, :n_cand] >= 0)


def test_exact_knn_matches_cdist():
    X = datagen.mixture(800, 8, 5, "int255", 19)
    Q = datagen.queries(20, 8, 5, "int255", 19)
    ids, dist = orc.exact_knn(X, Q, 10)
    full = cdist(Q.astype(np.float64), X.astype(np.float64), "sqeuclidean")
    for q in range(20):
        order = np.lexsort((np.arange(800), full[q]))[:10]
        assert np.array_equal(ids[q], order)


# -- chunked divide and conquer (Sec. 3) ------------------------------------------------

def test_chunked_single_chunk_reduces_to_plain_fit():
    X = datagen.mixture(3000, 8, 10, "cont", 20)
    gC, codes, r, local = orc.pq_fit_chunked(X, [0, 3000], 2, 16, 6, 5)
    # the pooled dataset is the chunk's own codewords; the global fit on it reproduces them
    for m in range(2):
        assert {tuple(v) for v in gC[m]} == {tuple(v) for v in local[0, m]}
    codes_local = orc.pq_encode(X, local[0])
    np.testing.assert_allclose(r, orc.pq_rmse(X, codes_local, local[0]), rtol=1e-12)


def test_chunked_multi_chunk_decomposes_into_plain_fits():
    """Sec. 3 divide and conquer, step by step on four uneven chunks: chunk c's codebooks are the
    plain fit of its own rows seeded with draw c of the chunk stream; the global model is the plain
    fit, seeded with the caller's seed, of the centroid dataset whose row c*Ks + k concatenates
    codeword k of every subspace of chunk c; codes and RMSE are the global model's.  Catches a wrong
    chunk row offset, a wrong per-chunk seed and a wrong pooled-row layout."""
    X = datagen.mixture(9000, 12, 30, "cont", 22)
    off = np.array([0, 1700, 2300, 6100, 9000], dtype=np.int64)
    M, Ks, iters, seed = 3, 32, 4, 0x1234ABCD
    gC, codes, r, local = orc.pq_fit_chunked(X, off, M, Ks, iters, seed)
    n_chunks = len(off) - 1
    for c in range(n_chunks):
        seed_c = orc.draw(seed, 0xFFFFFFFE, c)
        want, _ = orc.pq_fit(X[off[c]:off[c + 1]], M, Ks, iters, seed_c)
        assert np.array_equal(local[c], want), f"chunk {c}"
    # the centroid dataset, assembled here from the local codebooks: [n_chunks*Ks][D]
    pooled = np.concatenate([np.concatenate([local[c, m] for m in range(M)], axis=1) for c in range(n_chunks)])
    assert pooled.shape == (n_chunks * Ks, X.shape[1])
    want_g, _ = orc.pq_fit(pooled, M, Ks, iters, seed)
    assert np.array_equal(gC, want_g)
    assert np.array_equal(codes, orc.pq_encode(X, want_g))
    assert r == orc.pq_rmse(X, codes, want_g)
    # chunks fitted on their own rows differ from one another (the offsets matter)
    assert not np.array_equal(local[0], local[1])


def test_chunked_rmse_close_to_single_fit():
    """Sec. 3: the global model fitted on pooled chunk codewords reconstructs about as well as one fit."""
    X = datagen.mixture(12000, 8, 24, "cont", 21)
    off = [0, 2500, 5200, 9000, 12000]
    _, _, r_chunk, _ = orc.pq_fit_chunked(X, off, 2, 16, 10, 6)
    cb, _ = orc.pq_fit(X, 2, 16, 10, 6)
    r_single = orc.pq_rmse(X, orc.pq_encode(X, cb), cb)
    assert abs(r_chunk - r_single) / r_single < 0.1


# -- soft-assignment refinement ------------------------------------------------------------

def test_softpq_gradients_match_finite_differences():
    rng = np.random.default_rng(4)
    X = rng.normal(size=(7, 6))
    cb = rng.normal(size=(2, 5, 3))
    tau = 0.7
    dC, dX = orc.softpq_backward(X, cb, tau)
    h = 1e-6
    for arr, grad in ((cb, dC), (X, dX)):
        num = np.zeros_like(arr)
        it = np.nditer(arr, flags=["multi_index"])
        for _ in it:
            i = it.multi_index
            old = arr[i]
            arr[i] = old + h
            lp = orc.softpq_forward(X, cb, tau)
            arr[i] = old - h
            lm = orc.softpq_forward(X, cb, tau)
            arr[i] = old
            num[i] = (lp - lm) / (2 * h)
        np.testing.assert_allclose(grad, num, rtol=1e-6, atol=1e-9)


def _fd4(f, x0, h):
    """Fourth-order central difference of f at x0 (truncation error O(h^4))."""
    return (f(x0 - 2 * h) - 8 * f(x0 - h) + 8 * f(x0 + h) - f(x0 + 2 * h)) / (12 * h)


@pytest.mark.slow
def test_softpq_gradients_match_finite_differences_at_refinement_size():
    """The refinement workload's shape (N=1000, D=256, M=32, Ks=256, tau=0.1) in FP64: 200
    seeded-random entries each of dL/dC and dL/dX against central finite differences, relative
    error below 1e-6.  L is a sum over subspaces and rows of the same function, so the
    difference quotient of an entry of subspace m is taken on that subspace's slice (and, for
    X, on its row: L = (1/N) sum_n L_n); eight entries are also checked on the full loss."""
    N, D, M, Ks, tau = 1000, 256, 32, 256, 0.1
    ds = D // M
    X = datagen.mixture(N, D, 256, "cont", 99).astype(np.float64)
    rng = np.random.default_rng(1)
    cb = X[rng.integers(0, N, Ks)].reshape(Ks, M, ds).transpose(1, 0, 2).copy()
    cb += 0.01 * rng.standard_normal(cb.shape)
    dC, dX = orc.softpq_backward(X, cb, tau)
    h = 1e-3
    worst = 0.0

    def check(num, ana):
        nonlocal worst
        err = abs(num - ana)
        assert err <= 1e-6 * abs(ana) + 1e-13, (num, ana)
        worst = max(worst, err / max(abs(ana), 1e-300))

    for _ in range(200):
        m, k, j = int(rng.integers(M)), int(rng.integers(Ks)), int(rng.integers(ds))
        Xs = np.ascontiguousarray(X[:, m * ds:(m + 1) * ds])

        def f_c(v):
            c = cb[m].copy()
            c[k, j] = v
            return orc.softpq_forward(Xs, c[None], tau)
        check(_fd4(f_c, cb[m, k, j], h), dC[m, k, j])
    for _ in range(200):
        n, d = int(rng.integers(N)), int(rng.integers(D))
        m = d // ds
        cm = cb[m][None].copy()

        def f_x(v):
            x = X[n:n + 1, m * ds:(m + 1) * ds].copy()
            x[0, d - m * ds] = v
            return orc.softpq_forward(x, cm, tau) / N
        check(_fd4(f_x, X[n, d], h), dX[n, d])
    # a few entries through the whole loss (all rows and subspaces)
    for e in range(8):
        arr, grad = (cb, dC) if e % 2 == 0 else (X, dX)
        i = tuple(int(rng.integers(s)) for s in arr.shape)
        old = arr[i]

        def f_full(v):
            arr[i] = v
            try:
                return orc.softpq_forward(X, cb, tau)
            finally:
                arr[i] = old
        check(_fd4(f_full, old, h), grad[i])
    print("largest relative error", worst)


def test_softpq_limits():
    rng = np.random.default_rng(5)
    X = rng.normal(size=(50, 4))
    cb = rng.normal(size=(2, 6, 2))
    # tau -> 0: hard assignment, loss = SSE / N
    X32 = X.astype(np.float32)
    cb32 = cb.astype(np.float32)
    _, mind, gap = orc.assign(X32, cb32)
    tau0 = gap.min() / 200.0  # second-best weight below exp(-200)
    hard = orc.softpq_forward(X32.astype(np.float64), cb32.astype(np.float64), tau0)
    np.testing.assert_allclose(hard, mind.sum() / 50, rtol=1e-9)
    # tau -> inf: uniform weights, xhat = mean codeword
    big = orc.softpq_forward(X, cb, 1e12)
    mean_cw = np.concatenate([cb[m].mean(axis=0) for m in range(2)])
    np.testing.assert_allclose(big, ((X - mean_cw) ** 2).sum() / 50, rtol=1e-9)


# -- weighted centroid dataset (Sec. 3 variant) ----------------------------------------------

def test_pq_fit_counts_are_the_last_update_members():
    X = datagen.mixture(4000, 8, 10, "cont", 60)
    C, cnt = orc.pq_fit_counts(X, 2, 16, 5, 61)
    ref, _ = orc.pq_fit(X, 2, 16, 5, 61)
    assert np.array_equal(C, ref)
    prev, _ = orc.pq_fit(X, 2, 16, 4, 61)
    codes, _, _ = orc.assign(X, prev)
    for m in range(2):
        assert np.array_equal(cnt[m], np.bincount(codes[:, m], minlength=16))
    upd, _ = orc.update(X, codes, prev)
    assert np.array_equal(upd, C)
    # each chunk codeword is the mean of its members: the count-weighted mean of the codewords is
    # the mean of all rows
    for m in range(2):
        wmean = (cnt[m][:, None] * C[m].astype(np.float64)).sum(axis=0) / cnt[m].sum()
        np.testing.assert_allclose(wmean, X[:, 4 * m:4 * m + 4].astype(np.float64).mean(axis=0), rtol=1e-6, atol=1e-7)


def test_pq_fit_weighted_unit_weights_is_the_plain_fit():
    X = datagen.mixture(3000, 12, 10, "cont", 62)
    C = orc.pq_fit_weighted(X, np.ones((3000, 3), dtype=np.int64), 3, 16, 6, 63)
    ref, _ = orc.pq_fit(X, 3, 16, 6, 63)
    assert np.array_equal(C, ref)


def test_pq_fit_weighted_update_is_a_weighted_mean_and_weights_are_multiplicities():
    rng = np.random.default_rng(64)
    P = datagen.mixture(600, 8, 6, "cont", 64)
    W = rng.integers(0, 4, size=(600, 2)).astype(np.int64)
    W[:, 1] = W[:, 0]  # the same multiplicity in both subspaces
    C0 = orc.kmeanspp(P, 2, 8, 65)
    C1 = orc.pq_fit_weighted(P, W, 2, 8, 1, 65)
    codes, _, _ = orc.assign(P, C0)
    for m in range(2):
        for k in range(8):
            sel = codes[:, m] == k
            w = W[sel, m].astype(np.float64)
            if w.sum() == 0:
                assert np.array_equal(C1[m, k], C0[m, k])
                continue
            ref = (w[:, None] * P[sel, 4 * m:4 * m + 4].astype(np.float64)).sum(axis=0) / w.sum()
            np.testing.assert_allclose(C1[m, k], ref, rtol=2e-7, atol=1e-7)
    # the same step on the data with every point repeated W times (weight = multiplicity)
    Pe = np.repeat(P, W[:, 0], axis=0)
    ce = np.repeat(codes, W[:, 0], axis=0)
    upd, _ = orc.update(Pe, ce, C0)
    np.testing.assert_allclose(C1, upd, rtol=2e-7, atol=1e-7)


def test_chunked_weighted_decomposes_into_weighted_fits():
    X = datagen.mixture(8000, 12, 30, "cont", 66)
    off = np.array([0, 1500, 4000, 8000], dtype=np.int64)
    M, Ks, iters, seed = 3, 32, 4, 67
    gC, codes, r, local, W = orc.pq_fit_chunked_weighted(X, off, M, Ks, iters, seed)
    gu, _, ru, local_u = orc.pq_fit_chunked(X, off, M, Ks, iters, seed)
    assert np.array_equal(local, local_u)  # the same local fits
    for c in range(3):
        Cc, cnt = orc.pq_fit_counts(X[off[c]:off[c + 1]], M, Ks, iters, orc.draw(seed, 0xFFFFFFFE, c))
        assert np.array_equal(Cc, local[c])
        assert np.array_equal(W[c * Ks:(c + 1) * Ks], cnt.T)
        assert W[c * Ks:(c + 1) * Ks].sum(axis=0).tolist() == [off[c + 1] - off[c]] * M
    pooled = np.concatenate([np.concatenate([local[c, m] for m in range(M)], axis=1) for c in range(3)])
    want = orc.pq_fit_weighted(pooled, W, M, Ks, iters, seed)
    assert np.array_equal(gC, want)
    assert np.array_equal(codes, orc.pq_encode(X, want))
    assert r == orc.pq_rmse(X, codes, want)
    print("RMSE weighted", r, "unweighted", ru)


# -- optimized PQ ------------------------------------------------------------------------------

def _random_rotation(d, seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).standard_normal((d, d)))
    return q * np.sign(np.diag(r))


def test_opq_procrustes_recovers_a_known_rotation():
    X = datagen.mixture(2000, 16, 8, "cont", 70).astype(np.float64)
    Q = _random_rotation(16, 71)
    R = orc.opq_procrustes(X, X @ Q)
    np.testing.assert_allclose(R, Q, atol=1e-10)
    # and it minimises ||X R - Y|| over rotations: no random rotation does better
    Y = X @ Q + 0.05 * np.random.default_rng(72).standard_normal(X.shape)
    R = orc.opq_procrustes(X, Y)
    best = np.linalg.norm(X @ R - Y)
    for s in range(20):
        assert np.linalg.norm(X @ _random_rotation(16, 100 + s) - Y) >= best
    np.testing.assert_allclose(R @ R.T, np.eye(16), atol=1e-12)


def test_opq_fit_distortion_never_rises_and_zero_rounds_is_plain_pq():
    # rows with correlated dimensions, where a rotation helps PQ
    base = datagen.mixture(4000, 16, 12, "cont", 73).astype(np.float64)
    X = (base @ _random_rotation(16, 74) * np.linspace(2.0, 0.2, 16)).astype(np.float32)
    R0, cb0, _ = orc.opq_fit(X, 4, 16, 0, 5, 75)
    assert np.array_equal(R0, np.eye(16, dtype=np.float32))
    ref, _ = orc.pq_fit(X, 4, 16, 5, 75)
    assert np.array_equal(cb0, ref)
    R, cb, dist = orc.opq_fit(X, 4, 16, 6, 3, 75)
    assert np.all(np.diff(dist) <= 1e-6 * dist[0])
    np.testing.assert_allclose(R.astype(np.float64) @ R.T, np.eye(16), atol=1e-5)
    Y = orc.opq_rotate(X, R)
    r_opq = orc.pq_rmse(Y, orc.pq_encode(Y, cb), cb)
    r_pq = orc.pq_rmse(X, orc.pq_encode(X, ref), ref)
    assert r_opq < r_pq  # the rotation lowers the reconstruction error on correlated data
