"""Failure detection without a GPU fault: a device-side wait that runs out, and a scratch
allocation that fails, both reported through the C ABI's status codes.

The wait is the k-means++ seeding's inter-block barrier (a poll of global memory; the
seeding has no bulk copies in flight), with its poll budget lowered to one poll so that
the blocks that arrive first give up.  Every block then returns, the error word holds
PQ_ETIMEOUT, pq_sync_status reports and clears it, and the next call succeeds.  The
allocation failure is injected on the host: the call returns PQ_ENOMEM before it
launches anything, and the next call succeeds.
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


def test_seeding_wait_that_runs_out_reports_timeout(pq):
    X = datagen.mixture(60_000, 32, 20, "cont", 31)
    Xd = torch.from_numpy(X).cuda()
    M, Ks, seed = 4, 64, 77
    pq.sync_status()
    timeouts = 0
    try:
        for _ in range(3):
            pq.lib().pq_test_set_spin_limit(1)
            pq.init_kmeanspp(Xd, M, Ks, seed)  # enqueued; the failure is asynchronous
            try:
                pq.sync_status()
            except pq.PqError as e:
                assert e.status == pq.PQ_ETIMEOUT
                timeouts += 1
                break
    finally:
        pq.lib().pq_test_set_spin_limit(0)
    assert timeouts == 1
    pq.sync_status()  # the error word was cleared
    got = pq.init_kmeanspp(Xd, M, Ks, seed)
    pq.sync_status()
    assert np.array_equal(got.cpu().numpy(), orc.kmeanspp(X, M, Ks, seed))


@pytest.mark.parametrize("after", [0, 2])
def test_injected_allocation_failure_returns_enomem(pq, after):
    X = datagen.mixture(20_000, 32, 20, "cont", 32)
    Xd = torch.from_numpy(X).cuda()
    l0 = pq.launch_count()
    try:
        pq.lib().pq_test_fail_alloc_after(after)
        with pytest.raises(pq.PqError) as e:
            pq.fit(Xd, 4, 32, iters=2, seed=3)
        assert e.value.status == pq.PQ_ENOMEM
        assert b"injected" in pq.lib().pq_last_error()
    finally:
        pq.lib().pq_test_fail_alloc_after(-1)
    assert pq.launch_count() == l0  # the call stopped before its first kernel
    pq.sync_status()
    got = pq.fit(Xd, 4, 32, iters=2, seed=3)
    ref, _ = orc.pq_fit(X, 4, 32, 2, 3)
    np.testing.assert_allclose(got.cpu().numpy(), ref, rtol=0, atol=1e-5 * np.abs(ref).max())


def test_persistent_batched_fit_wait_that_runs_out_reports_timeout(pq):
    """The persistent batched fit: a unit of pass t + 1 waits for the previous pass of its (chunk,
    subspace group).  Here a pass has fewer units than there are resident CTAs, so CTAs take
    pass-1 units while pass 0 still runs; with a one-poll budget those waits run out, the CTAs
    leave, the call finishes, and pq_sync_status reports PQ_ETIMEOUT once.  The next call, with
    the default budget, gives the same model as a call before the failure."""
    X = datagen.mixture(200_000, 32, 20, "cont", 33)
    Xd = torch.from_numpy(X).cuda()
    off = [0, 90_000, 200_000]
    M, Ks = 4, 64
    pq.tune_clear()
    pq.sync_status()
    ref_cb, ref_codes, _ = pq.fit_chunked(Xd, off, M, Ks, iters=6, seed=5, prec="bf16", want_rmse=False)
    pq.sync_status()
    ref_cb, ref_codes = ref_cb.clone(), ref_codes.clone()
    try:
        pq.lib().pq_test_set_spin_limit(1)
        pq.fit_chunked(Xd, off, M, Ks, iters=6, seed=5, prec="bf16", want_rmse=False)
        with pytest.raises(pq.PqError) as e:
            pq.sync_status()
        assert e.value.status == pq.PQ_ETIMEOUT
    finally:
        pq.lib().pq_test_set_spin_limit(0)
    pq.sync_status()  # the error word was cleared
    cb, codes, _ = pq.fit_chunked(Xd, off, M, Ks, iters=6, seed=5, prec="bf16", want_rmse=False)
    pq.sync_status()
    assert torch.equal(cb, ref_cb) and torch.equal(codes, ref_codes)
