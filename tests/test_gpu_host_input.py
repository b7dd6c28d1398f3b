"""pq_fit_encode_host: fit + encode of rows in page-locked host memory, the seeding reading its
subsample from host memory while the matrix is copied to the device.  Its codebooks and codes
are identical to those of the device calls on the same rows (which are pinned to the oracle by
the fit and encode parity tests)."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2604_21645_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_21645_gb300 import pqgb
    return pqgb


@pytest.mark.parametrize("prec,N,D,M,Ks", [("bf16", 50_011, 64, 8, 256), ("fp32", 30_007, 96, 12, 256),
                                           ("bf16", 26_000, 128, 16, 256), ("fp32", 3_001, 32, 4, 16)])
def test_host_input_matches_device_calls(pq, prec, N, D, M, Ks):
    X = datagen.mixture(N, D, 50, "cont", 9100 + N)
    Xh = torch.from_numpy(X).pin_memory()
    cb_h, codes_h = pq.fit_encode_host(Xh, M, Ks, iters=4, seed=77, prec=prec)
    Xd = torch.from_numpy(X).cuda()
    cb = pq.fit(Xd, M, Ks, iters=4, seed=77, prec=prec)
    codes = pq.encode(Xd, cb, prec=prec)
    assert torch.equal(cb_h, cb.cpu())
    assert torch.equal(codes_h, codes.cpu())


def test_host_input_without_codes_and_async(pq):
    X = datagen.mixture(20_000, 64, 30, "int255", 9201)
    Xh = torch.from_numpy(X).pin_memory()
    cb_h, none = pq.fit_encode_host(Xh, 8, 256, iters=2, seed=5, prec="bf16", want_codes=False, sync=False)
    torch.cuda.current_stream().synchronize()
    assert none is None
    cb = pq.fit(torch.from_numpy(X).cuda(), 8, 256, iters=2, seed=5, prec="bf16")
    assert torch.equal(cb_h, cb.cpu())


def test_host_input_rejects_pageable_memory(pq):
    X = np.zeros((1000, 32), dtype=np.float32)  # ordinary (pageable) host memory
    cb = torch.empty((4, 16, 8), dtype=torch.float32).pin_memory()
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = pq.lib().pq_fit_encode_host(C.c_void_p(X.ctypes.data), 1000, 32, 4, 16, 2, 1, pq.PQ_PREC_FP32,
                                     C.c_void_p(cb.data_ptr()), None, st)
    assert rc == pq.PQ_EINVAL
    with pytest.raises(ValueError):
        pq.fit_encode_host(torch.from_numpy(X), 4, 16)
