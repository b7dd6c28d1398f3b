"""pq_lloyd_noalloc: the allocation-free Lloyd iterations, checked against pq_fit.

Some callers cannot let a library allocate device memory during a call (their
GPU memory is reserved up front by their own allocator, or an allocation in a
latency-bound loop could block or fail).  For them pq_lloyd_noalloc keeps its
scratch in a fixed array compiled into the library.  This test calls it through
the C ABI twice in a row, on different inputs, and compares each result with
pq_fit's and the oracle's from the same initial codebooks at the codeword
tolerance used by the other parity tests (1e-5 relative), and reads the device's
free memory and its stream-ordered pool around the second call to show that the
call allocates nothing.  Because every call shares the fixed array,
the second call also shows that nothing stale from the first leaks into it.
The file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle as orc
from paper_2604_21645_gb300 import datagen
from tests.parity import assert_codebooks_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_21645_gb300 import pqgb
    return pqgb


def _noalloc_via_abi(pq, X, init, iters, out=None):
    out = torch.empty_like(init) if out is None else out
    N, D = X.shape
    M, Ks, _ = init.shape
    st = pq.lib().pq_lloyd_noalloc(C.c_void_p(X.data_ptr()), N, D, M, Ks, iters, C.c_void_p(init.data_ptr()),
                                   C.c_void_p(out.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == pq.PQ_OK, pq.lib().pq_last_error()
    torch.cuda.synchronize()
    return out


class _DeviceMemory:
    """Device memory seen through the CUDA driver: free bytes, and the in-use high watermark of the
    device's default stream-ordered pool (the pool cudaMallocAsync draws from)."""

    USED_MEM_HIGH = 8  # CU_MEMPOOL_ATTR_USED_MEM_HIGH

    def __init__(self):
        self.cu = C.CDLL("libcuda.so.1")
        dev = C.c_int()
        assert self.cu.cuDeviceGet(C.byref(dev), torch.cuda.current_device()) == 0
        self.pool = C.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(C.byref(self.pool), dev) == 0

    def free_bytes(self):
        free, total = C.c_size_t(), C.c_size_t()
        assert self.cu.cuMemGetInfo_v2(C.byref(free), C.byref(total)) == 0
        return free.value

    def reset_pool_high(self):
        zero = C.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH, C.byref(zero)) == 0

    def pool_high(self):
        v = C.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, self.USED_MEM_HIGH, C.byref(v)) == 0
        return v.value


@pytest.mark.parametrize("n,d,m,ks,kind", [(50_000, 128, 16, 256, "int255")])
def test_noalloc_matches_pq_fit_on_two_calls(pq, n, d, m, ks, kind):
    cases = [
        datagen.mixture(n, d, 200, kind, 901),
        datagen.mixture(12_345, 64, 32, "cont", 902),
    ]
    shapes = [(m, ks), (8, 100)]
    mem = _DeviceMemory()
    for call, (X, (M, Ks)) in enumerate(zip(cases, shapes)):
        init = orc.kmeanspp(X, M, Ks, 5)
        Xd = torch.from_numpy(X).cuda()
        initd = torch.from_numpy(init).cuda()
        got = torch.empty_like(initd)
        torch.cuda.synchronize()
        mem.reset_pool_high()
        free0 = mem.free_bytes()
        _noalloc_via_abi(pq, Xd, initd, 3, got)
        if call == 1:
            # the first call on the device may load the library's code and look up its array; from
            # the second call on, nothing is allocated: no free memory taken, no pool memory in use
            assert mem.free_bytes() == free0
            assert mem.pool_high() == 0
        want = pq.fit(Xd, M, Ks, iters=3, init=initd)
        assert_codebooks_close(got.cpu().numpy(), want.cpu().numpy())
        ref, _ = orc.pq_fit(X, M, Ks, 3, 0, init=init)
        assert_codebooks_close(got.cpu().numpy(), ref)


def test_noalloc_rejects_unsupported_width_before_any_work(pq):
    X = torch.zeros((300, 48), dtype=torch.float32, device="cuda")
    init = torch.ones((2, 16, 24), dtype=torch.float32, device="cuda")  # Ds = 24
    out = torch.zeros_like(init)
    st = pq.lib().pq_lloyd_noalloc(C.c_void_p(X.data_ptr()), 300, 48, 2, 16, 1, C.c_void_p(init.data_ptr()),
                                   C.c_void_p(out.data_ptr()), None)
    torch.cuda.synchronize()
    assert st == pq.PQ_ENOTSUP
    assert torch.count_nonzero(out).item() == 0  # the codebook copy was not enqueued


def test_noalloc_rejects_shapes_beyond_its_scratch(pq):
    # One block per subspace needs M*Ks*(8*Ds + 4) bytes: D=4096, M=128 (Ds=32), Ks=256 needs 8.5 MB > 8 MiB.
    X = torch.zeros((256, 4096), dtype=torch.float32, device="cuda")
    init = torch.zeros((128, 256, 32), dtype=torch.float32, device="cuda")
    out = torch.empty_like(init)
    st = pq.lib().pq_lloyd_noalloc(C.c_void_p(X.data_ptr()), 256, 4096, 128, 256, 1, C.c_void_p(init.data_ptr()),
                                   C.c_void_p(out.data_ptr()), None)
    assert st == pq.PQ_EINVAL
    assert b"fixed scratch" in pq.lib().pq_last_error()
