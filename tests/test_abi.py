"""The C ABI library loads, exports every declared entry point, and rejects bad
arguments before touching the GPU (CPU only: no compute call is made)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pqgb.h")
LIB = os.path.join(ROOT, "paper_2604_21645_gb300", "libpqgb.so")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b((?:pq|ivf|softpq|opq)_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        import __graft_entry__
        __graft_entry__.build()
    return C.CDLL(LIB)


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert "pq_fit" in names and "ivf_search" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_exports_match_header():
    from paper_2604_21645_gb300 import pqgb
    assert sorted(pqgb.EXPORTS) == declared()


def _status(lib, name, *args):
    f = getattr(lib, name)
    f.restype = C.c_int
    return f(*args)


def test_argument_errors_before_any_launch(lib):
    lib.pq_last_error.restype = C.c_char_p
    vp = C.c_void_p
    i64 = C.c_int64
    # D not a multiple of M
    assert _status(lib, "pq_fit", vp(16), i64(1000), 30, 4, 256, 5, C.c_uint64(0), 0, None, vp(16), None,
                   None) == -1
    assert b"multiple" in lib.pq_last_error()
    # Ks out of range
    assert _status(lib, "pq_fit", vp(16), i64(1000), 32, 4, 257, 5, C.c_uint64(0), 0, None, vp(16), None,
                   None) == -1
    # N < Ks
    assert _status(lib, "pq_fit", vp(16), i64(100), 32, 4, 256, 5, C.c_uint64(0), 0, None, vp(16), None,
                   None) == -1
    # null codebooks
    assert _status(lib, "pq_fit", vp(16), i64(1000), 32, 4, 256, 5, C.c_uint64(0), 0, None, None, None,
                   None) == -1
    # unknown precision
    assert _status(lib, "pq_fit", vp(16), i64(1000), 32, 4, 256, 5, C.c_uint64(0), 7, None, vp(16), None,
                   None) == -1
    # misaligned X
    assert _status(lib, "pq_fit", vp(18), i64(1000), 32, 4, 256, 5, C.c_uint64(0), 0, None, vp(16), None,
                   None) == -1
    assert b"aligned" in lib.pq_last_error()
    # too many iterations
    assert _status(lib, "pq_fit", vp(16), i64(1000), 32, 4, 256, 65, C.c_uint64(0), 0, None, vp(16), None,
                   None) == -1
    # decode with nothing to do
    assert _status(lib, "pq_decode_rmse", vp(16), vp(16), None, i64(10), 32, 4, 256, None, None, None) == -1
    # ivf: nlist > N, null handle
    assert _status(lib, "ivf_build", vp(16), vp(16), i64(10), 32, 4, 11, 5, C.c_uint64(0), 0, C.byref(vp()),
                   None) == -1
    assert _status(lib, "ivf_build", vp(16), vp(16), i64(10), 32, 4, 2, 5, C.c_uint64(0), 0, None, None) == -1
    # search on a null index
    assert _status(lib, "ivf_search", None, vp(16), 256, vp(16), i64(4), 1, 10, vp(16), vp(16), None) == -1
    # chunked form and its tuner: chunk smaller than Ks, offsets not starting at 0
    off = (C.c_int64 * 3)(0, 10, 1000)
    assert _status(lib, "pq_fit_chunked", vp(16), off, 2, 32, 4, 64, 5, C.c_uint64(0), 0, vp(16), vp(16), None,
                   None) == -1
    off2 = (C.c_int64 * 2)(5, 1000)
    assert _status(lib, "pq_tune_chunked", vp(16), off2, 1, 32, 4, 64, 0, None, None, None) == -1
    # soft PQ: tau must be positive, Ds must be 4, 8 or 16
    f = lib.softpq_forward
    f.restype = C.c_int
    f.argtypes = [vp, i64, C.c_int32, C.c_int32, C.c_int32, vp, C.c_float, vp, vp]
    assert f(vp(16), 10, 64, 8, 256, vp(16), 0.0, vp(16), None) == -1
    assert f(vp(16), 10, 96, 8, 256, vp(16), 0.1, vp(16), None) == -5


def test_launch_counter_starts_at_zero(lib):
    lib.pq_launch_count.restype = C.c_int64
    assert lib.pq_launch_count() >= 0


def test_host_input_call_checks_its_tensors_before_any_launch():
    import torch

    from paper_2604_21645_gb300 import pqgb
    X = torch.zeros((512, 32), dtype=torch.float32)  # pageable CPU memory
    with pytest.raises(ValueError):
        pqgb.fit_encode_host(X, 4, 16)
    with pytest.raises(TypeError):
        pqgb.fit_encode_host(X.numpy(), 4, 16)
