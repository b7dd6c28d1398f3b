"""ctypes binding of ``libpqgb.so`` (C ABI in ``include/pqgb.h``).

Argument marshalling only: tensors are checked for device, dtype, shape and
contiguity and their device pointers are passed with the current CUDA stream.
Every step of the computation runs in the library's kernels; there is no CPU
or PyTorch fallback, and importing this module raises if the library has not
been built.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpqgb.so")

PQ_OK, PQ_EINVAL, PQ_ENOMEM, PQ_ECUDA, PQ_ETIMEOUT, PQ_ENOTSUP, PQ_EINTERNAL = 0, -1, -2, -3, -4, -5, -6
PQ_PREC_FP32, PQ_PREC_BF16 = 0, 1
PREC = {"fp32": PQ_PREC_FP32, "bf16": PQ_PREC_BF16}
STATS_MAX_ITERS = 64
EXPORTS = ("pq_fit", "pq_init_kmeanspp", "pq_encode", "pq_decode_rmse", "ivf_build", "ivf_search", "ivf_get_info",
           "ivf_copy_coarse", "ivf_copy_lists", "ivf_free", "pq_sync_status", "pq_last_error", "pq_launch_count",
           "pq_profile_enable", "pq_profile_collect", "pq_profile_names", "pq_lloyd_noalloc", "pq_fit_chunked",
           "softpq_forward", "softpq_backward", "pq_tune_chunked", "pq_tune_clear", "pq_fit_encode_host",
           "pq_test_set_spin_limit", "pq_test_fail_alloc_after", "ivf_build_codes", "ivf_copy_centers",
           "ivf_clone_empty", "ivf_add", "ivf_merge", "pq_fit_chunked_weighted", "opq_fit", "opq_rotate",
           "opq_procrustes")


class PqStats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("reserved", C.c_int32), ("fp64_rechecks", C.c_int64),
                ("empty_clusters", C.c_int64), ("kernel_launches", C.c_int64),
                ("sse", C.c_double * STATS_MAX_ITERS)]

    def as_dict(self):
        return {"iters": self.iters, "fp64_rechecks": self.fp64_rechecks, "empty_clusters": self.empty_clusters,
                "kernel_launches": self.kernel_launches, "sse": list(self.sse[:self.iters])}


class PqError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libpqgb status {status}: {msg}")
        self.status = status


def load_library(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    p, i64, i32, u64, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_uint64, C.c_double
    sigs = {
        "pq_fit": (i32, [p, i64, i32, i32, i32, i32, u64, i32, p, p, C.POINTER(PqStats), p]),
        "pq_init_kmeanspp": (i32, [p, i64, i32, i32, i32, u64, p, p]),
        "pq_encode": (i32, [p, i64, i32, i32, i32, p, i32, p, p, C.POINTER(PqStats), p]),
        "pq_decode_rmse": (i32, [p, p, p, i64, i32, i32, i32, p, C.POINTER(dbl), p]),
        "ivf_build": (i32, [p, p, i64, i32, i32, i32, i32, u64, i32, C.POINTER(p), p]),
        "ivf_search": (i32, [p, p, i32, p, i64, i32, i32, p, p, p]),
        "ivf_get_info": (i32, [p, C.POINTER(i64), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]),
        "ivf_copy_coarse": (i32, [p, p, p]),
        "ivf_copy_lists": (i32, [p, p, p, p, p]),
        "ivf_free": (None, [p]),
        "pq_sync_status": (i32, [p]),
        "pq_last_error": (C.c_char_p, []),
        "pq_launch_count": (i64, []),
        "pq_profile_enable": (i32, [i32]),
        "pq_profile_collect": (i32, [C.c_char_p, C.POINTER(i64), C.POINTER(dbl)]),
        "pq_profile_names": (i32, [C.c_char_p, i32]),
        "pq_lloyd_noalloc": (i32, [p, i64, i32, i32, i32, i32, p, p, p]),
        "pq_fit_chunked": (i32, [p, C.POINTER(i64), i32, i32, i32, i32, i32, u64, i32, p, p, C.POINTER(dbl), p]),
        "softpq_forward": (i32, [p, i64, i32, i32, i32, p, C.c_float, p, p]),
        "pq_tune_chunked": (i32, [p, C.POINTER(i64), i32, i32, i32, i32, i32, C.POINTER(i32), C.POINTER(C.c_float), p]),
        "pq_tune_clear": (i32, []),
        "softpq_backward": (i32, [p, i64, i32, i32, i32, p, C.c_float, p, p, p, p]),
        "pq_fit_encode_host": (i32, [p, i64, i32, i32, i32, i32, u64, i32, p, p, p]),
        "pq_test_set_spin_limit": (i32, [C.c_uint32]),
        "pq_test_fail_alloc_after": (i32, [i32]),
        "ivf_build_codes": (i32, [p, p, i64, i32, i32, i32, i32, i32, u64, i32, C.POINTER(p), p]),
        "ivf_copy_centers": (i32, [p, p, p]),
        "ivf_clone_empty": (i32, [p, C.POINTER(p)]),
        "ivf_add": (i32, [p, p, p, i64, i32, p]),
        "ivf_merge": (i32, [p, p, p]),
        "pq_fit_chunked_weighted": (i32, [p, C.POINTER(i64), i32, i32, i32, i32, i32, u64, i32, p, p,
                                          C.POINTER(dbl), p]),
        "opq_fit": (i32, [p, i64, i32, i32, i32, i32, i32, u64, i32, p, p, p]),
        "opq_rotate": (i32, [p, i64, i32, p, p, p]),
        "opq_procrustes": (i32, [p, p, i64, i32, p, p]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = load_library()


def lib() -> C.CDLL:
    return _lib


def _check(status):
    if status != PQ_OK:
        raise PqError(status, _lib.pq_last_error().decode(errors="replace"))


def _stream(t: torch.Tensor | None = None):
    dev = t.device if t is not None else torch.device("cuda", torch.cuda.current_device())
    return C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _need(t, dtype, ndim, name):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if t.dim() != ndim:
        raise ValueError(f"{name} must have {ndim} dims, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


def launch_count() -> int:
    return _lib.pq_launch_count()


def profile_enable(on: bool = True):
    """Start (clearing old records) or stop per-kernel CUDA-event timing inside the library."""
    _check(_lib.pq_profile_enable(1 if on else 0))


def profile_collect() -> dict:
    """{kernel name: {"launches": n, "ms": summed device time}} of the recorded launches (synchronizes)."""
    buf = C.create_string_buffer(8192)
    _check(_lib.pq_profile_names(buf, len(buf)))
    out = {}
    for name in filter(None, buf.value.decode().split(",")):
        cnt, ms = C.c_int64(), C.c_double()
        _check(_lib.pq_profile_collect(name.encode(), C.byref(cnt), C.byref(ms)))
        out[name] = {"launches": cnt.value, "ms": ms.value}
    return out


def sync_status(stream=None):
    _check(_lib.pq_sync_status(stream if stream is not None else _stream()))


def init_kmeanspp(X: torch.Tensor, M: int, Ks: int, seed: int) -> torch.Tensor:
    """k-means++ seeding of the M subspace codebooks (the first step of ``fit``)."""
    px = _need(X, torch.float32, 2, "X")
    N, D = X.shape
    cb = torch.empty((M, Ks, D // M), dtype=torch.float32, device=X.device)
    with torch.cuda.device(X.device):
        _check(_lib.pq_init_kmeanspp(px, N, D, M, Ks, seed & (2**64 - 1), C.c_void_p(cb.data_ptr()), _stream(X)))
    return cb


def fit(X: torch.Tensor, M: int, Ks: int = 256, iters: int = 20, seed: int = 0, prec: str = "fp32",
        init: torch.Tensor | None = None, out: torch.Tensor | None = None, stats: bool = False):
    """PQ fit (Sec. 2.1): returns codebooks [M][Ks][D/M] (and a stats dict if ``stats``)."""
    px = _need(X, torch.float32, 2, "X")
    N, D = X.shape
    if out is None:
        out = torch.empty((M, Ks, D // M), dtype=torch.float32, device=X.device)
    po = _need(out, torch.float32, 3, "out")
    pi = _need(init, torch.float32, 3, "init") if init is not None else None
    st = PqStats() if stats else None
    with torch.cuda.device(X.device):
        _check(_lib.pq_fit(px, N, D, M, Ks, iters, seed & (2**64 - 1), PREC[prec], pi, po,
                           C.byref(st) if st is not None else None, _stream(X)))
    return (out, st.as_dict()) if stats else out


def _need_pinned(t, dtype, ndim, name):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.is_cuda or not t.is_pinned():
        raise ValueError(f"{name} must be a CPU tensor in pinned memory")
    if t.dtype != dtype or t.dim() != ndim or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {ndim}-dim {dtype} tensor")
    return C.c_void_p(t.data_ptr())


def fit_encode_host(X: torch.Tensor, M: int, Ks: int = 256, iters: int = 20, seed: int = 0, prec: str = "fp32",
                    codebooks: torch.Tensor | None = None, codes: torch.Tensor | None = None, want_codes: bool = True,
                    device=None, sync: bool = True):
    """fit + encode of pinned host rows in one call (``pq_fit_encode_host``).

    The seeding reads its subsample from host memory while X is copied to the device on a
    second stream.  Returns pinned CPU tensors (codebooks [M][Ks][D/M], codes [N][M] or None);
    with ``sync=False`` they are complete once the device's current stream has passed the call.
    """
    px = _need_pinned(X, torch.float32, 2, "X")
    N, D = X.shape
    if codebooks is None:
        codebooks = torch.empty((M, Ks, D // M), dtype=torch.float32).pin_memory()
    pcb = _need_pinned(codebooks, torch.float32, 3, "codebooks")
    pcd = None
    if want_codes:
        if codes is None:
            codes = torch.empty((N, M), dtype=torch.uint8).pin_memory()
        pcd = _need_pinned(codes, torch.uint8, 2, "codes")
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    with torch.cuda.device(dev):
        st = C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
        _check(_lib.pq_fit_encode_host(px, N, D, M, Ks, iters, seed & (2**64 - 1), PREC[prec], pcb, pcd, st))
        if sync:
            torch.cuda.current_stream(dev).synchronize()
    return codebooks, (codes if want_codes else None)


def lloyd_noalloc(X: torch.Tensor, init: torch.Tensor, iters: int, out: torch.Tensor | None = None) -> torch.Tensor:
    """Lloyd iterations from ``init`` without any device allocation inside the library.

    For callers that must not allocate device memory during the call (memory reserved up
    front by their own allocator, or a latency-bound loop): the scratch is a fixed array
    inside the library.  ``out`` (allocate it beforehand) receives the codebooks.
    Concurrent calls that overlap on the GPU share that array and must be serialized.
    """
    px = _need(X, torch.float32, 2, "X")
    pi = _need(init, torch.float32, 3, "init")
    N, D = X.shape
    M, Ks, _ = init.shape
    if out is None:
        out = torch.empty_like(init)
    po = _need(out, torch.float32, 3, "out")
    with torch.cuda.device(X.device):
        _check(_lib.pq_lloyd_noalloc(px, N, D, M, Ks, iters, pi, po, _stream(X)))
    return out


def fit_chunked(X: torch.Tensor, chunk_offsets, M: int, Ks: int = 256, iters: int = 20, seed: int = 0,
                prec: str = "fp32", want_rmse: bool = True, weighted: bool = False):
    """Divide-and-conquer PQ (Sec. 3): per-chunk fits, pooled codewords, global refit, global encode.

    ``chunk_offsets`` is a host sequence of n_chunks + 1 row offsets.  ``weighted`` weights each
    pooled codeword by its member count in its chunk's last update.  Returns
    (global codebooks [M][Ks][D/M], codes [N][M] uint8, RMSE or None).
    """
    px = _need(X, torch.float32, 2, "X")
    N, D = X.shape
    off = (C.c_int64 * len(chunk_offsets))(*[int(v) for v in chunk_offsets])
    n_chunks = len(chunk_offsets) - 1
    if n_chunks < 1 or off[n_chunks] != N:
        raise ValueError("chunk_offsets must end at N")
    cb = torch.empty((M, Ks, D // M), dtype=torch.float32, device=X.device)
    codes = torch.empty((N, M), dtype=torch.uint8, device=X.device)
    r = C.c_double(0.0)
    with torch.cuda.device(X.device):
        fn = _lib.pq_fit_chunked_weighted if weighted else _lib.pq_fit_chunked
        _check(fn(px, off, n_chunks, D, M, Ks, iters, seed & (2**64 - 1), PREC[prec], C.c_void_p(cb.data_ptr()),
                  C.c_void_p(codes.data_ptr()), C.byref(r) if want_rmse else None, _stream(X)))
    return cb, codes, (r.value if want_rmse else None)


def opq_fit(X: torch.Tensor, M: int, Ks: int = 256, outer: int = 5, pq_iters: int = 5, seed: int = 0,
            prec: str = "fp32"):
    """Optimized PQ: (R [D][D], codebooks [M][Ks][D/M]) with the codebooks those of X R."""
    px = _need(X, torch.float32, 2, "X")
    N, D = X.shape
    R = torch.empty((D, D), dtype=torch.float32, device=X.device)
    cb = torch.empty((M, Ks, D // M), dtype=torch.float32, device=X.device)
    with torch.cuda.device(X.device):
        _check(_lib.opq_fit(px, N, D, M, Ks, outer, pq_iters, seed & (2**64 - 1), PREC[prec],
                            C.c_void_p(R.data_ptr()), C.c_void_p(cb.data_ptr()), _stream(X)))
    return R, cb


def opq_rotate(X: torch.Tensor, R: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    """X R (rows rotated into the space the OPQ codebooks quantize)."""
    px = _need(X, torch.float32, 2, "X")
    pr = _need(R, torch.float32, 2, "R")
    if out is None:
        out = torch.empty_like(X)
    po = _need(out, torch.float32, 2, "out")
    with torch.cuda.device(X.device):
        _check(_lib.opq_rotate(px, X.shape[0], X.shape[1], pr, po, _stream(X)))
    return out


def opq_procrustes(X: torch.Tensor, Y: torch.Tensor) -> torch.Tensor:
    """The orthogonal R minimising ||X R - Y||_F."""
    px = _need(X, torch.float32, 2, "X")
    py = _need(Y, torch.float32, 2, "Y")
    D = X.shape[1]
    R = torch.empty((D, D), dtype=torch.float32, device=X.device)
    with torch.cuda.device(X.device):
        _check(_lib.opq_procrustes(px, py, X.shape[0], D, C.c_void_p(R.data_ptr()), _stream(X)))
    return R


def softpq_forward(X: torch.Tensor, codebooks: torch.Tensor, tau: float, out: torch.Tensor | None = None):
    """Soft-assignment reconstruction loss L (device float32 scalar); see softpq.SoftPQLoss."""
    px = _need(X, torch.float32, 2, "X")
    pc = _need(codebooks, torch.float32, 3, "codebooks")
    N, D = X.shape
    M, Ks, _ = codebooks.shape
    if out is None:
        out = torch.empty((), dtype=torch.float32, device=X.device)
    po = _need(out, torch.float32, 0, "loss")
    with torch.cuda.device(X.device):
        _check(_lib.softpq_forward(px, N, D, M, Ks, pc, float(tau), po, _stream(X)))
    return out


def softpq_backward(X: torch.Tensor, codebooks: torch.Tensor, tau: float, grad_loss: torch.Tensor | None = None,
                    need_dx: bool = True):
    """(dL/dcodebooks, dL/dX or None), scaled by the device scalar ``grad_loss`` when given."""
    px = _need(X, torch.float32, 2, "X")
    pc = _need(codebooks, torch.float32, 3, "codebooks")
    N, D = X.shape
    M, Ks, _ = codebooks.shape
    pg = _need(grad_loss, torch.float32, 0, "grad_loss") if grad_loss is not None else None
    dC = torch.empty_like(codebooks)
    dX = torch.empty_like(X) if need_dx else None
    with torch.cuda.device(X.device):
        _check(_lib.softpq_backward(px, N, D, M, Ks, pc, float(tau), pg, C.c_void_p(dC.data_ptr()),
                                    C.c_void_p(dX.data_ptr()) if dX is not None else None, _stream(X)))
    return dC, dX


def tune_chunked(X: torch.Tensor, chunk_offsets, M: int, Ks: int = 256, prec: str = "fp32"):
    """Autotune the batched pass of fit_chunked for this shape; returns (CTAs per subspace group, pass ms)."""
    px = _need(X, torch.float32, 2, "X")
    N, D = X.shape
    off = (C.c_int64 * len(chunk_offsets))(*[int(v) for v in chunk_offsets])
    n_chunks = len(chunk_offsets) - 1
    if n_chunks < 1 or off[n_chunks] != N:
        raise ValueError("chunk_offsets must end at N")
    ctas, ms = C.c_int32(0), C.c_float(0.0)
    with torch.cuda.device(X.device):
        _check(_lib.pq_tune_chunked(px, off, n_chunks, D, M, Ks, PREC[prec], C.byref(ctas), C.byref(ms), _stream(X)))
    return ctas.value, ms.value


def tune_clear():
    _check(_lib.pq_tune_clear())


def encode(X: torch.Tensor, codebooks: torch.Tensor, prec: str = "fp32", out: torch.Tensor | None = None,
           sse: torch.Tensor | None = None, stats: bool = False):
    """PQ encode (Sec. 2.1): uint8 codes [N][M]; ``sse`` (device float64 [1]) receives sum (x - xhat)^2."""
    px = _need(X, torch.float32, 2, "X")
    pc = _need(codebooks, torch.float32, 3, "codebooks")
    N, D = X.shape
    M, Ks, _ = codebooks.shape
    if out is None:
        out = torch.empty((N, M), dtype=torch.uint8, device=X.device)
    po = _need(out, torch.uint8, 2, "codes")
    ps = _need(sse, torch.float64, 1, "sse") if sse is not None else None
    st = PqStats() if stats else None
    with torch.cuda.device(X.device):
        _check(_lib.pq_encode(px, N, D, M, Ks, pc, PREC[prec], po, ps, C.byref(st) if st is not None else None,
                              _stream(X)))
    return (out, st.as_dict()) if stats else out


def decode_rmse(codes: torch.Tensor, codebooks: torch.Tensor, X: torch.Tensor | None = None,
                want_xhat: bool = False):
    """Decode and RMSE (Sec. 2.1, Sec. 3): returns (xhat or None, rmse or None)."""
    pcodes = _need(codes, torch.uint8, 2, "codes")
    pc = _need(codebooks, torch.float32, 3, "codebooks")
    N, M = codes.shape
    _, Ks, ds = codebooks.shape
    D = M * ds
    px = _need(X, torch.float32, 2, "X") if X is not None else None
    xhat = torch.empty((N, D), dtype=torch.float32, device=codes.device) if want_xhat else None
    r = C.c_double(0.0)
    with torch.cuda.device(codes.device):
        _check(_lib.pq_decode_rmse(pcodes, pc, px, N, D, M, Ks, C.c_void_p(xhat.data_ptr()) if xhat is not None
                                   else None, C.byref(r) if X is not None else None, _stream(codes)))
    return xhat, (r.value if X is not None else None)


class IVFIndex:
    """Inverted-file index over PQ codes (Sec. 2.2, Sec. 3.1); owns a library handle."""

    def __init__(self, handle: int, device: torch.device):
        self._h = C.c_void_p(handle)
        self.device = device
        N, D, M, nl = C.c_int64(), C.c_int32(), C.c_int32(), C.c_int32()
        _check(_lib.ivf_get_info(self._h, C.byref(N), C.byref(D), C.byref(M), C.byref(nl)))
        self.N, self.D, self.M, self.nlist = N.value, D.value, M.value, nl.value

    @classmethod
    def build(cls, X: torch.Tensor, codes: torch.Tensor, nlist: int, iters: int = 25, seed: int = 0,
              prec: str = "fp32") -> "IVFIndex":
        px = _need(X, torch.float32, 2, "X")
        pc = _need(codes, torch.uint8, 2, "codes")
        N, D = X.shape
        M = codes.shape[1]
        h = C.c_void_p()
        with torch.cuda.device(X.device):
            _check(_lib.ivf_build(px, pc, N, D, M, nlist, iters, seed & (2**64 - 1), PREC[prec], C.byref(h),
                                  _stream(X)))
        return cls(h.value, X.device)

    @classmethod
    def build_codes(cls, codes: torch.Tensor, codebooks: torch.Tensor, nlist: int, iters: int = 25, seed: int = 0,
                    prec: str = "fp32") -> "IVFIndex":
        """Code-space index (Rii): centre codes by k-means over the PQ codes, lists by symmetric distance."""
        pc = _need(codes, torch.uint8, 2, "codes")
        pb = _need(codebooks, torch.float32, 3, "codebooks")
        N, M = codes.shape
        _, Ks, ds = codebooks.shape
        h = C.c_void_p()
        with torch.cuda.device(codes.device):
            _check(_lib.ivf_build_codes(pc, pb, N, M * ds, M, Ks, nlist, iters, seed & (2**64 - 1), PREC[prec],
                                        C.byref(h), _stream(codes)))
        idx = cls(h.value, codes.device)
        idx.code_space = True
        return idx

    code_space = False

    def centers(self) -> torch.Tensor:
        """Centre codes [nlist][M] of a code-space index."""
        out = torch.empty((self.nlist, self.M), dtype=torch.uint8, device=self.device)
        with torch.cuda.device(self.device):
            _check(_lib.ivf_copy_centers(self._h, C.c_void_p(out.data_ptr()), _stream(out)))
        return out

    def clone_empty(self) -> "IVFIndex":
        """A new index with the same coarse quantizer and no rows."""
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            _check(_lib.ivf_clone_empty(self._h, C.byref(h)))
        idx = IVFIndex(h.value, self.device)
        idx.code_space = self.code_space
        return idx

    def add(self, codes: torch.Tensor, X: torch.Tensor | None = None, prec: str = "fp32"):
        """Appends rows (ids N, N+1, ...) to the lists of their nearest coarse centres."""
        pc = _need(codes, torch.uint8, 2, "codes")
        px = _need(X, torch.float32, 2, "X") if X is not None else None
        with torch.cuda.device(codes.device):
            _check(_lib.ivf_add(self._h, px, pc, codes.shape[0], PREC[prec], _stream(codes)))
        self._refresh()
        return self

    def merge(self, other: "IVFIndex"):
        """Appends every row of `other` (same coarse quantizer), its ids shifted past this index's rows."""
        with torch.cuda.device(self.device):
            _check(_lib.ivf_merge(self._h, other._h, _stream()))
        self._refresh()
        return self

    def _refresh(self):
        N = C.c_int64()
        _check(_lib.ivf_get_info(self._h, C.byref(N), None, None, None))
        self.N = N.value

    def search(self, codebooks: torch.Tensor, Q: torch.Tensor, nprobe: int, k: int, out_ids=None, out_d=None):
        pc = _need(codebooks, torch.float32, 3, "codebooks")
        pq = _need(Q, torch.float32, 2, "Q")
        nq = Q.shape[0]
        if out_ids is None:
            out_ids = torch.empty((nq, k), dtype=torch.int64, device=Q.device)
        if out_d is None:
            out_d = torch.empty((nq, k), dtype=torch.float32, device=Q.device)
        pi = _need(out_ids, torch.int64, 2, "ids")
        pd = _need(out_d, torch.float32, 2, "dists")
        with torch.cuda.device(Q.device):
            _check(_lib.ivf_search(self._h, pc, codebooks.shape[1], pq, nq, nprobe, k, pi, pd, _stream(Q)))
        return out_ids, out_d

    def coarse(self) -> torch.Tensor:
        out = torch.empty((self.nlist, self.D), dtype=torch.float32, device=self.device)
        with torch.cuda.device(self.device):
            _check(_lib.ivf_copy_coarse(self._h, C.c_void_p(out.data_ptr()), _stream(out)))
        return out

    def lists(self):
        off = torch.empty(self.nlist + 1, dtype=torch.int64, device=self.device)
        ids = torch.empty(self.N, dtype=torch.int64, device=self.device)
        codes = torch.empty((self.N, self.M), dtype=torch.uint8, device=self.device)
        with torch.cuda.device(self.device):
            _check(_lib.ivf_copy_lists(self._h, C.c_void_p(off.data_ptr()), C.c_void_p(ids.data_ptr()),
                                       C.c_void_p(codes.data_ptr()), _stream(off)))
        return off, ids, codes

    def close(self):
        if self._h:
            _lib.ivf_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
