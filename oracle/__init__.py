"""FP64 CPU oracle for the PQ + IVF-ADC path (ctypes wrapper over ``pq_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only
callers.  The CUDA library never imports, links or runs anything here, and this
module imports nothing from the CUDA package.

Every function restates a step of the method described in Sec. 2.1 (PQ fit,
encode, decode), Sec. 2.1/Sec. 3 (RMSE), Sec. 2.2 and Sec. 3.1 (inverted index,
k-nearest query) and Sec. 3 (chunked fit, centroid dataset, global refit); the
readings taken where the paper is silent are listed in the C source header.

Parity pins: all functions are pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (brute force on tiny inputs, library routines,
closed forms, invariants, the published SplitMix64 output).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pq_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc if it is missing or older than its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            p = C.c_void_p
            i64, i32, u64, dbl = C.c_int64, C.c_int, C.c_uint64, C.c_double
            sig = {
                "orc_sm64": (u64, [u64, u64]),
                "orc_draw": (u64, [u64, u64, u64]),
                "orc_scale53": (i64, [u64, i64]),
                "orc_kmeanspp": (i32, [p, i64, i32, i32, i32, u64, p]),
                "orc_assign": (None, [p, i64, i32, i32, i32, p, p, p, p]),
                "orc_update": (i32, [p, i64, i32, i32, i32, p, p, p]),
                "orc_pq_fit": (i32, [p, i64, i32, i32, i32, i32, u64, p, p, p]),
                "orc_pq_encode": (i32, [p, i64, i32, i32, i32, p, p]),
                "orc_pq_decode": (None, [p, i64, i32, i32, i32, p, p]),
                "orc_pq_rmse": (dbl, [p, p, i64, i32, i32, i32, p]),
                "orc_ivf_build": (i32, [p, p, i64, i32, i32, i32, i32, u64, p, p, p, p, p]),
                "orc_ivf_search": (i32, [p, p, p, p, i32, i32, i32, i32, p, p, i64, i32, i32, p, p, p]),
                "orc_exact_knn": (i32, [p, i64, i32, p, i64, i32, p, p]),
                "orc_pq_fit_chunked": (i32, [p, p, i32, i32, i32, i32, i32, u64, p, p, p, p]),
                "orc_softpq_forward": (dbl, [p, i64, i32, i32, i32, p, dbl]),
                "orc_softpq_backward": (None, [p, i64, i32, i32, i32, p, dbl, p, p]),
                "orc_num_threads": (i32, []),
                "orc_pq_fit_counts": (i32, [p, i64, i32, i32, i32, i32, u64, p, p]),
                "orc_pq_fit_weighted": (i32, [p, p, i64, i32, i32, i32, i32, u64, p]),
                "orc_pq_fit_chunked_weighted": (i32, [p, p, i32, i32, i32, i32, i32, u64, p, p, p, p, p]),
                "orc_sdc_table": (None, [p, i32, i32, i32, p]),
                "orc_pick_distinct": (i32, [i64, i32, u64, p]),
                "orc_assign_codes": (None, [p, i64, i32, i32, p, p, i32, p, p]),
                "orc_update_centers": (i32, [p, i64, i32, i32, p, p, i32, p]),
                "orc_ivf_build_codes": (i32, [p, i64, i32, i32, i32, p, i32, i32, u64, p, p, p, p, p, p]),
                "orc_ivf_search_codes": (i32, [p, p, p, p, i32, i32, i32, i32, p, p, i64, i32, i32, p, p, p]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def num_threads() -> int:
    return _load().orc_num_threads()


# -- counter-based generator ---------------------------------------------------

def sm64(seed: int, i: int) -> int:
    """Output number i of a SplitMix64 generator seeded with ``seed``."""
    return _load().orc_sm64(seed & (2**64 - 1), i)


def draw(seed: int, stream: int, i: int) -> int:
    return _load().orc_draw(seed & (2**64 - 1), stream, i)


def scale53(r53: int, n: int) -> int:
    return _load().orc_scale53(r53, n)


# -- PQ (Sec. 2.1) -------------------------------------------------------------

def kmeanspp(X, M: int, Ks: int, seed: int) -> np.ndarray:
    X = _f32(X)
    N, D = X.shape
    out = np.empty((M, Ks, D // M), dtype=np.float32)
    _check(_load().orc_kmeanspp(_ptr(X), N, D, M, Ks, seed & (2**64 - 1), _ptr(out)), "kmeanspp")
    return out


def assign(X, codebooks):
    """Nearest codeword per (row, subspace): (codes int32, min distance, top-two gap)."""
    X = _f32(X)
    cb = _f32(codebooks)
    N, D = X.shape
    M, Ks, _ = cb.shape
    codes = np.empty((N, M), dtype=np.int32)
    mind = np.empty((N, M), dtype=np.float64)
    gap = np.empty((N, M), dtype=np.float64)
    _load().orc_assign(_ptr(X), N, D, M, Ks, _ptr(cb), _ptr(codes), _ptr(mind), _ptr(gap))
    return codes, mind, gap


def update(X, codes, codebooks):
    """One centroid update; returns (new codebooks, member counts)."""
    X = _f32(X)
    cb = _f32(codebooks).copy()
    codes = np.ascontiguousarray(codes, dtype=np.int32)
    N, D = X.shape
    M, Ks, _ = cb.shape
    counts = np.empty((M, Ks), dtype=np.int64)
    _check(_load().orc_update(_ptr(X), N, D, M, Ks, _ptr(codes), _ptr(cb), _ptr(counts)), "update")
    return cb, counts


def pq_fit(X, M: int, Ks: int, iters: int, seed: int, init=None):
    """PQ fit; returns (codebooks [M][Ks][Ds] float32, per-iteration SSE)."""
    X = _f32(X)
    N, D = X.shape
    out = np.empty((M, Ks, D // M), dtype=np.float32)
    sse = np.zeros(max(iters, 1), dtype=np.float64)
    init_a = None if init is None else _f32(init)
    _check(_load().orc_pq_fit(_ptr(X), N, D, M, Ks, iters, seed & (2**64 - 1), _ptr(init_a), _ptr(out),
                              _ptr(sse)), "pq_fit")
    return out, sse[:iters]


def pq_encode(X, codebooks) -> np.ndarray:
    X = _f32(X)
    cb = _f32(codebooks)
    N, D = X.shape
    M, Ks, _ = cb.shape
    codes = np.empty((N, M), dtype=np.uint8)
    _check(_load().orc_pq_encode(_ptr(X), N, D, M, Ks, _ptr(cb), _ptr(codes)), "pq_encode")
    return codes


def pq_decode(codes, codebooks) -> np.ndarray:
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    cb = _f32(codebooks)
    N, M = codes.shape
    _, Ks, ds = cb.shape
    out = np.empty((N, M * ds), dtype=np.float32)
    _load().orc_pq_decode(_ptr(codes), N, M * ds, M, Ks, _ptr(cb), _ptr(out))
    return out


def pq_rmse(X, codes, codebooks) -> float:
    X = _f32(X)
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    cb = _f32(codebooks)
    N, D = X.shape
    M, Ks, _ = cb.shape
    return _load().orc_pq_rmse(_ptr(X), _ptr(codes), N, D, M, Ks, _ptr(cb))


# -- inverted index (Sec. 2.2, Sec. 3.1) -----------------------------------------

def ivf_build(X, codes, nlist: int, iters: int, seed: int):
    """Returns dict(coarse, offsets, ids, list_codes, list_of_row)."""
    X = _f32(X)
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    N, D = X.shape
    M = codes.shape[1]
    coarse = np.empty((nlist, D), dtype=np.float32)
    offsets = np.empty(nlist + 1, dtype=np.int64)
    ids = np.empty(N, dtype=np.int64)
    lc = np.empty((N, M), dtype=np.uint8)
    lor = np.empty(N, dtype=np.int32)
    _check(_load().orc_ivf_build(_ptr(X), _ptr(codes), N, D, M, nlist, iters, seed & (2**64 - 1), _ptr(coarse),
                                 _ptr(offsets), _ptr(ids), _ptr(lc), _ptr(lor)), "ivf_build")
    return {"coarse": coarse, "offsets": offsets, "ids": ids, "list_codes": lc, "list_of_row": lor}


def ivf_search(index, codebooks, Q, nprobe: int, k: int):
    """Returns (ids int64 [nq][k], ADC distances float64 [nq][k], probed lists int32 [nq][nprobe])."""
    Q = _f32(Q)
    cb = _f32(codebooks)
    nq, D = Q.shape
    M, Ks, _ = cb.shape
    nlist = index["coarse"].shape[0]
    ids = np.empty((nq, k), dtype=np.int64)
    dist = np.empty((nq, k), dtype=np.float64)
    probes = np.empty((nq, nprobe), dtype=np.int32)
    _check(_load().orc_ivf_search(_ptr(_f32(index["coarse"])), _ptr(index["offsets"]), _ptr(index["ids"]),
                                  _ptr(index["list_codes"]), nlist, D, M, Ks, _ptr(cb), _ptr(Q), nq, nprobe, k,
                                  _ptr(ids), _ptr(dist), _ptr(probes)), "ivf_search")
    return ids, dist, probes


def exact_knn(X, Q, k: int):
    X = _f32(X)
    Q = _f32(Q)
    N, D = X.shape
    nq = Q.shape[0]
    ids = np.empty((nq, k), dtype=np.int64)
    dist = np.empty((nq, k), dtype=np.float64)
    _check(_load().orc_exact_knn(_ptr(X), N, D, _ptr(Q), nq, k, _ptr(ids), _ptr(dist)), "exact_knn")
    return ids, dist


# -- code-space coarse quantizer (Rii, Sec. 3.1) ---------------------------------

def sdc_table(codebooks) -> np.ndarray:
    """DT[m][k][j] = ||c_{m,k} - c_{m,j}||^2 (FP64)."""
    cb = _f32(codebooks)
    M, Ks, ds = cb.shape
    DT = np.empty((M, Ks, Ks), dtype=np.float64)
    _load().orc_sdc_table(_ptr(cb), M, Ks, ds, _ptr(DT))
    return DT


def pick_distinct(N: int, nlist: int, seed: int) -> np.ndarray:
    out = np.empty(nlist, dtype=np.int64)
    _check(_load().orc_pick_distinct(N, nlist, seed & (2**64 - 1), _ptr(out)), "pick_distinct")
    return out


def assign_codes(codes, DT, centers):
    """Nearest centre code of every row code by symmetric distance: (lists int32, SDC float64)."""
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    centers = np.ascontiguousarray(centers, dtype=np.uint8)
    DT = np.ascontiguousarray(DT, dtype=np.float64)
    N, M = codes.shape
    Ks = DT.shape[1]
    lst = np.empty(N, dtype=np.int32)
    dist = np.empty(N, dtype=np.float64)
    _load().orc_assign_codes(_ptr(codes), N, M, Ks, _ptr(DT), _ptr(centers), centers.shape[0], _ptr(lst), _ptr(dist))
    return lst, dist


def update_centers(codes, DT, lists, centers):
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    out = np.ascontiguousarray(centers, dtype=np.uint8).copy()
    DT = np.ascontiguousarray(DT, dtype=np.float64)
    lists = np.ascontiguousarray(lists, dtype=np.int32)
    N, M = codes.shape
    _check(_load().orc_update_centers(_ptr(codes), N, M, DT.shape[1], _ptr(DT), _ptr(lists), out.shape[0],
                                      _ptr(out)), "update_centers")
    return out


def ivf_build_codes(codes, codebooks, nlist: int, iters: int, seed: int):
    """Code-space index.  Returns dict(centers, offsets, ids, list_codes, list_of_row, obj)."""
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    cb = _f32(codebooks)
    N, M = codes.shape
    _, Ks, ds = cb.shape
    centers = np.empty((nlist, M), dtype=np.uint8)
    offsets = np.empty(nlist + 1, dtype=np.int64)
    ids = np.empty(N, dtype=np.int64)
    lc = np.empty((N, M), dtype=np.uint8)
    lor = np.empty(N, dtype=np.int32)
    obj = np.zeros(max(iters, 1), dtype=np.float64)
    _check(_load().orc_ivf_build_codes(_ptr(codes), N, M, Ks, ds, _ptr(cb), nlist, iters, seed & (2**64 - 1),
                                       _ptr(centers), _ptr(offsets), _ptr(ids), _ptr(lc), _ptr(lor), _ptr(obj)),
           "ivf_build_codes")
    return {"centers": centers, "offsets": offsets, "ids": ids, "list_codes": lc, "list_of_row": lor,
            "obj": obj[:iters]}


def ivf_search_codes(index, codebooks, Q, nprobe: int, k: int):
    """Returns (ids int64 [nq][k], ADC distances float64 [nq][k], probed lists int32 [nq][nprobe])."""
    Q = _f32(Q)
    cb = _f32(codebooks)
    nq, D = Q.shape
    M, Ks, _ = cb.shape
    centers = np.ascontiguousarray(index["centers"], dtype=np.uint8)
    nlist = centers.shape[0]
    ids = np.empty((nq, k), dtype=np.int64)
    dist = np.empty((nq, k), dtype=np.float64)
    probes = np.empty((nq, nprobe), dtype=np.int32)
    _check(_load().orc_ivf_search_codes(_ptr(centers), _ptr(index["offsets"]), _ptr(index["ids"]),
                                        _ptr(index["list_codes"]), nlist, D, M, Ks, _ptr(cb), _ptr(Q), nq, nprobe,
                                        k, _ptr(ids), _ptr(dist), _ptr(probes)), "ivf_search_codes")
    return ids, dist, probes


# -- chunked divide and conquer (Sec. 3) -----------------------------------------

def pq_fit_chunked(X, chunk_offsets, M: int, Ks: int, iters: int, seed: int):
    """Returns (global codebooks, codes, RMSE, local codebooks [n_chunks][M][Ks][Ds])."""
    X = _f32(X)
    off = np.ascontiguousarray(chunk_offsets, dtype=np.int64)
    n_chunks = off.shape[0] - 1
    N, D = X.shape
    assert off[-1] == N
    gC = np.empty((M, Ks, D // M), dtype=np.float32)
    codes = np.empty((N, M), dtype=np.uint8)
    rmse = np.zeros(1, dtype=np.float64)
    local = np.empty((n_chunks, M, Ks, D // M), dtype=np.float32)
    _check(_load().orc_pq_fit_chunked(_ptr(X), _ptr(off), n_chunks, D, M, Ks, iters, seed & (2**64 - 1), _ptr(gC),
                                      _ptr(codes), _ptr(rmse), _ptr(local)), "pq_fit_chunked")
    return gC, codes, float(rmse[0]), local


def pq_fit_counts(X, M: int, Ks: int, iters: int, seed: int):
    """PQ fit; returns (codebooks, member counts [M][Ks] of the last update)."""
    X = _f32(X)
    N, D = X.shape
    out = np.empty((M, Ks, D // M), dtype=np.float32)
    cnt = np.empty((M, Ks), dtype=np.int64)
    _check(_load().orc_pq_fit_counts(_ptr(X), N, D, M, Ks, iters, seed & (2**64 - 1), _ptr(out), _ptr(cnt)),
           "pq_fit_counts")
    return out, cnt


def pq_fit_weighted(P, W, M: int, Ks: int, iters: int, seed: int):
    """Weighted PQ fit of points P [n][D] with weights W [n][M] (int64)."""
    P = _f32(P)
    W = np.ascontiguousarray(W, dtype=np.int64)
    n, D = P.shape
    out = np.empty((M, Ks, D // M), dtype=np.float32)
    _check(_load().orc_pq_fit_weighted(_ptr(P), _ptr(W), n, D, M, Ks, iters, seed & (2**64 - 1), _ptr(out)),
           "pq_fit_weighted")
    return out


def pq_fit_chunked_weighted(X, chunk_offsets, M: int, Ks: int, iters: int, seed: int):
    """Returns (global codebooks, codes, RMSE, local codebooks, weights [n_chunks*Ks][M])."""
    X = _f32(X)
    off = np.ascontiguousarray(chunk_offsets, dtype=np.int64)
    n_chunks = off.shape[0] - 1
    N, D = X.shape
    gC = np.empty((M, Ks, D // M), dtype=np.float32)
    codes = np.empty((N, M), dtype=np.uint8)
    rmse = np.zeros(1, dtype=np.float64)
    local = np.empty((n_chunks, M, Ks, D // M), dtype=np.float32)
    W = np.empty((n_chunks * Ks, M), dtype=np.int64)
    _check(_load().orc_pq_fit_chunked_weighted(_ptr(X), _ptr(off), n_chunks, D, M, Ks, iters, seed & (2**64 - 1),
                                               _ptr(gC), _ptr(codes), _ptr(rmse), _ptr(local), _ptr(W)),
           "pq_fit_chunked_weighted")
    return gC, codes, float(rmse[0]), local, W


# -- optimized PQ (Sec. 2.1 "Optimized PQ", Sec. 3.1) -------------------------------------

def opq_rotate(X, R) -> np.ndarray:
    """Rotated rows X R, computed in FP64 and rounded once to float32."""
    return (np.asarray(X, dtype=np.float64) @ np.asarray(R, dtype=np.float64)).astype(np.float32)


def opq_procrustes(X, Yh) -> np.ndarray:
    """The orthogonal R minimising ||X R - Yh||_F: R = U V^T for X^T Yh = U S V^T (FP64 SVD)."""
    A = np.asarray(X, dtype=np.float64).T @ np.asarray(Yh, dtype=np.float64)
    U, _, Vt = np.linalg.svd(A)
    return U @ Vt


def opq_fit(X, M: int, Ks: int, outer: int, pq_iters: int, seed: int):
    """Optimized PQ by alternating minimisation (non-parametric OPQ): R = I and a PQ fit of X; then
    `outer` times: encode the rotated rows, decode, R = Procrustes(X, reconstruction), refit the
    codebooks on X R from the previous ones (pq_iters Lloyd iterations).  Returns
    (R [D][D] float32, codebooks, distortion ||X R - Yh||^2 before each rotation update)."""
    X = _f32(X)
    D = X.shape[1]
    R = np.eye(D, dtype=np.float32)
    Y = opq_rotate(X, R)
    cb, _ = pq_fit(Y, M, Ks, pq_iters, seed)
    dist = []
    for _ in range(outer):
        Yh = pq_decode(pq_encode(Y, cb), cb)
        dist.append(float(((Y.astype(np.float64) - Yh) ** 2).sum()))
        R = opq_procrustes(X, Yh).astype(np.float32)
        Y = opq_rotate(X, R)
        cb, _ = pq_fit(Y, M, Ks, pq_iters, 0, init=cb)
    return R, cb, dist


# -- soft-assignment refinement ----------------------------------------------------

def softpq_forward(X, codebooks, tau: float) -> float:
    X = np.ascontiguousarray(X, dtype=np.float64)
    cb = np.ascontiguousarray(codebooks, dtype=np.float64)
    N, D = X.shape
    M, Ks, _ = cb.shape
    return _load().orc_softpq_forward(_ptr(X), N, D, M, Ks, _ptr(cb), tau)


def softpq_backward(X, codebooks, tau: float):
    """Returns (dL/dcodebooks, dL/dX) in FP64."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    cb = np.ascontiguousarray(codebooks, dtype=np.float64)
    N, D = X.shape
    M, Ks, _ = cb.shape
    dC = np.empty_like(cb)
    dX = np.empty_like(X)
    _load().orc_softpq_backward(_ptr(X), N, D, M, Ks, _ptr(cb), tau, _ptr(dC), _ptr(dX))
    return dC, dX
