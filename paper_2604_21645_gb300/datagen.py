"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the method (no distances, no k-means, no
encoding): it only draws the input matrices, query sets and chunk sizes that
both sides consume bit-identically.

The paper's own data (a 6.7M x 48 SoilGrids sample split into 400 chunks of
16,750 rows, Section 3) is not available, so seeded Gaussian mixtures of the
shapes below stand in for it:

* ``kind="cont"``   : component means mu_c ~ U[-1, 1]^D, x = mu_z + 0.1 * eps
* ``kind="int255"`` : mu_c ~ U[0, 255]^D, x = clip(rint(mu_z + 20 * eps), 0, 255)
  (integer-valued floats, the value range of a SIFT-like descriptor set)

z is a uniform component id, eps ~ N(0, I).  Everything is computed in float64
and rounded once to float32.  Rows are drawn in independent blocks of 65,536
(one PCG64 stream per block, keyed by ``SeedSequence([seed, 1, block])``) so
large matrices can be generated on several threads with a result that does not
depend on the thread count.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

BLOCK_ROWS = 1 << 16
_M64 = (1 << 64) - 1


def _rng(seed: int, *keys: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed & _M64, *keys])))


def mixture_means(seed: int, n_comp: int, d: int, kind: str) -> np.ndarray:
    rng = _rng(seed, 0)
    if kind == "cont":
        return rng.uniform(-1.0, 1.0, size=(n_comp, d))
    if kind == "int255":
        return rng.uniform(0.0, 255.0, size=(n_comp, d))
    raise ValueError(f"unknown mixture kind {kind!r}")


def _block(seed, b, rows, d, means, kind):
    rng = _rng(seed, 1, b)
    z = rng.integers(0, means.shape[0], size=rows)
    eps = rng.standard_normal((rows, d))
    if kind == "cont":
        x = means[z] + 0.1 * eps
    else:
        x = np.clip(np.rint(means[z] + 20.0 * eps), 0.0, 255.0)
    return x.astype(np.float32)


def mixture(n: int, d: int, n_comp: int, kind: str, seed: int, threads: int | None = None) -> np.ndarray:
    """Return an (n, d) float32 C-contiguous matrix drawn from the seeded mixture."""
    means = mixture_means(seed, n_comp, d, kind)
    out = np.empty((n, d), dtype=np.float32)
    nb = (n + BLOCK_ROWS - 1) // BLOCK_ROWS

    def fill(b):
        r0 = b * BLOCK_ROWS
        r1 = min(n, r0 + BLOCK_ROWS)
        out[r0:r1] = _block(seed, b, r1 - r0, d, means, kind)

    if threads is None:
        threads = min(16, os.cpu_count() or 1)
    if nb <= 1 or threads <= 1:
        for b in range(nb):
            fill(b)
    else:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(fill, range(nb)))
    return out


def queries(nq: int, d: int, n_comp: int, kind: str, seed: int) -> np.ndarray:
    """Queries from the same mixture (same means), drawn from an independent row stream."""
    means = mixture_means(seed, n_comp, d, kind)
    out = np.empty((nq, d), dtype=np.float32)
    nb = (nq + BLOCK_ROWS - 1) // BLOCK_ROWS
    for b in range(nb):
        r0 = b * BLOCK_ROWS
        r1 = min(nq, r0 + BLOCK_ROWS)
        out[r0:r1] = _block(seed + 1, (1 << 20) + b, r1 - r0, d, means, kind)
    return out


def chunk_sizes(n_chunks: int, median: float, log_sigma: float, lo: int, hi: int, seed: int) -> np.ndarray:
    """Lognormal chunk row counts (the paper splits data row-wise into chunks, Section 3)."""
    rng = _rng(seed, 2)
    s = rng.lognormal(mean=np.log(median), sigma=log_sigma, size=n_chunks)
    return np.clip(np.rint(s), lo, hi).astype(np.int64)


@dataclass(frozen=True)
class Workload:
    """A named synthetic workload with the sizes of one of the target configurations."""
    name: str
    n: int
    d: int
    m: int
    ks: int
    iters: int
    n_comp: int
    kind: str
    seed: int
    nlist: int = 0
    ivf_iters: int = 25
    nq: int = 0
    nprobe: int = 0
    topk: int = 0
    n_chunks: int = 0
    tau: float = 0.0
    extra: dict = field(default_factory=dict)

    @property
    def init_seed(self) -> int:
        return self.seed + 7

    @property
    def coarse_seed(self) -> int:
        return self.seed + 7 + 2

    def data(self, n: int | None = None) -> np.ndarray:
        return mixture(self.n if n is None else n, self.d, self.n_comp, self.kind, self.seed)

    def queries(self, nq: int | None = None) -> np.ndarray:
        return queries(self.nq if nq is None else nq, self.d, self.n_comp, self.kind, self.seed)


BASE_SEED = 0x5EED0000

# Plain PQ fit+encode, 10k x 64, M=8, Ks=256, 20 Lloyd iterations.
PQ_SMALL = Workload("pq_10k_d64_m8", 10_000, 64, 8, 256, 20, 32, "cont", BASE_SEED + 1)
# PQ + inverted index, 1M x 128 integer-valued, M=16, Ks=256, 25 iterations,
# nlist=1024, 10k queries, nprobe=16, top-100.
IVF_MEDIUM = Workload("ivf_1m_d128_m16_nlist1024", 1_000_000, 128, 16, 256, 25, 1000, "int255",
                      BASE_SEED + 2, nlist=1024, ivf_iters=25, nq=10_000, nprobe=16, topk=100)
# Precision form, 10M x 128 integer-valued, 4,096 components, M=16, Ks=256, 20 iterations.
PQ_10M = Workload("pq_10m_d128_m16", 10_000_000, 128, 16, 256, 20, 4096, "int255", BASE_SEED + 3)
# Search over the precision form's rows: the 10M x 128 rows above (same seed, same mixture) in an
# inverted index of nlist=1024 lists, 10k queries from the mixture, nprobe=16, top-100.  Its 160 MB
# of codes exceed the 129 MB L2, so the scan reads them from HBM.
IVF_10M = Workload("ivf_10m_d128_m16_nlist1024", 10_000_000, 128, 16, 256, 20, 4096, "int255", BASE_SEED + 3,
                   nlist=1024, ivf_iters=25, nq=10_000, nprobe=16, topk=100)
# Batched chunked form: 64 lognormal chunks (median 200k), D=96, M=12, Ks=256, 20 iterations.
CHUNKED = Workload("chunked_64x_d96_m12", 0, 96, 12, 256, 20, 256, "cont", BASE_SEED + 4, n_chunks=64,
                   extra={"median": 200_000, "log_sigma": 1.0, "lo": 10_000, "hi": 2_000_000})
# Differentiable refinement: 1M x 256, M=32, Ks=256, tau=0.1.
SOFTPQ = Workload("softpq_1m_d256_m32", 1_000_000, 256, 32, 256, 0, 256, "cont", BASE_SEED + 5, tau=0.1)

WORKLOADS = {w.name: w for w in (PQ_SMALL, IVF_MEDIUM, PQ_10M, IVF_10M, CHUNKED, SOFTPQ)}


def chunk_offsets(w: Workload, n_chunks: int | None = None) -> np.ndarray:
    """Row offsets (n_chunks + 1) of the lognormal chunks of a chunked workload."""
    e = w.extra
    sizes = chunk_sizes(n_chunks or w.n_chunks, e["median"], e["log_sigma"], e["lo"], e["hi"], w.seed)
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
