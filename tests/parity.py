"""Comparison helpers for GPU-vs-oracle parity (tolerances stated per check)."""
import numpy as np

# Codeword tolerance: 1e-5 relative to the largest magnitude in the subspace codebook.
CENTROID_RTOL = 1e-5
# Reconstruction RMSE tolerance: 1e-4 relative.
RMSE_RTOL = 1e-4
# Ranked query results: distances within 1e-5 relative; an id may differ from
# the oracle's only where the oracle's own distances tie within 1e-5 relative.
TOPK_RTOL = 1e-5


def assert_codebooks_close(got, ref, rtol=CENTROID_RTOL):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape
    for m in range(ref.shape[0]):
        scale = max(np.abs(ref[m]).max(), 1e-30)
        err = np.abs(got[m] - ref[m]).max()
        assert err <= rtol * scale, f"subspace {m}: max |diff| {err} > {rtol} * {scale}"


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def check_topk(gpu_ids, gpu_d, ref_ids, ref_d, rtol=TOPK_RTOL):
    """Returns the number of id mismatches explained by near-ties; asserts there are no others."""
    gpu_ids = np.asarray(gpu_ids)
    ref_ids = np.asarray(ref_ids)
    gpu_d = np.asarray(gpu_d, dtype=np.float64)
    ref_d = np.asarray(ref_d, dtype=np.float64)
    nq, k = ref_ids.shape
    ties = 0
    for q in range(nq):
        valid = ref_ids[q] >= 0
        assert np.array_equal(gpu_ids[q] >= 0, valid), f"query {q}: different result counts"
        rd = ref_d[q][valid]
        gd = gpu_d[q][valid]
        np.testing.assert_allclose(gd, rd, rtol=rtol, atol=1e-6 * (rd.max() if rd.size else 1.0))
        pos = {int(i): r for r, i in enumerate(ref_ids[q]) if i >= 0}
        for r in np.nonzero(gpu_ids[q] != ref_ids[q])[0]:
            gid = int(gpu_ids[q, r])
            if gid in pos:
                r2 = pos[gid]
                assert abs(ref_d[q, r2] - ref_d[q, r]) <= rtol * max(ref_d[q, r], 1e-30), \
                    f"query {q} rank {r}: id {gid} is rank {r2} in the oracle without a near-tie"
            else:
                last = ref_d[q][valid][-1]
                assert abs(gpu_d[q, r] - last) <= rtol * max(last, 1e-30), \
                    f"query {q} rank {r}: id {gid} not in the oracle's top-{k} and not tied with its last"
            ties += 1
    return ties
