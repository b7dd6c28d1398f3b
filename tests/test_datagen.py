"""The seeded input generators: the same rows whatever the thread count (one PCG64 stream per
block of rows), different rows for different seeds, and the value ranges of the two mixtures."""
import numpy as np

from paper_2604_21645_gb300 import datagen


def test_mixture_is_independent_of_thread_count():
    a = datagen.mixture(140_001, 24, 17, "cont", 31, threads=1)
    b = datagen.mixture(140_001, 24, 17, "cont", 31, threads=4)
    assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
    assert np.array_equal(a, b)


def test_mixture_depends_on_seed_and_kind():
    a = datagen.mixture(5_000, 16, 8, "int255", 1)
    b = datagen.mixture(5_000, 16, 8, "int255", 2)
    assert not np.array_equal(a, b)
    assert a.min() >= 0 and a.max() <= 255 and np.array_equal(a, np.rint(a))
    c = datagen.mixture(5_000, 16, 8, "cont", 1)
    assert np.abs(c).max() < 2.0
