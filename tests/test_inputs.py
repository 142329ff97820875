"""The seeded input generators both sides consume: deterministic, regenerable
by band, and shaped as their docstrings state (CPU)."""
import numpy as np
import pytest

from paper_2510_03631_gb300 import inputs


def test_db_digits_bands_regenerate_the_same_matrix():
    full = inputs.db_digits(300, 1000, 256, seed=4)
    for r0, rc in ((0, 1), (7, 13), (299, 1), (64, 200)):
        assert np.array_equal(inputs.db_digits(300, 1000, 256, seed=4, row_start=r0, row_count=rc), full[r0:r0 + rc])
    assert not np.array_equal(full, inputs.db_digits(300, 1000, 256, seed=5))


@pytest.mark.parametrize("p", [2, 16, 256])
def test_db_digits_are_below_p(p):
    assert int(inputs.db_digits(64, 512, p, seed=1).max()) < p


def test_sorted_entries_are_sorted_with_bounded_gaps():
    x = inputs.sorted_entries(100000, seed=3, max_gap=31)
    gaps = np.diff(x.astype(np.int64))
    assert x.dtype == np.uint32 and (gaps >= 0).all() and gaps.max() <= 31
    assert 10 < gaps.mean() < 21   # uniform on [0, 31]: mean 15.5
    assert np.array_equal(x, inputs.sorted_entries(100000, seed=3, max_gap=31))
    assert not np.array_equal(x, inputs.sorted_entries(100000, seed=4, max_gap=31))


def test_noise_is_a_rounded_gaussian_within_its_tail_cut():
    e = inputs.noise(200000, seed=2)
    assert e.dtype == np.int32 and np.abs(e).max() <= 64
    assert abs(float(e.mean())) < 0.1 and 6.0 < float(e.std()) < 6.8   # sigma = 6.4
