"""Checks of the seeded input generators against closed forms (no GPU)."""
import math

import numpy as np

import workloads as wl


def test_counter_based_slices_agree():
    full = wl.uniform(10_000, 16, 8, seed=42)
    part = wl.uniform(3_000, 16, 8, seed=42, first=5_000)
    np.testing.assert_array_equal(full[5_000:8_000], part)
    # payload word is the global index
    np.testing.assert_array_equal(part[:, 8:].copy().view("<u8").ravel(), np.arange(5_000, 8_000))


def test_seeds_differ_and_threads_do_not_matter():
    a = wl.uniform(200_000, 24, 16, seed=1)
    b = wl.uniform(200_000, 24, 16, seed=2)
    assert not np.array_equal(a, b)
    c = np.empty_like(a)
    wl.lib().wl_fill_uniform(c.ctypes.data, 200_000, 24, 16, 1, 0, 1)   # single thread
    np.testing.assert_array_equal(a, c)


def test_uniform_bytes_are_uniform():
    a = wl.uniform(400_000, 8, 8, seed=3)
    top = a[:, 7].astype(np.float64)
    assert abs(top.mean() - 127.5) < 1.0
    counts = np.bincount(a[:, 7], minlength=256)
    chi2 = ((counts - 400_000 / 256) ** 2 / (400_000 / 256)).sum()
    assert chi2 < 400  # 255 dof


def test_zipf_top_rank_share_matches_closed_form():
    # Zipf(1) over 2^32 ranks: P(rank 1) = 1 / H_{2^32} ~ 4.39%
    n = 200_000
    ranks = wl.zipf_ranks(3, range(n))
    p1 = 1.0 / wl.harmonic(2 ** 32)
    assert abs(p1 - 0.0439) < 0.0005
    share = float(np.mean(ranks == 1))
    assert abs(share - p1) < 5 * math.sqrt(p1 * (1 - p1) / n)
    p2 = 0.5 * p1
    assert abs(float(np.mean(ranks == 2)) - p2) < 5 * math.sqrt(p2 * (1 - p2) / n)
    assert ranks.min() >= 1 and ranks.max() <= 2 ** 32


def test_zipf_keys_are_bijective_image_of_ranks():
    recs = wl.zipf(50_000, 16, seed=3)
    keys = recs[:, :8].copy().view("<u8").ravel()
    ranks = wl.zipf_ranks(3, range(50_000))
    mapped = np.array([wl.zipf_key_of_rank(3, int(r)) for r in ranks], dtype=np.uint64)
    np.testing.assert_array_equal(keys, mapped)
    # equal ranks <-> equal keys
    assert len(np.unique(keys)) == len(np.unique(ranks))


def test_kmer_high_word_from_1024_prefixes():
    recs = wl.kmer(100_000, 24, seed=4)
    hi = recs[:, 8:16].copy().view("<u8").ravel()
    table = wl.kmer_table(4)
    assert len(np.unique(table)) == 1024
    assert np.isin(hi, table).all()
    assert 1000 <= len(np.unique(hi)) <= 1024
    idx = recs[:, 16:24].copy().view("<u8").ravel()
    np.testing.assert_array_equal(idx, np.arange(100_000))


def test_log_uniform_mean_closed_form():
    m = 100_000
    s = wl.log_uniform(m, 1, 10 ** 6, seed=5)
    assert s.min() >= 1 and s.max() <= 10 ** 6
    # continuous log-uniform on [1, 10^6+1): mean (b - a) / ln(b / a); floor subtracts ~1/2
    mean = 10 ** 6 / math.log(10 ** 6 + 1) - 0.5
    assert abs(s.mean() - mean) < 5 * 1.8e5 / math.sqrt(m)


def test_batched_sizes_are_capped():
    s = wl.batched_sizes()
    assert len(s) == 100_000
    assert int(s.sum()) <= 2_000_000_000
    assert s.min() >= 1
