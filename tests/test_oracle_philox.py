"""Pins for oracle/philox.py: statistical properties and the counter layout
(the word stream itself is unpinned: no known-answer vectors in the tree)."""
import numpy as np
import scipy.stats as st

from oracle import philox


def test_counter_layout_is_prefix_stable():
    a = philox.gaussian(3, 1000, seed=12345)
    b = philox.gaussian(5, 1003, seed=12345)
    np.testing.assert_array_equal(a, b[:3, :1000])
    r1 = philox.rademacher(2, 300, seed=9)
    r2 = philox.rademacher(4, 1000, seed=9)
    np.testing.assert_array_equal(r1, r2[:2, :300])


def test_seeds_and_streams_differ():
    a = philox.gaussian_words(1, 4096, seed=1)
    b = philox.gaussian_words(1, 4096, seed=2)
    c = philox.gaussian_words(1, 4096, seed=1 + (1 << 32))
    assert np.mean(a == b) < 0.01 and np.mean(a == c) < 0.01


def test_word_uniformity():
    w = philox.gaussian_words(4, 1 << 16, seed=77).reshape(-1)
    # top byte histogram: chi-square against uniform
    hist = np.bincount((w >> 24).astype(np.int64), minlength=256)
    chi2 = st.chisquare(hist)
    assert chi2.pvalue > 1e-4
    # every bit is set about half the time
    bits = np.array([(w >> b) & 1 for b in range(32)]).mean(axis=1)
    assert np.all(np.abs(bits - 0.5) < 0.01)


def test_gaussian_moments_and_ks():
    z = philox.gaussian(8, 1 << 15, seed=3).reshape(-1)
    assert abs(z.mean()) < 5 / np.sqrt(len(z))
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / len(z))
    assert st.kstest(z, "norm").pvalue > 1e-4
    # neighbouring elements and neighbouring vectors are uncorrelated
    Z = philox.gaussian(2, 1 << 16, seed=3)
    assert abs(np.corrcoef(Z[0], Z[1])[0, 1]) < 5 / np.sqrt(Z.shape[1])
    assert abs(np.corrcoef(Z[0][:-1], Z[0][1:])[0, 1]) < 5 / np.sqrt(Z.shape[1])


def test_rademacher_balance():
    r = philox.rademacher(16, 1 << 14, seed=5)
    assert set(np.unique(r)) == {-1.0, 1.0}
    assert abs(r.mean()) < 5 / np.sqrt(r.size)
