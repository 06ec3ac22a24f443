"""Pins for the oracle's counter-based sketch generator (Definition 2.1 random
Gaussian TT; Philox4x32-10 of Salmon et al., SC'11)."""
import os

import numpy as np
import pytest

from oracle import philox
from tests.conftest import read_kat

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def test_philox_known_answer_vectors(golden_dir):
    rows = read_kat(os.path.join(golden_dir, "philox4x32_10_kat.txt"))
    assert len(rows) == 3
    for ctr, key, out in rows:
        got = philox.philox4x32_10(np.array(ctr, dtype=np.uint32), key)
        assert [int(v) for v in got] == out


def test_philox_vectorised_matches_scalar():
    rng = np.random.default_rng(7)
    ctr = rng.integers(0, 2 ** 32, size=(64, 4), dtype=np.uint64).astype(np.uint32)
    key = (0x12345678, 0x9abcdef0)
    batch = philox.philox4x32_10(ctr, key)
    for j in range(64):
        assert np.array_equal(batch[j], philox.philox4x32_10(ctr[j], key))


def test_uniform_mapping_is_exact_and_open():
    # smallest and largest words map to 2^-53 and 1 - 2^-53 exactly
    lo = philox.uniforms_from_words(np.uint32(0), np.uint32(0))
    hi = philox.uniforms_from_words(np.uint32(0xFFFFFFFF), np.uint32(0xFFFFFFFF))
    assert lo == 2.0 ** -53
    assert hi == 1.0 - 2.0 ** -53
    # the 52 kept bits: (x0 >> 6) high, (x1 >> 6) low
    u = philox.uniforms_from_words(np.uint32(1 << 6), np.uint32(3 << 6))
    assert u == ((1 << 26) + 3 + 0.5) * 2.0 ** -52


def test_gaussian_moments():
    core = philox.sketch_core(seed=11, core=0, shape=(1, 200000, 1))
    g = core.ravel() * np.sqrt(200000.0)      # undo the 1/sqrt(l n l) scale
    n = g.size
    assert abs(g.mean()) < 5.0 / np.sqrt(n)
    assert abs(g.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
    # kurtosis of N(0,1) is 3
    assert abs(np.mean(g ** 4) - 3.0) < 0.1


def test_sketch_core_variance_definition_2_1():
    a, n, b = 30, 40, 50
    core = philox.sketch_core(seed=3, core=2, shape=(a, n, b))
    var = core.var()
    expect = 1.0 / (a * n * b)
    assert abs(var / expect - 1.0) < 0.03


def test_streams_are_distinct_and_reproducible():
    c0 = philox.sketch_core(5, 0, (4, 8, 4))
    c0b = philox.sketch_core(5, 0, (4, 8, 4))
    c1 = philox.sketch_core(5, 1, (4, 8, 4))
    c0p = philox.sketch_core(5, 0, (4, 8, 4), pair=1)
    s6 = philox.sketch_core(6, 0, (4, 8, 4))
    assert np.array_equal(c0, c0b)
    for other in (c1, c0p, s6):
        assert not np.allclose(c0, other)
        corr = np.corrcoef(c0.ravel(), other.ravel())[0, 1]
        assert abs(corr) < 0.35
