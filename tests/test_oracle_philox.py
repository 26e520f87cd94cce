"""Oracle pins for the counter-based Gaussian test matrices (Sec. 2.5)."""
import numpy as np
import pytest

from conftest import golden_path
from oracle import philox


def test_known_answer_vectors():
    for line in open(golden_path("philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        out = philox.philox4x32_10(v[0], v[1], v[2], v[3], v[4], v[5])
        assert [int(o) for o in out] == v[6:10]


def test_gaussian_moments_and_normality():
    scipy_stats = pytest.importorskip("scipy.stats")
    g = philox.gaussian(2, philox.STREAM_OMEGA, 3, np.arange(20000), np.arange(10)).ravel()
    assert abs(g.mean()) < 0.01
    assert abs(g.var() - 1.0) < 0.02
    assert scipy_stats.kstest(g, "norm").pvalue > 1e-3
    # the two Box-Muller outputs of one counter are uncorrelated
    g2 = philox.gaussian(2, 0, 3, np.arange(20000), np.arange(2))
    assert abs(np.corrcoef(g2[:, 0], g2[:, 1])[0, 1]) < 0.03


def test_geometry_independence():
    full = philox.gaussian(9, 0, 1, np.arange(100), np.arange(12))
    part = philox.gaussian(9, 0, 1, np.arange(40, 60), np.arange(3, 9))
    assert np.array_equal(full[40:60, 3:9], part)
    other_level = philox.gaussian(9, 0, 2, np.arange(100), np.arange(12))
    assert not np.allclose(full, other_level)


def test_round_bf16():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 1.0 + 2.0 ** -9, 3.0e-39])
    got = philox.round_bf16(x)
    # ties go to even mantissa: 1 + 2^-8 -> 1, 1 + 3*2^-8 -> 1 + 2^-6
    assert got[0] == 1.0 and got[1] == 1.0 and got[2] == 1.0 + 2.0 ** -6
    assert got[3] == -2.5 and got[4] == 1.0
    bits = got.astype(np.float32).view(np.uint32)
    assert np.all(bits & 0xFFFF == 0)
    g = philox.gaussian(1, 0, 0, np.arange(1000), np.arange(4)).ravel()
    rb = philox.round_bf16(g)
    assert np.max(np.abs(rb - g) / np.abs(g)) <= 2.0 ** -8
