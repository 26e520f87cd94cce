"""The matrix-free log-kernel black box computes its entries from two tables
(log|x_i - x_j| = S[|i - j|] + P[i + j]).  Pins of that factorization against
the direct definition of the kernel on the ellipse, on the CPU."""
import numpy as np

import workloads as W


def test_factorization_matches_the_distance_formula():
    N = 1000
    x = W.ellipse_points(N)
    rng = np.random.default_rng(3)
    i = rng.integers(0, N, 5000)
    j = rng.integers(0, N, 5000)
    keep = i != j
    i, j = i[keep], j[keep]
    direct = np.log(np.hypot(x[i, 0] - x[j, 0], x[i, 1] - x[j, 1]))
    d, f = np.pi * (i - j) / N, np.pi * (i + j) / N
    via = np.log(np.abs(np.sin(d))) + 0.5 * np.log1p(3.0 * np.sin(f) ** 2)
    assert np.max(np.abs(via - direct)) < 1e-12
    # a hand case: antipodal points (1, 0) and (-1, 0) are 2 apart
    assert abs(np.log(abs(np.sin(np.pi / 2))) + 0.5 * np.log1p(3.0) - np.log(2.0)) < 1e-15


def test_fp32_entries_within_one_ulp_and_symmetric():
    """With the tables as float pairs, an entry is within about one FP32 ulp of the
    FP64 formula rounded once (where the two terms cancel, near distance 1, the
    high parts subtract exactly and the low parts carry the rest); the matrix is
    exactly symmetric with ones on the diagonal."""
    N = 777
    A = W.log_kernel_tab(N)
    ref = W.log_kernel(N)  # FP64 formula rounded once to FP32
    ulp = np.abs(A.view(np.int32).astype(np.int64) - ref.view(np.int32).astype(np.int64))
    assert ulp.max() <= 1 and np.mean(ulp == 0) > 0.8
    assert np.array_equal(A, A.T)
    assert np.all(np.diag(A) == 1.0)
