"""Gaussian test matrices for randomized sampling (Sec. 2.5; Figs. HODLR / HBS).

The paper draws Omega with ``randn``.  To make the draws reproducible and
independent of launch geometry, entry (i, c) of the level-l Gaussian field is a
pure function of (seed, stream, level, i, c), built from the counter-based
generator Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
as easy as 1, 2, 3", SC'11) and the Box-Muller transform, both written here from
their published definitions:

* Philox4x32 round: (hi0, lo0) = mulhilo(0xD2511F53, c0),
  (hi1, lo1) = mulhilo(0xCD9E8D57, c2),
  c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); between rounds the key is
  bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85).  Ten rounds.
* counter = (i, c >> 1, level, stream), key = (seed mod 2^32, seed >> 32).
* u1 = (w0 * 2^21 + (w1 >> 11) + 1/2) * 2^-53, u2 likewise from (w2, w3);
  rho = sqrt(-2 ln u1), theta = 2 pi u2; even c takes rho cos(theta), odd c
  takes rho sin(theta).  All in FP64.
* Mixed precision: the FP64 value is rounded to FP32 (round to nearest even)
  and then to BF16 (round to nearest even on the FP32 bit pattern); the
  rounded value is the test matrix entry for both the oracle and the device.

Pinned by tests/test_oracle_philox.py: Random123 known-answer vectors for
Philox4x32-10, and moments / normality of the Gaussian field.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint32(0x9E3779B9)
W1 = np.uint32(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)

STREAM_OMEGA = 0   # level test matrices of the compression sweeps
STREAM_ESTIMATE = 1  # unit vectors of the error estimate E (Sec. 5)


def _mulhilo(a: np.uint64, b: np.ndarray):
    p = a * b.astype(np.uint64)
    return (p >> np.uint64(32)).astype(np.uint32), (p & MASK32).astype(np.uint32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds on arrays of 32-bit counters with a 2x32-bit key."""
    c0 = np.asarray(c0, dtype=np.uint32)
    c1 = np.asarray(c1, dtype=np.uint32)
    c2 = np.asarray(c2, dtype=np.uint32)
    c3 = np.asarray(c3, dtype=np.uint32)
    k0 = np.uint32(k0)
    k1 = np.uint32(k1)
    with np.errstate(over="ignore"):
        for rnd in range(10):
            if rnd > 0:
                k0 = np.uint32(k0 + W0)
                k1 = np.uint32(k1 + W1)
            hi0, lo0 = _mulhilo(M0, c0)
            hi1, lo1 = _mulhilo(M1, c2)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def _uniform53(hi: np.ndarray, lo: np.ndarray) -> np.ndarray:
    m = hi.astype(np.float64) * 2.0 ** 21 + (lo >> np.uint32(11)).astype(np.float64)
    return (m + 0.5) * 2.0 ** -53


def gaussian(seed: int, stream: int, level: int, rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """FP64 standard normal entries G(i, c) for the outer product of rows x cols."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    I, C = np.meshgrid(rows, cols, indexing="ij")
    k0 = seed & 0xFFFFFFFF
    k1 = (seed >> 32) & 0xFFFFFFFF
    w0, w1, w2, w3 = philox4x32_10(I.astype(np.uint32), (C >> 1).astype(np.uint32),
                                   np.full(I.shape, level, np.uint32),
                                   np.full(I.shape, stream, np.uint32), k0, k1)
    u1 = _uniform53(w0, w1)
    u2 = _uniform53(w2, w3)
    rho = np.sqrt(-2.0 * np.log(u1))
    theta = 2.0 * np.pi * u2
    return np.where((C & 1) == 0, rho * np.cos(theta), rho * np.sin(theta))


def round_bf16(x: np.ndarray) -> np.ndarray:
    """FP64 -> FP32 (RNE) -> BF16 (RNE on the FP32 bits), returned as FP64."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))) & np.uint64(0xFFFF0000)
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def level_field(seed: int, level: int, N: int, r: int, mixed: bool) -> np.ndarray:
    """The N x r Gaussian field of one level (rounded to BF16 values if mixed)."""
    g = gaussian(seed, STREAM_OMEGA, level, np.arange(N), np.arange(r))
    return round_bf16(g) if mixed else g
