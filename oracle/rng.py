"""Counter-based Gaussian probes for the peeling construction (oracle side).

TEST INFRASTRUCTURE: the oracle is a slow CPU reference used only by the
tests, the smoke check and the CPU-baseline leg of the benchmark.

The randomized construction (Section 3.3) draws Gaussian probe blocks level
by level.  Because the probes are drawn inside the method, the oracle and the
CUDA path each implement the same counter-based generator from its published
definition:

* SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014): the i-th output of a generator seeded with s is
  mix(s + (i+1) * 0x9E3779B97F4A7C15 mod 2^64), where mix is the 64-bit
  finaliser  z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27;
  z *= 0x94D049BB133111EB; z ^= z>>31.
* Box-Muller (Box and Muller, 1958): z = sqrt(-2 ln u1) cos(2 pi u2).

Keying: key = mix(seed XOR mix(stream * 2^16 + level)); the Gaussian at
(row, col) uses counter c = col * 2^32 + row and the two SplitMix64 outputs
with indices 2c and 2c+1 of the generator seeded with key; u1 = (b1>>11 + 1) 2^-53
lies in (0, 1], u2 = (b2>>11) 2^-53 in [0, 1).
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)

STREAM_PROBE = 1      # range-finder probes
STREAM_POWER = 2      # start vector of the 2-norm power iteration
STREAM_ERR = 3        # start vector of the error power iteration
STREAM_GLOBAL = 5     # probes of the global low-rank range finder
STREAM_COLORED = 8    # probes of the coloured (strong-structure) range pass


def mix64(z):
    """SplitMix64 output finaliser on uint64 arrays (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z ^ (z >> np.uint64(30))
        z = z * M1
        z = z ^ (z >> np.uint64(27))
        z = z * M2
        z = z ^ (z >> np.uint64(31))
    return z


def stream_key(seed: int, stream: int, level: int) -> np.uint64:
    inner = mix64(np.uint64((stream << 16) + level))
    return mix64(np.uint64(seed) ^ inner)


def splitmix_at(key, idx):
    """Output number idx (0-based) of SplitMix64 seeded with key."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(np.uint64(key) + (idx + np.uint64(1)) * GOLDEN)


def gaussian(seed: int, stream: int, level: int, rows, cols) -> np.ndarray:
    """Gaussian values g(row, col) for broadcastable integer arrays rows, cols."""
    rows = np.asarray(rows, dtype=np.uint64)
    cols = np.asarray(cols, dtype=np.uint64)
    key = stream_key(seed, stream, level)
    with np.errstate(over="ignore"):
        c = (cols << np.uint64(32)) + rows
        b1 = splitmix_at(key, np.uint64(2) * c)
        b2 = splitmix_at(key, np.uint64(2) * c + np.uint64(1))
    u1 = ((b1 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = (b2 >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def gaussian_block(seed: int, stream: int, level: int, nrows: int, col0: int, ncols: int) -> np.ndarray:
    """nrows x ncols block of g(row, col0 + j), rows 0..nrows-1 (tree order)."""
    r = np.arange(nrows, dtype=np.uint64)[:, None]
    c = np.arange(col0, col0 + ncols, dtype=np.uint64)[None, :]
    return gaussian(seed, stream, level, r, c)
