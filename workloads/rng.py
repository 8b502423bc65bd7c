"""Counter-based SplitMix64 random numbers (Steele, Lea & Flood, OOPSLA 2014).

Every synthetic input of this project is drawn from here, so that the oracle
side and the CUDA side receive bit-identical arrays.  Value number ``i`` of
stream ``s`` under ``seed`` is the SplitMix64 finaliser applied to
``key(seed, s) + (i + 1) * GOLDEN`` (mod 2**64), i.e. the i-th output of a
SplitMix64 generator whose state starts at ``key``.  No state is carried
between calls, so any slice of a stream can be regenerated on its own.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
DEFAULT_SEED = 20111003


def _mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    """Start state of stream ``stream``: two finaliser rounds over (seed, stream)."""
    s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    t = np.uint64(stream & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        return _mix(np.array([_mix(np.array([s]))[0] ^ (t * GOLDEN + np.uint64(0x632BE59BD9B4E019))]))[0]


def u64(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """Raw 64-bit outputs ``start .. start+n-1`` of one stream."""
    key = stream_key(seed, stream)
    ctr = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key + ctr * GOLDEN)


def uniform(seed: int, stream: int, n: int, lo: float = 0.0, hi: float = 1.0,
            start: int = 0) -> np.ndarray:
    """Doubles in [lo, hi) from the top 53 bits of each output."""
    u = (u64(seed, stream, n, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def integers(seed: int, stream: int, n: int, count: int, start: int = 0) -> np.ndarray:
    """Integers in [0, count) (floor of a uniform double; count << 2**53)."""
    return np.floor(uniform(seed, stream, n, 0.0, float(count), start)).astype(np.int64)
