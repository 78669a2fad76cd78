"""Counter-based random numbers for the seeded workloads.

SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) used as a stateless hash of (seed, stream, index):
the i-th number of a stream never depends on how many numbers were drawn
before it, so the generator, the device path and the CPU checker can all
draw the same values by counter.  Only numpy integer arithmetic is used, so
the bits are identical on x86-64 and aarch64.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_S30 = np.uint64(30)
_S27 = np.uint64(27)
_S31 = np.uint64(31)
_S11 = np.uint64(11)


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser applied element-wise (wrapping uint64)."""
    z = np.asarray(z, dtype=np.uint64).copy()
    z ^= z >> _S30
    z *= _M1
    z ^= z >> _S27
    z *= _M2
    z ^= z >> _S31
    return z


def _stream_key(seed: int, stream: int) -> np.uint64:
    a = mix64(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))
    b = mix64(np.array([(stream * 0x2545F4914F6CDD1D) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))
    return (a ^ b)[0]


def bits(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n 64-bit words of stream `stream` of `seed`, starting at counter `offset`."""
    key = _stream_key(seed, stream)
    ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    return mix64(ctr * _GOLDEN + key)


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles uniform in [0, 1) (53 random bits each)."""
    return (bits(seed, stream, n, offset) >> _S11).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normal doubles by the Box-Muller transform."""
    m = (n + 1) // 2
    u1 = uniform(seed, stream, m, 0)
    u2 = uniform(seed, stream, m, m)
    r = np.sqrt(-2.0 * np.log1p(-u1))  # 1-u1 in (0, 1]
    z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
    return z[:n]
