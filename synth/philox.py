"""Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11), vectorised over numpy uint64 arrays.

Holds no arithmetic of the blocked linear method: it only turns (key, counter) pairs into
random bits, 53-bit uniforms and Box-Muller normals.  The CUDA twin in synth/csrc/synth.cu
implements the same published definition; the two agree bit for bit on the integer output.
"""
import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox rounds on 4x32-bit counters (uint64 arrays holding 32-bit values)."""
    c0 = np.asarray(c0, dtype=np.uint64) & _MASK
    c1 = np.asarray(c1, dtype=np.uint64) & _MASK
    c2 = np.asarray(c2, dtype=np.uint64) & _MASK
    c3 = np.asarray(c3, dtype=np.uint64) & _MASK
    k0 = np.uint64(k0) & _MASK
    k1 = np.uint64(k1) & _MASK
    for r in range(10):
        if r:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0          # < 2^64, exact in uint64
        p1 = _M1 * c2
        hi0, lo0 = p0 >> _S32, p0 & _MASK
        hi1, lo1 = p1 >> _S32, p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def _u53(a, b):
    """Uniform on the open interval (0, 1) from two 32-bit words: 53 random bits + 1/2 ulp."""
    return ((a >> np.uint64(5)).astype(np.float64) * 67108864.0
            + (b >> np.uint64(6)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def uniform(seed, opt, tag, idx):
    """One U(0,1) per 64-bit index; key=(seed, opt), counter=(idx_lo, idx_hi, tag, 0)."""
    idx = np.asarray(idx, dtype=np.uint64)
    x0, x1, _, _ = philox4x32_10(idx & _MASK, idx >> _S32, np.uint64(tag), np.uint64(0), seed, opt)
    return _u53(x0, x1)


def normal(seed, opt, tag, idx):
    """One N(0,1) per 64-bit index by Box-Muller: sqrt(-2 ln u1) * cos(2 pi u2)."""
    idx = np.asarray(idx, dtype=np.uint64)
    x0, x1, x2, x3 = philox4x32_10(idx & _MASK, idx >> _S32, np.uint64(tag), np.uint64(0), seed, opt)
    u1 = _u53(x0, x1)
    u2 = _u53(x2, x3)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
