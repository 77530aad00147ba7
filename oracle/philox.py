"""Philox4x32-10 counter-based generator and the Gaussian stream built on it.

The generator is Philox4x32 with 10 rounds from Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC'11): each round maps the
counter ``(c0, c1, c2, c3)`` with key ``(k0, k1)`` to
``(hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))`` with
``M0 = 0xD2511F53``, ``M1 = 0xCD9E8D57``, and the key is bumped by the Weyl
constants ``(0x9E3779B9, 0xBB67AE85)`` between rounds.

Gaussian stream (the definition both sides implement): element ``e`` of the
stream ``(seed, stream)`` uses counter ``(lo(e//2), hi(e//2), lo(stream),
hi(stream))`` and key ``(lo(seed), hi(seed))``.  The four output words give two
uniforms ``u = ((w_a << 32 | w_b) >> 11 + 0.5) * 2^-53`` in (0, 1), and the
Box-Muller pair ``sqrt(-2 ln u1) (cos, sin)(2 pi u2)``; element ``e`` takes the
cosine branch when even and the sine branch when odd.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Vectorised Philox4x32-10.  ``ctr`` has shape ``(..., 4)`` and ``key``
    shape ``(..., 2)`` (uint32 values); returns the four output words."""
    c = [np.asarray(ctr[..., i], dtype=np.uint64) & MASK for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint64) & MASK
    k1 = np.asarray(key[..., 1], dtype=np.uint64) & MASK
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c = [(hi1 ^ c[1] ^ k0) & MASK, lo1, (hi0 ^ c[3] ^ k1) & MASK, lo0]
    return np.stack([x.astype(np.uint32) for x in c], axis=-1)


def gaussian(count: int, seed: int, stream: int, std: float = 1.0) -> np.ndarray:
    """``count`` elements of the Gaussian stream ``(seed, stream)`` times
    ``std``, in float64."""
    e = np.arange(count, dtype=np.uint64)
    c = e >> np.uint64(1)
    ctr = np.stack([c & MASK, c >> np.uint64(32),
                    np.full_like(c, np.uint64(stream) & MASK),
                    np.full_like(c, np.uint64(stream) >> np.uint64(32))], axis=-1)
    key = np.stack([np.full_like(c, np.uint64(seed) & MASK),
                    np.full_like(c, np.uint64(seed) >> np.uint64(32))], axis=-1)
    w = philox4x32_10(ctr, key).astype(np.uint64)
    a = ((w[:, 0] << np.uint64(32)) | w[:, 1]) >> np.uint64(11)
    b = ((w[:, 2] << np.uint64(32)) | w[:, 3]) >> np.uint64(11)
    u1 = (a.astype(np.float64) + 0.5) * 2.0 ** -53
    u2 = (b.astype(np.float64) + 0.5) * 2.0 ** -53
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    even = (e & np.uint64(1)) == 0
    return np.where(even, rad * np.cos(ang), rad * np.sin(ang)) * std


# Stream ids of the solver's random draws.
STREAM_SKETCH = 1      # Khatri-Rao factor k uses stream STREAM_SKETCH * 1024 + k
STREAM_DRM = 2         # TT-DRM core k uses stream STREAM_DRM * 1024 + k


def sketch_factors(ns, s, seed):
    """Khatri-Rao factors ``S_k`` (``[s, n_k]``, variance ``s^{-1/d}``) drawn
    from the Gaussian stream, factor k from stream ``1024 + k``."""
    d = len(ns)
    std = float(s) ** (-0.5 / d)
    return [gaussian(s * n, seed, STREAM_SKETCH * 1024 + k, std).reshape(s, n)
            for k, n in enumerate(ns)]


def drm_cores(ns, ells, seed):
    """TT-DRM cores ``[l_{k-1}, n_k, l_k]`` with variance ``1/(l_{k-1} n_k l_k)``
    drawn from streams ``2048 + k``."""
    out = []
    for k, n in enumerate(ns):
        a, b = ells[k], ells[k + 1]
        std = 1.0 / np.sqrt(a * n * b)
        out.append(gaussian(a * n * b, seed, STREAM_DRM * 1024 + k, std).reshape(a, n, b))
    return out
