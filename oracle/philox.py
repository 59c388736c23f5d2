"""Philox4x64-10 and the method's Gaussian draws (oracle side).

Test infrastructure only (see the package docstring).

Philox4x64-10 is the counter-based generator of Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC'11): a 4x64-bit counter is
mapped through 10 rounds of two 64x64->128-bit multiplies, with the key bumped
by two Weyl constants between rounds. This module restates that published
definition; the CUDA side has its own, independent implementation of the same
definition, and the two share no code.

Draw convention used by both sides of the method (the paper only asks for
G ~ N(0,1)^{d x l} in Alg. 1 and x uniform on the unit sphere in Alg. 6):

* key     = (seed, 0)
* counter = (block, buffer b, attempt r, tag) with tag 1 for G, 2 for x
* block j yields four words w0..w3; each becomes a uniform
  u = ((w >> 40) + 0.5) * 2**-24 in (0, 1)
* Box-Muller: (u0, u1) -> sqrt(-2 ln u0) * (cos 2 pi u1, sin 2 pi u1), and the
  same for (u2, u3); normal number 4j+k is the k-th of the four.
* G[j, c] (row-major d x l) is normal number j*l + c of tag 1;
  x is normals 0..d-1 of tag 2, divided by their Euclidean norm.
"""
import numpy as np

# Multipliers and Weyl key increments of Philox4x64 (SC'11, Sec. 3.3 / Table 2).
PHILOX_M0 = 0xD2E7470EE14C6C93
PHILOX_M1 = 0xCA5A826395121157
PHILOX_W0 = 0x9E3779B97F4A7C15
PHILOX_W1 = 0xBB67AE8584CAA73B

TAG_G = 1
TAG_VS = 2

_MASK32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo64(a, b):
    """Full 64x64 -> 128-bit product of uint64 arrays, as (hi, lo)."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    a_lo, a_hi = a & _MASK32, a >> _S32
    b_lo, b_hi = b & _MASK32, b >> _S32
    ll = a_lo * b_lo
    lh = a_lo * b_hi
    hl = a_hi * b_lo
    hh = a_hi * b_hi
    mid = (ll >> _S32) + (lh & _MASK32) + (hl & _MASK32)
    lo = (ll & _MASK32) | ((mid & _MASK32) << _S32)
    hi = hh + (lh >> _S32) + (hl >> _S32) + (mid >> _S32)
    return hi, lo


def philox4x64_10(counter, key):
    """Philox4x64 with 10 rounds.

    counter: uint64 array of shape (..., 4); key: pair of ints.
    Returns uint64 array of shape (..., 4).
    """
    ctr = np.array(counter, dtype=np.uint64, copy=True)
    x0, x1, x2, x3 = ctr[..., 0], ctr[..., 1], ctr[..., 2], ctr[..., 3]
    k0 = np.uint64(key[0] & 0xFFFFFFFFFFFFFFFF)
    k1 = np.uint64(key[1] & 0xFFFFFFFFFFFFFFFF)
    m0, m1 = np.uint64(PHILOX_M0), np.uint64(PHILOX_M1)
    w0, w1 = np.uint64(PHILOX_W0), np.uint64(PHILOX_W1)
    with np.errstate(over="ignore"):
        for rnd in range(10):
            hi0, lo0 = _mulhilo64(m0, x0)
            hi1, lo1 = _mulhilo64(m1, x2)
            x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
            if rnd != 9:
                k0 = k0 + w0
                k1 = k1 + w1
    return np.stack([x0, x1, x2, x3], axis=-1)


def uniforms24(words):
    """Map 64-bit words to uniforms ((w >> 40) + 0.5) * 2^-24 in (0, 1)."""
    return ((np.asarray(words, dtype=np.uint64) >> np.uint64(40)).astype(np.float64) + 0.5) * 2.0 ** -24


def box_muller(u_a, u_b):
    """Two independent N(0,1) numbers from two uniforms (Box and Muller, 1958)."""
    rad = np.sqrt(-2.0 * np.log(u_a))
    ang = 2.0 * np.pi * u_b
    return rad * np.cos(ang), rad * np.sin(ang)


def normals(seed, b, r, tag, count):
    """The first `count` normal numbers of stream (seed, b, r, tag), float64."""
    nblk = (count + 3) // 4
    ctr = np.zeros((nblk, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(nblk, dtype=np.uint64)
    ctr[:, 1] = np.uint64(b)
    ctr[:, 2] = np.uint64(r)
    ctr[:, 3] = np.uint64(tag)
    words = philox4x64_10(ctr, (seed, 0))
    u = uniforms24(words)
    z0, z1 = box_muller(u[:, 0], u[:, 1])
    z2, z3 = box_muller(u[:, 2], u[:, 3])
    out = np.stack([z0, z1, z2, z3], axis=1).reshape(-1)
    return out[:count]


def gaussian_G(seed, b, r, d, ell):
    """G ~ N(0,1)^{d x l} of Alg. 1 for buffer b, attempt r (row-major)."""
    return normals(seed, b, r, TAG_G, d * ell).reshape(d, ell)


def sphere_x(seed, b, r, d):
    """x uniform on the unit sphere of R^d for Alg. 6 (normalised Gaussian)."""
    z = normals(seed, b, r, TAG_VS, d)
    return z / np.linalg.norm(z)
