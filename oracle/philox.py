"""Random input Theta ~ N(0, 1/d) of Alg. 1 and Eq. 4's Z^(0), from a seed.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product library has
its own, separately written generator and never imports this module.

The paper only says that Z^(0) = Theta is Gaussian noise with variance 1/d
(Sec. III-A, Eq. 4; the random input of Alg. 1). To make that noise reproducible on both
sides, row i / column c of Theta is a fixed function of (seed, i, c):

* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
  as 1, 2, 3", SC 2011) maps the 256-bit counter (i, q, 0, 0) and the 128-bit
  key (seed, 0) to four 64-bit words; q = c // 8 is the column block.
* Each 64-bit word is split into its low and high 32-bit halves, giving eight
  32-bit words w_0..w_7 (word k -> half k % 2 of output k // 2).
* Each w_k gives a uniform u_k = ((w_k >> 8) + 1) * 2^-24 in (0, 1]; the value
  is exact in both fp32 and fp64, and never 0, so log(u) is finite.
* Box-Muller on the pairs (u_{2p}, u_{2p+1}):
      r = sqrt(-2 ln u_{2p}),  z_{2p} = r cos(2 pi u_{2p+1}),
      z_{2p+1} = r sin(2 pi u_{2p+1}),
  giving eight independent standard normals for columns 8q .. 8q+7.
* Theta[i, c] = z_{c % 8} * x_scale with x_scale = 1/sqrt(d) (the paper's
  variance 1/d) unless another scale is asked for.

Rows depend only on (seed, i), so the rows of old nodes do not change when a
streaming graph grows (each step of Alg. 2 still draws a fresh N(0, 1/d) matrix
for a fresh seed).
"""
import numpy as np

_M32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)

# Philox4x64 round multipliers and Weyl key increments (Salmon et al. 2011).
PHILOX_M0 = np.uint64(0xD2E7470EE14C6C93)
PHILOX_M1 = np.uint64(0xCA5A826395121157)
PHILOX_W0 = np.uint64(0x9E3779B97F4A7C15)
PHILOX_W1 = np.uint64(0xBB67AE8584CAA73B)


def _mulhilo64(a, b):
    """Full 128-bit product of two uint64 arrays, returned as (hi, lo) uint64."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    a_lo, a_hi = a & _M32, a >> _S32
    b_lo, b_hi = b & _M32, b >> _S32
    p0 = a_lo * b_lo
    p1 = a_lo * b_hi
    p2 = a_hi * b_lo
    p3 = a_hi * b_hi
    mid = (p0 >> _S32) + (p1 & _M32) + (p2 & _M32)  # < 3 * 2^32, no overflow
    lo = (p0 & _M32) | ((mid & _M32) << _S32)
    hi = p3 + (p1 >> _S32) + (p2 >> _S32) + (mid >> _S32)
    return hi, lo


def philox4x64_10(ctr, key):
    """Philox4x64 with 10 rounds.

    ctr: uint64 array of shape (..., 4); key: uint64 array of shape (..., 2)
    (broadcastable). Returns the four output words, shape (..., 4).
    """
    ctr = np.array(ctr, dtype=np.uint64, copy=True)
    key = np.array(key, dtype=np.uint64, copy=True)
    c0, c1, c2, c3 = ctr[..., 0], ctr[..., 1], ctr[..., 2], ctr[..., 3]
    k0 = np.broadcast_to(key[..., 0], c0.shape).copy()
    k1 = np.broadcast_to(key[..., 1], c0.shape).copy()
    with np.errstate(over="ignore"):
        for rnd in range(10):
            if rnd > 0:  # the key is bumped between rounds
                k0 = k0 + PHILOX_W0
                k1 = k1 + PHILOX_W1
            hi0, lo0 = _mulhilo64(PHILOX_M0, c0)
            hi1, lo1 = _mulhilo64(PHILOX_M1, c2)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1)


def uniforms_from_words(x):
    """Four 64-bit Philox words (..., 4) -> eight uniforms in (0, 1], shape (..., 8)."""
    x = np.asarray(x, dtype=np.uint64)
    w = np.empty(x.shape[:-1] + (8,), dtype=np.uint64)
    w[..., 0::2] = x & _M32
    w[..., 1::2] = x >> _S32
    return ((w >> np.uint64(8)) + np.uint64(1)).astype(np.float64) * (2.0 ** -24)


def box_muller(u):
    """Uniform pairs (..., 8) -> eight standard normals (..., 8), in fp64."""
    u = np.asarray(u, dtype=np.float64)
    ua, ub = u[..., 0::2], u[..., 1::2]
    r = np.sqrt(-2.0 * np.log(ua))
    z = np.empty_like(u)
    z[..., 0::2] = r * np.cos(2.0 * np.pi * ub)
    z[..., 1::2] = r * np.sin(2.0 * np.pi * ub)
    return z


def theta_input(seed, N, d, x_scale=None, row0=0):
    """Theta in R^{N x d} (fp64) for rows row0 .. row0+N-1; d must be a multiple of 8."""
    if d % 8 != 0:
        raise ValueError("d must be a multiple of 8")
    if x_scale is None:
        x_scale = 1.0 / np.sqrt(d)
    nq = d // 8
    rows = np.arange(row0, row0 + N, dtype=np.uint64)
    ctr = np.zeros((N, nq, 4), dtype=np.uint64)
    ctr[..., 0] = rows[:, None]
    ctr[..., 1] = np.arange(nq, dtype=np.uint64)[None, :]
    key = np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF), np.uint64(0)], dtype=np.uint64)
    words = philox4x64_10(ctr, key)
    z = box_muller(uniforms_from_words(words))  # (N, nq, 8)
    return z.reshape(N, d) * float(x_scale)
