"""Philox4x32-10 counter-based generator and the sample streams built on it.

Test infrastructure (see ``oracle/__init__``).

The generator follows its published definition (J. Salmon, M. Moraes,
R. Dror, D. Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11):
a 128-bit counter (c0,c1,c2,c3) and a 64-bit key (k0,k1); each of ten rounds
multiplies c0 and c2 by the two round multipliers, keeps the 64-bit products'
halves, swaps words and XORs the high halves with the other counter words and
the key; the key is bumped by the two Weyl constants between rounds.

The paper draws its samples from the ``vegas`` library's generator
(Sec. 3A); here a counter-based stream is fixed instead, so that the GPU
and this oracle consume identical samples.  Stream definition (a reading):

  key     = (seed mod 2^32, seed div 2^32)
  counter = (block, iteration, call, task)

For a task evaluated with N samples in D dimensions, uniform number
u = s*D + d (sample s, dimension d) is taken from

  * mode "f32": block u div 4, 32-bit word u mod 4, value x 2^-32 in [0, 1)
    (so that the VEGAS increment floor(x nb / 2^32) and its fraction are the
    high and low halves of the integer product x nb)
  * mode "f64": block u div 2, words (2(u mod 2), 2(u mod 2)+1) = (x0, x1),
                value (((x0 >> 6) 2^26 + (x1 >> 6)) + 1/2) 2^-52 in (0, 1)

Both are exact in FP64, so every order of evaluation gives the same number on
every machine.
"""
import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds on arrays of counters; returns four uint32 arrays.

    ``c0..c3`` are broadcastable integer arrays (values < 2^32); ``k0, k1`` are
    Python ints.  Arithmetic is done in uint64 so that the 32x32 products are
    exact.
    """
    c0, c1, c2, c3 = np.broadcast_arrays(*(np.asarray(c, dtype=np.uint64) for c in (c0, c1, c2, c3)))
    c0, c1, c2, c3 = (c.copy() for c in (c0, c1, c2, c3))
    k0 = np.uint64(k0 & 0xFFFFFFFF)
    k1 = np.uint64(k1 & 0xFFFFFFFF)
    m0 = np.uint64(PHILOX_M0)
    m1 = np.uint64(PHILOX_M1)
    for _ in range(10):
        prod0 = m0 * c0                      # exact: both factors < 2^32
        prod1 = m1 * c2
        hi0, lo0 = prod0 >> np.uint64(32), prod0 & _MASK32
        hi1, lo1 = prod1 >> np.uint64(32), prod1 & _MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + np.uint64(PHILOX_W0)) & _MASK32
        k1 = (k1 + np.uint64(PHILOX_W1)) & _MASK32
    return tuple(c.astype(np.uint32) for c in (c0, c1, c2, c3))


def _words(seed, task, iteration, call, first_block, n_blocks):
    """uint32 words of blocks [first_block, first_block + n_blocks), block-major."""
    blocks = np.arange(first_block, first_block + n_blocks, dtype=np.uint64)
    out = philox4x32_10(blocks, iteration, call, task, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return np.stack(out, axis=1).reshape(-1)


def uniforms(seed, task, iteration, call, n_samples, dim, mode="f64", first_sample=0):
    """Uniforms of samples [first_sample, first_sample + n_samples) as an
    (n_samples, dim) float64 array, following the stream definition above."""
    u0 = first_sample * dim
    n_u = n_samples * dim
    if n_u == 0:
        return np.zeros((n_samples, dim))
    if mode == "f32":
        b0 = u0 // 4
        b1 = (u0 + n_u - 1) // 4 + 1
        w = _words(seed, task, iteration, call, b0, b1 - b0)
        x = w[u0 - 4 * b0: u0 - 4 * b0 + n_u].astype(np.float64)
        v = x * 2.0 ** -32
    elif mode == "f64":
        b0 = u0 // 2
        b1 = (u0 + n_u - 1) // 2 + 1
        w = _words(seed, task, iteration, call, b0, b1 - b0).reshape(-1, 2)
        pair = w[u0 - 2 * b0: u0 - 2 * b0 + n_u]    # (x0, x1) per uniform
        hi = np.floor(pair[:, 0].astype(np.float64) / 64.0)   # x0 >> 6 (26 bits)
        lo = np.floor(pair[:, 1].astype(np.float64) / 64.0)   # x1 >> 6 (26 bits)
        v = ((hi * 2.0 ** 26 + lo) + 0.5) * 2.0 ** -52
    else:
        raise ValueError(mode)
    return v.reshape(n_samples, dim)
