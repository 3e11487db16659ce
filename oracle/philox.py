"""Philox4x32-10 and the Rademacher noise vectors of the Hutchinson estimator.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper draws the noise vectors x_j with i.i.d. entries uniform on {+1, -1}
(Sec. 1, text after Eq. 1: "Rademacher vectors").  The paper does not say how
the signs are generated; this library's reading is a counter-based generator
so that every (seed, sample, dof) triple has one fixed sign on any device:

* generator: Philox4x32 with 10 rounds, as defined by Salmon, Moraes, Dror and
  Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11): a 4x32-bit
  counter, a 2x32-bit key, per round two 32x32->64-bit products with the
  multipliers 0xD2511F53 and 0xCD9E8D57, and a Weyl key schedule with the
  increments 0x9E3779B9 and 0xBB67AE85;
* noise: dof i of sample j (i = 12*lex_site + 3*spin + colour) takes bit
  (i mod 128) of the 128-bit block Philox(counter=(i // 128, j, 0, 0),
  key=(seed & 0xffffffff, seed >> 32)); word (i mod 128)//32, bit i mod 32.
  Bit 0 gives +1 and bit 1 gives -1.  The imaginary part is 0 (real noise).
* random starts for the multigrid setup (Sec. 2, "n different random initial
  guesses"): null vector v, dof i takes re from bit 2*(i mod 64) and im from
  bit 2*(i mod 64)+1 of Philox(counter=(i // 64, v, 1, 0), key as above), each
  bit mapped 0 -> +1, 1 -> -1.

Pinned by the published Philox4x32-10 known-answer vectors
(``tests/golden/philox4x32_10_kat.txt``) and by the moments of the noise.
"""

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Philox4x32-10 block function (Salmon et al., SC'11).

    ``ctr``: uint array (..., 4) of 32-bit counter words; ``key``: pair of
    32-bit key words, either a tuple or an array (..., 2).  Returns a uint32
    array (..., 4).  Vectorised over leading dimensions.
    """
    c = np.asarray(ctr, dtype=np.uint64) & _MASK32
    k = np.asarray(key, dtype=np.uint64) & _MASK32
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0 = np.broadcast_to(k[..., 0], c0.shape).copy()
    k1 = np.broadcast_to(k[..., 1], c0.shape).copy()
    for rnd in range(10):
        if rnd > 0:  # key schedule: add the Weyl constants before rounds 2..10
            k0 = (k0 + np.uint64(_W0)) & _MASK32
            k1 = (k1 + np.uint64(_W1)) & _MASK32
        p0 = _M0 * c0  # exact: both factors < 2^32, product < 2^64
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def _seed_key(seed):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint64)


def rademacher(ndof, seed, samples):
    """Real Rademacher noise, shape (ndof, len(samples)), values +-1.0.

    Row i is the dof 12*lex_site + 3*spin + colour; column j is the global
    sample index ``samples[j]`` (the estimator's x_j, Sec. 1).
    """
    samples = np.asarray(samples, dtype=np.int64)
    i = np.arange(ndof, dtype=np.int64)
    blk = i // 128
    nblk = int(blk[-1]) + 1 if ndof else 0
    key = _seed_key(seed)
    out = np.empty((ndof, samples.size), dtype=np.float64)
    for col, j in enumerate(samples):
        ctr = np.zeros((nblk, 4), dtype=np.uint64)
        ctr[:, 0] = np.arange(nblk, dtype=np.uint64)
        ctr[:, 1] = np.uint64(int(j) & 0xFFFFFFFF)
        words = philox4x32_10(ctr, key)  # (nblk, 4)
        w = words[blk, (i % 128) // 32].astype(np.uint64)
        bit = (w >> (i % 32).astype(np.uint64)) & np.uint64(1)
        out[:, col] = 1.0 - 2.0 * bit.astype(np.float64)
    return out


def random_starts(ndof, seed, nvec):
    """Complex +-1 +-i starting vectors for the adaptive setup, (ndof, nvec)."""
    i = np.arange(ndof, dtype=np.int64)
    blk = i // 64
    nblk = int(blk[-1]) + 1 if ndof else 0
    key = _seed_key(seed)
    out = np.empty((ndof, nvec), dtype=np.complex128)
    pos = 2 * (i % 64)
    for v in range(nvec):
        ctr = np.zeros((nblk, 4), dtype=np.uint64)
        ctr[:, 0] = np.arange(nblk, dtype=np.uint64)
        ctr[:, 1] = np.uint64(v)
        ctr[:, 2] = np.uint64(1)
        words = philox4x32_10(ctr, key)
        w_re = words[blk, pos // 32].astype(np.uint64)
        w_im = words[blk, (pos + 1) // 32].astype(np.uint64)
        b_re = (w_re >> (pos % 32).astype(np.uint64)) & np.uint64(1)
        b_im = (w_im >> ((pos + 1) % 32).astype(np.uint64)) & np.uint64(1)
        out[:, v] = (1.0 - 2.0 * b_re) + 1j * (1.0 - 2.0 * b_im)
    return out
