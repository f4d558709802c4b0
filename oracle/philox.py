"""Counter-based random numbers for the oracle: Philox4x32-10 and Box-Muller.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package;
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.

The paper's HMC kernel draws "one independent momentum per state variable per
chain" (Section 2.1, "Case Study: HMC") and a uniform for the
Metropolis-Hastings test, but names no generator.  Both this oracle and the
CUDA path implement the same counter-based generator, Philox4x32 with 10
rounds, from its published definition (Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11), so the two sides draw
identical 32-bit words without sharing code.  Only the conversion of those
words to floats differs: here it is done in float64.

Stream layout (the same reading is used on both sides):
  key     = (seed & 0xffffffff, seed >> 32)
  counter = (block j, chain c, transition t, stream tag s)
  s = 0: momentum; word 4j+i of chain c feeds state dimension 4j+i via
         Box-Muller on the pairs (w0, w1) and (w2, w3).
  s = 1: Metropolis-Hastings uniform; word 0 of block 0.
  Uniforms are u = (w + 0.5) * 2**-32, strictly inside (0, 1).
"""
import numpy as np

# Multipliers and Weyl key increments of Philox4x32 (Salmon et al. 2011, Table 2
# and Section 4.2).
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)

TAG_MOMENTUM = 0
TAG_ACCEPT = 1


def philox4x32_10(counter, key):
    """Apply 10 Philox rounds to an (n, 4) array of uint32 counters.

    ``key`` is a pair of uint32 (k0, k1).  Each round multiplies words 0 and 2
    by the two constants, splits the 64-bit products into high and low halves,
    and forms (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is bumped by
    the Weyl constants between rounds.  Returns an (n, 4) uint32 array.
    """
    c = np.asarray(counter, dtype=np.uint64).reshape(-1, 4) & _MASK
    c0, c1, c2, c3 = (c[:, i].copy() for i in range(4))
    k0 = np.uint64(int(key[0]) & 0xFFFFFFFF)
    k1 = np.uint64(int(key[1]) & 0xFFFFFFFF)
    for _ in range(10):
        p0 = _M0 * c0            # < 2**64: both factors are below 2**32
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & _MASK, lo1, (hi0 ^ c3 ^ k1) & _MASK, lo0
        k0 = (k0 + _W0) & _MASK
        k1 = (k1 + _W1) & _MASK
    return np.stack([c0, c1, c2, c3], axis=1).astype(np.uint32)


def seed_key(seed):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return (seed & 0xFFFFFFFF, seed >> 32)


def words_to_uniform(w):
    """Map uint32 words to float64 uniforms (w + 1/2) / 2**32 in (0, 1)."""
    return (np.asarray(w, dtype=np.float64) + 0.5) * 2.0 ** -32


def box_muller(w_a, w_b):
    """Two uint32 words -> two independent N(0,1) draws (Box and Muller 1958):
    r = sqrt(-2 log u_a), (r cos 2 pi u_b, r sin 2 pi u_b)."""
    ua = words_to_uniform(w_a)
    ub = words_to_uniform(w_b)
    r = np.sqrt(-2.0 * np.log(ua))
    return r * np.cos(2.0 * np.pi * ub), r * np.sin(2.0 * np.pi * ub)


def momentum(seed, transition, num_chains, dim, chain_offset=0):
    """Momentum p ~ N(0, I) of shape (num_chains, dim) for one transition.

    Chain c uses counters (j, chain_offset + c, transition, TAG_MOMENTUM) for
    j = 0 .. ceil(dim / 4) - 1; unused normals past ``dim`` are dropped.
    """
    nblk = (dim + 3) // 4
    j, c = np.meshgrid(np.arange(nblk), np.arange(num_chains) + chain_offset,
                       indexing="xy")
    ctr = np.stack([j.ravel(), c.ravel(),
                    np.full(j.size, transition & 0xFFFFFFFF),
                    np.full(j.size, TAG_MOMENTUM)], axis=1)
    w = philox4x32_10(ctr, seed_key(seed))
    z0, z1 = box_muller(w[:, 0], w[:, 1])
    z2, z3 = box_muller(w[:, 2], w[:, 3])
    z = np.stack([z0, z1, z2, z3], axis=1).reshape(num_chains, nblk * 4)
    return z[:, :dim]


def accept_uniform(seed, transition, num_chains, chain_offset=0):
    """Uniform u in (0, 1) per chain for the Metropolis-Hastings test."""
    c = np.arange(num_chains) + chain_offset
    ctr = np.stack([np.zeros_like(c), c,
                    np.full(c.size, transition & 0xFFFFFFFF),
                    np.full(c.size, TAG_ACCEPT)], axis=1)
    w = philox4x32_10(ctr, seed_key(seed))
    return words_to_uniform(w[:, 0])
