"""Counter-based random numbers for the diffusion modules -- TEST INFRASTRUCTURE ONLY.

The paper (Section 4.3, ``module_rng_init`` / ``generate_random_nums``) creates one
cuRAND generator per device, seeded with ``task + 83 * device``, and materialises
arrays of double-precision random numbers for the turbulent-diffusion, mesoscale
and convection modules each time step (the ``randoms_t`` struct).  The method
here keeps the seed form but replaces the stored arrays by a counter-based
generator evaluated where the numbers are used:

* Philox4x32 with 10 rounds, as published by Salmon, Moraes, Dror and Shaw,
  "Parallel Random Numbers: As Easy as 1, 2, 3" (SC'11): a 4 x 32-bit counter
  and a 2 x 32-bit key; each round multiplies counter words 0 and 2 by two
  fixed odd multipliers, exchanges/xors the high and low product halves with
  words 1 and 3 and the key, and the key is bumped by two Weyl increments
  between rounds.
* counter = (particle id, global step index, stream, release id) with
  stream 0 = turbulent diffusion, 1 = mesoscale diffusion;
  key = (seed & 0xffffffff, seed >> 32).  Keying on the particle id (not its
  array slot) makes results independent of the particle order.
* Uniform u = ((x >> 9) + 1/2) * 2^-23, exactly representable in float32 and
  float64, so both precisions see the same u in (0, 1).
* Box-Muller: for word pairs (x0, x1) and (x2, x3),
  z_a = sqrt(-2 ln u_a) cos(2 pi u_b), z_b = sqrt(-2 ln u_a) sin(2 pi u_b).
"""
from __future__ import annotations

import numpy as np

MASK32 = np.uint64(0xFFFFFFFF)
# Round multipliers and Weyl key increments of Philox4x32 as published in the SC'11 paper.
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint64(0x9E3779B9)
PHILOX_W1 = np.uint64(0xBB67AE85)

STREAM_TURB = 0
STREAM_MESO = 1


def philox4x32(c0, c1, c2, c3, k0, k1, rounds: int = 10):
    """Philox4x32-``rounds`` of counter (c0..c3) under key (k0, k1).

    Arguments are integer arrays/scalars holding 32-bit values; the result is a
    tuple of four uint32 arrays.  Products are formed exactly in uint64.
    """
    x = [np.asarray(c, dtype=np.uint64) & MASK32 for c in (c0, c1, c2, c3)]
    x = list(np.broadcast_arrays(*x))
    x = [a.copy() for a in x]
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for r in range(rounds):
        if r > 0:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        prod0 = PHILOX_M0 * x[0]
        prod1 = PHILOX_M1 * x[2]
        hi0, lo0 = prod0 >> np.uint64(32), prod0 & MASK32
        hi1, lo1 = prod1 >> np.uint64(32), prod1 & MASK32
        x = [hi1 ^ x[1] ^ k0, lo1, hi0 ^ x[3] ^ k1, lo0]
    return tuple(a.astype(np.uint32) for a in x)


def seed_key(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def default_seed(task: int = 0, device: int = 0) -> int:
    """Seed of the paper's generator for MPI task ``task`` on GPU ``device`` (Section 4.3)."""
    return task + 83 * device


def uniform23(x):
    """uint32 word -> uniform in (0, 1) from its top 23 bits (exact in float32)."""
    x = np.asarray(x, dtype=np.uint32)
    return ((x >> np.uint32(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def box_muller(ua, ub):
    r = np.sqrt(-2.0 * np.log(ua))
    ang = 2.0 * np.pi * ub
    return r * np.cos(ang), r * np.sin(ang)


def words(pid, step, stream, release, seed):
    """Raw Philox words for particles ``pid`` at global step ``step`` on ``stream``."""
    k0, k1 = seed_key(seed)
    return philox4x32(pid, step, stream, release, k0, k1)


def normals4(pid, step, stream, release, seed):
    """Four standard normals per particle from one Philox call (float64)."""
    x0, x1, x2, x3 = words(pid, step, stream, release, seed)
    z0, z1 = box_muller(uniform23(x0), uniform23(x1))
    z2, z3 = box_muller(uniform23(x2), uniform23(x3))
    return z0, z1, z2, z3
