"""Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11) and the draws the
sampler makes from it (oracle).

One block: 128-bit key (k0, k1), 256-bit counter (x0, x1, x2, x3); ten rounds of
  (hi0, lo0) = M0 * x0,  (hi1, lo1) = M1 * x2            (64 x 64 -> 128-bit products)
  (x0, x1, x2, x3) <- (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0)
  (k0, k1) <- (k0 + W0, k1 + W1)                          (mod 2^64)
with the published multipliers M0, M1 and Weyl increments W0, W1 below.

Stream layout used by the sampler (each chain has its own key, so chains are independent):
  key     = (seed, chain)
  counter = (block, iteration, purpose, 0),  purpose 0 = momentum normals, 1 = MH uniform
Normals: block b yields z[4b .. 4b+3] by Box-Muller on the pairs (x0, x1) and (x2, x3):
  u1 = ((x >> 11) + 1) 2^-53 in (0, 1],  u2 = (x >> 11) 2^-53 in [0, 1)
  z_a = sqrt(-2 log u1) cos(2 pi u2),   z_b = sqrt(-2 log u1) sin(2 pi u2)
MH uniform: r = (x0 >> 11) 2^-53 of block 0.
"""
import numpy as np

MASK = (1 << 64) - 1
M0 = 0xD2E7470EE14C6C93
M1 = 0xCA5A826395121157
W0 = 0x9E3779B97F4A7C15
W1 = 0xBB67AE8584CAA73B

PURPOSE_MOMENTUM = 0
PURPOSE_ACCEPT = 1


def philox4x64_10(counter, key):
    """One Philox4x64-10 block: returns four 64-bit words (Python ints)."""
    x0, x1, x2, x3 = (int(v) & MASK for v in counter)
    k0, k1 = (int(v) & MASK for v in key)
    for _ in range(10):
        p0 = M0 * x0
        p1 = M1 * x2
        hi0, lo0 = p0 >> 64, p0 & MASK
        hi1, lo1 = p1 >> 64, p1 & MASK
        x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
        k0 = (k0 + W0) & MASK
        k1 = (k1 + W1) & MASK
    return [x0, x1, x2, x3]


def _u_open0(x):
    return ((x >> 11) + 1) * (2.0 ** -53)


def _u_closed0(x):
    return (x >> 11) * (2.0 ** -53)


def normals(seed, chain, iteration, d):
    """d standard normals for the momentum draw of `iteration` of `chain`."""
    z = np.empty(4 * ((d + 3) // 4))
    for b in range(len(z) // 4):
        w = philox4x64_10((b, iteration, PURPOSE_MOMENTUM, 0), (seed, chain))
        for pair in range(2):
            u1 = _u_open0(w[2 * pair])
            u2 = _u_closed0(w[2 * pair + 1])
            r = np.sqrt(-2.0 * np.log(u1))
            z[4 * b + 2 * pair] = r * np.cos(2.0 * np.pi * u2)
            z[4 * b + 2 * pair + 1] = r * np.sin(2.0 * np.pi * u2)
    return z[:d]


def mh_uniform(seed, chain, iteration):
    """The uniform r in [0, 1) of the Metropolis-Hastings test of `iteration` of `chain`."""
    w = philox4x64_10((0, iteration, PURPOSE_ACCEPT, 0), (seed, chain))
    return _u_closed0(w[0])
