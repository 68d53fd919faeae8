"""Philox4x32-10 counter-based random number generator, FP64 uniform and
normal draws used by the Landau initial condition.

Test infrastructure only (see ``oracle/__init__.py``).

Definition followed: J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11. One Philox-4x32 round
maps counter (c0, c1, c2, c3) and key (k0, k1) to
    (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
with M0 = 0xD2511F53, M1 = 0xCD9E8D57; between rounds the key is bumped by the
Weyl constants (0x9E3779B9, 0xBB67AE85). Ten rounds.

Stream layout (shared convention with the GPU side, each side implementing it
on its own): particle p uses counters (p_lo, p_hi, j, 0) for j = 0..3 and key
(seed_lo, seed_hi). Each call yields four 32-bit words (a, b, c, d) and two
uniforms in (0, 1) with 53-bit resolution:
    u = ((a >> 5) * 2**26 + (b >> 6) + 0.5) * 2**-53,  u' = same for (c, d).
Call 0 -> (u_x, u_y); call 1 -> (u_z, unused); call 2 -> Box-Muller pair
(vx, vy); call 3 -> Box-Muller pair, first value is vz. The sum-form initial
density takes its rejection trials from calls 4, 5, 6, ... (two a trial).
"""
import numpy as np

MASK32 = np.uint64(0xFFFFFFFF)
M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox-4x32 rounds on uint32 values held in uint64 arrays."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & MASK32 for v in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & MASK32
    k1 = np.asarray(k1, dtype=np.uint64) & MASK32
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c0          # < 2**64: exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def uniform_pair(words_a, words_b):
    """53-bit uniform in the open interval (0, 1) from two 32-bit words."""
    a = (words_a >> np.uint64(5)).astype(np.float64)
    b = (words_b >> np.uint64(6)).astype(np.float64)
    return (a * 67108864.0 + b + 0.5) * (1.0 / 9007199254740992.0)


def particle_uniforms(p_index, seed):
    """The eight uniforms of particles ``p_index`` (uint64 array) for ``seed``.

    Returns an array of shape (4, 2, n): [call j][first/second uniform][particle].
    """
    return particle_uniforms_calls(p_index, seed, range(4))


def particle_uniforms_calls(p_index, seed, calls):
    """Uniforms of Philox calls ``calls`` (counter c2 = call) of particles
    ``p_index``: shape (len(calls), 2, n), as particle_uniforms."""
    p = np.asarray(p_index, dtype=np.uint64)
    lo = p & MASK32
    hi = p >> np.uint64(32)
    k0 = np.uint64(seed) & MASK32
    k1 = (np.uint64(seed) >> np.uint64(32)) & MASK32
    calls = list(calls)
    out = np.empty((len(calls), 2, p.size), dtype=np.float64)
    for i, j in enumerate(calls):
        a, b, c, d = philox4x32_10(lo, hi, np.full_like(lo, j), np.zeros_like(lo), k0, k1)
        out[i, 0] = uniform_pair(a, b)
        out[i, 1] = uniform_pair(c, d)
    return out


def box_muller(u1, u2):
    """Two independent N(0, 1) draws from two uniforms in (0, 1) (Box & Muller 1958)."""
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    return rad * np.cos(ang), rad * np.sin(ang)
