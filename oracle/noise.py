"""Z4 noise in the LapH subspace from a counter-based generator.

Sec. IV: a Z_4 noise vector rho(t, i, alpha) is identified by a 16-bit noise
id s and a 16-bit configuration id k, combined into a 32-bit seed m; every
element is drawn from two bits of a random stream in a fixed order.  The paper
draws the bits from the Mersenne twister; this build uses the counter-based
Philox4x32-10 generator instead (Salmon, Moraes, Dror, Shaw, SC'11), so each
element is independently addressable on a GPU.  Reading taken:
    m   = (k << 16) | s
    idx = (t * 4 + alpha) * N_v + n
    w   = Philox4x32-10(counter = (idx, 0, 0, 0), key = (m, 0x4C415048))
    v   = w[0] & 3,   rho(t, alpha, n) = i^v.

Philox4x32-10, from its published definition: ten rounds of
    (hi0, lo0) = mulhilo(0xD2511F53, c0),  (hi1, lo1) = mulhilo(0xCD9E8D57, c2)
    c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
with the key bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85) before
every round after the first.
"""
import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)
KEY1_LAPH = 0x4C415048


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10.  Inputs are integer arrays (or scalars) < 2^32."""
    c = [np.asarray(v, dtype=np.uint64) & _MASK for v in (c0, c1, c2, c3)]
    k0 = int(k0) & 0xFFFFFFFF
    k1 = int(k1) & 0xFFFFFFFF
    for r in range(10):
        if r > 0:
            k0 = (k0 + _W0) & 0xFFFFFFFF
            k1 = (k1 + _W1) & 0xFFFFFFFF
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c = [hi1 ^ c[1] ^ np.uint64(k0), lo1, hi0 ^ c[3] ^ np.uint64(k1), lo0]
    return [v.astype(np.uint32) for v in c]


def noise_seed(noise_id: int, config_id: int) -> int:
    return ((config_id & 0xFFFF) << 16) | (noise_id & 0xFFFF)


def z4_codes(nt: int, nv: int, noise_id: int, config_id: int) -> np.ndarray:
    """uint8 codes v[t, alpha, n] in {0,1,2,3}; rho = i^v."""
    idx = np.arange(nt * 4 * nv, dtype=np.uint64)
    w = philox4x32_10(idx, 0, 0, 0, noise_seed(noise_id, config_id), KEY1_LAPH)
    return (w[0] & 3).astype(np.uint8).reshape(nt, 4, nv)


def z4_values(codes: np.ndarray) -> np.ndarray:
    return (1j) ** codes.astype(np.int64)


# ---------------------------------------------------------------- the paper's generator (oracle only)
# Sec. IV draws the Z4 elements from the Mersenne twister, two bits at a time in a fixed
# order.  Written from its published definition (Matsumoto and Nishimura, ACM TOMACS 8, 1998):
# MT19937 with the 1998/2002 seeding rule init_genrand.  Reading taken for the parts the paper
# leaves open: the generator is seeded with m = (k << 16) | s; element idx = (t*4 + alpha)*N_v + n
# takes bits 2j, 2j+1 (j = idx mod 16) of output word idx // 16, least significant pair first.
# The GPU path keeps the counter-based generator above; this mode exists for fidelity checks.

_MT_N, _MT_M = 624, 397


def mt19937_words(seed: int, count: int) -> np.ndarray:
    """The first `count` 32-bit outputs of MT19937 seeded by init_genrand(seed)."""
    mt = [0] * _MT_N
    mt[0] = seed & 0xFFFFFFFF
    for i in range(1, _MT_N):
        mt[i] = (1812433253 * (mt[i - 1] ^ (mt[i - 1] >> 30)) + i) & 0xFFFFFFFF
    out = []
    idx = _MT_N
    while len(out) < count:
        if idx >= _MT_N:
            for i in range(_MT_N):
                y = (mt[i] & 0x80000000) | (mt[(i + 1) % _MT_N] & 0x7FFFFFFF)
                mt[i] = mt[(i + _MT_M) % _MT_N] ^ (y >> 1) ^ (0x9908B0DF if y & 1 else 0)
            idx = 0
        y = mt[idx]
        idx += 1
        y ^= y >> 11
        y ^= (y << 7) & 0x9D2C5680
        y ^= (y << 15) & 0xEFC60000
        y ^= y >> 18
        out.append(y & 0xFFFFFFFF)
    return np.array(out, dtype=np.uint64)


def z4_codes_mt(nt: int, nv: int, noise_id: int, config_id: int) -> np.ndarray:
    """uint8 codes v[t, alpha, n] from MT19937 two bits at a time (the paper's generator)."""
    n = nt * 4 * nv
    words = mt19937_words(noise_seed(noise_id, config_id), (n + 15) // 16)
    idx = np.arange(n, dtype=np.uint64)
    codes = (words[idx // np.uint64(16)] >> (np.uint64(2) * (idx % np.uint64(16)))) & np.uint64(3)
    return codes.astype(np.uint8).reshape(nt, 4, nv)
