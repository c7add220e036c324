"""Philox4x64-10 and the Z4 noise (oracle).

The Hutchinson samples of Sec. 1 (Eq. Hutchinson) use iid entries with
E x_i = 0 and E conj(x_i) x_j = delta_ij; the paper takes the Z4 distribution
x_i in {1, -1, i, -i} with probability 1/4 each (Eq. z4).  The draw is made
reproducible and order-free with the counter-based Philox4x64-10 generator of
Salmon, Moraes, Dror and Shaw ("Parallel random numbers: as easy as 1, 2, 3",
SC'11), written here from that definition in plain uint64 numpy arithmetic:

  round(c, k):  (hi0, lo0) = M0 * c0,  (hi1, lo1) = M1 * c2      (128-bit)
                c' = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
  10 rounds; after each round but the last the key is bumped by the Weyl
  constants (k0 += W0, k1 += W1).

Z4 map (the reading taken here; the paper fixes only the
distribution): entry i of a noise vector draws the Philox block with counter
(i >> 2, sample, term, aux) and key (seed, 0), takes word i & 3 of it and sets
r = word >> 62 and x_i = i^r  (r = 0, 1, 2, 3 -> 1, i, -1, -i).
"""
import numpy as np

M0 = np.uint64(0xD2E7470EE14C6C93)
M1 = np.uint64(0xCA5A826395121157)
W0 = np.uint64(0x9E3779B97F4A7C15)
W1 = np.uint64(0xBB67AE8584CAA73B)
_M32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def mulhilo64(a, b):
    """(hi, lo) of the 128-bit product of uint64 arrays, from 32-bit halves."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    al, ah = a & _M32, a >> _S32
    bl, bh = b & _M32, b >> _S32
    p0 = al * bl
    p1 = al * bh
    p2 = ah * bl
    p3 = ah * bh
    mid = (p0 >> _S32) + (p1 & _M32) + (p2 & _M32)
    lo = (p0 & _M32) | ((mid & _M32) << _S32)
    hi = p3 + (p1 >> _S32) + (p2 >> _S32) + (mid >> _S32)
    return hi, lo


def philox4x64_10(ctr, key):
    """ctr: (..., 4) uint64, key: (..., 2) uint64 -> (..., 4) uint64."""
    c = [np.asarray(ctr[..., i], dtype=np.uint64).copy() for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint64).copy()
    k1 = np.asarray(key[..., 1], dtype=np.uint64).copy()
    with np.errstate(over='ignore'):
        for r in range(10):
            if r > 0:
                k0 = k0 + W0
                k1 = k1 + W1
            hi0, lo0 = mulhilo64(M0, c[0])
            hi1, lo1 = mulhilo64(M1, c[2])
            c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack(c, axis=-1)


Z4_VALUES = np.array([1.0, 1.0j, -1.0, -1.0j], dtype=np.complex128)


def z4_codes(n, seed, sample, term, aux=0, index=None):
    """r_i in {0,1,2,3} for entries i (all of 0..n-1 when index is None)."""
    i = np.arange(n, dtype=np.uint64) if index is None else np.asarray(index, dtype=np.uint64)
    ctr = np.zeros(i.shape + (4,), dtype=np.uint64)
    ctr[..., 0] = i >> np.uint64(2)
    ctr[..., 1] = np.uint64(sample)
    ctr[..., 2] = np.uint64(term)
    ctr[..., 3] = np.uint64(aux)
    key = np.zeros(i.shape + (2,), dtype=np.uint64)
    key[..., 0] = np.uint64(seed)
    words = philox4x64_10(ctr, key)
    w = np.take_along_axis(words, (i & np.uint64(3)).astype(np.int64)[..., None], axis=-1)[..., 0]
    return (w >> np.uint64(62)).astype(np.int64)


def z4_vector(n, seed, sample, term, aux=0):
    """Full-support Z4 vector of length n (Eq. z4)."""
    return Z4_VALUES[z4_codes(n, seed, sample, term, aux)]


def z4_slice_vector(dims, dof, t, seed, sample, term, aux=0):
    """Z4 vector supported on time slice t of a lattice with `dof` per site:
    entries on slice t are drawn with their full-volume index, all others 0."""
    Lx, Ly, Lz, Lt = dims
    n = Lx * Ly * Lz * Lt * dof
    per_slice = Lx * Ly * Lz * dof
    x = np.zeros(n, dtype=np.complex128)
    idx = np.arange(t * per_slice, (t + 1) * per_slice)
    x[idx] = Z4_VALUES[z4_codes(n, seed, sample, term, aux, index=idx)]
    return x


# term identifiers used for the noise counter (the counter's third word)
TERM_PLAIN = 0
TERM_O = 16          # + level (0-based)
TERM_F = 32          # + level (0-based)
TERM_COARSEST = 48
TERM_CONNECTED = 64  # aux = source time slice
TERM_DISCONNECTED = 80  # aux = time slice
TERM_M = 144         # + level (0-based): oblique M_l


def term_id(kind, level=0):
    return {'plain': TERM_PLAIN, 'O': TERM_O + level, 'F': TERM_F + level,
            'coarsest': TERM_COARSEST, 'connected': TERM_CONNECTED,
            'disconnected': TERM_DISCONNECTED}[kind]
