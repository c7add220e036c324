"""Counter-based synthetic gauge field (test infrastructure of the oracle).

The paper measures on real gauge ensembles (Sec. 4); this project stands in
synthetic SU(3) links U_mu(x) = exp(i eps H) with H a random traceless
Hermitian matrix per link.  The library can draw them on the device
(mgmlmc_gen_gauge); this module restates that draw in plain numpy/scipy so
that a test can compare the device field with an independent computation.

Definition (the same one the library's header states):
* link L = 4 s + mu (canonical site s, direction mu);
* 20 words: Philox4x64-10 of counters (L, j, 128, 0), j = 0..4, key (seed, 0)
  (the oracle's own Philox, oracle.noise.philox4x64_10);
* entry e = 3 a + b of A from words 2e, 2e + 1: uniforms
  u = ((w >> 12) + 1/2) 2^-52 in [2^-53, 1 - 2^-53] (exact in FP64: the sum
  stays below 2^52), Box-Muller
  A_e = sqrt(-2 ln u1) (cos 2 pi u2 + i sin 2 pi u2) / sqrt 2, so E|A_e|^2 = 1;
* H = (A + A^H)/2 - tr(H)/3 I;  U = exp(i eps H) (scipy.linalg.expm).
"""
import numpy as np
import scipy.linalg

from . import noise

TERM_GAUGE = 128


def link_words(L, seed):
    """(n, 20) uint64 Philox words of the links L (array of link indices)."""
    L = np.asarray(L, dtype=np.uint64)
    n = L.size
    ctr = np.zeros((n, 5, 4), dtype=np.uint64)
    ctr[:, :, 0] = L[:, None]
    ctr[:, :, 1] = np.arange(5, dtype=np.uint64)[None, :]
    ctr[:, :, 2] = np.uint64(TERM_GAUGE)
    key = np.zeros((n, 5, 2), dtype=np.uint64)
    key[:, :, 0] = np.uint64(seed)
    return noise.philox4x64_10(ctr, key).reshape(n, 20)


def uniforms(words):
    """u = ((w >> 12) + 1/2) 2^-52, strictly inside (0, 1)."""
    return ((words >> np.uint64(12)).astype(np.float64) + 0.5) * 2.0 ** -52


def normal_matrices(L, seed):
    """(n, 3, 3) complex normal matrices A of the links L (Box-Muller)."""
    u = uniforms(link_words(L, seed))[:, :18]
    u1, u2 = u[:, 0::2], u[:, 1::2]
    rho = np.sqrt(-2.0 * np.log(u1)) / np.sqrt(2.0)
    A = rho * np.cos(2.0 * np.pi * u2) + 1j * rho * np.sin(2.0 * np.pi * u2)
    return A.reshape(-1, 3, 3)


def traceless_hermitian(A):
    H = 0.5 * (A + np.conj(np.swapaxes(A, -1, -2)))
    tr = np.trace(H, axis1=-2, axis2=-1).real / 3.0
    return H - tr[..., None, None] * np.eye(3)


def links(L, eps, seed):
    """(n, 3, 3) links exp(i eps H) of the link indices L."""
    H = traceless_hermitian(normal_matrices(L, seed))
    return np.array([scipy.linalg.expm(1j * eps * h) for h in H])


def gauge_field(dims, eps, seed):
    """Flat complex128 array of all 4 V links, canonical order U[s][mu][a][b]."""
    V = int(np.prod(dims))
    return links(np.arange(4 * V), eps, seed).reshape(-1)
