"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the
oracle's tests.

This module holds no arithmetic of the trace-estimation method.  It only
draws inputs: SU(3) gauge links U = exp(i eps H) with H a random traceless
Hermitian 3x3 matrix per link (the generator the workloads of this project
use in place of the paper's ensembles, which are not available), random
complex test vectors, and random complex right-hand sides.

Recipes (all numpy, FP64):
* gauge_field(dims, eps, seed): links in the canonical order U[s][mu][a][b];
  drawn in chunks of CHUNK links with numpy's default_rng(seed): for each
  chunk the real parts of A (chunk x 3 x 3) then the imaginary parts, both
  standard normal scaled by 1/sqrt(2) (so E|A_ab|^2 = 1);
  H = (A + A^H)/2 - tr(.)/3, U = Q exp(i eps Lambda) Q^H with H = Q Lambda Q^H.
  det U = exp(i eps tr H) = 1.  eps = 0 gives the free field U = 1.
* random_su3(n, seed, eps): the same construction for n independent matrices.
* complex_normal(shape, seed): iid complex normal entries, E|z|^2 = 1.
* random_test_vectors(n, ntv, seed): (n, ntv) complex normal columns.
"""
import numpy as np

CHUNK = 1 << 18


def _hermitian_exp(A, eps):
    H = 0.5 * (A + np.conj(np.swapaxes(A, -1, -2)))
    tr = np.trace(H, axis1=-2, axis2=-1).real / 3.0
    H = H - tr[..., None, None] * np.eye(3)
    w, Q = np.linalg.eigh(H)
    return (Q * np.exp(1j * eps * w)[..., None, :]) @ np.conj(np.swapaxes(Q, -1, -2))


def random_su3(n, seed, eps=1.0):
    """n SU(3) matrices exp(i eps H) drawn as documented above."""
    rng = np.random.default_rng(seed)
    out = np.empty((n, 3, 3), dtype=np.complex128)
    for a in range(0, n, CHUNK):
        b = min(n, a + CHUNK)
        re = rng.standard_normal((b - a, 3, 3))
        im = rng.standard_normal((b - a, 3, 3))
        out[a:b] = _hermitian_exp((re + 1j * im) / np.sqrt(2.0), eps)
    return out


def gauge_field(dims, eps, seed):
    """Flat complex128 array of 4 V links, canonical order U[s][mu][a][b]."""
    V = int(np.prod(dims))
    if eps == 0.0:
        return unit_gauge(dims)
    return random_su3(4 * V, seed, eps).reshape(-1)


def unit_gauge(dims):
    V = int(np.prod(dims))
    U = np.zeros((4 * V, 3, 3), dtype=np.complex128)
    U[:, 0, 0] = U[:, 1, 1] = U[:, 2, 2] = 1.0
    return U.reshape(-1)


def complex_normal(shape, seed):
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im) / np.sqrt(2.0)


def random_test_vectors(n, ntv, seed):
    """(n, ntv) complex normal test vectors (column k is test vector k)."""
    return complex_normal((n, ntv), seed)
