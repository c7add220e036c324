"""Inexact deflation of Hutchinson's estimator (oracle, test infrastructure).

Sec. 2.1 ('Deflation for the Dirac operator', Eq. deflated-estimator):

    tr(D^-1) ~ (1/N) sum_n x_n^H (I - V_k V_k^H) D^-1 x_n + tr(V_k^H D^-1 V_k),

with V_k approximate eigenvectors of Q = Gamma5 D for its smallest
eigenvalues (equivalently right singular vectors of D for its smallest
singular values).  The paper's experiments build V_k by five steps of an
inverse block power method on Q with inner solves to 1e-6 (Sec. 4.2).

Steps restated here, in this order:
* start: column j of V is the Z4 vector of sample j of noise stream 176,
  orthonormalised by two-pass Gram-Schmidt in column order;
* each power step: W = Q^-1 V = D^-1 Gamma5 V, then V = orthonormalised W;
* exact part: tr(V^H D^-1 V) = sum_j v_j^H D^-1 v_j (k solves);
* sample: z = D^-1 x, X = x^H z - (V^H x)^H (V^H z), x the Z4 vector of
  sample k of noise stream 160.
"""
import numpy as np

from . import noise as nz
from .dirac import apply_gamma5
from .multigrid import mgs_orthonormalise

TERM_DEFL = 160
TERM_DEFL_START = 176


def orthonormalise(V):
    """two-pass Gram-Schmidt of the columns of V (n, k), in column order."""
    return mgs_orthonormalise(V[None, None])[0, 0]


def start_vectors(n, k, seed):
    return np.stack([nz.z4_vector(n, seed, j, TERM_DEFL_START) for j in range(k)], axis=1)


def block_power(solve, n, k, iters, seed):
    """V (n, k) after `iters` inverse block power steps on Gamma5 D;
    solve(b) returns D^-1 b."""
    V = orthonormalise(start_vectors(n, k, seed))
    for _ in range(iters):
        W = np.stack([solve(apply_gamma5(V[:, j])) for j in range(k)], axis=1)
        V = orthonormalise(W)
    return V


def exact_part(solve, V):
    return sum(np.vdot(V[:, j], solve(V[:, j])) for j in range(V.shape[1]))


def sample(solve, V, seed, k):
    x = nz.z4_vector(V.shape[0], seed, k, TERM_DEFL)
    z = solve(x)
    return np.vdot(x, z) - np.vdot(V.conj().T @ x, V.conj().T @ z)
