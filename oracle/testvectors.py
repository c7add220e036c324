"""Test vectors refined toward low eigenvectors of Gamma5 D_l (oracle, test
infrastructure).

Sec. 2.2 builds P_l from N_tv test vectors that approximate eigenvectors of
D_l for its smallest eigenvalues; the same section cites a construction from
exact eigenvectors of the Hermitian Gamma5 D.  Sec. 4 uses rough ones
(residual about 1e-1); Sec. 5 reports lower variance with more test vectors
computed to an eigen-residual of 1e-3 to 1e-4.  The paper does not say how
the accurate ones are computed.  This module fixes one way, in this order:

* Q_l = Gamma5_l D_l with Gamma5_l = +1 on the first half of every site's
  dofs and -1 on the second (spins 0, 1 against 2, 3 on the fine level,
  chirality on coarser ones); Q_l^-1 v = D_l^-1 Gamma5_l v;
* block V (n, m), m >= N_tv: the level's current N_tv test vectors followed
  by m - N_tv Z4 columns (noise stream 192 + l, sample = column index),
  orthonormalised by two-pass Gram-Schmidt in column order;
* step (Rutishauser's simultaneous iteration, 'ritzit', Numer. Math. 16
  (1970), with the Ritz step taken on Q^-2): W = Q^-1 V, G = W^H W =
  Y diag(mu) Y^H with mu descending, V <- W Y diag(mu)^-1/2 (orthonormal).
  Q^-2 is positive definite and its largest eigenvalues 1/lambda^2 belong
  to the smallest |lambda| of Q, so no spurious interior Ritz value can
  appear, as it does for a Rayleigh-Ritz step on the indefinite Q itself;
* after every step (and once for the start block): theta_j = v_j^H Q v_j and
  the eigen-residual rho_j = ||Q v_j - theta_j v_j|| of the unit columns;
* steps run while max_{j < N_tv} rho_j > tol (tol > 0) and fewer than
  `iters` have run;
* phase: each returned column is scaled by a unit complex number so that its
  entry of largest modulus (the first, on a tie) is real and positive.

The first N_tv columns are the refined test vectors.
"""
import numpy as np

from . import noise as nz
from .deflation import orthonormalise
from .dirac import apply_gamma5

TERM_TV_EXTRA = 192


def gamma5_level(v, dof):
    """Gamma5_l: the sign of the second half of every site's dofs flipped."""
    return apply_gamma5(v, dof)


def start_block(V0, m, level, seed):
    """(n, m) start block: the N_tv given columns, then Z4 columns."""
    n, k = V0.shape
    extra = [nz.z4_vector(n, seed, j, TERM_TV_EXTRA + level) for j in range(k, m)]
    return np.concatenate([np.asarray(V0, dtype=np.complex128)] + [e[:, None] for e in extra], axis=1)


def ritz_step(W):
    """(U, mu): U = W Y diag(mu)^-1/2 with W^H W = Y diag(mu) Y^H, mu
    descending; U is orthonormal and spans span(W)."""
    G = W.conj().T @ W
    G = 0.5 * (G + G.conj().T)
    mu, Y = np.linalg.eigh(G)
    order = np.argsort(-mu, kind='stable')
    mu, Y = mu[order], Y[:, order]
    return W @ (Y / np.sqrt(mu)[None, :]), mu


def rayleigh_quotients(V, QV):
    """theta_j = v_j^H Q v_j (real: Q Hermitian) and rho_j = ||Q v_j - theta_j v_j||."""
    theta = np.real(np.sum(V.conj() * QV, axis=0))
    rho = np.linalg.norm(QV - V * theta[None, :], axis=0)
    return theta, rho


def canonical_phase(V):
    """each column times the unit number that makes its largest-modulus entry
    (first on a tie) real and positive."""
    V = np.array(V, dtype=np.complex128, copy=True)
    for j in range(V.shape[1]):
        i = int(np.argmax(np.abs(V[:, j])))
        a = abs(V[i, j])
        V[:, j] *= np.conj(V[i, j]) / a
        V[i, j] = a  # exactly real, not real up to rounding
    return V


def refine(apply_D, solve, V0, dof, m, iters, tol, level, seed):
    """Refined test vectors of one level.

    apply_D(v) = D_l v, solve(b) = D_l^-1 b, V0 (n, N_tv) the current test
    vectors, dof the level's dofs per site.  Returns (V (n, N_tv), theta,
    rho, steps) with theta, rho of the N_tv returned columns and steps the
    inverse-iteration steps taken."""
    k = V0.shape[1]
    if m < k:
        raise ValueError('block smaller than the number of test vectors')

    def Q(v):
        return gamma5_level(apply_D(v), dof)

    def quotients(V):
        return rayleigh_quotients(V, np.stack([Q(V[:, j]) for j in range(V.shape[1])], axis=1))

    V = orthonormalise(start_block(V0, m, level, seed))
    theta, rho = quotients(V)
    steps = 0
    while not (tol > 0 and rho[:k].max() <= tol) and steps < iters:
        W = np.stack([solve(gamma5_level(V[:, j], dof)) for j in range(m)], axis=1)
        V, _ = ritz_step(W)
        theta, rho = quotients(V)
        steps += 1
    return canonical_phase(V[:, :k]), theta[:k], rho[:k], steps
