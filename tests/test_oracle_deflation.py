"""Pins of the inexact-deflation oracle (oracle/deflation.py) against what
the mathematics fixes: the trace split of Eq. deflated-estimator holds for
any orthonormal V; with the exact eigenvectors of Q = Gamma5 D for the k
smallest |eigenvalues| the deflated Frobenius norm reaches its optimum
||D^-1||_F^2 - sum_{i<=k} sigma_i(D^-1)^2 (Eq. Frobenius-reduction-singular);
the block power iteration converges to that subspace; a sample equals the
dense quadratic form; the estimator is unbiased."""
import numpy as np
import pytest

from oracle import deflation as odf, dirac, noise as nz, solve
from paper_2509_11424_gb300 import synth

DIMS = (2, 2, 2, 4)


@pytest.fixture(scope='module')
def op():
    U = synth.gauge_field(DIMS, 0.5, 41)
    A = dirac.wilson_matrix(U, -0.3, DIMS).tocsr()
    Dd = A.toarray()
    Dinv = np.linalg.inv(Dd)
    sol = solve.LevelSolver(A)
    return Dd, Dinv, sol


def _gamma5(n):
    return np.diag(np.tile(np.array([1.0] * 6 + [-1.0] * 6), n // 12))


def test_split_holds_for_any_orthonormal_basis(op):
    Dd, Dinv, _ = op
    n = Dd.shape[0]
    V = odf.orthonormalise(synth.complex_normal((n, 10), 3))
    assert np.max(np.abs(V.conj().T @ V - np.eye(10))) < 1e-13
    Pi = V @ V.conj().T
    lhs = np.trace((np.eye(n) - Pi) @ Dinv) + np.trace(V.conj().T @ Dinv @ V)
    assert abs(lhs - np.trace(Dinv)) < 1e-11 * abs(np.trace(Dinv))


def test_exact_eigenvectors_give_optimal_frobenius_reduction(op):
    Dd, Dinv, _ = op
    n = Dd.shape[0]
    k = 12
    lam, W = np.linalg.eigh(_gamma5(n) @ Dd)        # Q Hermitian
    idx = np.argsort(np.abs(lam))[:k]
    V = W[:, idx]
    sig = np.linalg.svd(Dinv, compute_uv=False)     # descending
    want = np.linalg.norm(Dinv, 'fro') ** 2 - np.sum(sig[:k] ** 2)
    got = np.linalg.norm((np.eye(n) - V @ V.conj().T) @ Dinv, 'fro') ** 2
    assert abs(got - want) < 1e-9 * want


def test_block_power_converges_to_smallest_eigenspace(op):
    Dd, Dinv, sol = op
    n = Dd.shape[0]
    # k = 5: the gap |lambda_5| / |lambda_6| of Q = Gamma5 D is 0.954 on this
    # field, so the subspace error shrinks like 0.954^iterations
    k = 5
    lam, W = np.linalg.eigh(_gamma5(n) @ Dd)
    idx = np.argsort(np.abs(lam))
    rate = abs(lam[idx[k - 1]]) / abs(lam[idx[k]])
    assert rate < 0.96
    Vex = W[:, idx[:k]]
    V = odf.block_power(sol, n, k, 400, 5)
    assert np.max(np.abs(V.conj().T @ V - np.eye(k))) < 1e-12
    # principal angles between span(V) and the exact subspace: cosines -> 1
    cos = np.linalg.svd(Vex.conj().T @ V, compute_uv=False)
    assert np.min(cos) > 1 - 1e-8
    # five steps already deflate: the Frobenius norm drops below plain
    V5 = odf.block_power(sol, n, 8, 5, 5)
    f5 = np.linalg.norm((np.eye(n) - V5 @ V5.conj().T) @ Dinv, 'fro')
    assert f5 < np.linalg.norm(Dinv, 'fro')


def test_samples_and_unbiasedness(op):
    Dd, Dinv, sol = op
    n = Dd.shape[0]
    V = odf.block_power(sol, n, 6, 5, 7)
    T = (np.eye(n) - V @ V.conj().T) @ Dinv
    for k in range(3):
        x = nz.z4_vector(n, 9, k, odf.TERM_DEFL)
        assert abs(odf.sample(sol, V, 9, k) - np.vdot(x, T @ x)) < 1e-10
    ex = odf.exact_part(sol, V)
    assert abs(ex - np.trace(V.conj().T @ Dinv @ V)) < 1e-10
    N = 400
    X = np.array([odf.sample(sol, V, 9, k) for k in range(N)])
    off = T - np.diag(np.diag(T))
    se = np.sqrt(np.sum(np.abs(off) ** 2) / N)
    assert abs(X.mean() + ex - np.trace(Dinv)) < 4 * se
