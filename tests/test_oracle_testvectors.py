"""Pins of the test-vector refinement oracle (oracle/testvectors.py) against
what the mathematics fixes: on an operator built with a planted spectrum the
refined vectors are the planted eigenvectors and the Ritz values the planted
eigenvalues; on a Wilson operator they match a dense Hermitian
eigen-decomposition of Gamma5 D; Ritz pairs satisfy the Galerkin condition
and are Rayleigh quotients; the stopping rule takes the fewest steps that
meet the tolerance; Gamma5-hermiticity survives the chirality-split
aggregation, so Q_l is Hermitian on every level."""
import numpy as np
import pytest

from oracle import dirac, multigrid as omg, noise as nz, testvectors as otv
from oracle.deflation import orthonormalise
from paper_2509_11424_gb300 import synth

DIMS = (2, 2, 2, 4)


def _unitary(n, seed):
    q, r = np.linalg.qr(synth.complex_normal((n, n), seed))
    return q * (np.diag(r) / np.abs(np.diag(r)))[None, :]


def _g5(n, dof=12):
    return np.diag(np.tile(np.array([1.0] * (dof // 2) + [-1.0] * (dof // 2)), n // dof))


@pytest.fixture(scope='module')
def planted():
    """D = Gamma5 Q with Q = U diag(lam) U^H: the spectrum of Q is lam."""
    n = 96
    rng = np.random.default_rng(5)
    lam = np.concatenate([[0.05, -0.07, 0.11, -0.16, 0.23, 0.31],
                          rng.uniform(1.0, 3.0, n - 6) * rng.choice([-1, 1], n - 6)])
    U = _unitary(n, 17)
    Q = (U * lam[None, :]) @ U.conj().T
    D = _g5(n) @ Q
    return n, lam, U, D


def test_planted_spectrum_is_recovered(planted):
    n, lam, U, D = planted
    Dinv = np.linalg.inv(D)
    k = 4
    V0 = synth.complex_normal((n, k), 3)
    V, theta, rho, steps = otv.refine(lambda v: D @ v, lambda b: Dinv @ b, V0, 12, k + 2, 200, 1e-11, 0, 9)
    order = np.argsort(np.abs(lam))[:k]
    assert np.max(np.abs(theta - lam[order])) < 1e-11
    assert rho.max() <= 1e-11 and 0 < steps < 200
    want = otv.canonical_phase(U[:, order])
    assert np.max(np.abs(V - want)) < 1e-9


def test_ritz_step_on_an_invariant_subspace_is_exact(planted):
    n, lam, U, D = planted
    Q = _g5(n) @ D
    idx = [7, 2, 30]
    V = U[:, idx] @ _unitary(3, 8)             # same span, mixed basis
    Uo, mu = otv.ritz_step(np.linalg.solve(Q, V))
    theta, rho = otv.rayleigh_quotients(Uo, Q @ Uo)
    want = lam[idx][np.argsort(np.abs(lam[idx]))]
    assert np.all(np.abs(theta - want) < 1e-12 * np.abs(want))
    assert np.max(np.abs(mu - 1.0 / want ** 2)) < 1e-12 * np.max(mu)
    assert rho.max() < 1e-12


def test_ritz_step_galerkin_condition(planted):
    """for any orthonormal V and W = Q^-1 V the step returns orthonormal
    columns u_j spanning span(W) with V^H (Q^-1 u_j - mu_j Q u_j) = 0, i.e.
    Q u_j sqrt(mu_j) are the Ritz vectors of Q^-2 on span(V)."""
    n, lam, U, D = planted
    Q = _g5(n) @ D
    Qinv = np.linalg.inv(Q)
    V = orthonormalise(synth.complex_normal((n, 7), 4))
    W = Qinv @ V
    Uo, mu = otv.ritz_step(W)
    assert np.all(np.diff(mu) <= 0) and np.all(mu > 0)
    assert np.max(np.abs(Uo.conj().T @ Uo - np.eye(7))) < 1e-12
    # span: W = U (U^H W)
    assert np.max(np.abs(W - Uo @ (Uo.conj().T @ W))) < 1e-12 * np.max(np.abs(W))
    for j in range(7):
        u = Uo[:, j]
        assert np.max(np.abs(V.conj().T @ (Qinv @ u - mu[j] * (Q @ u)))) < 1e-11 * mu[j]


def test_rayleigh_quotients_definition(planted):
    n, lam, U, D = planted
    Q = _g5(n) @ D
    V = orthonormalise(synth.complex_normal((n, 3), 6))
    theta, rho = otv.rayleigh_quotients(V, Q @ V)
    for j in range(3):
        v = V[:, j]
        rq = np.vdot(v, Q @ v)
        assert abs(rq.imag) < 1e-13 and abs(rq.real - theta[j]) < 1e-13
        assert abs(np.linalg.norm(Q @ v - rq.real * v) - rho[j]) < 1e-13
    # an exact eigenvector has residual 0 and its eigenvalue as quotient
    th, r = otv.rayleigh_quotients(U[:, :1], Q @ U[:, :1])
    assert abs(th[0] - lam[0]) < 1e-13 and r[0] < 1e-13


@pytest.fixture(scope='module')
def wilson():
    U = synth.gauge_field(DIMS, 0.5, 41)
    D = dirac.wilson_matrix(U, -0.3, DIMS).toarray()
    return D, np.linalg.inv(D)


def test_wilson_low_modes_match_dense_eigendecomposition(wilson):
    D, Dinv = wilson
    n = D.shape[0]
    k = 6
    V0 = synth.random_test_vectors(n, k, 3001)
    V, theta, rho, steps = otv.refine(lambda v: D @ v, lambda b: Dinv @ b, V0, 12, k + 6, 500, 1e-10, 0, 4)
    lam = np.linalg.eigvalsh(_g5(n) @ D)
    lam = lam[np.argsort(np.abs(lam))][:k]
    assert np.max(np.abs(theta - lam)) < 1e-10
    assert rho.max() <= 1e-10
    Q = _g5(n) @ D
    assert np.max(np.linalg.norm(Q @ V - V * theta[None, :], axis=0)) < 1e-9
    # canonical phase: the largest-modulus entry of every column real positive
    i = np.argmax(np.abs(V), axis=0)
    top = V[i, np.arange(k)]
    assert np.all(top.real > 0) and np.max(np.abs(top.imag)) == 0.0


def test_stopping_rule_takes_fewest_steps(wilson):
    D, Dinv = wilson
    n = D.shape[0]
    V0 = synth.random_test_vectors(n, 4, 3002)
    args = (lambda v: D @ v, lambda b: Dinv @ b, V0, 12, 8)
    _, _, rho, steps = otv.refine(*args, 100, 1e-3, 0, 6)
    assert rho.max() <= 1e-3 and steps >= 1
    _, _, rho_less, steps_less = otv.refine(*args, steps - 1, 1e-3, 0, 6)
    assert steps_less == steps - 1 and rho_less.max() > 1e-3
    # tol = 0: exactly `iters` steps
    assert otv.refine(*args, 3, 0.0, 0, 6)[3] == 3
    # no step: Ritz vectors of the start block itself
    _, theta0, _, s0 = otv.refine(*args, 0, 0.0, 0, 6)
    assert s0 == 0 and theta0.shape == (4,)


def test_start_block_and_phase():
    n, k, m = 48, 3, 5
    V0 = synth.complex_normal((n, k), 1)
    B = otv.start_block(V0, m, 1, 77)
    assert np.array_equal(B[:, :k], V0)
    for j in range(k, m):
        assert np.array_equal(B[:, j], nz.z4_vector(n, 77, j, otv.TERM_TV_EXTRA + 1))
    W = synth.complex_normal((n, 4), 2)
    C = otv.canonical_phase(W)
    assert np.max(np.abs(otv.canonical_phase(W * np.exp(1j * np.array([0.3, -2.0, 1.0, 3.1]))) - C)) < 1e-15
    assert np.max(np.abs(np.abs(C) - np.abs(W))) < 1e-15
    # a tie takes the first entry
    T = np.zeros((4, 1), dtype=complex)
    T[1, 0], T[3, 0] = 1j, -1.0
    assert np.array_equal(otv.canonical_phase(T)[:, 0], np.array([0, 1, 0, 1j]))  # times -i
    with pytest.raises(ValueError):
        otv.refine(None, None, V0, 12, k - 1, 1, 0.0, 0, 1)


def test_coarse_gamma5_hermiticity():
    """P commutes with Gamma5 (chirality-split aggregates), so Gamma5_c D_c
    is Hermitian and the refinement applies on coarse levels as on the fine
    one."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.4, 5)
    A = dirac.wilson_stencil(U, -0.2, dims)
    tv = synth.random_test_vectors(dirac.volume(dims) * 12, 6, 11)
    h = omg.Hierarchy(A, dims, [(2, 2, 2, 2)], [tv])
    Dc = h.matrix(1).toarray()
    Qc = _g5(Dc.shape[0], 12) @ Dc
    assert np.max(np.abs(Qc - Qc.conj().T)) < 1e-13 * np.max(np.abs(Qc))
    # and Gamma5_l as the oracle applies it is that matrix
    v = synth.complex_normal(Dc.shape[0], 3)
    assert np.array_equal(otv.gamma5_level(v, 12), _g5(Dc.shape[0], 12) @ v)
