"""Pins of the oracle's estimators: exact identities from dense inverses,
closed forms, brute-force optimality and statistical laws with fixed seeds."""
import numpy as np
import pytest

from oracle import dirac, estimators as est, exact, multigrid as mg, solve
from paper_2509_11424_gb300 import synth

from test_oracle_noise_mg import make_hier


def solvers_for(h):
    return [solve.LevelSolver(h.matrix(l)) for l in range(h.n_levels)]


@pytest.fixture(scope='module')
def two_level():
    # config-1 shape: 4^4, eps 0.3, m0 -0.2, 2^4 aggregates, 8 test vectors
    h = make_hier((4, 4, 4, 4), [(2, 2, 2, 2)], [8], eps=0.3, m0=-0.2, seed=1001)
    return h, exact.DenseTerms(h), solvers_for(h)


@pytest.fixture(scope='module')
def three_level():
    h = make_hier((4, 4, 4, 4), [(2, 2, 2, 2), (2, 2, 2, 2)], [4, 3], eps=0.4, m0=-0.1, seed=7)
    return h, exact.DenseTerms(h), solvers_for(h)


@pytest.mark.parametrize('fx', ['two_level', 'three_level'])
def test_orthogonal_split_telescopes(fx, request):
    """sum tr(O_l) + sum tr(F_l) + tr(D_L^-1) = tr(D^-1) (Eq.
    smultigrid-multilevel-monte-carlo), exactly, from dense inverses."""
    h, dt, _ = request.getfixturevalue(fx)
    total = sum(np.trace(M) for _, M in dt.terms())
    assert abs(total - np.trace(dt.Dinv[0])) < 1e-10 * abs(np.trace(dt.Dinv[0]))
    # Frobenius norm cannot grow under the two-sided orthogonal projection (Sec. 3)
    for l in range(h.n_levels - 1):
        P = dt.P[l]
        Q = np.eye(P.shape[0]) - P @ P.conj().T
        assert np.linalg.norm(dt.O(l)) <= np.linalg.norm(Q @ dt.Dinv[l]) * (1 + 1e-12)
        assert np.linalg.norm(Q @ dt.Dinv[l]) <= np.linalg.norm(dt.Dinv[l]) * (1 + 1e-12)


def test_samples_equal_quadratic_forms(three_level):
    """each per-sample value equals x^H T x with the dense term matrix T and
    the same Z4 vector (O, F, coarsest, plain)."""
    h, dt, sol = three_level
    E = est.Estimators(h, sol, seed=2001)
    from oracle import noise as nz
    terms = dict(dt.terms())
    for k in range(3):
        for l in range(h.n_levels - 1):
            x = nz.z4_vector(h.size(l), 2001, k, nz.TERM_O + l)
            assert abs(E.O(l, k) - np.vdot(x, terms['O%d' % l] @ x)) < 1e-9
            x = nz.z4_vector(h.size(l + 1), 2001, k, nz.TERM_F + l)
            assert abs(E.F(l, k) - np.vdot(x, terms['F%d' % l] @ x)) < 1e-9
        x = nz.z4_vector(h.size(2), 2001, k, nz.TERM_COARSEST)
        assert abs(E.coarsest(k) - np.vdot(x, terms['coarsest'] @ x)) < 1e-9
        x = nz.z4_vector(h.size(0), 2001, k, nz.TERM_PLAIN)
        assert abs(E.plain(k) - np.vdot(x, dt.Dinv[0] @ x)) < 1e-9


def test_sample_variance_matches_numpy():
    X = synth.complex_normal(37, 4) * 3 + 1j
    mu, var = est.sample_stats(X)
    assert abs(mu - np.mean(X)) < 1e-14
    assert abs(var - np.var(X, ddof=1)) < 1e-13


def test_mlmc_allocation_is_optimal():
    """N_l of Eq. MLMC-Nl meets the variance target and no other feasible
    allocation (random perturbations along the constraint) is cheaper."""
    rng = np.random.default_rng(3)
    V = rng.uniform(0.1, 50, 4)
    C = rng.uniform(0.01, 3, 4)
    eps = 0.05
    N, cost = est.mlmc_allocation(V, C, eps)
    assert abs(np.sum(V / N) - eps ** 2) < 1e-12
    assert abs(np.sum(N * C) - cost) < 1e-9 * cost
    for _ in range(2000):
        M = N * np.exp(rng.normal(0, 0.3, 4))
        M *= np.sum(V / M) / eps ** 2  # rescale onto the constraint
        assert np.sum(M * C) >= cost * (1 - 1e-12)


def test_terms_unbiased_and_variance_law(two_level):
    """fixed seed 2002, N = 300: every term's sample mean lies within 4 SE of
    its exact trace, and its sample variance lies within a wide band around
    the Z4 law ||offdiag(T)||_F^2."""
    h, dt, sol = two_level
    E = est.Estimators(h, sol, seed=2002)
    exact_terms = dict(dt.terms())
    N = 300
    for name, sampler in E.orthogonal_terms():
        X = np.array([sampler(k) for k in range(N)])
        mu, var = est.sample_stats(X)
        T = exact_terms[name]
        se = np.sqrt(exact.offdiag_fro2(T) / N)
        assert abs(mu - np.trace(T)) < 4 * se + 1e-12, name
        law = exact.offdiag_fro2(T)
        assert 0.6 * law < var < 1.5 * law, (name, var, law)


def test_correlator_split_and_free_field():
    """G = sum_rs G_rs exactly; the plain dense G(t) of the free field equals
    the momentum sum; G is real, positive and G(t) = G(T - t)."""
    dims = (2, 2, 2, 8)
    h = make_hier(dims, [(2, 2, 2, 2), (1, 1, 1, 2)], [4, 3], eps=0.4, m0=0.1, seed=31)
    dt = exact.DenseTerms(h)
    B = dt.B_matrices()
    assert np.max(np.abs(sum(B) - dt.Dinv[0])) < 1e-11
    G = exact.correlator_exact(B, dims)
    Gplain = exact.correlator_exact([dt.Dinv[0]], dims)[0, 0]
    assert np.max(np.abs(G.sum(axis=(0, 1)) - Gplain)) < 1e-10
    assert np.max(np.abs(Gplain.imag)) < 1e-12 and np.all(Gplain.real > 0)
    # free field closed form
    dims = (2, 2, 4, 6)
    M = dirac.wilson_matrix(synth.unit_gauge(dims), 0.05, dims).toarray()
    Gf = exact.correlator_exact([np.linalg.inv(M)], dims)[0, 0]
    want = exact.free_field_correlator(dims, 0.05)
    assert np.max(np.abs(Gf - want)) < 1e-12 * np.max(want)
    T = dims[3]
    assert np.allclose(want[1:], want[1:][::-1])


def test_correlator_operators_and_samples():
    """the oracle's B_r x and Gamma5 B_r^H Gamma5 x equal the dense
    operators, and the sample mean of X_rs(t) (fixed seed 2003, N = 40)
    lies within 5 SE of the exact G_rs(t)."""
    dims = (2, 2, 2, 8)
    h = make_hier(dims, [(2, 2, 2, 2), (1, 1, 1, 2)], [4, 3], eps=0.4, m0=0.1, seed=31)
    dt = exact.DenseTerms(h)
    B = dt.B_matrices()
    sol = solvers_for(h)
    E = est.Estimators(h, sol, seed=2003)
    x = synth.complex_normal(h.size(0), 8)
    g5 = exact.gamma5_matrix(h.size(0) // 12)
    for br, Bm in zip(E.B_apply(x), B):
        assert np.max(np.abs(br - Bm @ x)) < 1e-11
    for bt, Bm in zip(E.Btilde_apply(x), B):
        assert np.max(np.abs(bt - g5 @ Bm.conj().T @ g5 @ x)) < 1e-11
    Gex = exact.correlator_exact(B, dims)
    N = 40
    S = np.array([E.connected(k) for k in range(N)])
    mu = S.mean(axis=0)
    se = S.std(axis=0, ddof=1) / np.sqrt(N)
    z = np.abs(mu - Gex) / np.maximum(se, 1e-14)
    assert np.all(z[se > 1e-12] < 5.0)
    # plain correlator samples estimate the plain G
    P = np.array([E.connected_plain(k) for k in range(N)])
    Gp = Gex.sum(axis=(0, 1))
    zp = np.abs(P.mean(axis=0) - Gp) / (P.std(axis=0, ddof=1) / np.sqrt(N))
    assert np.all(zp < 5.0)


def test_disconnected_exact_and_free_field():
    dims = (2, 2, 2, 8)
    h = make_hier(dims, [(2, 2, 2, 2)], [4], eps=0.4, m0=0.1, seed=33)
    dt = exact.DenseTerms(h)
    B = dt.B_matrices()
    for t in (1, 5):
        loops = exact.loop_exact(B, dims, t)
        full = exact.loop_exact([dt.Dinv[0]], dims, t)[0]
        assert abs(loops.sum() - full) < 1e-11
        assert abs(full.imag) < 1e-12  # Gamma5 D^-1 is Hermitian
    M = dirac.wilson_matrix(synth.unit_gauge(dims), 0.1, dims).toarray()
    free = exact.loop_exact([np.linalg.inv(M)], dims, 2)[0]
    assert abs(free) < 1e-12
    # samples: within 5 SE, fixed seed 2004
    E = est.Estimators(h, solvers_for(h), seed=2004)
    X = np.array([E.disconnected(k, 1) for k in range(200)])
    mu = X.mean(axis=0)
    se = np.sqrt(np.sum(np.abs(X - mu) ** 2, axis=0) / (200 - 1) / 200)
    assert np.all(np.abs(mu - exact.loop_exact(B, dims, 1)) < 5 * se)


def _dense_M(h, dt, l):
    """M_l = D_l^-1 - P_l D_{l+1}^-1 P_l^H from dense inverses (Eq.
    oblique-deflation), written from the definition."""
    P = dt.P[l]
    return dt.Dinv[l] - P @ dt.Dinv[l + 1] @ P.conj().T


@pytest.mark.parametrize('fx', ['two_level', 'three_level'])
def test_oblique_split_telescopes_and_projects(fx, request):
    """sum_l tr(M_l) + tr(D_L^-1) = tr(D^-1) (Eq.
    oblique_multigrid-multilevel-monte-carlo) exactly; Pi_l = P D_{l+1}^-1
    P^H D_l is a projection (Galerkin) but not an orthogonal one, and
    M_l = (I - Pi_l) D_l^-1."""
    h, dt, _ = request.getfixturevalue(fx)
    L = h.n_levels
    total = sum(np.trace(_dense_M(h, dt, l)) for l in range(L - 1)) + np.trace(dt.Dinv[L - 1])
    assert abs(total - np.trace(dt.Dinv[0])) < 1e-10 * abs(np.trace(dt.Dinv[0]))
    for l in range(L - 1):
        D = h.matrix(l).toarray()
        P = dt.P[l]
        Pi = P @ dt.Dinv[l + 1] @ P.conj().T @ D
        assert np.max(np.abs(Pi @ Pi - Pi)) < 1e-10 * np.max(np.abs(Pi))
        assert np.max(np.abs(Pi - Pi.conj().T)) > 1e-3  # oblique
        I = np.eye(D.shape[0])
        assert np.max(np.abs((I - Pi) @ dt.Dinv[l] - _dense_M(h, dt, l))) < 1e-10 * np.max(np.abs(dt.Dinv[l]))


def test_oblique_samples_equal_quadratic_forms(three_level):
    h, dt, sol = three_level
    E = est.Estimators(h, sol, seed=2011)
    from oracle import noise as nz
    for k in range(3):
        for l in range(h.n_levels - 1):
            x = nz.z4_vector(h.size(l), 2011, k, nz.TERM_M + l)
            assert abs(E.M(l, k) - np.vdot(x, _dense_M(h, dt, l) @ x)) < 1e-9
    names = [n for n, _ in E.oblique_terms()]
    assert names == ['M0', 'M1', 'coarsest']


def test_oblique_terms_unbiased_and_variance_law(two_level):
    """fixed seed 2012, N = 300: the M_0 sample mean within 4 SE of tr(M_0),
    its sample variance near the Z4 law ||offdiag(M_0)||_F^2."""
    h, dt, sol = two_level
    E = est.Estimators(h, sol, seed=2012)
    T = _dense_M(h, dt, 0)
    N = 300
    X = np.array([E.M(0, k) for k in range(N)])
    mu, var = est.sample_stats(X)
    law = exact.offdiag_fro2(T)
    assert abs(mu - np.trace(T)) < 4 * np.sqrt(law / N) + 1e-12
    assert 0.6 * law < var < 1.5 * law, (var, law)


def test_oblique_correlator_and_loop_operators():
    """oblique split of the correlator and loops (Eq. G-traditional, Eq.
    trace_equality_disconnected): sum_l B_l = D^-1 exactly; each B_l is its
    own Gamma5-adjoint (Gamma5 B_l^H Gamma5 = B_l, from Gamma5-hermiticity on
    every level); the oracle's B_l x and its literal Gamma5 B_l^H Gamma5 x
    equal the dense operators; the correlator and loop samples (seeds 2005,
    2006) lie within 5 SE of the exact G_ij(t) and tr(Gamma5 B_l(t, t))."""
    dims = (2, 2, 2, 8)
    h = make_hier(dims, [(2, 2, 2, 2), (1, 1, 1, 2)], [4, 3], eps=0.4, m0=0.1, seed=31)
    dt = exact.DenseTerms(h)
    B = dt.B_matrices_oblique()
    assert len(B) == h.n_levels
    assert np.max(np.abs(sum(B) - dt.Dinv[0])) < 1e-11
    g5 = exact.gamma5_matrix(h.size(0) // 12)
    for Bm in B:
        assert np.max(np.abs(g5 @ Bm.conj().T @ g5 - Bm)) < 1e-11
    E = est.Estimators(h, solvers_for(h), seed=2005)
    x = synth.complex_normal(h.size(0), 9)
    for br, bt, Bm in zip(E.B_apply_oblique(x), E.Btilde_apply_oblique(x), B):
        assert np.max(np.abs(br - Bm @ x)) < 1e-11
        assert np.max(np.abs(bt - Bm @ x)) < 1e-11
    Gex = exact.correlator_exact(B, dims)
    Gplain = exact.correlator_exact([dt.Dinv[0]], dims)[0, 0]
    assert np.max(np.abs(Gex.sum(axis=(0, 1)) - Gplain)) < 1e-10
    N = 40
    S = np.array([E.connected(k, kind='oblique') for k in range(N)])
    mu = S.mean(axis=0)
    se = S.std(axis=0, ddof=1) / np.sqrt(N)
    z = np.abs(mu - Gex) / np.maximum(se, 1e-14)
    assert np.all(z[se > 1e-12] < 5.0)
    E2 = est.Estimators(h, solvers_for(h), seed=2006)
    X = np.array([E2.disconnected(k, 3, kind='oblique') for k in range(200)])
    mu = X.mean(axis=0)
    se = np.sqrt(np.sum(np.abs(X - mu) ** 2, axis=0) / (200 - 1) / 200)
    loops = exact.loop_exact(B, dims, 3)
    assert abs(loops.sum() - exact.loop_exact([dt.Dinv[0]], dims, 3)[0]) < 1e-11
    assert np.all(np.abs(mu - loops) < 5 * se)
