"""Test-vector refinement (mgmlmc_refine_test_vectors) against the oracle
(oracle/testvectors.py): with a fixed number of steps the Rayleigh
quotients, eigen-residuals, the rebuilt P_l and every estimator sample equal
the oracle's on the same start block, on the fine and on a coarse level;
with a tolerance the device stops with every returned vector within it,
checked with the oracle's own operator; bad arguments are refused."""
import numpy as np
import pytest

from oracle import estimators as oest, multigrid as omg, solve as osolve, testvectors as otv

pytestmark = pytest.mark.gpu

torch = pytest.importorskip('torch')
if not torch.cuda.is_available():
    pytest.skip('needs a CUDA GPU', allow_module_level=True)

from gpu_util import Setup, rel, require_lib  # noqa: E402

M = require_lib()

# Tolerances: the device solves to a 1e-12 relative residual (errors below
# 1e-10 at these condition numbers); the oracle solves directly.  Perturbing
# the oracle's solves by 1e-11 moved theta, rho, P and the samples by at most
# 4e-11 over six steps, so 1e-8 (1e-7 for samples) leaves a wide margin.
TOL_Q, TOL_P, TOL_X = 1e-8, 1e-8, 1e-7


def _three():
    return Setup((4, 4, 4, 8), [(2, 2, 2, 2), (2, 2, 2, 2)], [6, 4], eps=0.4, m0=-0.1, gseed=77)


@pytest.mark.parametrize('level', [0, 1])
def test_refinement_matches_oracle(level):
    s = _three()
    try:
        h0 = s.hier
        A_l = h0.matrix(level)
        dof = h0.A[level].shape[2]
        k = s.ntvs[level]
        m, steps_req, seed = k + 4, 6, 4321
        th, rh, steps = M.mgmlmc_refine_test_vectors(s.ctx, level, m, steps_req, 0.0, 1e-12, seed)
        sol = osolve.LevelSolver(A_l)
        V, th_o, rh_o, st_o = otv.refine(lambda v: A_l @ v, sol.solve, s.tvs[level], dof, m, steps_req, 0.0,
                                         level, seed)
        assert steps == st_o == steps_req
        assert np.max(np.abs(th - th_o)) < TOL_Q
        assert np.max(np.abs(rh - rh_o)) < TOL_Q
        # the returned vectors and the rebuilt hierarchy
        got = M.mgmlmc_get_test_vectors(s.ctx, level)
        assert rel(got.T, V) < TOL_P
        tvs = list(s.tvs)
        tvs[level] = V
        h = omg.Hierarchy(h0.A[0], s.dims, s.blocks, tvs)
        for l in range(2):
            Q = h.P[l].Q
            out = np.zeros(Q.size, dtype=np.complex128)
            M.mgmlmc_get_prolongator(s.ctx, l, out)
            assert rel(out.reshape(Q.shape), Q) < TOL_P, l
        E = oest.Estimators(h, [osolve.LevelSolver(h.matrix(l)) for l in range(3)], seed=2424)
        N = 4
        res = M.mgmlmc_estimate_trace(s.ctx, M.est_params(M.EST_ORTHOGONAL, [N] * 5, batch=4, seed=2424))
        terms = dict(E.orthogonal_terms())
        for r, name in zip(res, ['O0', 'O1', 'F0', 'F1', 'coarsest']):
            X = np.array([terms[name](q) for q in range(N)])
            mu, var = oest.sample_stats(X)
            assert abs(complex(r['mean_re'], r['mean_im']) - mu) < TOL_X * max(1.0, abs(mu)), name
            assert abs(r['var'] - var) < TOL_X * max(1.0, var), name
    finally:
        s.close()


def test_refinement_stops_at_tolerance():
    """config-1 shape, 16-column block, eigen-residual 1e-3 (Sec. 5's
    accuracy): every returned vector meets it under the oracle's operator,
    and the vectors are orthonormal with their largest entry real positive."""
    s = Setup((4, 4, 4, 4), [(2, 2, 2, 2)], [8], eps=0.3, m0=-0.2)
    try:
        tol = 1e-3
        th, rh, steps = M.mgmlmc_refine_test_vectors(s.ctx, 0, 16, 400, tol, 1e-10, 99)
        assert 0 < steps < 400
        assert rh.max() <= tol
        V = M.mgmlmc_get_test_vectors(s.ctx, 0).T
        D = s.hier.matrix(0)
        QV = otv.gamma5_level((D @ V).T.reshape(-1), 12).reshape(V.shape[1], -1).T
        theta, rho = otv.rayleigh_quotients(V, QV)
        assert np.max(np.abs(V.conj().T @ V - np.eye(8))) < 1e-10
        assert np.max(np.abs(theta - th)) < 1e-9
        assert np.max(np.abs(rho - rh)) < 1e-9 and rho.max() <= tol * (1 + 1e-6)
        i = np.argmax(np.abs(V), axis=0)
        top = V[i, np.arange(8)]
        assert np.all(top.real > 0) and np.all(top.imag == 0.0)
        # the hierarchy was rebuilt from them and still solves
        h = omg.Hierarchy(s.hier.A[0], s.dims, s.blocks, [V])
        Q = h.P[0].Q
        out = np.zeros(Q.size, dtype=np.complex128)
        M.mgmlmc_get_prolongator(s.ctx, 0, out)
        assert rel(out.reshape(Q.shape), Q) < 1e-12
        r = M.mgmlmc_estimate_trace(s.ctx, M.est_params(M.EST_ORTHOGONAL, [2, 2, 2], batch=2, seed=5))
        assert all(t['max_residual'] <= 1.5e-12 for t in r)
    finally:
        s.close()


def test_refinement_arguments():
    s = Setup((4, 4, 4, 4), [(2, 2, 2, 2)], [8], eps=0.3, m0=-0.2, oracle=False)
    try:
        for args in ((1, 12, 1, 0.0, 1e-10),     # the coarsest level has no test vectors
                     (-1, 12, 1, 0.0, 1e-10),
                     (0, 7, 1, 0.0, 1e-10),      # block smaller than N_tv
                     (0, 129, 1, 0.0, 1e-10),
                     (0, 12, -1, 0.0, 1e-10),
                     (0, 12, 1, -1.0, 1e-10),
                     (0, 12, 1, 0.0, 0.0),
                     (0, 12, 1, 0.0, 1.0)):
            with pytest.raises(M.MgmlmcError) as e:
                M.mgmlmc_refine_test_vectors(s.ctx, *args, 1)
            assert e.value.status == 1, args
        # zero steps: the orthonormalised start block, hierarchy rebuilt
        th, rh, steps = M.mgmlmc_refine_test_vectors(s.ctx, 0, 8, 0, 0.0, 1e-10, 1)
        assert steps == 0 and th.shape == (8,) and np.all(rh > 0)
        V = M.mgmlmc_get_test_vectors(s.ctx, 0).T
        assert np.max(np.abs(V.conj().T @ V - np.eye(8))) < 1e-12
    finally:
        s.close()
