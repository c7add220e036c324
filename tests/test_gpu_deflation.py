"""Inexact deflation (Sec. 2.1, Eq. deflated-estimator) through the C-ABI
against the oracle (oracle/deflation.py): the basis built with 1e-12 inner
solves spans the oracle's subspace, so the exact part tr(V^H D^-1 V) and
the per-sample values of x^H (I - V V^H) D^-1 x agree to solve accuracy
(1e-8 relative); the deflated estimate of tr(D^-1) lies within 3 SE of the
dense exact trace; bad arguments and a missing basis give error statuses."""
import numpy as np
import pytest

from oracle import deflation as odf, estimators as oest, solve as osolve

pytestmark = pytest.mark.gpu

torch = pytest.importorskip('torch')
if not torch.cuda.is_available():
    pytest.skip('needs a CUDA GPU', allow_module_level=True)

from gpu_util import Setup, require_lib  # noqa: E402

M = require_lib()


@pytest.fixture(scope='module')
def cfg():
    s = Setup((4, 4, 4, 4), [(2, 2, 2, 2)], [8], eps=0.3, m0=-0.2)
    yield s
    s.close()


def test_deflation_matches_oracle(cfg):
    with pytest.raises(M.MgmlmcError):  # no basis yet
        M.mgmlmc_estimate_trace(cfg.ctx, M.est_params(M.EST_DEFLATED, [4], batch=4, seed=62))
    k, iters = 8, 3
    exact, sec = M.mgmlmc_deflation_build(cfg.ctx, k, iters, 1e-12, 61)
    assert sec > 0
    A = cfg.hier.matrix(0)
    sol = osolve.LevelSolver(A)
    n = A.shape[0]
    V = odf.block_power(sol, n, k, iters, 61)
    want = odf.exact_part(sol, V)
    assert abs(exact - want) < 1e-8 * abs(want)
    N = 10
    res = M.mgmlmc_estimate_trace(cfg.ctx, M.est_params(M.EST_DEFLATED, [N], batch=4, seed=62))
    assert [r['term'] for r in res] == [M.TERM_DEFL, M.TERM_DEFL_EXACT]
    X = np.array([odf.sample(sol, V, 62, q) for q in range(N)])
    mu, var = oest.sample_stats(X)
    r = res[0]
    assert r['n'] == N and r['max_residual'] <= 1.5e-12
    assert abs(complex(r['mean_re'], r['mean_im']) - mu) < 1e-8 * abs(mu)
    assert abs(r['var'] - var) < 1e-6 * var
    assert abs(complex(res[1]['mean_re'], res[1]['mean_im']) - exact) == 0.0
    assert res[1]['var'] == 0.0


def test_deflation_ragged_block_matches_oracle(cfg):
    """k = 11 columns: the build's solves and the estimator's projections run
    in batches of 8 and 3; exact part and samples against the oracle."""
    k, iters = 11, 2
    exact, _ = M.mgmlmc_deflation_build(cfg.ctx, k, iters, 1e-12, 64)
    A = cfg.hier.matrix(0)
    sol = osolve.LevelSolver(A)
    V = odf.block_power(sol, A.shape[0], k, iters, 64)
    want = odf.exact_part(sol, V)
    assert abs(exact - want) < 1e-8 * abs(want)
    N = 6
    res = M.mgmlmc_estimate_trace(cfg.ctx, M.est_params(M.EST_DEFLATED, [N], batch=4, seed=65))
    X = np.array([odf.sample(sol, V, 65, q) for q in range(N)])
    mu, _ = oest.sample_stats(X)
    assert res[0]['n'] == N
    assert abs(complex(res[0]['mean_re'], res[0]['mean_im']) - mu) < 1e-8 * abs(mu)


def test_deflated_trace_unbiased_and_bad_args(cfg):
    exact_tr = np.trace(np.linalg.inv(cfg.hier.matrix(0).toarray()))
    ex, _ = M.mgmlmc_deflation_build(cfg.ctx, 16, 5, 1e-6, 63)
    res = M.mgmlmc_estimate_trace(cfg.ctx, M.est_params(M.EST_DEFLATED, [200], batch=25, seed=64))
    est = complex(res[0]['mean_re'], res[0]['mean_im']) + ex
    se = np.sqrt(res[0]['var'] / res[0]['n'])
    assert abs(est - exact_tr) < 3 * se
    for k, it, tol in ((0, 5, 1e-6), (129, 5, 1e-6), (8, -1, 1e-6), (8, 5, 0.0)):
        with pytest.raises(M.MgmlmcError):
            M.mgmlmc_deflation_build(cfg.ctx, k, it, tol, 1)
