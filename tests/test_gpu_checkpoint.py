"""Checkpoint and resume with the public entry points: the test vectors a
hierarchy was built from (mgmlmc_get_test_vectors), imported into a new
context, rebuild the same P and coarse operators bit for bit; an estimate
split over two calls by first_sample gives the samples of one call, and the
raw accumulators merge by addition."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip('torch')
if not torch.cuda.is_available():
    pytest.skip('needs a CUDA GPU', allow_module_level=True)

from gpu_util import require_lib  # noqa: E402
from paper_2509_11424_gb300 import synth  # noqa: E402

M = require_lib()
DIMS = (4, 4, 4, 8)
BLOCKS = [(2, 2, 2, 2), (2, 2, 2, 2)]
NTV = [6, 4]


def _context(U, imported=None):
    ctx = M.mgmlmc_create(DIMS, torch.cuda.current_stream())
    M.mgmlmc_set_gauge(ctx, U)
    M.mgmlmc_set_mass(ctx, -0.1)
    M.mgmlmc_set_solver(ctx)
    for l, V in enumerate(imported or []):
        M.mgmlmc_set_test_vectors(ctx, l, np.ascontiguousarray(V), V.shape[0], V.shape[1], on_device=False)
    M.mgmlmc_build_hierarchy(ctx, M.mg_params(BLOCKS, NTV, setup_rounds=2, setup_iters=10, seed=3100))
    return ctx


def _operators(ctx):
    ops = []
    for l in range(2):
        info = M.mgmlmc_level_info(ctx, l)
        ntv = M.mgmlmc_level_info(ctx, l + 1)[1] // 2
        P = np.zeros(info[2] * ntv, dtype=np.complex128)
        M.mgmlmc_get_prolongator(ctx, l, P)
        ops.append(P)
    for l in (1, 2):
        _, dof, n = M.mgmlmc_level_info(ctx, l)
        A = np.zeros(n * 9 * dof, dtype=np.complex128)
        M.mgmlmc_get_coarse_op(ctx, l, A)
        ops.append(A)
    return ops


def test_hierarchy_rebuilds_from_saved_test_vectors():
    U = synth.gauge_field(DIMS, 0.4, 77)
    a = _context(U)
    b = None
    try:
        saved = [M.mgmlmc_get_test_vectors(a, l) for l in range(2)]
        assert [v.shape for v in saved] == [(6, 4 * 4 * 4 * 8 * 12), (4, 2 * 2 * 2 * 4 * 12)]
        b = _context(U, saved)
        for x, y in zip(_operators(a), _operators(b)):
            assert np.array_equal(x, y)
        for l in range(2):
            assert np.array_equal(M.mgmlmc_get_test_vectors(b, l), saved[l])
    finally:
        M.mgmlmc_destroy(a)
        if b is not None:
            M.mgmlmc_destroy(b)


def test_estimate_resumes_by_first_sample():
    U = synth.gauge_field(DIMS, 0.4, 77)
    ctx = _context(U)
    try:
        N = 8
        one = M.mgmlmc_estimate_trace(ctx, M.est_params(M.EST_ORTHOGONAL, [N] * 5, batch=4, seed=2500))
        h1 = M.mgmlmc_estimate_trace(ctx, M.est_params(M.EST_ORTHOGONAL, [N // 2] * 5, batch=4, seed=2500))
        h2 = M.mgmlmc_estimate_trace(ctx, M.est_params(M.EST_ORTHOGONAL, [N // 2] * 5, batch=4, seed=2500,
                                                       first_sample=N // 2))
        for r, p, q in zip(one, h1, h2):
            assert r['term'] == p['term'] == q['term']
            assert p['n'] + q['n'] == r['n'] == N
            for key in ('sum_re', 'sum_im', 'sum_abs2'):
                assert abs(p[key] + q[key] - r[key]) <= 1e-12 * max(1.0, abs(r[key])), (r['term'], key)
            n = r['n']
            mean = complex(p['sum_re'] + q['sum_re'], p['sum_im'] + q['sum_im']) / n
            var = (p['sum_abs2'] + q['sum_abs2'] - n * abs(mean) ** 2) / (n - 1)
            assert abs(mean - complex(r['mean_re'], r['mean_im'])) <= 1e-12 * max(1.0, abs(mean))
            assert abs(var - r['var']) <= 1e-9 * max(1.0, r['var'])
    finally:
        M.mgmlmc_destroy(ctx)
