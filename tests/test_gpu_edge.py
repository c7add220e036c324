"""Edge cases through the C-ABI: rejected lattice shapes and arguments give
MGMLMC_ERR_ARG (status 1) and leave the process and the context usable;
zero samples per term give empty results; a right-hand-side count above the
batch sizes the kernels use (33) and a single site row still match the
oracle."""
import numpy as np
import pytest

from oracle import dirac
from paper_2509_11424_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip('torch')
if not torch.cuda.is_available():
    pytest.skip('needs a CUDA GPU', allow_module_level=True)

from gpu_util import Setup, dev, host, rel, require_lib  # noqa: E402

M = require_lib()


@pytest.mark.parametrize('dims', [(1, 4, 4, 4), (4, 4, 4, 0), (4, 4, 4, -2), (2048, 2048, 2048, 2048)])
def test_bad_lattice_shapes(dims):
    with pytest.raises(M.MgmlmcError) as e:
        M.mgmlmc_create(dims, torch.cuda.current_stream())
    assert e.value.status == 1


def test_bad_arguments_keep_context_usable():
    s = Setup((4, 4, 4, 4), [(2, 2, 2, 2)], [8], eps=0.3, m0=-0.2)
    try:
        n = s.hier.size(0)
        x = dev(synth.complex_normal((1, n), 5))
        y = torch.empty_like(x)
        for level, nrhs, inp, out in ((0, 0, x, y), (0, -1, x, y), (2, 1, x, y), (-1, 1, x, y),
                                      (0, 1, None, y), (0, 1, x, None)):
            with pytest.raises(M.MgmlmcError) as e:
                M.mgmlmc_apply(s.ctx, M.OP_D, level, M.FP64, inp, out, nrhs)
            assert e.value.status == 1
        with pytest.raises(M.MgmlmcError):
            M.mgmlmc_apply(s.ctx, M.OP_D, 0, 7, x, y, 1)  # unknown precision
        M.mgmlmc_apply(s.ctx, M.OP_D, 0, M.FP64, x, y, 1)
        assert rel(host(y)[0], dirac.apply_wilson(s.U, host(x)[0], -0.2, s.dims)) < 1e-12
        res = M.mgmlmc_estimate_trace(s.ctx, M.est_params(M.EST_ORTHOGONAL, [0, 0, 0], batch=4, seed=9))
        assert [r['n'] for r in res] == [0, 0, 0]
        assert all(r['mean_re'] == 0.0 and r['var'] == 0.0 for r in res)
    finally:
        s.close()


@pytest.mark.parametrize('dims,nrhs', [((4, 4, 4, 4), 33), ((2, 2, 2, 2), 1), ((32, 2, 2, 2), 3)])
def test_dslash_rhs_counts_and_thin_lattices(dims, nrhs):
    U = synth.gauge_field(dims, 0.6, 11)
    ctx = M.mgmlmc_create(dims, torch.cuda.current_stream())
    try:
        M.mgmlmc_set_gauge(ctx, U)
        M.mgmlmc_set_mass(ctx, -0.1)
        n = dirac.volume(dims) * 12
        x = synth.complex_normal((nrhs, n), 12)
        y = torch.empty((nrhs, n), dtype=torch.complex128, device='cuda')
        M.mgmlmc_apply(ctx, M.OP_D, 0, M.FP64, dev(x), y, nrhs)
        y32 = torch.empty((nrhs, n), dtype=torch.complex64, device='cuda')
        M.mgmlmc_apply(ctx, M.OP_D, 0, M.FP32, dev(x, torch.complex64), y32, nrhs)
        got, got32 = host(y), host(y32)
        for r in (0, nrhs - 1):
            want = dirac.apply_wilson(U, x[r], -0.1, dims)
            assert rel(got[r], want) < 1e-12
            want32 = dirac.apply_wilson(U, x[r].astype(np.complex64).astype(np.complex128), -0.1, dims)
            assert rel(got32[r], want32) < 1e-5
    finally:
        M.mgmlmc_destroy(ctx)
