"""The device-generated gauge field (mgmlmc_gen_gauge) against the oracle's
restatement of the same counter-based draw (oracle/gauge.py), through the
Wilson operator: D built from the device links applied to random vectors
equals the oracle's D built from the oracle's links (FP64 1e-12, FP32
1e-5), eps = 0 gives the free field, the draw is reproducible, and a
non-finite eps is rejected with the context still usable."""
import numpy as np
import pytest

from oracle import dirac, gauge as ogauge
from paper_2509_11424_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip('torch')
if not torch.cuda.is_available():
    pytest.skip('needs a CUDA GPU', allow_module_level=True)

from gpu_util import dev, host, rel, require_lib  # noqa: E402

M = require_lib()


def apply_d(ctx, x, prec):
    ct = torch.complex128 if prec == M.FP64 else torch.complex64
    y = torch.empty(x.shape, dtype=ct, device='cuda')
    M.mgmlmc_apply(ctx, M.OP_D, 0, prec, dev(x, ct), y, x.shape[0])
    return host(y)


@pytest.mark.parametrize('dims,eps,seed', [((4, 4, 4, 4), 0.4, 1002), ((6, 4, 4, 8), 0.7, 5),
                                           ((3, 2, 2, 2), 1.3, 9)])
def test_generated_field_matches_oracle(dims, eps, seed):
    ctx = M.mgmlmc_create(dims, torch.cuda.current_stream())
    try:
        M.mgmlmc_gen_gauge(ctx, eps, seed)
        M.mgmlmc_set_mass(ctx, -0.2)
        U = ogauge.gauge_field(dims, eps, seed)
        n = dirac.volume(dims) * 12
        x = synth.complex_normal((2, n), 31)
        y64 = apply_d(ctx, x, M.FP64)
        y32 = apply_d(ctx, x.astype(np.complex64), M.FP32)
        for r in range(2):
            want = dirac.apply_wilson(U, x[r], -0.2, dims)
            assert rel(y64[r], want) < 1e-12
            want32 = dirac.apply_wilson(U, x[r].astype(np.complex64).astype(np.complex128), -0.2, dims)
            assert rel(y32[r], want32) < 1e-5
    finally:
        M.mgmlmc_destroy(ctx)


def test_free_field_reproducible_and_bad_eps():
    dims = (4, 2, 2, 4)
    n = dirac.volume(dims) * 12
    x = synth.complex_normal((1, n), 32)
    ctx = M.mgmlmc_create(dims, torch.cuda.current_stream())
    try:
        M.mgmlmc_set_mass(ctx, 0.1)
        M.mgmlmc_gen_gauge(ctx, 0.0, 77)
        free = dirac.apply_wilson(synth.unit_gauge(dims), x[0], 0.1, dims)
        assert rel(apply_d(ctx, x, M.FP64)[0], free) < 1e-14
        M.mgmlmc_gen_gauge(ctx, 0.5, 77)
        a = apply_d(ctx, x, M.FP64)
        M.mgmlmc_gen_gauge(ctx, 0.5, 77)
        assert np.array_equal(apply_d(ctx, x, M.FP64), a)
        M.mgmlmc_gen_gauge(ctx, 0.5, 78)
        assert rel(apply_d(ctx, x, M.FP64), a) > 1e-3
        with pytest.raises(M.MgmlmcError):
            M.mgmlmc_gen_gauge(ctx, float('nan'), 1)
        M.mgmlmc_gen_gauge(ctx, 0.5, 77)  # still usable
        assert np.array_equal(apply_d(ctx, x, M.FP64), a)
    finally:
        M.mgmlmc_destroy(ctx)
