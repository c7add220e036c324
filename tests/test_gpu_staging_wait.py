"""Failure detection on the GPU without a fault: the coarse-stencil kernels
stage a site's blocks with one bulk copy onto an mbarrier and wait for it
with a bound (1 s of the GPU's global timer).  mgmlmc_test_staging_extra
arms that barrier with 16 bytes more than the copy delivers, so the copy
lands in full but the wait runs out: the call must return MGMLMC_ERR_CUDA,
and with the injection off the same context must compute the right result
again."""
import numpy as np
import pytest

from paper_2509_11424_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip('torch')
if not torch.cuda.is_available():
    pytest.skip('needs a CUDA GPU', allow_module_level=True)

from gpu_util import Setup, dev, host, rel  # noqa: E402


# variant 0 with 9 right-hand sides: the one-site-per-block kernel (more
# than the 8 of the pipelined one); variant 1: the tensor-core kernel;
# variant 5: the persistent tensor-core kernel (its bulk copy of the first
# site runs out; the CTA then waits, bounded, for it once more and for
# nothing else in flight)
@pytest.mark.parametrize('variant,nr', [(0, 9), (1, 2), (5, 2)])
def test_staging_wait_runs_out_and_context_survives(variant, nr):
    # a 2^4 coarse lattice of 16 sites: one wave of blocks waits its 2 x 1 s
    s = Setup((4, 4, 4, 4), [(2, 2, 2, 2)], [16], eps=0.3, m0=-0.2, gseed=81)
    M = s.M
    from paper_2509_11424_gb300.mgmlmc import MgmlmcError
    try:
        A1 = s.hier.matrix(1).tocsr()
        n1 = A1.shape[0]
        x = synth.complex_normal((nr, n1), 82)
        y = torch.empty((nr, n1), dtype=torch.complex64, device='cuda')
        M.mgmlmc_set_kernel_variant(s.ctx, M.VARIANT_STENCIL_FP32, variant)
        M.mgmlmc_test_staging_extra(s.ctx, 16)
        try:
            with pytest.raises(MgmlmcError) as e:
                M.mgmlmc_apply(s.ctx, M.OP_D, 1, M.FP32, dev(x, torch.complex64), y, nr)
        finally:
            M.mgmlmc_test_staging_extra(s.ctx, 0)
        assert e.value.status == 4 and 'bounded wait' in str(e.value)
        # usable again, right result
        M.mgmlmc_apply(s.ctx, M.OP_D, 1, M.FP32, dev(x, torch.complex64), y, nr)
        got = host(y)
        want = np.array([A1 @ v.astype(np.complex64).astype(np.complex128) for v in x])
        assert rel(got, want) < {0: 1e-5, 1: 3e-3, 5: 1e-2}[variant]
    finally:
        M.mgmlmc_set_kernel_variant(s.ctx, M.VARIANT_STENCIL_FP32, 0)
        s.close()


def test_pipelined_stencil_wait_runs_out_and_context_survives():
    """The same for the pipelined stencil (variant 0 at 32 dofs per site and
    at most 8 right-hand sides): its CTAs keep two bulk copies in flight and
    wait for both (bounded) before leaving after a failed wait."""
    s = Setup((4, 4, 4, 4), [(2, 2, 2, 2)], [16], eps=0.3, m0=-0.2, gseed=83)
    M = s.M
    from paper_2509_11424_gb300.mgmlmc import MgmlmcError
    try:
        A1 = s.hier.matrix(1).tocsr()
        n1 = A1.shape[0]
        x = synth.complex_normal((2, n1), 84)
        y = torch.empty((2, n1), dtype=torch.complex64, device='cuda')
        M.mgmlmc_test_staging_extra(s.ctx, 32)
        try:
            with pytest.raises(MgmlmcError) as e:
                M.mgmlmc_apply(s.ctx, M.OP_D, 1, M.FP32, dev(x, torch.complex64), y, 2)
        finally:
            M.mgmlmc_test_staging_extra(s.ctx, 0)
        assert e.value.status == 4
        M.mgmlmc_apply(s.ctx, M.OP_D, 1, M.FP32, dev(x, torch.complex64), y, 2)
        want = np.array([A1 @ v.astype(np.complex64).astype(np.complex128) for v in x])
        assert rel(host(y), want) < 1e-5
    finally:
        s.close()
