"""GPU smoothers against the oracle's restatement (oracle/smoother.py): SAP
on the fine level (2^4 and 4^4 blocks) and MR on the fine and a coarse level,
FP64 to 1e-11 and FP32 to 1e-4 relative (element by element, see rel); and
full solves with the SAP smoother reaching the 1e-12 residual measured with
the oracle's own D.

Why 1e-4 for FP32 SAP, not the 1e-5 of a single FP32 operator: SAP is not
linear in the input.  Every block MR step takes alpha = <q, r> / <q, q> from
block sums that the kernel forms in FP32 (12 products per thread added in
order, a 5-level warp tree, then up to 8 warp sums in order: about 25
roundings of u = 2^-24 = 6e-8, i.e. ~1.5e-6 relative per alpha), and the
test runs 2 sweeps x 4 block iterations = 8 such steps in sequence on every
block, each feeding the next residual.  The compounded error is therefore of
order 8 x 1.5e-6 ~ 1.2e-5 on top of the ~6e-8-per-flop rounding of the
block operator itself; 1e-4 leaves a factor ~8 of margin over that estimate.
The FP64 runs of the same kernels pin the algorithm to 1e-11."""
import numpy as np
import pytest

from oracle import dirac, smoother as osm
from paper_2509_11424_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip('torch')
if not torch.cuda.is_available():
    pytest.skip('needs a CUDA GPU', allow_module_level=True)

from gpu_util import Setup, dev, host, rel  # noqa: E402


# the library picks SAP blocks of 8x4x4x2 where every direction holds an even
# number of them (16x8x8x4 here), else 4^4, else 2^4
@pytest.mark.parametrize('dims,bshape,blocks', [((4, 4, 4, 8), (2, 2, 2, 2), [(2, 2, 2, 2)]),
                                                ((8, 8, 8, 8), (4, 4, 4, 4), [(4, 4, 4, 4)]),
                                                ((16, 8, 8, 4), (8, 4, 4, 2), [(4, 4, 4, 4)])])
@pytest.mark.parametrize('prec,tol', [(0, 1e-11), (1, 1e-4)])
def test_sap_smoother_matches_oracle(dims, bshape, blocks, prec, tol):
    s = Setup(dims, blocks, [4], eps=0.4, m0=0.1, gseed=91, oracle=False,
              solver=dict(smoother=1, sap_iters=4, smoother_steps=2))
    try:
        M = s.M
        Mx = dirac.wilson_matrix(s.U, 0.1, dims)
        n = Mx.shape[0]
        b = synth.complex_normal((2, n), 92)
        ct = torch.complex128 if prec == 0 else torch.complex64
        out = torch.empty((2, n), dtype=ct, device='cuda')
        M.mgmlmc_apply(s.ctx, M.OP_SMOOTH, 0, prec, dev(b, ct), out, 2)
        got = host(out)
        for r in range(2):
            want = osm.sap_smooth(Mx, dims, bshape, b[r], sweeps=2, iters=4)
            assert rel(got[r], want) < tol
    finally:
        s.close()


@pytest.mark.parametrize('dims', [(16, 8, 8, 4), (8, 8, 8, 8)])
@pytest.mark.parametrize('nrhs', [1, 2, 3, 4])
def test_sap_variants_identical(dims, nrhs):
    """The staged (variant 0) and paired (variant 1) FP32 SAP kernels
    (8x4x4x2 blocks on 16x8x8x4, 4^4 on 8^4; two right-hand sides per thread
    block, an odd count leaving one idle) against the general ones (variant
    2), two sweeps so that the fused face terms and the face pass both run:
    the same sums in the same order, so the results agree bit for bit; the
    default variant is held to the oracle above."""
    s = Setup(dims, [(4, 4, 4, 4)], [4], eps=0.4, m0=0.1, gseed=97, oracle=False,
              solver=dict(smoother=1, sap_iters=4, smoother_steps=2))
    try:
        M = s.M
        assert M.mgmlmc_kernel_variants(M.VARIANT_SAP_FP32) == 3
        n = M.mgmlmc_level_info(s.ctx, 0)[2]
        b = dev(synth.complex_normal((nrhs, n), 98), torch.complex64)
        outs = []
        for v in (0, 1, 2):
            M.mgmlmc_set_kernel_variant(s.ctx, M.VARIANT_SAP_FP32, v)
            assert M.mgmlmc_get_kernel_variant(s.ctx, M.VARIANT_SAP_FP32, nrhs) == v
            out = torch.empty((nrhs, n), dtype=torch.complex64, device='cuda')
            M.mgmlmc_apply(s.ctx, M.OP_SMOOTH, 0, 1, b, out, nrhs)
            outs.append(out)
        assert torch.equal(outs[0], outs[2])
        assert torch.equal(outs[1], outs[2])
        assert float(outs[0].abs().max()) > 0
    finally:
        s.close()


def test_mr_smoother_matches_oracle():
    dims = (4, 4, 4, 8)
    s = Setup(dims, [(2, 2, 2, 2)], [4], eps=0.4, m0=0.1, gseed=93, solver=dict(smoother_steps=3, coarse_smoother_steps=3))
    try:
        M = s.M
        for level in (0, 1):
            Mx = s.hier.matrix(level)
            n = Mx.shape[0]
            b = synth.complex_normal((2, n), 94 + level)
            out = torch.empty((2, n), dtype=torch.complex128, device='cuda')
            M.mgmlmc_apply(s.ctx, M.OP_SMOOTH, level, 0, dev(b), out, 2)
            got = host(out)
            for r in range(2):
                assert rel(got[r], osm.mr_smooth(Mx, b[r], 3)) < 1e-11
    finally:
        s.close()


@pytest.mark.parametrize('prec', [0, 1])
def test_solve_with_sap(prec):
    dims = (8, 8, 8, 8)
    s = Setup(dims, [(4, 4, 4, 4), (2, 2, 2, 2)], [8, 6], eps=0.4, m0=-0.2, gseed=95, oracle=False,
              solver=dict(smoother=1, sap_iters=4, smoother_steps=1, coarse_iters=4, precision=prec,
                          inner_tol=1e-6))
    try:
        M = s.M
        Mx = dirac.wilson_matrix(s.U, -0.2, dims)
        n = Mx.shape[0]
        b = synth.complex_normal((3, n), 96)
        x = torch.empty((3, n), dtype=torch.complex128, device='cuda')
        M.mgmlmc_apply(s.ctx, M.OP_SOLVE, 0, M.FP64, dev(b), x, 3)
        xs = host(x)
        for r in range(3):
            assert np.linalg.norm(b[r] - Mx @ xs[r]) / np.linalg.norm(b[r]) < 1.5e-12
    finally:
        s.close()
