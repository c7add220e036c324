"""The tensor-core (tcgen05 kind::tf32) coarse stencil D_{l+1} = P^H D_l P
(Sec. 2.2, Galerkin) against the oracle, element by element, and inside the
solver.

Tolerance, derived from the arithmetic: the tensor cores take each FP32
operand as TF32, keeping 10 of its 23 mantissa bits, so every operand
carries a relative error of at most u = 2^-10 (truncation; 2^-11 if
rounded), and the products are accumulated in FP32.  Every real and
imaginary part of the output is a sum of K = 9 x 2 x 32 products a_k b_k, so
  |got - exact| <= 2 u sum_k |a_k| |b_k| + (FP32 accumulation, K 2^-24 sum_k |a_k b_k|)
and sum_k |a_k| |b_k| <= (|A|_1 |x|_1) with |z|_1 = |Re z| + |Im z| taken
entry by entry.  The test asserts that bound (with 2.1 u + 300 * 2^-24 in
place of 2 u + K 2^-24) for every entry, against the oracle's FP64 stencil
applied to the FP32-rounded input."""
import numpy as np
import pytest

from oracle import dirac
from paper_2509_11424_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip('torch')
if not torch.cuda.is_available():
    pytest.skip('needs a CUDA GPU', allow_module_level=True)

from gpu_util import Setup, dev, host  # noqa: E402

U_TF32 = 2.0 ** -10
K_FP32 = 300 * 2.0 ** -24


@pytest.fixture(scope='module')
def tc():
    """8^4 lattice, 2^4 aggregates with 16 test vectors: level 1 is 4^4 with
    32 dofs per site (the tensor-core path), level 2 a 2^4 lattice."""
    s = Setup((8, 8, 8, 8), [(2, 2, 2, 2), (2, 2, 2, 2)], [16, 4], eps=0.4, m0=-0.2, gseed=71)
    yield s
    s.close()


def bound_check(got, x32, A1, u=U_TF32):
    """|got - A1 x| within the bound for operands rounded with relative error
    u, entry by entry (real and imaginary parts separately)."""
    want = A1 @ x32
    Aabs = abs(A1.real) + abs(A1.imag)
    xabs = np.abs(x32.real) + np.abs(x32.imag)
    bnd = (2.1 * u + K_FP32) * (Aabs @ xabs) + 1e-30
    ok_re = np.abs(got.real - want.real) <= bnd
    ok_im = np.abs(got.imag - want.imag) <= bnd
    return bool(ok_re.all() and ok_im.all()), float(np.max(np.abs(got - want) / bnd))


# variants 4 and 5: BF16 operands (kind::f16), both rounded to nearest:
# relative error <= 2^-9 per operand, the same bound with u = 2^-9
@pytest.mark.parametrize('variant', [1, 2, 4, 5])
@pytest.mark.parametrize('nrhs', [1, 8, 32, 37])
def test_tensor_stencil_matches_oracle(tc, variant, nrhs):
    M = tc.M
    A1 = tc.hier.matrix(1).tocsr()
    n1 = A1.shape[0]
    x = synth.complex_normal((nrhs, n1), 500 + nrhs)
    x32 = x.astype(np.complex64).astype(np.complex128)
    y = torch.empty((nrhs, n1), dtype=torch.complex64, device='cuda')
    M.mgmlmc_set_kernel_variant(tc.ctx, M.VARIANT_STENCIL_FP32, variant)
    try:
        M.mgmlmc_apply(tc.ctx, M.OP_D, 1, M.FP32, dev(x, torch.complex64), y, nrhs)
        got = host(y).astype(np.complex128)
    finally:
        M.mgmlmc_set_kernel_variant(tc.ctx, M.VARIANT_STENCIL_FP32, 0)
    u = 2.0 ** -9 if variant in (4, 5) else U_TF32
    for r in range(nrhs):
        ok, worst = bound_check(got[r], x32[r], A1, u)
        assert ok, (variant, nrhs, r, worst)


@pytest.mark.parametrize('nrhs', [1, 8, 32, 37])
def test_persistent_tensor_stencil_identical(tc, nrhs):
    """Variant 5, the persistent two-stage form of the BF16 tensor-core
    stencil (152 thread blocks walking the 256 sites of the 4^4 level, so
    most walk two), bit-identical to variant 4: the same MMAs in the same
    order per site.  37 right-hand sides exceed its 32 and run variant 4."""
    M = tc.M
    n1 = tc.hier.matrix(1).shape[0]
    xd = dev(synth.complex_normal((nrhs, n1), 550 + nrhs), torch.complex64)
    outs = []
    try:
        for v in (4, 5):
            M.mgmlmc_set_kernel_variant(tc.ctx, M.VARIANT_STENCIL_FP32, v)
            y = torch.empty((nrhs, n1), dtype=torch.complex64, device='cuda')
            M.mgmlmc_apply(tc.ctx, M.OP_D, 1, M.FP32, xd, y, nrhs)
            outs.append(y)
    finally:
        M.mgmlmc_set_kernel_variant(tc.ctx, M.VARIANT_STENCIL_FP32, 0)
    assert torch.equal(outs[0], outs[1])
    assert float(outs[0].abs().max()) > 0


@pytest.mark.parametrize('nrhs', [1, 4, 5, 8])
def test_fp32_stencil_pipelined_matches_oracle_and_staged_kernel(tc, nrhs):
    """Variant 0 at 32 dofs per site: up to 8 right-hand sides run in the
    pipelined kernel (persistent blocks, two-stage bulk-copy ring), more in
    the one-site-per-block kernel.  Both against the oracle to the FP32
    tolerance 1e-5 element-wise, and bit-identical to each other (the same
    products summed in the same order)."""
    from gpu_util import rel
    M = tc.M
    A1 = tc.hier.matrix(1).tocsr()
    n1 = A1.shape[0]
    x = synth.complex_normal((9, n1), 600 + nrhs)
    xd = dev(x, torch.complex64)
    y = torch.empty((nrhs, n1), dtype=torch.complex64, device='cuda')
    y9 = torch.empty((9, n1), dtype=torch.complex64, device='cuda')
    M.mgmlmc_apply(tc.ctx, M.OP_D, 1, M.FP32, xd[:nrhs].contiguous(), y, nrhs)  # pipelined
    M.mgmlmc_apply(tc.ctx, M.OP_D, 1, M.FP32, xd, y9, 9)                          # staged
    got, got9 = host(y), host(y9)
    assert np.array_equal(got, got9[:nrhs])
    x32 = x.astype(np.complex64).astype(np.complex128)
    for r in range(nrhs):
        assert rel(got[r], A1 @ x32[r]) < 1e-5


@pytest.mark.parametrize('variant', [3, 6, 7])
@pytest.mark.parametrize('nrhs', [1, 4, 7])
def test_bf16_stencil_matches_oracle(tc, variant, nrhs):
    """Variants 3, 6 and 7: the blocks stored as BF16 pairs (round to nearest,
    relative error <= 2^-9 per real entry), FP32 products and sums (6 and 7
    stream them with one warp per site or per direction).  Bound per output entry, real and imaginary
    parts: 2^-9 sum_k |a_k| |b_k| from the storage rounding, plus FP32
    accumulation (300 x 2^-24 of the same sum)."""
    M = tc.M
    A1 = tc.hier.matrix(1).tocsr()
    n1 = A1.shape[0]
    x = synth.complex_normal((nrhs, n1), 700 + nrhs)
    x32 = x.astype(np.complex64).astype(np.complex128)
    y = torch.empty((nrhs, n1), dtype=torch.complex64, device='cuda')
    M.mgmlmc_set_kernel_variant(tc.ctx, M.VARIANT_STENCIL_FP32, variant)
    try:
        M.mgmlmc_apply(tc.ctx, M.OP_D, 1, M.FP32, dev(x, torch.complex64), y, nrhs)
        got = host(y).astype(np.complex128)
    finally:
        M.mgmlmc_set_kernel_variant(tc.ctx, M.VARIANT_STENCIL_FP32, 0)
    want = np.array([A1 @ v for v in x32])
    Aabs = abs(A1.real) + abs(A1.imag)
    for r in range(nrhs):
        bnd = (2.0 ** -9 + K_FP32) * (Aabs @ (np.abs(x32[r].real) + np.abs(x32[r].imag))) + 1e-30
        assert np.all(np.abs(got[r].real - want[r].real) <= bnd), r
        assert np.all(np.abs(got[r].imag - want[r].imag) <= bnd), r
        assert np.max(np.abs(got[r] - want[r])) > 0  # it is not the FP32 result


@pytest.fixture(scope='module')
def walk():
    """16^3 x 32 lattice with 2^4 aggregates twice (16 test vectors each,
    device gauge field, no setup iterations): level 1 is 8^3 x 16 (8192
    sites) and level 2 4^3 x 8 (512 sites), both with 32 dofs per site.  At
    level 1 every warp of the streaming kernel walks several sites, so the
    prefetch of the next (site, direction) item crosses site boundaries."""
    from gpu_util import require_lib
    M = require_lib()
    ctx = M.mgmlmc_create((16, 16, 16, 32), torch.cuda.current_stream())
    M.mgmlmc_gen_gauge(ctx, 0.4, 91)
    M.mgmlmc_set_mass(ctx, -0.3)
    M.mgmlmc_build_hierarchy(ctx, M.mg_params([(2, 2, 2, 2), (2, 2, 2, 2)], [16, 16], setup_rounds=0, seed=92))
    yield M, ctx
    M.mgmlmc_destroy(ctx)


@pytest.mark.parametrize('level', [1, 2])
@pytest.mark.parametrize('nrhs', [1, 2, 3, 4, 5, 8])
def test_streaming_stencil_identical_to_pipelined(walk, level, nrhs):
    """Variants 6 (one warp per site, row-chunked BF16 blocks streamed into
    registers, packed FP32 pair arithmetic) and 7 (one thread block per site,
    a warp per direction) bit-identical to variant 3 (the pipelined kernel on
    the same BF16 values): the same fused multiply-adds per direction in the
    same order, the nine direction sums added in the same order.  Odd counts
    leave the last packed lane unused."""
    M, ctx = walk
    _, dof, n = M.mgmlmc_level_info(ctx, level)
    assert dof == 32
    xd = dev(synth.complex_normal((nrhs, n), 900 + 10 * level + nrhs), torch.complex64)
    outs = []
    try:
        for v in (3, 6, 7):
            M.mgmlmc_set_kernel_variant(ctx, M.VARIANT_STENCIL_FP32, v)
            y = torch.full((nrhs, n), float('nan'), dtype=torch.complex64, device='cuda')
            M.mgmlmc_apply(ctx, M.OP_D, level, M.FP32, xd, y, nrhs)
            outs.append(y)
    finally:
        M.mgmlmc_set_kernel_variant(ctx, M.VARIANT_STENCIL_FP32, 0)
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
    assert bool(torch.isfinite(outs[1]).all()) and float(outs[1].abs().max()) > 0


@pytest.mark.parametrize('gs', [2, 1])
def test_solve_with_preconditioner_variants(tc, gs):
    """The tensor-core and BF16 stencils inside the multigrid preconditioner
    of FP32 inner solves, with two or one Gram-Schmidt passes and
    post-smoothing only on the fine level: every level-0 solve still reaches
    the 1e-12 true residual measured with the oracle's D (the FP64 defect
    correction decides)."""
    M = tc.M
    A0 = tc.hier.matrix(0).tocsr()
    n = A0.shape[0]
    b = synth.complex_normal((3, n), 801)
    M.mgmlmc_set_solver(tc.ctx, precision=M.FP32, restart=8, coarse_restart=16, smoother=1, smoother_steps=1,
                        coarse_iters=4, inner_tol=1e-6, gram_schmidt_passes=gs, post_smoothing_only=gs % 2)
    try:
        for v in (1, 3, 4, 5, 6, 7, -2):
            M.mgmlmc_set_kernel_variant(tc.ctx, M.VARIANT_STENCIL_FP32, v)
            # with the BF16 stencils, BF16-stored P in the preconditioner too
            M.mgmlmc_set_kernel_variant(tc.ctx, M.VARIANT_TRANSFER_FP32, 1 if v in (3, 4, 5, 6, 7) else 0)
            x = torch.empty((3, n), dtype=torch.complex128, device='cuda')
            M.mgmlmc_apply(tc.ctx, M.OP_SOLVE, 0, M.FP64, dev(b), x, 3)
            xs = host(x)
            for r in range(3):
                assert np.linalg.norm(b[r] - A0 @ xs[r]) / np.linalg.norm(b[r]) < 1.5e-12, v
    finally:
        M.mgmlmc_set_kernel_variant(tc.ctx, M.VARIANT_STENCIL_FP32, 0)
        M.mgmlmc_set_kernel_variant(tc.ctx, M.VARIANT_TRANSFER_FP32, 0)
        M.mgmlmc_set_solver(tc.ctx)
