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


def bound_check(got, x32, A1):
    """|got - A1 x| within the TF32 bound, entry by entry (real and imaginary
    parts separately)."""
    want = A1 @ x32
    Aabs = abs(A1.real) + abs(A1.imag)
    xabs = np.abs(x32.real) + np.abs(x32.imag)
    bnd = (2.1 * U_TF32 + K_FP32) * (Aabs @ xabs) + 1e-30
    ok_re = np.abs(got.real - want.real) <= bnd
    ok_im = np.abs(got.imag - want.imag) <= bnd
    return bool(ok_re.all() and ok_im.all()), float(np.max(np.abs(got - want) / bnd))


@pytest.mark.parametrize('variant', [1, 2])
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
    for r in range(nrhs):
        ok, worst = bound_check(got[r], x32[r], A1)
        assert ok, (variant, nrhs, r, worst)
