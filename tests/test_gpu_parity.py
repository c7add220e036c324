"""GPU parity tests: every step of the hot path through the C-ABI against the
FP64 oracle on the same seeded inputs.

Tolerances (written here, derived from the arithmetic):
* gathers, indexing, noise: bit-exact;
* FP64 operator applications: 1e-12 relative (norm-wise);
* FP32 operator applications: 1e-5 relative against the FP64 oracle;
* level solves: true relative residual <= 1e-12 measured with the oracle's
  own D, and solution within cond * 1e-12 of the oracle's direct solve;
* per-sample estimator values: solves to 1e-12 make each sample exact to
  about cond * 1e-12, so sample means agree to 1e-8 relative.
"""
import numpy as np
import pytest

from oracle import dirac, estimators as oest, exact, multigrid as omg, noise as onz, solve as osolve
from paper_2509_11424_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip('torch')
if not torch.cuda.is_available():
    pytest.skip('needs a CUDA GPU', allow_module_level=True)

from gpu_util import Setup, dev, host, rel, require_lib  # noqa: E402

M = require_lib()
ODD = (6, 4, 4, 8)


@pytest.fixture(scope='module')
def cfg1():
    """config-1 shape: 4^4, eps 0.3, m0 -0.2, 2^4 aggregates, 8 test vectors."""
    s = Setup((4, 4, 4, 4), [(2, 2, 2, 2)], [8], eps=0.3, m0=-0.2)
    yield s
    s.close()


@pytest.fixture(scope='module')
def three():
    """three levels on 4^3 x 8: 2^4 then 2^4 aggregates, ragged coarse lattice
    (1 x 1 x 1 x 2) at the coarsest level."""
    s = Setup((4, 4, 4, 8), [(2, 2, 2, 2), (2, 2, 2, 2)], [6, 4], eps=0.4, m0=-0.1, gseed=77)
    yield s
    s.close()


# --------------------------------------------------------------- Wilson D
@pytest.mark.parametrize('dims', [(4, 4, 4, 4), ODD, (2, 2, 2, 2), (8, 2, 6, 4)])
def test_dslash_fp64(dims):
    U = synth.gauge_field(dims, 0.5, 5)
    ctx = M.mgmlmc_create(dims, torch.cuda.current_stream())
    try:
        M.mgmlmc_set_gauge(ctx, U)
        M.mgmlmc_set_mass(ctx, -0.3)
        n = dirac.volume(dims) * 12
        x = synth.complex_normal((3, n), 6)
        xd = dev(x)
        yd = torch.empty_like(xd)
        M.mgmlmc_apply(ctx, M.OP_D, 0, M.FP64, xd, yd, 3)
        y = host(yd)
        for r in range(3):
            want = dirac.apply_wilson(U, x[r], -0.3, dims)
            assert rel(y[r], want) < 1e-12
    finally:
        M.mgmlmc_destroy(ctx)


# V % 32 != 0 for (6, 2, 2, 3) and (3, 2, 2, 2); 32-site tiles straddle x rows
# for L_x = 12 and 48; (16, 4, 4, 4) puts two x rows in one tile
FP32_DIMS = [(4, 4, 4, 4), ODD, (6, 2, 2, 3), (3, 2, 2, 2), (12, 4, 2, 2), (48, 2, 2, 2),
             (16, 4, 4, 4)]


@pytest.mark.parametrize('dims', FP32_DIMS)
@pytest.mark.parametrize('nrhs', [2, 5])
def test_dslash_fp32(dims, nrhs):
    """Every FP32 kernel variant (1 or 2 right-hand sides per thread, several
    register budgets) against
    the oracle to 1e-5, and all variants bit-identical to each other (they add
    the same terms in the same order)."""
    U = synth.gauge_field(dims, 0.5, 7)
    ctx = M.mgmlmc_create(dims, torch.cuda.current_stream())
    try:
        M.mgmlmc_set_gauge(ctx, U)
        M.mgmlmc_set_mass(ctx, 0.1)
        n = dirac.volume(dims) * 12
        x = synth.complex_normal((nrhs, n), 8).astype(np.complex64)
        xd = dev(x, torch.complex64)
        outs = []
        nv = M.mgmlmc_kernel_variants(M.VARIANT_DSLASH_FP32)
        assert nv >= 1
        for v in range(nv):
            M.mgmlmc_set_kernel_variant(ctx, M.VARIANT_DSLASH_FP32, v)
            assert M.mgmlmc_get_kernel_variant(ctx, M.VARIANT_DSLASH_FP32, nrhs) == v
            yd = torch.full_like(xd, float('nan'))
            M.mgmlmc_apply(ctx, M.OP_D, 0, M.FP32, xd, yd, nrhs)
            outs.append(host(yd))
        for r in range(nrhs):
            want = dirac.apply_wilson(U, x[r].astype(np.complex128), 0.1, dims)
            assert rel(outs[0][r], want) < 1e-5
        for o in outs[1:]:
            assert np.array_equal(o, outs[0])
        # the internal order: component i of site s at ((i // 2) V + s) * 2 + i % 2
        V = dirac.volume(dims)
        xi = torch.empty_like(xd)
        M.mgmlmc_reorder(ctx, xd, xi, nrhs, 1)
        want_order = x.reshape(nrhs, V, 6, 2).transpose(0, 2, 1, 3).reshape(nrhs, -1)
        assert np.array_equal(host(xi), want_order)
        yi = torch.empty_like(xd)
        M.mgmlmc_apply(ctx, M.OP_D | M.LAYOUT_INTERNAL, 0, M.FP32, xi, yi, nrhs)
        yc = torch.empty_like(xd)
        M.mgmlmc_reorder(ctx, yi, yc, nrhs, 0)
        assert np.array_equal(host(yc), outs[0])
        # autotuned choice: made on the first call, then reported
        M.mgmlmc_set_kernel_variant(ctx, M.VARIANT_DSLASH_FP32, M.VARIANT_AUTOTUNE)
        assert M.mgmlmc_get_kernel_variant(ctx, M.VARIANT_DSLASH_FP32, nrhs) == -2
        yd = torch.empty_like(xd)
        M.mgmlmc_apply(ctx, M.OP_D, 0, M.FP32, xd, yd, nrhs)
        assert np.array_equal(host(yd), outs[0])
        assert M.mgmlmc_get_kernel_variant(ctx, M.VARIANT_DSLASH_FP32, nrhs) in range(nv)
    finally:
        M.mgmlmc_destroy(ctx)


@pytest.mark.parametrize('dims', [(4, 4, 4, 4), (6, 2, 2, 3), (16, 4, 4, 4)])
def test_dslash_bf16(dims):
    """BF16 storage, FP32 arithmetic: against the oracle applied to the same
    bf16-rounded inputs (links FP64 -> FP32 -> bf16 as the library does,
    spinors bf16).  What remains is the round-to-nearest of each output
    component, at most 2^-9 relative, so 3e-3 norm-wise.  The internal-order
    call (reorder, LAYOUT_INTERNAL, reorder back) is bit-identical."""
    U = synth.gauge_field(dims, 0.5, 7)
    nrhs = 3
    ctx = M.mgmlmc_create(dims, torch.cuda.current_stream())
    try:
        M.mgmlmc_set_gauge(ctx, U)
        M.mgmlmc_set_mass(ctx, 0.1)
        n = dirac.volume(dims) * 12
        x = synth.complex_normal((nrhs, n), 8).astype(np.complex64)
        xb = torch.from_numpy(x.view(np.float32)).to(torch.bfloat16).cuda()     # (nrhs, 2n) re, im
        yb = torch.empty_like(xb)
        M.mgmlmc_apply(ctx, M.OP_D, 0, M.BF16, xb, yb, nrhs)
        got = yb.float().cpu().numpy().view(np.complex64).astype(np.complex128)
        xr = xb.float().cpu().numpy().view(np.complex64).astype(np.complex128)
        Ur = torch.from_numpy(U.astype(np.complex64).view(np.float32)).to(torch.bfloat16).float()
        Ur = Ur.numpy().view(np.complex64).astype(np.complex128)
        for r in range(nrhs):
            want = dirac.apply_wilson(Ur, xr[r], 0.1, dims)
            assert rel(got[r], want) < 3e-3
        xi, yi, yc = torch.empty_like(xb), torch.empty_like(xb), torch.empty_like(xb)
        M.mgmlmc_reorder_bf16(ctx, xb, xi, nrhs, 1)
        M.mgmlmc_apply(ctx, M.OP_D | M.LAYOUT_INTERNAL, 0, M.BF16, xi, yi, nrhs)
        M.mgmlmc_reorder_bf16(ctx, yi, yc, nrhs, 0)
        assert torch.equal(yc, yb)
        with pytest.raises(M.MgmlmcError):
            M.mgmlmc_apply(ctx, M.OP_PROJECT, 0, M.BF16, xb, yb, nrhs)
    finally:
        M.mgmlmc_destroy(ctx)


def test_dslash_variant_bad_args():
    nv = M.mgmlmc_kernel_variants(M.VARIANT_DSLASH_FP32)
    ns = M.mgmlmc_kernel_variants(M.VARIANT_STENCIL_FP32)
    nsap = M.mgmlmc_kernel_variants(M.VARIANT_SAP_FP32)
    assert nv == 7 and ns == 8 and nsap == 3
    assert M.mgmlmc_kernel_variants(M.VARIANT_TRANSFER_FP32) == 2
    assert M.mgmlmc_kernel_variants(4) == -1
    ctx = M.mgmlmc_create((4, 4, 4, 4), torch.cuda.current_stream())
    try:
        for kern, v in ((0, nv), (0, -1), (0, -3), (1, ns), (1, -1), (2, nsap), (2, -1), (2, -2), (3, 2), (3, -1),
                        (4, 0)):
            with pytest.raises(M.MgmlmcError):
                M.mgmlmc_set_kernel_variant(ctx, kern, v)
    finally:
        M.mgmlmc_destroy(ctx)


def test_gamma5(cfg1):
    n = cfg1.hier.size(0)
    x = synth.complex_normal(n, 9)
    yd = torch.empty(n, dtype=torch.complex128, device='cuda')
    M.mgmlmc_apply(cfg1.ctx, M.OP_GAMMA5, 0, M.FP64, dev(x), yd, 1)
    assert np.array_equal(host(yd), dirac.apply_gamma5(x))


def test_free_field_plane_wave_on_gpu():
    dims = ODD
    chi = synth.complex_normal((4, 3), 10)
    psi, Dpsi = exact.free_field_plane_wave(dims, -0.4, (1, 2, 3, 5), chi)
    ctx = M.mgmlmc_create(dims, torch.cuda.current_stream())
    try:
        M.mgmlmc_set_gauge(ctx, synth.unit_gauge(dims))
        M.mgmlmc_set_mass(ctx, -0.4)
        yd = torch.empty(psi.size, dtype=torch.complex128, device='cuda')
        M.mgmlmc_apply(ctx, M.OP_D, 0, M.FP64, dev(psi), yd, 1)
        assert np.max(np.abs(host(yd) - Dpsi)) < 1e-13
    finally:
        M.mgmlmc_destroy(ctx)


# --------------------------------------------------------------- noise
@pytest.mark.parametrize('slice_', [-1, 0, 5])
def test_z4_noise_bit_exact(three, slice_):
    for level in (0, 1, 2):
        dims, dof, n = M.mgmlmc_level_info(three.ctx, level)
        sl = -1 if slice_ < 0 else slice_ % dims[3]
        out = torch.empty((3, n), dtype=torch.complex128, device='cuda')
        M.mgmlmc_noise(three.ctx, level, 123456789, 40, onz.TERM_O + level, 7, sl, out, 3)
        got = host(out)
        for r in range(3):
            if sl < 0:
                want = onz.z4_vector(n, 123456789, 40 + r, onz.TERM_O + level, 7)
            else:
                want = onz.z4_slice_vector(dims, dof, sl, 123456789, 40 + r, onz.TERM_O + level, 7)
            assert np.array_equal(got[r], want)


# --------------------------------------------------------------- hierarchy
def test_prolongator_parity(three):
    for l in range(2):
        Q = three.hier.P[l].Q  # (nagg, 2, rows, ntv)
        out = np.zeros(Q.size, dtype=np.complex128)
        M.mgmlmc_get_prolongator(three.ctx, l, out)
        assert rel(out.reshape(Q.shape), Q) < 1e-12


@pytest.mark.parametrize('fx', ['cfg1', 'three'])
def test_coarse_operator_parity(fx, request):
    s = request.getfixturevalue(fx)
    for l in range(1, s.hier.n_levels):
        A = s.hier.A[l]
        out = np.zeros(A.size, dtype=np.complex128)
        M.mgmlmc_get_coarse_op(s.ctx, l, out)
        assert rel(out.reshape(A.shape), A) < 1e-12


@pytest.mark.parametrize('prec', [0, 1])
def test_transfer_and_coarse_ops(three, prec):
    tol = 1e-12 if prec == 0 else 1e-5
    ct = torch.complex128 if prec == 0 else torch.complex64
    h = three.hier
    for l in range(2):
        n, nc = h.size(l), h.size(l + 1)
        x = synth.complex_normal((2, n), 20 + l)
        xc = synth.complex_normal((2, nc), 30 + l)
        out_c = torch.empty((2, nc), dtype=ct, device='cuda')
        out_f = torch.empty((2, n), dtype=ct, device='cuda')
        M.mgmlmc_apply(three.ctx, M.OP_RESTRICT, l, prec, dev(x, ct), out_c, 2)
        M.mgmlmc_apply(three.ctx, M.OP_PROLONG, l, prec, dev(xc, ct), out_f, 2)
        rc, pf = host(out_c), host(out_f)
        M.mgmlmc_apply(three.ctx, M.OP_PROJECT, l, prec, dev(x, ct), out_f, 2)
        pj = host(out_f)
        for r in range(2):
            assert rel(rc[r], h.P[l].restrict(x[r])) < tol
            assert rel(pf[r], h.P[l].prolong(xc[r])) < tol
            assert rel(pj[r], h.P[l].project_out(x[r])) < tol
    for l in range(1, 3):
        n = h.size(l)
        x = synth.complex_normal((2, n), 40 + l)
        out = torch.empty((2, n), dtype=ct, device='cuda')
        M.mgmlmc_apply(three.ctx, M.OP_D, l, prec, dev(x, ct), out, 2)
        y = host(out)
        for r in range(2):
            assert rel(y[r], dirac.apply_stencil(h.A[l], x[r], h.dims[l])) < tol


def test_transfer_bf16_storage(three):
    """Transfer variant 1: P stored as BF16 pairs (round to nearest, relative
    error <= 2^-9 per real entry), FP32 products and sums.  Every entry of
    P^H x or P x_c is a sum of products p_k x_k, so per output entry, real and
    imaginary parts: |got - exact| <= 2^-9 sum_k |p_k|_1 |x_k|_1 (storage)
    plus the FP32 accumulation, K 2^-24 of the same sum (K <= 2 x 192 here),
    with |z|_1 = |Re z| + |Im z|; asserted against the oracle's P applied to
    the FP32-rounded input.  The projector keeps the exact P: OP_PROJECT
    equals variant 0 bit for bit."""
    h = three.hier
    u = 2.0 ** -9 + 400 * 2.0 ** -24
    try:
        for l in range(2):
            Pm = h.P[l].matrix()
            Pabs = abs(Pm.real) + abs(Pm.imag)
            n, nc = h.size(l), h.size(l + 1)
            x = synth.complex_normal((2, n), 120 + l).astype(np.complex64).astype(np.complex128)
            xc = synth.complex_normal((2, nc), 130 + l).astype(np.complex64).astype(np.complex128)
            out_c = torch.empty((2, nc), dtype=torch.complex64, device='cuda')
            out_f = torch.empty((2, n), dtype=torch.complex64, device='cuda')
            pj = []
            for v in (0, 1):
                M.mgmlmc_set_kernel_variant(three.ctx, M.VARIANT_TRANSFER_FP32, v)
                M.mgmlmc_apply(three.ctx, M.OP_PROJECT, l, 1, dev(x, torch.complex64), out_f, 2)
                pj.append(out_f.clone())
            assert torch.equal(pj[0], pj[1])
            assert M.mgmlmc_get_kernel_variant(three.ctx, M.VARIANT_TRANSFER_FP32, 2) == 1
            M.mgmlmc_apply(three.ctx, M.OP_RESTRICT, l, 1, dev(x, torch.complex64), out_c, 2)
            M.mgmlmc_apply(three.ctx, M.OP_PROLONG, l, 1, dev(xc, torch.complex64), out_f, 2)
            rc, pf = host(out_c).astype(np.complex128), host(out_f).astype(np.complex128)
            for r in range(2):
                want = h.P[l].restrict(x[r])
                bnd = u * (Pabs.T @ (np.abs(x[r].real) + np.abs(x[r].imag))) + 1e-30
                assert np.all(np.abs(rc[r].real - want.real) <= bnd), (l, r)
                assert np.all(np.abs(rc[r].imag - want.imag) <= bnd), (l, r)
                assert np.max(np.abs(rc[r] - want)) > 1e-6 * np.max(np.abs(want))  # not the FP32 P
                want = h.P[l].prolong(xc[r])
                bnd = u * (Pabs @ (np.abs(xc[r].real) + np.abs(xc[r].imag))) + 1e-30
                assert np.all(np.abs(pf[r].real - want.real) <= bnd), (l, r)
                assert np.all(np.abs(pf[r].imag - want.imag) <= bnd), (l, r)
    finally:
        M.mgmlmc_set_kernel_variant(three.ctx, M.VARIANT_TRANSFER_FP32, 0)


def test_coarsest_trace(three):
    tr = M.mgmlmc_coarsest_trace(three.ctx)
    want = np.trace(np.linalg.inv(three.hier.matrix(2).toarray()))
    assert abs(tr - want) < 1e-10 * abs(want)


# --------------------------------------------------------------- solves
@pytest.mark.parametrize('level', [0, 1, 2])
def test_solve_fp64(three, level):
    h = three.hier
    n = h.size(level)
    b = synth.complex_normal((3, n), 50 + level)
    xd = torch.empty((3, n), dtype=torch.complex128, device='cuda')
    M.mgmlmc_apply(three.ctx, M.OP_SOLVE, level, M.FP64, dev(b), xd, 3)
    x = host(xd)
    Mx = h.matrix(level)
    sol = osolve.LevelSolver(Mx)
    for r in range(3):
        res = np.linalg.norm(b[r] - Mx @ x[r]) / np.linalg.norm(b[r])
        assert res < 1.5e-12, res
        assert rel(x[r], sol(b[r])) < 1e-9


def test_solve_mixed_precision():
    s = Setup((4, 4, 4, 8), [(2, 2, 2, 2), (2, 2, 2, 2)], [6, 4], eps=0.4, m0=-0.1, gseed=77,
              solver=dict(precision=1, inner_tol=1e-5))
    try:
        h = s.hier
        b = synth.complex_normal((2, h.size(0)), 60)
        xd = torch.empty((2, h.size(0)), dtype=torch.complex128, device='cuda')
        M.mgmlmc_apply(s.ctx, M.OP_SOLVE, 0, M.FP64, dev(b), xd, 2)
        x = host(xd)
        Mx = h.matrix(0)
        for r in range(2):
            assert np.linalg.norm(b[r] - Mx @ x[r]) / np.linalg.norm(b[r]) < 1.5e-12
    finally:
        s.close()


@pytest.mark.parametrize('ntv', [32, 50, 64, 96])
def test_wide_coarse_operator(ntv):
    """N_tv = 32 (64 dofs per coarse site: too large for the TMA-staged
    kernel's shared memory, so the plain staged stencil kernel), 50, 64 and
    96 (100, 128, 192 dofs: the wide coarse-stencil kernel, 100 with a
    partial last row tile): D_1 in FP64 (1e-12) and FP32 (1e-5) against the
    oracle's Galerkin operator, and a level-0 solve through this hierarchy to
    the 1.5e-12 residual measured with the oracle's D."""
    s = Setup((4, 4, 4, 4), [(2, 2, 2, 2)], [ntv], eps=0.3, m0=-0.2)
    try:
        A1 = s.hier.matrix(1)
        n1 = A1.shape[0]
        x = synth.complex_normal((3, n1), 91)
        y = torch.empty((3, n1), dtype=torch.complex128, device='cuda')
        M.mgmlmc_apply(s.ctx, M.OP_D, 1, M.FP64, dev(x), y, 3)
        got = host(y)
        y32 = torch.empty((3, n1), dtype=torch.complex64, device='cuda')
        M.mgmlmc_apply(s.ctx, M.OP_D, 1, M.FP32, dev(x, torch.complex64), y32, 3)
        got32 = host(y32)
        for r in range(3):
            assert rel(got[r], A1 @ x[r]) < 1e-12
            assert rel(got32[r], A1 @ x[r].astype(np.complex64).astype(np.complex128)) < 1e-5
        A0 = s.hier.matrix(0)
        b = synth.complex_normal((2, A0.shape[0]), 92)
        z = torch.empty((2, A0.shape[0]), dtype=torch.complex128, device='cuda')
        M.mgmlmc_apply(s.ctx, M.OP_SOLVE, 0, M.FP64, dev(b), z, 2)
        zs = host(z)
        for r in range(2):
            assert np.linalg.norm(b[r] - A0 @ zs[r]) / np.linalg.norm(b[r]) < 1.5e-12
        # P for more right-hand sides than 48 KB of staged coefficients hold
        # in one launch (40 x N_tv complex doubles > 48 KB from N_tv = 77)
        nr = 40
        xc = synth.complex_normal((nr, n1), 93)
        f = torch.empty((nr, A0.shape[0]), dtype=torch.complex128, device='cuda')
        M.mgmlmc_apply(s.ctx, M.OP_PROLONG, 0, M.FP64, dev(xc), f, nr)
        fs = host(f)
        for r in (0, 31, 32, nr - 1):
            assert rel(fs[r], s.hier.P[0].prolong(xc[r])) < 1e-12
    finally:
        s.close()


# --------------------------------------------------------------- estimators
def test_trace_estimator_samples_match_oracle(three):
    """identical noise, identical P: per-term sample means and variances of
    the GPU estimator equal the oracle's to solve accuracy."""
    h = three.hier
    sol = [osolve.LevelSolver(h.matrix(l)) for l in range(3)]
    E = oest.Estimators(h, sol, seed=2222)
    N = 10
    res = M.mgmlmc_estimate_trace(three.ctx, M.est_params(M.EST_ORTHOGONAL, [N] * 5, batch=4, seed=2222))
    names = ['O0', 'O1', 'F0', 'F1', 'coarsest']
    terms = dict(E.orthogonal_terms())
    for i, (r, name) in enumerate(zip(res, names)):
        X = np.array([terms[name](k) for k in range(N)])
        mu, var = oest.sample_stats(X)
        assert r['n'] == N
        assert abs(complex(r['mean_re'], r['mean_im']) - mu) < 1e-8 * max(1.0, abs(mu)), name
        assert abs(r['var'] - var) < 1e-7 * max(1.0, var), name
        assert r['max_residual'] <= 1.5e-12
        # sample by sample, not only through the mean and the variance
        got = M.mgmlmc_last_samples(three.ctx, i, N)
        assert got.shape == (N,)
        assert np.max(np.abs(got - X)) < 1e-8 * max(1.0, np.max(np.abs(X))), name
    plain = M.mgmlmc_estimate_trace(three.ctx, M.est_params(M.EST_PLAIN, [N], batch=3, seed=2222))[0]
    X = np.array([E.plain(k) for k in range(N)])
    assert abs(complex(plain['mean_re'], plain['mean_im']) - X.mean()) < 1e-8 * abs(X.mean())
    got = M.mgmlmc_last_samples(three.ctx, 0, N)
    assert np.max(np.abs(got - X)) < 1e-8 * np.max(np.abs(X))


def test_trace_samples_config1_per_sample(cfg1):
    """config-1 (4^4, two levels): every per-sample value X_k of the
    orthogonal terms O_0, F_0 and the coarsest term and of plain Hutchinson
    equals the oracle's x_k^H A x_k on identical noise and P (1e-8: solves to
    1e-12 times the condition number ~10)."""
    h = cfg1.hier
    sol = [osolve.LevelSolver(h.matrix(l)) for l in range(2)]
    N = 24
    E = oest.Estimators(h, sol, seed=2424)
    M.mgmlmc_estimate_trace(cfg1.ctx, M.est_params(M.EST_ORTHOGONAL, [N] * 3, batch=8, seed=2424))
    for i, (name, f) in enumerate(E.orthogonal_terms()):
        X = np.array([f(k) for k in range(N)])
        got = M.mgmlmc_last_samples(cfg1.ctx, i, N)
        assert np.max(np.abs(got - X)) < 1e-8 * max(1.0, np.max(np.abs(X))), name
    M.mgmlmc_estimate_trace(cfg1.ctx, M.est_params(M.EST_PLAIN, [N], batch=8, seed=2424))
    X = np.array([E.plain(k) for k in range(N)])
    assert np.max(np.abs(M.mgmlmc_last_samples(cfg1.ctx, 0, N) - X)) < 1e-8 * np.max(np.abs(X))


def test_oblique_estimator_samples_match_oracle(three):
    """the oblique decomposition (Eq. oblique_multigrid-multilevel-monte-carlo):
    identical noise and P, per-term sample means and variances of M_0, M_1 and
    the coarsest term equal the oracle's to solve accuracy; the term codes are
    MGMLMC_TERM_M + level."""
    h = three.hier
    sol = [osolve.LevelSolver(h.matrix(l)) for l in range(3)]
    E = oest.Estimators(h, sol, seed=2233)
    N = 10
    res = M.mgmlmc_estimate_trace(three.ctx, M.est_params(M.EST_OBLIQUE, [N] * 3, batch=4, seed=2233))
    assert [r['term'] for r in res] == [M.TERM_M, M.TERM_M + 1, M.TERM_COARSEST]
    for r, (name, sampler) in zip(res, E.oblique_terms()):
        X = np.array([sampler(k) for k in range(N)])
        mu, var = oest.sample_stats(X)
        assert r['n'] == N
        assert abs(complex(r['mean_re'], r['mean_im']) - mu) < 1e-8 * max(1.0, abs(mu)), name
        assert abs(r['var'] - var) < 1e-7 * max(1.0, var), name
        assert r['max_residual'] <= 1.5e-12


def test_oblique_trace_unbiased_config1(cfg1):
    """config-1: oblique MG-MLMC (N = 200 per term) within 3 SE of the dense
    exact tr(D^-1)."""
    exact_tr = np.trace(np.linalg.inv(cfg1.hier.matrix(0).toarray()))
    res = M.mgmlmc_estimate_trace(cfg1.ctx, M.est_params(M.EST_OBLIQUE, [200, 200], batch=25, seed=2311))
    est = sum(complex(r['mean_re'], r['mean_im']) for r in res)
    se = np.sqrt(sum(r['var'] / r['n'] for r in res))
    assert abs(est - exact_tr) < 3 * se


def test_four_level_hierarchy_matches_oracle():
    """L = 4 (the ABI's maximum): 8x4x4x8 -> 4x2x2x4 -> 2x2x2x2 -> 1x1x1x1
    coarse lattices, N_tv = 6, 4, 3.  Every level solve reaches 1.5e-12 with
    the oracle's operator; the 7 orthogonal and the 4 oblique terms match the
    oracle per sample on identical noise and P (1e-8)."""
    s = Setup((8, 4, 4, 8), [(2, 2, 2, 2), (2, 1, 1, 2), (2, 2, 2, 2)], [6, 4, 3],
              eps=0.4, m0=-0.1, gseed=55)
    try:
        h = s.hier
        assert h.n_levels == 4
        for l in range(4):
            A = h.matrix(l)
            b = synth.complex_normal((2, A.shape[0]), 93 + l)
            z = torch.empty((2, A.shape[0]), dtype=torch.complex128, device='cuda')
            M.mgmlmc_apply(s.ctx, M.OP_SOLVE, l, M.FP64, dev(b), z, 2)
            zs = host(z)
            for r in range(2):
                assert np.linalg.norm(b[r] - A @ zs[r]) / np.linalg.norm(b[r]) < 1.5e-12, l
        sol = [osolve.LevelSolver(h.matrix(l)) for l in range(4)]
        N = 5
        E = oest.Estimators(h, sol, seed=2244)
        res = M.mgmlmc_estimate_trace(s.ctx, M.est_params(M.EST_ORTHOGONAL, [N] * 7, batch=5, seed=2244))
        terms = dict(E.orthogonal_terms())
        names = ['O0', 'O1', 'O2', 'F0', 'F1', 'F2', 'coarsest']
        assert len(res) == 7
        for i, (r, name) in enumerate(zip(res, names)):
            X = np.array([terms[name](k) for k in range(N)])
            mu = X.mean()
            assert abs(complex(r['mean_re'], r['mean_im']) - mu) < 1e-8 * max(1.0, abs(mu)), name
            got = M.mgmlmc_last_samples(s.ctx, i, N)
            assert np.max(np.abs(got - X)) < 1e-8 * max(1.0, np.max(np.abs(X))), name
        res = M.mgmlmc_estimate_trace(s.ctx, M.est_params(M.EST_OBLIQUE, [N] * 4, batch=5, seed=2245))
        E2 = oest.Estimators(h, sol, seed=2245)
        assert len(res) == 4
        for r, (name, sampler) in zip(res, E2.oblique_terms()):
            mu = np.mean([sampler(k) for k in range(N)])
            assert abs(complex(r['mean_re'], r['mean_im']) - mu) < 1e-8 * max(1.0, abs(mu)), name
    finally:
        s.close()


def test_trace_unbiased_config1(cfg1):
    """config-1: orthogonal MG-MLMC (N = 200 per term, seed 2301) and plain
    Hutchinson (N = 200) each within 3 SE of the dense exact tr(D^-1)."""
    exact_tr = np.trace(np.linalg.inv(cfg1.hier.matrix(0).toarray()))
    res = M.mgmlmc_estimate_trace(cfg1.ctx, M.est_params(M.EST_ORTHOGONAL, [200, 200, 200], batch=25, seed=2301))
    est = sum(complex(r['mean_re'], r['mean_im']) for r in res)
    se = np.sqrt(sum(r['var'] / r['n'] for r in res))
    assert abs(est - exact_tr) < 3 * se
    p = M.mgmlmc_estimate_trace(cfg1.ctx, M.est_params(M.EST_PLAIN, [200], batch=25, seed=2302))[0]
    assert abs(complex(p['mean_re'], p['mean_im']) - exact_tr) < 3 * np.sqrt(p['var'] / p['n'])


def test_connected_correlator_matches_oracle():
    dims = (2, 2, 2, 8)
    s = Setup(dims, [(2, 2, 2, 2), (1, 1, 1, 2)], [4, 3], eps=0.4, m0=0.1, gseed=31)
    try:
        h = s.hier
        sol = [osolve.LevelSolver(h.matrix(l)) for l in range(3)]
        E = oest.Estimators(h, sol, seed=4040)
        N = 3
        mean, var = M.mgmlmc_connected_correlator(s.ctx, M.EST_ORTHOGONAL, N, 4040, 0, 8, 5)
        X = np.array([E.connected(k) for k in range(N)])
        assert np.max(np.abs(mean - X.mean(axis=0))) < 1e-9 * np.max(np.abs(X.mean(axis=0)))
        mp, vp = M.mgmlmc_connected_correlator(s.ctx, M.EST_PLAIN, N, 4040, 0, 8, 1)
        Xp = np.array([E.connected_plain(k) for k in range(N)])
        assert np.max(np.abs(mp[0, 0] - Xp.mean(axis=0))) < 1e-9 * np.max(np.abs(Xp.mean(axis=0)))
        # unbiasedness against the exact split (Eq. connected-G, Eq. G-split):
        # the dense G_rs(t) of the oracle's dense operators, every (r, s, t)
        # within 5 standard errors of the mean of 256 samples (fixed seed)
        B = exact.DenseTerms(h).B_matrices()
        G = exact.correlator_exact(B, dims)
        Ns = 256
        mean, var = M.mgmlmc_connected_correlator(s.ctx, M.EST_ORTHOGONAL, Ns, 4042, 0, 8, 5)
        assert G.shape == mean.shape
        se = np.sqrt(var / Ns)
        assert np.all(np.abs(mean - G) <= 5 * se + 1e-12 * np.max(np.abs(G)))
        # and the sum over (r, s) is the full correlator G(t)
        assert np.allclose(G.sum(axis=(0, 1)), exact.correlator_exact([np.linalg.inv(h.matrix(0).toarray())],
                                                                     dims)[0, 0], rtol=1e-10, atol=0)
    finally:
        s.close()


def test_disconnected_loop_matches_oracle():
    dims = (2, 2, 2, 8)
    s = Setup(dims, [(2, 2, 2, 2), (1, 1, 1, 2)], [4, 3], eps=0.4, m0=0.1, gseed=33)
    try:
        h = s.hier
        sol = [osolve.LevelSolver(h.matrix(l)) for l in range(3)]
        E = oest.Estimators(h, sol, seed=5050)
        N = 12
        mean, var = M.mgmlmc_disconnected_loop(s.ctx, M.EST_ORTHOGONAL, 3, N, 5050, 0, 5)
        X = np.array([E.disconnected(k, 3) for k in range(N)])
        assert np.max(np.abs(mean - X.mean(axis=0))) < 1e-9 * np.max(np.abs(X.mean(axis=0)))
        mp, _ = M.mgmlmc_disconnected_loop(s.ctx, M.EST_PLAIN, 3, N, 5050, 0, 1)
        Xp = np.array([E.disconnected_plain(k, 3) for k in range(N)])
        assert abs(mp[0] - Xp.mean()) < 1e-9 * abs(Xp.mean())
    finally:
        s.close()


def test_oblique_correlator_and_loop_match_oracle():
    """the oblique split (R = L operators B_l of Eq. G-traditional) of the
    connected correlator and of the disconnected loop: GPU means equal the
    oracle's on identical noise and P (the oracle applies Gamma5 B^H Gamma5
    literally with adjoint solves, the library uses that it equals B)."""
    dims = (2, 2, 2, 8)
    s = Setup(dims, [(2, 2, 2, 2), (1, 1, 1, 2)], [4, 3], eps=0.4, m0=0.1, gseed=31)
    try:
        h = s.hier
        sol = [osolve.LevelSolver(h.matrix(l)) for l in range(3)]
        E = oest.Estimators(h, sol, seed=4141)
        N = 3
        mean, var = M.mgmlmc_connected_correlator(s.ctx, M.EST_OBLIQUE, N, 4141, 0, 8, 5)
        X = np.array([E.connected(k, kind='oblique') for k in range(N)])
        assert mean.shape == X.shape[1:]
        assert np.max(np.abs(mean - X.mean(axis=0))) < 1e-9 * np.max(np.abs(X.mean(axis=0)))
        E2 = oest.Estimators(h, sol, seed=5151)
        N = 12
        mean, var = M.mgmlmc_disconnected_loop(s.ctx, M.EST_OBLIQUE, 3, N, 5151, 0, 5)
        Xd = np.array([E2.disconnected(k, 3, kind='oblique') for k in range(N)])
        assert mean.shape == Xd.shape[1:]
        assert np.max(np.abs(mean - Xd.mean(axis=0))) < 1e-9 * np.max(np.abs(Xd.mean(axis=0)))
    finally:
        s.close()


# --------------------------------------------------------------- failures
def test_failures_return_status_and_context_survives(three):
    from paper_2509_11424_gb300.mgmlmc import MgmlmcError
    n = three.hier.size(0)
    b = dev(synth.complex_normal(n, 70))
    x = torch.empty_like(b)
    M.mgmlmc_set_solver(three.ctx, max_iter=1)
    with pytest.raises(MgmlmcError) as e:
        M.mgmlmc_apply(three.ctx, M.OP_SOLVE, 0, M.FP64, b, x, 1)
    assert e.value.status == 5
    M.mgmlmc_set_solver(three.ctx)
    M.mgmlmc_apply(three.ctx, M.OP_SOLVE, 0, M.FP64, b, x, 1)  # usable again
    with pytest.raises(MgmlmcError) as e:
        M.mgmlmc_apply(three.ctx, 99, 0, M.FP64, b, x, 1)
    assert e.value.status == 1
    with pytest.raises(MgmlmcError):
        M.mgmlmc_set_solver(three.ctx, restart=0)


def test_nan_gauge_rejected():
    from paper_2509_11424_gb300.mgmlmc import MgmlmcError
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 1).copy()
    U[17] = np.nan
    ctx = M.mgmlmc_create(dims, torch.cuda.current_stream())
    try:
        with pytest.raises(MgmlmcError) as e:
            M.mgmlmc_set_gauge(ctx, U)
        assert e.value.status == 6
        with pytest.raises(MgmlmcError) as e:
            M.mgmlmc_build_hierarchy(ctx, M.mg_params([(2, 2, 2, 2)], [4]))
        assert e.value.status == 2
    finally:
        M.mgmlmc_destroy(ctx)


def test_fine_batch_and_released_workspaces_keep_samples(three):
    """fine_batch (the level-0 memory bound) only regroups the right-hand
    sides of the fine-level solves: the per-sample values of every
    orthogonal term agree with the ungrouped run to the solves' accuracy,
    also after mgmlmc_release_workspaces freed every work buffer."""
    N = 10
    p = M.est_params(M.EST_ORTHOGONAL, [N] * 5, batch=5, seed=2626)
    M.mgmlmc_estimate_trace(three.ctx, p)
    ref = [M.mgmlmc_last_samples(three.ctx, i, N) for i in range(5)]
    try:
        M.mgmlmc_set_solver(three.ctx, fine_batch=2)
        M.mgmlmc_release_workspaces(three.ctx)
        res = M.mgmlmc_estimate_trace(three.ctx, p)
        assert [r['n'] for r in res] == [N] * 5
        for i in range(5):
            got = M.mgmlmc_last_samples(three.ctx, i, N)
            assert np.max(np.abs(got - ref[i])) < 1e-8 * max(1.0, np.max(np.abs(ref[i]))), i
    finally:
        M.mgmlmc_set_solver(three.ctx)
