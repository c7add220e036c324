"""Parity at the benchmark's full size (16^4, eps 0.4, seed 1002, the
oracle-chosen m0) in the launch configuration bench.py times (32 right-hand
sides, its solver settings): Dslash FP64 / FP32 element by element, Z4 noise
bit-exact, P orthonormal and the Galerkin relation D_1 = P^H D P checked on
vectors with the oracle's D, the coarse operators Gamma5-hermitian, and the
level-0 solves reaching the 1e-12 residual measured with the oracle's D."""
import json
import os

import numpy as np
import pytest

from oracle import dirac, noise as onz
from paper_2509_11424_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip('torch')
if not torch.cuda.is_available():
    pytest.skip('needs a CUDA GPU', allow_module_level=True)

from gpu_util import dev, host, rel, require_lib  # noqa: E402

M = require_lib()
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DIMS = (16, 16, 16, 16)
B = 32  # right-hand sides per launch, as bench.py runs them


@pytest.fixture(scope='module')
def full():
    import bench
    m0 = json.load(open(os.path.join(ROOT, 'tests', 'golden', 'mass_16x16x16x16.json')))['m0']
    U = synth.gauge_field(DIMS, bench.EPS_GAUGE, bench.GAUGE_SEED)
    ctx = M.mgmlmc_create(DIMS, torch.cuda.current_stream())
    M.mgmlmc_set_gauge(ctx, U)
    M.mgmlmc_set_mass(ctx, m0)
    M.mgmlmc_set_solver(ctx, precision=M.FP32, **bench.SOLVER)
    M.mgmlmc_build_hierarchy(ctx, M.mg_params(bench.BLOCKS, bench.NTV, setup_rounds=6, setup_iters=30,
                                               seed=bench.TV_SEED))
    Mx = dirac.wilson_matrix(U, m0, DIMS).tocsr()
    yield ctx, U, m0, Mx
    M.mgmlmc_destroy(ctx)


@pytest.mark.parametrize('prec,tol', [(0, 1e-12), (1, 1e-5)])
def test_dslash_full_size(full, prec, tol):
    ctx, U, m0, Mx = full
    n = Mx.shape[0]
    x = synth.complex_normal((B, n), 401)
    ct = torch.complex128 if prec == 0 else torch.complex64
    y = torch.empty((B, n), dtype=ct, device='cuda')
    M.mgmlmc_apply(ctx, M.OP_D, 0, prec, dev(x, ct), y, B)
    got = host(y)
    for r in range(B):
        assert rel(got[r], Mx @ x[r].astype(np.complex128 if prec == 0 else np.complex64).astype(np.complex128)) < tol


def test_noise_full_size_bit_exact(full):
    ctx = full[0]
    n = full[3].shape[0]
    out = torch.empty((B, n), dtype=torch.complex128, device='cuda')
    M.mgmlmc_noise(ctx, 0, 2002, 16, onz.TERM_O, 0, -1, out, B)
    got = host(out)
    for r in (0, B - 1):
        assert np.array_equal(got[r], onz.z4_vector(n, 2002, 16 + r, onz.TERM_O))


def test_galerkin_and_orthonormality_full_size(full):
    ctx, U, m0, Mx = full
    _, dof1, n1 = M.mgmlmc_level_info(ctx, 1)
    n = Mx.shape[0]
    xc = synth.complex_normal((2, n1), 402)
    f = torch.empty((2, n), dtype=torch.complex128, device='cuda')
    back = torch.empty((2, n1), dtype=torch.complex128, device='cuda')
    M.mgmlmc_apply(ctx, M.OP_PROLONG, 0, 0, dev(xc), f, 2)
    M.mgmlmc_apply(ctx, M.OP_RESTRICT, 0, 0, f, back, 2)
    assert rel(host(back), xc) < 1e-13  # P^H P = I
    # D_1 xc == P^H (D (P xc)) with the oracle's D in the middle
    Dpx = dev(np.array([Mx @ v for v in host(f)]))
    want = torch.empty((2, n1), dtype=torch.complex128, device='cuda')
    M.mgmlmc_apply(ctx, M.OP_RESTRICT, 0, 0, Dpx, want, 2)
    got = torch.empty((2, n1), dtype=torch.complex128, device='cuda')
    M.mgmlmc_apply(ctx, M.OP_D, 1, 0, dev(xc), got, 2)
    assert rel(host(got), host(want)) < 1e-12
    # Gamma5c-hermiticity of D_1: <g5 a, D_1 b> = <D_1 a, g5 b>... as (g5 D_1)^H = g5 D_1
    a, b = synth.complex_normal(n1, 403), synth.complex_normal(n1, 404)
    Da = torch.empty(n1, dtype=torch.complex128, device='cuda')
    Db = torch.empty(n1, dtype=torch.complex128, device='cuda')
    M.mgmlmc_apply(ctx, M.OP_D, 1, 0, dev(a), Da, 1)
    M.mgmlmc_apply(ctx, M.OP_D, 1, 0, dev(dirac.apply_gamma5(b, dof1)), Db, 1)
    lhs = np.vdot(host(Da), b)
    rhs = np.vdot(dirac.apply_gamma5(a, dof1), host(Db))
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_solve_full_size(full):
    ctx, U, m0, Mx = full
    n = Mx.shape[0]
    b = np.array([onz.z4_vector(n, 2002, k, onz.TERM_PLAIN) for k in range(B)])
    x = torch.empty((B, n), dtype=torch.complex128, device='cuda')
    M.mgmlmc_apply(ctx, M.OP_SOLVE, 0, M.FP64, dev(b), x, B)
    xs = host(x)
    for r in range(B):
        assert np.linalg.norm(b[r] - Mx @ xs[r]) / np.linalg.norm(b[r]) < 1.5e-12


def test_estimator_samples_full_size():
    """Per-sample values of every orthogonal term at the benchmark's size and
    batch (16^4, 32 right-hand sides per launch, mixed-precision solver with
    SAP) against the oracle on identical noise and identical P (test vectors
    imported from the seeded generator on both sides).  The coarse terms O_1,
    F_1 and the coarsest term are compared on all 32 samples (the oracle
    factors the coarse operators); the fine terms O_0 and F_0, whose oracle
    samples each need an unpreconditioned GMRES solve of the 786,432-dof
    system (~430 iterations), on the batch's last sample (O_0) and sample 7
    (F_0), the two solves run side by side.  Each
    sample is exact to the solves' 1e-12 times the condition number (~45), so
    1e-8 relative to the largest sample of the term."""
    import concurrent.futures as cf

    import bench
    from oracle import estimators as oest, multigrid as omg, solve as osolve
    m0 = json.load(open(os.path.join(ROOT, 'tests', 'golden', 'mass_16x16x16x16.json')))['m0']
    U = synth.gauge_field(DIMS, bench.EPS_GAUGE, bench.GAUGE_SEED)
    ctx = M.mgmlmc_create(DIMS, torch.cuda.current_stream())
    try:
        M.mgmlmc_set_gauge(ctx, U)
        M.mgmlmc_set_mass(ctx, m0)
        M.mgmlmc_set_solver(ctx, precision=M.FP32, **bench.SOLVER)
        tvs, cur, dof = [], DIMS, 12
        for l, (b, k) in enumerate(zip(bench.BLOCKS, bench.NTV)):
            n = int(np.prod(cur)) * dof
            tv = synth.random_test_vectors(n, k, 3900 + l)
            tvs.append(tv)
            M.mgmlmc_set_test_vectors(ctx, l, np.ascontiguousarray(tv.T), k, n, on_device=False)
            cur = tuple(c // bb for c, bb in zip(cur, b))
            dof = 2 * k
        M.mgmlmc_build_hierarchy(ctx, M.mg_params(bench.BLOCKS, bench.NTV, setup_rounds=0))
        seed = 2929
        M.mgmlmc_estimate_trace(ctx, M.est_params(M.EST_ORTHOGONAL, [B] * 5, batch=B, seed=seed))
        got = [M.mgmlmc_last_samples(ctx, i, B) for i in range(5)]
    finally:
        M.mgmlmc_destroy(ctx)
    h = omg.Hierarchy(dirac.wilson_stencil(U, m0, DIMS), DIMS, bench.BLOCKS, tvs)
    sol = [osolve.LevelSolver(h.matrix(l)) for l in range(3)]
    terms = dict(oest.Estimators(h, sol, seed=seed).orthogonal_terms())
    order = ['O0', 'O1', 'F0', 'F1', 'coarsest']
    picks = {'O0': [B - 1], 'F0': [7], 'O1': range(B), 'F1': range(B), 'coarsest': range(B)}
    jobs = [(name, k) for name in order for k in picks[name]]
    fine = [j for j in jobs if j[0] in ('O0', 'F0')]
    with cf.ThreadPoolExecutor(max_workers=len(fine)) as ex:
        fut = {j: ex.submit(terms[j[0]], j[1]) for j in fine}
        want = {j: terms[j[0]](j[1]) for j in jobs if j not in fut}
        want.update({j: f.result() for j, f in fut.items()})
    for i, name in enumerate(order):
        scale = max(abs(want[(name, k)]) for k in picks[name])
        for k in picks[name]:
            assert abs(got[i][k] - want[(name, k)]) < 1e-8 * max(1.0, scale), (name, k)
