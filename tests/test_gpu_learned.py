"""The learned gauge-covariant smoother on the GPU: forward pass and FP64
loss / weight gradients against the oracle (oracle/learned.py), training on
solver-produced residuals lowering the loss, and solves with the trained
learned step (SAP + network) converging to the 1e-12 residual (measured with
the oracle's D) in no more outer iterations than with SAP alone, and the
network as the initial guess of the fine-level solves."""
import numpy as np
import pytest

from oracle import dirac, learned as oln
from paper_2509_11424_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip('torch')
if not torch.cuda.is_available():
    pytest.skip('needs a CUDA GPU', allow_module_level=True)

from gpu_util import Setup, dev, host, rel, require_lib  # noqa: E402

M = require_lib()
DIMS = (4, 4, 4, 8)


def weights_for(C, seed):
    shapes = [(9, C, 1, 4, 4), (9, C, C, 4, 4), (9, 1, C, 4, 4)]
    return [0.3 * synth.complex_normal(s, seed + i) for i, s in enumerate(shapes)]


@pytest.fixture(scope='module')
def net_ctx():
    U = synth.gauge_field(DIMS, 0.4, 301)
    ctx = M.mgmlmc_create(DIMS, torch.cuda.current_stream())
    M.mgmlmc_set_gauge(ctx, U)
    M.mgmlmc_set_mass(ctx, 0.2)
    M.mgmlmc_learned_init(ctx, 3, 7)
    Ws = weights_for(3, 310)
    flat = np.concatenate([w.reshape(-1) for w in Ws])
    assert flat.size == M.mgmlmc_learned_size(ctx)
    M.mgmlmc_learned_weights(ctx, flat.view(np.float64).copy(), 1)
    yield ctx, U, Ws
    M.mgmlmc_destroy(ctx)


@pytest.mark.parametrize('prec,tol', [(0, 1e-12), (1, 1e-5)])
def test_forward_matches_oracle(net_ctx, prec, tol):
    ctx, U, Ws = net_ctx
    n = dirac.volume(DIMS) * 12
    r = synth.complex_normal((2, n), 320)
    ct = torch.complex128 if prec == 0 else torch.complex64
    out = torch.empty((2, n), dtype=ct, device='cuda')
    M.mgmlmc_apply(ctx, M.OP_NET, 0, prec, dev(r, ct), out, 2)
    got = host(out)
    for b in range(2):
        want = oln.network_forward(Ws, r[b], U, DIMS)[-1][0]
        assert rel(got[b], want) < tol


def test_loss_and_gradient_match_oracle(net_ctx):
    ctx, U, Ws = net_ctx
    n = dirac.volume(DIMS) * 12
    r = synth.complex_normal((2, n), 330)
    grad = np.zeros(2 * M.mgmlmc_learned_size(ctx))
    L = M.mgmlmc_learned_loss_grad(ctx, dev(r), 2, grad)
    D = lambda v: dirac.apply_wilson(U, v, 0.2, DIMS)
    DH = lambda v: dirac.apply_gamma5(D(dirac.apply_gamma5(v)))
    Lw, gw = 0.0, [np.zeros_like(w) for w in Ws]
    for b in range(2):
        l, g = oln.loss_and_grads(Ws, r[b], U, DIMS, D, DH)
        Lw += l
        gw = [a + c for a, c in zip(gw, g)]
    assert abs(L - Lw) < 1e-10 * abs(Lw)
    want = np.concatenate([g.reshape(-1) for g in gw])
    assert rel(grad.view(np.complex128), want) < 1e-10


def test_training_lowers_loss_and_trained_solves_converge():
    dims = (8, 8, 8, 8)
    s = Setup(dims, [(4, 4, 4, 4), (2, 2, 2, 2)], [8, 6], eps=0.4, m0=-0.2, gseed=340, oracle=False,
              solver=dict(smoother=1, sap_iters=4, smoother_steps=1, coarse_iters=4, precision=1,
                          inner_tol=1e-6))
    try:
        ctx = s.ctx
        res = M.mgmlmc_learned_train(ctx, channels=4, steps=60, batch=4, pool=64, lr=2e-3, seed=341)
        assert res['pairs'] == 64 and np.isfinite(res['loss_last'])
        assert res['loss_last'] < 0.9 * res['loss_init'], res
        Mx = dirac.wilson_matrix(s.U, -0.2, dims)
        n = Mx.shape[0]
        b = synth.complex_normal((2, n), 342)
        x = torch.empty((2, n), dtype=torch.complex128, device='cuda')

        def solve_iters():
            M.mgmlmc_apply(ctx, M.OP_SOLVE, 0, M.FP64, dev(b), x, 2)
            xs = host(x)
            for r in range(2):
                assert np.linalg.norm(b[r] - Mx @ xs[r]) / np.linalg.norm(b[r]) < 1.5e-12
            return M.mgmlmc_last_solve_stats(ctx)[0]

        M.mgmlmc_set_solver(ctx, smoother=2, smoother_steps=1, coarse_iters=4, precision=1, inner_tol=1e-6)
        it_learned = solve_iters()
        assert M.mgmlmc_learned_stats(ctx) == 0
        M.mgmlmc_set_solver(ctx, smoother=1, smoother_steps=1, coarse_iters=4, precision=1, inner_tol=1e-6)
        it_sap = solve_iters()
        print('outer iterations: SAP + learned step %d, SAP alone %d' % (it_learned, it_sap))
        assert it_learned <= it_sap, (it_learned, it_sap)
    finally:
        s.close()


def test_learned_initial_guess():
    """The network as the initial guess of the fine-level solves (solver
    option learned_guess), trained on the right-hand sides the estimator's
    O_0 solves start from (training source 1: projected Z4 noise).  Training lowers the loss; on a projected
    right-hand side c (unit norm) the trained network's guess leaves a
    smaller residual ||c - alpha D N(c)|| (alpha residual-minimising) than
    the untrained one, i.e. what training gains; solves that start from the
    guess reach the 1e-12 true residual (the oracle's D) and the solution of
    the solves that start from zero to 1e-9."""
    dims = (8, 8, 8, 8)
    solver = dict(smoother=1, sap_iters=4, smoother_steps=1, coarse_iters=4, precision=1, inner_tol=1e-6)
    s = Setup(dims, [(4, 4, 4, 4), (2, 2, 2, 2)], [8, 6], eps=0.4, m0=-0.2, gseed=350, oracle=False,
              solver=solver)
    try:
        ctx = s.ctx
        Mx = dirac.wilson_matrix(s.U, -0.2, dims)
        n = Mx.shape[0]
        b = synth.complex_normal((2, n), 352)
        pb = torch.empty((2, n), dtype=torch.complex128, device='cuda')
        M.mgmlmc_apply(ctx, M.OP_PROJECT, 0, M.FP64, dev(b), pb, 2)
        c = host(pb)
        c = c / np.linalg.norm(c, axis=1, keepdims=True)

        def guess_residual():
            e = torch.empty((2, n), dtype=torch.complex128, device='cuda')
            M.mgmlmc_apply(ctx, M.OP_NET, 0, M.FP64, dev(c), e, 2)
            out = []
            for r, er in enumerate(host(e)):
                q = Mx @ er
                al = np.vdot(q, c[r]) / np.vdot(q, q)
                out.append(np.linalg.norm(c[r] - al * q))
            return np.array(out)

        M.mgmlmc_learned_init(ctx, 1, 353)
        rho0 = guess_residual()
        res = M.mgmlmc_learned_train(ctx, channels=1, steps=80, batch=4, pool=64, lr=2e-3, seed=353, source=1)
        assert res['pairs'] == 64 and res['loss_last'] < res['loss_init'], res
        rho = guess_residual()
        print('guess residual: untrained %s, trained %s' % (rho0, rho))
        assert np.all(rho < rho0) and np.all(rho < 1.0), (rho0, rho)

        x = torch.empty((2, n), dtype=torch.complex128, device='cuda')
        sols, iters = [], []
        for guess in (0, 1):
            M.mgmlmc_set_solver(ctx, learned_guess=guess, **solver)
            M.mgmlmc_apply(ctx, M.OP_SOLVE, 0, M.FP64, dev(b), x, 2)
            xs = host(x)
            for r in range(2):
                assert np.linalg.norm(b[r] - Mx @ xs[r]) / np.linalg.norm(b[r]) < 1.5e-12, guess
            sols.append(xs)
            iters.append(M.mgmlmc_last_solve_stats(ctx)[0])
        print('outer iterations: from zero %d, from the learned guess %d' % tuple(iters))
        assert rel(sols[1], sols[0]) < 1e-9
        # out-of-range option values are refused, the context stays usable
        with pytest.raises(M.MgmlmcError):
            M.mgmlmc_set_solver(ctx, learned_guess=2, **solver)
        with pytest.raises(M.MgmlmcError):
            M.mgmlmc_learned_train(ctx, channels=1, steps=1, batch=1, pool=1, source=2)
        M.mgmlmc_set_solver(ctx, **solver)
    finally:
        s.close()
