"""Pins of the oracle's gauge-covariant network: with the Wilson hop
matrices as weights one layer is the Dirac operator; gauge covariance; the
adjoint identity; gradients against central finite differences."""
import numpy as np
import pytest

from oracle import dirac, learned
from paper_2509_11424_gb300 import synth

DIMS = (2, 4, 2, 4)


def wilson_weights(m0):
    W = np.zeros((9, 1, 1, 4, 4), dtype=np.complex128)
    W[0, 0, 0] = (4 + m0) * np.eye(4)
    for mu in range(4):
        W[1 + 2 * mu, 0, 0] = -0.5 * (np.eye(4) - dirac.GAMMA[mu])
        W[2 + 2 * mu, 0, 0] = -0.5 * (np.eye(4) + dirac.GAMMA[mu])
    return W


def test_layer_with_wilson_hops_is_D():
    U = synth.gauge_field(DIMS, 0.5, 1)
    psi = synth.complex_normal(dirac.volume(DIMS) * 12, 2)
    out = learned.layer_forward(wilson_weights(-0.3), psi[None], U, DIMS)[0]
    assert np.max(np.abs(out - dirac.apply_wilson(U, psi, -0.3, DIMS))) < 1e-13


def rand_W(Cout, Cin, seed):
    return synth.complex_normal((9, Cout, Cin, 4, 4), seed)


def test_gauge_covariance():
    U = synth.gauge_field(DIMS, 0.5, 3)
    V = dirac.volume(DIMS)
    g = synth.random_su3(V, 4, eps=3.0).reshape(-1)
    Ug = dirac.gauge_transform_links(U, g, DIMS)
    psi = synth.complex_normal((2, V * 12), 5)
    W = rand_W(3, 2, 6)
    a = learned.layer_forward(W, np.array([dirac.gauge_transform_spinor(p, g, DIMS) for p in psi]), Ug, DIMS)
    b = np.array([dirac.gauge_transform_spinor(p, g, DIMS) for p in learned.layer_forward(W, psi, U, DIMS)])
    assert np.max(np.abs(a - b)) < 1e-12


def test_adjoint_identity():
    U = synth.gauge_field(DIMS, 0.5, 7)
    V = dirac.volume(DIMS)
    W = rand_W(3, 2, 8)
    a = synth.complex_normal((3, V * 12), 9)
    b = synth.complex_normal((2, V * 12), 10)
    lhs = np.vdot(a, learned.layer_forward(W, b, U, DIMS))
    rhs = np.vdot(learned.layer_adjoint(W, a, U, DIMS), b)
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_gradients_against_finite_differences():
    U = synth.gauge_field(DIMS, 0.5, 11)
    V = dirac.volume(DIMS)
    m0 = 0.2
    D = lambda v: dirac.apply_wilson(U, v, m0, DIMS)
    DH = lambda v: dirac.apply_gamma5(D(dirac.apply_gamma5(v)))
    Ws = learned.init_weights(3, 1.0 / (4 + m0), 12, noise=0.2)
    r = synth.complex_normal(V * 12, 13)
    L, grads = learned.loss_and_grads(Ws, r, U, DIMS, D, DH)
    h = 1e-6
    rng = np.random.default_rng(14)
    for layer in range(3):
        for _ in range(4):
            idx = tuple(int(rng.integers(0, s)) for s in Ws[layer].shape)
            for part, scale in ((1.0, 're'), (1j, 'im')):
                Wp = [w.copy() for w in Ws]
                Wm = [w.copy() for w in Ws]
                Wp[layer][idx] += h * part
                Wm[layer][idx] -= h * part
                Lp, _ = learned.loss_and_grads(Wp, r, U, DIMS, D, DH)
                Lm, _ = learned.loss_and_grads(Wm, r, U, DIMS, D, DH)
                fd = (Lp - Lm) / (2 * h)
                g = grads[layer][idx]
                an = 2 * (g.real if scale == 're' else g.imag)
                assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (layer, idx, scale, fd, an)
