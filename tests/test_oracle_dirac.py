"""Pins of the oracle's Wilson-Dirac operator against facts fixed by the
mathematics (closed forms, identities, hand-built cases), not against itself."""
import numpy as np
import pytest

from oracle import dirac, exact
from paper_2509_11424_gb300 import synth

ODD = (6, 4, 4, 8)  # non-power-of-two extents catch index mix-ups


def rand_spinor(dims, seed):
    return synth.complex_normal(dirac.volume(dims) * 12, seed)


def test_gamma_algebra():
    g, g5 = dirac.GAMMA, dirac.GAMMA5
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            ac = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(ac, 2 * np.eye(4) * (mu == nu))
        assert np.allclose(g5 @ g[mu] + g[mu] @ g5, 0)
    # chiral basis: Gamma_5 is diagonal, flipping the sign of spins 2, 3 (Sec. 2)
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))


@pytest.mark.parametrize('dims,m0', [((4, 2, 2, 4), -0.2), ((2, 4, 2, 2), 0.3)])
def test_free_field_spectrum_closed_form(dims, m0):
    """U = 1: the dense spectrum equals m(p) +- i|sin p|, 6-fold, with
    antiperiodic time momenta."""
    M = dirac.wilson_matrix(synth.unit_gauge(dims), m0, dims).toarray()
    ev = np.linalg.eigvals(M)
    ref = exact.free_field_eigenvalues(dims, m0)
    key = lambda z: np.lexsort((np.round(z.imag, 9), np.round(z.real, 9)))
    assert np.allclose(ev[key(ev)], ref[key(ref)], atol=1e-10)


@pytest.mark.parametrize('n', [(0, 0, 0, 0), (1, 2, 3, 5), (5, 3, 1, 7)])
def test_plane_wave_any_size(n):
    """exp(i p.x) chi is mapped to (m(p) + i gamma.sin p) chi exp(i p.x)."""
    chi = synth.complex_normal((4, 3), 7)
    psi, Dpsi = exact.free_field_plane_wave(ODD, -0.4, n, chi)
    out = dirac.apply_wilson(synth.unit_gauge(ODD), psi, -0.4, ODD)
    assert np.max(np.abs(out - Dpsi)) < 1e-13


def test_gamma5_hermiticity():
    """(Gamma_5 D)^H = Gamma_5 D for a random SU(3) field (Sec. 2)."""
    U = synth.gauge_field(ODD, 0.5, 11)
    a, b = rand_spinor(ODD, 1), rand_spinor(ODD, 2)
    D = lambda v: dirac.apply_wilson(U, v, -0.3, ODD)
    g5 = dirac.apply_gamma5
    lhs = np.vdot(D(a), b)
    rhs = np.vdot(g5(a), D(g5(b)))
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_gauge_covariance():
    """D[U^g] G psi = G D[U] psi with U^g_mu(x) = g(x) U_mu(x) g(x+mu)^H."""
    U = synth.gauge_field(ODD, 0.4, 12)
    V = dirac.volume(ODD)
    g = synth.random_su3(V, 13, eps=3.0).reshape(-1)
    Ug = dirac.gauge_transform_links(U, g, ODD)
    psi = rand_spinor(ODD, 3)
    lhs = dirac.apply_wilson(Ug, dirac.gauge_transform_spinor(psi, g, ODD), 0.1, ODD)
    rhs = dirac.gauge_transform_spinor(dirac.apply_wilson(U, psi, 0.1, ODD), g, ODD)
    assert np.max(np.abs(lhs - rhs)) < 1e-12


def test_single_link_by_hand():
    """One non-trivial link U_mu(x0); a delta source at x0 + mu and at x0
    checks hop direction, site numbering and the link/adjoint placement."""
    dims = ODD
    V = dirac.volume(dims)
    Lx, Ly, Lz, Lt = dims
    x0 = (2, 1, 2, 5)
    s0 = x0[0] + Lx * (x0[1] + Ly * (x0[2] + Lz * x0[3]))
    W = synth.random_su3(1, 21, eps=1.0)[0]
    one = np.eye(4)
    for mu, stride in enumerate([1, Lx, Lx * Ly, Lx * Ly * Lz]):
        U = synth.unit_gauge(dims).reshape(V, 4, 3, 3).copy()
        U[s0, mu] = W
        chi = synth.complex_normal((4, 3), 30 + mu)
        # source at x0 + mu: the forward hop of site x0 sees W chi
        s1 = s0 + stride  # x0 + mu stays inside the lattice for this x0
        psi = np.zeros((V, 4, 3), dtype=np.complex128)
        psi[s1] = chi
        out = dirac.apply_wilson(U.reshape(-1), psi.reshape(-1), 0.0, dims).reshape(V, 4, 3)
        want = -0.5 * (one - dirac.GAMMA[mu]) @ chi @ W.T
        assert np.allclose(out[s0], want, atol=1e-14)
        # source at x0: the backward hop of site x0 + mu sees W^H chi
        psi = np.zeros((V, 4, 3), dtype=np.complex128)
        psi[s0] = chi
        out = dirac.apply_wilson(U.reshape(-1), psi.reshape(-1), 0.0, dims).reshape(V, 4, 3)
        want = -0.5 * (one + dirac.GAMMA[mu]) @ chi @ np.conj(W)
        assert np.allclose(out[s1], want, atol=1e-14)


def test_time_boundary_sign():
    """A hop across t = Lt-1 -> 0 carries -1 (antiperiodic fermions)."""
    dims = (2, 2, 2, 4)
    V = dirac.volume(dims)
    psi = np.zeros((V, 4, 3), dtype=np.complex128)
    chi = synth.complex_normal((4, 3), 5)
    psi[0] = chi  # site (0,0,0,0)
    out = dirac.apply_wilson(synth.unit_gauge(dims), psi.reshape(-1), 0.0, dims).reshape(V, 4, 3)
    s_last = 0 + 2 * 2 * 2 * 3  # (0,0,0,Lt-1): its forward t-neighbour is site 0
    want = +0.5 * (np.eye(4) - dirac.GAMMA[3]) @ chi
    assert np.allclose(out[s_last], want, atol=1e-14)


@pytest.mark.parametrize('dims', [ODD, (2, 2, 2, 2)])
def test_stencil_and_matrix_forms_agree(dims):
    U = synth.gauge_field(dims, 0.6, 40)
    psi = rand_spinor(dims, 41)
    y = dirac.apply_wilson(U, psi, -0.25, dims)
    A = dirac.wilson_stencil(U, -0.25, dims)
    assert np.max(np.abs(dirac.apply_stencil(A, psi, dims) - y)) < 1e-13
    assert np.max(np.abs(dirac.stencil_matrix(A, dims) @ psi - y)) < 1e-13


def test_free_field_trace_4444():
    """Dense tr(D^-1) on 4^4 at m0 = -0.2 equals the momentum sum."""
    dims = (4, 4, 4, 4)
    M = dirac.wilson_matrix(synth.unit_gauge(dims), -0.2, dims).toarray()
    tr = np.trace(np.linalg.inv(M)).real
    assert abs(tr - exact.free_field_trace(dims, -0.2)) < 1e-9
    assert abs(tr - 745.10307568270) < 1e-8
