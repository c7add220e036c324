"""Pins of the oracle's counter-based gauge field (oracle/gauge.py) against
what the mathematics fixes, independent of the oracle's own code paths:
SU(3) membership, the exponential against an eigen-decomposition formula,
the uniform map's end points, Gaussian statistics of the Box-Muller draws,
the second moments of H, eps = 0 and the first-order expansion."""
import numpy as np
import pytest

from oracle import gauge

scipy_stats = pytest.importorskip('scipy.stats')


def test_links_are_su3():
    U = gauge.links(np.arange(512), 0.7, 11)
    I = np.eye(3)
    assert np.max(np.abs(U @ np.conj(np.swapaxes(U, -1, -2)) - I)) < 1e-13
    assert np.max(np.abs(np.linalg.det(U) - 1.0)) < 1e-13


def test_exponential_equals_eigen_form():
    L = np.arange(64)
    eps = 0.9
    H = gauge.traceless_hermitian(gauge.normal_matrices(L, 5))
    w, Q = np.linalg.eigh(H)
    want = (Q * np.exp(1j * eps * w)[:, None, :]) @ np.conj(np.swapaxes(Q, -1, -2))
    assert np.max(np.abs(gauge.links(L, eps, 5) - want)) < 1e-13


def test_uniform_map_end_points():
    w = np.array([0, 2 ** 64 - 1, 2 ** 63], dtype=np.uint64)
    u = gauge.uniforms(w)
    assert u[0] == 2.0 ** -53
    assert u[1] == 1.0 - 2.0 ** -53
    assert u[2] == 0.5 + 2.0 ** -53
    assert np.all((u > 0) & (u < 1))


def test_box_muller_draws_are_standard_complex_normal():
    A = gauge.normal_matrices(np.arange(1 << 14), 123).reshape(-1)  # 147456 values
    n = A.size
    re, im = A.real * np.sqrt(2.0), A.imag * np.sqrt(2.0)   # each should be N(0, 1)
    for x in (re, im):
        assert abs(x.mean()) < 5.0 / np.sqrt(n)
        assert abs(x.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
        kurt = np.mean(x ** 4) / np.mean(x ** 2) ** 2
        assert abs(kurt - 3.0) < 0.05
        assert scipy_stats.kstest(x, 'norm').pvalue > 1e-3
    assert abs(np.mean(re * im)) < 5.0 / np.sqrt(n)
    assert abs(np.mean(np.abs(A) ** 2) - 1.0) < 0.02


def test_hermitian_part_second_moments():
    H = gauge.traceless_hermitian(gauge.normal_matrices(np.arange(1 << 14), 9))
    assert np.max(np.abs(H - np.conj(np.swapaxes(H, -1, -2)))) == 0.0
    assert np.max(np.abs(np.trace(H, axis1=1, axis2=2))) < 1e-14
    off = np.concatenate([H[:, 0, 1], H[:, 0, 2], H[:, 1, 2]])
    # H_ab = (A_ab + conj A_ba)/2 with E|A|^2 = 1: E|H_ab|^2 = 1/2
    assert abs(np.mean(np.abs(off) ** 2) - 0.5) < 0.02
    # H_aa = Re A_aa - mean of the three: variance (1/2)(1 - 1/3) = 1/3
    diag = np.concatenate([H[:, a, a].real for a in range(3)])
    assert abs(np.var(diag) - 1.0 / 3.0) < 0.02


def test_free_field_and_first_order():
    L = np.arange(32)
    assert np.max(np.abs(gauge.links(L, 0.0, 3) - np.eye(3))) == 0.0
    eps = 1e-6
    H = gauge.traceless_hermitian(gauge.normal_matrices(L, 3))
    U = gauge.links(L, eps, 3)
    assert np.max(np.abs(U - (np.eye(3) + 1j * eps * H))) < 10 * eps ** 2


def test_reproducible_and_seed_dependent():
    a = gauge.gauge_field((2, 2, 2, 2), 0.5, 1)
    assert np.array_equal(a, gauge.gauge_field((2, 2, 2, 2), 0.5, 1))
    assert np.max(np.abs(a - gauge.gauge_field((2, 2, 2, 2), 0.5, 2))) > 0.1
    # a link depends on its own index only
    L = np.arange(4 * 16)
    assert np.array_equal(gauge.links(L[5:6], 0.5, 1)[0], a.reshape(-1, 3, 3)[5])
