"""Pins of the oracle's noise generator, transfer operators and Galerkin
coarse operators."""
import itertools

import numpy as np
import pytest

from oracle import dirac, multigrid as mg, noise as nz
from paper_2509_11424_gb300 import synth


# ---------------------------------------------------------------- Philox / Z4
@pytest.mark.parametrize('ctr,key', [
    ((1, 0, 0, 0), (0, 0)),
    ((5, 7, 11, 13), (123456789, 987654321)),
    ((2 ** 64 - 1, 3, 2 ** 63, 1), (2 ** 64 - 5, 17)),
    ((0x243F6A8885A308D3, 0x13198A2E03707344, 0xA4093822299F31D0, 0x082EFA98EC4E6C89),
     (0x452821E638D01377, 0xBE5466CF34E90C6C)),
])
def test_philox_matches_numpy_bit_generator(ctr, key):
    """numpy's Philox bit generator is Philox4x64-10; its first block after
    setting counter c - 1 is the block of counter c."""
    c = sum(int(v) << (64 * i) for i, v in enumerate(ctr))
    cm1 = (c - 1) % (1 << 256)
    state_ctr = np.array([(cm1 >> (64 * i)) & (2 ** 64 - 1) for i in range(4)], dtype=np.uint64)
    bg = np.random.Philox(counter=state_ctr, key=np.array(key, dtype=np.uint64))
    want = bg.random_raw(4)
    got = nz.philox4x64_10(np.array(ctr, dtype=np.uint64), np.array(key, dtype=np.uint64))
    assert np.array_equal(got, want)


def test_mulhilo_against_python_ints():
    rng = np.random.default_rng(0)
    a = rng.integers(0, 2 ** 63, 200, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    b = rng.integers(0, 2 ** 63, 200, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    hi, lo = nz.mulhilo64(a, b)
    for x, y, h, l in zip(a, b, hi, lo):
        p = int(x) * int(y)
        assert int(h) == p >> 64 and int(l) == p & (2 ** 64 - 1)


def test_z4_distribution():
    x = nz.z4_vector(400000, 2024, 3, nz.TERM_PLAIN)
    assert np.allclose(np.abs(x), 1.0)
    counts = np.array([np.sum(np.isclose(x, v)) for v in nz.Z4_VALUES])
    assert counts.sum() == x.size
    chi2 = np.sum((counts - x.size / 4) ** 2 / (x.size / 4))
    assert chi2 < 16.3  # 3 dof, p = 0.001
    # E conj(x_i) x_{i+1} = 0 and neighbouring entries independent
    assert abs(np.mean(np.conj(x[:-1]) * x[1:])) < 0.01


def test_z4_streams_differ_and_repeat():
    a = nz.z4_codes(1000, 1, 0, nz.TERM_O)
    assert np.array_equal(a, nz.z4_codes(1000, 1, 0, nz.TERM_O))
    for other in [nz.z4_codes(1000, 2, 0, nz.TERM_O), nz.z4_codes(1000, 1, 1, nz.TERM_O),
                  nz.z4_codes(1000, 1, 0, nz.TERM_O + 1), nz.z4_codes(1000, 1, 0, nz.TERM_O, aux=1)]:
        assert np.mean(a == other) < 0.35


def test_z4_slice_vector_support_and_values():
    dims = (4, 2, 2, 6)
    x = nz.z4_slice_vector(dims, 12, 3, 9, 4, nz.TERM_CONNECTED, aux=3)
    full = nz.z4_vector(dirac.volume(dims) * 12, 9, 4, nz.TERM_CONNECTED, aux=3)
    per = 4 * 2 * 2 * 12
    assert np.all(x[:3 * per] == 0) and np.all(x[4 * per:] == 0)
    assert np.array_equal(x[3 * per:4 * per], full[3 * per:4 * per])


def test_z4_variance_law_exhaustive():
    """Var[x^H A x] = ||offdiag(A)||_F^2 over all 4^n Z4 vectors (Eq.
    variance-Frobenius-Relation), by enumeration, n = 5."""
    n = 5
    A = synth.complex_normal((n, n), 77)
    vals = []
    for r in itertools.product(range(4), repeat=n):
        x = nz.Z4_VALUES[list(r)]
        vals.append(np.vdot(x, A @ x))
    vals = np.array(vals)
    assert abs(vals.mean() - np.trace(A)) < 1e-12
    var = np.mean(np.abs(vals - vals.mean()) ** 2)
    off = np.sum(np.abs(A) ** 2) - np.sum(np.abs(np.diag(A)) ** 2)
    assert abs(var - off) < 1e-10


# ------------------------------------------------------------ transfer, MGS
def test_mgs_equals_qr_with_positive_diagonal():
    V = synth.complex_normal((1, 2, 40, 6), 5)
    Q = mg.mgs_orthonormalise(V)
    for c in range(2):
        q, r = np.linalg.qr(V[0, c])
        ph = np.diag(r) / np.abs(np.diag(r))
        assert np.allclose(Q[0, c], q * ph[None, :], atol=1e-13)
        assert np.allclose(Q[0, c].conj().T @ Q[0, c], np.eye(6), atol=1e-14)


def make_hier(dims, blocks, ntvs, eps=0.3, m0=-0.2, seed=100):
    U = synth.gauge_field(dims, eps, seed)
    A = dirac.wilson_stencil(U, m0, dims)
    tvs = []
    dof = 12
    cur = dims
    for l, (b, k) in enumerate(zip(blocks, ntvs)):
        n = dirac.volume(cur) * dof
        tvs.append(synth.random_test_vectors(n, k, seed + 10 + l))
        cur = tuple(c // bb for c, bb in zip(cur, b))
        dof = 2 * k
    return mg.Hierarchy(A, dims, blocks, tvs)


@pytest.mark.parametrize('dims,block,ntv', [((4, 4, 4, 4), (2, 2, 2, 2), 4),
                                            ((6, 4, 4, 8), (3, 2, 4, 2), 3)])
def test_projector_identities(dims, block, ntv):
    h = make_hier(dims, [block], [ntv])
    P = h.P[0].matrix()
    PH = P.conj().T
    assert abs(PH @ P - np.eye(P.shape[1])).max() < 1e-13
    x = synth.complex_normal(P.shape[0], 3)
    Pi = lambda v: h.P[0].prolong(h.P[0].restrict(v))
    assert np.max(np.abs(Pi(Pi(x)) - Pi(x))) < 1e-13
    y = synth.complex_normal(P.shape[0], 4)
    assert abs(np.vdot(y, Pi(x)) - np.vdot(Pi(y), x)) < 1e-12 * np.linalg.norm(x) * np.linalg.norm(y)
    # matrix form == restrict / prolong
    assert np.max(np.abs(PH @ x - h.P[0].restrict(x))) < 1e-13
    xc = synth.complex_normal(P.shape[1], 5)
    assert np.max(np.abs(P @ xc - h.P[0].prolong(xc))) < 1e-13
    # Gamma_5 P = P Gamma_5c: chirality-split aggregation
    g5 = dirac.apply_gamma5
    g5c = lambda v: dirac.apply_gamma5(v, 2 * ntv)
    assert np.max(np.abs(g5(h.P[0].prolong(xc)) - h.P[0].prolong(g5c(xc)))) < 1e-13
    # the span of P contains every test vector restricted to an aggregate block
    tv = synth.random_test_vectors(P.shape[0], ntv, 100 + 10)
    assert np.max(np.abs(Pi(tv[:, 0]) - tv[:, 0])) < 1e-12


@pytest.mark.parametrize('dims,blocks,ntvs', [
    ((4, 4, 4, 4), [(2, 2, 2, 2)], [4]),            # coarse extent 2 everywhere
    ((4, 4, 4, 4), [(4, 2, 2, 2)], [3]),            # coarse extent 1 in x
    ((4, 4, 4, 4), [(2, 2, 2, 2), (2, 2, 2, 2)], [3, 2]),
    ((6, 4, 4, 8), [(3, 2, 2, 4)], [2]),
])
def test_galerkin_equals_dense_product(dims, blocks, ntvs):
    """stencil-form D_{l+1} assembled to a matrix == P^H D_l P (Sec. 2.2)."""
    h = make_hier(dims, blocks, ntvs)
    for l in range(len(blocks)):
        D = h.matrix(l).toarray()
        P = h.P[l].matrix().toarray()
        want = P.conj().T @ D @ P
        got = h.matrix(l + 1).toarray()
        assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))
        # coarse Gamma_5c-hermiticity
        m = 2 * ntvs[l]
        g = np.diag(np.tile(np.r_[np.ones(m // 2), -np.ones(m // 2)], got.shape[0] // m))
        assert np.max(np.abs((g @ got).conj().T - g @ got)) < 1e-12 * np.max(np.abs(got))


def test_coarse_stencil_apply_matches_matrix():
    h = make_hier((4, 4, 4, 4), [(2, 2, 2, 2)], [4])
    x = synth.complex_normal(h.size(1), 9)
    y1 = dirac.apply_stencil(h.A[1], x, h.dims[1])
    y2 = h.matrix(1) @ x
    assert np.max(np.abs(y1 - y2)) < 1e-13
