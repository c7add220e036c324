"""The host Jacobi eigensolver of the test-vector refinement
(paper_2509_11424_gb300/csrc/herm_eig.h), compiled with the host compiler and
checked against what an eigen-decomposition must satisfy: A Z = Z diag(w),
Z unitary, and the eigenvalues of numpy's Hermitian solver, on random,
diagonal, degenerate, rank-deficient and 1 x 1 matrices up to m = 128."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2509_11424_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, '..', 'paper_2509_11424_gb300', 'csrc')


@pytest.fixture(scope='module')
def prog(tmp_path_factory):
    cxx = shutil.which('g++') or shutil.which('c++')
    if cxx is None:
        pytest.skip('no host C++ compiler')
    exe = str(tmp_path_factory.mktemp('heig') / 'herm_eig_check')
    subprocess.run([cxx, '-O2', '-std=c++17', '-I', CSRC, os.path.join(HERE, 'herm_eig_check.cpp'), '-o', exe],
                   check=True)
    return exe


def _run(exe, A):
    m = A.shape[0]
    txt = '%d\n' % m + '\n'.join('%.17g %.17g' % (a.real, a.imag) for a in A.reshape(-1))
    out = subprocess.run([exe], input=txt, capture_output=True, text=True, check=True).stdout.split('\n')
    sweeps = int(out[0])
    w = np.array([float(x) for x in out[1:1 + m]])
    Z = np.array([complex(*map(float, r.split())) for r in out[1 + m:1 + m + m * m]]).reshape(m, m)
    return sweeps, w, Z


def _check(exe, A):
    sweeps, w, Z = _run(exe, A)
    m = A.shape[0]
    scale = max(np.linalg.norm(A), 1e-300)
    assert sweeps >= 0
    assert np.max(np.abs(Z.conj().T @ Z - np.eye(m))) < 1e-13 * m
    assert np.max(np.abs(A @ Z - Z * w[None, :])) < 1e-13 * scale * np.sqrt(m)
    assert np.max(np.abs(np.sort(w) - np.linalg.eigvalsh(A))) < 1e-13 * scale * np.sqrt(m)


@pytest.mark.parametrize('m', [1, 2, 5, 33, 128])
def test_random_hermitian(prog, m):
    X = synth.complex_normal((m, m), m)
    _check(prog, 0.5 * (X + X.conj().T))


def test_gram_matrix_like_refinement(prog):
    """W^H W of a block whose columns differ in norm by 1e4, as the
    refinement's Gram matrices do."""
    W = synth.complex_normal((400, 24), 3) * np.logspace(0, 4, 24)[None, :]
    _check(prog, W.conj().T @ W)


def test_special_matrices(prog):
    _check(prog, np.diag([3.0, -1.0, 2.0, 2.0]).astype(complex))
    _check(prog, np.zeros((3, 3), dtype=complex))
    U, _ = np.linalg.qr(synth.complex_normal((6, 6), 8))
    _check(prog, (U * np.array([1.0, 1.0, 1.0, -2.0, -2.0, 5.0])[None, :]) @ U.conj().T)   # degenerate
    v = synth.complex_normal((7, 2), 9)
    _check(prog, v @ v.conj().T)                                                          # rank 2
