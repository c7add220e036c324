"""Pins of the oracle's smoothers against facts independent of their code:
the one-step MR closed form and its optimality, and SAP with exact block
solves (many MR steps) against multiplicative Schwarz written with direct
block solves."""
import numpy as np

from oracle import dirac, smoother
from paper_2509_11424_gb300 import synth


def test_mr_one_step_closed_form_and_optimal():
    dims = (4, 2, 2, 4)
    M = dirac.wilson_matrix(synth.gauge_field(dims, 0.4, 3), 0.2, dims)
    b = synth.complex_normal(M.shape[0], 4)
    z = smoother.mr_smooth(M, b, 1)
    Db = M @ b
    al = np.vdot(Db, b) / np.vdot(Db, Db)
    assert np.allclose(z, al * b, atol=1e-14)
    res = np.linalg.norm(b - M @ z)
    for d in (1e-3, -1e-3, 1e-3j, -1e-3j):
        assert np.linalg.norm(b - (al + d) * Db) > res
    # residual never grows over several steps
    norms = [np.linalg.norm(b - M @ smoother.mr_smooth(M, b, k)) for k in range(6)]
    assert all(norms[k + 1] <= norms[k] * (1 + 1e-12) for k in range(5))


def test_sap_exact_blocks_is_multiplicative_schwarz():
    dims, block = (4, 4, 2, 4), (2, 2, 1, 2)
    M = dirac.wilson_matrix(synth.gauge_field(dims, 0.3, 5), 0.5, dims).tocsr()
    b = synth.complex_normal(M.shape[0], 6)
    z = smoother.sap_smooth(M, dims, block, b, sweeps=1, iters=300)
    # direct restatement: colour 0 blocks solved exactly, residual updated,
    # then colour 1 blocks solved exactly
    V = dirac.volume(dims)
    c = dirac.site_coords(dims) // np.array(block)
    nb = np.array(dims) // np.array(block)
    blk = c[:, 0] + nb[0] * (c[:, 1] + nb[1] * (c[:, 2] + nb[2] * c[:, 3]))
    col = c.sum(axis=1) % 2
    zz = np.zeros_like(b)
    r = b.copy()
    for cc in (0, 1):
        for B in np.unique(blk[col == cc]):
            idx = (np.nonzero(blk == B)[0][:, None] * 12 + np.arange(12)).reshape(-1)
            zz[idx] += np.linalg.solve(M[idx][:, idx].toarray(), r[idx])
        r = b - M @ zz
    assert np.max(np.abs(z - zz)) < 1e-10 * np.max(np.abs(zz))
    # after the sweep the residual vanishes on the colour visited last
    last = np.repeat(col == 1, 12)
    assert np.max(np.abs(r[last])) < 1e-10 * np.max(np.abs(b))
