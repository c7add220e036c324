"""Smoothers of the multigrid level solves (oracle).

The paper solves every level with DD-alpha-AMG (Sec. 4), whose smoother is
the Schwarz alternating procedure (SAP); the paper states no details and the
smoother only changes how fast a solve reaches its tolerance, never what it
returns.  The oracle restates the two smoothers the library uses, so that the
CUDA smoothers can be checked step by step:

* minimal residual (MR), `steps` steps from z = 0 on D z = b:
    q = D r,  alpha = <q, r> / <q, q>,  z += alpha r,  r -= alpha q;
* SAP: the lattice is cut into blocks of extent `block` (an even number in
  every direction), coloured by the parity of the block coordinates; a sweep
  visits colour 0 then colour 1; every block B of the active colour runs
  `iters` MR steps on D_BB e = r_B with D_BB the block of D restricted to
  the sites of B (hops leaving B dropped), then z_B += e; after each colour
  the residual r = b - D z is recomputed from its definition.
An MR step whose <q, q> has underflowed (below 1e-280) takes alpha = 0.
"""
import numpy as np

from .dirac import site_coords, volume


def mr_smooth(M, b, steps):
    z = np.zeros_like(b)
    r = np.array(b, dtype=np.complex128)
    for _ in range(steps):
        q = M @ r
        qq = np.vdot(q, q).real
        al = np.vdot(q, r) / qq if qq > 1e-280 else 0.0
        z = z + al * r
        r = r - al * q
    return z


def sap_smooth(M, dims, block, b, sweeps, iters, dof=12):
    V = volume(dims)
    c = site_coords(dims)
    bc = c // np.array(block)
    nb = np.array(dims) // np.array(block)
    assert np.all(nb % 2 == 0), 'SAP needs an even number of blocks per direction'
    blk = bc[:, 0] + nb[0] * (bc[:, 1] + nb[1] * (bc[:, 2] + nb[2] * bc[:, 3]))
    color = bc.sum(axis=1) % 2
    Mc = M.tocsr()
    z = np.zeros(V * dof, dtype=np.complex128)
    r = np.array(b, dtype=np.complex128)
    for _ in range(sweeps):
        for col in (0, 1):
            for B in np.unique(blk[color == col]):
                sites = np.nonzero(blk == B)[0]
                idx = (sites[:, None] * dof + np.arange(dof)[None, :]).reshape(-1)
                DBB = Mc[idx][:, idx].toarray()
                rho = r[idx].copy()
                e = np.zeros_like(rho)
                for _ in range(iters):
                    q = DBB @ rho
                    qq = np.vdot(q, q).real
                    al = np.vdot(q, rho) / qq if qq > 1e-280 else 0.0
                    e = e + al * rho
                    rho = rho - al * q
                z[idx] += e
            r = b - Mc @ z
    return z
