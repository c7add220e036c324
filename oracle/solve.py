"""Level solves for the oracle.

Sec. 4 solves every level system D_l z = y to a relative residual of 1e-12
(with DD-alpha-AMG).  What such a solve returns is D_l^{-1} y up to that
tolerance, so the oracle takes the plain definition: a sparse direct LU
factorisation (SuperLU via scipy) for the small lattices the parity tests use,
and, for lattices too large to factor, scipy's restarted GMRES(64) driven to
the same relative residual (BiCGStab stagnates on the indefinite Wilson
operators near the most ill-conditioned masses, GMRES does not).  Solves with
D_l^H use the same factorisation transposed, or GMRES on D_l^H.
"""
import numpy as np
import scipy.sparse.linalg as spla

LU_MAX_N = 40000


class LevelSolver:
    def __init__(self, M, tol=1e-12, maxiter=400, restart=64):
        self.M = M.tocsc()
        self.n = M.shape[0]
        self.tol = tol
        self.maxiter = maxiter
        self.restart = restart
        self.lu = spla.splu(self.M) if self.n <= LU_MAX_N else None
        self.last_iters = 0

    def _iterative(self, M, b):
        it = [0]

        def cb(_):
            it[0] += 1

        x, info = spla.gmres(M, b, rtol=self.tol, atol=0.0, restart=self.restart,
                             maxiter=self.maxiter, callback=cb, callback_type='pr_norm')
        self.last_iters = it[0]
        if info != 0:
            raise RuntimeError('oracle GMRES did not converge (info=%d)' % info)
        return x

    def solve(self, b):
        """z = D^{-1} b."""
        b = np.asarray(b, dtype=np.complex128)
        if self.lu is not None:
            return self.lu.solve(b)
        return self._iterative(self.M.tocsr(), b)

    def solve_adjoint(self, b):
        """z = D^{-H} b."""
        b = np.asarray(b, dtype=np.complex128)
        if self.lu is not None:
            return self.lu.solve(b, trans='H')
        return self._iterative(self.M.conj().T.tocsr(), b)

    def __call__(self, b):
        return self.solve(b)
