"""Stochastic trace estimators of the paper, step by step (oracle).

* Hutchinson (Sec. 1, Eq. Hutchinson): tr(A) ~ (1/N) sum_k x_k^H A x_k.
* Sample variance (Sec. 4): V = 1/(N-1) sum_i |X_i - mean|^2 (complex X).
* MLMC allocation (Sec. 2.2, Eq. MLMC-Nl; the inner sum index is N_l):
  N_l = eps^-2 sqrt(V_l / C_l) sum_i sqrt(V_i C_i); total cost
  (sum_l sqrt(V_l C_l))^2 / eps^2.
* Orthogonal multigrid MLMC (Sec. 3, Eq. OandF_def and
  Eq. smultigrid-multilevel-monte-carlo):
     tr(D^-1) = sum_{l<L} tr(O_l) + sum_{l<L} tr(F_l) + tr(D_L^-1),
     O_l = (I - P_l P_l^H) D_l^-1 (I - P_l P_l^H),
     F_l = P_l^H D_l^-1 P_l - D_{l+1}^-1.
  O_l sample (Sec. 3): y = (I - P P^H) x, solve D_l z = y, X = y^H z.
  F_l sample: x on level l+1, X = (P x)^H D_l^-1 (P x) - x^H D_{l+1}^-1 x.
* Oblique multigrid MLMC (Sec. 2.2, Eq. oblique-deflation and
  Eq. oblique_multigrid-multilevel-monte-carlo):
     tr(D^-1) = sum_{l<L} tr(M_l) + tr(D_L^-1),
     M_l = D_l^-1 - P_l D_{l+1}^-1 R_l = (I - Pi_l) D_l^-1, R_l = P_l^H,
     Pi_l = P_l D_{l+1}^-1 R_l D_l (an oblique projection by Galerkin).
  M_l sample: x on level l, X = x^H D_l^-1 x - (R_l x)^H D_{l+1}^-1 (R_l x).
* Connected correlator (Sec. 1.1, Eq. connected-G; Sec. 4.1, Eq.
  full_ops_orth and Eq. G-split), orthogonal split with
     J_l = (I - P_l P_l^H) D_l^-1,
     K_l = P_l P_l^H D_l^-1 - P_l D_{l+1}^-1 P_l^H,
     B_l = Phat_{l-1} J_l Phat_{l-1}^H,  B_{L-1+l} = Phat_{l-1} K_l Phat_{l-1}^H,
     B_{2L-1} = Phat_{L-1} D_L^-1 Phat_{L-1}^H,
  G_rs(t) = (1/T) sum_t' tr(B_r(t+t',t') Gamma5 B_s(t',t+t') Gamma5).
  Readings: the accumulated prolongation attached to a level-l operator is
  Phat_{l-1} (Phat_0 = I; the printed subscripts do not match the operator
  dimensions), the last term of the split of D_l^-1 is P_l D_{l+1}^-1 P_l^H,
  and the trace is sampled with Z4 noise x on source slice t' through
  Gamma5 B_s(t',t+t') Gamma5 = [Btil_s(t+t',t')]^H, Btil = Gamma5 B^H Gamma5:
     X_rs(t) = (1/T) sum_t' (Btil_s x)|_{t+t'}^H (B_r x)|_{t+t'}.
  The oracle applies Btil literally (solves with D_l^H).
  Oblique split (Eq. G-traditional, same reading of Phat):
     B_l = Phat_{l-1} (D_l^-1 - P_l D_{l+1}^-1 P_l^H) Phat_{l-1}^H, l < L,
     B_L = Phat_{L-1} D_L^-1 Phat_{L-1}^H.
* Disconnected loop (Sec. 4.3, Eq. trace_equality_disconnected):
  tr(Gamma5 D^-1(t,t)) = sum_r tr(Gamma5 B_r(t,t)); sample X_r = x^H Gamma5 B_r x
  with x on slice t.
"""
import numpy as np

from . import noise as nz
from .dirac import apply_gamma5


def sample_stats(X):
    """mean and the unbiased complex sample variance of Sec. 4."""
    X = np.asarray(X, dtype=np.complex128)
    N = X.size
    mu = X.mean()
    var = np.sum(np.abs(X - mu) ** 2) / (N - 1) if N > 1 else np.nan
    return mu, var


def mlmc_allocation(V, C, eps):
    """N_l (real-valued, before rounding) and the minimum total cost."""
    V = np.asarray(V, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    S = np.sum(np.sqrt(V * C))
    N = S * np.sqrt(V / C) / eps ** 2
    return N, S ** 2 / eps ** 2


class Estimators:
    """Per-sample values of every estimator on a Hierarchy with exact level
    solvers solvers[l] (LevelSolver)."""

    def __init__(self, hier, solvers, seed):
        self.h = hier
        self.sol = solvers
        self.seed = seed

    # --- tr(D^-1) ---------------------------------------------------------
    def plain(self, k):
        x = nz.z4_vector(self.h.size(0), self.seed, k, nz.TERM_PLAIN)
        return np.vdot(x, self.sol[0](x))

    def O(self, l, k):
        x = nz.z4_vector(self.h.size(l), self.seed, k, nz.TERM_O + l)
        y = self.h.P[l].project_out(x)
        z = self.sol[l](y)
        return np.vdot(y, z)

    def F(self, l, k):
        x = nz.z4_vector(self.h.size(l + 1), self.seed, k, nz.TERM_F + l)
        y = self.h.P[l].prolong(x)
        z1 = self.sol[l](y)
        z2 = self.sol[l + 1](x)
        return np.vdot(y, z1) - np.vdot(x, z2)

    def M(self, l, k):
        x = nz.z4_vector(self.h.size(l), self.seed, k, nz.TERM_M + l)
        z1 = self.sol[l](x)
        xc = self.h.P[l].restrict(x)
        z2 = self.sol[l + 1](xc)
        return np.vdot(x, z1) - np.vdot(xc, z2)

    def coarsest(self, k):
        L = self.h.n_levels - 1
        x = nz.z4_vector(self.h.size(L), self.seed, k, nz.TERM_COARSEST)
        return np.vdot(x, self.sol[L](x))

    def orthogonal_terms(self):
        """[(name, sampler)] in the order O_0..O_{L-2}, F_0..F_{L-2}, coarsest."""
        L = self.h.n_levels
        out = [('O%d' % l, lambda k, l=l: self.O(l, k)) for l in range(L - 1)]
        out += [('F%d' % l, lambda k, l=l: self.F(l, k)) for l in range(L - 1)]
        out.append(('coarsest', self.coarsest))
        return out

    def oblique_terms(self):
        """[(name, sampler)] in the order M_0..M_{L-2}, coarsest."""
        L = self.h.n_levels
        out = [('M%d' % l, lambda k, l=l: self.M(l, k)) for l in range(L - 1)]
        out.append(('coarsest', self.coarsest))
        return out

    # --- correlator / loop operators ---------------------------------------
    def _gamma5_level(self, v, l):
        return apply_gamma5(v, self.h.A[l].shape[2])

    def B_apply(self, x):
        """[B_r x] (fine vectors), r in the order J_0..J_{L-2}, K_0..K_{L-2},
        coarsest (0-based levels)."""
        h, sol = self.h, self.sol
        L = h.n_levels
        J, K = [], []
        for l in range(L - 1):
            u = h.restrict_from_fine(x, l)
            P = h.P[l]
            Du = sol[l](u)
            J.append(h.prolong_to_fine(P.project_out(Du), l))
            Kl = P.prolong(P.restrict(Du)) - P.prolong(sol[l + 1](P.restrict(u)))
            K.append(h.prolong_to_fine(Kl, l))
        uL = h.restrict_from_fine(x, L - 1)
        last = h.prolong_to_fine(sol[L - 1](uL), L - 1)
        return J + K + [last]

    def Btilde_apply(self, x):
        """[Gamma5 B_r^H Gamma5 x], literally, with D_l^{-H} solves."""
        h, sol = self.h, self.sol
        L = h.n_levels
        g5x = apply_gamma5(x)
        J, K = [], []
        for l in range(L - 1):
            P = h.P[l]
            u = h.restrict_from_fine(g5x, l)
            # J^H = D_l^{-H} (I - P P^H)
            Jh = sol[l].solve_adjoint(P.project_out(u))
            # K^H = D_l^{-H} P P^H - P D_{l+1}^{-H} P^H
            Kh = sol[l].solve_adjoint(P.prolong(P.restrict(u))) \
                - P.prolong(sol[l + 1].solve_adjoint(P.restrict(u)))
            J.append(apply_gamma5(h.prolong_to_fine(Jh, l)))
            K.append(apply_gamma5(h.prolong_to_fine(Kh, l)))
        uL = h.restrict_from_fine(g5x, L - 1)
        last = apply_gamma5(h.prolong_to_fine(sol[L - 1].solve_adjoint(uL), L - 1))
        return J + K + [last]

    def B_apply_oblique(self, x):
        """[B_l x] of the oblique split: M_l = D_l^-1 - P_l D_{l+1}^-1 P_l^H
        between Phat_{l-1}^H and Phat_{l-1}, then the coarsest."""
        h, sol = self.h, self.sol
        L = h.n_levels
        out = []
        for l in range(L - 1):
            u = h.restrict_from_fine(x, l)
            P = h.P[l]
            Ml = sol[l](u) - P.prolong(sol[l + 1](P.restrict(u)))
            out.append(h.prolong_to_fine(Ml, l))
        uL = h.restrict_from_fine(x, L - 1)
        return out + [h.prolong_to_fine(sol[L - 1](uL), L - 1)]

    def Btilde_apply_oblique(self, x):
        """[Gamma5 B_l^H Gamma5 x] of the oblique split, literally (D^{-H})."""
        h, sol = self.h, self.sol
        L = h.n_levels
        g5x = apply_gamma5(x)
        out = []
        for l in range(L - 1):
            P = h.P[l]
            u = h.restrict_from_fine(g5x, l)
            Mh = sol[l].solve_adjoint(u) - P.prolong(sol[l + 1].solve_adjoint(P.restrict(u)))
            out.append(apply_gamma5(h.prolong_to_fine(Mh, l)))
        uL = h.restrict_from_fine(g5x, L - 1)
        return out + [apply_gamma5(h.prolong_to_fine(sol[L - 1].solve_adjoint(uL), L - 1))]

    def _ops(self, kind):
        if kind == 'oblique':
            return self.B_apply_oblique, self.Btilde_apply_oblique, self.h.n_levels
        return self.B_apply, self.Btilde_apply, 2 * (self.h.n_levels - 1) + 1

    def _slice_dots(self, a, b):
        """per time slice sum of conj(a) b over a fine vector."""
        dims = self.h.dims[0]
        T = dims[3]
        return np.einsum('ti,ti->t', np.conj(a.reshape(T, -1)), b.reshape(T, -1))

    def connected(self, k, sources=None, kind='orthogonal'):
        """X_rs(t) for sample k (array (R, R, T)), averaging over the source
        slices t' (all T when sources is None); kind 'orthogonal' (R = 2L-1)
        or 'oblique' (R = L)."""
        dims = self.h.dims[0]
        T = dims[3]
        src = range(T) if sources is None else sources
        Bop, Btop, R = self._ops(kind)
        X = np.zeros((R, R, T), dtype=np.complex128)
        for tp in src:
            x = nz.z4_slice_vector(dims, 12, tp, self.seed, k, nz.TERM_CONNECTED, aux=tp)
            b = Bop(x)
            bt = Btop(x)
            for r in range(R):
                for s in range(R):
                    d = self._slice_dots(bt[s], b[r])  # index: absolute slice
                    X[r, s] += np.roll(d, -tp)          # -> separation t
        return X / len(src)

    def connected_plain(self, k, sources=None):
        dims = self.h.dims[0]
        T = dims[3]
        src = range(T) if sources is None else sources
        X = np.zeros(T, dtype=np.complex128)
        for tp in src:
            x = nz.z4_slice_vector(dims, 12, tp, self.seed, k, nz.TERM_CONNECTED, aux=tp)
            z = self.sol[0](x)
            zt = apply_gamma5(self.sol[0].solve_adjoint(apply_gamma5(x)))
            X += np.roll(self._slice_dots(zt, z), -tp)
        return X / len(src)

    def disconnected(self, k, t, kind='orthogonal'):
        """X_r = x^H Gamma5 B_r x, x on slice t, for every r (array (R,))."""
        dims = self.h.dims[0]
        x = nz.z4_slice_vector(dims, 12, t, self.seed, k, nz.TERM_DISCONNECTED, aux=t)
        b = self._ops(kind)[0](x)
        return np.array([np.vdot(x, apply_gamma5(br)) for br in b])

    def disconnected_plain(self, k, t):
        dims = self.h.dims[0]
        x = nz.z4_slice_vector(dims, 12, t, self.seed, k, nz.TERM_DISCONNECTED, aux=t)
        return np.vdot(x, apply_gamma5(self.sol[0](x)))
