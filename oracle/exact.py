"""Exact targets that the estimators estimate (oracle).

* Dense inverses on tiny lattices give tr(D^-1) and every term of the
  orthogonal split (Sec. 3, Eq. OandF_def) exactly, plus the Z4 variance of
  each term, ||offdiag(A)||_F^2 / N (Sec. 1, Eq. variance-Frobenius-Relation;
  the printed left side says tr(D) where A is meant).
* Free field (U = 1): D is diagonal in momentum space,
     D(p) = m(p) + i sum_mu gamma_mu sin p_mu,  m(p) = m0 + sum_mu (1 - cos p_mu),
  with p_k = 2 pi n_k / L_k in space and p_4 = 2 pi (n_4 + 1/2) / T in time
  (antiperiodic), so the eigenvalues are m(p) +- i |sin p| (6-fold each) and
  tr D^-1 = sum_p 12 m(p) / (m(p)^2 + |sin p|^2).
"""
import numpy as np

from .dirac import GAMMA, GAMMA5, volume


def momenta(dims):
    Lx, Ly, Lz, Lt = dims
    px = 2 * np.pi * np.arange(Lx) / Lx
    py = 2 * np.pi * np.arange(Ly) / Ly
    pz = 2 * np.pi * np.arange(Lz) / Lz
    pt = 2 * np.pi * (np.arange(Lt) + 0.5) / Lt
    return np.meshgrid(px, py, pz, pt, indexing='ij')


def free_field_eigenvalues(dims, m0):
    """All 12 V eigenvalues of the free Wilson operator."""
    p = momenta(dims)
    m = m0 + sum(1 - np.cos(q) for q in p)
    s = np.sqrt(sum(np.sin(q) ** 2 for q in p))
    lam = np.concatenate([(m + 1j * s).ravel(), (m - 1j * s).ravel()])
    return np.repeat(lam, 6)


def free_field_trace(dims, m0):
    p = momenta(dims)
    m = m0 + sum(1 - np.cos(q) for q in p)
    s2 = sum(np.sin(q) ** 2 for q in p)
    return float(np.sum(12 * m / (m ** 2 + s2)))


def free_field_plane_wave(dims, m0, n, chi):
    """(psi, D psi) for psi(x) = exp(i p.x) chi (chi: 4x3 spin-colour), with
    D psi from the momentum-space form; n: integer momentum labels."""
    Lx, Ly, Lz, Lt = dims
    p = np.array([2 * np.pi * n[0] / Lx, 2 * np.pi * n[1] / Ly,
                  2 * np.pi * n[2] / Lz, 2 * np.pi * (n[3] + 0.5) / Lt])
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing='ij')
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    Dp = (m0 + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(GAMMA[mu] * np.sin(p[mu]) for mu in range(4))
    psi = phase[..., None, None] * chi[None, None, None, None]
    Dchi = Dp @ chi
    return psi.reshape(-1), (phase[..., None, None] * Dchi[None, None, None, None]).reshape(-1)


def free_field_correlator(dims, m0):
    """G(t) of Eq. connected-G for U = 1 from momentum sums:
    G(t) = (3 / T^2) sum_{pvec} || S(pvec, t) ||_F^2,
    S(pvec, t) = sum_{p4} exp(i p4 t) D(pvec, p4)^-1 (4x4 spin)."""
    Lx, Ly, Lz, Lt = dims
    px = 2 * np.pi * np.arange(Lx) / Lx
    py = 2 * np.pi * np.arange(Ly) / Ly
    pz = 2 * np.pi * np.arange(Lz) / Lz
    p4 = 2 * np.pi * (np.arange(Lt) + 0.5) / Lt
    G = np.zeros(Lt)
    for a in px:
        for b in py:
            for c in pz:
                Dinv = []
                for q in p4:
                    p = (a, b, c, q)
                    Dp = (m0 + sum(1 - np.cos(v) for v in p)) * np.eye(4) \
                        + 1j * sum(GAMMA[mu] * np.sin(p[mu]) for mu in range(4))
                    Dinv.append(np.linalg.inv(Dp))
                Dinv = np.array(Dinv)
                for t in range(Lt):
                    S = np.einsum('q,qij->ij', np.exp(1j * p4 * t), Dinv)
                    G[t] += np.sum(np.abs(S) ** 2)
    return 3.0 * G / Lt ** 2


def offdiag_fro2(A):
    """||offdiag(A)||_F^2 for a dense matrix."""
    A = np.asarray(A)
    return float(np.sum(np.abs(A) ** 2) - np.sum(np.abs(np.diag(A)) ** 2))


class DenseTerms:
    """Dense level operators of a Hierarchy and the exact values of the
    orthogonal split (tiny lattices only)."""

    def __init__(self, hier):
        self.h = hier
        L = hier.n_levels
        self.Dinv = [np.linalg.inv(hier.matrix(l).toarray()) for l in range(L)]
        self.P = [hier.P[l].matrix().toarray() for l in range(L - 1)]

    def O(self, l):
        P = self.P[l]
        Q = np.eye(P.shape[0]) - P @ P.conj().T
        return Q @ self.Dinv[l] @ Q

    def F(self, l):
        P = self.P[l]
        return P.conj().T @ self.Dinv[l] @ P - self.Dinv[l + 1]

    def terms(self):
        """[(name, dense matrix)] in the estimator's term order."""
        L = self.h.n_levels
        out = [('O%d' % l, self.O(l)) for l in range(L - 1)]
        out += [('F%d' % l, self.F(l)) for l in range(L - 1)]
        out.append(('coarsest', self.Dinv[L - 1]))
        return out

    def Phat(self, l):
        """accumulated prolongation level l -> level 0 (identity for l = 0)."""
        n0 = self.h.size(0)
        M = np.eye(n0, dtype=np.complex128)
        for k in range(l):
            M = M @ self.P[k]
        return M

    def B_matrices(self):
        """dense B_r (fine x fine) in the order J_0.., K_0.., coarsest."""
        L = self.h.n_levels
        J, K = [], []
        for l in range(L - 1):
            Ph = self.Phat(l)
            P = self.P[l]
            Pi = P @ P.conj().T
            Jl = (np.eye(P.shape[0]) - Pi) @ self.Dinv[l]
            Kl = Pi @ self.Dinv[l] - P @ self.Dinv[l + 1] @ P.conj().T
            J.append(Ph @ Jl @ Ph.conj().T)
            K.append(Ph @ Kl @ Ph.conj().T)
        Ph = self.Phat(L - 1)
        return J + K + [Ph @ self.Dinv[L - 1] @ Ph.conj().T]


    def B_matrices_oblique(self):
        """dense B_l of the oblique split (Sec. 4.1, Eq. G-traditional):
        Phat_{l-1} (D_l^-1 - P_l D_{l+1}^-1 P_l^H) Phat_{l-1}^H, then
        Phat_{L-1} D_L^-1 Phat_{L-1}^H."""
        L = self.h.n_levels
        out = []
        for l in range(L - 1):
            Ph = self.Phat(l)
            P = self.P[l]
            out.append(Ph @ (self.Dinv[l] - P @ self.Dinv[l + 1] @ P.conj().T) @ Ph.conj().T)
        Ph = self.Phat(L - 1)
        return out + [Ph @ self.Dinv[L - 1] @ Ph.conj().T]


def gamma5_matrix(n_sites, dof=12):
    d = np.ones(dof)
    d[dof // 2:] = -1
    return np.diag(np.tile(d, n_sites))


def correlator_exact(B, dims):
    """G_rs(t) = (1/T) sum_t' tr(B_r(t+t',t') Gamma5 B_s(t',t+t') Gamma5) for
    dense B (list), array (R, R, T); plain G(t) is the sum over r, s."""
    T = dims[3]
    n = B[0].shape[0]
    ns = n // T
    g5 = np.tile(np.array([1.0] * 6 + [-1.0] * 6), n // 12)
    R = len(B)
    G = np.zeros((R, R, T), dtype=np.complex128)

    def blk(M, a, b):
        return M[a * ns:(a + 1) * ns, b * ns:(b + 1) * ns]

    for t in range(T):
        for tp in range(T):
            a = (t + tp) % T
            for r in range(R):
                Br = blk(B[r], a, tp)
                for s in range(R):
                    Bs = g5[tp * ns:(tp + 1) * ns, None] * blk(B[s], tp, a) * g5[None, a * ns:(a + 1) * ns]
                    G[r, s, t] += np.trace(Br @ Bs)
    return G / T


def loop_exact(B, dims, t):
    """tr(Gamma5 B_r(t,t)) for dense B (list)."""
    T = dims[3]
    n = B[0].shape[0]
    ns = n // T
    g5 = np.tile(np.array([1.0] * 6 + [-1.0] * 6), ns // 12)
    return np.array([np.sum(g5 * np.diag(M)[t * ns:(t + 1) * ns]) for M in B])


__all__ = ['free_field_eigenvalues', 'free_field_trace', 'free_field_plane_wave',
           'free_field_correlator', 'offdiag_fro2', 'DenseTerms', 'correlator_exact',
           'loop_exact', 'volume', 'GAMMA5']
