"""Wilson-Dirac operator in FP64 (oracle).

The paper works with the lattice Dirac operator D on a 4-D lattice with 12
degrees of freedom per site, 4 spin x 3 colour (Sec. 1), and uses only its
Gamma_5-hermiticity, (Gamma_5 D)^H = Gamma_5 D with Gamma_5 diagonal and
flipping the sign of half of the spin components (Sec. 2, 'Deflation for the
Dirac operator').  It never writes D out.  The reading taken here is the
standard Wilson discretisation

  (D psi)(x) = (4 + m0) psi(x)
               - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x)       psi(x + mu)
                            + (1 + gamma_mu) U_mu(x - mu)^H psi(x - mu) ]

in the Euclidean chiral basis
  gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]  (k = 1, 2, 3),
  gamma_4 = [[0, 1], [1, 0]],
  gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1),
periodic in space and antiperiodic in time for the fermion field.

Layouts (the canonical host layout shared with the C-ABI):
  site   s = x + Lx (y + Ly (z + Lz t)),  dims = (Lx, Ly, Lz, Lt)
  spinor index (s * 4 + spin) * 3 + colour
  link   U[s][mu][a][b], mu = 0..3 = x, y, z, t; U_mu(x) maps colour at x+mu
         to colour at x.
"""
import numpy as np
import scipy.sparse as sp

SIGMA = (
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
)


def gamma_matrices():
    """gamma_1..gamma_4 and gamma_5 in the chiral basis stated above."""
    z = np.zeros((2, 2), dtype=np.complex128)
    e = np.eye(2, dtype=np.complex128)
    g = []
    for k in range(3):
        g.append(np.block([[z, -1j * SIGMA[k]], [1j * SIGMA[k], z]]))
    g.append(np.block([[z, e], [e, z]]))
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return g, g5


GAMMA, GAMMA5 = gamma_matrices()


def volume(dims):
    return int(dims[0] * dims[1] * dims[2] * dims[3])


def _axis(mu):
    # numpy field shape is (Lt, Lz, Ly, Lx, ...): direction mu lives on axis 3-mu
    return 3 - mu


def _field(v, dims, inner):
    return np.asarray(v).reshape((dims[3], dims[2], dims[1], dims[0]) + inner)


def shift_forward(f, mu, antiperiodic_t=True):
    """g(x) = f(x + mu_hat), with the fermion time-boundary sign."""
    g = np.roll(f, -1, axis=_axis(mu))
    if mu == 3 and antiperiodic_t:
        g[-1] = -g[-1]  # sites at t = Lt-1 received f(t = 0) across the boundary
    return g


def shift_backward(f, mu, antiperiodic_t=True):
    """g(x) = f(x - mu_hat), with the fermion time-boundary sign."""
    g = np.roll(f, 1, axis=_axis(mu))
    if mu == 3 and antiperiodic_t:
        g[0] = -g[0]
    return g


def apply_wilson(U, psi, m0, dims):
    """y = D psi, matrix-free, straight from the formula in the module docstring."""
    psi_f = _field(psi, dims, (4, 3))
    U_f = _field(U, dims, (4, 3, 3))
    out = (4.0 + m0) * psi_f
    for mu in range(4):
        Umu = U_f[..., mu, :, :]
        # forward hop: (1 - gamma_mu) U_mu(x) psi(x + mu)
        a = np.einsum('...ab,...sb->...sa', Umu, shift_forward(psi_f, mu))
        a = a - np.einsum('st,...tb->...sb', GAMMA[mu], a)
        # backward hop: (1 + gamma_mu) U_mu(x - mu)^H psi(x - mu)
        Ub = np.roll(Umu, 1, axis=_axis(mu))
        b = np.einsum('...ba,...sb->...sa', Ub.conj(), shift_backward(psi_f, mu))
        b = b + np.einsum('st,...tb->...sb', GAMMA[mu], b)
        out = out - 0.5 * (a + b)
    return out.reshape(-1)


def apply_gamma5(psi, dof=12):
    """Gamma_5 on a fine vector: +1 on spins 0,1 and -1 on spins 2,3."""
    f = np.asarray(psi).reshape(-1, dof).copy()
    f[:, dof // 2:] *= -1
    return f.reshape(-1)


def gauge_transform_links(U, g, dims):
    """U^g_mu(x) = g(x) U_mu(x) g(x + mu)^H (links are periodic)."""
    U_f = _field(U, dims, (4, 3, 3))
    g_f = _field(g, dims, (3, 3))
    out = np.empty_like(U_f)
    for mu in range(4):
        gn = np.roll(g_f, -1, axis=_axis(mu))
        out[..., mu, :, :] = g_f @ U_f[..., mu, :, :] @ np.conj(np.swapaxes(gn, -1, -2))
    return out.reshape(-1)


def gauge_transform_spinor(psi, g, dims):
    """(G psi)(x) = g(x) psi(x) colour-wise at every spin."""
    f = _field(psi, dims, (4, 3))
    g_f = _field(g, dims, (3, 3))
    return np.einsum('...ab,...sb->...sa', g_f, f).reshape(-1)


# ---------------------------------------------------------------------------
# Stencil-block form: (D x)(s) = sum_d A[s, d] x(nbr(s, d)), d = 0 self,
# d = 1 + 2 mu forward (+mu), d = 2 + 2 mu backward (-mu).  Boundary signs are
# folded into the blocks so the neighbour map is plain periodic.  This is the
# same operator as apply_wilson written as 9 dense 12x12 blocks per site; the
# Galerkin coarse operators of every level use the same form.
# ---------------------------------------------------------------------------

def neighbor_table(dims):
    """nbr[s, d] for d = 0..8 on a periodic lattice of extents dims."""
    Lx, Ly, Lz, Lt = dims
    V = volume(dims)
    s = np.arange(V)
    c = [s % Lx, (s // Lx) % Ly, (s // (Lx * Ly)) % Lz, s // (Lx * Ly * Lz)]
    L = dims

    def idx(cc):
        return cc[0] + L[0] * (cc[1] + L[1] * (cc[2] + L[2] * cc[3]))

    nbr = np.empty((V, 9), dtype=np.int64)
    nbr[:, 0] = s
    for mu in range(4):
        f = list(c)
        f[mu] = (c[mu] + 1) % L[mu]
        b = list(c)
        b[mu] = (c[mu] - 1) % L[mu]
        nbr[:, 1 + 2 * mu] = idx(f)
        nbr[:, 2 + 2 * mu] = idx(b)
    return nbr


def site_coords(dims):
    Lx, Ly, Lz, Lt = dims
    s = np.arange(volume(dims))
    return np.stack([s % Lx, (s // Lx) % Ly, (s // (Lx * Ly)) % Lz, s // (Lx * Ly * Lz)], axis=1)


def wilson_stencil(U, m0, dims):
    """A[s, d] (12 x 12) for the Wilson operator; dof = spin * 3 + colour."""
    V = volume(dims)
    U = np.asarray(U).reshape(V, 4, 3, 3)
    nbr = neighbor_table(dims)
    t = site_coords(dims)[:, 3]
    Lt = dims[3]
    A = np.zeros((V, 9, 12, 12), dtype=np.complex128)
    A[:, 0] = (4.0 + m0) * np.eye(12)
    one = np.eye(4, dtype=np.complex128)
    for mu in range(4):
        pm = one - GAMMA[mu]
        pp = one + GAMMA[mu]
        sgn_f = np.ones(V)
        sgn_b = np.ones(V)
        if mu == 3:
            sgn_f[t == Lt - 1] = -1.0
            sgn_b[t == 0] = -1.0
        Uf = U[:, mu]
        Ub = np.conj(np.swapaxes(U[nbr[:, 2 + 2 * mu], mu], -1, -2))
        A[:, 1 + 2 * mu] = -0.5 * sgn_f[:, None, None] * np.einsum('st,vab->vsatb', pm, Uf).reshape(V, 12, 12)
        A[:, 2 + 2 * mu] = -0.5 * sgn_b[:, None, None] * np.einsum('st,vab->vsatb', pp, Ub).reshape(V, 12, 12)
    return A


def apply_stencil(A, x, dims):
    """y(s) = sum_d A[s, d] x(nbr(s, d))."""
    V, nd, dof, _ = A.shape
    xs = np.asarray(x).reshape(V, dof)
    nbr = neighbor_table(dims)
    y = np.zeros((V, dof), dtype=np.complex128)
    for d in range(nd):
        y += np.einsum('vij,vj->vi', A[:, d], xs[nbr[:, d]])
    return y.reshape(-1)


def stencil_matrix(A, dims, hop_filter=None):
    """Sparse matrix of the stencil; hop_filter(d) -> bool mask over sites
    selects which (site, direction) blocks are kept (all when None)."""
    V, nd, dof, _ = A.shape
    nbr = neighbor_table(dims)
    rows, cols, vals = [], [], []
    ii, jj = np.meshgrid(np.arange(dof), np.arange(dof), indexing='ij')
    for d in range(nd):
        keep = np.ones(V, dtype=bool) if hop_filter is None else hop_filter(d)
        s = np.nonzero(keep)[0]
        if s.size == 0:
            continue
        r = (s[:, None, None] * dof + ii[None]).reshape(-1)
        c = (nbr[s, d][:, None, None] * dof + jj[None]).reshape(-1)
        rows.append(r)
        cols.append(c)
        vals.append(A[s, d].reshape(-1))
    n = V * dof
    if not vals:
        return sp.csr_matrix((n, n), dtype=np.complex128)
    M = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return M.tocsr()


def wilson_matrix(U, m0, dims):
    return stencil_matrix(wilson_stencil(U, m0, dims), dims)
