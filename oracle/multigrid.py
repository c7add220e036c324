"""Aggregation-based transfer operators and Galerkin coarse operators (oracle).

Sec. 2.2 (multigrid MLMC): R_l = P_l^H with P_l^H P_l = I, and the coarse
operators are the Galerkin products D_{l+1} = R_l D_l P_l.  Sec. 3 builds the
orthogonal projector P_l P_l^H from the same P_l.  P_l is built from N_tv test
vectors (Sec. 2.2, setup phase; Sec. 4: rough approximations to low modes).

Readings taken where the paper is silent:
* aggregates are rectangular blocks of `block` sites; each aggregate is split
  by chirality: the first half of a site's dofs (spins 0, 1 on the fine
  level; the first N_tv coarse dofs on coarser levels) is chirality +, the
  second half chirality -;
* per (aggregate, chirality) the restrictions of the N_tv test vectors are
  orthonormalised with modified Gram-Schmidt run twice, in test-vector order;
  the resulting orthonormal columns are the block of P for that pair;
* coarse dof of (aggregate X, chirality c, test vector k) is
  X * 2 N_tv + c * N_tv + k;
* the coarse operator is stored in the same 9-block stencil form as the fine
  one.  The block for direction d of coarse site X collects exactly the fine
  hops of direction d that leave aggregate X (d = 1..8), and block 0 collects
  the diagonal and every hop that stays inside X.  On a coarse lattice of
  extent 2, X + mu and X - mu coincide but their blocks stay separate.
"""
import numpy as np
import scipy.sparse as sp

from .dirac import neighbor_table, site_coords, volume, stencil_matrix


class Aggregation:
    """Block aggregation of a lattice with `dof` dofs per site into blocks of
    extent `block` (per direction), chirality-split."""

    def __init__(self, dims, block, dof):
        self.dims = tuple(int(d) for d in dims)
        self.block = tuple(int(b) for b in block)
        if any(d % b for d, b in zip(self.dims, self.block)):
            raise ValueError('block must divide the lattice')
        self.cdims = tuple(d // b for d, b in zip(self.dims, self.block))
        self.dof = int(dof)
        self.half = self.dof // 2
        V = volume(self.dims)
        c = site_coords(self.dims)
        b = self.block
        cc = c // np.array(b)
        cd = self.cdims
        self.agg = cc[:, 0] + cd[0] * (cc[:, 1] + cd[1] * (cc[:, 2] + cd[2] * cc[:, 3]))
        r = c % np.array(b)
        self.site_in_agg = r[:, 0] + b[0] * (r[:, 1] + b[1] * (r[:, 2] + b[2] * r[:, 3]))
        self.nagg = volume(self.cdims)
        self.sites_per_agg = volume(self.block)
        self.rows = self.sites_per_agg * self.half
        # fine dof index of (aggregate, chirality, row)
        idx = np.empty((self.nagg, 2, self.rows), dtype=np.int64)
        s = np.arange(V)
        for d in range(self.dof):
            ch, dd = divmod(d, self.half)
            idx[self.agg, ch, self.site_in_agg * self.half + dd] = s * self.dof + d
        self.index = idx

    def gather(self, v):
        """v (n,) or (n, k) -> (nagg, 2, rows[, k]) in aggregate order."""
        return np.asarray(v)[self.index]


def mgs_orthonormalise(Vb):
    """Modified Gram-Schmidt, two passes, in column order, on each
    (aggregate, chirality) block: Vb (nagg, 2, rows, ntv) -> Q of same shape."""
    Q = np.array(Vb, dtype=np.complex128, copy=True)
    ntv = Q.shape[-1]
    for j in range(ntv):
        w = Q[..., j].copy()
        for _ in range(2):
            for i in range(j):
                qi = Q[..., i]
                h = np.sum(np.conj(qi) * w, axis=-1)
                w = w - h[..., None] * qi
        nrm = np.sqrt(np.sum(np.abs(w) ** 2, axis=-1))
        Q[..., j] = w / nrm[..., None]
    return Q


class Prolongator:
    """P_l for one level: block-diagonal over (aggregate, chirality), each
    block the orthonormalised test vectors of that pair."""

    def __init__(self, agg: Aggregation, test_vectors):
        tv = np.asarray(test_vectors, dtype=np.complex128)
        self.agg = agg
        self.ntv = tv.shape[1]
        self.Q = mgs_orthonormalise(agg.gather(tv))  # (nagg, 2, rows, ntv)
        self.n_fine = volume(agg.dims) * agg.dof
        self.n_coarse = agg.nagg * 2 * self.ntv
        self.coarse_dof = 2 * self.ntv

    def restrict(self, x):
        """x_c = P^H x, coarse layout (X, c, k)."""
        xb = self.agg.gather(x)  # (nagg, 2, rows)
        return np.einsum('acrk,acr->ack', np.conj(self.Q), xb).reshape(-1)

    def prolong(self, xc):
        """x = P x_c."""
        xc = np.asarray(xc).reshape(self.agg.nagg, 2, self.ntv)
        yb = np.einsum('acrk,ack->acr', self.Q, xc)
        y = np.zeros(self.n_fine, dtype=np.complex128)
        y[self.agg.index.reshape(-1)] = yb.reshape(-1)
        return y

    def project_out(self, x):
        """(I - P P^H) x (Sec. 3, two-sided projection)."""
        return np.asarray(x) - self.prolong(self.restrict(x))

    def matrix(self):
        """P as a sparse n_fine x n_coarse matrix."""
        a = self.agg
        rows = np.broadcast_to(a.index[..., None], a.index.shape + (self.ntv,))
        cols = (np.arange(a.nagg)[:, None, None, None] * 2 * self.ntv
                + np.arange(2)[None, :, None, None] * self.ntv
                + np.arange(self.ntv)[None, None, None, :])
        cols = np.broadcast_to(cols, rows.shape)
        return sp.csr_matrix((self.Q.reshape(-1), (rows.reshape(-1), cols.reshape(-1))),
                             shape=(self.n_fine, self.n_coarse))


def hop_class(agg: Aggregation):
    """cls[s, d]: 0 if the hop (s, d) stays in the aggregate of s (always for
    d = 0), else d."""
    nbr = neighbor_table(agg.dims)
    same = agg.agg[nbr] == agg.agg[:, None]
    cls = np.where(same, 0, np.arange(9)[None, :])
    return cls


def galerkin(A, prol: Prolongator):
    """Coarse stencil blocks Ac[X, d] (2 N_tv square) of D_{l+1} = P^H D_l P,
    split by hop direction as described in the module docstring."""
    agg = prol.agg
    dims = agg.dims
    cls = hop_class(agg)
    Pm = prol.matrix()
    PH = Pm.conj().T.tocsr()
    cn = neighbor_table(agg.cdims)
    nc = agg.nagg
    m = prol.coarse_dof
    Ac = np.zeros((nc, 9, m, m), dtype=np.complex128)
    for h in range(9):
        Dh = stencil_matrix(A, dims, hop_filter=lambda d, h=h: cls[:, d] == h)
        C = (PH @ (Dh @ Pm)).tocsr()
        for X in range(nc):
            Y = cn[X, h]
            Ac[X, h] = C[X * m:(X + 1) * m, Y * m:(Y + 1) * m].toarray()
    return Ac


class Hierarchy:
    """Operators of all levels: A[l] (stencil blocks of D_l), dims[l], and
    prolongators P[l] between level l and l+1 (0-based levels)."""

    def __init__(self, A_fine, dims, blocks, test_vectors):
        self.A = [np.asarray(A_fine)]
        self.dims = [tuple(dims)]
        self.P = []
        for l, (blk, tv) in enumerate(zip(blocks, test_vectors)):
            dof = self.A[l].shape[2]
            agg = Aggregation(self.dims[l], blk, dof)
            prol = Prolongator(agg, tv)
            self.P.append(prol)
            self.A.append(galerkin(self.A[l], prol))
            self.dims.append(agg.cdims)

    @property
    def n_levels(self):
        return len(self.A)

    def size(self, l):
        return volume(self.dims[l]) * self.A[l].shape[2]

    def matrix(self, l):
        return stencil_matrix(self.A[l], self.dims[l])

    def prolong_to_fine(self, v, l):
        """P_hat_{l} v: level l -> level 0 (P_1 ... P_l in the paper's 1-based
        notation)."""
        for k in range(l - 1, -1, -1):
            v = self.P[k].prolong(v)
        return v

    def restrict_from_fine(self, v, l):
        for k in range(l):
            v = self.P[k].restrict(v)
        return v
