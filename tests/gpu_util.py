"""Helpers shared by the GPU parity tests: device buffers through torch,
contexts of the C-ABI library, and oracle hierarchies built from the same
imported test vectors."""
import os

import numpy as np
import pytest

from oracle import dirac, multigrid as omg
from paper_2509_11424_gb300 import synth

torch = pytest.importorskip('torch')


def require_lib():
    from paper_2509_11424_gb300 import build, mgmlmc
    srcs = build.sources()
    lib = build.LIB
    if not os.path.exists(lib) or any(os.path.getmtime(s) > os.path.getmtime(lib) for s in srcs):
        build.build()
    return mgmlmc


def dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    """Relative error of a against b, element by element as well as by norm:
    the larger of ||a - b|| / ||b|| and max_i |a_i - b_i| / max_i |b_i|.  The
    second keeps one wrong entry (a boundary or tail site) from hiding in the
    norm of a large vector."""
    a, b = np.ravel(a), np.ravel(b)
    d = np.abs(a - b)
    norm = float(np.linalg.norm(d) / max(np.linalg.norm(b), 1e-300))
    elem = float(d.max(initial=0.0) / max(np.abs(b).max(initial=0.0), 1e-300))
    return max(norm, elem)


class Setup:
    """A GPU context and the matching oracle hierarchy, both built from the
    same gauge field and imported test vectors."""

    def __init__(self, dims, blocks, ntvs, eps=0.3, m0=-0.2, gseed=1001, tvseed=3001,
                 solver=None, oracle=True):
        M = require_lib()
        self.M = M
        self.dims = tuple(dims)
        self.blocks = blocks
        self.ntvs = ntvs
        self.m0 = m0
        self.U = synth.gauge_field(dims, eps, gseed)
        self.ctx = M.mgmlmc_create(dims, torch.cuda.current_stream())
        M.mgmlmc_set_gauge(self.ctx, self.U, on_device=False)
        M.mgmlmc_set_mass(self.ctx, m0)
        M.mgmlmc_set_solver(self.ctx, **(solver or {}))
        # test vectors: level l vectors have the level's length
        self.tvs = []
        cur, dof = tuple(dims), 12
        for l, (b, k) in enumerate(zip(blocks, ntvs)):
            n = int(np.prod(cur)) * dof
            tv = synth.random_test_vectors(n, k, tvseed + l)
            self.tvs.append(tv)
            M.mgmlmc_set_test_vectors(self.ctx, l, np.ascontiguousarray(tv.T), k, n, on_device=False)
            cur = tuple(c // bb for c, bb in zip(cur, b))
            dof = 2 * k
        M.mgmlmc_build_hierarchy(self.ctx, M.mg_params(blocks, ntvs, setup_rounds=0))
        self.hier = None
        if oracle:
            A = dirac.wilson_stencil(self.U, m0, dims)
            self.hier = omg.Hierarchy(A, dims, blocks, self.tvs)

    def close(self):
        if self.ctx:
            self.M.mgmlmc_destroy(self.ctx)
            self.ctx = None
