"""Choose the Wilson mass m0 of the 16^4 benchmark workload with the oracle.

The workload asks for an ill-conditioned operator (a condition number of
about 1e3).  On the synthetic field U = exp(i 0.4 H) (seed 1002) with
antiperiodic time boundary conditions the smallest singular value of D is
bounded away from zero by the lowest time momentum, so 1e3 is not reachable;
this script scans m0 on a grid and keeps the most ill-conditioned point.

For each m0: sigma_max by 30 power iterations on D^H D; sigma_min by 5 steps
of inverse iteration on D^H D, (D^H D)^-1 v = D^-1 Gamma5 D^-1 Gamma5 v
(Gamma5-hermiticity), each solve by the oracle's GMRES to 1e-6, and the
Rayleigh quotient rho = (w^H v) / (w^H w) of the last step (an upper bound
of sigma_min^2).  One process per grid point, each single-threaded.  Calls only oracle/ and the seeded input generator.
Writes tests/golden/mass_16x16x16x16.json.  Run: python tests/golden/tune_mass.py
"""
import json
import multiprocessing as mp
import os
import sys
import time

for _v in ('OMP_NUM_THREADS', 'OPENBLAS_NUM_THREADS', 'MKL_NUM_THREADS'):
    os.environ[_v] = '1'  # one BLAS thread per scan process

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

DIMS = (16, 16, 16, 16)
GRID = [-0.35, -0.40, -0.45, -0.50, -0.55]


def condition(m0):
    from oracle import dirac, solve
    from paper_2509_11424_gb300 import synth
    t0 = time.time()
    U = synth.gauge_field(DIMS, 0.4, 1002)
    M = dirac.wilson_matrix(U, m0, DIMS).tocsr()
    g5 = dirac.apply_gamma5
    v = synth.complex_normal(M.shape[0], 11)
    v /= np.linalg.norm(v)
    for _ in range(30):
        v = g5(M @ g5(M @ v))
        s = np.linalg.norm(v)
        v /= s
    smax = np.sqrt(s)
    sol = solve.LevelSolver(M, tol=1e-6)
    v = synth.complex_normal(M.shape[0], 12)
    v /= np.linalg.norm(v)
    for _ in range(5):
        w = sol(g5(sol(g5(v))))
        rho = (np.vdot(w, v) / np.vdot(w, w)).real
        v = w / np.linalg.norm(w)
    smin = np.sqrt(rho)
    return dict(m0=m0, sigma_max=smax, sigma_min=smin, cond=smax / smin, seconds=time.time() - t0)


def main():
    ctx = mp.get_context('spawn')
    with ctx.Pool(len(GRID)) as pool:
        res = pool.map(condition, GRID)
    best = max(res, key=lambda r: r['cond'])
    out = dict(workload='16^4, U = exp(i 0.4 H) seed 1002, antiperiodic time',
               method='oracle: power iteration (sigma_max), inverse iteration with GMRES 1e-6 (sigma_min)',
               grid=res, m0=best['m0'], cond=best['cond'])
    with open(os.path.join(HERE, 'mass_16x16x16x16.json'), 'w') as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == '__main__':
    main()
