"""Oracle statistics of the 16^4 benchmark workload, for the CPU arm of
bench.py.

For the mass chosen by tune_mass.py (read from mass_16x16x16x16.json) this
script runs the plain Hutchinson estimator of tr(D^-1) (Sec. 1, Eq.
Hutchinson) with the oracle: Z4 noise (seed 2002, plain-term stream, samples
0..N-1), each sample x^H D^-1 x with the oracle's GMRES(64) solve to the
1e-12 relative residual of Sec. 4.  It records the sample mean, the sample
variance of Sec. 4 and the GMRES iterations and seconds per solve, and adds
them to mass_16x16x16x16.json under "oracle_plain".  Calls only oracle/ and
the seeded input generator.  Run: python tests/golden/oracle_workload.py [N]
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import dirac, estimators, noise, solve  # noqa: E402
from paper_2509_11424_gb300 import synth  # noqa: E402

DIMS = (16, 16, 16, 16)


def main(N=6):
    path = os.path.join(HERE, 'mass_16x16x16x16.json')
    info = json.load(open(path))
    m0 = info['m0']
    U = synth.gauge_field(DIMS, 0.4, 1002)
    M = dirac.wilson_matrix(U, m0, DIMS).tocsr()
    sol = solve.LevelSolver(M, tol=1e-12)
    X, iters, secs = [], [], []
    for k in range(N):
        x = noise.z4_vector(M.shape[0], 2002, k, noise.TERM_PLAIN)
        t0 = time.time()
        z = sol(x)
        secs.append(time.time() - t0)
        iters.append(sol.last_iters)
        X.append(np.vdot(x, z))
        print('sample %d: X = %s, %d iterations, %.1f s' % (k, X[-1], iters[-1], secs[-1]), flush=True)
    mu, var = estimators.sample_stats(np.array(X))
    info['oracle_plain'] = dict(n=N, mean=[mu.real, mu.imag], var=var, gmres_iters=iters,
                                seconds=secs, noise_seed=2002, solver='GMRES(64) to 1e-12')
    with open(path, 'w') as f:
        json.dump(info, f, indent=1)
    print(json.dumps(info['oracle_plain'], indent=1))


if __name__ == '__main__':
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 6)
