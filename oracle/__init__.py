"""Plain, slow FP64 CPU oracle for orthogonal-projector multigrid multilevel
Monte Carlo (MG-MLMC) trace estimation in lattice QCD (Frommer et al.,
arXiv:2509.11424).

This package is TEST INFRASTRUCTURE.  Only the test-suite, the smoke check in
``__graft_entry__`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` may import it.  The CUDA library never imports, links or calls
anything in here, and nothing in here imports the CUDA library or its Python
binding: the two share no code, no tables and no constants.  Inputs (gauge
fields, test vectors) reach both sides from the seeded generators in
``paper_2509_11424_gb300.synth``, which hold none of the method's arithmetic;
the one random stream the method itself draws (the Z4 noise) is produced on
each side by its own Philox4x64-10 implementation written from the generator's
published definition.

Every function restates the paper's definitions in numpy/scipy, in FP64, with
no blocking, fusion or reordering beyond what the definition states:

* ``dirac``      the Wilson-Dirac operator D (Sec. 1: 12 dof per site) and
                 Gamma_5 (Sec. 2, 'Deflation for the Dirac operator').
* ``noise``      Philox4x64-10 and the Z4 distribution (Sec. 1, Eq. z4).
* ``gauge``      the counter-based synthetic gauge field exp(i eps H) that
                 the library can draw on the device (stand-in for the
                 ensembles of Sec. 4), with the same published Philox.
* ``multigrid``  aggregation, per-aggregate orthonormalised P, R = P^H,
                 Galerkin D_{l+1} = P^H D_l P (Sec. 2.2, Eq. Al_def and the
                 Galerkin paragraph; Sec. 3).
* ``solve``      exact level solves (the 1e-12 solves of Sec. 4 are D_l^{-1}
                 up to tolerance; the oracle solves directly).
* ``estimators`` Hutchinson (Eq. Hutchinson), the orthogonal decomposition
                 (Eq. OandF_def, Eq. smultigrid-multilevel-monte-carlo), the
                 sample variance of Sec. 4, the MLMC allocation (Eq. MLMC-Nl),
                 the connected correlator split (Eq. connected-G, Eq.
                 full_ops_orth, Eq. G-split) and the disconnected loop
                 (Eq. trace_equality_disconnected).
* ``exact``      exact targets: dense inverses on tiny lattices and free-field
                 closed forms in momentum space.
* ``smoother``, ``learned``  the MR/SAP smoothers and the gauge-covariant
                 learned layers the solver uses.
* ``deflation``  inexact deflation of Hutchinson's estimator (Sec. 2.1,
                 Eq. deflated-estimator; inverse block power on Gamma5 D).
* ``testvectors`` test vectors refined toward the low eigenvectors of
                 Gamma5 D_l to a chosen eigen-residual (Sec. 2.2 setup phase,
                 Sec. 5 outlook), by simultaneous inverse iteration.
"""
