/*
 * mgmlmc.h -- C ABI of the GB300 (sm_103a) library for orthogonal-projector
 * multigrid multilevel Monte Carlo trace estimation in lattice QCD
 * (Frommer, Jimenez-Merchan, Knechtli, Korzec, Ramirez-Hidalgo,
 * arXiv:2509.11424).
 *
 * The library computes, on one GPU, the estimators of the paper:
 *   tr(D^-1) = sum_{l<L} tr(O_l) + sum_{l<L} tr(F_l) + tr(D_L^-1)      (Sec. 3)
 *   O_l = (I - P_l P_l^H) D_l^-1 (I - P_l P_l^H),
 *   F_l = P_l^H D_l^-1 P_l - D_{l+1}^-1                   (Eq. OandF_def)
 * each term by Hutchinson's method with Z4 noise (Sec. 1, Eq. Hutchinson and
 * Eq. z4), with every level solve D_l z = y driven to a relative residual
 * (1e-12 in the paper, Sec. 4) by FGMRES preconditioned with a multigrid
 * cycle that starts at level l.  It also estimates the connected
 * pseudoscalar correlator G(t) (Eq. connected-G) through the orthogonal split
 * of Eq. full_ops_orth / Eq. G-split, and the disconnected loops
 * tr(Gamma5 D^-1(t,t)) (Eq. trace_equality_disconnected).
 *
 * Conventions
 *   Levels are 0-based here: level 0 is the fine lattice (the paper's l = 1).
 *   Complex numbers are interleaved (re, im) pairs of double (FP64) or
 *   float (FP32).
 *   Canonical layouts (host and device buffers passed to this API):
 *     site s = x + Lx (y + Ly (z + Lz t)), dims = {Lx, Ly, Lz, Lt};
 *     fine vector: index (s * 4 + spin) * 3 + colour (12 per site);
 *     coarse vector at level l >= 1: index (X * 2 N_tv + c * N_tv + k) for
 *       coarse site X (same ordering as s on the coarse lattice), chirality
 *       c in {0, 1} and test vector k;
 *     links: U[s][mu][a][b], mu = 0..3 = x, y, z, t (4 * 9 complex per site);
 *     multi-vectors (nrhs right-hand sides): nrhs vectors stored one after
 *       the other, each in the canonical vector layout.
 *   The Wilson operator (the paper uses only its Gamma5-hermiticity, Sec. 2):
 *     (D psi)(x) = (4 + m0) psi(x) - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                                   + (1 + gamma_mu) U_mu(x-mu)^H psi(x-mu) ]
 *   in the chiral basis (gamma_5 = diag(1, 1, -1, -1)), periodic in space,
 *   antiperiodic in time.
 *   Z4 noise (Eq. z4): entry i of a noise vector for (seed, sample, term, aux)
 *     takes word (i & 3) of Philox4x64-10 with counter
 *     (i >> 2, sample, term, aux) and key (seed, 0), r = word >> 62 and
 *     x_i = i^r.  term = 0 plain Hutchinson, 16 + l for O_l, 32 + l for F_l,
 *     48 for the coarsest level, 64 for connected-correlator sources
 *     (aux = source slice), 80 for disconnected loops (aux = slice),
 *     96 + l for the start vectors of the test-vector setup, 144 + l for
 *     the oblique M_l, 160 for deflated samples, 176 for the deflation
 *     start columns (sample = column), 192 + l for the extra start columns
 *     of the test-vector refinement (sample = column).
 *
 * Ownership and streams
 *   The context owns every device buffer it allocates; caller buffers are
 *   only read or written during the call.  Every kernel is launched on the
 *   stream given to mgmlmc_create (0 = legacy default stream).  Calls that
 *   return host results synchronise that stream.  A context is not
 *   thread-safe; use one context per host thread.
 *
 * Errors
 *   Every call returns an mgmlmc_status and never aborts the process.
 *   mgmlmc_last_error() returns a description of the last failure of that
 *   context.  A solve that hits its iteration cap or meets a NaN/Inf returns
 *   MGMLMC_ERR_NOT_CONVERGED / MGMLMC_ERR_NUMERIC; the context stays usable.
 */
#ifndef MGMLMC_H
#define MGMLMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MGMLMC_MAX_LEVELS 4

typedef struct mgmlmc_ctx mgmlmc_ctx;

typedef enum {
  MGMLMC_OK = 0,
  MGMLMC_ERR_ARG = 1,            /* invalid argument */
  MGMLMC_ERR_STATE = 2,          /* call out of order (e.g. no hierarchy yet) */
  MGMLMC_ERR_OOM = 3,            /* device allocation failed */
  MGMLMC_ERR_CUDA = 4,           /* a CUDA runtime call failed */
  MGMLMC_ERR_NOT_CONVERGED = 5,  /* iteration cap reached */
  MGMLMC_ERR_NUMERIC = 6         /* NaN / Inf / breakdown */
} mgmlmc_status;

/* MGMLMC_BF16 (bfloat16 storage, FP32 arithmetic) is accepted by
 * mgmlmc_apply for MGMLMC_OP_D on level 0 only; the solver runs FP64 or
 * FP32. */
typedef enum { MGMLMC_FP64 = 0, MGMLMC_FP32 = 1, MGMLMC_BF16 = 2 } mgmlmc_precision;

/* Multigrid hierarchy (Sec. 2.2: aggregation-based P_l with P_l^H P_l = I,
 * Galerkin D_{l+1} = P_l^H D_l P_l; Sec. 4: test vectors are rough
 * approximations, residual ~1e-1, to low modes). */
typedef struct {
  int n_levels;                        /* L, 1 .. MGMLMC_MAX_LEVELS */
  int block[MGMLMC_MAX_LEVELS - 1][4]; /* aggregate extents for level l -> l+1 */
  int n_tv[MGMLMC_MAX_LEVELS - 1];     /* test vectors for level l -> l+1,
                                          1 .. 128 and at most the rows of a
                                          (aggregate, chirality) block */
  int setup_rounds;   /* rounds of approximate inverse iteration */
  int setup_iters;    /* Krylov iterations per round (rough solves) */
  uint64_t seed;      /* seed of the initial random test vectors */
} mgmlmc_mg_params;

/* Level solver: FGMRES(restart) preconditioned by a multigrid K-cycle that
 * starts at the level being solved (Sec. 4: all levels to 1e-12).  With
 * MGMLMC_FP32 each inner FP32 solve of the FP64 defect correction reduces its
 * residual by inner_tol, or by the smaller factor 2 tol / r that is left to
 * do (r the largest relative true residual over the right-hand sides), and
 * also ends when a restart cycle fails to halve its true residual (the
 * precision floor of FP32 on an ill-conditioned level); the outer loop
 * continues from it until the true FP64 residual meets tol. */
typedef struct {
  double tol;          /* relative residual target ||b - D x|| / ||b|| */
  int max_iter;        /* cap on outer FGMRES iterations per solve */
  int restart;         /* FGMRES restart length, 1 .. 64 */
  int smoother_steps;  /* minimal-residual smoothing steps per cycle */
  int coarse_iters;    /* FGMRES iterations on intermediate levels */
  int precision;       /* MGMLMC_FP64: all FP64.  MGMLMC_FP32: FP32 inner
                          solves inside FP64 defect correction */
  double inner_tol;    /* FP32 inner relative tolerance (defect correction) */
  int smoother;        /* fine level: MGMLMC_SMOOTHER_SAP (red/black Schwarz
                          blocks, MR inside each block) or MGMLMC_SMOOTHER_MR;
                          coarse levels always use MR.  SAP needs an even
                          number of blocks in every direction (blocks of
                          8 x 4 x 4 x 2, else 4^4, else 2^4); otherwise MR is
                          used. */
  int sap_iters;       /* MR iterations inside each SAP block */
  int coarse_smoother_steps; /* MR steps of the smoother on levels >= 1 */
  int coarse_restart;  /* FGMRES restart length of the solves on levels >= 1
                          (their vectors are small), 1 .. 64; 0 = restart */
  int post_smoothing_only; /* 1: on the fine level the multigrid cycle
                          smooths after the coarse-grid correction only (no
                          pre-smoothing; coarser levels keep both);
                          0 (default): before and after on every level */
  int gram_schmidt_passes; /* classical Gram-Schmidt passes of the FP32
                          FGMRES Arnoldi step: 1, or 2 (0 = 2, the default);
                          FP64 solves always run 2 */
  int fine_batch;      /* memory bound of the fine level: mgmlmc_estimate_trace
                          solves level-0 systems (the O_0, F_0, M_0 and plain
                          terms) in blocks of at most fine_batch right-hand
                          sides; 0 = the estimator's batch.  Samples, noise
                          counters and results do not depend on it. */
  int learned_guess;   /* 1: FP32 solves on the fine level start from the
                          trained network's guess instead of zero: with
                          c = b / ||b||, x0 = ||b|| alpha N(c), alpha =
                          <D N(c), c> / ||D N(c)||^2 (the residual-minimising
                          step), and the FP32 residual c - alpha D N(c),
                          scaled back, as the first defect; every later defect
                          is the true FP64 residual, which alone decides
                          convergence (needs mgmlmc_learned_init or _train;
                          any smoother).  mgmlmc_estimate_trace does not use
                          it for the fine solve of F_0, whose right-hand side
                          P_0 x lies in the range of P_0 (the coarse-grid
                          correction already covers it; measured, the guess
                          cost iterations there).  0 (default): x0 = 0. */
} mgmlmc_solver_params;

#define MGMLMC_SMOOTHER_MR 0
#define MGMLMC_SMOOTHER_SAP 1
#define MGMLMC_SMOOTHER_LEARNED 2 /* fine level: SAP sweeps followed by one
                                     step along the trained network's output,
                                     z += alpha N(r) with the residual-minimising
                                     alpha (see mgmlmc_learned_train); a solve
                                     that does not converge within max_iter / 4
                                     is redone with SAP alone (counted in
                                     mgmlmc_learned_stats) */
#define MGMLMC_SMOOTHER_NET 3     /* fine level: the trained network in place of
                                     SAP, smoother_steps residual-minimising
                                     steps z += alpha N(r) per smoothing, with
                                     the same SAP fallback */

/* PLAIN: Hutchinson (Sec. 1, Eq. Hutchinson).  ORTHOGONAL: Sec. 3, Eq.
 * smultigrid-multilevel-monte-carlo (terms O_l, F_l, coarsest).  OBLIQUE:
 * Sec. 2.2, Eq. oblique_multigrid-multilevel-monte-carlo, the earlier
 * decomposition the paper compares against: terms M_l = D_l^-1 -
 * P_l D_{l+1}^-1 P_l^H (Eq. oblique-deflation), sampled as
 * x^H D_l^-1 x - (P_l^H x)^H D_{l+1}^-1 (P_l^H x), then the coarsest. */
typedef enum {
  MGMLMC_EST_PLAIN = 0,
  MGMLMC_EST_ORTHOGONAL = 1,
  MGMLMC_EST_OBLIQUE = 2,
  MGMLMC_EST_DEFLATED = 3  /* Sec. 2.1, Eq. deflated-estimator: needs
                              mgmlmc_deflation_build; terms DEFL (n_samples[0]
                              samples) and DEFL_EXACT (the exact part) */
} mgmlmc_estimator;

/* Term codes of the results (same numbers as the noise term ids). */
#define MGMLMC_TERM_PLAIN 0
#define MGMLMC_TERM_O 16        /* + level */
#define MGMLMC_TERM_F 32        /* + level */
#define MGMLMC_TERM_COARSEST 48
#define MGMLMC_TERM_M 144       /* + level: oblique M_l */
#define MGMLMC_TERM_DEFL 160    /* x^H (I - V V^H) D^-1 x */
#define MGMLMC_TERM_DEFL_EXACT 161 /* tr(V^H D^-1 V), n = 1, variance 0 */
#define MGMLMC_TERM_DEFL_START 176 /* noise stream of the start vectors */
#define MGMLMC_TERM_TV_EXTRA 192   /* + level: extra start columns of
                                      mgmlmc_refine_test_vectors */

typedef struct {
  int kind;          /* mgmlmc_estimator */
  int n_samples[2 * MGMLMC_MAX_LEVELS]; /* per term in the order
                       O_0..O_{L-2}, F_0..F_{L-2}, coarsest; oblique:
                       M_0..M_{L-2}, coarsest; plain: [0] */
  int batch;         /* right-hand sides solved together, >= 1 */
  uint64_t seed;     /* noise seed */
  uint64_t first_sample; /* sample counter of the first sample */
} mgmlmc_est_params;

typedef struct {
  int term;            /* MGMLMC_TERM_* code */
  int n;               /* samples taken */
  double mean_re, mean_im;
  double var;          /* 1/(N-1) sum |X_i - mean|^2 (Sec. 4) */
  double sum_re, sum_im, sum_abs2; /* raw accumulators (resume / merge) */
  double seconds;      /* device time spent on this term */
  double iters_mean;   /* mean outer iterations per level solve */
  double max_residual; /* largest true relative residual of its solves */
} mgmlmc_term_result;

/* ---- context -------------------------------------------------------------- */

/* Create a context for a lattice of extents dims[4] (each >= 2, even
 * extents not required, aggregation needs divisibility; 12 V < 2^31 with V
 * the number of sites).  stream is a cudaStream_t (NULL = legacy default
 * stream).  Uses the current device.  MGMLMC_ERR_ARG for other extents. */
mgmlmc_status mgmlmc_create(const int dims[4], void *stream, mgmlmc_ctx **out);
/* Release every device buffer of the context.  NULL is accepted. */
void mgmlmc_destroy(mgmlmc_ctx *ctx);
/* Description of the last failure (never NULL). */
const char *mgmlmc_last_error(const mgmlmc_ctx *ctx);

/* Gauge field (Sec. 1: 4-D lattice, 12 dof per site): 4 * V * 9 complex
 * double in the canonical link layout; host pointer (on_device = 0) or
 * device pointer (on_device = 1).  Invalidates the hierarchy. */
mgmlmc_status mgmlmc_set_gauge(mgmlmc_ctx *ctx, const double *U, int on_device);
/* Generate the gauge field on the device instead: synthetic SU(3) links
 * U_mu(x) = exp(i eps H) standing in for the paper's ensembles (Sec. 4 uses
 * real ones), H a random traceless Hermitian matrix per link.  Link
 * L = 4 s + mu draws the 20 Philox4x64-10 words of counters (L, j, 128, 0),
 * j = 0..4, key (seed, 0); entry e (row-major) of A uses words 2e, 2e + 1
 * as uniforms u = ((w >> 12) + 1/2) 2^-52 (inside (0, 1)) and Box-Muller,
 * A_e = sqrt(-2 ln u1) (cos 2 pi u2 + i sin 2 pi u2) / sqrt 2; then
 * H = (A + A^H)/2 - tr(.)/3 and U = exp(i eps H) in FP64.  eps = 0 gives the
 * free field.  Invalidates the hierarchy; MGMLMC_ERR_ARG for a non-finite
 * eps. */
mgmlmc_status mgmlmc_gen_gauge(mgmlmc_ctx *ctx, double eps, uint64_t seed);
/* Copy the context's gauge field out, in the layout mgmlmc_set_gauge takes
 * (4 * V * 9 complex double), to a host (on_device = 0) or device
 * (on_device = 1) buffer: checkpoints of a field drawn by mgmlmc_gen_gauge,
 * or its transfer to another context. */
mgmlmc_status mgmlmc_get_gauge(mgmlmc_ctx *ctx, double *U, int on_device);
/* Bare mass m0 of the Wilson operator.  Invalidates the hierarchy. */
mgmlmc_status mgmlmc_set_mass(mgmlmc_ctx *ctx, double m0);
/* Solver parameters (defaults: tol 1e-12, max_iter 2000, restart 16,
 * smoother_steps 4, coarse_iters 8, FP64, MR smoother, sap_iters 4,
 * coarse_smoother_steps 4).  smoother_steps counts the fine-level smoother
 * applications (SAP sweeps or MR steps) of each pre- and post-smoothing; the
 * learned step, when selected, follows the SAP sweeps of the post-smoother. */
mgmlmc_status mgmlmc_set_solver(mgmlmc_ctx *ctx, const mgmlmc_solver_params *p);
/* Import the N_tv test vectors of level `level` (0 .. L-2): n_tv vectors of
 * length n (the level's vector length), one after the other (canonical
 * layout, complex double), host or device.  The library keeps a copy; a later
 * mgmlmc_build_hierarchy uses them for that level instead of its own setup
 * (the parity hook: P and D_{l+1} become deterministic functions of the given
 * vectors) and fails with MGMLMC_ERR_ARG if n or n_tv do not match. */
mgmlmc_status mgmlmc_set_test_vectors(mgmlmc_ctx *ctx, int level, const double *V,
                                      int n_tv, int64_t n, int on_device);
/* Build P_l (per-aggregate, per-chirality modified Gram-Schmidt run twice),
 * D_{l+1} = P_l^H D_l P_l for every level and the dense inverse of the
 * coarsest operator. */
mgmlmc_status mgmlmc_build_hierarchy(mgmlmc_ctx *ctx, const mgmlmc_mg_params *p);
/* Size information of a level: dims[4] of its lattice, dofs per site and
 * vector length (complex entries). */
mgmlmc_status mgmlmc_level_info(const mgmlmc_ctx *ctx, int level, int dims[4],
                                int *dof, int64_t *n);

/* ---- estimators ----------------------------------------------------------- */

/* tr(D^-1) by plain Hutchinson (kind 0) or by the orthogonal multilevel
 * split (kind 1) or the oblique one (kind 2).  Writes one
 * mgmlmc_term_result per term (plain: 1; orthogonal: 2(L-1)+1 in the order
 * O_0.., F_0.., coarsest; oblique: L in the order M_0.., coarsest) into
 * out[max_terms] and their count into *n_terms. */
mgmlmc_status mgmlmc_estimate_trace(mgmlmc_ctx *ctx, const mgmlmc_est_params *p,
                                    mgmlmc_term_result *out, int max_terms, int *n_terms);
/* The per-sample values X_k of Hutchinson's estimator (Sec. 1, Eq.
 * Hutchinson: X_k = x_k^H A x_k for the term's operator A) of term `index`
 * (0-based position in the result array) of the last mgmlmc_estimate_trace
 * call on this context, in sample order: out[2k], out[2k + 1] = re, im of
 * sample first_sample + k.  *n receives the sample count; MGMLMC_ERR_ARG when
 * it exceeds max_samples or there is no such term (a failed estimate keeps
 * none). */
mgmlmc_status mgmlmc_last_samples(mgmlmc_ctx *ctx, int index, double *out, int max_samples, int *n);
/* Inexact deflation basis (Sec. 2.1, 'Deflation for the Dirac operator';
 * the paper's setting in Sec. 4.2 is k = 128, iters = 5, tol = 1e-6): the k
 * start columns are the Z4 vectors of samples 0..k-1 of noise stream
 * MGMLMC_TERM_DEFL_START, orthonormalised (Gram-Schmidt, two passes, column
 * order); each of `iters` inverse block power steps forms D^-1 Gamma5 V with
 * the hierarchy's solver at relative tolerance tol and re-orthonormalises.
 * Then the exact part tr(V^H D^-1 V) is computed with k solves at the
 * solver's own tolerance and returned in exact[2] (re, im) with the device
 * seconds of the whole build.  The build's solves run in FP64 whatever the
 * solver's precision.  1 <= k <= min(128, n); requires a hierarchy;
 * a new gauge field, mass or hierarchy discards the basis. */
mgmlmc_status mgmlmc_deflation_build(mgmlmc_ctx *ctx, int k, int iters, double tol, uint64_t seed,
                                     double *exact, double *seconds);
/* Test vectors of level `level` refined toward the eigenvectors of
 * Q_l = Gamma5_l D_l for its smallest |eigenvalues| (Sec. 2.2: the setup
 * phase builds P_l from test vectors approximating low modes; Sec. 5: more
 * accurate ones, to eigen-residual 1e-3 .. 1e-4, lower the variance).
 * Gamma5_l is +1 on the first half of a site's dofs and -1 on the second.
 * Block of n_vec columns (N_tv <= n_vec <= min(128, n)): the level's
 * current N_tv test vectors, then Z4 columns of samples N_tv .. n_vec-1 of
 * noise stream MGMLMC_TERM_TV_EXTRA + level, orthonormalised (Gram-Schmidt,
 * two passes, column order).  Each step: W = D_l^-1 Gamma5_l V with FP64
 * solves to relative tolerance solve_tol, W^H W = Y diag(mu) Y^H with mu
 * descending, V = W Y diag(mu)^-1/2 (simultaneous iteration with the Ritz
 * step on Q_l^-2).  Steps stop after max_iters, or earlier once every one
 * of the first N_tv columns has ||Q v - theta v|| <= eig_tol with
 * theta = v^H Q v (eig_tol = 0: exactly max_iters steps).  Those columns,
 * each scaled so that its first entry of largest modulus is real and
 * positive, become the level's test vectors (as if set by
 * mgmlmc_set_test_vectors; the levels above keep theirs), and the hierarchy
 * is rebuilt with the parameters of the last mgmlmc_build_hierarchy.
 * Outputs (each may be NULL): theta[N_tv], eig_res[N_tv] of the returned
 * columns, *steps taken.  Requires a hierarchy; level < L - 1. */
mgmlmc_status mgmlmc_refine_test_vectors(mgmlmc_ctx *ctx, int level, int n_vec, int max_iters,
                                         double eig_tol, double solve_tol, uint64_t seed,
                                         double *theta, double *eig_res, int *steps);
/* Exact trace of the coarsest-level inverse, tr(D_L^-1), from its dense
 * inverse (Sec. 3 allows a direct computation of this term). */
mgmlmc_status mgmlmc_coarsest_trace(mgmlmc_ctx *ctx, double *re, double *im);

/* Connected correlator split (Eq. G-split), orthogonal operators of Eq.
 * full_ops_orth with R = 2L-1 terms.  For samples k = first .. first+n-1 and
 * every source slice t' in [0, T) (all slices), with Z4 noise x on slice t':
 *   X_rs(t) = (1/T) sum_t' (Btil_s x)|_{t+t'}^H (B_r x)|_{t+t'},
 *   Btil = Gamma5 B^H Gamma5.
 * kind 0 (plain) uses the single operator D^-1 (R = 1); kind 2 (oblique)
 * the R = L operators B_l of Eq. G-traditional,
 *   B_l = Phat_{l-1} (D_l^-1 - P_l D_{l+1}^-1 P_l^H) Phat_{l-1}^H, then
 *   Phat_{L-1} D_L^-1 Phat_{L-1}^H  (here Btil = B).  Output (host):
 * mean[R][R][T] and var[R][R][T] complex mean / real variance over samples. */
mgmlmc_status mgmlmc_connected_correlator(mgmlmc_ctx *ctx, int kind, int n_samples,
                                          uint64_t seed, uint64_t first_sample,
                                          double *mean, double *var, int *R);
/* Disconnected loop tr(Gamma5 D^-1(t,t)) = sum_r tr(Gamma5 B_r(t,t)) (Eq.
 * trace_equality_disconnected) with the operators of the correlator's kind
 * (plain R = 1, orthogonal 2L-1, oblique L): samples X_r = x^H Gamma5 B_r x
 * with Z4 noise x on slice t.  Output mean[R] complex, var[R] real. */
mgmlmc_status mgmlmc_disconnected_loop(mgmlmc_ctx *ctx, int kind, int t, int n_samples,
                                       uint64_t seed, uint64_t first_sample,
                                       double *mean, double *var, int *R);

/* ---- operator hooks (device buffers, canonical layouts) ------------------ */

typedef enum {
  MGMLMC_OP_D = 0,        /* out = D_l in                      (level l)       */
  MGMLMC_OP_RESTRICT = 1, /* out = P_l^H in      (level l -> level l+1)         */
  MGMLMC_OP_PROLONG = 2,  /* out = P_l in        (level l+1 -> level l)         */
  MGMLMC_OP_PROJECT = 3,  /* out = (I - P_l P_l^H) in            (level l)      */
  MGMLMC_OP_SOLVE = 4,    /* out = D_l^-1 in by the MG-preconditioned solver   */
  MGMLMC_OP_GAMMA5 = 5,   /* out = Gamma5 in (level l)                         */
  MGMLMC_OP_SMOOTH = 6,   /* out = z after the level's smoother (SAP on level 0
                             when selected, else MR; smoother_steps sweeps)
                             applied to D_l z = in from z = 0                 */
  MGMLMC_OP_NET = 7       /* out = N(in), the learned network (level 0)       */
} mgmlmc_op;

/* OR-ed into op of mgmlmc_apply: level-0 MGMLMC_FP32 vectors are already in
 * the library's internal order (see mgmlmc_reorder), so no reordering pass
 * runs around the operator.  Other levels and precisions are unaffected. */
#define MGMLMC_LAYOUT_INTERNAL 0x100

/* Apply an operator to nrhs device vectors.  precision selects the storage
 * type of in/out (complex double for MGMLMC_FP64, complex float for
 * MGMLMC_FP32; MGMLMC_OP_SOLVE accepts MGMLMC_FP64 only, its internal
 * precision is the solver's; MGMLMC_BF16, complex bfloat16 storage with
 * FP32 arithmetic, is accepted for MGMLMC_OP_D on level 0).  in and out
 * must not overlap (MGMLMC_ERR_ARG if their byte ranges intersect).  Level-0 FP32 and BF16 vectors are reordered to and from
 * the internal order around the operator unless op carries
 * MGMLMC_LAYOUT_INTERNAL. */
mgmlmc_status mgmlmc_apply(mgmlmc_ctx *ctx, int op, int level, int precision,
                           const void *in, void *out, int nrhs);
/* Reorder nrhs level-0 complex-float device vectors between the canonical
 * layout and the internal one, where the library keeps FP32 fine-level
 * vectors structure-of-arrays: complex component i (spin-major, 0..11) of
 * site s at ((i / 2) V + s) * 2 + i % 2, so that consecutive sites are
 * contiguous for each pair of components.  to_internal = 1: in canonical,
 * out internal; 0: the reverse.  in and out must not overlap. */
mgmlmc_status mgmlmc_reorder(mgmlmc_ctx *ctx, const void *in, void *out, int nrhs,
                             int to_internal);
/* The same for level-0 complex-bfloat16 vectors (pairs re, im of bf16, the
 * MGMLMC_BF16 storage of mgmlmc_apply): internally component i of site s is
 * the pair ((i / 4) V + s) * 4 + i % 4, 16-byte chunks of four components. */
mgmlmc_status mgmlmc_reorder_bf16(mgmlmc_ctx *ctx, const void *in, void *out, int nrhs,
                                  int to_internal);
/* The projection of MGMLMC_OP_PROJECT, out = (I - P_l P_l^H) in, without any
 * device allocation during the call.  The paper has no counterpart: this is
 * for callers that cannot allocate device memory while they run -- code
 * inside a CUDA stream capture that must not create allocations, processes
 * whose device memory is reserved up front by a pool they do not control,
 * or loops that forbid allocator calls on their critical path.  in/out are
 * device buffers as for mgmlmc_apply (complex double for MGMLMC_FP64,
 * complex float for MGMLMC_FP32), nrhs vectors of level `level`; in and out
 * must be distinct (MGMLMC_ERR_ARG if their byte ranges intersect).
 * The coarse intermediate P_l^H in lives in a fixed device array of 2 MiB
 * (131072 complex doubles, 262144 complex floats) that every GPU loading the
 * library holds until exit; calls with nrhs * n_{l+1} beyond that return
 * MGMLMC_ERR_ARG.  The first call on a device looks the array's address up
 * (once per device), so make that first call before any stream capture.
 * Every call shares the array: calls whose kernels overlap on the GPU race on
 * it and must be serialised by the caller.  The array is fully overwritten
 * before it is read, so no clearing is needed between calls. */
mgmlmc_status mgmlmc_project_noalloc(mgmlmc_ctx *ctx, int level, int precision, const void *in,
                                     void *out, int nrhs);
/* Z4 noise (Eq. z4) of `level` for samples first_sample .. + nrhs - 1 into a
 * device multi-vector (complex double).  slice < 0: full support; otherwise
 * supported on time slice `slice` of that level's lattice. */
mgmlmc_status mgmlmc_noise(mgmlmc_ctx *ctx, int level, uint64_t seed, uint64_t first_sample,
                           uint64_t term, uint64_t aux, int slice, double *out, int nrhs);
/* Copy P_l to host as [aggregate][chirality][row][k] complex double, row =
 * site_in_aggregate * dof/2 + (dof within chirality); site_in_aggregate
 * ordered like s inside the block. */
mgmlmc_status mgmlmc_get_prolongator(mgmlmc_ctx *ctx, int level, double *out);
/* Copy the N_tv test vectors P_l was built from to host as [k][n] complex
 * double (n the level's vector length): imported, set up, or refined by
 * mgmlmc_refine_test_vectors.  Passing them back through
 * mgmlmc_set_test_vectors reproduces the hierarchy.  level < L - 1. */
mgmlmc_status mgmlmc_get_test_vectors(mgmlmc_ctx *ctx, int level, double *out);
/* Copy the stencil blocks of D_l (level >= 1) to host as
 * [X][d][i][j] complex double, d = 0 self, 1 + 2 mu (+mu), 2 + 2 mu (-mu);
 * block d of X collects the fine hops of direction d leaving aggregate X,
 * block 0 the diagonal and the hops staying inside X. */
mgmlmc_status mgmlmc_get_coarse_op(mgmlmc_ctx *ctx, int level, double *out);
/* Free every device work buffer the context has grown (Krylov bases,
 * smoother and estimator vectors, reduction and transfer scratch) and the
 * captured graphs that use them; the gauge field, the hierarchy (P_l, D_l,
 * the coarsest inverse, the kept test vectors), a deflation basis and the
 * learned network stay.  Later calls allocate what they need again.  For
 * callers that switch between configurations of very different memory
 * footprint on a large lattice (e.g. FP32 and FP64 solvers, or batch sizes). */
mgmlmc_status mgmlmc_release_workspaces(mgmlmc_ctx *ctx);
/* Failure injection for tests (process-wide, not in the paper): the
 * coarse-stencil kernels arm the mbarrier of their shared-memory staging
 * copy with extra_bytes (a multiple of 16, at most 4096) more than the copy
 * delivers, so the copy lands in full but the barrier never completes: the
 * kernel's bounded wait (1 s of the GPU's global timer, then a second one
 * before the block leaves) runs out, the kernel sets its error flag and the
 * call that launched it returns MGMLMC_ERR_CUDA with the context usable.  0
 * (the default) restores normal operation. */
mgmlmc_status mgmlmc_test_staging_extra(mgmlmc_ctx *ctx, int extra_bytes);
/* Statistics of the last solve: outer iterations (max over rhs) and true
 * relative residual (max over rhs). */
mgmlmc_status mgmlmc_last_solve_stats(const mgmlmc_ctx *ctx, int *iters, double *residual);

/* ---- learned smoother ------------------------------------------------------
 * Not in the paper.  A gauge-covariant convolutional network stands in for the
 * fine-level smoother: three linear layers, channels 1 -> C -> C -> 1,
 *   phi[o](x) = sum_c sum_h W[h][o][c] (T_h psi[c])(x),
 * h = 0 identity, 1 + 2 mu: U_mu(x) psi(x + mu), 2 + 2 mu: U_mu(x - mu)^H
 * psi(x - mu) (fermion boundary sign), W[h][o][c] a complex 4x4 spin matrix.
 * Weights are stored layer by layer, each [h][o][c][4][4] complex double.
 * Training minimises sum_b ||r_b - D N(r_b)||^2 / ||r_b||^2 over residuals
 * r_b that the solver itself produces (the residuals left by the SAP
 * post-smoother of its multigrid cycles, i.e. what the learned step sees);
 * with the error e = D^-1 r this is ||N(r) - e||^2 in the D^H D norm.
 * The true FP64 residual still decides every solve, so estimates stay
 * unbiased whatever the network does. */
typedef struct {
  int channels;   /* C, 1 .. 32 (16 for the workload) */
  int steps;      /* Adam steps */
  int batch;      /* residuals per step */
  int pool;       /* residual / error pairs collected from the solver */
  double lr;      /* Adam learning rate */
  uint64_t seed;  /* seed of the weight initialisation and of the noise of the
                     solves that produce the pairs */
  int source;     /* 0: the residuals the SAP post-smoother leaves during solves
                     of Z4 right-hand sides (the network as a smoothing step);
                     1: the right-hand sides of the estimator's O_0
                     solves, projected Z4 noise (I - P_0 P_0^H) x, for the
                     network as the initial guess (learned_guess); no solves
                     are needed to collect them */
} mgmlmc_train_params;

typedef struct {
  int steps, pairs;
  double loss_init;   /* mean loss of the initial (Jacobi-like) network */
  double loss_first;  /* mean loss over the first 10 steps */
  double loss_last;   /* mean loss over the last 10 steps */
  double seconds;     /* wall time of collection + training */
} mgmlmc_train_result;

/* (Re)initialise the network: channel 0 carries the input through the layers
 * scaled to a Jacobi step 1/(4 + m0), every other weight small (Z4 draws of
 * size 0.01 from the library's Philox stream). */
mgmlmc_status mgmlmc_learned_init(mgmlmc_ctx *ctx, int channels, uint64_t seed);
/* Number of complex weights of all layers together. */
mgmlmc_status mgmlmc_learned_size(const mgmlmc_ctx *ctx, int64_t *n_complex);
/* Copy all weights to (set = 0) or from (set = 1) a host array of
 * 2 * n_complex doubles. */
mgmlmc_status mgmlmc_learned_weights(mgmlmc_ctx *ctx, double *host, int set);
/* FP64 loss and gradient dL/dW* (host, 2 * n_complex doubles) of a batch of
 * nrhs fine-level device vectors r (complex double). */
mgmlmc_status mgmlmc_learned_loss_grad(mgmlmc_ctx *ctx, const double *r, int nrhs, double *loss,
                                       double *grad_host);
/* Collect p->pool residuals from solves with the current solver, then run
 * p->steps Adam steps on the GPU (FP32 forward/backward, FP64 weights). */
mgmlmc_status mgmlmc_learned_train(mgmlmc_ctx *ctx, const mgmlmc_train_params *p,
                                   mgmlmc_train_result *out);
/* Solves that fell back from the learned smoother to SAP. */
mgmlmc_status mgmlmc_learned_stats(const mgmlmc_ctx *ctx, int64_t *fallbacks);

/* ---- measurement --------------------------------------------------------- */

/* Kernel classes timed by mgmlmc_profile. */
#define MGMLMC_KERNEL_WILSON_FP64 0
#define MGMLMC_KERNEL_WILSON_FP32 1
#define MGMLMC_KERNEL_STENCIL_FP64 2
#define MGMLMC_KERNEL_STENCIL_FP32 3
#define MGMLMC_KERNEL_SAP_FP64 4 /* one SAP sweep (both colours) */
#define MGMLMC_KERNEL_SAP_FP32 5
#define MGMLMC_KERNEL_TRANSFER 6 /* P^H and P inside the multigrid cycle */
#define MGMLMC_KERNEL_ORTHO 7    /* Gram-Schmidt of the FGMRES basis */
#define MGMLMC_KERNEL_NET 8      /* learned step: network forward */
#define MGMLMC_KERNEL_COARSEST 9 /* dense coarsest apply inside the cycle */

/* Number of CUDA kernels this library has launched in this process (all
 * contexts), for counting the launches of a timed region. */
int64_t mgmlmc_kernel_launches(void);
/* Enable (1) or disable (0) per-launch timing of the operator kernels with
 * CUDA events on the context's stream, and reset the counters. */
mgmlmc_status mgmlmc_profile(mgmlmc_ctx *ctx, int enable);
/* Counters of one kernel class since the last mgmlmc_profile: launches,
 * summed device milliseconds, summed algorithmic bytes (unique data: for the
 * Wilson operator nrhs input and output spinors plus 4 links per site; for a
 * coarse stencil the 9 blocks, at their stored size, plus input and output
 * per site; for a SAP sweep the 4 links once, and per right-hand side the
 * residual, z and e read or written by the block and face passes, 8 spinors
 * per site) and summed algorithmic flops (1368 per site and rhs for Wilson;
 * 72 m^2 per coarse site and rhs for a stencil with m dofs per site;
 * 1368 sap_iters + 684 per site and rhs for a SAP sweep).  Synchronises the
 * stream. */
mgmlmc_status mgmlmc_profile_stats(mgmlmc_ctx *ctx, int kernel_class, int64_t *launches,
                                   double *ms, double *bytes, double *flops);

/* ---- kernel variants ------------------------------------------------------ */

/* Kernels with selectable variants. */
#define MGMLMC_VARIANT_DSLASH_FP32 0
/* The FP32 coarse stencil D_l, l >= 1 (Galerkin, Sec. 2.2): 0 = FP32 on the
 * CUDA cores (default); 1, 2 = the 5th-generation tensor cores (tcgen05.mma
 * kind::tf32, operands staged in shared memory by a bulk copy, FP32
 * accumulators in tensor memory) for levels with 32 dofs per site (N_tv =
 * 16; other levels keep variant 0): the products take the operands as TF32
 * (10-bit mantissa, relative rounding <= 2^-11 per operand) and accumulate
 * in FP32, so results differ from variant 0 by that rounding; 1 issues
 * M = 64 MMAs (two accumulators, real and imaginary parts of the blocks
 * stacked), 2 the same as M = 128 MMAs whose extra rows are discarded (the
 * same numbers, twice the tensor work); 3 = the blocks stored as BF16 pairs
 * (half the bytes, relative rounding <= 2^-9 per entry) with FP32
 * arithmetic, for up to 8 right-hand sides at 32 dofs per site (variant 0
 * otherwise); 4 = the tensor cores with BF16 operands (tcgen05.mma
 * kind::f16, relative rounding <= 2^-9 per operand, FP32 accumulation, half
 * the bytes of variant 1); 5 = variant 4 as a persistent kernel (one thread
 * block per SM walking the sites with two shared-memory stages and two
 * tensor-memory accumulators, so one site's MMAs and tile copy overlap the
 * gathers and epilogue of others; identical results; up to 32 right-hand
 * sides, variant 4 beyond); 6 = variant 3's BF16 blocks and sums with one
 * warp per coarse site streaming its blocks from memory in 16-byte row
 * chunks (a second BF16 copy of the blocks in that layout; results
 * identical to variant 3; up to 8 right-hand sides at 32 dofs per site,
 * variant 0 otherwise); 7 = variant 6 with one thread block per coarse site
 * and a warp per direction (more parallel work on coarse lattices with few
 * sites; identical results).  Variant 0 runs up to 8 right-hand sides at 32 dofs per site in
 * a pipelined kernel (persistent blocks, a two-stage ring of bulk copies
 * over sites) with results identical to the one-site-per-block kernels.
 * -2 = autotune among 0, 1, 3, 4, 5, 6 and 7 per (level, nrhs) on the first call
 * outside graph capture (opt-in,
 * since the choice changes the rounding).  Inside a solve the variant applies
 * to the multigrid preconditioner only (smoothers, coarse-grid corrections);
 * the Krylov operator of every FGMRES keeps variant 0, so the FP32 inner
 * solves reach their tolerance as with FP32 throughout, and the FP64 defect
 * correction decides convergence with the true residual either way. */
#define MGMLMC_VARIANT_STENCIL_FP32 1
/* The FP32 SAP sweep on the fine level (the smoother of Sec. 4's
 * DD-alpha-AMG solver).  With two or more right-hand sides and blocks of
 * 8 x 4 x 4 x 2 or 4^4 sites, one block and two right-hand sides per thread
 * block: 0 (default) = one thread per site and right-hand side, the block's
 * links and the solution it updates staged in shared memory by asynchronous
 * copies that overlap the residual load; 1 = one thread per site carrying
 * both right-hand sides in packed FP32 pairs (.f32x2 instructions).  Other
 * cases, and 2 = throughout, the general kernels.  Every variant updates the
 * faces of each colour in a separate pass over that colour's sites, and all
 * compute the same sums in the same order: identical results. */
#define MGMLMC_VARIANT_SAP_FP32 2
/* FP32 restriction P_l^H and prolongation P_l (Sec. 2.2): 0 (default) = P in
 * FP32; 1 = P stored as BF16 (round to nearest, relative error <= 2^-9 per
 * entry; FP32 arithmetic; half the bytes of the dominant operand), for the
 * transfers inside the multigrid preconditioner and for MGMLMC_OP_RESTRICT /
 * MGMLMC_OP_PROLONG on FP32 vectors.  The orthogonal projector
 * I - P_l P_l^H of the estimators always uses the exact P. */
#define MGMLMC_VARIANT_TRANSFER_FP32 3
/* Choose the variant of a kernel for later calls: for the FP32 fine Wilson
 * operator -2 = autotune (default: the first call per right-hand-side count
 * outside graph capture times every variant on that call's operands and
 * keeps the fastest), 0 .. 6 = fixed: one thread per site; 0 .. 4 in
 * 128-thread blocks, 0 and 1 one right-hand side per thread with registers
 * for 6 or 8 resident blocks per SM; 2 and 3 two right-hand sides per thread
 * with registers for 4 or 5 blocks; 4 one right-hand side with the next
 * operand set loaded while the current one is used (4 blocks); 5 and 6 put 4
 * or 8 right-hand sides of the same 32 sites in the warps of one block, so
 * those warps read the sites' links from L1 after the first.
 * Every variant computes the same sums in the same order.  Returns
 * MGMLMC_ERR_ARG for an unknown kernel or variant. */
mgmlmc_status mgmlmc_set_kernel_variant(mgmlmc_ctx *ctx, int kernel, int variant);
/* Number of fixed variants of a kernel (-1 for an unknown kernel). */
int mgmlmc_kernel_variants(int kernel);
/* The variant that calls with nrhs right-hand sides use (-2 while an
 * autotuned choice is not yet made; for the stencil, that of level 1). */
mgmlmc_status mgmlmc_get_kernel_variant(const mgmlmc_ctx *ctx, int kernel, int nrhs,
                                        int *variant);

#ifdef __cplusplus
}
#endif
#endif /* MGMLMC_H */
