// Host-side launchers of the mgmlmc kernels.  Every launcher enqueues on the
// given stream and returns immediately; buffers are device pointers.
// Multi-vectors hold nrhs vectors of length n one after the other; a Krylov
// basis holds k multi-vectors one after the other (stride nrhs * n).
#pragma once

#include "common.cuh"

namespace mg {

// Blocks per reduction output (deterministic: depends on n only).
int reduce_blocks(int64_t n);
// Scratch of the single-pass reductions: reduce_blocks(n) partial sums per
// output, and one ticket per output that is zero between calls (the block
// that finishes an output last resets it).  Tickets belong to one stream at
// a time: concurrent reductions need separate ticket arrays.
constexpr int kTickets = 1 << 16;
struct RedScratch {
  double2 *partial;
  unsigned *ticket;  // kTickets entries
};

// ------------------------------------------------------------------ BLAS-1
// out[r] = sum_i conj(x_r[i]) y_r[i]   (double2 results on the device)
template <typename T>
void dot(const C<T> *x, const C<T> *y, int64_t n, int nrhs, double2 *out, RedScratch scr,
         cudaStream_t s);
// h[r * ldh + j] = <V_j,r , w_r> for j < k (basis stride vstride)
template <typename T>
void multi_dot(const C<T> *V, int64_t vstride, int k, const C<T> *w, int64_t n, int nrhs,
               double2 *h, int ldh, RedScratch scr, cudaStream_t s);
// w_r += sign * sum_{j<k} h[r * ldh + j] V_j,r
template <typename T>
void multi_axpy(const C<T> *V, int64_t vstride, int k, C<T> *w, int64_t n, int nrhs,
                const double2 *h, int ldh, double sign, cudaStream_t s);
// y = a x + b y   (host scalars, all rhs)
template <typename T>
void axpby(double a, const C<T> *x, double b, C<T> *y, int64_t n, int nrhs, cudaStream_t s);
// y_r = x_r * scal[r]  (real per-rhs factors on the device)
template <typename T>
void scale_rhs(const C<T> *x, C<T> *y, const double *scal, int64_t n, int nrhs, cudaStream_t s);
// minimal-residual step for every rhs: alpha = <q, r> / <q, q>;
// z += alpha r; r -= alpha q.  dots[r] = <q, r>, nq[r].x = <q, q>
template <typename T>
void mr_update(C<T> *z, C<T> *r, const C<T> *q, const double2 *dqr, const double2 *nq,
               int64_t n, int nrhs, cudaStream_t s);
// minimal-residual step along a given direction e with q = D e:
// alpha = <q, r> / <q, q>; z += alpha e; r -= alpha q
template <typename T>
void mr_dir_update(C<T> *z, C<T> *r, const C<T> *e, const C<T> *q, const double2 *dqr,
                   const double2 *nq, int64_t n, int nrhs, cudaStream_t s);
// out = in converted between precisions
template <typename To, typename From>
void convert(const C<From> *in, C<To> *out, int64_t n, cudaStream_t s);
// y += x (x in lower precision, y in higher)
template <typename T, typename Tlo>
void add_lo(const C<Tlo> *x, C<T> *y, int64_t n, cudaStream_t s);
// y_r = x_r * scal[r] (null scal: 1) between the canonical order and the
// fine level's structure-of-arrays order (to_soa: x canonical -> y SoA, else
// y canonical), converting precision; V sites of 12 complex per vector
template <typename To, typename From>
void relayout(const C<From> *x, C<To> *y, const double *scal, int64_t V, int nrhs, bool to_soa,
              cudaStream_t s);
// y_r = x_r * scal[r] converting precision (scal real, device)
template <typename To, typename From>
void convert_scale(const C<From> *x, C<To> *y, const double *scal, int64_t n, int nrhs,
                   cudaStream_t s);

// ------------------------------------------------------------------ FGMRES
// Small per-rhs state of a batched FGMRES cycle (device arrays).
struct GmresState {
  int m;          // restart length
  int nrhs;
  double2 *H;     // [nrhs][(m+1) * m]  column-major: H[r][j * (m+1) + i]
  double2 *h1;    // [nrhs][m+1] first Gram-Schmidt coefficients
  double2 *h2;    // [nrhs][m+1] second (re-orthogonalisation) coefficients
  double *cs;     // [nrhs][m]
  double2 *sn;    // [nrhs][m]
  double2 *g;     // [nrhs][m+1]
  double2 *y;     // [nrhs][m]
  double2 *nrm;   // [nrhs] ||w||^2 in .x
  double *inv;    // [nrhs] scale factor for the next basis vector
  double *res;    // [nrhs] residual estimate |g_{i+1}|
  double *target; // [nrhs] absolute tolerance per rhs
  int *active;    // [nrhs] 1 while the rhs iterates in this cycle
  int *nit;       // [nrhs] iterations done in this cycle
};
// initial: beta = sqrt(nrm.x); g = (beta, 0...); inv = 1/beta; active per
// beta > target
void gmres_start(GmresState st, cudaStream_t s);
// fold the Gram-Schmidt coefficients and ||w||^2 of iteration i
void gmres_arnoldi(GmresState st, int i, cudaStream_t s);
// y = H^-1 g per rhs (upper triangular of size nit[r])
void gmres_solve(GmresState st, cudaStream_t s);

// ------------------------------------------------------------------ operators
// D psi for nrhs right-hand sides.  FP64: canonical vectors and links U.
// FP32: structure-of-arrays vectors (soa_index) and links UDs, 16-byte
// aligned; variant 0 .. wilson_fp32_variants() - 1 picks right-hand sides per
// thread (1 or 2) and the register budget (resident blocks per SM).
template <typename T>
void wilson_apply(const C<T> *in, C<T> *out, const C<T> *U, const C<T> *UDs, Geom g, double m0,
                  int nrhs, int variant, cudaStream_t s);
int wilson_fp32_variants();
// nlinks synthetic SU(3) links U = exp(i eps H) from a counter-based draw
// (seed): Philox4x64-10 words -> Box-Muller normals A -> H = (A + A^H)/2 -
// tr/3 -> matrix exponential; U row-major per link, canonical link order
void gauge_generate(double2 *U, int64_t nlinks, double eps, uint64_t seed, cudaStream_t s);
// BF16 storage, FP32 arithmetic: D psi for nrhs vectors of complex bf16 in
// the chunked structure-of-arrays order (pair ((i/4) V + s) * 4 + i % 4),
// links Ub from link_bf16; 16-byte aligned
void wilson_apply_bf16(const void *in, void *out, const void *Ub, Geom g, double m0, int nrhs,
                       cudaStream_t s);
// Ub[mu][a][b][s] = bf16(U[s][mu][a][b]) (round to nearest)
void link_bf16(const float2 *U, void *Ub, int V, cudaStream_t s);
// canonical complex-bf16 [rhs][site][12] <-> the chunked order above
void relayout_bf16(const void *x, void *y, int64_t V, int nrhs, bool to_soa, cudaStream_t s);
// UDs[mu][a][b][s] = U[s][mu][a][b]
void link_soa(const float2 *U, float2 *UDs, int V, cudaStream_t s);
// the 9 hop-class parts of D (Galerkin): out9[h] for h = 0..8, single rhs.
template <typename T>
void wilson_split(const C<T> *in, C<T> *out9, const C<T> *U, Geom g, double m0, const int b[4],
                  cudaStream_t s);
// coarse stencil with transposed blocks AT[X][d][j][i]; when they fit, the 9
// blocks of a site are staged by one TMA bulk copy; err[0] = 2 if a copy
// does not complete within the bounded wait
template <typename T>
void stencil_apply(const C<T> *in, C<T> *out, const C<T> *AT, Geom g, int nrhs, int *err,
                   cudaStream_t s);
// Tensor-core (tcgen05 kind::tf32) coarse stencil for 32 dofs per site:
// ATC holds each site's nine stacked [Re A_d; Im A_d] tiles in the MMA's
// shared-memory image (stencil_tile_tc builds it from the canonical A);
// FP32 vectors, TF32 products, FP32 accumulation.  layout 0: M = 64 MMAs,
// 1: M = 128 MMAs with half the rows discarded, 2: BF16 operands (kind::f16,
// M = 64) (see kernels_tc.cu).  err[0] = 3 if a bounded wait runs out.
// With bf16 the tiles hold BF16 values (kind::f16 MMAs, layout 2).
bool stencil_tc_supported(const Geom &g);
size_t stencil_tc_elems(const Geom &g);
void stencil_tile_tc(const double2 *A, void *ATC, bool bf16, const Geom &g, cudaStream_t s);
void stencil_apply_tc(const float2 *in, float2 *out, const void *ATC, Geom g, int nrhs, int *err, int layout,
                      cudaStream_t s);
// Pipelined FP32 coarse stencil for 32 dofs per site and 1 .. 8 right-hand
// sides: persistent CTAs with a two-stage ring of bulk copies over sites.
// AT: the transposed blocks as FP32 (identical results to stencil_apply) or,
// bf16 = true, as BF16 pairs from stencil_to_bf16 (FP32 arithmetic).
// err[0] = 2 if a bounded wait runs out.
bool stencil_pipe_supported(const Geom &g);
void stencil_apply_pipe(const float2 *in, float2 *out, const void *AT, bool bf16, Geom g, int nrhs, int *err,
                        cudaStream_t s);
void stencil_to_bf16(const float2 *AT32, void *ATB, int64_t count, cudaStream_t s);
// Streaming BF16 coarse stencil for 32 dofs per site and 1 .. 8 right-hand
// sides: one warp per site (per_site: one thread block per site, a warp per
// direction), the blocks in the row-chunked BF16 layout that
// stencil_to_stream builds from the transposed FP32 blocks (count complex
// entries); the same results as the BF16 pipelined kernel.
void stencil_apply_stream(const float2 *in, float2 *out, const void *AS, Geom g, int nrhs, bool per_site,
                          cudaStream_t s);
void stencil_to_stream(const float2 *AT32, void *AS, int64_t count, cudaStream_t s);
// AT = blockwise transpose of the canonical A[X][d][i][j] (nblocks = 9 V)
template <typename To>
void stencil_transpose(const double2 *A, C<To> *AT, int64_t nblocks, int m, cudaStream_t s);
// (<q, r>, <q, q>) for every rhs in one pass: out_qr[r], out_qq[r]
template <typename T>
void dot_qr(const C<T> *q, const C<T> *r, int64_t n, int nrhs, double2 *out_qr, double2 *out_qq,
            RedScratch scr, cudaStream_t s);
template <typename T>
void stencil_split(const C<T> *in, C<T> *out9, const C<T> *A, Geom g, const int b[4],
                   cudaStream_t s);
// soa: fine-level vectors in the structure-of-arrays order
template <typename T>
void gamma5_apply(const C<T> *in, C<T> *out, int64_t nsites, int dof, int nrhs, cudaStream_t s,
                  bool soa = false);

// ------------------------------------------------------------------ SAP
// blocks b tile the lattice with an even block count in every direction
bool sap_feasible(const Geom &g, const int b[4]);
template <typename T> size_t sap_smem_bytes(const int b[4], int rs);
// one red/black sweep: r (residual, exact on exit), z += correction, e scratch;
// FP32: structure-of-arrays vectors and links (UDs), FP64: canonical.
// variant 0: the staged FP32 block kernels where they apply (two or more
// right-hand sides, blocks 8 x 4 x 4 x 2 or 4^4), 1: the paired ones there,
// 2: the general kernels throughout; all give identical results
int sap_variants();
template <typename T>
void sap_sweep(C<T> *r, C<T> *z, C<T> *e, const C<T> *U, Geom g, const int b[4], double m0,
               int block_iters, int nrhs, cudaStream_t s, int variant = 0);

// ------------------------------------------------------------------ learned smoother
// gauge-covariant layer phi[o] = sum_c sum_h W[h][o][c] T_h psi[c]; activations
// [b][c] vectors of the fine level (FP32 structure-of-arrays with the links
// UDs, FP64 canonical [site][12] with U), weights [h][o][c][4][4]
template <typename T>
void glayer_forward(const C<T> *in, C<T> *out, const C<T> *W, const C<T> *U, Geom g, int Cin,
                    int Cout, int B, cudaStream_t s);
// input gradient: out[c] = sum_o sum_h W[h][o][c]^H T_rev(h) gin[o]
template <typename T>
void glayer_adjoint(const C<T> *gin, C<T> *out, const C<T> *W, const C<T> *U, Geom g, int Cin,
                    int Cout, int B, cudaStream_t s);
int glayer_wgrad_chunks(const Geom &g);
// out[h][o][c][16] = sum_b sum_x gin[b][o](x) (T_h in[b][c])(x)^H (colour summed)
template <typename T>
void glayer_wgrad(const C<T> *gin, const C<T> *in, const C<T> *U, Geom g, int Cin, int Cout, int B,
                  double2 *partial, double2 *out, cudaStream_t s);
// Adam (t = step count from 1) on complex weights given dL/dW* (times scale)
void adam_step(double2 *W, const double2 *grad, double2 *m, double2 *v, int64_t count, double lr,
               double b1, double b2, double eps, int t, double scale, cudaStream_t s);

// ------------------------------------------------------------------ transfer
// P is stored [X][c][k][row] (row fastest).
template <typename T>
void restrict_op(const C<T> *in, C<T> *out, const C<T> *P, const AggMap &m, int nrhs,
                 cudaStream_t s);
// out = P in (beta = 0) or out = beta * out + P in
template <typename T>
void prolong_op(const C<T> *in, C<T> *out, const C<T> *P, const AggMap &m, int nrhs, double beta,
                cudaStream_t s);
// the same with P stored as BF16 pairs (from stencil_to_bf16; relative
// rounding <= 2^-9 per entry, FP32 arithmetic): the transfers inside the
// multigrid preconditioner of FP32 solves
void restrict_op_bf16(const float2 *in, float2 *out, const void *P, const AggMap &m, int nrhs, cudaStream_t s);
void prolong_op_bf16(const float2 *in, float2 *out, const void *P, const AggMap &m, int nrhs, double beta,
                     cudaStream_t s);
// out = P e_col: column `col` of every aggregate's block (col = c * ntv + k)
void probe_column(double2 *out, const double2 *P, const AggMap &m, int col, cudaStream_t s);
// P from ntv test vectors V[k][n]: per (aggregate, chirality) modified
// Gram-Schmidt run twice in k order.  status[0] set to 1 on a zero norm.
void build_prolongator(const double2 *V, double2 *P, const AggMap &m, int *status,
                       cudaStream_t s);
// A[X][h][i][col] = cols[h][X * dof + i] for h = 0..8
void galerkin_scatter(const double2 *cols, double2 *A, Geom coarse, int col, cudaStream_t s);
// convert / transpose P to the canonical host order [X][c][row][k]
void prolongator_to_canonical(const double2 *P, double2 *out, const AggMap &m, cudaStream_t s);

// ------------------------------------------------------------------ noise
// Z4 noise, samples sample0 .. sample0 + nrhs - 1 (Philox4x64-10).  When
// slice >= 0 only entries of time slice `slice` are non-zero.
template <typename T>
void z4_noise(C<T> *out, Geom g, uint64_t seed, uint64_t sample0, uint64_t term, uint64_t aux,
              int slice, int nrhs, cudaStream_t s);
// per-slice dots: out[r][t] = sum_{i in slice t} conj(a_r[i]) b_r[i]
template <typename T>
void slice_dot(const C<T> *a, const C<T> *b, Geom g, int nrhs, double2 *out, cudaStream_t s);

// ------------------------------------------------------------------ dense
void dense_from_stencil(const double2 *A, double2 *M, Geom g, cudaStream_t s);
// in-place Gauss-Jordan inverse with partial pivoting of the n x n row-major
// M (work: 2 n^2 complex + n); status[0] = 1 on a zero pivot
void dense_invert(double2 *M, double2 *work, int n, int *status, cudaStream_t s);
void dense_trace(const double2 *M, int n, double2 *out, cudaStream_t s);

// ------------------------------------------------------------------ checks
// flag[0] = 1 when any entry of x is NaN / Inf
template <typename T>
void check_finite(const C<T> *x, int64_t n, int *flag, cudaStream_t s);

}  // namespace mg
