// Host orchestration of the multigrid hierarchy, the batched MG-preconditioned
// FGMRES level solves and the MG-MLMC estimators.  Everything numeric runs in
// the kernels of kernels.h on one stream; the host holds scalars only.
#pragma once

#include <complex>
#include <map>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/mgmlmc.h"
#include "kernels.h"

namespace mg {

struct Level {
  Geom g{};
  bool fine = false;
  double2 *U64 = nullptr;  // fine links [V][4][3][3]
  float2 *UD32 = nullptr;  // FP32 links structure-of-arrays [4][3][3][V] (FP32 kernels)
  float *Ub16 = nullptr;   // bf16 links structure-of-arrays (one bf16 pair per float slot)
  double2 *A64 = nullptr;   // coarse stencil, canonical [V][9][dof][dof]
  double2 *AT64 = nullptr;  // the same blocks transposed [V][9][j][i] (apply)
  float2 *AT32 = nullptr;
  float *ATC = nullptr;     // tensor-core tiles (32 dofs per site only), see stencil_tile_tc
  void *ATCB = nullptr;     // the same tiles in BF16 (kind::f16 MMAs)
  float *ATB16 = nullptr;   // AT32 as bf16 pairs (32 dofs per site only), preconditioner variant
  float *ATS = nullptr;     // the same BF16 pairs row-chunked for the streaming kernel (variant 6)
  bool has_next = false;
  AggMap agg{};            // to level + 1
  double2 *P64 = nullptr;  // [X][c][k][row]
  float2 *P32 = nullptr;
  float *PB16 = nullptr;   // P32 as bf16 pairs (transfer variant 1)
  double2 *Dinv64 = nullptr;  // coarsest: dense inverse, row-major
  float2 *Dinv32 = nullptr;
};

struct SolveInfo {
  int iters = 0;          // outer iterations (max over rhs)
  double residual = 0.0;  // true relative residual (max over rhs)
  bool converged = true;
};

struct TermAcc {
  int term = 0;
  int n = 0;
  double sre = 0, sim = 0, sabs2 = 0;
  double seconds = 0;
  double iters_sum = 0;
  int solves = 0;
  double max_res = 0;
  std::vector<std::complex<double>> samples;
};

// Per-kernel-class timing collected with CUDA events on the engine's stream
// while profiling is enabled (mgmlmc_profile).
enum KClass {
  K_WILSON64 = 0,
  K_WILSON32 = 1,
  K_STENCIL64 = 2,
  K_STENCIL32 = 3,
  K_SAP64 = 4,
  K_SAP32 = 5,
  K_TRANSFER = 6,   // restriction + prolongation inside the cycle
  K_ORTHO = 7,      // Gram-Schmidt of the FGMRES basis (all levels)
  K_NET = 8,        // learned step (network forward)
  K_COARSEST = 9,   // dense coarsest-level apply inside the cycle
  K_NCLASS = 12
};
struct KStat {
  int64_t launches = 0;
  double ms = 0.0;
  double bytes = 0.0;  // algorithmic bytes
  double flops = 0.0;  // algorithmic flops
};

// Learned smoother: three gauge-covariant layers, channels 1 -> C -> C -> 1.
struct Net {
  int C = 0;
  int cin[3] = {0, 0, 0}, cout[3] = {0, 0, 0};
  int64_t cnt[3] = {0, 0, 0};  // complex weights per layer
  double2 *W64[3] = {nullptr, nullptr, nullptr};
  float2 *W32[3] = {nullptr, nullptr, nullptr};
  double2 *m[3] = {nullptr, nullptr, nullptr};
  double2 *v[3] = {nullptr, nullptr, nullptr};
  int adam_t = 0;
  int64_t fallbacks = 0;
};

class Engine {
 public:
  Engine(const int dims[4], cudaStream_t s);
  ~Engine();
  Engine(const Engine &) = delete;
  Engine &operator=(const Engine &) = delete;

  void set_gauge(const double *U, bool on_device);
  void get_gauge(double *U, bool on_device);
  // U = exp(i eps H) generated on the device (kernels.h gauge_generate)
  void gen_gauge(double eps, uint64_t seed);
  void set_mass(double m0);
  void set_solver(const mgmlmc_solver_params &p);
  void set_test_vectors(int level, const double *V, int ntv, int64_t n, bool on_device);
  void build_hierarchy(const mgmlmc_mg_params &p);

  int n_levels() const { return (int)levels_.size(); }
  const Level &level(int l) const { return levels_.at(l); }
  bool ready() const { return ready_; }

  // operator hooks (device buffers)
  template <typename T> void apply_D(int l, const C<T> *in, C<T> *out, int nrhs);
  // level-0 D on complex-bf16 vectors in the chunked internal order
  void apply_D_bf16(const void *in, void *out, int nrhs);
  template <typename T> void restrict_to(int l, const C<T> *in, C<T> *out, int nrhs);
  template <typename T> void prolong_from(int l, const C<T> *in, C<T> *out, int nrhs, double beta);
  template <typename T> void project_out(int l, const C<T> *in, C<T> *out, int nrhs);
  template <typename T> void smooth_apply(int l, const C<T> *in, C<T> *out, int nrhs);
  // z = D_l^-1 b (FP64 interface; the solver precision is set by set_solver)
  SolveInfo solve(int l, const double2 *b, double2 *x, int nrhs);
  void noise(int l, uint64_t seed, uint64_t sample0, uint64_t term, uint64_t aux, int slice,
             double2 *out, int nrhs);

  void estimate_trace(const mgmlmc_est_params &p, std::vector<TermAcc> &out);
  void coarsest_trace(double *re, double *im);
  void connected(int kind, int n_samples, uint64_t seed, uint64_t first, std::vector<double> &mean,
                 std::vector<double> &var, int &R);
  void disconnected(int kind, int t, int n_samples, uint64_t seed, uint64_t first,
                    std::vector<double> &mean, std::vector<double> &var, int &R);

  // learned smoother
  void net_init(int channels, uint64_t seed);
  int64_t net_size() const;
  void net_weights(double *host, bool set);
  template <typename T> void net_forward(const C<T> *in, C<T> *out, int B);
  // loss sum_b ||r_b - D N(r_b)||^2 / ||r_b||^2 and dL/dW* (device, [layer][cnt])
  template <typename T> double net_loss_grad(const C<T> *r, int B, double2 *grad);
  void net_train(const mgmlmc_train_params &p, mgmlmc_train_result &out);
  int64_t net_fallbacks() const { return net_.fallbacks; }

  // inexact deflation (Eq. deflated-estimator): V_k by `iters` inverse block
  // power steps on Gamma5 D with inner solves to tol, then the exact part
  // tr(V^H D^-1 V) at the solver's tolerance
  void deflation_build(int k, int iters, double tol, uint64_t seed, std::complex<double> &exact,
                       double &seconds);
  int deflation_k() const { return defl_k_; }

  // test vectors of level l refined toward the low eigenvectors of
  // Q_l = Gamma5_l D_l (Sec. 2.2 setup phase, Sec. 5): block of m >= N_tv
  // columns, at most `iters` simultaneous inverse-iteration steps with the
  // Ritz step on Q_l^-2 and FP64 solves to solve_tol, stopping once every
  // returned column has ||Q v - theta v|| <= tol (tol > 0); the hierarchy is
  // then rebuilt from them.  theta / rho / steps: Rayleigh quotients and
  // eigen-residuals of the N_tv returned columns, steps taken.
  void refine_test_vectors(int l, int m, int iters, double tol, double solve_tol, uint64_t seed,
                           std::vector<double> &theta, std::vector<double> &rho, int &steps);

  void get_prolongator(int l, double *host);
  void get_test_vectors(int l, double *host);
  void get_coarse_op(int l, double *host);

  SolveInfo last_solve;
  cudaStream_t stream = nullptr;       // internal non-blocking stream: all work runs here
  void *blas_ = nullptr;               // cuBLAS handle bound to `stream` (the coarsest-level GEMM)
  void *blas_ws_ = nullptr;            // its fixed workspace, so that it can run under graph capture
  cudaStream_t user_stream = nullptr;  // the caller's stream given at creation
  // order the internal stream after the caller's earlier work / the caller's
  // stream after ours (every API call is bracketed by these)
  void enter();
  void leave();
  void set_graphs(bool on) { graphs_on_ = on; if (!on) drop_graphs(); }
  // free every workspace (and the graphs that use them) except the levels'
  // test vectors; later calls allocate what they need again
  void release_workspaces();
  // MGMLMC_ERR_CUDA (and the flag cleared) if a coarse-stencil kernel's
  // bounded staging wait ran out since the last check; synchronises
  void check_staging();

  void profile(bool on);
  KStat kstat(int cls);
  // engine-owned FP32 scratch on level 0 (reordering caller vectors)
  float2 *scratch32(const std::string &name, size_t count) { return ws<float>(name, 0, count); }

  // FP32 Dslash kernel variant per rhs count: -2 = autotune on the first call
  // outside graph capture (every variant timed on that call's operands, the
  // fastest kept), 0 .. wilson_fp32_variants() - 1 = fixed
  void set_dslash_variant(int v);
  int dslash_variant(int nrhs) const;
  // FP32 coarse stencil per rhs count: 0 = FP32 CUDA cores, 1 = tcgen05
  // TF32 with M = 64 MMAs, 2 = the same with M = 128 MMAs, 3 = BF16-stored
  // blocks with FP32 arithmetic, 4 = tcgen05 with BF16 operands, -2 = the
  // fastest of 0, 1, 3, 4, 5, 6, 7 on the first call outside capture; 5 =
  // variant 4 as a persistent pipelined kernel (up to 32 right-hand sides);
  // 6 = variant 3's arithmetic with one warp per site streaming the blocks
  // (up to 8 right-hand sides; identical results to 3); 7 = 6 with one
  // thread block per site, a warp per direction (small coarse lattices)
  void set_stencil_variant(int v);
  int stencil_variant(int l, int nrhs) const;
  static int stencil_variants();
  // FP32 SAP sweep: 0 = the staged block kernels where they apply, 1 = the
  // paired ones, 2 = the general ones (identical results)
  void set_sap_variant(int v);
  int sap_variant() const { return sap_variant_; }
  // FP32 restriction / prolongation (mgmlmc_apply and the multigrid
  // preconditioner; never the projector): 0 = P in FP32, 1 = P stored as BF16
  void set_transfer_variant(int v);
  int transfer_variant() const { return transfer_variant_; }

 private:
  template <typename T> C<T> *ws(const std::string &name, int l, size_t count);
  // free one named workspace (only for buffers no captured graph uses)
  void ws_release(const std::string &name, int l, bool dbl);
  void contraction_vectors(int kind, int nb, double2 *x, double2 *B, double2 *Bt);
  template <typename T> const C<T> *Pmat(int l) const;
  // the aggregation map of level l for vectors of type T (FP32 level-0
  // vectors are structure-of-arrays)
  template <typename T> AggMap agg_of(int l) const;
  template <typename T> const C<T> *Dinv(int l) const;

  template <typename T> void smooth(int l, C<T> *z, C<T> *res, int nrhs);
  template <typename T> void precond(int l, const C<T> *r, C<T> *z, int nrhs);
  // out = Minv in for the dense coarsest-level inverse (n x n, row-major) and
  // nrhs vectors of n: one complex GEMM in cuBLAS (FP32 or FP64 arithmetic,
  // no reduced-precision math mode)
  template <typename T> void coarsest_apply(const C<T> *Minv, const C<T> *in, C<T> *out, int n, int nrhs);
  // the preconditioner of an outer solve: replayed from a CUDA graph captured
  // once per (level, nrhs, precision, operand addresses) unless profiling or
  // graphs are off
  template <typename T> void precond_top(int l, const C<T> *r, C<T> *z, int nrhs);
  // batched FGMRES; fixed = run exactly max_iter iterations with no host check
  template <typename T>
  // stall_exit: stop once a restart cycle fails to halve the true residual
  SolveInfo fgmres(int l, const C<T> *b, C<T> *x, int nrhs, double tol, int max_iter, int m,
                   bool use_precond, bool fixed, bool stall_exit = false);
  int restart_of(int l) const;  // FGMRES restart length of level l's solves
  SolveInfo solve_mixed(int l, const double2 *b, double2 *x, int nrhs);
  void galerkin(int l);
  void setup_test_vectors(int l, double2 *V, int ntv, const mgmlmc_mg_params &p);
  // larger test-vector sets are not kept after the build (see build_hierarchy)
  static constexpr double kKeepTestVectorBytes = 8e9;
  void free_hierarchy();
  void release();  // frees everything the context holds; safe on a partly built one
  void gauge_derived();  // FP32 and structure-of-arrays copies of the new links
  void sync();

  int dims_[4];
  Geom fine_{};
  int sap_b_[4] = {0, 0, 0, 0};  // SAP block extents (0: SAP not possible)
  double m0_ = 0.0;
  bool have_gauge_ = false;
  bool ready_ = false;
  mgmlmc_solver_params sp_{};
  bool guess_off_ = false;  // the learned guess skips the solve in progress (F_l fine solves)
  std::vector<Level> levels_;
  std::map<int, std::vector<double>> imported_host_;  // level -> ntv * n complex
  mgmlmc_mg_params mgp_{};  // parameters of the last successful build
  std::map<std::string, std::pair<void *, size_t>> ws_;
  double2 *scal_ = nullptr;     // small scalar scratch
  double2 *partial_ = nullptr;  // reduction partials
  unsigned *tickets_ = nullptr;  // reduction tickets (kTickets, zero between calls)
  size_t partial_cap_ = 0;
  int *flag_dev_ = nullptr;
  static constexpr size_t kPinnedBytes = 1 << 20;
  static constexpr size_t kBlasWorkspace = 32u << 20;
  void *pinned_ = nullptr;
  size_t pinned_cap_ = 0;
  void *pinned(size_t bytes);
  bool prof_ = false;
  struct Pending { int cls; cudaEvent_t a, b; double bytes, flops; };
  std::vector<Pending> pending_;
  std::vector<cudaEvent_t> events_;
  KStat kst_[K_NCLASS];
  cudaEvent_t take_event();
  void prof_resolve();
  // event pair around a launch sequence of one kernel class (no-op unless profiling)
  cudaEvent_t prof_begin();
  void prof_end(cudaEvent_t a, int cls, double bytes, double flops);
  RedScratch partials(size_t count);
  Net net_;
  void net_free();
  bool recording_ = false;    // copy level-0 post-smoother inputs into the training pool
  bool post_smooth_ = false;  // set while the post-smoother of a cycle runs
  float2 *pool_ = nullptr;    // [pool_cap][n0] FP32
  int pool_n_ = 0, pool_cap_ = 0;
  template <typename T> void record(const C<T> *res, int nrhs);
  bool graphs_on_ = true;
  bool capturing_ = false;
  struct GraphEntry {
    cudaGraphExec_t exec;
    int64_t kernels;  // kernel nodes in the graph
  };
  // (level, nrhs, sizeof(T), input, output) -> captured preconditioner
  std::map<std::tuple<int, int, int, const void *, void *>, GraphEntry> graphs_;
  void drop_graphs();
  cudaEvent_t ev_enter_ = nullptr, ev_leave_ = nullptr;
  int dslash_force_ = -2;
  double2 *defl_V_ = nullptr;  // [k][n0] orthonormal columns
  int defl_k_ = 0;
  std::complex<double> defl_exact_{0.0, 0.0};
  double defl_seconds_ = 0.0;
  void orthonormalise_cols(double2 *V, int k, int64_t n);
  std::map<int, int> dslash_tuned_;
  int stencil_force_ = 0;
  int sap_variant_ = 0;
  int transfer_variant_ = 0;
  int precond_depth_ = 0;  // > 0 while the multigrid preconditioner runs
  int solving_ = 0;        // > 0 inside solve()
  std::map<std::pair<int, int>, int> stencil_tuned_;  // (level, nrhs) -> variant
  int stencil_pick(int l, int nrhs, const float2 *in, float2 *out);
  void stencil_run(int l, int v, const float2 *in, float2 *out, int nrhs);
  int dslash_pick(int nrhs, const float2 *in, float2 *out);
};

}  // namespace mg
