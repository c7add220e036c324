// Host orchestration: hierarchy construction (Sec. 2.2 and Sec. 4: test
// vectors, aggregation-based P_l with P_l^H P_l = I, Galerkin D_{l+1}),
// the batched MG-preconditioned FGMRES level solves (the role DD-alpha-AMG
// plays in Sec. 4: every level solved to a relative residual), and the
// estimators of Sec. 3 / Sec. 4.
#include "engine.h"
#include "herm_eig.h"

#include <cublas_v2.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>

namespace mg {

namespace {
template <typename T> T *dalloc(size_t count) {
  void *p = nullptr;
  MG_CUDA(cudaMalloc(&p, count * sizeof(T) + 64));
  return static_cast<T *>(p);
}
template <typename T> void dfree(T *&p) {
  if (p) cudaFree(p);
  p = nullptr;
}
// a pair of timing events, destroyed on every exit (a failed step throws)
struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  EventPair() {
    MG_CUDA(cudaEventCreate(&a));
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      throw Error(MGMLMC_ERR_CUDA, "cudaEventCreate failed");
    }
  }
  ~EventPair() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
  EventPair(const EventPair &) = delete;
  EventPair &operator=(const EventPair &) = delete;
};
// a device buffer freed on every exit
template <typename T> struct DevBuf {
  T *p = nullptr;
  explicit DevBuf(size_t count) : p(dalloc<T>(count)) {}
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
};

__global__ void target_kernel(double *target, const double2 *nrm, double tol, int nrhs) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nrhs) target[r] = tol * sqrt(fmax(nrm[r].x, 0.0));
}
__global__ void inv_norm_kernel(double *out, double *nrm_out, const double2 *nrm, int nrhs) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nrhs) {
    const double v = sqrt(fmax(nrm[r].x, 0.0));
    out[r] = v > 0.0 ? 1.0 / v : 0.0;
    nrm_out[r] = v;
  }
}
}  // namespace

Engine::Engine(const int dims[4], cudaStream_t s) : user_stream(s) {
  // validate before acquiring anything: a throwing constructor runs no destructor
  for (int i = 0; i < 4; ++i)
    if (dims[i] < 2) throw Error(MGMLMC_ERR_ARG, "lattice extents must be >= 2");
  const int64_t V = (int64_t)dims[0] * dims[1] * dims[2] * dims[3];
  // sites are int, and 12 V must index a vector with int arithmetic in places
  if (V * 12 >= ((int64_t)1 << 31)) throw Error(MGMLMC_ERR_ARG, "lattice too large (12 V >= 2^31)");
  for (int i = 0; i < 4; ++i) {
    dims_[i] = dims[i];
    fine_.L[i] = dims[i];
  }
  fine_.V = (int)V;
  fine_.dof = 12;
  sp_.tol = 1e-12;
  sp_.max_iter = 2000;
  sp_.restart = 16;
  sp_.smoother_steps = 4;
  sp_.coarse_iters = 8;
  sp_.precision = MGMLMC_FP64;
  sp_.inner_tol = 1e-6;
  sp_.smoother = MGMLMC_SMOOTHER_MR;
  sp_.sap_iters = 4;
  sp_.coarse_smoother_steps = 4;
  // SAP blocks of 256 sites, 8 x 4 x 4 x 2, when every direction holds an
  // even number of them: a block's x rows are then 128 bytes per FP32
  // structure-of-arrays chunk and 64 bytes per link plane, whole memory
  // bursts (the 4-site rows of 4^4 blocks use half of each burst, the other
  // half belonging to the neighbouring block of the other colour); else 4^4,
  // else 2^4
  const int shapes[3][4] = {{8, 4, 4, 2}, {4, 4, 4, 4}, {2, 2, 2, 2}};
  for (const auto &b : shapes) {
    if (sap_feasible(fine_, b)) {
      for (int i = 0; i < 4; ++i) sap_b_[i] = b[i];
      break;
    }
  }
  levels_.resize(1);
  levels_[0].g = fine_;
  levels_[0].fine = true;
  // a throwing constructor runs no destructor: release what was acquired
  try {
    MG_CUDA(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
    {
      cublasHandle_t h = nullptr;
      if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) throw Error(MGMLMC_ERR_CUDA, "cublasCreate failed");
      blas_ = h;
      MG_CUDA(cudaMalloc(&blas_ws_, kBlasWorkspace));
      if (cublasSetStream(h, stream) != CUBLAS_STATUS_SUCCESS ||
          cublasSetWorkspace(h, blas_ws_, kBlasWorkspace) != CUBLAS_STATUS_SUCCESS)
        throw Error(MGMLMC_ERR_CUDA, "cuBLAS stream or workspace setup failed");
    }
    MG_CUDA(cudaEventCreateWithFlags(&ev_enter_, cudaEventDisableTiming));
    MG_CUDA(cudaEventCreateWithFlags(&ev_leave_, cudaEventDisableTiming));
    levels_[0].U64 = dalloc<double2>((size_t)V * 36);
    levels_[0].UD32 = dalloc<float2>((size_t)V * 36);
    levels_[0].Ub16 = dalloc<float>((size_t)V * 36);  // 36 bf16 pairs of 4 bytes per site
    scal_ = dalloc<double2>(4096);
    flag_dev_ = dalloc<int>(16);
    MG_CUDA(cudaMemset(flag_dev_, 0, 16 * sizeof(int)));
    tickets_ = dalloc<unsigned>(kTickets);
    MG_CUDA(cudaMemset(tickets_, 0, kTickets * sizeof(unsigned)));
  } catch (...) {
    release();
    throw;
  }
}

Engine::~Engine() { release(); }

void Engine::release() {
  if (stream) cudaStreamSynchronize(stream);
  if (blas_) cublasDestroy(static_cast<cublasHandle_t>(blas_));
  blas_ = nullptr;
  if (blas_ws_) cudaFree(blas_ws_);
  blas_ws_ = nullptr;
  free_hierarchy();
  net_free();
  if (pool_) cudaFree(pool_);
  pool_ = nullptr;
  dfree(levels_[0].U64);
  dfree(levels_[0].UD32);
  dfree(levels_[0].Ub16);
  for (auto &kv : ws_) cudaFree(kv.second.first);
  ws_.clear();
  for (auto &p : pending_) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  pending_.clear();
  for (auto e : events_) cudaEventDestroy(e);
  events_.clear();
  dfree(scal_);
  dfree(partial_);
  dfree(tickets_);
  dfree(flag_dev_);
  if (pinned_) cudaFreeHost(pinned_);
  pinned_ = nullptr;
  if (ev_enter_) cudaEventDestroy(ev_enter_);
  if (ev_leave_) cudaEventDestroy(ev_leave_);
  ev_enter_ = ev_leave_ = nullptr;
  if (stream) cudaStreamDestroy(stream);
  stream = nullptr;
}

void Engine::enter() {
  MG_CUDA(cudaEventRecord(ev_enter_, user_stream));
  MG_CUDA(cudaStreamWaitEvent(stream, ev_enter_, 0));
}

void Engine::leave() {
  MG_CUDA(cudaEventRecord(ev_leave_, stream));
  MG_CUDA(cudaStreamWaitEvent(user_stream, ev_leave_, 0));
}

void Engine::drop_graphs() {
  if (graphs_.empty()) return;
  cudaStreamSynchronize(stream);
  for (auto &kv : graphs_) cudaGraphExecDestroy(kv.second.exec);
  graphs_.clear();
}

void Engine::sync() {
  MG_CUDA(cudaStreamSynchronize(stream));
  if (!pending_.empty()) prof_resolve();
}

cudaEvent_t Engine::take_event() {
  if (events_.empty()) {
    cudaEvent_t e;
    MG_CUDA(cudaEventCreate(&e));
    return e;
  }
  cudaEvent_t e = events_.back();
  events_.pop_back();
  return e;
}

void Engine::prof_resolve() {
  for (const Pending &p : pending_) {
    float ms = 0.f;
    MG_CUDA(cudaEventElapsedTime(&ms, p.a, p.b));
    KStat &k = kst_[p.cls];
    k.launches += 1;
    k.ms += ms;
    k.bytes += p.bytes;
    k.flops += p.flops;
    events_.push_back(p.a);
    events_.push_back(p.b);
  }
  pending_.clear();
}

cudaEvent_t Engine::prof_begin() {
  if (!prof_ || capturing_) return nullptr;
  cudaEvent_t a = take_event();
  MG_CUDA(cudaEventRecord(a, stream));
  return a;
}

void Engine::prof_end(cudaEvent_t a, int cls, double bytes, double flops) {
  if (!a) return;
  cudaEvent_t b = take_event();
  MG_CUDA(cudaEventRecord(b, stream));
  pending_.push_back({cls, a, b, bytes, flops});
}

void Engine::profile(bool on) {
  sync();
  prof_ = on;
  for (auto &k : kst_) k = KStat{};
}

KStat Engine::kstat(int cls) {
  if (cls < 0 || cls >= K_NCLASS) throw Error(MGMLMC_ERR_ARG, "kernel class out of range");
  sync();
  return kst_[cls];
}

// One pinned staging buffer of fixed size, allocated once: callers may keep
// the pointer across nested solver calls (it is never reallocated).  Every
// use copies, synchronises and consumes before the next use.
void *Engine::pinned(size_t bytes) {
  if (!pinned_) {
    MG_CUDA(cudaMallocHost(&pinned_, kPinnedBytes));
    pinned_cap_ = kPinnedBytes;
  }
  if (bytes > pinned_cap_) throw Error(MGMLMC_ERR_ARG, "too many right-hand sides for the staging buffer");
  return pinned_;
}

RedScratch Engine::partials(size_t count) {
  if (count > partial_cap_) {
    if (capturing_) throw Error(MGMLMC_ERR_STATE, "reduction scratch growth during graph capture");
    drop_graphs();
    sync();
    dfree(partial_);
    partial_ = dalloc<double2>(count);
    partial_cap_ = count;
  }
  return RedScratch{partial_, tickets_};
}

template <typename T> C<T> *Engine::ws(const std::string &name, int l, size_t count) {
  const std::string key = name + "#" + std::to_string(l) + (sizeof(T) == 8 ? "d" : "f");
  const size_t bytes = count * sizeof(C<T>);
  auto it = ws_.find(key);
  if (it != ws_.end() && it->second.second >= bytes) return static_cast<C<T> *>(it->second.first);
  if (it != ws_.end()) {
    if (capturing_) throw Error(MGMLMC_ERR_STATE, "workspace growth during graph capture");
    drop_graphs();  // captured graphs may reference the old buffer
    sync();
    cudaFree(it->second.first);
    ws_.erase(it);
  }
  void *p = nullptr;
  MG_CUDA(cudaMalloc(&p, bytes + 256));
  ws_[key] = {p, bytes};
  return static_cast<C<T> *>(p);
}

void Engine::ws_release(const std::string &name, int l, bool dbl) {
  const std::string key = name + "#" + std::to_string(l) + (dbl ? "d" : "f");
  auto it = ws_.find(key);
  if (it == ws_.end()) return;
  drop_graphs();  // a captured graph may hold the buffer's address
  sync();
  cudaFree(it->second.first);
  ws_.erase(it);
}

template <> const C<double> *Engine::Pmat<double>(int l) const { return levels_[l].P64; }
template <> const C<float> *Engine::Pmat<float>(int l) const { return levels_[l].P32; }
template <> const C<double> *Engine::Dinv<double>(int l) const { return levels_[l].Dinv64; }
template <> const C<float> *Engine::Dinv<float>(int l) const { return levels_[l].Dinv32; }

// ------------------------------------------------------------------ inputs
void Engine::set_gauge(const double *U, bool on_device) {
  const size_t cnt = (size_t)fine_.V * 36;
  MG_CUDA(cudaMemcpyAsync(levels_[0].U64, U, cnt * sizeof(double2),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, stream));
  MG_CUDA(cudaMemsetAsync(flag_dev_, 0, sizeof(int), stream));
  check_finite<double>(levels_[0].U64, (int64_t)cnt, flag_dev_, stream);
  int flag = 0;
  MG_CUDA(cudaMemcpyAsync(&flag, flag_dev_, sizeof(int), cudaMemcpyDeviceToHost, stream));
  sync();
  if (flag) {
    have_gauge_ = false;
    throw Error(MGMLMC_ERR_NUMERIC, "gauge field contains NaN or Inf");
  }
  gauge_derived();
}

void Engine::get_gauge(double *U, bool on_device) {
  if (!have_gauge_) throw Error(MGMLMC_ERR_STATE, "no gauge field");
  MG_CUDA(cudaMemcpyAsync(U, levels_[0].U64, (size_t)fine_.V * 36 * sizeof(double2),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, stream));
  sync();
}

void Engine::gen_gauge(double eps, uint64_t seed) {
  if (!std::isfinite(eps)) throw Error(MGMLMC_ERR_ARG, "eps must be finite");
  gauge_generate(levels_[0].U64, (int64_t)fine_.V * 4, eps, seed, stream);
  gauge_derived();
}

void Engine::gauge_derived() {
  const size_t cnt = (size_t)fine_.V * 36;
  // the canonical FP32 links are only the intermediate of the two layouts the
  // FP32 and BF16 kernels read
  DevBuf<float2> u32(cnt);
  convert<float, double>(levels_[0].U64, u32.p, (int64_t)cnt, stream);
  link_soa(u32.p, levels_[0].UD32, fine_.V, stream);
  link_bf16(u32.p, levels_[0].Ub16, fine_.V, stream);
  sync();
  have_gauge_ = true;
  free_hierarchy();
}

void Engine::set_mass(double m0) {
  if (!std::isfinite(m0)) throw Error(MGMLMC_ERR_ARG, "mass must be finite");
  m0_ = m0;
  free_hierarchy();
}

int Engine::restart_of(int l) const {
  return (l > 0 && sp_.coarse_restart > 0) ? sp_.coarse_restart : sp_.restart;
}

void Engine::set_solver(const mgmlmc_solver_params &p) {
  if (!(p.tol > 0.0) || p.max_iter < 1 || p.restart < 1 || p.restart > 64 || p.smoother_steps < 0 ||
      p.coarse_restart < 0 || p.coarse_restart > 64 || (p.post_smoothing_only != 0 && p.post_smoothing_only != 1) ||
      p.gram_schmidt_passes < 0 || p.gram_schmidt_passes > 2 ||
      p.coarse_iters < 1 || p.coarse_iters > 64 ||
      (p.precision != MGMLMC_FP64 && p.precision != MGMLMC_FP32) ||
      (p.precision == MGMLMC_FP32 && !(p.inner_tol > 0.0 && p.inner_tol < 1.0)) ||
      (p.smoother != MGMLMC_SMOOTHER_MR && p.smoother != MGMLMC_SMOOTHER_SAP &&
       p.smoother != MGMLMC_SMOOTHER_LEARNED && p.smoother != MGMLMC_SMOOTHER_NET) || p.sap_iters < 1 ||
      p.coarse_smoother_steps < 0 ||
      p.sap_iters > 64 || p.fine_batch < 0 || (p.learned_guess != 0 && p.learned_guess != 1))
    throw Error(MGMLMC_ERR_ARG, "invalid solver parameters");
  drop_graphs();  // captured preconditioners bake in smoother / inner iteration counts
  sp_ = p;
}

void Engine::set_test_vectors(int level, const double *V, int ntv, int64_t n, bool on_device) {
  if (level < 0 || level >= MGMLMC_MAX_LEVELS - 1 || ntv < 1 || ntv > 128 || n < 1 || !V)
    throw Error(MGMLMC_ERR_ARG, "set_test_vectors: bad level, count, length or pointer");
  std::vector<double> &h = imported_host_[level];
  h.assign((size_t)ntv * n * 2, 0.0);
  MG_CUDA(cudaMemcpyAsync(h.data(), V, h.size() * sizeof(double),
                          on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, stream));
  sync();
  free_hierarchy();
}

void Engine::free_hierarchy() {
  drop_graphs();
  for (size_t l = 0; l < levels_.size(); ++l) {
    Level &L = levels_[l];
    dfree(L.P64);
    dfree(L.P32);
    dfree(L.PB16);
    dfree(L.Dinv64);
    dfree(L.Dinv32);
    if (l > 0) {
      dfree(L.A64);
      dfree(L.AT64);
      dfree(L.AT32);
      dfree(L.ATC);
      if (L.ATCB) cudaFree(L.ATCB);
      L.ATCB = nullptr;
      dfree(L.ATB16);
      dfree(L.ATS);
    }
    L.has_next = false;
  }
  levels_.resize(1);
  ready_ = false;
  dfree(defl_V_);
  defl_V_ = nullptr;
  defl_k_ = 0;
}

// ------------------------------------------------------------------ operators
void Engine::set_dslash_variant(int v) {
  const int nv = wilson_fp32_variants();
  if (v < -2 || v == -1 || v >= nv) throw Error(MGMLMC_ERR_ARG, "dslash variant out of range");
  dslash_force_ = v;
  dslash_tuned_.clear();
  drop_graphs();
}

int Engine::dslash_variant(int nrhs) const {
  if (dslash_force_ != -2) return dslash_force_;
  auto it = dslash_tuned_.find(nrhs);
  return it == dslash_tuned_.end() ? -2 : it->second;
}

int Engine::stencil_variants() { return 8; }

void Engine::set_transfer_variant(int v) {
  if (v < 0 || v > 1) throw Error(MGMLMC_ERR_ARG, "transfer variant out of range");
  transfer_variant_ = v;
  drop_graphs();
}

void Engine::set_sap_variant(int v) {
  if (v < 0 || v >= sap_variants()) throw Error(MGMLMC_ERR_ARG, "SAP variant out of range");
  sap_variant_ = v;
  drop_graphs();
}

void Engine::set_stencil_variant(int v) {
  if (v < -2 || v == -1 || v >= stencil_variants()) throw Error(MGMLMC_ERR_ARG, "stencil variant out of range");
  stencil_force_ = v;
  stencil_tuned_.clear();
  drop_graphs();
}

int Engine::stencil_variant(int l, int nrhs) const {
  if (stencil_force_ != -2) return stencil_force_;
  auto it = stencil_tuned_.find({l, nrhs});
  return it == stencil_tuned_.end() ? -2 : it->second;
}

// 0: FP32 (the pipelined kernel where it applies, same sums as the
// one-site-per-CTA kernels); 1, 2: tensor cores (TF32); 3: BF16-stored
// blocks, FP32 arithmetic (pipelined kernel, up to 8 right-hand sides);
// 4: tensor cores with BF16 operands; 5: 4 as a persistent pipelined kernel;
// 6: 3's sums with one warp per site streaming the row-chunked blocks;
// 7: 6 with one thread block per site (a warp per direction)
void Engine::stencil_run(int l, int v, const float2 *in, float2 *out, int nrhs) {
  const Level &L = levels_[l];
  const bool pipe = stencil_pipe_supported(L.g) && nrhs <= 8;
  if ((v == 1 || v == 2) && L.ATC) stencil_apply_tc(in, out, L.ATC, L.g, nrhs, flag_dev_ + 1, v - 1, stream);
  else if (v == 4 && L.ATCB) stencil_apply_tc(in, out, L.ATCB, L.g, nrhs, flag_dev_ + 1, 2, stream);
  else if (v == 5 && L.ATCB) stencil_apply_tc(in, out, L.ATCB, L.g, nrhs, flag_dev_ + 1, 3, stream);
  else if (v == 3 && L.ATB16 && pipe) stencil_apply_pipe(in, out, L.ATB16, true, L.g, nrhs, flag_dev_ + 1, stream);
  else if ((v == 6 || v == 7) && L.ATS && nrhs <= 8) stencil_apply_stream(in, out, L.ATS, L.g, nrhs, v == 7, stream);
  else if (pipe) stencil_apply_pipe(in, out, L.AT32, false, L.g, nrhs, flag_dev_ + 1, stream);
  else stencil_apply<float>(in, out, L.AT32, L.g, nrhs, flag_dev_ + 1, stream);
}

// the tensor-core variants compute TF32 products, so the variant changes the
// numbers: autotuning (-2) is an opt-in; every variant is timed on the
// caller's operands and the fastest kept per (level, nrhs)
int Engine::stencil_pick(int l, int nrhs, const float2 *in, float2 *out) {
  // inside a solve the variant serves the multigrid preconditioner only;
  // every FGMRES keeps the FP32 stencil as its Krylov operator
  if (solving_ > 0 && precond_depth_ == 0) return 0;
  if (stencil_force_ != -2) return levels_[l].ATC ? stencil_force_ : 0;
  if (!levels_[l].ATC) return 0;
  auto it = stencil_tuned_.find({l, nrhs});
  if (it != stencil_tuned_.end()) return it->second;
  if (capturing_) return 0;
  EventPair ev;
  int pick = 0;
  float best = 1e30f;
  // variant 2 is variant 1 with twice the tensor work: not a candidate
  for (int v : {0, 1, 3, 4, 5, 6, 7}) {
    if (v == 3 && !(levels_[l].ATB16 && nrhs <= 8)) continue;
    if ((v == 6 || v == 7) && !(levels_[l].ATS && nrhs <= 8)) continue;
    stencil_run(l, v, in, out, nrhs);
    MG_CUDA(cudaEventRecord(ev.a, stream));
    for (int rep = 0; rep < 3; ++rep) stencil_run(l, v, in, out, nrhs);
    MG_CUDA(cudaEventRecord(ev.b, stream));
    MG_CUDA(cudaEventSynchronize(ev.b));
    float ms = 0.f;
    MG_CUDA(cudaEventElapsedTime(&ms, ev.a, ev.b));
    if (ms < best) { best = ms; pick = v; }
  }
  stencil_tuned_[{l, nrhs}] = pick;
  return pick;
}

int Engine::dslash_pick(int nrhs, const float2 *in, float2 *out) {
  if (dslash_force_ != -2) return dslash_force_;
  auto it = dslash_tuned_.find(nrhs);
  if (it != dslash_tuned_.end()) return it->second;
  if (capturing_) return 0;
  // every variant computes the same sums in the same order, so timing them on
  // the caller's operands leaves `out` correct whichever runs last
  const Level &L = levels_[0];
  EventPair ev;
  cudaEvent_t a = ev.a, b = ev.b;
  int pick = 0;
  float best = 1e30f;
  for (int v = 0; v < wilson_fp32_variants(); ++v) {
    wilson_apply<float>(in, out, nullptr, L.UD32, L.g, m0_, nrhs, v, stream);
    MG_CUDA(cudaEventRecord(a, stream));
    for (int rep = 0; rep < 3; ++rep)
      wilson_apply<float>(in, out, nullptr, L.UD32, L.g, m0_, nrhs, v, stream);
    MG_CUDA(cudaEventRecord(b, stream));
    MG_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    MG_CUDA(cudaEventElapsedTime(&ms, a, b));
    if (ms < best) { best = ms; pick = v; }
  }
  dslash_tuned_[nrhs] = pick;
  return pick;
}

template <typename T> void Engine::apply_D(int l, const C<T> *in, C<T> *out, int nrhs) {
  const Level &L = levels_.at(l);
  cudaEvent_t a = nullptr;
  const bool prof = prof_ && !capturing_;
  if (prof) {
    a = take_event();
    MG_CUDA(cudaEventRecord(a, stream));
  }
  const double cs = (double)sizeof(C<T>);
  double bytes, flops;
  int cls;
  if (L.fine) {
    if constexpr (sizeof(T) == 8) {
      wilson_apply<double>(in, out, L.U64, nullptr, L.g, m0_, nrhs, -1, stream);
    } else {
      const int v = dslash_pick(nrhs, in, out);
      wilson_apply<float>(in, out, nullptr, L.UD32, L.g, m0_, nrhs, v, stream);
    }
    // unique data: nrhs spinors in and out, 4 links per site; 1368 flop per site
    bytes = (double)L.g.V * (24.0 * nrhs + 36.0) * cs;
    flops = 1368.0 * L.g.V * nrhs;
    cls = sizeof(T) == 8 ? K_WILSON64 : K_WILSON32;
  } else {
    // bytes of one complex block entry as stored (BF16 variants: 4)
    double bs = cs;
    if constexpr (sizeof(T) == 8) {
      stencil_apply<T>(in, out, L.AT64, L.g, nrhs, flag_dev_ + 1, stream);
    } else {
      const int v = stencil_pick(l, nrhs, in, out);
      stencil_run(l, v, in, out, nrhs);
      if ((v == 3 && L.ATB16 && nrhs <= 8) || ((v == 6 || v == 7) && L.ATS && nrhs <= 8) || ((v == 4 || v == 5) && L.ATCB))
        bs = 4.0;
    }
    const double m = L.g.dof;
    bytes = (double)L.g.V * (9.0 * m * m * bs + 2.0 * m * nrhs * cs);
    flops = 8.0 * 9.0 * m * m * L.g.V * nrhs;
    cls = sizeof(T) == 8 ? K_STENCIL64 : K_STENCIL32;
  }
  if (prof) {
    cudaEvent_t b = take_event();
    MG_CUDA(cudaEventRecord(b, stream));
    pending_.push_back({cls, a, b, bytes, flops});
  }
}

void Engine::apply_D_bf16(const void *in, void *out, int nrhs) {
  if (!have_gauge_) throw Error(MGMLMC_ERR_STATE, "no gauge field");
  const Level &L = levels_[0];
  wilson_apply_bf16(in, out, L.Ub16, L.g, m0_, nrhs, stream);
}

// Minv is row-major, i.e. column-major Minv^T; the vectors are the columns
// of a column-major n x nrhs matrix: out = (Minv^T)^T in
template <typename T> void Engine::coarsest_apply(const C<T> *Minv, const C<T> *in, C<T> *out, int n, int nrhs) {
  if (nrhs <= 0 || n <= 0) return;
  cublasHandle_t h = static_cast<cublasHandle_t>(blas_);
  cublasStatus_t st;
  if constexpr (sizeof(T) == 4) {
    const cuComplex one = make_cuComplex(1.f, 0.f), zero = make_cuComplex(0.f, 0.f);
    st = cublasCgemm(h, CUBLAS_OP_T, CUBLAS_OP_N, n, nrhs, n, &one, reinterpret_cast<const cuComplex *>(Minv), n,
                     reinterpret_cast<const cuComplex *>(in), n, &zero, reinterpret_cast<cuComplex *>(out), n);
  } else {
    const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
    st = cublasZgemm(h, CUBLAS_OP_T, CUBLAS_OP_N, n, nrhs, n, &one,
                     reinterpret_cast<const cuDoubleComplex *>(Minv), n, reinterpret_cast<const cuDoubleComplex *>(in),
                     n, &zero, reinterpret_cast<cuDoubleComplex *>(out), n);
  }
  if (st != CUBLAS_STATUS_SUCCESS) throw Error(MGMLMC_ERR_CUDA, "cuBLAS GEMM of the coarsest level failed");
}
template void Engine::coarsest_apply<float>(const float2 *, const float2 *, float2 *, int, int);
template void Engine::coarsest_apply<double>(const double2 *, const double2 *, double2 *, int, int);

template <typename T> AggMap Engine::agg_of(int l) const {
  AggMap m = levels_.at(l).agg;
  m.soa = (sizeof(T) == 4 && l == 0) ? 1 : 0;  // FP32 fine vectors are structure-of-arrays
  return m;
}
template <typename T> void Engine::restrict_to(int l, const C<T> *in, C<T> *out, int nrhs) {
  if constexpr (sizeof(T) == 4) {
    if (transfer_variant_ == 1 && levels_[l].PB16) {
      restrict_op_bf16(in, out, levels_[l].PB16, agg_of<T>(l), nrhs, stream);
      return;
    }
  }
  restrict_op<T>(in, out, Pmat<T>(l), agg_of<T>(l), nrhs, stream);
}
template <typename T>
void Engine::prolong_from(int l, const C<T> *in, C<T> *out, int nrhs, double beta) {
  if constexpr (sizeof(T) == 4) {
    if (transfer_variant_ == 1 && levels_[l].PB16) {
      prolong_op_bf16(in, out, levels_[l].PB16, agg_of<T>(l), nrhs, beta, stream);
      return;
    }
  }
  prolong_op<T>(in, out, Pmat<T>(l), agg_of<T>(l), nrhs, beta, stream);
}
template <typename T> void Engine::project_out(int l, const C<T> *in, C<T> *out, int nrhs) {
  const int64_t n = levels_[l].g.n(), nc = levels_[l + 1].g.n();
  C<T> *xc = ws<T>("proj_c", l + 1, (size_t)nc * nrhs);
  restrict_op<T>(in, xc, Pmat<T>(l), agg_of<T>(l), nrhs, stream);
  prolong_op<T>(xc, out, Pmat<T>(l), agg_of<T>(l), nrhs, 0.0, stream);
  axpby<T>(1.0, in, -1.0, out, n, nrhs, stream);
}

void Engine::noise(int l, uint64_t seed, uint64_t sample0, uint64_t term, uint64_t aux, int slice,
                   double2 *out, int nrhs) {
  const Level &L = levels_.at(l);
  if (slice >= L.g.L[3]) throw Error(MGMLMC_ERR_ARG, "slice out of range");
  z4_noise<double>(out, L.g, seed, sample0, term, aux, slice, nrhs, stream);
}

// ------------------------------------------------------------------ MG cycle
// Smoothing: res holds r - D z on entry and exit.  Level 0: SAP sweeps
// (MGMLMC_SMOOTHER_SAP), followed for MGMLMC_SMOOTHER_LEARNED by one learned
// step z += alpha N(res) with the residual-minimising alpha (so the step can
// only lower ||res||); other levels / MR: minimal-residual steps.
template <typename T> void Engine::smooth(int l, C<T> *z, C<T> *res, int nrhs) {
  const int64_t n = levels_[l].g.n();
  const bool learned = l == 0 && sp_.smoother == MGMLMC_SMOOTHER_LEARNED;
  if (l == 0 && sp_.smoother == MGMLMC_SMOOTHER_NET) {
    // the network in place of SAP: smoother_steps residual-minimising steps
    // z += alpha N(res), res -= alpha D N(res)
    if (!net_.C) throw Error(MGMLMC_ERR_STATE, "network smoother selected but the network is not initialised");
    C<T> *e = ws<T>("sape", l, (size_t)n * nrhs);
    C<T> *q = ws<T>("smq", l, (size_t)n * nrhs);
    double2 *d = ws<double>("netd", l, 2 * (size_t)nrhs);
    for (int s = 0; s < sp_.smoother_steps; ++s) {
      cudaEvent_t pa = prof_begin();
      net_forward<T>(res, e, nrhs);
      prof_end(pa, K_NET, 0.0, 0.0);
      apply_D<T>(0, e, q, nrhs);
      dot_qr<T>(q, res, n, nrhs, d, d + nrhs, partials((size_t)reduce_blocks(n) * nrhs * 2), stream);
      mr_dir_update<T>(z, res, e, q, d, d + nrhs, n, nrhs, stream);
    }
    return;
  }
  if (l == 0 && (sp_.smoother == MGMLMC_SMOOTHER_SAP || learned) && sap_b_[0] > 0) {
    C<T> *e = ws<T>("sape", l, (size_t)n * nrhs);
    const C<T> *U;
    if constexpr (sizeof(T) == 8) U = levels_[0].U64; else U = levels_[0].UD32;
    const Geom &g = levels_[0].g;
    // per sweep: the block kernels read the links (once, shared by the
    // right-hand sides), the residual and z and write z, e and the residual;
    // the face passes read e and the residual and write the residual, each
    // site once: 36 + 12 * (5 + 3) complex per site and right-hand side;
    // flops: sap_iters block operators (1368 per site) + the face hops
    const double bytes = (double)g.V * (36.0 + 96.0 * nrhs) * sizeof(C<T>);
    const double flops = (double)g.V * nrhs * (1368.0 * sp_.sap_iters + 684.0);
    for (int s = 0; s < sp_.smoother_steps; ++s) {
      cudaEvent_t a = prof_begin();
      sap_sweep<T>(res, z, e, U, g, sap_b_, m0_, sp_.sap_iters, nrhs, stream, sap_variant_);
      prof_end(a, sizeof(T) == 8 ? K_SAP64 : K_SAP32, bytes, flops);
    }
    // training pairs: the residuals the learned step will see -- after SAP,
    // in the post-smoother, i.e. once the coarse grid has acted
    if (post_smooth_) record<T>(res, nrhs);
    if (learned && post_smooth_) {
      if (!net_.C) throw Error(MGMLMC_ERR_STATE, "learned smoother selected but the network is not initialised");
      C<T> *q = ws<T>("smq", l, (size_t)n * nrhs);
      double2 *d = ws<double>("netd", l, 2 * (size_t)nrhs);
      cudaEvent_t pa = prof_begin();
      net_forward<T>(res, e, nrhs);
      prof_end(pa, K_NET, 0.0, 0.0);
      apply_D<T>(0, e, q, nrhs);
      dot_qr<T>(q, res, n, nrhs, d, d + nrhs, partials((size_t)reduce_blocks(n) * nrhs * 2), stream);
      mr_dir_update<T>(z, res, e, q, d, d + nrhs, n, nrhs, stream);
    }
    return;
  }
  C<T> *q = ws<T>("smq", l, (size_t)n * nrhs);
  double2 *d = ws<double>("smd", l, 2 * (size_t)nrhs);
  const int steps = l == 0 ? sp_.smoother_steps : sp_.coarse_smoother_steps;
  for (int s = 0; s < steps; ++s) {
    apply_D<T>(l, res, q, nrhs);
    dot_qr<T>(q, res, n, nrhs, d, d + nrhs, partials((size_t)reduce_blocks(n) * nrhs * 2), stream);
    mr_update<T>(z, res, q, d, d + nrhs, n, nrhs, stream);
  }
}

template <typename T> void Engine::smooth_apply(int l, const C<T> *in, C<T> *out, int nrhs) {
  const int64_t n = levels_.at(l).g.n();
  C<T> *res = ws<T>("smres", l, (size_t)n * nrhs);
  MG_CUDA(cudaMemcpyAsync(res, in, sizeof(C<T>) * n * nrhs, cudaMemcpyDeviceToDevice, stream));
  MG_CUDA(cudaMemsetAsync(out, 0, sizeof(C<T>) * n * nrhs, stream));
  smooth<T>(l, out, res, nrhs);
}
template void Engine::smooth_apply<double>(int, const C<double> *, C<double> *, int);
template void Engine::smooth_apply<float>(int, const C<float> *, C<float> *, int);

// z = M r: pre-smoothing, coarse-grid correction (recursive K-cycle: a few
// FGMRES iterations on the next level, exact dense solve on the coarsest),
// post-smoothing.
template <typename T> void Engine::precond(int l, const C<T> *r, C<T> *z, int nrhs) {
  // operator applications below belong to the preconditioner: the FP32
  // stencil variant applies there (not to the Krylov operator of a solve)
  struct Depth {
    int &d;
    explicit Depth(int &x) : d(x) { ++d; }
    ~Depth() { --d; }
  } depth(precond_depth_);
  const Level &L = levels_[l];
  const int64_t n = L.g.n();
  if (l == n_levels() - 1) {
    coarsest_apply<T>(Dinv<T>(l), r, z, (int)n, nrhs);
    return;
  }
  const int64_t nc = levels_[l + 1].g.n();
  C<T> *res = ws<T>("mgres", l, (size_t)n * nrhs);
  // q = D z of the post-smoothing residual shares the smoothers' work vector
  // (dead whenever the smoother runs)
  C<T> *q = ws<T>("smq", l, (size_t)n * nrhs);
  C<T> *rc = ws<T>("mgrc", l + 1, (size_t)nc * nrhs);
  C<T> *ec = ws<T>("mgec", l + 1, (size_t)nc * nrhs);
  MG_CUDA(cudaMemsetAsync(z, 0, sizeof(C<T>) * n * nrhs, stream));
  MG_CUDA(cudaMemcpyAsync(res, r, sizeof(C<T>) * n * nrhs, cudaMemcpyDeviceToDevice, stream));
  if (!(sp_.post_smoothing_only && l == 0)) smooth<T>(l, z, res, nrhs);
  cudaEvent_t pr = prof_begin();
  restrict_to<T>(l, res, rc, nrhs);
  prof_end(pr, K_TRANSFER, 0.0, 0.0);
  if (l + 1 == n_levels() - 1) {
    cudaEvent_t pd = prof_begin();
    coarsest_apply<T>(Dinv<T>(l + 1), rc, ec, (int)nc, nrhs);
    prof_end(pd, K_COARSEST, 0.0, 0.0);
  } else {
    fgmres<T>(l + 1, rc, ec, nrhs, 0.0, sp_.coarse_iters, sp_.coarse_iters, true, true);
  }
  cudaEvent_t pp = prof_begin();
  prolong_from<T>(l, ec, z, nrhs, 1.0);
  prof_end(pp, K_TRANSFER, 0.0, 0.0);
  if ((l == 0 ? sp_.smoother_steps : sp_.coarse_smoother_steps) > 0) {
    apply_D<T>(l, z, q, nrhs);
    MG_CUDA(cudaMemcpyAsync(res, r, sizeof(C<T>) * n * nrhs, cudaMemcpyDeviceToDevice, stream));
    axpby<T>(-1.0, q, 1.0, res, n, nrhs, stream);
    post_smooth_ = true;
    smooth<T>(l, z, res, nrhs);
    post_smooth_ = false;
  }
}

// The graphs are keyed by the operand addresses as well: an outer FGMRES
// cycle preconditions V_i into Z_i, i < m, whose addresses are fixed while
// its workspaces live, so m graphs per (level, nrhs, precision) replay the
// cycle on the caller's vectors directly (no staging copies in and out).
template <typename T> void Engine::precond_top(int l, const C<T> *r, C<T> *z, int nrhs) {
  if (!graphs_on_ || prof_ || recording_ || l == n_levels() - 1) {
    precond<T>(l, r, z, nrhs);
    return;
  }
  const auto key = std::make_tuple(l, nrhs, (int)sizeof(T), (const void *)r, (void *)z);
  auto it = graphs_.find(key);
  if (it == graphs_.end()) {
    // eager run: sizes every workspace the captured sequence touches (z gets
    // the result; the captured replay recomputes the same values)
    precond<T>(l, r, z, nrhs);
    sync();
    cudaGraph_t graph = nullptr;
    MG_CUDA(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
    capturing_ = true;
    const int64_t launches_before = launch_counter().load();
    try {
      precond<T>(l, r, z, nrhs);
    } catch (...) {
      capturing_ = false;
      cudaStreamEndCapture(stream, &graph);
      if (graph) cudaGraphDestroy(graph);
      throw;
    }
    capturing_ = false;
    MG_CUDA(cudaStreamEndCapture(stream, &graph));
    cudaGraphExec_t exec = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    MG_CUDA(e);
    graphs_[key] = GraphEntry{exec, launch_counter().load() - launches_before};
    return;  // z already holds the eager result
  }
  MG_CUDA(cudaGraphLaunch(it->second.exec, stream));
  MG_COUNT(it->second.kernels);  // the kernels replayed by the graph
}

// ------------------------------------------------------------------ FGMRES
template <typename T>
SolveInfo Engine::fgmres(int l, const C<T> *b, C<T> *x, int nrhs, double tol, int max_iter, int m,
                         bool use_precond, bool fixed, bool stall_exit) {
  double prev_worst = 1e300;
  const Level &L = levels_[l];
  const int64_t n = L.g.n();
  const int64_t vs = n * nrhs;
  const std::string tag = fixed ? "k" : "t";
  // basis V_0..V_m; the new direction of iteration i is formed in V_{i+1}
  // itself (orthogonalised and normalised in place), so no extra work vector
  C<T> *V = ws<T>("gmV" + tag, l, (size_t)(m + 1) * vs);
  C<T> *Z = use_precond ? ws<T>("gmZ" + tag, l, (size_t)m * vs) : nullptr;
  GmresState st;
  st.m = m;
  st.nrhs = nrhs;
  st.H = ws<double>("gsH" + tag, l, (size_t)nrhs * (m + 1) * m);
  st.h1 = ws<double>("gsh1" + tag, l, (size_t)nrhs * (m + 1));
  st.h2 = ws<double>("gsh2" + tag, l, (size_t)nrhs * (m + 1));
  st.sn = ws<double>("gssn" + tag, l, (size_t)nrhs * m);
  st.g = ws<double>("gsg" + tag, l, (size_t)nrhs * (m + 1));
  st.y = ws<double>("gsy" + tag, l, (size_t)nrhs * m);
  st.nrm = ws<double>("gsnrm" + tag, l, (size_t)nrhs);
  double2 *sc = ws<double>("gssc" + tag, l, (size_t)nrhs * 3 + (size_t)nrhs * m / 2 + 8);
  st.cs = reinterpret_cast<double *>(sc);
  st.inv = st.cs + (size_t)nrhs * m;
  st.res = st.inv + nrhs;
  st.target = st.res + nrhs;
  int *iw = reinterpret_cast<int *>(ws<double>("gsi" + tag, l, (size_t)nrhs + 4));
  st.active = iw;
  st.nit = iw + nrhs;
  double2 *part_k = nullptr;
  auto part = [&](int k) { return partials((size_t)reduce_blocks(n) * nrhs * k); };
  (void)part_k;

  // classical Gram-Schmidt twice, or once for FP32 solves when the solver
  // parameters ask for it (the second coefficients then stay zero)
  const bool two_pass = sizeof(T) == 8 || sp_.gram_schmidt_passes != 1;
  if (!two_pass) MG_CUDA(cudaMemsetAsync(st.h2, 0, sizeof(double2) * nrhs * (m + 1), stream));
  dot<T>(b, b, n, nrhs, st.nrm, part(1), stream);
  target_kernel<<<(nrhs + 63) / 64, 64, 0, stream>>>(st.target, st.nrm, tol, nrhs);
  MG_LAUNCH_CHECK();
  std::vector<double> bn;
  const double *bn_host = nullptr;
  if (!fixed) {
    double2 *h = static_cast<double2 *>(pinned(sizeof(double2) * nrhs));
    MG_CUDA(cudaMemcpyAsync(h, st.nrm, sizeof(double2) * nrhs, cudaMemcpyDeviceToHost, stream));
    sync();
    bn.assign(nrhs, 0.0);
    for (int r = 0; r < nrhs; ++r) bn[r] = std::sqrt(std::max(h[r].x, 0.0));
    bn_host = bn.data();
  }
  MG_CUDA(cudaMemsetAsync(x, 0, sizeof(C<T>) * vs, stream));
  MG_CUDA(cudaMemcpyAsync(V, b, sizeof(C<T>) * vs, cudaMemcpyDeviceToDevice, stream));

  SolveInfo info;
  int total = 0;
  for (;;) {
    dot<T>(V, V, n, nrhs, st.nrm, part(1), stream);
    gmres_start(st, stream);
    scale_rhs<T>(V, V, st.inv, n, nrhs, stream);
    int it = 0;
    for (int i = 0; i < m; ++i) {
      C<T> *vi = V + i * vs;
      C<T> *zi = use_precond ? Z + i * vs : vi;
      C<T> *w = V + (i + 1) * vs;
      if (use_precond) {
        if (fixed) precond<T>(l, vi, zi, nrhs);
        else precond_top<T>(l, vi, zi, nrhs);
      }
      apply_D<T>(l, zi, w, nrhs);
      cudaEvent_t po = prof_begin();
      multi_dot<T>(V, vs, i + 1, w, n, nrhs, st.h1, m + 1, part(i + 1), stream);
      multi_axpy<T>(V, vs, i + 1, w, n, nrhs, st.h1, m + 1, -1.0, stream);
      if (two_pass) {
        multi_dot<T>(V, vs, i + 1, w, n, nrhs, st.h2, m + 1, part(i + 1), stream);
        multi_axpy<T>(V, vs, i + 1, w, n, nrhs, st.h2, m + 1, -1.0, stream);
      }
      dot<T>(w, w, n, nrhs, st.nrm, part(1), stream);
      // unique data of CGS2 (CGS1): the i+1 basis vectors twice (once) for the
      // dots and twice (once) for the updates, w read/written 9 (5) times
      prof_end(po, K_ORTHO,
               (double)vs * sizeof(C<T>) * (two_pass ? 4.0 * (i + 1) + 9.0 : 2.0 * (i + 1) + 5.0), 0.0);
      gmres_arnoldi(st, i, stream);
      scale_rhs<T>(w, w, st.inv, n, nrhs, stream);
      ++it;
      ++total;
      if (total >= max_iter) break;
      if (!fixed) {
        int *ah = static_cast<int *>(pinned(sizeof(int) * nrhs));
        MG_CUDA(cudaMemcpyAsync(ah, st.active, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, stream));
        sync();
        bool any = false;
        for (int r = 0; r < nrhs; ++r) any |= ah[r] != 0;
        if (!any) break;
      }
    }
    gmres_solve(st, stream);
    multi_axpy<T>(use_precond ? Z : V, vs, it, x, n, nrhs, st.y, m, 1.0, stream);
    if (fixed && total >= max_iter) break;
    // true residual (V_1 as the work vector: the cycle's basis is spent)
    apply_D<T>(l, x, V + vs, nrhs);
    MG_CUDA(cudaMemcpyAsync(V, b, sizeof(C<T>) * vs, cudaMemcpyDeviceToDevice, stream));
    axpby<T>(-1.0, V + vs, 1.0, V, n, nrhs, stream);
    if (fixed) continue;
    dot<T>(V, V, n, nrhs, st.nrm, part(1), stream);
    double2 *h = static_cast<double2 *>(pinned(sizeof(double2) * nrhs));
    MG_CUDA(cudaMemcpyAsync(h, st.nrm, sizeof(double2) * nrhs, cudaMemcpyDeviceToHost, stream));
    sync();
    double worst = 0.0;
    bool bad = false;
    for (int r = 0; r < nrhs; ++r) {
      const double rn = std::sqrt(std::max(h[r].x, 0.0));
      if (!std::isfinite(h[r].x)) bad = true;
      const double rel = bn_host[r] > 0.0 ? rn / bn_host[r] : 0.0;
      worst = std::max(worst, rel);
    }
    info.residual = worst;
    if (bad) {
      info.converged = false;
      info.iters = total;
      throw Error(MGMLMC_ERR_NUMERIC, "solver produced NaN/Inf (level " + std::to_string(l) + ")");
    }
    if (worst <= tol) break;
    if (total >= max_iter) {
      info.converged = false;
      break;
    }
    // an inner solve of the defect correction ends at the precision floor
    // of its arithmetic: a restart cycle that did not halve the true
    // residual returns what it has (the FP64 outer loop continues from it)
    if (stall_exit && worst > 0.5 * prev_worst) {
      info.converged = false;
      break;
    }
    prev_worst = worst;
  }
  info.iters = total;
  return info;
}

// FP64 defect correction around FP32 inner solves.  One FP64 work vector t:
// the residual of the current x (b itself before the first correction), then
// the correction e converted up, then D x and b - D x again.
SolveInfo Engine::solve_mixed(int l, const double2 *b, double2 *x, int nrhs) {
  const int64_t n = levels_[l].g.n();
  const int64_t vs = n * nrhs;
  double2 *t = ws<double>("dct", l, (size_t)vs);
  float2 *r32 = ws<float>("dcr32", l, (size_t)vs);
  float2 *e32 = ws<float>("dce32", l, (size_t)vs);
  double2 *nr = ws<double>("dcn", l, (size_t)nrhs * 2);
  double *inv = reinterpret_cast<double *>(ws<double>("dcinv", l, (size_t)nrhs));
  double *rn = reinterpret_cast<double *>(ws<double>("dcrn", l, (size_t)nrhs));
  dot<double>(b, b, n, nrhs, nr, partials((size_t)reduce_blocks(n) * nrhs), stream);
  double2 *h = static_cast<double2 *>(pinned(sizeof(double2) * nrhs));
  MG_CUDA(cudaMemcpyAsync(h, nr, sizeof(double2) * nrhs, cudaMemcpyDeviceToHost, stream));
  sync();
  std::vector<double> bn(nrhs);
  for (int q = 0; q < nrhs; ++q) bn[q] = std::sqrt(std::max(h[q].x, 0.0));
  MG_CUDA(cudaMemsetAsync(x, 0, sizeof(double2) * vs, stream));
  const double2 *r = b;  // residual of x = 0
  if (l == 0 && sp_.learned_guess && !guess_off_) {
    // the network's guess: with c = b / ||b|| (FP32 fine layout), e = N(c)
    // and q = D e, x0 = ||b|| alpha e and c - alpha q is the first defect
    // (its FP32 rounding is corrected by the true FP64 residual after the
    // first inner solve)
    if (!net_.C) throw Error(MGMLMC_ERR_STATE, "learned guess selected but the network is not initialised");
    float2 *q32 = ws<float>("smq", 0, (size_t)vs);
    float2 *z32 = ws<float>("sape", 0, (size_t)vs);
    double2 *dq = ws<double>("netd", 0, 2 * (size_t)nrhs);
    inv_norm_kernel<<<(nrhs + 63) / 64, 64, 0, stream>>>(inv, rn, nr, nrhs);
    MG_LAUNCH_CHECK();
    relayout<float, double>(b, r32, inv, levels_[0].g.V, nrhs, true, stream);
    cudaEvent_t pa = prof_begin();
    net_forward<float>(r32, e32, nrhs);
    prof_end(pa, K_NET, 0.0, 0.0);
    apply_D<float>(0, e32, q32, nrhs);
    dot_qr<float>(q32, r32, n, nrhs, dq, dq + nrhs, partials((size_t)reduce_blocks(n) * nrhs * 2), stream);
    MG_CUDA(cudaMemsetAsync(z32, 0, sizeof(float2) * vs, stream));
    mr_dir_update<float>(z32, r32, e32, q32, dq, dq + nrhs, n, nrhs, stream);
    relayout<double, float>(z32, x, rn, levels_[0].g.V, nrhs, false, stream);
    relayout<double, float>(r32, t, rn, levels_[0].g.V, nrhs, false, stream);
    r = t;
  }
  SolveInfo info;
  int total = 0;
  for (int outer = 0;; ++outer) {
    dot<double>(r, r, n, nrhs, nr, partials((size_t)reduce_blocks(n) * nrhs), stream);
    MG_CUDA(cudaMemcpyAsync(h, nr, sizeof(double2) * nrhs, cudaMemcpyDeviceToHost, stream));
    sync();
    double worst = 0.0;
    for (int q = 0; q < nrhs; ++q) {
      if (!std::isfinite(h[q].x)) throw Error(MGMLMC_ERR_NUMERIC, "defect correction: NaN/Inf");
      worst = std::max(worst, bn[q] > 0 ? std::sqrt(std::max(h[q].x, 0.0)) / bn[q] : 0.0);
    }
    info.residual = worst;
    if (worst <= sp_.tol) break;
    if (total >= sp_.max_iter || outer >= 100) {
      info.converged = false;
      break;
    }
    inv_norm_kernel<<<(nrhs + 63) / 64, 64, 0, stream>>>(inv, rn, nr, nrhs);
    MG_LAUNCH_CHECK();
    if (l == 0) relayout<float, double>(r, r32, inv, levels_[0].g.V, nrhs, true, stream);
    else convert_scale<float, double>(r, r32, inv, n, nrhs, stream);
    // the inner solve reduces its residual by inner_tol, or by only what is
    // left to reach tol (with a factor 2 of margin) when that is less: the
    // least converged right-hand side sets it, so it suffices for all
    const double itol = std::max(sp_.inner_tol, std::min(0.5, 0.5 * sp_.tol / std::max(worst, 1e-300)));
    SolveInfo in = fgmres<float>(l, r32, e32, nrhs, itol, sp_.max_iter - total, restart_of(l), true, false, true);
    total += in.iters;
    if (l == 0) relayout<double, float>(e32, t, rn, levels_[0].g.V, nrhs, false, stream);
    else convert_scale<double, float>(e32, t, rn, n, nrhs, stream);
    axpby<double>(1.0, t, 1.0, x, n, nrhs, stream);
    apply_D<double>(l, x, t, nrhs);
    axpby<double>(1.0, b, -1.0, t, n, nrhs, stream);  // t = b - D x
    r = t;
  }
  info.iters = total;
  return info;
}

SolveInfo Engine::solve(int l, const double2 *b, double2 *x, int nrhs) {
  if (!ready_) throw Error(MGMLMC_ERR_STATE, "hierarchy not built");
  struct Solving {
    int &d;
    explicit Solving(int &x) : d(x) { ++d; }
    ~Solving() { --d; }
  } solving(solving_);
  const int64_t n = levels_.at(l).g.n();
  SolveInfo info;
  if (l == n_levels() - 1) {
    coarsest_apply<double>(levels_[l].Dinv64, b, x, (int)n, nrhs);
    info.iters = 0;
    info.residual = 0.0;
  } else if (l == 0 && (sp_.smoother == MGMLMC_SMOOTHER_LEARNED || sp_.smoother == MGMLMC_SMOOTHER_NET)) {
    // learned smoother first; the true residual judges it, SAP takes over
    // when it does not converge within a quarter of the iteration budget
    const int mode = sp_.smoother;
    const int full = sp_.max_iter;
    sp_.max_iter = std::max(1, full / 4);
    bool ok = true;
    try {
      info = sp_.precision == MGMLMC_FP32
                 ? solve_mixed(l, b, x, nrhs)
                 : fgmres<double>(l, b, x, nrhs, sp_.tol, sp_.max_iter, restart_of(l), true, false);
      ok = info.converged;
    } catch (const Error &e) {
      if (e.code != MGMLMC_ERR_NUMERIC && e.code != MGMLMC_ERR_NOT_CONVERGED) {
        sp_.max_iter = full;
        throw;
      }
      ok = false;
    }
    sp_.max_iter = full;
    if (!ok) {
      ++net_.fallbacks;
      sp_.smoother = MGMLMC_SMOOTHER_SAP;
      drop_graphs();
      try {
        info = sp_.precision == MGMLMC_FP32
                   ? solve_mixed(l, b, x, nrhs)
                   : fgmres<double>(l, b, x, nrhs, sp_.tol, sp_.max_iter, restart_of(l), true, false);
      } catch (...) {
        sp_.smoother = mode;
        drop_graphs();
        throw;
      }
      sp_.smoother = mode;
      drop_graphs();
    }
  } else if (sp_.precision == MGMLMC_FP32) {
    info = solve_mixed(l, b, x, nrhs);
  } else {
    info = fgmres<double>(l, b, x, nrhs, sp_.tol, sp_.max_iter, restart_of(l), true, false);
  }
  last_solve = info;
  check_staging();
  if (!info.converged)
    throw Error(MGMLMC_ERR_NOT_CONVERGED,
                "level " + std::to_string(l) + " solve stopped after " + std::to_string(info.iters) +
                    " iterations at relative residual " + std::to_string(info.residual));
  return info;
}

// ------------------------------------------------------------------ setup
void Engine::galerkin(int l) {
  Level &f = levels_[l];
  Level &c = levels_[l + 1];
  const AggMap &m = f.agg;
  const int64_t nf = f.g.n(), nc = c.g.n();
  const int dofc = c.g.dof;
  double2 *probe = ws<double>("galp", l, (size_t)nf);
  double2 *out9 = ws<double>("gal9", l, (size_t)9 * nf);
  double2 *cols = ws<double>("galc", l, (size_t)9 * nc);
  const size_t acnt = (size_t)c.g.V * 9 * dofc * dofc;
  c.A64 = dalloc<double2>(acnt);
  c.AT64 = dalloc<double2>(acnt);
  c.AT32 = dalloc<float2>(acnt);
  for (int col = 0; col < dofc; ++col) {
    probe_column(probe, f.P64, m, col, stream);
    if (f.fine) wilson_split<double>(probe, out9, f.U64, f.g, m0_, m.b, stream);
    else stencil_split<double>(probe, out9, f.A64, f.g, m.b, stream);
    restrict_op<double>(out9, cols, f.P64, m, 9, stream);
    galerkin_scatter(cols, c.A64, c.g, col, stream);
  }
  stencil_transpose<double>(c.A64, c.AT64, (int64_t)c.g.V * 9, dofc, stream);
  stencil_transpose<float>(c.A64, c.AT32, (int64_t)c.g.V * 9, dofc, stream);
  if (stencil_tc_supported(c.g)) {
    c.ATC = dalloc<float>(stencil_tc_elems(c.g));
    stencil_tile_tc(c.A64, c.ATC, false, c.g, stream);
    c.ATCB = dalloc<float>((stencil_tc_elems(c.g) + 1) / 2);  // BF16 elements, two per float slot
    stencil_tile_tc(c.A64, c.ATCB, true, c.g, stream);
  }
  if (stencil_pipe_supported(c.g)) {
    c.ATB16 = dalloc<float>(acnt);  // one bf16 pair (4 bytes) per complex entry
    stencil_to_bf16(c.AT32, c.ATB16, (int64_t)acnt, stream);
    c.ATS = dalloc<float>(acnt);
    stencil_to_stream(c.AT32, c.ATS, (int64_t)acnt, stream);
  }
}

void Engine::build_hierarchy(const mgmlmc_mg_params &p) {
  if (!have_gauge_) throw Error(MGMLMC_ERR_STATE, "set the gauge field first");
  if (p.n_levels < 1 || p.n_levels > MGMLMC_MAX_LEVELS) throw Error(MGMLMC_ERR_ARG, "n_levels out of range");
  free_hierarchy();
  // geometry of every level first (argument checks before any allocation)
  std::vector<Geom> geo(p.n_levels);
  std::vector<AggMap> maps(p.n_levels);
  geo[0] = fine_;
  for (int l = 0; l + 1 < p.n_levels; ++l) {
    AggMap &m = maps[l];
    m.fine = geo[l];
    const int ntv = p.n_tv[l];
    if (ntv < 1 || ntv > 128) throw Error(MGMLMC_ERR_ARG, "n_tv must be in 1..128");
    Geom cg{};
    int64_t cv = 1;
    int sites = 1;
    for (int i = 0; i < 4; ++i) {
      const int b = p.block[l][i];
      if (b < 1 || geo[l].L[i] % b) throw Error(MGMLMC_ERR_ARG, "block must divide the lattice");
      m.b[i] = b;
      cg.L[i] = geo[l].L[i] / b;
      cv *= cg.L[i];
      sites *= b;
    }
    cg.V = (int)cv;
    cg.dof = 2 * ntv;
    m.coarse = cg;
    m.ntv = ntv;
    m.half = geo[l].dof / 2;
    m.sites = sites;
    m.rows = sites * m.half;
    if (ntv > m.rows) throw Error(MGMLMC_ERR_ARG, "more test vectors than rows per aggregate");
    if ((size_t)m.rows * sizeof(double2) > 48 * 1024)
      throw Error(MGMLMC_ERR_ARG, "aggregate too large (rows * 16 B must fit 48 KB)");
    geo[l + 1] = cg;
  }
  const int64_t ncoarsest = geo[p.n_levels - 1].n();
  if (ncoarsest > 20000) throw Error(MGMLMC_ERR_ARG, "coarsest level too large for the dense inverse");

  levels_.resize(p.n_levels);
  for (int l = 1; l < p.n_levels; ++l) {
    levels_[l] = Level{};
    levels_[l].g = geo[l];
  }
  for (int l = 0; l + 1 < p.n_levels; ++l) {
    Level &f = levels_[l];
    f.agg = maps[l];
    f.has_next = true;
    const int64_t n = f.g.n();
    const int ntv = maps[l].ntv;
    double2 *V = ws<double>("tv", l, (size_t)ntv * n);
    auto imp = imported_host_.find(l);
    if (imp != imported_host_.end()) {
      if ((int64_t)imp->second.size() != (int64_t)ntv * n * 2)
        throw Error(MGMLMC_ERR_ARG, "imported test vectors have the wrong size for level " + std::to_string(l));
      MG_CUDA(cudaMemcpyAsync(V, imp->second.data(), sizeof(double2) * ntv * n, cudaMemcpyHostToDevice, stream));
    } else {
      z4_noise<double>(V, f.g, p.seed, 0, 96 + l, 0, -1, ntv, stream);
      if (p.setup_rounds > 0) setup_test_vectors(l, V, ntv, p);
    }
    f.P64 = dalloc<double2>((size_t)ntv * n);
    f.P32 = dalloc<float2>((size_t)ntv * n);
    f.PB16 = dalloc<float>((size_t)ntv * n);
    MG_CUDA(cudaMemsetAsync(flag_dev_, 0, sizeof(int), stream));
    build_prolongator(V, f.P64, f.agg, flag_dev_, stream);
    convert<float, double>(f.P64, f.P32, (int64_t)ntv * n, stream);
    stencil_to_bf16(f.P32, f.PB16, (int64_t)ntv * n, stream);
    int flag = 0;
    MG_CUDA(cudaMemcpyAsync(&flag, flag_dev_, sizeof(int), cudaMemcpyDeviceToHost, stream));
    sync();
    if (flag) throw Error(MGMLMC_ERR_NUMERIC, "test vectors are linearly dependent on an aggregate");
    galerkin(l);
  }
  // coarsest level: dense inverse (FP64 Gauss-Jordan with partial pivoting)
  Level &c = levels_.back();
  const int n = (int)c.g.n();
  if (c.fine) {
    // one level only: the coarsest operator is the Wilson operator itself
    throw Error(MGMLMC_ERR_ARG, "n_levels must be >= 2");
  }
  c.Dinv64 = dalloc<double2>((size_t)n * n);
  c.Dinv32 = dalloc<float2>((size_t)n * n);
  double2 *work = ws<double>("gj", 0, (size_t)2 * n * n + n + 8);
  dense_from_stencil(c.A64, c.Dinv64, c.g, stream);
  MG_CUDA(cudaMemsetAsync(flag_dev_, 0, sizeof(int), stream));
  dense_invert(c.Dinv64, work, n, flag_dev_, stream);
  convert<float, double>(c.Dinv64, c.Dinv32, (int64_t)n * n, stream);
  int flag = 0;
  MG_CUDA(cudaMemcpyAsync(&flag, flag_dev_, sizeof(int), cudaMemcpyDeviceToHost, stream));
  sync();
  if (flag) throw Error(MGMLMC_ERR_NUMERIC, "coarsest operator is singular");
  // the build's scratch is not needed by the solves: give it back (large
  // lattices need the room for the Krylov bases); a level's test vectors are
  // kept for mgmlmc_get_test_vectors unless they exceed kKeepTestVectorBytes
  for (const char *name : {"galp", "gal9", "galc", "tvx", "tv32", "tvx32", "gj"})
    for (int l = 0; l < p.n_levels; ++l) {
      ws_release(name, l, true);
      ws_release(name, l, false);
    }
  for (int l = 0; l + 1 < p.n_levels; ++l)
    if ((double)levels_[l].agg.ntv * levels_[l].g.n() * sizeof(double2) > kKeepTestVectorBytes)
      ws_release("tv", l, true);
  mgp_ = p;
  ready_ = true;
}

// Sec. 4 setup: `setup_rounds` rounds of v <- w / ||w||, w the result of
// `setup_iters` unpreconditioned GMRES iterations on D_l w = v (a rough
// solve).  All N_tv columns at once would need a GMRES basis of N_tv (m + 1)
// level vectors, more than a large lattice leaves free, so the columns go in
// groups sized to the free device memory; every column sees the same
// iterations whatever the grouping.  When the solver runs FP32 inner solves
// the setup runs in FP32 too (the vectors only need a rough residual).
void Engine::setup_test_vectors(int l, double2 *V, int ntv, const mgmlmc_mg_params &p) {
  const Geom &g = levels_[l].g;
  const int64_t n = g.n();
  const int it = std::max(1, p.setup_iters);
  const int m = std::min(it, 64);
  const bool fp32 = sp_.precision == MGMLMC_FP32;
  const double es = fp32 ? sizeof(float2) : sizeof(double2);
  size_t freeb = 0, totalb = 0;
  MG_CUDA(cudaMemGetInfo(&freeb, &totalb));
  // per column: the basis (m + 1), the iterate, the converted input
  const double per_col = (double)n * es * (m + 3);
  const int group = std::max(1, std::min(ntv, (int)(0.7 * (double)freeb / per_col)));
  double *inv = reinterpret_cast<double *>(ws<double>("tvinv", l, (size_t)ntv));
  double *nr = reinterpret_cast<double *>(ws<double>("tvnr", l, (size_t)ntv));
  double2 *d = ws<double>("tvd", l, (size_t)ntv);
  for (int c0 = 0; c0 < ntv; c0 += group) {
    const int gs = std::min(group, ntv - c0);
    double2 *Vg = V + (size_t)c0 * n;
    for (int round = 0; round < p.setup_rounds; ++round) {
      if (fp32) {
        float2 *v32 = ws<float>("tv32", l, (size_t)gs * n);
        float2 *x32 = ws<float>("tvx32", l, (size_t)gs * n);
        if (l == 0) relayout<float, double>(Vg, v32, nullptr, g.V, gs, true, stream);
        else convert<float, double>(Vg, v32, (int64_t)gs * n, stream);
        fgmres<float>(l, v32, x32, gs, 0.0, it, m, false, true);
        dot<float>(x32, x32, n, gs, d, partials((size_t)reduce_blocks(n) * gs), stream);
        inv_norm_kernel<<<(gs + 63) / 64, 64, 0, stream>>>(inv, nr, d, gs);
        MG_LAUNCH_CHECK();
        if (l == 0) relayout<double, float>(x32, Vg, inv, g.V, gs, false, stream);
        else convert_scale<double, float>(x32, Vg, inv, n, gs, stream);
      } else {
        double2 *X = ws<double>("tvx", l, (size_t)gs * n);
        fgmres<double>(l, Vg, X, gs, 0.0, it, m, false, true);
        dot<double>(X, X, n, gs, d, partials((size_t)reduce_blocks(n) * gs), stream);
        inv_norm_kernel<<<(gs + 63) / 64, 64, 0, stream>>>(inv, nr, d, gs);
        MG_LAUNCH_CHECK();
        scale_rhs<double>(X, Vg, inv, n, gs, stream);
      }
    }
  }
  // the fixed-length GMRES workspaces of the setup (recreated on demand)
  for (const char *name : {"gmVk", "gmZk", "gsHk", "gsh1k", "gsh2k", "gssnk", "gsgk", "gsyk", "gsnrmk",
                           "gssck", "gsik"}) {
    ws_release(name, l, true);
    ws_release(name, l, false);
  }
}

void Engine::check_staging() {
  // a staging wait of a coarse-stencil kernel that ran out of its bound sets
  // flag_dev_[1] (2: CUDA-core kernel, 3: tensor-core kernel)
  int tma_err = 0;
  MG_CUDA(cudaMemcpyAsync(&tma_err, flag_dev_ + 1, sizeof(int), cudaMemcpyDeviceToHost, stream));
  sync();
  if (tma_err) {
    MG_CUDA(cudaMemsetAsync(flag_dev_ + 1, 0, sizeof(int), stream));
    sync();
    throw Error(MGMLMC_ERR_CUDA, "a shared-memory staging copy did not complete within its bounded wait");
  }
}

void Engine::release_workspaces() {
  drop_graphs();
  sync();
  for (auto it = ws_.begin(); it != ws_.end();) {
    if (it->first.rfind("tv#", 0) == 0) {  // a level's test vectors
      ++it;
      continue;
    }
    cudaFree(it->second.first);
    it = ws_.erase(it);
  }
}

// ------------------------------------------------------------------ estimators
namespace {
struct TermDef {
  int code, level, kind, N;  // kind 0 plain, 1 O, 2 F, 3 coarsest
};
}  // namespace

void Engine::estimate_trace(const mgmlmc_est_params &p, std::vector<TermAcc> &out) {
  if (!ready_) throw Error(MGMLMC_ERR_STATE, "hierarchy not built");
  const int L = n_levels();
  std::vector<TermDef> terms;
  if (p.kind == MGMLMC_EST_PLAIN) {
    terms.push_back({MGMLMC_TERM_PLAIN, 0, 0, p.n_samples[0]});
  } else if (p.kind == MGMLMC_EST_ORTHOGONAL) {
    int idx = 0;
    for (int l = 0; l + 1 < L; ++l) terms.push_back({MGMLMC_TERM_O + l, l, 1, p.n_samples[idx++]});
    for (int l = 0; l + 1 < L; ++l) terms.push_back({MGMLMC_TERM_F + l, l, 2, p.n_samples[idx++]});
    terms.push_back({MGMLMC_TERM_COARSEST, L - 1, 3, p.n_samples[idx++]});
  } else if (p.kind == MGMLMC_EST_DEFLATED) {
    if (!defl_V_) throw Error(MGMLMC_ERR_STATE, "no deflation basis (mgmlmc_deflation_build)");
    terms.push_back({MGMLMC_TERM_DEFL, 0, 5, p.n_samples[0]});
  } else if (p.kind == MGMLMC_EST_OBLIQUE) {
    int idx = 0;
    for (int l = 0; l + 1 < L; ++l) terms.push_back({MGMLMC_TERM_M + l, l, 4, p.n_samples[idx++]});
    terms.push_back({MGMLMC_TERM_COARSEST, L - 1, 3, p.n_samples[idx++]});
  } else {
    throw Error(MGMLMC_ERR_ARG, "unknown estimator kind");
  }
  for (const TermDef &td : terms)
    if (td.N < 0) throw Error(MGMLMC_ERR_ARG, "negative sample count");
  const int B = std::max(1, p.batch);
  EventPair ev;
  cudaEvent_t e0 = ev.a, e1 = ev.b;
  out.clear();
  for (const TermDef &td : terms) {
    TermAcc acc;
    acc.term = td.code;
    std::vector<std::complex<double>> X;
    // terms that solve on the fine level take its memory bound (fine_batch)
    const int Bt = (td.level == 0 && td.kind != 3 && sp_.fine_batch > 0) ? std::min(B, sp_.fine_batch) : B;
    for (int k0 = 0; k0 < td.N; k0 += Bt) {
      const int nb = std::min(Bt, td.N - k0);
      const uint64_t s0 = p.first_sample + (uint64_t)k0;
      double2 *res = ws<double>("est_res", 0, 2 * (size_t)nb);
      MG_CUDA(cudaEventRecord(e0, stream));
      const int l = td.level;
      const int64_t n = levels_[l].g.n();
      if (td.kind == 0) {
        double2 *x = ws<double>("estx", l, (size_t)nb * n), *z = ws<double>("estz", l, (size_t)nb * n);
        noise(l, p.seed, s0, MGMLMC_TERM_PLAIN, 0, -1, x, nb);
        SolveInfo si = solve(l, x, z, nb);
        acc.iters_sum += si.iters;
        acc.solves += 1;
        acc.max_res = std::max(acc.max_res, si.residual);
        dot<double>(x, z, n, nb, res, partials((size_t)reduce_blocks(n) * nb), stream);
      } else if (td.kind == 1) {
        // the noise x is drawn into z's buffer and projected into y; the
        // solve then overwrites z (two level-l vectors instead of three)
        double2 *y = ws<double>("esty", l, (size_t)nb * n), *z = ws<double>("estz", l, (size_t)nb * n);
        noise(l, p.seed, s0, MGMLMC_TERM_O + l, 0, -1, z, nb);
        project_out<double>(l, z, y, nb);
        SolveInfo si = solve(l, y, z, nb);
        acc.iters_sum += si.iters;
        acc.solves += 1;
        acc.max_res = std::max(acc.max_res, si.residual);
        dot<double>(y, z, n, nb, res, partials((size_t)reduce_blocks(n) * nb), stream);
      } else if (td.kind == 2) {
        const int64_t nc = levels_[l + 1].g.n();
        double2 *x = ws<double>("estxc", l + 1, (size_t)nb * nc), *y = ws<double>("esty", l, (size_t)nb * n);
        double2 *z1 = ws<double>("estz", l, (size_t)nb * n), *z2 = ws<double>("estzc", l + 1, (size_t)nb * nc);
        noise(l + 1, p.seed, s0, MGMLMC_TERM_F + l, 0, -1, x, nb);
        prolong_from<double>(l, x, y, nb, 0.0);
        // y = P x lies in the range of P, which the coarse-grid correction
        // covers: the learned guess is not used for it
        guess_off_ = true;
        SolveInfo s1;
        try {
          s1 = solve(l, y, z1, nb);
        } catch (...) {
          guess_off_ = false;
          throw;
        }
        guess_off_ = false;
        SolveInfo s2 = solve(l + 1, x, z2, nb);
        acc.iters_sum += s1.iters + s2.iters;
        acc.solves += 2;
        acc.max_res = std::max(acc.max_res, std::max(s1.residual, s2.residual));
        dot<double>(y, z1, n, nb, res, partials((size_t)reduce_blocks(n) * nb), stream);
        dot<double>(x, z2, nc, nb, res + nb, partials((size_t)reduce_blocks(nc) * nb), stream);
      } else if (td.kind == 5) {
        // deflated sample: x^H z - (V^H x)^H (V^H z), z = D^-1 x
        const int k = defl_k_;
        double2 *x = ws<double>("estx", 0, (size_t)nb * n), *z = ws<double>("estz", 0, (size_t)nb * n);
        double2 *cx = ws<double>("dfcx", 0, (size_t)nb * k), *cz = ws<double>("dfcz", 0, (size_t)nb * k);
        noise(0, p.seed, s0, MGMLMC_TERM_DEFL, 0, -1, x, nb);
        SolveInfo si = solve(0, x, z, nb);
        acc.iters_sum += si.iters;
        acc.solves += 1;
        acc.max_res = std::max(acc.max_res, si.residual);
        dot<double>(x, z, n, nb, res, partials((size_t)reduce_blocks(n) * nb), stream);
        for (int q = 0; q < nb; ++q) {
          multi_dot<double>(defl_V_, n, k, x + (size_t)q * n, n, 1, cx + (size_t)q * k, k,
                            partials((size_t)reduce_blocks(n) * k), stream);
          multi_dot<double>(defl_V_, n, k, z + (size_t)q * n, n, 1, cz + (size_t)q * k, k,
                            partials((size_t)reduce_blocks(n) * k), stream);
        }
        std::vector<double2> hx((size_t)nb * k), hz((size_t)nb * k);
        MG_CUDA(cudaMemcpyAsync(hx.data(), cx, sizeof(double2) * nb * k, cudaMemcpyDeviceToHost, stream));
        MG_CUDA(cudaMemcpyAsync(hz.data(), cz, sizeof(double2) * nb * k, cudaMemcpyDeviceToHost, stream));
        sync();
        // fold the projected part into res[nb + q] so the common code subtracts it
        std::vector<double2> sub((size_t)nb);
        for (int q = 0; q < nb; ++q) {
          std::complex<double> s(0.0, 0.0);
          for (int j = 0; j < k; ++j)
            s += std::conj(std::complex<double>(hx[(size_t)q * k + j].x, hx[(size_t)q * k + j].y)) *
                 std::complex<double>(hz[(size_t)q * k + j].x, hz[(size_t)q * k + j].y);
          sub[q] = make_double2(s.real(), s.imag());
        }
        MG_CUDA(cudaMemcpyAsync(res + nb, sub.data(), sizeof(double2) * nb, cudaMemcpyHostToDevice, stream));
        sync();
      } else if (td.kind == 4) {
        // oblique M_l (Eq. oblique-deflation): x^H D_l^-1 x - (P^H x)^H D_{l+1}^-1 (P^H x)
        const int64_t nc = levels_[l + 1].g.n();
        double2 *x = ws<double>("estx", l, (size_t)nb * n), *z1 = ws<double>("estz", l, (size_t)nb * n);
        double2 *xc = ws<double>("estxc", l + 1, (size_t)nb * nc), *z2 = ws<double>("estzc", l + 1, (size_t)nb * nc);
        noise(l, p.seed, s0, MGMLMC_TERM_M + l, 0, -1, x, nb);
        SolveInfo s1 = solve(l, x, z1, nb);
        restrict_to<double>(l, x, xc, nb);
        SolveInfo s2 = solve(l + 1, xc, z2, nb);
        acc.iters_sum += s1.iters + s2.iters;
        acc.solves += 2;
        acc.max_res = std::max(acc.max_res, std::max(s1.residual, s2.residual));
        dot<double>(x, z1, n, nb, res, partials((size_t)reduce_blocks(n) * nb), stream);
        dot<double>(xc, z2, nc, nb, res + nb, partials((size_t)reduce_blocks(nc) * nb), stream);
      } else {
        double2 *x = ws<double>("estx", l, (size_t)nb * n), *z = ws<double>("estz", l, (size_t)nb * n);
        noise(l, p.seed, s0, MGMLMC_TERM_COARSEST, 0, -1, x, nb);
        coarsest_apply<double>(levels_[l].Dinv64, x, z, (int)n, nb);
        dot<double>(x, z, n, nb, res, partials((size_t)reduce_blocks(n) * nb), stream);
      }
      MG_CUDA(cudaEventRecord(e1, stream));
      double2 *h = static_cast<double2 *>(pinned(sizeof(double2) * 2 * nb));
      MG_CUDA(cudaMemcpyAsync(h, res, sizeof(double2) * 2 * nb, cudaMemcpyDeviceToHost, stream));
      sync();
      float ms = 0.f;
      MG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      acc.seconds += ms * 1e-3;
      for (int q = 0; q < nb; ++q) {
        std::complex<double> v(h[q].x, h[q].y);
        if (td.kind == 2 || td.kind == 4 || td.kind == 5) v -= std::complex<double>(h[nb + q].x, h[nb + q].y);
        X.push_back(v);
      }
    }
    acc.n = (int)X.size();
    for (auto &v : X) {
      acc.sre += v.real();
      acc.sim += v.imag();
      acc.sabs2 += std::norm(v);
    }
    acc.samples = X;
    out.push_back(acc);
  }
  if (p.kind == MGMLMC_EST_DEFLATED) {
    // the non-stochastic part tr(V^H D^-1 V), computed when the basis was built
    TermAcc acc;
    acc.term = MGMLMC_TERM_DEFL_EXACT;
    acc.n = 1;
    acc.sre = defl_exact_.real();
    acc.sim = defl_exact_.imag();
    acc.sabs2 = std::norm(defl_exact_);
    acc.seconds = defl_seconds_;
    acc.samples = {defl_exact_};
    out.push_back(acc);
  }
}

// columns of V ([k][n]) orthonormalised by classical Gram-Schmidt run twice,
// in column order
void Engine::orthonormalise_cols(double2 *V, int k, int64_t n) {
  double2 *h = ws<double>("gsh", 0, (size_t)k + 1);
  for (int j = 0; j < k; ++j) {
    double2 *v = V + (size_t)j * n;
    for (int pass = 0; pass < 2 && j > 0; ++pass) {
      multi_dot<double>(V, n, j, v, n, 1, h, j, partials((size_t)reduce_blocks(n) * j), stream);
      multi_axpy<double>(V, n, j, v, n, 1, h, j, -1.0, stream);
    }
    dot<double>(v, v, n, 1, h + k, partials((size_t)reduce_blocks(n)), stream);
    double2 nn;
    MG_CUDA(cudaMemcpyAsync(&nn, h + k, sizeof(double2), cudaMemcpyDeviceToHost, stream));
    sync();
    if (!(nn.x > 0.0) || !std::isfinite(nn.x))
      throw Error(MGMLMC_ERR_NUMERIC, "orthonormalisation: dependent or non-finite column");
    axpby<double>(1.0 / std::sqrt(nn.x), v, 0.0, v, n, 1, stream);
  }
}

void Engine::deflation_build(int k, int iters, double tol, uint64_t seed,
                             std::complex<double> &exact, double &seconds) {
  if (!ready_) throw Error(MGMLMC_ERR_STATE, "hierarchy not built");
  const int64_t n = levels_[0].g.n();
  if (k < 1 || k > 128 || k > n) throw Error(MGMLMC_ERR_ARG, "deflation: k must be in [1, min(128, n)]");
  if (iters < 0 || !(tol > 0.0 && tol < 1.0)) throw Error(MGMLMC_ERR_ARG, "deflation: bad iters or tol");
  EventPair ev;
  cudaEvent_t a = ev.a, b = ev.b;
  MG_CUDA(cudaEventRecord(a, stream));
  dfree(defl_V_);
  defl_V_ = nullptr;
  defl_k_ = 0;
  double2 *V = dalloc<double2>((size_t)k * n);
  try {
    double2 *g = ws<double>("dfg", 0, (size_t)8 * n);
    double2 *W = ws<double>("dfw", 0, (size_t)k * n);
    noise(0, seed, 0, MGMLMC_TERM_DEFL_START, 0, -1, V, k);
    orthonormalise_cols(V, k, n);
    // the build solves in FP64: the basis columns approach the low modes of
    // Gamma5 D, on which the FP32 inner solves of the mixed scheme stalled
    // near a 1e-6 relative residual (16^4 benchmark field)
    const mgmlmc_solver_params keep = sp_;
    sp_.precision = MGMLMC_FP64;
    sp_.tol = tol;
    try {
      for (int it = 0; it < iters; ++it) {
        for (int j0 = 0; j0 < k; j0 += 8) {  // W = D^-1 Gamma5 V, 8 columns at a time
          const int nb = std::min(8, k - j0);
          gamma5_apply<double>(V + (size_t)j0 * n, g, levels_[0].g.V, 12, nb, stream);
          solve(0, g, W + (size_t)j0 * n, nb);
        }
        orthonormalise_cols(W, k, n);
        MG_CUDA(cudaMemcpyAsync(V, W, sizeof(double2) * k * n, cudaMemcpyDeviceToDevice, stream));
      }
      // exact part, sum_j v_j^H D^-1 v_j, at the solver's tolerance
      sp_.tol = keep.tol;
      for (int j0 = 0; j0 < k; j0 += 8) {
        const int nb = std::min(8, k - j0);
        solve(0, V + (size_t)j0 * n, W + (size_t)j0 * n, nb);
      }
    } catch (...) {
      sp_ = keep;
      throw;
    }
    sp_ = keep;
    double2 *d = ws<double>("dfd", 0, (size_t)k);
    dot<double>(V, W, n, k, d, partials((size_t)reduce_blocks(n) * k), stream);
    std::vector<double2> hd((size_t)k);
    MG_CUDA(cudaMemcpyAsync(hd.data(), d, sizeof(double2) * k, cudaMemcpyDeviceToHost, stream));
    MG_CUDA(cudaEventRecord(b, stream));
    sync();
    std::complex<double> s(0.0, 0.0);
    for (int j = 0; j < k; ++j) s += std::complex<double>(hd[j].x, hd[j].y);
    float ms = 0.f;
    MG_CUDA(cudaEventElapsedTime(&ms, a, b));
    defl_V_ = V;
    defl_k_ = k;
    defl_exact_ = s;
    defl_seconds_ = ms * 1e-3;
  } catch (...) {
    cudaFree(V);
    ws_release("dfw", 0, true);
    ws_release("dfg", 0, true);
    throw;
  }
  // the k x n work columns are needed only while building
  ws_release("dfw", 0, true);
  ws_release("dfg", 0, true);
  exact = defl_exact_;
  seconds = defl_seconds_;
}

// ------------------------------------------------------- test-vector refinement
// Simultaneous inverse iteration on Q_l = Gamma5_l D_l (Rutishauser's
// 'ritzit', with the Ritz step on Q_l^-2, which is positive definite, so the
// wanted low modes of the indefinite Q_l are its exterior ones):
//   start: the level's N_tv test vectors, then m - N_tv Z4 columns (noise
//          term 192 + l, samples N_tv .. m-1), orthonormalised;
//   step:  W = Q^-1 V = D^-1 Gamma5 V (FP64 solves to solve_tol),
//          W^H W = Y diag(mu) Y^H (host Jacobi), mu descending,
//          V = W Y diag(mu)^-1/2;
//   check: theta_j = v_j^H Q v_j, rho_j = ||Q v_j - theta_j v_j||.
// The first N_tv columns, each turned so that its largest-modulus entry is
// real and positive, replace the level's test vectors as if imported; the
// levels above keep the vectors they were built from, and the hierarchy is
// rebuilt with the parameters of the last build.
void Engine::refine_test_vectors(int l, int m, int iters, double tol, double solve_tol, uint64_t seed,
                                 std::vector<double> &theta, std::vector<double> &rho, int &steps) {
  if (!ready_) throw Error(MGMLMC_ERR_STATE, "hierarchy not built");
  if (l < 0 || l + 1 >= n_levels()) throw Error(MGMLMC_ERR_ARG, "refine: the level has no test vectors");
  const int k = levels_[l].agg.ntv;
  const Geom G = levels_[l].g;
  const int64_t n = G.n();
  if (m < k || m > 128 || m > n) throw Error(MGMLMC_ERR_ARG, "refine: block size must be in [N_tv, min(128, n)]");
  if (iters < 0 || !(tol >= 0.0) || !(solve_tol > 0.0 && solve_tol < 1.0))
    throw Error(MGMLMC_ERR_ARG, "refine: bad iteration count or tolerance");
  auto built_tv = [&](int j, size_t count) -> double2 * {
    auto it = ws_.find("tv#" + std::to_string(j) + "d");
    if (it == ws_.end() || it->second.second < count * sizeof(double2))
      throw Error(MGMLMC_ERR_STATE, "refine: the build's test vectors are gone");
    return static_cast<double2 *>(it->second.first);
  };
  const mgmlmc_mg_params params = mgp_;
  std::vector<double> hv((size_t)2 * k * n);
  std::vector<double> th(m), rh(m);
  {
    DevBuf<double2> Vb((size_t)m * n), Wb((size_t)m * n);
    double2 *V = Vb.p, *W = Wb.p;
    double2 *g = ws<double>("rfg", l, (size_t)8 * n);
    double2 *d = ws<double>("rfd", 0, (size_t)m);
    double2 *hc = ws<double>("rfc", 0, (size_t)m * m);
    MG_CUDA(cudaMemcpyAsync(V, built_tv(l, (size_t)k * n), sizeof(double2) * k * n, cudaMemcpyDeviceToDevice,
                            stream));
    if (m > k) z4_noise<double>(V + (size_t)k * n, G, seed, (uint64_t)k, 192 + l, 0, -1, m - k, stream);
    orthonormalise_cols(V, m, n);
    std::vector<double2> h((size_t)m * m);
    auto fetch = [&](const double2 *src, size_t count) {
      MG_CUDA(cudaMemcpyAsync(h.data(), src, sizeof(double2) * count, cudaMemcpyDeviceToHost, stream));
      sync();
    };
    // theta_r = Re <v_r, Q v_r>, rho_r = ||Q v_r - theta_r v_r|| (W is scratch)
    auto quotients = [&]() {
      for (int j0 = 0; j0 < m; j0 += 8)
        apply_D<double>(l, V + (size_t)j0 * n, W + (size_t)j0 * n, std::min(8, m - j0));
      gamma5_apply<double>(W, W, G.V, G.dof, m, stream);
      dot<double>(V, W, n, m, d, partials((size_t)reduce_blocks(n) * m), stream);
      fetch(d, m);
      for (int r = 0; r < m; ++r) {
        th[r] = h[r].x;
        axpby<double>(-th[r], V + (size_t)r * n, 1.0, W + (size_t)r * n, n, 1, stream);
      }
      dot<double>(W, W, n, m, d, partials((size_t)reduce_blocks(n) * m), stream);
      fetch(d, m);
      for (int r = 0; r < m; ++r) rh[r] = std::sqrt(std::max(h[r].x, 0.0));
    };
    auto step = [&]() {
      for (int j0 = 0; j0 < m; j0 += 8) {
        const int nb = std::min(8, m - j0);
        gamma5_apply<double>(V + (size_t)j0 * n, g, G.V, G.dof, nb, stream);
        solve(l, g, W + (size_t)j0 * n, nb);
      }
      // hc[r m + j] = <W_j, W_r> = (W^H W)_jr
      for (int r = 0; r < m; ++r)
        multi_dot<double>(W, n, m, W + (size_t)r * n, n, 1, hc + (size_t)r * m, m,
                          partials((size_t)reduce_blocks(n) * m), stream);
      fetch(hc, (size_t)m * m);
      std::vector<std::complex<double>> Gm((size_t)m * m), Y;
      for (int j = 0; j < m; ++j)
        for (int r = 0; r < m; ++r) {
          const std::complex<double> a(h[(size_t)r * m + j].x, h[(size_t)r * m + j].y);
          const std::complex<double> b(h[(size_t)j * m + r].x, h[(size_t)j * m + r].y);
          Gm[(size_t)j * m + r] = 0.5 * (a + std::conj(b));
        }
      std::vector<double> mu;
      if (herm_eig_jacobi(Gm, m, mu, Y) < 0) throw Error(MGMLMC_ERR_NUMERIC, "refine: eigensolver did not converge");
      std::vector<int> order(m);
      for (int j = 0; j < m; ++j) order[j] = j;
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return mu[a] > mu[b]; });
      for (int r = 0; r < m; ++r) {
        const int o = order[r];
        if (!(mu[o] > 0.0) || !std::isfinite(mu[o])) throw Error(MGMLMC_ERR_NUMERIC, "refine: rank-deficient block");
        const double f = 1.0 / std::sqrt(mu[o]);
        for (int j = 0; j < m; ++j) {
          const std::complex<double> c = Y[(size_t)j * m + o] * f;
          h[(size_t)r * m + j] = make_double2(c.real(), c.imag());
        }
      }
      MG_CUDA(cudaMemcpyAsync(hc, h.data(), sizeof(double2) * m * m, cudaMemcpyHostToDevice, stream));
      MG_CUDA(cudaMemsetAsync(V, 0, sizeof(double2) * m * n, stream));
      for (int r = 0; r < m; ++r)  // v_r = sum_j W_j C_jr
        multi_axpy<double>(W, n, m, V + (size_t)r * n, n, 1, hc + (size_t)r * m, m, 1.0, stream);
      sync();  // h is rewritten by the next fetch
    };
    const mgmlmc_solver_params keep = sp_;
    sp_.precision = MGMLMC_FP64;
    sp_.tol = solve_tol;
    try {
      quotients();
      steps = 0;
      auto converged = [&]() {
        if (!(tol > 0.0)) return false;
        double mx = 0.0;
        for (int j = 0; j < k; ++j) mx = std::max(mx, rh[j]);
        return mx <= tol;
      };
      while (!converged() && steps < iters) {
        step();
        quotients();
        ++steps;
      }
    } catch (...) {
      sp_ = keep;
      ws_release("rfg", l, true);
      throw;
    }
    sp_ = keep;
    ws_release("rfg", l, true);
    MG_CUDA(cudaMemcpyAsync(hv.data(), V, sizeof(double2) * k * n, cudaMemcpyDeviceToHost, stream));
    sync();
  }
  // canonical phase: the first entry of largest modulus real and positive
  for (int j = 0; j < k; ++j) {
    double *v = hv.data() + (size_t)2 * j * n;
    int64_t im = 0;
    double best = -1.0;
    for (int64_t i = 0; i < n; ++i) {
      const double a = std::hypot(v[2 * i], v[2 * i + 1]);
      if (a > best) {
        best = a;
        im = i;
      }
    }
    const std::complex<double> ph = std::conj(std::complex<double>(v[2 * im], v[2 * im + 1])) / best;
    for (int64_t i = 0; i < n; ++i) {
      const std::complex<double> x = std::complex<double>(v[2 * i], v[2 * i + 1]) * ph;
      v[2 * i] = x.real();
      v[2 * i + 1] = x.imag();
    }
    v[2 * im] = best;
    v[2 * im + 1] = 0.0;
  }
  // the levels above keep exactly the vectors they were built from
  for (int j = 0; j < l; ++j) {
    const int kj = levels_[j].agg.ntv;
    const int64_t nj = levels_[j].g.n();
    std::vector<double> hj((size_t)2 * kj * nj);
    MG_CUDA(cudaMemcpyAsync(hj.data(), built_tv(j, (size_t)kj * nj), sizeof(double2) * kj * nj,
                            cudaMemcpyDeviceToHost, stream));
    sync();
    imported_host_[j] = std::move(hj);
  }
  imported_host_[l] = std::move(hv);
  theta.assign(th.begin(), th.begin() + k);
  rho.assign(rh.begin(), rh.begin() + k);
  build_hierarchy(params);
}

void Engine::coarsest_trace(double *re, double *im) {
  if (!ready_) throw Error(MGMLMC_ERR_STATE, "hierarchy not built");
  const Level &c = levels_.back();
  double2 *d = ws<double>("ctr", 0, 1);
  dense_trace(c.Dinv64, (int)c.g.n(), d, stream);
  double2 h;
  MG_CUDA(cudaMemcpyAsync(&h, d, sizeof(double2), cudaMemcpyDeviceToHost, stream));
  sync();
  *re = h.x;
  *im = h.y;
}

void Engine::get_prolongator(int l, double *host) {
  if (!ready_ || l < 0 || l + 1 >= n_levels()) throw Error(MGMLMC_ERR_ARG, "no prolongator at that level");
  const Level &f = levels_[l];
  const size_t cnt = (size_t)f.agg.coarse.V * 2 * f.agg.ntv * f.agg.rows;
  double2 *tmp = ws<double>("pcan", l, cnt);
  prolongator_to_canonical(f.P64, tmp, f.agg, stream);
  MG_CUDA(cudaMemcpyAsync(host, tmp, cnt * sizeof(double2), cudaMemcpyDeviceToHost, stream));
  sync();
}

// the build leaves each level's test vectors in its "tv" workspace
void Engine::get_test_vectors(int l, double *host) {
  if (!ready_ || l < 0 || l + 1 >= n_levels()) throw Error(MGMLMC_ERR_ARG, "no test vectors at that level");
  const size_t cnt = (size_t)levels_[l].agg.ntv * levels_[l].g.n();
  auto it = ws_.find("tv#" + std::to_string(l) + "d");
  if (it == ws_.end() || it->second.second < cnt * sizeof(double2))
    throw Error(MGMLMC_ERR_STATE, "the build's test vectors are gone");
  MG_CUDA(cudaMemcpyAsync(host, it->second.first, cnt * sizeof(double2), cudaMemcpyDeviceToHost, stream));
  sync();
}

void Engine::get_coarse_op(int l, double *host) {
  if (!ready_ || l < 1 || l >= n_levels()) throw Error(MGMLMC_ERR_ARG, "no coarse operator at that level");
  const Level &c = levels_[l];
  const size_t cnt = (size_t)c.g.V * 9 * c.g.dof * c.g.dof;
  MG_CUDA(cudaMemcpyAsync(host, c.A64, cnt * sizeof(double2), cudaMemcpyDeviceToHost, stream));
  sync();
}

template void Engine::apply_D<double>(int, const C<double> *, C<double> *, int);
template void Engine::apply_D<float>(int, const C<float> *, C<float> *, int);
template void Engine::restrict_to<double>(int, const C<double> *, C<double> *, int);
template void Engine::restrict_to<float>(int, const C<float> *, C<float> *, int);
template void Engine::prolong_from<double>(int, const C<double> *, C<double> *, int, double);
template void Engine::prolong_from<float>(int, const C<float> *, C<float> *, int, double);
template void Engine::project_out<double>(int, const C<double> *, C<double> *, int);
template void Engine::project_out<float>(int, const C<float> *, C<float> *, int);

}  // namespace mg

namespace mg {
template C<double> *Engine::ws<double>(const std::string &, int, size_t);
template C<float> *Engine::ws<float>(const std::string &, int, size_t);
}  // namespace mg
