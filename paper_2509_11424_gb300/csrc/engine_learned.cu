// The learned smoother: a three-layer gauge-covariant network, its loss and
// gradients, training on residuals the solver produces (Adam on the GPU), and
// its use as the fine-level smoother.  Not part of the paper; the
// trace estimators stay unbiased because every solve is still judged by its
// true FP64 residual.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "engine.h"

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
__global__ void neg_inv_kernel(double *out, const double2 *nrm, int B) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < B) out[r] = nrm[r].x > 0.0 ? -1.0 / nrm[r].x : 0.0;
}
}  // namespace

void Engine::net_free() {
  for (int i = 0; i < 3; ++i) {
    dfree(net_.W64[i]);
    dfree(net_.W32[i]);
    dfree(net_.m[i]);
    dfree(net_.v[i]);
  }
  net_.C = 0;
}

void Engine::net_init(int channels, uint64_t seed) {
  if (channels < 1 || channels > 32) throw Error(MGMLMC_ERR_ARG, "channels must be in 1..32");
  drop_graphs();
  net_free();
  net_.C = channels;
  const int cin[3] = {1, channels, channels}, cout[3] = {channels, channels, 1};
  for (int i = 0; i < 3; ++i) {
    net_.cin[i] = cin[i];
    net_.cout[i] = cout[i];
    net_.cnt[i] = (int64_t)9 * cout[i] * cin[i] * 16;
    net_.W64[i] = dalloc<double2>(net_.cnt[i]);
    net_.W32[i] = dalloc<float2>(net_.cnt[i]);
    net_.m[i] = dalloc<double2>(net_.cnt[i]);
    net_.v[i] = dalloc<double2>(net_.cnt[i]);
    MG_CUDA(cudaMemsetAsync(net_.m[i], 0, sizeof(double2) * net_.cnt[i], stream));
    MG_CUDA(cudaMemsetAsync(net_.v[i], 0, sizeof(double2) * net_.cnt[i], stream));
    // small Z4 draws from the library's own Philox stream (term 112 + layer)
    Geom flat{};
    flat.L[0] = (int)net_.cnt[i];
    flat.L[1] = flat.L[2] = flat.L[3] = 1;
    flat.V = (int)net_.cnt[i];
    flat.dof = 1;
    z4_noise<double>(net_.W64[i], flat, seed, 0, 112 + i, 0, -1, 1, stream);
    axpby<double>(0.0, net_.W64[i], 0.01, net_.W64[i], net_.cnt[i], 1, stream);
  }
  // channel 0 carries the input; the last layer scales it to a Jacobi step
  std::vector<double2> h;
  for (int i = 0; i < 3; ++i) {
    h.resize(net_.cnt[i]);
    MG_CUDA(cudaMemcpyAsync(h.data(), net_.W64[i], sizeof(double2) * net_.cnt[i], cudaMemcpyDeviceToHost, stream));
    sync();
    const double sc = i == 2 ? 1.0 / (4.0 + m0_) : 1.0;
    for (int s = 0; s < 4; ++s) h[s * 4 + s].x += sc;  // W[h=0][o=0][c=0] = I (scaled)
    MG_CUDA(cudaMemcpyAsync(net_.W64[i], h.data(), sizeof(double2) * net_.cnt[i], cudaMemcpyHostToDevice, stream));
    convert<float, double>(net_.W64[i], net_.W32[i], net_.cnt[i], stream);
  }
  net_.adam_t = 0;
  sync();
}

int64_t Engine::net_size() const { return net_.cnt[0] + net_.cnt[1] + net_.cnt[2]; }

void Engine::net_weights(double *host, bool set) {
  if (!net_.C) throw Error(MGMLMC_ERR_STATE, "network not initialised");
  size_t off = 0;
  for (int i = 0; i < 3; ++i) {
    const size_t bytes = sizeof(double2) * net_.cnt[i];
    if (set) {
      MG_CUDA(cudaMemcpyAsync(net_.W64[i], host + 2 * off, bytes, cudaMemcpyHostToDevice, stream));
      convert<float, double>(net_.W64[i], net_.W32[i], net_.cnt[i], stream);
    } else {
      MG_CUDA(cudaMemcpyAsync(host + 2 * off, net_.W64[i], bytes, cudaMemcpyDeviceToHost, stream));
    }
    off += net_.cnt[i];
  }
  if (set) drop_graphs();
  sync();
}

template <typename T> void Engine::net_forward(const C<T> *in, C<T> *out, int B) {
  if (!net_.C) throw Error(MGMLMC_ERR_STATE, "network not initialised");
  const Level &L = levels_[0];
  const int64_t n = L.g.n();
  C<T> *a1 = ws<T>("neta1", 0, (size_t)net_.C * B * n);
  C<T> *a2 = ws<T>("neta2", 0, (size_t)net_.C * B * n);
  const C<T> *U;
  const C<T> *W[3];
  if constexpr (sizeof(T) == 8) {
    U = L.U64;
    for (int i = 0; i < 3; ++i) W[i] = net_.W64[i];
  } else {
    U = L.UD32;  // structure-of-arrays links for the FP32 (SoA) activations
    for (int i = 0; i < 3; ++i) W[i] = net_.W32[i];
  }
  glayer_forward<T>(in, a1, W[0], U, L.g, 1, net_.C, B, stream);
  glayer_forward<T>(a1, a2, W[1], U, L.g, net_.C, net_.C, B, stream);
  glayer_forward<T>(a2, out, W[2], U, L.g, net_.C, 1, B, stream);
}

template <typename T> double Engine::net_loss_grad(const C<T> *r, int B, double2 *grad) {
  const Level &L = levels_[0];
  const int64_t n = L.g.n();
  const int Cc = net_.C;
  C<T> *out = ws<T>("netout", 0, (size_t)B * n);
  C<T> *t1 = ws<T>("nett1", 0, (size_t)B * n);
  C<T> *t2 = ws<T>("nett2", 0, (size_t)B * n);
  C<T> *g2 = ws<T>("netg2", 0, (size_t)Cc * B * n);
  C<T> *g1 = ws<T>("netg1", 0, (size_t)Cc * B * n);
  double2 *nr = ws<double>("netnr", 0, (size_t)2 * B + 2);
  double *sc = reinterpret_cast<double *>(ws<double>("netsc", 0, (size_t)B));
  double2 *part = ws<double>("netpart", 0, (size_t)glayer_wgrad_chunks(L.g) * 9 * Cc * Cc * 16);
  net_forward<T>(r, out, B);
  C<T> *a1 = ws<T>("neta1", 0, (size_t)Cc * B * n);
  C<T> *a2 = ws<T>("neta2", 0, (size_t)Cc * B * n);
  // v = r - D N(r) in t2
  apply_D<T>(0, out, t1, B);
  MG_CUDA(cudaMemcpyAsync(t2, r, sizeof(C<T>) * n * B, cudaMemcpyDeviceToDevice, stream));
  axpby<T>(-1.0, t1, 1.0, t2, n, B, stream);
  dot<T>(r, r, n, B, nr, partials((size_t)reduce_blocks(n) * B), stream);
  dot<T>(t2, t2, n, B, nr + B, partials((size_t)reduce_blocks(n) * B), stream);
  std::vector<double2> h(2 * B);
  MG_CUDA(cudaMemcpyAsync(h.data(), nr, sizeof(double2) * 2 * B, cudaMemcpyDeviceToHost, stream));
  // G3 = -D^H v / ||r||^2 = -Gamma5 D Gamma5 v / ||r||^2  (in out)
  constexpr bool soa = sizeof(T) == 4;
  gamma5_apply<T>(t2, t1, L.g.V, 12, B, stream, soa);
  apply_D<T>(0, t1, out, B);
  gamma5_apply<T>(out, t1, L.g.V, 12, B, stream, soa);
  neg_inv_kernel<<<(B + 63) / 64, 64, 0, stream>>>(sc, nr, B);
  MG_LAUNCH_CHECK();
  scale_rhs<T>(t1, out, sc, n, B, stream);
  const C<T> *U;
  const C<T> *W[3];
  if constexpr (sizeof(T) == 8) {
    U = L.U64;
    for (int i = 0; i < 3; ++i) W[i] = net_.W64[i];
  } else {
    U = L.UD32;  // structure-of-arrays links for the FP32 (SoA) activations
    for (int i = 0; i < 3; ++i) W[i] = net_.W32[i];
  }
  double2 *gW[3] = {grad, grad + net_.cnt[0], grad + net_.cnt[0] + net_.cnt[1]};
  glayer_wgrad<T>(out, a2, U, L.g, Cc, 1, B, part, gW[2], stream);
  glayer_adjoint<T>(out, g2, W[2], U, L.g, Cc, 1, B, stream);
  glayer_wgrad<T>(g2, a1, U, L.g, Cc, Cc, B, part, gW[1], stream);
  glayer_adjoint<T>(g2, g1, W[1], U, L.g, Cc, Cc, B, stream);
  glayer_wgrad<T>(g1, r, U, L.g, 1, Cc, B, part, gW[0], stream);
  sync();
  double loss = 0.0;
  for (int b = 0; b < B; ++b) loss += h[b].x > 0 ? h[B + b].x / h[b].x : 0.0;
  return loss;
}

template <typename T> void Engine::record(const C<T> *res, int nrhs) {
  if (!recording_ || pool_n_ >= pool_cap_) return;
  const int64_t n = levels_[0].g.n();
  const int k = std::min(nrhs, pool_cap_ - pool_n_);
  // the pool holds FP32 fine-level vectors, i.e. structure-of-arrays
  if constexpr (sizeof(T) == 8)
    relayout<float, double>(res, pool_ + (size_t)pool_n_ * n, nullptr, levels_[0].g.V, k, true, stream);
  else MG_CUDA(cudaMemcpyAsync(pool_ + (size_t)pool_n_ * n, res, sizeof(float2) * n * k, cudaMemcpyDeviceToDevice, stream));
  pool_n_ += k;
}

void Engine::net_train(const mgmlmc_train_params &p, mgmlmc_train_result &out) {
  if (!ready_) throw Error(MGMLMC_ERR_STATE, "hierarchy not built");
  if (p.steps < 1 || p.batch < 1 || p.batch > 64 || p.pool < p.batch || !(p.lr > 0.0) ||
      (p.source != 0 && p.source != 1))
    throw Error(MGMLMC_ERR_ARG, "invalid training parameters");
  if (p.source == 1 && n_levels() < 2)
    throw Error(MGMLMC_ERR_ARG, "training source 1 needs a coarse level (the projector of the O_0 term)");
  const auto t0 = std::chrono::steady_clock::now();
  if (net_.C != p.channels) net_init(p.channels, p.seed);
  const int64_t n = levels_[0].g.n();
  // 1. residual / error pairs from the solver: the inputs of its fine-level
  //    smoother during solves of Z4 right-hand sides (SAP when the learned
  //    smoother is selected, so the pairs never depend on the network), or
  //    (source 1) the right-hand sides its fine-level solves start from
  const int saved = sp_.smoother, saved_guess = sp_.learned_guess;
  if (sp_.smoother == MGMLMC_SMOOTHER_LEARNED || sp_.smoother == MGMLMC_SMOOTHER_NET)
    sp_.smoother = MGMLMC_SMOOTHER_SAP;
  sp_.learned_guess = 0;
  drop_graphs();
  if (pool_) cudaFree(pool_);
  pool_ = nullptr;
  pool_cap_ = p.pool;
  pool_n_ = 0;
  {
    void *q = nullptr;
    MG_CUDA(cudaMalloc(&q, sizeof(float2) * (size_t)p.pool * n + 256));
    pool_ = static_cast<float2 *>(q);
  }
  const int nb = 8;
  double2 *b = ws<double>("trb", 0, (size_t)nb * n), *x = ws<double>("trx", 0, (size_t)nb * n);
  recording_ = true;
  try {
    if (p.source == 1) {
      // the right-hand sides of the estimator's O_0 solves, (I - P P^H) x
      // for fine Z4 noise x (noise stream 113 of the training seed)
      for (int k = 0; pool_n_ < pool_cap_ && k < 400; ++k) {
        z4_noise<double>(b, levels_[0].g, p.seed, (uint64_t)k * nb, 113, 0, -1, nb, stream);
        project_out<double>(0, b, x, nb);
        record<double>(x, nb);
      }
    } else {
      for (int k = 0; pool_n_ < pool_cap_ && k < 400; ++k) {
        z4_noise<double>(b, levels_[0].g, p.seed, (uint64_t)k * nb, 113, 0, -1, nb, stream);
        solve(0, b, x, nb);
      }
    }
  } catch (...) {
    recording_ = false;
    sp_.smoother = saved;
    sp_.learned_guess = saved_guess;
    throw;
  }
  recording_ = false;
  sp_.smoother = saved;
  sp_.learned_guess = saved_guess;
  drop_graphs();
  const int P = pool_n_;
  if (P < p.batch) throw Error(MGMLMC_ERR_STATE, "too few training pairs collected");
  // 2. Adam on the GPU (FP32 forward / backward, FP64 master weights)
  const int64_t tot = net_size();
  double2 *grad = ws<double>("trgrad", 0, (size_t)tot);
  float2 *batch = ws<float>("trbatch", 0, (size_t)p.batch * n);
  std::vector<double> losses;
  auto fill = [&](int step) {
    for (int j = 0; j < p.batch; ++j) {
      const int idx = (int)(((int64_t)step * p.batch + j) % P);
      MG_CUDA(cudaMemcpyAsync(batch + (size_t)j * n, pool_ + (size_t)idx * n, sizeof(float2) * n,
                              cudaMemcpyDeviceToDevice, stream));
    }
  };
  fill(0);
  out.loss_init = net_loss_grad<float>(batch, p.batch, grad) / p.batch;
  for (int step = 0; step < p.steps; ++step) {
    fill(step);
    const double L = net_loss_grad<float>(batch, p.batch, grad) / p.batch;
    losses.push_back(L);
    if (!std::isfinite(L)) throw Error(MGMLMC_ERR_NUMERIC, "training loss is not finite");
    ++net_.adam_t;
    for (int i = 0; i < 3; ++i) {
      double2 *g = grad + (i == 0 ? 0 : (i == 1 ? net_.cnt[0] : net_.cnt[0] + net_.cnt[1]));
      adam_step(net_.W64[i], g, net_.m[i], net_.v[i], net_.cnt[i], p.lr, 0.9, 0.999, 1e-8, net_.adam_t,
                1.0 / p.batch, stream);
      convert<float, double>(net_.W64[i], net_.W32[i], net_.cnt[i], stream);
    }
  }
  sync();
  const int w = std::min<int>(10, (int)losses.size());
  double f = 0, l = 0;
  for (int i = 0; i < w; ++i) {
    f += losses[i];
    l += losses[losses.size() - 1 - i];
  }
  out.steps = p.steps;
  out.pairs = P;
  out.loss_first = f / w;
  out.loss_last = l / w;
  out.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  cudaFree(pool_);
  pool_ = nullptr;
  pool_cap_ = pool_n_ = 0;
}

template void Engine::net_forward<double>(const C<double> *, C<double> *, int);
template void Engine::net_forward<float>(const C<float> *, C<float> *, int);
template double Engine::net_loss_grad<double>(const C<double> *, int, double2 *);
template double Engine::net_loss_grad<float>(const C<float> *, int, double2 *);
template void Engine::record<double>(const C<double> *, int);
template void Engine::record<float>(const C<float> *, int);

}  // namespace mg
