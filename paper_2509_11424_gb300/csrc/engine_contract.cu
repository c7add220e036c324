// Correlator and loop estimators on top of the level solves.
//
// Connected pseudoscalar correlator (Eq. connected-G) through the orthogonal
// split of Eq. full_ops_orth / Eq. G-split, with the accumulated prolongation
// of a level-l operator taken as Phat_{l-1} (Phat_0 = I):
//   B_l         = Phat_{l-1} J_l Phat_{l-1}^H,  J_l = (I - P_l P_l^H) D_l^-1
//   B_{L-1+l}   = Phat_{l-1} K_l Phat_{l-1}^H,  K_l = P_l P_l^H D_l^-1 - P_l D_{l+1}^-1 P_l^H
//   B_{2L-1}    = Phat_{L-1} D_L^-1 Phat_{L-1}^H
// Each term is sampled with Z4 noise x on a source slice t' through
//   G_rs(t) = (1/T) sum_t' tr(B_r(t+t',t') [Btil_s(t+t',t')]^H),
//   Btil = Gamma5 B^H Gamma5,
// i.e. X_rs(t) = (1/T) sum_t' (Btil_s x)|_{t+t'}^H (B_r x)|_{t+t'}.
// Because Gamma5 P_l = P_l Gamma5c and D_l is Gamma5-hermitian on every
// level (Galerkin), Btil needs no adjoint solves:
//   Jtil_l = D_l^-1 (I - P P^H),   Ktil_l = D_l^-1 P P^H - P D_{l+1}^-1 P^H,
// so two level-l solves per level give every B and Btil:
//   s1 = D_l^-1 (I - P P^H) u,  s2 = D_l^-1 P P^H u,  D_l^-1 u = s1 + s2.
//
// Oblique split (Sec. 4.1, the B_l of Eq. G-traditional, same reading of
// the accumulated prolongation):
//   B_l = Phat_{l-1} (D_l^-1 - P_l D_{l+1}^-1 P_l^H) Phat_{l-1}^H, l < L,
//   B_L = Phat_{L-1} D_L^-1 Phat_{L-1}^H;
// here Btil = Gamma5 B^H Gamma5 = B (Gamma5-hermiticity on every level), so
// one solve per level gives every B_l: with u_l = Phat_{l-1}^H x and
// d_l = D_l^-1 u_l, B_l x = Phat_{l-1} (d_l - P_l d_{l+1}).
//
// Disconnected loop (Eq. trace_equality_disconnected): X_r = x^H Gamma5 B_r x
// with Z4 noise x on slice t.
#include <algorithm>
#include <complex>

#include "engine.h"

namespace mg {

// B (and, for the correlator, Btil) for nb right-hand sides x on level 0.
// Layout of B, Bt: [R][nb][n0].  Plain: R = 1, B = D^-1 x; orthogonal:
// R = 2L - 1; oblique: R = L.
void Engine::contraction_vectors(int kind, int nb, double2 *x, double2 *B, double2 *Bt) {
  const int L = n_levels();
  const int64_t n0 = levels_[0].g.n();
  const int64_t s0 = (int64_t)nb * n0;
  if (kind == MGMLMC_EST_PLAIN) {
    solve(0, x, B, nb);
    if (Bt) MG_CUDA(cudaMemcpyAsync(Bt, B, sizeof(double2) * s0, cudaMemcpyDeviceToDevice, stream));
    return;
  }
  if (kind == MGMLMC_EST_OBLIQUE) {
    std::vector<double2 *> u(L), d(L);
    u[0] = x;
    for (int l = 0; l < L; ++l) {
      const int64_t n = levels_[l].g.n();
      if (l + 1 < L) {
        u[l + 1] = ws<double>("cvu", l + 1, (size_t)nb * levels_[l + 1].g.n());
        restrict_to<double>(l, u[l], u[l + 1], nb);
      }
      d[l] = ws<double>("cvd", l, (size_t)nb * n);
      solve(l, u[l], d[l], nb);  // the coarsest level: its dense inverse
    }
    for (int l = 0; l < L; ++l) {
      const int64_t n = levels_[l].g.n();
      double2 *v = d[l];
      if (l + 1 < L) {
        v = ws<double>("cvtmp", l, (size_t)nb * n);
        prolong_from<double>(l, d[l + 1], v, nb, 0.0);      // P d_{l+1}
        axpby<double>(1.0, d[l], -1.0, v, n, nb, stream);  // d_l - P d_{l+1}
      }
      // Phat_{l-1} v into B_l
      double2 *cur = v;
      for (int k = l - 1; k >= 0; --k) {
        double2 *nxt = (k == 0) ? B + (size_t)l * s0 : ws<double>("cvf", k, (size_t)nb * levels_[k].g.n());
        prolong_from<double>(k, cur, nxt, nb, 0.0);
        cur = nxt;
      }
      if (l == 0)
        MG_CUDA(cudaMemcpyAsync(B, v, sizeof(double2) * s0, cudaMemcpyDeviceToDevice, stream));
    }
    if (Bt)
      MG_CUDA(cudaMemcpyAsync(Bt, B, sizeof(double2) * s0 * L, cudaMemcpyDeviceToDevice, stream));
    return;
  }
  const int R = 2 * (L - 1) + 1;
  std::vector<double2 *> u(L), s1(L), s2(L), d(L);
  u[0] = x;
  for (int l = 0; l + 1 < L; ++l) {
    const int64_t n = levels_[l].g.n(), nc = levels_[l + 1].g.n();
    u[l + 1] = ws<double>("cvu", l + 1, (size_t)nb * nc);
    double2 *pu = ws<double>("cvpu", l, (size_t)nb * n);
    double2 *qu = ws<double>("cvqu", l, (size_t)nb * n);
    s1[l] = ws<double>("cvs1", l, (size_t)nb * n);
    s2[l] = ws<double>("cvs2", l, (size_t)nb * n);
    d[l] = ws<double>("cvd", l, (size_t)nb * n);
    restrict_to<double>(l, u[l], u[l + 1], nb);
    prolong_from<double>(l, u[l + 1], pu, nb, 0.0);
    MG_CUDA(cudaMemcpyAsync(qu, u[l], sizeof(double2) * nb * n, cudaMemcpyDeviceToDevice, stream));
    axpby<double>(-1.0, pu, 1.0, qu, n, nb, stream);
    if (Bt) {
      solve(l, qu, s1[l], nb);
      solve(l, pu, s2[l], nb);
      MG_CUDA(cudaMemcpyAsync(d[l], s1[l], sizeof(double2) * nb * n, cudaMemcpyDeviceToDevice, stream));
      axpby<double>(1.0, s2[l], 1.0, d[l], n, nb, stream);
    } else {
      solve(l, u[l], d[l], nb);
    }
  }
  {
    const int l = L - 1;
    const int64_t n = levels_[l].g.n();
    d[l] = ws<double>("cvd", l, (size_t)nb * n);
    coarsest_apply<double>(levels_[l].Dinv64, u[l], d[l], (int)n, nb);
  }
  // level-l vector -> fine vector (Phat_l) into dst
  auto to_fine = [&](int l, double2 *v, double2 *dst) {
    if (l == 0) {
      MG_CUDA(cudaMemcpyAsync(dst, v, sizeof(double2) * s0, cudaMemcpyDeviceToDevice, stream));
      return;
    }
    double2 *cur = v;
    for (int k = l - 1; k >= 0; --k) {
      double2 *nxt = (k == 0) ? dst : ws<double>("cvf", k, (size_t)nb * levels_[k].g.n());
      prolong_from<double>(k, cur, nxt, nb, 0.0);
      cur = nxt;
    }
  };
  for (int l = 0; l + 1 < L; ++l) {
    const int64_t n = levels_[l].g.n();
    double2 *pd = ws<double>("cvpd", l, (size_t)nb * n);   // P P^H D_l^-1 u
    double2 *pc = ws<double>("cvpc", l, (size_t)nb * n);   // P D_{l+1}^-1 P^H u
    double2 *tmp = ws<double>("cvtmp", l, (size_t)nb * n);
    double2 *dc = ws<double>("cvdc", l + 1, (size_t)nb * levels_[l + 1].g.n());
    restrict_to<double>(l, d[l], dc, nb);
    prolong_from<double>(l, dc, pd, nb, 0.0);
    prolong_from<double>(l, d[l + 1], pc, nb, 0.0);
    // J u = d - P P^H d
    MG_CUDA(cudaMemcpyAsync(tmp, d[l], sizeof(double2) * nb * n, cudaMemcpyDeviceToDevice, stream));
    axpby<double>(-1.0, pd, 1.0, tmp, n, nb, stream);
    to_fine(l, tmp, B + (size_t)l * s0);
    // K u = P P^H d - P c
    MG_CUDA(cudaMemcpyAsync(tmp, pd, sizeof(double2) * nb * n, cudaMemcpyDeviceToDevice, stream));
    axpby<double>(-1.0, pc, 1.0, tmp, n, nb, stream);
    to_fine(l, tmp, B + (size_t)(L - 1 + l) * s0);
    if (Bt) {
      to_fine(l, s1[l], Bt + (size_t)l * s0);
      MG_CUDA(cudaMemcpyAsync(tmp, s2[l], sizeof(double2) * nb * n, cudaMemcpyDeviceToDevice, stream));
      axpby<double>(-1.0, pc, 1.0, tmp, n, nb, stream);
      to_fine(l, tmp, Bt + (size_t)(L - 1 + l) * s0);
    }
  }
  to_fine(L - 1, d[L - 1], B + (size_t)(R - 1) * s0);
  if (Bt)
    MG_CUDA(cudaMemcpyAsync(Bt + (size_t)(R - 1) * s0, B + (size_t)(R - 1) * s0, sizeof(double2) * s0,
                            cudaMemcpyDeviceToDevice, stream));
}

void Engine::connected(int kind, int n_samples, uint64_t seed, uint64_t first,
                       std::vector<double> &mean, std::vector<double> &var, int &R) {
  if (!ready_) throw Error(MGMLMC_ERR_STATE, "hierarchy not built");
  if (kind != MGMLMC_EST_PLAIN && kind != MGMLMC_EST_ORTHOGONAL && kind != MGMLMC_EST_OBLIQUE)
    throw Error(MGMLMC_ERR_ARG, "unknown kind");
  if (n_samples < 1) throw Error(MGMLMC_ERR_ARG, "n_samples must be >= 1");
  const int L = n_levels();
  const Geom &g0 = levels_[0].g;
  const int T = g0.L[3];
  const int64_t n0 = g0.n(), ns = n0 / T;
  R = kind == MGMLMC_EST_PLAIN ? 1 : kind == MGMLMC_EST_OBLIQUE ? L : 2 * (L - 1) + 1;
  const int G = std::min(T, 8);  // source slices solved together
  std::vector<std::complex<double>> sum((size_t)R * R * T), cur((size_t)R * R * T);
  std::vector<double> sabs((size_t)R * R * T, 0.0);
  double2 *x = ws<double>("ccx", 0, (size_t)G * n0);
  double2 *B = ws<double>("ccB", 0, (size_t)R * G * n0);
  double2 *Bt = ws<double>("ccBt", 0, (size_t)R * G * n0);
  double2 *h = ws<double>("cch", 0, (size_t)T * R);
  for (int k = 0; k < n_samples; ++k) {
    std::fill(cur.begin(), cur.end(), std::complex<double>(0.0, 0.0));
    for (int t0 = 0; t0 < T; t0 += G) {
      const int nb = std::min(G, T - t0);
      for (int q = 0; q < nb; ++q)
        noise(0, seed, first + (uint64_t)k, 64, (uint64_t)(t0 + q), t0 + q, x + (size_t)q * n0, 1);
      contraction_vectors(kind, nb, x, B, Bt);
      const int64_t s0 = (int64_t)nb * n0;
      for (int r = 0; r < R; ++r) {
        for (int q = 0; q < nb; ++q) {
          // h[t * R + s] = <slice t of Bt_s, slice t of B_r> for source t0 + q
          multi_dot<double>(Bt + (size_t)q * n0, s0, R, B + (size_t)r * s0 + (size_t)q * n0, ns, T, h, R,
                            partials((size_t)reduce_blocks(ns) * T * R), stream);
          std::vector<double2> hh((size_t)T * R);
          MG_CUDA(cudaMemcpyAsync(hh.data(), h, sizeof(double2) * T * R, cudaMemcpyDeviceToHost, stream));
          sync();
          const int tp = t0 + q;
          for (int s = 0; s < R; ++s)
            for (int t = 0; t < T; ++t) {
              const double2 v = hh[(size_t)((t + tp) % T) * R + s];
              cur[((size_t)r * R + s) * T + t] += std::complex<double>(v.x, v.y) / (double)T;
            }
        }
      }
    }
    for (size_t i = 0; i < cur.size(); ++i) {
      sum[i] += cur[i];
      sabs[i] += std::norm(cur[i]);
    }
  }
  mean.assign(2 * sum.size(), 0.0);
  var.assign(sum.size(), 0.0);
  const double N = (double)n_samples;
  for (size_t i = 0; i < sum.size(); ++i) {
    const std::complex<double> mu = sum[i] / N;
    mean[2 * i] = mu.real();
    mean[2 * i + 1] = mu.imag();
    var[i] = n_samples > 1 ? std::max(0.0, (sabs[i] - N * std::norm(mu)) / (N - 1.0)) : 0.0;
  }
}

void Engine::disconnected(int kind, int t, int n_samples, uint64_t seed, uint64_t first,
                          std::vector<double> &mean, std::vector<double> &var, int &R) {
  if (!ready_) throw Error(MGMLMC_ERR_STATE, "hierarchy not built");
  if (kind != MGMLMC_EST_PLAIN && kind != MGMLMC_EST_ORTHOGONAL && kind != MGMLMC_EST_OBLIQUE)
    throw Error(MGMLMC_ERR_ARG, "unknown kind");
  const Geom &g0 = levels_[0].g;
  if (t < 0 || t >= g0.L[3]) throw Error(MGMLMC_ERR_ARG, "time slice out of range");
  if (n_samples < 1) throw Error(MGMLMC_ERR_ARG, "n_samples must be >= 1");
  const int L = n_levels();
  const int64_t n0 = g0.n();
  R = kind == MGMLMC_EST_PLAIN ? 1 : kind == MGMLMC_EST_OBLIQUE ? L : 2 * (L - 1) + 1;
  const int G = 8;
  double2 *x = ws<double>("dlx", 0, (size_t)G * n0);
  double2 *g5x = ws<double>("dlg", 0, (size_t)G * n0);
  double2 *B = ws<double>("dlB", 0, (size_t)R * G * n0);
  double2 *res = ws<double>("dlr", 0, (size_t)R * G);
  std::vector<std::complex<double>> sum(R);
  std::vector<double> sabs(R, 0.0);
  for (int k0 = 0; k0 < n_samples; k0 += G) {
    const int nb = std::min(G, n_samples - k0);
    noise(0, seed, first + (uint64_t)k0, 80, (uint64_t)t, t, x, nb);
    gamma5_apply<double>(x, g5x, g0.V, 12, nb, stream);
    contraction_vectors(kind, nb, x, B, nullptr);
    for (int r = 0; r < R; ++r)
      dot<double>(g5x, B + (size_t)r * nb * n0, n0, nb, res + (size_t)r * nb,
                  partials((size_t)reduce_blocks(n0) * nb), stream);
    std::vector<double2> hh((size_t)R * nb);
    MG_CUDA(cudaMemcpyAsync(hh.data(), res, sizeof(double2) * R * nb, cudaMemcpyDeviceToHost, stream));
    sync();
    for (int r = 0; r < R; ++r)
      for (int q = 0; q < nb; ++q) {
        const std::complex<double> v(hh[(size_t)r * nb + q].x, hh[(size_t)r * nb + q].y);
        sum[r] += v;
        sabs[r] += std::norm(v);
      }
  }
  mean.assign(2 * R, 0.0);
  var.assign(R, 0.0);
  const double N = (double)n_samples;
  for (int r = 0; r < R; ++r) {
    const std::complex<double> mu = sum[r] / N;
    mean[2 * r] = mu.real();
    mean[2 * r + 1] = mu.imag();
    var[r] = n_samples > 1 ? std::max(0.0, (sabs[r] - N * std::norm(mu)) / (N - 1.0)) : 0.0;
  }
}

}  // namespace mg
