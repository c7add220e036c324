// extern "C" boundary of libmgmlmc.so (declared in include/mgmlmc.h).  Every
// entry point catches the engine's exceptions and turns them into a status
// code plus a message retrievable with mgmlmc_last_error().
#include <complex>
#include <cstring>
#include <new>
#include <string>

#include "ctx.h"

namespace {
thread_local std::string g_create_error;

template <typename F> mgmlmc_status guard(mgmlmc_ctx *ctx, F &&f) {
  if (!ctx) return MGMLMC_ERR_ARG;
  try {
    ctx->eng->enter();
    struct Leave {
      mg::Engine *e;
      ~Leave() {
        try { e->leave(); } catch (...) {}
      }
    } leave{ctx->eng};
    f();
    return MGMLMC_OK;
  } catch (const mg::Error &e) {
    ctx->err = e.what();
    // a failed kernel launch may leave a sticky error state; surface it
    return (mgmlmc_status)e.code;
  } catch (const std::bad_alloc &) {
    ctx->err = "host allocation failed";
    return MGMLMC_ERR_OOM;
  } catch (const std::exception &e) {
    ctx->err = e.what();
    return MGMLMC_ERR_ARG;
  }
}

mg::Engine &E(mgmlmc_ctx *ctx) { return *ctx->eng; }
}  // namespace

extern "C" {

mgmlmc_status mgmlmc_create(const int dims[4], void *stream, mgmlmc_ctx **out) {
  if (!dims || !out) return MGMLMC_ERR_ARG;
  *out = nullptr;
  mgmlmc_ctx *ctx = new (std::nothrow) mgmlmc_ctx();
  if (!ctx) return MGMLMC_ERR_OOM;
  try {
    ctx->eng = new mg::Engine(dims, static_cast<cudaStream_t>(stream));
  } catch (const mg::Error &e) {
    g_create_error = e.what();
    delete ctx;
    return (mgmlmc_status)e.code;
  } catch (const std::exception &e) {
    g_create_error = e.what();
    delete ctx;
    return MGMLMC_ERR_OOM;
  }
  *out = ctx;
  return MGMLMC_OK;
}

void mgmlmc_destroy(mgmlmc_ctx *ctx) {
  if (!ctx) return;
  delete ctx->eng;
  delete ctx;
}

const char *mgmlmc_last_error(const mgmlmc_ctx *ctx) {
  if (!ctx) return g_create_error.c_str();
  return ctx->err.c_str();
}

mgmlmc_status mgmlmc_set_gauge(mgmlmc_ctx *ctx, const double *U, int on_device) {
  return guard(ctx, [&] {
    if (!U) throw mg::Error(MGMLMC_ERR_ARG, "U is NULL");
    E(ctx).set_gauge(U, on_device != 0);
  });
}

mgmlmc_status mgmlmc_get_gauge(mgmlmc_ctx *ctx, double *U, int on_device) {
  return guard(ctx, [&] {
    if (!U) throw mg::Error(MGMLMC_ERR_ARG, "U is NULL");
    E(ctx).get_gauge(U, on_device != 0);
  });
}

mgmlmc_status mgmlmc_deflation_build(mgmlmc_ctx *ctx, int k, int iters, double tol, uint64_t seed,
                                     double *exact, double *seconds) {
  return guard(ctx, [&] {
    std::complex<double> ex;
    double sec = 0.0;
    E(ctx).deflation_build(k, iters, tol, seed, ex, sec);
    if (exact) {
      exact[0] = ex.real();
      exact[1] = ex.imag();
    }
    if (seconds) *seconds = sec;
  });
}

mgmlmc_status mgmlmc_refine_test_vectors(mgmlmc_ctx *ctx, int level, int n_vec, int max_iters,
                                         double eig_tol, double solve_tol, uint64_t seed,
                                         double *theta, double *eig_res, int *steps) {
  return guard(ctx, [&] {
    std::vector<double> th, rh;
    int st = 0;
    E(ctx).refine_test_vectors(level, n_vec, max_iters, eig_tol, solve_tol, seed, th, rh, st);
    if (theta) std::memcpy(theta, th.data(), th.size() * sizeof(double));
    if (eig_res) std::memcpy(eig_res, rh.data(), rh.size() * sizeof(double));
    if (steps) *steps = st;
  });
}

mgmlmc_status mgmlmc_gen_gauge(mgmlmc_ctx *ctx, double eps, uint64_t seed) {
  return guard(ctx, [&] { E(ctx).gen_gauge(eps, seed); });
}

mgmlmc_status mgmlmc_set_mass(mgmlmc_ctx *ctx, double m0) {
  return guard(ctx, [&] { E(ctx).set_mass(m0); });
}

mgmlmc_status mgmlmc_set_solver(mgmlmc_ctx *ctx, const mgmlmc_solver_params *p) {
  return guard(ctx, [&] {
    if (!p) throw mg::Error(MGMLMC_ERR_ARG, "params is NULL");
    E(ctx).set_solver(*p);
  });
}

mgmlmc_status mgmlmc_set_test_vectors(mgmlmc_ctx *ctx, int level, const double *V, int n_tv,
                                      int64_t n, int on_device) {
  return guard(ctx, [&] { E(ctx).set_test_vectors(level, V, n_tv, n, on_device != 0); });
}

mgmlmc_status mgmlmc_build_hierarchy(mgmlmc_ctx *ctx, const mgmlmc_mg_params *p) {
  return guard(ctx, [&] {
    if (!p) throw mg::Error(MGMLMC_ERR_ARG, "params is NULL");
    E(ctx).build_hierarchy(*p);
  });
}

mgmlmc_status mgmlmc_level_info(const mgmlmc_ctx *cctx, int level, int dims[4], int *dof,
                                int64_t *n) {
  mgmlmc_ctx *ctx = const_cast<mgmlmc_ctx *>(cctx);
  return guard(ctx, [&] {
    if (level < 0 || level >= E(ctx).n_levels()) throw mg::Error(MGMLMC_ERR_ARG, "level out of range");
    const mg::Geom &g = E(ctx).level(level).g;
    if (dims)
      for (int i = 0; i < 4; ++i) dims[i] = g.L[i];
    if (dof) *dof = g.dof;
    if (n) *n = g.n();
  });
}

mgmlmc_status mgmlmc_estimate_trace(mgmlmc_ctx *ctx, const mgmlmc_est_params *p,
                                    mgmlmc_term_result *out, int max_terms, int *n_terms) {
  return guard(ctx, [&] {
    if (!p || !out || !n_terms) throw mg::Error(MGMLMC_ERR_ARG, "NULL argument");
    std::vector<mg::TermAcc> acc;
    ctx->last_samples.clear();
    E(ctx).estimate_trace(*p, acc);
    if ((int)acc.size() > max_terms) throw mg::Error(MGMLMC_ERR_ARG, "max_terms too small");
    *n_terms = (int)acc.size();
    for (const mg::TermAcc &a : acc) ctx->last_samples.push_back(a.samples);
    for (size_t i = 0; i < acc.size(); ++i) {
      const mg::TermAcc &a = acc[i];
      mgmlmc_term_result &r = out[i];
      std::memset(&r, 0, sizeof(r));
      r.term = a.term;
      r.n = a.n;
      r.sum_re = a.sre;
      r.sum_im = a.sim;
      r.sum_abs2 = a.sabs2;
      r.seconds = a.seconds;
      r.iters_mean = a.solves > 0 ? a.iters_sum / a.solves : 0.0;
      r.max_residual = a.max_res;
      if (a.n > 0) {
        r.mean_re = a.sre / a.n;
        r.mean_im = a.sim / a.n;
        double v = 0.0;
        for (const auto &x : a.samples) v += std::norm(x - std::complex<double>(r.mean_re, r.mean_im));
        r.var = a.n > 1 ? v / (a.n - 1) : 0.0;
      }
    }
  });
}

mgmlmc_status mgmlmc_last_samples(mgmlmc_ctx *ctx, int index, double *out, int max_samples, int *n) {
  return guard(ctx, [&] {
    if (!n) throw mg::Error(MGMLMC_ERR_ARG, "NULL argument");
    if (index < 0 || index >= (int)ctx->last_samples.size())
      throw mg::Error(MGMLMC_ERR_ARG, "no such term in the last estimate");
    const auto &X = ctx->last_samples[index];
    *n = (int)X.size();
    if ((int)X.size() > max_samples || (!out && !X.empty()))
      throw mg::Error(MGMLMC_ERR_ARG, "output holds fewer samples than the term has");
    for (size_t k = 0; k < X.size(); ++k) {
      out[2 * k] = X[k].real();
      out[2 * k + 1] = X[k].imag();
    }
  });
}

mgmlmc_status mgmlmc_test_staging_extra(mgmlmc_ctx *ctx, int extra_bytes) {
  return guard(ctx, [&] {
    if (extra_bytes < 0 || extra_bytes > 4096 || extra_bytes % 16)
      throw mg::Error(MGMLMC_ERR_ARG, "extra_bytes must be a multiple of 16 in 0 .. 4096");
    mg::set_staging_extra_bytes((unsigned)extra_bytes);
  });
}

mgmlmc_status mgmlmc_release_workspaces(mgmlmc_ctx *ctx) {
  return guard(ctx, [&] { E(ctx).release_workspaces(); });
}

mgmlmc_status mgmlmc_coarsest_trace(mgmlmc_ctx *ctx, double *re, double *im) {
  return guard(ctx, [&] {
    if (!re || !im) throw mg::Error(MGMLMC_ERR_ARG, "NULL argument");
    E(ctx).coarsest_trace(re, im);
  });
}

mgmlmc_status mgmlmc_connected_correlator(mgmlmc_ctx *ctx, int kind, int n_samples, uint64_t seed,
                                          uint64_t first_sample, double *mean, double *var, int *R) {
  return guard(ctx, [&] {
    if (!mean || !var || !R) throw mg::Error(MGMLMC_ERR_ARG, "NULL argument");
    std::vector<double> m, v;
    int r = 0;
    E(ctx).connected(kind, n_samples, seed, first_sample, m, v, r);
    std::memcpy(mean, m.data(), m.size() * sizeof(double));
    std::memcpy(var, v.data(), v.size() * sizeof(double));
    *R = r;
  });
}

mgmlmc_status mgmlmc_disconnected_loop(mgmlmc_ctx *ctx, int kind, int t, int n_samples, uint64_t seed,
                                       uint64_t first_sample, double *mean, double *var, int *R) {
  return guard(ctx, [&] {
    if (!mean || !var || !R) throw mg::Error(MGMLMC_ERR_ARG, "NULL argument");
    std::vector<double> m, v;
    int r = 0;
    E(ctx).disconnected(kind, t, n_samples, seed, first_sample, m, v, r);
    std::memcpy(mean, m.data(), m.size() * sizeof(double));
    std::memcpy(var, v.data(), v.size() * sizeof(double));
    *R = r;
  });
}

mgmlmc_status mgmlmc_reorder(mgmlmc_ctx *ctx, const void *in, void *out, int nrhs,
                             int to_internal) {
  return guard(ctx, [&] {
    mg::Engine &e = E(ctx);
    if (!in || !out || nrhs < 1) throw mg::Error(MGMLMC_ERR_ARG, "bad buffers or nrhs");
    mg::relayout<float, float>((const float2 *)in, (float2 *)out, nullptr, e.level(0).g.V, nrhs,
                               to_internal != 0, e.stream);
  });
}

mgmlmc_status mgmlmc_reorder_bf16(mgmlmc_ctx *ctx, const void *in, void *out, int nrhs,
                                  int to_internal) {
  return guard(ctx, [&] {
    mg::Engine &e = E(ctx);
    if (!in || !out || nrhs < 1) throw mg::Error(MGMLMC_ERR_ARG, "bad buffers or nrhs");
    mg::relayout_bf16(in, out, e.level(0).g.V, nrhs, to_internal != 0, e.stream);
  });
}

mgmlmc_status mgmlmc_apply(mgmlmc_ctx *ctx, int op_flags, int level, int precision, const void *in,
                           void *out, int nrhs) {
  return guard(ctx, [&] {
    mg::Engine &e = E(ctx);
    const bool internal = (op_flags & MGMLMC_LAYOUT_INTERNAL) != 0;
    const int op = op_flags & ~MGMLMC_LAYOUT_INTERNAL;
    if (!in || !out || nrhs < 1) throw mg::Error(MGMLMC_ERR_ARG, "bad buffers or nrhs");
    if (precision == MGMLMC_BF16) {
      if (op != MGMLMC_OP_D || level != 0)
        throw mg::Error(MGMLMC_ERR_ARG, "BF16 storage is available for the level-0 Wilson operator only");
      const mg::Geom &g = e.level(0).g;
      const size_t bytes = (size_t)g.n() * nrhs * 4;
      require_disjoint(in, bytes, out, bytes);
      const void *src = in;
      void *dst = out;
      if (!internal) {
        void *t = e.scratch32("api_in_bf16", (bytes + 7) / 8);
        mg::relayout_bf16(in, t, g.V, nrhs, true, e.stream);
        src = t;
        dst = e.scratch32("api_out_bf16", (bytes + 7) / 8);
      }
      e.apply_D_bf16(src, dst, nrhs);
      if (!internal) mg::relayout_bf16(dst, out, g.V, nrhs, false, e.stream);
      MG_CUDA(cudaGetLastError());
      return;
    }
    if (precision != MGMLMC_FP64 && precision != MGMLMC_FP32) throw mg::Error(MGMLMC_ERR_ARG, "bad precision");
    if (level < 0 || level >= e.n_levels()) throw mg::Error(MGMLMC_ERR_ARG, "level out of range");
    const bool dp = precision == MGMLMC_FP64;
    const bool needs_next = op == MGMLMC_OP_RESTRICT || op == MGMLMC_OP_PROLONG || op == MGMLMC_OP_PROJECT;
    if (needs_next && (!e.ready() || level + 1 >= e.n_levels()))
      throw mg::Error(MGMLMC_ERR_STATE, "no transfer operator at that level");
    if (level > 0 && !e.ready()) throw mg::Error(MGMLMC_ERR_STATE, "hierarchy not built");
    {
      const size_t es = dp ? sizeof(double2) : sizeof(float2);
      const size_t nl = (size_t)e.level(level).g.n();
      const size_t nn = needs_next ? (size_t)e.level(level + 1).g.n() : nl;
      const size_t nin = op == MGMLMC_OP_PROLONG ? nn : nl, nout = op == MGMLMC_OP_RESTRICT ? nn : nl;
      require_disjoint(in, nin * nrhs * es, out, nout * nrhs * es);
    }
    const bool fine_op = op == MGMLMC_OP_D || op == MGMLMC_OP_RESTRICT || op == MGMLMC_OP_PROLONG ||
                         op == MGMLMC_OP_PROJECT || op == MGMLMC_OP_SMOOTH || op == MGMLMC_OP_NET;
    if (!dp && level == 0 && fine_op && !internal) {
      // FP32 level-0 vectors live structure-of-arrays inside the library:
      // the caller's canonical buffers are reordered in and out
      const mg::Geom &g = e.level(0).g;
      const size_t cnt = (size_t)g.n() * nrhs;
      const bool fin = op != MGMLMC_OP_PROLONG, fout = op != MGMLMC_OP_RESTRICT;
      const float2 *src = (const float2 *)in;
      float2 *dst = (float2 *)out;
      if (fin) {
        float2 *t = e.scratch32("api_in32", cnt);
        mg::relayout<float, float>(src, t, nullptr, g.V, nrhs, true, e.stream);
        src = t;
      }
      if (fout) dst = e.scratch32("api_out32", cnt);
      switch (op) {
        case MGMLMC_OP_D: e.apply_D<float>(0, src, dst, nrhs); break;
        case MGMLMC_OP_RESTRICT: e.restrict_to<float>(0, src, dst, nrhs); break;
        case MGMLMC_OP_PROLONG: e.prolong_from<float>(0, src, dst, nrhs, 0.0); break;
        case MGMLMC_OP_PROJECT: e.project_out<float>(0, src, dst, nrhs); break;
        case MGMLMC_OP_SMOOTH: e.smooth_apply<float>(0, src, dst, nrhs); break;
        default: e.net_forward<float>(src, dst, nrhs); break;
      }
      if (fout) mg::relayout<float, float>(dst, (float2 *)out, nullptr, g.V, nrhs, false, e.stream);
      MG_CUDA(cudaGetLastError());
      return;
    }
    switch (op) {
      case MGMLMC_OP_D:
        if (dp) e.apply_D<double>(level, (const double2 *)in, (double2 *)out, nrhs);
        else e.apply_D<float>(level, (const float2 *)in, (float2 *)out, nrhs);
        if (level > 0) e.check_staging();  // a bounded wait of the stencil ran out
        break;
      case MGMLMC_OP_RESTRICT:
        if (dp) e.restrict_to<double>(level, (const double2 *)in, (double2 *)out, nrhs);
        else e.restrict_to<float>(level, (const float2 *)in, (float2 *)out, nrhs);
        break;
      case MGMLMC_OP_PROLONG:
        if (dp) e.prolong_from<double>(level, (const double2 *)in, (double2 *)out, nrhs, 0.0);
        else e.prolong_from<float>(level, (const float2 *)in, (float2 *)out, nrhs, 0.0);
        break;
      case MGMLMC_OP_PROJECT:
        if (dp) e.project_out<double>(level, (const double2 *)in, (double2 *)out, nrhs);
        else e.project_out<float>(level, (const float2 *)in, (float2 *)out, nrhs);
        break;
      case MGMLMC_OP_SOLVE:
        if (!dp) throw mg::Error(MGMLMC_ERR_ARG, "solve takes FP64 buffers");
        e.solve(level, (const double2 *)in, (double2 *)out, nrhs);
        break;
      case MGMLMC_OP_SMOOTH:
        if (dp) e.smooth_apply<double>(level, (const double2 *)in, (double2 *)out, nrhs);
        else e.smooth_apply<float>(level, (const float2 *)in, (float2 *)out, nrhs);
        break;
      case MGMLMC_OP_NET:
        if (level != 0) throw mg::Error(MGMLMC_ERR_ARG, "the network acts on level 0");
        if (dp) e.net_forward<double>((const double2 *)in, (double2 *)out, nrhs);
        else e.net_forward<float>((const float2 *)in, (float2 *)out, nrhs);
        break;
      case MGMLMC_OP_GAMMA5: {
        const mg::Geom &g = e.level(level).g;
        if (dp) mg::gamma5_apply<double>((const double2 *)in, (double2 *)out, g.V, g.dof, nrhs, e.stream);
        else mg::gamma5_apply<float>((const float2 *)in, (float2 *)out, g.V, g.dof, nrhs, e.stream);
        break;
      }
      default:
        throw mg::Error(MGMLMC_ERR_ARG, "unknown op");
    }
    MG_CUDA(cudaGetLastError());
  });
}

mgmlmc_status mgmlmc_noise(mgmlmc_ctx *ctx, int level, uint64_t seed, uint64_t first_sample,
                           uint64_t term, uint64_t aux, int slice, double *out, int nrhs) {
  return guard(ctx, [&] {
    mg::Engine &e = E(ctx);
    if (!out || nrhs < 1) throw mg::Error(MGMLMC_ERR_ARG, "bad buffer or nrhs");
    if (level < 0 || level >= e.n_levels()) throw mg::Error(MGMLMC_ERR_ARG, "level out of range");
    e.noise(level, seed, first_sample, term, aux, slice, (double2 *)out, nrhs);
  });
}

mgmlmc_status mgmlmc_get_prolongator(mgmlmc_ctx *ctx, int level, double *out) {
  return guard(ctx, [&] {
    if (!out) throw mg::Error(MGMLMC_ERR_ARG, "NULL argument");
    E(ctx).get_prolongator(level, out);
  });
}

mgmlmc_status mgmlmc_get_test_vectors(mgmlmc_ctx *ctx, int level, double *out) {
  return guard(ctx, [&] {
    if (!out) throw mg::Error(MGMLMC_ERR_ARG, "NULL argument");
    E(ctx).get_test_vectors(level, out);
  });
}

mgmlmc_status mgmlmc_get_coarse_op(mgmlmc_ctx *ctx, int level, double *out) {
  return guard(ctx, [&] {
    if (!out) throw mg::Error(MGMLMC_ERR_ARG, "NULL argument");
    E(ctx).get_coarse_op(level, out);
  });
}

mgmlmc_status mgmlmc_last_solve_stats(const mgmlmc_ctx *cctx, int *iters, double *residual) {
  mgmlmc_ctx *ctx = const_cast<mgmlmc_ctx *>(cctx);
  return guard(ctx, [&] {
    if (iters) *iters = E(ctx).last_solve.iters;
    if (residual) *residual = E(ctx).last_solve.residual;
  });
}

mgmlmc_status mgmlmc_learned_init(mgmlmc_ctx *ctx, int channels, uint64_t seed) {
  return guard(ctx, [&] { E(ctx).net_init(channels, seed); });
}

mgmlmc_status mgmlmc_learned_size(const mgmlmc_ctx *cctx, int64_t *n_complex) {
  mgmlmc_ctx *ctx = const_cast<mgmlmc_ctx *>(cctx);
  return guard(ctx, [&] {
    if (!n_complex) throw mg::Error(MGMLMC_ERR_ARG, "NULL argument");
    *n_complex = E(ctx).net_size();
  });
}

mgmlmc_status mgmlmc_learned_weights(mgmlmc_ctx *ctx, double *host, int set) {
  return guard(ctx, [&] {
    if (!host) throw mg::Error(MGMLMC_ERR_ARG, "NULL argument");
    E(ctx).net_weights(host, set != 0);
  });
}

mgmlmc_status mgmlmc_learned_loss_grad(mgmlmc_ctx *ctx, const double *r, int nrhs, double *loss,
                                       double *grad_host) {
  return guard(ctx, [&] {
    mg::Engine &e = E(ctx);
    if (!r || !loss || !grad_host || nrhs < 1) throw mg::Error(MGMLMC_ERR_ARG, "bad arguments");
    const int64_t tot = e.net_size();
    if (tot <= 0) throw mg::Error(MGMLMC_ERR_STATE, "network not initialised");
    double2 *g = nullptr;
    MG_CUDA(cudaMalloc(&g, sizeof(double2) * tot));
    try {
      *loss = e.net_loss_grad<double>((const double2 *)r, nrhs, g);
      MG_CUDA(cudaMemcpy(grad_host, g, sizeof(double2) * tot, cudaMemcpyDeviceToHost));
    } catch (...) {
      cudaFree(g);
      throw;
    }
    cudaFree(g);
  });
}

mgmlmc_status mgmlmc_learned_train(mgmlmc_ctx *ctx, const mgmlmc_train_params *p,
                                   mgmlmc_train_result *out) {
  return guard(ctx, [&] {
    if (!p || !out) throw mg::Error(MGMLMC_ERR_ARG, "NULL argument");
    std::memset(out, 0, sizeof(*out));
    E(ctx).net_train(*p, *out);
  });
}

mgmlmc_status mgmlmc_learned_stats(const mgmlmc_ctx *cctx, int64_t *fallbacks) {
  mgmlmc_ctx *ctx = const_cast<mgmlmc_ctx *>(cctx);
  return guard(ctx, [&] {
    if (fallbacks) *fallbacks = E(ctx).net_fallbacks();
  });
}

int64_t mgmlmc_kernel_launches(void) { return mg::launch_counter().load(); }

mgmlmc_status mgmlmc_profile(mgmlmc_ctx *ctx, int enable) {
  return guard(ctx, [&] { E(ctx).profile(enable != 0); });
}

mgmlmc_status mgmlmc_profile_stats(mgmlmc_ctx *ctx, int kernel_class, int64_t *launches,
                                   double *ms, double *bytes, double *flops) {
  return guard(ctx, [&] {
    const mg::KStat k = E(ctx).kstat(kernel_class);
    if (launches) *launches = k.launches;
    if (ms) *ms = k.ms;
    if (bytes) *bytes = k.bytes;
    if (flops) *flops = k.flops;
  });
}

int mgmlmc_kernel_variants(int kernel) {
  if (kernel == MGMLMC_VARIANT_DSLASH_FP32) return mg::wilson_fp32_variants();
  if (kernel == MGMLMC_VARIANT_STENCIL_FP32) return mg::Engine::stencil_variants();
  if (kernel == MGMLMC_VARIANT_SAP_FP32) return mg::sap_variants();
  if (kernel == MGMLMC_VARIANT_TRANSFER_FP32) return 2;
  return -1;
}

mgmlmc_status mgmlmc_set_kernel_variant(mgmlmc_ctx *ctx, int kernel, int variant) {
  return guard(ctx, [&] {
    if (kernel == MGMLMC_VARIANT_DSLASH_FP32) E(ctx).set_dslash_variant(variant);
    else if (kernel == MGMLMC_VARIANT_STENCIL_FP32) E(ctx).set_stencil_variant(variant);
    else if (kernel == MGMLMC_VARIANT_SAP_FP32) E(ctx).set_sap_variant(variant);
    else if (kernel == MGMLMC_VARIANT_TRANSFER_FP32) E(ctx).set_transfer_variant(variant);
    else throw mg::Error(MGMLMC_ERR_ARG, "unknown kernel");
  });
}

mgmlmc_status mgmlmc_get_kernel_variant(const mgmlmc_ctx *cctx, int kernel, int nrhs,
                                        int *variant) {
  mgmlmc_ctx *ctx = const_cast<mgmlmc_ctx *>(cctx);
  return guard(ctx, [&] {
    if (!variant) throw mg::Error(MGMLMC_ERR_ARG, "variant is null");
    if (kernel == MGMLMC_VARIANT_DSLASH_FP32) *variant = E(ctx).dslash_variant(nrhs);
    else if (kernel == MGMLMC_VARIANT_STENCIL_FP32) *variant = E(ctx).stencil_variant(1, nrhs);
    else if (kernel == MGMLMC_VARIANT_SAP_FP32) *variant = E(ctx).sap_variant();
    else if (kernel == MGMLMC_VARIANT_TRANSFER_FP32) *variant = E(ctx).transfer_variant();
    else throw mg::Error(MGMLMC_ERR_ARG, "unknown kernel");
  });
}

}  // extern "C"
