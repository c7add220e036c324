// mgmlmc_project_noalloc: the orthogonal projection out = (I - P_l P_l^H) in
// of mgmlmc_apply(MGMLMC_OP_PROJECT) for callers that must not allocate
// device memory during the call -- code running inside a CUDA stream capture
// that is not allowed to create allocations, processes whose device memory
// is reserved up front by a pool they do not control, or real-time loops that
// forbid allocator calls on the critical path.  The projection needs one
// intermediate buffer, the coarse vector P_l^H in; here it lives in a
// file-scope device array instead of a workspace the context would allocate
// on first use.
//
// The array is a per-device global: every GPU that loads this library holds
// it (2 MiB) until the process exits.  All calls on a device share it, so two
// calls whose kernels overlap on the GPU (different streams, or different
// contexts on the same device) race on it; serialise such calls.  Each call
// writes the coarse intermediate completely before reading it, so nothing has
// to be cleared between calls.
#include <mutex>

#include "ctx.h"

namespace {

constexpr int64_t kScratchComplexDoubles = int64_t(1) << 17;  // 2 MiB
__device__ __align__(256) double2 g_project_scratch[kScratchComplexDoubles];

constexpr int kMaxDevices = 64;
void *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device with that device current.
void *scratch_address() {
  int dev = 0;
  MG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) throw mg::Error(MGMLMC_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    MG_CUDA(cudaGetSymbolAddress(&p, g_project_scratch));
    g_scratch_ptr[dev] = p;
  }
  return g_scratch_ptr[dev];
}

}  // namespace

extern "C" mgmlmc_status mgmlmc_project_noalloc(mgmlmc_ctx *ctx, int level, int precision,
                                                const void *in, void *out, int nrhs) {
  if (!ctx) return MGMLMC_ERR_ARG;
  try {
    mg::Engine &e = *ctx->eng;
    if (!in || !out || nrhs < 1) throw mg::Error(MGMLMC_ERR_ARG, "bad buffers or nrhs");
    if (precision != MGMLMC_FP64 && precision != MGMLMC_FP32) throw mg::Error(MGMLMC_ERR_ARG, "bad precision");
    if (!e.ready() || level < 0 || level + 1 >= e.n_levels())
      throw mg::Error(MGMLMC_ERR_STATE, "no transfer operator at that level");
    const mg::Level &L = e.level(level);
    const int64_t n = L.g.n();
    const int64_t nc = L.agg.coarse.n();
    const int64_t capacity = precision == MGMLMC_FP64 ? kScratchComplexDoubles : 2 * kScratchComplexDoubles;
    if (nc * nrhs > capacity)
      throw mg::Error(MGMLMC_ERR_ARG,
                      "project_noalloc: nrhs * coarse length = " + std::to_string(nc * nrhs) +
                          " exceeds the fixed scratch of " + std::to_string(capacity) + " complex entries");
    const size_t es = precision == MGMLMC_FP64 ? sizeof(double2) : sizeof(float2);
    require_disjoint(in, (size_t)n * nrhs * es, out, (size_t)n * nrhs * es);
    void *scratch = scratch_address();
    e.enter();
    struct Leave {
      mg::Engine *e;
      ~Leave() {
        try { e->leave(); } catch (...) {}
      }
    } leave{&e};
    if (precision == MGMLMC_FP64) {
      auto *tmp = static_cast<double2 *>(scratch);
      mg::restrict_op<double>((const double2 *)in, tmp, L.P64, L.agg, nrhs, e.stream);
      mg::prolong_op<double>(tmp, (double2 *)out, L.P64, L.agg, nrhs, 0.0, e.stream);
      mg::axpby<double>(1.0, (const double2 *)in, -1.0, (double2 *)out, n, nrhs, e.stream);
    } else {
      auto *tmp = static_cast<float2 *>(scratch);
      mg::restrict_op<float>((const float2 *)in, tmp, L.P32, L.agg, nrhs, e.stream);
      mg::prolong_op<float>(tmp, (float2 *)out, L.P32, L.agg, nrhs, 0.0, e.stream);
      mg::axpby<float>(1.0, (const float2 *)in, -1.0, (float2 *)out, n, nrhs, e.stream);
    }
    return MGMLMC_OK;
  } catch (const mg::Error &err) {
    ctx->err = err.what();
    return (mgmlmc_status)err.code;
  } catch (const std::exception &err) {
    ctx->err = err.what();
    return MGMLMC_ERR_ARG;
  }
}
