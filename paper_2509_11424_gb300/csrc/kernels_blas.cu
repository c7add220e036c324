// Level-1 vector kernels (batched over right-hand sides) and the per-rhs
// small-matrix kernels of batched FGMRES.
//
// Reductions are deterministic: a fixed number of blocks (a function of n
// only) writes partial sums that the last block to finish adds in block
// order, so a result never depends on scheduling.  Sums are accumulated in
// FP64 for both storage precisions.
#include "kernels.h"

#include <map>
#include <mutex>
#include <utility>

namespace mg {

namespace {
constexpr int RB = 256;  // reduction block size

__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// block-wide sum; valid in thread 0
__device__ __forceinline__ double2 block_sum(double2 v) {
  __shared__ double2 sh[RB / 32];
  v = warp_sum(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < (int)(blockDim.x >> 5)) ? sh[l] : make_double2(0.0, 0.0);
    v = warp_sum(v);
  }
  __syncthreads();
  return v;
}

// Single-pass reductions.  Block b of output g sums its chunk, writes the
// partial, and takes a ticket; the block that draws the last ticket adds the
// NB partials of g in block order (so the result never depends on
// scheduling) and puts the ticket back to zero.  Nothing waits on anything.
__device__ __forceinline__ bool last_block(unsigned *ticket) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();  // this block's partial is visible before its ticket
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  return last;
}

__device__ __forceinline__ double2 sum_partials(const double2 *p, int NB) {
  __threadfence();
  double2 acc = make_double2(0.0, 0.0);
  for (int b = threadIdx.x; b < NB; b += blockDim.x) {
    const double2 v = __ldcg(p + b);
    acc.x += v.x;
    acc.y += v.y;
  }
  return block_sum(acc);
}

// out[r * ldh + j] = sum conj(x_j,r) y_r; output g = j * nrhs + r, its NB
// partials at partial[g * NB ..]
template <typename T>
__global__ void dot_kernel(const C<T> *__restrict__ x, int64_t xstride, const C<T> *__restrict__ y,
                           int64_t n, int64_t chunk, double2 *__restrict__ partial,
                           unsigned *__restrict__ ticket, double2 *__restrict__ out, int ldh) {
  const int b = blockIdx.x, r = blockIdx.y, j = blockIdx.z;
  const int64_t g = (int64_t)j * gridDim.y + r;
  const C<T> *xr = x + j * xstride + r * n;
  const C<T> *yr = y + r * n;
  const int64_t beg = (int64_t)b * chunk;
  const int64_t end = beg + chunk < n ? beg + chunk : n;
  // per-thread partial in the storage precision over the few elements a
  // thread visits (reduce_blocks keeps that short; FP32 FMAs run ~58x faster
  // than FP64 ones on this part), then FP64 across threads and blocks
  C<T> acc = mk<T>((T)0, (T)0);
  for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x) {
    const C<T> a = xr[i], c = yr[i];
    acc = cfmac(a, c, acc);
  }
  const double2 tot = block_sum(make_double2((double)acc.x, (double)acc.y));
  if (threadIdx.x == 0) partial[g * gridDim.x + b] = tot;
  if (!last_block(ticket + g)) return;
  const double2 s = sum_partials(partial + g * gridDim.x, gridDim.x);
  if (threadIdx.x == 0) {
    out[r * ldh + j] = s;
    ticket[g] = 0u;
  }
}

// oqr[r] = <q_r, r_r>, oqq[r] = <q_r, q_r>; output r, partials at
// partial[(2 r + o) * NB ..]
template <typename T>
__global__ void dot_qr_kernel(const C<T> *__restrict__ q, const C<T> *__restrict__ rr, int64_t n,
                              int64_t chunk, double2 *__restrict__ partial,
                              unsigned *__restrict__ ticket, double2 *__restrict__ oqr,
                              double2 *__restrict__ oqq) {
  const int b = blockIdx.x, r = blockIdx.y;
  const C<T> *qr = q + r * n;
  const C<T> *xr = rr + r * n;
  const int64_t beg = (int64_t)b * chunk;
  const int64_t end = beg + chunk < n ? beg + chunk : n;
  C<T> ta = mk<T>((T)0, (T)0);
  T tc = (T)0;
  for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x) {
    const C<T> u = qr[i], v = xr[i];
    ta = cfmac(u, v, ta);
    tc = fma(u.x, u.x, fma(u.y, u.y, tc));
  }
  const double2 a = block_sum(make_double2((double)ta.x, (double)ta.y));
  const double2 c = block_sum(make_double2((double)tc, 0.0));
  if (threadIdx.x == 0) {
    partial[((int64_t)r * 2 + 0) * gridDim.x + b] = a;
    partial[((int64_t)r * 2 + 1) * gridDim.x + b] = c;
  }
  if (!last_block(ticket + r)) return;
  const double2 sa = sum_partials(partial + ((int64_t)r * 2 + 0) * gridDim.x, gridDim.x);
  const double2 sc = sum_partials(partial + ((int64_t)r * 2 + 1) * gridDim.x, gridDim.x);
  if (threadIdx.x == 0) {
    oqr[r] = sa;
    oqq[r] = sc;
    ticket[r] = 0u;
  }
}

template <typename T>
__global__ void multi_axpy_kernel(const C<T> *__restrict__ V, int64_t vstride, int k,
                                  C<T> *__restrict__ w, int64_t n, const double2 *__restrict__ h,
                                  int ldh, double sign) {
  __shared__ C<T> coef[128];
  const int r = blockIdx.y;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double2 c = h[r * ldh + j];
    coef[j] = mk<T>((T)(sign * c.x), (T)(sign * c.y));
  }
  __syncthreads();
  C<T> *wr = w + r * n;
  const C<T> *Vr = V + r * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    C<T> acc = wr[i];
    for (int j = 0; j < k; ++j) acc = cfma(coef[j], Vr[j * vstride + i], acc);
    wr[i] = acc;
  }
}

template <typename T>
__global__ void axpby_kernel(T a, const C<T> *__restrict__ x, T b, C<T> *__restrict__ y,
                             int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    C<T> xv = x[i], yv = y[i];
    yv.x = a * xv.x + b * yv.x;
    yv.y = a * xv.y + b * yv.y;
    y[i] = yv;
  }
}

template <typename T>
__global__ void scale_rhs_kernel(const C<T> *x, C<T> *y,  // may alias (in-place scaling)
                                 const double *__restrict__ scal, int64_t n) {
  const int r = blockIdx.y;
  const T f = (T)scal[r];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[r * n + i] = cscale(x[r * n + i], f);
}

template <typename T>
__global__ void mr_update_kernel(C<T> *__restrict__ z, C<T> *__restrict__ res,
                                 const C<T> *__restrict__ q, const double2 *__restrict__ dqr,
                                 const double2 *__restrict__ nq, int64_t n) {
  const int r = blockIdx.y;
  const double qq = nq[r].x;
  const double2 d = dqr[r];
  const C<T> al = qq > 0.0 ? mk<T>((T)(d.x / qq), (T)(d.y / qq)) : mk<T>((T)0, (T)0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = r * n + i;
    C<T> rv = res[o];
    z[o] = cfma(al, rv, z[o]);
    res[o] = cfma(cneg(al), q[o], rv);
  }
}

// z += alpha e; r -= alpha q with alpha = <q, r> / <q, q> per rhs
template <typename T>
__global__ void mr_dir_kernel(C<T> *__restrict__ z, C<T> *__restrict__ res, const C<T> *__restrict__ e,
                              const C<T> *__restrict__ q, const double2 *__restrict__ dqr,
                              const double2 *__restrict__ nq, int64_t n) {
  const int r = blockIdx.y;
  const double qq = nq[r].x;
  const double2 d = dqr[r];
  const C<T> al = qq > 1e-280 ? mk<T>((T)(d.x / qq), (T)(d.y / qq)) : mk<T>((T)0, (T)0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = r * n + i;
    z[o] = cfma(al, e[o], z[o]);
    res[o] = cfma(cneg(al), q[o], res[o]);
  }
}

template <typename To, typename From>
__global__ void convert_kernel(const C<From> *__restrict__ in, C<To> *__restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = cvt<To>(in[i]);
}

template <typename To, typename From>
__global__ void convert_scale_kernel(const C<From> *__restrict__ in, C<To> *__restrict__ out,
                                     const double *__restrict__ scal, int64_t n) {
  const int r = blockIdx.y;
  const double f = scal[r];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    C<From> v = in[r * n + i];
    out[r * n + i] = mk<To>((To)(v.x * f), (To)(v.y * f));
  }
}

// y_r = x_r * scal[r] (scal may be null: 1) between the canonical order
// [site][12] and the fine level's structure-of-arrays order (to_soa: x
// canonical, y SoA; else the reverse), converting precision.  One thread per
// (site, chunk of two components), chunks of a site on consecutive threads.
template <typename To, typename From>
__global__ void relayout_kernel(const C<From> *__restrict__ x, C<To> *__restrict__ y,
                                const double *__restrict__ scal, int64_t V, bool to_soa) {
  const int r = blockIdx.y;
  const double f = scal ? scal[r] : 1.0;
  const int64_t n = V * 12;
  const C<From> *xr = x + r * n;
  C<To> *yr = y + r * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < V * 6;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = e / 6;
    const int k = (int)(e - s * 6);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int64_t ic = s * 12 + 2 * k + j, is = soa_index(s, 2 * k + j, V);
      const C<From> v = xr[to_soa ? ic : is];
      yr[to_soa ? is : ic] = mk<To>((To)(v.x * f), (To)(v.y * f));
    }
  }
}

template <typename T, typename Tlo>
__global__ void add_lo_kernel(const C<Tlo> *__restrict__ x, C<T> *__restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    C<T> v = y[i];
    C<Tlo> a = x[i];
    v.x += (T)a.x;
    v.y += (T)a.y;
    y[i] = v;
  }
}

template <typename T>
__global__ void finite_kernel(const C<T> *__restrict__ x, int64_t n, int *flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    C<T> v = x[i];
    if (!isfinite(v.x) || !isfinite(v.y)) {
      *flag = 1;
      return;
    }
  }
}

inline int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

// ----------------------------------------------------------------- FGMRES
__device__ __forceinline__ double2 dcmul(double2 a, double2 b) { return cmul(a, b); }

__global__ void gmres_start_kernel(GmresState st) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= st.nrhs) return;
  const int m = st.m;
  const double beta = sqrt(fmax(st.nrm[r].x, 0.0));
  for (int i = 0; i <= m; ++i) st.g[r * (m + 1) + i] = make_double2(0.0, 0.0);
  st.g[r * (m + 1)] = make_double2(beta, 0.0);
  for (int i = 0; i < m; ++i) st.y[r * m + i] = make_double2(0.0, 0.0);
  st.res[r] = beta;
  st.nit[r] = 0;
  const int act = (beta > st.target[r]) && isfinite(beta);
  st.active[r] = act;
  st.inv[r] = (act && beta > 0.0) ? 1.0 / beta : 0.0;
}

__global__ void gmres_arnoldi_kernel(GmresState st, int i) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= st.nrhs || !st.active[r]) return;
  const int m = st.m;
  double2 *H = st.H + (int64_t)r * (m + 1) * m;
  double2 *col = H + i * (m + 1);
  for (int j = 0; j <= i; ++j) {
    double2 a = st.h1[r * (m + 1) + j], b = st.h2[r * (m + 1) + j];
    col[j] = make_double2(a.x + b.x, a.y + b.y);
  }
  const double hn = sqrt(fmax(st.nrm[r].x, 0.0));
  col[i + 1] = make_double2(hn, 0.0);
  // previous rotations
  for (int j = 0; j < i; ++j) {
    const double c = st.cs[r * m + j];
    const double2 s = st.sn[r * m + j];
    const double2 a = col[j], b = col[j + 1];
    col[j] = cadd(cscale(a, c), dcmul(s, b));
    col[j + 1] = csub(cscale(b, c), dcmul(cconj(s), a));
  }
  // new rotation zeroing col[i+1] (real, >= 0)
  const double2 a = col[i];
  const double b = col[i + 1].x;
  const double aa = sqrt(cabs2(a));
  const double rr = sqrt(aa * aa + b * b);
  double c;
  double2 s;
  if (rr == 0.0) {
    c = 1.0;
    s = make_double2(0.0, 0.0);
  } else if (aa == 0.0) {
    c = 0.0;
    s = make_double2(1.0, 0.0);
    col[i] = make_double2(rr, 0.0);
  } else {
    c = aa / rr;
    const double2 ph = make_double2(a.x / aa, a.y / aa);
    s = cscale(ph, b / rr);
    col[i] = cscale(ph, rr);
  }
  col[i + 1] = make_double2(0.0, 0.0);
  st.cs[r * m + i] = c;
  st.sn[r * m + i] = s;
  double2 *g = st.g + r * (m + 1);
  const double2 gi = g[i];
  g[i + 1] = cneg(dcmul(cconj(s), gi));
  g[i] = cscale(gi, c);
  const double res = sqrt(cabs2(g[i + 1]));
  st.res[r] = res;
  st.nit[r] = i + 1;
  const bool done = !(res > st.target[r]) || hn == 0.0 || !isfinite(res) || rr == 0.0;
  if (done) {
    st.active[r] = 0;
    st.inv[r] = 0.0;
  } else {
    st.inv[r] = 1.0 / hn;
  }
}

__global__ void gmres_solve_kernel(GmresState st) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= st.nrhs) return;
  const int m = st.m;
  const int k = st.nit[r];
  const double2 *H = st.H + (int64_t)r * (m + 1) * m;
  const double2 *g = st.g + r * (m + 1);
  double2 *y = st.y + r * m;
  for (int j = k; j < m; ++j) y[j] = make_double2(0.0, 0.0);
  for (int j = k - 1; j >= 0; --j) {
    double2 acc = g[j];
    for (int l = j + 1; l < k; ++l) acc = csub(acc, dcmul(H[l * (m + 1) + j], y[l]));
    const double2 d = H[j * (m + 1) + j];
    const double dd = cabs2(d);
    y[j] = dd > 0.0 ? make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd)
                    : make_double2(0.0, 0.0);
  }
}
}  // namespace

std::atomic<int64_t> &launch_counter() {
  static std::atomic<int64_t> c{0};
  return c;
}

namespace {
std::atomic<unsigned> g_staging_extra{0};
}
void set_staging_extra_bytes(unsigned bytes) { g_staging_extra.store(bytes); }
unsigned staging_extra_bytes() { return g_staging_extra.load(); }

void smem_optin(const void *func, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void *, int>, int> done;  // (kernel, device) -> bytes set
  int dev = 0;
  MG_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  auto key = std::make_pair(func, dev);
  auto it = done.find(key);
  if (it != done.end() && it->second >= bytes) return;
  MG_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done[key] = bytes;
}

// blocks of the first reduction stage: chunks of >= 4096 elements, at most
// 4096 blocks, so a thread of a 256-wide block sums at most ~16 elements for
// vectors up to 16.7 M entries (and proportionally more beyond)
int reduce_blocks(int64_t n) {
  int64_t b = (n + 4095) / 4096;
  if (b < 1) b = 1;
  if (b > 4096) b = 4096;
  return (int)b;
}

template <typename T>
void dot(const C<T> *x, const C<T> *y, int64_t n, int nrhs, double2 *out, RedScratch scr,
         cudaStream_t s) {
  const int NB = reduce_blocks(n);
  const int64_t chunk = (n + NB - 1) / NB;
  if (nrhs > kTickets) throw Error(1, "reduction: too many outputs for the ticket array");
  dot_kernel<T><<<dim3(NB, nrhs, 1), RB, 0, s>>>(x, 0, y, n, chunk, scr.partial, scr.ticket, out, 1);
  MG_LAUNCH_CHECK();
}

template <typename T>
void dot_qr(const C<T> *q, const C<T> *r, int64_t n, int nrhs, double2 *out_qr, double2 *out_qq,
            RedScratch scr, cudaStream_t s) {
  const int NB = reduce_blocks(n);
  const int64_t chunk = (n + NB - 1) / NB;
  if (nrhs > kTickets) throw Error(1, "reduction: too many outputs for the ticket array");
  dot_qr_kernel<T><<<dim3(NB, nrhs), RB, 0, s>>>(q, r, n, chunk, scr.partial, scr.ticket, out_qr, out_qq);
  MG_LAUNCH_CHECK();
}

template <typename T>
void multi_dot(const C<T> *V, int64_t vstride, int k, const C<T> *w, int64_t n, int nrhs,
               double2 *h, int ldh, RedScratch scr, cudaStream_t s) {
  const int NB = reduce_blocks(n);
  const int64_t chunk = (n + NB - 1) / NB;
  if ((int64_t)k * nrhs > kTickets) throw Error(1, "reduction: too many outputs for the ticket array");
  dot_kernel<T><<<dim3(NB, nrhs, k), RB, 0, s>>>(V, vstride, w, n, chunk, scr.partial, scr.ticket, h, ldh);
  MG_LAUNCH_CHECK();
}

template <typename T>
void multi_axpy(const C<T> *V, int64_t vstride, int k, C<T> *w, int64_t n, int nrhs,
                const double2 *h, int ldh, double sign, cudaStream_t s) {
  if (k <= 0) return;
  if (k > 128) throw Error(1, "multi_axpy: k > 128");
  const int gx = (grid_for(n) + nrhs - 1) / nrhs + 1;
  multi_axpy_kernel<T><<<dim3(gx, nrhs), 256, 0, s>>>(V, vstride, k, w, n, h, ldh, sign);
  MG_LAUNCH_CHECK();
}

template <typename T>
void axpby(double a, const C<T> *x, double b, C<T> *y, int64_t n, int nrhs, cudaStream_t s) {
  axpby_kernel<T><<<grid_for(n * nrhs), 256, 0, s>>>((T)a, x, (T)b, y, n * nrhs);
  MG_LAUNCH_CHECK();
}

template <typename T>
void scale_rhs(const C<T> *x, C<T> *y, const double *scal, int64_t n, int nrhs, cudaStream_t s) {
  const int gx = (grid_for(n) + nrhs - 1) / nrhs + 1;
  scale_rhs_kernel<T><<<dim3(gx, nrhs), 256, 0, s>>>(x, y, scal, n);
  MG_LAUNCH_CHECK();
}

template <typename T>
void mr_update(C<T> *z, C<T> *r, const C<T> *q, const double2 *dqr, const double2 *nq, int64_t n,
               int nrhs, cudaStream_t s) {
  const int gx = (grid_for(n) + nrhs - 1) / nrhs + 1;
  mr_update_kernel<T><<<dim3(gx, nrhs), 256, 0, s>>>(z, r, q, dqr, nq, n);
  MG_LAUNCH_CHECK();
}

template <typename T>
void mr_dir_update(C<T> *z, C<T> *r, const C<T> *e, const C<T> *q, const double2 *dqr,
                   const double2 *nq, int64_t n, int nrhs, cudaStream_t s) {
  const int gx = (grid_for(n) + nrhs - 1) / nrhs + 1;
  mr_dir_kernel<T><<<dim3(gx, nrhs), 256, 0, s>>>(z, r, e, q, dqr, nq, n);
  MG_LAUNCH_CHECK();
}

template <typename To, typename From>
void convert(const C<From> *in, C<To> *out, int64_t n, cudaStream_t s) {
  convert_kernel<To, From><<<grid_for(n), 256, 0, s>>>(in, out, n);
  MG_LAUNCH_CHECK();
}

template <typename To, typename From>
void convert_scale(const C<From> *x, C<To> *y, const double *scal, int64_t n, int nrhs,
                   cudaStream_t s) {
  const int gx = (grid_for(n) + nrhs - 1) / nrhs + 1;
  convert_scale_kernel<To, From><<<dim3(gx, nrhs), 256, 0, s>>>(x, y, scal, n);
  MG_LAUNCH_CHECK();
}

template <typename To, typename From>
void relayout(const C<From> *x, C<To> *y, const double *scal, int64_t V, int nrhs, bool to_soa,
              cudaStream_t s) {
  const int gx = (grid_for(V * 6) + nrhs - 1) / nrhs + 1;
  relayout_kernel<To, From><<<dim3(gx, nrhs), 256, 0, s>>>(x, y, scal, V, to_soa);
  MG_LAUNCH_CHECK();
}

template <typename T, typename Tlo>
void add_lo(const C<Tlo> *x, C<T> *y, int64_t n, cudaStream_t s) {
  add_lo_kernel<T, Tlo><<<grid_for(n), 256, 0, s>>>(x, y, n);
  MG_LAUNCH_CHECK();
}

template <typename T>
void check_finite(const C<T> *x, int64_t n, int *flag, cudaStream_t s) {
  finite_kernel<T><<<grid_for(n), 256, 0, s>>>(x, n, flag);
  MG_LAUNCH_CHECK();
}

void gmres_start(GmresState st, cudaStream_t s) {
  gmres_start_kernel<<<(st.nrhs + 63) / 64, 64, 0, s>>>(st);
  MG_LAUNCH_CHECK();
}
void gmres_arnoldi(GmresState st, int i, cudaStream_t s) {
  gmres_arnoldi_kernel<<<(st.nrhs + 63) / 64, 64, 0, s>>>(st, i);
  MG_LAUNCH_CHECK();
}
void gmres_solve(GmresState st, cudaStream_t s) {
  gmres_solve_kernel<<<(st.nrhs + 63) / 64, 64, 0, s>>>(st);
  MG_LAUNCH_CHECK();
}

#define INST(T)                                                                                  \
  template void dot<T>(const C<T> *, const C<T> *, int64_t, int, double2 *, RedScratch,         \
                       cudaStream_t);                                                            \
  template void multi_dot<T>(const C<T> *, int64_t, int, const C<T> *, int64_t, int, double2 *,  \
                             int, RedScratch, cudaStream_t);                                     \
  template void multi_axpy<T>(const C<T> *, int64_t, int, C<T> *, int64_t, int, const double2 *, \
                              int, double, cudaStream_t);                                        \
  template void axpby<T>(double, const C<T> *, double, C<T> *, int64_t, int, cudaStream_t);      \
  template void scale_rhs<T>(const C<T> *, C<T> *, const double *, int64_t, int, cudaStream_t);  \
  template void mr_update<T>(C<T> *, C<T> *, const C<T> *, const double2 *, const double2 *,     \
                             int64_t, int, cudaStream_t);                                        \
  template void check_finite<T>(const C<T> *, int64_t, int *, cudaStream_t);               \
  template void dot_qr<T>(const C<T> *, const C<T> *, int64_t, int, double2 *, double2 *,        \
                          RedScratch, cudaStream_t);                                           \
  template void mr_dir_update<T>(C<T> *, C<T> *, const C<T> *, const C<T> *, const double2 *,    \
                                 const double2 *, int64_t, int, cudaStream_t);
INST(double)
INST(float)
template void convert<float, double>(const C<double> *, C<float> *, int64_t, cudaStream_t);
template void convert<double, float>(const C<float> *, C<double> *, int64_t, cudaStream_t);
template void convert_scale<float, double>(const C<double> *, C<float> *, const double *, int64_t,
                                           int, cudaStream_t);
template void convert_scale<double, double>(const C<double> *, C<double> *, const double *,
                                            int64_t, int, cudaStream_t);
template void convert_scale<double, float>(const C<float> *, C<double> *, const double *, int64_t,
                                           int, cudaStream_t);
template void relayout<float, double>(const C<double> *, C<float> *, const double *, int64_t, int,
                                      bool, cudaStream_t);
template void relayout<double, float>(const C<float> *, C<double> *, const double *, int64_t, int,
                                      bool, cudaStream_t);
template void relayout<float, float>(const C<float> *, C<float> *, const double *, int64_t, int,
                                     bool, cudaStream_t);
template void add_lo<double, float>(const C<float> *, C<double> *, int64_t, cudaStream_t);
template void add_lo<double, double>(const C<double> *, C<double> *, int64_t, cudaStream_t);

}  // namespace mg
