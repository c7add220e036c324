// Shared device/host helpers of the mgmlmc CUDA library: complex arithmetic
// on float2 / double2, lattice geometry, error plumbing.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>

namespace mg {

// ----------------------------------------------------------------- complex
template <typename T> struct Cplx;
template <> struct Cplx<double> { using type = double2; };
template <> struct Cplx<float> { using type = float2; };
template <typename T> using C = typename Cplx<T>::type;

template <typename T> __host__ __device__ __forceinline__ C<T> mk(T re, T im) {
  C<T> z; z.x = re; z.y = im; return z;
}
template <typename V> __host__ __device__ __forceinline__ V cadd(V a, V b) { a.x += b.x; a.y += b.y; return a; }
template <typename V> __host__ __device__ __forceinline__ V csub(V a, V b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename V> __host__ __device__ __forceinline__ V cconj(V a) { a.y = -a.y; return a; }
template <typename V> __host__ __device__ __forceinline__ V cneg(V a) { a.x = -a.x; a.y = -a.y; return a; }
// i * a and -i * a
template <typename V> __host__ __device__ __forceinline__ V cmuli(V a) { V r; r.x = -a.y; r.y = a.x; return r; }
template <typename V> __host__ __device__ __forceinline__ V cmulmi(V a) { V r; r.x = a.y; r.y = -a.x; return r; }
template <typename V, typename S> __host__ __device__ __forceinline__ V cscale(V a, S s) { a.x *= s; a.y *= s; return a; }
template <typename V> __host__ __device__ __forceinline__ V cmul(V a, V b) {
  V r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// conj(a) * b
template <typename V> __host__ __device__ __forceinline__ V cmulc(V a, V b) {
  V r; r.x = a.x * b.x + a.y * b.y; r.y = a.x * b.y - a.y * b.x; return r;
}
// acc += a * b
template <typename V> __host__ __device__ __forceinline__ V cfma(V a, V b, V acc) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
// acc += conj(a) * b
template <typename V> __host__ __device__ __forceinline__ V cfmac(V a, V b, V acc) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
  return acc;
}
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }

template <typename To, typename From> __host__ __device__ __forceinline__ C<To> cvt(From a) {
  C<To> r; r.x = (To)a.x; r.y = (To)a.y; return r;
}

// ---- packed FP32 pairs: two values in the lanes of a 64-bit register pair,
// advanced by one .f32x2 instruction; each lane rounds exactly as the scalar
// instruction would, so a paired computation reproduces the scalar one bit
// for bit
struct P2 {
  unsigned long long v;
};
__device__ __forceinline__ P2 p2(float lo, float hi) {
  P2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 p2split(P2 a) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(a.v));
  return r;
}
__device__ __forceinline__ P2 p2fma(P2 a, P2 b, P2 c) {
  P2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}
__device__ __forceinline__ P2 p2add(P2 a, P2 b) {
  P2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ P2 p2sub(P2 a, P2 b) {
  P2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ P2 p2mul(P2 a, P2 b) {
  P2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ P2 p2neg(P2 a) { return p2mul(a, p2(-1.f, -1.f)); }

// ----------------------------------------------------------------- geometry
// A 4-D periodic lattice with `dof` complex entries per site.  Site index
// s = x + L0 (y + L1 (z + L2 t)).
struct Geom {
  int L[4];
  int V;
  int dof;
  __host__ __device__ int64_t n() const { return (int64_t)V * dof; }
  __host__ __device__ __forceinline__ void coords(int s, int c[4]) const {
    c[0] = s % L[0]; s /= L[0];
    c[1] = s % L[1]; s /= L[1];
    c[2] = s % L[2];
    c[3] = s / L[2];
  }
  __host__ __device__ __forceinline__ int index(const int c[4]) const {
    return c[0] + L[0] * (c[1] + L[1] * (c[2] + L[2] * c[3]));
  }
  // neighbour of s in direction d (0 self, 1 + 2 mu forward, 2 + 2 mu backward)
  __host__ __device__ __forceinline__ int neighbor(int s, int d) const {
    if (d == 0) return s;
    int c[4];
    coords(s, c);
    int mu = (d - 1) >> 1;
    if (d & 1) c[mu] = (c[mu] + 1 == L[mu]) ? 0 : c[mu] + 1;
    else c[mu] = (c[mu] == 0) ? L[mu] - 1 : c[mu] - 1;
    return index(c);
  }
};

// FP32 vectors of the fine level are stored structure-of-arrays: complex
// component i (0..11, spin-major) of site s sits at ((i >> 1) V + s) * 2 +
// (i & 1), so the 16-byte chunk i >> 1 of consecutive sites is contiguous and
// a thread-per-site access is coalesced.  FP64 fine vectors and every coarse
// vector keep the canonical order s * dof + i.
__host__ __device__ __forceinline__ int64_t soa_index(int64_t s, int i, int64_t V) {
  return ((int64_t)(i >> 1) * V + s) * 2 + (i & 1);
}
template <bool SOA>
__host__ __device__ __forceinline__ int64_t fidx(int64_t s, int i, int64_t V) {
  return SOA ? soa_index(s, i, V) : s * 12 + i;
}

// the 12 components of site s of a fine vector: FP32 structure-of-arrays
// vectors as six 16-byte chunks (two components each, one load per chunk, so
// a warp's access covers whole sectors), FP64 ones canonical
template <typename T>
__device__ __forceinline__ void load_fine_site(const C<T> *v, int64_t s, int64_t V, C<T> (&p)[12]) {
  if constexpr (sizeof(T) == 4) {
    const float4 *c = reinterpret_cast<const float4 *>(v);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const float4 q = c[(int64_t)k * V + s];
      p[2 * k] = mk<T>(q.x, q.y);
      p[2 * k + 1] = mk<T>(q.z, q.w);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 12; ++i) p[i] = v[s * 12 + i];
  }
}
template <typename T>
__device__ __forceinline__ void store_fine_site(C<T> *v, int64_t s, int64_t V, const C<T> (&p)[12]) {
  if constexpr (sizeof(T) == 4) {
    float4 *c = reinterpret_cast<float4 *>(v);
#pragma unroll
    for (int k = 0; k < 6; ++k)
      c[(int64_t)k * V + s] = make_float4(p[2 * k].x, p[2 * k].y, p[2 * k + 1].x, p[2 * k + 1].y);
  } else {
#pragma unroll
    for (int i = 0; i < 12; ++i) v[s * 12 + i] = p[i];
  }
}



// Block aggregation of a level (Sec. 2.2): aggregates are blocks of extent
// b[4]; rows of an (aggregate, chirality) pair are site_in_block * half + d.
struct AggMap {
  Geom fine;      // level l
  Geom coarse;    // level l+1 lattice (dof = 2 ntv)
  int b[4];
  int ntv;
  int half;       // fine.dof / 2
  int sites;      // sites per aggregate
  int rows;       // sites * half
  int soa = 0;    // fine vectors in the FP32 fine-level (structure-of-arrays) order
  // fine dof index of (aggregate X, chirality c, row)
  __host__ __device__ __forceinline__ int64_t fine_index(int X, int c, int row) const {
    int cc[4];
    coarse.coords(X, cc);
    int sia = row / half, d = row - sia * half;
    int r[4];
    r[0] = sia % b[0]; sia /= b[0];
    r[1] = sia % b[1]; sia /= b[1];
    r[2] = sia % b[2];
    r[3] = sia / b[2];
    int f[4];
    for (int i = 0; i < 4; ++i) f[i] = cc[i] * b[i] + r[i];
    if (soa) return soa_index(fine.index(f), c * half + d, fine.V);
    return (int64_t)fine.index(f) * fine.dof + c * half + d;
  }
  // aggregate, chirality and row of fine dof i
  __host__ __device__ __forceinline__ void locate(int64_t i, int &X, int &c, int &row) const {
    int s = (int)(i / fine.dof);
    int dd = (int)(i - (int64_t)s * fine.dof);
    c = dd / half;
    int d = dd - c * half;
    int f[4];
    fine.coords(s, f);
    int cc[4], r[4];
    for (int k = 0; k < 4; ++k) { cc[k] = f[k] / b[k]; r[k] = f[k] - cc[k] * b[k]; }
    X = coarse.index(cc);
    int sia = r[0] + b[0] * (r[1] + b[1] * (r[2] + b[2] * r[3]));
    row = sia * half + d;
  }
};

// ----------------------------------------------------------------- errors
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};

#define MG_CUDA(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      throw ::mg::Error(e_ == cudaErrorMemoryAllocation ? 3 : 4,                       \
                        std::string(#call) + ": " + cudaGetErrorString(e_));           \
  } while (0)

// process-wide count of kernel launches issued by this library
std::atomic<int64_t> &launch_counter();
#define MG_COUNT(k) ::mg::launch_counter().fetch_add((k), std::memory_order_relaxed)
#define MG_LAUNCH_CHECK()          \
  do {                             \
    MG_COUNT(1);                   \
    MG_CUDA(cudaGetLastError());   \
  } while (0)

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Device-side waits (mbarrier polls) give up after kWaitNs of the GPU's
// global timer and report through an error flag instead of hanging.
constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Failure injection for tests: extra bytes the staging barriers of the coarse
// stencil kernels expect beyond what their bulk copy delivers (0 in normal
// operation; a positive value makes their bounded wait run out).
void set_staging_extra_bytes(unsigned bytes);
unsigned staging_extra_bytes();

// Raise the dynamic shared-memory limit of kernel `func` to `bytes` on the
// current device.  The attribute is per device, so the call is made once per
// (kernel, device) and remembered under a lock: launchers may run on several
// host threads and devices.
void smem_optin(const void *func, int bytes);

// streaming multiprocessors of the current device (cached per device)
int sm_count();

}  // namespace mg
