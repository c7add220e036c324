// Wilson-Dirac operator on the fine lattice (the paper's D; Sec. 1 and the
// Gamma5-hermiticity of Sec. 2), Gamma5, and the Z4 noise generator.
//
//   (D psi)(x) = (4 + m0) psi(x) - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
//                                 + (1 + gamma_mu) U_mu(x-mu)^H psi(x-mu) ]
//
// Chiral basis: gamma_mu = [[0, B_mu], [B_mu^H, 0]] with B_k = -i sigma_k and
// B_4 = 1, so (1 -+ gamma_mu) has rank 2 per colour: with the upper/lower
// spin halves u, l of psi,
//   (1 - gamma) psi = ( h, -B^H h ),  h = u - B l,
//   (1 + gamma) psi = ( h,  B^H h ),  h = u + B l.
// Each hop therefore multiplies two colour vectors by the link instead of
// four.  Time is antiperiodic for the fermion field.
#include "kernels.h"

namespace mg {

namespace {

// (B_mu l)_a for a = 0, 1 given the lower spins l0 = psi_2, l1 = psi_3
template <int MU, typename V> __device__ __forceinline__ V Bl(int a, V l0, V l1) {
  if (MU == 0) return a == 0 ? cmulmi(l1) : cmulmi(l0);   // -i sigma_1
  if (MU == 1) return a == 0 ? cneg(l1) : l0;              // -i sigma_2
  if (MU == 2) return a == 0 ? cmulmi(l0) : cmuli(l1);     // -i sigma_3
  return a == 0 ? l0 : l1;                                 // 1
}
// (B_mu^H v)_a
template <int MU, typename V> __device__ __forceinline__ V Bh(int a, V v0, V v1) {
  if (MU == 0) return a == 0 ? cmuli(v1) : cmuli(v0);
  if (MU == 1) return a == 0 ? v1 : cneg(v0);
  if (MU == 2) return a == 0 ? cmuli(v0) : cmulmi(v1);
  return a == 0 ? v0 : v1;
}

template <typename T>
__device__ __forceinline__ void load_spinor(const C<T> *__restrict__ p, C<T> (&s)[12]) {
  if constexpr (sizeof(T) == 4) {
    // 96 B per site: six 16-byte loads through the read-only path
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const float4 v = __ldg(q + i);
      s[2 * i] = mk<T>(v.x, v.y);
      s[2 * i + 1] = mk<T>(v.z, v.w);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 12; ++i) s[i] = __ldg(p + i);
  }
}
template <typename T>
__device__ __forceinline__ void load_link(const C<T> *__restrict__ p, C<T> (&u)[9]) {
#pragma unroll
  for (int i = 0; i < 9; ++i) u[i] = __ldg(p + i);
}
template <typename T>
__device__ __forceinline__ void store_spinor(C<T> *__restrict__ p, const C<T> (&s)[12]) {
  if constexpr (sizeof(T) == 4) {
    float4 *q = reinterpret_cast<float4 *>(p);
#pragma unroll
    for (int i = 0; i < 6; ++i) q[i] = make_float4(s[2 * i].x, s[2 * i].y, s[2 * i + 1].x, s[2 * i + 1].y);
  } else {
#pragma unroll
    for (int i = 0; i < 12; ++i) p[i] = s[i];
  }
}

// contribution of one hop in direction MU (FWD: from x+mu through U_mu(x);
// otherwise from x-mu through U_mu(x-mu)^H), scaled by k = -1/2 * boundary
// sign, added to acc.
template <int MU, bool FWD, typename T>
__device__ __forceinline__ void hop(const C<T> (&p)[12], const C<T> (&u)[9], T k, C<T> (&acc)[12]) {
  const T sg = FWD ? (T)-1 : (T)1;
  C<T> h[2][3];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      C<T> b = Bl<MU>(a, p[6 + c], p[9 + c]);
      h[a][c] = cadd(p[3 * a + c], cscale(b, sg));
    }
  C<T> v[2][3];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      C<T> z = mk<T>((T)0, (T)0);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (FWD) z = cfma(u[3 * c + b], h[a][b], z);   // U h
        else z = cfmac(u[3 * b + c], h[a][b], z);      // U^H h
      }
      v[a][c] = z;
    }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      // real scale factors: two FMAs per complex entry
      acc[3 * a + c].x = fma(k, v[a][c].x, acc[3 * a + c].x);
      acc[3 * a + c].y = fma(k, v[a][c].y, acc[3 * a + c].y);
      const C<T> w = Bh<MU>(a, v[0][c], v[1][c]);
      acc[6 + 3 * a + c].x = fma(sg * k, w.x, acc[6 + 3 * a + c].x);
      acc[6 + 3 * a + c].y = fma(sg * k, w.y, acc[6 + 3 * a + c].y);
    }
}

template <int MU, typename T, bool SPLIT>
__device__ __forceinline__ void dir_pair(const C<T> *__restrict__ in, const C<T> *__restrict__ U,
                                         const Geom &g, int s, const int (&c)[4], const int *b,
                                         C<T> (&acc)[12], C<T> *__restrict__ out9,
                                         int64_t nstride) {
  // forward
  {
    int cn[4] = {c[0], c[1], c[2], c[3]};
    cn[MU] = (c[MU] + 1 == g.L[MU]) ? 0 : c[MU] + 1;
    const int sn = g.index(cn);
    const T k = (MU == 3 && cn[3] == 0) ? (T)0.5 : (T)-0.5;
    C<T> p[12], u[9];
    load_spinor<T>(in + (int64_t)sn * 12, p);
    load_link<T>(U + ((int64_t)s * 4 + MU) * 9, u);
    if (!SPLIT) {
      hop<MU, true, T>(p, u, k, acc);
    } else {
      const bool cross = (c[MU] / b[MU]) != (cn[MU] / b[MU]);
      if (cross) {
        C<T> t[12];
#pragma unroll
        for (int i = 0; i < 12; ++i) t[i] = mk<T>((T)0, (T)0);
        hop<MU, true, T>(p, u, k, t);
        C<T> *o = out9 + (1 + 2 * MU) * nstride + (int64_t)s * 12;
#pragma unroll
        for (int i = 0; i < 12; ++i) o[i] = t[i];
      } else {
        hop<MU, true, T>(p, u, k, acc);
        C<T> *o = out9 + (1 + 2 * MU) * nstride + (int64_t)s * 12;
#pragma unroll
        for (int i = 0; i < 12; ++i) o[i] = mk<T>((T)0, (T)0);
      }
    }
  }
  // backward
  {
    int cn[4] = {c[0], c[1], c[2], c[3]};
    cn[MU] = (c[MU] == 0) ? g.L[MU] - 1 : c[MU] - 1;
    const int sn = g.index(cn);
    const T k = (MU == 3 && c[3] == 0) ? (T)0.5 : (T)-0.5;
    C<T> p[12], u[9];
    load_spinor<T>(in + (int64_t)sn * 12, p);
    load_link<T>(U + ((int64_t)sn * 4 + MU) * 9, u);
    if (!SPLIT) {
      hop<MU, false, T>(p, u, k, acc);
    } else {
      const bool cross = (c[MU] / b[MU]) != (cn[MU] / b[MU]);
      C<T> *o = out9 + (2 + 2 * MU) * nstride + (int64_t)s * 12;
      if (cross) {
        C<T> t[12];
#pragma unroll
        for (int i = 0; i < 12; ++i) t[i] = mk<T>((T)0, (T)0);
        hop<MU, false, T>(p, u, k, t);
#pragma unroll
        for (int i = 0; i < 12; ++i) o[i] = t[i];
      } else {
        hop<MU, false, T>(p, u, k, acc);
#pragma unroll
        for (int i = 0; i < 12; ++i) o[i] = mk<T>((T)0, (T)0);
      }
    }
  }
}

template <typename T, bool SPLIT>
__global__ void __launch_bounds__(128) wilson_kernel(const C<T> *__restrict__ in,
                                                     C<T> *__restrict__ out,
                                                     const C<T> *__restrict__ U, Geom g, T diag,
                                                     int b0, int b1, int b2, int b3) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  const int64_t n = (int64_t)g.V * 12;
  const C<T> *inr = in + blockIdx.y * n;
  C<T> *outr = out + (SPLIT ? 0 : blockIdx.y * n);
  const int b[4] = {b0, b1, b2, b3};
  int c[4];
  g.coords(s, c);
  C<T> acc[12];
  {
    const C<T> *ps = inr + (int64_t)s * 12;
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = cscale(ps[i], diag);
  }
  dir_pair<0, T, SPLIT>(inr, U, g, s, c, b, acc, outr, n);
  dir_pair<1, T, SPLIT>(inr, U, g, s, c, b, acc, outr, n);
  dir_pair<2, T, SPLIT>(inr, U, g, s, c, b, acc, outr, n);
  dir_pair<3, T, SPLIT>(inr, U, g, s, c, b, acc, outr, n);
  store_spinor<T>(outr + (int64_t)s * 12, acc);
}

// ------------------------------------------------------------------ staged FP32
// The FP32 hop term with the spinor operands staged through shared memory.
// One warp owns 32 consecutive sites of one right-hand side.  For each of the
// nine spinor sets it needs (the centre, then the eight neighbours) the warp
// gathers the 32 records with lane-contiguous cp.async copies: round r of
// lane l moves 16-byte chunk (32 r + l) of the 32 records, so one warp
// instruction covers 512 contiguous bytes whenever the neighbours are
// contiguous (every direction except at a wrap), where a thread-per-site load
// would touch 32 records spread over 3 KB.  A record lands in a 128-byte row
// of shared memory with chunk k in slot k ^ (row & 7): the reads of eight
// consecutive lanes hit eight distinct bank groups and the copies at most
// five.  A ring of S stages keeps S-1 sets in flight while one is consumed.
// Links are stored structure-of-arrays, UDs[mu][a][b][s], so a lane's own
// link components are coalesced across the warp either way: DIRECT loads
// them into registers two hops ahead, otherwise they ride in the same stage
// as the spinors (slot [component][lane]).
namespace staged {
constexpr int kRow = 128;                 // bytes per staged spinor record
constexpr int kSpinBytes = 32 * kRow;     // one staged spinor set
constexpr int kLinkBytes = 9 * 32 * 8;    // one staged link set
template <bool DIRECT> constexpr int stage_bytes() { return DIRECT ? kSpinBytes : kSpinBytes + kLinkBytes; }
constexpr int kWarps = 4;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ void cp16(void *smem, const void *g) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(g) : "memory");
}
__device__ __forceinline__ void cp8(void *smem, const void *g) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(a), "l"(g) : "memory");
}
__device__ __forceinline__ void commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void wait_groups() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
// byte offset of chunk k of record q in a staged spinor set
__device__ __forceinline__ int slot(int q, int k) { return q * kRow + ((k ^ (q & 7)) << 4); }

struct Tile {
  const float2 *in;   // this right-hand side
  const float2 *UDs;  // structure-of-arrays links
  Geom g;
  float diag;
  unsigned char *smem;  // this warp's S stages
  int lane, s0, s;      // s: own site, clamped into the lattice
  int c[4];
  float2 acc[12];
};

// source site of operand set I for this lane: 0 the site itself, 1 + 2 mu the
// forward neighbour, 2 + 2 mu the backward neighbour
template <int I> __device__ __forceinline__ int item_site(const Tile &t) {
  if (I == 0) return t.s;
  constexpr int mu = (I - 1) / 2;
  int cn[4] = {t.c[0], t.c[1], t.c[2], t.c[3]};
  if (I & 1) cn[mu] = (t.c[mu] + 1 == t.g.L[mu]) ? 0 : t.c[mu] + 1;
  else cn[mu] = (t.c[mu] == 0) ? t.g.L[mu] - 1 : t.c[mu] - 1;
  return t.g.index(cn);
}
// the link of hop I (U_mu(x) forward, U_mu(x - mu) backward), component k
template <int I> __device__ __forceinline__ const float2 *link_ptr(const Tile &t, int ns, int k) {
  constexpr int mu = (I - 1) / 2;
  const int ls = (I & 1) ? t.s : ns;
  return t.UDs + ((int64_t)(mu * 9 + k)) * t.g.V + ls;
}

template <int I, int S, bool DIRECT> __device__ __forceinline__ void issue(Tile &t) {
  unsigned char *st = t.smem + (I % S) * stage_bytes<DIRECT>();
  const int ns = item_site<I>(t);
#pragma unroll
  for (int r = 0; r < 6; ++r) {
    const int f = r * 32 + t.lane, q = f / 6, k = f - 6 * q;
    const int src = __shfl_sync(kFull, ns, q);
    cp16(st + slot(q, k), t.in + (int64_t)src * 12 + 2 * k);
  }
  if constexpr (I > 0 && !DIRECT) {
    float2 *lk = reinterpret_cast<float2 *>(st + kSpinBytes);
#pragma unroll
    for (int k = 0; k < 9; ++k) cp8(lk + k * 32 + t.lane, link_ptr<I>(t, ns, k));
  }
}

template <int I> __device__ __forceinline__ void load_link_direct(const Tile &t, float2 (&u)[9]) {
  if constexpr (I >= 1 && I <= 8) {
    const int ns = item_site<I>(t);
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k] = __ldg(link_ptr<I>(t, ns, k));
  }
}

template <int I, int S, bool DIRECT>
__device__ __forceinline__ void consume(Tile &t, const float2 (&ud)[9]) {
  const unsigned char *st = t.smem + (I % S) * stage_bytes<DIRECT>();
  float2 p[12];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float4 v = *reinterpret_cast<const float4 *>(st + slot(t.lane, k));
    p[2 * k] = make_float2(v.x, v.y);
    p[2 * k + 1] = make_float2(v.z, v.w);
  }
  if constexpr (I == 0) {
#pragma unroll
    for (int i = 0; i < 12; ++i) t.acc[i] = cscale(p[i], t.diag);
  } else {
    constexpr int mu = (I - 1) / 2;
    constexpr bool fwd = (I & 1) != 0;
    float2 u[9];
    if constexpr (DIRECT) {
#pragma unroll
      for (int k = 0; k < 9; ++k) u[k] = ud[k];
    } else {
      const float2 *lk = reinterpret_cast<const float2 *>(st + kSpinBytes);
#pragma unroll
      for (int k = 0; k < 9; ++k) u[k] = lk[k * 32 + t.lane];
    }
    // antiperiodic time: hops across the t boundary change sign
    const bool wrap = mu == 3 && (fwd ? t.c[3] + 1 == t.g.L[3] : t.c[3] == 0);
    hop<mu, fwd, float>(p, u, wrap ? 0.5f : -0.5f, t.acc);
  }
}

template <int I, int S, bool DIRECT> __device__ __forceinline__ void prologue(Tile &t) {
  if constexpr (I < S - 1) {
    issue<I, S, DIRECT>(t);
    commit();
    prologue<I + 1, S, DIRECT>(t);
  }
}

// step I: issue set I + S - 1, (DIRECT) load the links of hop I + 2, wait for
// set I and consume it.  u0, u1: the directly loaded links of hops I, I + 1.
template <int I, int S, bool DIRECT>
__device__ __forceinline__ void steps(Tile &t, float2 (&u0)[9], float2 (&u1)[9]) {
  if constexpr (I + S - 1 <= 8) issue<I + S - 1, S, DIRECT>(t);
  commit();  // possibly empty: keeps the group count uniform
  float2 u2[9];
  if constexpr (DIRECT) load_link_direct<I + 2>(t, u2);
  wait_groups<S - 1>();
  __syncwarp();
  consume<I, S, DIRECT>(t, u0);
  __syncwarp();
  if constexpr (I < 8) steps<I + 1, S, DIRECT>(t, u1, u2);
}
}  // namespace staged

template <int S, bool DIRECT>
__global__ void __launch_bounds__(staged::kWarps * 32, 3)
    wilson_staged_kernel(const float2 *__restrict__ in, float2 *__restrict__ out,
                         const float2 *__restrict__ UDs, Geom g, float diag, int nrhs) {
  using namespace staged;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int w = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + w;
  const int ntiles = (g.V + 31) >> 5;
  if (gw >= (int64_t)ntiles * nrhs) return;  // whole warps only: no block barrier below
  const int tile = (int)(gw / nrhs);
  const int r = (int)(gw - (int64_t)tile * nrhs);
  const int64_t n = (int64_t)g.V * 12;
  Tile t;
  t.in = in + r * n;
  t.UDs = UDs;
  t.g = g;
  t.diag = diag;
  t.smem = smem_raw + w * S * stage_bytes<DIRECT>();
  t.lane = threadIdx.x & 31;
  t.s0 = tile * 32;
  t.s = min(t.s0 + t.lane, g.V - 1);
  g.coords(t.s, t.c);
  float2 u0[9], u1[9];
  if constexpr (DIRECT) load_link_direct<1>(t, u1);
  prologue<0, S, DIRECT>(t);
  steps<0, S, DIRECT>(t, u0, u1);
  wait_groups<0>();
  // transpose the result through stage 0 and store 512 contiguous bytes per
  // warp instruction
  unsigned char *st = t.smem;
#pragma unroll
  for (int k = 0; k < 6; ++k)
    *reinterpret_cast<float4 *>(st + slot(t.lane, k)) =
        make_float4(t.acc[2 * k].x, t.acc[2 * k].y, t.acc[2 * k + 1].x, t.acc[2 * k + 1].y);
  __syncwarp();
  float4 *o = reinterpret_cast<float4 *>(out + r * n + (int64_t)t.s0 * 12);
#pragma unroll
  for (int rr = 0; rr < 6; ++rr) {
    const int f = rr * 32 + t.lane, q = f / 6, k = f - 6 * q;
    if (t.s0 + q < g.V) o[f] = *reinterpret_cast<const float4 *>(st + slot(q, k));
  }
}

// UDs[mu][a][b][s] = U[s][mu][a][b]
__global__ void link_soa_kernel(const float2 *__restrict__ U, float2 *__restrict__ UDs, int V) {
  const int64_t total = (int64_t)V * 36;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i / 36;
    const int comp = (int)(i - s * 36);  // mu * 9 + k
    UDs[(int64_t)comp * V + s] = U[i];
  }
}

template <typename T>
__global__ void gamma5_kernel(const C<T> *__restrict__ in, C<T> *__restrict__ out, int64_t total,
                              int dof) {
  const int half = dof / 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int d = (int)(i % dof);
    out[i] = d < half ? in[i] : cneg(in[i]);
  }
}

// ------------------------------------------------------------------ Philox
// Philox4x64-10 (Salmon et al., SC'11): 10 rounds of
//   (hi0, lo0) = M0 c0, (hi1, lo1) = M1 c2,
//   c = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0),
// the key bumped by the Weyl constants between rounds.
struct U64x4 { uint64_t v[4]; };
__device__ __forceinline__ U64x4 philox4x64_10(U64x4 c, uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    const uint64_t lo0 = M0 * c.v[0], hi0 = __umul64hi(M0, c.v[0]);
    const uint64_t lo1 = M1 * c.v[2], hi1 = __umul64hi(M1, c.v[2]);
    U64x4 o;
    o.v[0] = hi1 ^ c.v[1] ^ k0;
    o.v[1] = lo1;
    o.v[2] = hi0 ^ c.v[3] ^ k1;
    o.v[3] = lo0;
    c = o;
  }
  return c;
}

template <typename T>
__global__ void z4_kernel(C<T> *__restrict__ out, int64_t n, uint64_t seed, uint64_t sample0,
                          uint64_t term, uint64_t aux, int64_t lo, int64_t hi) {
  const int r = blockIdx.y;
  C<T> *o = out + r * n;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q * 4 < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = q * 4;
    const bool any = (i0 + 4 > lo) && (i0 < hi);
    U64x4 w;
    if (any) {
      U64x4 c;
      c.v[0] = (uint64_t)q;
      c.v[1] = sample0 + (uint64_t)r;
      c.v[2] = term;
      c.v[3] = aux;
      w = philox4x64_10(c, seed, 0ull);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t i = i0 + j;
      if (i >= n) break;
      C<T> x = mk<T>((T)0, (T)0);
      if (any && i >= lo && i < hi) {
        const int code = (int)(w.v[j] >> 62);
        x = code == 0 ? mk<T>((T)1, (T)0)
                      : code == 1 ? mk<T>((T)0, (T)1) : code == 2 ? mk<T>((T)-1, (T)0) : mk<T>((T)0, (T)-1);
      }
      o[i] = x;
    }
  }
}

inline int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

}  // namespace

namespace {
template <int S, bool DIRECT>
void launch_staged(const float2 *in, float2 *out, const float2 *UDs, Geom g, float diag, int nrhs,
                   cudaStream_t s) {
  constexpr int smem = staged::kWarps * S * staged::stage_bytes<DIRECT>();
  static bool attr = false;
  if (!attr) {
    MG_CUDA(cudaFuncSetAttribute(wilson_staged_kernel<S, DIRECT>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    attr = true;
  }
  const int64_t warps = (int64_t)((g.V + 31) / 32) * nrhs;
  wilson_staged_kernel<S, DIRECT><<<div_up(warps, staged::kWarps), staged::kWarps * 32, smem, s>>>(
      in, out, UDs, g, diag, nrhs);
  MG_LAUNCH_CHECK();
}
}  // namespace

int wilson_staged_variants() { return 4; }

template <typename T>
void wilson_apply(const C<T> *in, C<T> *out, const C<T> *U, const C<T> *UDs, Geom g, double m0,
                  int nrhs, int variant, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    const bool aligned = (((uintptr_t)in | (uintptr_t)out) & 15) == 0;
    if (UDs && aligned && variant >= 0) {
      const float diag = (float)(4.0 + m0);
      switch (variant) {
        case 0: launch_staged<2, false>(in, out, UDs, g, diag, nrhs, s); return;
        case 1: launch_staged<3, false>(in, out, UDs, g, diag, nrhs, s); return;
        case 2: launch_staged<2, true>(in, out, UDs, g, diag, nrhs, s); return;
        default: launch_staged<3, true>(in, out, UDs, g, diag, nrhs, s); return;
      }
    }
  }
  dim3 grid(div_up(g.V, 128), nrhs);
  wilson_kernel<T, false><<<grid, 128, 0, s>>>(in, out, U, g, (T)(4.0 + m0), 1, 1, 1, 1);
  MG_LAUNCH_CHECK();
}

void link_soa(const float2 *U, float2 *UDs, int V, cudaStream_t s) {
  link_soa_kernel<<<grid_for((int64_t)V * 36), 256, 0, s>>>(U, UDs, V);
  MG_LAUNCH_CHECK();
}

template <typename T>
void wilson_split(const C<T> *in, C<T> *out9, const C<T> *U, Geom g, double m0, const int b[4],
                  cudaStream_t s) {
  dim3 grid(div_up(g.V, 128), 1);
  wilson_kernel<T, true><<<grid, 128, 0, s>>>(in, out9, U, g, (T)(4.0 + m0), b[0], b[1], b[2], b[3]);
  MG_LAUNCH_CHECK();
}

template <typename T>
void gamma5_apply(const C<T> *in, C<T> *out, int64_t nsites, int dof, int nrhs, cudaStream_t s) {
  const int64_t total = nsites * dof * nrhs;
  gamma5_kernel<T><<<grid_for(total), 256, 0, s>>>(in, out, total, dof);
  MG_LAUNCH_CHECK();
}

template <typename T>
void z4_noise(C<T> *out, Geom g, uint64_t seed, uint64_t sample0, uint64_t term, uint64_t aux,
              int slice, int nrhs, cudaStream_t s) {
  const int64_t n = g.n();
  int64_t lo = 0, hi = n;
  if (slice >= 0) {
    const int64_t per = n / g.L[3];
    lo = per * slice;
    hi = lo + per;
  }
  const int gx = grid_for((n + 3) / 4);
  z4_kernel<T><<<dim3(gx, nrhs), 256, 0, s>>>(out, n, seed, sample0, term, aux, lo, hi);
  MG_LAUNCH_CHECK();
}

#define INST(T)                                                                               \
  template void wilson_apply<T>(const C<T> *, C<T> *, const C<T> *, const C<T> *, Geom, double, \
                                int, int, cudaStream_t);                                      \
  template void wilson_split<T>(const C<T> *, C<T> *, const C<T> *, Geom, double, const int *, \
                                cudaStream_t);                                                \
  template void gamma5_apply<T>(const C<T> *, C<T> *, int64_t, int, int, cudaStream_t);       \
  template void z4_noise<T>(C<T> *, Geom, uint64_t, uint64_t, uint64_t, uint64_t, int, int,   \
                            cudaStream_t);
INST(double)
INST(float)

}  // namespace mg
