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

#include <cuda_bf16.h>

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

// ------------------------------------------------------------------ FP32 SoA
// The FP32 operator on the fine level, where spinors are stored
// structure-of-arrays (chunk k = components 2k, 2k+1 of all sites
// contiguous) and links likewise, UDs[mu][a][b][s].  One thread per site and
// R right-hand sides: every load of a warp is 32 consecutive 16-byte chunks
// (8-byte for links), the neighbour loads of the x direction hit the lines
// the centre load brought into L1, and each link is read once for R spinors
// from registers and once per right-hand-side group from L2 (the groups of a
// site range are neighbouring blocks).
// The nine operand sets (centre, then the hops x+, x-, y+, ..., t-) are
// consumed in order; with PIPE they form a register pipeline (set I + 1 is
// loaded while set I is consumed, two sets of loads in flight per thread).
namespace soa {
template <int R> struct Ctx {
  const float4 *P[R];
  const float2 *UDs;
  Geom g;
  int64_t V;
  int s, nr;
  int c[4];
  float diag;
  float2 acc[R][12];
};

template <int I, int R> __device__ __forceinline__ int item_site(const Ctx<R> &t) {
  if (I == 0) return t.s;
  constexpr int mu = (I - 1) / 2;
  int cn[4] = {t.c[0], t.c[1], t.c[2], t.c[3]};
  if (I & 1) cn[mu] = (t.c[mu] + 1 == t.g.L[mu]) ? 0 : t.c[mu] + 1;
  else cn[mu] = (t.c[mu] == 0) ? t.g.L[mu] - 1 : t.c[mu] - 1;
  return t.g.index(cn);
}

template <int I, int R>
__device__ __forceinline__ void load_item(const Ctx<R> &t, float4 (&p)[R][6], float2 (&u)[9]) {
  const int sn = item_site<I, R>(t);
#pragma unroll
  for (int q = 0; q < R; ++q)
    if (q < t.nr) {
#pragma unroll
      for (int k = 0; k < 6; ++k) p[q][k] = __ldg(t.P[q] + k * t.V + sn);
    }
  if constexpr (I > 0) {
    constexpr int mu = (I - 1) / 2;
    const float2 *u0 = t.UDs + (int64_t)mu * 9 * t.V + ((I & 1) ? t.s : sn);
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k] = __ldg(u0 + k * t.V);
  }
}

template <int I, int R>
__device__ __forceinline__ void use_item(Ctx<R> &t, const float4 (&p)[R][6], const float2 (&u)[9]) {
#pragma unroll
  for (int q = 0; q < R; ++q) {
    if (q < t.nr) {
      float2 v[12];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        v[2 * k] = make_float2(p[q][k].x, p[q][k].y);
        v[2 * k + 1] = make_float2(p[q][k].z, p[q][k].w);
      }
      if constexpr (I == 0) {
#pragma unroll
        for (int i = 0; i < 12; ++i) t.acc[q][i] = cscale(v[i], t.diag);
      } else {
        constexpr int mu = (I - 1) / 2;
        constexpr bool fwd = (I & 1) != 0;
        // antiperiodic time: hops across the t boundary change sign
        const bool wrap = mu == 3 && (fwd ? t.c[3] + 1 == t.g.L[3] : t.c[3] == 0);
        hop<mu, fwd, float>(v, u, wrap ? 0.5f : -0.5f, t.acc[q]);
      }
    }
  }
}

template <int I, int R>
__device__ __forceinline__ void step(Ctx<R> &t, float4 (&pc)[R][6], float2 (&uc)[9],
                                     float4 (&pn)[R][6], float2 (&un)[9]) {
  if constexpr (I < 8) load_item<I + 1, R>(t, pn, un);
  use_item<I, R>(t, pc, uc);
  if constexpr (I < 8) step<I + 1, R>(t, pn, un, pc, uc);
}
// the same sets one after the other: load, consume (scheduling left to the
// compiler, fewer registers)
template <int I, int R> __device__ __forceinline__ void serial(Ctx<R> &t) {
  float4 p[R][6];
  float2 u[9];
  load_item<I, R>(t, p, u);
  use_item<I, R>(t, p, u);
  if constexpr (I < 8) serial<I + 1, R>(t);
}
}  // namespace soa

template <int R, int BS, int MINB, bool PIPE>
__global__ void __launch_bounds__(BS, MINB) wilson_soa_kernel(const float2 *__restrict__ in,
                                                        float2 *__restrict__ out,
                                                        const float2 *__restrict__ UDs, Geom g,
                                                        float diag, int nrhs) {
  // the right-hand-side group varies fastest over consecutive blocks, so the
  // blocks sharing a site range (and its links) run close together in time
  const int ng = (nrhs + R - 1) / R;
  const int sb = (int)(blockIdx.x / ng), rg = (int)(blockIdx.x - (unsigned)sb * ng);
  const int s = sb * BS + threadIdx.x;
  if (s >= g.V) return;
  const int r0 = rg * R;
  const int64_t n = (int64_t)g.V * 12;
  soa::Ctx<R> t;
  t.nr = nrhs - r0 < R ? nrhs - r0 : R;
#pragma unroll
  for (int q = 0; q < R; ++q)
    t.P[q] = reinterpret_cast<const float4 *>(in + (r0 + (q < t.nr ? q : 0)) * n);
  t.UDs = UDs;
  t.g = g;
  t.V = g.V;
  t.s = s;
  t.diag = diag;
  g.coords(s, t.c);
  if constexpr (PIPE) {
    float4 pa[R][6], pb[R][6];
    float2 ua[9], ub[9];
    soa::load_item<0, R>(t, pa, ua);
    soa::step<0, R>(t, pa, ua, pb, ub);
  } else {
    soa::serial<0, R>(t);
  }
#pragma unroll
  for (int q = 0; q < R; ++q) {
    if (q < t.nr) {
      float4 *o = reinterpret_cast<float4 *>(out + (r0 + q) * n);
#pragma unroll
      for (int k = 0; k < 6; ++k)
        o[k * t.V + s] = make_float4(t.acc[q][2 * k].x, t.acc[q][2 * k].y, t.acc[q][2 * k + 1].x,
                                     t.acc[q][2 * k + 1].y);
    }
  }
}

// The right-hand sides of a group in the warps of one CTA: warp w of a CTA
// of 32 RW threads takes right-hand side r0 + w of the same 32 sites, so the
// links (and the neighbour sites' index arithmetic) of those sites are read
// by RW warps of one SM: from L1 after the first, instead of once per
// right-hand side from L2.  Same sums in the same order as the kernel above.
template <int RW, int MINB>
__global__ void __launch_bounds__(32 * RW, MINB) wilson_soa_rw_kernel(const float2 *__restrict__ in,
                                                                  float2 *__restrict__ out,
                                                                  const float2 *__restrict__ UDs, Geom g,
                                                                  float diag, int nrhs) {
  const int ng = (nrhs + RW - 1) / RW;
  const int sb = (int)(blockIdx.x / ng), rg = (int)(blockIdx.x - (unsigned)sb * ng);
  const int s = sb * 32 + (int)(threadIdx.x & 31);
  const int q = rg * RW + (int)(threadIdx.x >> 5);
  if (s >= g.V || q >= nrhs) return;
  const int64_t n = (int64_t)g.V * 12;
  soa::Ctx<1> t;
  t.nr = 1;
  t.P[0] = reinterpret_cast<const float4 *>(in + q * n);
  t.UDs = UDs;
  t.g = g;
  t.V = g.V;
  t.s = s;
  t.diag = diag;
  g.coords(s, t.c);
  soa::serial<0, 1>(t);
  float4 *o = reinterpret_cast<float4 *>(out + q * n);
#pragma unroll
  for (int k = 0; k < 6; ++k)
    o[k * t.V + s] = make_float4(t.acc[0][2 * k].x, t.acc[0][2 * k].y, t.acc[0][2 * k + 1].x,
                                 t.acc[0][2 * k + 1].y);
}

// ------------------------------------------------------------------ BF16
// BF16 storage, FP32 arithmetic.  Spinors structure-of-arrays in 16-byte
// chunks of 4 complex entries: component i of site s is bf16 pair
// ((i / 4) V + s) * 4 + i % 4 (3 chunks per site, 48 B); links
// structure-of-arrays as bf16 pairs, [mu][a][b][s].  One thread per site:
// each load of a warp is 32 consecutive 16-byte (spinor) or 4-byte (link)
// words; results are rounded to nearest on the store.
__device__ __forceinline__ void bf_load(const uint4 *__restrict__ P, int64_t V, int s, float2 (&p)[12]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const uint4 v = __ldg(P + k * V + s);
    const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      __nv_bfloat162 b;
      memcpy(&b, &w[j], 4);
      p[4 * k + j] = __bfloat1622float2(b);
    }
  }
}

template <int MU, bool FWD>
__device__ __forceinline__ void bf_dir(const uint4 *__restrict__ P, const __nv_bfloat162 *__restrict__ Ub,
                                       const Geom &g, int s, const int (&c)[4], float2 (&acc)[12]) {
  int cn[4] = {c[0], c[1], c[2], c[3]};
  if (FWD) cn[MU] = (c[MU] + 1 == g.L[MU]) ? 0 : c[MU] + 1;
  else cn[MU] = (c[MU] == 0) ? g.L[MU] - 1 : c[MU] - 1;
  const int sn = g.index(cn);
  const int64_t V = g.V;
  float2 u[9], p[12];
  const __nv_bfloat162 *u0 = Ub + (int64_t)MU * 9 * V + (FWD ? s : sn);
#pragma unroll
  for (int k = 0; k < 9; ++k) u[k] = __bfloat1622float2(u0[k * V]);
  bf_load(P, V, sn, p);
  const bool wrap = MU == 3 && (FWD ? c[3] + 1 == g.L[3] : c[3] == 0);
  hop<MU, FWD, float>(p, u, wrap ? 0.5f : -0.5f, acc);
}

__global__ void __launch_bounds__(128, 6) wilson_bf16_kernel(const uint4 *__restrict__ in, uint4 *__restrict__ out,
                                                             const __nv_bfloat162 *__restrict__ Ub, Geom g,
                                                             float diag) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  const int64_t V = g.V;
  const uint4 *P = in + blockIdx.y * 3 * V;
  int c[4];
  g.coords(s, c);
  float2 acc[12];
  bf_load(P, V, s, acc);
#pragma unroll
  for (int i = 0; i < 12; ++i) acc[i] = cscale(acc[i], diag);
  bf_dir<0, true>(P, Ub, g, s, c, acc);
  bf_dir<0, false>(P, Ub, g, s, c, acc);
  bf_dir<1, true>(P, Ub, g, s, c, acc);
  bf_dir<1, false>(P, Ub, g, s, c, acc);
  bf_dir<2, true>(P, Ub, g, s, c, acc);
  bf_dir<2, false>(P, Ub, g, s, c, acc);
  bf_dir<3, true>(P, Ub, g, s, c, acc);
  bf_dir<3, false>(P, Ub, g, s, c, acc);
  uint4 *o = out + blockIdx.y * 3 * V;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    unsigned w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const __nv_bfloat162 b = __float22bfloat162_rn(acc[4 * k + j]);
      memcpy(&w[j], &b, 4);
    }
    o[k * V + s] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// bf16 structure-of-arrays links from the FP32 canonical ones
__global__ void link_bf16_kernel(const float2 *__restrict__ U, __nv_bfloat162 *__restrict__ Ub, int V) {
  const int64_t total = (int64_t)V * 36;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i / 36;
    const int comp = (int)(i - s * 36);
    Ub[(int64_t)comp * V + s] = __float22bfloat162_rn(U[i]);
  }
}

// canonical complex-bf16 vectors (re, im pairs, [site][12]) <-> the chunked
// structure-of-arrays order above
__global__ void relayout_bf16_kernel(const __nv_bfloat162 *__restrict__ x, __nv_bfloat162 *__restrict__ y,
                                     int64_t V, bool to_soa) {
  const int64_t n = V * 12;
  const __nv_bfloat162 *xr = x + blockIdx.y * n;
  __nv_bfloat162 *yr = y + blockIdx.y * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = e / 12;
    const int i = (int)(e - s * 12);
    const int64_t is = ((int64_t)(i >> 2) * V + s) * 4 + (i & 3);
    if (to_soa) yr[is] = xr[e];
    else yr[e] = xr[is];
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

// per site the upper half of the dofs keeps its sign, the lower half flips;
// in the structure-of-arrays order (vec > 0: complex entries per vector) the
// lower half is the second half of each vector
template <typename T>
__global__ void gamma5_kernel(const C<T> *__restrict__ in, C<T> *__restrict__ out, int64_t total,
                              int dof, int64_t vec) {
  const int half = dof / 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool upper = vec > 0 ? (i % vec) < vec / 2 : (int)(i % dof) < half;
    out[i] = upper ? in[i] : cneg(in[i]);
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

// ------------------------------------------------------------------ gauge
// Synthetic links U = exp(i eps H), H traceless Hermitian.  Link L = 4 s + mu
// draws the 20 Philox4x64-10 words of counters (L, j, 128, 0), j = 0..4, key
// (seed, 0); entry e (row-major) of A uses words 2e, 2e + 1 as uniforms
// u = ((w >> 12) + 1/2) 2^-52 in (0, 1) (exact: the sum stays below 2^52)
// and Box-Muller:
// A_e = sqrt(-2 ln u1) (cos 2 pi u2 + i sin 2 pi u2) / sqrt 2, E|A_e|^2 = 1.
// H = (A + A^H) / 2 - tr / 3; the exponential by scaling (Frobenius norm
// <= 1/4), a degree-16 Taylor polynomial and repeated squaring, all FP64.
constexpr uint64_t kTermGauge = 128;

__device__ __forceinline__ void mat3_mul(const double2 (&a)[9], const double2 (&b)[9],
                                         double2 (&c)[9]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double2 z = make_double2(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < 3; ++k) z = cfma(a[3 * i + k], b[3 * k + j], z);
      c[3 * i + j] = z;
    }
}

__global__ void gauge_kernel(double2 *__restrict__ U, int64_t nlinks, double eps, uint64_t seed) {
  for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < nlinks;
       L += (int64_t)gridDim.x * blockDim.x) {
    uint64_t w[20];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      U64x4 c;
      c.v[0] = (uint64_t)L;
      c.v[1] = (uint64_t)j;
      c.v[2] = kTermGauge;
      c.v[3] = 0ull;
      const U64x4 r = philox4x64_10(c, seed, 0ull);
#pragma unroll
      for (int k = 0; k < 4; ++k) w[4 * j + k] = r.v[k];
    }
    double2 A[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const double u1 = ((double)(w[2 * e] >> 12) + 0.5) * 0x1p-52;
      const double u2 = ((double)(w[2 * e + 1] >> 12) + 0.5) * 0x1p-52;
      const double rho = sqrt(-2.0 * log(u1)) * 0.70710678118654752440;
      double sn, cs;
      sincospi(2.0 * u2, &sn, &cs);
      A[e] = make_double2(rho * cs, rho * sn);
    }
    double2 X[9];
    double nrm2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        // H_ab = (A_ab + conj(A_ba)) / 2, X = i eps H
        const double hr = 0.5 * (A[3 * a + b].x + A[3 * b + a].x);
        const double hi = 0.5 * (A[3 * a + b].y - A[3 * b + a].y);
        X[3 * a + b] = make_double2(-eps * hi, eps * hr);
      }
    const double tr = (X[0].y + X[4].y + X[8].y) / 3.0;  // X diagonal is i eps H_aa
    X[0].y -= tr;
    X[4].y -= tr;
    X[8].y -= tr;
#pragma unroll
    for (int e = 0; e < 9; ++e) nrm2 += X[e].x * X[e].x + X[e].y * X[e].y;
    int k = 0;
    double scale = 1.0;
    while (nrm2 * scale * scale > 0.0625 && k < 60) {
      scale *= 0.5;
      ++k;
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) X[e] = cscale(X[e], scale);
    double2 E[9], T[9], Tn[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) E[e] = T[e] = make_double2((e % 4 == 0) ? 1.0 : 0.0, 0.0);
    for (int m = 1; m <= 16; ++m) {
      mat3_mul(T, X, Tn);
#pragma unroll
      for (int e = 0; e < 9; ++e) {
        T[e] = cscale(Tn[e], 1.0 / m);
        E[e] = cadd(E[e], T[e]);
      }
    }
    for (int q = 0; q < k; ++q) {
      mat3_mul(E, E, Tn);
#pragma unroll
      for (int e = 0; e < 9; ++e) E[e] = Tn[e];
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) U[L * 9 + e] = E[e];
  }
}

inline int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

}  // namespace

namespace {
template <int RW, int MINB>
void launch_soa_rw(const float2 *in, float2 *out, const float2 *UDs, Geom g, float diag, int nrhs,
                   cudaStream_t s) {
  const int64_t blocks = (int64_t)div_up(g.V, 32) * div_up(nrhs, RW);
  if (blocks > 0x7fffffff) throw Error(1, "lattice too large for one launch");
  wilson_soa_rw_kernel<RW, MINB><<<(unsigned)blocks, 32 * RW, 0, s>>>(in, out, UDs, g, diag, nrhs);
  MG_LAUNCH_CHECK();
}

template <int R, int MINB, bool PIPE>
void launch_soa(const float2 *in, float2 *out, const float2 *UDs, Geom g, float diag, int nrhs,
                cudaStream_t s) {
  constexpr int BS = 128;
  const int64_t blocks = (int64_t)div_up(g.V, BS) * div_up(nrhs, R);
  if (blocks > 0x7fffffff) throw Error(1, "lattice too large for one launch");
  wilson_soa_kernel<R, BS, MINB, PIPE><<<(unsigned)blocks, BS, 0, s>>>(in, out, UDs, g, diag, nrhs);
  MG_LAUNCH_CHECK();
}
}  // namespace

int wilson_fp32_variants() { return 7; }

template <typename T>
void wilson_apply(const C<T> *in, C<T> *out, const C<T> *U, const C<T> *UDs, Geom g, double m0,
                  int nrhs, int variant, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if ((((uintptr_t)in | (uintptr_t)out) & 15) != 0 || !UDs)
      throw Error(1, "FP32 fine vectors and links must be 16-byte aligned structure-of-arrays");
    const float diag = (float)(4.0 + m0);
    // (right-hand sides per thread, resident 128-thread blocks per SM the
    // register budget is cut for, register pipeline)
    switch (variant) {
      case 1: launch_soa<1, 8, false>(in, out, UDs, g, diag, nrhs, s); return;
      case 2: launch_soa<2, 4, false>(in, out, UDs, g, diag, nrhs, s); return;
      case 3: launch_soa<2, 5, false>(in, out, UDs, g, diag, nrhs, s); return;
      case 4: launch_soa<1, 4, true>(in, out, UDs, g, diag, nrhs, s); return;
      case 5: launch_soa_rw<4, 5>(in, out, UDs, g, diag, nrhs, s); return;
      case 6: launch_soa_rw<8, 2>(in, out, UDs, g, diag, nrhs, s); return;
      default: launch_soa<1, 6, false>(in, out, UDs, g, diag, nrhs, s); return;
    }
  } else {
    (void)UDs;
    (void)variant;
    dim3 grid(div_up(g.V, 128), nrhs);
    wilson_kernel<T, false><<<grid, 128, 0, s>>>(in, out, U, g, (T)(4.0 + m0), 1, 1, 1, 1);
    MG_LAUNCH_CHECK();
  }
}

void wilson_apply_bf16(const void *in, void *out, const void *Ub, Geom g, double m0, int nrhs,
                       cudaStream_t s) {
  if ((((uintptr_t)in | (uintptr_t)out) & 15) != 0 || !Ub)
    throw Error(1, "BF16 fine vectors must be 16-byte aligned");
  dim3 grid(div_up(g.V, 128), nrhs);
  wilson_bf16_kernel<<<grid, 128, 0, s>>>(static_cast<const uint4 *>(in), static_cast<uint4 *>(out),
                                          static_cast<const __nv_bfloat162 *>(Ub), g, (float)(4.0 + m0));
  MG_LAUNCH_CHECK();
}

void link_bf16(const float2 *U, void *Ub, int V, cudaStream_t s) {
  link_bf16_kernel<<<grid_for((int64_t)V * 36), 256, 0, s>>>(U, static_cast<__nv_bfloat162 *>(Ub), V);
  MG_LAUNCH_CHECK();
}

void relayout_bf16(const void *x, void *y, int64_t V, int nrhs, bool to_soa, cudaStream_t s) {
  const int gx = (grid_for(V * 12) + nrhs - 1) / nrhs + 1;
  relayout_bf16_kernel<<<dim3(gx, nrhs), 256, 0, s>>>(static_cast<const __nv_bfloat162 *>(x),
                                                      static_cast<__nv_bfloat162 *>(y), V, to_soa);
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
void gamma5_apply(const C<T> *in, C<T> *out, int64_t nsites, int dof, int nrhs, cudaStream_t s,
                  bool soa) {
  const int64_t total = nsites * dof * nrhs;
  gamma5_kernel<T><<<grid_for(total), 256, 0, s>>>(in, out, total, dof, soa ? nsites * dof : 0);
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

void gauge_generate(double2 *U, int64_t nlinks, double eps, uint64_t seed, cudaStream_t s) {
  gauge_kernel<<<grid_for(nlinks), 256, 0, s>>>(U, nlinks, eps, seed);
  MG_LAUNCH_CHECK();
}

#define INST(T)                                                                               \
  template void wilson_apply<T>(const C<T> *, C<T> *, const C<T> *, const C<T> *, Geom, double, \
                                int, int, cudaStream_t);                                      \
  template void wilson_split<T>(const C<T> *, C<T> *, const C<T> *, Geom, double, const int *, \
                                cudaStream_t);                                                \
  template void gamma5_apply<T>(const C<T> *, C<T> *, int64_t, int, int, cudaStream_t, bool); \
  template void z4_noise<T>(C<T> *, Geom, uint64_t, uint64_t, uint64_t, uint64_t, int, int,   \
                            cudaStream_t);
INST(double)
INST(float)

}  // namespace mg
