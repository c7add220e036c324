// Schwarz alternating procedure (SAP) smoother on the fine lattice: the
// domain-decomposition smoother of the paper's solver (DD-alpha-AMG, Sec. 4)
// written for one GPU.
//
// The lattice is cut into blocks of extent b[4]; blocks are coloured red /
// black by the parity of their block coordinates (every direction must hold
// an even number of blocks, so neighbouring blocks always differ in colour).
// One sweep visits red then black blocks.  For every block B of the active
// colour, in parallel, a few minimal-residual iterations solve
// D_BB e_B = r_B with the block-local Wilson operator (hops that leave B are
// dropped); then z_B += e_B, the residual inside B becomes the block MR
// residual, and the residual of the other colour loses the hops of e that
// cross block faces.  The residual r = b - D z is exact at the end of the
// sweep.  That last update runs as a face pass over the other colour's
// sites after each colour's blocks: red blocks, face pass on the black
// sites, black blocks, face pass on the red sites (four launches per sweep).
//
// Three block kernels, for FP32 blocks of 256 sites with every extent >= 2
// (8 x 4 x 4 x 2 and 4^4) and two or more right-hand sides: the staged one
// (the default) gives each thread one (site, right-hand side), the block's
// links and the z it updates arriving in shared memory by asynchronous
// copies that overlap the residual load; the paired one gives each thread
// one site and two right-hand sides held in the two lanes of packed
// registers (.f32x2 arithmetic: one instruction and one link read from
// shared memory serve both; fewer instructions, but its 197 KB of shared
// memory leaves 8 warps per SM).  The general one below serves FP64, other
// block shapes and single right-hand sides.  All compute the same sums in
// the same order.
//
// One CTA per (active block, rhs), one thread per site of the block; the
// right-hand side varies fastest over the grid, so the CTAs of a block share
// its links through L2.  The block's links and its residual live in shared
// memory for all block iterations (FP32: 256 sites x (36 + 12) complex = 98
// KB), so the MR iterations touch HBM once per sweep.  FP32 vectors and
// links are in the fine level's structure-of-arrays order, FP64 ones
// canonical.
#include "kernels.h"

namespace mg {

namespace {

template <typename T> constexpr bool kSoa = sizeof(T) == 4;

// the 9 colour entries of U_mu(site): FP32 structure-of-arrays links
// U[mu][a][b][V], FP64 canonical [V][mu][a][b]
template <typename T>
__device__ __forceinline__ void link_at(const C<T> *__restrict__ U, int64_t V, int64_t site, int mu,
                                        C<T> (&u)[9]) {
#pragma unroll
  for (int k = 0; k < 9; ++k)
    u[k] = kSoa<T> ? U[(int64_t)(mu * 9 + k) * V + site] : U[(site * 4 + mu) * 9 + k];
}

struct SapGeom {
  Geom g;
  int b[4];   // block extents
  int nb[4];  // blocks per direction
  int sites;  // sites per block
};

template <int MU, typename V> __device__ __forceinline__ V sBl(int a, V l0, V l1) {
  if (MU == 0) return a == 0 ? cmulmi(l1) : cmulmi(l0);
  if (MU == 1) return a == 0 ? cneg(l1) : l0;
  if (MU == 2) return a == 0 ? cmulmi(l0) : cmuli(l1);
  return a == 0 ? l0 : l1;
}
template <int MU, typename V> __device__ __forceinline__ V sBh(int a, V v0, V v1) {
  if (MU == 0) return a == 0 ? cmuli(v1) : cmuli(v0);
  if (MU == 1) return a == 0 ? v1 : cneg(v0);
  if (MU == 2) return a == 0 ? cmuli(v0) : cmulmi(v1);
  return a == 0 ? v0 : v1;
}

// acc += k * (1 -+ gamma_MU) (U or U^H) p   (same algebra as the full operator)
template <int MU, bool FWD, typename T>
__device__ __forceinline__ void shop(const C<T> *p, const C<T> *u, T k, C<T> (&acc)[12]) {
  const T sg = FWD ? (T)-1 : (T)1;
  C<T> h[2][3];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) h[a][c] = cadd(p[3 * a + c], cscale(sBl<MU>(a, p[6 + c], p[9 + c]), sg));
  C<T> v[2][3];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      C<T> z = mk<T>((T)0, (T)0);
#pragma unroll
      for (int bb = 0; bb < 3; ++bb) {
        if (FWD) z = cfma(u[3 * c + bb], h[a][bb], z);
        else z = cfmac(u[3 * bb + c], h[a][bb], z);
      }
      v[a][c] = z;
    }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      acc[3 * a + c].x = fma(k, v[a][c].x, acc[3 * a + c].x);
      acc[3 * a + c].y = fma(k, v[a][c].y, acc[3 * a + c].y);
      const C<T> w = sBh<MU>(a, v[0][c], v[1][c]);
      acc[6 + 3 * a + c].x = fma(sg * k, w.x, acc[6 + 3 * a + c].x);
      acc[6 + 3 * a + c].y = fma(sg * k, w.y, acc[6 + 3 * a + c].y);
    }
}

// block index (of all blocks) of the i-th block of colour `color`
__device__ __forceinline__ void active_block(const SapGeom &sg, int i, int color, int (&bc)[4]) {
  const int half = sg.nb[0] >> 1;
  const int k = i % half;
  int rest = i / half;
  bc[1] = rest % sg.nb[1];
  rest /= sg.nb[1];
  bc[2] = rest % sg.nb[2];
  bc[3] = rest / sg.nb[2];
  bc[0] = 2 * k + ((color + bc[1] + bc[2] + bc[3]) & 1);
}

// sum (v0, v1, v2) over the block in the storage precision (warp shuffles,
// then the per-warp sums in a fixed order), result in out3 for all threads;
// FP32 sums here keep the block MR iterations off the slow FP64 pipe
template <typename T>
__device__ __forceinline__ void block_reduce3(T v0, T v1, T v2, T *s, T *out3) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v0 += __shfl_down_sync(0xffffffffu, v0, o);
    v1 += __shfl_down_sync(0xffffffffu, v1, o);
    v2 += __shfl_down_sync(0xffffffffu, v2, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  if (l == 0) {
    s[3 * w] = v0;
    s[3 * w + 1] = v1;
    s[3 * w + 2] = v2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    T a = 0, b = 0, c = 0;
    for (int i = 0; i < nw; ++i) {
      a += s[3 * i];
      b += s[3 * i + 1];
      c += s[3 * i + 2];
    }
    out3[0] = a;
    out3[1] = b;
    out3[2] = c;
  }
  __syncthreads();
}

// block_reduce3 over the threads of one right-hand-side slot of a CTA that
// holds RS slots of `sites` threads each (sites a multiple of 32): lt is the
// thread's index within its slot, s / out3 the slot's scratch
template <typename T>
__device__ __forceinline__ void slot_reduce3(T v0, T v1, T v2, T *s, T *out3, int lt, int nw) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v0 += __shfl_down_sync(0xffffffffu, v0, o);
    v1 += __shfl_down_sync(0xffffffffu, v1, o);
    v2 += __shfl_down_sync(0xffffffffu, v2, o);
  }
  const int w = lt >> 5, l = lt & 31;
  if (l == 0) {
    s[3 * w] = v0;
    s[3 * w + 1] = v1;
    s[3 * w + 2] = v2;
  }
  __syncthreads();
  if (lt == 0) {
    T a = 0, b = 0, c = 0;
    for (int i = 0; i < nw; ++i) {
      a += s[3 * i];
      b += s[3 * i + 1];
      c += s[3 * i + 2];
    }
    out3[0] = a;
    out3[1] = b;
    out3[2] = c;
  }
  __syncthreads();
}

// rho [12][sites] and Us [4 * 9][sites] are component-major in shared memory:
// the threads of a warp (consecutive sites of the block) read consecutive
// words, free of bank conflicts
template <typename T, int DIR>
__device__ __forceinline__ void local_hops(const C<T> *rho, const C<T> *Us, const int (&lc)[4],
                                           const int *b, int lsite, int sites, C<T> (&acc)[12]) {
  int stride = 1;
  for (int i = 0; i < DIR; ++i) stride *= b[i];
  // the time-boundary sign never applies inside a block: blocks tile the
  // lattice without wrapping
  if (lc[DIR] + 1 < b[DIR]) {
    const int ln = lsite + stride;
    C<T> p[12], u[9];
#pragma unroll
    for (int i = 0; i < 12; ++i) p[i] = rho[i * sites + ln];
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k] = Us[(DIR * 9 + k) * sites + lsite];
    shop<DIR, true, T>(p, u, (T)-0.5, acc);
  }
  if (lc[DIR] > 0) {
    const int ln = lsite - stride;
    C<T> p[12], u[9];
#pragma unroll
    for (int i = 0; i < 12; ++i) p[i] = rho[i * sites + ln];
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k] = Us[(DIR * 9 + k) * sites + ln];
    shop<DIR, false, T>(p, u, (T)-0.5, acc);
  }
}

// residual of the inactive colour: r(x) -= hops of e that cross a block face
// into x from a block of the active colour.
template <int MU, typename T>
__device__ __forceinline__ void cross_pair(const C<T> *__restrict__ ev, const C<T> *__restrict__ U,
                                           const SapGeom &sg, int s, const int (&c)[4],
                                           C<T> (&acc)[12], T sign = (T)1) {
  const Geom &g = sg.g;
  {
    int cn[4] = {c[0], c[1], c[2], c[3]};
    cn[MU] = (c[MU] + 1 == g.L[MU]) ? 0 : c[MU] + 1;
    if (c[MU] / sg.b[MU] != cn[MU] / sg.b[MU]) {
      const int sn = g.index(cn);
      const T k = sign * ((MU == 3 && cn[3] == 0) ? (T)0.5 : (T)-0.5);
      C<T> p[12], u[9];
      load_fine_site<T>(ev, sn, g.V, p);
      link_at<T>(U, g.V, s, MU, u);
      shop<MU, true, T>(p, u, k, acc);
    }
  }
  {
    int cn[4] = {c[0], c[1], c[2], c[3]};
    cn[MU] = (c[MU] == 0) ? g.L[MU] - 1 : c[MU] - 1;
    if (c[MU] / sg.b[MU] != cn[MU] / sg.b[MU]) {
      const int sn = g.index(cn);
      const T k = sign * ((MU == 3 && c[3] == 0) ? (T)0.5 : (T)-0.5);
      C<T> p[12], u[9];
      load_fine_site<T>(ev, sn, g.V, p);
      link_at<T>(U, g.V, sn, MU, u);
      shop<MU, false, T>(p, u, k, acc);
    }
  }
}

// The same for blocks of extent >= 2 in MU, where at most one of the two hops
// of a site leaves its block: one set of loads per direction instead of two
// (the threads of a warp that cross forward and those that cross backward
// load together), the sum unchanged.
template <int MU, typename T>
__device__ __forceinline__ void cross_one(const C<T> *__restrict__ ev, const C<T> *__restrict__ U,
                                          const Geom &g, int s, const int (&c)[4], int lcm, int bm,
                                          C<T> (&acc)[12], T sign) {
  const bool fwd = lcm == bm - 1;
  if (!fwd && lcm != 0) return;
  int cn[4] = {c[0], c[1], c[2], c[3]};
  if (fwd) cn[MU] = (c[MU] + 1 == g.L[MU]) ? 0 : c[MU] + 1;
  else cn[MU] = (c[MU] == 0) ? g.L[MU] - 1 : c[MU] - 1;
  const int sn = g.index(cn);
  const bool tb = MU == 3 && (fwd ? cn[3] == 0 : c[3] == 0);
  const T k = sign * (tb ? (T)0.5 : (T)-0.5);
  C<T> p[12], u[9];
  load_fine_site<T>(ev, sn, g.V, p);
  link_at<T>(U, g.V, fwd ? s : sn, MU, u);
  if (fwd) shop<MU, true, T>(p, u, k, acc);
  else shop<MU, false, T>(p, u, k, acc);
}

template <int MU, typename T>
__device__ __forceinline__ void cross_dir(const C<T> *__restrict__ ev, const C<T> *__restrict__ U,
                                          const SapGeom &sg, int s, const int (&c)[4], int lcm,
                                          C<T> (&acc)[12], T sign) {
  if (sg.b[MU] >= 2) cross_one<MU, T>(ev, U, sg.g, s, c, lcm, sg.b[MU], acc, sign);
  else cross_pair<MU, T>(ev, U, sg, s, c, acc, sign);
}

// 16-byte asynchronous global -> shared copies (completion awaited with
// cp.async.wait_group, which ends when the copies land)
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <int B0, int B1, int B2, int B3> struct SapShape {
  static constexpr int S = B0 * B1 * B2 * B3;
  static constexpr int b(int i) { return i == 0 ? B0 : i == 1 ? B1 : i == 2 ? B2 : B3; }
  static constexpr int stride(int i) { return i == 0 ? 1 : i == 1 ? B0 : i == 2 ? B0 * B1 : B0 * B1 * B2; }
};

// the 12 components of a site from [6][S] float4 chunks in shared memory
template <int S>
__device__ __forceinline__ void chunk_site(const float4 *v, int site, float2 (&p)[12]) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float4 q = v[k * S + site];
    p[2 * k] = make_float2(q.x, q.y);
    p[2 * k + 1] = make_float2(q.z, q.w);
  }
}

// block-local hops of direction DIR on the staged residual (compile-time
// block geometry; same sums as local_hops)
template <int DIR, class SH>
__device__ __forceinline__ void staged_hops(const float4 *rho, const float2 *Us, const int (&lc)[4], int ls,
                                            float2 (&acc)[12]) {
  constexpr int S = SH::S, st = SH::stride(DIR), bd = SH::b(DIR);
  if (lc[DIR] + 1 < bd) {
    float2 p[12], u[9];
    chunk_site<S>(rho, ls + st, p);
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k] = Us[(DIR * 9 + k) * S + ls];
    shop<DIR, true, float>(p, u, -0.5f, acc);
  }
  if (lc[DIR] > 0) {
    const int ln = ls - st;
    float2 p[12], u[9];
    chunk_site<S>(rho, ln, p);
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k] = Us[(DIR * 9 + k) * S + ln];
    shop<DIR, false, float>(p, u, -0.5f, acc);
  }
}

// Staged FP32 block kernel: one CTA per (active block, pair of right-hand
// sides), one thread per (site, right-hand side).  Shared memory: links
// [36][S] float2, residuals [2][6][S] float4, the z being updated [2][6][S]
// float4, reduction partials (172 KB at S = 256).  The links (shared by both
// slots) and z are asynchronous copies issued before the residual load and
// the face terms, awaited before the first block iteration; the MR iterations
// and every sum follow sap_block_kernel exactly (bit-identical results).
template <int B0, int B1, int B2, int B3>
__global__ void __launch_bounds__(2 * B0 * B1 * B2 * B3, 1)
    sap_block_staged_kernel(float2 *__restrict__ r, float2 *__restrict__ z, float2 *e_out,
                            const float2 *__restrict__ U, SapGeom sg, float diag, int color, int iters,
                            int nrhs) {
  using SH = SapShape<B0, B1, B2, B3>;
  constexpr int S = SH::S, NW = S / 32;
  static_assert(S % 32 == 0 && B0 % 2 == 0 && B1 >= 2 && B2 >= 2 && B3 >= 2, "staged SAP block shape");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *Us = reinterpret_cast<float2 *>(smem_raw);
  float4 *vbase = reinterpret_cast<float4 *>(Us + 36 * S);
  const int slot = (int)threadIdx.x / S;
  const int ls = (int)threadIdx.x - slot * S;
  float4 *rho = vbase + slot * 6 * S;
  float4 *zs = vbase + (2 + slot) * 6 * S;
  float *red = reinterpret_cast<float *>(vbase + 4 * 6 * S) + slot * 3 * NW;
  const Geom &g = sg.g;
  const int64_t n = g.n(), V = g.V;
  const int ngr = (nrhs + 1) >> 1;
  const int rq = (int)(blockIdx.x % (unsigned)ngr) * 2 + slot;
  const bool live = rq < nrhs;  // a slot past the last right-hand side computes on zeros
  const int rr = live ? rq : nrhs - 1;
  float2 *rv = r + rr * n;
  float2 *zv = z + rr * n;
  float2 *ev = e_out + rr * n;
  int bc[4];
  active_block(sg, (int)(blockIdx.x / (unsigned)ngr), color, bc);
  const int lc[4] = {ls % B0, (ls / B0) % B1, (ls / (B0 * B1)) % B2, ls / (B0 * B1 * B2)};
  int gc[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) gc[i] = bc[i] * SH::b(i) + lc[i];
  const int s = g.index(gc);
  {
    // links: 16-byte copies of site pairs (x rows hold an even number of
    // sites starting at an even x), 9 per thread at S = 256
    int oc[4] = {bc[0] * B0, bc[1] * B1, bc[2] * B2, bc[3] * B3};
    const int64_t s0 = g.index(oc);
    static_assert((18 * S) % (2 * S) == 0, "link chunks per thread");
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const int j = q * 2 * S + (int)threadIdx.x;
      const int comp = j / (S / 2), l0 = 2 * (j - comp * (S / 2));
      const int lx = l0 % B0, ly = (l0 / B0) % B1, lz = (l0 / (B0 * B1)) % B2, lt = l0 / (B0 * B1 * B2);
      const int64_t gs = s0 + lx + (int64_t)g.L[0] * (ly + g.L[1] * (lz + (int64_t)g.L[2] * lt));
      cp_async16(Us + comp * S + l0, U + (int64_t)comp * V + gs);
    }
    if (live) {
      const float4 *zc = reinterpret_cast<const float4 *>(zv);
#pragma unroll
      for (int k = 0; k < 6; ++k) cp_async16(zs + k * S + ls, zc + (int64_t)k * V + s);
    }
    cp_async_commit();
  }
  float2 rh[12];
  if (live) {
    load_fine_site<float>(rv, s, V, rh);
  } else {
#pragma unroll
    for (int i = 0; i < 12; ++i) rh[i] = make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int k = 0; k < 6; ++k)
    rho[k * S + ls] = make_float4(rh[2 * k].x, rh[2 * k].y, rh[2 * k + 1].x, rh[2 * k + 1].y);
  float2 e[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) e[i] = make_float2(0.f, 0.f);
  cp_async_wait_all();
  __syncthreads();
  for (int it = 0; it < iters; ++it) {
    float2 q[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) q[i] = cscale(rh[i], diag);
    staged_hops<0, SH>(rho, Us, lc, ls, q);
    staged_hops<1, SH>(rho, Us, lc, ls, q);
    staged_hops<2, SH>(rho, Us, lc, ls, q);
    staged_hops<3, SH>(rho, Us, lc, ls, q);
    float qr_re = 0.f, qr_im = 0.f, qq = 0.f;
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      const float2 p = rh[i];
      qr_re = fmaf(q[i].x, p.x, fmaf(q[i].y, p.y, qr_re));
      qr_im = fmaf(q[i].x, p.y, fmaf(-q[i].y, p.x, qr_im));
      qq = fmaf(q[i].x, q[i].x, fmaf(q[i].y, q[i].y, qq));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      qr_re += __shfl_down_sync(0xffffffffu, qr_re, o);
      qr_im += __shfl_down_sync(0xffffffffu, qr_im, o);
      qq += __shfl_down_sync(0xffffffffu, qq, o);
    }
    if ((ls & 31) == 0) {
      red[3 * (ls >> 5)] = qr_re;
      red[3 * (ls >> 5) + 1] = qr_im;
      red[3 * (ls >> 5) + 2] = qq;
    }
    __syncthreads();
    // every thread sums the per-warp partials in warp order (the order of
    // slot_reduce3), so no second barrier is needed
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      a0 += red[3 * w];
      a1 += red[3 * w + 1];
      a2 += red[3 * w + 2];
    }
    const float2 al = a2 > 1e-30f ? make_float2(a0 / a2, a1 / a2) : make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      const float2 p = rh[i];
      e[i] = cfma(al, p, e[i]);
      rh[i] = cfma(cneg(al), q[i], p);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k)
      rho[k * S + ls] = make_float4(rh[2 * k].x, rh[2 * k].y, rh[2 * k + 1].x, rh[2 * k + 1].y);
    __syncthreads();
  }
  if (!live) return;
  {
    float2 zz[12];
    chunk_site<S>(zs, ls, zz);
#pragma unroll
    for (int i = 0; i < 12; ++i) zz[i] = cadd(zz[i], e[i]);
    store_fine_site<float>(zv, s, V, zz);
  }
  store_fine_site<float>(ev, s, V, e);
  store_fine_site<float>(rv, s, V, rh);
}

// ---- paired FP32 arithmetic (P2 and the p2* helpers of common.cuh): the
// same component of two right-hand sides in the two lanes of a register pair

// the spin-projection and reconstruction rules of sBl / sBh as data: the
// result's real (imaginary) part is sign * (real or imaginary part) of one
// of two inputs
struct SpinRule {
  int src, xc, xs, yc, ys;  // input 0/1; x from component xc (0 re, 1 im) with sign xs; y likewise
};
template <int MU> __host__ __device__ constexpr SpinRule rule_bl(int a) {
  return MU == 0 ? (a == 0 ? SpinRule{1, 1, 1, 0, -1} : SpinRule{0, 1, 1, 0, -1})
       : MU == 1 ? (a == 0 ? SpinRule{1, 0, -1, 1, -1} : SpinRule{0, 0, 1, 1, 1})
       : MU == 2 ? (a == 0 ? SpinRule{0, 1, 1, 0, -1} : SpinRule{1, 1, -1, 0, 1})
                 : (a == 0 ? SpinRule{0, 0, 1, 1, 1} : SpinRule{1, 0, 1, 1, 1});
}
template <int MU> __host__ __device__ constexpr SpinRule rule_bh(int a) {
  return MU == 0 ? (a == 0 ? SpinRule{1, 1, -1, 0, 1} : SpinRule{0, 1, -1, 0, 1})
       : MU == 1 ? (a == 0 ? SpinRule{1, 0, 1, 1, 1} : SpinRule{0, 0, -1, 1, -1})
       : MU == 2 ? (a == 0 ? SpinRule{0, 1, -1, 0, 1} : SpinRule{1, 1, 1, 0, -1})
                 : (a == 0 ? SpinRule{0, 0, 1, 1, 1} : SpinRule{1, 0, 1, 1, 1});
}

// shop for a pair of right-hand sides: acc += k (1 -+ gamma_MU) (U or U^H) p
// with p, acc as (real, imaginary) pairs and the link entries as broadcast
// pairs (uR = (re, re), uI = (im, im)); kt = (k, k), kp = (sg k, sg k),
// kn = -kp.  Every lane performs the scalar shop's operations in its order.
template <int MU, bool FWD>
__device__ __forceinline__ void shop2(const P2 (&pR)[12], const P2 (&pI)[12], const P2 (&uR)[9],
                                      const P2 (&uI)[9], P2 kt, P2 kp, P2 kn, P2 (&aR)[12], P2 (&aI)[12]) {
  constexpr int sg = FWD ? -1 : 1;
  P2 hR[2][3], hI[2][3];
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    constexpr int dummy = 0;
    (void)dummy;
    const SpinRule r = rule_bl<MU>(a);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const P2 sx = r.xc == 0 ? pR[6 + 3 * r.src + c] : pI[6 + 3 * r.src + c];
      const P2 sy = r.yc == 0 ? pR[6 + 3 * r.src + c] : pI[6 + 3 * r.src + c];
      hR[a][c] = sg * r.xs > 0 ? p2add(pR[3 * a + c], sx) : p2sub(pR[3 * a + c], sx);
      hI[a][c] = sg * r.ys > 0 ? p2add(pI[3 * a + c], sy) : p2sub(pI[3 * a + c], sy);
    }
  }
  P2 nh[2][3];  // the negated component the complex product needs: -Im h (forward), -Re h (backward)
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) nh[a][c] = p2neg(FWD ? hI[a][c] : hR[a][c]);
  P2 vR[2][3], vI[2][3];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      P2 zr = p2(0.f, 0.f), zi = p2(0.f, 0.f);
#pragma unroll
      for (int bb = 0; bb < 3; ++bb) {
        if (FWD) {  // z += u[c][bb] h
          const int k = 3 * c + bb;
          zr = p2fma(uR[k], hR[a][bb], zr);
          zr = p2fma(uI[k], nh[a][bb], zr);
          zi = p2fma(uR[k], hI[a][bb], zi);
          zi = p2fma(uI[k], hR[a][bb], zi);
        } else {  // z += conj(u[bb][c]) h
          const int k = 3 * bb + c;
          zr = p2fma(uR[k], hR[a][bb], zr);
          zr = p2fma(uI[k], hI[a][bb], zr);
          zi = p2fma(uR[k], hI[a][bb], zi);
          zi = p2fma(uI[k], nh[a][bb], zi);
        }
      }
      vR[a][c] = zr;
      vI[a][c] = zi;
    }
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const SpinRule r = rule_bh<MU>(a);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      aR[3 * a + c] = p2fma(kt, vR[a][c], aR[3 * a + c]);
      aI[3 * a + c] = p2fma(kt, vI[a][c], aI[3 * a + c]);
      const P2 wx = r.xc == 0 ? vR[r.src][c] : vI[r.src][c];
      const P2 wy = r.yc == 0 ? vR[r.src][c] : vI[r.src][c];
      aR[6 + 3 * a + c] = p2fma(r.xs > 0 ? kp : kn, wx, aR[6 + 3 * a + c]);
      aI[6 + 3 * a + c] = p2fma(r.ys > 0 ? kp : kn, wy, aI[6 + 3 * a + c]);
    }
  }
}

// the 12 components of a site from [12][S] (re pair, im pair) entries
template <int S>
__device__ __forceinline__ void pair_site(const ulonglong2 *v, int site, P2 (&pR)[12], P2 (&pI)[12]) {
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    const ulonglong2 t = v[i * S + site];
    pR[i].v = t.x;
    pI[i].v = t.y;
  }
}

template <int DIR, class SH>
__device__ __forceinline__ void pair_hops(const ulonglong2 *rho, const ulonglong2 *Us, const int (&lc)[4], int ls,
                                          P2 kt, P2 kpf, P2 knf, P2 kpb, P2 knb, P2 (&aR)[12], P2 (&aI)[12]) {
  constexpr int S = SH::S, st = SH::stride(DIR), bd = SH::b(DIR);
  if (lc[DIR] + 1 < bd) {
    P2 pR[12], pI[12], uR[9], uI[9];
    pair_site<S>(rho, ls + st, pR, pI);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const ulonglong2 t = Us[(DIR * 9 + k) * S + ls];
      uR[k].v = t.x;
      uI[k].v = t.y;
    }
    shop2<DIR, true>(pR, pI, uR, uI, kt, kpf, knf, aR, aI);
  }
  if (lc[DIR] > 0) {
    const int ln = ls - st;
    P2 pR[12], pI[12], uR[9], uI[9];
    pair_site<S>(rho, ln, pR, pI);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const ulonglong2 t = Us[(DIR * 9 + k) * S + ln];
      uR[k].v = t.x;
      uI[k].v = t.y;
    }
    shop2<DIR, false>(pR, pI, uR, uI, kt, kpb, knb, aR, aI);
  }
}

// Paired FP32 block kernel: one CTA per (active block, pair of right-hand
// sides), one thread per site holding both right-hand sides in the lanes of
// packed registers, so one instruction advances both and one link read from
// shared memory serves both.  Shared memory: links [36][S] as (re, re, im,
// im), the residual pair [12][S] as (re0, re1, im0, im1), reduction
// partials (197 KB at S = 256).  Same sums as sap_block_kernel.
template <int B0, int B1, int B2, int B3>
__global__ void __launch_bounds__(B0 * B1 * B2 * B3, 1)
    sap_block_pair_kernel(float2 *__restrict__ r, float2 *__restrict__ z, float2 *e_out,
                          const float2 *__restrict__ U, SapGeom sg, float diag, int color, int iters,
                          int nrhs) {
  using SH = SapShape<B0, B1, B2, B3>;
  constexpr int S = SH::S, NW = S / 32;
  static_assert(S % 32 == 0 && B0 >= 2 && B1 >= 2 && B2 >= 2 && B3 >= 2, "paired SAP block shape");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ulonglong2 *Us = reinterpret_cast<ulonglong2 *>(smem_raw);  // [36][S]
  ulonglong2 *rho = Us + 36 * S;                                // [12][S]
  float *red = reinterpret_cast<float *>(rho + 12 * S);        // [6][NW]
  const int ls = (int)threadIdx.x;
  const Geom &g = sg.g;
  const int64_t n = g.n(), V = g.V;
  const int ngr = (nrhs + 1) >> 1;
  const int r0 = (int)(blockIdx.x % (unsigned)ngr) * 2;
  const bool live1 = r0 + 1 < nrhs;  // the second lane computes on zeros past the last right-hand side
  int bc[4];
  active_block(sg, (int)(blockIdx.x / (unsigned)ngr), color, bc);
  const int lc[4] = {ls % B0, (ls / B0) % B1, (ls / (B0 * B1)) % B2, ls / (B0 * B1 * B2)};
  int gc[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) gc[i] = bc[i] * SH::b(i) + lc[i];
  const int s = g.index(gc);
  // links of this site, broadcast pairs
#pragma unroll
  for (int k = 0; k < 36; ++k) {
    const float2 u = __ldg(U + (int64_t)k * V + s);
    Us[k * S + ls] = make_ulonglong2(p2(u.x, u.x).v, p2(u.y, u.y).v);
  }
  float2 rh0[12], rh1[12];
  load_fine_site<float>(r + r0 * n, s, V, rh0);
  if (live1) {
    load_fine_site<float>(r + (r0 + 1) * n, s, V, rh1);
  } else {
#pragma unroll
    for (int i = 0; i < 12; ++i) rh1[i] = make_float2(0.f, 0.f);
  }
  P2 rR[12], rI[12], eR[12], eI[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    rR[i] = p2(rh0[i].x, rh1[i].x);
    rI[i] = p2(rh0[i].y, rh1[i].y);
    rho[i * S + ls] = make_ulonglong2(rR[i].v, rI[i].v);
    eR[i] = p2(0.f, 0.f);
    eI[i] = p2(0.f, 0.f);
  }
  __syncthreads();
  const P2 dg = p2(diag, diag);
  const P2 kt = p2(-0.5f, -0.5f);
  // bottom-half factors sg k (forward sg = -1: +0.5; backward sg = +1: -0.5) and their negatives
  const P2 kpf = p2(0.5f, 0.5f), knf = p2(-0.5f, -0.5f), kpb = p2(-0.5f, -0.5f), knb = p2(0.5f, 0.5f);
  for (int it = 0; it < iters; ++it) {
    P2 qR[12], qI[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      qR[i] = p2mul(rR[i], dg);
      qI[i] = p2mul(rI[i], dg);
    }
    pair_hops<0, SH>(rho, Us, lc, ls, kt, kpf, knf, kpb, knb, qR, qI);
    pair_hops<1, SH>(rho, Us, lc, ls, kt, kpf, knf, kpb, knb, qR, qI);
    pair_hops<2, SH>(rho, Us, lc, ls, kt, kpf, knf, kpb, knb, qR, qI);
    pair_hops<3, SH>(rho, Us, lc, ls, kt, kpf, knf, kpb, knb, qR, qI);
    P2 dre = p2(0.f, 0.f), dim = p2(0.f, 0.f), dqq = p2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      dre = p2fma(qR[i], rR[i], p2fma(qI[i], rI[i], dre));
      dim = p2fma(qR[i], rI[i], p2fma(qI[i], p2neg(rR[i]), dim));
      dqq = p2fma(qR[i], qR[i], p2fma(qI[i], qI[i], dqq));
    }
    float2 v0 = p2split(dre), v1 = p2split(dim), v2 = p2split(dqq);
    float red6[6] = {v0.x, v1.x, v2.x, v0.y, v1.y, v2.y};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int j = 0; j < 6; ++j) red6[j] += __shfl_down_sync(0xffffffffu, red6[j], o);
    if ((ls & 31) == 0) {
#pragma unroll
      for (int j = 0; j < 6; ++j) red[j * NW + (ls >> 5)] = red6[j];
    }
    __syncthreads();
    float sums[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      float a = 0.f;
#pragma unroll
      for (int w = 0; w < NW; ++w) a += red[j * NW + w];
      sums[j] = a;
    }
    const float2 al0 = sums[2] > 1e-30f ? make_float2(sums[0] / sums[2], sums[1] / sums[2]) : make_float2(0.f, 0.f);
    const float2 al1 = sums[5] > 1e-30f ? make_float2(sums[3] / sums[5], sums[4] / sums[5]) : make_float2(0.f, 0.f);
    const P2 aR = p2(al0.x, al1.x), aI = p2(al0.y, al1.y);
    const P2 naR = p2(-al0.x, -al1.x), naI = p2(-al0.y, -al1.y);
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      // e += al rh (cfma), then rh = rh - al q (cfma with -al)
      eR[i] = p2fma(naI, rI[i], p2fma(aR, rR[i], eR[i]));
      eI[i] = p2fma(aI, rR[i], p2fma(aR, rI[i], eI[i]));
      const P2 nr = p2fma(aI, qI[i], p2fma(naR, qR[i], rR[i]));
      const P2 ni = p2fma(naI, qR[i], p2fma(naR, qI[i], rI[i]));
      rR[i] = nr;
      rI[i] = ni;
      rho[i * S + ls] = make_ulonglong2(rR[i].v, rI[i].v);
    }
    __syncthreads();
  }
  // unpack: lane 0 -> right-hand side r0, lane 1 -> r0 + 1
  float2 e0[12], e1[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    const float2 er = p2split(eR[i]), ei = p2split(eI[i]);
    const float2 rr_ = p2split(rR[i]), ri = p2split(rI[i]);
    e0[i] = make_float2(er.x, ei.x);
    e1[i] = make_float2(er.y, ei.y);
    rh0[i] = make_float2(rr_.x, ri.x);
    rh1[i] = make_float2(rr_.y, ri.y);
  }
  {
    float2 zz[12];
    load_fine_site<float>(z + r0 * n, s, V, zz);
#pragma unroll
    for (int i = 0; i < 12; ++i) zz[i] = cadd(zz[i], e0[i]);
    store_fine_site<float>(z + r0 * n, s, V, zz);
    store_fine_site<float>(e_out + r0 * n, s, V, e0);
    store_fine_site<float>(r + r0 * n, s, V, rh0);
  }
  if (live1) {
    float2 zz[12];
    load_fine_site<float>(z + (r0 + 1) * n, s, V, zz);
#pragma unroll
    for (int i = 0; i < 12; ++i) zz[i] = cadd(zz[i], e1[i]);
    store_fine_site<float>(z + (r0 + 1) * n, s, V, zz);
    store_fine_site<float>(e_out + (r0 + 1) * n, s, V, e1);
    store_fine_site<float>(r + (r0 + 1) * n, s, V, rh1);
  }
}

// One colour of one SAP sweep.  r: residual (in/out), z: solution (+= e),
// e: correction of this colour (written for the face update of the other
// colour's sites).
// RS right-hand sides per CTA (RS = 2 needs blocks of a multiple of 32
// sites): the block's links are staged once for all of them, each slot of
// `sites` threads iterates on its own right-hand side.  FP32 with RS = 1:
// two CTAs per SM (98 KB of shared memory each); RS = 2: one of 512 threads
// (123 KB); FP64 (196 KB) fits one, so it takes the whole register file.
template <typename T, int RS>
__global__ void __launch_bounds__(256 * RS, (sizeof(T) == 4 && RS == 1) ? 2 : 1)
    sap_block_kernel(C<T> *__restrict__ r, C<T> *__restrict__ z, C<T> *e_out, const C<T> *__restrict__ U,
                     SapGeom sg, T diag, int color, int iters, int nrhs) {
  extern __shared__ unsigned char smem_raw[];
  const int sites = sg.sites;
  const int slot = RS == 1 ? 0 : (int)threadIdx.x / sites;
  const int ls = (int)threadIdx.x - slot * sites;
  C<T> *Us = reinterpret_cast<C<T> *>(smem_raw);     // [4][9][sites]
  C<T> *rho = Us + sites * 36 + slot * sites * 12;    // [slot][12][sites]
  T *red = reinterpret_cast<T *>(Us + sites * 36 + RS * sites * 12) + slot * 100;  // per slot
  T *out3 = red + 96;
  const int64_t n = sg.g.n();
  // the right-hand-side group varies fastest over the grid: the CTAs of one
  // block run together and read its links from L2 after the first of them
  const int ngr = (nrhs + RS - 1) / RS;
  const int rq = (int)(blockIdx.x % (unsigned)ngr) * RS + slot;
  const bool live = rq < nrhs;  // a slot past the last right-hand side computes on zeros
  const int rr = live ? rq : nrhs - 1;
  C<T> *rv = r + rr * n;
  C<T> *zv = z + rr * n;
  C<T> *ev = e_out + rr * n;
  int bc[4];
  active_block(sg, (int)(blockIdx.x / (unsigned)ngr), color, bc);
  int lc[4];
  {
    int t = ls;
    lc[0] = t % sg.b[0]; t /= sg.b[0];
    lc[1] = t % sg.b[1]; t /= sg.b[1];
    lc[2] = t % sg.b[2];
    lc[3] = t / sg.b[2];
  }
  int gc[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) gc[i] = bc[i] * sg.b[i] + lc[i];
  const int s = sg.g.index(gc);
  // stage links (once for all slots) and the residual of the block
  const int64_t V = sg.g.V;
  for (int i = slot; i < 36; i += RS) Us[i * sites + ls] = kSoa<T> ? U[(int64_t)i * V + s] : U[(int64_t)s * 36 + i];
  C<T> rh[12];  // this site's residual, kept in registers (its slot in rho is for the neighbours)
  {
    if (live) {
      load_fine_site<T>(rv, s, V, rh);
    } else {
#pragma unroll
      for (int i = 0; i < 12; ++i) rh[i] = mk<T>((T)0, (T)0);
    }
#pragma unroll
    for (int i = 0; i < 12; ++i) rho[i * sites + ls] = rh[i];
  }
  C<T> e[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) e[i] = mk<T>((T)0, (T)0);
  __syncthreads();
  for (int it = 0; it < iters; ++it) {
    C<T> q[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) q[i] = cscale(rh[i], diag);
    local_hops<T, 0>(rho, Us, lc, sg.b, ls, sites, q);
    local_hops<T, 1>(rho, Us, lc, sg.b, ls, sites, q);
    local_hops<T, 2>(rho, Us, lc, sg.b, ls, sites, q);
    local_hops<T, 3>(rho, Us, lc, sg.b, ls, sites, q);
    T qr_re = 0, qr_im = 0, qq = 0;
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      const C<T> p = rh[i];
      qr_re = fma(q[i].x, p.x, fma(q[i].y, p.y, qr_re));
      qr_im = fma(q[i].x, p.y, fma(-q[i].y, p.x, qr_im));
      qq = fma(q[i].x, q[i].x, fma(q[i].y, q[i].y, qq));
    }
    if (RS == 1) block_reduce3<T>(qr_re, qr_im, qq, red, out3);
    else slot_reduce3<T>(qr_re, qr_im, qq, red, out3, ls, sites >> 5);
    const T den = out3[2];
    const T tiny = sizeof(T) == 4 ? (T)1e-30 : (T)1e-280;
    const C<T> al = den > tiny ? mk<T>(out3[0] / den, out3[1] / den) : mk<T>((T)0, (T)0);
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      const C<T> p = rh[i];
      e[i] = cfma(al, p, e[i]);
      rh[i] = cfma(cneg(al), q[i], p);
      rho[i * sites + ls] = rh[i];
    }
    __syncthreads();
  }
  if (!live) return;
  {
    C<T> zz[12];
    load_fine_site<T>(zv, s, V, zz);
#pragma unroll
    for (int i = 0; i < 12; ++i) zz[i] = cadd(zz[i], e[i]);
    store_fine_site<T>(zv, s, V, zz);
  }
  store_fine_site<T>(ev, s, V, e);
  store_fine_site<T>(rv, s, V, rh);
}

// The boundary pass over the sites of the blocks of colour `color` only
// (whole warps of one colour, instead of half the lanes of every warp idle),
// one load set per direction where the block extent allows it; the same sum
// as sap_boundary_kernel.  Right-hand side fastest over the grid.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1) sap_face_kernel(C<T> *__restrict__ r, const C<T> *__restrict__ e,
                                                       const C<T> *__restrict__ U, SapGeom sg, int color,
                                                       int nrhs) {
  const int rr = (int)(blockIdx.x % (unsigned)nrhs);
  const int64_t q = (int64_t)(blockIdx.x / (unsigned)nrhs) * blockDim.x + threadIdx.x;
  if (q >= sg.g.V / 2) return;
  const int bi = (int)(q / sg.sites), ls = (int)(q - (int64_t)bi * sg.sites);
  int bc[4];
  active_block(sg, bi, color, bc);
  int lc[4];
  {
    int t = ls;
    lc[0] = t % sg.b[0]; t /= sg.b[0];
    lc[1] = t % sg.b[1]; t /= sg.b[1];
    lc[2] = t % sg.b[2];
    lc[3] = t / sg.b[2];
  }
  int c[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) c[i] = bc[i] * sg.b[i] + lc[i];
  const int s = sg.g.index(c);
  const int64_t n = sg.g.n();
  const C<T> *ev = e + rr * n;
  C<T> *rv = r + rr * n;
  C<T> acc[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) acc[i] = mk<T>((T)0, (T)0);
  cross_dir<0, T>(ev, U, sg, s, c, lc[0], acc, (T)1);
  cross_dir<1, T>(ev, U, sg, s, c, lc[1], acc, (T)1);
  cross_dir<2, T>(ev, U, sg, s, c, lc[2], acc, (T)1);
  cross_dir<3, T>(ev, U, sg, s, c, lc[3], acc, (T)1);
  C<T> res[12];
  load_fine_site<T>(rv, s, sg.g.V, res);
#pragma unroll
  for (int i = 0; i < 12; ++i) res[i] = csub(res[i], acc[i]);
  store_fine_site<T>(rv, s, sg.g.V, res);
}

template <int B0, int B1, int B2, int B3>
void launch_pair(float2 *r, float2 *z, float2 *e, const float2 *U, const SapGeom &sg, float diag, int color,
                 int iters, int nrhs, unsigned grid, cudaStream_t st) {
  constexpr int S = B0 * B1 * B2 * B3;
  const int sm = 48 * S * 16 + 6 * (S / 32) * 4;
  smem_optin((const void *)sap_block_pair_kernel<B0, B1, B2, B3>, sm);
  sap_block_pair_kernel<B0, B1, B2, B3><<<grid, S, sm, st>>>(r, z, e, U, sg, diag, color, iters, nrhs);
}

template <int B0, int B1, int B2, int B3>
void launch_staged(float2 *r, float2 *z, float2 *e, const float2 *U, const SapGeom &sg, float diag, int color,
                   int iters, int nrhs, unsigned grid, cudaStream_t st) {
  constexpr int S = B0 * B1 * B2 * B3;
  const int sm = 36 * S * 8 + 4 * 6 * S * 16 + 2 * 3 * (S / 32) * 4;
  smem_optin((const void *)sap_block_staged_kernel<B0, B1, B2, B3>, sm);
  sap_block_staged_kernel<B0, B1, B2, B3><<<grid, 2 * S, sm, st>>>(r, z, e, U, sg, diag, color, iters, nrhs);
}

}  // namespace

int sap_variants() { return 3; }

bool sap_feasible(const Geom &g, const int b[4]) {
  int sites = 1;
  for (int i = 0; i < 4; ++i) {
    if (b[i] < 1 || g.L[i] % b[i]) return false;
    if ((g.L[i] / b[i]) % 2) return false;
    sites *= b[i];
  }
  return sites <= 256 && sites >= 2;
}

template <typename T>
size_t sap_smem_bytes(const int b[4], int rs) {
  const int sites = b[0] * b[1] * b[2] * b[3];
  return (size_t)sites * (36 + 12 * rs) * sizeof(C<T>) + (size_t)rs * 100 * sizeof(T);
}

template <typename T>
void sap_sweep(C<T> *r, C<T> *z, C<T> *e, const C<T> *U, Geom g, const int b[4], double m0,
               int block_iters, int nrhs, cudaStream_t s, int variant) {
  SapGeom sg;
  sg.g = g;
  sg.sites = 1;
  int nblocks = 1;
  for (int i = 0; i < 4; ++i) {
    sg.b[i] = b[i];
    sg.nb[i] = g.L[i] / b[i];
    sg.sites *= b[i];
    nblocks *= sg.nb[i];
  }
  // two right-hand sides per CTA share the block's staged links where the
  // shared memory allows it (FP32, whole warps per right-hand side)
  const bool two = sizeof(T) == 4 && nrhs >= 2 && sg.sites % 32 == 0 && sg.sites <= 256;
  const int rs = two ? 2 : 1;
  const size_t sm = sap_smem_bytes<T>(b, rs);
  if (sm > 220 * 1024) throw Error(1, "SAP block too large for shared memory");
  const unsigned grid = (unsigned)(nblocks / 2) * (unsigned)((nrhs + rs - 1) / rs);
  const float dg = (float)(4.0 + m0);
  bool b8 = false, b4 = false;
  if constexpr (sizeof(T) == 4) {
    b8 = two && b[0] == 8 && b[1] == 4 && b[2] == 4 && b[3] == 2;
    b4 = two && b[0] == 4 && b[1] == 4 && b[2] == 4 && b[3] == 4;
  }
  // red blocks; the black sites take the red corrections across their
  // faces; black blocks; the red sites take the black corrections (r exact
  // again).  The face updates run over one colour's sites at a time in their
  // own kernel, where many resident warps hide the latency of the gathers.
  for (int color = 0; color < 2; ++color) {
    if (color == 1) {
      sap_face_kernel<T><<<(unsigned)div_up(g.V / 2, 256) * (unsigned)nrhs, 256, 0, s>>>(r, e, U, sg, 1, nrhs);
      MG_LAUNCH_CHECK();
    }
    if constexpr (sizeof(T) == 4) {
      if (variant == 0 && b8) launch_staged<8, 4, 4, 2>(r, z, e, U, sg, dg, color, block_iters, nrhs, grid, s);
      else if (variant == 0 && b4) launch_staged<4, 4, 4, 4>(r, z, e, U, sg, dg, color, block_iters, nrhs, grid, s);
      else if (variant == 1 && b8) launch_pair<8, 4, 4, 2>(r, z, e, U, sg, dg, color, block_iters, nrhs, grid, s);
      else if (variant == 1 && b4) launch_pair<4, 4, 4, 4>(r, z, e, U, sg, dg, color, block_iters, nrhs, grid, s);
      else if (two) {
        smem_optin((const void *)sap_block_kernel<T, 2>, (int)sm);
        sap_block_kernel<T, 2><<<grid, 2 * sg.sites, sm, s>>>(r, z, e, U, sg, (T)dg, color, block_iters, nrhs);
      } else {
        smem_optin((const void *)sap_block_kernel<T, 1>, (int)sm);
        sap_block_kernel<T, 1><<<grid, sg.sites, sm, s>>>(r, z, e, U, sg, (T)dg, color, block_iters, nrhs);
      }
    } else {
      smem_optin((const void *)sap_block_kernel<T, 1>, (int)sm);
      sap_block_kernel<T, 1><<<grid, sg.sites, sm, s>>>(r, z, e, U, sg, (T)(4.0 + m0), color, block_iters, nrhs);
    }
    MG_LAUNCH_CHECK();
  }
  sap_face_kernel<T><<<(unsigned)div_up(g.V / 2, 256) * (unsigned)nrhs, 256, 0, s>>>(r, e, U, sg, 0, nrhs);
  MG_LAUNCH_CHECK();
}

template void sap_sweep<double>(C<double> *, C<double> *, C<double> *, const C<double> *, Geom,
                                const int *, double, int, int, cudaStream_t, int);
template void sap_sweep<float>(C<float> *, C<float> *, C<float> *, const C<float> *, Geom,
                               const int *, double, int, int, cudaStream_t, int);
template size_t sap_smem_bytes<double>(const int *, int);
template size_t sap_smem_bytes<float>(const int *, int);

}  // namespace mg
