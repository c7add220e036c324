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
// sweep.  That last update is done for the black sites by the black blocks
// themselves as they stage their residual (the red corrections across their
// faces enter before their iterations start), and for the red sites by one
// boundary pass after the black blocks: three launches per sweep.
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

// One colour of one SAP sweep.  r: residual (in/out), z: solution (+= e),
// e: correction of this colour (written for the boundary update).  With
// fuse_in the block's residual first takes the hops of the other colour's
// corrections across its faces (the boundary update of the previous pass,
// done here on the block's own sites instead of by a separate kernel).
// RS right-hand sides per CTA (RS = 2 needs blocks of a multiple of 32
// sites): the block's links are staged once for all of them, each slot of
// `sites` threads iterates on its own right-hand side.  FP32 with RS = 1:
// two CTAs per SM (98 KB of shared memory each); RS = 2: one of 512 threads
// (123 KB); FP64 (196 KB) fits one, so it takes the whole register file.
template <typename T, int RS>
__global__ void __launch_bounds__(256 * RS, (sizeof(T) == 4 && RS == 1) ? 2 : 1)
    sap_block_kernel(C<T> *__restrict__ r, C<T> *__restrict__ z, C<T> *e_out, const C<T> *__restrict__ U,
                     SapGeom sg, T diag, int color, int iters, int nrhs, int fuse_in) {
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
    if (fuse_in && live) {
      // the other colour's blocks are the face neighbours: their fresh
      // corrections e enter this block's residual, r -= hops of e
      cross_pair<0, T>(ev, U, sg, s, gc, rh, (T)-1);
      cross_pair<1, T>(ev, U, sg, s, gc, rh, (T)-1);
      cross_pair<2, T>(ev, U, sg, s, gc, rh, (T)-1);
      cross_pair<3, T>(ev, U, sg, s, gc, rh, (T)-1);
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

template <typename T>
__global__ void sap_boundary_kernel(C<T> *__restrict__ r, const C<T> *__restrict__ e,
                                    const C<T> *__restrict__ U, SapGeom sg, int color, int nrhs) {
  // right-hand side fastest over the grid: the CTAs of one site range share
  // its links through L2
  const int rr = (int)(blockIdx.x % (unsigned)nrhs);
  const int s = (int)(blockIdx.x / (unsigned)nrhs) * blockDim.x + threadIdx.x;
  if (s >= sg.g.V) return;
  int c[4];
  sg.g.coords(s, c);
  const int par = (c[0] / sg.b[0] + c[1] / sg.b[1] + c[2] / sg.b[2] + c[3] / sg.b[3]) & 1;
  if (par == color) return;  // residual of active blocks was written by the block kernel
  const int64_t n = sg.g.n();
  const C<T> *ev = e + rr * n;
  C<T> *rv = r + rr * n;
  C<T> acc[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) acc[i] = mk<T>((T)0, (T)0);
  cross_pair<0, T>(ev, U, sg, s, c, acc);
  cross_pair<1, T>(ev, U, sg, s, c, acc);
  cross_pair<2, T>(ev, U, sg, s, c, acc);
  cross_pair<3, T>(ev, U, sg, s, c, acc);
  C<T> res[12];
  load_fine_site<T>(rv, s, sg.g.V, res);
#pragma unroll
  for (int i = 0; i < 12; ++i) res[i] = csub(res[i], acc[i]);
  store_fine_site<T>(rv, s, sg.g.V, res);
}

}  // namespace

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
               int block_iters, int nrhs, cudaStream_t s) {
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
  // red blocks; black blocks, which first take the red corrections across
  // their faces; then the red sites take the black corrections (r exact again)
  for (int color = 0; color < 2; ++color) {
    if constexpr (sizeof(T) == 4) {
      if (two) {
        smem_optin((const void *)sap_block_kernel<T, 2>, (int)sm);
        sap_block_kernel<T, 2><<<grid, 2 * sg.sites, sm, s>>>(r, z, e, U, sg, (T)(4.0 + m0), color,
                                                              block_iters, nrhs, color);
        MG_LAUNCH_CHECK();
        continue;
      }
    }
    {
      smem_optin((const void *)sap_block_kernel<T, 1>, (int)sm);
      sap_block_kernel<T, 1><<<grid, sg.sites, sm, s>>>(r, z, e, U, sg, (T)(4.0 + m0), color, block_iters,
                                                        nrhs, color);
    }
    MG_LAUNCH_CHECK();
  }
  sap_boundary_kernel<T><<<(unsigned)div_up(g.V, 128) * (unsigned)nrhs, 128, 0, s>>>(r, e, U, sg, 1, nrhs);
  MG_LAUNCH_CHECK();
}

template void sap_sweep<double>(C<double> *, C<double> *, C<double> *, const C<double> *, Geom,
                                const int *, double, int, int, cudaStream_t);
template void sap_sweep<float>(C<float> *, C<float> *, C<float> *, const C<float> *, Geom,
                               const int *, double, int, int, cudaStream_t);
template size_t sap_smem_bytes<double>(const int *, int);
template size_t sap_smem_bytes<float>(const int *, int);

}  // namespace mg
