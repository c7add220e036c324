// Coarse-level kernels: the Galerkin stencil D_{l+1} = P_l^H D_l P_l (Sec.
// 2.2) stored as 9 dense (2 N_tv)^2 blocks per coarse site, the transfer
// operators P_l / P_l^H built per aggregate and chirality, the Galerkin
// construction, and the dense coarsest-level inverse.
#include "kernels.h"

#include <cuda_bf16.h>

#include <mutex>

namespace mg {

namespace {

inline int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

template <typename V> __device__ __forceinline__ V warp_csum(V v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// y(X) = sum_d A[X][d] x(nbr(X, d)) with the blocks stored transposed,
// AT[X][d][j][i], so that the m threads of one direction read a block column
// with one coalesced access.  Block = (m, 9) threads: thread (i, d) forms row
// i of direction d for RG right-hand sides at a time from the neighbour
// vectors staged in shared memory; the 9 partial rows are then summed in
// shared memory by the d = 0 threads.  Each block entry is read once per RG
// right-hand sides.
template <typename T, int RG>
__global__ void stencil_t_kernel(const C<T> *__restrict__ in, C<T> *__restrict__ out,
                                 const C<T> *__restrict__ AT, Geom g, int nrhs) {
  extern __shared__ unsigned char smem_raw[];
  const int m = g.dof;
  C<T> *xs = reinterpret_cast<C<T> *>(smem_raw);  // [9][RG][m]
  C<T> *part = xs + 9 * RG * m;                   // [9][RG][m]
  const int X = blockIdx.x;
  const int i = threadIdx.x, d = threadIdx.y;
  const int64_t n = g.n();
  const int nb = g.neighbor(X, d);
  const C<T> *Ad = AT + ((int64_t)X * 9 + d) * m * m;
  for (int r0 = 0; r0 < nrhs; r0 += RG) {
    const int rg = nrhs - r0 < RG ? nrhs - r0 : RG;
#pragma unroll
    for (int r = 0; r < RG; ++r)
      if (r < rg) xs[(d * RG + r) * m + i] = in[(int64_t)(r0 + r) * n + (int64_t)nb * m + i];
    __syncthreads();
    C<T> acc[RG];
#pragma unroll
    for (int r = 0; r < RG; ++r) acc[r] = mk<T>((T)0, (T)0);
    const C<T> *xd = xs + d * RG * m;
#pragma unroll 4
    for (int j = 0; j < m; ++j) {
      const C<T> a = __ldg(Ad + (int64_t)j * m + i);
#pragma unroll
      for (int r = 0; r < RG; ++r) acc[r] = cfma(a, xd[r * m + j], acc[r]);
    }
#pragma unroll
    for (int r = 0; r < RG; ++r) part[(d * RG + r) * m + i] = acc[r];
    __syncthreads();
    if (d == 0) {
      for (int r = 0; r < rg; ++r) {
        C<T> v = part[r * m + i];
#pragma unroll
        for (int dd = 1; dd < 9; ++dd) v = cadd(v, part[(dd * RG + r) * m + i]);
        out[(int64_t)(r0 + r) * n + (int64_t)X * m + i] = v;
      }
    }
    __syncthreads();
  }
}

// Wide coarse operators (m > 64 dofs per site, e.g. 2 N_tv = 100, 128, 256):
// one CTA of 8 warps per (site, 32-row tile).  Lane l owns row i0 + l, so
// the reads of AT[X][d][j][i0..i0+31] are 32 consecutive entries; warp w
// takes the columns j = w, w + 8, ... of every direction.  The neighbour
// vectors of the 9 directions for RG right-hand sides are staged in shared
// memory; the 8 warp partials of a row are added in warp order.
template <typename T, int RG>
__global__ void __launch_bounds__(256) stencil_wide_kernel(const C<T> *__restrict__ in,
                                                           C<T> *__restrict__ out,
                                                           const C<T> *__restrict__ AT, Geom g,
                                                           int nrhs) {
  extern __shared__ unsigned char smem_raw[];
  const int m = g.dof;
  C<T> *xs = reinterpret_cast<C<T> *>(smem_raw);  // [9][RG][m]
  C<T> *part = xs + 9 * RG * m;                   // [8 warps][RG][32]
  const int X = blockIdx.x, i0 = blockIdx.y * 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = i0 + lane;
  const bool row_ok = i < m;
  const int64_t n = g.n();
  for (int r0 = 0; r0 < nrhs; r0 += RG) {
    const int rg = nrhs - r0 < RG ? nrhs - r0 : RG;
    __syncthreads();
    for (int e = threadIdx.x; e < 9 * RG * m; e += blockDim.x) {
      const int d = e / (RG * m), rem = e - d * RG * m, r = rem / m, j = rem - r * m;
      xs[e] = r < rg ? in[(int64_t)(r0 + r) * n + (int64_t)g.neighbor(X, d) * m + j] : mk<T>((T)0, (T)0);
    }
    __syncthreads();
    C<T> acc[RG];
#pragma unroll
    for (int r = 0; r < RG; ++r) acc[r] = mk<T>((T)0, (T)0);
    if (row_ok) {
      for (int d = 0; d < 9; ++d) {
        const C<T> *Ad = AT + ((int64_t)X * 9 + d) * m * m;
        const C<T> *xd = xs + d * RG * m;
        for (int j = w; j < m; j += 8) {
          const C<T> a = __ldg(Ad + (int64_t)j * m + i);
#pragma unroll
          for (int r = 0; r < RG; ++r) acc[r] = cfma(a, xd[r * m + j], acc[r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < RG; ++r) part[(w * RG + r) * 32 + lane] = acc[r];
    __syncthreads();
    if (w == 0 && row_ok) {
      for (int r = 0; r < rg; ++r) {
        C<T> v = part[r * 32 + lane];
#pragma unroll
        for (int ww = 1; ww < 8; ++ww) v = cadd(v, part[(ww * RG + r) * 32 + lane]);
        out[(int64_t)(r0 + r) * n + (int64_t)X * m + i] = v;
      }
    }
  }
}

template <typename T, int RG>
void launch_wide(const C<T> *in, C<T> *out, const C<T> *AT, Geom g, int nrhs, cudaStream_t s) {
  const int m = g.dof;
  const size_t sm = (size_t)(9 * RG * m + 8 * RG * 32) * sizeof(C<T>);
  smem_optin((const void *)stencil_wide_kernel<T, RG>, 200 * 1024);
  if (sm > 200 * 1024) throw Error(1, "coarse stencil: too many dofs per site");
  stencil_wide_kernel<T, RG><<<dim3(g.V, (m + 31) / 32), 256, sm, s>>>(in, out, AT, g, nrhs);
  MG_LAUNCH_CHECK();
}

// ---- TMA bulk staging (cp.async.bulk + mbarrier) --------------------------
__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *mbar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes)
               : "memory");
}
// one bulk copy global -> this CTA's shared memory; 16-byte aligned
// addresses and a byte count that is a multiple of 16
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(mbar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(mbar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: false (and *err set) if the copy did not land in time
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *mbar, unsigned parity, int *err) {
  const unsigned long long t0 = global_ns();
  for (int it = 0; it < (1 << 26); ++it) {
    if (mbar_try_wait(mbar, parity)) return true;
    if ((it & 63) == 63 && global_ns() - t0 > kWaitNs) break;
  }
  if (err) atomicExch(err, 2);
  return false;
}

// Same contraction as stencil_t_kernel, with the site's 9 transposed blocks
// (9 m^2 complex, contiguous) brought into shared memory by one TMA bulk copy
// issued by thread 0 while the others stage the neighbour vectors; every
// block entry is then read from shared memory for all right-hand sides.
template <typename T, int RG>
__global__ void stencil_tma_kernel(const C<T> *__restrict__ in, C<T> *__restrict__ out,
                                   const C<T> *__restrict__ AT, Geom g, int nrhs, int *err,
                                   unsigned extra_tx) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar;
  const int m = g.dof;
  C<T> *As = reinterpret_cast<C<T> *>(smem_raw);  // [9][j][i]
  C<T> *xs = As + 9 * m * m;                        // [9][RG][m]
  C<T> *part = xs + 9 * RG * m;                     // [9][RG][m]
  const int X = blockIdx.x;
  const int i = threadIdx.x, d = threadIdx.y;
  const int tid = d * blockDim.x + i;
  const int64_t n = g.n();
  const unsigned bytes = (unsigned)(9u * m * m * sizeof(C<T>));
  if (tid == 0) mbar_init(&mbar, 1);
  __syncthreads();
  if (tid == 0) {
    mbar_expect_tx(&mbar, bytes + extra_tx);  // extra_tx = 0 but in failure-injection tests
    bulk_g2s(As, AT + (int64_t)X * 9 * m * m, bytes, &mbar);
  }
  const int nb = g.neighbor(X, d);
  bool ready = false;
  for (int r0 = 0; r0 < nrhs; r0 += RG) {
    const int rg = nrhs - r0 < RG ? nrhs - r0 : RG;
#pragma unroll
    for (int r = 0; r < RG; ++r)
      if (r < rg) xs[(d * RG + r) * m + i] = in[(int64_t)(r0 + r) * n + (int64_t)nb * m + i];
    if (!ready) {
      ready = mbar_wait_bounded(&mbar, 0, err);
      // the whole block gives up together (no thread may be left at a
      // barrier); a copy still in flight gets a second bounded wait first
      if (__syncthreads_or(ready ? 0 : 1)) {
        if (!ready) mbar_wait_bounded(&mbar, 0, nullptr);
        return;
      }
    }
    __syncthreads();
    C<T> acc[RG];
#pragma unroll
    for (int r = 0; r < RG; ++r) acc[r] = mk<T>((T)0, (T)0);
    const C<T> *xd = xs + d * RG * m;
    const C<T> *Ad = As + d * m * m;
#pragma unroll 4
    for (int j = 0; j < m; ++j) {
      const C<T> a = Ad[j * m + i];
#pragma unroll
      for (int r = 0; r < RG; ++r) acc[r] = cfma(a, xd[r * m + j], acc[r]);
    }
#pragma unroll
    for (int r = 0; r < RG; ++r) part[(d * RG + r) * m + i] = acc[r];
    __syncthreads();
    if (d == 0) {
      for (int r = 0; r < rg; ++r) {
        C<T> v = part[r * m + i];
#pragma unroll
        for (int dd = 1; dd < 9; ++dd) v = cadd(v, part[(dd * RG + r) * m + i]);
        out[(int64_t)(r0 + r) * n + (int64_t)X * m + i] = v;
      }
    }
    __syncthreads();
  }
}

// Pipelined form for few right-hand sides (nrhs <= RG): a persistent CTA
// walks over coarse sites X = blockIdx.x, + gridDim.x, ... with a two-stage
// ring of bulk copies, so the next site's 9 blocks stream in while the
// current one is multiplied (one site per CTA leaves the copy latency
// exposed when there is little arithmetic per block).  Thread (i, d) forms
// row i of direction d as in stencil_tma_kernel, in the same order, from
// blocks stored as S: float2 (FP32, identical results) or __nv_bfloat162
// (BF16 storage for the multigrid preconditioner: half the bytes, the
// products and sums in FP32).
__device__ __forceinline__ float2 ld_blk(const float2 *p) { return *p; }
__device__ __forceinline__ float2 ld_blk(const __nv_bfloat162 *p) { return __bfloat1622float2(*p); }

template <typename S, int RG>
__global__ void __launch_bounds__(32 * 9, 1) stencil_pipe_kernel(const float2 *__restrict__ in,
                                                                float2 *__restrict__ out,
                                                                const S *__restrict__ AT, Geom g, int nrhs,
                                                                int *err, unsigned extra_tx) {
  constexpr int m = 32;
  constexpr int TILE = 9 * m * m;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[2];
  S *As = reinterpret_cast<S *>(smem_raw);                         // [2][9][j][i]
  float2 *xs = reinterpret_cast<float2 *>(smem_raw + 2 * TILE * sizeof(S));  // [9][RG][m]
  float2 *part = xs + 9 * RG * m;                                  // [9][RG][m]
  const int i = threadIdx.x, d = threadIdx.y, tid = d * 32 + i;
  const int64_t n = g.n();
  const unsigned bytes = (unsigned)(TILE * sizeof(S));
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
  }
  __syncthreads();
  // the copies of the CTA's first two sites
  if (tid == 0) {
    for (int st = 0; st < 2; ++st) {
      const int X = blockIdx.x + st * gridDim.x;
      if (X < g.V) {
        mbar_expect_tx(&bar[st], bytes + extra_tx);  // extra_tx = 0 but in failure-injection tests
        bulk_g2s(As + st * TILE, AT + (int64_t)X * TILE, bytes, &bar[st]);
      }
    }
  }
  unsigned phase[2] = {0u, 0u};
  bool pending[2] = {blockIdx.x < (unsigned)g.V, blockIdx.x + gridDim.x < (unsigned)g.V};
  int k = 0;
  bool failed = false;
  // the neighbour values of the next site are loaded into registers while
  // the current one computes (one site ahead, like the block copies)
  float2 xn[RG];
  if ((int)blockIdx.x < g.V) {
    const int nb = g.neighbor(blockIdx.x, d);
#pragma unroll
    for (int r = 0; r < RG; ++r)
      xn[r] = r < nrhs ? __ldg(in + (int64_t)r * n + (int64_t)nb * m + i) : make_float2(0.f, 0.f);
  }
  for (int X = blockIdx.x; X < g.V; X += gridDim.x, ++k) {
    const int st = k & 1;
#pragma unroll
    for (int r = 0; r < RG; ++r) xs[(d * RG + r) * m + i] = xn[r];
    if (X + (int)gridDim.x < g.V) {
      const int nb = g.neighbor(X + (int)gridDim.x, d);
#pragma unroll
      for (int r = 0; r < RG; ++r)
        xn[r] = r < nrhs ? __ldg(in + (int64_t)r * n + (int64_t)nb * m + i) : make_float2(0.f, 0.f);
    }
    const bool ready = mbar_wait_bounded(&bar[st], phase[st], err);
    if (__syncthreads_or(ready ? 0 : 1)) {
      failed = true;
      break;
    }
    phase[st] ^= 1u;
    pending[st] = false;
    float2 acc[RG];
#pragma unroll
    for (int r = 0; r < RG; ++r) acc[r] = make_float2(0.f, 0.f);
    const float2 *xd = xs + d * RG * m;
    const S *Ad = As + st * TILE + d * m * m;
#pragma unroll 4
    for (int j = 0; j < m; ++j) {
      const float2 a = ld_blk(Ad + j * m + i);
#pragma unroll
      for (int r = 0; r < RG; ++r) acc[r] = cfma(a, xd[r * m + j], acc[r]);
    }
#pragma unroll
    for (int r = 0; r < RG; ++r) part[(d * RG + r) * m + i] = acc[r];
    __syncthreads();
    // every thread is done with this stage: refill it two sites ahead
    if (tid == 0) {
      const int Xn = X + 2 * (int)gridDim.x;
      if (Xn < g.V) {
        mbar_expect_tx(&bar[st], bytes + extra_tx);
        bulk_g2s(As + st * TILE, AT + (int64_t)Xn * TILE, bytes, &bar[st]);
      }
    }
    pending[st] = X + 2 * (int)gridDim.x < g.V;
    if (d == 0) {
      for (int r = 0; r < nrhs; ++r) {
        float2 v = part[r * m + i];
#pragma unroll
        for (int dd = 1; dd < 9; ++dd) v = cadd(v, part[(dd * RG + r) * m + i]);
        out[(int64_t)r * n + (int64_t)X * m + i] = v;
      }
    }
    __syncthreads();
  }
  if (failed && tid == 0) {
    // copies still in flight must land before the CTA leaves (bounded)
    for (int st = 0; st < 2; ++st)
      if (pending[st]) mbar_wait_bounded(&bar[st], phase[st], nullptr);
  }
}

// BF16 pairs of the transposed blocks (round to nearest)
__global__ void stencil_bf16_kernel(const float2 *__restrict__ AT32, __nv_bfloat162 *__restrict__ ATB,
                                    int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    ATB[e] = __float22bfloat162_rn(AT32[e]);
}


// ---- streaming BF16 coarse stencil for 32 dofs per site and up to 8
// right-hand sides: one warp per coarse site, lane i forming row i.
//
// The blocks are stored row-chunked, AS[X][d][c][i][q] = A(X, d)[i][4c + q]
// as BF16 pairs (real part in the low half), so lane i's four entries of a
// chunk are one 16-byte load and a warp's load is 512 contiguous bytes: the
// blocks stream from HBM straight into registers, with no shared-memory
// staging and no barrier.  A warp walks its items (site, direction) in
// order and loads item t + 1 (eight chunks and the neighbour's vector
// entries) while it computes item t.  The neighbour's 32 entries reach every
// lane through a per-warp shared-memory buffer (two buffers, one __syncwarp
// per item), packed as right-hand-side pairs (re_a, re_b, im_a, im_b) so
// that one broadcast load feeds four paired .f32x2 FMAs.
//
// Per direction each lane accumulates over j in order, from zero, with the
// same fused multiply-adds as cfma; the nine direction sums are added in
// direction order.  This is the order of stencil_pipe_kernel on the same
// BF16 values, so the two give identical results.
// neighbour of site X in direction d (Geom::neighbor without a local
// coordinate array: selects instead of a dynamically indexed one)
__device__ __forceinline__ int stream_neighbor(const Geom &g, int X, int d) {
  if (d == 0) return X;
  const int mu = (d - 1) >> 1;
  const int L0 = g.L[0], L1 = g.L[1], L2 = g.L[2], L3 = g.L[3];
  int s = X;
  const int x0 = s % L0;
  s /= L0;
  const int x1 = s % L1;
  s /= L1;
  const int x2 = s % L2, x3 = s / L2;
  const int c = mu == 0 ? x0 : mu == 1 ? x1 : mu == 2 ? x2 : x3;
  const int ext = mu == 0 ? L0 : mu == 1 ? L1 : mu == 2 ? L2 : L3;
  const int stride = mu == 0 ? 1 : mu == 1 ? L0 : mu == 2 ? L0 * L1 : L0 * L1 * L2;
  if (d & 1) return c + 1 == ext ? X - c * stride : X + stride;
  return c == 0 ? X + (ext - 1) * stride : X - stride;
}

template <int RP>
__device__ __forceinline__ void stream_load(const uint4 *__restrict__ AS, const float2 *__restrict__ in, int64_t n,
                                            const Geom &g, int X, int d, int nrhs, int lane, uint4 (&a)[8],
                                            float2 (&xv)[2 * RP]) {
  const uint4 *src = AS + ((int64_t)X * 9 + d) * 256 + lane;
#pragma unroll
  for (int c = 0; c < 8; ++c) a[c] = __ldg(src + c * 32);
  const int nb = stream_neighbor(g, X, d);
#pragma unroll
  for (int r = 0; r < 2 * RP; ++r)
    xv[r] = r < nrhs ? __ldg(in + (int64_t)r * n + (int64_t)nb * 32 + lane) : make_float2(0.f, 0.f);
}

// one item (site, direction) of a lane: row `lane` of the block, whose
// four-entry chunks are ac[c], times the neighbour's entries xs[j][rhs pair];
// per right-hand side the fused multiply-adds of cfma, over j in order, from
// zero
template <int RP>
__device__ __forceinline__ void stream_item(const uint4 (&ac)[8], const float4 *xs, P2 (&accR)[RP],
                                            P2 (&accI)[RP]) {
#pragma unroll
  for (int rp = 0; rp < RP; ++rp) accR[rp] = accI[rp] = p2(0.f, 0.f);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const unsigned wd[4] = {ac[c].x, ac[c].y, ac[c].z, ac[c].w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float ar = __uint_as_float(wd[q] << 16), ai = __uint_as_float(wd[q] & 0xffff0000u);
      const P2 AX = p2(ar, ar), NAY = p2(-ai, -ai), AY = p2(ai, ai);
      const float4 *xj = xs + (4 * c + q) * RP;
#pragma unroll
      for (int rp = 0; rp < RP; ++rp) {
        const float4 x4 = xj[rp];
        const P2 XR = p2(x4.x, x4.y), XI = p2(x4.z, x4.w);
        // cfma: re += ar xr, re += -ai xi; im += ar xi, im += ai xr
        accR[rp] = p2fma(AX, XR, accR[rp]);
        accR[rp] = p2fma(NAY, XI, accR[rp]);
        accI[rp] = p2fma(AX, XI, accI[rp]);
        accI[rp] = p2fma(AY, XR, accI[rp]);
      }
    }
  }
}

template <int RP>
__global__ void __launch_bounds__(256, 2) stencil_stream_kernel(const float2 *__restrict__ in,
                                                                float2 *__restrict__ out,
                                                                const uint4 *__restrict__ AS, Geom g, int nrhs) {
  __shared__ __align__(16) float4 xbuf[8][2][32 * RP];  // per warp: two buffers [j][rhs pair]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t n = g.n();
  const int gw = (int)blockIdx.x * 8 + w, nw = (int)gridDim.x * 8;
  const int nsites = gw < g.V ? (g.V - 1 - gw) / nw + 1 : 0;
  const int items = nsites * 9;
  if (items == 0) return;
  uint4 a[8];
  float2 xv[2 * RP];
  stream_load<RP>(AS, in, n, g, gw, 0, nrhs, lane, a, xv);
  P2 totR[RP], totI[RP];
#pragma unroll
  for (int rp = 0; rp < RP; ++rp) totR[rp] = totI[rp] = p2(0.f, 0.f);
  for (int t = 0; t < items; ++t) {
    const int d = t % 9;
    const int X = gw + (t / 9) * nw;
    float4 *xs = xbuf[w][t & 1];
#pragma unroll
    for (int rp = 0; rp < RP; ++rp)
      xs[lane * RP + rp] = make_float4(xv[2 * rp].x, xv[2 * rp + 1].x, xv[2 * rp].y, xv[2 * rp + 1].y);
    __syncwarp();
    uint4 ac[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) ac[c] = a[c];
    if (t + 1 < items) {
      const int t1 = t + 1;
      stream_load<RP>(AS, in, n, g, gw + (t1 / 9) * nw, t1 % 9, nrhs, lane, a, xv);
    }
    P2 accR[RP], accI[RP];
    stream_item<RP>(ac, xs, accR, accI);
#pragma unroll
    for (int rp = 0; rp < RP; ++rp) {
      totR[rp] = d == 0 ? accR[rp] : p2add(totR[rp], accR[rp]);
      totI[rp] = d == 0 ? accI[rp] : p2add(totI[rp], accI[rp]);
    }
    if (d == 8) {
#pragma unroll
      for (int rp = 0; rp < RP; ++rp) {
        const float2 re = p2split(totR[rp]), im = p2split(totI[rp]);
        if (2 * rp < nrhs) out[(int64_t)(2 * rp) * n + (int64_t)X * 32 + lane] = make_float2(re.x, im.x);
        if (2 * rp + 1 < nrhs) out[(int64_t)(2 * rp + 1) * n + (int64_t)X * 32 + lane] = make_float2(re.y, im.y);
      }
    }
  }
}

// The same items with one thread block per coarse site and one warp per
// direction (for coarse lattices with fewer sites than the walking kernel
// has warps): warp d forms direction d's partial rows, warp 0 adds the nine
// partials in direction order.  Identical results to stencil_stream_kernel.
template <int RP>
__global__ void __launch_bounds__(288) stencil_stream_site_kernel(const float2 *__restrict__ in,
                                                                 float2 *__restrict__ out,
                                                                 const uint4 *__restrict__ AS, Geom g,
                                                                 int nrhs) {
  __shared__ __align__(16) float4 xbuf[9][32 * RP];
  __shared__ __align__(16) float4 part[9][RP][32];  // (re_a, re_b, im_a, im_b) per lane
  const int lane = threadIdx.x & 31, d = threadIdx.x >> 5;
  const int X = blockIdx.x;
  const int64_t n = g.n();
  uint4 a[8];
  float2 xv[2 * RP];
  stream_load<RP>(AS, in, n, g, X, d, nrhs, lane, a, xv);
  float4 *xs = xbuf[d];
#pragma unroll
  for (int rp = 0; rp < RP; ++rp)
    xs[lane * RP + rp] = make_float4(xv[2 * rp].x, xv[2 * rp + 1].x, xv[2 * rp].y, xv[2 * rp + 1].y);
  __syncwarp();
  P2 accR[RP], accI[RP];
  stream_item<RP>(a, xs, accR, accI);
#pragma unroll
  for (int rp = 0; rp < RP; ++rp) {
    const float2 re = p2split(accR[rp]), im = p2split(accI[rp]);
    part[d][rp][lane] = make_float4(re.x, re.y, im.x, im.y);
  }
  __syncthreads();
  if (d != 0) return;
#pragma unroll
  for (int rp = 0; rp < RP; ++rp) {
    float4 v = part[0][rp][lane];
    P2 totR = p2(v.x, v.y), totI = p2(v.z, v.w);
#pragma unroll
    for (int dd = 1; dd < 9; ++dd) {
      v = part[dd][rp][lane];
      totR = p2add(totR, p2(v.x, v.y));
      totI = p2add(totI, p2(v.z, v.w));
    }
    const float2 re = p2split(totR), im = p2split(totI);
    if (2 * rp < nrhs) out[(int64_t)(2 * rp) * n + (int64_t)X * 32 + lane] = make_float2(re.x, im.x);
    if (2 * rp + 1 < nrhs) out[(int64_t)(2 * rp + 1) * n + (int64_t)X * 32 + lane] = make_float2(re.y, im.y);
  }
}

// AS[blk][c][i][q] = AT32[blk][4c + q][i] as a BF16 pair (round to nearest),
// blk = 9 X + d
__global__ void stencil_stream_layout_kernel(const float2 *__restrict__ AT32, __nv_bfloat162 *__restrict__ AS,
                                             int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t blk = e >> 10;
    const int w = (int)(e & 1023);
    const int q = w & 3, i = (w >> 2) & 31, c = w >> 7;
    AS[e] = __float22bfloat162_rn(AT32[(blk << 10) + (4 * c + q) * 32 + i]);
  }
}

template <typename S, int RG>
void launch_pipe(const float2 *in, float2 *out, const S *AT, Geom g, int nrhs, int *err, cudaStream_t s) {
  const size_t sm = (size_t)2 * 9 * 32 * 32 * sizeof(S) + (size_t)2 * 9 * RG * 32 * sizeof(float2);
  smem_optin((const void *)stencil_pipe_kernel<S, RG>, (int)sm);
  // as many CTAs as fit at once (shared memory bound: 1 per SM for FP32
  // blocks, 2 for BF16), each walking over its share of the sites
  const int per_sm = sm * 2 <= 220 * 1024 ? 2 : 1;
  const int grid = (int)std::min<int64_t>(g.V, (int64_t)sm_count() * per_sm);
  stencil_pipe_kernel<S, RG><<<grid, dim3(32, 9), sm, s>>>(in, out, AT, g, nrhs, err, staging_extra_bytes());
  MG_LAUNCH_CHECK();
}

// AT[X][d][j][i] = A[X][d][i][j], converted to the storage type To.
template <typename To>
__global__ void stencil_transpose_kernel(const double2 *__restrict__ A, C<To> *__restrict__ AT,
                                         int64_t nblocks, int m) {
  const int64_t total = nblocks * m * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t blk = e / ((int64_t)m * m);
    const int rem = (int)(e - blk * m * m);
    const int j = rem / m, i = rem - j * m;  // e indexes AT[blk][j][i]
    AT[e] = cvt<To>(A[blk * m * m + (int64_t)i * m + j]);
  }
}

// the 9 hop-class parts of a coarse stencil (Galerkin on the next level):
// out9[h] row i of X = sum over d of class h of A[X][d] x(nbr(X, d)).
template <typename T>
__global__ void stencil_split_kernel(const C<T> *__restrict__ in, C<T> *__restrict__ out9,
                                     const C<T> *__restrict__ A, Geom g, int b0, int b1, int b2,
                                     int b3) {
  const int X = blockIdx.x;
  const int m = g.dof;
  const int64_t n = g.n();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b[4] = {b0, b1, b2, b3};
  int c[4];
  g.coords(X, c);
  int cls[9], nb[9];
  cls[0] = 0;
  nb[0] = X;
  for (int d = 1; d < 9; ++d) {
    const int mu = (d - 1) >> 1;
    int cn[4] = {c[0], c[1], c[2], c[3]};
    if (d & 1) cn[mu] = (c[mu] + 1 == g.L[mu]) ? 0 : c[mu] + 1;
    else cn[mu] = (c[mu] == 0) ? g.L[mu] - 1 : c[mu] - 1;
    nb[d] = g.index(cn);
    cls[d] = (c[mu] / b[mu]) != (cn[mu] / b[mu]) ? d : 0;
  }
  const C<T> *AX = A + (int64_t)X * 9 * m * m;
  for (int i = warp; i < m; i += (blockDim.x >> 5)) {
    C<T> acc[9];
#pragma unroll
    for (int h = 0; h < 9; ++h) acc[h] = mk<T>((T)0, (T)0);
#pragma unroll
    for (int d = 0; d < 9; ++d) {
      const C<T> *Ar = AX + ((int64_t)d * m + i) * m;
      C<T> v = mk<T>((T)0, (T)0);
      for (int j = lane; j < m; j += 32) v = cfma(Ar[j], in[(int64_t)nb[d] * m + j], v);
      v = warp_csum(v);
      acc[cls[d]] = cadd(acc[cls[d]], v);
    }
    if (lane == 0) {
#pragma unroll
      for (int h = 0; h < 9; ++h) out9[h * n + (int64_t)X * m + i] = acc[h];
    }
  }
}

// ------------------------------------------------------------------ transfer
// out[r][X][c*ntv + k] = sum_row conj(P[X][c][k][row]) in_r[fine(X, c, row)]
// One block per (aggregate, chirality); RG right-hand sides are staged in
// shared memory per pass so each P entry is read once per RG of them.
// entries of P as stored: FP64 / FP32 complex, or BF16 pairs (FP32 arithmetic)
__device__ __forceinline__ double2 ldp(const double2 *p) { return __ldg(p); }
__device__ __forceinline__ float2 ldp(const float2 *p) { return __ldg(p); }
__device__ __forceinline__ float2 ldp(const __nv_bfloat162 *p) {
  const unsigned u = __ldg(reinterpret_cast<const unsigned *>(p));
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u));
}

template <typename T, int RG, typename PS = C<T>>
__global__ void restrict_kernel(const C<T> *__restrict__ in, C<T> *__restrict__ out,
                                const PS *__restrict__ P, AggMap m, int nrhs) {
  extern __shared__ unsigned char smem_raw[];
  C<T> *xs = reinterpret_cast<C<T> *>(smem_raw);  // [RG][rows]
  const int X = blockIdx.x >> 1, c = blockIdx.x & 1;
  const int64_t nf = m.fine.n(), nc = m.coarse.n();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const PS *PX = P + ((int64_t)(X * 2 + c) * m.ntv) * m.rows;
  for (int r0 = 0; r0 < nrhs; r0 += RG) {
    const int rg = nrhs - r0 < RG ? nrhs - r0 : RG;
    __syncthreads();
    for (int row = threadIdx.x; row < m.rows; row += blockDim.x) {
      const int64_t fi = m.fine_index(X, c, row);
#pragma unroll
      for (int r = 0; r < RG; ++r)
        if (r < rg) xs[r * m.rows + row] = in[(int64_t)(r0 + r) * nf + fi];
    }
    __syncthreads();
    for (int k = warp; k < m.ntv; k += nw) {
      const PS *Pk = PX + (int64_t)k * m.rows;
      C<T> acc[RG];
#pragma unroll
      for (int r = 0; r < RG; ++r) acc[r] = mk<T>((T)0, (T)0);
      // unrolled so that several rows' loads of P are in flight per lane
      // (the sums keep their order)
#pragma unroll 4
      for (int row = lane; row < m.rows; row += 32) {
        const C<T> a = ldp(Pk + row);
#pragma unroll
        for (int r = 0; r < RG; ++r) acc[r] = cfmac(a, xs[r * m.rows + row], acc[r]);
      }
#pragma unroll
      for (int r = 0; r < RG; ++r) {
        const C<T> v = warp_csum(acc[r]);
        if (lane == 0 && r < rg) out[(int64_t)(r0 + r) * nc + (int64_t)X * m.coarse.dof + c * m.ntv + k] = v;
      }
    }
  }
}

// out_r[fine(X, c, row)] = beta out + sum_k P[X][c][k][row] in_r[X][c*ntv + k]
// One block per (aggregate, chirality); each thread owns rows and applies the
// column segment of P to RG right-hand sides at a time.
template <typename T, int RG, typename PS = C<T>>
__global__ void prolong_kernel(const C<T> *__restrict__ in, C<T> *__restrict__ out,
                               const PS *__restrict__ P, AggMap m, int nrhs, T beta) {
  extern __shared__ unsigned char smem_raw[];
  C<T> *cs = reinterpret_cast<C<T> *>(smem_raw);  // [nrhs][ntv]
  const int X = blockIdx.x >> 1, c = blockIdx.x & 1;
  const int64_t nf = m.fine.n(), nc = m.coarse.n();
  for (int e = threadIdx.x; e < nrhs * m.ntv; e += blockDim.x) {
    const int r = e / m.ntv, k = e - r * m.ntv;
    cs[e] = in[(int64_t)r * nc + (int64_t)X * m.coarse.dof + c * m.ntv + k];
  }
  __syncthreads();
  const PS *PX = P + ((int64_t)(X * 2 + c) * m.ntv) * m.rows;
  for (int row = threadIdx.x; row < m.rows; row += blockDim.x) {
    const int64_t fi = m.fine_index(X, c, row);
    for (int r0 = 0; r0 < nrhs; r0 += RG) {
      const int rg = nrhs - r0 < RG ? nrhs - r0 : RG;
      C<T> acc[RG];
#pragma unroll
      for (int r = 0; r < RG; ++r) acc[r] = mk<T>((T)0, (T)0);
      // unrolled so that several test vectors' loads of P are in flight
      // (the sums keep their order)
#pragma unroll 4
      for (int k = 0; k < m.ntv; ++k) {
        const C<T> a = ldp(PX + (int64_t)k * m.rows + row);
#pragma unroll
        for (int r = 0; r < RG; ++r)
          if (r < rg) acc[r] = cfma(a, cs[(r0 + r) * m.ntv + k], acc[r]);
      }
#pragma unroll
      for (int r = 0; r < RG; ++r) {
        if (r < rg) {
          C<T> *o = out + (int64_t)(r0 + r) * nf + fi;
          *o = beta == (T)0 ? acc[r] : cadd(cscale(*o, beta), acc[r]);
        }
      }
    }
  }
}

__global__ void probe_kernel(double2 *__restrict__ out, const double2 *__restrict__ P, AggMap m,
                             int col) {
  const int cc = col / m.ntv, k = col - cc * m.ntv;
  const int64_t nf = m.fine.n();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nf;
       i += (int64_t)gridDim.x * blockDim.x) {
    int X, c, row;
    m.locate(i, X, c, row);
    out[i] = (c == cc) ? P[((int64_t)(X * 2 + c) * m.ntv + k) * m.rows + row] : make_double2(0.0, 0.0);
  }
}

__device__ __forceinline__ double2 block_csum(double2 v, double2 *sh) {
  v = warp_csum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 t = make_double2(0.0, 0.0);
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { t.x += sh[i].x; t.y += sh[i].y; }
    sh[32] = t;
  }
  __syncthreads();
  double2 r = sh[32];
  __syncthreads();
  return r;
}

// P[X][c][k][:] = MGS-orthonormalised (twice, in k order) restriction of the
// test vectors V[k] to aggregate X, chirality c.
__global__ void mgs_kernel(const double2 *__restrict__ V, double2 *__restrict__ P, AggMap m,
                           int *status) {
  __shared__ double2 sh[33];
  const int X = blockIdx.x >> 1, c = blockIdx.x & 1;
  const int64_t nf = m.fine.n();
  double2 *PX = P + ((int64_t)(X * 2 + c) * m.ntv) * m.rows;
  for (int k = 0; k < m.ntv; ++k) {
    double2 *w = PX + (int64_t)k * m.rows;
    for (int row = threadIdx.x; row < m.rows; row += blockDim.x)
      w[row] = V[k * nf + m.fine_index(X, c, row)];
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      for (int j = 0; j < k; ++j) {
        const double2 *q = PX + (int64_t)j * m.rows;
        double2 acc = make_double2(0.0, 0.0);
        for (int row = threadIdx.x; row < m.rows; row += blockDim.x) acc = cfmac(q[row], w[row], acc);
        const double2 h = block_csum(acc, sh);
        for (int row = threadIdx.x; row < m.rows; row += blockDim.x) w[row] = csub(w[row], cmul(h, q[row]));
        __syncthreads();
      }
    }
    double2 acc = make_double2(0.0, 0.0);
    for (int row = threadIdx.x; row < m.rows; row += blockDim.x) acc.x += cabs2(w[row]);
    const double nrm = sqrt(block_csum(acc, sh).x);
    if (!(nrm > 0.0) && threadIdx.x == 0) *status = 1;
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    for (int row = threadIdx.x; row < m.rows; row += blockDim.x) w[row] = cscale(w[row], inv);
    __syncthreads();
  }
}

__global__ void galerkin_scatter_kernel(const double2 *__restrict__ cols, double2 *__restrict__ A,
                                        Geom g, int col) {
  const int m = g.dof;
  const int64_t nc = g.n();
  const int64_t total = 9 * nc;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int h = (int)(e / nc);
    const int64_t rem = e - h * nc;
    const int X = (int)(rem / m), i = (int)(rem - (int64_t)X * m);
    A[(((int64_t)X * 9 + h) * m + i) * m + col] = cols[e];
  }
}

__global__ void p_canonical_kernel(const double2 *__restrict__ P, double2 *__restrict__ out, AggMap m) {
  const int64_t total = (int64_t)m.coarse.V * 2 * m.ntv * m.rows;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    // e over [X][c][row][k]
    const int k = (int)(e % m.ntv);
    const int64_t t = e / m.ntv;
    const int row = (int)(t % m.rows);
    const int64_t xc = t / m.rows;
    out[e] = P[(xc * m.ntv + k) * m.rows + row];
  }
}

// ------------------------------------------------------------------ dense
__global__ void dense_build_kernel(const double2 *__restrict__ A, double2 *__restrict__ M, Geom g) {
  const int m = g.dof;
  const int64_t n = g.n();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / n, col = e - row * n;
    const int X = (int)(row / m), i = (int)(row - (int64_t)X * m);
    const int Y = (int)(col / m), j = (int)(col - (int64_t)Y * m);
    double2 v = make_double2(0.0, 0.0);
    for (int d = 0; d < 9; ++d)
      if (g.neighbor(X, d) == Y) v = cadd(v, A[(((int64_t)X * 9 + d) * m + i) * m + j]);
    M[e] = v;
  }
}

__global__ void gj_pivot_kernel(const double2 *__restrict__ M, int n, int k, int *piv,
                                double2 *pivval, int *status) {
  __shared__ double bv[1024];
  __shared__ int bi[1024];
  double best = -1.0;
  int idx = k;
  for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
    const double a = cabs2(M[(int64_t)i * n + k]);
    if (a > best) { best = a; idx = i; }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = idx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double b2 = bv[threadIdx.x + o];
      const int i2 = bi[threadIdx.x + o];
      if (b2 > bv[threadIdx.x] || (b2 == bv[threadIdx.x] && i2 < bi[threadIdx.x])) {
        bv[threadIdx.x] = b2;
        bi[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *piv = bi[0];
    *pivval = M[(int64_t)bi[0] * n + k];
    if (!(bv[0] > 0.0)) *status = 1;
  }
}

// column k of M after the row swap k <-> piv, with f[k] = 0 (read only).
__global__ void gj_factor_kernel(const double2 *__restrict__ M, int n, int k, const int *piv,
                                 double2 *__restrict__ f) {
  const int p = *piv;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int src = (i == p) ? k : i;
    f[i] = (i == k) ? make_double2(0.0, 0.0) : M[(int64_t)src * n + k];
  }
}

// swap rows k and piv of M and Inv and divide row k by the pivot.
__global__ void gj_swap_kernel(double2 *__restrict__ M, double2 *__restrict__ Inv, int n, int k,
                               const int *piv, const double2 *pivval) {
  const int p = *piv;
  const double2 pv = *pivval;
  const double d = cabs2(pv);
  const double2 ip = d > 0.0 ? make_double2(pv.x / d, -pv.y / d) : make_double2(0.0, 0.0);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < 2 * n; j += gridDim.x * blockDim.x) {
    double2 *B = j < n ? M : Inv;
    const int jj = j < n ? j : j - n;
    const double2 a = B[(int64_t)k * n + jj];
    const double2 b = B[(int64_t)p * n + jj];
    B[(int64_t)k * n + jj] = cmul(b, ip);
    if (p != k) B[(int64_t)p * n + jj] = a;
  }
}

__global__ void gj_elim_kernel(double2 *__restrict__ M, double2 *__restrict__ Inv, int n, int k,
                               const double2 *__restrict__ f) {
  const int64_t total = (int64_t)n * 2 * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / (2 * n));
    const int j = (int)(e - (int64_t)i * 2 * n);
    if (i == k) continue;
    const double2 fi = f[i];
    if (fi.x == 0.0 && fi.y == 0.0) continue;
    double2 *B = j < n ? M : Inv;
    const int jj = j < n ? j : j - n;
    B[(int64_t)i * n + jj] = csub(B[(int64_t)i * n + jj], cmul(fi, B[(int64_t)k * n + jj]));
  }
}

__global__ void eye_kernel(double2 *__restrict__ M, int n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e - i * n;
    M[e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
}

// out_r = Minv in_r: warp per row, lanes over columns, RG right-hand sides
// per pass so each matrix entry is loaded once per RG of them.
__global__ void dense_trace_kernel(const double2 *__restrict__ M, int n, double2 *out) {
  __shared__ double2 sh[33];
  double2 acc = make_double2(0.0, 0.0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc = cadd(acc, M[(int64_t)i * n + i]);
  acc = block_csum(acc, sh);
  if (threadIdx.x == 0) *out = acc;
}

}  // namespace

int sm_count() {
  static std::mutex mu;
  static int cached[64] = {0};
  int dev = 0;
  MG_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (dev >= 0 && dev < 64 && cached[dev]) return cached[dev];
  int n = 0;
  MG_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  if (dev >= 0 && dev < 64) cached[dev] = n;
  return n;
}

template <typename T>
void stencil_apply(const C<T> *in, C<T> *out, const C<T> *AT, Geom g, int nrhs, int *err,
                   cudaStream_t s) {
  constexpr int RG = sizeof(T) == 4 ? 8 : 4;
  const int m = g.dof;
  // the (m, 9)-thread kernels below need 9 m threads of ~80 registers, which
  // one SM holds only up to m ~ 91; wider operators take the tiled kernel
  if (m > 64) {
    // wide operators: as many right-hand sides per pass as ~96 KB of staged
    // neighbour vectors allow
    const size_t per = (size_t)9 * m * sizeof(C<T>);
    if (per * 4 <= 96 * 1024) launch_wide<T, 4>(in, out, AT, g, nrhs, s);
    else if (per * 2 <= 96 * 1024) launch_wide<T, 2>(in, out, AT, g, nrhs, s);
    else launch_wide<T, 1>(in, out, AT, g, nrhs, s);
    return;
  }
  const size_t sm_tma = (size_t)(9 * m * m + 2 * 9 * RG * m) * sizeof(C<T>);
  if (sm_tma <= 200 * 1024) {
    smem_optin((const void *)stencil_tma_kernel<T, RG>, 200 * 1024);
    stencil_tma_kernel<T, RG><<<g.V, dim3(m, 9), sm_tma, s>>>(in, out, AT, g, nrhs, err, staging_extra_bytes());
    MG_LAUNCH_CHECK();
    return;
  }
  const size_t sm = (size_t)2 * 9 * RG * m * sizeof(C<T>);
  smem_optin((const void *)stencil_t_kernel<T, RG>, 200 * 1024);
  stencil_t_kernel<T, RG><<<g.V, dim3(m, 9), sm, s>>>(in, out, AT, g, nrhs);
  MG_LAUNCH_CHECK();
}

bool stencil_pipe_supported(const Geom &g) { return g.dof == 32; }

void stencil_apply_pipe(const float2 *in, float2 *out, const void *AT, bool bf16, Geom g, int nrhs, int *err,
                        cudaStream_t s) {
  if (!stencil_pipe_supported(g) || nrhs > 8 || nrhs < 1)
    throw Error(1, "pipelined stencil: 32 dofs per site and 1 .. 8 right-hand sides");
  if ((((uintptr_t)in | (uintptr_t)out | (uintptr_t)AT) & 15) != 0)
    throw Error(1, "pipelined stencil: operands must be 16-byte aligned");
  if (bf16) {
    if (nrhs <= 4) launch_pipe<__nv_bfloat162, 4>(in, out, (const __nv_bfloat162 *)AT, g, nrhs, err, s);
    else launch_pipe<__nv_bfloat162, 8>(in, out, (const __nv_bfloat162 *)AT, g, nrhs, err, s);
  } else {
    if (nrhs <= 4) launch_pipe<float2, 4>(in, out, (const float2 *)AT, g, nrhs, err, s);
    else launch_pipe<float2, 8>(in, out, (const float2 *)AT, g, nrhs, err, s);
  }
}

void stencil_apply_stream(const float2 *in, float2 *out, const void *AS, Geom g, int nrhs, bool per_site,
                          cudaStream_t s) {
  if (!stencil_pipe_supported(g) || nrhs > 8 || nrhs < 1)
    throw Error(1, "streaming stencil: 32 dofs per site and 1 .. 8 right-hand sides");
  if ((((uintptr_t)in | (uintptr_t)out | (uintptr_t)AS) & 15) != 0)
    throw Error(1, "streaming stencil: operands must be 16-byte aligned");
  if (per_site) {
    const uint4 *a = static_cast<const uint4 *>(AS);
    if (nrhs <= 2) stencil_stream_site_kernel<1><<<g.V, 288, 0, s>>>(in, out, a, g, nrhs);
    else if (nrhs <= 4) stencil_stream_site_kernel<2><<<g.V, 288, 0, s>>>(in, out, a, g, nrhs);
    else stencil_stream_site_kernel<4><<<g.V, 288, 0, s>>>(in, out, a, g, nrhs);
    MG_LAUNCH_CHECK();
    return;
  }
  // one warp per site, eight per block, at most two resident blocks per SM
  // worth of warps: each warp walks its share of the sites
  const int grid = (int)std::min<int64_t>((g.V + 7) / 8, (int64_t)sm_count() * 2);
  const uint4 *a = static_cast<const uint4 *>(AS);
  if (nrhs <= 2) stencil_stream_kernel<1><<<grid, 256, 0, s>>>(in, out, a, g, nrhs);
  else if (nrhs <= 4) stencil_stream_kernel<2><<<grid, 256, 0, s>>>(in, out, a, g, nrhs);
  else stencil_stream_kernel<4><<<grid, 256, 0, s>>>(in, out, a, g, nrhs);
  MG_LAUNCH_CHECK();
}

void stencil_to_stream(const float2 *AT32, void *AS, int64_t count, cudaStream_t s) {
  stencil_stream_layout_kernel<<<grid_for(count), 256, 0, s>>>(AT32, (__nv_bfloat162 *)AS, count);
  MG_LAUNCH_CHECK();
}

void stencil_to_bf16(const float2 *AT32, void *ATB, int64_t count, cudaStream_t s) {
  stencil_bf16_kernel<<<grid_for(count), 256, 0, s>>>(AT32, (__nv_bfloat162 *)ATB, count);
  MG_LAUNCH_CHECK();
}

template <typename To>
void stencil_transpose(const double2 *A, C<To> *AT, int64_t nblocks, int m, cudaStream_t s) {
  stencil_transpose_kernel<To><<<grid_for(nblocks * m * m), 256, 0, s>>>(A, AT, nblocks, m);
  MG_LAUNCH_CHECK();
}
template void stencil_transpose<double>(const double2 *, C<double> *, int64_t, int, cudaStream_t);
template void stencil_transpose<float>(const double2 *, C<float> *, int64_t, int, cudaStream_t);

template <typename T>
void stencil_split(const C<T> *in, C<T> *out9, const C<T> *A, Geom g, const int b[4],
                   cudaStream_t s) {
  stencil_split_kernel<T><<<g.V, 256, 0, s>>>(in, out9, A, g, b[0], b[1], b[2], b[3]);
  MG_LAUNCH_CHECK();
}

template <typename T>
void restrict_op(const C<T> *in, C<T> *out, const C<T> *P, const AggMap &m, int nrhs,
                 cudaStream_t s) {
  constexpr int RG = 4;
  const size_t sm = (size_t)RG * m.rows * sizeof(C<T>);
  if (sm > 200 * 1024) throw Error(1, "restrict: aggregate too large for shared memory");
  smem_optin((const void *)restrict_kernel<T, RG>, 200 * 1024);
  restrict_kernel<T, RG><<<m.coarse.V * 2, 256, sm, s>>>(in, out, P, m, nrhs);
  MG_LAUNCH_CHECK();
}

template <typename T>
void prolong_op(const C<T> *in, C<T> *out, const C<T> *P, const AggMap &m, int nrhs, double beta,
                cudaStream_t s) {
  // the coarse coefficients of every right-hand side of a launch are staged
  // in 48 KB of shared memory: launch groups of right-hand sides that fit
  const int per = (int)((48 * 1024) / ((size_t)m.ntv * sizeof(C<T>)));
  if (per < 1) throw Error(1, "prolong: too many test vectors");
  const int64_t nf = m.fine.n(), nc = m.coarse.n();
  for (int r0 = 0; r0 < nrhs; r0 += per) {
    const int rg = nrhs - r0 < per ? nrhs - r0 : per;
    const size_t sm = (size_t)rg * m.ntv * sizeof(C<T>);
    prolong_kernel<T, 4><<<m.coarse.V * 2, 256, sm, s>>>(in + (int64_t)r0 * nc, out + (int64_t)r0 * nf, P, m,
                                                         rg, (T)beta);
    MG_LAUNCH_CHECK();
  }
}

void restrict_op_bf16(const float2 *in, float2 *out, const void *P, const AggMap &m, int nrhs, cudaStream_t s) {
  constexpr int RG = 4;
  const size_t sm = (size_t)RG * m.rows * sizeof(float2);
  if (sm > 200 * 1024) throw Error(1, "restrict: aggregate too large for shared memory");
  smem_optin((const void *)restrict_kernel<float, RG, __nv_bfloat162>, 200 * 1024);
  restrict_kernel<float, RG, __nv_bfloat162>
      <<<m.coarse.V * 2, 256, sm, s>>>(in, out, static_cast<const __nv_bfloat162 *>(P), m, nrhs);
  MG_LAUNCH_CHECK();
}

void prolong_op_bf16(const float2 *in, float2 *out, const void *P, const AggMap &m, int nrhs, double beta,
                     cudaStream_t s) {
  const int per = (int)((48 * 1024) / ((size_t)m.ntv * sizeof(float2)));
  if (per < 1) throw Error(1, "prolong: too many test vectors");
  const int64_t nf = m.fine.n(), nc = m.coarse.n();
  for (int r0 = 0; r0 < nrhs; r0 += per) {
    const int rg = nrhs - r0 < per ? nrhs - r0 : per;
    const size_t sm = (size_t)rg * m.ntv * sizeof(float2);
    prolong_kernel<float, 4, __nv_bfloat162><<<m.coarse.V * 2, 256, sm, s>>>(
        in + (int64_t)r0 * nc, out + (int64_t)r0 * nf, static_cast<const __nv_bfloat162 *>(P), m, rg, (float)beta);
    MG_LAUNCH_CHECK();
  }
}

void probe_column(double2 *out, const double2 *P, const AggMap &m, int col, cudaStream_t s) {
  probe_kernel<<<grid_for(m.fine.n()), 256, 0, s>>>(out, P, m, col);
  MG_LAUNCH_CHECK();
}

void build_prolongator(const double2 *V, double2 *P, const AggMap &m, int *status, cudaStream_t s) {
  mgs_kernel<<<m.coarse.V * 2, 256, 0, s>>>(V, P, m, status);
  MG_LAUNCH_CHECK();
}

void galerkin_scatter(const double2 *cols, double2 *A, Geom coarse, int col, cudaStream_t s) {
  galerkin_scatter_kernel<<<grid_for(9 * coarse.n()), 256, 0, s>>>(cols, A, coarse, col);
  MG_LAUNCH_CHECK();
}

void prolongator_to_canonical(const double2 *P, double2 *out, const AggMap &m, cudaStream_t s) {
  p_canonical_kernel<<<grid_for((int64_t)m.coarse.V * 2 * m.ntv * m.rows), 256, 0, s>>>(P, out, m);
  MG_LAUNCH_CHECK();
}

void dense_from_stencil(const double2 *A, double2 *M, Geom g, cudaStream_t s) {
  dense_build_kernel<<<grid_for(g.n() * g.n()), 256, 0, s>>>(A, M, g);
  MG_LAUNCH_CHECK();
}

void dense_invert(double2 *M, double2 *work, int n, int *status, cudaStream_t s) {
  double2 *Inv = work;
  double2 *f = work + (int64_t)n * n;
  double2 *pivval = f + n;
  int *piv = reinterpret_cast<int *>(pivval + 1);
  eye_kernel<<<grid_for((int64_t)n * n), 256, 0, s>>>(Inv, n);
  for (int k = 0; k < n; ++k) {
    gj_pivot_kernel<<<1, 1024, 0, s>>>(M, n, k, piv, pivval, status);
    gj_factor_kernel<<<grid_for(n), 256, 0, s>>>(M, n, k, piv, f);
    gj_swap_kernel<<<grid_for(2 * n), 256, 0, s>>>(M, Inv, n, k, piv, pivval);
    gj_elim_kernel<<<grid_for((int64_t)n * 2 * n), 256, 0, s>>>(M, Inv, n, k, f);
  }
  MG_CUDA(cudaMemcpyAsync(M, Inv, sizeof(double2) * n * n, cudaMemcpyDeviceToDevice, s));
  MG_COUNT(4 * (int64_t)n);
  MG_LAUNCH_CHECK();
}

void dense_trace(const double2 *M, int n, double2 *out, cudaStream_t s) {
  dense_trace_kernel<<<1, 256, 0, s>>>(M, n, out);
  MG_LAUNCH_CHECK();
}

#define INST(T)                                                                                 \
  template void stencil_apply<T>(const C<T> *, C<T> *, const C<T> *, Geom, int, int *,         \
                                 cudaStream_t);                                                 \
  template void stencil_split<T>(const C<T> *, C<T> *, const C<T> *, Geom, const int *,         \
                                 cudaStream_t);                                                 \
  template void restrict_op<T>(const C<T> *, C<T> *, const C<T> *, const AggMap &, int,         \
                               cudaStream_t);                                                   \
  template void prolong_op<T>(const C<T> *, C<T> *, const C<T> *, const AggMap &, int, double,  \
                              cudaStream_t);                                                    \

INST(double)
INST(float)

}  // namespace mg
