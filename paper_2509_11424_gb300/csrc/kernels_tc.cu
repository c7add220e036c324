// Coarse stencil D_{l+1} = P_l^H D_l P_l (Sec. 2.2, Galerkin) on the
// 5th-generation tensor cores: tcgen05.mma kind::tf32 with operands in
// shared memory and FP32 accumulators in tensor memory (TMEM).
//
// For one coarse site X with m = 32 dofs (N_tv = 16) and a chunk of N
// right-hand sides the stencil is nine complex products
//   out = sum_d A_d B_d,   A_d = A(X, d) (32 x 32),  B_d = in[nbr(X, d)] (32 x N).
// With the real and imaginary parts of A_d stacked into one 64-row tile
// S_d = [Ar; Ai] (64 x 32 real), two accumulators of 64 x N collect
//   acc1 = sum_d S_d Br_d = [Ar Br; Ai Br],   acc2 = sum_d S_d Bi_d = [Ar Bi; Ai Bi],
// and the epilogue forms Re = acc1_top - acc2_bottom, Im = acc2_top + acc1_bottom.
// Each (direction, K-step of 8) is two MMAs of M = 64, N, K = 8.
//
// Data movement: the stacked tiles of a site (9 x 8 KB) are stored in HBM
// already in the shared-memory image the MMA descriptors describe (canonical
// K-major core matrices of 8 rows x 16 bytes, no swizzle), so one bulk copy
// (cp.async.bulk onto an mbarrier) brings them in; the 128 threads gather the
// neighbour vectors into the same core-matrix form meanwhile.  One elected
// thread issues the 72 MMAs of a chunk and commits them to an mbarrier;
// every wait is bounded and a timeout sets the error flag, waits (bounded)
// for the work in flight, releases the tensor memory and leaves.
//
// Precision: kind::tf32 reads FP32 operands as TF32 (10-bit mantissa);
// kind::f16 takes BF16 operands (8-bit mantissa, half the bytes and twice the
// tensor rate); both accumulate in FP32.  Neither is the FP32 stencil: the
// library uses them inside the multigrid preconditioner of the FP32 inner
// solves of the FP64 defect correction, where the true FP64 residual still
// decides convergence.
#include "kernels.h"

#include <cuda_bf16.h>

namespace mg {

namespace {

constexpr int kTcM = 32;                          // dofs per coarse site this path serves
constexpr int kTcTileElems = 64 * kTcM;           // one stacked [Ar; Ai] tile
constexpr int kTcMaxN = 32;                       // right-hand sides per MMA chunk
constexpr int kTcThreads = 128;

// operand element types: TF32 (FP32 storage, kind::tf32, K = 8 per MMA) and
// BF16 (kind::f16, K = 16 per MMA); a core-matrix row is 16 bytes = KC
// elements, each MMA spans two core matrices along K
template <typename E> struct TcOp;
template <> struct TcOp<float> {
  static constexpr int KC = 4, KMMA = 8;
  static constexpr uint32_t fmt = 2;  // TF32
};
template <> struct TcOp<__nv_bfloat16> {
  static constexpr int KC = 8, KMMA = 16;
  static constexpr uint32_t fmt = 1;  // BF16
};

__device__ __forceinline__ unsigned saddr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tc_mbar_init(uint64_t *mbar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(mbar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void tc_expect_tx(uint64_t *mbar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(mbar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tc_bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(saddr(dst)),
      "l"(src), "r"(bytes), "r"(saddr(mbar))
      : "memory");
}
__device__ __forceinline__ bool tc_try_wait(uint64_t *mbar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(saddr(mbar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait on one phase of an mbarrier (kWaitNs of the global timer)
__device__ __forceinline__ bool tc_wait(uint64_t *mbar, unsigned parity) {
  const unsigned long long t0 = global_ns();
  for (int it = 0; it < (1 << 26); ++it) {
    if (tc_try_wait(mbar, parity)) return true;
    if ((it & 63) == 63 && global_ns() - t0 > kWaitNs) break;
  }
  return false;
}

// shared-memory matrix descriptor (tcgen05): start address, leading (K)
// and stride (M/N) byte offsets of the core matrices, all in 16-byte units;
// bits 46-47 = 1 (descriptor version), no swizzle
__device__ __forceinline__ uint64_t smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// instruction descriptor: FP32 accumulator (bits 4-5 = 1), A and B format
// (bits 7-9, 10-12: TF32 = 2 under kind::tf32, BF16 = 1 under kind::f16),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t mma_idesc(uint32_t fmt, int M, int N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <typename E>
__device__ __forceinline__ void mma_op(unsigned tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       unsigned accumulate) {
  if constexpr (sizeof(E) == 4) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}
__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(mbar))
               : "memory");
}

// 32 lanes x 32 consecutive 32-bit columns of tensor memory into v
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float (&v)[32]) {
  unsigned r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Accumulator row held by TMEM lane 32 warp + lane (-1: none of the 64
// rows).  LAYOUT 0: M = 64 MMAs, whose accumulator rows 16w .. 16w + 15 sit
// in the first 16 lanes of warp w's lane quarter (checked against the
// oracle; row i in lane i does not hold for M = 64).  LAYOUT 2: M = 128 MMAs
// (row i in lane i) whose rows 64..127 read the next core matrices of the
// tile and are discarded: twice the tensor work, the same result.
template <int LAYOUT> __device__ __forceinline__ int acc_row_of_lane(int warp, int lane) {
  if (LAYOUT == 0) return lane < 16 ? 16 * warp + lane : -1;
  return warp < 2 ? 32 * warp + lane : -1;
}

// four complex values (re, im) as the quad of real parts and the quad of
// imaginary parts in the operand element type
__device__ __forceinline__ void split_store(float *re_dst, float *im_dst, float2 a, float2 b, float2 c, float2 d) {
  *reinterpret_cast<float4 *>(re_dst) = make_float4(a.x, b.x, c.x, d.x);
  *reinterpret_cast<float4 *>(im_dst) = make_float4(a.y, b.y, c.y, d.y);
}

// smem: [A tiles 9 x 64 x 32 E][B: 9 dirs x {re, im} x (N x 32 E)][acc staging 2 x 64 x 32 FP32]
template <typename E, int LAYOUT>
__global__ void __launch_bounds__(kTcThreads) stencil_tc_kernel(const float2 *__restrict__ in,
                                                               float2 *__restrict__ out,
                                                               const E *__restrict__ ATC, Geom g,
                                                               int nrhs, int *err, unsigned extra_tx) {
  using Op = TcOp<E>;
  constexpr int KC = Op::KC;
  constexpr unsigned kSiteBytes = 9u * kTcTileElems * sizeof(E);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar_a, bar_mma;
  __shared__ unsigned tmem_slot;
  __shared__ int fail;
  E *As = reinterpret_cast<E *>(smem_raw);
  E *Bs = As + 9 * kTcTileElems;                                           // [d][part][N x 32]
  float *St = reinterpret_cast<float *>(Bs + 9 * 2 * kTcMaxN * kTcM);      // [2 acc][64 rows][kTcMaxN]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int X = blockIdx.x;
  const int64_t n = g.n();

  if (tid == 0) {
    tc_mbar_init(&bar_a, 1);
    tc_mbar_init(&bar_mma, 1);
    fail = 0;
  }
  if (warp == 0) {
    // 64 columns: two accumulators of up to 32 columns each
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                 "r"(64)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_slot;
  if (tid == 0) {
    tc_expect_tx(&bar_a, kSiteBytes + extra_tx);  // extra_tx: failure-injection tests only
    tc_bulk_g2s(As, ATC + (int64_t)X * 9 * kTcTileElems, kSiteBytes, &bar_a);
  }
  int nbr[9];
#pragma unroll
  for (int d = 0; d < 9; ++d) nbr[d] = g.neighbor(X, d);

  unsigned mma_phase = 0;
  bool a_ready = false;
  for (int r0 = 0; r0 < nrhs; r0 += kTcMaxN) {
    const int rc = nrhs - r0 < kTcMaxN ? nrhs - r0 : kTcMaxN;
    const int N = LAYOUT == 1 ? (rc + 15) & ~15 : (rc + 7) & ~7;  // MMA N (M = 128 needs N % 16 == 0)
    // gather B: element (n, k) of part p of direction d at
    // ((k / KC) * N + n) * KC + k % KC (core matrices of 8 rows x 16 bytes).
    // A fixed trip count (the full chunk of 32 right-hand sides), all loads
    // issued before the first conversion: one round trip to memory instead
    // of one per item.
    {
      constexpr int kItems = 9 * (kTcM / KC) * kTcMaxN;
      constexpr int kIters = (kItems + kTcThreads - 1) / kTcThreads;
      constexpr int kLd = KC / 2;  // 16-byte loads per item (two complex values each)
      const int total = 9 * (kTcM / KC) * N;
      float4 v[kIters][kLd];
#pragma unroll
      for (int it = 0; it < kIters; ++it) {
        const int t = tid + it * kTcThreads;
        const int nn = t % N, c = (t / N) % (kTcM / KC), d = t / ((kTcM / KC) * N);
        const bool ok = t < total && nn < rc;
        const float4 *src = reinterpret_cast<const float4 *>(in + (int64_t)(r0 + (ok ? nn : 0)) * n +
                                                             (int64_t)nbr[ok ? d : 0] * kTcM + KC * c);
#pragma unroll
        for (int q = 0; q < kLd; ++q) v[it][q] = ok ? __ldg(src + q) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int it = 0; it < kIters; ++it) {
        const int t = tid + it * kTcThreads;
        if (t < total) {
          const int nn = t % N, c = (t / N) % (kTcM / KC), d = t / ((kTcM / KC) * N);
          E *base = Bs + (size_t)(d * 2) * kTcMaxN * kTcM;
          E *re_dst = base + ((size_t)c * N + nn) * KC;
          E *im_dst = base + kTcMaxN * kTcM + ((size_t)c * N + nn) * KC;
          if constexpr (sizeof(E) == 4) {
            split_store(reinterpret_cast<float *>(re_dst), reinterpret_cast<float *>(im_dst),
                        make_float2(v[it][0].x, v[it][0].y), make_float2(v[it][0].z, v[it][0].w),
                        make_float2(v[it][1].x, v[it][1].y), make_float2(v[it][1].z, v[it][1].w));
          } else {
            __nv_bfloat162 re[4], im[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              re[q] = __floats2bfloat162_rn(v[it][q].x, v[it][q].z);
              im[q] = __floats2bfloat162_rn(v[it][q].y, v[it][q].w);
            }
            *reinterpret_cast<uint4 *>(re_dst) = *reinterpret_cast<const uint4 *>(re);
            *reinterpret_cast<uint4 *>(im_dst) = *reinterpret_cast<const uint4 *>(im);
          }
        }
      }
    }
    // make the generic-proxy stores visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    int bad = 0;
    if (!a_ready) {
      a_ready = tc_wait(&bar_a, 0);
      bad = a_ready ? 0 : 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    bad = __syncthreads_or(bad);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (bad) break;
    if (tid == 0) {
      const uint32_t idesc = mma_idesc(Op::fmt, LAYOUT == 1 ? 128 : 64, N);
      const unsigned a0 = saddr(As), b0 = saddr(Bs);
      for (int d = 0; d < 9; ++d) {
        for (int kc = 0; kc < kTcM / Op::KMMA; ++kc) {
          // A: core matrix (row group gr, K chunk c) at c * 1024 + gr * 128
          const uint64_t ad = smem_desc(a0 + d * kTcTileElems * (unsigned)sizeof(E) + kc * 2 * 1024, 1024, 128);
          // B: (n group, K chunk c) at c * N * 16 + ng * 128
          const unsigned bre = b0 + (unsigned)(d * 2) * kTcMaxN * kTcM * (unsigned)sizeof(E) + kc * 2 * N * 16;
          const unsigned bim = bre + kTcMaxN * kTcM * (unsigned)sizeof(E);
          const unsigned acc = (d > 0 || kc > 0) ? 1u : 0u;
          mma_op<E>(tmem, ad, smem_desc(bre, N * 16, 128), idesc, acc);
          mma_op<E>(tmem + kTcMaxN, ad, smem_desc(bim, N * 16, 128), idesc, acc);
        }
      }
      mma_commit(&bar_mma);
    }
    __syncwarp();
    const bool done = tc_wait(&bar_mma, mma_phase);
    mma_phase ^= 1u;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    bad = __syncthreads_or(done ? 0 : 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (bad) {
      // the MMAs may still run: a second bounded wait before the tensor
      // memory is released
      fail = 1;
      if (!done) tc_wait(&bar_mma, mma_phase ^ 1u);
      break;
    }
    // epilogue: each warp reads its 32 lanes of both accumulators
    {
      float v1[32], v2[32];
      const unsigned lane_base = (unsigned)(32 * warp) << 16;
      tmem_ld32(tmem + lane_base, v1);
      tmem_ld32(tmem + lane_base + kTcMaxN, v2);
      const int row = acc_row_of_lane<LAYOUT == 1 ? 2 : 0>(warp, lane);
      if (row >= 0) {
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          St[row * kTcMaxN + c] = v1[c];
          St[64 * kTcMaxN + row * kTcMaxN + c] = v2[c];
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // Re = Ar Br - Ai Bi (acc1 top - acc2 bottom), Im = Ar Bi + Ai Br
    for (int t = tid; t < rc * kTcM; t += kTcThreads) {
      const int r = t / kTcM, i = t % kTcM;
      const float re = St[i * kTcMaxN + r] - St[64 * kTcMaxN + (32 + i) * kTcMaxN + r];
      const float im = St[64 * kTcMaxN + i * kTcMaxN + r] + St[(32 + i) * kTcMaxN + r];
      out[(int64_t)(r0 + r) * n + (int64_t)X * kTcM + i] = make_float2(re, im);
    }
    __syncthreads();
  }
  if (!a_ready) {
    // the bulk copy may still be writing shared memory
    fail = 1;
    tc_wait(&bar_a, 0);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64) : "memory");
  if (tid == 0 && fail && err) atomicExch(err, 3);
}

// Persistent pipelined form of the BF16 kernel for up to 32 right-hand
// sides: one CTA per SM walks the sites X = blockIdx.x + i gridDim.x with two
// shared-memory stages and two TMEM accumulator sets.  Iteration i issues the
// neighbour loads of site i, writes out site i - 1 (its MMAs ran meanwhile),
// stores site i's operands, and has one thread start site i's MMAs and the
// bulk copy of site i + 1's tiles, so the tensor work and the tile copy of
// one site overlap the gathers and the epilogue of its neighbours in the
// walk.  The MMAs and their order per site are those of stencil_tc_kernel:
// identical results.  Every wait is bounded; on a timeout the CTA sets the
// error flag, waits (bounded) for its MMAs and copies in flight, releases its
// tensor memory and leaves.
// smem: [2 stages][A tiles 9 x 64 x 32][B 9 x {re, im} x 32 x 32] BF16, then
// [64 x 32 x 2] FP32 accumulator staging
__global__ void __launch_bounds__(kTcThreads, 1)
    stencil_tc_pipe_kernel(const float2 *__restrict__ in, float2 *__restrict__ out,
                           const __nv_bfloat16 *__restrict__ ATC, Geom g, int nrhs, int *err,
                           unsigned extra_tx) {
  using E = __nv_bfloat16;
  using Op = TcOp<E>;
  constexpr int KC = Op::KC;
  constexpr unsigned kSiteBytes = 9u * kTcTileElems * sizeof(E);
  constexpr int kStageElems = 9 * kTcTileElems + 9 * 2 * kTcMaxN * kTcM;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar_a[2], bar_mma[2];
  __shared__ unsigned tmem_slot;
  E *stage0 = reinterpret_cast<E *>(smem_raw);
  float *St = reinterpret_cast<float *>(stage0 + 2 * kStageElems);  // [2 acc][64 rows][kTcMaxN]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t n = g.n();
  const int count = g.V > (int)blockIdx.x ? (g.V - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int N = (nrhs + 7) & ~7;
  if (tid == 0) {
    for (int q = 0; q < 2; ++q) {
      tc_mbar_init(&bar_a[q], 1);
      tc_mbar_init(&bar_mma[q], 1);
    }
  }
  if (warp == 0) {
    // two stages x two accumulators of 32 columns
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                 "r"(128)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_slot;
  // work in flight per stage and the parity of the phase that will end it
  bool a_pending[2] = {false, false}, mma_pending[2] = {false, false};
  unsigned a_par[2] = {0u, 0u}, mma_par[2] = {0u, 0u};
  if (count > 0) {
    if (tid == 0) {
      tc_expect_tx(&bar_a[0], kSiteBytes + extra_tx);  // extra_tx: failure-injection tests only
      tc_bulk_g2s(stage0, ATC + (int64_t)blockIdx.x * 9 * kTcTileElems, kSiteBytes, &bar_a[0]);
    }
    a_pending[0] = true;
  }
  bool failed = false;
  constexpr int kItems = 9 * (kTcM / KC) * kTcMaxN;
  constexpr int kIters = (kItems + kTcThreads - 1) / kTcThreads;
  const int total = 9 * (kTcM / KC) * N;
  for (int i = 0; i <= count && !failed; ++i) {
    const int s = i & 1;
    const int X = (int)blockIdx.x + i * (int)gridDim.x;
    float4 v[kIters][4];
    if (i < count) {
      int nbr[9];
#pragma unroll
      for (int d = 0; d < 9; ++d) nbr[d] = g.neighbor(X, d);
#pragma unroll
      for (int it = 0; it < kIters; ++it) {
        const int t = tid + it * kTcThreads;
        const int nn = t % N, c = (t / N) % (kTcM / KC), d = t / ((kTcM / KC) * N);
        const bool ok = t < total && nn < nrhs;
        const float4 *src = reinterpret_cast<const float4 *>(in + (int64_t)(ok ? nn : 0) * n +
                                                             (int64_t)nbr[ok ? d : 0] * kTcM + KC * c);
#pragma unroll
        for (int q = 0; q < 4; ++q) v[it][q] = ok ? __ldg(src + q) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    if (i > 0) {
      // epilogue of site i - 1 (stage s ^ 1)
      const int sp = s ^ 1;
      const bool done = tc_wait(&bar_mma[sp], ((i - 1) >> 1) & 1);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      const int bad = __syncthreads_or(done ? 0 : 1);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (bad) {
        failed = true;
        break;
      }
      mma_pending[sp] = false;
      {
        float v1[32], v2[32];
        const unsigned lane_base = (unsigned)(32 * warp) << 16;
        tmem_ld32(tmem + lane_base + sp * 64, v1);
        tmem_ld32(tmem + lane_base + sp * 64 + kTcMaxN, v2);
        const int row = acc_row_of_lane<0>(warp, lane);
        if (row >= 0) {
#pragma unroll
          for (int c = 0; c < 32; ++c) {
            St[row * kTcMaxN + c] = v1[c];
            St[64 * kTcMaxN + row * kTcMaxN + c] = v2[c];
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int Xp = X - (int)gridDim.x;
      for (int t = tid; t < nrhs * kTcM; t += kTcThreads) {
        const int r = t / kTcM, k = t % kTcM;
        const float re = St[k * kTcMaxN + r] - St[64 * kTcMaxN + (32 + k) * kTcMaxN + r];
        const float im = St[64 * kTcMaxN + k * kTcMaxN + r] + St[(32 + k) * kTcMaxN + r];
        out[(int64_t)r * n + (int64_t)Xp * kTcM + k] = make_float2(re, im);
      }
    }
    if (i == count) break;
    // operands of site i into stage s (its previous MMAs, site i - 2, are done)
    E *As = stage0 + s * kStageElems;
    E *Bs = As + 9 * kTcTileElems;
#pragma unroll
    for (int it = 0; it < kIters; ++it) {
      const int t = tid + it * kTcThreads;
      if (t < total) {
        const int nn = t % N, c = (t / N) % (kTcM / KC), d = t / ((kTcM / KC) * N);
        E *base = Bs + (size_t)(d * 2) * kTcMaxN * kTcM;
        E *re_dst = base + ((size_t)c * N + nn) * KC;
        E *im_dst = base + kTcMaxN * kTcM + ((size_t)c * N + nn) * KC;
        __nv_bfloat162 re[4], im[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          re[q] = __floats2bfloat162_rn(v[it][q].x, v[it][q].z);
          im[q] = __floats2bfloat162_rn(v[it][q].y, v[it][q].w);
        }
        *reinterpret_cast<uint4 *>(re_dst) = *reinterpret_cast<const uint4 *>(re);
        *reinterpret_cast<uint4 *>(im_dst) = *reinterpret_cast<const uint4 *>(im);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const bool landed = tc_wait(&bar_a[s], (i >> 1) & 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    const int bad = __syncthreads_or(landed ? 0 : 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (bad) {
      failed = true;
      break;
    }
    a_pending[s] = false;
    if (tid == 0) {
      const uint32_t idesc = mma_idesc(Op::fmt, 64, N);
      const unsigned a0 = saddr(As), b0 = saddr(Bs);
      const unsigned acc0 = tmem + s * 64;
      for (int d = 0; d < 9; ++d) {
        for (int kc = 0; kc < kTcM / Op::KMMA; ++kc) {
          const uint64_t ad = smem_desc(a0 + d * kTcTileElems * (unsigned)sizeof(E) + kc * 2 * 1024, 1024, 128);
          const unsigned bre = b0 + (unsigned)(d * 2) * kTcMaxN * kTcM * (unsigned)sizeof(E) + kc * 2 * N * 16;
          const unsigned bim = bre + kTcMaxN * kTcM * (unsigned)sizeof(E);
          const unsigned acc = (d > 0 || kc > 0) ? 1u : 0u;
          mma_op<E>(acc0, ad, smem_desc(bre, N * 16, 128), idesc, acc);
          mma_op<E>(acc0 + kTcMaxN, ad, smem_desc(bim, N * 16, 128), idesc, acc);
        }
      }
      mma_commit(&bar_mma[s]);
      if (i + 1 < count) {
        // stage s ^ 1's tiles were read by site i - 1's MMAs, complete above
        tc_expect_tx(&bar_a[s ^ 1], kSiteBytes + extra_tx);
        tc_bulk_g2s(stage0 + (s ^ 1) * kStageElems, ATC + (int64_t)(X + (int)gridDim.x) * 9 * kTcTileElems,
                    kSiteBytes, &bar_a[s ^ 1]);
      }
    }
    mma_pending[s] = true;
    mma_par[s] = (i >> 1) & 1;
    if (i + 1 < count) {
      a_pending[s ^ 1] = true;
      a_par[s ^ 1] = ((i + 1) >> 1) & 1;
    }
    __syncwarp();
  }
  if (failed) {
    // copies and MMAs still in flight: bounded waits before the memory goes
    for (int q = 0; q < 2; ++q) {
      if (a_pending[q]) tc_wait(&bar_a[q], a_par[q]);
      if (mma_pending[q]) tc_wait(&bar_mma[q], mma_par[q]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128) : "memory");
  if (tid == 0 && failed && err) atomicExch(err, 3);
}

// ATC[X][d][c][gr][r][q] = element (row 8 gr + r, k = KC c + q) of the
// stacked tile [Re A; Im A] of block d of site X (A canonical [X][d][i][j]),
// in the operand type E
template <typename E>
__global__ void stencil_tile_tc_kernel(const double2 *__restrict__ A, E *__restrict__ ATC, int64_t nsites) {
  constexpr int KC = TcOp<E>::KC;
  const int64_t total = nsites * 9 * kTcTileElems;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t blk = e / kTcTileElems;  // X * 9 + d
    const int w = (int)(e - blk * kTcTileElems);
    const int q = w % KC, r = (w / KC) & 7, gr = (w / (8 * KC)) & 7, c = w / (64 * KC);
    const int row = 8 * gr + r, k = KC * c + q;
    const double2 a = A[blk * kTcM * kTcM + (int64_t)(row & 31) * kTcM + k];
    const float v = (float)(row < 32 ? a.x : a.y);
    if constexpr (sizeof(E) == 4) ATC[e] = v;
    else ATC[e] = __float2bfloat16_rn(v);
  }
}

}  // namespace

bool stencil_tc_supported(const Geom &g) { return g.dof == kTcM; }

size_t stencil_tc_elems(const Geom &g) { return (size_t)g.V * 9 * kTcTileElems; }

void stencil_tile_tc(const double2 *A, void *ATC, bool bf16, const Geom &g, cudaStream_t s) {
  if (!stencil_tc_supported(g)) throw Error(1, "tensor-core stencil: needs 32 dofs per coarse site");
  const int64_t total = (int64_t)g.V * 9 * kTcTileElems;
  const int64_t blocks = (total + 255) / 256;
  const int grid = (int)(blocks < 152 * 16 ? blocks : 152 * 16);
  if (bf16) stencil_tile_tc_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(A, (__nv_bfloat16 *)ATC, g.V);
  else stencil_tile_tc_kernel<float><<<grid, 256, 0, s>>>(A, (float *)ATC, g.V);
  MG_LAUNCH_CHECK();
}

template <typename E, int LAYOUT>
static void launch_tc(const float2 *in, float2 *out, const E *ATC, Geom g, int nrhs, int *err, cudaStream_t s) {
  const size_t sm = (size_t)(9 * kTcTileElems + 9 * 2 * kTcMaxN * kTcM) * sizeof(E) +
                    (size_t)2 * 64 * kTcMaxN * sizeof(float);
  smem_optin((const void *)stencil_tc_kernel<E, LAYOUT>, (int)sm);
  stencil_tc_kernel<E, LAYOUT><<<g.V, kTcThreads, sm, s>>>(in, out, ATC, g, nrhs, err, staging_extra_bytes());
  MG_LAUNCH_CHECK();
}

void stencil_apply_tc(const float2 *in, float2 *out, const void *ATC, Geom g, int nrhs, int *err, int layout,
                      cudaStream_t s) {
  if (!stencil_tc_supported(g)) throw Error(1, "tensor-core stencil: needs 32 dofs per coarse site");
  if ((((uintptr_t)in | (uintptr_t)out | (uintptr_t)ATC) & 15) != 0)
    throw Error(1, "tensor-core stencil: operands must be 16-byte aligned");
  if (layout == 3 && nrhs >= 1 && nrhs <= kTcMaxN) {
    const size_t sm = (size_t)2 * (9 * kTcTileElems + 9 * 2 * kTcMaxN * kTcM) * sizeof(__nv_bfloat16) +
                      (size_t)2 * 64 * kTcMaxN * sizeof(float);
    smem_optin((const void *)stencil_tc_pipe_kernel, (int)sm);
    const int grid = g.V < sm_count() ? g.V : sm_count();
    stencil_tc_pipe_kernel<<<grid, kTcThreads, sm, s>>>(in, out, (const __nv_bfloat16 *)ATC, g, nrhs, err,
                                                       staging_extra_bytes());
    MG_LAUNCH_CHECK();
    return;
  }
  if (layout == 2 || layout == 3) launch_tc<__nv_bfloat16, 0>(in, out, (const __nv_bfloat16 *)ATC, g, nrhs, err, s);
  else if (layout == 1) launch_tc<float, 1>(in, out, (const float *)ATC, g, nrhs, err, s);
  else launch_tc<float, 0>(in, out, (const float *)ATC, g, nrhs, err, s);
}

}  // namespace mg
