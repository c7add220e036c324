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
// Precision: the tensor cores read the FP32 operands as TF32 (10-bit
// mantissa) and accumulate in FP32.  The result is therefore not the FP32
// stencil; it is used inside the FP32 inner solves of the FP64 defect
// correction, where the true FP64 residual still decides convergence.
#include "kernels.h"

namespace mg {

namespace {

constexpr int kTcM = 32;                          // dofs per coarse site this path serves
constexpr int kTcTileFloats = 64 * kTcM;          // one stacked [Ar; Ai] tile
constexpr int kTcSiteBytes = 9 * kTcTileFloats * 4;  // 73728
constexpr int kTcMaxN = 32;                       // right-hand sides per MMA chunk
constexpr int kTcThreads = 128;

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
// instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t tf32_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(unsigned tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         unsigned accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
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

// smem: [A tiles 9 x 8 KB][B: 9 dirs x {re, im} x (N x 32 floats)][acc staging]
template <int LAYOUT>
__global__ void __launch_bounds__(kTcThreads) stencil_tc_kernel(const float2 *__restrict__ in,
                                                               float2 *__restrict__ out,
                                                               const float *__restrict__ ATC, Geom g,
                                                               int nrhs, int *err, unsigned extra_tx) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar_a, bar_mma;
  __shared__ unsigned tmem_slot;
  __shared__ int fail;
  float *As = reinterpret_cast<float *>(smem_raw);
  float *Bs = As + 9 * kTcTileFloats;          // [d][part][N x 32]
  float *St = Bs + 9 * 2 * kTcMaxN * kTcM;       // [2 acc][64 rows][kTcMaxN]
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
    tc_expect_tx(&bar_a, (unsigned)kTcSiteBytes + extra_tx);  // extra_tx: failure-injection tests only
    tc_bulk_g2s(As, ATC + (int64_t)X * (kTcSiteBytes / 4), (unsigned)kTcSiteBytes, &bar_a);
  }
  int nbr[9];
#pragma unroll
  for (int d = 0; d < 9; ++d) nbr[d] = g.neighbor(X, d);

  unsigned mma_phase = 0;
  bool a_ready = false;
  for (int r0 = 0; r0 < nrhs; r0 += kTcMaxN) {
    const int rc = nrhs - r0 < kTcMaxN ? nrhs - r0 : kTcMaxN;
    const int N = LAYOUT == 2 ? (rc + 15) & ~15 : (rc + 7) & ~7;  // MMA N (M = 128 needs N % 16 == 0)
    // gather B: element (n, k) of part p of direction d at
    // ((k/4) * N + n) * 4 + k%4 floats (core matrices of 8 rows x 16 bytes)
    for (int t = tid; t < 9 * 8 * N; t += kTcThreads) {
      const int nn = t % N, c = (t / N) & 7, d = t / (8 * N);
      float4 re = make_float4(0.f, 0.f, 0.f, 0.f), im = re;
      if (nn < rc) {
        const float4 *src = reinterpret_cast<const float4 *>(in + (int64_t)(r0 + nn) * n +
                                                             (int64_t)nbr[d] * kTcM + 4 * c);
        const float4 a = __ldg(src), b = __ldg(src + 1);  // 4 complex: (re, im) pairs
        re = make_float4(a.x, a.z, b.x, b.z);
        im = make_float4(a.y, a.w, b.y, b.w);
      }
      float *base = Bs + (size_t)(d * 2) * kTcMaxN * kTcM;
      reinterpret_cast<float4 *>(base)[c * N + nn] = re;
      reinterpret_cast<float4 *>(base + kTcMaxN * kTcM)[c * N + nn] = im;
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
      const uint32_t idesc = tf32_idesc(LAYOUT == 2 ? 128 : 64, N);
      const unsigned a0 = saddr(As), b0 = saddr(Bs);
      for (int d = 0; d < 9; ++d) {
        for (int kc = 0; kc < 4; ++kc) {
          // A: core matrix (row group gr, K chunk c) at c * 1024 + gr * 128
          const uint64_t ad = smem_desc(a0 + d * kTcTileFloats * 4 + kc * 2 * 1024, 1024, 128);
          // B: (n group, K chunk c) at c * N * 16 + ng * 128
          const unsigned bre = b0 + (unsigned)(d * 2) * kTcMaxN * kTcM * 4 + kc * 2 * N * 16;
          const unsigned bim = bre + kTcMaxN * kTcM * 4;
          const unsigned acc = (d > 0 || kc > 0) ? 1u : 0u;
          mma_tf32(tmem, ad, smem_desc(bre, N * 16, 128), idesc, acc);
          mma_tf32(tmem + kTcMaxN, ad, smem_desc(bim, N * 16, 128), idesc, acc);
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
      const int row = acc_row_of_lane<LAYOUT>(warp, lane);
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

// ATC[X][d][c][gr][r][q] = element (row 8 gr + r, k = 4 c + q) of the stacked
// tile [Re A; Im A] of block d of site X (A canonical [X][d][i][j])
__global__ void stencil_tile_tc_kernel(const double2 *__restrict__ A, float *__restrict__ ATC, int64_t nsites) {
  const int64_t total = nsites * 9 * kTcTileFloats;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t blk = e / kTcTileFloats;  // X * 9 + d
    const int w = (int)(e - blk * kTcTileFloats);
    const int q = w & 3, r = (w >> 2) & 7, gr = (w >> 5) & 7, c = w >> 8;
    const int row = 8 * gr + r, k = 4 * c + q;
    const double2 a = A[blk * kTcM * kTcM + (int64_t)(row & 31) * kTcM + k];
    ATC[e] = (float)(row < 32 ? a.x : a.y);
  }
}

}  // namespace

bool stencil_tc_supported(const Geom &g) { return g.dof == kTcM; }

size_t stencil_tc_floats(const Geom &g) { return (size_t)g.V * 9 * kTcTileFloats; }

void stencil_tile_tc(const double2 *A, float *ATC, const Geom &g, cudaStream_t s) {
  if (!stencil_tc_supported(g)) throw Error(1, "tensor-core stencil: needs 32 dofs per coarse site");
  const int64_t total = (int64_t)g.V * 9 * kTcTileFloats;
  const int64_t blocks = (total + 255) / 256;
  stencil_tile_tc_kernel<<<(int)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, s>>>(A, ATC, g.V);
  MG_LAUNCH_CHECK();
}

void stencil_apply_tc(const float2 *in, float2 *out, const float *ATC, Geom g, int nrhs, int *err, int layout,
                      cudaStream_t s) {
  if (!stencil_tc_supported(g)) throw Error(1, "tensor-core stencil: needs 32 dofs per coarse site");
  if ((((uintptr_t)in | (uintptr_t)out | (uintptr_t)ATC) & 15) != 0)
    throw Error(1, "tensor-core stencil: operands must be 16-byte aligned");
  const size_t sm = (size_t)(9 * kTcTileFloats + 9 * 2 * kTcMaxN * kTcM + 2 * 64 * kTcMaxN) * sizeof(float);
  if (layout == 1) {
    smem_optin((const void *)stencil_tc_kernel<2>, (int)sm);
    stencil_tc_kernel<2><<<g.V, kTcThreads, sm, s>>>(in, out, ATC, g, nrhs, err,
                                                             staging_extra_bytes());
  } else {
    smem_optin((const void *)stencil_tc_kernel<0>, (int)sm);
    stencil_tc_kernel<0><<<g.V, kTcThreads, sm, s>>>(in, out, ATC, g, nrhs, err,
                                                             staging_extra_bytes());
  }
  MG_LAUNCH_CHECK();
}

}  // namespace mg
