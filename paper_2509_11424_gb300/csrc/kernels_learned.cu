// Gauge-covariant convolution layers of the learned smoother: forward,
// adjoint (input gradient), weight gradient, and the Adam update.
//
//   phi[o](x) = sum_c sum_h W[h][o][c] (T_h psi[c])(x)
//
// h = 0 identity, 1 + 2 mu: U_mu(x) psi(x + mu), 2 + 2 mu: U_mu(x - mu)^H
// psi(x - mu), with the fermion sign on hops across the time boundary;
// W[h][o][c] is a complex 4x4 matrix on the spin index.  Activations are
// [b][c] fine-level vectors (FP32 in the structure-of-arrays order with
// structure-of-arrays links, FP64 canonical [site][12]); weights
// [h][o][c][4][4].  The adjoint uses that
// the adjoint of hop h is the reversed hop and the adjoint of W is W^H.
#include "kernels.h"

namespace mg {

namespace {

inline int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

template <typename T> constexpr bool kSoa = sizeof(T) == 4;

// transported spinor t = T_h psi at site s (12 complex), sign folded in
template <typename T>
__device__ __forceinline__ void transported(const C<T> *__restrict__ psi, const C<T> *__restrict__ U,
                                            const Geom &g, int s, const int (&c)[4], int h,
                                            C<T> (&t)[12]) {
  const int64_t V = g.V;
  if (h == 0) {
    load_fine_site<T>(psi, s, V, t);
    return;
  }
  const int mu = (h - 1) >> 1;
  const bool fwd = h & 1;
  int cn[4] = {c[0], c[1], c[2], c[3]};
  T sign = (T)1;
  if (fwd) {
    cn[mu] = (c[mu] + 1 == g.L[mu]) ? 0 : c[mu] + 1;
    if (mu == 3 && cn[3] == 0) sign = (T)-1;
  } else {
    cn[mu] = (c[mu] == 0) ? g.L[mu] - 1 : c[mu] - 1;
    if (mu == 3 && c[3] == 0) sign = (T)-1;
  }
  const int sn = g.index(cn);
  const int ls = fwd ? s : sn;
  C<T> uu[9];
#pragma unroll
  for (int i = 0; i < 9; ++i)
    uu[i] = kSoa<T> ? __ldg(U + (int64_t)(mu * 9 + i) * V + ls) : __ldg(U + ((int64_t)ls * 4 + mu) * 9 + i);
  C<T> v[12];
  load_fine_site<T>(psi, sn, V, v);
#pragma unroll
  for (int sp = 0; sp < 4; ++sp) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      C<T> z = mk<T>((T)0, (T)0);
#pragma unroll
      for (int b = 0; b < 3; ++b)
        z = fwd ? cfma(uu[3 * a + b], v[sp * 3 + b], z) : cfmac(uu[3 * b + a], v[sp * 3 + b], z);
      t[sp * 3 + a] = cscale(z, sign);
    }
  }
}

// forward: one thread per site computing OG output channels at once, so each
// transported input T_h psi[c] is formed once for the whole group;
// blockIdx.x = (site range, sample) with the sample fastest, so the blocks
// of one site range run together and read its links from L2 after the
// first; blockIdx.y = output group
template <typename T, int OG>
__global__ void __launch_bounds__(128) glayer_forward_kernel(const C<T> *__restrict__ in,
                                                             C<T> *__restrict__ out,
                                                             const C<T> *__restrict__ W,
                                                             const C<T> *__restrict__ U, Geom g,
                                                             int Cin, int Cout, int nb) {
  extern __shared__ unsigned char smem_raw[];
  C<T> *Ws = reinterpret_cast<C<T> *>(smem_raw);  // [h][c][og][16] for this group
  const int o0 = blockIdx.y * OG, b = (int)(blockIdx.x % (unsigned)nb);
  const int og = Cout - o0 < OG ? Cout - o0 : OG;
  for (int e = threadIdx.x; e < 9 * Cin * OG * 16; e += blockDim.x) {
    const int h = e / (Cin * OG * 16), rem = e - h * Cin * OG * 16;
    const int c = rem / (OG * 16), rem2 = rem - c * OG * 16, k = rem2 / 16, q = rem2 % 16;
    Ws[e] = k < og ? W[(((int64_t)h * Cout + o0 + k) * Cin + c) * 16 + q] : mk<T>((T)0, (T)0);
  }
  __syncthreads();
  const int s = (int)(blockIdx.x / (unsigned)nb) * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  const int64_t n = g.n();
  int cc[4];
  g.coords(s, cc);
  C<T> acc[OG][12];
#pragma unroll
  for (int k = 0; k < OG; ++k)
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[k][i] = mk<T>((T)0, (T)0);
  for (int c = 0; c < Cin; ++c) {
    const C<T> *psi = in + ((int64_t)b * Cin + c) * n;
    for (int h = 0; h < 9; ++h) {
      C<T> t[12];
      transported<T>(psi, U, g, s, cc, h, t);
#pragma unroll
      for (int k = 0; k < OG; ++k) {
        const C<T> *w = Ws + ((h * Cin + c) * OG + k) * 16;
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
          for (int sq = 0; sq < 4; ++sq) {
            const C<T> wv = w[sp * 4 + sq];
#pragma unroll
            for (int a = 0; a < 3; ++a) acc[k][sp * 3 + a] = cfma(wv, t[sq * 3 + a], acc[k][sp * 3 + a]);
          }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < OG; ++k) {
    if (k < og) {
      store_fine_site<T>(out + ((int64_t)b * Cout + o0 + k) * n, s, g.V, acc[k]);
    }
  }
}

// adjoint: out[c](x) = sum_o sum_h W[h][o][c]^H (T_rev(h) gin[o])(x)
template <typename T>
__global__ void __launch_bounds__(128) glayer_adjoint_kernel(const C<T> *__restrict__ gin,
                                                             C<T> *__restrict__ out,
                                                             const C<T> *__restrict__ W,
                                                             const C<T> *__restrict__ U, Geom g,
                                                             int Cin, int Cout, int nb) {
  extern __shared__ unsigned char smem_raw[];
  C<T> *Ws = reinterpret_cast<C<T> *>(smem_raw);  // [h][o][16] for this c
  // blockIdx.x = (site range, sample), the sample fastest (as the forward)
  const int c = blockIdx.y, b = (int)(blockIdx.x % (unsigned)nb);
  for (int e = threadIdx.x; e < 9 * Cout * 16; e += blockDim.x) {
    const int h = e / (Cout * 16), rem = e - h * Cout * 16, o = rem / 16, k = rem % 16;
    Ws[e] = W[(((int64_t)h * Cout + o) * Cin + c) * 16 + k];
  }
  __syncthreads();
  const int s = (int)(blockIdx.x / (unsigned)nb) * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  const int64_t n = g.n();
  int cc[4];
  g.coords(s, cc);
  C<T> acc[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) acc[i] = mk<T>((T)0, (T)0);
  for (int o = 0; o < Cout; ++o) {
    const C<T> *gp = gin + ((int64_t)b * Cout + o) * n;
    for (int h = 0; h < 9; ++h) {
      const int hr = h == 0 ? 0 : ((h & 1) ? h + 1 : h - 1);
      C<T> t[12];
      transported<T>(gp, U, g, s, cc, hr, t);
      const C<T> *w = Ws + (h * Cout + o) * 16;
#pragma unroll
      for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int sq = 0; sq < 4; ++sq) {
          const C<T> wv = w[sq * 4 + sp];  // (W^H)[sp][sq] = conj(W[sq][sp])
#pragma unroll
          for (int a = 0; a < 3; ++a) acc[sp * 3 + a] = cfmac(wv, t[sq * 3 + a], acc[sp * 3 + a]);
        }
    }
  }
  C<T> *o_ = out + ((int64_t)b * Cin + c) * n;
#pragma unroll
  for (int i = 0; i < 12; ++i) o_[fidx<kSoa<T>>(s, i, g.V)] = acc[i];
}

__device__ __forceinline__ double2 warp_sum2(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// weight-gradient partials: block (chunk, c*9 + h, o) sums over its sites
// and all samples g[o](x) (T_h psi[c])(x)^H (16 spin entries, colour summed)
template <typename T>
__global__ void __launch_bounds__(256) glayer_wgrad_kernel(const C<T> *__restrict__ gin,
                                                           const C<T> *__restrict__ in,
                                                           const C<T> *__restrict__ U, Geom g,
                                                           int Cin, int Cout, int B, int chunk,
                                                           double2 *__restrict__ partial) {
  __shared__ double2 sh[16][8];
  const int ch = blockIdx.y / 9, h = blockIdx.y % 9, o = blockIdx.z;
  const int64_t n = g.n();
  C<T> acc[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) acc[k] = mk<T>((T)0, (T)0);
  const int beg = blockIdx.x * chunk, end = min(g.V, beg + chunk);
  for (int s = beg + threadIdx.x; s < end; s += blockDim.x) {
    int cc[4];
    g.coords(s, cc);
    for (int b = 0; b < B; ++b) {
      C<T> t[12];
      transported<T>(in + ((int64_t)b * Cin + ch) * n, U, g, s, cc, h, t);
      const C<T> *gp = gin + ((int64_t)b * Cout + o) * n;
      C<T> gv[12];
#pragma unroll
      for (int i = 0; i < 12; ++i) gv[i] = gp[fidx<kSoa<T>>(s, i, g.V)];
#pragma unroll
      for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int sq = 0; sq < 4; ++sq)
#pragma unroll
          for (int a = 0; a < 3; ++a)
            acc[sp * 4 + sq] = cfmac(t[sq * 3 + a], gv[sp * 3 + a], acc[sp * 4 + sq]);  // g conj(t)
    }
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    double2 v = warp_sum2(make_double2((double)acc[k].x, (double)acc[k].y));
    if (l == 0) sh[k][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < 16) {
    double2 t = make_double2(0.0, 0.0);
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      t.x += sh[threadIdx.x][i].x;
      t.y += sh[threadIdx.x][i].y;
    }
    // layout [chunk][h][o][c][16]
    partial[((((int64_t)blockIdx.x * 9 + h) * Cout + o) * Cin + ch) * 16 + threadIdx.x] = t;
  }
}

__global__ void wgrad_sum_kernel(const double2 *__restrict__ partial, int nchunks, int64_t count,
                                 double2 *__restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    double2 t = make_double2(0.0, 0.0);
    for (int k = 0; k < nchunks; ++k) {
      const double2 p = partial[(int64_t)k * count + e];
      t.x += p.x;
      t.y += p.y;
    }
    out[e] = t;
  }
}

// Adam on the real and imaginary parts of every complex weight; grad holds
// dL/dW* (so the real-parameter gradient is 2 grad); scale divides the
// accumulated gradient (batch mean).
__global__ void adam_kernel(double2 *__restrict__ W, const double2 *__restrict__ grad,
                            double2 *__restrict__ m, double2 *__restrict__ v, int64_t count,
                            double lr, double b1, double b2, double epsv, double bc1, double bc2,
                            double scale) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double gx = 2.0 * grad[e].x * scale, gy = 2.0 * grad[e].y * scale;
    double2 mm = m[e], vv = v[e];
    mm.x = b1 * mm.x + (1 - b1) * gx;
    mm.y = b1 * mm.y + (1 - b1) * gy;
    vv.x = b2 * vv.x + (1 - b2) * gx * gx;
    vv.y = b2 * vv.y + (1 - b2) * gy * gy;
    m[e] = mm;
    v[e] = vv;
    double2 w = W[e];
    w.x -= lr * (mm.x / bc1) / (sqrt(vv.x / bc2) + epsv);
    w.y -= lr * (mm.y / bc1) / (sqrt(vv.y / bc2) + epsv);
    W[e] = w;
  }
}

}  // namespace

template <typename T, int OG>
static void glayer_forward_og(const C<T> *in, C<T> *out, const C<T> *W, const C<T> *U, Geom g, int Cin,
                              int Cout, int B, cudaStream_t s) {
  const size_t sm = (size_t)9 * Cin * OG * 16 * sizeof(C<T>);
  smem_optin((const void *)glayer_forward_kernel<T, OG>, 160 * 1024);
  glayer_forward_kernel<T, OG><<<dim3((unsigned)div_up(g.V, 128) * (unsigned)B, div_up(Cout, OG), 1), 128, sm,
                                 s>>>(in, out, W, U, g, Cin, Cout, B);
  MG_LAUNCH_CHECK();
}

template <typename T>
void glayer_forward(const C<T> *in, C<T> *out, const C<T> *W, const C<T> *U, Geom g, int Cin,
                    int Cout, int B, cudaStream_t s) {
  if (Cout == 1) glayer_forward_og<T, 1>(in, out, W, U, g, Cin, Cout, B, s);
  else if (Cout == 2) glayer_forward_og<T, 2>(in, out, W, U, g, Cin, Cout, B, s);
  else glayer_forward_og<T, 4>(in, out, W, U, g, Cin, Cout, B, s);
}

template <typename T>
void glayer_adjoint(const C<T> *gin, C<T> *out, const C<T> *W, const C<T> *U, Geom g, int Cin,
                    int Cout, int B, cudaStream_t s) {
  const size_t sm = (size_t)9 * Cout * 16 * sizeof(C<T>);
  smem_optin((const void *)glayer_adjoint_kernel<T>, 100 * 1024);
  glayer_adjoint_kernel<T><<<dim3((unsigned)div_up(g.V, 128) * (unsigned)B, Cin, 1), 128, sm, s>>>(gin, out, W, U,
                                                                                                  g, Cin, Cout, B);
  MG_LAUNCH_CHECK();
}

int glayer_wgrad_chunks(const Geom &g) {
  const int chunk = 4096;
  return div_up(g.V, chunk);
}

template <typename T>
void glayer_wgrad(const C<T> *gin, const C<T> *in, const C<T> *U, Geom g, int Cin, int Cout, int B,
                  double2 *partial, double2 *out, cudaStream_t s) {
  const int chunk = 4096;
  const int nchunks = div_up(g.V, chunk);
  glayer_wgrad_kernel<T><<<dim3(nchunks, Cin * 9, Cout), 256, 0, s>>>(gin, in, U, g, Cin, Cout, B, chunk,
                                                                        partial);
  MG_LAUNCH_CHECK();
  const int64_t count = (int64_t)9 * Cout * Cin * 16;
  wgrad_sum_kernel<<<grid_for(count), 256, 0, s>>>(partial, nchunks, count, out);
  MG_LAUNCH_CHECK();
}

void adam_step(double2 *W, const double2 *grad, double2 *m, double2 *v, int64_t count, double lr,
               double b1, double b2, double eps, int t, double scale, cudaStream_t s) {
  const double bc1 = 1.0 - pow(b1, t), bc2 = 1.0 - pow(b2, t);
  adam_kernel<<<grid_for(count), 256, 0, s>>>(W, grad, m, v, count, lr, b1, b2, eps, bc1, bc2, scale);
  MG_LAUNCH_CHECK();
}

#define INST(T)                                                                                 \
  template void glayer_forward<T>(const C<T> *, C<T> *, const C<T> *, const C<T> *, Geom, int,  \
                                  int, int, cudaStream_t);                                      \
  template void glayer_adjoint<T>(const C<T> *, C<T> *, const C<T> *, const C<T> *, Geom, int,  \
                                  int, int, cudaStream_t);                                      \
  template void glayer_wgrad<T>(const C<T> *, const C<T> *, const C<T> *, Geom, int, int, int,  \
                                double2 *, double2 *, cudaStream_t);
INST(double)
INST(float)

}  // namespace mg
