// Learned initialiser (no counterpart in the paper): forward and backward
// kernels of  x -> relu(W1 x + b1) -> relu(W2 . + b2) -> reshape 16x4^3 -> convT(16->16) -> relu
// -> convT(16->8) -> relu -> convT(8->2) -> 32^3 x 2,  convT = 3D transposed convolution with
// kernel 4, stride 2, padding 1:  out[co][o] = b[co] + sum_ci sum_k in[ci][i] w[ci][co][k],
// o = 2 i - 1 + k per axis.  W1, W2 are read as BF16, everything accumulates in FP32.  All
// reductions are deterministic (fixed per-thread order, fixed trees, no atomics).
#include <cuda_bf16.h>

#include <algorithm>

#include "k_nn.h"
#include "mw_internal.h"

namespace mwk {
namespace {

constexpr int TM = 64, TN = 64, TK = 16;

template <typename TB>
__device__ __forceinline__ float ldb(const TB* p) {
  return (float)*p;
}
template <>
__device__ __forceinline__ float ldb<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}

// C[m][n] = sum_k A(m, k) B(k, n) (+ bias[n]); A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn].
// Optional ReLU copy H.  64 x 64 tiles, 4 x 4 outputs per thread.  Split K: the CTA of
// blockIdx.z sums k in [z kchunk, (z + 1) kchunk) and, when P is given, writes its partial
// sums to P[z][m][n] for gemm_reduce_kernel (bias and ReLU are applied there).
template <typename TB>
__global__ void __launch_bounds__(256) gemm_kernel(const float* __restrict__ A, int64_t sam, int64_t sak,
                                                   const TB* __restrict__ B, int64_t sbk, int64_t sbn,
                                                   const float* __restrict__ bias, float* __restrict__ C,
                                                   float* __restrict__ H, int M, int N, int Kfull, int kchunk,
                                                   float* __restrict__ P) {
  __shared__ float As[TK][TM + 1];
  __shared__ float Bs[TK][TN + 1];
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
  const int kbeg = blockIdx.z * kchunk, Kd = min(Kfull, kbeg + kchunk);
  float acc[4][4] = {};
  for (int k0 = kbeg; k0 < Kd; k0 += TK) {
    for (int e = threadIdx.x; e < TK * TM; e += 256) {
      // consecutive threads walk the contiguous axis of each operand
      int k, m;
      if (sak == 1) {
        k = e % TK;
        m = e / TK;
      } else {
        m = e % TM;
        k = e / TM;
      }
      const int gm = m0 + m, gk = k0 + k;
      As[k][m] = (gm < M && gk < Kd) ? A[(int64_t)gm * sam + (int64_t)gk * sak] : 0.f;
    }
    for (int e = threadIdx.x; e < TK * TN; e += 256) {
      int k, n;
      if (sbk == 1) {
        k = e % TK;
        n = e / TK;
      } else {
        n = e % TN;
        k = e / TN;
      }
      const int gn = n0 + n, gk = k0 + k;
      Bs[k][n] = (gn < N && gk < Kd) ? ldb(B + (int64_t)gk * sbk + (int64_t)gn * sbn) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < TK; ++k) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][tr + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tc + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + tr + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tc + 16 * j;
      if (gn >= N) continue;
      if (P) {
        P[((int64_t)blockIdx.z * M + gm) * N + gn] = acc[i][j];
        continue;
      }
      const float v = acc[i][j] + (bias ? bias[gn] : 0.f);
      C[(int64_t)gm * N + gn] = v;
      if (H) H[(int64_t)gm * N + gn] = v > 0.f ? v : 0.f;
    }
  }
}

// C = sum_z P[z] (z ascending) + bias, H = relu(C).
__global__ void gemm_reduce_kernel(const float* __restrict__ P, int nz, const float* __restrict__ bias,
                                   float* __restrict__ C, float* __restrict__ H, int M, int N) {
  const int64_t MN = (int64_t)M * N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < MN; i += (int64_t)gridDim.x * blockDim.x) {
    float v = 0.f;
    for (int z = 0; z < nz; ++z) v += P[z * MN + i];
    if (bias) v += bias[i % N];
    C[i] = v;
    if (H) H[i] = v > 0.f ? v : 0.f;
  }
}

// Column sums of dZ [B][N] -> db [N] (fixed order).
__global__ void colsum_kernel(const float* __restrict__ dz, int B, int N, float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += dz[(int64_t)b * N + n];
  db[n] = s;
}

__global__ void relu_back_kernel(const float* __restrict__ z, const float* __restrict__ dh, float* __restrict__ dz,
                                 int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dz[i] = z[i] > 0.f ? dh[i] : 0.f;
}

// convT forward, gather form: one thread per output position (b, o), all Co channels at once;
// per axis the inputs i with o = 2i - 1 + k are i = (o + 1 - k) / 2 for the two k of matching
// parity.  The layer's weights sit in shared memory; every input value is read once per output
// position.  Per output the sum runs over ci, then kz, ky, kx ascending.
template <int CO>
__global__ void __launch_bounds__(256) convT_fwd_kernel(const float* __restrict__ x, const float* __restrict__ w,
                                                        const float* __restrict__ b, float* __restrict__ a,
                                                        float* __restrict__ g, int B, int Ci, int D) {
  extern __shared__ float sw[];                     // [Ci][CO][64]
  for (int q = threadIdx.x; q < Ci * CO * 64; q += blockDim.x) sw[q] = w[q];
  __syncthreads();
  const int Do = 2 * D;
  const int64_t V = (int64_t)Do * Do * Do;
  const int64_t total = (int64_t)B * V;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = t % V;
    const int bb = (int)(t / V);
    const int ox = (int)(o % Do), oy = (int)((o / Do) % Do), oz = (int)(o / ((int64_t)Do * Do));
    float s[CO];
#pragma unroll
    for (int co = 0; co < CO; ++co) s[co] = b[co];
    for (int ci = 0; ci < Ci; ++ci) {
      const float* xc = x + ((int64_t)bb * Ci + ci) * D * D * D;
      const float* wc = sw + ci * CO * 64;
      for (int kz = (oz + 1) & 1; kz < 4; kz += 2) {
        const int iz = (oz + 1 - kz) >> 1;
        if (iz < 0 || iz >= D) continue;
        for (int ky = (oy + 1) & 1; ky < 4; ky += 2) {
          const int iy = (oy + 1 - ky) >> 1;
          if (iy < 0 || iy >= D) continue;
          for (int kx = (ox + 1) & 1; kx < 4; kx += 2) {
            const int ix = (ox + 1 - kx) >> 1;
            if (ix < 0 || ix >= D) continue;
            const float xv = xc[(iz * D + iy) * D + ix];
            const int kk = (kz * 4 + ky) * 4 + kx;
#pragma unroll
            for (int co = 0; co < CO; ++co) s[co] = fmaf(xv, wc[co * 64 + kk], s[co]);
          }
        }
      }
    }
#pragma unroll
    for (int co = 0; co < CO; ++co) {
      const int64_t idx = ((int64_t)bb * CO + co) * V + o;
      a[idx] = s[co];
      if (g) g[idx] = s[co] > 0.f ? s[co] : 0.f;
    }
  }
}

// convT backward-data: dx[b][ci][i] = sum_co sum_k w[ci][co][k] dy[b][co][2i - 1 + k]; one thread
// per input position (b, i) and group of CIG channels (the group is blockIdx.y, so layers with
// few positions still fill the GPU), the group's weights in shared memory.  Per output the sum
// runs over co, then kz, ky, kx ascending.
template <int CIG>
__global__ void __launch_bounds__(256) convT_bwd_data_kernel(const float* __restrict__ dy,
                                                             const float* __restrict__ w, float* __restrict__ dx,
                                                             int B, int Co, int D, int Ci) {
  extern __shared__ float sw[];                     // [CIG][Co][64] of channels ci0 ..
  const int ci0 = blockIdx.y * CIG;
  for (int q = threadIdx.x; q < CIG * Co * 64; q += blockDim.x) sw[q] = w[(size_t)ci0 * Co * 64 + q];
  __syncthreads();
  const int Do = 2 * D;
  const int64_t V = (int64_t)D * D * D;
  const int64_t total = (int64_t)B * V;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % V;
    const int bb = (int)(t / V);
    const int ix = (int)(i % D), iy = (int)((i / D) % D), iz = (int)(i / ((int64_t)D * D));
    float s[CIG];
#pragma unroll
    for (int ci = 0; ci < CIG; ++ci) s[ci] = 0.f;
    for (int co = 0; co < Co; ++co) {
      const float* yc = dy + ((int64_t)bb * Co + co) * Do * Do * Do;
      for (int kz = 0; kz < 4; ++kz) {
        const int oz = 2 * iz - 1 + kz;
        if (oz < 0 || oz >= Do) continue;
        for (int ky = 0; ky < 4; ++ky) {
          const int oy = 2 * iy - 1 + ky;
          if (oy < 0 || oy >= Do) continue;
          for (int kx = 0; kx < 4; ++kx) {
            const int ox = 2 * ix - 1 + kx;
            if (ox < 0 || ox >= Do) continue;
            const float yv = yc[(oz * Do + oy) * Do + ox];
            const int kk = (kz * 4 + ky) * 4 + kx;
#pragma unroll
            for (int ci = 0; ci < CIG; ++ci) s[ci] = fmaf(yv, sw[(ci * Co + co) * 64 + kk], s[ci]);
          }
        }
      }
    }
#pragma unroll
    for (int ci = 0; ci < CIG; ++ci) dx[((int64_t)bb * Ci + ci0 + ci) * V + i] = s[ci];
  }
}

// convT backward-weights, dW[ci][co][k] = sum_b sum_i x[b][ci][i] dy[b][co][2i - 1 + k], in two
// fixed-order passes.  Pass 1: block (ci, co, kz, chunk) walks its chunk of the B D^3 input
// positions for the 16 taps of one kz plane; thread t takes positions t, t + 256, ... and keeps
// the 16 tap sums in registers; the block then sums the 256 threads' values tap by tap (thread
// order, through shared memory) into part[chunk][ci][co][k].
// Pass 2 sums the chunks in order.
constexpr int kBwdWThreads = 256;
__global__ void __launch_bounds__(kBwdWThreads) convT_bwd_w_kernel(const float* __restrict__ x,
                                                                   const float* __restrict__ dy,
                                                                   float* __restrict__ part, int B, int Ci, int Co,
                                                                   int D, int64_t chunk) {
  __shared__ float red[kBwdWThreads][17];
  const int pair = blockIdx.x >> 2, kz = blockIdx.x & 3;
  const int ci = pair / Co, co = pair % Co;
  const int Do = 2 * D;
  const int64_t V = (int64_t)D * D * D, total = (int64_t)B * V;
  const int64_t p0 = (int64_t)blockIdx.y * chunk, p1 = min(total, p0 + chunk);
  float acc[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) acc[k] = 0.f;
  for (int64_t t = p0 + threadIdx.x; t < p1; t += kBwdWThreads) {
    const int64_t i = t % V;
    const int bb = (int)(t / V);
    const int ix = (int)(i % D), iy = (int)((i / D) % D), iz = (int)(i / ((int64_t)D * D));
    const int oz = 2 * iz - 1 + kz;
    if (oz < 0 || oz >= Do) continue;
    const float xv = x[((int64_t)bb * Ci + ci) * V + i];
    const float* yc = dy + ((int64_t)bb * Co + co) * Do * Do * Do + (int64_t)oz * Do * Do;
#pragma unroll
    for (int ky = 0; ky < 4; ++ky) {
      const int oy = 2 * iy - 1 + ky;
#pragma unroll
      for (int kx = 0; kx < 4; ++kx) {
        const int ox = 2 * ix - 1 + kx;
        if (oy >= 0 && oy < Do && ox >= 0 && ox < Do)
          acc[ky * 4 + kx] = fmaf(xv, yc[(int64_t)oy * Do + ox], acc[ky * 4 + kx]);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) red[threadIdx.x][k] = acc[k];
  __syncthreads();
  if (threadIdx.x < 16) {
    float sum = 0.f;
    for (int q = 0; q < kBwdWThreads; ++q) sum += red[q][threadIdx.x];
    part[(((int64_t)blockIdx.y * Ci + ci) * Co + co) * 64 + kz * 16 + threadIdx.x] = sum;
  }
}

// dw[q] = sum over chunks of part[chunk][q] (chunk order), q over Ci Co 64.
__global__ void convT_bwd_w_final_kernel(const float* __restrict__ part, int nchunk, int64_t n, float* __restrict__ dw) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  float s = 0.f;
  for (int c = 0; c < nchunk; ++c) s += part[(int64_t)c * n + q];
  dw[q] = s;
}

// per-channel sums of dy [B][Co][V] -> db [Co] in two fixed-order passes: block (co, b) writes
// the tree sum of its (channel, sample) slab to part[co][b]; then db[co] = sum_b part[co][b].
__global__ void chansum_kernel(const float* __restrict__ dy, int B, int Co, int64_t V, float* __restrict__ part) {
  __shared__ float red[256];
  const int co = blockIdx.x, b = blockIdx.y;
  float s = 0.f;
  for (int64_t v = threadIdx.x; v < V; v += 256) s += dy[((int64_t)b * Co + co) * V + v];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[co * B + b] = red[0];
}

__global__ void chansum_final_kernel(const float* __restrict__ part, int B, int Co, float* __restrict__ db) {
  const int co = blockIdx.x * blockDim.x + threadIdx.x;
  if (co >= Co) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += part[co * B + b];
  db[co] = s;
}

// MSE: dy = 2 (y - t) / n, per-block partial sums of (y - t)^2 in FP64.
__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ t, int64_t n, float* __restrict__ dy,
                           double* __restrict__ part) {
  __shared__ double red[256];
  double s = 0.0;
  const float sc = 2.0f / (float)n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    dy[i] = sc * d;
    s += (double)d * d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void sum_parts_kernel(const double* __restrict__ part, int n, double scale, double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] * scale;
}

// Adam (Kingma & Ba) with bias correction; bc1 = 1 - b1^t, bc2 = 1 - b2^t.
__global__ void adam_kernel(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float bc1,
                            float bc2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16_rn(a[i]);
}

__global__ void gather_rows_kernel(const float* __restrict__ src, const int32_t* __restrict__ idx, int n,
                                   int64_t width, float* __restrict__ dst) {
  const int64_t total = (int64_t)n * width;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / width, c = t % width;
    dst[t] = src[(int64_t)idx[r] * width + c];
  }
}

// Mean over the 35 points of the order-4 barycentric lattice of each tet (points
// (i v0 + j v1 + k v2 + l v3) / 4, i + j + k + l = 4) of the trilinear interpolant of a
// cell-centred [2][G][G][G] grid over box [lo, hi] (0 outside the box): an average of the grid
// over the tet.  out [T][2] += (Re, Im).
__global__ void grid_to_tets_kernel(const float* __restrict__ grid, int G, double lx, double ly, double lz, double hx,
                                    double hy, double hz, const double* __restrict__ xyz,
                                    const int32_t* __restrict__ tets, int64_t T, double* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  double v[4][3];
  for (int a = 0; a < 4; ++a)
    for (int d = 0; d < 3; ++d) v[a][d] = xyz[3 * (int64_t)tets[4 * t + a] + d];
  const double lo[3] = {lx, ly, lz}, hi[3] = {hx, hy, hz};
  double acc0 = 0.0, acc1 = 0.0;
  for (int i = 0; i <= 4; ++i)
    for (int j = 0; i + j <= 4; ++j)
      for (int k = 0; i + j + k <= 4; ++k) {
        const int l = 4 - i - j - k;
        double c[3];
        for (int d = 0; d < 3; ++d) c[d] = (i * v[0][d] + j * v[1][d] + k * v[2][d] + l * v[3][d]) * 0.25;
        bool in = true;
        double f[3];
        int i0[3];
        for (int d = 0; d < 3; ++d) {
          if (c[d] < lo[d] || c[d] > hi[d]) in = false;
          const double u = (c[d] - lo[d]) / (hi[d] - lo[d]) * G - 0.5;
          double fl = floor(u);
          fl = fmin(fmax(fl, 0.0), (double)(G - 2));
          i0[d] = (int)fl;
          f[d] = fmin(fmax(u - fl, 0.0), 1.0);
        }
        if (!in) continue;
        for (int dz = 0; dz < 2; ++dz)
          for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
              const double wgt = (dz ? f[2] : 1 - f[2]) * (dy ? f[1] : 1 - f[1]) * (dx ? f[0] : 1 - f[0]);
              const int64_t cell = ((int64_t)(i0[2] + dz) * G + i0[1] + dy) * G + i0[0] + dx;
              acc0 += wgt * grid[cell];
              acc1 += wgt * grid[(int64_t)G * G * G + cell];
            }
      }
  out[2 * t] += acc0 / 35.0;
  out[2 * t + 1] += acc1 / 35.0;
}

inline int gsb(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

}  // namespace

// K chunks for a GEMM of `tiles` 64x64 tiles: enough CTAs for two per SM, chunks of at least
// 256 along K, a whole number of TK steps, and the partials within the workspace.
static int k_splits(int tiles, int M, int N, int K, size_t ws_floats, int& kchunk) {
  int z = std::max(1, std::min(K / 256, (2 * 152 + tiles - 1) / tiles));
  while (z > 1 && (size_t)z * M * N > ws_floats) --z;
  kchunk = ((K + z - 1) / z + TK - 1) / TK * TK;
  return (K + kchunk - 1) / kchunk;
}

template <typename TB>
static void gemm_launch(const float* A, int64_t sam, int64_t sak, const TB* B, int64_t sbk, int64_t sbn,
                        const float* bias, float* C, float* H, int M, int N, int K, float* ws, size_t ws_floats,
                        cudaStream_t s) {
  const int tiles = ((N + TN - 1) / TN) * ((M + TM - 1) / TM);
  int kchunk = K;
  const int z = ws ? k_splits(tiles, M, N, K, ws_floats, kchunk) : 1;
  dim3 g((N + TN - 1) / TN, (M + TM - 1) / TM, z);
  if (z == 1) {
    note_launch(1);
    gemm_kernel<TB><<<g, 256, 0, s>>>(A, sam, sak, B, sbk, sbn, bias, C, H, M, N, K, K, nullptr);
    return;
  }
  note_launch(2);
  gemm_kernel<TB><<<g, 256, 0, s>>>(A, sam, sak, B, sbk, sbn, bias, C, H, M, N, K, kchunk, ws);
  const int64_t MN = (int64_t)M * N;
  gemm_reduce_kernel<<<(int)std::min<int64_t>((MN + 255) / 256, 152 * 8), 256, 0, s>>>(ws, z, bias, C, H, M, N);
}

void nn_gemm_bf16(const float* A, int64_t sam, int64_t sak, const void* Bw, int64_t sbk, int64_t sbn,
                  const float* bias, float* C, float* H, int M, int N, int K, cudaStream_t s, float* ws,
                  size_t ws_floats) {
  gemm_launch<__nv_bfloat16>(A, sam, sak, (const __nv_bfloat16*)Bw, sbk, sbn, bias, C, H, M, N, K, ws, ws_floats, s);
}
void nn_gemm_f32(const float* A, int64_t sam, int64_t sak, const float* Bf, int64_t sbk, int64_t sbn,
                 const float* bias, float* C, float* H, int M, int N, int K, cudaStream_t s, float* ws,
                 size_t ws_floats) {
  gemm_launch<float>(A, sam, sak, Bf, sbk, sbn, bias, C, H, M, N, K, ws, ws_floats, s);
}
void nn_colsum(const float* dz, int B, int N, float* db, cudaStream_t s) {
  note_launch(1);
  colsum_kernel<<<(N + 255) / 256, 256, 0, s>>>(dz, B, N, db);
}
void nn_relu_back(const float* z, const float* dh, float* dz, int64_t n, cudaStream_t s) {
  note_launch(1);
  relu_back_kernel<<<gsb(n), 256, 0, s>>>(z, dh, dz, n);
}
// The transposed convolutions keep a layer's weights (up to 16 x 16 x 64 floats, 64 KB) in
// dynamic shared memory.
static void allow_conv_smem() {
  static bool done = false;
  if (done) return;
  const int sm = 16 * 16 * 64 * (int)sizeof(float);
  cudaFuncSetAttribute(convT_fwd_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(convT_fwd_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(convT_fwd_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(convT_bwd_data_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(convT_bwd_data_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(convT_bwd_data_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  done = true;
}

void nn_convT_fwd(const float* x, const float* w, const float* b, float* a, float* g, int B, int Ci, int Co, int D,
                  cudaStream_t s) {
  allow_conv_smem();
  note_launch(1);
  const int64_t n = (int64_t)B * 8 * D * D * D;
  const size_t sm = sizeof(float) * Ci * Co * 64;
  switch (Co) {
    case 2:
      convT_fwd_kernel<2><<<gsb(n), 256, sm, s>>>(x, w, b, a, g, B, Ci, D);
      break;
    case 8:
      convT_fwd_kernel<8><<<gsb(n), 256, sm, s>>>(x, w, b, a, g, B, Ci, D);
      break;
    default:
      convT_fwd_kernel<16><<<gsb(n), 256, sm, s>>>(x, w, b, a, g, B, Ci, D);
      break;
  }
}
void nn_convT_bwd(const float* x, const float* w, const float* dy, float* dx, float* dw, float* db, int B, int Ci,
                  int Co, int D, float* part, float* wpart, cudaStream_t s) {
  allow_conv_smem();
  note_launch(dx ? 5 : 4);
  if (dx) {
    // channel groups so that every layer launches about two waves of blocks
    const int64_t n = (int64_t)B * D * D * D;
    const int nb = gsb(n);
    const int cig = nb * (Ci / 8) >= 2 * 152 ? 8 : (nb * (Ci / 4) >= 2 * 152 ? 4 : 1);
    const dim3 grid((unsigned)nb, (unsigned)(Ci / cig));
    const size_t sm = sizeof(float) * cig * Co * 64;
    if (cig == 8)
      convT_bwd_data_kernel<8><<<grid, 256, sm, s>>>(dy, w, dx, B, Co, D, Ci);
    else if (cig == 4)
      convT_bwd_data_kernel<4><<<grid, 256, sm, s>>>(dy, w, dx, B, Co, D, Ci);
    else
      convT_bwd_data_kernel<1><<<grid, 256, sm, s>>>(dy, w, dx, B, Co, D, Ci);
  }
  {
    // enough (ci, co, chunk) blocks for every SM twice, chunks of whole thread rounds, at most
    // kConvChunks chunks (the workspace holds kConvChunks x Ci x Co x 64 partial sums)
    const int64_t total = (int64_t)B * D * D * D;
    int nchunk = (int)std::min<int64_t>(kConvChunks, std::max<int64_t>(1, (2 * 152 + Ci * Co - 1) / (Ci * Co)));
    int64_t chunk = (total + nchunk - 1) / nchunk;
    chunk = (chunk + kBwdWThreads - 1) / kBwdWThreads * kBwdWThreads;
    nchunk = (int)((total + chunk - 1) / chunk);
    convT_bwd_w_kernel<<<dim3(Ci * Co * 4, nchunk), kBwdWThreads, 0, s>>>(x, dy, wpart, B, Ci, Co, D, chunk);
    const int64_t n = (int64_t)Ci * Co * 64;
    convT_bwd_w_final_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(wpart, nchunk, n, dw);
  }
  chansum_kernel<<<dim3(Co, B), 256, 0, s>>>(dy, B, Co, (int64_t)8 * D * D * D, part);
  chansum_final_kernel<<<1, 32, 0, s>>>(part, B, Co, db);
}
void nn_mse(const float* y, const float* t, int64_t n, float* dy, double* part, double* loss, cudaStream_t s) {
  note_launch(2);
  const int nb = 256;
  mse_kernel<<<nb, 256, 0, s>>>(y, t, n, dy, part);
  sum_parts_kernel<<<1, 256, 0, s>>>(part, nb, 1.0 / (double)n, loss);
}
void nn_adam(float* th, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2, float eps, int step,
             cudaStream_t s) {
  note_launch(1);
  const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<gsb(n), 256, 0, s>>>(th, g, m, v, n, lr, b1, b2, eps, bc1, bc2);
}
void nn_to_bf16(const float* a, void* b, int64_t n, cudaStream_t s) {
  note_launch(1);
  to_bf16_kernel<<<gsb(n), 256, 0, s>>>(a, (__nv_bfloat16*)b, n);
}
void nn_gather_rows(const float* src, const int32_t* idx, int n, int64_t width, float* dst, cudaStream_t s) {
  note_launch(1);
  gather_rows_kernel<<<gsb((int64_t)n * width), 256, 0, s>>>(src, idx, n, width, dst);
}
void nn_grid_to_tets(const float* grid, int G, const double* box, const double* xyz, const int32_t* tets, int64_t T,
                     double* out, cudaStream_t s) {
  note_launch(1);
  grid_to_tets_kernel<<<(unsigned)((T + 127) / 128), 128, 0, s>>>(grid, G, box[0], box[1], box[2], box[3], box[4],
                                                                   box[5], xyz, tets, T, out);
}

}  // namespace mwk
