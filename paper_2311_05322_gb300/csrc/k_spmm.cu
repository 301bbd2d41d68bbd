// K3: complex SpMM Y = A X over a block of R right-hand sides stored edge-major with the RHS
// index fastest ([E][R]), so the threads of one row read one contiguous span of X per nonzero.
// Threads of a row split the R columns (CPL consecutive columns each); rows are spread over
// the grid.  FP64 variant (FP64 arithmetic) and FP32 variant (FP32 arithmetic, FP32 accumulate).
#include "mw_internal.h"

namespace mwk {
namespace {

template <typename T>
struct Cx;
template <>
struct Cx<double2> {
  using S = double;
};
template <>
struct Cx<float2> {
  using S = float;
};

template <typename T>
__device__ __forceinline__ void cmac(T& acc, T a, T x) {
  acc.x = fma(a.x, x.x, acc.x);
  acc.x = fma(-a.y, x.y, acc.x);
  acc.y = fma(a.x, x.y, acc.y);
  acc.y = fma(a.y, x.x, acc.y);
}

// Stored X value as the arithmetic type: itself, or a complex BF16 pair (real in the low half)
// widened to complex FP32.
template <typename T>
__device__ __forceinline__ T xval(T v) {
  return v;
}
__device__ __forceinline__ float2 xval(uint32_t u) {
  return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}

// A row's terms are taken in batches of NB: the NB column indices, then the NB gathers of X (all
// in flight together), then the complex FMAs in term order.  The gathers are latency-bound
// (about 16 terms per row, each a 128-256 byte row of X), so the batch raises the loads in
// flight per warp; the sums keep the canonical term order.  XT is the stored type of X: T, or
// uint32_t for complex BF16 pairs (T = float2).
template <typename T, int CPL, typename XT = T>
__global__ void __launch_bounds__(512) spmm_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                   const T* __restrict__ A, const XT* __restrict__ X, T* __restrict__ Y,
                                                   int64_t E, int R, int tpr_log2) {
  constexpr int NB = 8 / CPL;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t row = g >> tpr_log2;
  const int c0 = (int)(g & ((1 << tpr_log2) - 1)) * CPL;
  if (row >= E || c0 >= R) return;
  T acc[CPL];
#pragma unroll
  for (int q = 0; q < CPL; ++q) acc[q] = T{0, 0};
  const int64_t b = rp[row], e = rp[row + 1];
  int64_t k = b;
  for (; k + NB <= e; k += NB) {
    int cc[NB];
    XT xv[NB][CPL];
#pragma unroll
    for (int u = 0; u < NB; ++u) cc[u] = ci[k + u];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const XT* xr = X + (int64_t)cc[u] * R + c0;
#pragma unroll
      for (int q = 0; q < CPL; ++q)
        if (c0 + q < R) xv[u][q] = xr[q];
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const T a = A[k + u];
#pragma unroll
      for (int q = 0; q < CPL; ++q)
        if (c0 + q < R) cmac(acc[q], a, xval(xv[u][q]));
    }
  }
  for (; k < e; ++k) {
    const T a = A[k];
    const XT* xr = X + (int64_t)ci[k] * R + c0;
#pragma unroll
    for (int q = 0; q < CPL; ++q)
      if (c0 + q < R) cmac(acc[q], a, xval(xr[q]));
  }
  T* yr = Y + row * R + c0;
#pragma unroll
  for (int q = 0; q < CPL; ++q)
    if (c0 + q < R) yr[q] = acc[q];
}

// r = b - A x in FP64 with per-block, per-column partial sums of |r|^2 (deterministic).  ZX: x = 0
// (the first outer step): the row sums are +0 and the row loop is skipped.
template <int CPL, bool ZX>
__global__ void __launch_bounds__(256) residual_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                       const double2* __restrict__ A, const double2* __restrict__ X,
                                                       const double2* __restrict__ B, double2* __restrict__ Rv,
                                                       double* __restrict__ part, int64_t E, int R, int tpr_log2) {
  __shared__ double red[256 * CPL];
  const int tpr = 1 << tpr_log2;
  const int rows_per_block = 256 >> tpr_log2;
  const int lane_c = threadIdx.x & (tpr - 1);
  const int c0 = lane_c * CPL;
  double nrm[CPL];
#pragma unroll
  for (int q = 0; q < CPL; ++q) nrm[q] = 0.0;
  for (int64_t row = (int64_t)blockIdx.x * rows_per_block + (threadIdx.x >> tpr_log2); row < E;
       row += (int64_t)gridDim.x * rows_per_block) {
    if (c0 >= R) continue;
    double2 acc[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) acc[q] = make_double2(0.0, 0.0);
    for (int64_t k = ZX ? 0 : rp[row]; k < (ZX ? 0 : rp[row + 1]); ++k) {
      const double2 a = A[k];
      const double2* xr = X + (int64_t)ci[k] * R + c0;
#pragma unroll
      for (int q = 0; q < CPL; ++q)
        if (c0 + q < R) cmac(acc[q], a, xr[q]);
    }
#pragma unroll
    for (int q = 0; q < CPL; ++q)
      if (c0 + q < R) {
        const double2 bb = B[row * R + c0 + q];
        const double2 r = make_double2(bb.x - acc[q].x, bb.y - acc[q].y);
        Rv[row * R + c0 + q] = r;
        nrm[q] += r.x * r.x + r.y * r.y;
      }
  }
#pragma unroll
  for (int q = 0; q < CPL; ++q) red[threadIdx.x * CPL + q] = nrm[q];
  __syncthreads();
  if ((int)threadIdx.x < tpr) {
    for (int q = 0; q < CPL; ++q) {
      const int c = c0 + q;
      if (c >= R) continue;
      double s = 0.0;
      for (int r = 0; r < rows_per_block; ++r) s += red[(r * tpr + lane_c) * CPL + q];
      part[(int64_t)blockIdx.x * R + c] = s;
    }
  }
}

struct Shape {
  int cpl, tpr_log2;
};
inline Shape shape_for(int R) {
  int cpl = (R + 31) / 32;
  if (cpl > 2) cpl = 4;
  if (cpl > 4) cpl = 4;
  int tpr = (R + cpl - 1) / cpl;
  int l = 0;
  while ((1 << l) < tpr) ++l;
  return {cpl, l};
}

template <typename T>
void spmm_launch(const int64_t* rp, const int32_t* ci, const T* A, const T* X, T* Y, int64_t E, int R,
                 cudaStream_t s, int threads) {
  if (threads != 128 && threads != 256 && threads != 512) threads = 256;
  note_launch(1);
  Shape sh = shape_for(R);
  if (R > 128) {
    // wide blocks: process 128 columns at a time is not supported by the layout; caller splits.
    return;
  }
  const int64_t nthr = E << sh.tpr_log2;
  const int blocks = (int)((nthr + threads - 1) / threads);
  switch (sh.cpl) {
    case 1:
      spmm_kernel<T, 1><<<blocks, threads, 0, s>>>(rp, ci, A, X, Y, E, R, sh.tpr_log2);
      break;
    case 2:
      spmm_kernel<T, 2><<<blocks, threads, 0, s>>>(rp, ci, A, X, Y, E, R, sh.tpr_log2);
      break;
    default:
      spmm_kernel<T, 4><<<blocks, threads, 0, s>>>(rp, ci, A, X, Y, E, R, sh.tpr_log2);
      break;
  }
}

// Halo-tiled FP32 SpMM.  One CTA takes one block of the SpMM plan (rows in Morton order whose
// column set, the halo, holds at most kHaloMax edges; at most kHaloRows rows and kHaloNnz
// nonzeros) and one chunk of kHaloCols columns.  Staging, all at the CTA's start:
//  - the halo's rows of X (kHaloCols complex values each) by 16-byte cp.async copies, 8 threads
//    per row;
//  - the block's nonzero values, halo-local columns, row offsets and row ids by coalesced loads.
// Then each half-warp computes one row from shared memory only: its 16 lanes hold 16 columns.
// A row's terms are accumulated in the canonical column order with the same complex FMA
// sequence as spmm_kernel, so both kernels give bit-identical results.
constexpr int kHaloCols = 16;
constexpr int kHaloThreads = 256;
constexpr size_t kHaloSmem = (size_t)kHaloMax * kHaloCols * 8 + (size_t)kHaloNnz * 8 + (kHaloRows + 1) * 4 +
                             (size_t)kHaloRows * 4 + (size_t)kHaloNnz * 2;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

__global__ void __launch_bounds__(kHaloThreads, 2)
    spmm_halo_kernel(const int64_t* __restrict__ blk_row, const int64_t* __restrict__ blk_halo,
                     const int32_t* __restrict__ halo, const int32_t* __restrict__ rows,
                     const int64_t* __restrict__ rptr, const uint16_t* __restrict__ lcol,
                     const float2* __restrict__ A, const float2* __restrict__ X, float2* __restrict__ Y, int R,
                     int nchunk) {
  extern __shared__ float4 smem4[];
  float2* sX = reinterpret_cast<float2*>(smem4);
  float2* sA = sX + (size_t)kHaloMax * kHaloCols;
  int32_t* sR = reinterpret_cast<int32_t*>(sA + kHaloNnz);   // local row offsets [nrow + 1]
  int32_t* sG = sR + kHaloRows + 1;                            // global row ids [nrow]
  uint16_t* sL = reinterpret_cast<uint16_t*>(sG + kHaloRows);  // halo-local columns [nnz]
  const int64_t b = blockIdx.x / nchunk;
  const int ch = (int)(blockIdx.x - b * nchunk);
  const int c0 = ch * kHaloCols;
  const int ncol = min(kHaloCols, R - c0);       // even: R is even and c0 a multiple of 16
  const int64_t h0 = blk_halo[b], H = blk_halo[b + 1] - h0;
  const int64_t r0 = blk_row[b], nrow = blk_row[b + 1] - r0;
  const int part = threadIdx.x & 7;
  if (2 * part < ncol)
    for (int64_t i = threadIdx.x >> 3; i < H; i += kHaloThreads / 8)
      cp_async16(sX + i * kHaloCols + 2 * part, X + (int64_t)halo[h0 + i] * R + c0 + 2 * part);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  const int64_t k0 = rptr[r0], nnz = rptr[r0 + nrow] - k0;
  for (int64_t q = threadIdx.x; q < nnz; q += kHaloThreads) {
    sA[q] = A[k0 + q];
    sL[q] = lcol[k0 + q];
  }
  for (int64_t i = threadIdx.x; i <= nrow; i += kHaloThreads) {
    sR[i] = (int32_t)(rptr[r0 + i] - k0);
    if (i < nrow) sG[i] = rows[r0 + i];
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  const int lane = threadIdx.x & 31, half = lane >> 4, col = lane & 15;
  const int warp = threadIdx.x >> 5;
  for (int i = 2 * warp + half; i < (int)nrow; i += 2 * (kHaloThreads / 32)) {
    float2 acc = make_float2(0.f, 0.f);
    const int kb = sR[i], ke = sR[i + 1];
#pragma unroll 4
    for (int k = kb; k < ke; ++k) cmac(acc, sA[k], sX[(int)sL[k] * kHaloCols + col]);
    if (col < ncol) Y[(int64_t)sG[i] * R + c0 + col] = acc;
  }
}

// out[q] = in[src[q]]: the FP32 values in the plan's blocked order.
__global__ void gather_f2_kernel(const float2* __restrict__ in, const int32_t* __restrict__ src, int64_t n,
                                 float2* __restrict__ out) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    out[q] = in[src[q]];
}

}  // namespace

void spmm_f64(const int64_t* rp, const int32_t* ci, const double2* A, const double2* X, double2* Y, int64_t E, int R,
              cudaStream_t s, int threads) {
  spmm_launch<double2>(rp, ci, A, X, Y, E, R, s, threads);
}
void spmm_f32(const int64_t* rp, const int32_t* ci, const float2* A, const float2* X, float2* Y, int64_t E, int R,
              cudaStream_t s, int threads) {
  spmm_launch<float2>(rp, ci, A, X, Y, E, R, s, threads);
}

bool spmm_halo_f32(const SpmmDev& p, const float2* A, const float2* X, float2* Y, int R, cudaStream_t s) {
  if (!p.n_block || p.halo_max > kHaloMax || R < 2 || R > 128 || (R & 1) || ((uintptr_t)X & 15)) return false;
  const size_t smem = kHaloSmem;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(spmm_halo_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  const int nchunk = (R + kHaloCols - 1) / kHaloCols;
  note_launch(1);
  spmm_halo_kernel<<<(unsigned)(p.n_block * nchunk), kHaloThreads, smem, s>>>(p.blk_row, p.blk_halo, p.halo, p.rows,
                                                                           p.rptr, p.lcol, A, X, Y, R, nchunk);
  return true;
}

void spmm_f32_bx(const int64_t* rp, const int32_t* ci, const float2* A, const void* X, float2* Y, int64_t E, int R,
                 cudaStream_t s, int threads) {
  if (threads != 128 && threads != 256 && threads != 512) threads = 256;
  if (R > 128) return;
  note_launch(1);
  const Shape sh = shape_for(R);
  const int64_t nthr = E << sh.tpr_log2;
  const int blocks = (int)((nthr + threads - 1) / threads);
  const uint32_t* Xb = (const uint32_t*)X;
  switch (sh.cpl) {
    case 1:
      spmm_kernel<float2, 1, uint32_t><<<blocks, threads, 0, s>>>(rp, ci, A, Xb, Y, E, R, sh.tpr_log2);
      break;
    case 2:
      spmm_kernel<float2, 2, uint32_t><<<blocks, threads, 0, s>>>(rp, ci, A, Xb, Y, E, R, sh.tpr_log2);
      break;
    default:
      spmm_kernel<float2, 4, uint32_t><<<blocks, threads, 0, s>>>(rp, ci, A, Xb, Y, E, R, sh.tpr_log2);
      break;
  }
}

void spmm_plan_values(const SpmmDev& p, const float2* A32, int64_t nnz, float2* out, cudaStream_t s) {
  note_launch(1);
  gather_f2_kernel<<<152 * 8, 256, 0, s>>>(A32, p.src, nnz, out);
}

int residual_f64(const int64_t* rp, const int32_t* ci, const double2* A, const double2* X, const double2* B,
                 double2* Rv, double* part, int64_t E, int R, cudaStream_t s, bool zero_x) {
  note_launch(1);
  Shape sh = shape_for(R);
  const int blocks = 152 * 4;
  switch (sh.cpl) {
    case 1:
      if (zero_x)
        residual_kernel<1, true><<<blocks, 256, 0, s>>>(rp, ci, A, X, B, Rv, part, E, R, sh.tpr_log2);
      else
        residual_kernel<1, false><<<blocks, 256, 0, s>>>(rp, ci, A, X, B, Rv, part, E, R, sh.tpr_log2);
      break;
    case 2:
      if (zero_x)
        residual_kernel<2, true><<<blocks, 256, 0, s>>>(rp, ci, A, X, B, Rv, part, E, R, sh.tpr_log2);
      else
        residual_kernel<2, false><<<blocks, 256, 0, s>>>(rp, ci, A, X, B, Rv, part, E, R, sh.tpr_log2);
      break;
    default:
      if (zero_x)
        residual_kernel<4, true><<<blocks, 256, 0, s>>>(rp, ci, A, X, B, Rv, part, E, R, sh.tpr_log2);
      else
        residual_kernel<4, false><<<blocks, 256, 0, s>>>(rp, ci, A, X, B, Rv, part, E, R, sh.tpr_log2);
      break;
  }
  return blocks;
}

}  // namespace mwk

// ---------------------------------------------------------------------------------------
// FP64-accurate residual on the FP32 pipes (double-float arithmetic).
//
// GB300 runs FP64 at about 1/64 of its FP32 rate, so the outer residual r = b - A x of the
// mixed solver keeps A and x as unevaluated sums of two floats (hi + lo, about 48 significant
// bits) and forms every product with the exact FMA product error and every sum with Knuth's
// error-free two-sum; only b - (s_hi + s_lo) and |r|^2 are FP64.  The intrinsics (__fmul_rn,
// __fadd_rn, __fsub_rn) are never contracted, which keeps the transformations exact.
// ---------------------------------------------------------------------------------------
namespace mwk {
namespace {

// (s_h, s_l) += (a_h + a_l) * (x_h + x_l), the a_l * x_l term dropped.
__device__ __forceinline__ void df_mac(float& s_h, float& s_l, float a_h, float a_l, float x_h, float x_l) {
  const float p_h = __fmul_rn(a_h, x_h);
  const float p_e = fmaf(a_h, x_h, -p_h);                 // exact error of the product
  const float p_l = fmaf(a_h, x_l, fmaf(a_l, x_h, p_e));
  const float t = __fadd_rn(s_h, p_h);                     // two-sum(s_h, p_h)
  const float bp = __fsub_rn(t, s_h);
  const float e = __fadd_rn(__fsub_rn(s_h, __fsub_rn(t, bp)), __fsub_rn(p_h, bp));
  s_l = __fadd_rn(s_l, __fadd_rn(p_l, e));
  s_h = t;
}

// A_df[k] = (re_hi, re_lo, im_hi, im_lo) of a complex FP64 value.
__global__ void split_df_kernel(const double2* __restrict__ a, float4* __restrict__ o, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = a[i];
    const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
    o[i] = make_float4(rh, __double2float_rn(v.x - (double)rh), ih, __double2float_rn(v.y - (double)ih));
  }
}

// r = b - A x (or y = A x when B is null) with per-block, per-column partial |r|^2, as
// residual_kernel but in double-float arithmetic.
template <int CPL>
__global__ void __launch_bounds__(256) residual_df_kernel(const int64_t* __restrict__ rp,
                                                          const int32_t* __restrict__ ci,
                                                          const float4* __restrict__ A, const float4* __restrict__ X,
                                                          const double2* __restrict__ B, double2* __restrict__ Rv,
                                                          double* __restrict__ part, int64_t E, int R, int tpr_log2) {
  __shared__ double red[256 * CPL];
  const int tpr = 1 << tpr_log2;
  const int rows_per_block = 256 >> tpr_log2;
  const int lane_c = threadIdx.x & (tpr - 1);
  const int c0 = lane_c * CPL;
  double nrm[CPL];
#pragma unroll
  for (int q = 0; q < CPL; ++q) nrm[q] = 0.0;
  for (int64_t row = (int64_t)blockIdx.x * rows_per_block + (threadIdx.x >> tpr_log2); row < E;
       row += (int64_t)gridDim.x * rows_per_block) {
    if (c0 >= R) continue;
    float rh[CPL], rl[CPL], ih[CPL], il[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) rh[q] = rl[q] = ih[q] = il[q] = 0.f;
    for (int64_t k = rp[row]; k < rp[row + 1]; ++k) {
      const float4 a = A[k];
      const float4* xr = X + (int64_t)ci[k] * R + c0;
#pragma unroll
      for (int q = 0; q < CPL; ++q)
        if (c0 + q < R) {
          const float4 x = xr[q];
          df_mac(rh[q], rl[q], a.x, a.y, x.x, x.y);       // + ar xr
          df_mac(rh[q], rl[q], -a.z, -a.w, x.z, x.w);     // - ai xi
          df_mac(ih[q], il[q], a.x, a.y, x.z, x.w);       // + ar xi
          df_mac(ih[q], il[q], a.z, a.w, x.x, x.y);       // + ai xr
        }
    }
#pragma unroll
    for (int q = 0; q < CPL; ++q)
      if (c0 + q < R) {
        const double yr = (double)rh[q] + (double)rl[q], yi = (double)ih[q] + (double)il[q];
        double2 r;
        if (B) {
          const double2 bb = B[row * R + c0 + q];
          r = make_double2(bb.x - yr, bb.y - yi);
        } else {
          r = make_double2(yr, yi);
        }
        Rv[row * R + c0 + q] = r;
        nrm[q] += r.x * r.x + r.y * r.y;
      }
  }
#pragma unroll
  for (int q = 0; q < CPL; ++q) red[threadIdx.x * CPL + q] = nrm[q];
  __syncthreads();
  if ((int)threadIdx.x < tpr) {
    for (int q = 0; q < CPL; ++q) {
      const int c = c0 + q;
      if (c >= R) continue;
      double s = 0.0;
      for (int r = 0; r < rows_per_block; ++r) s += red[(r * tpr + lane_c) * CPL + q];
      part[(int64_t)blockIdx.x * R + c] = s;
    }
  }
}

// (b_h + b_l) - (y_h + y_l) rounded to FP32: the high parts' difference with its exact error
// (two-sum), then the low parts.
__device__ __forceinline__ float df_sub_round(float b_h, float b_l, float y_h, float y_l) {
  const float s = __fsub_rn(b_h, y_h);
  const float bp = __fsub_rn(s, b_h);
  const float e = __fadd_rn(__fsub_rn(b_h, __fsub_rn(s, bp)), __fsub_rn(-y_h, bp));
  return __fadd_rn(s, __fadd_rn(__fsub_rn(b_l, y_l), e));
}

// (a_h, a_l) += (b_h, b_l): two-sum of the high parts, low parts added to the error.
__device__ __forceinline__ void df_add(float& a_h, float& a_l, float b_h, float b_l) {
  const float t = __fadd_rn(a_h, b_h);
  const float bp = __fsub_rn(t, a_h);
  const float e = __fadd_rn(__fsub_rn(a_h, __fsub_rn(t, bp)), __fsub_rn(b_h, bp));
  a_l = __fadd_rn(__fadd_rn(a_l, b_l), e);
  a_h = t;
}

// The outer residual of the mixed solver: r = b - A x with b, A and x in double-float, every
// product and sum as in residual_df_kernel, r rounded once to FP32 complex (the inner solver's
// start vector is FP32) and |r|^2 of the rounded r promoted to FP64 per row (per-block,
// per-column partials).  Two FP64 operations per element instead of eleven.  The nonzeros of a
// row alternate between two independent double-float accumulators (two dependency chains in
// flight), joined by a double-float add at the end of the row.  ZX: x = 0 (the first outer step),
// so every product and sum of a row is +0 and the row loop is skipped: the same r and norms.
template <int CPL, bool ZX>
__global__ void __launch_bounds__(256) residual_df32_kernel(const int64_t* __restrict__ rp,
                                                            const int32_t* __restrict__ ci,
                                                            const float4* __restrict__ A, const float4* __restrict__ X,
                                                            const float4* __restrict__ Bdf, float2* __restrict__ Rv,
                                                            double* __restrict__ part, int64_t E, int R, int tpr_log2) {
  __shared__ double red[256 * CPL];
  const int tpr = 1 << tpr_log2;
  const int rows_per_block = 256 >> tpr_log2;
  const int lane_c = threadIdx.x & (tpr - 1);
  const int c0 = lane_c * CPL;
  double nrm[CPL];
#pragma unroll
  for (int q = 0; q < CPL; ++q) nrm[q] = 0.0;
  for (int64_t row = (int64_t)blockIdx.x * rows_per_block + (threadIdx.x >> tpr_log2); row < E;
       row += (int64_t)gridDim.x * rows_per_block) {
    if (c0 >= R) continue;
    float rh[CPL], rl[CPL], ih[CPL], il[CPL], rh2[CPL], rl2[CPL], ih2[CPL], il2[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) rh[q] = rl[q] = ih[q] = il[q] = rh2[q] = rl2[q] = ih2[q] = il2[q] = 0.f;
    const int64_t kb = ZX ? 0 : rp[row], ke = ZX ? 0 : rp[row + 1];
    int64_t k = kb;
    for (; k + 1 < ke; k += 2) {
      const float4 a = A[k], a2 = A[k + 1];
      const float4* xr = X + (int64_t)ci[k] * R + c0;
      const float4* xr2 = X + (int64_t)ci[k + 1] * R + c0;
#pragma unroll
      for (int q = 0; q < CPL; ++q)
        if (c0 + q < R) {
          const float4 x = xr[q], x2 = xr2[q];
          df_mac(rh[q], rl[q], a.x, a.y, x.x, x.y);
          df_mac(rh2[q], rl2[q], a2.x, a2.y, x2.x, x2.y);
          df_mac(ih[q], il[q], a.x, a.y, x.z, x.w);
          df_mac(ih2[q], il2[q], a2.x, a2.y, x2.z, x2.w);
          df_mac(rh[q], rl[q], -a.z, -a.w, x.z, x.w);
          df_mac(rh2[q], rl2[q], -a2.z, -a2.w, x2.z, x2.w);
          df_mac(ih[q], il[q], a.z, a.w, x.x, x.y);
          df_mac(ih2[q], il2[q], a2.z, a2.w, x2.x, x2.y);
        }
    }
    if (k < ke) {
      const float4 a = A[k];
      const float4* xr = X + (int64_t)ci[k] * R + c0;
#pragma unroll
      for (int q = 0; q < CPL; ++q)
        if (c0 + q < R) {
          const float4 x = xr[q];
          df_mac(rh[q], rl[q], a.x, a.y, x.x, x.y);
          df_mac(ih[q], il[q], a.x, a.y, x.z, x.w);
          df_mac(rh[q], rl[q], -a.z, -a.w, x.z, x.w);
          df_mac(ih[q], il[q], a.z, a.w, x.x, x.y);
        }
    }
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
      df_add(rh[q], rl[q], rh2[q], rl2[q]);
      df_add(ih[q], il[q], ih2[q], il2[q]);
    }
#pragma unroll
    for (int q = 0; q < CPL; ++q)
      if (c0 + q < R) {
        const float4 bb = Bdf[row * R + c0 + q];
        const float re = df_sub_round(bb.x, bb.y, rh[q], rl[q]);
        const float im = df_sub_round(bb.z, bb.w, ih[q], il[q]);
        Rv[row * R + c0 + q] = make_float2(re, im);
        nrm[q] += (double)fmaf(re, re, __fmul_rn(im, im));
      }
  }
#pragma unroll
  for (int q = 0; q < CPL; ++q) red[threadIdx.x * CPL + q] = nrm[q];
  __syncthreads();
  if ((int)threadIdx.x < tpr) {
    for (int q = 0; q < CPL; ++q) {
      const int c = c0 + q;
      if (c >= R) continue;
      double s = 0.0;
      for (int r = 0; r < rows_per_block; ++r) s += red[(r * tpr + lane_c) * CPL + q];
      part[(int64_t)blockIdx.x * R + c] = s;
    }
  }
}

}  // namespace

void split_df(const double2* a, float4* o, int64_t n, cudaStream_t s) {
  note_launch(1);
  int64_t b = (n + 255) / 256;
  split_df_kernel<<<(int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16), 256, 0, s>>>(a, o, n);
}

int residual_df(const int64_t* rp, const int32_t* ci, const float4* A, const float4* X, const double2* B, double2* Rv,
                double* part, int64_t E, int R, cudaStream_t s) {
  note_launch(1);
  Shape sh = shape_for(R);
  const int blocks = 152 * 4;
  switch (sh.cpl) {
    case 1:
      residual_df_kernel<1><<<blocks, 256, 0, s>>>(rp, ci, A, X, B, Rv, part, E, R, sh.tpr_log2);
      break;
    case 2:
      residual_df_kernel<2><<<blocks, 256, 0, s>>>(rp, ci, A, X, B, Rv, part, E, R, sh.tpr_log2);
      break;
    default:
      residual_df_kernel<4><<<blocks, 256, 0, s>>>(rp, ci, A, X, B, Rv, part, E, R, sh.tpr_log2);
      break;
  }
  return blocks;
}

int residual_df32(const int64_t* rp, const int32_t* ci, const float4* A, const float4* X, const float4* Bdf, float2* Rv,
                  double* part, int64_t E, int R, cudaStream_t s, bool zero_x) {
  note_launch(1);
  Shape sh = shape_for(R);
  const int blocks = 152 * 4;
  switch (sh.cpl) {
    case 1:
      if (zero_x)
        residual_df32_kernel<1, true><<<blocks, 256, 0, s>>>(rp, ci, A, X, Bdf, Rv, part, E, R, sh.tpr_log2);
      else
        residual_df32_kernel<1, false><<<blocks, 256, 0, s>>>(rp, ci, A, X, Bdf, Rv, part, E, R, sh.tpr_log2);
      break;
    case 2:
      if (zero_x)
        residual_df32_kernel<2, true><<<blocks, 256, 0, s>>>(rp, ci, A, X, Bdf, Rv, part, E, R, sh.tpr_log2);
      else
        residual_df32_kernel<2, false><<<blocks, 256, 0, s>>>(rp, ci, A, X, Bdf, Rv, part, E, R, sh.tpr_log2);
      break;
    default:
      if (zero_x)
        residual_df32_kernel<4, true><<<blocks, 256, 0, s>>>(rp, ci, A, X, Bdf, Rv, part, E, R, sh.tpr_log2);
      else
        residual_df32_kernel<4, false><<<blocks, 256, 0, s>>>(rp, ci, A, X, Bdf, Rv, part, E, R, sh.tpr_log2);
      break;
  }
  return blocks;
}

}  // namespace mwk
