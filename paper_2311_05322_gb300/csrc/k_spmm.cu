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

template <typename T, int CPL>
__global__ void __launch_bounds__(256) spmm_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                   const T* __restrict__ A, const T* __restrict__ X, T* __restrict__ Y,
                                                   int64_t E, int R, int tpr_log2) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t row = g >> tpr_log2;
  const int c0 = (int)(g & ((1 << tpr_log2) - 1)) * CPL;
  if (row >= E || c0 >= R) return;
  T acc[CPL];
#pragma unroll
  for (int q = 0; q < CPL; ++q) acc[q] = T{0, 0};
  const int64_t b = rp[row], e = rp[row + 1];
  for (int64_t k = b; k < e; ++k) {
    const T a = A[k];
    const T* xr = X + (int64_t)ci[k] * R + c0;
#pragma unroll
    for (int q = 0; q < CPL; ++q)
      if (c0 + q < R) cmac(acc[q], a, xr[q]);
  }
  T* yr = Y + row * R + c0;
#pragma unroll
  for (int q = 0; q < CPL; ++q)
    if (c0 + q < R) yr[q] = acc[q];
}

// r = b - A x in FP64 with per-block, per-column partial sums of |r|^2 (deterministic).
template <int CPL>
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
    for (int64_t k = rp[row]; k < rp[row + 1]; ++k) {
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
                 cudaStream_t s) {
  note_launch(1);
  Shape sh = shape_for(R);
  if (R > 128) {
    // wide blocks: process 128 columns at a time is not supported by the layout; caller splits.
    return;
  }
  const int64_t threads = E << sh.tpr_log2;
  const int blocks = (int)((threads + 255) / 256);
  switch (sh.cpl) {
    case 1:
      spmm_kernel<T, 1><<<blocks, 256, 0, s>>>(rp, ci, A, X, Y, E, R, sh.tpr_log2);
      break;
    case 2:
      spmm_kernel<T, 2><<<blocks, 256, 0, s>>>(rp, ci, A, X, Y, E, R, sh.tpr_log2);
      break;
    default:
      spmm_kernel<T, 4><<<blocks, 256, 0, s>>>(rp, ci, A, X, Y, E, R, sh.tpr_log2);
      break;
  }
}

}  // namespace

void spmm_f64(const int64_t* rp, const int32_t* ci, const double2* A, const double2* X, double2* Y, int64_t E, int R,
              cudaStream_t s) {
  spmm_launch<double2>(rp, ci, A, X, Y, E, R, s);
}
void spmm_f32(const int64_t* rp, const int32_t* ci, const float2* A, const float2* X, float2* Y, int64_t E, int R,
              cudaStream_t s) {
  spmm_launch<float2>(rp, ci, A, X, Y, E, R, s);
}

int residual_f64(const int64_t* rp, const int32_t* ci, const double2* A, const double2* X, const double2* B,
                 double2* Rv, double* part, int64_t E, int R, cudaStream_t s) {
  note_launch(1);
  Shape sh = shape_for(R);
  const int blocks = 152 * 4;
  switch (sh.cpl) {
    case 1:
      residual_kernel<1><<<blocks, 256, 0, s>>>(rp, ci, A, X, B, Rv, part, E, R, sh.tpr_log2);
      break;
    case 2:
      residual_kernel<2><<<blocks, 256, 0, s>>>(rp, ci, A, X, B, Rv, part, E, R, sh.tpr_log2);
      break;
    default:
      residual_kernel<4><<<blocks, 256, 0, s>>>(rp, ci, A, X, B, Rv, part, E, R, sh.tpr_log2);
      break;
  }
  return blocks;
}

}  // namespace mwk
