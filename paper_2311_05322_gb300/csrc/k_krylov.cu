// K6-K8, K15: batched Arnoldi (classical Gram-Schmidt), Givens least squares and solution update
// of restarted, right-preconditioned (flexible) GMRES, all columns of a block at once.
//
// Layout: Krylov vectors V[i] are [E][R] (column index fastest) at V + i * vstride.  All
// reductions are deterministic: per-block partial sums reduced in a fixed order.  Dot products
// of FP32 vectors multiply and sum in FP32 over chunks of kChunk rows and accumulate the chunk
// sums in FP64; FP64 vectors use FP64 throughout.
//
// Per-column GMRES state (one entry per column c of the block, m = restart length):
//   H[c][j][i]   Hessenberg column j (i <= j+1) after rotations, complex FP64, (m+1) per column j
//   cs[c][2j], cs[c][2j+1]   Givens pair (c_j, s_j) mapping (a, b) -> (sqrt(|a|^2+|b|^2), 0)
//   g[c][i]      rotated right-hand side beta e_1
//   target[c]    residual-estimate target of this cycle
//   done[c]      1 once the column stopped (converged, breakdown or out of steps)
//   kcol[c]      Arnoldi steps used by the column in this cycle
#include <algorithm>
#include <cstdint>

#include "mw_async.cuh"
#include "mw_internal.h"

namespace mwk {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxVecPerWarp = 8;   // restart m <= 63 => nvec <= 64 = 8 warps x 8
constexpr int kChunk = 16;          // FP32 rows summed before promotion to FP64
constexpr int kBlocks = 152 * 4;

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

template <typename T>
struct Traits;
template <>
struct Traits<double2> {
  using S = double;
};
template <>
struct Traits<float2> {
  using S = float;
};

struct Shape {
  int cpl, tpr_log2;
};
inline Shape shape_for(int R) {
  int cpl = (R + 31) / 32;
  if (cpl > 2) cpl = 4;
  int tpr = (R + cpl - 1) / cpl;
  int l = 0;
  while ((1 << l) < tpr) ++l;
  return {cpl, l};
}

// h_part[p][i][c] = sum over the rows of part p of conj(V_i[e][c]) * w[e][c].
// Warp k of a block serves vectors i = k, k + 16, ... (nvec >= 16); for nvec < 16 the 16
// warps split into S = 16 / nvec row slots per vector.  A warp walks its rows in passes of kUnroll
// rows with all loads of a pass issued together (V_i from HBM, w shared by the block's warps
// through L1); each pass is summed in the vector precision and added to an FP64 accumulator.
// No block-level synchronisation.  Part index p = block * S + slot.
constexpr int kDotThreads = 512;
constexpr int kDotWarps = kDotThreads / 32;
constexpr int kDotVecPerWarp = 4;   // nvec <= 64 = 16 warps x 4

template <typename T, int CPL>
__global__ void __launch_bounds__(kDotThreads) cgs_dots_kernel(const T* __restrict__ V, int64_t vstride, int nvec,
                                                            const T* __restrict__ w, int64_t E, int R, int tpr_log2,
                                                            int S, double2* __restrict__ part) {
  using Sc = typename Traits<T>::S;
  // rows in flight per thread: the same bytes per thread for every CPL and precision
  constexpr int kUnroll = (16 / CPL) / (sizeof(T) / 8) > 0 ? (16 / CPL) / (sizeof(T) / 8) : 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tpr = 1 << tpr_log2;
  const int rpw = 32 >> tpr_log2;           // rows per warp pass
  const int lrow = lane >> tpr_log2;
  const int c0 = (lane & (tpr - 1)) * CPL;
  int i_first, i_step, slot;
  bool idle = false;
  if (nvec >= kDotWarps) {
    i_first = warp;
    i_step = kDotWarps;
    slot = 0;
  } else {
    idle = warp >= nvec * S;
    i_first = warp % nvec;
    i_step = 1 << 30;
    slot = warp / nvec;
  }
  const int nmine = idle ? 0 : (i_first < nvec ? (nvec - 1 - i_first) / i_step + 1 : 0);
  double2 acc[kDotVecPerWarp][CPL];
#pragma unroll
  for (int a = 0; a < kDotVecPerWarp; ++a)
#pragma unroll
    for (int q = 0; q < CPL; ++q) acc[a][q] = make_double2(0.0, 0.0);
  const bool active_c = c0 < R && !idle;
  // Block iterations take contiguous chunks of kUnroll * rpw * S rows; slot q of the chunk owns
  // the contiguous sub-range [q * kUnroll * rpw, (q + 1) * kUnroll * rpw), and thread (lrow, u)
  // reads row sub + u * rpw + lrow, so a warp streams kUnroll * rpw consecutive rows.
  const int64_t chunk = (int64_t)kUnroll * rpw * S;
  if (active_c) {
    for (int64_t cb = (int64_t)blockIdx.x * chunk; cb < E; cb += (int64_t)gridDim.x * chunk) {
      const int64_t sub = cb + (int64_t)slot * kUnroll * rpw + lrow;
#pragma unroll
      for (int a = 0; a < kDotVecPerWarp; ++a) {
        if (a < nmine) {
          const int i = i_first + a * i_step;
          const T* Vi = V + (int64_t)i * vstride;
          T vv[kUnroll][CPL], xx[kUnroll][CPL];
#pragma unroll
          for (int u = 0; u < kUnroll; ++u) {
            const int64_t row = sub + (int64_t)u * rpw;
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
              const bool ok = row < E && c0 + q < R;
              vv[u][q] = ok ? Vi[row * R + c0 + q] : T{0, 0};
              xx[u][q] = ok ? __ldg(&w[row * R + c0 + q]) : T{0, 0};
            }
          }
#pragma unroll
          for (int q = 0; q < CPL; ++q) {
            Sc sr = 0, si = 0;
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
              sr = fma(vv[u][q].x, xx[u][q].x, sr);
              sr = fma(vv[u][q].y, xx[u][q].y, sr);
              si = fma(vv[u][q].x, xx[u][q].y, si);
              si = fma(-vv[u][q].y, xx[u][q].x, si);
            }
            acc[a][q].x += (double)sr;
            acc[a][q].y += (double)si;
          }
        }
      }
    }
  }
  // reduce over the rows of the warp (lanes with equal column)
#pragma unroll
  for (int a = 0; a < kDotVecPerWarp; ++a) {
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
      double x = acc[a][q].x, y = acc[a][q].y;
      for (int off = tpr; off < 32; off <<= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, off);
        y += __shfl_xor_sync(0xffffffffu, y, off);
      }
      acc[a][q] = make_double2(x, y);
    }
  }
  if (lrow == 0 && active_c) {
    const int64_t p = (int64_t)blockIdx.x * S + slot;
#pragma unroll
    for (int a = 0; a < kDotVecPerWarp; ++a) {
      if (a < nmine) {
        const int i = i_first + a * i_step;
#pragma unroll
        for (int q = 0; q < CPL; ++q)
          if (c0 + q < R) part[(p * nvec + i) * R + c0 + q] = acc[a][q];
      }
    }
  }
}

// Streaming form of the same dots for 16 <= R <= 128 with 16-byte aligned vectors.  The rows
// are cut into tiles of TR = G * bd_rows<T>() rows (G = 256 / R row groups), about 16 KB per
// vector; block b takes a contiguous range of tiles.  Warp 0 lane 0 streams, per tile, w and
// then V_i0 .. V_i0+nv-1 through a ring of NS shared-memory stages with bulk copies;
// the 256 consumer threads (warps 1-8) map thread (c, g) = (t % R, t / R) to column c and the
// tile rows g, g + G, ...  Each consumer keeps its w rows in registers for the whole tile,
// forms its FP32 (FP64) partial of conj(V_i) w over its bd_rows<T>() rows, and the G partials of a
// column are summed in the vector precision in a fixed order by thread (c, i % G), which adds
// the tile sum to an FP64 accumulator in shared memory (so FP32 vectors are summed in FP32 over
// chunks of TR rows; FP64 instructions, slow on this part, stay at a few per tile and column).
// Vector groups of VG = min(64, 2048 / R) vectors are swept in turn (w is re-read per sweep).
// Part index p = block.  The element beyond the last 16-byte boundary of a ragged last tile
// (odd rows * R in FP32) is read from global memory.  Every wait is bounded; on timeout the
// kernel records an error code, skips the remaining waits and copies (still executing the
// same named barriers), drains its outstanding copies and returns.
constexpr int kBdConsumers = 256;
// A consumer warp releases a ring stage once all its lanes are done with it: one arrival per
// warp on the stage's empty barrier (which expects kBdConsumers / 32) instead of one per thread.
__device__ __forceinline__ void release_stage(uint64_t* bar) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(bar);
}
constexpr int kBdThreads = kBdConsumers + 32;
constexpr int kBdStages = 4;      // default ring depth; 2..kBdMaxStages accepted (same result)
constexpr int kBdMaxStages = 6;
constexpr int kBdStageBytes = 16384;
template <typename T>
__host__ __device__ constexpr int bd_rows() {
  return 64 / (int)sizeof(T);   // 8 rows (FP32 complex), 4 rows (FP64 complex)
}
constexpr int kBdGroup = 4;     // basis vectors whose partials share one named barrier
// partial buffer: 2 (double buffer) x kBdGroup x 256 entries of the vector type
__host__ __device__ inline size_t bd_red_bytes(size_t es) { return 2 * kBdGroup * kBdConsumers * es; }
// VG * R <= 2048 accumulators of 16 bytes
inline size_t bd_smem_bytes(int R, int NS, size_t es) {
  const int VG = std::min(64, 2048 / R);
  return (size_t)NS * kBdStageBytes + bd_red_bytes(es) + (size_t)VG * R * sizeof(double2) +
         2 * NS * sizeof(uint64_t) + 16;
}
constexpr size_t kBdMaxSmem = (size_t)kBdMaxStages * kBdStageBytes + 2 * kBdGroup * kBdConsumers * sizeof(double2) +
                              2048 * sizeof(double2) + 2 * kBdMaxStages * sizeof(uint64_t) + 16;

template <typename T>
__global__ void __launch_bounds__(kBdThreads, 2)
    cgs_dots_bulk_kernel(const T* __restrict__ V, int64_t vstride, int nvec, const T* __restrict__ w, int64_t E,
                         int R, int G, int VG, int NS, double2* __restrict__ part, int32_t* __restrict__ err) {
  using Sc = typename Traits<T>::S;
  constexpr int RPT = bd_rows<T>();
  constexpr int kStageElems = kBdStageBytes / (int)sizeof(T);
  extern __shared__ __align__(128) uint8_t bd_smem[];
  T* stage = reinterpret_cast<T*>(bd_smem);
  T* red = reinterpret_cast<T*>(bd_smem + (size_t)NS * kBdStageBytes);   // [2][kBdGroup][256]
  double2* acc = reinterpret_cast<double2*>(bd_smem + (size_t)NS * kBdStageBytes + bd_red_bytes(sizeof(T)));
  uint64_t* full = reinterpret_cast<uint64_t*>(acc + (size_t)VG * R);
  uint64_t* empty = full + NS;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + NS);

  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kBdConsumers / 32);   // one arrival per consumer warp
    }
    *abort_flag = 0;
    mbar_init_fence();
  }
  __syncthreads();

  const int TR = G * RPT;
  const int64_t nt = (E + TR - 1) / TR;
  const int64_t t0 = nt * blockIdx.x / gridDim.x, t1 = nt * (blockIdx.x + 1) / gridDim.x;
  const int nsweep = (nvec + VG - 1) / VG;

  if (tid < 32) {
    if (tid != 0) return;
    // producer: ring position st with phase bit ph (st advances per item, ph flips per lap)
    int64_t it = 0;
    int st = 0;
    uint32_t ph = 0;
    bool stop = false;
    for (int sw = 0; sw < nsweep && !stop; ++sw) {
      const int i0 = sw * VG, nv = min(VG, nvec - i0);
      for (int64_t t = t0; t < t1 && !stop; ++t) {
        const int64_t r0 = t * TR;
        const int64_t rows = E - r0 < TR ? E - r0 : (int64_t)TR;
        const uint32_t bytes = (uint32_t)((rows * R * (int64_t)sizeof(T)) & ~(int64_t)15);
        for (int q = -1; q < nv; ++q) {
          if (it >= NS && !mbar_wait(&empty[st], ph ^ 1u)) {
            atomicCAS(err, 0, 11);
            *abort_flag = 1;
          }
          if (*abort_flag) {
            stop = true;
            break;
          }
          const T* src = (q < 0 ? w : V + (int64_t)(i0 + q) * vstride) + r0 * R;
          if (bytes > 0) {
            mbar_expect_tx(&full[st], bytes);
            bulk_g2s(stage + (size_t)st * kStageElems, src, bytes, &full[st]);
          } else {
            mbar_arrive(&full[st]);
          }
          ++it;
          if (++st == NS) {
            st = 0;
            ph ^= 1u;
          }
        }
      }
    }
    // drain: every issued copy has landed before this thread leaves (the latest use of stage
    // k < st is in the current lap, of stage k >= st in the previous one, if any)
    for (int k = 0; k < NS; ++k) {
      if (k >= st && it < NS) continue;
      if (!mbar_wait(&full[k], k < st ? ph : ph ^ 1u)) atomicCAS(err, 0, 12);
    }
    return;
  }

  // consumers
  const int ct = tid - 32;
  const int c = ct % R, g = ct / R;
  const bool act = g < G;
  int st = 0;        // ring position and phase bit, as the producer's
  uint32_t ph = 0;
  int64_t nred = 0;
  auto wait_full = [&]() {
    if (*abort_flag) return;
    if (!mbar_wait(&full[st], ph)) {
      atomicCAS(err, 0, 13);
      *abort_flag = 1;
    }
  };
  auto advance = [&]() {
    if (++st == NS) {
      st = 0;
      ph ^= 1u;
    }
  };
  for (int sw = 0; sw < nsweep; ++sw) {
    const int i0 = sw * VG, nv = min(VG, nvec - i0);
    if (act)
      for (int q = g; q < nv; q += G) acc[q * R + c] = make_double2(0.0, 0.0);
    for (int64_t t = t0; t < t1; ++t) {
      const int64_t r0 = t * TR;
      const int64_t rows = E - r0 < TR ? E - r0 : (int64_t)TR;
      const int64_t ncop = ((rows * R * (int64_t)sizeof(T)) & ~(int64_t)15) / (int64_t)sizeof(T);
      // w tile -> registers
      T wr[RPT];
      {
        wait_full();
        const T* sm = stage + (size_t)st * kStageElems;
        const T* gl = w + r0 * R;
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
          const int row = k * G + g;
          const int f = row * R + c;
          wr[k] = T{0, 0};
          if (act && row < rows) wr[k] = f < ncop ? sm[f] : gl[f];
        }
        release_stage(&empty[st]);
        advance();
      }
      // partials of up to kBdGroup consecutive vectors, then one barrier and their reductions
      for (int q0 = 0, qg0 = 0; q0 < nv; q0 += kBdGroup) {
        const int ng = min(kBdGroup, nv - q0);
        T* rb = red + (size_t)(nred & 1) * kBdGroup * kBdConsumers;
        for (int u = 0; u < ng; ++u) {
          wait_full();
          const T* sm = stage + (size_t)st * kStageElems;
          const T* gl = V + (int64_t)(i0 + q0 + u) * vstride + r0 * R;
          Sc pr = 0, pi = 0;
#pragma unroll
          for (int k = 0; k < RPT; ++k) {
            const int row = k * G + g;
            const int f = row * R + c;
            if (act && row < rows) {
              const T v = f < ncop ? sm[f] : gl[f];
              pr = fma(v.x, wr[k].x, pr);
              pr = fma(v.y, wr[k].y, pr);
              pi = fma(v.x, wr[k].y, pi);
              pi = fma(-v.y, wr[k].x, pi);
            }
          }
          release_stage(&empty[st]);
          advance();
          rb[u * kBdConsumers + ct] = T{pr, pi};
        }
        ++nred;
        asm volatile("bar.sync 1, %0;" ::"n"(kBdConsumers) : "memory");
        for (int u = 0, qg = qg0; u < ng; ++u, qg = (qg + 1 == G ? 0 : qg + 1)) {
          if (act && g == qg) {
            const T* ru = rb + u * kBdConsumers;
            Sc sr = 0, si = 0;
#pragma unroll 8
            for (int g2 = 0; g2 < G; ++g2) {
              const T v = ru[g2 * R + c];
              sr += v.x;
              si += v.y;
            }
            double2 a = acc[(q0 + u) * R + c];
            a.x += (double)sr;
            a.y += (double)si;
            acc[(q0 + u) * R + c] = a;
          }
        }
        qg0 = (qg0 + ng) % G;
      }
    }
    if (act)
      for (int q = g; q < nv; q += G) part[((int64_t)blockIdx.x * nvec + i0 + q) * R + c] = acc[q * R + c];
  }
}

// h[i][c] = sum_p part[p][i][c]: one warp per entry, lanes take parts lane, lane + 32, ...,
// then a fixed shuffle tree (deterministic).
// With vscale (the basis kept unscaled, V_i = vscale[i][c] * Vu_i), h[i][c] is scaled by it.
__global__ void reduce_h_kernel(const double2* __restrict__ part, int nparts, int nvec, int R, double2* __restrict__ h,
                                const double* __restrict__ vscale) {
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= nvec * R) return;
  double x = 0.0, y = 0.0;
  for (int p = lane; p < nparts; p += 32) {
    const double2 v = part[(int64_t)p * nvec * R + t];
    x += v.x;
    y += v.y;
  }
  for (int off = 16; off > 0; off >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, off);
    y += __shfl_xor_sync(0xffffffffu, y, off);
  }
  if (lane == 0) {
    const double sc = vscale ? vscale[t] : 1.0;
    h[t] = make_double2(x * sc, y * sc);
  }
}

// w[e][c] -= sum_i h[i][c] V_i[e][c]; partial sums of |w|^2 per block and column.
template <typename T, int CPL>
__global__ void __launch_bounds__(kThreads) cgs_update_kernel(const T* __restrict__ V, int64_t vstride, int nvec,
                                                              const double2* __restrict__ h, T* __restrict__ w,
                                                              int64_t E, int R, int tpr_log2,
                                                              double* __restrict__ npart,
                                                              const double* __restrict__ vscale) {
  using Sc = typename Traits<T>::S;
  extern __shared__ unsigned char smem_raw[];
  T* hs = reinterpret_cast<T*>(smem_raw);                          // [nvec][R]
  double* red = reinterpret_cast<double*>(smem_raw + sizeof(T) * nvec * R + 16);  // [kThreads][CPL]
  for (int t = threadIdx.x; t < nvec * R; t += kThreads) {
    const double2 v = h[t];
    const double sc = vscale ? vscale[t] : 1.0;   // coefficient of the unscaled basis vector
    hs[t] = T{(Sc)(v.x * sc), (Sc)(v.y * sc)};
  }
  __syncthreads();
  const int tpr = 1 << tpr_log2;
  const int rows_per_block = kThreads >> tpr_log2;
  const int lc = threadIdx.x & (tpr - 1);
  const int c0 = lc * CPL;
  double nrm[CPL];
#pragma unroll
  for (int q = 0; q < CPL; ++q) nrm[q] = 0.0;
  if (c0 < R) {
    for (int64_t row = (int64_t)blockIdx.x * rows_per_block + (threadIdx.x >> tpr_log2); row < E;
         row += (int64_t)gridDim.x * rows_per_block) {
      T acc[CPL];
      T* wr = w + row * R + c0;
#pragma unroll
      for (int q = 0; q < CPL; ++q)
        if (c0 + q < R) acc[q] = wr[q];
      for (int i = 0; i < nvec; ++i) {
        const T* vr = V + (int64_t)i * vstride + row * R + c0;
#pragma unroll
        for (int q = 0; q < CPL; ++q)
          if (c0 + q < R) {
            const T v = vr[q], hh = hs[i * R + c0 + q];
            acc[q].x = fma(-hh.x, v.x, acc[q].x);
            acc[q].x = fma(hh.y, v.y, acc[q].x);
            acc[q].y = fma(-hh.x, v.y, acc[q].y);
            acc[q].y = fma(-hh.y, v.x, acc[q].y);
          }
      }
#pragma unroll
      for (int q = 0; q < CPL; ++q)
        if (c0 + q < R) {
          wr[q] = acc[q];
          nrm[q] += (double)(acc[q].x * acc[q].x + acc[q].y * acc[q].y);
        }
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
      for (int r = 0; r < rows_per_block; ++r) s += red[(r * tpr + lc) * CPL + q];
      npart[(int64_t)blockIdx.x * R + c] = s;
    }
  }
}

// Streaming form of the update for 16 <= R <= 128 with 16-byte aligned vectors, on the tiles,
// ring and thread map of cgs_dots_bulk_kernel: per tile the producer streams w and then V_0 ..
// V_nvec-1; consumer (c, g) holds its kBdRows w rows of column c in registers, applies
// w -= h_i V_i for each arriving tile in the order of cgs_update_kernel (the same operations per
// element, so w is bit-identical), and stores its rows back.  |w|^2 is promoted to FP64 per row
// and summed per thread; the G row groups of a column are summed in a fixed order at the end
// (one partial per block and column).  h is staged in shared memory as T.  Bounded waits as in
// the dots kernel.
template <typename T>
__global__ void __launch_bounds__(kBdThreads, 2)
    cgs_update_bulk_kernel(const T* __restrict__ V, int64_t vstride, int nvec, const double2* __restrict__ h,
                           T* __restrict__ w, int64_t E, int R, int G, int NS, double* __restrict__ npart,
                           int32_t* __restrict__ err, const double* __restrict__ vscale) {
  using Sc = typename Traits<T>::S;
  constexpr int RPT = bd_rows<T>();
  constexpr int kStageElems = kBdStageBytes / (int)sizeof(T);
  extern __shared__ __align__(128) uint8_t bu_smem[];
  T* stage = reinterpret_cast<T*>(bu_smem);
  T* hs = reinterpret_cast<T*>(bu_smem + (size_t)NS * kBdStageBytes);                 // [nvec][R]
  double* red = reinterpret_cast<double*>(hs + (size_t)nvec * R + 2);                 // [G][R]
  uint64_t* full = reinterpret_cast<uint64_t*>(red + (size_t)kBdConsumers);
  uint64_t* empty = full + NS;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + NS);

  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kBdConsumers / 32);   // one arrival per consumer warp
    }
    *abort_flag = 0;
    mbar_init_fence();
  }
  for (int t = tid; t < nvec * R; t += kBdThreads) {
    const double2 v = h[t];
    const double sc = vscale ? vscale[t] : 1.0;   // coefficient of the unscaled basis vector
    hs[t] = T{(Sc)(v.x * sc), (Sc)(v.y * sc)};
  }
  __syncthreads();

  const int TR = G * RPT;
  const int64_t nt = (E + TR - 1) / TR;
  const int64_t t0 = nt * blockIdx.x / gridDim.x, t1 = nt * (blockIdx.x + 1) / gridDim.x;

  if (tid < 32) {
    if (tid != 0) return;
    // producer: ring position st with phase bit ph
    int64_t it = 0;
    int st = 0;
    uint32_t ph = 0;
    bool stop = false;
    for (int64_t t = t0; t < t1 && !stop; ++t) {
      const int64_t r0 = t * TR;
      const int64_t rows = E - r0 < TR ? E - r0 : (int64_t)TR;
      const uint32_t bytes = (uint32_t)((rows * R * (int64_t)sizeof(T)) & ~(int64_t)15);
      for (int q = -1; q < nvec; ++q) {
        if (it >= NS && !mbar_wait(&empty[st], ph ^ 1u)) {
          atomicCAS(err, 0, 21);
          *abort_flag = 1;
        }
        if (*abort_flag) {
          stop = true;
          break;
        }
        const T* src = (q < 0 ? w : V + (int64_t)q * vstride) + r0 * R;
        if (bytes > 0) {
          mbar_expect_tx(&full[st], bytes);
          bulk_g2s(stage + (size_t)st * kStageElems, src, bytes, &full[st]);
        } else {
          mbar_arrive(&full[st]);
        }
        ++it;
        if (++st == NS) {
          st = 0;
          ph ^= 1u;
        }
      }
    }
    for (int k = 0; k < NS; ++k) {
      if (k >= st && it < NS) continue;
      if (!mbar_wait(&full[k], k < st ? ph : ph ^ 1u)) atomicCAS(err, 0, 22);
    }
    return;
  }

  // consumers
  const int ct = tid - 32;
  const int c = ct % R, g = ct / R;
  const bool act = g < G;
  int st = 0;
  uint32_t ph = 0;
  auto wait_full = [&]() {
    if (*abort_flag) return;
    if (!mbar_wait(&full[st], ph)) {
      atomicCAS(err, 0, 23);
      *abort_flag = 1;
    }
  };
  auto advance = [&]() {
    if (++st == NS) {
      st = 0;
      ph ^= 1u;
    }
  };
  double nrm = 0.0;
  for (int64_t t = t0; t < t1; ++t) {
    const int64_t r0 = t * TR;
    const int64_t rows = E - r0 < TR ? E - r0 : (int64_t)TR;
    const int64_t ncop = ((rows * R * (int64_t)sizeof(T)) & ~(int64_t)15) / (int64_t)sizeof(T);
    T acc[RPT];
    {
      wait_full();
      const T* sm = stage + (size_t)st * kStageElems;
      const T* gl = w + r0 * R;
#pragma unroll
      for (int k = 0; k < RPT; ++k) {
        const int row = k * G + g;
        const int f = row * R + c;
        acc[k] = T{0, 0};
        if (act && row < rows) acc[k] = f < ncop ? sm[f] : gl[f];
      }
      release_stage(&empty[st]);
      advance();
    }
    for (int i = 0; i < nvec; ++i) {
      wait_full();
      const T* sm = stage + (size_t)st * kStageElems;
      const T* gl = V + (int64_t)i * vstride + r0 * R;
      const T hh = act ? hs[i * R + c] : T{0, 0};
#pragma unroll
      for (int k = 0; k < RPT; ++k) {
        const int row = k * G + g;
        const int f = row * R + c;
        if (act && row < rows) {
          const T v = f < ncop ? sm[f] : gl[f];
          acc[k].x = fma(-hh.x, v.x, acc[k].x);
          acc[k].x = fma(hh.y, v.y, acc[k].x);
          acc[k].y = fma(-hh.x, v.y, acc[k].y);
          acc[k].y = fma(-hh.y, v.x, acc[k].y);
        }
      }
      release_stage(&empty[st]);
      advance();
    }
    if (act && !*abort_flag) {
      T* wr = w + r0 * R;
#pragma unroll
      for (int k = 0; k < RPT; ++k) {
        const int row = k * G + g;
        if (row < rows) {
          wr[row * R + c] = acc[k];
          nrm += (double)(acc[k].x * acc[k].x + acc[k].y * acc[k].y);
        }
      }
    }
  }
  red[ct] = nrm;
  asm volatile("bar.sync 1, %0;" ::"n"(kBdConsumers) : "memory");
  if (act && g == 0) {
    double sum = 0.0;
    for (int g2 = 0; g2 < G; ++g2) sum += red[g2 * R + c];
    npart[(int64_t)blockIdx.x * R + c] = sum;
  }
}

inline size_t bu_smem_bytes(int R, int nvec, int NS) {
  return (size_t)NS * kBdStageBytes + ((size_t)nvec * R + 2) * 16 + kBdConsumers * sizeof(double) +
         2 * NS * sizeof(uint64_t) + 16;
}

template <typename T, int CPL>
__global__ void __launch_bounds__(kThreads) colnorm2_kernel(const T* __restrict__ x, int64_t E, int R, int tpr_log2,
                                                            double* __restrict__ npart) {
  __shared__ double red[kThreads * CPL];
  const int tpr = 1 << tpr_log2;
  const int rows_per_block = kThreads >> tpr_log2;
  const int lc = threadIdx.x & (tpr - 1);
  const int c0 = lc * CPL;
  double nrm[CPL];
#pragma unroll
  for (int q = 0; q < CPL; ++q) nrm[q] = 0.0;
  if (c0 < R)
    for (int64_t row = (int64_t)blockIdx.x * rows_per_block + (threadIdx.x >> tpr_log2); row < E;
         row += (int64_t)gridDim.x * rows_per_block)
#pragma unroll
      for (int q = 0; q < CPL; ++q)
        if (c0 + q < R) {
          const T v = x[row * R + c0 + q];
          nrm[q] += (double)v.x * v.x + (double)v.y * v.y;
        }
#pragma unroll
  for (int q = 0; q < CPL; ++q) red[threadIdx.x * CPL + q] = nrm[q];
  __syncthreads();
  if ((int)threadIdx.x < tpr)
    for (int q = 0; q < CPL; ++q) {
      const int c = c0 + q;
      if (c >= R) continue;
      double s = 0.0;
      for (int r = 0; r < rows_per_block; ++r) s += red[(r * tpr + lc) * CPL + q];
      npart[(int64_t)blockIdx.x * R + c] = s;
    }
}

__global__ void reduce_cols_kernel(const double* __restrict__ part, int nparts, int R, double* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= R) return;
  double s = 0.0;
  for (int p = 0; p < nparts; ++p) s += part[(int64_t)p * R + c];
  out[c] = s;
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 conjd(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// One thread per column: Hessenberg column j from h[0..j] and ||w||, previous rotations,
// new rotation, residual estimate |g[j+1]| against the target.
// One warp per column: the lanes sum the column's norm partials (fixed order: lane l takes parts
// l, l + 32, ..., then an xor-shuffle tree) and stage the new Hessenberg column and the stored
// rotations in shared memory; lane 0 applies the rotations (a sequential chain) and forms the
// new one; the lanes write the column back.
constexpr int kGivensWarps = 4;
__global__ void __launch_bounds__(32 * kGivensWarps) givens_kernel(
    const double2* __restrict__ h, const double* __restrict__ npart, int nparts, int j, int m, int R,
    double2* __restrict__ H, double2* __restrict__ cs, double2* __restrict__ g, const double* __restrict__ target,
    int32_t* __restrict__ done, int32_t* __restrict__ kcol, double* __restrict__ scale, int32_t* __restrict__ active) {
  __shared__ double2 hs_all[kGivensWarps][64], rc_all[kGivensWarps][64], rs_all[kGivensWarps][64];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * kGivensWarps + wib;
  if (c >= R) return;
  if (done[c]) {
    if (lane == 0) scale[c] = 0.0;
    return;
  }
  double2* hs = hs_all[wib];
  double2* rc = rc_all[wib];
  double2* rs = rs_all[wib];
  double nn = 0.0;
  for (int p = lane; p < nparts; p += 32) nn += npart[(int64_t)p * R + c];
  for (int off = 16; off > 0; off >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, off);
  const double hn = sqrt(nn);
  double2* Hc = H + ((int64_t)c * m + j) * (m + 1);
  double2* csc = cs + (int64_t)c * 2 * m;
  for (int i = lane; i <= j; i += 32) hs[i] = h[i * R + c];
  for (int i = lane; i < j; i += 32) {
    rc[i] = csc[2 * i];
    rs[i] = csc[2 * i + 1];
  }
  __syncwarp();
  if (lane == 0) {
    hs[j + 1] = make_double2(hn, 0.0);
    for (int i = 0; i < j; ++i) {
      const double2 ci = rc[i], si = rs[i];
      const double2 a = hs[i], b = hs[i + 1];
      hs[i] = cadd(cmul(ci, a), cmul(si, b));
      hs[i + 1] = cadd(cmul(make_double2(-si.x, si.y), a), cmul(conjd(ci), b));  // -conj(s) a + conj(c) b
    }
    const double2 a = hs[j], b = hs[j + 1];
    const double den = sqrt(cabs2(a) + cabs2(b));
    double2 cj, sj;
    if (den == 0.0) {
      cj = make_double2(1.0, 0.0);
      sj = make_double2(0.0, 0.0);
    } else {
      cj = make_double2(a.x / den, -a.y / den);   // conj(a)/den
      sj = make_double2(b.x / den, -b.y / den);   // conj(b)/den
    }
    csc[2 * j] = cj;
    csc[2 * j + 1] = sj;
    hs[j] = make_double2(den, 0.0);
    hs[j + 1] = make_double2(0.0, 0.0);
    double2* gc = g + (int64_t)c * (m + 1);
    const double2 gj = gc[j];
    gc[j + 1] = cmul(make_double2(-sj.x, sj.y), gj);   // -conj(s) g_j
    gc[j] = cmul(cj, gj);
    const double res = sqrt(cabs2(gc[j + 1]));
    const bool stop = (res <= target[c]) || (hn == 0.0) || (j + 1 >= m) || !(res == res);
    kcol[c] = j + 1;
    if (stop) {
      done[c] = 1;
      scale[c] = 0.0;
    } else {
      scale[c] = 1.0 / hn;
      atomicAdd(active, 1);
    }
  }
  __syncwarp();
  for (int i = lane; i <= j + 1; i += 32) Hc[i] = hs[i];
}

template <typename T>
__global__ void scale_cols_kernel(T* __restrict__ v, const double* __restrict__ sc, int64_t E, int R) {
  using Sc = typename Traits<T>::S;
  const int64_t n = E * R;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const Sc s = (Sc)sc[i % R];
    T x = v[i];
    x.x *= s;
    x.y *= s;
    v[i] = x;
  }
}

// Start of a cycle: ||r|| from partials, per-column target and state; columns already within
// tol of ||b|| are marked done.
__global__ void start_state_kernel(const double* __restrict__ npart, int nparts, int R, const double* __restrict__ bnorm,
                                   double tol, double inner_tol, int fp64_mode, double* __restrict__ rnorm,
                                   double2* __restrict__ g, double* __restrict__ target, int32_t* __restrict__ done,
                                   int32_t* __restrict__ kcol, int m) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= R) return;
  double nn = 0.0;
  for (int p = 0; p < nparts; ++p) nn += npart[(int64_t)p * R + c];
  const double rn = sqrt(nn);
  rnorm[c] = rn;
  const double goal = tol * bnorm[c];
  const bool conv = !(rn > goal);
  done[c] = conv ? 1 : 0;
  kcol[c] = 0;
  double2* gc = g + (int64_t)c * (m + 1);
  for (int i = 0; i <= m; ++i) gc[i] = make_double2(0.0, 0.0);
  gc[0] = make_double2(rn, 0.0);
  // FP64 mode: aim a little below tol so the recomputed true residual passes;
  // mixed mode: reduce the residual by inner_tol (never below half the final goal).
  target[c] = fp64_mode ? 0.5 * goal : fmax(inner_tol * rn, 0.5 * goal);
}

template <typename T>
__global__ void normalize_start_kernel(const double2* __restrict__ r, const double* __restrict__ rnorm,
                                       const int32_t* __restrict__ done, int64_t E, int R, T* __restrict__ v0) {
  using Sc = typename Traits<T>::S;
  const int64_t n = E * R;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % R);
    const double s = done[c] ? 0.0 : 1.0 / rnorm[c];
    const double2 x = r[i];
    v0[i] = T{(Sc)(x.x * s), (Sc)(x.y * s)};
  }
}

// v0 = r / |r| per column from an FP32 residual (mixed mode): the column scales are formed once
// per block in shared memory, the column index advances with the grid stride.
__global__ void normalize_start32_kernel(const float2* __restrict__ r, const double* __restrict__ rnorm,
                                         const int32_t* __restrict__ done, int64_t E, int R, float2* __restrict__ v0) {
  extern __shared__ float sc[];
  for (int c = threadIdx.x; c < R; c += blockDim.x) sc[c] = done[c] ? 0.f : (float)(1.0 / rnorm[c]);
  __syncthreads();
  const int64_t n = E * R;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int step = (int)(stride % R);
  int c = (int)(i0 % R);
  for (int64_t i = i0; i < n; i += stride) {
    const float2 x = r[i];
    const float s = sc[c];
    v0[i] = make_float2(x.x * s, x.y * s);
    c += step;
    if (c >= R) c -= R;
  }
}

// Back substitution R y = g per column (R upper triangular after the rotations).
__global__ void hessenberg_solve_kernel(const double2* __restrict__ H, const double2* __restrict__ g,
                                        const int32_t* __restrict__ kcol, int m, int R, double2* __restrict__ y) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= R) return;
  const int k = kcol[c];
  double2* yc = y + (int64_t)c * m;
  const double2* gc = g + (int64_t)c * (m + 1);
  for (int i = k; i < m; ++i) yc[i] = make_double2(0.0, 0.0);
  for (int i = k - 1; i >= 0; --i) {
    double2 s = gc[i];
    for (int l = i + 1; l < k; ++l) {
      const double2 hv = H[((int64_t)c * m + l) * (m + 1) + i];
      const double2 p = cmul(hv, yc[l]);
      s.x -= p.x;
      s.y -= p.y;
    }
    const double2 d = H[((int64_t)c * m + i) * (m + 1) + i];
    const double dd = cabs2(d);
    yc[i] = dd > 0.0 ? make_double2((s.x * d.x + s.y * d.y) / dd, (s.y * d.x - s.x * d.y) / dd)
                     : make_double2(0.0, 0.0);
  }
}

// x[e][c] += sum_{i < kcol[c]} y[c][i] Z_i[e][c]; correction formed in the basis precision,
// added to x in FP64.
template <typename T>
__global__ void update_x_kernel(const T* __restrict__ Z, int64_t zstride, const double2* __restrict__ y,
                                const int32_t* __restrict__ kcol, int m, double2* __restrict__ x, int64_t E, int R) {
  using Sc = typename Traits<T>::S;
  const int64_t n = E * R;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % R);
    const int k = kcol[c];
    Sc dr = 0, di = 0;
    for (int l = 0; l < k; ++l) {
      const T z = Z[(int64_t)l * zstride + i];
      const double2 yy = y[(int64_t)c * m + l];
      const Sc yr = (Sc)yy.x, yi = (Sc)yy.y;
      dr = fma(yr, z.x, dr);
      dr = fma(-yi, z.y, dr);
      di = fma(yr, z.y, di);
      di = fma(yi, z.x, di);
    }
    double2 xv = x[i];
    xv.x += (double)dr;
    xv.y += (double)di;
    x[i] = xv;
  }
}

// The same update with Z stored as complex BF16 pairs (4 bytes per value, real in the low half):
// the correction is formed in FP32 from the widened values and added to x in FP64.
__global__ void update_x_bx_kernel(const uint32_t* __restrict__ Z, int64_t zstride, const double2* __restrict__ y,
                                   const int32_t* __restrict__ kcol, int m, double2* __restrict__ x, int64_t E, int R) {
  const int64_t n = E * R;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % R);
    const int k = kcol[c];
    float dr = 0.f, di = 0.f;
    for (int l = 0; l < k; ++l) {
      const uint32_t u = Z[(int64_t)l * zstride + i];
      const float zx = __uint_as_float(u << 16), zy = __uint_as_float(u & 0xffff0000u);
      const double2 yy = y[(int64_t)c * m + l];
      const float yr = (float)yy.x, yi = (float)yy.y;
      dr = fmaf(yr, zx, dr);
      dr = fmaf(-yi, zy, dr);
      di = fmaf(yr, zy, di);
      di = fmaf(yi, zx, di);
    }
    double2 xv = x[i];
    xv.x += (double)dr;
    xv.y += (double)di;
    x[i] = xv;
  }
}

// Stored value of Z widened to the arithmetic type: itself, or a complex BF16 pair (real in the
// low half) as complex FP32.
__device__ __forceinline__ float2 zval(float2 v) { return v; }
__device__ __forceinline__ double2 zval(double2 v) { return v; }
__device__ __forceinline__ float2 zval(uint32_t u) {
  return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}

// Streaming form of the solution update for 16 <= R <= 128 with 16-byte aligned bases, on the tiles,
// ring and thread map of cgs_dots_bulk_kernel: the producer streams Z_0 .. Z_{kmax-1} per tile
// (kmax = the largest kcol of the block); consumer (c, g) forms the correction of its rows of
// column c in the basis precision with the operations of update_x_kernel, in the same order
// (bit-identical x), and adds it to x in FP64.  y is staged in shared memory as T.  ZT is the
// stored type of Z: T, or uint32_t for complex BF16 pairs (T = float2; the widened values enter
// the same operations as update_x_bx_kernel's, bit-identical to it); the tiles keep
// bd_rows<T>() rows per row group, so BF16 tiles fill half a stage.
template <typename T, typename ZT = T>
__global__ void __launch_bounds__(kBdThreads, 2)
    update_x_bulk_kernel(const ZT* __restrict__ Z, int64_t zstride, const double2* __restrict__ y,
                         const int32_t* __restrict__ kcol, int m, double2* __restrict__ x, int64_t E, int R, int G,
                         int NS, int32_t* __restrict__ err) {
  using Sc = typename Traits<T>::S;
  constexpr int RPT = bd_rows<T>();
  constexpr int kStageElems = kBdStageBytes / (int)sizeof(ZT);
  extern __shared__ __align__(128) uint8_t ux_smem[];
  ZT* stage = reinterpret_cast<ZT*>(ux_smem);
  T* ys = reinterpret_cast<T*>(ux_smem + (size_t)NS * kBdStageBytes);   // [m][R]
  int32_t* ks = reinterpret_cast<int32_t*>(ys + (size_t)m * R);          // [R]
  uint64_t* full = reinterpret_cast<uint64_t*>(ks + ((R + 3) & ~3));
  uint64_t* empty = full + NS;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + NS);
  __shared__ int kmax_s;

  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kBdConsumers / 32);   // one arrival per consumer warp
    }
    *abort_flag = 0;
    int km = 0;
    for (int c = 0; c < R; ++c) km = max(km, min(kcol[c], m));
    kmax_s = km;
    mbar_init_fence();
  }
  for (int t = tid; t < R; t += kBdThreads) ks[t] = kcol[t];
  for (int t = tid; t < m * R; t += kBdThreads) {
    const int l = t / R, c = t - l * R;
    const double2 v = y[(int64_t)c * m + l];
    ys[t] = T{(Sc)v.x, (Sc)v.y};
  }
  __syncthreads();
  const int kmax = kmax_s;

  const int TR = G * RPT;
  const int64_t nt = (E + TR - 1) / TR;
  const int64_t t0 = nt * blockIdx.x / gridDim.x, t1 = nt * (blockIdx.x + 1) / gridDim.x;

  if (tid < 32) {
    if (tid != 0) return;
    int64_t it = 0;
    int st = 0;
    uint32_t ph = 0;
    bool stop = false;
    for (int64_t t = t0; t < t1 && !stop; ++t) {
      const int64_t r0 = t * TR;
      const int64_t rows = E - r0 < TR ? E - r0 : (int64_t)TR;
      const uint32_t bytes = (uint32_t)((rows * R * (int64_t)sizeof(ZT)) & ~(int64_t)15);
      for (int l = 0; l < kmax; ++l) {
        if (it >= NS && !mbar_wait(&empty[st], ph ^ 1u)) {
          atomicCAS(err, 0, 31);
          *abort_flag = 1;
        }
        if (*abort_flag) {
          stop = true;
          break;
        }
        const ZT* src = Z + (int64_t)l * zstride + r0 * R;
        if (bytes > 0) {
          mbar_expect_tx(&full[st], bytes);
          bulk_g2s(stage + (size_t)st * kStageElems, src, bytes, &full[st]);
        } else {
          mbar_arrive(&full[st]);
        }
        ++it;
        if (++st == NS) {
          st = 0;
          ph ^= 1u;
        }
      }
    }
    for (int k = 0; k < NS; ++k) {
      if (k >= st && it < NS) continue;
      if (!mbar_wait(&full[k], k < st ? ph : ph ^ 1u)) atomicCAS(err, 0, 32);
    }
    return;
  }

  const int ct = tid - 32;
  const int c = ct % R, g = ct / R;
  const bool act = g < G;
  const int kc = act ? ks[c] : 0;
  int st = 0;
  uint32_t ph = 0;
  for (int64_t t = t0; t < t1; ++t) {
    const int64_t r0 = t * TR;
    const int64_t rows = E - r0 < TR ? E - r0 : (int64_t)TR;
    const int64_t ncop = ((rows * R * (int64_t)sizeof(ZT)) & ~(int64_t)15) / (int64_t)sizeof(ZT);
    Sc dr[RPT], di[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) dr[k] = di[k] = 0;
    for (int l = 0; l < kmax; ++l) {
      if (!*abort_flag && !mbar_wait(&full[st], ph)) {
        atomicCAS(err, 0, 33);
        *abort_flag = 1;
      }
      if (act && l < kc) {
        const ZT* sm = stage + (size_t)st * kStageElems;
        const ZT* gl = Z + (int64_t)l * zstride + r0 * R;
        const T yy = ys[l * R + c];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
          const int row = k * G + g;
          const int f = row * R + c;
          if (row < rows) {
            const T z = zval(f < ncop ? sm[f] : gl[f]);
            dr[k] = fma(yy.x, z.x, dr[k]);
            dr[k] = fma(-yy.y, z.y, dr[k]);
            di[k] = fma(yy.x, z.y, di[k]);
            di[k] = fma(yy.y, z.x, di[k]);
          }
        }
      }
      release_stage(&empty[st]);
      if (++st == NS) {
        st = 0;
        ph ^= 1u;
      }
    }
    if (act && !*abort_flag) {
      double2* xr = x + r0 * R;
#pragma unroll
      for (int k = 0; k < RPT; ++k) {
        const int row = k * G + g;
        if (row < rows) {
          double2 xv = xr[row * R + c];
          xv.x += (double)dr[k];
          xv.y += (double)di[k];
          xr[row * R + c] = xv;
        }
      }
    }
  }
}

inline size_t ux_smem_bytes(int R, int m, int NS) {
  return (size_t)NS * kBdStageBytes + (size_t)m * R * 16 + ((R + 3) & ~3) * 4 + 2 * NS * sizeof(uint64_t) + 16;
}

template <typename T, typename ZT = T>
bool update_x_bulk(const ZT* Z, int64_t zstride, const double2* y, const int32_t* kcol, int m, double2* x, int64_t E,
                   int R, int32_t* err, cudaStream_t s) {
  const bool aligned = ((uintptr_t)Z % 16 == 0) && ((zstride * sizeof(ZT)) % 16 == 0);
  if (!err || !aligned || R < 16 || R > 128 || m < 1) return false;
  static bool attr = false;   // one per instantiation
  if (!attr) {
    // 226 KB: the kernel's static shared memory shares the 227 KB per block
    attr = cudaFuncSetAttribute(update_x_bulk_kernel<T, ZT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                226 * 1024) == cudaSuccess;
  }
  int NS = kBdStages;
  while (NS > 2 && ux_smem_bytes(R, m, NS) > (size_t)226 * 1024) --NS;
  update_x_bulk_kernel<T, ZT><<<152 * 2, kBdThreads, ux_smem_bytes(R, m, NS), s>>>(Z, zstride, y, kcol, m, x, E, R,
                                                                                  kBdConsumers / R, NS, err);
  return true;
}

inline int gs_blocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 8 ? (b > 0 ? b : 1) : 152 * 8);
}

template <typename T>
int dots_launch(const T* V, int64_t vstride, int nvec, const T* w, int64_t E, int R, double2* part, int32_t* err,
                cudaStream_t s, int stages) {
  note_launch(1);
  const bool aligned = ((uintptr_t)V % 16 == 0) && ((uintptr_t)w % 16 == 0) && ((vstride * sizeof(T)) % 16 == 0);
  if (err && aligned && R >= 16 && R <= 128 && nvec >= 1) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(cgs_dots_bulk_kernel<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kBdMaxSmem);
      cudaFuncSetAttribute(cgs_dots_bulk_kernel<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kBdMaxSmem);
      attr = true;
    }
    const int G = kBdConsumers / R;
    const int VG = std::min(64, 2048 / R);
    const int nb = 152 * 2;
    const int NS = stages >= 2 && stages <= kBdMaxStages ? stages : kBdStages;
    cgs_dots_bulk_kernel<T>
        <<<nb, kBdThreads, bd_smem_bytes(R, NS, sizeof(T)), s>>>(V, vstride, nvec, w, E, R, G, VG, NS, part, err);
    return nb;
  }
  Shape sh = shape_for(R);
  const int S = nvec >= kDotWarps ? 1 : kDotWarps / nvec;
  switch (sh.cpl) {
    case 1:
      cgs_dots_kernel<T, 1><<<kBlocks, kDotThreads, 0, s>>>(V, vstride, nvec, w, E, R, sh.tpr_log2, S, part);
      break;
    case 2:
      cgs_dots_kernel<T, 2><<<kBlocks, kDotThreads, 0, s>>>(V, vstride, nvec, w, E, R, sh.tpr_log2, S, part);
      break;
    default:
      cgs_dots_kernel<T, 4><<<kBlocks, kDotThreads, 0, s>>>(V, vstride, nvec, w, E, R, sh.tpr_log2, S, part);
      break;
  }
  return kBlocks * S;
}

template <typename T>
int update_launch(const T* V, int64_t vstride, int nvec, const double2* h, T* w, int64_t E, int R, double* npart,
                  cudaStream_t s, int32_t* err, int stages, const double* vscale) {
  note_launch(1);
  const bool aligned = ((uintptr_t)V % 16 == 0) && ((uintptr_t)w % 16 == 0) && ((vstride * sizeof(T)) % 16 == 0);
  if (err && aligned && R >= 16 && R <= 128 && nvec >= 1) {
    static bool attr = false;
    if (!attr) {
      attr = cudaFuncSetAttribute(cgs_update_bulk_kernel<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  226 * 1024) == cudaSuccess &&
             cudaFuncSetAttribute(cgs_update_bulk_kernel<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  226 * 1024) == cudaSuccess;
    }
    int NS = stages >= 2 && stages <= kBdMaxStages ? stages : kBdStages;
    while (NS > 2 && bu_smem_bytes(R, nvec, NS) > (size_t)226 * 1024) --NS;
    const int G = kBdConsumers / R;
    const int nb = 152 * 2;
    cgs_update_bulk_kernel<T>
        <<<nb, kBdThreads, bu_smem_bytes(R, nvec, NS), s>>>(V, vstride, nvec, h, w, E, R, G, NS, npart, err, vscale);
    return nb;
  }
  Shape sh = shape_for(R);
  const size_t smem = sizeof(T) * nvec * R + 16 + sizeof(double) * kThreads * sh.cpl;
  static bool attr = false;
  if (!attr) {
    const int mx = 200 * 1024;
    cudaFuncSetAttribute(cgs_update_kernel<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(cgs_update_kernel<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(cgs_update_kernel<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    attr = true;
  }
  switch (sh.cpl) {
    case 1:
      cgs_update_kernel<T, 1>
          <<<kBlocks, kThreads, smem, s>>>(V, vstride, nvec, h, w, E, R, sh.tpr_log2, npart, vscale);
      break;
    case 2:
      cgs_update_kernel<T, 2>
          <<<kBlocks, kThreads, smem, s>>>(V, vstride, nvec, h, w, E, R, sh.tpr_log2, npart, vscale);
      break;
    default:
      cgs_update_kernel<T, 4>
          <<<kBlocks, kThreads, smem, s>>>(V, vstride, nvec, h, w, E, R, sh.tpr_log2, npart, vscale);
      break;
  }
  return kBlocks;
}

__global__ void fill_f64_kernel(double* __restrict__ x, int n, double v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = v;
}

// Deterministic pseudo-random fill in [-1, 1) (timing inputs of the launch-shape tuner).
template <typename F>
__global__ void fill_pattern_kernel(F* __restrict__ x, int64_t n, uint32_t seed, double scale) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)i * 2654435761u ^ seed;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    x[i] = (F)(scale * ((double)(h >> 8) * (1.0 / 8388608.0) - 1.0));
  }
}

// Sets the conditional handles of one captured Arnoldi step: the step's bodies run while some
// column of the block is still active.
struct StepHandles {
  cudaGraphConditionalHandle h[kMaxStepHandles];
  int n;
};
__global__ void set_step_conditions_kernel(StepHandles sh, const int32_t* __restrict__ active) {
  const unsigned v = *active != 0 ? 1u : 0u;
  for (int i = 0; i < sh.n; ++i) cudaGraphSetConditional(sh.h[i], v);
}

}  // namespace

void fill_f64(double* x, int n, double v, cudaStream_t s) {
  note_launch(1);
  fill_f64_kernel<<<(n + 255) / 256 < 64 ? (n + 255) / 256 : 64, 256, 0, s>>>(x, n, v);
}
void fill_pattern_f32(float* x, int64_t n, uint32_t seed, cudaStream_t s, double scale) {
  note_launch(1);
  fill_pattern_kernel<float><<<gs_blocks(n), 256, 0, s>>>(x, n, seed, scale);
}
void fill_pattern_f64(double* x, int64_t n, uint32_t seed, cudaStream_t s, double scale) {
  note_launch(1);
  fill_pattern_kernel<double><<<gs_blocks(n), 256, 0, s>>>(x, n, seed, scale);
}

void set_step_conditions(const unsigned long long* handles, int n, const int32_t* active, cudaStream_t s) {
  note_launch(1);
  StepHandles sh;
  sh.n = n < kMaxStepHandles ? n : kMaxStepHandles;
  for (int i = 0; i < sh.n; ++i) sh.h[i] = (cudaGraphConditionalHandle)handles[i];
  set_step_conditions_kernel<<<1, 1, 0, s>>>(sh, active);
}

int cgs_dots_f64(const double2* V, int64_t vstride, int nvec, const double2* w, int64_t E, int R, double2* part,
                 int32_t* err, cudaStream_t s, int stages) {
  return dots_launch<double2>(V, vstride, nvec, w, E, R, part, err, s, stages);
}
int cgs_dots_f32(const float2* V, int64_t vstride, int nvec, const float2* w, int64_t E, int R, double2* part,
                 int32_t* err, cudaStream_t s, int stages) {
  return dots_launch<float2>(V, vstride, nvec, w, E, R, part, err, s, stages);
}
void reduce_h(const double2* part, int nparts, int nvec, int R, double2* h, cudaStream_t s, const double* vscale) {
  note_launch(1);
  const int n = nvec * R;
  reduce_h_kernel<<<(n * 32 + 255) / 256, 256, 0, s>>>(part, nparts, nvec, R, h, vscale);
}
int cgs_update_f64(const double2* V, int64_t vstride, int nvec, const double2* h, double2* w, int64_t E, int R,
                   double* npart, cudaStream_t s, int32_t* err, int stages, const double* vscale) {
  return update_launch<double2>(V, vstride, nvec, h, w, E, R, npart, s, err, stages, vscale);
}
int cgs_update_f32(const float2* V, int64_t vstride, int nvec, const double2* h, float2* w, int64_t E, int R,
                   double* npart, cudaStream_t s, int32_t* err, int stages, const double* vscale) {
  return update_launch<float2>(V, vstride, nvec, h, w, E, R, npart, s, err, stages, vscale);
}
int colnorm2_f64(const double2* x, int64_t E, int R, double* npart, cudaStream_t s) {
  note_launch(1);
  Shape sh = shape_for(R);
  switch (sh.cpl) {
    case 1:
      colnorm2_kernel<double2, 1><<<kBlocks, kThreads, 0, s>>>(x, E, R, sh.tpr_log2, npart);
      break;
    case 2:
      colnorm2_kernel<double2, 2><<<kBlocks, kThreads, 0, s>>>(x, E, R, sh.tpr_log2, npart);
      break;
    default:
      colnorm2_kernel<double2, 4><<<kBlocks, kThreads, 0, s>>>(x, E, R, sh.tpr_log2, npart);
      break;
  }
  return kBlocks;
}
void reduce_cols(const double* part, int nparts, int R, double* out, cudaStream_t s) {
  note_launch(1);
  reduce_cols_kernel<<<(R + 127) / 128, 128, 0, s>>>(part, nparts, R, out);
}
void givens_step(const double2* h, const double* npart, int nparts, int j, int m, int R, double2* H, double2* cs,
                 double2* gvec, double* target, int32_t* done, int32_t* kcol, double* scale, int32_t* active_count,
                 cudaStream_t s) {
  note_launch(1);
  givens_kernel<<<(R + kGivensWarps - 1) / kGivensWarps, 32 * kGivensWarps, 0, s>>>(
      h, npart, nparts, j, m, R, H, cs, gvec, target, done, kcol, scale, active_count);
}
void scale_cols_f64(double2* v, const double* scale, int64_t E, int R, cudaStream_t s) {
  note_launch(1);
  scale_cols_kernel<double2><<<gs_blocks(E * R), 256, 0, s>>>(v, scale, E, R);
}
void scale_cols_f32(float2* v, const double* scale, int64_t E, int R, cudaStream_t s) {
  note_launch(1);
  scale_cols_kernel<float2><<<gs_blocks(E * R), 256, 0, s>>>(v, scale, E, R);
}
void start_state(const double* npart, int nparts, int R, const double* bnorm, double tol, double inner_tol,
                 int fp64_mode, double* rnorm, double2* gvec, double* target, int32_t* done, int32_t* kcol, int m,
                 cudaStream_t s) {
  note_launch(1);
  start_state_kernel<<<(R + 127) / 128, 128, 0, s>>>(npart, nparts, R, bnorm, tol, inner_tol, fp64_mode, rnorm, gvec,
                                                      target, done, kcol, m);
}
void normalize_start_f64(const double2* r, const double* rnorm, const int32_t* done, int64_t E, int R, double2* v0,
                         cudaStream_t s) {
  note_launch(1);
  normalize_start_kernel<double2><<<gs_blocks(E * R), 256, 0, s>>>(r, rnorm, done, E, R, v0);
}
void normalize_start_f32(const double2* r, const double* rnorm, const int32_t* done, int64_t E, int R, float2* v0,
                         cudaStream_t s) {
  note_launch(1);
  normalize_start_kernel<float2><<<gs_blocks(E * R), 256, 0, s>>>(r, rnorm, done, E, R, v0);
}
void normalize_start32(const float2* r, const double* rnorm, const int32_t* done, int64_t E, int R, float2* v0,
                       cudaStream_t s) {
  note_launch(1);
  normalize_start32_kernel<<<gs_blocks(E * R), 256, sizeof(float) * R, s>>>(r, rnorm, done, E, R, v0);
}
void solve_hessenberg(const double2* H, const double2* gvec, const int32_t* kcol, int m, int R, double2* y,
                      cudaStream_t s) {
  note_launch(1);
  hessenberg_solve_kernel<<<(R + 127) / 128, 128, 0, s>>>(H, gvec, kcol, m, R, y);
}
void update_x_f64(const double2* Z, int64_t zstride, const double2* y, const int32_t* kcol, int m, double2* x,
                  int64_t E, int R, cudaStream_t s, int32_t* err) {
  note_launch(1);
  if (update_x_bulk<double2>(Z, zstride, y, kcol, m, x, E, R, err, s)) return;
  update_x_kernel<double2><<<gs_blocks(E * R), 256, 0, s>>>(Z, zstride, y, kcol, m, x, E, R);
}
void update_x_bx(const void* Z, int64_t zstride, const double2* y, const int32_t* kcol, int m, double2* x, int64_t E,
                 int R, cudaStream_t s, int32_t* err) {
  note_launch(1);
  if (update_x_bulk<float2, uint32_t>((const uint32_t*)Z, zstride, y, kcol, m, x, E, R, err, s)) return;
  update_x_bx_kernel<<<gs_blocks(E * R), 256, 0, s>>>((const uint32_t*)Z, zstride, y, kcol, m, x, E, R);
}
void update_x_f32(const float2* Z, int64_t zstride, const double2* y, const int32_t* kcol, int m, double2* x,
                  int64_t E, int R, cudaStream_t s, int32_t* err) {
  note_launch(1);
  if (update_x_bulk<float2>(Z, zstride, y, kcol, m, x, E, R, err, s)) return;
  update_x_kernel<float2><<<gs_blocks(E * R), 256, 0, s>>>(Z, zstride, y, kcol, m, x, E, R);
}

}  // namespace mwk
