// Sparse subdomain solves of the ORAS preconditioner (Sec. IV-C): multifrontal LU on a
// nested-dissection tree per subdomain, FP32 complex.
//
// Factorisation, per subdomain, fronts row-major in a workspace:
//   1. mf_assemble_kernel: the original entries of B_s (element and face terms, as in the dense
//      local assembly, plus ones on the diagonal of metal and padding pivots), pulled per front
//      entry in a fixed order;
//   2. per tree height, leaves first: mf_extend_add_kernel adds the children's Schur complements
//      into each front, the partial Gauss-Jordan eliminates its pivots, and mf_extract_kernel keeps
//      TL | TR (the pivot rows) and BL (the update rows' pivot columns).
// Solve z = B_s^-1 r for R columns, every subdomain at once, per height:
//   forward (leaves first):  rhs_k = [r(pivots); 0] + the children's w mapped into the front,
//                            t_k = TL rhs_k(p),  w_k = rhs_k(u) + BL rhs_k(p);
//   backward (root first):   x(pivots of k) = t_k - TR x(update dofs of k);
//   then z(owned) = x(owned).
// The products are one task-list GEMM launch per height and direction (mf_gemm_kernel).
#include <algorithm>

#include "k_mf.h"
#include "mw_internal.h"

namespace mwk {
namespace {

__device__ __forceinline__ double2 csqrt_pr(double a, double b) {
  const double r = sqrt(a * a + b * b);
  const double re = sqrt(0.5 * (r + a));
  double im = sqrt(fmax(0.0, 0.5 * (r - a)));
  if (b < 0.0) im = -im;
  return make_double2(re, im);
}

// One thread per front entry that receives original contributions; the value is summed in FP64
// in the code order of the pull map, then rounded to FP32.
__global__ void mf_assemble_kernel(const int64_t* __restrict__ ptr, const int64_t* __restrict__ target,
                                   const int32_t* __restrict__ code, int64_t n_t, const int32_t* __restrict__ tet_ids,
                                   const double* __restrict__ KM, const double* __restrict__ eps, double k0,
                                   const double* __restrict__ Bsurf, const int32_t* __restrict__ surf_tet,
                                   double ebr, double ebi, const double2* __restrict__ zc, float2* __restrict__ ws) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_t) return;
  const double k0sq = k0 * k0;
  double re = 0.0, im = 0.0;
  for (int64_t q = ptr[i]; q < ptr[i + 1]; ++q) {
    const int32_t c = code[q];
    if (c == INT32_MIN) {
      re += 1.0;
    } else if (c >= 0) {
      const int64_t slot = c / 36;
      const int r = c - (int)slot * 36;
      const int64_t t = tet_ids[slot];
      const int pk = mw::packed6(r / 6, r % 6);
      const double Kv = KM[42 * t + pk], Mv = KM[42 * t + 21 + pk];
      re += Kv - (k0sq * eps[2 * t]) * Mv;
      im += -(k0sq * eps[2 * t + 1]) * Mv;
    } else {
      const int64_t q9 = -(int64_t)c - 1;
      const int64_t slot = q9 / 9;
      const int r = (int)(q9 - slot * 9);
      const double Bv = Bsurf[6 * slot + mw::packed3(r / 3, r % 3)];
      const int32_t it = surf_tet[slot];
      if (it < 0 && zc) {
        const double2 z = zc[-1 - it];
        re += z.x * Bv;
        im += z.y * Bv;
      } else {
        const double2 sq = it >= 0 ? csqrt_pr(eps[2 * (int64_t)it], eps[2 * (int64_t)it + 1]) : csqrt_pr(ebr, ebi);
        re += (-k0 * sq.y) * Bv;
        im += (k0 * sq.x) * Bv;
      }
    }
  }
  ws[target[i]] = make_float2((float)re, (float)im);
}

// Front entry (r, c) of node nodes[blockIdx.y] += sum over its children of S_child(inv(r), inv(c)).
__global__ void mf_extend_add_kernel(const int32_t* __restrict__ nodes, const int64_t* __restrict__ f,
                                     const int32_t* __restrict__ p, const int64_t* __restrict__ ws_off,
                                     const int64_t* __restrict__ child_ptr, const int32_t* __restrict__ child,
                                     const int64_t* __restrict__ inv_off, const int32_t* __restrict__ inv,
                                     float2* __restrict__ ws) {
  const int32_t k = nodes[blockIdx.y];
  const int64_t fk = f[k];
  const int64_t c0 = child_ptr[k], c1 = child_ptr[k + 1];
  if (c0 == c1) return;
  float2* F = ws + ws_off[k];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < fk * fk; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / fk, c = e - r * fk;
    float sx = 0.f, sy = 0.f;
    bool any = false;
    for (int64_t q = c0; q < c1; ++q) {
      const int32_t ch = child[q];
      const int32_t* m = inv + inv_off[ch];
      const int32_t a = m[r], b = m[c];
      if (a >= 0 && b >= 0) {
        const int64_t fc = f[ch], pc = p[ch];
        const float2 v = ws[ws_off[ch] + (pc + a) * fc + pc + b];
        sx += v.x;
        sy += v.y;
        any = true;
      }
    }
    if (any) {
      float2 v = F[e];
      v.x += sx;
      v.y += sy;
      F[e] = v;
    }
  }
}

// Keep the factors of nodes[blockIdx.y]: rows [0, p) of the front (TL | TR, p x f) then the
// pivot columns of rows [p, f) (BL, u x p).
__global__ void mf_extract_kernel(const int32_t* __restrict__ nodes, const int64_t* __restrict__ f,
                                  const int32_t* __restrict__ p, const int64_t* __restrict__ ws_off,
                                  const int64_t* __restrict__ fac_off, const float2* __restrict__ ws,
                                  float2* __restrict__ fac) {
  const int32_t k = nodes[blockIdx.y];
  const int64_t fk = f[k], pk = p[k], uk = fk - pk;
  const float2* F = ws + ws_off[k];
  float2* D = fac + fac_off[k];
  const int64_t n1 = pk * fk, n2 = uk * pk;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n1 + n2; e += (int64_t)gridDim.x * blockDim.x) {
    if (e < n1) {
      D[e] = F[e];
    } else {
      const int64_t q = e - n1, r = q / pk, c = q - r * pk;
      D[e] = F[(pk + r) * fk + c];
    }
  }
}

// Front right-hand sides as a pull: arena row out[i] = sum over src[ptr[i] .. ptr[i+1]) of the
// arena row src (>= 0) or input row -(src + 1), in list order (input first, then the children
// in child order, as the multifrontal forward sweep assembles them).  One thread per (row,
// column): a row's R columns are contiguous, so each source row is read coalesced.
__global__ void mf_pull_kernel(const int64_t* __restrict__ out, const int64_t* __restrict__ ptr,
                               const int64_t* __restrict__ src, int64_t n, const float2* __restrict__ in, int R,
                               float2* __restrict__ arena) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * R; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / R;
    const int c = (int)(t - i * R);
    float sx = 0.f, sy = 0.f;
    for (int64_t q = ptr[i]; q < ptr[i + 1]; ++q) {
      const int64_t g = src[q];
      const float2 v = g >= 0 ? arena[g * R + c] : in[(-g - 1) * R + c];
      sx += v.x;
      sy += v.y;
    }
    arena[out[i] * R + c] = make_float2(sx, sy);
  }
}

// The same pull with 4 consecutive complex columns per thread (R a multiple of 4) and NR rows
// per thread, rows i, i + nq, i + 2 nq, ... (nq = ceil(n / NR)): 32-byte loads and stores, and
// the rows' index chains run side by side.  Each row's sums are the same, in the same order.
template <int NR>
__global__ void mf_pull4_kernel(const int64_t* __restrict__ out, const int64_t* __restrict__ ptr,
                                const int64_t* __restrict__ src, int64_t n, const float2* __restrict__ in, int R,
                                float2* __restrict__ arena) {
  const int tpr = R / 4;
  const int64_t nq = (n + NR - 1) / NR;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nq * tpr) return;
  const int64_t i0 = t / tpr;
  const int c = (int)(t - i0 * tpr) * 4;
  float4 a[NR], b[NR];   // columns c, c+1 | c+2, c+3 of each row
  int64_t q[NR], qe[NR];
  bool more = false;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const int64_t i = i0 + r * nq;
    a[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    b[r] = a[r];
    q[r] = i < n ? ptr[i] : 0;
    qe[r] = i < n ? ptr[i + 1] : 0;
    more |= q[r] < qe[r];
  }
  while (more) {
    more = false;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (q[r] < qe[r]) {
        const int64_t g = src[q[r]++];
        const float4* v = reinterpret_cast<const float4*>(g >= 0 ? arena + g * R + c : in + (-g - 1) * R + c);
        const float4 v0 = v[0], v1 = v[1];
        a[r].x += v0.x;
        a[r].y += v0.y;
        a[r].z += v0.z;
        a[r].w += v0.w;
        b[r].x += v1.x;
        b[r].y += v1.y;
        b[r].z += v1.z;
        b[r].w += v1.w;
      }
      more |= q[r] < qe[r];
    }
  }
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const int64_t i = i0 + r * nq;
    if (i >= n) continue;
    float4* o = reinterpret_cast<float4*>(arena + out[i] * R + c);
    o[0] = a[r];
    o[1] = b[r];
  }
}

// Task-list GEMM: C = C0 + sign * A B for every task, A [m][k] (row stride lda) in the factor
// store, B [k][R] and C, C0 [m][R] in the vector arena.  Rows of B and C are either consecutive
// from an arena row or listed (b_idx / c_idx; a negative C row is skipped).  A CTA of 128
// threads computes a 64-row x 32-column tile, each thread 4 rows x 4 columns (rows tr + 16 i,
// columns tc + 8 j), over K chunks of 32 staged in shared memory; tile_task / tile_row0 list
// the 64-row tiles of all tasks.
constexpr int kMfRows = 64, kMfK = 32, kMfCols = 32, kMfThreads = 128;

//
// Split K: a tile with tile_slot >= 0 covers only K range [tile_k0, tile_k1) and writes its raw
// partial product to partial slot tile_slot ([64][R]); mf_reduce_kernel then sums the slots of
// each (task, row tile) in slot order and applies C0, the sign and the row list.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(gmem), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Shared-memory stages of the sweep GEMM: A [64][33] and B [32][33] complex FP32, two of each.
constexpr int kMfAStage = kMfRows * (kMfK + 1), kMfBStage = kMfK * (kMfCols + 1);
constexpr size_t kMfSmem = sizeof(float2) * 2 * (kMfAStage + kMfBStage);

__global__ void __launch_bounds__(kMfThreads) mf_gemm_kernel(const MfTask* __restrict__ tasks,
                                                             const MfTile* __restrict__ tiles,
                                                             const float2* __restrict__ fac,
                                                             const int32_t* __restrict__ idx, int R,
                                                             float2* __restrict__ arena,
                                                             float2* __restrict__ partial) {
  extern __shared__ float2 sm2[];
  const MfTile tl = tiles[blockIdx.x];
  const MfTask T = tasks[tl.task];
  const int64_t row0 = tl.row0;
  const int64_t kbeg = tl.k0, kend = min((int64_t)tl.k1, T.k);
  const int col0 = blockIdx.y * kMfCols;
  const int tr = threadIdx.x / 8, tc = threadIdx.x % 8;
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  const float2* A = fac + T.a_off;
  // copies of one K chunk into stage st (out-of-range entries are zero-filled)
  auto load = [&](int64_t k0, int st) {
    float2* As = sm2 + st * kMfAStage;
    float2* Bs = sm2 + 2 * kMfAStage + st * kMfBStage;
    for (int e = threadIdx.x; e < kMfRows * kMfK; e += kMfThreads) {
      const int r = e / kMfK, kk = e % kMfK;
      const int64_t gr = row0 + r, gk = k0 + kk;
      const bool ok = gr < T.m && gk < kend;
      cp_async8(As + r * (kMfK + 1) + kk, ok ? (const void*)(A + gr * T.lda + gk) : (const void*)A, ok);
    }
    for (int e = threadIdx.x; e < kMfK * kMfCols; e += kMfThreads) {
      const int kk = e / kMfCols, c = e % kMfCols;
      const int64_t gk = k0 + kk;
      const bool ok = gk < kend && col0 + c < R;
      const float2* src = arena;
      if (ok) {
        const int64_t brow = T.b_idx >= 0 ? (int64_t)idx[T.b_idx + gk] : T.b_row + gk;
        src = arena + brow * R + col0 + c;
      }
      cp_async8(Bs + kk * (kMfCols + 1) + c, src, ok);
    }
    cp_async_commit();
  };
  if (kbeg < kend) load(kbeg, 0);
  int st = 0;
  for (int64_t k0 = kbeg; k0 < kend; k0 += kMfK, st ^= 1) {
    if (k0 + kMfK < kend) {
      load(k0 + kMfK, st ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float2* As = sm2 + st * kMfAStage;
    const float2* Bs = sm2 + 2 * kMfAStage + st * kMfBStage;
#pragma unroll 4
    for (int kk = 0; kk < kMfK; ++kk) {
      float2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[(tr + 16 * i) * (kMfK + 1) + kk];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk * (kMfCols + 1) + tc + 8 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fmaf(a[i].x, b[j].x, acc[i][j].x);
          acc[i][j].x = fmaf(-a[i].y, b[j].y, acc[i][j].x);
          acc[i][j].y = fmaf(a[i].x, b[j].y, acc[i][j].y);
          acc[i][j].y = fmaf(a[i].y, b[j].x, acc[i][j].y);
        }
    }
    __syncthreads();
  }
  if (tl.slot >= 0) {
    float2* P = partial + (int64_t)tl.slot * kMfRows * R;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = col0 + tc + 8 * j;
        if (c < R) P[(int64_t)(tr + 16 * i) * R + c] = acc[i][j];
      }
    return;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gr = row0 + tr + 16 * i;
    if (gr >= T.m) continue;
    const int64_t crow = T.c_idx >= 0 ? (int64_t)idx[T.c_idx + gr] : T.c_row + gr;
    if (crow < 0) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = col0 + tc + 8 * j;
      if (c >= R) continue;
      float2 v = make_float2(T.sign * acc[i][j].x, T.sign * acc[i][j].y);
      if (T.c0_row >= 0) {
        const float2 c0 = arena[(T.c0_row + gr) * R + c];
        v.x += c0.x;
        v.y += c0.y;
      }
      arena[crow * R + c] = v;
    }
  }
}

// One CTA per split (task, row tile): the sum of its partial slots in slot order, then the
// epilogue of mf_gemm_kernel.
__global__ void mf_reduce_kernel(const MfTask* __restrict__ tasks, const MfSplit* __restrict__ splits,
                                 const float2* __restrict__ partial, const int32_t* __restrict__ idx, int R,
                                 float2* __restrict__ arena) {
  const MfSplit sp = splits[blockIdx.x];
  const MfTask T = tasks[sp.task];
  for (int e = threadIdx.x; e < kMfRows * R; e += blockDim.x) {
    const int r = e / R, c = e % R;
    const int64_t gr = sp.row0 + r;
    if (gr >= T.m) continue;
    const int64_t crow = T.c_idx >= 0 ? (int64_t)idx[T.c_idx + gr] : T.c_row + gr;
    if (crow < 0) continue;
    float sx = 0.f, sy = 0.f;
    for (int q = 0; q < sp.n_slots; ++q) {
      const float2 v = partial[((int64_t)(sp.slot0 + q) * kMfRows + r) * R + c];
      sx += v.x;
      sy += v.y;
    }
    float2 v = make_float2(T.sign * sx, T.sign * sy);
    if (T.c0_row >= 0) {
      const float2 c0 = arena[(T.c0_row + gr) * R + c];
      v.x += c0.x;
      v.y += c0.y;
    }
    arena[crow * R + c] = v;
  }
}

// z(own_glob[q]) = x(own_row[q]) for every owned dof.
__global__ void mf_owned_kernel(const int32_t* __restrict__ own_glob, const int64_t* __restrict__ own_row,
                                int64_t n_own, const float2* __restrict__ arena, int R, float2* __restrict__ z) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_own * R) return;
  const int64_t q = t / R;
  const int c = (int)(t - q * R);
  z[(int64_t)own_glob[q] * R + c] = arena[own_row[q] * R + c];
}

unsigned grid_for(int64_t n, int threads, int64_t cap = 152 * 32) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, cap));
}

}  // namespace

void mf_assemble(const int64_t* ptr, const int64_t* target, const int32_t* code, int64_t n_t, const int32_t* tet_ids,
                 const double* KM, const double* eps, double k0, const double* Bsurf, const int32_t* surf_tet,
                 double ebr, double ebi, const double2* zc, float2* ws, cudaStream_t s) {
  if (n_t <= 0) return;
  note_launch(1);
  mf_assemble_kernel<<<(unsigned)((n_t + 255) / 256), 256, 0, s>>>(ptr, target, code, n_t, tet_ids, KM, eps, k0,
                                                                    Bsurf, surf_tet, ebr, ebi, zc, ws);
}

void mf_extend_add(const int32_t* nodes, int n_nodes, int64_t fmax, const int64_t* f, const int32_t* p,
                   const int64_t* ws_off, const int64_t* child_ptr, const int32_t* child, const int64_t* inv_off,
                   const int32_t* inv, float2* ws, cudaStream_t s) {
  if (n_nodes <= 0) return;
  note_launch(1);
  dim3 g(grid_for(fmax * fmax, 256, 1024), n_nodes);
  mf_extend_add_kernel<<<g, 256, 0, s>>>(nodes, f, p, ws_off, child_ptr, child, inv_off, inv, ws);
}

void mf_extract(const int32_t* nodes, int n_nodes, int64_t max_entries, const int64_t* f, const int32_t* p,
                const int64_t* ws_off, const int64_t* fac_off, const float2* ws, float2* fac, cudaStream_t s) {
  if (n_nodes <= 0) return;
  note_launch(1);
  dim3 g(grid_for(max_entries, 256, 1024), n_nodes);
  mf_extract_kernel<<<g, 256, 0, s>>>(nodes, f, p, ws_off, fac_off, ws, fac);
}

void mf_gemm(const MfTask* tasks, const MfTile* tiles, int n_tiles, const MfSplit* splits, int n_splits,
             const float2* fac, const int32_t* idx, int R, float2* arena, float2* partial, cudaStream_t s) {
  if (n_tiles <= 0) return;
  note_launch(1);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(mf_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMfSmem);
    attr = true;
  }
  dim3 g((unsigned)n_tiles, (unsigned)((R + kMfCols - 1) / kMfCols));
  mf_gemm_kernel<<<g, kMfThreads, kMfSmem, s>>>(tasks, tiles, fac, idx, R, arena, partial);
  if (n_splits > 0) {
    note_launch(1);
    mf_reduce_kernel<<<n_splits, 256, 0, s>>>(tasks, splits, partial, idx, R, arena);
  }
}

void mf_reduce(const MfTask* tasks, const MfSplit* splits, int n_splits, const float2* partial, const int32_t* idx,
               int R, float2* arena, cudaStream_t s) {
  if (n_splits <= 0) return;
  note_launch(1);
  mf_reduce_kernel<<<n_splits, 256, 0, s>>>(tasks, splits, partial, idx, R, arena);
}

void mf_pull(const int64_t* out, const int64_t* ptr, const int64_t* src, int64_t n, const float2* in, int R,
             float2* arena, cudaStream_t s) {
  if (n <= 0) return;
  note_launch(1);
  if (R % 4 == 0 && R <= 128 && (((uintptr_t)in | (uintptr_t)arena) & 15) == 0) {
    // 4 complex columns and kPullRows rows per thread: a warp takes 32 kPullRows / (R / 4) rows
    // with independent load chains
    constexpr int kPullRows = 2;   // measured on the 16-subdomain shoulder: faster than 4 rows
    const int64_t thr = (n + kPullRows - 1) / kPullRows * (R / 4);
    mf_pull4_kernel<kPullRows><<<(unsigned)((thr + 255) / 256), 256, 0, s>>>(out, ptr, src, n, in, R, arena);
    return;
  }
  const int64_t thr = n * R;
  const int blocks = (int)std::min<int64_t>((thr + 255) / 256, 152 * 16);
  mf_pull_kernel<<<blocks, 256, 0, s>>>(out, ptr, src, n, in, R, arena);
}
void mf_owned(const int32_t* own_glob, const int64_t* own_row, int64_t n_own, const float2* arena, int R, float2* z,
              cudaStream_t s) {
  if (n_own <= 0) return;
  note_launch(1);
  const int64_t n = n_own * R;
  mf_owned_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(own_glob, own_row, n_own, arena, R, z);
}

}  // namespace mwk
