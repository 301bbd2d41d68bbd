// K4 on the tensor cores: z[own_s] = W_s r[dofs_s] for every subdomain s, as BF16 x BF16 -> FP32
// tcgen05 MMAs with the accumulator in tensor memory (Sec. IV-C: the subdomain solves of the
// one-level ORAS preconditioner, applied through precomputed owned-row inverses).
//
// Complex product as two real GEMMs on split planes.  W = Wr + i Wi is stored as two BF16 planes
// and the gathered input g = gr + i gi once, as B = [gr | gi] (N = 2 R_pad columns: column c
// holds gr_c, column R_pad + c holds gi_c).  Two accumulators D1 = Wr B and D2 = Wi B give
//   Re z_c = D1[c] - D2[R_pad + c],   Im z_c = D1[R_pad + c] + D2[c].
// Each complex input value is staged once (2 BF16), half the bytes of an interleaved real-GEMM
// form that needs (gr, -gi) and (gi, gr); the FLOPs and the W bytes are the same.
//
// Layouts.  All operands are K-major with the 128-byte swizzle: a tile row holds 64 BF16 of K
// (128 B, K = 64 subdomain dofs); the 16-byte chunk c of row r sits at chunk c ^ (r % 8); 8-row
// groups are 1024 B apart.  W_s is pre-tiled at setup into 128-row x 64-dof tile pairs (Wr tile,
// then Wi tile: 32 KB contiguous, in that swizzled order), so one bulk copy moves a pair into
// shared memory without a tensor map.  The gathered operand of each subdomain is written per
// apply into N x 64-dof tiles.
//
// Kernel roles (192 threads): warp 0 lane 0 issues the bulk copies, warp 1 allocates tensor
// memory and lane 0 issues the MMAs, warps 2-5 read the accumulator (tcgen05.ld) and scatter
// the owned rows.  Every mbarrier wait is bounded; on timeout the kernel records an error code,
// drains its outstanding copies (again bounded), frees tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "k_oras.h"
#include "k_oras_tc.h"
#include "k_mf.h"
#include "mw_async.cuh"
#include "mw_internal.h"

namespace mwk {
namespace {

constexpr int kTileM = 128;
constexpr int kTileKd = 64;                  // subdomain dofs (complex K) per tile
constexpr int kATileBytes = kTileM * 128;    // 16 KB
constexpr int kThreadsTc = 192;
// tcgen05 shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);        // start address
  d |= (uint64_t)1 << 16;                        // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;              // stride byte offset
  d |= (uint64_t)1 << 46;                        // descriptor version
  d |= (uint64_t)2 << 61;                        // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, M = 128, N.
__host__ __device__ constexpr uint32_t idesc_bf16(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of (row, k) in a K-major, 128-byte-swizzled tile with 64 BF16 per row.
__host__ __device__ __forceinline__ uint32_t swz(uint32_t row, uint32_t k) {
  return row * 128u + ((((k >> 3) ^ (row & 7u)) & 7u) << 4) + ((k & 7u) << 1);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat16 a = __float2bfloat16_rn(lo), b = __float2bfloat16_rn(hi);
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// ---------------------------------------------------------------------------------------
// Setup: owned rows of B_s^{-1} (FP32 or FP64 workspace) -> swizzled BF16 tile pairs (Wr, Wi).
// One block per (subdomain of the batch, m tile, k tile); one 32-bit word per two dofs and plane.
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void pack_w_kernel(const int64_t* __restrict__ nmat, const int64_t* __restrict__ off,
                              const T* __restrict__ ws, const int32_t* __restrict__ sub_ids,
                              const int64_t* __restrict__ own_ptr, const int32_t* __restrict__ own_local,
                              const int64_t* __restrict__ sub_wtile, const int32_t* __restrict__ sub_kt,
                              uint8_t* __restrict__ W) {
  const int b = blockIdx.z;
  const int s = sub_ids[b];
  const int64_t n = nmat[b];
  const int64_t nown = own_ptr[s + 1] - own_ptr[s];
  const int mt = blockIdx.y, kt = blockIdx.x;
  const int KT = sub_kt[s];
  if (kt >= KT || (int64_t)mt * kTileM >= nown) return;
  const T* A = ws + off[b];
  uint8_t* tr = W + ((size_t)sub_wtile[s] + ((size_t)mt * KT + kt) * 2) * kATileBytes;
  uint8_t* ti = tr + kATileBytes;
  constexpr int kPairs = kTileKd / 2;
  for (int w = threadIdx.x; w < kTileM * kPairs; w += blockDim.x) {
    const int r = w / kPairs, kp = w % kPairs;
    const int64_t q = (int64_t)mt * kTileM + r, k = (int64_t)kt * kTileKd + 2 * kp;
    float re0 = 0.f, im0 = 0.f, re1 = 0.f, im1 = 0.f;
    if (q < nown) {
      const T* row = A + (int64_t)own_local[own_ptr[s] + q] * n;
      if (k < n) {
        re0 = (float)row[k].x;
        im0 = (float)row[k].y;
      }
      if (k + 1 < n) {
        re1 = (float)row[k + 1].x;
        im1 = (float)row[k + 1].y;
      }
    }
    *reinterpret_cast<uint32_t*>(tr + swz(r, 2 * kp)) = pack_bf16(re0, re1);
    *reinterpret_cast<uint32_t*>(ti + swz(r, 2 * kp)) = pack_bf16(im0, im1);
  }
}

// The same tiles from strided FP32 blocks: "subdomain" q of the plan stacks up to two products
// with the same B, rows [0, m1) the product sign_1 A_1 of task first[q] and rows [m1, m1 + m2)
// the product sign_2 A_2 of task second[q] (second[q] < 0: none); A_i [m_i][k] has row stride
// lda_i at element a_off_i of src, both tasks have the same k, and the signs (+1 or -1) are
// exact in BF16.  One block per (q, m tile, k tile).
__global__ void pack_w_stacked_kernel(const MfTask* __restrict__ tasks, const int32_t* __restrict__ first,
                                      const int32_t* __restrict__ second, int q0,
                                      const int64_t* __restrict__ sub_wtile, const int32_t* __restrict__ sub_kt,
                                      const float2* __restrict__ src, uint8_t* __restrict__ W) {
  const int q = q0 + (int)blockIdx.z;
  const MfTask t1 = tasks[first[q]];
  const int j2 = second[q];
  const int64_t m2 = j2 >= 0 ? tasks[j2].m : 0;
  const int mt = blockIdx.y, kt = blockIdx.x;
  const int KT = sub_kt[q];
  if (kt >= KT || (int64_t)mt * kTileM >= t1.m + m2) return;
  uint8_t* tr = W + ((size_t)sub_wtile[q] + ((size_t)mt * KT + kt) * 2) * kATileBytes;
  uint8_t* ti = tr + kATileBytes;
  constexpr int kPairs = kTileKd / 2;
  for (int w = threadIdx.x; w < kTileM * kPairs; w += blockDim.x) {
    const int r = w / kPairs, kp = w % kPairs;
    const int64_t row = (int64_t)mt * kTileM + r, k = (int64_t)kt * kTileKd + 2 * kp;
    float re0 = 0.f, im0 = 0.f, re1 = 0.f, im1 = 0.f;
    if (row < t1.m + m2) {
      const MfTask t = row < t1.m ? t1 : tasks[j2];
      const float2* a = src + t.a_off + (row < t1.m ? row : row - t1.m) * t.lda;
      if (k < t.k) {
        re0 = t.sign * a[k].x;
        im0 = t.sign * a[k].y;
      }
      if (k + 1 < t.k) {
        re1 = t.sign * a[k + 1].x;
        im1 = t.sign * a[k + 1].y;
      }
    }
    *reinterpret_cast<uint32_t*>(tr + swz(r, 2 * kp)) = pack_bf16(re0, re1);
    *reinterpret_cast<uint32_t*>(ti + swz(r, 2 * kp)) = pack_bf16(im0, im1);
  }
}

// ---------------------------------------------------------------------------------------
// Apply, step 1: gathered operand tiles B' for every (subdomain, k tile).
// ---------------------------------------------------------------------------------------
// cscale (may be null): per-column factor of the input (a Krylov vector kept unscaled), applied
// in FP32 before the BF16 rounding.
__global__ void __launch_bounds__(128, 8) gather_b_kernel(const int32_t* __restrict__ gt_sub,
                                                       const int32_t* __restrict__ gt_kt,
                                                       const int64_t* __restrict__ dof_ptr,
                                                       const int32_t* __restrict__ dofs,
                                                       const float2* __restrict__ r, int R, int Rp,
                                                       uint8_t* __restrict__ Bt, const double* __restrict__ cscale,
                                                       int64_t ntiles) {
  // Blocks of 4 warps walk the tiles with a grid stride.  Per tile (64 dofs), warp w takes dofs
  // 16w .. 16w+15 and lane c the columns c, c + 32, ...: the dof indices come in one coalesced
  // load and are handed out by shuffles, the 16 values of a lane are independent loads, and each
  // lane writes its rows c (gr) and R_pad + c (gi) as two 16-byte swizzled chunks each.  The
  // tile is then copied out with coalesced 16-byte stores.
  extern __shared__ __align__(16) uint8_t tsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int N = 2 * Rp;
  const int nq = (Rp + 31) / 32;
  const int nvec16 = N * 128 / 16;
  for (int64_t g = blockIdx.x; g < ntiles; g += gridDim.x) {
    const int s = gt_sub[g], kt = gt_kt[g];
    const int64_t d0 = dof_ptr[s];
    const int64_t n = dof_ptr[s + 1] - d0;
    const int64_t k0 = (int64_t)kt * kTileKd + 16 * warp;
    const int idx = (lane < 16 && k0 + lane < n) ? dofs[d0 + k0 + lane] : -1;
    for (int q = 0; q < nq; ++q) {
      const int c = lane + 32 * q;
      float2 v[16];
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        const int e = __shfl_sync(0xffffffffu, idx, jj);
        v[jj] = (e >= 0 && c < R) ? r[(int64_t)e * R + c] : make_float2(0.f, 0.f);
      }
      if (c < R && cscale) {
        const float sc = (float)cscale[c];
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          v[jj].x *= sc;
          v[jj].y *= sc;
        }
      }
      if (c < Rp) {
        uint4 re0, re1, im0, im1;
        re0.x = pack_bf16(v[0].x, v[1].x);    re0.y = pack_bf16(v[2].x, v[3].x);
        re0.z = pack_bf16(v[4].x, v[5].x);    re0.w = pack_bf16(v[6].x, v[7].x);
        re1.x = pack_bf16(v[8].x, v[9].x);    re1.y = pack_bf16(v[10].x, v[11].x);
        re1.z = pack_bf16(v[12].x, v[13].x);  re1.w = pack_bf16(v[14].x, v[15].x);
        im0.x = pack_bf16(v[0].y, v[1].y);    im0.y = pack_bf16(v[2].y, v[3].y);
        im0.z = pack_bf16(v[4].y, v[5].y);    im0.w = pack_bf16(v[6].y, v[7].y);
        im1.x = pack_bf16(v[8].y, v[9].y);    im1.y = pack_bf16(v[10].y, v[11].y);
        im1.z = pack_bf16(v[12].y, v[13].y);  im1.w = pack_bf16(v[14].y, v[15].y);
        *reinterpret_cast<uint4*>(tsm + swz(c, 16 * warp)) = re0;
        *reinterpret_cast<uint4*>(tsm + swz(c, 16 * warp + 8)) = re1;
        *reinterpret_cast<uint4*>(tsm + swz(Rp + c, 16 * warp)) = im0;
        *reinterpret_cast<uint4*>(tsm + swz(Rp + c, 16 * warp + 8)) = im1;
      }
    }
    __syncthreads();
    uint4* tile = reinterpret_cast<uint4*>(Bt + (size_t)g * N * 128);
    for (int i = threadIdx.x; i < nvec16; i += blockDim.x) tile[i] = reinterpret_cast<const uint4*>(tsm)[i];
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Apply, step 2: one CTA per 128-row output tile of one subdomain.
// ---------------------------------------------------------------------------------------
struct TcArgs {
  const int32_t* mt_sub;
  const int32_t* mt_row0;
  const int64_t* sub_wtile;
  const int64_t* sub_gtile;
  const int32_t* sub_kt;
  const int64_t* own_ptr;
  const int32_t* own_glob;
  const int32_t* c0_glob;   // optional: row of z added to each output row (-1: none)
  int z_bf16;               // z holds complex BF16 pairs (4 bytes per value) instead of float2
  const uint8_t* W;
  const uint8_t* Bt;
  float2* z;
  int R, N, stages;
  uint32_t tmem_cols;
  int32_t* err;
};

__global__ void __launch_bounds__(kThreadsTc, 2) oras_tc_kernel(const TcArgs a) {
  extern __shared__ uint8_t dsm[];
  __shared__ __align__(8) uint64_t full_bar[8];
  __shared__ __align__(8) uint64_t empty_bar[8];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x;
  const int s = a.mt_sub[t];
  const int row0 = a.mt_row0[t];
  const int KT = a.sub_kt[s];
  const int S = a.stages;
  const uint32_t b_bytes = (uint32_t)a.N * 128u;
  const uint32_t a_bytes = 2u * kATileBytes;          // Wr and Wi tiles of one k tile
  const uint32_t stage_bytes = a_bytes + b_bytes;
  const uint8_t* Wt = a.W + ((size_t)a.sub_wtile[s] + (size_t)(row0 / kTileM) * KT * 2) * kATileBytes;
  const uint8_t* Bs = a.Bt + (size_t)a.sub_gtile[s] * b_bytes;

  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&full_bar[i], 1);
      mbar_init(&empty_bar[i], 1);
    }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      // producer: bulk copies of (Wr and Wi tiles, B tile) per k tile.  In the last m tile of a
      // subdomain only the 8-row swizzle groups that hold owned rows are copied: the other rows
      // of A feed only accumulator rows that the epilogue does not store.
      const int64_t nown_p = a.own_ptr[s + 1] - a.own_ptr[s];
      const int rows_valid = (int)min((int64_t)kTileM, nown_p - (int64_t)row0);
      const uint32_t a_part = (uint32_t)((rows_valid + 7) / 8) * 1024u;
      int issued = 0;
      for (int kt = 0; kt < KT; ++kt) {
        const int st = kt % S;
        if (kt >= S) {
          if (!mbar_wait(&empty_bar[st], ((kt / S) + 1) & 1)) {
            atomicCAS(a.err, 0, 1);
            abort_flag = 1;
            break;
          }
        }
        if (*(volatile int*)&abort_flag) break;
        uint8_t* sa = base + (size_t)st * stage_bytes;
        uint8_t* sb = sa + a_bytes;
        mbar_expect_tx(&full_bar[st], 2u * a_part + b_bytes);
        bulk_g2s(sa, Wt + (size_t)kt * a_bytes, a_part, &full_bar[st]);
        bulk_g2s(sa + kATileBytes, Wt + (size_t)kt * a_bytes + kATileBytes, a_part, &full_bar[st]);
        bulk_g2s(sb, Bs + (size_t)kt * b_bytes, b_bytes, &full_bar[st]);
        ++issued;
      }
      // drain: every issued copy has completed before this thread leaves
      for (int kt = (issued > S ? issued - S : 0); kt < issued; ++kt) {
        if (!mbar_wait(&full_bar[kt % S], (kt / S) & 1)) atomicCAS(a.err, 0, 2);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(a.N);
      for (int kt = 0; kt < KT; ++kt) {
        const int st = kt % S;
        if (!mbar_wait(&full_bar[st], (kt / S) & 1)) {
          atomicCAS(a.err, 0, 3);
          abort_flag = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sar = smem_u32(base + (size_t)st * stage_bytes);
        const uint32_t sai = sar + kATileBytes;
        const uint32_t sb = sar + a_bytes;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t acc = (kt > 0 || k > 0) ? 1u : 0u;
          mma_bf16(tmem, smem_desc(sar + 32u * k), smem_desc(sb + 32u * k), idesc, acc);               // D1 = Wr B
          mma_bf16(tmem + (uint32_t)a.N, smem_desc(sai + 32u * k), smem_desc(sb + 32u * k), idesc, acc);  // D2 = Wi B
        }
        mma_commit(&empty_bar[st]);
      }
      mma_commit(&done_bar);
    }
  } else {
    // epilogue: warps 2..5 cover tensor-memory lane quadrants (warp % 4).  The output row, the C0
    // row and C0's first 8 columns are looked up while the MMAs run.
    const int quad = warp & 3;
    const int row = quad * 32 + lane;
    const int64_t nown = a.own_ptr[s + 1] - a.own_ptr[s];
    const int64_t q = (int64_t)row0 + row;
    const int64_t og = q < nown ? (int64_t)a.own_glob[a.own_ptr[s] + q] : -1;   // negative: skipped
    const int64_t c0 = (og >= 0 && a.c0_glob) ? (int64_t)a.c0_glob[a.own_ptr[s] + q] : -1;
    const float2* c0r = c0 >= 0 ? a.z + c0 * a.R : nullptr;
    float2 nxt[8];
    auto fetch_c0 = [&](int cb) {
#pragma unroll
      for (int i = 0; i < 8; ++i) nxt[i] = (c0r && cb + i < a.R) ? c0r[cb + i] : make_float2(0.f, 0.f);
    };
    fetch_c0(0);
    bool ok = mbar_wait(&done_bar, 0);
    ok = __all_sync(0xffffffffu, ok);   // tcgen05.ld below is warp-collective
    if (!ok && lane == 0) atomicCAS(a.err, 0, 4);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool valid = ok && !abort_flag && og >= 0;
    float2* zr = valid ? a.z + og * a.R : nullptr;
    const int Rp = a.N / 2;
    const uint32_t lanes = tmem + ((uint32_t)(quad * 32) << 16);
    for (int cb = 0; cb < Rp; cb += 8) {
      // Re z = D1[c] - D2[Rp + c], Im z = D1[Rp + c] + D2[c] (plus the C0 row when given)
      float2 cur[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) cur[i] = nxt[i];
      if (cb + 8 < Rp) fetch_c0(cb + 8);
      float rr[8], ri[8], ir[8], ii[8];
      if (ok) {
        tmem_ld8(lanes + (uint32_t)cb, rr);                          // Wr gr
        tmem_ld8(lanes + (uint32_t)(Rp + cb), ri);                   // Wr gi
        tmem_ld8(lanes + (uint32_t)(a.N + cb), ir);                  // Wi gr
        tmem_ld8(lanes + (uint32_t)(a.N + Rp + cb), ii);             // Wi gi
      }
      if (valid) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int col = cb + i;
          if (col >= a.R) continue;
          float2 v = make_float2(rr[i] - ii[i], ri[i] + ir[i]);
          if (c0r) v = make_float2(v.x + cur[i].x, v.y + cur[i].y);
          if (a.z_bf16)
            reinterpret_cast<uint32_t*>(a.z)[og * a.R + col] = pack_bf16(v.x, v.y);
          else
            zr[col] = v;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
  }
}

// Persistent form of oras_tc_kernel for plans of many short tiles (the sparse sweeps): the CTAs
// take the 128-row output tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...; one copy ring runs
// across the CTA's tiles, and the accumulators are double-buffered in tensor memory (buffer
// i % 2 for the CTA's i-th tile), so the epilogue of one tile overlaps the copies and MMAs of
// the next.  Per tile: the same copies, MMAs in the same order and the same epilogue arithmetic
// as oras_tc_kernel, so z is bit-identical.  Waits are bounded: a wait that runs out records an
// error code and sets the abort flag, every role then stops, the producer drains its copies and
// the MMA warp waits (bounded) for its last MMAs before the accumulators are freed.
__global__ void __launch_bounds__(kThreadsTc, 2) oras_tc_persistent_kernel(const TcArgs a, int n_tiles) {
  extern __shared__ uint8_t dsm[];
  __shared__ __align__(8) uint64_t full_bar[8];
  __shared__ __align__(8) uint64_t empty_bar[8];
  __shared__ __align__(8) uint64_t acc_full[2];
  __shared__ __align__(8) uint64_t acc_empty[2];
  __shared__ __align__(8) uint64_t fin_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int S = a.stages;
  const uint32_t b_bytes = (uint32_t)a.N * 128u;
  const uint32_t a_bytes = 2u * kATileBytes;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  volatile int* abort_v = &abort_flag;

  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&full_bar[i], 1);
      mbar_init(&empty_bar[i], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);   // one arrival per epilogue warp
    }
    mbar_init(&fin_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(2u * a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      int64_t it = 0;   // k tiles issued by this CTA (running ring position)
      for (int t = blockIdx.x; t < n_tiles && !*abort_v; t += gridDim.x) {
        const int s = a.mt_sub[t];
        const int row0 = a.mt_row0[t];
        const int KT = a.sub_kt[s];
        const uint8_t* Wt = a.W + ((size_t)a.sub_wtile[s] + (size_t)(row0 / kTileM) * KT * 2) * kATileBytes;
        const uint8_t* Bs = a.Bt + (size_t)a.sub_gtile[s] * b_bytes;
        const int64_t nown_p = a.own_ptr[s + 1] - a.own_ptr[s];
        const int rows_valid = (int)min((int64_t)kTileM, nown_p - (int64_t)row0);
        const uint32_t a_part = (uint32_t)((rows_valid + 7) / 8) * 1024u;
        for (int kt = 0; kt < KT; ++kt, ++it) {
          const int st = (int)(it % S);
          if (it >= S && !mbar_wait(&empty_bar[st], (uint32_t)(((it / S) + 1) & 1))) {
            atomicCAS(a.err, 0, 11);
            *abort_v = 1;
          }
          if (*abort_v) break;
          uint8_t* sa = base + (size_t)st * stage_bytes;
          uint8_t* sb = sa + a_bytes;
          mbar_expect_tx(&full_bar[st], 2u * a_part + b_bytes);
          bulk_g2s(sa, Wt + (size_t)kt * a_bytes, a_part, &full_bar[st]);
          bulk_g2s(sa + kATileBytes, Wt + (size_t)kt * a_bytes + kATileBytes, a_part, &full_bar[st]);
          bulk_g2s(sb, Bs + (size_t)kt * b_bytes, b_bytes, &full_bar[st]);
        }
      }
      // drain: every issued copy has completed before this thread leaves
      for (int64_t k = (it > S ? it - S : 0); k < it; ++k)
        if (!mbar_wait(&full_bar[k % S], (uint32_t)((k / S) & 1))) atomicCAS(a.err, 0, 12);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(a.N);
      int64_t it = 0;
      int i = 0;   // tiles of this CTA
      for (int t = blockIdx.x; t < n_tiles && !*abort_v; t += gridDim.x, ++i) {
        const int KT = a.sub_kt[a.mt_sub[t]];
        const int buf = i & 1;
        if (i >= 2 && !mbar_wait(&acc_empty[buf], (uint32_t)(((i >> 1) + 1) & 1))) {
          atomicCAS(a.err, 0, 13);
          *abort_v = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc0 = tmem + (uint32_t)buf * a.tmem_cols;
        bool stop = false;
        for (int kt = 0; kt < KT; ++kt, ++it) {
          const int st = (int)(it % S);
          if (!mbar_wait(&full_bar[st], (uint32_t)((it / S) & 1))) {
            atomicCAS(a.err, 0, 14);
            *abort_v = 1;
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sar = smem_u32(base + (size_t)st * stage_bytes);
          const uint32_t sai = sar + kATileBytes;
          const uint32_t sb = sar + a_bytes;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint32_t acc = (kt > 0 || k > 0) ? 1u : 0u;
            mma_bf16(acc0, smem_desc(sar + 32u * k), smem_desc(sb + 32u * k), idesc, acc);
            mma_bf16(acc0 + (uint32_t)a.N, smem_desc(sai + 32u * k), smem_desc(sb + 32u * k), idesc, acc);
          }
          mma_commit(&empty_bar[st]);
        }
        if (stop) break;
        mma_commit(&acc_full[buf]);
      }
      // every MMA issued by this CTA has completed before the accumulators are freed
      mma_commit(&fin_bar);
      if (!mbar_wait(&fin_bar, 0)) atomicCAS(a.err, 0, 15);
    }
  } else {
    const int quad = warp & 3;
    const int row = quad * 32 + lane;
    const int Rp = a.N / 2;
    int i = 0;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++i) {
      const int s = a.mt_sub[t];
      const int row0 = a.mt_row0[t];
      const int buf = i & 1;
      const int64_t nown = a.own_ptr[s + 1] - a.own_ptr[s];
      const int64_t q = (int64_t)row0 + row;
      const int64_t og = q < nown ? (int64_t)a.own_glob[a.own_ptr[s] + q] : -1;
      const int64_t c0 = (og >= 0 && a.c0_glob) ? (int64_t)a.c0_glob[a.own_ptr[s] + q] : -1;
      const float2* c0r = c0 >= 0 ? a.z + c0 * a.R : nullptr;
      float2 nxt[8];
      auto fetch_c0 = [&](int cb) {
#pragma unroll
        for (int j = 0; j < 8; ++j) nxt[j] = (c0r && cb + j < a.R) ? c0r[cb + j] : make_float2(0.f, 0.f);
      };
      fetch_c0(0);
      bool ok = !*abort_v && mbar_wait(&acc_full[buf], (uint32_t)((i >> 1) & 1));
      ok = __all_sync(0xffffffffu, ok);   // tcgen05.ld below is warp-collective
      if (!ok) {
        if (lane == 0) {
          atomicCAS(a.err, 0, 16);
          *abort_v = 1;
        }
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const bool valid = og >= 0;
      float2* zr = valid ? a.z + og * a.R : nullptr;
      const uint32_t lanes = tmem + (uint32_t)buf * a.tmem_cols + ((uint32_t)(quad * 32) << 16);
      for (int cb = 0; cb < Rp; cb += 8) {
        float2 cur[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) cur[j] = nxt[j];
        if (cb + 8 < Rp) fetch_c0(cb + 8);
        float rr[8], ri[8], ir[8], ii[8];
        tmem_ld8(lanes + (uint32_t)cb, rr);
        tmem_ld8(lanes + (uint32_t)(Rp + cb), ri);
        tmem_ld8(lanes + (uint32_t)(a.N + cb), ir);
        tmem_ld8(lanes + (uint32_t)(a.N + Rp + cb), ii);
        if (valid) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int col = cb + j;
            if (col >= a.R) continue;
            float2 v = make_float2(rr[j] - ii[j], ri[j] + ir[j]);
            if (c0r) v = make_float2(v.x + cur[j].x, v.y + cur[j].y);
            if (a.z_bf16)
              reinterpret_cast<uint32_t*>(a.z)[og * a.R + col] = pack_bf16(v.x, v.y);
            else
              zr[col] = v;
          }
        }
      }
      // this warp's reads of the buffer are done: the MMA warp may overwrite it
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2u * a.tmem_cols)
                 : "memory");
  }
}

// Self-test of the bounded wait: waits on an mbarrier that expects two arrivals but receives
// one, so the phase never completes; the wait gives up after `limit` polls and the kernel
// reports MW_ETIMEOUT (5) in *code instead of hanging.
__global__ void bounded_wait_probe_kernel(long long limit, int32_t* code) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 2);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
    *code = mbar_wait(&bar, 0, limit) ? 0 : 5;
  }
}

inline int rpad(int R) { return (R + 7) / 8 * 8; }

}  // namespace

bool tc_plan_build(TcPlan& p, const mw::Subdomains& sd, const std::function<void*(size_t)>& alloc, cudaStream_t s) {
  p = TcPlan();
  const int ns = sd.n_sub;
  std::vector<int32_t> mt_sub, mt_row0, sub_kt(ns), gt_sub, gt_kt;
  std::vector<int64_t> sub_wtile(ns), sub_gtile(ns);
  int64_t wt = 0, gtile = 0;
  for (int q = 0; q < ns; ++q) {
    const int64_t n = sd.dof_ptr[q + 1] - sd.dof_ptr[q];
    const int64_t no = sd.own_ptr[q + 1] - sd.own_ptr[q];
    const int KT = (int)((n + kTileKd - 1) / kTileKd);
    const int MT = (int)((no + kTileM - 1) / kTileM);
    sub_kt[q] = KT;
    sub_wtile[q] = wt;
    sub_gtile[q] = gtile;
    for (int m = 0; m < MT; ++m) {
      mt_sub.push_back(q);
      mt_row0.push_back(m * kTileM);
    }
    for (int k = 0; k < KT; ++k) {
      gt_sub.push_back(q);
      gt_kt.push_back(k);
    }
    wt += (int64_t)MT * KT * 2;   // Wr and Wi tile per (m tile, k tile)
    gtile += KT;
  }
  p.n_sub = ns;
  p.n_mtiles = (int64_t)mt_sub.size();
  p.n_ktiles_total = gtile;
  p.w_tiles = wt;
  auto up = [&](const void* h, size_t bytes) {
    void* d = alloc(bytes);
    cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, s);
    return d;
  };
  p.mt_sub = (int32_t*)up(mt_sub.data(), sizeof(int32_t) * std::max<size_t>(mt_sub.size(), 1));
  p.mt_row0 = (int32_t*)up(mt_row0.data(), sizeof(int32_t) * std::max<size_t>(mt_row0.size(), 1));
  p.sub_wtile = (int64_t*)up(sub_wtile.data(), sizeof(int64_t) * ns);
  p.sub_gtile = (int64_t*)up(sub_gtile.data(), sizeof(int64_t) * ns);
  p.sub_kt = (int32_t*)up(sub_kt.data(), sizeof(int32_t) * ns);
  p.gt_sub = (int32_t*)up(gt_sub.data(), sizeof(int32_t) * std::max<size_t>(gt_sub.size(), 1));
  p.gt_kt = (int32_t*)up(gt_kt.data(), sizeof(int32_t) * std::max<size_t>(gt_kt.size(), 1));
  p.err = (int32_t*)alloc(sizeof(int32_t));
  cudaMemsetAsync(p.err, 0, sizeof(int32_t), s);
  cudaStreamSynchronize(s);  // host vectors go out of scope
  p.max_kt = 0;
  for (int q = 0; q < ns; ++q) p.max_kt = std::max(p.max_kt, sub_kt[q]);
  p.built = true;
  return true;
}

void tc_plan_free(TcPlan& p, const std::function<void(void*)>& dfree) {
  for (void* q : {(void*)p.mt_sub, (void*)p.mt_row0, (void*)p.sub_wtile, (void*)p.sub_gtile, (void*)p.sub_kt,
                  (void*)p.gt_sub, (void*)p.gt_kt, (void*)p.err})
    if (q) dfree(q);
  p = TcPlan();
}

void bounded_wait_probe(long long limit, int32_t* code, cudaStream_t s) {
  note_launch(1);
  bounded_wait_probe_kernel<<<1, 32, 0, s>>>(limit, code);
}

size_t tc_w_bytes(const TcPlan& p) { return (size_t)std::max<int64_t>(p.w_tiles, 1) * kATileBytes; }

size_t tc_scratch_bytes(const TcPlan& p, int R) {
  return (size_t)std::max<int64_t>(p.n_ktiles_total, 1) * 2 * rpad(R) * 128;
}

void tc_extract(const TcPlan& p, const OrasBatch& bt, const OrasTopo& tp, int ws_prec, const void* ws, void* W,
                cudaStream_t s) {
  note_launch(1);
  // grid: k tiles x m tiles of the largest subdomain in the batch x batch
  const int ktmax = (int)((bt.nmax + kTileKd - 1) / kTileKd);
  const int mtmax = (int)((bt.nmax + kTileM - 1) / kTileM);
  dim3 grid(ktmax, mtmax, bt.count);
  if (ws_prec == 0)
    pack_w_kernel<double2><<<grid, 256, 0, s>>>(bt.d_n, bt.d_off, (const double2*)ws, bt.d_sub, tp.own_ptr,
                                                 tp.own_local, p.sub_wtile, p.sub_kt, (uint8_t*)W);
  else
    pack_w_kernel<float2><<<grid, 256, 0, s>>>(bt.d_n, bt.d_off, (const float2*)ws, bt.d_sub, tp.own_ptr,
                                                tp.own_local, p.sub_wtile, p.sub_kt, (uint8_t*)W);
}

void tc_pack_stacked(const TcPlan& p, const MfTask* tasks, const int32_t* first, const int32_t* second, int n,
                     int ktmax, int mtmax, const float2* src, void* W, cudaStream_t s) {
  for (int q0 = 0; q0 < n; q0 += 65535) {
    const int cnt = std::min(65535, n - q0);
    note_launch(1);
    dim3 grid((unsigned)std::max(ktmax, 1), (unsigned)std::max(mtmax, 1), (unsigned)cnt);
    pack_w_stacked_kernel<<<grid, 256, 0, s>>>(tasks, first, second, q0, p.sub_wtile, p.sub_kt, src, (uint8_t*)W);
  }
}

int tc_stages(int N);
size_t tc_smem_bytes(int N, int stages);

int tc_stages(int N) {
  // about 100 KB of stages per CTA so that two CTAs share an SM
  const int stage = 2 * kATileBytes + N * 128;
  int st = (100 * 1024) / stage;
  return st > 6 ? 6 : (st < 2 ? 2 : st);
}

size_t tc_smem_bytes(int N, int stages) { return (size_t)stages * (2 * kATileBytes + N * 128) + 1024; }


int tc_max_stages(int R) {
  // the kernel holds 8 stage barriers; 1 KB of the 227 KB is left for its static shared memory
  const int N = 2 * rpad(R);
  int st = tc_min_stages;
  while (st < 8 && tc_smem_bytes(N, st + 1) <= (size_t)226 * 1024) ++st;
  return st;
}

void oras_apply_tc(const TcPlan& p, const OrasTopo& tp, const void* W, const float2* r, float2* z, int R,
                   void* scratch, cudaStream_t s, int stages, const double* in_scale, const int32_t* c0_glob,
                   bool z_bf16, bool persistent) {
  const int Rp = rpad(R);
  const int N = 2 * Rp;
  if (stages <= 0) stages = tc_stages(N);
  if (stages < tc_min_stages) stages = tc_min_stages;
  if (stages > tc_max_stages(R)) stages = tc_max_stages(R);
  note_launch(2);
  const size_t gsm = (size_t)N * 128;
  static size_t gattr = 0;
  if (gsm > 48 * 1024 && gsm > gattr) {
    cudaFuncSetAttribute(gather_b_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
    gattr = gsm;
  }
  const int64_t gblocks = std::min<int64_t>(p.n_ktiles_total, 152 * 8);    // one resident wave
  gather_b_kernel<<<(unsigned)std::max<int64_t>(gblocks, 1), 128, gsm, s>>>(
      p.gt_sub, p.gt_kt, tp.dof_ptr, tp.dofs, r, R, Rp, (uint8_t*)scratch, in_scale, p.n_ktiles_total);
  TcArgs a;
  a.mt_sub = p.mt_sub;
  a.mt_row0 = p.mt_row0;
  a.sub_wtile = p.sub_wtile;
  a.sub_gtile = p.sub_gtile;
  a.sub_kt = p.sub_kt;
  a.own_ptr = tp.own_ptr;
  a.own_glob = tp.own_glob;
  a.c0_glob = c0_glob;
  a.z_bf16 = z_bf16 ? 1 : 0;
  a.W = (const uint8_t*)W;
  a.Bt = (const uint8_t*)scratch;
  a.z = z;
  a.R = R;
  a.N = N;
  a.stages = stages;
  uint32_t cols = 32;
  while ((int)cols < 2 * N) cols <<= 1;   // two accumulators of N columns
  a.tmem_cols = cols;
  a.err = p.err;
  if (persistent && 2 * cols <= 512) {
    // two accumulator buffers per CTA; two CTAs per SM while both fit the 512 columns
    const int per_sm = 4 * cols <= 512 ? 2 : 1;
    size_t smem = tc_smem_bytes(N, stages);
    if (per_sm == 1 && smem < (size_t)120 * 1024) smem = (size_t)120 * 1024;
    static size_t pattr = 0;
    if (smem > pattr) {
      cudaFuncSetAttribute(oras_tc_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      pattr = smem;
    }
    const int grid = (int)std::min<int64_t>(p.n_mtiles, (int64_t)per_sm * 152);
    oras_tc_persistent_kernel<<<(unsigned)std::max(grid, 1), kThreadsTc, smem, s>>>(a, (int)p.n_mtiles);
    return;
  }
  // two CTAs of an SM must fit their tensor memory (512 columns per SM): above 256 columns the
  // shared-memory request keeps one CTA per SM
  size_t smem = tc_smem_bytes(N, stages);
  if (cols > 256 && smem < (size_t)120 * 1024) smem = (size_t)120 * 1024;
  static size_t attr = 0;
  if (smem > attr) {
    cudaFuncSetAttribute(oras_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = smem;
  }
  oras_tc_kernel<<<(unsigned)p.n_mtiles, kThreadsTc, smem, s>>>(a);
}


// ---------------------------------------------------------------------------------------
// Fixed scratch for the preconditioner apply that allocates nothing.
//
// Some callers cannot allocate device memory when they apply the preconditioner: code that
// runs while another framework owns the whole device heap, code that forbids allocation after
// initialisation (latency-critical or embedded loops), or callers on paths where an allocation
// would synchronise the device.  For them the gathered operand of the tensor-core apply lives
// in this file-scope array instead of a context buffer.  Every GPU that loads the library holds
// it until the process exits.  All calls share it and it keeps the last call's contents; the
// gather kernel rewrites every byte a call reads (zero padding included), so nothing needs
// clearing, but calls that overlap on the GPU race on it.
// ---------------------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

bool tc_noalloc_scratch(void** ptr, std::string& err) {
  // In host code the array's name is only a host-side handle; the device address is looked up
  // once per device, with that device current, and cached.
  static std::mutex mu;
  static void* addr[256] = {};
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 256) {
    err = std::string("cudaGetDevice failed: ") + cudaGetErrorString(e);
    return false;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      err = std::string("cudaGetSymbolAddress of the fixed scratch failed: ") + cudaGetErrorString(e);
      return false;
    }
    addr[dev] = p;
  }
  *ptr = addr[dev];
  return true;
}

}  // namespace mwk
