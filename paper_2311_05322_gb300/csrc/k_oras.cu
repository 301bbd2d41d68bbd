// K5 (ORAS setup) and the CUDA-core form of K4 (ORAS apply), Sec. IV-C.
//
// Setup, per subdomain s with n_s unknowns:
//   1. dense local matrix  B_s = sum_{T in s} (K^T - k0^2 eps_T M^T)
//                               + sum_{surface faces F of s} z_F B^F,
//      z_F = i k0 sqrt(eps_F) on an interface face, eps_F the eps of the inside tet (first-order
//      impedance transmission condition of Eq. m1 on the artificial boundary); on an outer face
//      z_F = i k0 sqrt(eps_bg), or with face classes (waveguide ports) the global boundary's
//      coefficient of that face (open, metal = 0, port = i beta_p); the rows and columns of
//      metal edges are then those of the identity, as in the global matrix;
//   2. in-place blocked Gauss-Jordan inversion without pivoting (the imaginary part of B_s is
//      symmetric positive definite for lossy media, so every leading block is nonsingular);
//   3. the owned rows of B_s^{-1} (restricted partition of unity, boolean D_s) are kept as
//      W_s [n_own][n_s] in the apply precision.
// Apply:  z[own_s] = W_s r[dofs_s]  for every s (owners partition the edges: no atomics).
#include "mw_internal.h"
#include "k_oras.h"

namespace mwk {
namespace {

template <typename T>
struct Tr;
template <>
struct Tr<double2> {
  using S = double;
};
template <>
struct Tr<float2> {
  using S = float;
};

__device__ __forceinline__ double2 csqrt_principal(double a, double b) {
  const double r = sqrt(a * a + b * b);
  const double re = sqrt(0.5 * (r + a));
  double im = sqrt(fmax(0.0, 0.5 * (r - a)));
  if (b < 0.0) im = -im;
  return make_double2(re, im);
}

// One warp per subdomain; tets then surface faces in list order, entries of one element by
// different lanes (never the same matrix entry), elements in sequence (ordered by __syncwarp).
// surf_tet codes: >= 0 inside tet of an interface face; -1 outer face with i k0 sqrt(eps_bg)
// when zc is null, else -1 - c for an outer face of class c with coefficient zc[c].
template <typename T>
__global__ void local_assemble_kernel(const int32_t* __restrict__ sub_ids, const int64_t* __restrict__ dof_ptr,
                                      const int32_t* __restrict__ dofs, const int64_t* __restrict__ tet_ptr,
                                      const int32_t* __restrict__ tet_ids, const int32_t* __restrict__ tet_loc,
                                      const int64_t* __restrict__ surf_ptr, const int32_t* __restrict__ surf_loc,
                                      const int32_t* __restrict__ surf_tet, const double* __restrict__ Bsurf,
                                      const double* __restrict__ KM, const double* __restrict__ eps, double k0,
                                      double eps_bg_re, double eps_bg_im, const double2* __restrict__ zc,
                                      const uint8_t* __restrict__ metal, const int64_t* __restrict__ ws_off,
                                      T* __restrict__ ws) {
  using Sc = typename Tr<T>::S;
  const int b = blockIdx.x;
  const int s = sub_ids[b];
  const int lane = threadIdx.x;
  const int64_t n = dof_ptr[s + 1] - dof_ptr[s];
  T* A = ws + ws_off[b];
  const double k0sq = k0 * k0;
  for (int64_t q = tet_ptr[s]; q < tet_ptr[s + 1]; ++q) {
    const int64_t t = tet_ids[q];
    const int32_t* loc = tet_loc + 6 * q;
    for (int e = lane; e < 36; e += 32) {
      const int m = e / 6, nn = e % 6;
      const int pk = mw::packed6(m, nn);
      const double Kv = KM[42 * t + pk], Mv = KM[42 * t + 21 + pk];
      const double re = Kv - (k0sq * eps[2 * t]) * Mv;
      const double im = -(k0sq * eps[2 * t + 1]) * Mv;
      T* p = A + (int64_t)loc[m] * n + loc[nn];
      T v = *p;
      v.x += (Sc)re;
      v.y += (Sc)im;
      *p = v;
    }
    __syncwarp();
  }
  const double2 sbg = csqrt_principal(eps_bg_re, eps_bg_im);
  for (int64_t q = surf_ptr[s]; q < surf_ptr[s + 1]; ++q) {
    if (lane < 9) {
      const int m = lane / 3, nn = lane % 3;
      const int32_t it = surf_tet[q];
      const double Bv = Bsurf[6 * q + mw::packed3(m, nn)];
      double re, im;
      if (it < 0 && zc) {
        const double2 z = zc[-1 - it];
        re = z.x * Bv;
        im = z.y * Bv;
      } else {
        const double2 sq = it >= 0 ? csqrt_principal(eps[2 * (int64_t)it], eps[2 * (int64_t)it + 1]) : sbg;
        // i k0 sqrt(eps) = (-k0 Im sqrt, k0 Re sqrt)
        re = (-k0 * sq.y) * Bv;
        im = (k0 * sq.x) * Bv;
      }
      T* p = A + (int64_t)surf_loc[3 * q + m] * n + surf_loc[3 * q + nn];
      T v = *p;
      v.x += (Sc)re;
      v.y += (Sc)im;
      *p = v;
    }
    __syncwarp();
  }
  if (metal) {
    const int32_t* gd = dofs + dof_ptr[s];
    for (int64_t i = 0; i < n; ++i) {
      if (!metal[gd[i]]) continue;
      for (int64_t j = lane; j < n; j += 32) {
        A[i * n + j] = T{0, 0};
        A[j * n + i] = T{0, 0};
      }
      __syncwarp();
      if (lane == 0) A[i * n + i] = T{1, 0};
      __syncwarp();
    }
  }
}

constexpr int NB = 32;

template <typename T>
__device__ __forceinline__ T cmul(T a, T b) {
  return T{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// Invert the NB x NB diagonal block at kb of every matrix in place (Gauss-Jordan, no pivoting)
// into Dinv[b].  Flags a pivot whose modulus is below tiny * (block max modulus).
template <typename T>
__global__ void gj_diag_kernel(const int64_t* __restrict__ nmat, const int64_t* __restrict__ off, T* __restrict__ ws,
                               int64_t kb, T* __restrict__ Dinv, int32_t* __restrict__ status,
                               const int64_t* __restrict__ lim) {
  using Sc = typename Tr<T>::S;
  __shared__ T D[NB][NB + 1];
  __shared__ Sc dmax;
  const int b = blockIdx.x;
  const int64_t n = nmat[b];
  const int64_t L = lim ? lim[b] : n;
  if (kb >= L) return;
  const int bs = (int)min((int64_t)NB, L - kb);
  const T* A = ws + off[b];
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int i = e / NB, j = e % NB;
    D[i][j] = (i < bs && j < bs) ? A[(kb + i) * n + kb + j] : T{(Sc)(i == j), 0};
  }
  if (threadIdx.x == 0) dmax = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    Sc mx = 0;
    for (int i = 0; i < bs; ++i) mx = fmax(mx, (Sc)sqrt((double)D[i][i].x * D[i][i].x + (double)D[i][i].y * D[i][i].y));
    dmax = mx;
  }
  __syncthreads();
  for (int k = 0; k < NB; ++k) {
    const T p = D[k][k];
    const Sc pm = p.x * p.x + p.y * p.y;
    const Sc tiny = (sizeof(Sc) == 4 ? (Sc)1e-12 : (Sc)1e-28) * dmax * dmax;
    T ip;
    if (!(pm > tiny)) {
      if (threadIdx.x == 0) atomicExch(status, 1);
      ip = T{0, 0};
    } else {
      ip = T{p.x / pm, -p.y / pm};
    }
    T vals[4];
    int cnt = 0;
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x, ++cnt) {
      const int i = e / NB, j = e % NB;
      T v;
      if (i == k && j == k) {
        v = ip;
      } else if (i == k) {
        v = cmul(D[k][j], ip);
      } else if (j == k) {
        const T t = cmul(D[i][k], ip);
        v = T{-t.x, -t.y};
      } else {
        const T t = cmul(cmul(D[i][k], ip), D[k][j]);
        v = T{D[i][j].x - t.x, D[i][j].y - t.y};
      }
      vals[cnt] = v;
    }
    __syncthreads();
    cnt = 0;
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x, ++cnt) D[e / NB][e % NB] = vals[cnt];
    __syncthreads();
  }
  T* Dv = Dinv + (int64_t)b * NB * NB;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) Dv[e] = D[e / NB][e % NB];
}

// A[K, j] <- Dinv A[K, j] for every column j outside K.
template <typename T>
__global__ void gj_rowpanel_kernel(const int64_t* __restrict__ nmat, const int64_t* __restrict__ off,
                                   T* __restrict__ ws, int64_t kb, const T* __restrict__ Dinv,
                                   const int64_t* __restrict__ lim) {
  using Sc = typename Tr<T>::S;
  __shared__ T D[NB][NB];
  const int b = blockIdx.y;
  const int64_t n = nmat[b];
  const int64_t L = lim ? lim[b] : n;
  if (kb >= L) return;
  const int bs = (int)min((int64_t)NB, L - kb);
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) D[e / NB][e % NB] = Dinv[(int64_t)b * NB * NB + e];
  __syncthreads();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n || (j >= kb && j < kb + bs)) return;
  T* A = ws + off[b];
  T col[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k) col[k] = k < bs ? A[(kb + k) * n + j] : T{0, 0};
  for (int i = 0; i < bs; ++i) {
    T acc{0, 0};
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      const T d = D[i][k];
      acc.x = fma(d.x, col[k].x, acc.x);
      acc.x = fma(-d.y, col[k].y, acc.x);
      acc.y = fma(d.x, col[k].y, acc.y);
      acc.y = fma(d.y, col[k].x, acc.y);
    }
    A[(kb + i) * n + j] = acc;
  }
}

// Rank-NB update A[I, J] -= A[I, K] A[K, J] for I, J outside K; 64 x 64 tiles, 4 x 4 per thread.
template <typename T>
__global__ void __launch_bounds__(256) gj_update_kernel(const int64_t* __restrict__ nmat,
                                                        const int64_t* __restrict__ off, T* __restrict__ ws,
                                                        int64_t kb, const int64_t* __restrict__ lim) {
  using Sc = typename Tr<T>::S;
  extern __shared__ unsigned char sm[];
  T* As = reinterpret_cast<T*>(sm);            // [64][NB]
  T* Bs = As + 64 * NB;                        // [NB][64]
  const int b = blockIdx.z;
  const int64_t n = nmat[b];
  const int64_t L = lim ? lim[b] : n;
  if (kb >= L) return;
  const int64_t i0 = (int64_t)blockIdx.y * 64, j0 = (int64_t)blockIdx.x * 64;
  if (i0 >= n || j0 >= n) return;
  const int bs = (int)min((int64_t)NB, L - kb);
  T* A = ws + off[b];
  for (int e = threadIdx.x; e < 64 * NB; e += 256) {
    const int r = e / NB, k = e % NB;
    const int64_t i = i0 + r;
    As[r * NB + k] = (i < n && k < bs) ? A[i * n + kb + k] : T{0, 0};
    const int kk = e / 64, c = e % 64;
    const int64_t j = j0 + c;
    Bs[kk * 64 + c] = (j < n && kk < bs) ? A[(kb + kk) * n + j] : T{0, 0};
  }
  __syncthreads();
  const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = T{0, 0};
#pragma unroll 4
  for (int k = 0; k < NB; ++k) {
    T av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = As[(tr + 16 * a) * NB + k];
#pragma unroll
    for (int c = 0; c < 4; ++c) bv[c] = Bs[k * 64 + tc + 16 * c];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        acc[a][c].x = fma(av[a].x, bv[c].x, acc[a][c].x);
        acc[a][c].x = fma(-av[a].y, bv[c].y, acc[a][c].x);
        acc[a][c].y = fma(av[a].x, bv[c].y, acc[a][c].y);
        acc[a][c].y = fma(av[a].y, bv[c].x, acc[a][c].y);
      }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t i = i0 + tr + 16 * a;
    if (i >= n || (i >= kb && i < kb + bs)) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t j = j0 + tc + 16 * c;
      if (j >= n || (j >= kb && j < kb + bs)) continue;
      T v = A[i * n + j];
      v.x -= acc[a][c].x;
      v.y -= acc[a][c].y;
      A[i * n + j] = v;
    }
  }
}

// A[i, K] <- -A[i, K] Dinv for rows outside K, A[K, K] <- Dinv.
template <typename T>
__global__ void gj_colpanel_kernel(const int64_t* __restrict__ nmat, const int64_t* __restrict__ off,
                                   T* __restrict__ ws, int64_t kb, const T* __restrict__ Dinv,
                                   const int64_t* __restrict__ lim) {
  __shared__ T D[NB][NB];
  const int b = blockIdx.y;
  const int64_t n = nmat[b];
  const int64_t L = lim ? lim[b] : n;
  if (kb >= L) return;
  const int bs = (int)min((int64_t)NB, L - kb);
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) D[e / NB][e % NB] = Dinv[(int64_t)b * NB * NB + e];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T* A = ws + off[b];
  if (i >= kb && i < kb + bs) {
    for (int j = 0; j < bs; ++j) A[i * n + kb + j] = D[i - kb][j];
    return;
  }
  T row[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k) row[k] = k < bs ? A[i * n + kb + k] : T{0, 0};
  for (int j = 0; j < bs; ++j) {
    T acc{0, 0};
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      const T d = D[k][j];
      acc.x = fma(row[k].x, d.x, acc.x);
      acc.x = fma(-row[k].y, d.y, acc.x);
      acc.y = fma(row[k].x, d.y, acc.y);
      acc.y = fma(row[k].y, d.x, acc.y);
    }
    A[i * n + kb + j] = T{-acc.x, -acc.y};
  }
}

// W_s[r][k] = Binv_s[own_local[r]][k], converted to the apply precision.
template <typename T, typename U>
__global__ void extract_owned_kernel(const int64_t* __restrict__ nmat, const int64_t* __restrict__ off,
                                     const T* __restrict__ ws, const int32_t* __restrict__ sub_ids,
                                     const int64_t* __restrict__ own_ptr, const int32_t* __restrict__ own_local,
                                     const int64_t* __restrict__ w_off, U* __restrict__ W) {
  using Su = decltype(U{}.x);
  const int b = blockIdx.y;
  const int s = sub_ids[b];
  const int64_t n = nmat[b];
  const int64_t nown = own_ptr[s + 1] - own_ptr[s];
  const T* A = ws + off[b];
  U* Ws = W + w_off[s];
  const int64_t total = nown * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / n, k = e - r * n;
    const T v = A[(int64_t)own_local[own_ptr[s] + r] * n + k];
    Ws[e] = U{(Su)v.x, (Su)v.y};
  }
}

// ---------------------------------------------------------------------------------------
// CUDA-core apply: a block computes a 32-row tile of z[own rows of s] for all R columns.
// ---------------------------------------------------------------------------------------
constexpr int TR = 32;   // rows per tile
constexpr int KC = 32;   // k chunk

template <typename T, int RMAX>
__global__ void __launch_bounds__(256) oras_apply_kernel(const int32_t* __restrict__ tile_sub,
                                                         const int32_t* __restrict__ tile_row0,
                                                         const int64_t* __restrict__ dof_ptr,
                                                         const int32_t* __restrict__ dofs,
                                                         const int64_t* __restrict__ own_ptr,
                                                         const int32_t* __restrict__ own_glob,
                                                         const int64_t* __restrict__ w_off, const T* __restrict__ W,
                                                         const T* __restrict__ r, T* __restrict__ z, int R) {
  __shared__ T Ws[TR][KC];
  __shared__ T Gs[KC][RMAX];
  const int s = tile_sub[blockIdx.x];
  const int row0 = tile_row0[blockIdx.x];
  const int64_t n = dof_ptr[s + 1] - dof_ptr[s];
  const int64_t nown = own_ptr[s + 1] - own_ptr[s];
  const int rows = (int)min((int64_t)TR, nown - row0);
  const T* Wt = W + w_off[s] + (int64_t)row0 * n;
  const int32_t* dv = dofs + dof_ptr[s];
  // thread -> (column c, row group)
  const int c = threadIdx.x % R;
  const int rg = threadIdx.x / R;
  const int ngroups = 256 / R;
  constexpr int MAXA = (TR * RMAX + 255) / 256;
  T acc[MAXA];
  const int my_rows = (rg < ngroups) ? (TR - rg + ngroups - 1) / ngroups : 0;
#pragma unroll
  for (int a = 0; a < MAXA; ++a) acc[a] = T{0, 0};
  for (int64_t k0 = 0; k0 < n; k0 += KC) {
    const int kc = (int)min((int64_t)KC, n - k0);
    for (int e = threadIdx.x; e < TR * KC; e += 256) {
      const int rr = e / KC, kk = e % KC;
      Ws[rr][kk] = (rr < rows && kk < kc) ? Wt[(int64_t)rr * n + k0 + kk] : T{0, 0};
    }
    for (int e = threadIdx.x; e < KC * R; e += 256) {
      const int kk = e / R, cc = e % R;
      Gs[kk][cc] = kk < kc ? r[(int64_t)dv[k0 + kk] * R + cc] : T{0, 0};
    }
    __syncthreads();
    if (rg < ngroups) {
#pragma unroll
      for (int a = 0; a < MAXA; ++a) {
        if (a >= my_rows) break;
        const int rr = rg + a * ngroups;
        T s2 = acc[a];
#pragma unroll 8
        for (int kk = 0; kk < KC; ++kk) {
          const T w = Ws[rr][kk], g = Gs[kk][c];
          s2.x = fma(w.x, g.x, s2.x);
          s2.x = fma(-w.y, g.y, s2.x);
          s2.y = fma(w.x, g.y, s2.y);
          s2.y = fma(w.y, g.x, s2.y);
        }
        acc[a] = s2;
      }
    }
    __syncthreads();
  }
  if (rg < ngroups)
#pragma unroll
    for (int a = 0; a < MAXA; ++a) {
      if (a >= my_rows) break;
      const int rr = rg + a * ngroups;
      if (rr < rows) z[(int64_t)own_glob[own_ptr[s] + row0 + rr] * R + c] = acc[a];
    }
}

// In-place blocked Gauss-Jordan over the first lim[b] pivots of every matrix (all of them when
// lim is null): the eliminated block becomes its inverse F11^-1, the rows right of it
// F11^-1 F12, the columns below it -F21 F11^-1 and the rest the Schur complement.
template <typename T>
void gj_all(const OrasBatch& bt, T* ws, T* dinv, int32_t* status, cudaStream_t st, const int64_t* lim = nullptr,
            int64_t lim_max = 0) {
  const int nb = bt.count;
  const int64_t nmax = bt.nmax;
  const size_t smem = sizeof(T) * 2 * 64 * NB;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(gj_update_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = true;
  }
  const int64_t kend = lim ? lim_max : nmax;
  for (int64_t kb = 0; kb < kend; kb += NB) {
    note_launch(4);
    gj_diag_kernel<T><<<nb, 256, 0, st>>>(bt.d_n, bt.d_off, ws, kb, dinv, status, lim);
    dim3 g1((unsigned)((nmax + 255) / 256), nb);
    gj_rowpanel_kernel<T><<<g1, 256, 0, st>>>(bt.d_n, bt.d_off, ws, kb, dinv, lim);
    dim3 g2((unsigned)((nmax + 63) / 64), (unsigned)((nmax + 63) / 64), nb);
    gj_update_kernel<T><<<g2, 256, smem, st>>>(bt.d_n, bt.d_off, ws, kb, lim);
    gj_colpanel_kernel<T><<<g1, 256, 0, st>>>(bt.d_n, bt.d_off, ws, kb, dinv, lim);
  }
}

}  // namespace

void oras_local_assemble(const OrasBatch& bt, const OrasTopo& tp, const double* Bsurf, const double* KM,
                         const double* eps, double k0, double ebr, double ebi, const double2* zc, const uint8_t* metal,
                         int prec, void* ws, cudaStream_t s) {
  note_launch(1);
  if (prec == 0)
    local_assemble_kernel<double2><<<bt.count, 32, 0, s>>>(bt.d_sub, tp.dof_ptr, tp.dofs, tp.tet_ptr, tp.tet_ids,
                                                            tp.tet_loc, tp.surf_ptr, tp.surf_loc, tp.surf_tet, Bsurf,
                                                            KM, eps, k0, ebr, ebi, zc, metal, bt.d_off, (double2*)ws);
  else
    local_assemble_kernel<float2><<<bt.count, 32, 0, s>>>(bt.d_sub, tp.dof_ptr, tp.dofs, tp.tet_ptr, tp.tet_ids,
                                                           tp.tet_loc, tp.surf_ptr, tp.surf_loc, tp.surf_tet, Bsurf,
                                                           KM, eps, k0, ebr, ebi, zc, metal, bt.d_off, (float2*)ws);
}

void oras_invert(const OrasBatch& bt, int prec, void* ws, void* dinv, int32_t* status, cudaStream_t s) {
  if (prec == 0)
    gj_all<double2>(bt, (double2*)ws, (double2*)dinv, status, s);
  else
    gj_all<float2>(bt, (float2*)ws, (float2*)dinv, status, s);
}

void partial_gj_f32(const OrasBatch& bt, const int64_t* lim, int64_t lim_max, float2* ws, float2* dinv,
                    int32_t* status, cudaStream_t s) {
  if (bt.count > 0 && lim_max > 0) gj_all<float2>(bt, ws, dinv, status, s, lim, lim_max);
}

void oras_extract(const OrasBatch& bt, const OrasTopo& tp, int ws_prec, const void* ws, int w_prec,
                  const int64_t* w_off, void* W, cudaStream_t s) {
  note_launch(1);
  dim3 g(256, bt.count);
  if (ws_prec == 0 && w_prec == 0)
    extract_owned_kernel<double2, double2><<<g, 256, 0, s>>>(bt.d_n, bt.d_off, (const double2*)ws, bt.d_sub,
                                                             tp.own_ptr, tp.own_local, w_off, (double2*)W);
  else if (ws_prec == 0 && w_prec == 1)
    extract_owned_kernel<double2, float2><<<g, 256, 0, s>>>(bt.d_n, bt.d_off, (const double2*)ws, bt.d_sub,
                                                            tp.own_ptr, tp.own_local, w_off, (float2*)W);
  else if (ws_prec == 1 && w_prec == 0)
    extract_owned_kernel<float2, double2><<<g, 256, 0, s>>>(bt.d_n, bt.d_off, (const float2*)ws, bt.d_sub,
                                                            tp.own_ptr, tp.own_local, w_off, (double2*)W);
  else
    extract_owned_kernel<float2, float2><<<g, 256, 0, s>>>(bt.d_n, bt.d_off, (const float2*)ws, bt.d_sub,
                                                           tp.own_ptr, tp.own_local, w_off, (float2*)W);
}

void oras_apply_cc(const OrasTopo& tp, int n_tiles, const int32_t* tile_sub, const int32_t* tile_row0, int prec,
                   const int64_t* w_off, const void* W, const void* r, void* z, int R, cudaStream_t s) {
  note_launch(1);
  if (prec == 0) {
    if (R <= 8)
      oras_apply_kernel<double2, 8><<<n_tiles, 256, 0, s>>>(tile_sub, tile_row0, tp.dof_ptr, tp.dofs, tp.own_ptr,
                                                            tp.own_glob, w_off, (const double2*)W,
                                                            (const double2*)r, (double2*)z, R);
    else if (R <= 32)
      oras_apply_kernel<double2, 32><<<n_tiles, 256, 0, s>>>(tile_sub, tile_row0, tp.dof_ptr, tp.dofs, tp.own_ptr,
                                                             tp.own_glob, w_off, (const double2*)W,
                                                             (const double2*)r, (double2*)z, R);
    else
      oras_apply_kernel<double2, 64><<<n_tiles, 256, 0, s>>>(tile_sub, tile_row0, tp.dof_ptr, tp.dofs, tp.own_ptr,
                                                             tp.own_glob, w_off, (const double2*)W,
                                                             (const double2*)r, (double2*)z, R);
  } else {
    if (R <= 8)
      oras_apply_kernel<float2, 8><<<n_tiles, 256, 0, s>>>(tile_sub, tile_row0, tp.dof_ptr, tp.dofs, tp.own_ptr,
                                                           tp.own_glob, w_off, (const float2*)W, (const float2*)r,
                                                           (float2*)z, R);
    else if (R <= 32)
      oras_apply_kernel<float2, 32><<<n_tiles, 256, 0, s>>>(tile_sub, tile_row0, tp.dof_ptr, tp.dofs, tp.own_ptr,
                                                            tp.own_glob, w_off, (const float2*)W, (const float2*)r,
                                                            (float2*)z, R);
    else
      oras_apply_kernel<float2, 64><<<n_tiles, 256, 0, s>>>(tile_sub, tile_row0, tp.dof_ptr, tp.dofs, tp.own_ptr,
                                                            tp.own_glob, w_off, (const float2*)W, (const float2*)r,
                                                            (float2*)z, R);
  }
}

}  // namespace mwk
