// K9 S-matrix extraction, K10 cost and adjoint sources, K11 per-tet gradient, K12 Tikhonov.
//
//   S_ij = q_i^T x_j,  q_i = w_i / n_i                                    (Eq. s1)
//     dipoles: w_i = s_i e_edge(i), n_i = 1;  ports: w_i,e = int_{port i} E_i . N_e,
//     n_i = int_{port i} |E_i|^2
//   J_data = 1/2 sum w_ij |S_ij - S^obs_ij|^2,  w = 1/|S^empty_ij|^2     (Eq. sahar:2)
//   c_ij = w_ij conj(S_ij - S^obs_ij),  adjoint sources sum_i c_ij q_i
//   G_T = sum_j lambda_j^T M^T x_j;  dJ/dRe eps_T += k0^2 Re G_T, dJ/dIm eps_T -= k0^2 Im G_T
//   R = 1/2 sum_{interior F} w_F |eps_T - eps_T'|^2,  w_F = |F| / |c_T - c_T'|
#include "k_adjoint.h"
#include "mw_internal.h"

namespace mwk {
namespace {

// One thread per (receiver i, transmitter j); the entries of q_i in list order.
__global__ void s_project_kernel(const double2* __restrict__ X, const int64_t* __restrict__ ptr,
                                 const int32_t* __restrict__ edge, const double* __restrict__ w,
                                 const double* __restrict__ nrm, int ns, int nl, double2* __restrict__ S) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ns * nl) return;
  const int i = t / nl, j = t % nl;
  double re = 0.0, im = 0.0;
  for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
    const double2 x = X[(int64_t)edge[k] * nl + j];
    re += w[k] * x.x;
    im += w[k] * x.y;
  }
  S[t] = make_double2(re / nrm[i], im / nrm[i]);
}

// Single block: deterministic tree reduction of the cost.
__global__ void adjoint_weights_kernel(const double2* __restrict__ S, const double2* __restrict__ So,
                                       const double2* __restrict__ Se, int64_t n, double2* __restrict__ C,
                                       double* __restrict__ J) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += 256) {
    const double2 d = make_double2(S[k].x - So[k].x, S[k].y - So[k].y);
    const double w = 1.0 / (Se[k].x * Se[k].x + Se[k].y * Se[k].y);
    C[k] = make_double2(w * d.x, -w * d.y);
    acc += 0.5 * w * (d.x * d.x + d.y * d.y);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) *J = red[0];
}

// One thread per (source edge u, column j), over the edge-major transpose of the source
// vectors: the (receiver i, entry k) pairs at edge u in receiver order, so the sum is
// deterministic even where receivers share an edge.  B[e_u][j] = sum (c_ij / n_i) w_k.
__global__ void adjoint_sources_kernel(const int64_t* __restrict__ tptr, const int32_t* __restrict__ tedge,
                                       const int32_t* __restrict__ tsrc, const int32_t* __restrict__ tk, int64_t nu,
                                       const double* __restrict__ w, const double* __restrict__ nrm,
                                       const double2* __restrict__ C, int ns, int j0, int nl,
                                       double2* __restrict__ B) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nu * nl) return;
  const int64_t u = t / nl;
  const int j = (int)(t - u * nl);
  double re = 0.0, im = 0.0;
  for (int64_t q = tptr[u]; q < tptr[u + 1]; ++q) {
    const int i = tsrc[q];
    const double2 c = C[i * ns + j0 + j];
    const double s = w[tk[q]];
    re += (c.x / nrm[i]) * s;
    im += (c.y / nrm[i]) * s;
  }
  B[(int64_t)tedge[u] * nl + j] = make_double2(re, im);
}

// Adjoint fields by reciprocity (receivers are the transmitters, A = A^T): the adjoint source
// of column j is sum_i (c_ij / n_i) w_i and A^-1 w_i = x_i / coef_i, so
// lambda_j = sum_i D_ij x_i with D_ij = c_ij / (n_i coef_i).  One thread per (edge, column).
__global__ void reciprocal_weights_kernel(const double2* __restrict__ C, const double* __restrict__ nrm,
                                          const double2* __restrict__ coef, int ns, double2* __restrict__ D) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ns * ns) return;
  const int i = t / ns;
  const double2 c = C[t], q = coef[i];
  // c / (n_i q)
  const double den = nrm[i] * (q.x * q.x + q.y * q.y);
  D[t] = make_double2((c.x * q.x + c.y * q.y) / den, (c.y * q.x - c.x * q.y) / den);
}

__global__ void reciprocal_combine_kernel(const double2* __restrict__ X, const double2* __restrict__ D, int ns,
                                          int64_t E, double2* __restrict__ L) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= E * ns) return;
  const int64_t e = t / ns;
  const int j = (int)(t - e * ns);
  double re = 0.0, im = 0.0;
  for (int i = 0; i < ns; ++i) {
    const double2 x = X[e * ns + i], d = D[i * ns + j];
    re = fma(x.x, d.x, re);
    re = fma(-x.y, d.y, re);
    im = fma(x.x, d.y, im);
    im = fma(x.y, d.x, im);
  }
  L[t] = make_double2(re, im);
}

// One warp per tet, lanes over the transmitter columns; the warp sums lambda_j^T M^T x_j
// over its columns with a fixed shuffle tree.
template <int CPL>
__global__ void __launch_bounds__(256) grad_tet_kernel(const int32_t* __restrict__ tet_edge,
                                                       const double* __restrict__ KM, int64_t T,
                                                       const double2* __restrict__ L, const double2* __restrict__ X,
                                                       int ns, double k0sq, double* __restrict__ g) {
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= T) return;
  int32_t e[6];
#pragma unroll
  for (int m = 0; m < 6; ++m) e[m] = tet_edge[6 * t + m];
  double M[21];
#pragma unroll
  for (int k = 0; k < 21; ++k) M[k] = KM[42 * t + 21 + k];
  double gr = 0.0, gi = 0.0;
#pragma unroll
  for (int q = 0; q < CPL; ++q) {
    const int j = lane + 32 * q;
    if (j >= ns) break;
    double2 x[6], l[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      x[m] = X[(int64_t)e[m] * ns + j];
      l[m] = L[(int64_t)e[m] * ns + j];
    }
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      double ur = 0.0, ui = 0.0;
#pragma unroll
      for (int n = 0; n < 6; ++n) {
        const double mv = M[mw::packed6(m, n)];
        ur = fma(mv, x[n].x, ur);
        ui = fma(mv, x[n].y, ui);
      }
      gr += l[m].x * ur - l[m].y * ui;
      gi += l[m].x * ui + l[m].y * ur;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    gr += __shfl_xor_sync(0xffffffffu, gr, off);
    gi += __shfl_xor_sync(0xffffffffu, gi, off);
  }
  if (lane == 0) {
    g[2 * t] += k0sq * gr;
    g[2 * t + 1] -= k0sq * gi;
  }
}

constexpr int kTikBlocks = 1024;

__global__ void tikhonov_kernel(const int32_t* __restrict__ nb, const double* __restrict__ w,
                                const double* __restrict__ eps, int64_t T, double* __restrict__ grad,
                                double* __restrict__ part) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (int64_t)gridDim.x * blockDim.x) {
    const double er = eps[2 * t], ei = eps[2 * t + 1];
    double gr = 0.0, gi = 0.0;
    for (int k = 0; k < 4; ++k) {
      const int32_t o = nb[4 * t + k];
      if (o < 0) continue;
      const double wk = w[4 * t + k];
      const double dr = er - eps[2 * (int64_t)o], di = ei - eps[2 * (int64_t)o + 1];
      gr += wk * dr;
      gi += wk * di;
      acc += 0.25 * wk * (dr * dr + di * di);
    }
    grad[2 * t] = gr;
    grad[2 * t + 1] = gi;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[1 + blockIdx.x] = red[0];
}

__global__ void final_sum_kernel(double* __restrict__ part, int n) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) acc += part[1 + i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[0] = red[0];
}

__global__ void sqrt_kernel(double* x, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = sqrt(x[i]);
}

__global__ void count_active_kernel(const int32_t* done, int R, int32_t* active) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < R && !done[i]) atomicAdd(active, 1);
}

}  // namespace

void s_project(const double2* X, const int64_t* ptr, const int32_t* edge, const double* w, const double* nrm, int ns,
               double2* S, cudaStream_t s, int nl) {
  if (nl < 0) nl = ns;
  note_launch(1);
  s_project_kernel<<<(ns * nl + 255) / 256, 256, 0, s>>>(X, ptr, edge, w, nrm, ns, nl, S);
}
void adjoint_weights(const double2* S, const double2* So, const double2* Se, int64_t n, double2* C, double* J,
                     cudaStream_t s) {
  note_launch(1);
  adjoint_weights_kernel<<<1, 256, 0, s>>>(S, So, Se, n, C, J);
}
void adjoint_sources(const int64_t* tptr, const int32_t* tedge, const int32_t* tsrc, const int32_t* tk, int64_t nu,
                     const double* w, const double* nrm, const double2* C, int ns, double2* B, int64_t E,
                     cudaStream_t s, int j0, int nl) {
  if (nl < 0) nl = ns;
  note_launch(1);
  cudaMemsetAsync(B, 0, sizeof(double2) * E * nl, s);
  const int64_t n = nu * nl;
  if (n > 0)
    adjoint_sources_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(tptr, tedge, tsrc, tk, nu, w, nrm, C, ns, j0,
                                                                        nl, B);
}
void grad_tet(const int32_t* tet_edge, const double* KM, int64_t T, const double2* L, const double2* X, int ns,
              double k0sq, double* g, cudaStream_t s) {
  note_launch(1);
  const int64_t threads = T * 32;
  const int blocks = (int)((threads + 255) / 256);
  if (ns <= 32)
    grad_tet_kernel<1><<<blocks, 256, 0, s>>>(tet_edge, KM, T, L, X, ns, k0sq, g);
  else if (ns <= 64)
    grad_tet_kernel<2><<<blocks, 256, 0, s>>>(tet_edge, KM, T, L, X, ns, k0sq, g);
  else
    grad_tet_kernel<4><<<blocks, 256, 0, s>>>(tet_edge, KM, T, L, X, ns, k0sq, g);
}
void reciprocal_adjoint(const double2* X, const double2* C, const double* nrm, const double2* coef, int ns, int64_t E,
                        double2* D, double2* L, cudaStream_t s) {
  note_launch(2);
  reciprocal_weights_kernel<<<(ns * ns + 255) / 256, 256, 0, s>>>(C, nrm, coef, ns, D);
  const int64_t n = E * ns;
  reciprocal_combine_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(X, D, ns, E, L);
}
void tikhonov(const int32_t* tet_nb, const double* w, const double* eps, int64_t T, double* grad, double* red,
              cudaStream_t s) {
  note_launch(2);
  tikhonov_kernel<<<kTikBlocks, 256, 0, s>>>(tet_nb, w, eps, T, grad, red);
  final_sum_kernel<<<1, 256, 0, s>>>(red, kTikBlocks);
}
void sqrt_inplace(double* x, int n, cudaStream_t s) {
  note_launch(1);
  sqrt_kernel<<<(n + 127) / 128, 128, 0, s>>>(x, n); }
void count_active(const int32_t* done, int R, int32_t* active, cudaStream_t s) {
  note_launch(1);
  count_active_kernel<<<(R + 127) / 128, 128, 0, s>>>(done, R, active);
}

}  // namespace mwk

namespace mwk {
namespace {
__global__ void axpy_kernel(double a, const double* __restrict__ x, double* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}
__global__ void add_scaled_scalar_kernel(double* J, double a, const double* r) { *J += a * r[0]; }
}  // namespace
void axpy_f64(double a, const double* x, double* y, int64_t n, cudaStream_t s) {
  note_launch(1);
  int64_t b = (n + 255) / 256;
  axpy_kernel<<<(int)(b < 1216 ? b : 1216), 256, 0, s>>>(a, x, y, n);
}
void add_scaled_scalar(double* J, double a, const double* r, cudaStream_t s) {
  note_launch(1);
  add_scaled_scalar_kernel<<<1, 1, 0, s>>>(J, a, r);
}
}  // namespace mwk
