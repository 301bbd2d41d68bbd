// K1 (element geometry) and K2 (eps -> matrix reassembly) for the edge-element form of Eq. (m2),
// plus right-hand sides, layout conversions and the Tikhonov face weights.
#include "mw_internal.h"

namespace mwk {

namespace {

__constant__ int c_edge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
__constant__ int c_face[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};

struct d3 {
  double x, y, z;
};
__device__ __forceinline__ d3 sub(d3 a, d3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ d3 cross(d3 a, d3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ d3 scale(d3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ d3 load3(const double* p, int64_t v) { return {p[3 * v], p[3 * v + 1], p[3 * v + 2]}; }

constexpr int kGeomThreads = 128;

// One thread per tet: barycentric gradients from cross products of the edge vectors,
//   grad l1 = (d2 x d3)/det, grad l2 = (d3 x d1)/det, grad l3 = (d1 x d2)/det, grad l0 = -sum,
// then K_mn = 4|T| s_m s_n (g_a x g_b).(g_c x g_d) and
// M_mn = s_m s_n |T|/20 [(1+d_ac) G_bd - (1+d_ad) G_bc - (1+d_bc) G_ad + (1+d_bd) G_ac].
// Output rows of 42 doubles (21 packed K, 21 packed M) staged in shared memory so the block
// writes one contiguous, coalesced span.
__global__ void __launch_bounds__(kGeomThreads) elem_geom_kernel(const double* __restrict__ xyz,
                                                                  const int32_t* __restrict__ tets,
                                                                  const int8_t* __restrict__ sign, int64_t T,
                                                                  double* __restrict__ KM, double* __restrict__ vol) {
  __shared__ double stage[kGeomThreads * 42];
  const int64_t t0 = (int64_t)blockIdx.x * kGeomThreads;
  const int64_t t = t0 + threadIdx.x;
  if (t < T) {
    const int4 v = reinterpret_cast<const int4*>(tets)[t];
    d3 P0 = load3(xyz, v.x), P1 = load3(xyz, v.y), P2 = load3(xyz, v.z), P3 = load3(xyz, v.w);
    d3 d1 = sub(P1, P0), d2 = sub(P2, P0), d3v = sub(P3, P0);
    double det = dot(d1, cross(d2, d3v));
    double inv = 1.0 / det;
    d3 g[4];
    g[1] = scale(cross(d2, d3v), inv);
    g[2] = scale(cross(d3v, d1), inv);
    g[3] = scale(cross(d1, d2), inv);
    g[0] = {-(g[1].x + g[2].x + g[3].x), -(g[1].y + g[2].y + g[3].y), -(g[1].z + g[2].z + g[3].z)};
    double V = fabs(det) / 6.0;
    vol[t] = V;
    double G[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) G[p][q] = dot(g[p], g[q]);
    d3 cr[6];
    double s[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      cr[m] = cross(g[c_edge[m][0]], g[c_edge[m][1]]);
      s[m] = (double)sign[6 * t + m];
    }
    double* out = stage + threadIdx.x * 42;
    int k = 0;
#pragma unroll
    for (int m = 0; m < 6; ++m)
#pragma unroll
      for (int n = m; n < 6; ++n) {
        const int a = c_edge[m][0], b = c_edge[m][1], c = c_edge[n][0], d = c_edge[n][1];
        const double ss = s[m] * s[n];
        out[k] = 4.0 * V * ss * dot(cr[m], cr[n]);
        const double br = (1.0 + (a == c)) * G[b][d] - (1.0 + (a == d)) * G[b][c] - (1.0 + (b == c)) * G[a][d] +
                          (1.0 + (b == d)) * G[a][c];
        out[21 + k] = ss * (V / 20.0) * br;
        ++k;
      }
  }
  __syncthreads();
  const int64_t nt = min((int64_t)kGeomThreads, T - t0);
  double* dst = KM + t0 * 42;
  for (int i = threadIdx.x; i < nt * 42; i += kGeomThreads) dst[i] = stage[i];
}

// One thread per face: surface gradients from the inverse metric of the edge vectors
// e1 = q1 - q0, e2 = q2 - q0:  grad l1 = Ginv11 e1 + Ginv12 e2, grad l2 = Ginv21 e1 + Ginv22 e2,
// grad l0 = -(grad l1 + grad l2), area = sqrt(det G)/2; then the 3x3 boundary mass matrix
// over the face edges (q0,q1) (q0,q2) (q1,q2) with int_F l_p l_q = |F|(1 + d_pq)/12.
__global__ void face_geom_kernel(const double* __restrict__ xyz, const int32_t* __restrict__ fv, int64_t F,
                                 double* __restrict__ Bf) {
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  d3 q0 = load3(xyz, fv[3 * f]), q1 = load3(xyz, fv[3 * f + 1]), q2 = load3(xyz, fv[3 * f + 2]);
  d3 e1 = sub(q1, q0), e2 = sub(q2, q0);
  double g11 = dot(e1, e1), g12 = dot(e1, e2), g22 = dot(e2, e2);
  double detg = g11 * g22 - g12 * g12;
  double i11 = g22 / detg, i12 = -g12 / detg, i22 = g11 / detg;
  d3 g[3];
  g[1] = {i11 * e1.x + i12 * e2.x, i11 * e1.y + i12 * e2.y, i11 * e1.z + i12 * e2.z};
  g[2] = {i12 * e1.x + i22 * e2.x, i12 * e1.y + i22 * e2.y, i12 * e1.z + i22 * e2.z};
  g[0] = {-(g[1].x + g[2].x), -(g[1].y + g[2].y), -(g[1].z + g[2].z)};
  double A = 0.5 * sqrt(detg);
  const int pe[3][2] = {{0, 1}, {0, 2}, {1, 2}};
  int k = 0;
  for (int m = 0; m < 3; ++m)
    for (int n = m; n < 3; ++n) {
      const int a = pe[m][0], b = pe[m][1], c = pe[n][0], d = pe[n][1];
      const double br = (1.0 + (a == c)) * dot(g[b], g[d]) - (1.0 + (a == d)) * dot(g[b], g[c]) -
                        (1.0 + (b == c)) * dot(g[a], g[d]) + (1.0 + (b == d)) * dot(g[a], g[c]);
      Bf[6 * f + k] = (A / 12.0) * br;
      ++k;
    }
}

// Tikhonov face weights |F| / |c_T - c_T'| for each tet and each of its 4 faces (0 on the boundary).
__global__ void tikhonov_weights_kernel(const double* __restrict__ xyz, const int32_t* __restrict__ tets,
                                        const int32_t* __restrict__ nb, int64_t T, double* __restrict__ w) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  d3 P[4];
  for (int i = 0; i < 4; ++i) P[i] = load3(xyz, tets[4 * t + i]);
  d3 c = {(P[0].x + P[1].x + P[2].x + P[3].x) * 0.25, (P[0].y + P[1].y + P[2].y + P[3].y) * 0.25,
          (P[0].z + P[1].z + P[2].z + P[3].z) * 0.25};
  for (int k = 0; k < 4; ++k) {
    const int32_t o = nb[4 * t + k];
    if (o < 0) {
      w[4 * t + k] = 0.0;
      continue;
    }
    d3 a = P[c_face[k][0]], b = P[c_face[k][1]], cc = P[c_face[k][2]];
    d3 n = cross(sub(b, a), sub(cc, a));
    double area = 0.5 * sqrt(dot(n, n));
    d3 Q[4];
    for (int i = 0; i < 4; ++i) Q[i] = load3(xyz, tets[4 * (int64_t)o + i]);
    d3 co = {(Q[0].x + Q[1].x + Q[2].x + Q[3].x) * 0.25, (Q[0].y + Q[1].y + Q[2].y + Q[3].y) * 0.25,
             (Q[0].z + Q[1].z + Q[2].z + Q[3].z) * 0.25};
    d3 dd = sub(c, co);
    w[4 * t + k] = area / sqrt(dot(dd, dd));
  }
}

// K2: one thread per matrix entry, pulling its contributions in tet order then face order:
//   A = sum_T (K^T - (k0^2 eps_T) M^T) + sum_F z_F B^F,
// z_F = i k0 sqrt(eps_bg) on every boundary face, or, with face classes (waveguide ports, Eq. m1),
// z_F = zc[fcls[F]]: i k0 sqrt(eps_bg) (open), 0 (metal), i beta_p (port p).  nzmask (optional)
// then replaces the rows and columns of metal edges by those of the identity (1: zero, 2: one).
// Writes the FP64 value and its FP32 rounding.
__global__ void reassemble_kernel(const int64_t* __restrict__ cptr, const int32_t* __restrict__ contrib, int64_t nnz,
                                  const double* __restrict__ KM, const double* __restrict__ Bf,
                                  const double* __restrict__ eps, double k0sq, double zb_re, double zb_im,
                                  const int32_t* __restrict__ fcls, const double2* __restrict__ zc,
                                  const uint8_t* __restrict__ nzmask, double2* __restrict__ A64,
                                  float2* __restrict__ A32) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nnz) return;
  double re = 0.0, im = 0.0;
  const int64_t b = cptr[p], e = cptr[p + 1];
  for (int64_t k = b; k < e; ++k) {
    const int32_t code = contrib[k];
    if (code >= 0) {
      const int64_t t = code / 36;
      const int r = code - (int)t * 36;
      const int pk = mw::packed6(r / 6, r % 6);
      const double Kv = KM[42 * t + pk];
      const double Mv = KM[42 * t + 21 + pk];
      const double cr = k0sq * eps[2 * t], ci = k0sq * eps[2 * t + 1];
      re = __dadd_rn(re, __dsub_rn(Kv, __dmul_rn(cr, Mv)));
      im = __dadd_rn(im, -__dmul_rn(ci, Mv));
    } else {
      const int64_t q = -(int64_t)code - 1;
      const int64_t f = q / 9;
      const int r = (int)(q - f * 9);
      const double Bv = Bf[6 * f + mw::packed3(r / 3, r % 3)];
      double zr = zb_re, zi = zb_im;
      if (fcls) {
        const double2 z = zc[fcls[f]];
        zr = z.x;
        zi = z.y;
      }
      re = __dadd_rn(re, __dmul_rn(zr, Bv));
      im = __dadd_rn(im, __dmul_rn(zi, Bv));
    }
  }
  if (nzmask) {
    const uint8_t m = nzmask[p];
    if (m) {
      re = m == 2 ? 1.0 : 0.0;
      im = 0.0;
    }
  }
  A64[p] = make_double2(re, im);
  if (A32) A32[p] = make_float2((float)re, (float)im);
}

// Right-hand sides b_j = c_j w_j of sparse source vectors (CSR over sources, edges distinct
// within a source): one thread per source.  Dipoles: one entry w = +-1, c = -i omega mu0;
// ports: the load vector w_j and c_j = 2 i beta_j (g = 2 i beta E^TE10, Eq. m2).
__global__ void source_rhs_kernel(const int64_t* __restrict__ ptr, const int32_t* __restrict__ edge,
                                  const double* __restrict__ w, const double2* __restrict__ coef, int j0, int nl,
                                  double2* __restrict__ B) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nl) return;
  const double2 c = coef[j0 + j];
  for (int64_t k = ptr[j0 + j]; k < ptr[j0 + j + 1]; ++k)
    B[(int64_t)edge[k] * nl + j] = make_double2(c.x * w[k], c.y * w[k]);
}

// Port face moments (Eq. m2 right-hand side and Eq. s1), one thread per port face F of port p:
//   mom[F][m] = int_F N_m . E_p,   nrm[F] = int_F |E_p|^2,
// E_p(x) = sin(pi ((x - o).u) / a) v (TE10), N_m = l_a grad l_b - l_b grad l_a for the face edges
// (q0,q1) (q0,q2) (q1,q2) (sorted vertices, so each points from its lower vertex), surface
// gradients as in face_geom_kernel.  Collapsed Gauss-Legendre rule: x = q0 + xi e1 + eta e2,
// eta = (1 - xi) t, dA = 2|F| (1 - xi) dxi dt, nq nodes gx / weights gw on [0, 1] per direction.
// pdesc [P][10] = origin, u, v, a.
__global__ void port_face_kernel(const double* __restrict__ xyz, const int32_t* __restrict__ fv,
                                 const int32_t* __restrict__ fport, int64_t F, const double* __restrict__ pdesc,
                                 const double* __restrict__ gx, const double* __restrict__ gw, int nq,
                                 double* __restrict__ mom, double* __restrict__ nrm) {
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const d3 q0 = load3(xyz, fv[3 * f]), q1 = load3(xyz, fv[3 * f + 1]), q2 = load3(xyz, fv[3 * f + 2]);
  const d3 e1 = sub(q1, q0), e2 = sub(q2, q0);
  const double g11 = dot(e1, e1), g12 = dot(e1, e2), g22 = dot(e2, e2);
  const double detg = g11 * g22 - g12 * g12;
  const double i11 = g22 / detg, i12 = -g12 / detg, i22 = g11 / detg;
  d3 g[3];
  g[1] = {i11 * e1.x + i12 * e2.x, i11 * e1.y + i12 * e2.y, i11 * e1.z + i12 * e2.z};
  g[2] = {i12 * e1.x + i22 * e2.x, i12 * e1.y + i22 * e2.y, i12 * e1.z + i22 * e2.z};
  g[0] = {-(g[1].x + g[2].x), -(g[1].y + g[2].y), -(g[1].z + g[2].z)};
  const double jac = sqrt(detg);  // 2|F|
  const double* P = pdesc + 10 * (int64_t)fport[f];
  const d3 o = {P[0], P[1], P[2]}, u = {P[3], P[4], P[5]}, v = {P[6], P[7], P[8]};
  const double inv_a = 1.0 / P[9];
  // N_m . v for the three face edges is linear in the barycentrics: (N_m . v) = l_a gv_b - l_b gv_a
  const double gv0 = dot(g[0], v), gv1 = dot(g[1], v), gv2 = dot(g[2], v);
  double m0 = 0.0, m1 = 0.0, m2 = 0.0, nn = 0.0;
  for (int i = 0; i < nq; ++i) {
    const double xi = gx[i];
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, an = 0.0;
    for (int j = 0; j < nq; ++j) {
      const double eta = (1.0 - xi) * gx[j];
      const double l0 = 1.0 - xi - eta, l1 = xi, l2 = eta;
      const d3 x = {q0.x + xi * e1.x + eta * e2.x, q0.y + xi * e1.y + eta * e2.y, q0.z + xi * e1.z + eta * e2.z};
      const double sv = sinpi(dot(sub(x, o), u) * inv_a);
      const double wj = gw[j] * sv;
      a0 += wj * (l0 * gv1 - l1 * gv0);
      a1 += wj * (l0 * gv2 - l2 * gv0);
      a2 += wj * (l1 * gv2 - l2 * gv1);
      an += wj * sv;
    }
    const double wi = gw[i] * (1.0 - xi);
    m0 += wi * a0;
    m1 += wi * a1;
    m2 += wi * a2;
    nn += wi * an;
  }
  mom[3 * f + 0] = jac * m0;
  mom[3 * f + 1] = jac * m1;
  mom[3 * f + 2] = jac * m2;
  nrm[f] = jac * nn * dot(v, v);
}

// Port load vectors: entry k (port p, edge e) sums the face moments listed for it, in face
// order; one thread per entry.  Port norms: one thread per port sums its faces in order.
__global__ void port_accumulate_kernel(const int64_t* __restrict__ eptr, const int32_t* __restrict__ econ,
                                       int64_t n_ent, const double* __restrict__ mom, double* __restrict__ w) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_ent) return;
  double acc = 0.0;
  for (int64_t q = eptr[k]; q < eptr[k + 1]; ++q) acc += mom[econ[q]];
  w[k] = acc;
}
__global__ void port_norm_kernel(const int64_t* __restrict__ fptr, int n_port, const double* __restrict__ nrm,
                                 double* __restrict__ pn) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_port) return;
  double acc = 0.0;
  for (int64_t f = fptr[p]; f < fptr[p + 1]; ++f) acc += nrm[f];
  pn[p] = acc;
}

__global__ void cast64to32_kernel(const double2* a, float2* b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = make_float2((float)a[i].x, (float)a[i].y);
}
__global__ void cast32to64_kernel(const float2* a, double2* b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = make_double2((double)a[i].x, (double)a[i].y);
}

// dst[c][r] = src[r][c] for a rows x cols matrix, tiled through shared memory; 1D grid of
// 32 x 32 tiles (column tiles fastest).
__global__ void transpose_kernel(const double2* __restrict__ src, double2* __restrict__ dst, int64_t rows,
                                 int64_t cols) {
  __shared__ double2 tile[32][33];
  const int64_t tiles_c = (cols + 31) / 32;
  const int64_t r0 = ((int64_t)blockIdx.x / tiles_c) * 32;
  const int64_t c0 = ((int64_t)blockIdx.x % tiles_c) * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[i][threadIdx.x] = src[r * cols + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) dst[c * rows + r] = tile[threadIdx.x][i];
  }
}

inline int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }
inline int grid_stride_blocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

}  // namespace

void elem_geom(const double* xyz, const int32_t* tets, const int8_t* sign, int64_t T, double* KM, double* vol,
               cudaStream_t s) {
  note_launch(1);
  elem_geom_kernel<<<blocks_for(T, kGeomThreads), kGeomThreads, 0, s>>>(xyz, tets, sign, T, KM, vol);
}
void face_geom(const double* xyz, const int32_t* fv, int64_t F, double* Bf, cudaStream_t s) {
  if (F > 0) note_launch(1);
  if (F > 0) face_geom_kernel<<<blocks_for(F, 128), 128, 0, s>>>(xyz, fv, F, Bf);
}
void tikhonov_weights(const double* xyz, const int32_t* tets, const int32_t* nb, int64_t T, double* w,
                      cudaStream_t s) {
  note_launch(1);
  tikhonov_weights_kernel<<<blocks_for(T, 128), 128, 0, s>>>(xyz, tets, nb, T, w);
}
void reassemble(const int64_t* cptr, const int32_t* contrib, int64_t nnz, const double* KM, const double* Bf,
                const double* eps, double k0sq, double zb_re, double zb_im, const int32_t* fcls, const double2* zc,
                const uint8_t* nzmask, double2* A64, float2* A32, cudaStream_t s) {
  note_launch(1);
  reassemble_kernel<<<blocks_for(nnz, 256), 256, 0, s>>>(cptr, contrib, nnz, KM, Bf, eps, k0sq, zb_re, zb_im, fcls,
                                                          zc, nzmask, A64, A32);
}
void source_rhs(const int64_t* ptr, const int32_t* edge, const double* w, const double2* coef, int ns, double2* B,
                int64_t E, cudaStream_t s, int j0, int nl) {
  if (nl < 0) nl = ns;
  note_launch(1);
  cudaMemsetAsync(B, 0, sizeof(double2) * E * nl, s);
  source_rhs_kernel<<<blocks_for(nl, 64), 64, 0, s>>>(ptr, edge, w, coef, j0, nl, B);
}
void port_face_moments(const double* xyz, const int32_t* fv, const int32_t* fport, int64_t F, const double* pdesc,
                       const double* gx, const double* gw, int nq, double* mom, double* nrm, cudaStream_t s) {
  note_launch(1);
  if (F > 0) port_face_kernel<<<blocks_for(F, 128), 128, 0, s>>>(xyz, fv, fport, F, pdesc, gx, gw, nq, mom, nrm);
}
void port_accumulate(const int64_t* eptr, const int32_t* econ, int64_t n_ent, const double* mom, double* w,
                     const int64_t* fptr, int n_port, const double* nrm, double* pn, cudaStream_t s) {
  note_launch(2);
  if (n_ent > 0) port_accumulate_kernel<<<blocks_for(n_ent, 128), 128, 0, s>>>(eptr, econ, n_ent, mom, w);
  port_norm_kernel<<<blocks_for(n_port, 64), 64, 0, s>>>(fptr, n_port, nrm, pn);
}
void cast_f64_to_f32(const double2* a, float2* b, int64_t n, cudaStream_t s) {
  note_launch(1);
  cast64to32_kernel<<<grid_stride_blocks(n), 256, 0, s>>>(a, b, n);
}
void cast_f32_to_f64(const float2* a, double2* b, int64_t n, cudaStream_t s) {
  note_launch(1);
  cast32to64_kernel<<<grid_stride_blocks(n), 256, 0, s>>>(a, b, n);
}
void transpose_in(const double2* src, double2* dst, int64_t E, int R, cudaStream_t s) {
  note_launch(1);
  // src [R][E] -> dst [E][R]
  const int64_t tiles = ((R + 31) / 32) * ((E + 31) / 32);
  transpose_kernel<<<(unsigned)tiles, dim3(32, 8), 0, s>>>(src, dst, R, E);
}
void transpose_out(const double2* src, double2* dst, int64_t E, int R, cudaStream_t s) {
  note_launch(1);
  // src [E][R] -> dst [R][E]
  const int64_t tiles = ((R + 31) / 32) * ((E + 31) / 32);
  transpose_kernel<<<(unsigned)tiles, dim3(32, 8), 0, s>>>(src, dst, E, R);
}

}  // namespace mwk
