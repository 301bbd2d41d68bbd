// Launchers of the S-matrix, adjoint-source, per-tet gradient and Tikhonov kernels (K9-K12).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mwk {
// S [ns][nl]: S_ij = (sum_k w_k X[edge_k][j]) / nrm_i over the entries of receiver i (CSR ptr),
// X [E][nl] the fields of nl transmitter columns (nl < 0: all ns).
void s_project(const double2* X, const int64_t* ptr, const int32_t* edge, const double* w, const double* nrm, int ns,
               double2* S, cudaStream_t s, int nl = -1);
void adjoint_weights(const double2* S, const double2* S_obs, const double2* S_empty, int64_t n, double2* C, double* J,
                     cudaStream_t s);
// B [E][nl] = 0, then B[tedge_u][j] = sum over the pairs of edge u of (C[i][j0 + j] / nrm_i) w[tk]
// for the transmitter columns j0 .. j0+nl-1 of C [ns][ns] (nl < 0: all ns, j0 = 0);
// tptr [nu+1], tedge [nu], tsrc / tk [pairs]: the edge-major transpose of the source vectors.
void adjoint_sources(const int64_t* tptr, const int32_t* tedge, const int32_t* tsrc, const int32_t* tk, int64_t nu,
                     const double* w, const double* nrm, const double2* C, int ns, double2* B, int64_t E,
                     cudaStream_t s, int j0 = 0, int nl = -1);
// Adjoint fields by reciprocity: L [E][ns] = X D with D_ij = C_ij / (nrm_i coef_i) (D: scratch
// [ns][ns]); X the forward fields of the same sources, C the adjoint weights [ns][ns].
void reciprocal_adjoint(const double2* X, const double2* C, const double* nrm, const double2* coef, int ns, int64_t E,
                        double2* D, double2* L, cudaStream_t s);
void grad_tet(const int32_t* tet_edge, const double* KM, int64_t T, const double2* L, const double2* X, int ns,
              double k0sq, double* g, cudaStream_t s);
void tikhonov(const int32_t* tet_nb, const double* w, const double* eps, int64_t T, double* grad, double* red,
              cudaStream_t s);
void sqrt_inplace(double* x, int n, cudaStream_t s);
void count_active(const int32_t* done, int R, int32_t* active, cudaStream_t s);
void axpy_f64(double a, const double* x, double* y, int64_t n, cudaStream_t s);
void add_scaled_scalar(double* J, double a, const double* r, cudaStream_t s);
}  // namespace mwk
