// Launchers of the S-matrix, adjoint-source, per-tet gradient and Tikhonov kernels (K9-K12).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mwk {
void s_extract(const double2* X, const int32_t* edge, const int8_t* sign, int ns, double2* S, cudaStream_t s);
void adjoint_weights(const double2* S, const double2* S_obs, const double2* S_empty, int64_t n, double2* C, double* J,
                     cudaStream_t s);
void adjoint_rhs(const int32_t* edge, const int8_t* sign, int ns, const double2* C, double2* B, int64_t E,
                 cudaStream_t s);
void grad_tet(const int32_t* tet_edge, const double* KM, int64_t T, const double2* L, const double2* X, int ns,
              double k0sq, double* g, cudaStream_t s);
void tikhonov(const int32_t* tet_nb, const double* w, const double* eps, int64_t T, double* grad, double* red,
              cudaStream_t s);
void sqrt_inplace(double* x, int n, cudaStream_t s);
void count_active(const int32_t* done, int R, int32_t* active, cudaStream_t s);
void axpy_f64(double a, const double* x, double* y, int64_t n, cudaStream_t s);
void add_scaled_scalar(double* J, double a, const double* r, cudaStream_t s);
}  // namespace mwk
