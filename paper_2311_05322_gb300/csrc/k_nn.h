// Launchers of the learned-initialiser kernels (k_nn.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mwk {
// C = A B (+ bias), optional H = relu(C).  ws (ws_floats floats, may be null): partial sums of a
// split K, used when the tile grid alone would leave SMs idle; the split sums in a fixed order.
void nn_gemm_bf16(const float* A, int64_t sam, int64_t sak, const void* Bw, int64_t sbk, int64_t sbn,
                  const float* bias, float* C, float* H, int M, int N, int K, cudaStream_t s, float* ws = nullptr,
                  size_t ws_floats = 0);
void nn_gemm_f32(const float* A, int64_t sam, int64_t sak, const float* Bf, int64_t sbk, int64_t sbn,
                 const float* bias, float* C, float* H, int M, int N, int K, cudaStream_t s, float* ws = nullptr,
                 size_t ws_floats = 0);
void nn_colsum(const float* dz, int B, int N, float* db, cudaStream_t s);
void nn_relu_back(const float* z, const float* dh, float* dz, int64_t n, cudaStream_t s);
void nn_convT_fwd(const float* x, const float* w, const float* b, float* a, float* g, int B, int Ci, int Co, int D,
                  cudaStream_t s);
// part: B * Co floats of per-(channel, sample) partial sums for the bias gradient; wpart:
// kConvChunks * Ci * Co * 64 floats of partial weight-gradient sums.
constexpr int kConvChunks = 64;
void nn_convT_bwd(const float* x, const float* w, const float* dy, float* dx, float* dw, float* db, int B, int Ci,
                  int Co, int D, float* part, float* wpart, cudaStream_t s);
void nn_mse(const float* y, const float* t, int64_t n, float* dy, double* part, double* loss, cudaStream_t s);
void nn_adam(float* th, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2, float eps, int step,
             cudaStream_t s);
void nn_to_bf16(const float* a, void* b, int64_t n, cudaStream_t s);
void nn_gather_rows(const float* src, const int32_t* idx, int n, int64_t width, float* dst, cudaStream_t s);
void nn_grid_to_tets(const float* grid, int G, const double* box, const double* xyz, const int32_t* tets, int64_t T,
                     double* out, cudaStream_t s);
}  // namespace mwk
