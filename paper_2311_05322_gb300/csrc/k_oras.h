// Device-side descriptors shared by the ORAS setup/apply launchers and the host driver.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mwk {

// Subdomain topology on the device (concatenated per-subdomain arrays, see mw::Subdomains).
struct OrasTopo {
  const int64_t* dof_ptr;
  const int32_t* dofs;
  const int64_t* own_ptr;
  const int32_t* own_local;
  const int32_t* own_glob;   // global edge of each owned row
  const int64_t* tet_ptr;
  const int32_t* tet_ids;
  const int32_t* tet_loc;
  const int64_t* surf_ptr;
  const int32_t* surf_loc;
  const int32_t* surf_tet;
};

// A batch of subdomains whose dense matrices share one workspace.
struct OrasBatch {
  int count;
  int64_t nmax;
  const int32_t* d_sub;   // [count] subdomain ids
  const int64_t* d_n;     // [count] n_s
  const int64_t* d_off;   // [count] element offset of each matrix in the workspace
};

// zc (optional): coefficients of the outer-face classes (surf_tet = -1 - class); metal
// (optional, [E]): edges whose local rows and columns become those of the identity.
void oras_local_assemble(const OrasBatch& bt, const OrasTopo& tp, const double* Bsurf, const double* KM,
                         const double* eps, double k0, double eps_bg_re, double eps_bg_im, const double2* zc,
                         const uint8_t* metal, int prec, void* ws, cudaStream_t s);
void oras_invert(const OrasBatch& bt, int prec, void* ws, void* dinv, int32_t* status, cudaStream_t s);
// Partial in-place Gauss-Jordan (FP32): eliminates the first lim[b] pivots (a multiple of 32) of
// each matrix of the batch; lim_max = the largest lim.
void partial_gj_f32(const OrasBatch& bt, const int64_t* lim, int64_t lim_max, float2* ws, float2* dinv,
                    int32_t* status, cudaStream_t s);
void oras_extract(const OrasBatch& bt, const OrasTopo& tp, int ws_prec, const void* ws, int w_prec,
                  const int64_t* w_off, void* W, cudaStream_t s);
void oras_apply_cc(const OrasTopo& tp, int n_tiles, const int32_t* tile_sub, const int32_t* tile_row0, int prec,
                   const int64_t* w_off, const void* W, const void* r, void* z, int R, cudaStream_t s);

}  // namespace mwk
