// Launchers of the multifrontal subdomain factorisation and solve (k_mf.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mwk {

// One product C = C0 + sign * A B of the solve (see mf_gemm_kernel).
struct MfTask {
  int64_t a_off;   // element offset of A [m][k] in the factor store
  int64_t lda;     // row stride of A
  int64_t m, k;
  int64_t b_row;   // first arena row of B, when b_idx < 0
  int64_t b_idx;   // offset of B's arena-row list in idx, or -1
  int64_t c_row;   // first arena row of C, when c_idx < 0
  int64_t c_idx;   // offset of C's arena-row list in idx (negative rows are skipped), or -1
  int64_t c0_row;  // first arena row of C0, or -1 (no C0)
  float sign;
  int32_t pad;
};

// One 64-row tile of a task over K range [k0, k1); slot >= 0: write the raw partial product to
// that partial slot (split K), slot < 0: the whole K range, with the task's epilogue.
struct MfTile {
  int32_t task;
  int32_t row0;
  int32_t k0, k1;
  int32_t slot;
};
// A (task, row tile) whose K range is split: partial slots slot0 .. slot0 + n_slots - 1.
struct MfSplit {
  int32_t task;
  int32_t row0;
  int32_t slot0, n_slots;
};
// Rows of a 64-row tile (the partial slot size is kMfTileRows x R).
constexpr int kMfTileRows = 64;

// Front entries target[i] of the workspace = sum of the contributions code[ptr[i] .. ptr[i+1]).
void mf_assemble(const int64_t* ptr, const int64_t* target, const int32_t* code, int64_t n_t, const int32_t* tet_ids,
                 const double* KM, const double* eps, double k0, const double* Bsurf, const int32_t* surf_tet,
                 double ebr, double ebi, const double2* zc, float2* ws, cudaStream_t s);
// Adds the children's Schur complements into the fronts of nodes[0 .. n_nodes).
void mf_extend_add(const int32_t* nodes, int n_nodes, int64_t fmax, const int64_t* f, const int32_t* p,
                   const int64_t* ws_off, const int64_t* child_ptr, const int32_t* child, const int64_t* inv_off,
                   const int32_t* inv, float2* ws, cudaStream_t s);
// Copies TL | TR and BL of the factored fronts into the factor store (max_entries = largest p f + u p).
void mf_extract(const int32_t* nodes, int n_nodes, int64_t max_entries, const int64_t* f, const int32_t* p,
                const int64_t* ws_off, const int64_t* fac_off, const float2* ws, float2* fac, cudaStream_t s);
// Front right-hand sides of one forward height as pull lists: arena row out[i] = sum of its
// listed arena rows (src >= 0) and input rows (-(src + 1)), for i < n (ptr relative to src).
void mf_pull(const int64_t* out, const int64_t* ptr, const int64_t* src, int64_t n, const float2* in, int R,
             float2* arena, cudaStream_t s);
// Tiles of one height (and direction) then, when some K ranges are split, the reduction of
// their partial slots.
void mf_gemm(const MfTask* tasks, const MfTile* tiles, int n_tiles, const MfSplit* splits, int n_splits,
             const float2* fac, const int32_t* idx, int R, float2* arena, float2* partial, cudaStream_t s);
// The reduction of mf_gemm alone: C = C0 + sign * (sum of the split's partial slots).
void mf_reduce(const MfTask* tasks, const MfSplit* splits, int n_splits, const float2* partial, const int32_t* idx,
               int R, float2* arena, cudaStream_t s);
void mf_owned(const int32_t* own_glob, const int64_t* own_row, int64_t n_own, const float2* arena, int R, float2* z,
              cudaStream_t s);

}  // namespace mwk
