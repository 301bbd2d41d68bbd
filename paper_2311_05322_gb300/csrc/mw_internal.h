// Internal declarations of libmw: context, host topology, device buffers and kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <climits>

#include <string>
#include <vector>

#include "../../include/mw.h"

namespace mw {

// Physical constants (SI).  Time convention e^{i omega t}.
constexpr double kC0 = 299792458.0;
constexpr double kMu0 = 4.0e-7 * 3.14159265358979323846;
constexpr double kPi = 3.14159265358979323846;

// Packed index of the symmetric 6x6 element matrix entry (m <= n): row-major upper triangle.
__host__ __device__ inline int packed6(int m, int n) {
  if (m > n) { int t = m; m = n; n = t; }
  return m * 6 - (m * (m - 1)) / 2 + (n - m);
}
// Packed index of the symmetric 3x3 face matrix entry.
__host__ __device__ inline int packed3(int m, int n) {
  if (m > n) { int t = m; m = n; n = t; }
  return m * 3 - (m * (m - 1)) / 2 + (n - m);
}

struct Error {
  mw_status code;
  std::string msg;
};

// ------------------------------------------------------------------------------------
// Host topology (canonical rules of the public header)
// ------------------------------------------------------------------------------------
struct Topology {
  int64_t n_vert = 0, n_tet = 0, n_edge = 0, n_face = 0, n_bface = 0, nnz = 0;
  std::vector<int32_t> tets;        // [T][4]
  std::vector<int32_t> edge_vert;   // [E][2]
  std::vector<int32_t> tet_edge;    // [T][6]
  std::vector<int8_t> tet_sign;     // [T][6]
  std::vector<int64_t> row_ptr;     // [E+1]
  std::vector<int32_t> col_idx;     // [nnz]
  // pull map: for each nnz position, contributions in tet order then face order;
  // code >= 0: tet t, local (m,n) -> t*36 + m*6 + n; code < 0: -(f*9 + m*3 + n) - 1.
  std::vector<int64_t> contrib_ptr; // [nnz+1]
  std::vector<int32_t> contrib;     // [36 T + 9 F_b]
  std::vector<int32_t> bface_vert;  // [F_b][3] sorted vertex ids
  std::vector<int32_t> bface_edge;  // [F_b][3] global edges (q0q1, q0q2, q1q2)
  std::vector<int32_t> tet_nb;      // [T][4] neighbour across the face opposite local vertex k, -1 = none
};

// Builds the topology; returns false and fills err on a bad mesh.
bool build_topology(int64_t n_vert, int64_t n_tet, const int32_t* tet_vert, Topology& topo, Error& err);

// Blocked layout of the SpMM for the halo-tiled kernel: rows in the Morton order of their edge
// midpoints, cut greedily into blocks whose column sets (halos) hold at most halo_max edges (and
// at most row_max rows and nnz_max nonzeros), so one block fits in shared memory.  Each row keeps its nonzeros in the canonical
// (ascending column) order, so a row's sum runs in the same order as with the canonical CSR.
struct SpmmPlan {
  int64_t n_block = 0;
  std::vector<int64_t> blk_row;    // [n_block+1] offsets into rows
  std::vector<int64_t> blk_halo;   // [n_block+1] offsets into halo
  std::vector<int32_t> halo;       // per block, ascending global columns
  std::vector<int32_t> rows;       // [E] global row of each blocked row
  std::vector<int64_t> rptr;       // [E+1] offsets of each blocked row's nonzeros
  std::vector<uint16_t> lcol;      // [nnz] halo-local column of each blocked nonzero
  std::vector<int32_t> src;        // [nnz] canonical position of each blocked nonzero
};
bool build_spmm_plan(const Topology& topo, const double* xyz, int halo_max, SpmmPlan& plan, Error& err,
                     int row_max = 1 << 30, int64_t nnz_max = INT64_MAX);

// Subdomains of the overlapping Schwarz preconditioner (host side).
struct Subdomains {
  int32_t n_sub = 0;
  std::vector<int32_t> owner;        // [E]
  std::vector<int64_t> dof_ptr;      // [n_sub+1]
  std::vector<int32_t> dofs;         // concatenated, ascending per subdomain
  std::vector<int64_t> own_ptr;      // [n_sub+1]
  std::vector<int32_t> own_local;    // local row index of each owned dof (ascending)
  std::vector<int64_t> tet_ptr;      // [n_sub+1]
  std::vector<int32_t> tet_ids;      // overlapped tets, ascending
  std::vector<int32_t> tet_loc;      // [sum tets][6] local dof index of each tet edge
  std::vector<int64_t> surf_ptr;     // [n_sub+1]
  std::vector<int32_t> surf_vert;    // [sum surf][3] sorted vertex ids of each surface face
  std::vector<int32_t> surf_loc;     // [sum surf][3] local dofs of the face edges (q0q1, q0q2, q1q2)
  std::vector<int32_t> surf_tet;     // [sum surf] inside tet (interface) or -1 (outer boundary)
};

bool build_subdomains(const Topology& topo, int32_t n_sub, const int32_t* tet_part, int32_t overlap,
                      Subdomains& sd, Error& err);

// Sparse local solves (multifrontal LU on a nested-dissection tree per subdomain).
// Every node k of a subdomain's tree owns a front of f_k = p_k + u_k rows: p_k pivots (its
// separator dofs, preal_k of them, padded with identity rows to a multiple of 32) followed by
// u_k update dofs (later-eliminated dofs coupled to the pivots or to a descendant's update).
// Partial Gauss-Jordan on the first p_k pivots leaves the factors
//   TL = F11^-1 [p][p], TR = F11^-1 F12 [p][u], BL = -F21 F11^-1 [u][p]
// and the Schur complement F22 - F21 F11^-1 F12, which the parent adds into its front.
struct Multifrontal {
  static constexpr int kPad = 32;
  int32_t n_nodes = 0, max_height = 0;
  std::vector<int32_t> sub;        // [nodes] subdomain of each node
  std::vector<int32_t> p, preal, u, height, parent;
  std::vector<int64_t> f;          // p + u
  std::vector<int64_t> fac_off;    // element offset of TL|TR ([p][f]) then BL ([u][p])
  int64_t fac_total = 0;
  std::vector<int64_t> piv_ptr;    // [nodes+1] real pivots (local dof index within the subdomain)
  std::vector<int32_t> piv_loc;
  std::vector<int64_t> upd_ptr;    // [nodes+1] update dofs in elimination order (local index)
  std::vector<int32_t> upd_loc;
  std::vector<int64_t> child_ptr;  // [nodes+1] children
  std::vector<int32_t> child;
  std::vector<int64_t> inv_off;    // [nodes] offset of the node's map into its parent's front rows
  std::vector<int32_t> inv;        // for child c: inv[inv_off[c] + r] = update index of parent row r, or -1
  std::vector<int64_t> sub_node_ptr;  // [n_sub+1] nodes of each subdomain (post-order, contiguous)
  // front assembly of the original entries, per subdomain: targets (row * f + col within the
  // node's front, plus the node's workspace offset) and contribution codes, sorted by target;
  // code >= 0: tet slot * 36 + m * 6 + n; code in [-2^30, 0): -1 - (surface slot * 9 + m * 3 + n);
  // kIdentity: a one on the diagonal (metal dof or padding pivot)
  static constexpr int32_t kIdentity = INT32_MIN;
  std::vector<int64_t> ws_off;     // [nodes] element offset of the front in its subdomain's workspace
  std::vector<int64_t> ws_size;    // [n_sub] elements of each subdomain's workspace
  std::vector<int64_t> asm_ptr;    // [targets+1] per subdomain concatenated (see asm_sub_ptr)
  std::vector<int64_t> asm_target;
  std::vector<int32_t> asm_code;
  std::vector<int64_t> asm_sub_ptr;  // [n_sub+1] ranges of targets per subdomain
};

// Builds the trees, the symbolic factorisation and the assembly maps for every subdomain.
// metal (optional, [E]): metal edges, whose rows and columns are those of the identity.
bool build_multifrontal(const Topology& topo, const Subdomains& sd, const std::vector<double>& xyz,
                        const uint8_t* metal, int leaf, Multifrontal& mf, Error& err);

// ------------------------------------------------------------------------------------
// Host L-BFGS (reverse communication)
// ------------------------------------------------------------------------------------
}  // namespace mw

// ------------------------------------------------------------------------------------
// Kernel launchers (k_*.cu).  All take the stream; none synchronises.
// ------------------------------------------------------------------------------------
namespace mwk {

// Count of kernel launches issued by the library (diagnostic; read through mw_kernel_launches).
void note_launch(int n);

struct c64 { float x, y; };

// K1 element geometry: Ke/Me [T][21] packed (signs applied), vol [T]; Bf [F][6] packed.
void elem_geom(const double* xyz, const int32_t* tets, const int8_t* sign, int64_t T, double* KM,
               double* vol, cudaStream_t s);
void face_geom(const double* xyz, const int32_t* face_vert, int64_t F, double* Bf, cudaStream_t s);
void tikhonov_weights(const double* xyz, const int32_t* tets, const int32_t* tet_nb, int64_t T, double* w,
                      cudaStream_t s);
// K2 reassembly for one frequency: A64/A32 [nnz].
// fcls [F_b] (optional): face class 0 open, 1 metal, 2 + p port p, with coefficients zc [2 + P];
// nzmask [nnz] (optional): 1 = zero the entry, 2 = set it to one (metal rows and columns).
void reassemble(const int64_t* cptr, const int32_t* contrib, int64_t nnz, const double* KM, const double* Bf,
                const double* eps, double k0sq, double zb_re, double zb_im, const int32_t* fcls, const double2* zc,
                const uint8_t* nzmask, double2* A64, float2* A32, cudaStream_t s);
// K3 SpMM: Y = A X, [E][R] layout with leading dimension ld (>= R).
// threads: block size, 128, 256 (default) or 512 (the result does not depend on it).
void spmm_f64(const int64_t* rp, const int32_t* ci, const double2* A, const double2* X, double2* Y, int64_t E,
              int R, cudaStream_t s, int threads = 256);
void spmm_f32(const int64_t* rp, const int32_t* ci, const float2* A, const float2* X, float2* Y, int64_t E, int R,
              cudaStream_t s, int threads = 256);
// Bounds of one block of the halo-tiled SpMM plan: columns (halo), rows and nonzeros.
constexpr int kHaloMax = 480, kHaloRows = 512, kHaloNnz = 4096;
// Device copy of mw::SpmmPlan (halo_max bounds every block's halo).
struct SpmmDev {
  int64_t n_block = 0;
  int halo_max = 0;
  const int64_t* blk_row = nullptr;
  const int64_t* blk_halo = nullptr;
  const int32_t* halo = nullptr;
  const int32_t* rows = nullptr;
  const int64_t* rptr = nullptr;
  const uint16_t* lcol = nullptr;
  const int32_t* src = nullptr;
};
// Y = A X with the halo-tiled kernel; A_blk holds the FP32 values in the plan's blocked order.
// Returns false (nothing launched) when the shape is not supported: R odd or above 128, or X
// not 16-byte aligned.  Bit-identical to spmm_f32.
bool spmm_halo_f32(const SpmmDev& p, const float2* A_blk, const float2* X, float2* Y, int R, cudaStream_t s);
// Y = A X (FP32) with X stored as complex BF16 pairs [E][R] (real in the low half).
void spmm_f32_bx(const int64_t* rp, const int32_t* ci, const float2* A, const void* X, float2* Y, int64_t E, int R,
                 cudaStream_t s, int threads = 256);
// A_blk[q] = A32[src[q]].
void spmm_plan_values(const SpmmDev& p, const float2* A32, int64_t nnz, float2* A_blk, cudaStream_t s);
// Split complex FP64 values into double-float (re_hi, re_lo, im_hi, im_lo).
void split_df(const double2* a, float4* o, int64_t n, cudaStream_t s);
// r = b - A x (y = A x when B is null) in double-float arithmetic on the FP32 pipes, with
// per-block partial |r|^2 as residual_f64; returns the number of blocks.
int residual_df(const int64_t* rp, const int32_t* ci, const float4* A, const float4* X, const double2* B,
                double2* Rv, double* part, int64_t E, int R, cudaStream_t s);
// The mixed solver's outer residual: b, A, x in double-float, r rounded to FP32 complex, partial
// ||r||^2 (FP64) per block and column; returns the number of blocks.
int residual_df32(const int64_t* rp, const int32_t* ci, const float4* A, const float4* X, const float4* Bdf,
                  float2* Rv, double* part, int64_t E, int R, cudaStream_t s, bool zero_x = false);
// v0 = r / rnorm per column (0 for done columns) from an FP32 residual.
void normalize_start32(const float2* r, const double* rnorm, const int32_t* done, int64_t E, int R, float2* v0,
                       cudaStream_t s);
// r = b - A x (FP64) and per-column partial ||r||^2 into part[nblk][R]; returns nblk used.
// zero_x: x is known to be 0 (the products are skipped; the same r and norms).
int residual_f64(const int64_t* rp, const int32_t* ci, const double2* A, const double2* X, const double2* B,
                 double2* Rv, double* part, int64_t E, int R, cudaStream_t s, bool zero_x = false);

// Krylov (K6-K8, K15)
// h_part = V^H w per part; returns the number of parts written.  `err` (device int, may be null)
// receives a nonzero code if a bounded wait of the streaming kernel gave up.  stages: ring depth
// of the streaming kernel, 2..6 (0 = default; the result does not depend on it).
int cgs_dots_f64(const double2* V, int64_t vstride, int nvec, const double2* w, int64_t E, int R,
                 double2* part, int32_t* err, cudaStream_t s, int stages = 0);
int cgs_dots_f32(const float2* V, int64_t vstride, int nvec, const float2* w, int64_t E, int R,
                 double2* part, int32_t* err, cudaStream_t s, int stages = 0);
constexpr int kCgsDotsMinStages = 2, kCgsDotsMaxStages = 6;
// Largest part count cgs_dots can return.
constexpr int kCgsDotsMaxParts = 152 * 4 * 8;
// Sets conditional-node handles (cudaGraphConditionalHandle values) of one captured Arnoldi
// step to (*active != 0); at most kMaxStepHandles handles.
constexpr int kMaxStepHandles = 8;
// Deterministic pseudo-random values in scale * [-1, 1) (timing inputs of the launch-shape tuner).
void fill_pattern_f32(float* x, int64_t n, uint32_t seed, cudaStream_t s, double scale = 1.0);
void fill_pattern_f64(double* x, int64_t n, uint32_t seed, cudaStream_t s, double scale = 1.0);
void set_step_conditions(const unsigned long long* handles, int n, const int32_t* active, cudaStream_t s);
// h[i][c] = sum_p part[p][i][c], times vscale[i][c] when given (basis kept unscaled).
void reduce_h(const double2* part, int nparts, int nvec, int R, double2* h, cudaStream_t s,
              const double* vscale = nullptr);
// w -= sum_i h_i V_i and per-part, per-column |w|^2 into npart[part][R]; returns the part count.
// err / stages as for cgs_dots (err null: the non-streaming kernel).  With vscale the basis is
// kept unscaled (V_i = vscale[i][c] Vu_i) and the coefficients become h_i * vscale_i.
int cgs_update_f64(const double2* V, int64_t vstride, int nvec, const double2* h, double2* w, int64_t E, int R,
                   double* npart, cudaStream_t s, int32_t* err = nullptr, int stages = 0,
                   const double* vscale = nullptr);
int cgs_update_f32(const float2* V, int64_t vstride, int nvec, const double2* h, float2* w, int64_t E, int R,
                   double* npart, cudaStream_t s, int32_t* err = nullptr, int stages = 0,
                   const double* vscale = nullptr);
// x[0..n) = v.
void fill_f64(double* x, int n, double v, cudaStream_t s);
int colnorm2_f64(const double2* x, int64_t E, int R, double* npart, cudaStream_t s);
// Givens step for Arnoldi column j; see k_krylov.cu for the state layout.
void givens_step(const double2* h, const double* npart, int nparts, int j, int m, int R, double2* H,
                 double2* cs, double2* gvec, double* target, int32_t* done, int32_t* kcol, double* scale,
                 int32_t* active_count, cudaStream_t s);
void scale_cols_f64(double2* v, const double* scale, int64_t E, int R, cudaStream_t s);
void scale_cols_f32(float2* v, const double* scale, int64_t E, int R, cudaStream_t s);
void solve_hessenberg(const double2* H, const double2* gvec, const int32_t* kcol, int m, int R, double2* y,
                      cudaStream_t s);
// x += sum_{l < kcol[c]} y[c][l] Z_l per column; err as for cgs_dots (null: the non-streaming kernel).
void update_x_f64(const double2* Z, int64_t zstride, const double2* y, const int32_t* kcol, int m, double2* x,
                  int64_t E, int R, cudaStream_t s, int32_t* err = nullptr);
void update_x_f32(const float2* Z, int64_t zstride, const double2* y, const int32_t* kcol, int m, double2* x,
                  int64_t E, int R, cudaStream_t s, int32_t* err = nullptr);
// The same with Z stored as complex BF16 pairs [E][R] per vector (real in the low half), vectors
// zstride values apart.
void update_x_bx(const void* Z, int64_t zstride, const double2* y, const int32_t* kcol, int m, double2* x, int64_t E,
                 int R, cudaStream_t s, int32_t* err);
void reduce_cols(const double* part, int nparts, int R, double* out, cudaStream_t s);

// layout conversions
void cast_f64_to_f32(const double2* a, float2* b, int64_t n, cudaStream_t s);
void cast_f32_to_f64(const float2* a, double2* b, int64_t n, cudaStream_t s);
// [R][E] (column-major, ABI) <-> [E][R] (internal)
void transpose_in(const double2* src, double2* dst, int64_t E, int R, cudaStream_t s);
void transpose_out(const double2* src, double2* dst, int64_t E, int R, cudaStream_t s);

// sources
// B [E][nl] = 0, then B[edge_k][j] = coef_{j0+j} w_k for the entries k of source j0 + j (CSR ptr
// [ns+1]), j < nl (nl < 0: all ns sources, j0 = 0).
void source_rhs(const int64_t* ptr, const int32_t* edge, const double* w, const double2* coef, int ns, double2* B,
                int64_t E, cudaStream_t s, int j0 = 0, int nl = -1);
// Port face moments: fv [F][3] sorted vertex ids, fport [F] port of each face, pdesc [P][10]
// (origin, u, v, a); outputs mom [F][3] and nrm [F].
void port_face_moments(const double* xyz, const int32_t* fv, const int32_t* fport, int64_t F, const double* pdesc,
                       const double* gx, const double* gw, int nq, double* mom, double* nrm, cudaStream_t s);
// w[k] = sum of mom[econ[eptr[k] .. eptr[k+1])]; pn[p] = sum of nrm[fptr[p] .. fptr[p+1]).
void port_accumulate(const int64_t* eptr, const int32_t* econ, int64_t n_ent, const double* mom, double* w,
                     const int64_t* fptr, int n_port, const double* nrm, double* pn, cudaStream_t s);

}  // namespace mwk
