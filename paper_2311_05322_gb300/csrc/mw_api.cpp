// libmw C-ABI: context, validation and orchestration of the hot path of arXiv 2311.05322.
// All arithmetic of the method runs in the kernels of k_*.cu; this file moves data, sizes
// workspaces, runs the GMRES control flow and the FP64 L-BFGS recursion on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "k_adjoint.h"
#include "k_mf.h"
#include "k_nn.h"
#include "k_oras.h"
#include "k_oras_tc.h"
#include "mw_internal.h"

#include <atomic>

using mw::Error;

static std::atomic<long long> g_launches{0};
void mwk::note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace mwk {
void start_state(const double* npart, int nparts, int R, const double* bnorm, double tol, double inner_tol,
                 int fp64_mode, double* rnorm, double2* gvec, double* target, int32_t* done, int32_t* kcol, int m,
                 cudaStream_t s);
void normalize_start_f64(const double2* r, const double* rnorm, const int32_t* done, int64_t E, int R, double2* v0,
                         cudaStream_t s);
void normalize_start_f32(const double2* r, const double* rnorm, const int32_t* done, int64_t E, int R, float2* v0,
                         cudaStream_t s);
}  // namespace mwk

namespace mwimpl {

constexpr int kMaxRestart = 63;

// Launch-shape value (mw_launch_shapes.spmm_threads) that selects the halo-tiled SpMM.
constexpr int kSpmmHaloShape = 1;
constexpr int kDotParts = mwk::kCgsDotsMaxParts;

// Distance between consecutive Krylov vectors, in complex elements: E * R rounded up to 32, so
// every vector starts on a 256-byte boundary (bulk copies need 16).
inline int64_t krylov_stride(int64_t E, int R) { return (E * R + 31) / 32 * 32; }
constexpr int kRedBlocks = 152 * 4;

struct Ctx;

struct Prec {
  bool ready = false;
  int apply_prec = 0;    // 0 FP64, 1 FP32, 2 BF16 (tensor cores)
  int factor_prec = 0;   // 0 FP64, 1 FP32
  int sparse_leaf = 64;  // nested-dissection leaf size of the sparse solves
  mw::Subdomains sd;
  // device copies
  int64_t *dof_ptr = nullptr, *own_ptr = nullptr, *tet_ptr = nullptr, *surf_ptr = nullptr;
  int32_t *dofs = nullptr, *own_local = nullptr, *own_glob = nullptr, *tet_ids = nullptr, *tet_loc = nullptr,
          *surf_loc = nullptr, *surf_tet = nullptr, *surf_vert = nullptr;
  double* Bsurf = nullptr;
  int n_tiles = 0;
  int32_t *tile_sub = nullptr, *tile_row0 = nullptr;
  int64_t* w_off = nullptr;          // element offsets of W_s (cc layouts)
  std::vector<void*> W;              // per frequency
  mwk::TcPlan tc;                    // BF16 tensor-core layout
  double sum_own_n = 0, sum_n = 0;   // sum_s n_own,s n_s and sum_s n_s
  // sparse (multifrontal) subdomain solves, apply_prec 4
  struct Mf {
    mw::Multifrontal sym;
    std::vector<void*> allocs;       // every device table below
    int64_t *f = nullptr, *ws_off = nullptr, *fac_off = nullptr, *piv_ptr = nullptr, *child_ptr = nullptr,
            *inv_off = nullptr, *rhs_row = nullptr, *w_row = nullptr, *own_row = nullptr, *asm_ptr = nullptr,
            *asm_target = nullptr, *sh_f = nullptr, *sh_off = nullptr, *sh_lim = nullptr;
    int32_t *p = nullptr, *preal = nullptr, *piv_glob = nullptr, *child = nullptr, *inv = nullptr, *idx = nullptr,
            *asm_code = nullptr, *sh_nodes = nullptr, *h_nodes = nullptr;
    mwk::MfTask* tasks = nullptr;
    mwk::MfTile* tiles = nullptr;
    mwk::MfSplit* splits = nullptr;
    // front right-hand sides of the forward sweep as pull lists: output arena row, and its
    // contributions (>= 0: arena row of a child's update; < 0: input row -(g + 1)), per height
    int64_t *pull_out = nullptr, *pull_ptr = nullptr, *pull_src = nullptr;
    std::vector<int64_t> pull_h;     // [H + 2] output-row ranges per height
    std::vector<int64_t> fwd_splits, bwd_splits;  // [H + 2] split ranges per height
    int64_t max_slots = 0;                         // partial slots of the largest launch
    std::vector<int64_t> sh_ptr;     // [(n_sub * (H + 1)) + 1] node ranges per (subdomain, height)
    std::vector<int64_t> sh_fmax, sh_pmax, sh_emax;
    std::vector<int64_t> h_ptr;      // [H + 2] node ranges per height (all subdomains)
    std::vector<int64_t> h_fmax;
    std::vector<int64_t> fwd_tiles, bwd_tiles;  // [H + 2] tile ranges per height
    int64_t arena_rows = 0, ws_max = 0, n_own = 0, max_sh = 0;
    std::vector<void*> fac;          // factors per frequency (FP32 complex; freed after BF16 packing)
    // BF16 tensor-core sweeps (apply_prec 5): one plan per launch (height x direction), whose
    // "subdomains" are the launch's products with K > 0; outputs go to partial slots that
    // mf_reduce turns into C = C0 + sign * A B
    struct TcLaunch {
      mwk::TcPlan plan;
      int64_t *dof_ptr = nullptr, *own_ptr = nullptr;
      int32_t *dofs = nullptr, *own_local = nullptr, *own_glob = nullptr;
      int32_t* c0_glob = nullptr;    // per output row: arena row of C0, or -1
      mwk::MfTask* tasks = nullptr;  // products with K > 0 (plan order), then those with K = 0
      mwk::MfSplit* splits = nullptr;
      int32_t *pk_first = nullptr, *pk_second = nullptr;   // tasks stacked in each plan "subdomain"
      int n_tc = 0, n_splits = 0, ktmax = 0, mtmax = 0;
      // the plan's B rows are rows of the input vector (the leaves' pivot entries), not arena
      // rows: the launch gathers straight from the input and the leaves' pull is skipped
      bool from_input = false;
      std::vector<void*> W;          // BF16 tiles per frequency
    };
    std::vector<TcLaunch> tcl;       // [2 (H + 1)]: forward heights, then backward heights
    int64_t tc_slots = 0;            // partial slots of the largest tensor-core launch
    size_t tc_scratch = 0;           // gathered-operand bytes of the largest plan at 128 columns
  } mf;
  mwk::OrasTopo topo() const {
    return {dof_ptr, dofs, own_ptr, own_local, own_glob, tet_ptr, tet_ids, tet_loc, surf_ptr, surf_loc, surf_tet};
  }
};

struct Work {
  int64_t E = 0;
  int R = 0, m = 0, prec = -1;
  void *V = nullptr, *Z = nullptr;   // Krylov and preconditioned bases, vectors krylov_stride apart
  int32_t* kerr = nullptr;     // bounded-wait error code of the streaming Gram-Schmidt kernel
  float4* xdf = nullptr;       // double-float copy of the iterate (mixed mode)
  float4* bdf = nullptr;       // double-float copy of the block's right-hand sides (mixed mode)
  float2* r32 = nullptr;       // outer residual rounded to FP32 (mixed mode)
  double* vscale = nullptr;    // [m+1][R] factors of the unscaled basis (BF16 tensor-core apply)
  double2 *r = nullptr, *x = nullptr, *part = nullptr, *h = nullptr, *H = nullptr, *cs = nullptr, *g = nullptr,
          *y = nullptr, *bblk = nullptr;
  double *npart = nullptr, *target = nullptr, *rnorm = nullptr, *bnorm = nullptr, *scale = nullptr;
  int32_t *done = nullptr, *kcol = nullptr, *active = nullptr;
  int32_t* h_active = nullptr;  // pinned
  double* h_vec = nullptr;      // pinned [R]
  int32_t* h_ivec = nullptr;    // pinned [R]
  void* tc_scratch = nullptr;   // BF16 gathered operand
  size_t tc_bytes = 0;
  void* mf_arena = nullptr;     // vectors of the sparse subdomain solves
  size_t mf_bytes = 0;
  void* mf_partial = nullptr;   // split-K partial products of the sparse solves
  size_t mf_pbytes = 0;
};

// Optional per-kernel-class timing with CUDA events on the context stream.
struct Profiler {
  uint32_t mask = 0;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> marks;
  double bytes[MW_K_NCLASS] = {};
  double flops[MW_K_NCLASS] = {};
  // device time and launches of classes timed inside replayed cycle graphs
  double graph_ms[MW_K_NCLASS] = {};
  int64_t graph_launches[MW_K_NCLASS] = {};
  cudaEvent_t get() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
};

// Learned-initialiser state: FP32 master parameters, BF16 copies of W1/W2, Adam moments,
// activations and gradients for up to `bcap` samples, and the resident training set.
struct NnState {
  int n_in = 0;
  int64_t np = 0;
  int bcap = 0;
  int step = 0;
  float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  void *W1b = nullptr, *W2b = nullptr;
  float *x = nullptr, *z1 = nullptr, *h1 = nullptr, *z2 = nullptr, *h2 = nullptr, *a1 = nullptr, *g1 = nullptr,
        *a2 = nullptr, *g2 = nullptr, *y = nullptr, *t = nullptr;
  float* gws = nullptr;       // split-K partial sums of the dense layers [32][bcap][1024]
  float* cpart = nullptr;     // per-(channel, sample) partial bias sums [bcap][16]
  float* wpart = nullptr;     // partial weight-gradient sums of the decoder [kConvChunks][16][16][64]
  float *dy = nullptr, *dg2 = nullptr, *da2 = nullptr, *dg1 = nullptr, *da1 = nullptr, *dh2 = nullptr,
        *dz2 = nullptr, *dh1 = nullptr, *dz1 = nullptr;
  double *part = nullptr, *loss = nullptr;
  float *data_x = nullptr, *data_t = nullptr;
  int64_t data_n = 0;
  int32_t* idx = nullptr;
  // parameter offsets (floats) in the flat layout W1 b1 W2 b2 C1 c1 C2 c2 C3 c3
  int64_t oW1, ob1, oW2, ob2, oC1, oc1, oC2, oc2, oC3, oc3;
};

// Launch shapes of the solve kernels for one block shape, picked by timing; none of them changes
// the arithmetic (see mw_autotune).  0 = default shape.
struct Tuned {
  int R = 0, wp = -1, m = 0;
  bool tc = false;                 // BF16 tensor-core preconditioner in use
  mw_launch_shapes sh{0, 0, 0, 256};
  std::vector<std::pair<int, double>> t[MW_TUNE_NKERNEL];  // (candidate, ms per launch) per kernel
};

// One restart cycle of the batched FGMRES captured as a CUDA graph: the start vector, m
// Arnoldi steps whose kernel segments sit in conditional (IF) nodes that run while a column of
// the block is active, the least-squares solve, the solution update and the copy of the
// per-column step counts to the host.  Valid while no device buffer it names has been freed
// (generation `gen`) and for the key below.
struct CycleGraph {
  cudaGraphExec_t exec = nullptr;
  uint64_t gen = 0, last_use = 0;
  int f = -1, R = 0, m = 0, wp = -1;
  bool use_p = false;
  const void* X = nullptr;
  uint32_t mask = 0;
  struct Mark {
    int cls, step;
    cudaEvent_t a, b;
    double bytes;
  };
  std::vector<Mark> marks;           // profiler events around the segments of each step
  int64_t fixed_launches = 0;        // kernels outside the steps
  int64_t step_launches = 0;         // kernels inside one step's conditional bodies
};

struct Ctx {
  int device = 0;
  Profiler prof;
  NnState nn;
  cudaStream_t stream = nullptr;
  std::string err;
  int64_t mem_cap = 0, mem_used = 0;
  std::map<void*, size_t> allocs;

  bool has_mesh = false;
  mw::Topology topo;
  std::vector<double> xyz;
  double* d_xyz = nullptr;
  int32_t *d_tets = nullptr, *d_col = nullptr, *d_contrib = nullptr, *d_bface_vert = nullptr, *d_tet_edge = nullptr,
          *d_tet_nb = nullptr;
  int8_t* d_sign = nullptr;
  int64_t *d_row = nullptr, *d_cptr = nullptr;
  double *d_KM = nullptr, *d_vol = nullptr, *d_Bf = nullptr, *d_tikw = nullptr;

  int n_freq = 0;
  std::vector<double> freqs;
  double eps_bg[2] = {0, 0};
  double* d_eps = nullptr;
  std::vector<double2*> A64;
  std::vector<float2*> A32;
  std::vector<float2*> A32b;       // FP32 values in the SpMM plan's blocked order
  mwk::SpmmDev spmm;               // halo-tiled SpMM plan (device copy)
  std::vector<float4*> Adf;    // double-float copy of A64 for the mixed solver's residual

  int n_src = 0;
  std::vector<int32_t> src_edge;   // dipole sources: edge and sign of each
  std::vector<int8_t> src_sign;
  // Sources as sparse vectors (dipoles: one entry each; ports: the port load vectors):
  // CSR over sources (q_ptr, q_edge, q_w = w_j entries), norms n_j, the edge-major transpose
  // (qt_ptr over distinct edges, qt_edge, and per pair the source and its entry index), and the
  // right-hand-side coefficient of each source per frequency (b_j = c_fj w_j).
  bool src_ports = false;
  std::vector<int64_t> q_ptr_h;
  int64_t *d_q_ptr = nullptr, *d_qt_ptr = nullptr;
  int32_t *d_q_edge = nullptr, *d_qt_edge = nullptr, *d_qt_src = nullptr, *d_qt_k = nullptr;
  double *d_q_w = nullptr, *d_q_norm = nullptr;
  int64_t n_qt = 0;
  std::vector<double2> src_coef;
  double2* d_src_coef = nullptr;

  // Boundary classes (waveguide ports and metal): empty = every boundary face open.
  int n_port = 0;
  std::vector<mw_port> ports;
  std::vector<int32_t> bface_cls;   // [F_b] 0 open, 1 metal, 2 + p port p
  std::vector<uint8_t> metal;       // [E] 1 = metal edge (empty: none)
  int32_t* d_bface_cls = nullptr;
  uint8_t *d_metal = nullptr, *d_nzmask = nullptr;
  std::vector<double2> zc_h;        // [n_freq][2 + n_port] face-class coefficients
  double2* d_zc = nullptr;

  Prec prec;
  Work work;
  std::vector<double2*> Xf;    // forward fields per frequency [E][n_src]
  std::vector<double2*> Lf;    // adjoint fields per frequency
  std::vector<double2*> Bfwd;  // forward right-hand sides per frequency
  // transmitter window of the column-sharded evaluation (mw_forward_cols / mw_gradient_cols):
  // fields, adjoint fields and right-hand sides per frequency [E][win_nl], S columns
  // [n_freq][n_src][win_nl]
  int win_j0 = 0, win_nl = 0, win_nf = 0, win_ns = 0;
  int adjoint_mode = 0;          // MW_ADJOINT_SOLVE or MW_ADJOINT_RECIPROCAL
  int sweep_persistent = 1;      // tensor-core sweeps: persistent CTAs over the tiles of a launch
  int z_bf16 = 1;                // preconditioned vectors of the tensor-core path stored in BF16
  double2* d_D = nullptr;        // reciprocity weights [n_src][n_src]
  std::vector<double2*> Xw, Lw, Bw, Bwa;
  double2* d_Sp = nullptr;
  double2* d_B = nullptr;      // RHS scratch [E][n_src]
  double2 *d_S = nullptr, *d_C = nullptr, *d_So = nullptr, *d_Se = nullptr;
  double *d_J = nullptr, *d_grad = nullptr, *d_gR = nullptr;
  std::vector<double2*> d_Badj;
  double* d_red = nullptr;     // reduction scratch
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  int mf_leaf = 256;         // nested-dissection leaf size for the next sparse preconditioner

  // tuned launch shapes
  bool autotune_on = true;
  std::vector<Tuned> tuned;

  // captured restart cycles
  bool graphs_on = false;
  uint64_t graph_gen = 1, graph_clock = 0;
  std::vector<CycleGraph> graphs;
  cudaStream_t cap_s = nullptr, body_s = nullptr;  // private capture streams
};

struct Fail {
  mw_status code;
  std::string msg;
};

#define CK(call)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) throw Fail{MW_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

void check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw Fail{MW_ECUDA, std::string(what) + ": " + cudaGetErrorString(e)};
}

template <typename T>
T* dalloc(Ctx* c, size_t n) {
  size_t bytes = std::max<size_t>(n * sizeof(T), 16);
  if (c->mem_cap > 0 && c->mem_used + (int64_t)bytes > c->mem_cap)
    throw Fail{MW_ENOMEM, "device memory cap exceeded (" + std::to_string(bytes) + " bytes requested)"};
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Fail{MW_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e)};
  }
  c->allocs[p] = bytes;
  c->mem_used += bytes;
  return (T*)p;
}

void dfree(Ctx* c, void* p) {
  if (!p) return;
  c->graph_gen++;  // a captured cycle may name this buffer
  auto it = c->allocs.find(p);
  if (it != c->allocs.end()) {
    c->mem_used -= it->second;
    c->allocs.erase(it);
  }
  cudaFree(p);
}

template <typename T>
T* upload(Ctx* c, const T* h, size_t n) {
  T* d = dalloc<T>(c, n);
  if (n) CK(cudaMemcpyAsync(d, h, n * sizeof(T), cudaMemcpyHostToDevice, c->stream));
  return d;
}

// Uploads a host vector that may be empty (an empty one gets a one-element zeroed buffer).
template <typename T>
T* upload_vec(Ctx* c, const std::vector<T>& h) {
  if (h.empty()) {
    const std::vector<T> one(1, T{});
    return upload(c, one.data(), 1);
  }
  return upload(c, h.data(), h.size());
}

// Copies h into d, reallocating d only when its size changes (keeps the address, and so any
// captured graph that names it, across repeated uploads of the same size).
template <typename T>
void upload_reuse(Ctx* c, T*& d, const std::vector<T>& h) {
  const size_t bytes = std::max<size_t>(h.size() * sizeof(T), 16);
  auto it = d ? c->allocs.find((void*)d) : c->allocs.end();
  if (!d || it == c->allocs.end() || it->second != bytes) {
    dfree(c, d);
    d = nullptr;
    d = dalloc<T>(c, h.size());
  }
  if (!h.empty()) CK(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream));
}

template <typename F>
mw_status guard(Ctx* c, F&& f) {
  if (!c) return MW_EINVAL;
  try {
    CK(cudaSetDevice(c->device));
    c->err.clear();
    f();
    return MW_OK;
  } catch (const Fail& e) {
    c->err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    c->err = "host allocation failed";
    return MW_ENOMEM;
  } catch (const std::exception& e) {
    c->err = e.what();
    return MW_EINVAL;
  }
}

void require(bool cond, mw_status code, const std::string& msg) {
  if (!cond) throw Fail{code, msg};
}
// Literal messages build a string only on failure (per-element checks of large inputs).
void require(bool cond, mw_status code, const char* msg) {
  if (!cond) throw Fail{code, std::string(msg)};
}

double k0_of(double f) { return 2.0 * mw::kPi * f / mw::kC0; }

void free_work(Ctx* c) {
  Work& w = c->work;
  for (void* p : {(void*)w.V, (void*)w.Z, (void*)w.xdf, (void*)w.r, (void*)w.x, (void*)w.part, (void*)w.h, (void*)w.H, (void*)w.cs,
                  (void*)w.g, (void*)w.y, (void*)w.npart, (void*)w.target, (void*)w.rnorm, (void*)w.bnorm,
                  (void*)w.scale, (void*)w.done, (void*)w.kcol, (void*)w.active, (void*)w.bblk, (void*)w.kerr, (void*)w.bdf, (void*)w.r32, (void*)w.vscale, w.tc_scratch, w.mf_arena, w.mf_partial})
    dfree(c, p);
  if (w.h_active) cudaFreeHost(w.h_active);
  if (w.h_vec) cudaFreeHost(w.h_vec);
  if (w.h_ivec) cudaFreeHost(w.h_ivec);
  w = Work();
}

void ensure_work(Ctx* c, int R, int m, int prec) {
  Work& w = c->work;
  const int64_t E = c->topo.n_edge;
  if (w.E == E && w.R >= R && w.m >= m && w.prec == prec) return;
  free_work(c);
  const size_t es = prec == 0 ? sizeof(double2) : sizeof(float2);
  const size_t n = (size_t)E * R;
  w.E = E;
  w.R = R;
  w.m = m;
  w.prec = prec;
  const size_t nv = (size_t)krylov_stride(E, R);
  w.V = dalloc<unsigned char>(c, es * nv * (m + 1));
  w.Z = dalloc<unsigned char>(c, es * nv * m);
  w.kerr = dalloc<int32_t>(c, 1);
  w.vscale = dalloc<double>(c, (size_t)(m + 1) * R);
  CK(cudaMemsetAsync(w.kerr, 0, sizeof(int32_t), c->stream));
  w.r = dalloc<double2>(c, n);
  w.x = dalloc<double2>(c, n);
  if (prec == 1) {
    w.xdf = dalloc<float4>(c, n);
    w.bdf = dalloc<float4>(c, n);
    w.r32 = dalloc<float2>(c, n);
  }
  w.bblk = dalloc<double2>(c, n);
  w.part = dalloc<double2>(c, (size_t)kDotParts * 8 * R > (size_t)kRedBlocks * (kMaxRestart + 1) * R
                                  ? (size_t)kDotParts * 8 * R
                                  : (size_t)kRedBlocks * (kMaxRestart + 1) * R);
  w.h = dalloc<double2>(c, (size_t)(kMaxRestart + 1) * R);
  w.H = dalloc<double2>(c, (size_t)R * m * (m + 1));
  w.cs = dalloc<double2>(c, (size_t)R * 2 * m);
  w.g = dalloc<double2>(c, (size_t)R * (m + 1));
  w.y = dalloc<double2>(c, (size_t)R * m);
  w.npart = dalloc<double>(c, (size_t)kRedBlocks * R);
  w.target = dalloc<double>(c, R);
  w.rnorm = dalloc<double>(c, R);
  w.bnorm = dalloc<double>(c, R);
  w.scale = dalloc<double>(c, R);
  w.done = dalloc<int32_t>(c, R);
  w.kcol = dalloc<int32_t>(c, R);
  w.active = dalloc<int32_t>(c, 1);
  CK(cudaMallocHost(&w.h_active, sizeof(int32_t)));
  CK(cudaMallocHost(&w.h_vec, sizeof(double) * R));
  CK(cudaMallocHost(&w.h_ivec, sizeof(int32_t) * R));
}

// ---------------------------------------------------------------------------------------
// preconditioner apply on basis vectors of the working precision
// ---------------------------------------------------------------------------------------
// Size the tensor-core apply's gathered-operand scratch before a capture (no allocation may
// happen while the stream is captured).
void ensure_prec_scratch(Ctx* c, int R) {
  Prec& p = c->prec;
  Work& w = c->work;
  if (p.ready && (p.apply_prec == 4 || p.apply_prec == 5)) {
    const size_t need = (size_t)p.mf.arena_rows * R * sizeof(float2);
    if (w.mf_bytes < need) {
      dfree(c, w.mf_arena);
      w.mf_arena = nullptr;
      w.mf_arena = dalloc<unsigned char>(c, need);
      w.mf_bytes = need;
    }
    const int64_t slots = std::max<int64_t>({p.mf.max_slots, p.mf.tc_slots, (int64_t)1});
    const size_t pneed = (size_t)slots * mwk::kMfTileRows * R * sizeof(float2);
    if (w.mf_pbytes < pneed) {
      dfree(c, w.mf_partial);
      w.mf_partial = nullptr;
      w.mf_partial = dalloc<unsigned char>(c, pneed);
      w.mf_pbytes = pneed;
    }
    if (p.apply_prec == 5 && w.tc_bytes < p.mf.tc_scratch) {
      dfree(c, w.tc_scratch);
      w.tc_scratch = nullptr;
      w.tc_scratch = dalloc<unsigned char>(c, p.mf.tc_scratch);
      w.tc_bytes = p.mf.tc_scratch;
    }
    return;
  }
  if (!p.ready || p.apply_prec != 2) return;
  const size_t need = mwk::tc_scratch_bytes(p.tc, R);
  if (w.tc_bytes < need) {
    dfree(c, w.tc_scratch);
    w.tc_scratch = dalloc<unsigned char>(c, need);
    w.tc_bytes = need;
  }
}

// ---------------------------------------------------------------------------------------
// sparse (multifrontal) subdomain solves
// ---------------------------------------------------------------------------------------
// z(owned rows) = sum_s R_s^T D_s B_s^-1 R_s v for R columns (FP32), every subdomain at once.
void apply_sparse(Ctx* c, int f, const float2* v, float2* z, int R) {
  Prec::Mf& m = c->prec.mf;
  Work& w = c->work;
  cudaStream_t s = c->stream;
  require(R >= 1 && R <= 128, MW_EINVAL, "the sparse preconditioner takes 1..128 columns");
  ensure_prec_scratch(c, R);
  float2* arena = (float2*)w.mf_arena;
  float2* partial = (float2*)w.mf_partial;
  const int H = m.sym.max_height;
  if (c->prec.apply_prec == 5) {
    auto run = [&](Prec::Mf::TcLaunch& L) {
      if (L.n_tc > 0) {
        // C = C0 + (sign A) B straight from the MMA epilogue into the arena
        const mwk::OrasTopo tp{L.dof_ptr, L.dofs, L.own_ptr, L.own_local, L.own_glob, nullptr, nullptr, nullptr,
                               nullptr, nullptr, nullptr};
        mwk::oras_apply_tc(L.plan, tp, L.W[f], L.from_input ? v : arena, arena, R, w.tc_scratch, s, 0, nullptr,
                           L.c0_glob, false, c->sweep_persistent != 0);
      }
      // products with K = 0: C = C0
      if (L.n_splits > 0) mwk::mf_reduce(L.tasks, L.splits, L.n_splits, partial, m.idx, R, arena, s);
    };
    for (int h = 0; h <= H; ++h) {
      if (!m.tcl[h].from_input)
        mwk::mf_pull(m.pull_out + m.pull_h[h], m.pull_ptr + m.pull_h[h], m.pull_src, m.pull_h[h + 1] - m.pull_h[h],
                     v, R, arena, s);
      run(m.tcl[h]);
    }
    for (int h = H; h >= 0; --h) run(m.tcl[H + 1 + h]);
    mwk::mf_owned(c->prec.own_glob, m.own_row, m.n_own, arena, R, z, s);
    return;
  }
  const float2* fac = (const float2*)m.fac[f];
  for (int h = 0; h <= H; ++h) {
    mwk::mf_pull(m.pull_out + m.pull_h[h], m.pull_ptr + m.pull_h[h], m.pull_src, m.pull_h[h + 1] - m.pull_h[h], v, R,
                 arena, s);
    mwk::mf_gemm(m.tasks, m.tiles + m.fwd_tiles[h], (int)(m.fwd_tiles[h + 1] - m.fwd_tiles[h]),
                 m.splits + m.fwd_splits[h], (int)(m.fwd_splits[h + 1] - m.fwd_splits[h]), fac, m.idx, R, arena,
                 partial, s);
  }
  for (int h = H; h >= 0; --h)
    mwk::mf_gemm(m.tasks, m.tiles + m.bwd_tiles[h], (int)(m.bwd_tiles[h + 1] - m.bwd_tiles[h]),
                 m.splits + m.bwd_splits[h], (int)(m.bwd_splits[h + 1] - m.bwd_splits[h]), fac, m.idx, R, arena,
                 partial, s);
  mwk::mf_owned(c->prec.own_glob, m.own_row, m.n_own, arena, R, z, s);
}

template <typename T>
T* mf_up(Ctx* c, Prec::Mf& m, const std::vector<T>& h) {
  T* d = upload_vec(c, h);
  m.allocs.push_back(d);
  return d;
}

void build_sparse_tc(Ctx* c, const std::vector<std::vector<mwk::MfTask>>& launches, const std::vector<int32_t>& idx,
                     const std::vector<int32_t>& leaf_in);

// Symbolic factorisation on the host, device tables, then the numeric factorisation of every
// subdomain for every frequency (FP32 fronts in a workspace, partial Gauss-Jordan per height).
void setup_sparse(Ctx* c) {
  Prec& P = c->prec;
  Prec::Mf& m = P.mf;
  const mw::Subdomains& sd = P.sd;
  Error err{MW_OK, ""};
  const uint8_t* metal = c->metal.empty() ? nullptr : c->metal.data();
  if (!mw::build_multifrontal(c->topo, sd, c->xyz, metal, P.sparse_leaf, m.sym, err)) throw Fail{err.code, err.msg};
  const mw::Multifrontal& y = m.sym;
  const int N = y.n_nodes, H = y.max_height, S = sd.n_sub;
  // arena rows: rhs (f), t (p), w (u) per node, then x (n_s) per subdomain
  std::vector<int64_t> rhs_row(N), t_row(N), w_row(N), x_row(S);
  int64_t rows = 0;
  for (int k = 0; k < N; ++k) { rhs_row[k] = rows; rows += y.f[k]; }
  for (int k = 0; k < N; ++k) { t_row[k] = rows; rows += y.p[k]; }
  for (int k = 0; k < N; ++k) { w_row[k] = rows; rows += y.u[k]; }
  for (int s = 0; s < S; ++s) { x_row[s] = rows; rows += sd.dof_ptr[s + 1] - sd.dof_ptr[s]; }
  require(rows < INT32_MAX, MW_EINVAL, "sparse preconditioner too large");
  m.arena_rows = rows;
  // pivots as global edges (forward input) and as arena rows of x; update dofs as arena rows of x
  std::vector<int32_t> piv_glob(y.piv_loc.size()), idx;
  std::vector<int64_t> bidx(N, -1), cidx(N, -1);
  for (int k = 0; k < N; ++k) {
    const int sub = y.sub[k];
    const int64_t d0 = sd.dof_ptr[sub];
    for (int64_t q = y.piv_ptr[k]; q < y.piv_ptr[k + 1]; ++q) piv_glob[q] = sd.dofs[d0 + y.piv_loc[q]];
    bidx[k] = (int64_t)idx.size();
    for (int64_t q = y.upd_ptr[k]; q < y.upd_ptr[k + 1]; ++q) idx.push_back((int32_t)(x_row[sub] + y.upd_loc[q]));
    cidx[k] = (int64_t)idx.size();
    const int32_t pr = y.preal[k];
    for (int32_t i = 0; i < y.p[k]; ++i)
      idx.push_back(i < pr ? (int32_t)(x_row[sub] + y.piv_loc[y.piv_ptr[k] + i]) : -1);
  }
  // nodes per height (all subdomains) and per (subdomain, height)
  std::vector<int32_t> h_nodes, sh_nodes;
  std::vector<int64_t> sh_f, sh_off, sh_lim;
  m.h_ptr.assign(1, 0);
  m.h_fmax.assign(H + 1, 0);
  for (int h = 0; h <= H; ++h) {
    for (int k = 0; k < N; ++k)
      if (y.height[k] == h) {
        h_nodes.push_back(k);
        m.h_fmax[h] = std::max(m.h_fmax[h], y.f[k]);
      }
    m.h_ptr.push_back((int64_t)h_nodes.size());
  }
  // pull lists of the front right-hand sides: row r of node k sums its input entry (a real
  // pivot) and the children's update rows mapped to r, in child order.  The update rows of a
  // leaf receive nothing (they are zero), so they are not listed, and its w product has no C0.
  std::vector<int64_t> pull_out, pull_ptr(1, 0), pull_src;
  m.pull_h.assign(1, 0);
  for (int h = 0; h <= H; ++h) {
    for (int64_t q = m.h_ptr[h]; q < m.h_ptr[h + 1]; ++q) {
      const int k = h_nodes[q];
      const bool leaf = y.child_ptr[k + 1] == y.child_ptr[k];
      const int64_t nr = leaf ? y.p[k] : y.f[k];
      for (int64_t r = 0; r < nr; ++r) {
        pull_out.push_back(rhs_row[k] + r);
        if (r < y.preal[k]) pull_src.push_back(-(int64_t)piv_glob[y.piv_ptr[k] + r] - 1);
        for (int64_t cq = y.child_ptr[k]; cq < y.child_ptr[k + 1]; ++cq) {
          const int32_t ch = y.child[cq];
          const int32_t a = y.inv[y.inv_off[ch] + r];
          if (a >= 0) pull_src.push_back(w_row[ch] + a);
        }
        pull_ptr.push_back((int64_t)pull_src.size());
      }
    }
    m.pull_h.push_back((int64_t)pull_out.size());
  }
  m.sh_ptr.assign(1, 0);
  for (int s = 0; s < S; ++s)
    for (int h = 0; h <= H; ++h) {
      int64_t fm = 0, pm = 0, em = 0;
      for (int64_t k = y.sub_node_ptr[s]; k < y.sub_node_ptr[s + 1]; ++k)
        if (y.height[k] == h) {
          sh_nodes.push_back((int32_t)k);
          sh_f.push_back(y.f[k]);
          sh_off.push_back(y.ws_off[k]);
          sh_lim.push_back(y.p[k]);
          fm = std::max(fm, y.f[k]);
          pm = std::max<int64_t>(pm, y.p[k]);
          em = std::max<int64_t>(em, (int64_t)y.p[k] * y.f[k] + (int64_t)y.u[k] * y.p[k]);
        }
      m.sh_ptr.push_back((int64_t)sh_nodes.size());
      m.sh_fmax.push_back(fm);
      m.sh_pmax.push_back(pm);
      m.sh_emax.push_back(em);
      m.max_sh = std::max<int64_t>(m.max_sh, m.sh_ptr.back() - m.sh_ptr[m.sh_ptr.size() - 2]);
    }
  // GEMM tasks of each height and direction (forward t and w, backward x) and their 64-row
  // tiles.  No tile covers more than kMfMaxTileK of K, so tiles of one launch take similar
  // times; a launch with fewer row tiles than kMfTargetCtas splits K further (chunks of at least
  // 256, aligned to 32) so that every SM gets work.  Split partial products are summed in slot
  // order by the reduction.
  constexpr int64_t kMfTargetCtas = 4 * 152, kMfMinSplitK = 256, kMfMaxTileK = 512;
  std::vector<mwk::MfTask> tasks;
  std::vector<mwk::MfTile> tiles;
  std::vector<mwk::MfSplit> splits;
  std::vector<std::vector<mwk::MfTask>> launches;   // forward heights, then backward heights
  auto emit_launch = [&](const std::vector<mwk::MfTask>& tl) {
    launches.push_back(tl);
    int64_t row_tiles = 0;
    for (const auto& t : tl) row_tiles += (t.m + 63) / 64;
    const int64_t want = row_tiles >= kMfTargetCtas ? 1 : (kMfTargetCtas + row_tiles - 1) / std::max<int64_t>(row_tiles, 1);
    int32_t slot = 0;
    for (const auto& t : tl) {
      const int32_t id = (int32_t)tasks.size();
      tasks.push_back(t);
      // split for parallelism in small launches, and always so that no tile's K exceeds kMfMaxTileK
      const int64_t ns = std::max<int64_t>({(int64_t)1, std::min<int64_t>(want, t.k / kMfMinSplitK),
                                           (t.k + kMfMaxTileK - 1) / kMfMaxTileK});
      const int64_t chunk = ns == 1 ? t.k : ((t.k + ns - 1) / ns + 31) / 32 * 32;
      for (int64_t r0 = 0; r0 < t.m; r0 += 64) {
        if (ns == 1) {
          tiles.push_back({id, (int32_t)r0, 0, (int32_t)std::max<int64_t>(t.k, 0), -1});
          continue;
        }
        const int32_t s0 = slot;
        for (int64_t k0 = 0; k0 < t.k; k0 += chunk)
          tiles.push_back({id, (int32_t)r0, (int32_t)k0, (int32_t)std::min(t.k, k0 + chunk), slot++});
        splits.push_back({id, (int32_t)r0, s0, slot - s0});
      }
    }
    m.max_slots = std::max<int64_t>(m.max_slots, slot);
  };
  m.fwd_tiles.assign(1, 0);
  m.fwd_splits.assign(1, 0);
  for (int h = 0; h <= H; ++h) {
    std::vector<mwk::MfTask> tl;
    for (int64_t q = m.h_ptr[h]; q < m.h_ptr[h + 1]; ++q) {
      const int k = h_nodes[q];
      const int64_t p = y.p[k], u = y.u[k], ff = y.f[k];
      if (p > 0) tl.push_back({y.fac_off[k], ff, p, p, rhs_row[k], -1, t_row[k], -1, -1, 1.f, 0});
      const bool leaf = y.child_ptr[k + 1] == y.child_ptr[k];
      if (u > 0) tl.push_back({y.fac_off[k] + p * ff, std::max<int64_t>(p, 1), u, p, rhs_row[k], -1, w_row[k], -1,
                               leaf ? -1 : rhs_row[k] + p, 1.f, 0});
    }
    emit_launch(tl);
    m.fwd_tiles.push_back((int64_t)tiles.size());
    m.fwd_splits.push_back((int64_t)splits.size());
  }
  m.bwd_tiles.assign(1, m.fwd_tiles.back());
  m.bwd_splits.assign(1, m.fwd_splits.back());
  for (int h = 0; h <= H; ++h) {
    std::vector<mwk::MfTask> tl;
    for (int64_t q = m.h_ptr[h]; q < m.h_ptr[h + 1]; ++q) {
      const int k = h_nodes[q];
      const int64_t p = y.p[k], u = y.u[k], ff = y.f[k];
      if (p > 0) tl.push_back({y.fac_off[k] + p, ff, p, u, -1, bidx[k], -1, cidx[k], t_row[k], -1.f, 0});
    }
    emit_launch(tl);
    m.bwd_tiles.push_back((int64_t)tiles.size());
    m.bwd_splits.push_back((int64_t)splits.size());
  }
  // owned rows of x
  std::vector<int64_t> own_row(sd.own_local.size());
  for (int s = 0; s < S; ++s)
    for (int64_t q = sd.own_ptr[s]; q < sd.own_ptr[s + 1]; ++q) own_row[q] = x_row[s] + sd.own_local[q];
  m.n_own = (int64_t)own_row.size();
  // every index the kernels will follow, checked against its buffer before the first launch
  {
    const char* bad = "internal: sparse preconditioner table out of range";
    const int64_t n_slot_t = (int64_t)sd.tet_ids.size(), n_slot_f = (int64_t)sd.surf_tet.size();
    for (int s = 0; s < S; ++s)
      for (int64_t i = y.asm_sub_ptr[s]; i < y.asm_sub_ptr[s + 1]; ++i) {
        require(y.asm_target[i] >= 0 && y.asm_target[i] < y.ws_size[s], MW_EINVAL, bad);
        require(y.asm_ptr[i] <= y.asm_ptr[i + 1] && y.asm_ptr[i + 1] <= (int64_t)y.asm_code.size(), MW_EINVAL, bad);
        for (int64_t q = y.asm_ptr[i]; q < y.asm_ptr[i + 1]; ++q) {
          const int32_t cd = y.asm_code[q];
          if (cd == mw::Multifrontal::kIdentity) continue;
          if (cd >= 0)
            require(cd / 36 < n_slot_t, MW_EINVAL, bad);
          else
            require((-(int64_t)cd - 1) / 9 < n_slot_f, MW_EINVAL, bad);
        }
      }
    for (int k = 0; k < N; ++k) {
      const int64_t p = y.p[k], u = y.u[k], ff = y.f[k];
      require(p % 32 == 0 && p >= y.preal[k] && ff == p + u, MW_EINVAL, bad);
      require(y.ws_off[k] >= 0 && y.ws_off[k] + ff * ff <= y.ws_size[y.sub[k]], MW_EINVAL, bad);
      require(y.fac_off[k] >= 0 && y.fac_off[k] + p * ff + u * p <= y.fac_total, MW_EINVAL, bad);
      require(rhs_row[k] + ff <= rows && t_row[k] + p <= rows && w_row[k] + u <= rows, MW_EINVAL, bad);
      for (int64_t q = y.child_ptr[k]; q < y.child_ptr[k + 1]; ++q) {
        const int32_t ch = y.child[q];
        require(ch >= 0 && ch < N && y.parent[ch] == k && y.sub[ch] == y.sub[k], MW_EINVAL, bad);
        require(y.inv_off[ch] >= 0 && y.inv_off[ch] + ff <= (int64_t)y.inv.size(), MW_EINVAL, bad);
        for (int64_t r = 0; r < ff; ++r) {
          const int32_t a = y.inv[y.inv_off[ch] + r];
          require(a >= -1 && a < y.u[ch], MW_EINVAL, bad);
        }
      }
    }
    for (int32_t g : piv_glob) require(g >= 0 && g < c->topo.n_edge, MW_EINVAL, bad);
    for (int32_t r : idx) require(r >= -1 && r < rows, MW_EINVAL, bad);
    for (const mwk::MfTask& t : tasks) {
      if (t.m > 0 && t.k > 0) require(t.a_off >= 0 && t.a_off + (t.m - 1) * t.lda + t.k <= y.fac_total, MW_EINVAL, bad);
      if (t.b_idx >= 0) {
        require(t.b_idx + t.k <= (int64_t)idx.size(), MW_EINVAL, bad);
        for (int64_t i = 0; i < t.k; ++i) require(idx[t.b_idx + i] >= 0, MW_EINVAL, bad);
      } else
        require(t.b_row >= 0 && t.b_row + t.k <= rows, MW_EINVAL, bad);
      if (t.c_idx >= 0)
        require(t.c_idx + t.m <= (int64_t)idx.size(), MW_EINVAL, bad);
      else
        require(t.c_row >= 0 && t.c_row + t.m <= rows, MW_EINVAL, bad);
      if (t.c0_row >= 0) require(t.c0_row + t.m <= rows, MW_EINVAL, bad);
    }
    for (int64_t r : own_row) require(r >= 0 && r < rows, MW_EINVAL, bad);
    for (int64_t r : pull_out) require(r >= 0 && r < rows, MW_EINVAL, bad);
    for (int64_t r : pull_src) require(r < rows && -r - 1 < c->topo.n_edge, MW_EINVAL, bad);
    require(pull_ptr.size() == pull_out.size() + 1 && pull_ptr.back() == (int64_t)pull_src.size(), MW_EINVAL, bad);
    for (const mwk::MfTile& tl : tiles) {
      require(tl.task >= 0 && tl.task < (int32_t)tasks.size() && tl.row0 >= 0 && tl.row0 < std::max<int64_t>(tasks[tl.task].m, 1),
              MW_EINVAL, bad);
      require(tl.k0 >= 0 && tl.k0 <= tl.k1 && tl.k1 <= tasks[tl.task].k && tl.slot < m.max_slots, MW_EINVAL, bad);
    }
    for (const mwk::MfSplit& sp : splits)
      require(sp.task >= 0 && sp.task < (int32_t)tasks.size() && sp.slot0 >= 0 && sp.slot0 + sp.n_slots <= m.max_slots,
              MW_EINVAL, bad);
  }
  std::vector<int32_t> pp(y.p.begin(), y.p.end());
  m.f = mf_up(c, m, y.f);
  m.ws_off = mf_up(c, m, y.ws_off);
  m.fac_off = mf_up(c, m, y.fac_off);
  m.piv_ptr = mf_up(c, m, y.piv_ptr);
  m.child_ptr = mf_up(c, m, y.child_ptr);
  m.inv_off = mf_up(c, m, y.inv_off);
  m.rhs_row = mf_up(c, m, rhs_row);
  m.w_row = mf_up(c, m, w_row);
  m.own_row = mf_up(c, m, own_row);
  m.pull_out = mf_up(c, m, pull_out);
  m.pull_ptr = mf_up(c, m, pull_ptr);
  m.pull_src = mf_up(c, m, pull_src.empty() ? std::vector<int64_t>(1, 0) : pull_src);
  m.asm_ptr = mf_up(c, m, y.asm_ptr);
  m.asm_target = mf_up(c, m, y.asm_target);
  m.sh_f = mf_up(c, m, sh_f);
  m.sh_off = mf_up(c, m, sh_off);
  m.sh_lim = mf_up(c, m, sh_lim);
  m.p = mf_up(c, m, pp);
  m.preal = mf_up(c, m, y.preal);
  m.piv_glob = mf_up(c, m, piv_glob);
  m.child = mf_up(c, m, y.child);
  m.inv = mf_up(c, m, y.inv);
  m.idx = mf_up(c, m, idx);
  m.asm_code = mf_up(c, m, y.asm_code);
  m.sh_nodes = mf_up(c, m, sh_nodes);
  m.h_nodes = mf_up(c, m, h_nodes);
  m.tasks = mf_up(c, m, tasks);
  m.tiles = mf_up(c, m, tiles);
  m.splits = mf_up(c, m, splits);
  for (int64_t v : y.ws_size) m.ws_max = std::max(m.ws_max, v);
  // numeric factorisation
  float2* ws = dalloc<float2>(c, std::max<int64_t>(m.ws_max, 1));
  float2* dinv = nullptr;
  int32_t* status = nullptr;
  try {
    dinv = dalloc<float2>(c, std::max<int64_t>(m.max_sh, 1) * 32 * 32);
    status = dalloc<int32_t>(c, 1);
    CK(cudaMemsetAsync(status, 0, sizeof(int32_t), c->stream));
    m.fac.assign(c->n_freq, nullptr);
    for (int f = 0; f < c->n_freq; ++f) {
      m.fac[f] = dalloc<float2>(c, std::max<int64_t>(y.fac_total, 1));
      const double k0 = k0_of(c->freqs[f]);
      const double2* zc = c->d_zc ? c->d_zc + (size_t)f * (2 + c->n_port) : nullptr;
      for (int s = 0; s < S; ++s) {
        CK(cudaMemsetAsync(ws, 0, sizeof(float2) * y.ws_size[s], c->stream));
        const int64_t t0 = y.asm_sub_ptr[s], t1 = y.asm_sub_ptr[s + 1];
        mwk::mf_assemble(m.asm_ptr + t0, m.asm_target + t0, m.asm_code, t1 - t0, P.tet_ids, c->d_KM, c->d_eps, k0,
                         P.Bsurf, P.surf_tet, c->eps_bg[0], c->eps_bg[1], zc, ws, c->stream);
        for (int h = 0; h <= H; ++h) {
          const size_t b = (size_t)s * (H + 1) + h;
          const int64_t q0 = m.sh_ptr[b], q1 = m.sh_ptr[b + 1];
          if (q1 == q0) continue;
          const int cnt = (int)(q1 - q0);
          if (h > 0)
            mwk::mf_extend_add(m.sh_nodes + q0, cnt, m.sh_fmax[b], m.f, m.p, m.ws_off, m.child_ptr, m.child,
                               m.inv_off, m.inv, ws, c->stream);
          mwk::OrasBatch bt{cnt, m.sh_fmax[b], m.sh_nodes + q0, m.sh_f + q0, m.sh_off + q0};
          mwk::partial_gj_f32(bt, m.sh_lim + q0, m.sh_pmax[b], ws, dinv, status, c->stream);
          mwk::mf_extract(m.sh_nodes + q0, cnt, m.sh_emax[b], m.f, m.p, m.ws_off, m.fac_off, ws, (float2*)m.fac[f],
                          c->stream);
        }
        check_launch("sparse factorisation");
      }
    }
    int32_t st = 0;
    CK(cudaMemcpyAsync(&st, status, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    require(st == 0, MW_ESINGULAR, "a front had a near-zero pivot");
  } catch (...) {
    dfree(c, ws);
    dfree(c, dinv);
    dfree(c, status);
    throw;
  }
  dfree(c, ws);
  dfree(c, dinv);
  dfree(c, status);
  if (P.apply_prec == 5) {
    // input row of each arena row that the leaves' pull fills (-1: an identity-padded pivot,
    // zero; -2: not such a row)
    std::vector<int32_t> leaf_in((size_t)rows, -2);
    for (int64_t i = m.pull_h[0]; i < m.pull_h[1]; ++i) {
      const int64_t n_src = pull_ptr[i + 1] - pull_ptr[i];
      if (n_src == 0)
        leaf_in[pull_out[i]] = -1;
      else if (n_src == 1 && pull_src[pull_ptr[i]] < 0)
        leaf_in[pull_out[i]] = (int32_t)(-pull_src[pull_ptr[i]] - 1);
    }
    build_sparse_tc(c, launches, idx, leaf_in);
  }
}

// BF16 tensor-core form of the sweeps: per launch, a tile plan whose "subdomains" are the
// products with K > 0 (inputs: the arena rows of B; outputs: the arena rows of C, with the
// arena rows of C0 added in the MMA epilogue), the BF16 tiles of their FP32 factor blocks times
// the product's sign for every frequency, and one reduction split per 64-row tile of the
// products with K = 0 (C = C0).  The FP32 factors are then freed.
void build_sparse_tc(Ctx* c, const std::vector<std::vector<mwk::MfTask>>& launches, const std::vector<int32_t>& idx,
                     const std::vector<int32_t>& leaf_in) {
  Prec& P = c->prec;
  Prec::Mf& m = P.mf;
  const char* bad = "internal: sparse tensor-core table out of range";
  m.tcl.resize(launches.size());
  for (size_t L = 0; L < launches.size(); ++L) {
    Prec::Mf::TcLaunch& T = m.tcl[L];
    std::vector<mwk::MfTask> ord;
    for (const auto& t : launches[L])
      if (t.k > 0) ord.push_back(t);
    T.n_tc = (int)ord.size();
    for (const auto& t : launches[L])
      if (t.k <= 0) ord.push_back(t);
    auto b_row_of = [&](const mwk::MfTask& t, int64_t i) {
      return t.b_idx >= 0 ? (int64_t)idx[t.b_idx + i] : t.b_row + i;
    };
    // the first forward launch (the leaves) reads its B rows from the input when every one of
    // them is a leaf pivot row that the pull would only copy
    T.from_input = L == 0 && T.n_tc > 0;
    for (int q = 0; q < T.n_tc && T.from_input; ++q)
      for (int64_t i = 0; i < ord[q].k && T.from_input; ++i) {
        const int64_t row = b_row_of(ord[q], i);
        T.from_input = row >= 0 && row < (int64_t)leaf_in.size() && leaf_in[row] >= -1;
      }
    // plan "subdomains": consecutive products with the same B (the forward t and w products of
    // a front) are stacked, so B is gathered once and their rows share the MMA tiles
    mw::Subdomains fake;
    fake.dof_ptr.assign(1, 0);
    fake.own_ptr.assign(1, 0);
    std::vector<int32_t> own_glob, c0_glob, first, second;
    std::vector<mwk::MfSplit> sp;
    int64_t slot = 0;
    for (int q = 0; q < T.n_tc;) {
      const mwk::MfTask& t = ord[q];
      int q2 = -1;
      if (q + 1 < T.n_tc) {
        const mwk::MfTask& u = ord[q + 1];
        if (u.k == t.k && u.b_idx == t.b_idx && (t.b_idx >= 0 || u.b_row == t.b_row)) q2 = q + 1;
      }
      first.push_back(q);
      second.push_back(q2);
      for (int64_t i = 0; i < t.k; ++i) {
        const int64_t row = b_row_of(t, i);
        require(row >= 0 && row < m.arena_rows, MW_EINVAL, bad);
        if (T.from_input) {
          const int32_t in = leaf_in[row];
          require(in >= -1 && in < c->topo.n_edge, MW_EINVAL, bad);
          fake.dofs.push_back(in);
        } else {
          fake.dofs.push_back((int32_t)row);
        }
      }
      fake.dof_ptr.push_back((int64_t)fake.dofs.size());
      int64_t r_out = 0;
      for (int qq : {q, q2}) {
        if (qq < 0) continue;
        const mwk::MfTask& tt = ord[qq];
        for (int64_t r = 0; r < tt.m; ++r, ++r_out) {
          const int64_t crow = tt.c_idx >= 0 ? (int64_t)idx[tt.c_idx + r] : tt.c_row + r;
          const int64_t c0 = tt.c0_row >= 0 ? tt.c0_row + r : -1;
          require(crow >= -1 && crow < m.arena_rows && c0 >= -1 && c0 < m.arena_rows, MW_EINVAL, bad);
          fake.own_local.push_back((int32_t)r_out);
          own_glob.push_back((int32_t)crow);
          c0_glob.push_back((int32_t)c0);
        }
      }
      fake.own_ptr.push_back((int64_t)fake.own_local.size());
      T.ktmax = std::max<int>(T.ktmax, (int)((t.k + 63) / 64));
      T.mtmax = std::max<int>(T.mtmax, (int)((r_out + 127) / 128));
      q += q2 >= 0 ? 2 : 1;
    }
    fake.n_sub = (int)first.size();
    for (int q = T.n_tc; q < (int)ord.size(); ++q)
      for (int64_t r0 = 0; r0 < ord[q].m; r0 += mwk::kMfTileRows) sp.push_back({q, (int32_t)r0, 0, 0});
    require(slot * mwk::kMfTileRows < INT32_MAX, MW_EINVAL, bad);
    m.tc_slots = std::max<int64_t>(m.tc_slots, slot);
    T.n_splits = (int)sp.size();
    T.tasks = mf_up(c, m, ord);
    T.splits = mf_up(c, m, sp);
    if (T.n_tc == 0) continue;
    T.pk_first = mf_up(c, m, first);
    T.pk_second = mf_up(c, m, second);
    T.dof_ptr = mf_up(c, m, fake.dof_ptr);
    T.dofs = mf_up(c, m, fake.dofs);
    T.own_ptr = mf_up(c, m, fake.own_ptr);
    T.own_local = mf_up(c, m, fake.own_local);
    T.own_glob = mf_up(c, m, own_glob);
    T.c0_glob = mf_up(c, m, c0_glob);
    require(mwk::tc_plan_build(T.plan, fake, [&](size_t b) { return (void*)dalloc<unsigned char>(c, b); }, c->stream),
            MW_EINVAL, "tensor-core plan of the sparse sweeps");
    m.tc_scratch = std::max(m.tc_scratch, mwk::tc_scratch_bytes(T.plan, 128));
    T.W.assign(c->n_freq, nullptr);
    for (int f = 0; f < c->n_freq; ++f) {
      T.W[f] = dalloc<unsigned char>(c, std::max<size_t>(mwk::tc_w_bytes(T.plan), 16));
      mwk::tc_pack_stacked(T.plan, T.tasks, T.pk_first, T.pk_second, fake.n_sub, T.ktmax, T.mtmax,
                           (const float2*)m.fac[f], T.W[f], c->stream);
    }
    check_launch("sparse tensor-core packing");
  }
  CK(cudaStreamSynchronize(c->stream));
  for (void*& q : m.fac) {
    dfree(c, q);
    q = nullptr;
  }
}

void apply_prec(Ctx* c, int f, int work_prec, const void* v, void* z, int R, int stages = 0,
                const double* in_scale = nullptr, bool z_bf16 = false) {
  Prec& p = c->prec;
  cudaStream_t s = c->stream;
  if (p.apply_prec == 4 || p.apply_prec == 5) {
    require(work_prec == 1, MW_EINVAL, "the sparse preconditioner needs the mixed-precision solve");
    apply_sparse(c, f, (const float2*)v, (float2*)z, R);
  } else if (p.apply_prec == 2) {
    require(work_prec == 1, MW_EINVAL, "BF16 preconditioner needs the mixed-precision solve");
    Work& w = c->work;
    ensure_prec_scratch(c, R);
    mwk::oras_apply_tc(p.tc, p.topo(), p.W[f], (const float2*)v, (float2*)z, R, w.tc_scratch, s, stages, in_scale,
                       nullptr, z_bf16);
  } else {
    const int need = work_prec;  // 0 FP64, 1 FP32
    require(p.apply_prec == need, MW_EINVAL,
            "preconditioner precision does not match the solve mode (FP64 mode needs an FP64-applied inverse)");
    require(R <= 64, MW_EINVAL, "the CUDA-core preconditioner apply takes at most 64 columns per launch");
    mwk::oras_apply_cc(p.topo(), p.n_tiles, p.tile_sub, p.tile_row0, p.apply_prec, p.w_off, p.W[f], v, z, R, s);
  }
  check_launch("oras apply");
}

// Records an event pair around the enclosed launches when the class is enabled.
struct ProfScope {
  Ctx* c;
  int cls;
  cudaEvent_t a = nullptr;
  // bytes / flops: algorithmic bytes moved and flops done by the enclosed launches (for
  // roofline fractions)
  ProfScope(Ctx* c_, int k, double bytes, double flops = 0.0) : c(c_), cls(k) {
    if (c->prof.mask & (1u << k)) {
      a = c->prof.get();
      cudaEventRecord(a, c->stream);
      c->prof.bytes[k] += bytes;
      c->prof.flops[k] += flops;
    }
  }
  ~ProfScope() {
    if (a) {
      cudaEvent_t b = c->prof.get();
      cudaEventRecord(b, c->stream);
      c->prof.marks.push_back({cls, {a, b}});
    }
  }
};

// Reads the bounded-wait error word of the tensor-core preconditioner apply (after the work
// that used it has completed on the stream) and turns a wait that ran out into MW_ETIMEOUT,
// clearing the word for the next call.
void check_tc_wait(Ctx* c) {
  if (!(c->prec.ready && c->prec.apply_prec == 2 && c->prec.tc.err)) return;
  int32_t e = 0;
  CK(cudaMemcpyAsync(&e, c->prec.tc.err, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (e != 0) {
    CK(cudaMemsetAsync(c->prec.tc.err, 0, sizeof(int32_t), c->stream));
    throw Fail{MW_ETIMEOUT, "tensor-core preconditioner apply: bounded wait ran out (code " + std::to_string(e) + ")"};
  }
}

// Algorithmic bytes of one preconditioner apply on R columns: the owned-row inverses once,
// the gathered subdomain inputs and the owned outputs.
// zb: the output z is stored as BF16 pairs (4 bytes per value)
double oras_bytes(Ctx* c, int R, bool zb = false) {
  const Prec& p = c->prec;
  if (p.apply_prec == 4) return 8.0 * (double)p.mf.sym.fac_total + 8.0 * R * (p.sum_n + (double)c->topo.n_edge);
  if (p.apply_prec == 5) return 4.0 * (double)p.mf.sym.fac_total + 8.0 * R * (p.sum_n + (double)c->topo.n_edge);
  const double wb = p.apply_prec == 0 ? 16.0 : (p.apply_prec == 1 ? 8.0 : 4.0);
  const double vb = p.apply_prec == 0 ? 16.0 : 8.0;
  return wb * p.sum_own_n + vb * R * (double)p.sum_n + (zb ? 4.0 : vb) * R * (double)c->topo.n_edge;
}

int read_active(Ctx* c) {
  CK(cudaMemcpyAsync(c->work.h_active, c->work.active, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return *c->work.h_active;
}

// r = b - A_f x with per-block partial norms: FP64 arithmetic into w.r in FP64 mode; in mixed
// mode double-float arithmetic on the FP32 pipes (same accuracy class) with b taken from w.bdf
// (split once per block solve) and r rounded to FP32 into w.r32, which is all the inner solver's
// start vector needs.
// zero_x: X is known to be 0 (the first outer step), so r = b without the products.
int outer_residual(Ctx* c, int f, int wp, const double2* X, const double2* B, int R, bool zero_x = false) {
  Work& w = c->work;
  const int64_t E = c->topo.n_edge;
  if (wp == 0)
    return mwk::residual_f64(c->d_row, c->d_col, c->A64[f], X, B, w.r, w.npart, E, R, c->stream, zero_x);
  if (!zero_x) mwk::split_df(X, w.xdf, E * R, c->stream);
  return mwk::residual_df32(c->d_row, c->d_col, c->Adf[f], w.xdf, w.bdf, w.r32, w.npart, E, R, c->stream, zero_x);
}

struct BlockStats {
  int outer = 0, steps = 0;
  bool have_relres = false;  // the last action was a residual check of the final x
};

// Solve A_f X = B for a block of R columns ([E][R] layout, FP64 in and out).
// Arguments of one restart cycle.
struct CycleArgs {
  int f, R, m, wp;
  bool use_p;
  double2* X;
  int64_t E, vstride;
  size_t es;
  Tuned t;
  // BF16 tensor-core apply: the basis is kept unscaled, V_i = vscale[i][c] * Vu_i, and the factor
  // is applied where a vector is read (the apply's gather, the dots' reduction, the update's
  // coefficients) instead of in a separate pass over each new vector
  bool lazy;
  // the preconditioned vectors Z are stored as complex BF16 pairs (tensor-core path): flexible
  // GMRES uses the stored Z both in A Z and in x += Z y, so their rounding only changes the
  // preconditioner
  bool zb;
  void* Vp(const Work& w, int i) const { return (unsigned char*)w.V + es * vstride * i; }
  void* Zp(const Work& w, int i) const {
    return use_p ? (unsigned char*)w.Z + (zb ? (size_t)4 : es) * vstride * i : Vp(w, i);
  }
};

// Arnoldi step j as segments (preconditioner apply, SpMM, Gram-Schmidt dots, Gram-Schmidt
// update, Givens and scaling); seg(cls, bytes, fn) runs fn, which launches on c->stream.
// FP32 SpMM of frequency f: the halo-tiled kernel for launch shape kSpmmHaloShape (when the
// shape allows it), else the row-per-warp kernel with `threads` per block.  Both sum every row
// in the same order, so the choice never changes a result bit.
bool spmm_halo_ok(Ctx* c, int R) {
  return c->spmm.n_block > 0 && R >= 2 && R <= 128 && R % 2 == 0 && (int)c->A32b.size() == c->n_freq;
}
void spmm32(Ctx* c, int f, const float2* X, float2* Y, int R, int threads) {
  if (threads == kSpmmHaloShape && spmm_halo_ok(c, R) && mwk::spmm_halo_f32(c->spmm, c->A32b[f], X, Y, R, c->stream))
    return;
  mwk::spmm_f32(c->d_row, c->d_col, c->A32[f], X, Y, c->topo.n_edge, R, c->stream, threads < 128 ? 256 : threads);
}
// The same with X stored as complex BF16 pairs: the row-per-warp kernel (256 threads for the
// halo shape, which has no BF16 form).
void spmm32_bx(Ctx* c, int f, const void* X, float2* Y, int R, int threads) {
  mwk::spmm_f32_bx(c->d_row, c->d_col, c->A32[f], X, Y, c->topo.n_edge, R, c->stream, threads < 128 ? 256 : threads);
}

template <class Seg>
void arnoldi_step(Ctx* c, const CycleArgs& a, int j, Seg&& seg) {
  Work& w = c->work;
  const int64_t E = a.E;
  const int R = a.R;
  const double* vs = a.lazy ? w.vscale : nullptr;
  if (a.use_p)
    seg(MW_K_ORAS, oras_bytes(c, R, a.zb), [&] {
      apply_prec(c, a.f, a.wp, a.Vp(w, j), a.Zp(w, j), R, a.t.sh.tc_stages, vs ? vs + (size_t)j * R : nullptr,
                 a.zb);
    });
  seg(MW_K_SPMM, (double)c->topo.nnz * (a.es + 4) + 8.0 * (E + 1) + (double)(a.es + (a.zb ? 4 : a.es)) * E * R, [&] {
    if (a.wp == 0)
      mwk::spmm_f64(c->d_row, c->d_col, c->A64[a.f], (const double2*)a.Zp(w, j), (double2*)a.Vp(w, j + 1), E, R,
                    c->stream, a.t.sh.spmm_threads);
    else if (a.zb)
      spmm32_bx(c, a.f, a.Zp(w, j), (float2*)a.Vp(w, j + 1), R, a.t.sh.spmm_threads);
    else
      spmm32(c, a.f, (const float2*)a.Zp(w, j), (float2*)a.Vp(w, j + 1), R, a.t.sh.spmm_threads);
  });
  seg(MW_K_CGS_DOTS, (double)a.es * E * R * (j + 2), [&] {
    const int np = a.wp == 0 ? mwk::cgs_dots_f64((const double2*)w.V, a.vstride, j + 1,
                                                 (const double2*)a.Vp(w, j + 1), E, R, w.part, w.kerr, c->stream,
                                                 a.t.sh.dots_stages)
                             : mwk::cgs_dots_f32((const float2*)w.V, a.vstride, j + 1,
                                                 (const float2*)a.Vp(w, j + 1), E, R, w.part, w.kerr, c->stream,
                                                 a.t.sh.dots_stages);
    mwk::reduce_h(w.part, np, j + 1, R, w.h, c->stream, vs);
  });
  int nu = 0;
  seg(MW_K_CGS_UPDATE, (double)a.es * E * R * (j + 3), [&] {
    nu = a.wp == 0 ? mwk::cgs_update_f64((const double2*)w.V, a.vstride, j + 1, w.h, (double2*)a.Vp(w, j + 1), E,
                                         R, w.npart, c->stream, w.kerr, a.t.sh.update_stages, vs)
                   : mwk::cgs_update_f32((const float2*)w.V, a.vstride, j + 1, w.h, (float2*)a.Vp(w, j + 1), E,
                                         R, w.npart, c->stream, w.kerr, a.t.sh.update_stages, vs);
  });
  seg(-1, 0.0, [&] {
    CK(cudaMemsetAsync(w.active, 0, sizeof(int32_t), c->stream));
    mwk::givens_step(w.h, w.npart, nu, j, a.m, R, w.H, w.cs, w.g, w.target, w.done, w.kcol,
                     vs ? w.vscale + (size_t)(j + 1) * R : w.scale, w.active, c->stream);
    if (!vs) {
      if (a.wp == 0)
        mwk::scale_cols_f64((double2*)a.Vp(w, j + 1), w.scale, E, R, c->stream);
      else
        mwk::scale_cols_f32((float2*)a.Vp(w, j + 1), w.scale, E, R, c->stream);
    }
  });
}
constexpr int kStepSegments = 5;

void cycle_start(Ctx* c, const CycleArgs& a) {
  Work& w = c->work;
  if (a.wp == 0)
    mwk::normalize_start_f64(w.r, w.rnorm, w.done, a.E, a.R, (double2*)a.Vp(w, 0), c->stream);
  else
    mwk::normalize_start32(w.r32, w.rnorm, w.done, a.E, a.R, (float2*)a.Vp(w, 0), c->stream);
  if (a.lazy) mwk::fill_f64(w.vscale, a.R, 1.0, c->stream);   // V_0 is stored scaled
}

// Least squares, x += Z y, and the per-column step counts into w.h_ivec (not yet synchronised).
void cycle_finish(Ctx* c, const CycleArgs& a) {
  Work& w = c->work;
  mwk::solve_hessenberg(w.H, w.g, w.kcol, a.m, a.R, w.y, c->stream);
  if (a.wp == 0)
    mwk::update_x_f64((const double2*)a.Zp(w, 0), a.vstride, w.y, w.kcol, a.m, a.X, a.E, a.R, c->stream, w.kerr);
  else
    if (a.zb)
      mwk::update_x_bx(a.Zp(w, 0), a.vstride, w.y, w.kcol, a.m, a.X, a.E, a.R, c->stream, w.kerr);
    else
      mwk::update_x_f32((const float2*)a.Zp(w, 0), a.vstride, w.y, w.kcol, a.m, a.X, a.E, a.R, c->stream, w.kerr);
  check_launch("solution update");
  CK(cudaMemcpyAsync(w.h_ivec, w.kcol, sizeof(int32_t) * a.R, cudaMemcpyDeviceToHost, c->stream));
}

// Eager cycle: the host reads the active-column count after every step.  Returns the steps run.
int cycle_eager(Ctx* c, const CycleArgs& a, int max_steps) {
  cycle_start(c, a);
  int j = 0;
  while (j < a.m) {
    arnoldi_step(c, a, j, [&](int cls, double bytes, auto&& fn) {
      if (cls >= 0) {
        ProfScope ps(c, cls, bytes);
        fn();
      } else {
        fn();
      }
    });
    check_launch("arnoldi step");
    ++j;
    if (read_active(c) == 0 || j >= max_steps) break;
  }
  cycle_finish(c, a);
  CK(cudaStreamSynchronize(c->stream));
  return j;
}

void destroy_graph(CycleGraph& G) {
  if (G.exec) cudaGraphExecDestroy(G.exec);
  for (auto& mk : G.marks) {
    cudaEventDestroy(mk.a);
    cudaEventDestroy(mk.b);
  }
  G = CycleGraph();
}

void drop_graphs(Ctx* c) {
  for (auto& G : c->graphs) destroy_graph(G);
  c->graphs.clear();
}

// Captures one cycle for the arguments `a` into conditional graph nodes.
CycleGraph capture_cycle(Ctx* c, const CycleArgs& a) {
  if (!c->cap_s) CK(cudaStreamCreateWithFlags(&c->cap_s, cudaStreamNonBlocking));
  if (!c->body_s) CK(cudaStreamCreateWithFlags(&c->body_s, cudaStreamNonBlocking));
  if (a.use_p) ensure_prec_scratch(c, a.R);
  Work& w = c->work;
  CycleGraph G;
  G.f = a.f;
  G.R = a.R;
  G.m = a.m;
  G.wp = a.wp;
  G.use_p = a.use_p;
  G.X = a.X;
  G.mask = c->prof.mask;
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  const cudaStream_t user = c->stream;
  const long long l0 = g_launches.load();
  bool capturing = false, body_capturing = false;
  try {
    CK(cudaStreamBeginCaptureToGraph(c->cap_s, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    capturing = true;
    c->stream = c->cap_s;
    cycle_start(c, a);
    long long body = 0;
    for (int j = 0; j < a.m; ++j) {
      unsigned long long hs[kStepSegments];
      for (int k = 0; k < kStepSegments; ++k) {
        cudaGraphConditionalHandle h;
        CK(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
        hs[k] = (unsigned long long)h;
      }
      mwk::set_step_conditions(hs, kStepSegments, w.active, c->cap_s);
      int k = 0;
      const long long ls = g_launches.load();
      arnoldi_step(c, a, j, [&](int cls, double bytes, auto&& fn) {
        const bool prof = cls >= 0 && (c->prof.mask & (1u << cls));
        CycleGraph::Mark mk{cls, j, nullptr, nullptr, bytes};
        if (prof) {
          CK(cudaEventCreate(&mk.a));
          CK(cudaEventCreate(&mk.b));
          G.marks.push_back(mk);
          CK(cudaEventRecordWithFlags(mk.a, c->cap_s, cudaEventRecordExternal));
        }
        cudaStreamCaptureStatus cst;
        cudaGraph_t cg = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        CK(cudaStreamGetCaptureInfo(c->cap_s, &cst, nullptr, &cg, &deps, nullptr, &nd));
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = (cudaGraphConditionalHandle)hs[k++];
        np.conditional.type = cudaGraphCondTypeIf;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        CK(cudaGraphAddNode(&node, cg, deps, nullptr, nd, &np));
        CK(cudaStreamUpdateCaptureDependencies(c->cap_s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
        CK(cudaStreamBeginCaptureToGraph(c->body_s, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeRelaxed));
        body_capturing = true;
        c->stream = c->body_s;
        fn();
        check_launch("captured arnoldi segment");
        c->stream = c->cap_s;
        cudaGraph_t bg = nullptr;
        CK(cudaStreamEndCapture(c->body_s, &bg));
        body_capturing = false;
        if (prof) CK(cudaEventRecordWithFlags(mk.b, c->cap_s, cudaEventRecordExternal));
      });
      if (j == 0) body = g_launches.load() - ls;
    }
    cycle_finish(c, a);
    cudaGraph_t out = nullptr;
    CK(cudaStreamEndCapture(c->cap_s, &out));
    capturing = false;
    c->stream = user;
    G.step_launches = body;
    G.fixed_launches = (g_launches.load() - l0) - (long long)a.m * body;
    g_launches.fetch_sub(g_launches.load() - l0);  // nothing ran yet
    CK(cudaGraphInstantiate(&G.exec, g, 0));
    cudaGraphDestroy(g);
  } catch (...) {
    c->stream = user;
    cudaGraph_t t = nullptr;
    if (body_capturing) cudaStreamEndCapture(c->body_s, &t);
    if (capturing) cudaStreamEndCapture(c->cap_s, &t);
    cudaGraphDestroy(g);
    g_launches.fetch_sub(g_launches.load() - l0);
    destroy_graph(G);
    cudaGetLastError();
    throw;
  }
  G.gen = c->graph_gen;
  return G;
}

// Graph cycle: one launch and one host synchronisation per restart cycle.  Returns the steps run
// (the largest per-column step count).
int cycle_graph(Ctx* c, const CycleArgs& a) {
  CycleGraph* G = nullptr;
  for (auto& g : c->graphs)
    if (g.gen == c->graph_gen && g.f == a.f && g.R == a.R && g.m == a.m && g.wp == a.wp && g.use_p == a.use_p &&
        g.X == a.X && g.mask == c->prof.mask) {
      G = &g;
      break;
    }
  if (!G) {
    // stale graphs name freed buffers; the cache holds a handful of live ones
    std::vector<CycleGraph> keep;
    for (auto& g : c->graphs) {
      if (g.gen == c->graph_gen && keep.size() < 7)
        keep.push_back(g);
      else
        destroy_graph(g);
    }
    c->graphs.swap(keep);
    c->graphs.push_back(capture_cycle(c, a));
    G = &c->graphs.back();
  }
  G->last_use = ++c->graph_clock;
  CK(cudaGraphLaunch(G->exec, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  Work& w = c->work;
  int steps = 0;
  for (int q = 0; q < a.R; ++q) steps = std::max(steps, (int)w.h_ivec[q]);
  g_launches.fetch_add(G->fixed_launches + (long long)steps * G->step_launches);
  for (auto& mk : G->marks) {
    if (mk.step >= steps) continue;
    float t = 0;
    CK(cudaEventElapsedTime(&t, mk.a, mk.b));
    c->prof.graph_ms[mk.cls] += t;
    c->prof.graph_launches[mk.cls] += 1;
    c->prof.bytes[mk.cls] += mk.bytes;
  }
  return steps;
}

// Mean device time per launch of fn (one untimed warm-up launch, then `reps` timed launches).
double time_launch(Ctx* c, const std::function<void()>& fn, int reps = 3) {
  cudaEvent_t a = nullptr, b = nullptr;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  fn();
  CK(cudaEventRecord(a, c->stream));
  for (int i = 0; i < reps; ++i) fn();
  CK(cudaEventRecord(b, c->stream));
  CK(cudaEventSynchronize(b));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  check_launch("launch-shape tuning");
  return ms / reps;
}

// Times every accepted launch shape of the preconditioner apply, the Gram-Schmidt dots and the
// SpMM for one block shape on pseudo-random inputs (frequency 0's operator and inverses) and
// keeps the fastest of each.  Uses the Krylov workspace as scratch.
Tuned autotune(Ctx* c, int R, int wp, int m, bool use_p) {
  const int64_t E = c->topo.n_edge;
  ensure_work(c, R, m, wp);
  Work& w = c->work;
  Tuned t;
  t.R = R;
  t.wp = wp;
  t.m = m;
  t.tc = use_p && c->prec.ready && c->prec.apply_prec == 2 && wp == 1;
  const int64_t vstride = krylov_stride(E, R);
  const size_t es = wp == 0 ? sizeof(double2) : sizeof(float2);
  auto Vp = [&](int i) { return (void*)((unsigned char*)w.V + es * vstride * i); };
  const int nvec = (m + 1) / 2;             // mid-cycle depth of the Gram-Schmidt pass
  const int out = std::min(nvec + 1, m);    // SpMM output vector (inside the m + 1 of the basis)
  for (int i = 0; i <= nvec; ++i) {
    if (wp == 0)
      mwk::fill_pattern_f64((double*)Vp(i), 2 * E * R, 977u * (i + 1), c->stream);
    else
      mwk::fill_pattern_f32((float*)Vp(i), 2 * E * R, 977u * (i + 1), c->stream);
  }
  auto pick = [](const std::vector<std::pair<int, double>>& v) {
    int best = v.front().first;
    double bt = v.front().second;
    for (auto& p : v)
      if (p.second < bt) {
        bt = p.second;
        best = p.first;
      }
    return best;
  };
  for (int th : {kSpmmHaloShape, 128, 256, 512}) {
    if (th == kSpmmHaloShape && !(wp == 1 && spmm_halo_ok(c, R))) continue;
    const double ms = time_launch(c, [&] {
      if (wp == 0)
        mwk::spmm_f64(c->d_row, c->d_col, c->A64[0], (const double2*)Vp(0), (double2*)Vp(out), E, R, c->stream,
                      th);
      else
        spmm32(c, 0, (const float2*)Vp(0), (float2*)Vp(out), R, th);
    });
    t.t[MW_TUNE_SPMM].push_back({th, ms});
  }
  t.sh.spmm_threads = pick(t.t[MW_TUNE_SPMM]);
  if (R >= 16 && R <= 128) {
    for (int st = mwk::kCgsDotsMinStages; st <= mwk::kCgsDotsMaxStages; ++st) {
      const double ms = time_launch(c, [&] {
        if (wp == 0)
          mwk::cgs_dots_f64((const double2*)w.V, vstride, nvec, (const double2*)Vp(nvec), E, R, w.part, w.kerr,
                            c->stream, st);
        else
          mwk::cgs_dots_f32((const float2*)w.V, vstride, nvec, (const float2*)Vp(nvec), E, R, w.part, w.kerr,
                            c->stream, st);
      });
      t.t[MW_TUNE_DOTS].push_back({st, ms});
    }
    t.sh.dots_stages = pick(t.t[MW_TUNE_DOTS]);
    // small coefficients keep the repeatedly updated vector bounded
    mwk::fill_pattern_f64((double*)w.h, 2 * (int64_t)nvec * R, 4099u, c->stream, 1e-3);
    for (int st = mwk::kCgsDotsMinStages; st <= mwk::kCgsDotsMaxStages; ++st) {
      const double ms = time_launch(c, [&] {
        if (wp == 0)
          mwk::cgs_update_f64((const double2*)w.V, vstride, nvec, w.h, (double2*)Vp(nvec), E, R, w.npart, c->stream,
                              w.kerr, st);
        else
          mwk::cgs_update_f32((const float2*)w.V, vstride, nvec, w.h, (float2*)Vp(nvec), E, R, w.npart, c->stream,
                              w.kerr, st);
      });
      t.t[MW_TUNE_UPDATE].push_back({st, ms});
    }
    t.sh.update_stages = pick(t.t[MW_TUNE_UPDATE]);
  }
  if (t.tc) {
    ensure_prec_scratch(c, R);
    for (int st = mwk::tc_min_stages; st <= mwk::tc_max_stages(R); ++st) {
      const double ms = time_launch(c, [&] { apply_prec(c, 0, wp, Vp(0), (unsigned char*)w.Z, R, st); });
      t.t[MW_TUNE_TC].push_back({st, ms});
    }
    t.sh.tc_stages = pick(t.t[MW_TUNE_TC]);
  }
  return t;
}

// Tuned launch shapes for a block shape (default shapes while automatic tuning is off).
Tuned tuned_for(Ctx* c, int R, int wp, int m, bool use_p) {
  if (!c->autotune_on) {
    Tuned d;
    d.R = R;
    d.wp = wp;
    d.m = m;
    return d;
  }
  const bool tc = use_p && c->prec.ready && c->prec.apply_prec == 2 && wp == 1;
  for (auto& t : c->tuned)
    if (t.R == R && t.wp == wp && t.m == m && t.tc == tc) return t;
  c->tuned.push_back(autotune(c, R, wp, m, use_p));
  return c->tuned.back();
}

// Solve A_f X = B for a block of R columns ([E][R] layout, FP64 in and out).
BlockStats solve_block(Ctx* c, int f, int R, const double2* B, double2* X, const mw_solve_opts& o,
                       std::vector<int32_t>& its_out) {
  const int64_t E = c->topo.n_edge;
  const int m = o.restart;
  const int wp = o.mode == MW_MODE_FP64 ? 0 : 1;
  const bool use_p = o.use_precond != 0;
  require(!use_p || c->prec.ready, MW_ESTATE, "preconditioner requested but not set up");
  ensure_work(c, R, m, wp);
  Work& w = c->work;
  cudaStream_t s = c->stream;
  CycleArgs a{f, R, m, wp, use_p, X, E, krylov_stride(E, R), wp == 0 ? sizeof(double2) : sizeof(float2),
              tuned_for(c, R, wp, m, use_p), use_p && c->prec.ready && c->prec.apply_prec == 2 && wp == 1, false};
  a.zb = a.lazy && c->z_bf16;

  CK(cudaMemsetAsync(X, 0, sizeof(double2) * E * R, s));
  if (wp == 1) mwk::split_df(B, w.bdf, E * R, s);
  int nb = mwk::colnorm2_f64(B, E, R, w.npart, s);
  mwk::reduce_cols(w.npart, nb, R, w.bnorm, s);
  mwk::sqrt_inplace(w.bnorm, R, s);
  std::vector<int32_t> its(R, 0);
  BlockStats st;
  const int max_outer = o.mode == MW_MODE_FP64 ? (o.max_it + m - 1) / m + 1 : std::max(1, o.max_outer);
  int total = 0;
  for (int outer = 0; outer < max_outer; ++outer) {
    {
      // the first step starts from X = 0: r = b, no products
      ProfScope ps(c, MW_K_RESIDUAL,
                   outer == 0 ? 24.0 * E * R : (double)c->topo.nnz * 20 + 8.0 * (E + 1) + 3.0 * 16 * E * R);
      nb = outer_residual(c, f, wp, X, B, R, outer == 0);
    }
    CK(cudaMemsetAsync(w.active, 0, sizeof(int32_t), s));
    mwk::start_state(w.npart, nb, R, w.bnorm, o.tol, o.inner_tol, wp == 0, w.rnorm, w.g, w.target, w.done, w.kcol,
                     m, s);
    mwk::count_active(w.done, R, w.active, s);
    check_launch("cycle start");
    st.outer++;
    st.have_relres = true;
    if (read_active(c) == 0 || total >= o.max_it) break;
    st.have_relres = false;
    // a cycle that may run all m steps is replayed from its captured graph
    const int steps = (c->graphs_on && o.max_it - total >= m) ? cycle_graph(c, a) : cycle_eager(c, a, o.max_it - total);
    total += steps;
    st.steps += steps;
    for (int q = 0; q < R; ++q) its[q] += w.h_ivec[q];
  }
  its_out = its;
  if (!st.have_relres) {
    // the loop ended after an update: measure the final residual
    nb = outer_residual(c, f, wp, X, B, R);
    mwk::reduce_cols(w.npart, nb, R, w.rnorm, s);
    mwk::sqrt_inplace(w.rnorm, R, s);
  }
  return st;
}

// True relative residuals of the block after solve_block (w.rnorm / w.bnorm, both sqrt'ed).
void block_relres(Ctx* c, int R, double* rel) {
  Work& w = c->work;
  std::vector<double> a(R), b(R);
  CK(cudaMemcpyAsync(a.data(), w.rnorm, sizeof(double) * R, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(b.data(), w.bnorm, sizeof(double) * R, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int q = 0; q < R; ++q) rel[q] = b[q] > 0 ? a[q] / b[q] : a[q];
}

// final true relative residuals of a block (FP64), into rel[R] on the host
void true_relres(Ctx* c, int f, int R, const double2* B, const double2* X, double* rel) {
  Work& w = c->work;
  cudaStream_t s = c->stream;
  const int64_t E = c->topo.n_edge;
  int nb = mwk::residual_f64(c->d_row, c->d_col, c->A64[f], X, B, w.r, w.npart, E, R, s);
  mwk::reduce_cols(w.npart, nb, R, w.rnorm, s);
  nb = mwk::colnorm2_f64(B, E, R, w.npart, s);
  mwk::reduce_cols(w.npart, nb, R, w.bnorm, s);
  std::vector<double> a(R), b(R);
  CK(cudaMemcpyAsync(a.data(), w.rnorm, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(b.data(), w.bnorm, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int q = 0; q < R; ++q) rel[q] = b[q] > 0 ? std::sqrt(a[q] / b[q]) : std::sqrt(a[q]);
}

mw_solve_opts norm_opts(const mw_solve_opts* o) {
  mw_solve_opts d{};
  d.mode = MW_MODE_FP64;
  d.restart = 50;
  d.batch = 0;
  d.max_it = 5000;
  d.tol = 1e-8;
  d.inner_tol = 1e-2;
  d.max_outer = 20;
  d.use_precond = 1;
  if (o) d = *o;
  require(d.mode == MW_MODE_FP64 || d.mode == MW_MODE_MIXED, MW_EINVAL, "unknown solve mode");
  require(d.restart >= 1 && d.restart <= kMaxRestart, MW_EINVAL, "restart must be in [1, 63]");
  require(d.tol > 0 && d.max_it >= 1, MW_EINVAL, "tol > 0 and max_it >= 1 required");
  if (d.inner_tol <= 0) d.inner_tol = 1e-2;
  if (d.max_outer <= 0) d.max_outer = 20;
  return d;
}

// Solve all frequencies for RHS blocks Bf[f] ([E][ncols]) into Xf[f]; fills stats.
void solve_all(Ctx* c, const mw_solve_opts& o, int ncols, const std::vector<const double2*>& Bf,
               const std::vector<double2*>& Xf, mw_solve_stats* stats) {
  const int64_t E = c->topo.n_edge;
  cudaStream_t s = c->stream;
  const int bsz = (o.batch <= 0 || o.batch > ncols) ? ncols : o.batch;
  require(bsz <= 128, MW_EINVAL, "at most 128 columns per Krylov launch (set batch)");
  {
    // launch shapes are tuned (once per shape) before the solve phase is timed
    const int wp = o.mode == MW_MODE_FP64 ? 0 : 1;
    require(o.use_precond == 0 || c->prec.ready, MW_ESTATE, "preconditioner requested but not set up");
    tuned_for(c, bsz, wp, o.restart, o.use_precond != 0);
    if (ncols % bsz) tuned_for(c, ncols % bsz, wp, o.restart, o.use_precond != 0);
  }
  std::vector<int32_t> its_all(c->n_freq * ncols, 0);
  std::vector<double> rel_all(c->n_freq * ncols, 0.0);
  int outer = 0, steps = 0;
  CK(cudaEventRecord(c->ev0, s));
  for (int f = 0; f < c->n_freq; ++f) {
    for (int c0 = 0; c0 < ncols; c0 += bsz) {
      const int R = std::min(bsz, ncols - c0);
      const double2* B = Bf[f] + c0;
      double2* X = Xf[f] + c0;
      std::vector<int32_t> its;
      if (R == ncols) {
        BlockStats bs = solve_block(c, f, R, B, X, o, its);
        outer += bs.outer;
        steps += bs.steps;
        block_relres(c, R, rel_all.data() + f * ncols + c0);
      } else {
        ensure_work(c, R, o.restart, o.mode == MW_MODE_FP64 ? 0 : 1);
        Work& w = c->work;
        CK(cudaMemcpy2DAsync(w.bblk, sizeof(double2) * R, B, sizeof(double2) * ncols, sizeof(double2) * R, E,
                             cudaMemcpyDeviceToDevice, s));
        // w.x is reused as the block solution
        BlockStats bs = solve_block(c, f, R, w.bblk, w.x, o, its);
        outer += bs.outer;
        steps += bs.steps;
        block_relres(c, R, rel_all.data() + f * ncols + c0);
        CK(cudaMemcpy2DAsync(X, sizeof(double2) * ncols, w.x, sizeof(double2) * R, sizeof(double2) * R, E,
                             cudaMemcpyDeviceToDevice, s));
      }
      for (int q = 0; q < R; ++q) its_all[f * ncols + c0 + q] = its[q];
    }
  }
  CK(cudaEventRecord(c->ev1, s));
  CK(cudaEventSynchronize(c->ev1));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  check_tc_wait(c);
  if (c->prec.ready && c->prec.apply_prec == 5)
    for (auto& L : c->prec.mf.tcl) {
      if (!L.plan.err) continue;
      int32_t e = 0;
      CK(cudaMemcpy(&e, L.plan.err, sizeof(int32_t), cudaMemcpyDeviceToHost));
      if (e != 0) {
        CK(cudaMemsetAsync(L.plan.err, 0, sizeof(int32_t), s));
        throw Fail{MW_ETIMEOUT, "tensor-core sparse sweep: bounded wait ran out (code " + std::to_string(e) + ")"};
      }
    }
  if (c->work.kerr) {
    int32_t e = 0;
    CK(cudaMemcpy(&e, c->work.kerr, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (e != 0) {
      CK(cudaMemsetAsync(c->work.kerr, 0, sizeof(int32_t), s));
      throw Fail{MW_ETIMEOUT, "streaming Gram-Schmidt dots: bounded wait ran out (code " + std::to_string(e) + ")"};
    }
  }
  int nconv = 0;
  double mx = 0;
  for (double r : rel_all) {
    if (r <= o.tol) ++nconv;
    mx = std::max(mx, r);
  }
  if (stats) {
    stats->n_cols = c->n_freq * ncols;
    stats->n_converged = nconv;
    stats->outer_steps = outer;
    stats->arnoldi_steps = steps;
    stats->max_relres = mx;
    stats->solve_ms = ms;
    if (stats->iters) std::memcpy(stats->iters, its_all.data(), sizeof(int32_t) * its_all.size());
    if (stats->relres) std::memcpy(stats->relres, rel_all.data(), sizeof(double) * rel_all.size());
  }
  if (nconv < c->n_freq * ncols)
    throw Fail{MW_ENOCONV, "GMRES: " + std::to_string(c->n_freq * ncols - nconv) + " columns missed tol (max relres " +
                               std::to_string(mx) + ")"};
}

// i beta of a TE10 port: beta = -i sqrt((pi/a)^2 - k0^2 eps_fill) (principal root), so
// i beta = sqrt((pi/a)^2 - k0^2 eps_fill); eps_fill has im <= 0, so the radicand has im >= 0.
double2 port_ibeta(const mw_port& p, double k0) {
  const double kc = mw::kPi / p.a;
  const double zr = kc * kc - k0 * k0 * p.eps_fill[0], zi = -k0 * k0 * p.eps_fill[1];
  const double r = std::hypot(zr, zi);
  return make_double2(std::sqrt(0.5 * (r + zr)), std::sqrt(std::max(0.0, 0.5 * (r - zr))));
}

// Right-hand-side coefficients c_fj of every source for every frequency: -i omega mu0 for a
// dipole, 2 i beta_fj for a port (g = 2 i beta E^TE10).
void upload_source_coefs(Ctx* c) {
  const int ns = c->n_src, nf = c->n_freq;
  const std::vector<double2> old = c->src_coef;
  c->src_coef.assign((size_t)nf * ns, make_double2(0, 0));
  for (int f = 0; f < nf; ++f)
    for (int j = 0; j < ns; ++j) {
      if (c->src_ports) {
        const double2 ib = port_ibeta(c->ports[j], k0_of(c->freqs[f]));
        c->src_coef[(size_t)f * ns + j] = make_double2(2.0 * ib.x, 2.0 * ib.y);
      } else {
        c->src_coef[(size_t)f * ns + j] = make_double2(0.0, -2.0 * mw::kPi * c->freqs[f] * mw::kMu0);
      }
    }
  if (c->d_src_coef && old.size() == c->src_coef.size() &&
      std::memcmp(old.data(), c->src_coef.data(), sizeof(double2) * old.size()) == 0)
    return;  // unchanged: no copy, so a solve loop keeps its buffers and captured graphs
  upload_reuse(c, c->d_src_coef, c->src_coef);
}

void build_source_rhs(Ctx* c, int f, double2* B) {
  mwk::source_rhs(c->d_q_ptr, c->d_q_edge, c->d_q_w, c->d_src_coef + (size_t)f * c->n_src, c->n_src, B,
                  c->topo.n_edge, c->stream);
  check_launch("source rhs");
}

void free_sources(Ctx* c) {
  for (void* q : {(void*)c->d_q_ptr, (void*)c->d_qt_ptr, (void*)c->d_q_edge, (void*)c->d_qt_edge, (void*)c->d_qt_src,
                  (void*)c->d_qt_k, (void*)c->d_q_w, (void*)c->d_q_norm, (void*)c->d_src_coef})
    dfree(c, q);
  c->d_q_ptr = c->d_qt_ptr = nullptr;
  c->d_q_edge = c->d_qt_edge = c->d_qt_src = c->d_qt_k = nullptr;
  c->d_q_w = c->d_q_norm = nullptr;
  c->d_src_coef = nullptr;
  c->n_qt = 0;
  c->q_ptr_h.clear();
  for (auto p : c->Xf) dfree(c, p);
  for (auto p : c->Lf) dfree(c, p);
  for (auto p : c->Bfwd) dfree(c, p);
  for (auto p : c->d_Badj) dfree(c, p);
  c->Xf.clear();
  c->Lf.clear();
  c->Bfwd.clear();
  c->d_Badj.clear();
  c->n_src = 0;
}

// Installs n sources given as CSR (host ptr / edges) with entry values and norms already on
// the device (ownership passes to the context); builds the edge-major transpose.
void install_sources(Ctx* c, int n, bool ports, const std::vector<int64_t>& ptr, const std::vector<int32_t>& edge,
                     double* d_w, double* d_norm) {
  free_sources(c);
  c->n_src = n;
  c->src_ports = ports;
  c->q_ptr_h = ptr;
  c->d_q_ptr = upload(c, ptr.data(), ptr.size());
  c->d_q_edge = upload_vec(c, edge);
  c->d_q_w = d_w;
  c->d_q_norm = d_norm;
  // transpose: pairs (edge, source, entry) sorted by edge, then source
  std::vector<std::array<int32_t, 3>> pr;
  pr.reserve(edge.size());
  for (int j = 0; j < n; ++j)
    for (int64_t k = ptr[j]; k < ptr[j + 1]; ++k) pr.push_back({edge[k], j, (int32_t)k});
  std::sort(pr.begin(), pr.end());
  std::vector<int64_t> tptr(1, 0);
  std::vector<int32_t> tedge, tsrc, tk;
  for (size_t i = 0; i < pr.size(); ++i) {
    if (i == 0 || pr[i][0] != pr[i - 1][0]) {
      if (i) tptr.push_back((int64_t)i);
      tedge.push_back(pr[i][0]);
    }
    tsrc.push_back(pr[i][1]);
    tk.push_back(pr[i][2]);
  }
  if (!pr.empty()) tptr.push_back((int64_t)pr.size());
  c->n_qt = (int64_t)tedge.size();
  c->d_qt_ptr = upload(c, tptr.data(), tptr.size());
  c->d_qt_edge = upload_vec(c, tedge);
  c->d_qt_src = upload_vec(c, tsrc);
  c->d_qt_k = upload_vec(c, tk);
}

// Face-class coefficient table [n_freq][2 + n_port]: i k0 sqrt(eps_bg) (open), 0 (metal),
// i beta_p (port p), uploaded to d_zc.
void upload_face_classes(Ctx* c, double si, double sr) {
  if (c->bface_cls.empty()) return;
  const int nc = 2 + c->n_port;
  c->zc_h.assign((size_t)c->n_freq * nc, make_double2(0, 0));
  for (int f = 0; f < c->n_freq; ++f) {
    const double k0 = k0_of(c->freqs[f]);
    c->zc_h[(size_t)f * nc] = make_double2(-k0 * si, k0 * sr);
    for (int p = 0; p < c->n_port; ++p) c->zc_h[(size_t)f * nc + 2 + p] = port_ibeta(c->ports[p], k0);
  }
  upload_reuse(c, c->d_zc, c->zc_h);
}

// A_f for every frequency from d_eps (Eq. m2 with the boundary classes), plus its FP32 and
// double-float copies.
void reassemble_all(Ctx* c) {
  const int64_t nnz = c->topo.nnz;
  const double* eb = c->eps_bg;
  const double r = std::hypot(eb[0], eb[1]);
  const double sr = std::sqrt(0.5 * (r + eb[0]));
  double si = std::sqrt(std::max(0.0, 0.5 * (r - eb[0])));
  if (eb[1] < 0) si = -si;
  upload_face_classes(c, si, sr);
  const int nc = 2 + c->n_port;
  const int64_t T = c->topo.n_tet, Fb = c->topo.n_bface;
  // pull map and offsets, element matrices and eps read once, FP64 and FP32 values written;
  // the double-float split reads the FP64 values and writes their (hi, lo) pairs (32 B per
  // nonzero); the SpMM plan's blocked copy reads a source index and an FP32 value and writes it
  // (20 B)
  const double rbytes = 8.0 * (nnz + 1) + 4.0 * (36.0 * T + 9.0 * Fb) + (42.0 * 8 + 16) * T + 48.0 * Fb + 24.0 * nnz;
  for (int f = 0; f < c->n_freq; ++f) {
    const double k0 = k0_of(c->freqs[f]);
    ProfScope ps(c, MW_K_REASSEMBLE, rbytes + (32.0 + 20.0) * nnz);
    mwk::reassemble(c->d_cptr, c->d_contrib, nnz, c->d_KM, c->d_Bf, c->d_eps, k0 * k0, -k0 * si, k0 * sr,
                    c->d_bface_cls, c->d_zc ? c->d_zc + (size_t)f * nc : nullptr, c->d_nzmask, c->A64[f], c->A32[f],
                    c->stream);
    mwk::split_df(c->A64[f], c->Adf[f], nnz, c->stream);
    if (c->A32b.size() == c->A32.size() && c->A32b[f]) mwk::spmm_plan_values(c->spmm, c->A32[f], nnz, c->A32b[f], c->stream);
  }
  check_launch("reassemble");
}

void alloc_fields(Ctx* c, std::vector<double2*>& v) {
  const int64_t n = c->topo.n_edge * (int64_t)c->n_src;
  if ((int)v.size() == c->n_freq && !v.empty()) return;
  for (auto p : v) dfree(c, p);
  v.assign(c->n_freq, nullptr);
  for (int f = 0; f < c->n_freq; ++f) v[f] = dalloc<double2>(c, n);
}

void forward(Ctx* c, const mw_solve_opts& o, mw_solve_stats* stats) {
  require(c->has_mesh && c->n_freq > 0, MW_ESTATE, "assemble first");
  require(c->n_src > 0, MW_ESTATE, "set sources first");
  alloc_fields(c, c->Xf);
  alloc_fields(c, c->Bfwd);   // source right-hand sides, kept between evaluations
  upload_source_coefs(c);
  std::vector<const double2*> Bs(c->n_freq);
  for (int f = 0; f < c->n_freq; ++f) {
    build_source_rhs(c, f, c->Bfwd[f]);
    Bs[f] = c->Bfwd[f];
  }
  solve_all(c, o, c->n_src, Bs, c->Xf, stats);
}

void release_prec(Ctx* c) {
  Prec& p = c->prec;
  for (void* q : {(void*)p.dof_ptr, (void*)p.own_ptr, (void*)p.tet_ptr, (void*)p.surf_ptr, (void*)p.dofs,
                  (void*)p.own_local, (void*)p.own_glob, (void*)p.tet_ids, (void*)p.tet_loc, (void*)p.surf_loc,
                  (void*)p.surf_tet, (void*)p.surf_vert, (void*)p.Bsurf, (void*)p.tile_sub, (void*)p.tile_row0,
                  (void*)p.w_off})
    dfree(c, q);
  for (void* q : p.W) dfree(c, q);
  for (void* q : p.mf.allocs) dfree(c, q);
  for (void* q : p.mf.fac) dfree(c, q);
  for (auto& L : p.mf.tcl) {
    for (void* q : L.W) dfree(c, q);
    mwk::tc_plan_free(L.plan, [&](void* q) { dfree(c, q); });
  }
  mwk::tc_plan_free(p.tc, [&](void* q) { dfree(c, q); });
  p = Prec();
  c->tuned.clear();
}

void free_window(Ctx* c);

void release_mesh(Ctx* c) {
  drop_graphs(c);
  release_prec(c);
  free_work(c);
  for (auto p : c->Xf) dfree(c, p);
  for (auto p : c->Lf) dfree(c, p);
  for (auto p : c->Bfwd) dfree(c, p);
  c->Xf.clear();
  c->Lf.clear();
  c->Bfwd.clear();
  for (auto p : c->A64) dfree(c, p);
  for (auto p : c->A32) dfree(c, p);
  for (auto p : c->A32b) dfree(c, p);
  for (auto p : c->Adf) dfree(c, p);
  c->A64.clear();
  c->A32.clear();
  c->A32b.clear();
  c->Adf.clear();
  for (const void* q : {(const void*)c->spmm.blk_row, (const void*)c->spmm.blk_halo, (const void*)c->spmm.halo,
                        (const void*)c->spmm.rows, (const void*)c->spmm.rptr, (const void*)c->spmm.lcol,
                        (const void*)c->spmm.src})
    dfree(c, const_cast<void*>(q));
  c->spmm = mwk::SpmmDev();
  for (void* q : {(void*)c->d_xyz, (void*)c->d_tets, (void*)c->d_col, (void*)c->d_contrib, (void*)c->d_bface_vert,
                  (void*)c->d_tet_edge, (void*)c->d_tet_nb, (void*)c->d_sign, (void*)c->d_row, (void*)c->d_cptr,
                  (void*)c->d_KM, (void*)c->d_vol, (void*)c->d_Bf, (void*)c->d_tikw, (void*)c->d_eps,
                  (void*)c->d_bface_cls, (void*)c->d_metal, (void*)c->d_nzmask, (void*)c->d_zc, (void*)c->d_B,
                  (void*)c->d_red, (void*)c->d_S,
                  (void*)c->d_C, (void*)c->d_So, (void*)c->d_Se, (void*)c->d_J, (void*)c->d_grad, (void*)c->d_gR})
    dfree(c, q);
  for (auto p : c->d_Badj) dfree(c, p);
  c->d_Badj.clear();
  free_window(c);
  dfree(c, c->d_D);
  c->d_D = nullptr;
  c->d_S = c->d_C = c->d_So = c->d_Se = nullptr;
  c->d_J = c->d_grad = c->d_gR = nullptr;
  c->d_xyz = nullptr;
  c->d_tets = c->d_col = c->d_contrib = c->d_bface_vert = c->d_tet_edge = c->d_tet_nb = nullptr;
  c->d_sign = nullptr;
  c->d_row = c->d_cptr = nullptr;
  c->d_KM = c->d_vol = c->d_Bf = c->d_tikw = c->d_eps = nullptr;
  c->d_bface_cls = nullptr;
  c->d_metal = c->d_nzmask = nullptr;
  c->d_zc = nullptr;
  free_sources(c);
  c->src_edge.clear();
  c->src_sign.clear();
  c->src_ports = false;
  c->n_port = 0;
  c->ports.clear();
  c->bface_cls.clear();
  c->metal.clear();
  c->zc_h.clear();
  c->d_B = nullptr;
  c->d_red = nullptr;
  c->has_mesh = false;
  c->n_freq = 0;
}

void free_window(Ctx* c) {
  for (auto* v : {&c->Xw, &c->Lw, &c->Bw, &c->Bwa}) {
    for (auto p : *v) dfree(c, p);
    v->clear();
  }
  dfree(c, c->d_Sp);
  c->d_Sp = nullptr;
  c->win_j0 = c->win_nl = c->win_nf = c->win_ns = 0;
}

// Drops the assembled matrices, the preconditioner and every stored field (the boundary
// changed: assemble again).
void drop_assembly(Ctx* c) {
  free_window(c);
  drop_graphs(c);
  release_prec(c);
  for (auto p : c->A64) dfree(c, p);
  for (auto p : c->A32) dfree(c, p);
  for (auto p : c->A32b) dfree(c, p);
  for (auto p : c->Adf) dfree(c, p);
  c->A64.clear();
  c->A32.clear();
  c->A32b.clear();
  c->Adf.clear();
  for (auto p : c->Xf) dfree(c, p);
  for (auto p : c->Lf) dfree(c, p);
  for (auto p : c->Bfwd) dfree(c, p);
  for (auto p : c->d_Badj) dfree(c, p);
  c->Xf.clear();
  c->Lf.clear();
  c->Bfwd.clear();
  c->d_Badj.clear();
  c->n_freq = 0;
}

// Boundary face with sorted vertices (a, b, c): index into bface_vert (sorted triples), or -1.
int64_t find_bface(const mw::Topology& t, int32_t a, int32_t b, int32_t cc) {
  int64_t lo = 0, hi = t.n_bface;
  while (lo < hi) {
    const int64_t mid = (lo + hi) / 2;
    const int32_t* q = t.bface_vert.data() + 3 * mid;
    const bool less = q[0] != a ? q[0] < a : (q[1] != b ? q[1] < b : q[2] < cc);
    if (less)
      lo = mid + 1;
    else
      hi = mid;
  }
  if (lo < t.n_bface) {
    const int32_t* q = t.bface_vert.data() + 3 * lo;
    if (q[0] == a && q[1] == b && q[2] == cc) return lo;
  }
  return -1;
}

// Edge (lo, hi), lo < hi: its id (the rank of the pair in lexicographic order), or -1.
int64_t find_edge_id(const mw::Topology& t, int32_t a, int32_t b) {
  int64_t lo = 0, hi = t.n_edge;
  while (lo < hi) {
    const int64_t mid = (lo + hi) / 2;
    const int32_t* q = t.edge_vert.data() + 2 * mid;
    if (q[0] < a || (q[0] == a && q[1] < b))
      lo = mid + 1;
    else
      hi = mid;
  }
  if (lo < t.n_edge && t.edge_vert[2 * lo] == a && t.edge_vert[2 * lo + 1] == b) return lo;
  return -1;
}

// Gauss-Legendre nodes and weights mapped to [0, 1]: Newton's method on P_n from the
// three-term recurrence (n P_n = (2n - 1) z P_{n-1} - (n - 1) P_{n-2}).
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(mw::kPi * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) <= 1e-16) break;
    }
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);  // (2 / ((1 - z^2) P_n'^2)) / 2
  }
}

constexpr int kPortQuad = 10;  // collapsed Gauss-Legendre points per direction on port faces

}  // namespace mwimpl

using namespace mwimpl;

// =======================================================================================
// C ABI
// =======================================================================================
struct mw_ctx : Ctx {};

extern "C" {

mw_status mw_create(mw_ctx** out, int device, void* stream) {
  if (!out) return MW_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return MW_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return MW_ECUDA;
  std::unique_ptr<mw_ctx> c(new mw_ctx());
  c->device = device;
  c->stream = (cudaStream_t)stream;
  if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) return MW_ECUDA;
  *out = c.release();
  return MW_OK;
}

void mw_destroy(mw_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  release_mesh(c);
  for (auto& kv : c->allocs) cudaFree(kv.first);
  if (c->cap_s) cudaStreamDestroy(c->cap_s);
  if (c->body_s) cudaStreamDestroy(c->body_s);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  delete c;
}

const char* mw_last_error(const mw_ctx* c) { return c ? c->err.c_str() : "null context"; }

mw_status mw_set_memory_cap(mw_ctx* c, int64_t bytes) {
  return guard(c, [&] {
    require(bytes >= 0, MW_EINVAL, "cap must be >= 0");
    c->mem_cap = bytes;
  });
}

mw_status mw_set_graphs(mw_ctx* c, int32_t enable) {
  return guard(c, [&] {
    c->graphs_on = enable != 0;
    if (!c->graphs_on) drop_graphs(c);
  });
}

mw_status mw_set_autotune(mw_ctx* c, int32_t enable) {
  return guard(c, [&] {
    c->autotune_on = enable != 0;
    if (!c->autotune_on) c->tuned.clear();
  });
}

mw_status mw_set_launch_shapes(mw_ctx* c, int32_t n_cols, int32_t mode, int32_t restart,
                               const mw_launch_shapes* shapes) {
  return guard(c, [&] {
    require(shapes != nullptr, MW_EINVAL, "null shapes");
    require(n_cols >= 1 && n_cols <= 128, MW_EINVAL, "n_cols must be in 1..128");
    require(mode == MW_MODE_FP64 || mode == MW_MODE_MIXED, MW_EINVAL, "bad mode");
    require(restart >= 1 && restart <= kMaxRestart, MW_EINVAL, "restart must be in 1..63");
    const mw_launch_shapes& q = *shapes;
    require(q.tc_stages == 0 || (q.tc_stages >= mwk::tc_min_stages && q.tc_stages <= mwk::tc_max_stages(n_cols)),
            MW_EINVAL, "tc_stages outside the accepted range for this block width");
    for (int v : {q.dots_stages, q.update_stages})
      require(v == 0 || (v >= mwk::kCgsDotsMinStages && v <= mwk::kCgsDotsMaxStages), MW_EINVAL,
              "dots_stages and update_stages must be 0 or 2..6");
    require(q.spmm_threads == 0 || q.spmm_threads == kSpmmHaloShape || q.spmm_threads == 128 ||
                q.spmm_threads == 256 || q.spmm_threads == 512,
            MW_EINVAL, "spmm_threads must be 0, 1, 128, 256 or 512");
    const int wp = mode == MW_MODE_FP64 ? 0 : 1;
    Tuned t;
    t.R = n_cols;
    t.wp = wp;
    t.m = restart;
    t.tc = c->prec.ready && c->prec.apply_prec == 2 && wp == 1;
    t.sh = q;
    if (t.sh.spmm_threads == 0) t.sh.spmm_threads = 256;
    for (auto& u : c->tuned)
      if (u.R == t.R && u.wp == t.wp && u.m == t.m && u.tc == t.tc) {
        u = t;
        return;
      }
    c->tuned.push_back(t);
  });
}

mw_status mw_autotune(mw_ctx* c, int32_t n_cols, int32_t mode, int32_t restart, mw_tune_report* out) {
  return guard(c, [&] {
    require(c->has_mesh && c->n_freq > 0, MW_ESTATE, "assemble before tuning");
    require(n_cols >= 1 && n_cols <= 128, MW_EINVAL, "n_cols must be in 1..128");
    require(mode == MW_MODE_FP64 || mode == MW_MODE_MIXED, MW_EINVAL, "bad mode");
    require(restart >= 1 && restart <= kMaxRestart, MW_EINVAL, "restart must be in 1..63");
    const int wp = mode == MW_MODE_FP64 ? 0 : 1;
    Tuned t = autotune(c, n_cols, wp, restart, c->prec.ready);
    if (c->autotune_on) {
      bool put = false;
      for (auto& u : c->tuned)
        if (u.R == t.R && u.wp == t.wp && u.m == t.m && u.tc == t.tc) {
          u = t;
          put = true;
        }
      if (!put) c->tuned.push_back(t);
    }
    if (out) {
      *out = mw_tune_report{};
      out->n_cols = n_cols;
      out->mode = mode;
      out->restart = restart;
      out->chosen = t.sh;
      if (t.t[MW_TUNE_TC].empty()) out->chosen.tc_stages = 0;
      if (t.t[MW_TUNE_DOTS].empty()) out->chosen.dots_stages = 0;
      if (t.t[MW_TUNE_UPDATE].empty()) out->chosen.update_stages = 0;
      for (int k = 0; k < MW_TUNE_NKERNEL; ++k) {
        out->n_cand[k] = (int32_t)std::min<size_t>(t.t[k].size(), 8);
        for (int i = 0; i < out->n_cand[k]; ++i) {
          out->cand[k][i] = t.t[k][i].first;
          out->ms[k][i] = t.t[k][i].second;
        }
      }
    }
  });
}

mw_status mw_set_mesh(mw_ctx* c, int64_t n_vert, const double* xyz, int64_t n_tet, const int32_t* tv,
                      mw_mesh_info* out) {
  return guard(c, [&] {
    require(xyz && tv, MW_EINVAL, "null mesh arrays");
    release_mesh(c);
    Error err{MW_OK, ""};
    if (!mw::build_topology(n_vert, n_tet, tv, c->topo, err)) throw Fail{err.code, err.msg};
    for (int64_t i = 0; i < 3 * n_vert; ++i) require(std::isfinite(xyz[i]), MW_EINVAL, "non-finite vertex coordinate");
    c->xyz.assign(xyz, xyz + 3 * n_vert);
    mw::Topology& t = c->topo;
    c->d_xyz = upload(c, xyz, 3 * n_vert);
    c->d_tets = upload(c, t.tets.data(), t.tets.size());
    c->d_sign = upload(c, t.tet_sign.data(), t.tet_sign.size());
    c->d_tet_edge = upload(c, t.tet_edge.data(), t.tet_edge.size());
    c->d_row = upload(c, t.row_ptr.data(), t.row_ptr.size());
    c->d_col = upload(c, t.col_idx.data(), t.col_idx.size());
    c->d_cptr = upload(c, t.contrib_ptr.data(), t.contrib_ptr.size());
    c->d_contrib = upload(c, t.contrib.data(), t.contrib.size());
    c->d_bface_vert = upload(c, t.bface_vert.data(), t.bface_vert.size());
    c->d_tet_nb = upload(c, t.tet_nb.data(), t.tet_nb.size());
    {
      mw::SpmmPlan sp;
      if (!mw::build_spmm_plan(t, xyz, mwk::kHaloMax, sp, err, mwk::kHaloRows, mwk::kHaloNnz))
        throw Fail{err.code, err.msg};
      c->spmm.n_block = sp.n_block;
      c->spmm.halo_max = mwk::kHaloMax;
      c->spmm.blk_row = upload(c, sp.blk_row.data(), sp.blk_row.size());
      c->spmm.blk_halo = upload(c, sp.blk_halo.data(), sp.blk_halo.size());
      c->spmm.halo = upload(c, sp.halo.data(), sp.halo.size());
      c->spmm.rows = upload(c, sp.rows.data(), sp.rows.size());
      c->spmm.rptr = upload(c, sp.rptr.data(), sp.rptr.size());
      c->spmm.lcol = upload(c, sp.lcol.data(), sp.lcol.size());
      c->spmm.src = upload(c, sp.src.data(), sp.src.size());
    }
    c->d_KM = dalloc<double>(c, 42 * n_tet);
    c->d_vol = dalloc<double>(c, n_tet);
    c->d_Bf = dalloc<double>(c, 6 * std::max<int64_t>(t.n_bface, 1));
    c->d_tikw = dalloc<double>(c, 4 * n_tet);
    c->d_red = dalloc<double>(c, 4096);
    mwk::elem_geom(c->d_xyz, c->d_tets, c->d_sign, n_tet, c->d_KM, c->d_vol, c->stream);
    mwk::face_geom(c->d_xyz, c->d_bface_vert, t.n_bface, c->d_Bf, c->stream);
    mwk::tikhonov_weights(c->d_xyz, c->d_tets, c->d_tet_nb, n_tet, c->d_tikw, c->stream);
    check_launch("element geometry");
    // reject degenerate tets
    std::vector<double> vol(n_tet);
    CK(cudaMemcpyAsync(vol.data(), c->d_vol, sizeof(double) * n_tet, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int64_t e = 0; e < n_tet; ++e) require(vol[e] > 0 && std::isfinite(vol[e]), MW_EINVAL, "degenerate tet");
    c->has_mesh = true;
    if (out) *out = {t.n_vert, t.n_tet, t.n_edge, t.n_face, t.n_bface, t.nnz};
  });
}

mw_status mw_get_topology(mw_ctx* c, int32_t* edge_vert, int32_t* tet_edge, int8_t* tet_sign, int64_t* row_ptr,
                          int32_t* col_idx) {
  return guard(c, [&] {
    require(c->has_mesh, MW_ESTATE, "no mesh");
    const mw::Topology& t = c->topo;
    if (edge_vert) std::memcpy(edge_vert, t.edge_vert.data(), sizeof(int32_t) * t.edge_vert.size());
    if (tet_edge) std::memcpy(tet_edge, t.tet_edge.data(), sizeof(int32_t) * t.tet_edge.size());
    if (tet_sign) std::memcpy(tet_sign, t.tet_sign.data(), t.tet_sign.size());
    if (row_ptr) std::memcpy(row_ptr, t.row_ptr.data(), sizeof(int64_t) * t.row_ptr.size());
    if (col_idx) std::memcpy(col_idx, t.col_idx.data(), sizeof(int32_t) * t.col_idx.size());
  });
}

mw_status mw_get_element_matrices(mw_ctx* c, double* K, double* M, double* vol) {
  return guard(c, [&] {
    require(c->has_mesh, MW_ESTATE, "no mesh");
    const int64_t T = c->topo.n_tet;
    std::vector<double> km(42 * T);
    CK(cudaMemcpyAsync(km.data(), c->d_KM, sizeof(double) * km.size(), cudaMemcpyDeviceToHost, c->stream));
    if (vol) CK(cudaMemcpyAsync(vol, c->d_vol, sizeof(double) * T, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int64_t e = 0; e < T; ++e)
      for (int m = 0; m < 6; ++m)
        for (int n = 0; n < 6; ++n) {
          if (K) K[36 * e + 6 * m + n] = km[42 * e + mw::packed6(m, n)];
          if (M) M[36 * e + 6 * m + n] = km[42 * e + 21 + mw::packed6(m, n)];
        }
  });
}

mw_status mw_assemble(mw_ctx* c, int32_t n_freq, const double* freq_hz, const double* eps_r, const double* eps_bg) {
  return guard(c, [&] {
    require(c->has_mesh, MW_ESTATE, "set the mesh first");
    require(n_freq >= 1 && n_freq <= 64 && freq_hz && eps_r && eps_bg, MW_EINVAL, "bad assemble arguments");
    const int64_t T = c->topo.n_tet, nnz = c->topo.nnz;
    for (int f = 0; f < n_freq; ++f) require(freq_hz[f] > 0 && std::isfinite(freq_hz[f]), MW_EINVAL, "bad frequency");
    for (int64_t i = 0; i < 2 * T; ++i) require(std::isfinite(eps_r[i]), MW_EINVAL, "non-finite permittivity");
    require(std::isfinite(eps_bg[0]) && std::isfinite(eps_bg[1]), MW_EINVAL, "non-finite background permittivity");
    if (n_freq != c->n_freq) {
      for (auto p : c->A64) dfree(c, p);
      for (auto p : c->A32) dfree(c, p);
      for (auto p : c->A32b) dfree(c, p);
      for (auto p : c->Adf) dfree(c, p);
      c->A64.assign(n_freq, nullptr);
      c->A32.assign(n_freq, nullptr);
      c->A32b.assign(n_freq, nullptr);
      c->Adf.assign(n_freq, nullptr);
      for (int f = 0; f < n_freq; ++f) {
        c->A64[f] = dalloc<double2>(c, nnz);
        c->A32[f] = dalloc<float2>(c, nnz);
        c->A32b[f] = dalloc<float2>(c, nnz);
        c->Adf[f] = dalloc<float4>(c, nnz);
      }
      for (auto p : c->Xf) dfree(c, p);
      for (auto p : c->Lf) dfree(c, p);
      for (auto p : c->Bfwd) dfree(c, p);
      c->Xf.clear();
      c->Lf.clear();
      c->Bfwd.clear();
      if (c->prec.ready && (int)c->prec.W.size() != n_freq) release_prec(c);
    }
    c->n_freq = n_freq;
    c->freqs.assign(freq_hz, freq_hz + n_freq);
    c->eps_bg[0] = eps_bg[0];
    c->eps_bg[1] = eps_bg[1];
    if (!c->d_eps) c->d_eps = dalloc<double>(c, 2 * T);
    CK(cudaMemcpyAsync(c->d_eps, eps_r, sizeof(double) * 2 * T, cudaMemcpyHostToDevice, c->stream));
    reassemble_all(c);
  });
}

mw_status mw_get_matrix(mw_ctx* c, int32_t f, double* values) {
  return guard(c, [&] {
    require(f >= 0 && f < c->n_freq && values, MW_EINVAL, "bad frequency index or null output");
    CK(cudaMemcpyAsync(values, c->A64[f], sizeof(double2) * c->topo.nnz, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  });
}

mw_status mw_apply_matrix(mw_ctx* c, int32_t f, int32_t prec, const void* x, void* y, int32_t n_cols) {
  return guard(c, [&] {
    require(f >= 0 && f < c->n_freq && x && y && n_cols >= 1 && n_cols <= 128, MW_EINVAL, "bad apply_matrix args");
    if (prec == MW_PREC_FP64)
      mwk::spmm_f64(c->d_row, c->d_col, c->A64[f], (const double2*)x, (double2*)y, c->topo.n_edge, n_cols, c->stream);
    else if (prec == MW_PREC_FP32)
      mwk::spmm_f32(c->d_row, c->d_col, c->A32[f], (const float2*)x, (float2*)y, c->topo.n_edge, n_cols, c->stream);
    else if (prec == 4) {
      require(spmm_halo_ok(c, n_cols) && ((uintptr_t)x & 15) == 0, MW_EINVAL,
              "the halo-tiled SpMM takes an even column count up to 128 and a 16-byte aligned x");
      require(mwk::spmm_halo_f32(c->spmm, c->A32b[f], (const float2*)x, (float2*)y, n_cols, c->stream), MW_EINVAL,
              "halo-tiled SpMM: unsupported shape");
    }
    else if (prec == 5)
      mwk::spmm_f32_bx(c->d_row, c->d_col, c->A32[f], x, (float2*)y, c->topo.n_edge, n_cols, c->stream);
    else if (prec == 3) {
      const int64_t n = c->topo.n_edge * (int64_t)n_cols;
      float4* xd = dalloc<float4>(c, n);
      double* part = dalloc<double>(c, (size_t)152 * 4 * n_cols);
      mwk::split_df((const double2*)x, xd, n, c->stream);
      mwk::residual_df(c->d_row, c->d_col, c->Adf[f], xd, nullptr, (double2*)y, part, c->topo.n_edge, n_cols,
                       c->stream);
      CK(cudaStreamSynchronize(c->stream));
      dfree(c, xd);
      dfree(c, part);
    } else
      throw Fail{MW_EINVAL, "apply_matrix precision must be FP64 (0), FP32 (1) or double-float (3)"};
    check_launch("spmm");
  });
}

mw_status mw_set_sources(mw_ctx* c, int32_t n_src, const double* pos, const double* dir, int32_t* edge_out,
                         int8_t* sign_out) {
  return guard(c, [&] {
    require(c->has_mesh, MW_ESTATE, "set the mesh first");
    require(n_src >= 1 && n_src <= 4096 && pos && dir, MW_EINVAL, "bad source arguments");
    const mw::Topology& t = c->topo;
    std::vector<int32_t> cand;
    for (int64_t e = 0; e < t.n_edge; ++e) {
      const double* a = &c->xyz[3 * (int64_t)t.edge_vert[2 * e]];
      const double* b = &c->xyz[3 * (int64_t)t.edge_vert[2 * e + 1]];
      const double dx = b[0] - a[0], dy = b[1] - a[1], dz = b[2] - a[2];
      if (dz != 0 && std::fabs(dx) <= 1e-9 * std::fabs(dz) && std::fabs(dy) <= 1e-9 * std::fabs(dz))
        cand.push_back((int32_t)e);
    }
    require(!cand.empty(), MW_EINVAL, "mesh has no z-directed edge");
    c->src_edge.assign(n_src, 0);
    c->src_sign.assign(n_src, 1);
    for (int j = 0; j < n_src; ++j) {
      require(dir[3 * j] == 0 && dir[3 * j + 1] == 0 && dir[3 * j + 2] != 0, MW_EINVAL, "only z-directed dipoles");
      double best = INFINITY;
      int32_t be = -1;
      for (int32_t e : cand) {
        const double* a = &c->xyz[3 * (int64_t)t.edge_vert[2 * (int64_t)e]];
        const double* b = &c->xyz[3 * (int64_t)t.edge_vert[2 * (int64_t)e + 1]];
        double d2 = 0;
        for (int k = 0; k < 3; ++k) {
          const double mid = 0.5 * (a[k] + b[k]);
          const double d = mid - pos[3 * j + k];
          d2 = d2 + d * d;
        }
        if (d2 < best) {
          best = d2;
          be = e;
        }
      }
      const double* a = &c->xyz[3 * (int64_t)t.edge_vert[2 * (int64_t)be]];
      const double* b = &c->xyz[3 * (int64_t)t.edge_vert[2 * (int64_t)be + 1]];
      c->src_edge[j] = be;
      c->src_sign[j] = ((b[2] - a[2]) * dir[3 * j + 2] > 0) ? 1 : -1;
    }
    // one-entry source vectors w_j = s_j e_edge(j), norms 1
    std::vector<int64_t> ptr(n_src + 1);
    std::vector<double> w(n_src), nrm(n_src, 1.0);
    for (int j = 0; j <= n_src; ++j) ptr[j] = j;
    for (int j = 0; j < n_src; ++j) w[j] = (double)c->src_sign[j];
    double* d_w = upload(c, w.data(), w.size());
    double* d_n = nullptr;
    try {
      d_n = upload(c, nrm.data(), nrm.size());
      install_sources(c, n_src, false, ptr, c->src_edge, d_w, d_n);
    } catch (...) {
      if (c->d_q_w != d_w) dfree(c, d_w);
      if (c->d_q_norm != d_n) dfree(c, d_n);
      throw;
    }
    if (edge_out) std::memcpy(edge_out, c->src_edge.data(), sizeof(int32_t) * n_src);
    if (sign_out) std::memcpy(sign_out, c->src_sign.data(), n_src);
  });
}

mw_status mw_set_ports(mw_ctx* c, int32_t n_port, const mw_port* ports, int64_t n_face, const int32_t* face_vert,
                       const int32_t* face_label) {
  return guard(c, [&] {
    require(c->has_mesh, MW_ESTATE, "set the mesh first");
    require(n_port >= 0 && n_port <= 4096 && n_face >= 0 && (n_port == 0 || ports) &&
                (n_face == 0 || (face_vert && face_label)),
            MW_EINVAL, "bad port arguments");
    const mw::Topology& t = c->topo;
    for (int p = 0; p < n_port; ++p) {
      const mw_port& q = ports[p];
      bool fin = std::isfinite(q.a) && std::isfinite(q.eps_fill[0]) && std::isfinite(q.eps_fill[1]);
      for (int k = 0; k < 3; ++k) fin = fin && std::isfinite(q.origin[k]) && std::isfinite(q.u[k]) && std::isfinite(q.v[k]);
      require(fin, MW_EINVAL, "non-finite port descriptor");
      require(q.a > 0, MW_EINVAL, "port width a must be > 0");
      require(q.eps_fill[1] <= 0, MW_EINVAL, "port filling must be passive (Im eps_fill <= 0)");
      const double uu = q.u[0] * q.u[0] + q.u[1] * q.u[1] + q.u[2] * q.u[2];
      const double vv = q.v[0] * q.v[0] + q.v[1] * q.v[1] + q.v[2] * q.v[2];
      const double uv = q.u[0] * q.v[0] + q.u[1] * q.v[1] + q.u[2] * q.v[2];
      require(std::fabs(uu - 1) <= 1e-9 && std::fabs(vv - 1) <= 1e-9 && std::fabs(uv) <= 1e-9, MW_EINVAL,
              "port directions u, v must be orthonormal");
    }
    // vertex -> tets, to check that a listed inner face is a face of the mesh
    const int64_t V = t.n_vert, T = t.n_tet, E = t.n_edge;
    std::vector<int64_t> vtp(V + 1, 0);
    for (int64_t i = 0; i < 4 * T; ++i) vtp[t.tets[i] + 1]++;
    for (int64_t v = 0; v < V; ++v) vtp[v + 1] += vtp[v];
    std::vector<int32_t> vt(4 * T);
    {
      std::vector<int64_t> fill(vtp.begin(), vtp.end() - 1);
      for (int64_t i = 0; i < 4 * T; ++i) vt[fill[t.tets[i]]++] = (int32_t)(i / 4);
    }
    std::vector<int32_t> cls(t.n_bface, 0);
    std::vector<uint8_t> set(t.n_bface, 0), metal(E, 0);
    bool any_metal = false;
    for (int64_t k = 0; k < n_face; ++k) {
      int32_t a = face_vert[3 * k], b = face_vert[3 * k + 1], d = face_vert[3 * k + 2];
      require(a >= 0 && a < V && b >= 0 && b < V && d >= 0 && d < V, MW_EINVAL, "face vertex out of range");
      if (a > b) std::swap(a, b);
      if (b > d) std::swap(b, d);
      if (a > b) std::swap(a, b);
      require(a < b && b < d, MW_EINVAL, "face with repeated vertices");
      const int32_t lab = face_label[k];
      require(lab >= -1 && lab < n_port, MW_EINVAL, "face label out of range");
      const int64_t bf = find_bface(t, a, b, d);
      if (bf < 0) {
        require(lab == -1, MW_EINVAL, "a port face is not a boundary face");
        bool found = false;
        for (int64_t q = vtp[a]; q < vtp[a + 1] && !found; ++q) {
          const int32_t* tv = &t.tets[4 * (int64_t)vt[q]];
          bool hb = false, hd = false;
          for (int m = 0; m < 4; ++m) {
            hb = hb || tv[m] == b;
            hd = hd || tv[m] == d;
          }
          found = hb && hd;
        }
        require(found, MW_EINVAL, "listed face is not a face of the mesh");
      } else {
        const int32_t cv = lab == -1 ? 1 : 2 + lab;
        require(!set[bf] || cls[bf] == cv, MW_EINVAL, "face listed twice with different labels");
        set[bf] = 1;
        cls[bf] = cv;
      }
      if (lab == -1) {
        any_metal = true;
        metal[find_edge_id(t, a, b)] = 1;
        metal[find_edge_id(t, a, d)] = 1;
        metal[find_edge_id(t, b, d)] = 1;
      }
    }
    // faces of each port, in boundary-face order; entries (port, edge) with their face moments
    std::vector<int64_t> fptr(n_port + 1, 0);
    for (int64_t f = 0; f < t.n_bface; ++f)
      if (cls[f] >= 2) fptr[cls[f] - 2 + 1]++;
    for (int p = 0; p < n_port; ++p) {
      require(fptr[p + 1] > 0, MW_EINVAL, "a port has no face");
      fptr[p + 1] += fptr[p];
    }
    const int64_t Fp = fptr[n_port];
    std::vector<int32_t> pfv(3 * Fp), pport(Fp);
    std::vector<int64_t> pbf(Fp);
    {
      std::vector<int64_t> fill(fptr.begin(), fptr.end() - 1);
      for (int64_t f = 0; f < t.n_bface; ++f)
        if (cls[f] >= 2) {
          const int64_t i = fill[cls[f] - 2]++;
          pbf[i] = f;
          pport[i] = cls[f] - 2;
          for (int m = 0; m < 3; ++m) pfv[3 * i + m] = t.bface_vert[3 * f + m];
        }
    }
    std::vector<int64_t> qptr(1, 0), eptr(1, 0);
    std::vector<int32_t> qedge, econ;
    for (int p = 0; p < n_port; ++p) {
      std::vector<std::pair<int32_t, int32_t>> pr;  // (edge, moment index) in face order
      for (int64_t i = fptr[p]; i < fptr[p + 1]; ++i)
        for (int m = 0; m < 3; ++m) pr.push_back({t.bface_edge[3 * pbf[i] + m], (int32_t)(3 * i + m)});
      std::stable_sort(pr.begin(), pr.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
      for (size_t i = 0; i < pr.size(); ++i) {
        if (metal[pr[i].first]) continue;
        if (qedge.empty() || (int64_t)qedge.size() == qptr.back() || qedge.back() != pr[i].first) {
          qedge.push_back(pr[i].first);
          eptr.push_back(eptr.back());
        }
        econ.push_back(pr[i].second);
        eptr.back()++;
      }
      qptr.push_back((int64_t)qedge.size());
    }
    // identity rows and columns of metal edges
    std::vector<uint8_t> nzm;
    if (any_metal) {
      nzm.assign(t.nnz, 0);
      for (int64_t r = 0; r < E; ++r)
        for (int64_t k = t.row_ptr[r]; k < t.row_ptr[r + 1]; ++k) {
          const int32_t col = t.col_idx[k];
          if (metal[r] || metal[col]) nzm[k] = col == r ? 2 : 1;
        }
    }
    // commit: the boundary changed, so everything assembled from it goes
    drop_assembly(c);
    for (void* q : {(void*)c->d_bface_cls, (void*)c->d_metal, (void*)c->d_nzmask, (void*)c->d_zc}) dfree(c, q);
    c->d_bface_cls = nullptr;
    c->d_metal = c->d_nzmask = nullptr;
    c->d_zc = nullptr;
    c->n_port = n_port;
    c->ports.assign(ports, ports + n_port);
    const bool any_class = n_face > 0;
    c->bface_cls = any_class ? cls : std::vector<int32_t>();
    c->metal = any_metal ? metal : std::vector<uint8_t>();
    if (any_class) c->d_bface_cls = upload(c, cls.data(), cls.size());
    if (any_metal) {
      c->d_metal = upload(c, metal.data(), metal.size());
      c->d_nzmask = upload(c, nzm.data(), nzm.size());
    }
    if (c->src_ports) free_sources(c);  // the previous ports' sources are stale
    if (n_port == 0) return;
    // port load vectors and norms on the device
    std::vector<double> pdesc(10 * n_port), gx, gw;
    for (int p = 0; p < n_port; ++p) {
      for (int k = 0; k < 3; ++k) {
        pdesc[10 * p + k] = ports[p].origin[k];
        pdesc[10 * p + 3 + k] = ports[p].u[k];
        pdesc[10 * p + 6 + k] = ports[p].v[k];
      }
      pdesc[10 * p + 9] = ports[p].a;
    }
    gauss_legendre01(kPortQuad, gx, gw);
    std::vector<void*> tmp;
    double* d_w = nullptr;
    double* d_n = nullptr;
    try {
      int32_t* d_fv = upload(c, pfv.data(), pfv.size());
      tmp.push_back(d_fv);
      int32_t* d_fp = upload(c, pport.data(), pport.size());
      tmp.push_back(d_fp);
      double* d_pd = upload(c, pdesc.data(), pdesc.size());
      tmp.push_back(d_pd);
      double* d_gx = upload(c, gx.data(), gx.size());
      tmp.push_back(d_gx);
      double* d_gw = upload(c, gw.data(), gw.size());
      tmp.push_back(d_gw);
      double* d_mom = dalloc<double>(c, 3 * Fp);
      tmp.push_back(d_mom);
      double* d_nrm = dalloc<double>(c, Fp);
      tmp.push_back(d_nrm);
      int64_t* d_eptr = upload(c, eptr.data(), eptr.size());
      tmp.push_back(d_eptr);
      int32_t* d_econ = upload_vec(c, econ);
      tmp.push_back(d_econ);
      int64_t* d_fptr = upload(c, fptr.data(), fptr.size());
      tmp.push_back(d_fptr);
      d_w = dalloc<double>(c, std::max<size_t>(qedge.size(), 1));
      d_n = dalloc<double>(c, n_port);
      mwk::port_face_moments(c->d_xyz, d_fv, d_fp, Fp, d_pd, d_gx, d_gw, kPortQuad, d_mom, d_nrm, c->stream);
      mwk::port_accumulate(d_eptr, d_econ, (int64_t)qedge.size(), d_mom, d_w, d_fptr, n_port, d_nrm, d_n, c->stream);
      check_launch("port vectors");
      std::vector<double> nh(n_port);
      CK(cudaMemcpyAsync(nh.data(), d_n, sizeof(double) * n_port, cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
      for (int p = 0; p < n_port; ++p)
        require(std::isfinite(nh[p]) && nh[p] > 0, MW_EINVAL, "a port mode has zero norm on its faces");
      for (void* q : tmp) dfree(c, q);
      tmp.clear();
      install_sources(c, n_port, true, qptr, qedge, d_w, d_n);
    } catch (...) {
      for (void* q : tmp) dfree(c, q);
      if (c->d_q_w != d_w) dfree(c, d_w);
      if (c->d_q_norm != d_n) dfree(c, d_n);
      throw;
    }
    c->src_edge.clear();
    c->src_sign.clear();
  });
}

mw_status mw_get_port_vectors(mw_ctx* c, double* W, double* norms) {
  return guard(c, [&] {
    require(c->has_mesh && c->src_ports && c->n_src > 0, MW_ESTATE, "no port sources");
    const int P = c->n_src;
    const int64_t nq = c->q_ptr_h.back(), E = c->topo.n_edge;
    std::vector<double> w(std::max<int64_t>(nq, 1)), nh(P);
    std::vector<int32_t> edge(std::max<int64_t>(nq, 1));
    CK(cudaMemcpyAsync(w.data(), c->d_q_w, sizeof(double) * nq, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(edge.data(), c->d_q_edge, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(nh.data(), c->d_q_norm, sizeof(double) * P, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (W) {
      std::fill(W, W + E * P, 0.0);
      for (int p = 0; p < P; ++p)
        for (int64_t k = c->q_ptr_h[p]; k < c->q_ptr_h[p + 1]; ++k) W[(int64_t)edge[k] * P + p] = w[k];
    }
    if (norms) std::memcpy(norms, nh.data(), sizeof(double) * P);
  });
}

mw_status mw_setup_preconditioner(mw_ctx* c, int32_t n_sub, const int32_t* part, int32_t overlap, int32_t inv_prec) {
  return guard(c, [&] {
    require(c->has_mesh && c->n_freq > 0, MW_ESTATE, "assemble before setting up the preconditioner");
    require(inv_prec >= 0 && inv_prec <= 5, MW_EINVAL, "inv_prec must be 0 (FP64), 1 (FP32), 2 (BF16), 3 (FP32 "
                                                       "factorisation applied in FP64), 4 (sparse) or 5 (sparse, "
                                                       "BF16 tensor-core sweeps)");
    release_prec(c);
    Prec& p = c->prec;
    Error err{MW_OK, ""};
    if (!mw::build_subdomains(c->topo, n_sub, part, overlap, p.sd, err)) throw Fail{err.code, err.msg};
    const mw::Subdomains& sd = p.sd;
    p.apply_prec = inv_prec == 3 ? 0 : inv_prec;
    p.factor_prec = inv_prec == 0 ? 0 : 1;
    p.sparse_leaf = c->mf_leaf;
    p.dof_ptr = upload(c, sd.dof_ptr.data(), sd.dof_ptr.size());
    p.dofs = upload(c, sd.dofs.data(), sd.dofs.size());
    p.own_ptr = upload(c, sd.own_ptr.data(), sd.own_ptr.size());
    p.own_local = upload(c, sd.own_local.data(), sd.own_local.size());
    std::vector<int32_t> own_glob(sd.own_local.size());
    for (int s = 0; s < n_sub; ++s)
      for (int64_t q = sd.own_ptr[s]; q < sd.own_ptr[s + 1]; ++q)
        own_glob[q] = sd.dofs[sd.dof_ptr[s] + sd.own_local[q]];
    p.own_glob = upload(c, own_glob.data(), own_glob.size());
    p.tet_ptr = upload(c, sd.tet_ptr.data(), sd.tet_ptr.size());
    p.tet_ids = upload(c, sd.tet_ids.data(), sd.tet_ids.size());
    p.tet_loc = upload(c, sd.tet_loc.data(), sd.tet_loc.size());
    p.surf_ptr = upload(c, sd.surf_ptr.data(), sd.surf_ptr.size());
    p.surf_loc = upload(c, sd.surf_loc.data(), sd.surf_loc.size());
    {
      // outer faces carry their boundary class when classes are set: code -1 - class
      std::vector<int32_t> code(sd.surf_tet);
      if (!c->bface_cls.empty())
        for (size_t q = 0; q < code.size(); ++q)
          if (code[q] < 0) {
            const int32_t* v = &sd.surf_vert[3 * q];
            const int64_t bf = find_bface(c->topo, v[0], v[1], v[2]);
            require(bf >= 0, MW_EINVAL, "subdomain outer face is not a boundary face");
            code[q] = -1 - c->bface_cls[bf];
          }
      p.surf_tet = upload(c, code.data(), code.size());
    }
    p.surf_vert = upload(c, sd.surf_vert.data(), sd.surf_vert.size());
    const int64_t n_surf = (int64_t)sd.surf_tet.size();
    p.Bsurf = dalloc<double>(c, 6 * std::max<int64_t>(n_surf, 1));
    mwk::face_geom(c->d_xyz, p.surf_vert, n_surf, p.Bsurf, c->stream);
    if (inv_prec == 4 || inv_prec == 5) {
      for (int s = 0; s < n_sub; ++s) p.sum_n += (double)(sd.dof_ptr[s + 1] - sd.dof_ptr[s]);
      try {
        setup_sparse(c);
      } catch (...) {
        release_prec(c);
        throw;
      }
      p.ready = true;
      return;
    }
    // W offsets (cc layouts) and apply tiles
    std::vector<int64_t> woff(n_sub + 1, 0);
    std::vector<int32_t> tsub, trow;
    int64_t nmax = 0;
    for (int s = 0; s < n_sub; ++s) {
      const int64_t n = sd.dof_ptr[s + 1] - sd.dof_ptr[s], no = sd.own_ptr[s + 1] - sd.own_ptr[s];
      woff[s + 1] = woff[s] + n * no;
      p.sum_own_n += (double)n * no;
      p.sum_n += (double)n;
      nmax = std::max(nmax, n);
      for (int64_t r0 = 0; r0 < no; r0 += 32) {
        tsub.push_back(s);
        trow.push_back((int32_t)r0);
      }
    }
    p.n_tiles = (int)tsub.size();
    p.tile_sub = upload(c, tsub.data(), tsub.size());
    p.tile_row0 = upload(c, trow.data(), trow.size());
    p.w_off = upload(c, woff.data(), woff.size());
    if (p.apply_prec == 2)
      require(mwk::tc_plan_build(p.tc, sd, [&](size_t b) { return (void*)dalloc<unsigned char>(c, b); }, c->stream),
              MW_EINVAL, "BF16 tensor-core apply unavailable for this partition");
    const size_t wes = p.apply_prec == 0 ? sizeof(double2) : sizeof(float2);
    const size_t fes = p.factor_prec == 0 ? sizeof(double2) : sizeof(float2);
    // workspace batches
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    size_t budget = std::min<size_t>((size_t)8 << 30, free_b / 4);
    budget = std::max<size_t>(budget, (size_t)nmax * nmax * fes);
    std::vector<int32_t> bsub;
    std::vector<int64_t> bn, boff;
    int32_t* d_status = dalloc<int32_t>(c, 1);
    CK(cudaMemsetAsync(d_status, 0, sizeof(int32_t), c->stream));
    void* ws = dalloc<unsigned char>(c, budget);
    int32_t* d_bsub = dalloc<int32_t>(c, n_sub);
    int64_t* d_bn = dalloc<int64_t>(c, n_sub);
    int64_t* d_boff = dalloc<int64_t>(c, n_sub);
    void* dinv = dalloc<unsigned char>(c, (size_t)n_sub * 32 * 32 * fes);
    p.W.assign(c->n_freq, nullptr);
    try {
      for (int f = 0; f < c->n_freq; ++f) {
        if (p.apply_prec == 2)
          p.W[f] = dalloc<unsigned char>(c, mwk::tc_w_bytes(p.tc));
        else
          p.W[f] = dalloc<unsigned char>(c, wes * std::max<int64_t>(woff[n_sub], 1));
        const double k0 = k0_of(c->freqs[f]);
        int s = 0;
        while (s < n_sub) {
          bsub.clear();
          bn.clear();
          boff.clear();
          size_t used = 0;
          int64_t bmax = 0;
          while (s < n_sub) {
            const int64_t n = sd.dof_ptr[s + 1] - sd.dof_ptr[s];
            const size_t need = (size_t)n * n * fes;
            if (!bsub.empty() && used + need > budget) break;
            bsub.push_back(s);
            bn.push_back(n);
            boff.push_back((int64_t)(used / fes));
            used += need;
            used = (used + 255) / 256 * 256;
            bmax = std::max(bmax, n);
            ++s;
          }
          const int cnt = (int)bsub.size();
          CK(cudaMemcpyAsync(d_bsub, bsub.data(), sizeof(int32_t) * cnt, cudaMemcpyHostToDevice, c->stream));
          CK(cudaMemcpyAsync(d_bn, bn.data(), sizeof(int64_t) * cnt, cudaMemcpyHostToDevice, c->stream));
          CK(cudaMemcpyAsync(d_boff, boff.data(), sizeof(int64_t) * cnt, cudaMemcpyHostToDevice, c->stream));
          mwk::OrasBatch bt{cnt, bmax, d_bsub, d_bn, d_boff};
          CK(cudaMemsetAsync(ws, 0, used, c->stream));
          const double2* zc = c->d_zc ? c->d_zc + (size_t)f * (2 + c->n_port) : nullptr;
          mwk::oras_local_assemble(bt, p.topo(), p.Bsurf, c->d_KM, c->d_eps, k0, c->eps_bg[0], c->eps_bg[1], zc,
                                   c->d_metal, p.factor_prec, ws, c->stream);
          {
            // in-place Gauss-Jordan inversion: n^3 complex multiply-adds (8 n^3 real flops)
            double fl = 0;
            for (int64_t n : bn) fl += 8.0 * (double)n * n * n;
            ProfScope ps(c, MW_K_FACTOR, 0.0, fl);
            mwk::oras_invert(bt, p.factor_prec, ws, dinv, d_status, c->stream);
          }
          if (p.apply_prec == 2)
            mwk::tc_extract(p.tc, bt, p.topo(), p.factor_prec, ws, p.W[f], c->stream);
          else
            mwk::oras_extract(bt, p.topo(), p.factor_prec, ws, p.apply_prec, p.w_off, p.W[f], c->stream);
          check_launch("oras setup");
          // host vectors must outlive the async copies
          CK(cudaStreamSynchronize(c->stream));
        }
      }
      int32_t st = 0;
      CK(cudaMemcpy(&st, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost));
      require(st == 0, MW_ESINGULAR, "a subdomain matrix had a near-zero pivot");
    } catch (...) {
      dfree(c, ws);
      dfree(c, dinv);
      dfree(c, d_status);
      dfree(c, d_bsub);
      dfree(c, d_bn);
      dfree(c, d_boff);
      release_prec(c);
      throw;
    }
    dfree(c, ws);
    dfree(c, dinv);
    dfree(c, d_status);
    dfree(c, d_bsub);
    dfree(c, d_bn);
    dfree(c, d_boff);
    p.ready = true;
  });
}

mw_status mw_apply_preconditioner(mw_ctx* c, int32_t f, const void* r, void* z, int32_t n_cols) {
  return guard(c, [&] {
    require(c->prec.ready, MW_ESTATE, "no preconditioner");
    require(f >= 0 && f < c->n_freq && r && z && n_cols >= 1 && n_cols <= 128, MW_EINVAL, "bad arguments");
    const int64_t n = c->topo.n_edge * (int64_t)n_cols;
    if (c->prec.apply_prec == 0) {
      CK(cudaMemsetAsync(z, 0, sizeof(double2) * n, c->stream));
      apply_prec(c, f, 0, r, z, n_cols);
    } else {
      float2* a = dalloc<float2>(c, n);
      float2* b = dalloc<float2>(c, n);
      mwk::cast_f64_to_f32((const double2*)r, a, n, c->stream);
      CK(cudaMemsetAsync(b, 0, sizeof(float2) * n, c->stream));
      apply_prec(c, f, 1, a, b, n_cols);
      mwk::cast_f32_to_f64(b, (double2*)z, n, c->stream);
      CK(cudaStreamSynchronize(c->stream));
      dfree(c, a);
      dfree(c, b);
    }
    check_launch("apply preconditioner");
    check_tc_wait(c);
  });
}

mw_status mw_get_partition(mw_ctx* c, int32_t* owner, int32_t* sub_size) {
  return guard(c, [&] {
    require(c->prec.ready, MW_ESTATE, "no preconditioner");
    const mw::Subdomains& sd = c->prec.sd;
    if (owner) std::memcpy(owner, sd.owner.data(), sizeof(int32_t) * sd.owner.size());
    if (sub_size)
      for (int s = 0; s < sd.n_sub; ++s) sub_size[s] = (int32_t)(sd.dof_ptr[s + 1] - sd.dof_ptr[s]);
  });
}

mw_status mw_solve(mw_ctx* c, const mw_solve_opts* opts, void* fields, double* S, mw_solve_stats* stats) {
  mw_status st = guard(c, [&] {
    mw_solve_opts o = norm_opts(opts);
    mw_status conv = MW_OK;
    std::string msg;
    try {
      forward(c, o, stats);
    } catch (const Fail& e) {
      if (e.code != MW_ENOCONV) throw;
      conv = e.code;
      msg = e.msg;
    }
    const int64_t E = c->topo.n_edge;
    if (fields)
      for (int f = 0; f < c->n_freq; ++f)
        mwk::transpose_out(c->Xf[f], (double2*)fields + (int64_t)f * c->n_src * E, E, c->n_src, c->stream);
    if (S) {
      double2* dS = dalloc<double2>(c, (size_t)c->n_freq * c->n_src * c->n_src);
      for (int f = 0; f < c->n_freq; ++f)
        mwk::s_project(c->Xf[f], c->d_q_ptr, c->d_q_edge, c->d_q_w, c->d_q_norm, c->n_src,
                       dS + (size_t)f * c->n_src * c->n_src, c->stream);
      CK(cudaMemcpyAsync(S, dS, sizeof(double2) * c->n_freq * c->n_src * c->n_src, cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
      dfree(c, dS);
    }
    check_launch("solve outputs");
    CK(cudaStreamSynchronize(c->stream));
    if (conv != MW_OK) throw Fail{conv, msg};
  });
  return st;
}

mw_status mw_solve_rhs(mw_ctx* c, const mw_solve_opts* opts, int32_t n_cols, const void* b, void* x,
                       mw_solve_stats* stats) {
  return guard(c, [&] {
    require(c->has_mesh && c->n_freq > 0, MW_ESTATE, "assemble first");
    require(n_cols >= 1 && b && x, MW_EINVAL, "bad solve_rhs arguments");
    mw_solve_opts o = norm_opts(opts);
    const int64_t E = c->topo.n_edge;
    std::vector<double2*> Bi(c->n_freq), Xi(c->n_freq);
    std::vector<const double2*> Bc(c->n_freq);
    for (int f = 0; f < c->n_freq; ++f) {
      Bi[f] = dalloc<double2>(c, E * n_cols);
      Xi[f] = dalloc<double2>(c, E * n_cols);
      mwk::transpose_in((const double2*)b + (int64_t)f * n_cols * E, Bi[f], E, n_cols, c->stream);
      Bc[f] = Bi[f];
    }
    mw_status conv = MW_OK;
    std::string msg;
    try {
      solve_all(c, o, n_cols, Bc, Xi, stats);
    } catch (const Fail& e) {
      if (e.code != MW_ENOCONV) {
        for (int f = 0; f < c->n_freq; ++f) {
          dfree(c, Bi[f]);
          dfree(c, Xi[f]);
        }
        throw;
      }
      conv = e.code;
      msg = e.msg;
    }
    for (int f = 0; f < c->n_freq; ++f)
      mwk::transpose_out(Xi[f], (double2*)x + (int64_t)f * n_cols * E, E, n_cols, c->stream);
    CK(cudaStreamSynchronize(c->stream));
    for (int f = 0; f < c->n_freq; ++f) {
      dfree(c, Bi[f]);
      dfree(c, Xi[f]);
    }
    if (conv != MW_OK) throw Fail{conv, msg};
  });
}

// ---------------------------------------------------------------------------------------
// cost, adjoint and gradient
// ---------------------------------------------------------------------------------------
static void tikhonov_dev(Ctx* c, const double* d_eps, double* R_out, double* d_grad) {
  mwk::tikhonov(c->d_tet_nb, c->d_tikw, d_eps, c->topo.n_tet, d_grad, c->d_red, c->stream);
  double r = 0;
  CK(cudaMemcpyAsync(&r, c->d_red, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *R_out = r;
}

mw_status mw_tikhonov(mw_ctx* c, const double* eps_r, double* R_out, double* grad) {
  return guard(c, [&] {
    require(c->has_mesh && eps_r && R_out, MW_EINVAL, "bad tikhonov arguments");
    const int64_t T = c->topo.n_tet;
    double* de = upload(c, eps_r, 2 * T);
    double* dg = dalloc<double>(c, 2 * T);
    tikhonov_dev(c, de, R_out, dg);
    if (grad) {
      CK(cudaMemcpyAsync(grad, dg, sizeof(double) * 2 * T, cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
    }
    dfree(c, de);
    dfree(c, dg);
  });
}

// Device-resident gradient: S_obs/S_empty on the device, grad [T][2] device output, J to the host.
static void gradient_dev_impl(Ctx* c, const mw_solve_opts& o, const double2* dSo, const double2* dSe, double alpha,
                              double* J_out, double* dg) {
  require(c->has_mesh && c->n_freq > 0 && c->n_src > 0, MW_ESTATE, "assemble and set sources first");
  require(c->n_src <= 128, MW_EINVAL, "gradient supports at most 128 sources");
  const int64_t E = c->topo.n_edge, T = c->topo.n_tet;
  const int ns = c->n_src, nf = c->n_freq;
  const size_t nS = (size_t)nf * ns * ns;
  forward(c, o, nullptr);
  alloc_fields(c, c->Lf);
  if (!c->d_S) c->d_S = dalloc<double2>(c, 64 * 128 * 128);
  if (!c->d_C) c->d_C = dalloc<double2>(c, 64 * 128 * 128);
  if (!c->d_J) c->d_J = dalloc<double>(c, 4);
  if (c->d_Badj.size() != (size_t)nf) {
    for (auto p : c->d_Badj) dfree(c, p);
    c->d_Badj.assign(nf, nullptr);
    for (int f = 0; f < nf; ++f) c->d_Badj[f] = dalloc<double2>(c, E * ns);
  }
  for (int f = 0; f < nf; ++f)
    mwk::s_project(c->Xf[f], c->d_q_ptr, c->d_q_edge, c->d_q_w, c->d_q_norm, ns, c->d_S + (size_t)f * ns * ns,
                   c->stream);
  mwk::adjoint_weights(c->d_S, dSo, dSe, (int64_t)nS, c->d_C, c->d_J, c->stream);
  if (c->adjoint_mode == MW_ADJOINT_RECIPROCAL) {
    // receivers are the transmitters and A = A^T: the adjoint fields are combinations of the
    // forward fields, no adjoint solve
    if (!c->d_D) c->d_D = dalloc<double2>(c, 128 * 128);
    for (int f = 0; f < nf; ++f)
      mwk::reciprocal_adjoint(c->Xf[f], c->d_C + (size_t)f * ns * ns, c->d_q_norm, c->d_src_coef + (size_t)f * ns,
                              ns, E, c->d_D, c->Lf[f], c->stream);
    check_launch("reciprocal adjoint");
  } else {
    std::vector<const double2*> Bc(nf);
    for (int f = 0; f < nf; ++f) {
      mwk::adjoint_sources(c->d_qt_ptr, c->d_qt_edge, c->d_qt_src, c->d_qt_k, c->n_qt, c->d_q_w, c->d_q_norm,
                           c->d_C + (size_t)f * ns * ns, ns, c->d_Badj[f], E, c->stream);
      Bc[f] = c->d_Badj[f];
    }
    check_launch("adjoint sources");
    solve_all(c, o, ns, Bc, c->Lf, nullptr);
  }
  CK(cudaMemsetAsync(dg, 0, sizeof(double) * 2 * T, c->stream));
  for (int f = 0; f < nf; ++f) {
    const double k0 = k0_of(c->freqs[f]);
    // both fields read once, M^T and the tet's edges once, the gradient read and written; per
    // tet and column M x (36 real-by-complex FMAs) and lambda . (M x) (6 complex MACs)
    ProfScope ps(c, MW_K_GRADIENT, 2.0 * 16 * E * ns + (21.0 * 8 + 24 + 32) * T, 192.0 * T * ns);
    mwk::grad_tet(c->d_tet_edge, c->d_KM, T, c->Lf[f], c->Xf[f], ns, k0 * k0, dg, c->stream);
  }
  check_launch("gradient");
  double J = 0;
  if (alpha != 0.0) {
    if (!c->d_gR) c->d_gR = dalloc<double>(c, 2 * T);
    mwk::tikhonov(c->d_tet_nb, c->d_tikw, c->d_eps, T, c->d_gR, c->d_red, c->stream);
    mwk::axpy_f64(alpha, c->d_gR, dg, 2 * T, c->stream);
    mwk::add_scaled_scalar(c->d_J, alpha, c->d_red, c->stream);
    check_launch("tikhonov");
  }
  CK(cudaMemcpyAsync(&J, c->d_J, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *J_out = J;
}

// Column-sharded evaluation (one inversion evaluation split by transmitter columns over
// processes): the forward solves and S columns of transmitters [j0, j0+nl).
static void forward_cols_impl(Ctx* c, const mw_solve_opts& o, int j0, int nl, double* S_cols) {
  require(c->has_mesh && c->n_freq > 0 && c->n_src > 0, MW_ESTATE, "assemble and set sources first");
  require(j0 >= 0 && nl >= 1 && j0 + nl <= c->n_src && nl <= 128 && S_cols, MW_EINVAL, "bad column window");
  const int64_t E = c->topo.n_edge;
  const int ns = c->n_src, nf = c->n_freq;
  if (c->win_nl != nl || c->win_nf != nf || c->win_ns != ns) {
    free_window(c);
    for (auto* v : {&c->Xw, &c->Lw, &c->Bw, &c->Bwa}) {
      v->assign(nf, nullptr);
      for (int f = 0; f < nf; ++f) (*v)[f] = dalloc<double2>(c, E * nl);
    }
    c->d_Sp = dalloc<double2>(c, (size_t)nf * ns * nl);
    c->win_nl = nl;
    c->win_nf = nf;
    c->win_ns = ns;
  }
  c->win_j0 = j0;
  upload_source_coefs(c);
  std::vector<const double2*> Bs(nf);
  for (int f = 0; f < nf; ++f) {
    mwk::source_rhs(c->d_q_ptr, c->d_q_edge, c->d_q_w, c->d_src_coef + (size_t)f * ns, ns, c->Bw[f], E, c->stream,
                    j0, nl);
    Bs[f] = c->Bw[f];
  }
  check_launch("source rhs (window)");
  solve_all(c, o, nl, Bs, c->Xw, nullptr);
  for (int f = 0; f < nf; ++f)
    mwk::s_project(c->Xw[f], c->d_q_ptr, c->d_q_edge, c->d_q_w, c->d_q_norm, ns, c->d_Sp + (size_t)f * ns * nl,
                   c->stream, nl);
  check_launch("S columns");
  CK(cudaMemcpyAsync(S_cols, c->d_Sp, sizeof(double2) * nf * ns * nl, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
}

// The rest of the sharded evaluation for the window of the last forward_cols: cost and adjoint
// weights from the whole S, adjoint solves of the window's columns, and their part of the
// per-tet gradient (no Tikhonov term).
static void gradient_cols_impl(Ctx* c, const mw_solve_opts& o, const double* S_full, const double* S_obs,
                               const double* S_empty, double* J_out, double* grad_part) {
  require(c->win_nl > 0 && c->win_nf == c->n_freq && c->win_ns == c->n_src, MW_ESTATE,
          "call mw_forward_cols first");
  require(S_full && S_obs && S_empty && J_out && grad_part, MW_EINVAL, "null argument");
  const int64_t E = c->topo.n_edge, T = c->topo.n_tet;
  const int ns = c->n_src, nf = c->n_freq, j0 = c->win_j0, nl = c->win_nl;
  const size_t nS = (size_t)nf * ns * ns;
  if (!c->d_S) c->d_S = dalloc<double2>(c, 64 * 128 * 128);
  if (!c->d_C) c->d_C = dalloc<double2>(c, 64 * 128 * 128);
  if (!c->d_So) c->d_So = dalloc<double2>(c, 64 * 128 * 128);
  if (!c->d_Se) c->d_Se = dalloc<double2>(c, 64 * 128 * 128);
  if (!c->d_J) c->d_J = dalloc<double>(c, 4);
  if (!c->d_grad) c->d_grad = dalloc<double>(c, 2 * T);
  CK(cudaMemcpyAsync(c->d_S, S_full, sizeof(double2) * nS, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->d_So, S_obs, sizeof(double2) * nS, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->d_Se, S_empty, sizeof(double2) * nS, cudaMemcpyHostToDevice, c->stream));
  mwk::adjoint_weights(c->d_S, c->d_So, c->d_Se, (int64_t)nS, c->d_C, c->d_J, c->stream);
  std::vector<const double2*> Bc(nf);
  for (int f = 0; f < nf; ++f) {
    mwk::adjoint_sources(c->d_qt_ptr, c->d_qt_edge, c->d_qt_src, c->d_qt_k, c->n_qt, c->d_q_w, c->d_q_norm,
                         c->d_C + (size_t)f * ns * ns, ns, c->Bwa[f], E, c->stream, j0, nl);
    Bc[f] = c->Bwa[f];
  }
  check_launch("adjoint sources (window)");
  solve_all(c, o, nl, Bc, c->Lw, nullptr);
  CK(cudaMemsetAsync(c->d_grad, 0, sizeof(double) * 2 * T, c->stream));
  for (int f = 0; f < nf; ++f) {
    const double k0 = k0_of(c->freqs[f]);
    ProfScope ps(c, MW_K_GRADIENT, 2.0 * 16 * E * nl + (21.0 * 8 + 24 + 32) * T, 192.0 * T * nl);
    mwk::grad_tet(c->d_tet_edge, c->d_KM, T, c->Lw[f], c->Xw[f], nl, k0 * k0, c->d_grad, c->stream);
  }
  check_launch("gradient (window)");
  CK(cudaMemcpyAsync(J_out, c->d_J, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(grad_part, c->d_grad, sizeof(double) * 2 * T, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
}

mw_status mw_set_adjoint_mode(mw_ctx* c, int32_t mode) {
  return guard(c, [&] {
    require(mode == MW_ADJOINT_SOLVE || mode == MW_ADJOINT_RECIPROCAL, MW_EINVAL, "bad adjoint mode");
    c->adjoint_mode = mode;
  });
}

mw_status mw_set_z_storage(mw_ctx* c, int32_t bf16) {
  return guard(c, [&] {
    require(bf16 == 0 || bf16 == 1, MW_EINVAL, "bad Z storage");
    if (c->z_bf16 != bf16) drop_graphs(c);
    c->z_bf16 = bf16;
  });
}

mw_status mw_set_sweep_schedule(mw_ctx* c, int32_t persistent) {
  return guard(c, [&] {
    require(persistent == 0 || persistent == 1, MW_EINVAL, "bad sweep schedule");
    if (c->sweep_persistent != persistent) drop_graphs(c);
    c->sweep_persistent = persistent;
  });
}

mw_status mw_forward_cols(mw_ctx* c, const mw_solve_opts* opts, int32_t j0, int32_t n_cols, double* S_cols) {
  return guard(c, [&] {
    mw_solve_opts o = norm_opts(opts);
    forward_cols_impl(c, o, j0, n_cols, S_cols);
  });
}

mw_status mw_gradient_cols(mw_ctx* c, const mw_solve_opts* opts, const double* S_full, const double* S_obs,
                           const double* S_empty, double* J_out, double* grad_part) {
  return guard(c, [&] {
    mw_solve_opts o = norm_opts(opts);
    gradient_cols_impl(c, o, S_full, S_obs, S_empty, J_out, grad_part);
  });
}

static void gradient_impl(Ctx* c, const mw_solve_opts& o, const double* S_obs, const double* S_empty, double alpha,
                          double* J_out, double* grad, double* S_out) {
  require(c->has_mesh && c->n_freq > 0 && c->n_src > 0, MW_ESTATE, "assemble and set sources first");
  require(S_obs && S_empty && J_out, MW_EINVAL, "null S_obs / S_empty / J_out");
  const int64_t T = c->topo.n_tet;
  const size_t nS = (size_t)c->n_freq * c->n_src * c->n_src;
  if (!c->d_So) c->d_So = dalloc<double2>(c, 64 * 128 * 128);
  if (!c->d_Se) c->d_Se = dalloc<double2>(c, 64 * 128 * 128);
  if (!c->d_grad) c->d_grad = dalloc<double>(c, 2 * T);
  CK(cudaMemcpyAsync(c->d_So, S_obs, sizeof(double2) * nS, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->d_Se, S_empty, sizeof(double2) * nS, cudaMemcpyHostToDevice, c->stream));
  gradient_dev_impl(c, o, c->d_So, c->d_Se, alpha, J_out, c->d_grad);
  if (grad) CK(cudaMemcpyAsync(grad, c->d_grad, sizeof(double) * 2 * T, cudaMemcpyDeviceToHost, c->stream));
  if (S_out) CK(cudaMemcpyAsync(S_out, c->d_S, sizeof(double2) * nS, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
}

mw_status mw_gradient(mw_ctx* c, const mw_solve_opts* opts, const double* S_obs, const double* S_empty, double alpha,
                      double* J_out, double* grad, double* S_out) {
  return guard(c, [&] {
    mw_solve_opts o = norm_opts(opts);
    gradient_impl(c, o, S_obs, S_empty, alpha, J_out, grad, S_out);
  });
}

// ---------------------------------------------------------------------------------------
// L-BFGS, reverse communication (Sec. IV-D): mirrors the recursion stated in mw.h.
// ---------------------------------------------------------------------------------------
struct mw_lbfgs {
  int64_t n = 0;
  mw_inv_opts o{};
  int phase = 0;            // 0: expecting f(x0); 1: line search
  std::vector<double> x, g, d, xn;
  double f = 0, gd = 0, t = 1;
  int trials = 0, it = 0;
  std::vector<std::vector<double>> S, Y;
};

static double dotv(const std::vector<double>& a, const std::vector<double>& b) {
  double s = 0;
  for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
  return s;
}

static void lbfgs_direction(mw_lbfgs* st) {
  const int64_t n = st->n;
  std::vector<double>& d = st->d;
  auto steepest = [&]() {
    double mx = 0;
    for (int64_t i = 0; i < n; ++i) mx = std::max(mx, std::fabs(st->g[i]));
    mx = std::max(mx, 1e-300);
    for (int64_t i = 0; i < n; ++i) d[i] = -st->g[i] * (st->o.first_step / mx);
  };
  d.assign(n, 0.0);
  if (st->S.empty()) {
    steepest();
  } else {
    std::vector<double> q = st->g;
    const int k = (int)st->S.size();
    std::vector<double> rho(k), al(k);
    for (int i = k - 1; i >= 0; --i) {
      rho[i] = 1.0 / dotv(st->Y[i], st->S[i]);
      al[i] = rho[i] * dotv(st->S[i], q);
      for (int64_t e = 0; e < n; ++e) q[e] -= al[i] * st->Y[i][e];
    }
    const double gamma = dotv(st->S[k - 1], st->Y[k - 1]) / dotv(st->Y[k - 1], st->Y[k - 1]);
    for (int64_t e = 0; e < n; ++e) q[e] *= gamma;
    for (int i = 0; i < k; ++i) {
      const double b = rho[i] * dotv(st->Y[i], q);
      for (int64_t e = 0; e < n; ++e) q[e] += (al[i] - b) * st->S[i][e];
    }
    for (int64_t e = 0; e < n; ++e) d[e] = -q[e];
  }
  st->gd = dotv(st->g, d);
  if (!(st->gd < 0.0)) {
    steepest();
    st->gd = dotv(st->g, d);
  }
  st->t = 1.0;
  st->trials = 0;
}

extern "C" mw_status mw_lbfgs_create(mw_lbfgs** out, int64_t n, const mw_inv_opts* opts) {
  if (!out || n <= 0) return MW_EINVAL;
  mw_lbfgs* st = new (std::nothrow) mw_lbfgs();
  if (!st) return MW_ENOMEM;
  st->n = n;
  mw_inv_opts d{};
  d.m = 8;
  d.max_it = 20;
  d.c1 = 1e-4;
  d.max_ls = 10;
  d.first_step = 1.0;
  if (opts) d = *opts;
  if (d.m <= 0) d.m = 8;
  if (d.max_ls <= 0) d.max_ls = 10;
  if (d.c1 <= 0) d.c1 = 1e-4;
  if (d.first_step <= 0) d.first_step = 1.0;
  st->o = d;
  *out = st;
  return MW_OK;
}

extern "C" void mw_lbfgs_destroy(mw_lbfgs* st) { delete st; }

extern "C" mw_status mw_lbfgs_step(mw_lbfgs* st, double* x_io, double f, const double* g, int32_t* request) {
  if (!st || !x_io || !g || !request) return MW_EINVAL;
  if (!std::isfinite(f)) return MW_EINVAL;
  const int64_t n = st->n;
  auto propose = [&]() {
    st->xn.resize(n);
    for (int64_t i = 0; i < n; ++i) st->xn[i] = st->x[i] + st->t * st->d[i];
    std::memcpy(x_io, st->xn.data(), sizeof(double) * n);
    *request = 1;
  };
  auto finish = [&]() {
    std::memcpy(x_io, st->x.data(), sizeof(double) * n);
    *request = 0;
  };
  if (st->phase == 0) {
    st->x.assign(x_io, x_io + n);
    st->g.assign(g, g + n);
    st->f = f;
    st->it = 0;
    if (st->o.max_it <= 0 || (st->o.target_J > 0 && f <= st->o.target_J)) {
      finish();
      return MW_OK;
    }
    lbfgs_direction(st);
    st->phase = 1;
    propose();
    return MW_OK;
  }
  // line search: f, g at xn
  st->trials++;
  if (f <= st->f + st->o.c1 * st->t * st->gd) {
    std::vector<double> s(n), y(n);
    for (int64_t i = 0; i < n; ++i) {
      s[i] = st->xn[i] - st->x[i];
      y[i] = g[i] - st->g[i];
    }
    const double sy = dotv(s, y);
    if (sy > 1e-12 * std::sqrt(dotv(s, s)) * std::sqrt(dotv(y, y))) {
      st->S.push_back(s);
      st->Y.push_back(y);
      if ((int)st->S.size() > st->o.m) {
        st->S.erase(st->S.begin());
        st->Y.erase(st->Y.begin());
      }
    }
    st->x = st->xn;
    st->g.assign(g, g + n);
    st->f = f;
    st->it++;
    if (st->it >= st->o.max_it || (st->o.target_J > 0 && f <= st->o.target_J)) {
      finish();
      return MW_OK;
    }
    lbfgs_direction(st);
    propose();
    return MW_OK;
  }
  if (st->trials >= st->o.max_ls) {
    finish();
    return MW_OK;
  }
  st->t *= 0.5;
  propose();
  return MW_OK;
}

extern "C" mw_status mw_invert(mw_ctx* c, const mw_inv_opts* opts, const mw_solve_opts* sopts, const double* S_obs,
                               const double* S_empty, double* eps_io, mw_inv_history* hist) {
  return guard(c, [&] {
    require(c->has_mesh && c->n_freq > 0 && c->n_src > 0, MW_ESTATE, "assemble and set sources first");
    require(opts && S_obs && S_empty && eps_io, MW_EINVAL, "bad invert arguments");
    mw_solve_opts so = norm_opts(sopts);
    const int64_t T = c->topo.n_tet;
    mw_lbfgs* st = nullptr;
    if (mw_lbfgs_create(&st, 2 * T, opts) != MW_OK) throw Fail{MW_ENOMEM, "lbfgs state"};
    std::unique_ptr<mw_lbfgs, void (*)(mw_lbfgs*)> hold(st, mw_lbfgs_destroy);
    std::vector<double> x(eps_io, eps_io + 2 * T), g(2 * T);
    std::vector<double> freqs = c->freqs;
    const double ebg[2] = {c->eps_bg[0], c->eps_bg[1]};
    int32_t req = 1;
    int evals = 0, accepted = 0;
    cudaEvent_t e0;
    CK(cudaEventCreate(&e0));
    CK(cudaEventRecord(e0, c->stream));
    auto elapsed = [&]() {
      CK(cudaEventRecord(c->ev1, c->stream));
      CK(cudaEventSynchronize(c->ev1));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, e0, c->ev1));
      return ms * 1e-3;
    };
    int last_it = -1;
    while (req) {
      mw_status a = mw_assemble(c, c->n_freq, freqs.data(), x.data(), ebg);
      if (a != MW_OK) throw Fail{a, c->err};
      double J = 0;
      gradient_impl(c, so, S_obs, S_empty, opts->alpha, &J, g.data(), nullptr);
      ++evals;
      if (st->phase == 0 || st->it != last_it) {
        // first evaluation is the start point; accepted iterates are recorded below
      }
      const int it_before = st->it;
      const int phase_before = st->phase;
      mw_status s = mw_lbfgs_step(st, x.data(), J, g.data(), &req);
      if (s != MW_OK) throw Fail{s, "lbfgs step"};
      if (phase_before == 0) {
        if (hist && hist->J) hist->J[0] = J;
        if (hist && hist->seconds) hist->seconds[0] = elapsed();
      } else if (st->it != it_before) {
        ++accepted;
        if (hist && hist->J) hist->J[accepted] = J;
        if (hist && hist->seconds) hist->seconds[accepted] = elapsed();
      }
      last_it = st->it;
    }
    cudaEventDestroy(e0);
    std::memcpy(eps_io, x.data(), sizeof(double) * 2 * T);
    mw_status a = mw_assemble(c, c->n_freq, freqs.data(), x.data(), ebg);
    if (a != MW_OK) throw Fail{a, c->err};
    if (hist) {
      hist->iterations = accepted;
      hist->evaluations = evals;
    }
  });
}


int64_t mw_kernel_launches(void) { return (int64_t)g_launches.load(); }

mw_status mw_profile_enable(mw_ctx* c, uint32_t mask) {
  return guard(c, [&] {
    c->prof.mask = mask;
    c->prof.marks.clear();
    c->prof.used = 0;
    for (int k = 0; k < MW_K_NCLASS; ++k) {
      c->prof.bytes[k] = 0;
      c->prof.flops[k] = 0;
      c->prof.graph_ms[k] = 0;
      c->prof.graph_launches[k] = 0;
    }
  });
}

mw_status mw_profile_read(mw_ctx* c, double* ms, int64_t* launches, double* bytes, double* flops) {
  return guard(c, [&] {
    require(ms && launches, MW_EINVAL, "null outputs");
    for (int k = 0; k < MW_K_NCLASS; ++k) {
      ms[k] = c->prof.graph_ms[k];
      launches[k] = c->prof.graph_launches[k];
      if (bytes) bytes[k] = c->prof.bytes[k];
      if (flops) flops[k] = c->prof.flops[k];
      c->prof.bytes[k] = 0;
      c->prof.flops[k] = 0;
      c->prof.graph_ms[k] = 0;
      c->prof.graph_launches[k] = 0;
    }
    CK(cudaStreamSynchronize(c->stream));
    for (auto& m : c->prof.marks) {
      float t = 0;
      CK(cudaEventElapsedTime(&t, m.second.first, m.second.second));
      if (m.first >= 0 && m.first < MW_K_NCLASS) {
        ms[m.first] += t;
        launches[m.first] += 1;
      }
    }
    c->prof.marks.clear();
    c->prof.used = 0;
  });
}

mw_status mw_assemble_dev(mw_ctx* c, int32_t n_freq, const double* freq_hz, const void* eps_dev, const double* eps_bg) {
  return guard(c, [&] {
    require(c->has_mesh && c->n_freq == n_freq && n_freq >= 1 && freq_hz && eps_dev && eps_bg, MW_EINVAL,
            "assemble_dev needs a prior host assemble with the same frequency count");
    const int64_t T = c->topo.n_tet, nnz = c->topo.nnz;
    CK(cudaMemcpyAsync(c->d_eps, eps_dev, sizeof(double) * 2 * T, cudaMemcpyDeviceToDevice, c->stream));
    c->freqs.assign(freq_hz, freq_hz + n_freq);
    c->eps_bg[0] = eps_bg[0];
    c->eps_bg[1] = eps_bg[1];
    reassemble_all(c);
  });
}

mw_status mw_gradient_dev(mw_ctx* c, const mw_solve_opts* opts, const void* S_obs_dev, const void* S_empty_dev,
                          double alpha, double* J_out, void* grad_dev) {
  return guard(c, [&] {
    mw_solve_opts o = norm_opts(opts);
    require(S_obs_dev && S_empty_dev && J_out && grad_dev, MW_EINVAL, "null device argument");
    gradient_dev_impl(c, o, (const double2*)S_obs_dev, (const double2*)S_empty_dev, alpha, J_out, (double*)grad_dev);
  });
}


mw_status mw_krylov_dots(mw_ctx* c, int32_t nvec, const void* V_dev, int64_t vstride, const void* w_dev,
                         int64_t n_rows, int32_t n_cols, double* h_out) {
  return guard(c, [&] {
    require(nvec >= 1 && nvec <= 64 && V_dev && w_dev && h_out && n_rows >= 1 && n_cols >= 1 && n_cols <= 128 &&
                vstride >= n_rows * (int64_t)n_cols,
            MW_EINVAL, "bad arguments");
    double2* part = dalloc<double2>(c, (size_t)mwk::kCgsDotsMaxParts * nvec * n_cols);
    double2* h = dalloc<double2>(c, (size_t)nvec * n_cols);
    int32_t* err = dalloc<int32_t>(c, 1);
    CK(cudaMemsetAsync(err, 0, sizeof(int32_t), c->stream));
    const int np = mwk::cgs_dots_f32((const float2*)V_dev, vstride, nvec, (const float2*)w_dev, n_rows, n_cols, part,
                                     err, c->stream);
    mwk::reduce_h(part, np, nvec, n_cols, h, c->stream);
    int32_t e = 0;
    CK(cudaMemcpyAsync(h_out, h, sizeof(double2) * nvec * n_cols, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&e, err, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    dfree(c, part);
    dfree(c, h);
    dfree(c, err);
    check_launch("krylov dots");
    require(e == 0, MW_ETIMEOUT, "streaming Gram-Schmidt dots: bounded wait ran out");
  });
}

// Tensor-core preconditioner apply for callers that cannot allocate device memory: the
// gathered operand goes to the library's fixed scratch array, nothing else is allocated.
mw_status mw_apply_preconditioner_noalloc(mw_ctx* c, int32_t f, const void* r, void* z, int32_t n_cols) {
  return guard(c, [&] {
    require(c->prec.ready, MW_ESTATE, "no preconditioner");
    require(c->prec.apply_prec == 2, MW_EINVAL, "the allocation-free apply needs a BF16 (tensor-core) preconditioner");
    require(f >= 0 && f < c->n_freq && r && z && n_cols >= 1 && n_cols <= 128, MW_EINVAL, "bad arguments");
    const size_t need = mwk::tc_scratch_bytes(c->prec.tc, n_cols);
    require(need <= mwk::kNoAllocScratchBytes, MW_EINVAL,
            "gathered operand needs " + std::to_string(need) + " bytes, above the fixed scratch of " +
                std::to_string(mwk::kNoAllocScratchBytes) + " bytes (fewer columns or a smaller mesh)");
    void* scratch = nullptr;
    std::string err;
    if (!mwk::tc_noalloc_scratch(&scratch, err)) throw Fail{MW_ECUDA, err};
    mwk::oras_apply_tc(c->prec.tc, c->prec.topo(), c->prec.W[f], (const float2*)r, (float2*)z, n_cols, scratch,
                       c->stream);
    check_launch("allocation-free preconditioner apply");
    check_tc_wait(c);
  });
}


// =======================================================================================
// Learned initialiser (no counterpart in the paper): MLP + transposed-convolution decoder
// =======================================================================================
static constexpr int kHid = 1024, kG = 32, kOut = 2 * kG * kG * kG;

mw_status mw_spmm_plan_stats(int64_t n_vert, const double* xyz, int64_t n_tet, const int32_t* tet_vert, int32_t halo_max,
                             int64_t* stats) {
  if (!xyz || !tet_vert || !stats) return MW_EINVAL;
  try {
    mw::Topology t;
    Error err{MW_OK, ""};
    if (!mw::build_topology(n_vert, n_tet, tet_vert, t, err)) return err.code;
    mw::SpmmPlan p;
    // the library's own bounds when halo_max is the library's halo bound
    const bool lib = halo_max == mwk::kHaloMax;
    if (!mw::build_spmm_plan(t, xyz, halo_max, p, err, lib ? mwk::kHaloRows : 1 << 30,
                             lib ? (int64_t)mwk::kHaloNnz : INT64_MAX))
      return err.code;
    const int64_t E = t.n_edge;
    // every row exactly once; blocks cover the rows in order
    std::vector<int32_t> seen(E, 0);
    for (int32_t r : p.rows) {
      if (r < 0 || r >= E || seen[r]++) return MW_ECUDA;
    }
    if ((int64_t)p.rows.size() != E || p.blk_row.front() != 0 || p.blk_row.back() != E) return MW_ECUDA;
    if ((int64_t)p.rptr.size() != E + 1 || p.rptr.back() != t.nnz || (int64_t)p.lcol.size() != t.nnz) return MW_ECUDA;
    std::vector<int32_t> hit(t.nnz, 0);
    int64_t halo_sum = 0, halo_big = 0;
    for (int64_t b = 0; b < p.n_block; ++b) {
      const int64_t h0 = p.blk_halo[b], H = p.blk_halo[b + 1] - h0;
      if (H < 1 || H > halo_max || p.blk_row[b + 1] <= p.blk_row[b]) return MW_ECUDA;
      if (lib && (p.blk_row[b + 1] - p.blk_row[b] > mwk::kHaloRows ||
                  p.rptr[p.blk_row[b + 1]] - p.rptr[p.blk_row[b]] > mwk::kHaloNnz))
        return MW_ECUDA;
      for (int64_t j = h0 + 1; j < h0 + H; ++j)
        if (p.halo[j] <= p.halo[j - 1]) return MW_ECUDA;      // ascending, no repeats
      halo_sum += H;
      halo_big = std::max(halo_big, H);
      for (int64_t i = p.blk_row[b]; i < p.blk_row[b + 1]; ++i) {
        const int32_t r = p.rows[i];
        if (p.rptr[i + 1] - p.rptr[i] != t.row_ptr[r + 1] - t.row_ptr[r]) return MW_ECUDA;
        for (int64_t q = p.rptr[i]; q < p.rptr[i + 1]; ++q) {
          const int64_t k = p.src[q];
          // the canonical nonzero of the same row, in the same (ascending column) order
          if (k != t.row_ptr[r] + (q - p.rptr[i]) || hit[k]++) return MW_ECUDA;
          if (p.lcol[q] >= H || p.halo[h0 + p.lcol[q]] != t.col_idx[k]) return MW_ECUDA;
        }
      }
    }
    stats[0] = p.n_block;
    stats[1] = halo_sum;
    stats[2] = halo_big;
    stats[3] = t.nnz;
    return MW_OK;
  } catch (const std::bad_alloc&) {
    return MW_ENOMEM;
  }
}

mw_status mw_sparse_plan_stats(int64_t n_vert, const double* xyz, int64_t n_tet, const int32_t* tet_vert, int32_t n_sub,
                               const int32_t* part, int32_t overlap, int32_t leaf, int64_t* stats) {
  if (!xyz || !tet_vert || !part || !stats || leaf < 1) return MW_EINVAL;
  try {
    mw::Topology t;
    Error err{MW_OK, ""};
    if (!mw::build_topology(n_vert, n_tet, tet_vert, t, err)) return err.code;
    mw::Subdomains sd;
    if (!mw::build_subdomains(t, n_sub, part, overlap, sd, err)) return err.code;
    std::vector<double> xv(xyz, xyz + 3 * n_vert);
    mw::Multifrontal y;
    if (!mw::build_multifrontal(t, sd, xv, nullptr, leaf, y, err)) return err.code;
    // structural invariants of the plan
    int64_t max_f = 0, dense = 0;
    for (int s = 0; s < sd.n_sub; ++s) {
      const int64_t n = sd.dof_ptr[s + 1] - sd.dof_ptr[s];
      dense += n * n;
      std::vector<int32_t> seen(n, 0);
      for (int64_t k = y.sub_node_ptr[s]; k < y.sub_node_ptr[s + 1]; ++k) {
        for (int64_t q = y.piv_ptr[k]; q < y.piv_ptr[k + 1]; ++q) {
          const int32_t d = y.piv_loc[q];
          if (d < 0 || d >= n || seen[d]++) return MW_ECUDA;  // a dof pivots twice (or never, below)
        }
        if (y.p[k] % 32 || y.p[k] < y.preal[k] || y.f[k] != (int64_t)y.p[k] + y.u[k]) return MW_ECUDA;
        if (y.ws_off[k] + y.f[k] * y.f[k] > y.ws_size[s]) return MW_ECUDA;
        max_f = std::max(max_f, y.f[k]);
        // every update dof of a child appears in its parent's front at the row its map names
        const int32_t par = y.parent[k];
        if (par >= 0) {
          const int32_t* inv = y.inv.data() + y.inv_off[k];
          int64_t hit = 0;
          for (int64_t r = 0; r < y.f[par]; ++r) {
            const int32_t a = inv[r];
            if (a < -1 || a >= y.u[k]) return MW_ECUDA;
            if (a < 0) continue;
            ++hit;
            const int32_t dof = y.upd_loc[y.upd_ptr[k] + a];
            int32_t rowdof = -1;
            if (r < y.preal[par]) rowdof = y.piv_loc[y.piv_ptr[par] + r];
            else if (r >= y.p[par]) rowdof = y.upd_loc[y.upd_ptr[par] + (r - y.p[par])];
            if (rowdof != dof) return MW_ECUDA;
          }
          if (hit != y.u[k]) return MW_ECUDA;
        } else if (y.u[k] != 0) {
          return MW_ECUDA;                                      // a root has no update dofs
        }
      }
      for (int64_t d = 0; d < n; ++d)
        if (seen[d] != 1) return MW_ECUDA;
      for (int64_t i = y.asm_sub_ptr[s]; i < y.asm_sub_ptr[s + 1]; ++i)
        if (y.asm_target[i] < 0 || y.asm_target[i] >= y.ws_size[s]) return MW_ECUDA;
    }
    int64_t ws_max = 0;
    for (int64_t v : y.ws_size) ws_max = std::max(ws_max, v);
    stats[0] = y.n_nodes;
    stats[1] = y.max_height;
    stats[2] = max_f;
    stats[3] = y.fac_total;
    stats[4] = ws_max;
    stats[5] = dense;
    return MW_OK;
  } catch (...) {
    return MW_ENOMEM;
  }
}

int64_t mw_nn_param_count(int32_t n_in) {
  if (n_in <= 0) return -1;
  return (int64_t)kHid * n_in + kHid + (int64_t)kHid * kHid + kHid + 16 * 16 * 64 + 16 + 16 * 8 * 64 + 8 + 8 * 2 * 64 +
         2;
}

static void nn_free(Ctx* c) {
  NnState& n = c->nn;
  for (void* p : {(void*)n.theta, (void*)n.grad, (void*)n.m, (void*)n.v, n.W1b, n.W2b, (void*)n.x, (void*)n.z1,
                  (void*)n.h1, (void*)n.z2, (void*)n.h2, (void*)n.a1, (void*)n.g1, (void*)n.a2, (void*)n.g2,
                  (void*)n.y, (void*)n.t, (void*)n.dy, (void*)n.dg2, (void*)n.da2, (void*)n.dg1, (void*)n.da1,
                  (void*)n.dh2, (void*)n.dz2, (void*)n.dh1, (void*)n.dz1, (void*)n.part, (void*)n.loss,
                  (void*)n.gws, (void*)n.cpart, (void*)n.wpart,
                  (void*)n.data_x, (void*)n.data_t, (void*)n.idx})
    dfree(c, p);
  n = NnState();
}

static void nn_batch_buffers(Ctx* c, int B) {
  NnState& n = c->nn;
  if (B <= n.bcap) return;
  for (void* p : {(void*)n.x, (void*)n.z1, (void*)n.h1, (void*)n.z2, (void*)n.h2, (void*)n.a1, (void*)n.g1, (void*)n.a2,
                  (void*)n.g2, (void*)n.y, (void*)n.t, (void*)n.dy, (void*)n.dg2, (void*)n.da2, (void*)n.dg1,
                  (void*)n.da1, (void*)n.dh2, (void*)n.dz2, (void*)n.dh1, (void*)n.dz1, (void*)n.idx, (void*)n.gws,
                  (void*)n.cpart, (void*)n.wpart})
    dfree(c, p);
  n.wpart = dalloc<float>(c, (size_t)mwk::kConvChunks * 16 * 16 * 64);
  n.gws = dalloc<float>(c, (size_t)32 * B * kHid);
  n.cpart = dalloc<float>(c, (size_t)16 * B);
  n.x = dalloc<float>(c, (size_t)B * n.n_in);
  n.z1 = dalloc<float>(c, (size_t)B * kHid);
  n.h1 = dalloc<float>(c, (size_t)B * kHid);
  n.z2 = dalloc<float>(c, (size_t)B * kHid);
  n.h2 = dalloc<float>(c, (size_t)B * kHid);
  n.a1 = dalloc<float>(c, (size_t)B * 16 * 512);
  n.g1 = dalloc<float>(c, (size_t)B * 16 * 512);
  n.a2 = dalloc<float>(c, (size_t)B * 8 * 4096);
  n.g2 = dalloc<float>(c, (size_t)B * 8 * 4096);
  n.y = dalloc<float>(c, (size_t)B * kOut);
  n.t = dalloc<float>(c, (size_t)B * kOut);
  n.dy = dalloc<float>(c, (size_t)B * kOut);
  n.dg2 = dalloc<float>(c, (size_t)B * 8 * 4096);
  n.da2 = dalloc<float>(c, (size_t)B * 8 * 4096);
  n.dg1 = dalloc<float>(c, (size_t)B * 16 * 512);
  n.da1 = dalloc<float>(c, (size_t)B * 16 * 512);
  n.dh2 = dalloc<float>(c, (size_t)B * kHid);
  n.dz2 = dalloc<float>(c, (size_t)B * kHid);
  n.dh1 = dalloc<float>(c, (size_t)B * kHid);
  n.dz1 = dalloc<float>(c, (size_t)B * kHid);
  n.idx = dalloc<int32_t>(c, (size_t)B);
  n.bcap = B;
}

static void nn_refresh_bf16(Ctx* c) {
  NnState& n = c->nn;
  mwk::nn_to_bf16(n.theta + n.oW1, n.W1b, (int64_t)kHid * n.n_in, c->stream);
  mwk::nn_to_bf16(n.theta + n.oW2, n.W2b, (int64_t)kHid * kHid, c->stream);
}

// forward on n.x[0..B) -> n.y
static void nn_forward(Ctx* c, int B) {
  NnState& n = c->nn;
  const float* th = n.theta;
  cudaStream_t s = c->stream;
  const double Bd = B, ni = n.n_in, H = kHid;
  {
    // BF16 weights, FP32 inputs and biases read once; pre- and post-activation written
    ProfScope ps(c, MW_K_NN_GEMM, 2.0 * H * (ni + H) + 4.0 * Bd * (ni + H) + 8.0 * H + 16.0 * Bd * H,
                 2.0 * Bd * H * (ni + H));
    const size_t wsf = (size_t)32 * n.bcap * kHid;
    mwk::nn_gemm_bf16(n.x, n.n_in, 1, n.W1b, 1, n.n_in, th + n.ob1, n.z1, n.h1, B, kHid, n.n_in, s, n.gws, wsf);
    mwk::nn_gemm_bf16(n.h1, kHid, 1, n.W2b, 1, kHid, th + n.ob2, n.z2, n.h2, B, kHid, kHid, s, n.gws, wsf);
  }
  // each input voxel meets 4^3 taps per (ci, co) pair: 16x16 at 4^3, 16x8 at 8^3, 8x2 at 16^3
  ProfScope ps(c, MW_K_NN_CONV, 4.0 * Bd * (H + 2 * 2 * 16 * 512 + 2 * 8 * 4096 + kOut),
               2.0 * 64 * Bd * (16 * 16 * 64 + 16 * 8 * 512 + 8 * 2 * 4096));
  mwk::nn_convT_fwd(n.h2, th + n.oC1, th + n.oc1, n.a1, n.g1, B, 16, 16, 4, s);
  mwk::nn_convT_fwd(n.g1, th + n.oC2, th + n.oc2, n.a2, n.g2, B, 16, 8, 8, s);
  mwk::nn_convT_fwd(n.g2, th + n.oC3, th + n.oc3, n.y, nullptr, B, 8, 2, 16, s);
}

// loss against n.t and gradient into n.grad
static void nn_backward(Ctx* c, int B) {
  NnState& n = c->nn;
  const float* th = n.theta;
  float* g = n.grad;
  cudaStream_t s = c->stream;
  const double Bd = B, ni = n.n_in, H = kHid;
  {
    ProfScope ps(c, MW_K_NN_OTHER, 12.0 * Bd * kOut);
    mwk::nn_mse(n.y, n.t, (int64_t)B * kOut, n.dy, n.part, n.loss, s);
  }
  {
    // backward-data and backward-weight of each transposed convolution (twice the forward
    // flops; the first layer's input gradient is the reshaped dh2), ReLU masks between them
    ProfScope ps(c, MW_K_NN_CONV, 4.0 * Bd * (kOut + 3 * 2 * 8 * 4096 + 3 * 2 * 16 * 512 + 2 * H),
                 4.0 * 64 * Bd * (16 * 16 * 64 + 16 * 8 * 512 + 8 * 2 * 4096));
    mwk::nn_convT_bwd(n.g2, th + n.oC3, n.dy, n.dg2, g + n.oC3, g + n.oc3, B, 8, 2, 16, n.cpart, n.wpart, s);
    mwk::nn_relu_back(n.a2, n.dg2, n.da2, (int64_t)B * 8 * 4096, s);
    mwk::nn_convT_bwd(n.g1, th + n.oC2, n.da2, n.dg1, g + n.oC2, g + n.oc2, B, 16, 8, 8, n.cpart, n.wpart, s);
    mwk::nn_relu_back(n.a1, n.dg1, n.da1, (int64_t)B * 16 * 512, s);
    mwk::nn_convT_bwd(n.h2, th + n.oC1, n.da1, n.dh2, g + n.oC1, g + n.oc1, B, 16, 16, 4, n.cpart, n.wpart, s);
  }
  // dW2 = dz2^T h1, dh1 = dz2 W2 (BF16 W2), dW1 = dz1^T x; bias sums and ReLU masks between
  ProfScope ps(c, MW_K_NN_GEMM, 4.0 * H * (H + ni) + 2.0 * H * H + 4.0 * Bd * (ni + 6 * H) + 8.0 * H,
               2.0 * Bd * H * (2 * H + ni));
  mwk::nn_relu_back(n.z2, n.dh2, n.dz2, (int64_t)B * kHid, s);
  const size_t wsf = (size_t)32 * n.bcap * kHid;
  mwk::nn_gemm_f32(n.dz2, 1, kHid, n.h1, kHid, 1, nullptr, g + n.oW2, nullptr, kHid, kHid, B, s, n.gws, wsf);
  mwk::nn_colsum(n.dz2, B, kHid, g + n.ob2, s);
  mwk::nn_gemm_bf16(n.dz2, kHid, 1, n.W2b, kHid, 1, nullptr, n.dh1, nullptr, B, kHid, kHid, s, n.gws, wsf);
  mwk::nn_relu_back(n.z1, n.dh1, n.dz1, (int64_t)B * kHid, s);
  mwk::nn_gemm_f32(n.dz1, 1, kHid, n.x, n.n_in, 1, nullptr, g + n.oW1, nullptr, kHid, n.n_in, B, s, n.gws, wsf);
  mwk::nn_colsum(n.dz1, B, kHid, g + n.ob1, s);
}

mw_status mw_nn_init(mw_ctx* c, int32_t n_in, const float* theta) {
  return guard(c, [&] {
    require(n_in >= 1 && n_in <= (1 << 20) && theta, MW_EINVAL, "bad network arguments");
    nn_free(c);
    NnState& n = c->nn;
    n.n_in = n_in;
    n.np = mw_nn_param_count(n_in);
    int64_t o = 0;
    n.oW1 = o; o += (int64_t)kHid * n_in;
    n.ob1 = o; o += kHid;
    n.oW2 = o; o += (int64_t)kHid * kHid;
    n.ob2 = o; o += kHid;
    n.oC1 = o; o += 16 * 16 * 64;
    n.oc1 = o; o += 16;
    n.oC2 = o; o += 16 * 8 * 64;
    n.oc2 = o; o += 8;
    n.oC3 = o; o += 8 * 2 * 64;
    n.oc3 = o; o += 2;
    for (int64_t i = 0; i < n.np; ++i) require(std::isfinite(theta[i]), MW_EINVAL, "non-finite parameter");
    n.theta = upload(c, theta, n.np);
    n.grad = dalloc<float>(c, n.np);
    n.m = dalloc<float>(c, n.np);
    n.v = dalloc<float>(c, n.np);
    CK(cudaMemsetAsync(n.m, 0, sizeof(float) * n.np, c->stream));
    CK(cudaMemsetAsync(n.v, 0, sizeof(float) * n.np, c->stream));
    n.W1b = dalloc<uint16_t>(c, (size_t)kHid * n_in);
    n.W2b = dalloc<uint16_t>(c, (size_t)kHid * kHid);
    n.part = dalloc<double>(c, 256);
    n.loss = dalloc<double>(c, 1);
    nn_refresh_bf16(c);
    check_launch("nn init");
    CK(cudaStreamSynchronize(c->stream));
  });
}

mw_status mw_nn_get_params(mw_ctx* c, float* theta) {
  return guard(c, [&] {
    require(c->nn.theta && theta, MW_ESTATE, "network not initialised");
    CK(cudaMemcpyAsync(theta, c->nn.theta, sizeof(float) * c->nn.np, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  });
}

mw_status mw_nn_loss_grad(mw_ctx* c, int64_t nsamp, const float* x, const float* t, double* loss, float* grad) {
  return guard(c, [&] {
    NnState& n = c->nn;
    require(n.theta, MW_ESTATE, "network not initialised");
    require(nsamp >= 1 && nsamp <= 4096 && x && t && loss, MW_EINVAL, "bad arguments");
    nn_batch_buffers(c, (int)nsamp);
    CK(cudaMemcpyAsync(n.x, x, sizeof(float) * nsamp * n.n_in, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(n.t, t, sizeof(float) * nsamp * kOut, cudaMemcpyHostToDevice, c->stream));
    nn_forward(c, (int)nsamp);
    nn_backward(c, (int)nsamp);
    check_launch("nn loss/grad");
    CK(cudaMemcpyAsync(loss, n.loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (grad) CK(cudaMemcpyAsync(grad, n.grad, sizeof(float) * n.np, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  });
}

static uint64_t splitmix64_next(uint64_t& st) {
  st += 0x9E3779B97F4A7C15ull;
  uint64_t z = st;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

mw_status mw_nn_train(mw_ctx* c, const mw_nn_opts* o, int64_t nsamp, const float* x, const float* t,
                      mw_nn_stats* st) {
  return guard(c, [&] {
    NnState& n = c->nn;
    require(n.theta, MW_ESTATE, "network not initialised");
    require(o && nsamp >= 1 && x && t, MW_EINVAL, "bad training arguments");
    require(o->batch >= 1 && o->batch <= 4096 && o->epochs >= 0 && o->lr > 0, MW_EINVAL, "bad training options");
    for (auto p : {(void*)n.data_x, (void*)n.data_t}) dfree(c, p);
    n.data_x = upload(c, x, (size_t)nsamp * n.n_in);
    n.data_t = upload(c, t, (size_t)nsamp * kOut);
    n.data_n = nsamp;
    const int B = (int)std::min<int64_t>(o->batch, nsamp);
    nn_batch_buffers(c, B);
    std::vector<int32_t> perm(nsamp);
    cudaEvent_t e0;
    CK(cudaEventCreate(&e0));
    CK(cudaEventRecord(e0, c->stream));
    for (int ep = 0; ep < o->epochs; ++ep) {
      uint64_t rs = o->seed + 0x632BE59BD9B4E019ull * (uint64_t)(ep + 1);
      for (int64_t i = 0; i < nsamp; ++i) perm[i] = (int32_t)i;
      for (int64_t i = nsamp - 1; i > 0; --i) {                 // Fisher-Yates
        const int64_t j = (int64_t)(splitmix64_next(rs) % (uint64_t)(i + 1));
        std::swap(perm[i], perm[j]);
      }
      double ep_loss = 0;
      for (int64_t b0 = 0; b0 < nsamp; b0 += B) {
        const int nb = (int)std::min<int64_t>(B, nsamp - b0);
        CK(cudaMemcpyAsync(n.idx, perm.data() + b0, sizeof(int32_t) * nb, cudaMemcpyHostToDevice, c->stream));
        {
          ProfScope ps(c, MW_K_NN_OTHER, 8.0 * nb * ((double)n.n_in + kOut));
          mwk::nn_gather_rows(n.data_x, n.idx, nb, n.n_in, n.x, c->stream);
          mwk::nn_gather_rows(n.data_t, n.idx, nb, kOut, n.t, c->stream);
        }
        nn_forward(c, nb);
        nn_backward(c, nb);
        n.step++;
        {
          // Adam reads the parameters, gradient and both moments and writes three of them back;
          // the BF16 copies of W1 and W2 are refreshed from the new parameters
          ProfScope ps(c, MW_K_NN_OTHER,
                       28.0 * (double)n.np + 6.0 * (double)kHid * ((double)n.n_in + kHid));
          mwk::nn_adam(n.theta, n.grad, n.m, n.v, n.np, o->lr, o->beta1, o->beta2, o->eps, n.step, c->stream);
          nn_refresh_bf16(c);
        }
        double l = 0;
        CK(cudaMemcpyAsync(&l, n.loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));   // perm slice and loss are host memory
        ep_loss += l * nb;
      }
      check_launch("nn train");
      if (st && st->epoch_loss) st->epoch_loss[ep] = ep_loss / (double)nsamp;
    }
    CK(cudaEventRecord(c->ev1, c->stream));
    CK(cudaEventSynchronize(c->ev1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, c->ev1));
    cudaEventDestroy(e0);
    if (st) {
      st->epochs_run = o->epochs;
      st->seconds = ms * 1e-3;
    }
  });
}

mw_status mw_nn_infer(mw_ctx* c, int64_t nsamp, const float* x, float* y) {
  return guard(c, [&] {
    NnState& n = c->nn;
    require(n.theta, MW_ESTATE, "network not initialised");
    require(nsamp >= 1 && x && y, MW_EINVAL, "bad inference arguments");
    const int B = (int)std::min<int64_t>(nsamp, 256);
    nn_batch_buffers(c, B);
    for (int64_t b0 = 0; b0 < nsamp; b0 += B) {
      const int nb = (int)std::min<int64_t>(B, nsamp - b0);
      CK(cudaMemcpyAsync(n.x, x + b0 * n.n_in, sizeof(float) * nb * n.n_in, cudaMemcpyHostToDevice, c->stream));
      nn_forward(c, nb);
      CK(cudaMemcpyAsync(y + b0 * kOut, n.y, sizeof(float) * nb * kOut, cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
    }
    check_launch("nn infer");
  });
}

mw_status mw_nn_grid_to_tets(mw_ctx* c, const float* grid, int32_t G, const double* box, double* deps) {
  return guard(c, [&] {
    require(c->has_mesh && grid && box && deps && G >= 2 && G <= 1024, MW_EINVAL, "bad grid arguments");
    const int64_t T = c->topo.n_tet;
    float* dg = upload(c, grid, (size_t)2 * G * G * G);
    double* out = dalloc<double>(c, 2 * T);
    CK(cudaMemsetAsync(out, 0, sizeof(double) * 2 * T, c->stream));
    mwk::nn_grid_to_tets(dg, G, box, c->d_xyz, c->d_tets, T, out, c->stream);
    check_launch("grid to tets");
    CK(cudaMemcpyAsync(deps, out, sizeof(double) * 2 * T, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    dfree(c, dg);
    dfree(c, out);
  });
}


mw_status mw_selftest_bounded_wait(mw_ctx* c, int64_t spins, int32_t* code_out) {
  return guard(c, [&] {
    require(code_out && spins >= 1 && spins <= (int64_t)1 << 26, MW_EINVAL, "spins in [1, 2^26]");
    int32_t* d = dalloc<int32_t>(c, 1);
    CK(cudaMemsetAsync(d, 0xff, sizeof(int32_t), c->stream));
    mwk::bounded_wait_probe((long long)spins, d, c->stream);
    check_launch("bounded wait probe");
    CK(cudaMemcpyAsync(code_out, d, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    dfree(c, d);
  });
}

}  // extern "C"
