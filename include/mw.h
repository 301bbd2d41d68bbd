/*
 * libmw - GB300-native hot path of the microwave-tomography method of arXiv 2311.05322
 * ("Numerical Modeling for Shoulder Injury Detection Using Microwave Imaging").
 *
 * The library solves the time-harmonic Maxwell problem of Eq. (m1)/(m2) with lowest-order
 * Nedelec (Whitney) edge elements on tetrahedra (Sec. IV-D), one solve per transmitter, by
 * GMRES with a one-level ORAS domain-decomposition preconditioner (Sec. IV-C), computes the
 * S-matrix (dipole form of Eq. s1), the cost of Eq. (sahar:2), its adjoint gradient and an
 * L-BFGS inversion step (Sec. IV-D).  All arithmetic of these steps runs in the library's own
 * sm_103a kernels; the host side only validates, orchestrates and runs L-BFGS in FP64.
 *
 * Conventions
 *   - Every call returns an mw_status; MW_OK == 0.  No exception crosses the ABI.  On error,
 *     mw_last_error(ctx) holds a one-line message (valid until the next call on ctx).
 *   - Complex numbers are interleaved (re, im) pairs of double (or float where stated), layout
 *     compatible with C99 double _Complex and std::complex<double>.
 *   - Time convention e^{i omega t} (Sec. IV-B): lossy media have Im eps_r < 0.
 *   - Indices are int32_t, counts int64_t.  Host input arrays are owned by the caller and
 *     copied in before the call returns.  Device pointers are caller-owned CUDA allocations on
 *     the context's device.  The context owns every internal device buffer.
 *   - All device work is enqueued on the stream given to mw_create.  Calls that return host
 *     data synchronise that stream before returning; the others return after enqueueing.
 *   - A context is not thread-safe; use one context per host thread.
 *   - Edge numbering: a global edge is the vertex pair (lo, hi), lo < hi, numbered by
 *     lexicographic rank; local tet edges are (0,1) (0,2) (0,3) (1,2) (1,3) (2,3) and carry
 *     sign +1 when the local tail has the smaller global vertex id.  The matrix pattern holds
 *     every pair of edges sharing a tet, columns ascending.
 */
#ifndef MW_H
#define MW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t mw_status;
enum {
  MW_OK = 0,
  MW_EINVAL = 1,    /* invalid argument (null pointer, size or index out of range, bad mesh) */
  MW_ECUDA = 2,     /* a CUDA runtime call or kernel launch failed */
  MW_ENOMEM = 3,    /* device allocation failed (or would exceed the context's memory cap) */
  MW_ENOCONV = 4,   /* a solve stopped before reaching its tolerance; outputs hold the last iterate */
  MW_ETIMEOUT = 5,  /* a device-side bounded wait ran out; the kernel returned early */
  MW_ESTATE = 6,    /* call out of order (e.g. solve before assemble) */
  MW_ESINGULAR = 7  /* a subdomain matrix had a (near-)zero pivot */
};

typedef enum {
  MW_PREC_FP64 = 0,
  MW_PREC_FP32 = 1,
  MW_PREC_BF16 = 2,
  MW_PREC_SPARSE = 4,
  MW_PREC_SPARSE_BF16 = 5
} mw_precision;
typedef enum { MW_MODE_FP64 = 0, MW_MODE_MIXED = 1 } mw_mode;

typedef struct mw_ctx mw_ctx;

typedef struct {
  int64_t n_vert, n_tet, n_edge, n_face, n_bface, nnz;
} mw_mesh_info;

/* Options of one solve phase (GMRES(m) + ORAS, Sec. IV-C).
 *   mode      MW_MODE_FP64: FP64 everywhere (operator, preconditioner apply, Krylov basis).
 *             MW_MODE_MIXED: GMRES-IR - FP64 outer residual b - A x and update of x; inner
 *             flexible GMRES with FP32 operator and basis, preconditioner applied in the
 *             precision chosen at setup (BF16 on the tensor cores, or FP32), FP64 Hessenberg
 *             least squares.
 *   restart   Krylov dimension m per cycle (1..63).
 *   batch     columns per Krylov launch; 0 = all columns of a frequency in one block launch.
 *   max_it    cap on Arnoldi steps per column over the whole solve.
 *   tol       target FP64 true relative residual ||b - A x||_2 / ||b||_2 per column.
 *   inner_tol mixed mode: relative residual reduction asked of each inner cycle (default 1e-2:
 *             short inner cycles over a shallow basis; the outer FP64 residual decides
 *             convergence, so the result's tolerance does not depend on it).
 *   max_outer mixed mode: cap on outer refinement steps.
 *   use_precond 1 = ORAS (mw_setup_preconditioner first), 0 = unpreconditioned. */
typedef struct {
  int32_t mode;
  int32_t restart;
  int32_t batch;
  int32_t max_it;
  double tol;
  double inner_tol;
  int32_t max_outer;
  int32_t use_precond;
} mw_solve_opts;

/* Per-solve statistics.  iters/relres are optional caller arrays of n_cols entries. */
typedef struct {
  int32_t n_cols;          /* columns solved (n_freq * n_src) */
  int32_t n_converged;     /* columns with FP64 true relres <= tol */
  int32_t outer_steps;     /* outer residual evaluations */
  int32_t arnoldi_steps;   /* Arnoldi steps executed (max over columns of a launch, summed) */
  double max_relres;       /* largest final FP64 true relative residual */
  double solve_ms;         /* device time of the solve phase (CUDA events on the stream) */
  int32_t* iters;          /* [n_cols] Arnoldi steps per column, or NULL */
  double* relres;          /* [n_cols] final true relative residual per column, or NULL */
} mw_solve_stats;

/* ---- context ---------------------------------------------------------------------- */
/* Create a context on CUDA device `device`; all work goes to `cuda_stream` (a cudaStream_t,
 * NULL = the legacy default stream). */
mw_status mw_create(mw_ctx** ctx, int device, void* cuda_stream);
void mw_destroy(mw_ctx* ctx);
const char* mw_last_error(const mw_ctx* ctx);
/* Cap on the context's device allocations in bytes (0 = no cap).  Exceeding it gives MW_ENOMEM. */
mw_status mw_set_memory_cap(mw_ctx* ctx, int64_t bytes);
/* Restart cycles as CUDA graphs (default off).  With enable != 0, a Krylov cycle that may run all
 * `restart` steps is captured once (per frequency, block width, restart length, precision,
 * output buffer and profiler mask) and replayed with one launch and one host synchronisation
 * per cycle: each Arnoldi step's kernels sit in conditional graph nodes that run while a column
 * of the block is still active (Sec. IV-C's GMRES, unchanged arithmetic: same kernels, same
 * order, bit-identical results).  Capture is part of setup; a capture is dropped when a buffer
 * it names is freed (new mesh, preconditioner or workspace).  Every captured step slot costs a
 * few microseconds of conditional-node evaluation even when skipped, so cycles that stop well
 * before `restart` steps run faster eagerly.  enable = 0 (the default) runs cycles eagerly, with
 * a host check of the active-column count after every step, and frees the graphs. */
mw_status mw_set_graphs(mw_ctx* ctx, int32_t enable);

/* Launch-shape autotuner for the solve kernels (Sec. IV-C's GMRES + ORAS, arithmetic unchanged).
 * For one block shape (n_cols columns, solve mode, restart length) it times, with CUDA events on
 * the context stream and on pseudo-random inputs of the real operator and inverses, each accepted
 * launch shape of four kernels and keeps the fastest:
 *   tc_stages      pipeline depth of the BF16 tensor-core ORAS apply, 2..8 by shared memory
 *                  (only with a BF16 preconditioner in mixed mode);
 *   dots_stages    ring depth of the streaming Gram-Schmidt dots, 2..6 (16..128 columns);
 *   update_stages  ring depth of the streaming Gram-Schmidt update, 2..6 (16..128 columns);
 *   spmm_threads   threads per block of the row-per-warp SpMM, 128 / 256 / 512, or 1 for the
 *                  halo-tiled SpMM (FP32, even column counts).
 * None of these changes a result bit: the same arithmetic runs in the same order.  The choice is
 * kept per shape until the mesh or preconditioner changes.  Solves tune each new shape before
 * their timed phase while automatic tuning is on (mw_set_autotune, default on); mw_autotune
 * (re)tunes a shape now and reports it.  A value 0 means the kernel's default shape (and, in a
 * report, that the shape does not use the kernel). */
typedef struct {
  int32_t tc_stages, dots_stages, update_stages, spmm_threads;
} mw_launch_shapes;
enum { MW_TUNE_TC = 0, MW_TUNE_DOTS = 1, MW_TUNE_UPDATE = 2, MW_TUNE_SPMM = 3, MW_TUNE_NKERNEL = 4 };
typedef struct {
  int32_t n_cols, mode, restart;
  mw_launch_shapes chosen;
  int32_t n_cand[MW_TUNE_NKERNEL];   /* candidates timed per kernel (MW_TUNE_*) */
  int32_t cand[MW_TUNE_NKERNEL][8];  /* candidate values */
  double ms[MW_TUNE_NKERNEL][8];     /* mean device time per launch, ms */
} mw_tune_report;
mw_status mw_autotune(mw_ctx* ctx, int32_t n_cols, int32_t mode, int32_t restart, mw_tune_report* out);
/* Automatic tuning before the solve phase of each new block shape: enable != 0 (default) or 0
 * (default launch shapes; forgets tuned shapes). */
mw_status mw_set_autotune(mw_ctx* ctx, int32_t enable);
/* Pins the launch shapes of one block shape (ranges as above, 0 = the kernel's default), replacing
 * any tuned choice until the mesh or preconditioner changes.  Takes effect while automatic tuning
 * is on.  MW_EINVAL for a value outside its range. */
mw_status mw_set_launch_shapes(mw_ctx* ctx, int32_t n_cols, int32_t mode, int32_t restart,
                               const mw_launch_shapes* shapes);

/* ---- mesh (Sec. IV-A; Nedelec r = 1, Sec. IV-D) ------------------------------------- */
/* xyz [n_vert][3] metres; tet_vert [n_tet][4] vertex ids (any orientation, non-degenerate).
 * Builds the canonical edges, signs, faces, the CSR pattern and the assembly maps on the
 * host, uploads them and computes the element matrices on the GPU.  Fills *out. */
mw_status mw_set_mesh(mw_ctx* ctx, int64_t n_vert, const double* xyz, int64_t n_tet,
                      const int32_t* tet_vert, mw_mesh_info* out);
/* Copies of the topology (any pointer may be NULL): edge_vert [E][2] (lo < hi), tet_edge
 * [T][6], tet_sign [T][6], row_ptr [E+1], col_idx [nnz]. */
mw_status mw_get_topology(mw_ctx* ctx, int32_t* edge_vert, int32_t* tet_edge, int8_t* tet_sign,
                          int64_t* row_ptr, int32_t* col_idx);
/* Element matrices from the GPU (parity hook): K, M [T][6][6] and volumes [T] (any may be NULL). */
mw_status mw_get_element_matrices(mw_ctx* ctx, double* K, double* M, double* vol);

/* ---- assembly, Eq. (m2) with k^2 = k0^2 eps_r ---------------------------------------- */
/* A_f = K - k0_f^2 sum_T eps_T M^T + i k0_f sqrt(eps_bg) B for each frequency (Hz);
 * eps_r [n_tet][2] (re, im), eps_bg[2].  Re-run whenever eps changes.  With boundary classes
 * (mw_set_ports) B keeps only the open faces, port faces add i beta_p B^F, and metal edges
 * have identity rows and columns. */
mw_status mw_assemble(mw_ctx* ctx, int32_t n_freq, const double* freq_hz, const double* eps_r,
                      const double* eps_bg);
/* Values of A_f in the canonical pattern, host complex128 [nnz] (parity hook). */
mw_status mw_get_matrix(mw_ctx* ctx, int32_t f, double* values);
/* Y = A_f X on the device for n_cols columns, layout [E][n_cols] (column fastest),
 * complex128 (prec = MW_PREC_FP64, FP64 arithmetic) or complex64 (MW_PREC_FP32, FP32); prec = 3
 * takes complex128 in and out and computes in double-float arithmetic on the FP32 pipes (the
 * mixed solver's outer residual); prec = 4 is the FP32 product of the halo-tiled kernel (rows
 * in Morton-ordered blocks whose columns of X are staged in shared memory; even n_cols, x
 * 16-byte aligned), bit-identical to MW_PREC_FP32; prec = 5 takes x as complex BF16 pairs (4 bytes
 * per value, real in the low half) and writes complex64 y, equal to MW_PREC_FP32 applied to the
 * widened x. */
mw_status mw_apply_matrix(mw_ctx* ctx, int32_t f, int32_t prec, const void* x_dev, void* y_dev,
                          int32_t n_cols);

/* ---- sources (volume-source reading of Eq. m1) ----------------------------------------- */
/* z-directed dipoles: pos/dir [n_src][3].  Each maps to the z-directed edge whose midpoint is
 * nearest (ties: lowest edge id); outputs (optional) the edge and its sign (+1 when the
 * edge lo -> hi points along dir).  RHS b_j = -i omega mu0 s_j e_edge(j), S_ij = s_i x_j[edge_i].
 * Replaces port sources (port faces keep their boundary term). */
mw_status mw_set_sources(mw_ctx* ctx, int32_t n_src, const double* pos, const double* dir,
                         int32_t* src_edge_out, int8_t* src_sign_out);

/* ---- waveguide ports and metal walls (Eq. m1-m2 boundary terms, Eq. s1) --------------- */
/* A rectangular waveguide port on the outer boundary.  Its TE10 mode is
 *   E_p(x) = sin(pi ((x - origin) . u) / a) v,
 * with propagation constant beta_p = -i sqrt((pi / a)^2 - k0^2 eps_fill) (principal root, so
 * Im beta <= 0, and beta > 0 above cut-off in a lossless filling). */
typedef struct mw_port {
  double origin[3];   /* corner of the aperture (m) */
  double u[3];        /* unit broad-side direction: the mode varies along u over [0, a] */
  double v[3];        /* unit narrow-side direction: the mode's field points along v */
  double a;           /* broad-side width (m), > 0 */
  double eps_fill[2]; /* relative permittivity filling the guide (re, im), im <= 0 */
} mw_port;
/* Boundary classes of Eq. (m1) (Sec. IV-B).  face_vert [n_face][3] lists faces by vertex ids
 * (any order) and face_label [n_face] gives each a class:
 *   -1           metal (Gamma_m), any face of the mesh: every edge of the face is removed from
 *                the unknowns (kept as an identity row and column with zero right-hand side,
 *                so every field is zero there);
 *   p in [0, n)  port p (Gamma_t while p transmits, Gamma_r while it receives), boundary faces
 *                only: face term i beta_p B^F in place of the open one.
 * Unlisted boundary faces stay open (Gamma_o, i k0 sqrt(eps_bg) B^F).  With n_port >= 1 the
 * ports become the transmitters and receivers, replacing any dipoles (Eq. m2 and Eq. s1):
 *   b_j = 2 i beta_j w_j,   w_j,e = int_{port j} E_j . N_e   (g = 2 i beta E^TE10),
 *   S_ij = w_i^T x_j / n_i,   n_i = int_{port i} |E_i|^2,
 * the face integrals by a 10 x 10 collapsed Gauss-Legendre rule per face, on the GPU.
 * n_port = 0 sets metal faces only and keeps dipole sources.  Call after mw_set_mesh; it
 * drops the assembled matrices, the preconditioner and stored fields (assemble again).
 * Errors: MW_ESTATE without a mesh; MW_EINVAL for a vertex out of range, a listed triple
 * that is not a face of the mesh, a port face that is not a boundary face, a face listed twice
 * with different labels, a label out of range, a port without faces, a <= 0, u / v not
 * orthonormal, a non-finite value, or eps_fill with im > 0. */
mw_status mw_set_ports(mw_ctx* ctx, int32_t n_port, const mw_port* ports, int64_t n_face,
                       const int32_t* face_vert, const int32_t* face_label);
/* Port load vectors and norms (parity hook): W host [E][n_port] (w_p, zero on metal edges and
 * away from port p) and norms [n_port]; either may be NULL.  MW_ESTATE unless ports are the
 * current sources. */
mw_status mw_get_port_vectors(mw_ctx* ctx, double* W, double* norms);

/* ---- ORAS preconditioner (Sec. IV-C) ------------------------------------------------ */
/* tet_part [n_tet] in [0, n_sub); overlap_layers >= 0 vertex-neighbour layers; inv_prec
 * selects the stored precision of the subdomain inverses (FP64: FP64 factorisation, applied
 * in FP64; FP32: FP32 factorisation, FP32 apply; BF16: FP32 factorisation, BF16 tensor-core
 * apply).  MW_PREC_SPARSE keeps no dense inverse: each subdomain matrix is factorised as a
 * multifrontal LU on a nested-dissection tree (FP32, no pivoting), and the apply runs its
 * forward and backward sweeps on the GPU (mixed-precision solves only).  Its memory grows like
 * n_s^(4/3) per subdomain instead of n_s^2, so subdomains of 1e5 unknowns are practical.
 * MW_PREC_SPARSE_BF16 factorises the same way, then stores the factor blocks as BF16 tiles and
 * runs the sweeps' products on the tensor cores (tcgen05, FP32 accumulation and FP32 vectors). */
/* Builds for every assembled frequency from the current eps.  MW_ESINGULAR when a pivot
 * block is numerically singular. */
mw_status mw_setup_preconditioner(mw_ctx* ctx, int32_t n_sub, const int32_t* tet_part,
                                  int32_t overlap_layers, int32_t inv_prec);
/* Host-only check of the sparse subdomain plan (no context, no GPU): builds the topology, the
 * subdomains and the nested-dissection multifrontal structure that MW_PREC_SPARSE would use
 * with the given leaf size, and verifies its invariants (every dof a pivot exactly once, fronts
 * of padded pivots plus update dofs, each child's update dofs found in its parent's front at the
 * rows its map names, roots without update dofs, assembly targets inside the workspace).
 * stats[6] receives: tree nodes, tree height, largest front, factor entries, largest workspace
 * (entries), and sum_s n_s^2 (the dense inverses' entries).  MW_ECUDA reports a broken
 * invariant; MW_EINVAL bad arguments. */
mw_status mw_sparse_plan_stats(int64_t n_vert, const double* xyz, int64_t n_tet, const int32_t* tet_vert,
                               int32_t n_sub, const int32_t* tet_part, int32_t overlap_layers, int32_t leaf,
                               int64_t* stats);
/* Host-only check of the halo-tiled SpMM plan (no context, no GPU): builds the topology and the
 * plan mw_set_mesh uses (rows in the Morton order of their edge midpoints, cut into blocks whose
 * column sets hold at most halo_max edges) and verifies its invariants: every row once, blocks
 * in order, each block's halo ascending and within bound, each blocked nonzero mapped to the
 * canonical nonzero of its row in the same order, and every halo-local column naming that
 * nonzero's column; with halo_max = 480 (the library's bound) also the library's block bounds of
 * 512 rows and 4096 nonzeros.  stats[4] receives: blocks, summed halo sizes, largest halo,
 * nonzeros.
 * MW_ECUDA reports a broken invariant; MW_EINVAL bad arguments (64 <= halo_max <= 65535). */
mw_status mw_spmm_plan_stats(int64_t n_vert, const double* xyz, int64_t n_tet, const int32_t* tet_vert,
                             int32_t halo_max, int64_t* stats);
/* z = M_f^{-1} r on the device, complex128 [E][n_cols] in and out (parity hook).  Returns
 * after the apply has completed; MW_ETIMEOUT when a bounded wait of the tensor-core apply ran
 * out (z is then incomplete). */
mw_status mw_apply_preconditioner(mw_ctx* ctx, int32_t f, const void* r_dev, void* z_dev,
                                  int32_t n_cols);
/* Parity hook of the Arnoldi orthogonalisation's first half (GMRES, Sec. IV-C; Hermitian
 * inner product): h[i][c] = sum_rows conj(V_i[row][c]) w[row][c] for i < nvec, computed by the
 * same kernels as the mixed-precision solves (streaming bulk-copy kernel for 16..128 columns on
 * 16-byte aligned vectors, FP32 products summed in FP32 within a row tile, FP64 across tiles
 * and blocks, fixed reduction order).  V_dev: device complex64, vector i at V_dev + i*vstride
 * elements, each [n_rows][n_cols] with the column fastest; w_dev the same shape.  h_out: host
 * complex128 [nvec][n_cols].  1 <= nvec <= 64, 1 <= n_cols <= 128.  Synchronises; allocates
 * temporary device memory; MW_ETIMEOUT when a bounded wait ran out. */
mw_status mw_krylov_dots(mw_ctx* ctx, int32_t nvec, const void* V_dev, int64_t vstride, const void* w_dev,
                         int64_t n_rows, int32_t n_cols, double* h_out);
/* z = M_f^{-1} r with no device allocation.  The paper has no counterpart: this is an
 * integration aid.  It is for callers that cannot allocate device memory when they apply the
 * preconditioner, for example because another framework holds the device heap, because the
 * code must not allocate after initialisation, or because an allocation would synchronise the
 * device at that point.  Needs a BF16 (tensor-core) preconditioner.  r_dev / z_dev: device
 * complex64 [E][n_cols] (column fastest), 1 <= n_cols <= 128; z receives every row.
 * Scratch: the gathered operand lives in one fixed device array of 16 MiB that the library
 * holds on each GPU until the process exits; a call whose operand would exceed it returns
 * MW_EINVAL with the sizes.  The first call on a device looks the array's address up on that
 * device; make that first call before any stream capture.  All calls share the array, so calls
 * that overlap on the GPU (different streams or contexts without ordering) race; order them.
 * Returns after the apply has completed on the context's stream (it reads the apply's
 * bounded-wait error word); MW_ETIMEOUT when a wait ran out, z then being incomplete. */
mw_status mw_apply_preconditioner_noalloc(mw_ctx* ctx, int32_t f, const void* r_dev, void* z_dev,
                                          int32_t n_cols);
/* Owner subdomain of each edge [E] and unknowns per subdomain [n_sub] (either may be NULL). */
mw_status mw_get_partition(mw_ctx* ctx, int32_t* edge_owner, int32_t* sub_size);

/* ---- solves -------------------------------------------------------------------------- */
/* Forward solves for all n_freq * n_src source columns (column c = f * n_src + j).
 * fields_dev: NULL, or device complex128 [n_cols][E] receiving the fields.
 * S: NULL, or host complex128 [n_freq][n_src][n_src], S[f][i][j] = w_i^T x_{f,j} / n_i
 * (dipoles: p_i^T x_{f,j}; ports: the Eq. s1 projection, see mw_set_ports).
 * Returns MW_ENOCONV if some column missed tol (outputs then hold the last iterate). */
mw_status mw_solve(mw_ctx* ctx, const mw_solve_opts* opts, void* fields_dev, double* S,
                   mw_solve_stats* stats);
/* Solve A_f x = b for arbitrary right-hand sides: b_dev/x_dev device complex128
 * [n_freq][n_cols][E] (n_cols per frequency). */
mw_status mw_solve_rhs(mw_ctx* ctx, const mw_solve_opts* opts, int32_t n_cols, const void* b_dev,
                       void* x_dev, mw_solve_stats* stats);

/* ---- cost and gradient (Eq. sahar:2, Sec. IV-D) ------------------------------------- */
/* Forward solve, cost J = 1/2 sum w |S - S_obs|^2 + alpha R with w = 1/|S_empty|^2, adjoint
 * solve with sources c_ij = w_ij conj(S_ij - S_obs_ij), per-tet gradient
 * dJ/dRe eps_T = sum_f k0_f^2 Re G_T, dJ/dIm eps_T = -sum_f k0_f^2 Im G_T,
 * G_T = sum_j lambda_j^T M^T x_j, plus alpha dR (face-jump Tikhonov).
 * S_obs, S_empty host complex128 [n_freq][n_src][n_src]; grad host [n_tet][2] (may be NULL);
 * S_out (may be NULL) receives the forward S. */
mw_status mw_gradient(mw_ctx* ctx, const mw_solve_opts* opts, const double* S_obs,
                      const double* S_empty, double alpha, double* J_out, double* grad,
                      double* S_out);
/* Tikhonov term R and alpha-free gradient dR [n_tet][2] for eps [n_tet][2] (device kernel). */
mw_status mw_tikhonov(mw_ctx* ctx, const double* eps_r, double* R_out, double* grad);

/* ---- L-BFGS (Sec. IV-D) ------------------------------------------------------------ */
typedef struct {
  int32_t m;            /* history pairs (8) */
  int32_t max_it;       /* iterations */
  double c1;            /* Armijo constant (1e-4) */
  int32_t max_ls;       /* backtracking trials (10) */
  double first_step;    /* first step scaled so max_k |d_k| = first_step (1.0) */
  double alpha;         /* Tikhonov weight */
  double target_J;      /* stop once J <= target_J (0 = off) */
} mw_inv_opts;

typedef struct {
  int32_t iterations;    /* accepted iterates */
  int32_t evaluations;   /* cost+gradient evaluations */
  double* J;             /* [max_it + 1] cost per accepted iterate (J[0] at the start), or NULL */
  double* seconds;       /* [max_it + 1] wall time at each accepted iterate, or NULL */
} mw_inv_history;

/* Reverse-communication L-BFGS on a host vector x[n] (FP64): create, then call step with the
 * cost f and gradient g at the x it last asked for.  *request = 1: evaluate at x (written into
 * x_io); 0: converged or stopped, x_io holds the final iterate. */
typedef struct mw_lbfgs mw_lbfgs;
mw_status mw_lbfgs_create(mw_lbfgs** st, int64_t n, const mw_inv_opts* opts);
mw_status mw_lbfgs_step(mw_lbfgs* st, double* x_io, double f, const double* g, int32_t* request);
void mw_lbfgs_destroy(mw_lbfgs* st);
/* Full inversion: L-BFGS over [Re eps; Im eps] with mw_assemble + mw_gradient per
 * evaluation; eps_inout [n_tet][2].  The preconditioner set up before the call is reused. */
mw_status mw_invert(mw_ctx* ctx, const mw_inv_opts* opts, const mw_solve_opts* sopts,
                    const double* S_obs, const double* S_empty, double* eps_inout,
                    mw_inv_history* hist);

/* ---- learned initialiser (the paper has no learned part) -------------------------------- */
/* Network: x [n_in] -> relu(W1 x + b1) -> relu(W2 . + b2) (1024 wide) -> reshape 16x4x4x4 ->
 * convT(16->16) -> relu -> convT(16->8) -> relu -> convT(8->2) -> [2][32][32][32] (Re, Im of
 * Delta eps on a grid); convT = 3D transposed convolution, kernel 4, stride 2, padding 1.
 * W1 and W2 are applied in BF16, every sum accumulates in FP32.  Parameters are one flat FP32
 * vector: W1 [1024][n_in], b1, W2 [1024][1024], b2, C1 [16][16][4][4][4], c1, C2 [16][8][..],
 * c2, C3 [8][2][..], c3.  Initial values are the caller's (random draws stay outside). */
typedef struct {
  int32_t batch;       /* minibatch size */
  int32_t epochs;
  float lr, beta1, beta2, eps;   /* Adam */
  uint64_t seed;       /* splitmix64 seed of the per-epoch shuffles */
} mw_nn_opts;
typedef struct {
  int32_t epochs_run;
  double* epoch_loss;  /* [epochs] mean training loss per epoch, or NULL */
  double seconds;      /* device time of the training loop */
} mw_nn_stats;
/* Number of parameters for an input width (-1 if invalid). */
int64_t mw_nn_param_count(int32_t n_in);
/* (Re)create the network with parameters theta (host FP32, copied). Resets Adam. */
mw_status mw_nn_init(mw_ctx* ctx, int32_t n_in, const float* theta);
mw_status mw_nn_get_params(mw_ctx* ctx, float* theta);
/* Mean-squared-error loss of the network on n samples (x [n][n_in], t [n][2][32][32][32], host)
 * and its gradient with respect to the parameters (host, may be NULL). */
mw_status mw_nn_loss_grad(mw_ctx* ctx, int64_t n, const float* x, const float* t, double* loss, float* grad);
/* Minibatch Adam training on n samples (host arrays, copied to the device once). */
mw_status mw_nn_train(mw_ctx* ctx, const mw_nn_opts* opts, int64_t n, const float* x, const float* t,
                      mw_nn_stats* stats);
/* Network outputs y [n][2][32][32][32] for inputs x [n][n_in] (host). */
mw_status mw_nn_infer(mw_ctx* ctx, int64_t n, const float* x, float* y);
/* Average of a cell-centred grid [2][G][G][G] over box {lo x,y,z, hi x,y,z} on each tet of the
 * context's mesh: the mean of its trilinear interpolant (0 outside the box) over the 35 points of
 * the order-4 barycentric lattice of the tet; deps [n_tet][2] (host). */
mw_status mw_nn_grid_to_tets(mw_ctx* ctx, const float* grid, int32_t G, const double* box, double* deps);

/* How mw_gradient / mw_gradient_dev / mw_invert obtain the adjoint fields (Sec. IV-D):
 *   MW_ADJOINT_SOLVE (default): one adjoint solve per transmitter column, A lambda_j =
 *     sum_i (c_ij / n_i) w_i, with the same solver and preconditioner as the forward solves;
 *   MW_ADJOINT_RECIPROCAL: the receivers are the transmitters and A = A^T, so
 *     lambda_j = sum_i c_ij / (n_i coef_i) x_i exactly (coef_i the source coefficient of
 *     transmitter i), formed from the forward fields in FP64 without any adjoint solve.  The
 *     gradient is the same up to the forward solves' tolerance.
 * MW_EINVAL for another value. */
enum { MW_ADJOINT_SOLVE = 0, MW_ADJOINT_RECIPROCAL = 1 };
mw_status mw_set_adjoint_mode(mw_ctx* ctx, int32_t mode);

/* Storage of the preconditioned vectors z_j = M^-1 v_j of the inner FGMRES cycles when the
 * preconditioner is the BF16 tensor-core apply (MW_APPLY_TC; elsewhere it has no effect):
 *   1 (default): complex BF16 pairs, 4 bytes per value, written by the apply's epilogue and
 *     widened to FP32 where they are read (the SpMM A z_j and the update x += Z y);
 *   0: complex FP32, 8 bytes per value.
 * Flexible GMRES takes the stored z_j as they are in both places, so the rounding only perturbs
 * the preconditioner (already a BF16 product); the Arnoldi relation and the FP64 outer residual
 * are unchanged.  The paper has no counterpart (its preconditioned vectors are FP64).  Drops the
 * captured solve graphs when the setting changes.  MW_EINVAL for another value. */
mw_status mw_set_z_storage(mw_ctx* ctx, int32_t bf16);

/* Schedule of the BF16 tensor-core sweeps of MW_PREC_SPARSE_BF16 (Sec. IV-C's subdomain solves;
 * elsewhere no effect).  1 (default): each sweep launch runs persistent CTAs that take its
 * 128-row output tiles in turn, with one copy ring across their tiles and the accumulators
 * double-buffered in tensor memory, so one tile's epilogue overlaps the next tile's copies and
 * MMAs (up to 64 columns; wider blocks use the other schedule); 0: one CTA per tile.  The same
 * products in the same order either way: bit-identical results.  MW_EINVAL for another value. */
mw_status mw_set_sweep_schedule(mw_ctx* ctx, int32_t persistent);

/* ---- column-sharded evaluation (one evaluation split over processes by transmitters) ---
 * The transmitter columns of an evaluation are independent until the cost: process r solves
 * its own window of columns (mw_forward_cols), the S columns of all windows are all-gathered
 * by the caller (each process needs the whole S for the cost of Eq. sahar:2 and the adjoint
 * weights), every process solves the adjoints of its own window and forms that window's part of
 * the per-tet gradient (mw_gradient_cols), and the caller all-reduces (sums) the parts.  The
 * sum equals mw_gradient's data gradient; the Tikhonov term (mw_tikhonov) is added once. */
/* Forward solves of transmitters j0 .. j0+n_cols-1 (all assembled frequencies), kept for the
 * next mw_gradient_cols; S_cols: host complex128 [n_freq][n_src][n_cols], the S-matrix columns
 * of the window (Eq. s1: every receiver i, window column j).  1 <= n_cols <= 128, j0 + n_cols
 * <= n_src.  Synchronises. */
mw_status mw_forward_cols(mw_ctx* ctx, const mw_solve_opts* opts, int32_t j0, int32_t n_cols, double* S_cols);
/* For the window of the last mw_forward_cols (same eps): J_out = the data cost of the whole
 * S_full (host complex128 [n_freq][n_src][n_src], the gathered S), the adjoint solves of the
 * window's columns with c_ij = w_ij conj(S_full_ij - S_obs_ij), and grad_part (host [n_tet][2])
 * = that window's share of dJ/d(Re eps, Im eps).  MW_ESTATE without a prior window.
 * Synchronises. */
mw_status mw_gradient_cols(mw_ctx* ctx, const mw_solve_opts* opts, const double* S_full, const double* S_obs,
                           const double* S_empty, double* J_out, double* grad_part);

/* ---- device-resident variants (same operations, device pointers) ------------------- */
/* mw_assemble with eps_r on the device ([n_tet][2] doubles); needs a prior mw_assemble with the
 * same number of frequencies (which sized the matrices). */
mw_status mw_assemble_dev(mw_ctx* ctx, int32_t n_freq, const double* freq_hz, const void* eps_dev,
                          const double* eps_bg);
/* mw_gradient with S_obs / S_empty on the device and the gradient [n_tet][2] written to the
 * device; the cost J is returned to the host. */
mw_status mw_gradient_dev(mw_ctx* ctx, const mw_solve_opts* opts, const void* S_obs_dev,
                          const void* S_empty_dev, double alpha, double* J_out, void* grad_dev);

/* ---- diagnostics ------------------------------------------------------------------- */
/* Self-test of the device-side bounded waits used by the tensor-core kernels: one thread waits
 * on an mbarrier whose phase never completes, gives up after `spins` polls and writes
 * MW_ETIMEOUT into *code_out (0 would mean the phase completed).  The context stays usable. */
mw_status mw_selftest_bounded_wait(mw_ctx* ctx, int64_t spins, int32_t* code_out);
/* Kernel launches issued by this library in the process so far. */
int64_t mw_kernel_launches(void);
/* Kernel classes timed by the optional event profiler. */
enum {
  MW_K_SPMM = 0,        /* Arnoldi SpMM (K3) */
  MW_K_ORAS = 1,        /* ORAS apply (K4) */
  MW_K_CGS_DOTS = 2,    /* Gram-Schmidt dot products and their reduction (K6) */
  MW_K_CGS_UPDATE = 3,  /* Gram-Schmidt update and norm (K6) */
  MW_K_RESIDUAL = 4,    /* FP64 residual b - A x (K8) */
  MW_K_REASSEMBLE = 5,  /* eps -> A_f reassembly and the double-float split of A_f (K2) */
  MW_K_GRADIENT = 6,    /* per-tet adjoint gradient (K11) */
  MW_K_FACTOR = 7,      /* ORAS subdomain inverses: blocked Gauss-Jordan (K5 setup) */
  MW_K_NN_GEMM = 8,     /* learned initialiser: dense layers, forward and backward (K13) */
  MW_K_NN_CONV = 9,     /* learned initialiser: transposed convolutions, forward and backward (K14) */
  MW_K_NN_OTHER = 10,   /* learned initialiser: loss, activations, bias sums, Adam, batch gathers */
  MW_K_NCLASS = 11
};
/* Record CUDA events around the launches of the classes in mask (bit k = class k); 0 = off.
 * Events cost a few microseconds each. */
mw_status mw_profile_enable(mw_ctx* ctx, uint32_t class_mask);
/* Per class since enable: summed durations (ms), launch count, algorithmic bytes (the bytes
 * each launch must move at minimum: operands read once, results written once) and algorithmic
 * floating-point operations (real flops of the defining arithmetic, 0 for classes rated by
 * bytes); bytes and flops may be NULL; arrays of MW_K_NCLASS entries; resets the counters. */
mw_status mw_profile_read(mw_ctx* ctx, double* ms, int64_t* launches, double* bytes, double* flops);

#ifdef __cplusplus
}
#endif
#endif /* MW_H */
