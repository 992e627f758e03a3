/*
 * nnmg.h - C ABI of the GB300-native non-nested geometric multigrid library.
 *
 * The library solves the Poisson problem -lap u = f, u = 0 on the Dirichlet boundary, or
 * linear elasticity (option pde, Sec. 6.3), discretised by continuous Lagrange P1/P2
 * elements on simplicial meshes (triangles, tetrahedra), with the V-cycle of Chen & Wells,
 * "Multigrid on unstructured meshes with regions of low quality cells" (arXiv:2402.12947):
 *   - non-nested levels Omega_1 (finest) .. Omega_L, interpolation prolongation
 *     [P_l]_ij = phi_j^(l+1)(x_i), R_l = P_l^T, Galerkin A_{l+1} = P_l^T A_l P_l (Sec. 2);
 *   - the global-local combined smoother S_gc (Sec. 4.2): local residual correction S_c on
 *     the patches around low-quality cells (Sec. 4.1, Alg. 2, patches per Sec. 4.4), a
 *     Jacobi-preconditioned Chebyshev global smoother S_g (Sec. 3.2) with the adjusted
 *     largest eigenvalue (Sec. 5), or multicolour symmetric Gauss-Seidel, then S_c again;
 *   - the V-cycle of Alg. 1 and, as in Sec. 6.2, CG preconditioned by one V-cycle.
 *
 * Conventions shared by every call:
 *   - Levels are numbered 0 (finest, the paper's Omega_1) .. L-1 (coarsest).
 *   - Vectors live on the free DoFs of a level, in the library's numbering: vertices in
 *     the caller's vertex order, then (P2) one DoF per edge with edges in lexicographic
 *     order of their sorted vertex pair; Dirichlet DoFs are removed, order kept. Local
 *     DoF order inside a cell: vertices, then edges (0,1),(0,2),(1,2) in 2D and
 *     (0,1),(0,2),(0,3),(1,2),(1,3),(2,3) in 3D.
 *   - Dirichlet DoFs: vertices on a boundary facet (a facet of exactly one cell) allowed
 *     by the optional vertex mask; an edge DoF is Dirichlet when its edge lies in a
 *     boundary facet and both of its vertices are Dirichlet.
 *   - Pointers named *_dev are device pointers (cudaMalloc / PyTorch CUDA memory) owned
 *     by the caller; *_host pointers are host memory owned by the caller. The library
 *     copies every host input it keeps; the hierarchy owns all device memory it allocates.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Compute calls are asynchronous on that stream unless stated otherwise.
 *   - Every call returns an mg_status code; on failure, mg_last_error(h) (or
 *     mg_last_error(NULL) after a failed setup) returns a message. Nothing aborts the
 *     process and no call traps the GPU.
 *   - Index limits: free DoFs and nonzeros per level must be < 2^31.
 */
#ifndef NNMG_H
#define NNMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum mg_status {
  MG_OK = 0,
  MG_ERR_INVALID_ARG = 1,     /* bad pointer, size, level index or option */
  MG_ERR_DEGENERATE_CELL = 2, /* a cell of zero volume (gamma = 0) */
  MG_ERR_POINT_LOCATION = 3,  /* a fine DoF point lies in no coarse cell (tolerance 1e-12) */
  MG_ERR_NOT_SPD = 4,         /* a patch matrix or the coarsest matrix failed Cholesky */
  MG_ERR_NO_CONVERGENCE = 5,  /* maxit reached; the info struct is still filled */
  MG_ERR_BREAKDOWN = 6,       /* CG breakdown: p^T A p <= 0 or a non-finite scalar */
  MG_ERR_OOM = 7,             /* device or host allocation failed */
  MG_ERR_CUDA = 8,            /* a CUDA runtime error (message has the CUDA text) */
  MG_ERR_TIMEOUT = 9,         /* a bounded device-side wait gave up */
  MG_ERR_NO_DEVICE = 10       /* compute call on a hierarchy built with host_only = 1 */
};

/* Smoother order (option `smoother`). */
enum mg_smoother {
  MG_SMOOTHER_SANDWICH = 0,          /* S_c, S_g, S_c on both sides (Sec. 4.2) */
  MG_SMOOTHER_GLOBAL_THEN_LOCAL = 1, /* pre: S_g then S_c; post: S_c then S_g */
  MG_SMOOTHER_GLOBAL = 2             /* S_g only (no local correction) */
};

/* Global smoother S_g (option `global_smoother`). */
enum mg_global_smoother {
  MG_GLOBAL_CHEBYSHEV = 0, /* Chebyshev on D^-1 A, cheb_degree steps (Sec. 3.2) */
  MG_GLOBAL_SGS = 1        /* symmetric Gauss-Seidel (Sec. 3.1 and Sec. 6 experiments), in
                              the multicolour form: rows greedily coloured in library index
                              order, ignoring couplings |a_ij| <= 1e-12 sqrt(a_ii a_jj); one
                              application sweeps the colours 0..C-1 then C-1..0, each colour's
                              rows at once (x_i = (b_i - sum_{j != i} a_ij x_j) / a_ii). No
                              lambda_max is computed. */
};

/* Operator assembled on level 0 by mg_setup (option `pde`). */
enum mg_pde {
  MG_PDE_POISSON = 0,     /* -lap u = f, P1/P2 (Sec. 6.1-6.2) */
  MG_PDE_ELASTICITY = 1   /* -div sigma(u) = f, sigma = 2 mu eps(u) + lambda tr(eps(u)) I with
                             mu = E / (2 (1 + nu)), lambda = E nu / ((1 + nu)(1 - 2 nu))
                             (Sec. 6.3); vector P1/P2, DoF dim*k + c = component c of scalar
                             DoF k (components interleaved); P acts componentwise (P (x) I);
                             patches hold every component of their nodes; a Dirichlet node
                             is clamped in every component */
};

/* Device-internal DoF order of the smoothed levels (option `reorder`). Column indices are
 * stored as 16-bit offsets from a per-slice (per-row) base wherever the slice spans fewer
 * than 2^16 columns, so orders that keep neighbours close in index shrink the matrix. */
enum mg_reorder {
  MG_REORDER_NONE = 0,    /* the library numbering */
  MG_REORDER_RCM = 1,     /* reverse Cuthill-McKee of the matrix graph */
  MG_REORDER_SPATIAL = 2, /* Z-order (Morton) of the DoF points, vertex and edge DoFs
                             interleaved; the library numbering where a level has no points
                             (mg_setup_csr) */
  MG_REORDER_SPATIAL_COARSE = 3  /* MG_REORDER_SPATIAL on every level but the finest, which
                                    keeps the library numbering */
};

/* Arithmetic of the V-cycle (option `precision`). */
enum mg_precision {
  MG_PREC_FP64 = 0,   /* everything in FP64 */
  MG_PREC_MIXED = 1   /* V-cycle SpMVs/transfers/Chebyshev in FP32 (int32 indices) inside
                         FP64 CG; patch solves, patch residuals and the coarsest solve FP64 */
};

typedef struct mg_hierarchy mg_hierarchy_t;

/* One mesh level (Sec. 2: a triangulation Omega_l of the same domain; levels need not be
 * nested but must share the boundary). coords [nv*dim] (x,y[,z] per vertex), cells
 * [nc*(dim+1)] vertex ids (either orientation). dirichlet_vertex_mask [nv] or NULL (NULL:
 * the whole boundary is Dirichlet). All host memory, copied by mg_setup. */
typedef struct mg_mesh_t {
  int32_t dim;            /* 2 or 3 */
  int32_t reserved;
  int64_t nv;
  int64_t nc;
  const double* coords;
  const int32_t* cells;
  const uint8_t* dirichlet_vertex_mask;
} mg_mesh_t;

/* Options; fill with mg_default_options() and change fields. */
typedef struct mg_options_t {
  int32_t cheb_degree;     /* A-applications per Chebyshev smoother application (2) */
  int32_t nu;              /* smoother applications before and after the coarse correction (1) */
  int32_t patch_layers;    /* vertex-layer extensions of Omega_b into Omega_B (1, Eq. identify) */
  int32_t smoother;        /* enum mg_smoother (SANDWICH) */
  int32_t adjusted_lambda; /* 1: lambda_max of A_gg (Sec. 5); 0: of the whole operator (1) */
  int32_t precision;       /* enum mg_precision (FP64) */
  int32_t host_only;       /* 1: build the hierarchy on the host only (exports work, compute
                              calls return MG_ERR_NO_DEVICE) (0) */
  int32_t eig_maxit;       /* Lanczos step limit for lambda_max (600) */
  double lmin_ratio;       /* lambda_min = lmin_ratio * lambda_max (0.1, Sec. 3.2) */
  double lmax_safety;      /* lambda_max is multiplied by this factor (1.0) */
  double eig_tol;          /* Lanczos residual tolerance relative to lambda_max (1e-8) */
  const double* lambda_override; /* [L-1] host array of lambda_max per level, or NULL */
  int32_t use_graph;       /* 1: mg_solve runs as one CUDA graph with a device-side
                              convergence test (conditional while node) (1) */
  int32_t local_levels_mask; /* bit l set: local correction on level l (-1 = all) */
  double quality_threshold;  /* set by mg_setup from its argument; ignored by mg_setup_csr */
  int32_t sell_sigma;      /* SELL-32 slot order: rows sorted by length within windows of this
                              many rows (1 = natural order); 0 = autotune: time y = A x on the
                              device for windows {1, 256, 2048} per operator, keep the fastest (0) */
  int32_t reorder;         /* enum mg_reorder: the order in which the device stores each
                              level but the coarsest (vectors at the ABI stay in the library's
                              numbering) (NONE) */
  int32_t global_smoother; /* enum mg_global_smoother (CHEBYSHEV) */
  int32_t pde;             /* enum mg_pde (POISSON); mg_setup only */
  double young;            /* Young's modulus E for MG_PDE_ELASTICITY (6.9e10, Sec. 6.3) */
  double poisson_ratio;    /* Poisson's ratio nu for MG_PDE_ELASTICITY (0.33, Sec. 6.3) */
  int32_t small_level_dofs; /* the first level with at most this many DoFs, and every level
                              below it, run their part of each V-cycle inside one persistent
                              cooperative launch (phases separated by grid barriers) instead of
                              one launch per step; 0 = never (Chebyshev global smoother only)
                              (0) */
  int32_t fp32_patch_kappa; /* MIXED precision: a patch whose block has condition number
                              kappa_1 = ||A[B,B]||_1 ||A[B,B]^-1||_1 at most this value applies its
                              inverse in FP32 (FP32 copy of the inverse, FP32 products); the
                              ill-conditioned ones, and every patch in FP64 precision, stay FP64;
                              0 = all FP64 (10000) */
  int32_t tune_min_nnz;    /* with sell_sigma = 0: operators with fewer nonzeros than this take
                              a fixed rule instead of device timing (CSR vector, lanes per row
                              the smallest power of two >= half the mean row length, 4..32, at
                              most one device wave of threads; SELL with one lane per row for
                              operators of more than 155,648 rows);
                              below about a million nonzeros every candidate runs in a few
                              microseconds, bound by launch and memory latency, and timing
                              cannot separate them. 0 = time every operator (1 << 20) */
  int32_t reserved[1];
} mg_options_t;

/* Result of a solve. */
typedef struct mg_solve_info_t {
  int32_t iterations;        /* CG iterations (= V-cycle applications) */
  int32_t converged;         /* 1 if the recurrence residual reached rtol */
  double rel_residual;       /* ||r_k||_2 / ||b||_2 of the recurrence residual */
  double true_rel_residual;  /* ||b - A x||_2 / ||b||_2 recomputed in FP64 at exit */
} mg_solve_info_t;

/* CSR matrix handed to mg_setup_csr (host memory, copied). */
typedef struct mg_csr_t {
  int64_t nrows;
  int64_t ncols;
  const int32_t* rowptr;   /* [nrows+1], rowptr[0] = 0 */
  const int32_t* colidx;   /* [nnz], sorted within each row */
  const double* values;    /* [nnz] */
} mg_csr_t;

/* ---- set-up and teardown ------------------------------------------------------------ */

/* Default options (see the field comments). */
void mg_default_options(mg_options_t* opt);

/* Build the hierarchy from mesh levels (Sec. 2, Sec. 4.4, Sec. 5, Sec. 6): P1/P2 stiffness
 * on level 0; per level gamma = d R_I / R_C (Eq. radius_ratio, read as normalised to 1
 * for the regular simplex), Omega_b = {gamma < quality_threshold}, Omega_B by
 * patch_layers vertex extensions, patches B_d = vertex-connected components (free DoFs,
 * ascending, patches ordered by their smallest DoF); P_l by point location of the fine
 * DoF points in the coarse mesh; A_{l+1} = P_l^T A_l P_l; patch matrices A[B_d,B_d] and
 * the coarsest matrix factored by Cholesky (FP64); lambda_max of D^-1 A_l by Lanczos.
 * levels: host array [L] (L >= 2), degree 1 or 2. On success *out owns the hierarchy.
 * Errors: INVALID_ARG, DEGENERATE_CELL, POINT_LOCATION, NOT_SPD, OOM, CUDA. */
int mg_setup(const mg_mesh_t* levels, int32_t L, int32_t degree, double quality_threshold,
             const mg_options_t* opt, mg_hierarchy_t** out);

/* Build a hierarchy from algebraic data: A[L] level operators (SPD, square), P[L-1] with
 * P[l] mapping level l+1 to level l (nrows = n_l, ncols = n_{l+1}; R_l = P_l^T),
 * patch_ptr[l] ([np_l+1]) / patch_dofs[l] (disjoint DoF sets) per level (NULL = none),
 * lambda_max per level through opt->lambda_override (required). No Galerkin product is
 * formed: A[l] is used as given. Same ownership and errors as mg_setup. */
int mg_setup_csr(const mg_csr_t* A, const mg_csr_t* P, int32_t L,
                 const int32_t* const* patch_ptr, const int32_t* const* patch_dofs,
                 const int32_t* num_patches, const mg_options_t* opt, mg_hierarchy_t** out);

/* Free a hierarchy and all memory it owns (NULL is allowed). Synchronises the device. */
void mg_free(mg_hierarchy_t* h);

/* Message of the last failed call on h (NULL: of the last failed setup in this thread). */
const char* mg_last_error(const mg_hierarchy_t* h);

/* ---- queries and exports (host memory; work on host_only hierarchies) --------------- */

int32_t mg_num_levels(const mg_hierarchy_t* h);
int64_t mg_num_dofs(const mg_hierarchy_t* h, int32_t level);        /* free DoFs n_l */
int64_t mg_level_nnz(const mg_hierarchy_t* h, int32_t level);       /* nnz of A_l */
int64_t mg_transfer_nnz(const mg_hierarchy_t* h, int32_t level);    /* nnz of P_l (l < L-1) */
/* Number of patches and total patch DoFs on a level. */
int mg_num_patches(const mg_hierarchy_t* h, int32_t level, int32_t* num, int64_t* total_dofs);

/* A_l as CSR into caller arrays rowptr[n+1], colidx[nnz], values[nnz]. */
int mg_export_level(const mg_hierarchy_t* h, int32_t level, int32_t* rowptr, int32_t* colidx, double* values);
/* P_l (level l+1 -> l) as CSR: rowptr[n_l+1], colidx/values[nnz]. */
int mg_export_transfer(const mg_hierarchy_t* h, int32_t level, int32_t* rowptr, int32_t* colidx, double* values);
/* Patches of a level: ptr[num+1], dofs[total] (free DoF ids). */
int mg_export_patches(const mg_hierarchy_t* h, int32_t level, int32_t* ptr, int32_t* dofs);
/* Per patch of level l (the order of mg_export_patches): 1 if the local correction (Alg. 2)
 * applies its inverse in FP32 (MIXED precision, option fp32_patch_kappa), else 0, into
 * flags[num_patches] (host). Needs the device phase (INVALID_ARG for host-only hierarchies). */
int mg_export_patch_precision(const mg_hierarchy_t* h, int32_t level, int32_t* flags);
/* The multicolour SGS colouring of level l (library numbering): *ncolours, and colour[n]
 * (nullable) with each DoF's colour. INVALID_ARG unless global_smoother = MG_GLOBAL_SGS
 * and l is below the coarsest level. Works for host-only hierarchies. */
int mg_export_colouring(const mg_hierarchy_t* h, int32_t level, int32_t* ncolours, int32_t* colour);
/* lambda_max of D^-1 A_l, unadjusted and adjusted (Sec. 5), as estimated at setup (0 when
 * an override was given), and the value the smoother uses. */
int mg_eigs(const mg_hierarchy_t* h, int32_t level, double* lmax, double* lmax_adj, double* lmax_used);
/* Interpolation point of each free DoF: out[n_l*dim] (geometric hierarchies only). */
int mg_dof_coords(const mg_hierarchy_t* h, int32_t level, double* out);
/* gamma per cell of a level's mesh: out[nc] (geometric hierarchies only). */
int mg_cell_quality(const mg_hierarchy_t* h, int32_t level, double* out);
/* b_i = int f phi_i for a constant f on the free DoFs of level 0: out[n_0] host
 * (MG_PDE_POISSON hierarchies built by mg_setup). */
int mg_load_constant(const mg_hierarchy_t* h, double f, double* out_host);

/* ---- the hot path (device vectors, FP64 at the boundary) ---------------------------- */

/* One V-cycle of Alg. 1 in place: x_dev (initial guess in, new iterate out) for
 * A_0 x = b, b_dev/x_dev [n_0] FP64. In MIXED precision the cycle computes the correction
 * for the residual in FP32 (x += V(b - A x)). Asynchronous on `stream`, except for
 * hierarchies with a bounded device-side wait (small_level_dofs > 0, or the TMA-staged SpMV
 * forced), where it blocks to read the wait flags (MG_ERR_TIMEOUT as for mg_solve). */
int mg_vcycle(mg_hierarchy_t* h, const double* b_dev, double* x_dev, void* stream);

/* V-cycle-preconditioned CG (Sec. 6.2) from x = 0 until ||r||_2/||b||_2 <= rtol or maxit
 * iterations; x_dev receives the solution. Blocks until the solve has finished and fills
 * *info (may be NULL). Returns MG_OK, MG_ERR_NO_CONVERGENCE or MG_ERR_BREAKDOWN.
 * The solve runs as one CUDA graph (use_graph = 1) or per-kernel launches; with
 * small_level_dofs >= n_0 the whole solve is one persistent cooperative launch, and with a
 * smaller nonzero small_level_dofs each V-cycle's lower levels are.
 * MG_ERR_TIMEOUT (the result is then not valid) only where a bounded device-side wait can
 * run: a grid barrier of the persistent launch (small_level_dofs > 0) or the TMA-staged SpMV
 * (only with the environment variable NNMG_FORCE_LAYOUT=tma at set-up; the autotuner never
 * picks it). Every entry point that runs such work (mg_vcycle, mg_solve*, the single steps,
 * the server's requests) checks and clears the flag after its work and reports it this way;
 * the TMA flag is shared by every stream of the device. */
int mg_solve(mg_hierarchy_t* h, const double* b_dev, double* x_dev, double rtol, int32_t maxit,
             mg_solve_info_t* info, void* stream);

/* mg_solve with host vectors: copies b_host in, solves, copies the solution to x_host. */
int mg_solve_host(mg_hierarchy_t* h, const double* b_host, double* x_host, double rtol,
                  int32_t maxit, mg_solve_info_t* info, void* stream);

/* Stationary multigrid (Sec. 6.1): repeated V-cycles from x_dev until ||b-Ax||/||b|| <=
 * rtol or maxit cycles. Blocks; fills *info. */
int mg_solve_stationary(mg_hierarchy_t* h, const double* b_dev, double* x_dev, double rtol,
                        int32_t maxit, mg_solve_info_t* info, void* stream);

/* Solve n independent problems (their own hierarchies, all FP64 at the boundary). The
 * problems whose whole solve runs persistently (small_level_dofs >= n_0) are iterated
 * together in one persistent cooperative launch per precision on `stream` (their steps
 * merged phase by phase; a problem's result is bitwise the same as solved alone); the others
 * run their solve graphs on their own streams, overlapping on the device, joined back to
 * `stream`. The persistent group allocates (and frees) its program and partial sums on
 * `stream` during the call. Blocks; info[n] may be NULL. Returns the first non-OK status
 * (MG_ERR_TIMEOUT as for mg_solve). */
int mg_solve_batch(mg_hierarchy_t* const* hs, const double* const* b_dev, double* const* x_dev,
                   int32_t n, double rtol, int32_t maxit, mg_solve_info_t* info, void* stream);

/* b = int_{Gamma_2} t . v over the boundary facets of level 0 lying in the plane
 * x_axis = value (every vertex within 1e-12 of it), for MG_PDE_ELASTICITY hierarchies
 * built by mg_setup (Sec. 6.3: traction (1e3, 0, 0) on the face x = 6 of the lattice).
 * t: host [dim]; b_host: host [mg_num_dofs(h, 0)]. INVALID_ARG for other hierarchies. */
int mg_load_traction(const mg_hierarchy_t* h, int32_t axis, double value, const double* t, double* b_host);
/* b = int_Omega f . v for a constant body force f (host [dim]) on the free DoFs of level 0
 * (Sec. 6.3: f = (0, 0, -1e3) on the dumbbell-like structure), for MG_PDE_ELASTICITY
 * hierarchies built by mg_setup; b_host: host [mg_num_dofs(h, 0)]. */
int mg_load_body(const mg_hierarchy_t* h, const double* f, double* b_host);

/* ---- single steps of the hot path (device vectors in the hierarchy's V-cycle type:
 *      FP64 in FP64 mode; FP32 in MIXED mode is not exposed) -------------------------- */

/* y = A_l x. */
int mg_apply_A(mg_hierarchy_t* h, int32_t level, const double* x_dev, double* y_dev, void* stream);
/* One Chebyshev smoother application S_g of cheb_degree steps on level l, in place. */
int mg_chebyshev(mg_hierarchy_t* h, int32_t level, const double* b_dev, double* x_dev, void* stream);
/* One multicolour symmetric Gauss-Seidel application on level l (forward then backward
 * colour sweep, see MG_GLOBAL_SGS), in place. INVALID_ARG unless the hierarchy was built
 * with global_smoother = MG_GLOBAL_SGS. */
int mg_sgs(mg_hierarchy_t* h, int32_t level, const double* b_dev, double* x_dev, void* stream);
/* One local correction S_c on level l (Alg. 2), in place. */
int mg_local_correction(mg_hierarchy_t* h, int32_t level, const double* b_dev, double* x_dev, void* stream);
/* One combined smoother application on level l (post = 0: pre-smoothing order), in place. */
int mg_smooth(mg_hierarchy_t* h, int32_t level, int32_t post, const double* b_dev, double* x_dev, void* stream);
/* r = b - A_l x and bc = R_l r (Eq. 4); r_dev [n_l], bc_dev [n_{l+1}]. */
int mg_residual_restrict(mg_hierarchy_t* h, int32_t level, const double* b_dev, const double* x_dev,
                         double* r_dev, double* bc_dev, void* stream);
/* x_l += P_l xc (Alg. 1, coarse-grid correction); xc_dev [n_{l+1}], x_dev [n_l]. */
int mg_prolong_correct(mg_hierarchy_t* h, int32_t level, const double* xc_dev, double* x_dev, void* stream);
/* x = A_{L-1}^{-1} b on the coarsest level (direct solve). */
int mg_coarse_solve(mg_hierarchy_t* h, const double* b_dev, double* x_dev, void* stream);

/* Capture the V-cycle from level `level` down (Alg. 1 entered at that level with a zero
 * iterate on the level's current right-hand side; level 0 = the whole preconditioner) into
 * a CUDA graph and time `reps` replays on `stream` with CUDA events; returns the mean ms per
 * replay. The difference between consecutive levels is that level's in-graph cost. The
 * level's work vectors are overwritten. */
int mg_time_vcycle(mg_hierarchy_t* h, int32_t level, int32_t reps, void* stream, double* ms_per_cycle);

/* Time `reps` back-to-back launches of the fine-level fused Chebyshev SpMV kernel with CUDA
 * events on `stream`; returns the mean duration in ms and the kernel's algorithmic bytes
 * per launch (matrix once, vectors once). Vectors are the hierarchy's own work buffers. */
int mg_time_smoother_kernel(mg_hierarchy_t* h, int32_t reps, void* stream, double* ms_per_launch,
                            double* bytes_per_launch);

/* ---- solve server: continuous batching of solve requests on one GPU ----------------
 * (a serving pattern; the paper has no counterpart.)
 * Requests (a mesh hierarchy and a right-hand side) go through host set-up on worker
 * threads, wait for admission in submission order until their device-byte estimate fits
 * under the HBM budget and one of max_active slots is free, then are set up on the device
 * and solved by MG-PCG on their own stream, overlapping with the other active requests.
 * Completion frees the request's device memory and admits the next ones. */
typedef struct mg_server mg_server_t;

typedef struct mg_request_t {
  const mg_mesh_t* levels;     /* [L] host meshes, copied at submission */
  int32_t L;
  int32_t degree;              /* 1 or 2 */
  double quality_threshold;    /* 0.1 in the paper */
  const mg_options_t* opt;     /* NULL = defaults; use_graph is forced on */
  const double* b;             /* [n_b] right-hand side on the level-0 free DoFs, or NULL: f = 1
                                  (elasticity: a body force of 1 in every component) */
  int64_t n_b;
  double rtol;
  int32_t maxit;
  int32_t tune;                /* 0: every operator of the request takes the rule layout of
                                  tune_min_nnz whatever opt says (a request is solved once, so
                                  device timing runs at set-up would cost more than they save);
                                  1: opt's tune_min_nnz applies */
} mg_request_t;

typedef struct mg_request_result_t {
  int32_t status;              /* -1 while pending; then MG_OK or an error code */
  int32_t iterations;
  double rel_residual;
  double true_rel_residual;
  int64_t n;                   /* free DoFs of level 0 */
  int64_t device_bytes;        /* device memory the request held */
  double t_queue_ms;           /* submission -> host set-up start */
  double t_setup_ms;           /* host set-up */
  double t_wait_ms;            /* host set-up done -> admitted to the device */
  double t_device_ms;          /* admitted -> solution on the host (device set-up + solve) */
  double t_total_ms;           /* submission -> done */
  double t_solve_ms;           /* GPU time of the solve itself (CUDA events on the request's
                                  stream around the copies in and out and the MG-PCG) */
} mg_request_result_t;

typedef struct mg_server_stats_t {
  int64_t submitted, completed, failed;
  int64_t bytes_in_use, peak_bytes;
  int32_t active, peak_active, queued, reserved;
} mg_server_stats_t;

/* Create a server with an HBM budget (bytes), max_active concurrent requests on the device
 * and setup_threads host set-up workers. A request's host set-up runs its parallel loops on
 * a share of the host cores fixed when it starts: all of them when no other request is in host
 * set-up, a 1/(k+1) share beside k others (results do not depend on the share). */
int mg_server_create(int64_t hbm_budget_bytes, int32_t max_active, int32_t setup_threads, mg_server_t** out);
/* Queue a request (inputs copied); *id identifies it. Never blocks on the device. */
int mg_server_submit(mg_server_t* s, const mg_request_t* req, int64_t* id);
/* Current state of a request (status -1 while pending). */
int mg_server_poll(mg_server_t* s, int64_t id, mg_request_result_t* out);
/* Block until the request is done or timeout_s passes (MG_ERR_TIMEOUT). */
int mg_server_wait(mg_server_t* s, int64_t id, double timeout_s, mg_request_result_t* out);
/* Copy a finished request's solution (x_host[n], n = result.n; NULL to discard) and forget it. */
int mg_server_fetch(mg_server_t* s, int64_t id, double* x_host, int64_t n);
int mg_server_stats(mg_server_t* s, mg_server_stats_t* out);
/* Message of the last failed server call in this thread. */
const char* mg_server_last_error(void);
/* Finish the requests already admitted, fail the rest, free everything. */
void mg_server_destroy(mg_server_t* s);

/* ---- allocation-free variant (the paper has no counterpart) ---------------------------
 * x = X b for a dense symmetric n x n FP64 matrix X (row-major, device), the product the
 * coarsest-level direct solve applies, for callers that cannot allocate device memory
 * when they need it (all memory pre-reserved by another allocator, or a latency-critical
 * path where cudaMalloc/cudaFree would stall or synchronise the device). The split-K
 * partial sums live in a static device array of 2^20 doubles (8 MiB per device, held until
 * the process exits) instead of allocated scratch; no allocation happens in the call.
 * Limits: 1 <= n <= 65536, every such n admitted (at most 16 split-K chunks of at most 4096
 * columns); larger n: MG_ERR_INVALID_ARG, message in mg_last_error(NULL). A failed launch of
 * this call's own kernels: MG_ERR_CUDA (an earlier, unrelated sticky error is not reported
 * as this call's).
 * The first call on a device looks up the array's address with that device current;
 * make it before any stream capture. All calls share the array (each call writes every
 * partial it reads, so nothing needs clearing): calls whose kernels overlap on the GPU
 * race. X_dev, b_dev [n], x_dev [n] are caller-owned device pointers; asynchronous on
 * `stream`. */
int mg_dense_symv_static(const double* X_dev, int64_t n, const double* b_dev, double* x_dev, void* stream);

/* Mean device time of the FP64 CG product q = A_0 p with its p.q reduction (the k_ap kernel
 * and its one-block finish) over reps back-to-back launches on `stream` (CUDA events; blocks),
 * and its algorithmic bytes per launch (values and indices once, p and q once, metadata).
 * Overwrites the hierarchy's CG work vectors; measurement helper. */
int mg_time_cg_product(mg_hierarchy_t* h, int32_t reps, void* stream, double* ms, double* bytes);

/* Mean device time of one S_c solve launch on level l (the patch GEMVs of Alg. 2 over the
 * work list, on whatever residual the hierarchy holds; overwrites the level's iterate) over
 * reps launches on `stream` (blocks), with its algorithmic work: FMAs with FP64 inverses
 * (sum of n_d^2), FMAs with FP32 inverses, and the inverses' bytes. Measurement helper. */
int mg_time_patch_solve(mg_hierarchy_t* h, int32_t level, int32_t reps, void* stream, double* ms, double* fma64,
                        double* fma32, double* bytes);

/* FP64 FMA throughput of the current device (FMAs per second): independent FMA chains on
 * every SM, timed with CUDA events on `stream` (blocks; allocates and frees a small buffer).
 * The denominator of the FP64-ALU roofline of the patch solves and the coarsest solve. */
int mg_measure_fp64_fma(void* stream, double* fma_per_s);

/* Device bytes held by the hierarchy. */
int64_t mg_device_bytes(const mg_hierarchy_t* h);
/* Number of kernel launches of one V-cycle, and of one CG iteration (V-cycle included). */
int mg_launch_counts(const mg_hierarchy_t* h, int32_t* per_vcycle, int32_t* per_cg_iteration);

#ifdef __cplusplus
}
#endif

#endif /* NNMG_H */
