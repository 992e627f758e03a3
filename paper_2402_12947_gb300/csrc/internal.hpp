// Internal host-side data structures and set-up routines of the nnmg library.
#pragma once

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstring>
#include <functional>
#include <mutex>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime_api.h>

#include "nnmg.h"

namespace nnmg {

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

// Compressed sparse rows with 32-bit indices (row pointers fit: nnz < 2^31).
struct Csr {
  int64_t nrows = 0, ncols = 0;
  std::vector<int32_t> rp, ci;
  std::vector<double> v;
  int64_t nnz() const { return (int64_t)ci.size(); }
};

struct MeshH {
  int dim = 0;
  int64_t nv = 0, nc = 0;
  std::vector<double> x;        // [nv*dim]
  std::vector<int32_t> c;       // [nc*(dim+1)]
  std::vector<uint8_t> mask;    // [nv] Dirichlet-allowed vertices (empty = all)
};

struct DofMapH {
  int degree = 1, dim = 2, nloc = 3;
  int64_t ndofs = 0, nfree = 0, nv = 0;
  std::vector<int64_t> cell_dofs;   // [nc*nloc] all-DoF ids
  std::vector<int64_t> edges;       // [ne*2] sorted vertex pairs (P2)
  std::vector<double> points;       // [ndofs*dim]
  std::vector<uint8_t> dirichlet;   // [ndofs]
  std::vector<int64_t> free_index;  // [ndofs] free id or -1
  std::vector<int64_t> free_list;   // [nfree] all-DoF id of each free DoF
  std::vector<int64_t> bfaces;      // boundary facets as c*(dim+1) + (local vertex opposite)
};

// Boundary facets of a mesh with their free scalar DoFs (-1: Dirichlet), for surface loads:
// x [nf*dim*dim] the facet's vertex coordinates, dofs [nf*nfloc] its vertex DoFs then (P2)
// its edge DoFs.
struct BoundaryFaces {
  int dim = 0, degree = 1, nfloc = 0;
  std::vector<double> x;
  std::vector<int64_t> dofs;
};

// One level of the hierarchy as built on the host.
struct LevelH {
  Csr A;                     // free-DoF operator (assembled on level 0, Galerkin below)
  Csr P, R;                  // P: level l+1 -> l (rows n_l); R = P^T (empty on the coarsest)
  std::vector<double> dinv;  // 1 / diag(A)
  std::vector<int32_t> patch_ptr, patch_dofs;
  double lmax_unadj = 0, lmax_adj = 0, lmax = 0, lmin = 0;
  int lanczos_iters = 0;
  int dim = 0;
  std::vector<double> dof_points;   // [n*dim] (geometric hierarchies)
  std::vector<double> gamma;        // [nc]    (geometric hierarchies)
  std::vector<int32_t> colour;      // [n] multicolour SGS colouring (global_smoother = SGS)
  int32_t ncolours = 0;
};

// ---- threading helper ----
// Threads a parallel_for may use; set_thread_budget(k) limits the calling thread's loops
// to k threads (0 = all hardware threads).
int num_threads();
void set_thread_budget(int k);
void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)>& body);

// A CSR matrix built row by row in one parallel pass: each parallel_for block creates its
// scratch with make_state() and appends row i's sorted columns and values through
// fill(state, i, ci, v); the blocks are then copied into place behind the row pointers.
template <typename MakeState, typename Fill>
Csr csr_from_rows(int64_t nrows, int64_t ncols, MakeState&& make_state, Fill&& fill) {
  struct Block {
    int64_t lo = 0, hi = 0;
    std::vector<int64_t> end;  // running entry count after each row of the block
    std::vector<int32_t> ci;
    std::vector<double> v;
  };
  std::vector<Block> blocks;
  std::mutex mu;
  parallel_for(nrows, [&](int64_t lo, int64_t hi) {
    Block blk;
    blk.lo = lo, blk.hi = hi;
    blk.end.resize(hi - lo);
    auto st = make_state();
    for (int64_t i = lo; i < hi; ++i) {
      fill(st, i, blk.ci, blk.v);
      blk.end[i - lo] = (int64_t)blk.ci.size();
    }
    std::lock_guard<std::mutex> lk(mu);
    blocks.push_back(std::move(blk));
  });
  std::sort(blocks.begin(), blocks.end(), [](const Block& a, const Block& b) { return a.lo < b.lo; });
  Csr C;
  C.nrows = nrows;
  C.ncols = ncols;
  C.rp.assign(nrows + 1, 0);
  int64_t base = 0;
  for (const Block& blk : blocks) {
    for (int64_t i = blk.lo; i < blk.hi; ++i) {
      const int64_t e = base + blk.end[i - blk.lo];
      if (e > INT32_MAX) throw Error(MG_ERR_INVALID_ARG, "nnz exceeds 2^31");
      C.rp[i + 1] = (int32_t)e;
    }
    base += (int64_t)blk.ci.size();
  }
  C.ci.resize(base);
  C.v.resize(base);
  std::vector<std::thread> th;
  for (const Block& blk : blocks)
    th.emplace_back([&C, &blk] {
      if (blk.ci.empty()) return;
      std::memcpy(C.ci.data() + C.rp[blk.lo], blk.ci.data(), blk.ci.size() * sizeof(int32_t));
      std::memcpy(C.v.data() + C.rp[blk.lo], blk.v.data(), blk.v.size() * sizeof(double));
    });
  for (auto& t : th) t.join();
  return C;
}

// ---- setup_fem.cpp: DoF maps, assembly, quality, patches ----
DofMapH build_dofmap(const MeshH& m, int degree);
std::vector<double> radius_ratio(const MeshH& m);
Csr assemble_stiffness(const MeshH& m, const DofMapH& dm);
std::vector<double> load_constant(const MeshH& m, const DofMapH& dm, double f);
// Linear elasticity (Sec. 6.3): the operator on free vector DoFs, vector DoF dim*k + c =
// component c of free scalar DoF k; cell term mu (grad phi_a . grad phi_b) delta_ij +
// mu d_j phi_a d_i phi_b + lambda d_i phi_a d_j phi_b (trial phi_b e_j, test phi_a e_i).
Csr assemble_elasticity(const MeshH& m, const DofMapH& dm, double mu, double lam);
BoundaryFaces boundary_faces(const MeshH& m, const DofMapH& dm);
// b = int_{Gamma} t . v over the boundary facets in the plane x_axis = value (all vertices
// within tol), over the nfree*dim vector DoFs.
std::vector<double> traction_load(const BoundaryFaces& bf, int axis, double value, double tol, const double* t,
                                  int64_t nfree);
void local_patches(const MeshH& m, const DofMapH& dm, const std::vector<double>& gamma,
                   double threshold, int layers, std::vector<int32_t>& ptr, std::vector<int32_t>& dofs);

// ---- setup_algebra.cpp: transfer, sparse products, dense factorisations, eigenvalues ----
Csr prolongation(const DofMapH& fine, const MeshH& coarse_mesh, const DofMapH& coarse);
Csr transpose(const Csr& A);
// Coarse DoFs that P never reaches have empty rows in P^T A P: give them A_ii = 1.
Csr unit_diagonal_on_empty_rows(const Csr& A);
Csr spgemm(const Csr& A, const Csr& B);
// P (x) I_d: entry (i, j, v) becomes (d*i + c, d*j + c, v) for c < d.
Csr kron_identity(const Csr& P, int d);
// lambda_max of D^{-1/2} A D^{-1/2} restricted to rows/cols with keep[i] != 0 (NULL: all).
double lanczos_lmax(const Csr& A, const uint8_t* keep, double tol, int maxit, int* iters);
// Greedy colouring in index order: colour[i] = the smallest colour not held by a neighbour
// j < i with |a_ij| > 1e-12 sqrt(|a_ii a_jj|). Returns the number of colours.
int32_t greedy_colouring(const Csr& A, std::vector<int32_t>& colour);
// Pieces of the Lanczos iteration shared by the host and device versions: the scaling
// D^{-1/2} (0 on excluded rows), the deterministic unit start vector, and the largest
// eigenvalue of the tridiagonal T_m (a = diagonal, b[1..m-1] = off-diagonal) with the
// modulus of the last component of its unit eigenvector.
std::vector<double> lanczos_scaling(const Csr& A, const uint8_t* keep);
std::vector<double> lanczos_start(const std::vector<double>& s);
void tridiag_top(const std::vector<double>& a, const std::vector<double>& b, int m, double* theta, double* slast);
std::vector<double> dense_submatrix(const Csr& A, const int32_t* idx, int64_t n);
void spmv_host(const Csr& A, const double* x, double* y);

// Reverse Cuthill-McKee order of A's graph (perm[new] = old), per connected component.
std::vector<int32_t> rcm_order(const Csr& A);
// Z-order (Morton) of points [n*dim]: coordinates scaled to integers over the bounding box
// (31 bits in 2D, 21 in 3D), bits interleaved; equal codes keep index order.
std::vector<int32_t> morton_order(const std::vector<double>& pts, int dim);
// B[i, :] = A[rowperm[i], :] with columns mapped by colmap (old -> new); empty = identity.
Csr permute_csr(const Csr& A, const std::vector<int32_t>& rowperm, const std::vector<int32_t>& colmap);
std::vector<int32_t> inverse_perm(const std::vector<int32_t>& p);

// ---- hierarchy.cu: phases of a hierarchy's life used by the solve server ----
// Host phase of mg_setup (throws Error).
mg_hierarchy* build_host_hierarchy(const mg_mesh_t* levels, int32_t L, int32_t degree, double quality_threshold,
                                   const mg_options_t* opt);
// Device phase (upload, dense inverses, layouts, solve graph) on the hierarchy's stream.
void build_device_hierarchy(mg_hierarchy* h);
// Upper bound of the device bytes the device phase will allocate (host phase done).
int64_t estimate_device_bytes(const mg_hierarchy* h);
int64_t hierarchy_device_bytes(const mg_hierarchy* h);
int64_t hierarchy_dofs(const mg_hierarchy* h);
// b for f = 1 on the free DoFs of level 0 (geometric hierarchies; elasticity: f = 1 in
// every component).
std::vector<double> hierarchy_unit_load(const mg_hierarchy* h);
// Enqueue one MG-PCG solve on the hierarchy's own stream: b (page-locked host, n_0) in, the
// solution to x (page-locked host) and the CG state out, then record `done`.
// `start` (nullable) is recorded before the copy in.
void enqueue_host_solve(mg_hierarchy* h, const double* b, double* x, double rtol, int maxit, cudaEvent_t done,
                        cudaEvent_t start = nullptr);
// After `done` has completed: the solve's status and info.
int collect_host_solve(mg_hierarchy* h, mg_solve_info_t* info);
void destroy_hierarchy(mg_hierarchy* h);
// Message returned by mg_last_error(NULL) in the calling thread.
void set_last_error(const std::string& msg);
// Page-locked host staging buffers reused across requests (allocating page-locked memory
// would synchronise every stream of the device).
double* pinned_acquire(int64_t n);
void pinned_release(double* p);

}  // namespace nnmg
