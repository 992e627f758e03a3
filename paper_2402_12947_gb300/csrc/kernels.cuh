// Device kernels of the nnmg hot path (sm_103a) and their host launchers.
//
// Sparse operators are stored in SELL-32: rows grouped in slices of 32 (one warp), each
// slice padded to its longest row and stored column-major, so that thread `lane` of a
// warp owns row 32*s + lane and every load instruction of the warp reads 32 consecutive
// values (and 32 consecutive column indices). One thread accumulates one row in CSR
// column order, so no cross-lane reduction (and no extra FP64 additions) is needed:
// on GB300 the FP64 pipe (~0.6 TFMA/s) is close to the HBM rate for 12-byte nonzeros.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace nnmg {

template <typename T>
struct SellMat {
  int32_t nrows = 0, ncols = 0, nslices = 0;
  int64_t nnz = 0, padded = 0;
  int64_t* off = nullptr;   // [nslices+1] element offset of each slice (multiple of 32)
  int32_t* col = nullptr;   // [padded]
  T* val = nullptr;         // [padded]
  int32_t* perm = nullptr;  // [nrows] matrix row held by each slot, or null (identity)
  int32_t sigma = 1;        // window within which rows were sorted by length
  int32_t lanes = 1;        // 1: SELL-32 (off/col/val/perm); G > 1: CSR vector (rp/col/val)
  int32_t unroll = 1;       // SELL-32 row loop: 1 = steps of 4 + scalar remainder, 2 = predicated steps of 4, 3 = of 8
  int32_t pf = 0;           // SELL: slices ahead whose data a warp prefetches into L2 (0 = none)
  int32_t sub = 1;          // SELL: lanes per row (1, 2, 4); a slice holds 32/sub rows whose
                            // entries j of row r sit at lane r*sub + j%sub of step j/sub
  int32_t* rp = nullptr;    // [nrows+1] CSR row pointer (lanes > 1)
  // 16-bit column offsets: column = cbase[slice or row] + col16[k] where cbase >= 0; a
  // slice or row spanning more than 2^16 columns has cbase = -1 and reads col (which is
  // then null when every slice or row is narrow)
  uint16_t* col16 = nullptr;
  int32_t* cbase = nullptr; // [nslices] (SELL) or [nrows] (CSR vector)
  double idx_bytes = 0;     // index bytes of the nonzeros (2 or 4 each), for the roofline
  // TMA-staged variant (SELL, one lane per row, 32-bit indices): chunks[c] .. chunks[c+1]
  // are the slices of chunk c, at most tma_stage_entries<T>() padded entries; tma = 1 runs
  // the persistent kernel that streams the chunks into shared memory with bulk copies.
  int32_t* chunks = nullptr;
  int32_t nchunks = 0;
  int32_t tma = 0;
};

// Padded entries of one shared-memory stage of the TMA-staged SpMV (values and indices).
template <typename T>
__host__ __device__ constexpr int tma_stage_entries() {
  return sizeof(T) == 4 ? 4096 : 2048;
}
// A bounded wait in a kernel gave up (the kernel set a device flag and returned): reads and
// clears the flag through stream s (synchronises s).
bool take_wait_timeout(cudaStream_t s);
// One-time set-up of the TMA-staged kernels (call before capturing a graph that uses them).
void tma_prepare();

// Device-side state of the preconditioned CG recurrence (all FP64).
struct CgState {
  double bb, rz, pq, alpha, rr, beta, rtol2, rr_true;
  int32_t it, maxit, status, cont;   // status: 0 running, 1 converged, 2 maxit, 3 breakdown
};

// FIN_NORM: rr = the sum; FIN_TRUE: rr_true = the sum (|b - A x|^2 recomputed at exit)
enum FinishOp { FIN_BB = 0, FIN_RZ0 = 1, FIN_PQ = 2, FIN_RR = 3, FIN_RZ = 4, FIN_NORM = 5, FIN_TRUE = 6 };

// The CG state update that finishes a reduction with sum s (shared by the per-kernel solve and
// the persistent batched solve): FIN_BB starts the recurrence, FIN_PQ sets alpha (breakdown on
// a non-positive or non-finite p.q), FIN_RR counts the iteration and decides whether to go on
// (converged, maxit, breakdown; inside a captured graph also the while-node condition),
// FIN_RZ sets beta.
#ifdef __CUDACC__
// Absolute bound on CG iterations inside one solve, whatever maxit says.
constexpr int kMaxCgIterations = 100000;

__device__ inline void apply_finish(CgState* st, double s, int op, int use_cond, unsigned long long handle) {
  switch (op) {
    case FIN_BB:
      st->bb = s;
      st->it = 0;
      st->status = 0;
      st->cont = 1;
      break;
    case FIN_RZ0:
      st->rz = s;
      break;
    case FIN_PQ:
      if (st->bb == 0.0) {
        st->alpha = 0.0;
      } else if (!(s > 0.0) || !isfinite(s) || !isfinite(st->rz)) {
        st->alpha = 0.0;
        st->status = 3;
      } else {
        st->alpha = st->rz / s;
      }
      st->pq = s;
      break;
    case FIN_RR: {
      st->rr = s;
      int cont = 1;
      if (st->bb == 0.0) {  // b = 0: x = 0 is exact, no iteration
        st->status = 1;
        st->cont = 0;
        if (use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)handle, 0u);
        break;
      }
      st->it += 1;
      if (st->status == 3) cont = 0;
      else if (s <= st->rtol2 * st->bb) st->status = 1, cont = 0;
      else if (st->it >= st->maxit || st->it >= kMaxCgIterations) st->status = 2, cont = 0;
      if (!isfinite(s)) st->status = 3, cont = 0;
      st->cont = cont;
      if (use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)handle, (unsigned)cont);
      break;
    }
    case FIN_RZ:
      st->beta = s / st->rz;
      st->rz = s;
      break;
    case FIN_NORM:
      st->rr = s;
      break;
    case FIN_TRUE:
      st->rr_true = s;
      break;
  }
}

#endif

// A reduction fused into the kernel that produces it: every block writes its partial sum to
// part[block]; the last block to finish (an atomic ticket, reset by that block) sums the
// partials in a fixed order and applies `op` to the CG state. With use_cond set (inside a
// captured graph), FIN_RR also sets the while-node condition through `handle`: 1 to iterate
// again, 0 once converged, at maxit, or on breakdown.
struct Reduce {
  double* part;
  unsigned* ticket;
  CgState* st;
  int op, use_cond;
  unsigned long long handle;
};

// One S_c work item: rows row0 .. row0 + (kPatchRowsPerItem or, with PI_WARP_ROWS,
// kPatchRowsPerWarpItem) - 1 of a patch whose DoFs are pdofs[p0 .. p0 + n) and whose dense
// inverse starts at element inv of the FP64 arena, or, with PI_FP32 (well-conditioned patches
// of the mixed form), of the FP32 arena.
enum PatchItemMode { PI_FP32 = 1, PI_WARP_ROWS = 2 };
struct PatchItem {
  int32_t p0, n, row0, mode;
  int64_t inv;
};

constexpr int kBlock = 256;
constexpr int kPatchRowsPerItem = 32;   // rows of one patch per S_c work item (one lane each)
constexpr int kPatchRowsPerWarpItem = 8; // rows per item of a small patch (one warp each)
constexpr int kSmallPatch = 256;         // patches up to this size take warp-per-row items
constexpr int kMaxPatchDofs = 27000;    // largest patch (its residual is staged in shared memory)

// ---- SELL-32 SpMV family ----
template <typename T> void sell_spmv(const SellMat<T>& A, const T* x, T* y, cudaStream_t s);
template <typename T> void sell_resid(const SellMat<T>& A, const T* x, const T* b, T* r, cudaStream_t s);
// One Chebyshev step: r = b - A xin; d = cd d + cr dinv r (first: cd ignored); xout = xin + d.
template <typename T>
void sell_cheb(const SellMat<T>& A, const T* xin, const T* b, const T* dinv, T* d, T* xout, double cd, double cr,
               bool first, cudaStream_t s);
// The first Chebyshev step when x_in is zero except possibly on the rows listed in hrow
// (the rows coupled to patch DoFs, with their entries of A in hrp/hci/hv): r = b on all
// other rows, so their step needs no SpMV. nh = 0 when x_in is zero everywhere.
template <typename T>
void cheb_first_from_zero(int n, const T* b, const T* dinv, const T* xin, T* d, T* xout, double cr, int nh,
                          const int32_t* hrow, const int32_t* hrp, const int32_t* hci, const T* hv, cudaStream_t s);
// x += P xc.
template <typename T> void sell_prolong(const SellMat<T>& P, const T* xc, T* x, cudaStream_t s);
// x += P x_c and, in the same launch, the residual of the S_c that follows on the nt patch
// rows: rbuf[t] = res[pdofs[t]] - (A P)_{pdofs[t],:} x_c with res = b - A x before the
// correction and the rows of A P in ELL form (apci/apv, w slots per row, aplen[t] entries).
template <typename T>
void sell_prolong_pr(const SellMat<T>& P, const T* xc, T* x, int nt, int w, const int32_t* pdofs, const int32_t* aplen,
                     const int32_t* apci, const double* apv, const T* res, double* rbuf, cudaStream_t s);
// bc = R r and xc = 0 (xc has R.nrows entries).
template <typename T> void sell_restrict(const SellMat<T>& R, const T* r, T* bc, T* xc, cudaStream_t s);
// One colour of a multicolour Gauss-Seidel sweep: for each row r of M (the colour's rows,
// without the diagonal and without couplings inside the colour), i = rows[r] and
// x_i = dinv_i (b_i - (M x)_r).
template <typename T>
void sell_gs(const SellMat<T>& M, const int32_t* rows, const T* b, const T* dinv, T* x, cudaStream_t s);
// q = A p and p.q (FP64), reduced in the same launch: one resident wave of blocks walks the
// row blocks grid-stride, the last block to finish sums the block partials in order and
// applies rd.op to the CG state; rd.part needs an entry per block (at most one per row block).
void sell_ap(const SellMat<double>& A, const double* p, double* q, const Reduce& rd, cudaStream_t s);
int sell_blocks(int nrows, int lanes);

// ---- local correction S_c (two phases) ----
// S_c phase 1: rbuf[t] = b[pdofs[t]] - (A x)[pdofs[t]] for the nt patch rows, stored
// ELL-style with w slots per row (pci/pv [nt*w]), row t's plen[t] entries first, padding
// with value 0 and a valid column.
template <typename T>
void patch_residual(int nt, int w, const int32_t* pdofs, const int32_t* plen, const int32_t* pci, const double* pv,
                    const T* b, const T* x, double* rbuf, cudaStream_t s);
// Raise the dynamic shared-memory limit of the solve kernels (once, to kMaxPatchDofs) when a
// hierarchy has a patch above 48 KB of residual.
void patch_solve_setup(int max_patch);
// S_c phase 2, x_B += (A^[d])^{-1} r_B, one block per work item; rbuf == nullptr: the
// iterate is zero and the residual is b itself (phase 1 skipped).
template <typename T>
void patch_solve(int nitems, const PatchItem* items, const int32_t* pdofs, const double* inv, const float* inv32,
                 const double* rbuf, const T* b, T* x, int max_patch, cudaStream_t s);
// Start of a sandwich pre-smoothing from a zero iterate in one launch (plus the halo rows):
// x_B = (A^[d])^{-1} b_B on every patch, d = cr D^{-1} b and x_out = d on every row, then the
// rows coupled to patch DoFs (hrow, with their rows of A in hrp/hci/hv) recomputed with
// r = b - A x. x must be zero outside the patch DoFs on entry.
template <typename T>
void cheb_entry_local(int nitems, const PatchItem* items, const int32_t* pdofs, const double* inv, const float* inv32,
                      int max_patch, int n, const T* b, const T* dinv, T* x, T* d, T* xout, double cr, int nh,
                      const int32_t* hrow, const int32_t* hrp, const int32_t* hci, const T* hv, cudaStream_t s);

// ---- coarsest level: x = X b with X = A_L^{-1} dense symmetric (split-K, deterministic) ----
// Returns the status of its own two launches.
template <typename T>
cudaError_t dense_solve(int n, const double* X, const T* b, T* x, double* part, int kchunk, cudaStream_t s);
int dense_chunks(int n, int kchunk);

// ---- batched dense inversion (set-up): in-place Gauss-Jordan on symmetric positive
// (semi-)definite matrices. A pivot <= 1e-10 of its original diagonal excludes that DoF
// (zero row and column: the inverse of the remaining block); a negative or non-finite
// pivot flags the matrix as indefinite in bad[b]. Matrices sorted by size, descending.
struct GjBatch {
  int nmat = 0, max_n = 0;
  std::vector<int32_t> hn;     // host copy of the sizes
  int32_t* n = nullptr;        // [nmat]
  int64_t* off = nullptr;      // [nmat] offset of matrix b in M (row-major n_b x n_b)
  int64_t* voff = nullptr;     // [nmat] offset of matrix b in the per-DoF vectors
  double* M = nullptr;         // matrices, overwritten by their inverses
  double* diag0 = nullptr;     // original diagonals
  double *rowk = nullptr, *colk = nullptr;     // row and column k before pivot k (even k)
  double *rowk2 = nullptr, *colk2 = nullptr;   // the same for odd k
  double* piv = nullptr;       // [2 nmat] 1/p of the current pivot (0 if dropped), by parity of k
  int32_t* pdrop = nullptr;    // [2 nmat] the current pivot is dropped, by parity of k
  int32_t *bad = nullptr, *ndrop = nullptr;
};
void batched_spsd_inverse(const GjBatch& g, cudaStream_t s);
// max_i sum_j |M_ij| of each matrix of a batch (its 1-norm, M symmetric) into out[b].
void batched_norm1(const GjBatch& g, double* out, cudaStream_t s);

// ---- Lanczos (set-up): step j of nv <= 2 runs on the same scaled operator M (SELL-32, one
// lane per row), run r with vectors v[r], w[r], vprev[r] (length M.nrows), the rows it keeps
// keep[r] (null: all) and its scalar history hist[r] (alpha_k at 2k, beta_{k+1}^2 at 2k + 1):
// for j > 0 v = w / beta_j (vprev = the old v), then w = M v with alpha_j = w.v, then
// w -= alpha_j v + beta_j vprev (w = 0 outside keep) with beta_{j+1}^2 = |w|^2. The scalars
// stay on the device, so that several steps can be queued without a host round trip; each
// reduction is finished by the last block of the kernel that produces it (fixed order; part
// holds 2 x the blocks of one launch, ticket is a zeroed counter). ----
void lanczos_step(const SellMat<double>& M, int nv, double* const* v, double* const* w, double* const* vprev,
                  const uint8_t* const* keep, double* const* hist, int j, double* part, unsigned* ticket,
                  cudaStream_t s);

// ---- vectors ----
template <typename Src, typename Dst> void convert(int n, const Src* a, Dst* b, cudaStream_t s);
// b[i] = (Dst) a[perm[i]] (gather) and b[perm[i]] = (Dst) a[i] (scatter); perm == nullptr: convert.
template <typename Src, typename Dst> void gather(int n, const int32_t* perm, const Src* a, Dst* b, cudaStream_t s);
template <typename Src, typename Dst> void scatter(int n, const int32_t* perm, const Src* a, Dst* b, cudaStream_t s);
template <typename T> void axpy_from(int n, const T* z, double* x, cudaStream_t s);   // x += (double) z

// ---- CG (FP64 recurrence; the V-cycle vectors vb/vx are FP64 or FP32) ----
int cg_parts(int n);
// r = b, x = 0, reduction of b.b; V-cycle input vb = r (converted) and vx = 0.
template <typename T> void cg_init(int n, const double* b, double* r, double* x, T* vb, T* vx, const Reduce& rd, cudaStream_t s);
// x += alpha p, r -= alpha q, reduction of r.r; vb = r, vx = 0.
template <typename T>
void cg_update(int n, const CgState* st, const double* p, const double* q, double* x, double* r, T* vb, T* vx,
               const Reduce& rd, cudaStream_t s);
// reduction of r.z with z = (double) vx; with first: p = z.
template <typename T>
void cg_dotz(int n, const double* r, const T* vx, double* p, bool first, const Reduce& rd, cudaStream_t s);
// p = z + beta p with z = (double) vx.
template <typename T> void cg_pupdate(int n, const CgState* st, const T* vx, double* p, cudaStream_t s);
// reduction of |r|^2
void dot_self(int n, const double* r, const Reduce& rd, cudaStream_t s);

// ---- persistent execution of the lower V-cycle (persistent.cu) ----
// Task kinds. CSR tasks (G lanes per row, 32/G rows per warp unit; rows != null maps task row
// r to level row rows[r]): PK_CHEB_FIRST / PK_CHEB r = b - A x, d = c1 d + c2 D^-1 r (FIRST:
// d = c2 D^-1 r), y = x + d; PK_RESID y = b - A x; PK_RESTRICT y = A x and z = 0; PK_PROLONG
// y += A x; PK_SPMV y = A x. Elementwise (32 rows per unit): PK_CHEB0 d = c2 D^-1 b, y = x + d
// (x null: y = d); PK_COPY y = x. One patch row per unit (FP64): PK_PATCH_RES / PK_PATCH_RES_AP
// rbuf[r] = b[pdofs[r]] - (ELL row r of pv/pci, w slots, plen entries) . x; PK_PATCH_SOLVE
// y[g] += X_i . r over the row's patch (r = rbuf, or b[pdofs] when rbuf is null). One row per
// unit: PK_DENSE y_i = X_i . b (FP64, inv = row-major n x n; b from y64 when set, which the
// restriction into the coarsest level fills, so that b is converted to FP64 once).
// MG-PCG (FP64 recurrence, V-cycle vectors vb/vx of type T), 32 rows per unit unless CSR,
// each unit writing its partial sum to part[unit]: PK_CG_INIT r = b, x = 0, vb = r, vx = 0,
// partial b.b; PK_CG_AP (CSR, A_0 in FP64) q = A p, partial p.q; PK_CG_UPDATE x += alpha p,
// r -= alpha q, vb = r, vx = 0, partial r.r; PK_CG_DOTZ partial r.z with z = vx (w = 1: also
// p = z); PK_CG_PUPDATE p = z + beta p; PK_FINISH (one unit) sums part[0 .. w) in a fixed
// order and applies FinishOp op to the CG state st. A task with gate set does nothing once
// that CG state has stopped (gate->cont == 0).
enum PKind {
  PK_CHEB_FIRST = 1, PK_CHEB, PK_RESID, PK_RESTRICT, PK_PROLONG, PK_SPMV,
  PK_CHEB0, PK_COPY, PK_PATCH_RES, PK_PATCH_RES_AP, PK_PATCH_SOLVE, PK_DENSE,
  PK_CG_INIT, PK_CG_AP, PK_CG_UPDATE, PK_CG_DOTZ, PK_CG_PUPDATE, PK_FINISH
};
// One row of a patch solve: the patch's DoFs are pdofs[p0 .. p0 + n), this is its row i, whose
// inverse row starts at element inv of the arena.
struct PRow {
  int32_t p0, n, i, pad;
  int64_t inv;
};
struct PTask {
  int32_t kind, n, G, u0;        // u0: the task's first unit within its phase
  int32_t w, op;
  const int32_t *rp, *ci, *rows;
  const void* val;
  const void *x, *b, *dinv;
  void *d, *y, *z;
  double c1, c2;
  const int32_t *pdofs, *plen, *pci;
  const double* pv;
  double* rbuf;
  const PRow* prow;
  const double* inv;
  double* y64;                  // PK_RESTRICT: also y64 = (double) y; PK_DENSE: b read from here
  // MG-PCG
  const CgState* gate;
  CgState* st;
  double* part;
  const double* cb;
  double *cx, *cr, *cp, *cq;
  void *vb, *vx;
};
struct PPhase {
  int32_t t0, t1, units, check;   // tasks [t0, t1) and their units in total; check: see below
};
// Barrier state of one hierarchy's persistent launches (zero-initialised; count returns to 0
// after every complete barrier).
struct PBarrier {
  unsigned count, gen;
  int error, abort;
};
constexpr int kPersistentThreads = 1024;
constexpr int kPersistentBlocksPerSm = 1;
// Units of a task: CSR kinds 32/G rows per unit, elementwise 32 rows, patch and dense kinds one row.
inline int ptask_units(const PTask& t) {
  switch (t.kind) {
    case PK_CHEB0: case PK_COPY: case PK_CG_INIT: case PK_CG_UPDATE: case PK_CG_DOTZ: case PK_CG_PUPDATE:
      return (t.n + 31) / 32;
    case PK_PATCH_RES: case PK_PATCH_RES_AP: case PK_PATCH_SOLVE: case PK_DENSE: return t.n;
    case PK_FINISH: return 1;
    default: return (t.n + 32 / t.G - 1) / (32 / t.G);
  }
}
template <typename T> int persistent_grid();
// One cooperative launch walking phases[0 .. nhead) once with a grid barrier between phases;
// then, when nbody > 0, the body phases[nhead .. nhead + nbody) repeatedly: after the barrier
// that follows a body phase with check set, the loop ends unless some CG state of
// states[0 .. nstates) still has cont set (at most max_iter passes).
template <typename T>
cudaError_t persistent_launch(const PPhase* phases, int nhead, const PTask* tasks, PBarrier* bar, cudaStream_t s,
                              int nbody = 0, CgState* const* states = nullptr, int nstates = 0, int max_iter = 0);

void check_launch(const char* what);
// FP64 FMAs per second of the device (independent FMA chains on every SM, CUDA events).
double measure_fp64_fma(cudaStream_t s);

}  // namespace nnmg
