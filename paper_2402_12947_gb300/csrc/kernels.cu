// Device kernels of the nnmg hot path (sm_103a). See kernels.cuh for the data layout.
//
// Kernels and the steps they implement (Chen & Wells, arXiv:2402.12947):
//   sell_cheb      Chebyshev-Jacobi step of S_g (Sec. 3.2, Sec. 5): SpMV fused with the
//                  residual, the Jacobi scaling and the three-term update
//   sell_resid +   residual and restriction b_{l+1} = P_l^T (b_l - A_l u_l) (Eq. 4),
//   sell_restrict  R = P^T stored explicitly so that both are row-wise gathers
//   sell_prolong   coarse-grid correction u_l += P_l u_{l+1} (Alg. 1); sell_prolong_pr
//                  also forms the residual of the S_c that follows it
//   patch_*        local correction S_c (Sec. 4.1, Alg. 2): patch residual, then the dense
//                  FP64 solve with (A^[d])^{-1} and the scatter back
//   cheb_entry_local  S_c from a zero iterate and the first Chebyshev step in one launch
//   k_sell_tma     TMA-staged variant of the SpMV family (bulk copies into shared memory)
//   dense_solve    direct solve on the coarsest level (Alg. 1)
//   cg_*           CG preconditioned by one V-cycle (Sec. 6.2), deterministic reductions
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>
#include <stdexcept>
#include <string>
#include <type_traits>

#include "internal.hpp"
#include "kernels.cuh"

namespace nnmg {

void check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw Error(MG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

namespace {

// Streaming loads for matrix data (read once per pass; keep the vectors in L2).
__device__ __forceinline__ double ld_stream(const double* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }
__device__ __forceinline__ int32_t ld_stream(const int32_t* p) { return __ldcs(p); }

// Matrix operands of one launch, in one of two layouts:
//  * lanes == 1, SELL-32: slot `srow` (slice srow/32, lane srow%32) holds matrix row
//    perm[srow] (srow itself when perm is null); one thread accumulates one row;
//  * lanes == G > 1, CSR vector: G consecutive threads share row `slot`, stride over its
//    CSR entries (coalesced) and combine their partial sums with xor shuffles.
// Every vector access of an epilogue goes through the matrix row.
// Launch on stream s (plain stream order).
// Returns the launch's own status (callers that batch launches check check_launch later).
template <typename... KArgs, typename... Args>
cudaError_t launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.numAttrs = 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <typename T>
struct OpView {
  const int64_t* __restrict__ off;
  const int32_t* __restrict__ rp;
  const int32_t* __restrict__ col;
  const T* __restrict__ val;
  const int32_t* __restrict__ perm;
  const uint16_t* __restrict__ col16;   // 16-bit layouts: column = cbase + col16
  const int32_t* __restrict__ cbase;
  int nrows, nslices;
  int pf;   // SELL: bulk L2 prefetch of the slice pf slices ahead (0 = none)
};

// Asynchronous bulk prefetch of [p, p + bytes) into L2 (bytes a multiple of 16, p 16-byte
// aligned): no registers or shared memory, the copy engine streams it ahead of its use.
__device__ __forceinline__ void l2_prefetch(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint16_t ld_stream(const uint16_t* p) { return __ldcs(p); }

// Column index k: a 16-bit offset from the slice's/row's base column (narrow slices and
// rows), or the 32-bit index (cbase < 0 marks a slice or row too wide for 16 bits).
struct Col16 {
  const uint16_t* __restrict__ c;
  int base;
  __device__ __forceinline__ int operator()(int64_t k) const { return base + (int)ld_stream(c + k); }
};
struct Col32 {
  const int32_t* __restrict__ c;
  __device__ __forceinline__ int operator()(int64_t k) const { return ld_stream(c + k); }
};

// Sum over the w padded entries of one SELL-32 lane starting at element k (stride 32).
// PRED = false: four entries per step (their value and index loads together, then the x
// gathers, then the FMAs), the remaining w % 4 entries one at a time. PRED = true: every
// step takes STEP (4 or 8) entries, the last one predicated: the wider step keeps twice the
// loads in flight per thread at the cost of registers. All variants perform the same FMAs
// in the same order (identical results); which is fastest depends on the operator and
// precision.
template <typename T, bool PRED, int STEP = 4, typename C>
__device__ __forceinline__ T sell_lane(const T* __restrict__ vp, int64_t k, int w, C col, const T* __restrict__ x) {
  T acc = T(0);
  if constexpr (!PRED) {
    int j = 0;
    for (; j + 4 <= w; j += 4) {
      const T v0 = ld_stream(vp), v1 = ld_stream(vp + 32), v2 = ld_stream(vp + 64), v3 = ld_stream(vp + 96);
      const int c0 = col(k), c1 = col(k + 32), c2 = col(k + 64), c3 = col(k + 96);
      const T x0 = __ldg(x + c0), x1 = __ldg(x + c1), x2 = __ldg(x + c2), x3 = __ldg(x + c3);
      acc = fma(v0, x0, acc);
      acc = fma(v1, x1, acc);
      acc = fma(v2, x2, acc);
      acc = fma(v3, x3, acc);
      vp += 128;
      k += 128;
    }
    for (; j < w; ++j) {
      acc = fma(ld_stream(vp), __ldg(x + col(k)), acc);
      vp += 32;
      k += 32;
    }
  } else {
    for (int j = 0; j < w; j += STEP) {
      T v[STEP], xv[STEP];
      int c[STEP];
#pragma unroll
      for (int u = 0; u < STEP; ++u) v[u] = j + u < w ? ld_stream(vp + 32 * u) : T(0);
#pragma unroll
      for (int u = 0; u < STEP; ++u) c[u] = j + u < w ? col(k + 32 * u) : 0;
#pragma unroll
      for (int u = 0; u < STEP; ++u) xv[u] = j + u < w ? __ldg(x + c[u]) : T(0);
#pragma unroll
      for (int u = 0; u < STEP; ++u)
        if (j + u < w) acc = fma(v[u], xv[u], acc);
      vp += 32 * STEP;
      k += 32 * STEP;
    }
  }
  return acc;
}

template <typename T, bool C16, bool PRED, int STEP = 4>
__device__ __forceinline__ T sell_row(const OpView<T>& m, const T* __restrict__ x, int srow) {
  const int s = srow >> 5, lane = srow & 31;
  if (m.pf > 0 && lane == 0 && s + m.pf < m.nslices) {
    // the slice this warp's successor about pf / (resident warps) waves later will read
    const int t = s + m.pf;
    const int64_t a = m.off[t], e = m.off[t + 1];
    if (e > a) {
      l2_prefetch(m.val + a, (uint32_t)((e - a) * (int64_t)sizeof(T)));
      if (C16 && m.cbase[t] >= 0) l2_prefetch(m.col16 + a, (uint32_t)((e - a) * 2));
      else l2_prefetch(m.col + a, (uint32_t)((e - a) * 4));
    }
  }
  const int64_t o = m.off[s];
  const int w = (int)((m.off[s + 1] - o) >> 5);
  if constexpr (C16) {
    const int base = m.cbase[s];   // uniform across the warp (one slice per warp)
    if (base >= 0) return sell_lane<T, PRED, STEP>(m.val + o + lane, o + lane, w, Col16{m.col16, base}, x);
  }
  return sell_lane<T, PRED, STEP>(m.val + o + lane, o + lane, w, Col32{m.col}, x);
}

// CSR-vector partial sum of one lane of a G-lane group over row entries [k, k1), four
// strided entries per group, the last group predicated.
template <typename T, int G, typename C>
__device__ __forceinline__ T csrv_lane(const T* __restrict__ val, int k, int k1, C col, const T* __restrict__ x) {
  T a = T(0);
  for (; k < k1; k += 4 * G) {
    T v[4], xv[4];
    int c[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = k + u * G < k1 ? ld_stream(val + k + u * G) : T(0);
#pragma unroll
    for (int u = 0; u < 4; ++u) c[u] = k + u * G < k1 ? col(k + u * G) : 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) xv[u] = k + u * G < k1 ? __ldg(x + c[u]) : T(0);
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (k + u * G < k1) a = fma(v[u], xv[u], a);
  }
  return a;
}

// Kernel layout parameter G: 1 = SELL, one lane per row (steps of four, scalar remainder);
// 2 = the same with predicated steps; 6 = predicated steps of eight; 3 = SELL with 2 lanes
// per row and 5 = SELL with 4 lanes per row (predicated steps; a row's partial sums are
// combined by xor shuffles); G in {4, 8, 16, 32} = CSR vector with G lanes per row.
template <int G>
__host__ __device__ constexpr bool is_sell() {
  return G == 1 || G == 2 || G == 3 || G == 5 || G == 6;
}
template <int G>
__host__ __device__ constexpr int sell_sub() {
  return G == 3 ? 2 : (G == 5 ? 4 : 1);
}

// Row sum of the calling thread's row. Returns false for threads past the last row; for
// CSR vector every lane of a group receives the group's total (all lanes take part in the
// shuffles, so no lane leaves early).
template <typename T, int G, bool C16>
__device__ __forceinline__ bool op_row(const OpView<T>& m, const T* __restrict__ x, int& row, T& acc,
                                       int vblock = -1) {
  // vblock: the (virtual) block whose rows this thread serves (grid-stride kernels), else blockIdx.x
  const int tid = (vblock < 0 ? (int)blockIdx.x : vblock) * kBlock + threadIdx.x;
  if constexpr (is_sell<G>() && sell_sub<G>() == 1) {
    if (tid >= m.nrows) return false;
    row = m.perm ? m.perm[tid] : tid;
    acc = sell_row<T, C16, G != 1, G == 6 ? 8 : 4>(m, x, tid);
    return true;
  } else if constexpr (is_sell<G>()) {
    // one warp per slice (warp-uniform bounds), every lane runs the slice's steps and the
    // shuffles; lane l serves slot 32/S * slice + l / S
    constexpr int S = sell_sub<G>();
    const int sl = tid >> 5;
    T a = sl < m.nslices ? sell_row<T, C16, true>(m, x, tid) : T(0);
#pragma unroll
    for (int o = S / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    const int slot = sl * (32 / S) + ((tid & 31) / S);
    const bool valid = slot < m.nrows;
    row = valid ? (m.perm ? m.perm[slot] : slot) : 0;
    acc = a;
    return valid;
  } else {
    const int slot = tid / G, lane = tid & (G - 1);
    const bool valid = slot < m.nrows;
    row = valid ? slot : 0;
    T a = T(0);
    if (valid) {
      const int k0 = m.rp[row] + lane, k1 = m.rp[row + 1];
      const int base = C16 ? m.cbase[row] : -1;
      if (C16 && base >= 0) a = csrv_lane<T, G>(m.val, k0, k1, Col16{m.col16, base}, x);
      else a = csrv_lane<T, G>(m.val, k0, k1, Col32{m.col}, x);
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    acc = a;
    return valid;
  }
}

template <int G>
__device__ __forceinline__ bool group_leader() {
  if constexpr (is_sell<G>()) return (threadIdx.x & (sell_sub<G>() - 1)) == 0;
  else return (threadIdx.x & (G - 1)) == 0;
}

template <typename T, int G, bool C16>
__global__ void __launch_bounds__(kBlock) k_spmv(OpView<T> m, const T* __restrict__ x, T* __restrict__ y) {
  int row;
  T ax;
  if (!op_row<T, G, C16>(m, x, row, ax) || !group_leader<G>()) return;
  y[row] = ax;
}

template <typename T, int G, bool C16>
__global__ void __launch_bounds__(kBlock) k_resid(OpView<T> m, const T* __restrict__ x, const T* __restrict__ b,
                                                  T* __restrict__ r) {
  int row;
  T ax;
  if (!op_row<T, G, C16>(m, x, row, ax) || !group_leader<G>()) return;
  r[row] = b[row] - ax;
}

template <typename T, int G, bool C16, bool FIRST>
__global__ void __launch_bounds__(kBlock) k_cheb(OpView<T> m, const T* __restrict__ xin, const T* __restrict__ b,
                                                 const T* __restrict__ dinv, T* __restrict__ d, T* __restrict__ xout,
                                                 T cd, T cr) {
  int row;
  T ax;
  if (!op_row<T, G, C16>(m, xin, row, ax) || !group_leader<G>()) return;
  const T r = b[row] - ax;
  const T t = dinv[row] * r;
  const T dn = FIRST ? cr * t : fma(cd, d[row], cr * t);
  d[row] = dn;
  xout[row] = xin[row] + dn;
}

template <typename T, int G, bool C16>
__global__ void __launch_bounds__(kBlock) k_prolong(OpView<T> m, const T* __restrict__ xc, T* __restrict__ x) {
  int row;
  T ax;
  if (!op_row<T, G, C16>(m, xc, row, ax) || !group_leader<G>()) return;
  x[row] = x[row] + ax;
}

template <typename T, int G, bool C16>
__global__ void __launch_bounds__(kBlock) k_restrict(OpView<T> m, const T* __restrict__ r, T* __restrict__ bc,
                                                     T* __restrict__ xc) {
  int row;
  T ax;
  if (!op_row<T, G, C16>(m, r, row, ax) || !group_leader<G>()) return;
  bc[row] = ax;
  xc[row] = T(0);
}

// ---- TMA-staged SELL SpMV -------------------------------------------------------------
// A persistent kernel (grid = SMs x resident CTAs) for SELL with one lane per row and 32-bit
// indices. Chunk c (a run of whole slices, at most E padded entries) goes to CTA c mod grid.
// One producer thread streams each chunk's values and column indices into a shared-memory
// stage with two bulk copies (cp.async.bulk, completion counted on the stage's "full"
// mbarrier, L2 evict-first: the matrix is read once per pass, the vectors stay in L2); 16
// consumer warps take one slice each per step, read the slice's entries from shared memory,
// gather x from global memory and apply the epilogue to their rows, then release the stage
// on its "empty" mbarrier. The row sum has the same FMAs in the same order as the register
// variants. Every wait is bounded (about a second): on expiry the thread sets
// g_wait_timeout and stops; the producer still waits (bounded) for its copies in flight.
constexpr int kTmaConsumers = 16;
constexpr int kTmaThreads = 32 * (kTmaConsumers + 1);
constexpr int kTmaStages = 3;
constexpr int kTmaBarBytes = 128;

__device__ int g_wait_timeout;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
// Wait until the phase of parity `parity` has completed, for at most ~2^31 SM clocks (about
// a second); false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > (1ll << 31)) {
      atomicExch(&g_wait_timeout, 1);
      return false;
    }
  }
}
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
// bytes: a multiple of 16, both addresses 16-byte aligned
__device__ __forceinline__ void bulk_to_smem(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}

// Epilogues: load() reads the row's vector operands (issued before the row's gathers),
// store() finishes the row with the same arithmetic as the register kernels.
template <typename T, bool FIRST>
struct EpiCheb {
  const T *b, *dinv, *xin;
  T *d, *xout;
  T cd, cr;
  struct Pre {
    T b, dinv, d, xin;
  };
  __device__ __forceinline__ Pre load(int row) const {
    return Pre{b[row], dinv[row], FIRST ? T(0) : d[row], xin[row]};
  }
  __device__ __forceinline__ void store(int row, T ax, const Pre& p) const {
    const T r = p.b - ax;
    const T t = p.dinv * r;
    const T dn = FIRST ? cr * t : fma(cd, p.d, cr * t);
    d[row] = dn;
    xout[row] = p.xin + dn;
  }
};
template <typename T>
struct EpiResid {
  const T* b;
  T* r;
  struct Pre {
    T b;
  };
  __device__ __forceinline__ Pre load(int row) const { return Pre{b[row]}; }
  __device__ __forceinline__ void store(int row, T ax, const Pre& p) const { r[row] = p.b - ax; }
};
template <typename T>
struct EpiSpmv {
  T* y;
  struct Pre {};
  __device__ __forceinline__ Pre load(int) const { return Pre{}; }
  __device__ __forceinline__ void store(int row, T ax, const Pre&) const { y[row] = ax; }
};

template <typename T, typename Epi>
__global__ void __launch_bounds__(kTmaThreads, 1) k_sell_tma(OpView<T> m, const int32_t* __restrict__ chunks,
                                                             int nchunks, const T* __restrict__ x, Epi epi) {
  constexpr int E = tma_stage_entries<T>();
  extern __shared__ __align__(128) unsigned char tsm[];
  uint64_t* full = reinterpret_cast<uint64_t*>(tsm);
  uint64_t* empty = full + kTmaStages;
  T* sval = reinterpret_cast<T*>(tsm + kTmaBarBytes);
  int32_t* scol = reinterpret_cast<int32_t*>(tsm + kTmaBarBytes + (size_t)kTmaStages * E * sizeof(T));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTmaStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kTmaConsumers);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp == kTmaConsumers) {  // producer
    if (lane != 0) return;
    const uint64_t pol = l2_evict_first();
    int k = 0;
    for (int c = blockIdx.x; c < nchunks; c += gridDim.x, ++k) {
      const int s = k % kTmaStages;
      const int use = k / kTmaStages;
      if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1)) break;
      const int64_t e0 = m.off[chunks[c]], e1 = m.off[chunks[c + 1]];
      const uint32_t n = (uint32_t)(e1 - e0);
      if (n == 0) {
        mbar_arrive(&full[s]);
        continue;
      }
      mbar_expect_tx(&full[s], n * (uint32_t)(sizeof(T) + sizeof(int32_t)));
      bulk_to_smem(sval + (size_t)s * E, m.val + e0, n * (uint32_t)sizeof(T), &full[s], pol);
      bulk_to_smem(scol + (size_t)s * E, m.col + e0, n * (uint32_t)sizeof(int32_t), &full[s], pol);
    }
    // copies still in flight (normally consumed already) complete before the CTA exits
    for (int j = k > kTmaStages ? k - kTmaStages : 0; j < k; ++j) mbar_wait(&full[j % kTmaStages], (j / kTmaStages) & 1);
    return;
  }
  int k = 0;
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x, ++k) {
    const int s = k % kTmaStages;
    if (!mbar_wait(&full[s], (k / kTmaStages) & 1)) return;
    const int s0 = chunks[c], s1 = chunks[c + 1];
    const int64_t cb = m.off[s0];
    const T* vs = sval + (size_t)s * E;
    const int32_t* cs = scol + (size_t)s * E;
    for (int sl = s0 + warp; sl < s1; sl += kTmaConsumers) {
      const int slot = sl * 32 + lane;
      const bool live = slot < m.nrows;
      const int row = live ? (m.perm ? m.perm[slot] : slot) : 0;
      typename Epi::Pre pre{};
      if (live) pre = epi.load(row);
      const int64_t o = m.off[sl];
      const int w = (int)((m.off[sl + 1] - o) >> 5);
      const int b0 = (int)(o - cb) + lane;
      T acc = T(0);
      for (int j = 0; j < w; j += 8) {
        T v[8], xv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const bool ok = j + u < w;
          v[u] = ok ? vs[b0 + (j + u) * 32] : T(0);
          xv[u] = ok ? __ldg(x + cs[b0 + (j + u) * 32]) : T(0);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (j + u < w) acc = fma(v[u], xv[u], acc);
      }
      if (live) epi.store(row, acc, pre);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
}

// One colour of a multicolour Gauss-Seidel sweep. m holds the colour's rows without their
// diagonal and without couplings between rows of the colour; rows[] maps its rows to the
// level's. x_i = dinv_i (b_i - sum_j a_ij x_j). The kernel reads x (through xr) only at
// entries of other colours and writes only its own colour's entries.
template <typename T, int G, bool C16>
__global__ void __launch_bounds__(kBlock) k_gs(OpView<T> m, const int32_t* __restrict__ rows,
                                               const T* __restrict__ xr, const T* __restrict__ b,
                                               const T* __restrict__ dinv, T* x) {
  int r;
  T s;
  if (!op_row<T, G, C16>(m, xr, r, s) || !group_leader<G>()) return;
  const int i = rows[r];
  x[i] = dinv[i] * (b[i] - s);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum in a fixed order (warp shuffles, then the warps' sums by warp 0).
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double ws[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) ws[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  double t = 0.0;
  if (w == 0) {
    t = l < nw ? ws[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

constexpr int kCgBlocks = 152 * 4;
// Every thread of the block calls this with the block's partial s (valid in thread 0, as
// block_sum returns it). The last block to arrive sums all partials in index order.
__device__ void reduce_finish(double s, const Reduce& rd) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    rd.part[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(rd.ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;  // block-uniform
  __threadfence();
  // eight independent loads per step (up to 16k partials for the fine-level SpMV grid);
  // the summation order is fixed by the block size and the partial count
  const int np = (int)gridDim.x, bd = (int)blockDim.x;
  double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int i = threadIdx.x;
  for (; i + 7 * bd < np; i += 8 * bd) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = __ldcg(rd.part + i + u * bd);
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] += v[u];
  }
  for (; i < np; i += bd) acc[0] += __ldcg(rd.part + i);
  double t = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
  t = block_sum(t);
  if (threadIdx.x == 0) {
    apply_finish(rd.st, t, rd.op, rd.use_cond, rd.handle);
    *rd.ticket = 0u;
  }
}

// Every thread of the block calls this with the block's partials s[0 .. nv) (valid in thread 0),
// nv <= 2; the last block to arrive sums each run's partials in index order into *out[r] and
// resets the ticket. part holds gridDim.x entries per run.
__device__ void reduce_to2(int nv, const double* s, double* part, unsigned* ticket, double* const* out) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    for (int r = 0; r < nv; ++r) part[r * gridDim.x + blockIdx.x] = s[r];
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;  // block-uniform
  __threadfence();
  for (int r = 0; r < nv; ++r) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) acc += __ldcg(part + r * gridDim.x + i);
    acc = block_sum(acc);
    if (threadIdx.x == 0) *out[r] = acc;
    __syncthreads();   // block_sum's shared words are reused by the next run
  }
  if (threadIdx.x == 0) *ticket = 0u;
}

// One or two Lanczos runs on the same scaled operator S (set-up), advanced together: run r has
// its vectors v, w, vprev, the rows it keeps (null: all) and its scalar history (alpha_k at 2k,
// beta_{k+1}^2 at 2k + 1). Each run's arithmetic is that of a run alone.
struct LzRuns {
  int nv;
  double* v[2];
  double* w[2];
  double* vprev[2];
  const uint8_t* keep[2];
  double* hist[2];
};

// Step j: w = S v and alpha = w.v for every run in one launch (the operator's rows are read by
// the first run and found in cache by the second).
template <int G, bool C16>
__global__ void __launch_bounds__(kBlock) k_lz_spmv_dot(OpView<double> m, LzRuns z, int j, double* part,
                                                        unsigned* ticket) {
  double s[2] = {0.0, 0.0};
  double* out[2];
  for (int r = 0; r < z.nv; ++r) {
    int row;
    double ax;
    if (op_row<double, G, C16>(m, z.v[r], row, ax) && group_leader<G>()) {
      z.w[r][row] = ax;
      s[r] = ax * z.v[r][row];
    }
    s[r] = block_sum(s[r]);
    __syncthreads();
    out[r] = z.hist[r] + 2 * j;
  }
  reduce_to2(z.nv, s, part, ticket, out);
}

// q = A p with the p.q reduction in the same launch. The grid (one resident wave) walks
// the operator's blocks of rows (`nvb` virtual blocks, grid-stride, a fixed assignment), each
// thread accumulating p_i q_i of its rows in a register; one block reduction per block, then
// the last block to finish sums the block partials in order and applies the reduction's op
// (reduce_finish). On GB300 this operator pass is bound by the FP64 pipe (one FMA per nonzero):
// a block reduction for every 256 rows added about 30 % more FP64 instructions.
template <int G, bool C16>
__global__ void __launch_bounds__(kBlock) k_ap(OpView<double> m, int nvb, const double* __restrict__ p,
                                               double* __restrict__ q, Reduce rd) {
  double v = 0.0;
  for (int vb = blockIdx.x; vb < nvb; vb += gridDim.x) {   // block-uniform loop
    int row;
    double ap;
    if (op_row<double, G, C16>(m, p, row, ap, vb) && group_leader<G>()) {
      q[row] = ap;
      v = fma(p[row], ap, v);
    }
  }
  reduce_finish(block_sum(v), rd);
}

// First Chebyshev step from a zero iterate: r = b, d = cr D^{-1} b, x_out = x_in + d for
// every row (x_in is zero there) ...
template <typename T>
__global__ void __launch_bounds__(kBlock) k_cheb0_all(int n, const T* __restrict__ b, const T* __restrict__ dinv,
                                                      const T* __restrict__ xin, T* __restrict__ d,
                                                      T* __restrict__ xout, T cr) {
  const int i = blockIdx.x * kBlock + threadIdx.x;
  if (i >= n) return;
  const T t = dinv[i] * b[i];
  const T dn = cr * t;
  d[i] = dn;
  xout[i] = xin[i] + dn;
}

// ... then the rows coupled to patch DoFs (where x_in may be non-zero after S_c) are redone
// with their full row: r = b - A x_in. One warp per such row.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_cheb0_halo(int nh, const int32_t* __restrict__ hrow,
                                                       const int32_t* __restrict__ hrp, const int32_t* __restrict__ hci,
                                                       const T* __restrict__ hv, const T* __restrict__ b,
                                                       const T* __restrict__ dinv, const T* __restrict__ xin,
                                                       T* __restrict__ d, T* __restrict__ xout, T cr) {
  const int t = (blockIdx.x * kBlock + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  T ax = T(0);
  if (t < nh)
    for (int k = hrp[t] + lane; k < hrp[t + 1]; k += 32) ax = fma(hv[k], xin[hci[k]], ax);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ax += __shfl_xor_sync(0xffffffffu, ax, o);
  if (t >= nh || lane != 0) return;
  const int i = hrow[t];
  const T r = b[i] - ax;
  const T tt = dinv[i] * r;
  const T dn = cr * tt;
  d[i] = dn;
  xout[i] = xin[i] + dn;
}

// Sum of row t of an ELL block (w slots per row, the row's len entries first) against x,
// one warp per row, lane l taking entries l, l + 32, ...: the first 32 slots are loaded
// without waiting for the row length (padding slots hold value 0 and a valid column), the
// rest only up to len, so padded slots cost neither bytes nor FP64 FMAs beyond the first 32.
template <typename T>
__device__ __forceinline__ double ell_row_sum(int64_t r0, int w, int len, const int32_t* __restrict__ ci,
                                              const double* __restrict__ v, const T* __restrict__ x, int lane) {
  double s = 0.0;
  if (lane < w) {
    const double a = v[r0 + lane];
    const double xv = (double)x[ci[r0 + lane]];
    if (lane < len) s = fma(a, xv, s);
  }
  for (int k = lane + 32; k < len; k += 32) s = fma(v[r0 + k], (double)x[ci[r0 + k]], s);
  return warp_sum(s);
}

// S_c phase 1: r_B = b_B - (A x)_B for every patch row, one warp per row (FP64).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_patch_residual(int nt, int w, const int32_t* __restrict__ pdofs,
                                                           const int32_t* __restrict__ plen,
                                                           const int32_t* __restrict__ pci,
                                                           const double* __restrict__ pv, const T* __restrict__ b,
                                                           const T* __restrict__ x, double* __restrict__ rbuf) {
  const int t = (blockIdx.x * kBlock + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (t >= nt) return;  // warp-uniform
  const double bt = (double)b[pdofs[t]];
  const double s = ell_row_sum<T>((int64_t)t * w, w, plen[t], pci, pv, x, lane);
  if (lane == 0) rbuf[t] = bt - s;
}

// Coarse-grid correction x += P x_c fused with the residual of the S_c that follows it: the
// residual before the correction, res = b - A x (kept from the restriction), gives
// r_B = res_B - (A P)_B x_c on the patch rows, with the rows (A P)_{i,:} of the patch rows
// precomputed (ELL, w entries each, FP64). Blocks [0, nbp) run the prolongation, the others
// one warp per patch row. Neither part reads what the other writes.
template <typename T, int G, bool C16>
__global__ void __launch_bounds__(kBlock) k_prolong_pr(OpView<T> m, const T* __restrict__ xc, T* __restrict__ x,
                                                       int nbp, int nt, int w, const int32_t* __restrict__ pdofs,
                                                       const int32_t* __restrict__ aplen,
                                                       const int32_t* __restrict__ apci,
                                                       const double* __restrict__ apv, const T* __restrict__ res,
                                                       double* __restrict__ rbuf) {
  if ((int)blockIdx.x >= nbp) {  // block-uniform
    const int t = (((int)blockIdx.x - nbp) * kBlock + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (t >= nt) return;  // warp-uniform
    const double rt = (double)res[pdofs[t]];
    const double acc = ell_row_sum<T>((int64_t)t * w, w, aplen[t], apci, apv, xc, lane);
    if (lane == 0) rbuf[t] = rt - acc;
    return;
  }
  int row;
  T ax;
  if (!op_row<T, G, C16>(m, xc, row, ax) || !group_leader<G>()) return;
  x[row] = x[row] + ax;
}

// S_c phase 2: e = (A^[d])^{-1} r_B and x_B += e, one launch over the work list. A work item
// is kPatchRowsPerItem (32) consecutive rows of one patch, one block per item: lane l owns row
// i = row0 + l, and the block's eight warps split the columns, warp w taking j = w, w + 8, ...
// The inverse X is symmetric, so row i's entry j is read as X[j][i]: for each j the warp reads
// X[j][row0 .. row0 + 31], 256 contiguous bytes, and every FMA of a warp instruction is one of
// the product's (no per-row warp reduction). The eight partial sums of a row are added in
// warp order through shared memory. The patch residual is staged in shared memory first (b
// itself when the iterate is zero, rbuf == nullptr). Items sorted by patch size, largest first.
// FP32 items (mixed form, well-conditioned patches): X and the staged residual in FP32, FP32
// FMAs, the result added to x in FP64 and rounded to T.
constexpr int kPatchWarps = kBlock / 32;

template <typename T, typename V>
__device__ __forceinline__ void patch_item_rows(const PatchItem it, const int32_t* __restrict__ pdofs,
                                                const V* __restrict__ X, const double* rbuf,
                                                const T* __restrict__ b, T* __restrict__ x, V* rs) {
  __shared__ V red[kPatchWarps][32];
  const int p0 = it.p0, n = it.n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = it.row0 + lane;
  const bool ok = i < n;
  const int g = warp == 0 && ok ? pdofs[p0 + i] : 0;
  const T xg = warp == 0 && ok ? x[g] : T(0);
  for (int j = threadIdx.x; j < n; j += blockDim.x) rs[j] = (V)(rbuf ? rbuf[p0 + j] : (double)b[pdofs[p0 + j]]);
  __syncthreads();
  const V* Xc = X + it.row0 + lane;
  V e[2] = {V(0), V(0)};
  int j = warp;
  for (; j + 7 * kPatchWarps < n; j += 8 * kPatchWarps) {   // eight rows of X in flight per lane
    V v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = ok ? Xc[(int64_t)(j + u * kPatchWarps) * n] : V(0);
#pragma unroll
    for (int u = 0; u < 8; ++u) e[u & 1] = fma(v[u], rs[j + u * kPatchWarps], e[u & 1]);
  }
  for (; j < n; j += kPatchWarps) e[0] = fma(ok ? Xc[(int64_t)j * n] : V(0), rs[j], e[0]);
  red[warp][lane] = e[0] + e[1];
  __syncthreads();
  if (warp != 0 || !ok) return;
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < kPatchWarps; ++w) s += (double)red[w][lane];
  x[g] = (T)((double)xg + s);
}

// Small patches (n <= kSmallPatch): one warp per output row, lane l accumulating entries
// l, l + 32, ... of row i of X (contiguous), then the warp sums; the row's first 256 entries
// and its DoF id and value are loaded before the barrier that stages the residual, so an item
// costs about two dependent memory round trips.
template <typename T, typename V>
__device__ __forceinline__ void patch_item_warp(const PatchItem it, const int32_t* __restrict__ pdofs,
                                                const V* __restrict__ X, const double* rbuf,
                                                const T* __restrict__ b, T* __restrict__ x, V* rs) {
  constexpr int K = 8;
  const int p0 = it.p0, n = it.n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = it.row0 + warp;
  const bool ok = i < n;
  const V* Xi = X + (int64_t)(ok ? i : 0) * n;
  const int g = ok ? pdofs[p0 + i] : 0;
  const T xg = ok ? x[g] : T(0);
  V xr[K];
#pragma unroll
  for (int u = 0; u < K; ++u) xr[u] = ok && lane + 32 * u < n ? Xi[lane + 32 * u] : V(0);
  for (int j = threadIdx.x; j < n; j += blockDim.x) rs[j] = (V)(rbuf ? rbuf[p0 + j] : (double)b[pdofs[p0 + j]]);
  __syncthreads();
  if (!ok) return;  // warp-uniform; no block barrier follows
  V e = V(0);
#pragma unroll
  for (int u = 0; u < K; ++u)
    if (lane + 32 * u < n) e = fma(xr[u], rs[lane + 32 * u], e);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if (lane == 0) x[g] = (T)((double)xg + (double)e);
}

template <typename T>
__device__ __forceinline__ void patch_item(const PatchItem it, const int32_t* __restrict__ pdofs,
                                           const double* __restrict__ inv, const float* __restrict__ inv32,
                                           const double* rbuf, const T* __restrict__ b, T* __restrict__ x,
                                           double* rs) {
  const bool lo = (it.mode & PI_FP32) != 0;
  if (it.mode & PI_WARP_ROWS) {
    if (lo) patch_item_warp<T, float>(it, pdofs, inv32 + it.inv, rbuf, b, x, reinterpret_cast<float*>(rs));
    else patch_item_warp<T, double>(it, pdofs, inv + it.inv, rbuf, b, x, rs);
  } else {
    if (lo) patch_item_rows<T, float>(it, pdofs, inv32 + it.inv, rbuf, b, x, reinterpret_cast<float*>(rs));
    else patch_item_rows<T, double>(it, pdofs, inv + it.inv, rbuf, b, x, rs);
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_patch_solve(const PatchItem* __restrict__ items,
                                                        const int32_t* __restrict__ pdofs,
                                                        const double* __restrict__ inv,
                                                        const float* __restrict__ inv32, const double* rbuf,
                                                        const T* __restrict__ b, T* __restrict__ x) {
  extern __shared__ double rs[];
  patch_item<T>(items[blockIdx.x], pdofs, inv, inv32, rbuf, b, x, rs);
}

// Start of a pre-smoothing S_c, S_g, ... from a zero iterate, in one launch: blocks
// [0, nitems) run the S_c work items with residual b (x_B = (A^[d])^{-1} b_B into x), the
// others the first Chebyshev step for every row as if x were zero everywhere (d = cr D^{-1} b,
// x_out = d). The two parts write disjoint arrays (x; d and x_out). The rows coupled to patch
// DoFs, whose residual does see x_B, are redone afterwards by k_cheb0_halo.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_cheb0_entry(int nitems, const PatchItem* __restrict__ items,
                                                        const int32_t* __restrict__ pdofs,
                                                        const double* __restrict__ inv,
                                                        const float* __restrict__ inv32, int n,
                                                        const T* __restrict__ b, const T* __restrict__ dinv,
                                                        T* __restrict__ x, T* __restrict__ d, T* __restrict__ xout,
                                                        T cr) {
  extern __shared__ double rs[];
  if ((int)blockIdx.x < nitems) {  // block-uniform
    patch_item<T>(items[blockIdx.x], pdofs, inv, inv32, nullptr, b, x, rs);
    return;
  }
  const int i = ((int)blockIdx.x - nitems) * kBlock + threadIdx.x;
  if (i >= n) return;
  const T t = dinv[i] * b[i];
  const T dn = cr * t;
  d[i] = dn;
  xout[i] = dn;
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_dense_partial(int n, int kchunk, const double* __restrict__ X,
                                                          const T* __restrict__ b, double* __restrict__ part) {
  extern __shared__ double bs[];
  const int k0 = blockIdx.y * kchunk, k1 = min(n, k0 + kchunk);
  for (int j = k0 + threadIdx.x; j < k1; j += blockDim.x) bs[j - k0] = (double)b[j];
  __syncthreads();
  const int i = blockIdx.x * kBlock + threadIdx.x;
  if (i >= n) return;
  const double* Xi = X + i;
  // eight column loads issued together (coalesced across the block's rows), then their FMAs
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int j = k0; j < k1; j += 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = j + u < k1 ? Xi[(int64_t)(j + u) * n] : 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (j + u < k1) s[u & 3] = fma(v[u], bs[j + u - k0], s[u & 3]);
  }
  part[(int64_t)blockIdx.y * n + i] = (s[0] + s[1]) + (s[2] + s[3]);
}

// x_i = sum over chunks of part[c][i]: one warp per row, lanes over the chunks (fixed order).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_dense_reduce(int n, int nchunks, const double* __restrict__ part,
                                                         T* __restrict__ x) {
  const int i = (blockIdx.x * kBlock + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= n) return;  // warp-uniform
  double s = 0.0;
  for (int c = lane; c < nchunks; c += 32) s += part[(int64_t)c * n + i];
  s = warp_sum(s);
  if (lane == 0) x[i] = (T)s;
}

template <typename Src, typename Dst>
__global__ void k_convert(int n, const Src* __restrict__ a, Dst* __restrict__ b) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = (Dst)a[i];
}

template <typename Src, typename Dst>
__global__ void k_gather(int n, const int32_t* __restrict__ perm, const Src* __restrict__ a, Dst* __restrict__ b) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = (Dst)a[perm[i]];
}

template <typename Src, typename Dst>
__global__ void k_scatter(int n, const int32_t* __restrict__ perm, const Src* __restrict__ a, Dst* __restrict__ b) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[perm[i]] = (Dst)a[i];
}

template <typename T>
__global__ void k_axpy_from(int n, const T* __restrict__ z, double* __restrict__ x) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] += (double)z[i];
}

// The CG vector kernels walk the vectors grid-stride (608 blocks, 4 of 256 threads per SM)
// four strides per step: the step issues the loads of all four elements before their
// arithmetic, so that a thread has four elements' bytes in flight. Each thread's partial sum is
// accumulated in element order, so the reductions stay deterministic.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_cg_init(int n, const double* __restrict__ b, double* __restrict__ r,
                                                    double* __restrict__ x, T* __restrict__ vb, T* __restrict__ vx,
                                                    Reduce rd) {
  double s = 0.0;
  const int st = gridDim.x * kBlock;
  int i = blockIdx.x * kBlock + threadIdx.x;
  for (; i + 3 * st < n; i += 4 * st) {
    double bv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) bv[u] = b[i + u * st];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int k = i + u * st;
      r[k] = bv[u];
      x[k] = 0.0;
      if constexpr (!std::is_same<T, double>::value) vb[k] = (T)bv[u];  // FP64: vb is r itself
      vx[k] = T(0);
      s = fma(bv[u], bv[u], s);
    }
  }
  for (; i < n; i += st) {
    const double bi = b[i];
    r[i] = bi;
    x[i] = 0.0;
    if constexpr (!std::is_same<T, double>::value) vb[i] = (T)bi;
    vx[i] = T(0);
    s = fma(bi, bi, s);
  }
  reduce_finish(block_sum(s), rd);
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_cg_update(int n, const CgState* __restrict__ stt, const double* __restrict__ p,
                                                      const double* __restrict__ q, double* __restrict__ x,
                                                      double* __restrict__ r, T* __restrict__ vb, T* __restrict__ vx,
                                                      Reduce rd) {
  const double a = stt->alpha;
  double s = 0.0;
  const int st = gridDim.x * kBlock;
  int i = blockIdx.x * kBlock + threadIdx.x;
  for (; i + 3 * st < n; i += 4 * st) {
    double pv[4], qv[4], xv[4], rv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      pv[u] = p[i + u * st];
      qv[u] = q[i + u * st];
      xv[u] = x[i + u * st];
      rv[u] = r[i + u * st];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int k = i + u * st;
      x[k] = fma(a, pv[u], xv[u]);
      const double ri = fma(-a, qv[u], rv[u]);
      r[k] = ri;
      if constexpr (!std::is_same<T, double>::value) vb[k] = (T)ri;  // FP64: vb is r itself
      vx[k] = T(0);
      s = fma(ri, ri, s);
    }
  }
  for (; i < n; i += st) {
    x[i] = fma(a, p[i], x[i]);
    const double ri = fma(-a, q[i], r[i]);
    r[i] = ri;
    if constexpr (!std::is_same<T, double>::value) vb[i] = (T)ri;
    vx[i] = T(0);
    s = fma(ri, ri, s);
  }
  reduce_finish(block_sum(s), rd);
}

template <typename T, bool FIRST>
__global__ void __launch_bounds__(kBlock) k_cg_dotz(int n, const double* __restrict__ r, const T* __restrict__ vx,
                                                    double* __restrict__ p, Reduce rd) {
  double s = 0.0;
  const int st = gridDim.x * kBlock;
  int i = blockIdx.x * kBlock + threadIdx.x;
  for (; i + 3 * st < n; i += 4 * st) {
    double zv[4], rv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      zv[u] = (double)vx[i + u * st];
      rv[u] = r[i + u * st];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (FIRST) p[i + u * st] = zv[u];
      s = fma(rv[u], zv[u], s);
    }
  }
  for (; i < n; i += st) {
    const double zi = (double)vx[i];
    if (FIRST) p[i] = zi;
    s = fma(r[i], zi, s);
  }
  reduce_finish(block_sum(s), rd);
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_cg_pupdate(int n, const CgState* __restrict__ stt, const T* __restrict__ vx,
                                                       double* __restrict__ p) {
  const double beta = stt->beta;
  const int st = gridDim.x * kBlock;
  int i = blockIdx.x * kBlock + threadIdx.x;
  for (; i + 3 * st < n; i += 4 * st) {
    double zv[4], pv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      zv[u] = (double)vx[i + u * st];
      pv[u] = p[i + u * st];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) p[i + u * st] = fma(beta, pv[u], zv[u]);
  }
  for (; i < n; i += st) p[i] = fma(beta, p[i], (double)vx[i]);
}

__global__ void __launch_bounds__(kBlock) k_dot_self(int n, const double* __restrict__ r, Reduce rd) {
  double s = 0.0;
  const int st = gridDim.x * kBlock;
  int i = blockIdx.x * kBlock + threadIdx.x;
  for (; i + 3 * st < n; i += 4 * st) {
    double rv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) rv[u] = r[i + u * st];
#pragma unroll
    for (int u = 0; u < 4; ++u) s = fma(rv[u], rv[u], s);
  }
  for (; i < n; i += st) s = fma(r[i], r[i], s);
  reduce_finish(block_sum(s), rd);
}

inline int grid_for(int n, int per) { return (n + per - 1) / per; }

// ---- Lanczos on the scaled operator S (set-up) ----
// Step j: w -= alpha v + beta vprev with beta = sqrt(beta_j^2) (0 at j = 0), and w = 0 outside
// the run's kept rows; |w|^2 = beta_{j+1}^2 into the history (last block), for every run.
__global__ void __launch_bounds__(kBlock) k_lz_update(int n, LzRuns z, int j, double* part, unsigned* ticket) {
  double s[2] = {0.0, 0.0};
  double* out[2];
  for (int r = 0; r < z.nv; ++r) {
    const double a = z.hist[r][2 * j];
    const double beta = j > 0 ? sqrt(z.hist[r][2 * j - 1]) : 0.0;
    const double* __restrict__ v = z.v[r];
    const double* __restrict__ vp = z.vprev[r];
    const uint8_t* __restrict__ keep = z.keep[r];
    double* __restrict__ w = z.w[r];
    double acc = 0.0;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
      const double wi = keep && !keep[i] ? 0.0 : w[i] - (a * v[i] + beta * vp[i]);
      w[i] = wi;
      acc = fma(wi, wi, acc);
    }
    s[r] = block_sum(acc);
    __syncthreads();
    out[r] = z.hist[r] + 2 * j + 1;
  }
  reduce_to2(z.nv, s, part, ticket, out);
}

// Step j > 0: vprev = v, v = w / beta with beta = sqrt(beta_j^2), for every run.
__global__ void __launch_bounds__(kBlock) k_lz_next(int n, LzRuns z, int j) {
  for (int r = 0; r < z.nv; ++r) {
    const double inv_beta = 1.0 / sqrt(z.hist[r][2 * j - 1]);
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
      z.vprev[r][i] = z.v[r][i];
      z.v[r][i] = z.w[r][i] * inv_beta;
    }
  }
}

constexpr double kGjDrop = 1e-10;

// Pivot rule of the batched sweep (semi-definite blocks): pivot k of a matrix is dropped when
// its current value p is at most kGjDrop times the original diagonal d0 (row and column k of
// the result are then zero); p below -kGjDrop d0, a non-positive d0 or a non-finite p marks the
// matrix as not positive semi-definite. Otherwise the step is the Gauss-Jordan update with
// pinv = 1/p: M[k][k] = pinv, M[k][j] = M[k][j] pinv, M[i][k] = -M[i][k] pinv and
// M[i][j] = fma(-M[i][k] pinv, M[k][j], M[i][j]) with row and column k taken before the step.

// The large matrices' sweep, one launch per pivot. rowk / colk hold row k and column k of
// every active matrix as they are before pivot k, and piv / pdrop the pivot's 1/p and drop
// decision (written by the previous step, or by k_gj_snap0 for k = 0; the buffers alternate
// with the parity of k). Step k applies the update to every element in place (element (i, j)
// reads only M[i][j] and the snapshot), writes the updated row and column k + 1 into the other
// snapshot buffers, and the thread that computes the new M[k+1][k+1] decides pivot k + 1. The
// kernel is bound by the FP64 pipe: one division per pivot instead of one per thread, and the
// row factor -M[i][k]/p formed once per row of a thread's 8 x 2 elements (64 x 64 tiles).
__device__ __forceinline__ void gj_decide(const GjBatch& g, int b, int k, double p, double* piv, int32_t* pdrop) {
  const double d0 = g.diag0[g.voff[b] + k];
  const bool bad = !(d0 > 0.0) || !isfinite(p) || p < -kGjDrop * d0;
  const bool drop = bad || p <= kGjDrop * d0;
  piv[b] = drop ? 0.0 : 1.0 / p;
  pdrop[b] = drop ? 1 : 0;
  if (bad) g.bad[b] = 1;
  if (drop) g.ndrop[b] += 1;
}

__global__ void k_gj_snap0(GjBatch g) {
  const int b = blockIdx.x;
  const int n = g.n[b];
  const double* M = g.M + g.off[b];
  double* rk = g.rowk + g.voff[b];
  double* ck = g.colk + g.voff[b];
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    rk[j] = M[j];
    ck[j] = M[(int64_t)j * n];
  }
  if (threadIdx.x == 0 && n > 0) gj_decide(g, b, 0, M[0], g.piv, g.pdrop);
}

constexpr int kGjTile = 64;   // rows and columns of a k_gj_step tile (8 rows x 2 columns per thread)

__global__ void __launch_bounds__(kBlock) k_gj_step(GjBatch g, int k, int tiles_x, const double* __restrict__ rk_all,
                                                    const double* __restrict__ ck_all, double* __restrict__ rk_next,
                                                    double* __restrict__ ck_next, const double* __restrict__ piv,
                                                    const int32_t* __restrict__ pdrop, double* piv_next,
                                                    int32_t* pdrop_next) {
  const int b = blockIdx.y;
  const int n = g.n[b];
  if (k >= n) return;
  const int ti = blockIdx.x / tiles_x, tj = blockIdx.x - ti * tiles_x;
  if (ti * kGjTile >= n || tj * kGjTile >= n) return;   // block-uniform
  const int lane = threadIdx.x & 31;
  const int i0 = ti * kGjTile + (threadIdx.x >> 5) * 8;
  const int j0 = tj * kGjTile + lane;
  double* M = g.M + g.off[b];
  const double* rk = rk_all + g.voff[b];
  const double* ck = ck_all + g.voff[b];
  double* rn = rk_next + g.voff[b];
  double* cn = ck_next + g.voff[b];
  const double pinv = piv[b];
  const bool drop = pdrop[b] != 0;
  double rkj[2], f[8], m[8][2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int j = j0 + 32 * c;
    rkj[c] = j < n && !drop ? rk[j] : 0.0;
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = i0 + r;
    f[r] = i < n ? -ck[i] * pinv : 0.0;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int j = j0 + 32 * c;
      m[r][c] = i < n && j < n ? M[(int64_t)i * n + j] : 0.0;
    }
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = i0 + r;
    if (i >= n) break;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int j = j0 + 32 * c;
      if (j >= n) continue;
      double v;
      if (drop) {
        if (i != k && j != k) continue;   // unchanged, and neither snapshot nor pivot k + 1 is here
        v = 0.0;
      } else if (i == k && j == k) {
        v = pinv;
      } else if (i == k) {
        v = rkj[c] * pinv;
      } else if (j == k) {
        v = f[r];
      } else {
        v = fma(f[r], rkj[c], m[r][c]);
      }
      M[(int64_t)i * n + j] = v;
      m[r][c] = v;
    }
  }
  // row and column k + 1 after this step, and the decision on pivot k + 1
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = i0 + r;
    if (i >= n) break;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int j = j0 + 32 * c;
      if (j >= n) continue;
      if (i == k + 1) rn[j] = m[r][c];
      if (j == k + 1) cn[i] = m[r][c];
      if (i == k + 1 && j == k + 1) gj_decide(g, b, k + 1, m[r][c], piv_next, pdrop_next);
    }
  }
}

// The whole sweep of one small matrix (n <= kGjSmallN) in one block, the matrix held in shared
// memory: matrix first + blockIdx.x of the batch. Every pivot step is the one k_gj_step
// performs (same drop rule, same operations in the same order, so the same result), with
// block barriers in place of launch boundaries.
constexpr int kGjSmallN = 128;
constexpr size_t kGjSmallSmem = ((size_t)kGjSmallN * kGjSmallN + 2 * kGjSmallN) * sizeof(double);

__global__ void __launch_bounds__(kBlock) k_gj_small(GjBatch g, int first) {
  extern __shared__ double gs[];
  const int b = first + blockIdx.x;
  const int n = g.n[b];
  const int nn = n * n;
  double* S = gs;
  double* rk = gs + nn;   // row k before the pivot step
  double* fk = rk + n;    // row factors -M[i][k] / p of the current pivot
  __shared__ double pinv_s;
  __shared__ int drop_s;
  double* M = g.M + g.off[b];
  const double* d0v = g.diag0 + g.voff[b];
  for (int e = threadIdx.x; e < nn; e += blockDim.x) S[e] = M[e];
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      const double p = S[k * n + k];
      const double d0 = d0v[k];
      const bool bad = !(d0 > 0.0) || !isfinite(p) || p < -kGjDrop * d0;
      const bool drop = bad || p <= kGjDrop * d0;
      pinv_s = drop ? 0.0 : 1.0 / p;
      drop_s = drop ? 1 : 0;
      if (bad) g.bad[b] = 1;
      if (drop) g.ndrop[b] += 1;
    }
    __syncthreads();
    const bool drop = drop_s != 0;
    const double pinv = pinv_s;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      rk[j] = drop ? 0.0 : S[k * n + j];
      fk[j] = drop ? 0.0 : -S[j * n + k] * pinv;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
      const int i = e / n, j = e - i * n;
      if (drop) {
        if (i == k || j == k) S[e] = 0.0;
      } else if (i == k && j == k) {
        S[e] = pinv;
      } else if (i == k) {
        S[e] = rk[j] * pinv;
      } else if (j == k) {
        S[e] = fk[i];
      } else {
        S[e] = fma(fk[i], rk[j], S[e]);
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nn; e += blockDim.x) M[e] = S[e];
}

// max_i sum_j |M_ij| of matrix blockIdx.x of the batch (column sums: M is symmetric, so
// thread i reads column i, coalesced across the block).
__global__ void __launch_bounds__(kBlock) k_gj_norm1(GjBatch g, double* __restrict__ out) {
  __shared__ double best[kBlock];
  const int b = blockIdx.x;
  const int n = g.n[b];
  const double* M = g.M + g.off[b];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double sum = 0.0;
    for (int j = 0; j < n; ++j) sum += fabs(M[(int64_t)j * n + i]);
    m = fmax(m, sum);
  }
  best[threadIdx.x] = m;
  __syncthreads();
  for (int o = kBlock / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) best[threadIdx.x] = fmax(best[threadIdx.x], best[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[b] = best[0];
}

// FP64 FMA throughput: every thread runs 8 independent FMA chains of `iters` steps on values
// that stay bounded (a = a * c + d with |c| < 1), then writes their sum (so nothing is elided).
__global__ void __launch_bounds__(kBlock) k_fp64_fma(int iters, double c, double d, double* __restrict__ out) {
  double a[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) a[u] = (double)(threadIdx.x + u);
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = fma(a[u], c, d);
  }
  double s = 0.0;
#pragma unroll
  for (int u = 0; u < 8; ++u) s += a[u];
  out[blockIdx.x * kBlock + threadIdx.x] = s;
}

}  // namespace



void batched_spsd_inverse(const GjBatch& g, cudaStream_t s) {
  // matrices are sorted by size, largest first: the small ones take one block each for the
  // whole sweep (shared memory), the others one prep and one update launch per pivot
  int nlarge = 0;
  while (nlarge < g.nmat && g.hn[nlarge] > kGjSmallN) ++nlarge;
  if (nlarge < g.nmat) {
    const int ns = g.hn[nlarge];
    cudaFuncSetAttribute(k_gj_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGjSmallSmem);
    k_gj_small<<<g.nmat - nlarge, kBlock, ((size_t)ns * ns + 2 * ns) * sizeof(double), s>>>(g, nlarge);
  }
  if (nlarge == 0) return;
  // row/column snapshots and pivot decisions: rowk/colk/piv/pdrop for even k, the second
  // buffers (rowk2/colk2, piv + nmat, pdrop + nmat) for odd k
  k_gj_snap0<<<nlarge, kBlock, 0, s>>>(g);
  const int tiles_x = (g.hn[0] + kGjTile - 1) / kGjTile;
  int active = nlarge;
  for (int k = 0; k < g.max_n && active > 0; ++k) {
    while (active > 0 && g.hn[active - 1] <= k) --active;
    if (active == 0) break;
    const bool even = (k & 1) == 0;
    double* pv0 = g.piv + (even ? 0 : g.nmat);
    double* pv1 = g.piv + (even ? g.nmat : 0);
    int32_t* pd0 = g.pdrop + (even ? 0 : g.nmat);
    int32_t* pd1 = g.pdrop + (even ? g.nmat : 0);
    k_gj_step<<<dim3(tiles_x * tiles_x, active), kBlock, 0, s>>>(
        g, k, tiles_x, even ? g.rowk : g.rowk2, even ? g.colk : g.colk2, even ? g.rowk2 : g.rowk,
        even ? g.colk2 : g.colk, pv0, pd0, pv1, pd1);
  }
}

double measure_fp64_fma(cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8, iters = 4096;
  double* out = nullptr;
  if (cudaMallocAsync(&out, sizeof(double) * blocks * kBlock, s) != cudaSuccess) throw Error(MG_ERR_OOM, "probe buffer");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fp64_fma<<<blocks, kBlock, 0, s>>>(iters, 0.999999, 1e-3, out);   // warm-up
  cudaEventRecord(e0, s);
  k_fp64_fma<<<blocks, kBlock, 0, s>>>(iters, 0.999999, 1e-3, out);
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, s);
  check_launch("FP64 FMA probe");
  return (double)blocks * kBlock * 8.0 * iters / (ms * 1e-3);   // FMAs per second
}

void batched_norm1(const GjBatch& g, double* out, cudaStream_t s) {
  if (g.nmat > 0) k_gj_norm1<<<g.nmat, kBlock, 0, s>>>(g, out);
}

int sell_blocks(int nrows, int lanes) { return grid_for((int)std::min<int64_t>((int64_t)nrows * lanes, INT32_MAX), kBlock); }

// Blocks of one launch over an operator: a warp per SELL slice, or G threads per CSR row.
template <typename T>
int op_blocks(const SellMat<T>& A) {
  return A.lanes > 1 ? sell_blocks(A.nrows, A.lanes) : grid_for((int)std::min<int64_t>((int64_t)A.nslices * 32, INT32_MAX), kBlock);
}

template <typename T>
OpView<T> view(const SellMat<T>& A) {
  return OpView<T>{A.off, A.rp, A.col, A.val, A.perm, A.col16, A.cbase, A.nrows, A.nslices, A.lanes > 1 ? 0 : A.pf};
}

template <int G, bool C>
struct Lay {
  static constexpr int lanes = G;
  static constexpr bool c16 = C;
};

// Dispatch on the layout: f(Lay<G, C16>) with the kernel's layout parameter G (see is_sell)
// and index width.
template <typename F>
void by_layout(int lanes, int unroll, int sub, bool c16, F&& f) {
  auto go = [&](auto c) {
    constexpr bool C = decltype(c)::value;
    switch (lanes) {
      case 1:
        if (sub == 2) f(Lay<3, C>());
        else if (sub == 4) f(Lay<5, C>());
        else if (unroll == 2) f(Lay<2, C>());
        else if (unroll == 3) f(Lay<6, C>());
        else f(Lay<1, C>());
        break;
      case 4: f(Lay<4, C>()); break;
      case 8: f(Lay<8, C>()); break;
      case 16: f(Lay<16, C>()); break;
      case 32: f(Lay<32, C>()); break;
      default: throw Error(MG_ERR_INVALID_ARG, "unsupported lanes per row");
    }
  };
  if (c16) go(std::true_type());
  else go(std::false_type());
}

bool take_wait_timeout(cudaStream_t s) {
  static const int zero = 0;
  int v = 0;
  cudaMemcpyFromSymbolAsync(&v, g_wait_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  if (v) {
    cudaMemcpyToSymbolAsync(g_wait_timeout, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
  }
  return v != 0;
}

template <typename T>
constexpr size_t tma_smem() {
  return kTmaBarBytes + (size_t)kTmaStages * tma_stage_entries<T>() * (sizeof(T) + sizeof(int32_t));
}

// One-time set-up per instantiation (shared-memory limit, resident CTAs): thread-safe, and
// run by tma_prepare() before any graph capture.
template <typename T, typename Epi>
int tma_grid_cap() {
  static const int cap = [] {
    auto kernel = k_sell_tma<T, Epi>;
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma_smem<T>());
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kTmaThreads, tma_smem<T>());
    return std::max(1, sms * std::max(per, 1));
  }();
  return cap;
}

// Persistent launch of the TMA-staged SpMV with epilogue `epi`: as many CTAs as fit on the
// device at once (one per SM at this shared-memory size), at most one per chunk.
template <typename T, typename Epi>
void launch_tma(const SellMat<T>& A, const T* x, const Epi& epi, cudaStream_t s) {
  const int cap = tma_grid_cap<T, Epi>();
  auto kernel = k_sell_tma<T, Epi>;
  const size_t smem = tma_smem<T>();
  const int grid = std::min(cap, A.nchunks);
  if (grid <= 0) return;
  launch(kernel, grid, kTmaThreads, smem, s, view(A), A.chunks, A.nchunks, x, epi);
}

template <typename T>
void tma_prepare_t() {
  tma_grid_cap<T, EpiSpmv<T>>();
  tma_grid_cap<T, EpiResid<T>>();
  tma_grid_cap<T, EpiCheb<T, true>>();
  tma_grid_cap<T, EpiCheb<T, false>>();
}
void tma_prepare() {
  tma_prepare_t<float>();
  tma_prepare_t<double>();
}

template <typename T>
void sell_spmv(const SellMat<T>& A, const T* x, T* y, cudaStream_t s) {
  if (A.nrows == 0) return;
  if (A.tma) return launch_tma<T>(A, x, EpiSpmv<T>{y}, s);
  by_layout(A.lanes, A.unroll, A.sub, A.col16 != nullptr, [&](auto g) {
    using L = decltype(g);
    launch(k_spmv<T, L::lanes, L::c16>, op_blocks(A), kBlock, 0, s, view(A), x, y);
  });
}
template <typename T>
void sell_resid(const SellMat<T>& A, const T* x, const T* b, T* r, cudaStream_t s) {
  if (A.nrows == 0) return;
  if (A.tma) return launch_tma<T>(A, x, EpiResid<T>{b, r}, s);
  by_layout(A.lanes, A.unroll, A.sub, A.col16 != nullptr, [&](auto g) {
    using L = decltype(g);
    launch(k_resid<T, L::lanes, L::c16>, op_blocks(A), kBlock, 0, s, view(A), x, b, r);
  });
}
template <typename T>
void sell_cheb(const SellMat<T>& A, const T* xin, const T* b, const T* dinv, T* d, T* xout, double cd, double cr,
               bool first, cudaStream_t s) {
  if (A.nrows == 0) return;
  if (A.tma) {
    if (first) return launch_tma<T>(A, xin, EpiCheb<T, true>{b, dinv, xin, d, xout, (T)cd, (T)cr}, s);
    return launch_tma<T>(A, xin, EpiCheb<T, false>{b, dinv, xin, d, xout, (T)cd, (T)cr}, s);
  }
  by_layout(A.lanes, A.unroll, A.sub, A.col16 != nullptr, [&](auto g) {
    using L = decltype(g);
    constexpr int G = L::lanes;
    if (first)
      launch(k_cheb<T, G, L::c16, true>, op_blocks(A), kBlock, 0, s, view(A), xin, b, dinv, d, xout, (T)cd,
                                                                            (T)cr);
    else
      launch(k_cheb<T, G, L::c16, false>, op_blocks(A), kBlock, 0, s, view(A), xin, b, dinv, d, xout, (T)cd,
                                                                             (T)cr);
  });
}
template <typename T>
void sell_prolong_pr(const SellMat<T>& P, const T* xc, T* x, int nt, int w, const int32_t* pdofs, const int32_t* aplen,
                     const int32_t* apci, const double* apv, const T* res, double* rbuf, cudaStream_t s) {
  const int nbp = P.nrows == 0 ? 0 : op_blocks(P);
  if (nbp + nt == 0) return;
  by_layout(P.lanes, P.unroll, P.sub, P.col16 != nullptr, [&](auto g) {
    using L = decltype(g);
    launch(k_prolong_pr<T, L::lanes, L::c16>, nbp + grid_for(nt, kBlock / 32), kBlock, 0, s, view(P), xc, x, nbp, nt,
           w, pdofs, aplen, apci, apv, res, rbuf);
  });
}
template <typename T>
void sell_prolong(const SellMat<T>& P, const T* xc, T* x, cudaStream_t s) {
  if (P.nrows == 0) return;
  by_layout(P.lanes, P.unroll, P.sub, P.col16 != nullptr, [&](auto g) {
    using L = decltype(g);
    launch(k_prolong<T, L::lanes, L::c16>, op_blocks(P), kBlock, 0, s, view(P), xc, x);
  });
}
template <typename T>
void sell_restrict(const SellMat<T>& R, const T* r, T* bc, T* xc, cudaStream_t s) {
  if (R.nrows == 0) return;
  by_layout(R.lanes, R.unroll, R.sub, R.col16 != nullptr, [&](auto g) {
    using L = decltype(g);
    launch(k_restrict<T, L::lanes, L::c16>, op_blocks(R), kBlock, 0, s, view(R), r, bc, xc);
  });
}
template <typename T>
void sell_gs(const SellMat<T>& M, const int32_t* rows, const T* b, const T* dinv, T* x, cudaStream_t s) {
  if (M.nrows == 0) return;
  by_layout(M.lanes, M.unroll, M.sub, M.col16 != nullptr, [&](auto g) {
    using L = decltype(g);
    launch(k_gs<T, L::lanes, L::c16>, op_blocks(M), kBlock, 0, s, view(M), rows, x, b, dinv, x);
  });
}
void lanczos_step(const SellMat<double>& M, int nv, double* const* v, double* const* w, double* const* vprev,
                  const uint8_t* const* keep, double* const* hist, int j, double* part, unsigned* ticket,
                  cudaStream_t s) {
  LzRuns z{};
  z.nv = nv;
  for (int r = 0; r < nv; ++r) {
    z.v[r] = v[r];
    z.w[r] = w[r];
    z.vprev[r] = vprev[r];
    z.keep[r] = keep[r];
    z.hist[r] = hist[r];
  }
  const int n = M.nrows;
  if (j > 0) k_lz_next<<<cg_parts(n), kBlock, 0, s>>>(n, z, j);
  by_layout(M.lanes, M.unroll, M.sub, M.col16 != nullptr, [&](auto g) {
    using L = decltype(g);
    launch(k_lz_spmv_dot<L::lanes, L::c16>, op_blocks(M), kBlock, 0, s, view(M), z, j, part, ticket);
  });
  k_lz_update<<<cg_parts(n), kBlock, 0, s>>>(n, z, j, part, ticket);
}
// Blocks of one k_ap launch: one resident wave (SMs x the blocks of this instantiation that fit
// on an SM: four at its 60-62 registers), at most one per row block. With two waves (8 blocks
// per SM requested) the C2 product took 125.1 vs 122.2 us.
template <typename K>
int ap_wave(K kernel) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kBlock, 0);
  return std::max(1, sms * std::max(per, 1));
}

void sell_ap(const SellMat<double>& A, const double* p, double* q, const Reduce& rd, cudaStream_t s) {
  const int nvb = op_blocks(A);
  by_layout(A.lanes, A.unroll, A.sub, A.col16 != nullptr, [&](auto g) {
    using L = decltype(g);
    static const int wave = ap_wave(k_ap<L::lanes, L::c16>);
    launch(k_ap<L::lanes, L::c16>, std::max(1, std::min(nvb, wave)), kBlock, 0, s, view(A), nvb, p, q, rd);
  });
}

template <typename T>
void cheb_first_from_zero(int n, const T* b, const T* dinv, const T* xin, T* d, T* xout, double cr, int nh,
                          const int32_t* hrow, const int32_t* hrp, const int32_t* hci, const T* hv, cudaStream_t s) {
  if (n == 0) return;
  launch(k_cheb0_all<T>, grid_for(n, kBlock), kBlock, 0, s, n, b, dinv, xin, d, xout, (T)cr);
  if (nh > 0)
    launch(k_cheb0_halo<T>, grid_for(nh, kBlock / 32), kBlock, 0, s, nh, hrow, hrp, hci, hv, b, dinv, xin, d, xout, (T)cr);
}

template <typename T>
void patch_residual(int nt, int w, const int32_t* pdofs, const int32_t* plen, const int32_t* pci, const double* pv,
                    const T* b, const T* x, double* rbuf, cudaStream_t s) {
  if (nt == 0) return;
  launch(k_patch_residual<T>, grid_for(nt, kBlock / 32), kBlock, 0, s, nt, w, pdofs, plen, pci, pv, b, x, rbuf);
}

// The limit is a per-function attribute of the device's context, shared by every hierarchy in
// the process: it is raised once per device to the largest patch any hierarchy may have
// (27000 DoFs, 216,000 bytes) and never lowered, so that a hierarchy set up later (possibly
// on another thread) cannot shrink the limit under an earlier one's launches.
void patch_solve_setup(int max_patch) {
  static std::mutex mu;
  static bool done[64] = {};
  if ((size_t)max_patch * sizeof(double) <= 48 * 1024) return;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) throw Error(MG_ERR_CUDA, "no current device");
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return;
  const int smem = kMaxPatchDofs * (int)sizeof(double);
  const cudaError_t e[4] = {
      cudaFuncSetAttribute(k_patch_solve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
      cudaFuncSetAttribute(k_patch_solve<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
      cudaFuncSetAttribute(k_cheb0_entry<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
      cudaFuncSetAttribute(k_cheb0_entry<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)};
  for (cudaError_t x : e)
    if (x != cudaSuccess) throw Error(MG_ERR_CUDA, std::string("patch solve shared-memory limit: ") + cudaGetErrorString(x));
  done[dev] = true;
}

template <typename T>
void cheb_entry_local(int nitems, const PatchItem* items, const int32_t* pdofs, const double* inv, const float* inv32,
                      int max_patch, int n, const T* b, const T* dinv, T* x, T* d, T* xout, double cr, int nh,
                      const int32_t* hrow, const int32_t* hrp, const int32_t* hci, const T* hv, cudaStream_t s) {
  if (n == 0) return;
  const size_t smem = (size_t)max_patch * sizeof(double);
  launch(k_cheb0_entry<T>, nitems + grid_for(n, kBlock), kBlock, smem, s, nitems, items, pdofs, inv, inv32, n, b,
         dinv, x, d, xout, (T)cr);
  if (nh > 0)
    launch(k_cheb0_halo<T>, grid_for(nh, kBlock / 32), kBlock, 0, s, nh, hrow, hrp, hci, hv, b, dinv, x, d, xout, (T)cr);
}

template <typename T>
void patch_solve(int nitems, const PatchItem* items, const int32_t* pdofs, const double* inv, const float* inv32,
                 const double* rbuf, const T* b, T* x, int max_patch, cudaStream_t s) {
  if (nitems == 0) return;
  size_t smem = (size_t)max_patch * sizeof(double);
  launch(k_patch_solve<T>, nitems, kBlock, smem, s, items, pdofs, inv, inv32, rbuf, b, x);
}

int dense_chunks(int n, int kchunk) { return grid_for(n, kchunk); }

template <typename T>
cudaError_t dense_solve(int n, const double* X, const T* b, T* x, double* part, int kchunk, cudaStream_t s) {
  int nch = dense_chunks(n, kchunk);
  dim3 grid(grid_for(n, kBlock), nch);
  cudaError_t e = launch(k_dense_partial<T>, grid, kBlock, kchunk * sizeof(double), s, n, kchunk, X, b, part);
  if (e != cudaSuccess) return e;
  return launch(k_dense_reduce<T>, grid_for(n, kBlock / 32), kBlock, 0, s, n, nch, part, x);
}

template <typename Src, typename Dst>
void convert(int n, const Src* a, Dst* b, cudaStream_t s) {
  if (n == 0) return;
  launch(k_convert<Src, Dst>, std::min(grid_for(n, kBlock), kCgBlocks), kBlock, 0, s, n, a, b);
}
template <typename Src, typename Dst>
void gather(int n, const int32_t* perm, const Src* a, Dst* b, cudaStream_t s) {
  if (n == 0) return;
  if (!perm) return convert<Src, Dst>(n, a, b, s);
  launch(k_gather<Src, Dst>, std::min(grid_for(n, kBlock), kCgBlocks), kBlock, 0, s, n, perm, a, b);
}
template <typename Src, typename Dst>
void scatter(int n, const int32_t* perm, const Src* a, Dst* b, cudaStream_t s) {
  if (n == 0) return;
  if (!perm) return convert<Src, Dst>(n, a, b, s);
  launch(k_scatter<Src, Dst>, std::min(grid_for(n, kBlock), kCgBlocks), kBlock, 0, s, n, perm, a, b);
}

template <typename T>
void axpy_from(int n, const T* z, double* x, cudaStream_t s) {
  if (n == 0) return;
  launch(k_axpy_from<T>, std::min(grid_for(n, kBlock), kCgBlocks), kBlock, 0, s, n, z, x);
}

int cg_parts(int n) { return std::max(1, std::min(grid_for(n, kBlock), kCgBlocks)); }

template <typename T>
void cg_init(int n, const double* b, double* r, double* x, T* vb, T* vx, const Reduce& rd, cudaStream_t s) {
  launch(k_cg_init<T>, cg_parts(n), kBlock, 0, s, n, b, r, x, vb, vx, rd);
}
template <typename T>
void cg_update(int n, const CgState* st, const double* p, const double* q, double* x, double* r, T* vb, T* vx,
               const Reduce& rd, cudaStream_t s) {
  launch(k_cg_update<T>, cg_parts(n), kBlock, 0, s, n, st, p, q, x, r, vb, vx, rd);
}
template <typename T>
void cg_dotz(int n, const double* r, const T* vx, double* p, bool first, const Reduce& rd, cudaStream_t s) {
  if (first) launch(k_cg_dotz<T, true>, cg_parts(n), kBlock, 0, s, n, r, vx, p, rd);
  else launch(k_cg_dotz<T, false>, cg_parts(n), kBlock, 0, s, n, r, vx, p, rd);
}
template <typename T>
void cg_pupdate(int n, const CgState* st, const T* vx, double* p, cudaStream_t s) {
  launch(k_cg_pupdate<T>, cg_parts(n), kBlock, 0, s, n, st, vx, p);
}
void dot_self(int n, const double* r, const Reduce& rd, cudaStream_t s) {
  launch(k_dot_self, cg_parts(n), kBlock, 0, s, n, r, rd);
}

#define NNMG_INST(T)                                                                                             \
  template void sell_spmv<T>(const SellMat<T>&, const T*, T*, cudaStream_t);                                     \
  template void sell_resid<T>(const SellMat<T>&, const T*, const T*, T*, cudaStream_t);                          \
  template void sell_cheb<T>(const SellMat<T>&, const T*, const T*, const T*, T*, T*, double, double, bool,      \
                             cudaStream_t);                                                                      \
  template void sell_prolong<T>(const SellMat<T>&, const T*, T*, cudaStream_t);                                  \
  template void sell_prolong_pr<T>(const SellMat<T>&, const T*, T*, int, int, const int32_t*, const int32_t*,     \
                                   const int32_t*, const double*, const T*, double*, cudaStream_t);             \
  template void sell_restrict<T>(const SellMat<T>&, const T*, T*, T*, cudaStream_t);                             \
  template void sell_gs<T>(const SellMat<T>&, const int32_t*, const T*, const T*, T*, cudaStream_t);             \
  template void cheb_first_from_zero<T>(int, const T*, const T*, const T*, T*, T*, double, int, const int32_t*, \
                                        const int32_t*, const int32_t*, const T*, cudaStream_t);                 \
  template void patch_residual<T>(int, int, const int32_t*, const int32_t*, const int32_t*, const double*,       \
                                   const T*, const T*, double*, cudaStream_t);                            \
  template void patch_solve<T>(int, const PatchItem*, const int32_t*, const double*, const float*, const double*, \
                                const T*, T*, int, cudaStream_t);                                         \
  template void cheb_entry_local<T>(int, const PatchItem*, const int32_t*, const double*, const float*, int, int,  \
                                    const T*, const T*, T*, T*, T*, double, int, const int32_t*, const int32_t*, \
                                    const int32_t*, const T*, cudaStream_t);                                     \
  template cudaError_t dense_solve<T>(int, const double*, const T*, T*, double*, int, cudaStream_t);                    \
  template void axpy_from<T>(int, const T*, double*, cudaStream_t);                                              \
  template void cg_init<T>(int, const double*, double*, double*, T*, T*, const Reduce&, cudaStream_t);         \
  template void cg_update<T>(int, const CgState*, const double*, const double*, double*, double*, T*, T*,        \
                             const Reduce&, cudaStream_t);                                                       \
  template void cg_dotz<T>(int, const double*, const T*, double*, bool, const Reduce&, cudaStream_t);            \
  template void cg_pupdate<T>(int, const CgState*, const T*, double*, cudaStream_t);

NNMG_INST(double)
NNMG_INST(float)
template void convert<double, float>(int, const double*, float*, cudaStream_t);
template void convert<float, double>(int, const float*, double*, cudaStream_t);
template void convert<double, double>(int, const double*, double*, cudaStream_t);
template void convert<float, float>(int, const float*, float*, cudaStream_t);
template void gather<double, float>(int, const int32_t*, const double*, float*, cudaStream_t);
template void gather<double, double>(int, const int32_t*, const double*, double*, cudaStream_t);
template void scatter<float, double>(int, const int32_t*, const float*, double*, cudaStream_t);
template void scatter<double, double>(int, const int32_t*, const double*, double*, cudaStream_t);

}  // namespace nnmg
