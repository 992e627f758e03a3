// Persistent execution of the lower part of the V-cycle (Alg. 1 from a given level down to the
// coarsest and back) in one cooperative launch.
//
// On the small levels every step of the cycle moves a few megabytes, which the GPU streams
// in a microsecond or two, while a dependent kernel launch costs several: there the cycle
// is bound by launch and drain latency, not by memory. Here the host records the cycle's
// steps as a program of phases; each phase holds one or more independent tasks (a sparse
// product with its epilogue, the patch residuals, the patch solves, the coarsest dense
// product ...) cut into warp-sized units. One grid, as large as can be resident at once
// (cooperative launch), walks the phases: every warp takes the units u = warp, warp + W, ...
// of the phase (a fixed assignment, so results are deterministic), then the grid meets at a
// barrier before the next phase.
//
// Coherence: vectors written earlier in the same launch are read with plain (weak) loads,
// never through the read-only (non-coherent) path; matrices and the other set-up data, which
// no phase writes, use the read-only path. Every barrier is a device-scope release by each
// block before it arrives and an acquire after it leaves (the fences around the arrival
// counter), which makes every write before the barrier visible to plain loads after it.
//
// Every barrier wait is bounded (about a second of SM clocks); on expiry the waiting block
// sets the error word and the abort flag, and every block leaves at its next barrier, so the
// launch always ends. The host reads the error word after the solve.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.hpp"
#include "kernels.cuh"

namespace nnmg {
namespace {

// A vector that phases of this launch write: a plain load (never the read-only path).
template <typename T>
__device__ __forceinline__ T ldv(const T* p) {
  return *p;
}

__device__ __forceinline__ double pwarp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Grid-wide barrier with a bounded wait. Returns false when the launch is being abandoned
// (this block's wait expired, or another block's did).
__device__ bool grid_barrier(PBarrier* bar) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = &bar->gen;
    volatile int* abort = &bar->abort;
    const unsigned g = *gen;
    __threadfence();
    int good = 1;
    if (atomicAdd(&bar->count, 1u) == gridDim.x - 1) {
      bar->count = 0u;
      __threadfence();
      atomicExch(&bar->gen, g + 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g) {
        __nanosleep(32);
        if (*abort) {
          good = 0;
          break;
        }
        if (clock64() - t0 > (1ll << 31)) {
          atomicExch(&bar->error, 1);
          atomicExch(&bar->abort, 1);
          good = 0;
          break;
        }
      }
    }
    __threadfence();
    ok = good && !*abort;
  }
  __syncthreads();
  return ok != 0;
}

// Sum over the CSR row `row` by the G lanes of a group (gl = lane within the group), xor
// shuffles combining the group; every lane of the warp must call it (rows past the end pass
// row = -1 and contribute nothing).
template <typename T, int G>
__device__ __forceinline__ T group_row(const PTask& t, int row, int gl, const T* x) {
  T acc = T(0);
  if (row >= 0) {
    const int32_t* __restrict__ rp = t.rp;
    const int32_t* __restrict__ ci = t.ci;
    const T* __restrict__ val = static_cast<const T*>(t.val);
    const int k1 = __ldg(rp + row + 1);
    // four entries per lane per step: their value and index loads, then the gathers, then the
    // FMAs (the last step predicated)
    for (int k = __ldg(rp + row) + gl; k < k1; k += 4 * G) {
      T v[4], xv[4];
      int c[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = k + u * G < k1 ? __ldg(val + k + u * G) : T(0);
#pragma unroll
      for (int u = 0; u < 4; ++u) c[u] = k + u * G < k1 ? __ldg(ci + k + u * G) : 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) xv[u] = k + u * G < k1 ? ldv(x + c[u]) : T(0);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (k + u * G < k1) acc = fma(v[u], xv[u], acc);
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

// One unit of a CSR task: 32 / G rows, G lanes each.
template <typename T, int G>
__device__ __forceinline__ void csr_unit(const PTask& t, int unit, int lane) {
  constexpr int R = 32 / G;
  const int r = unit * R + lane / G, gl = lane & (G - 1);
  const int live = r < t.n ? r : -1;
  const int row = live >= 0 ? (t.rows ? __ldg(t.rows + live) : live) : -1;
  const T* x = static_cast<const T*>(t.x);
  const T ax = group_row<T, G>(t, live, gl, x);
  if (live < 0 || gl != 0) return;
  T* y = static_cast<T*>(t.y);
  const T* b = static_cast<const T*>(t.b);
  switch (t.kind) {
    case PK_CHEB_FIRST:
    case PK_CHEB: {   // r = b - A x; d = cd d + cr D^-1 r; y = x + d
      const T* dinv = static_cast<const T*>(t.dinv);
      T* d = static_cast<T*>(t.d);
      const T rr = ldv(b + row) - ax;
      const T tt = __ldg(dinv + row) * rr;
      const T cr = (T)t.c2;
      const T dn = t.kind == PK_CHEB_FIRST ? cr * tt : fma((T)t.c1, ldv(d + row), cr * tt);
      d[row] = dn;
      y[row] = ldv(x + row) + dn;
      break;
    }
    case PK_RESID:    // y = b - A x
      y[row] = ldv(b + row) - ax;
      break;
    case PK_RESTRICT:  // y = R x; z = 0 (the coarse iterate)
      y[row] = ax;
      static_cast<T*>(t.z)[row] = T(0);
      if (t.y64) t.y64[row] = (double)ax;
      break;
    case PK_PROLONG:   // y += P x
      y[row] = ldv(y + row) + ax;
      break;
    case PK_SPMV:
      y[row] = ax;
      break;
  }
}

template <typename T>
__device__ __forceinline__ void csr_dispatch(const PTask& t, int unit, int lane) {
  switch (t.G) {
    case 4: csr_unit<T, 4>(t, unit, lane); break;
    case 8: csr_unit<T, 8>(t, unit, lane); break;
    case 16: csr_unit<T, 16>(t, unit, lane); break;
    default: csr_unit<T, 32>(t, unit, lane); break;
  }
}

// q = A p on 32 / G rows of the FP64 level-0 operator, and the unit's partial p.q.
template <int G>
__device__ __forceinline__ void cg_ap_unit(const PTask& t, int unit, int lane) {
  constexpr int R = 32 / G;
  const int r = unit * R + lane / G, gl = lane & (G - 1);
  const int live = r < t.n ? r : -1;
  const double ax = group_row<double, G>(t, live, gl, t.cp);
  double v = 0.0;
  if (live >= 0 && gl == 0) {
    t.cq[live] = ax;
    v = ldv(t.cp + live) * ax;
  }
  v = pwarp_sum(v);
  if (lane == 0) t.part[unit] = v;
}

// One warp-unit of the other task kinds.
template <typename T>
__device__ __forceinline__ void run_unit(const PTask& t, int unit, int lane) {
  if (t.gate && !ldv(&t.gate->cont)) return;   // this problem's solve has stopped
  switch (t.kind) {
    case PK_CG_INIT:
    case PK_CG_UPDATE:
    case PK_CG_DOTZ:
    case PK_CG_PUPDATE: {
      const int i = unit * 32 + lane;
      T* vb = static_cast<T*>(t.vb);
      T* vx = static_cast<T*>(t.vx);
      double v = 0.0;
      if (i < t.n) {
        if (t.kind == PK_CG_INIT) {
          const double bi = ldv(t.cb + i);
          t.cr[i] = bi;
          t.cx[i] = 0.0;
          vb[i] = (T)bi;
          vx[i] = T(0);
          v = bi * bi;
        } else if (t.kind == PK_CG_UPDATE) {
          const double a = ldv(&t.st->alpha);
          t.cx[i] = fma(a, ldv(t.cp + i), ldv(t.cx + i));
          const double ri = fma(-a, ldv(t.cq + i), ldv(t.cr + i));
          t.cr[i] = ri;
          vb[i] = (T)ri;
          vx[i] = T(0);
          v = ri * ri;
        } else if (t.kind == PK_CG_DOTZ) {
          const double zi = (double)ldv(vx + i);
          if (t.w) t.cp[i] = zi;
          v = ldv(t.cr + i) * zi;
        } else {
          t.cp[i] = fma(ldv(&t.st->beta), ldv(t.cp + i), (double)ldv(vx + i));
        }
      }
      if (t.kind != PK_CG_PUPDATE) {
        v = pwarp_sum(v);
        if (lane == 0) t.part[unit] = v;
      }
      return;
    }
    case PK_CG_AP:
      switch (t.G) {
        case 4: cg_ap_unit<4>(t, unit, lane); break;
        case 8: cg_ap_unit<8>(t, unit, lane); break;
        case 16: cg_ap_unit<16>(t, unit, lane); break;
        default: cg_ap_unit<32>(t, unit, lane); break;
      }
      return;
    case PK_FINISH: {   // the partials in a fixed order: lane-strided, then the warp tree
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      int k = lane;
      for (; k + 96 < t.w; k += 128) {
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = ldv(t.part + k + 32 * u);
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] += v[u];
      }
      for (; k < t.w; k += 32) acc[0] += ldv(t.part + k);
      const double s = pwarp_sum((acc[0] + acc[1]) + (acc[2] + acc[3]));
      if (lane == 0) apply_finish(t.st, s, t.op, 0, 0);
      return;
    }
    case PK_CHEB0: {   // first step from a zero iterate: d = cr D^-1 b; y = x + d (32 rows)
      const int i = unit * 32 + lane;
      if (i >= t.n) return;
      const T* b = static_cast<const T*>(t.b);
      const T* dinv = static_cast<const T*>(t.dinv);
      const T dn = (T)t.c2 * (__ldg(dinv + i) * ldv(b + i));
      static_cast<T*>(t.d)[i] = dn;
      static_cast<T*>(t.y)[i] = t.x ? ldv(static_cast<const T*>(t.x) + i) + dn : dn;
      return;
    }
    case PK_COPY: {
      const int i = unit * 32 + lane;
      if (i < t.n) static_cast<T*>(t.y)[i] = ldv(static_cast<const T*>(t.x) + i);
      return;
    }
    case PK_PATCH_RES:     // rbuf[t] = b[g] - (A x)[g], or res[g] - ((A P) x_c)[g] (ELL row, FP64)
    case PK_PATCH_RES_AP: {
      const int r = unit;
      const int64_t o = (int64_t)r * t.w;
      const int len = __ldg(t.plen + r);
      const T* x = static_cast<const T*>(t.x);
      double s = 0.0;
      for (int k = lane; k < len; k += 32) s = fma(__ldg(t.pv + o + k), (double)ldv(x + __ldg(t.pci + o + k)), s);
      s = pwarp_sum(s);
      if (lane == 0) t.rbuf[r] = (double)ldv(static_cast<const T*>(t.b) + __ldg(t.pdofs + r)) - s;
      return;
    }
    case PK_PATCH_SOLVE: {   // x_g += sum_j X_ij r_j over the row's patch (FP64)
      const PRow pr = t.prow[unit];
      const double* Xi = t.inv + pr.inv;
      double e = 0.0;
      const T* b = static_cast<const T*>(t.b);
      for (int j = lane; j < pr.n; j += 4 * 32) {   // four inverse entries in flight per lane
        double xv[4], rv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[u] = j + 32 * u < pr.n ? __ldg(Xi + j + 32 * u) : 0.0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int jj = j + 32 * u;
          rv[u] = jj < pr.n ? (t.rbuf ? ldv(t.rbuf + pr.p0 + jj) : (double)ldv(b + __ldg(t.pdofs + pr.p0 + jj))) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (j + 32 * u < pr.n) e = fma(xv[u], rv[u], e);
      }
      e = pwarp_sum(e);
      if (lane == 0) {
        T* x = static_cast<T*>(t.y);
        const int g = __ldg(t.pdofs + pr.p0 + pr.i);
        x[g] = (T)((double)ldv(x + g) + e);
      }
      return;
    }
    case PK_DENSE: {   // y_i = sum_j X_ij b_j (FP64, X symmetric and row-major)
      const int i = unit;
      const double* Xi = t.inv + (int64_t)i * t.n;
      const T* b = static_cast<const T*>(t.b);
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      for (int j = lane; j < t.n; j += 8 * 32) {   // eight loads of X in flight per lane
        double xv[8], bv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) xv[u] = j + 32 * u < t.n ? __ldg(Xi + j + 32 * u) : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u)
          bv[u] = j + 32 * u < t.n ? (t.y64 ? ldv(t.y64 + j + 32 * u) : (double)ldv(b + j + 32 * u)) : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (j + 32 * u < t.n) acc[u & 3] = fma(xv[u], bv[u], acc[u & 3]);
      }
      const double s = pwarp_sum((acc[0] + acc[1]) + (acc[2] + acc[3]));
      if (lane == 0) static_cast<T*>(t.y)[i] = (T)s;
      return;
    }
    default:
      csr_dispatch<T>(t, unit, lane);
  }
}

// Every block must call this after the same barrier: true while some problem goes on.
__device__ bool any_active(CgState* const* states, int nstates) {
  __shared__ int act;
  if (threadIdx.x == 0) {
    int a = 0;
    for (int k = 0; k < nstates && !a; ++k) a = ldv(&states[k]->cont) != 0;
    act = a;
  }
  __syncthreads();
  return act != 0;
}

template <typename T>
__device__ __forceinline__ void run_phase(const PPhase& ph, const PTask* __restrict__ tasks, int gw, int nw, int lane) {
  int t = ph.t0;
  for (int u = gw; u < ph.units; u += nw) {
    while (t + 1 < ph.t1 && tasks[t + 1].u0 <= u) ++t;   // units ascend: tasks are visited in order
    run_unit<T>(tasks[t], u - tasks[t].u0, lane);
  }
}

template <typename T>
__global__ void __launch_bounds__(kPersistentThreads, kPersistentBlocksPerSm)
    k_persistent(const PPhase* __restrict__ phases, int nhead, int nbody, const PTask* __restrict__ tasks,
                 PBarrier* bar, CgState* const* states, int nstates, int max_iter) {
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  for (int p = 0; p < nhead; ++p) {
    run_phase<T>(phases[p], tasks, gw, nw, lane);
    if ((p + 1 < nhead || nbody > 0) && !grid_barrier(bar)) return;
  }
  for (int it = 0; it < max_iter && nbody > 0; ++it) {
    for (int p = nhead; p < nhead + nbody; ++p) {
      run_phase<T>(phases[p], tasks, gw, nw, lane);
      if (!grid_barrier(bar)) return;
      if (phases[p].check && !any_active(states, nstates)) return;
    }
  }
}

}  // namespace

template <typename T>
int persistent_grid() {
  static const int g = [] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persistent<T>, kPersistentThreads, 0);
    return sms * std::max(1, std::min(per, kPersistentBlocksPerSm));
  }();
  return g;
}

template <typename T>
cudaError_t persistent_launch(const PPhase* phases, int nhead, const PTask* tasks, PBarrier* bar, cudaStream_t s,
                              int nbody, CgState* const* states, int nstates, int max_iter) {
  if (nhead <= 0 && nbody <= 0) return cudaSuccess;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(persistent_grid<T>());
  cfg.blockDim = dim3(kPersistentThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_persistent<T>, phases, nhead, nbody, tasks, bar, states, nstates, max_iter);
}

template int persistent_grid<float>();
template int persistent_grid<double>();
template cudaError_t persistent_launch<float>(const PPhase*, int, const PTask*, PBarrier*, cudaStream_t, int,
                                              CgState* const*, int, int);
template cudaError_t persistent_launch<double>(const PPhase*, int, const PTask*, PBarrier*, cudaStream_t, int,
                                               CgState* const*, int, int);

}  // namespace nnmg
