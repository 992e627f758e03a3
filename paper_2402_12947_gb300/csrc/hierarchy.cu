// nnmg C ABI: hierarchy set-up, device residency, the V-cycle schedule and MG-PCG.
//
// Schedule of one V-cycle (Alg. 1 of Chen & Wells, zero initial guess on every level):
//   level l < L-1: nu x S (pre), r_l = b_l - A_l x_l, b_{l+1} = R_l r_l (x_{l+1} = 0),
//                  recurse, x_l += P_l x_{l+1}, nu x S (post)
//   level L-1:     x = A^{-1} b with the dense inverse (FP64)
// where S is the combined smoother of Sec. 4.2: S_c, cheb_degree fused Chebyshev steps,
// S_c (sandwich), or the global-then-local / global-only variants. Two launches are folded
// into neighbours without changing what is computed: the first pre-smoothing S_c (from
// x = 0, residual b) shares a launch with the first Chebyshev step, and the residual of the
// S_c that opens the post-smoothing, b - A(x + P x_c) = r_l - (A P) x_c, is formed in the
// prolongation's launch from the r_l kept by the restriction.
// MG-PCG (Sec. 6.2) keeps x, r, p, q, z and every scalar in FP64; in MIXED precision the
// V-cycle runs on FP32 copies of the operators (int32 indices) and of r, while the patch
// residuals and solves and the coarsest solve stay FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cctype>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <type_traits>

#include "internal.hpp"
#include "kernels.cuh"

namespace nnmg {

namespace {

thread_local std::string g_setup_error;

// Phase timer for set-up, printed to stderr when the environment sets NNMG_VERBOSE.
struct PhaseTimer {
  bool on = std::getenv("NNMG_VERBOSE") != nullptr;
  std::chrono::steady_clock::time_point t = std::chrono::steady_clock::now();
  void mark(const std::string& what) {
    if (!on) return;
    auto now = std::chrono::steady_clock::now();
    std::fprintf(stderr, "[nnmg setup] %-28s %8.3f s\n", what.c_str(),
                 std::chrono::duration<double>(now - t).count());
    t = now;
  }
};

#define CK(x)                                                                                            \
  do {                                                                                                   \
    cudaError_t e_ = (x);                                                                                \
    if (e_ != cudaSuccess)                                                                               \
      throw Error(e_ == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA,                            \
                  std::string(#x) + ": " + cudaGetErrorString(e_));                                      \
  } while (0)

// Device allocations owned by one hierarchy, stream-ordered on `stream` (cudaMallocAsync
// from the device's default pool, zero-filled; freed with cudaFreeAsync), so that building
// or freeing one hierarchy never synchronises the device under other hierarchies' solves.
struct DevMem {
  cudaStream_t stream = nullptr;
  std::vector<void*> ptrs;
  int64_t bytes = 0;
  template <typename T>
  T* alloc(size_t n) {
    if (n == 0) return nullptr;
    void* p = nullptr;
    CK(cudaMallocAsync(&p, n * sizeof(T), stream));
    ptrs.push_back(p);
    bytes += (int64_t)(n * sizeof(T));
    CK(cudaMemsetAsync(p, 0, n * sizeof(T), stream));
    return (T*)p;
  }
  // The host buffer may be released as soon as this returns (pageable copies are staged).
  template <typename T>
  T* upload(const T* src, size_t n) {
    T* p = alloc<T>(n);
    if (p) CK(cudaMemcpyAsync(p, src, n * sizeof(T), cudaMemcpyHostToDevice, stream));
    return p;
  }
  template <typename T>
  T* upload(const std::vector<T>& v) {
    return upload(v.data(), v.size());
  }
  void release() {
    for (void* p : ptrs) cudaFreeAsync(p, stream);
    ptrs.clear();
    bytes = 0;
  }
};

// Slot order of a SELL-32 layout: rows sorted by length (descending, stable) inside
// consecutive windows of `sigma` rows; identity for sigma <= 1.
std::vector<int32_t> sell_order(const Csr& A, int sigma) {
  std::vector<int32_t> ord(A.nrows);
  for (int64_t i = 0; i < A.nrows; ++i) ord[i] = (int32_t)i;
  if (sigma <= 1) return ord;
  for (int64_t w0 = 0; w0 < A.nrows; w0 += sigma) {
    int64_t w1 = std::min<int64_t>(A.nrows, w0 + sigma);
    std::stable_sort(ord.begin() + w0, ord.begin() + w1, [&](int32_t a, int32_t b) {
      return A.rp[a + 1] - A.rp[a] > A.rp[b + 1] - A.rp[b];
    });
  }
  return ord;
}

// Padded entries of the SELL layout with `sub` lanes per row (slices of 32/sub rows, each
// padded to its longest row rounded up to a multiple of sub) for a slot order.
int64_t sell_padded(const Csr& A, const std::vector<int32_t>& ord, int sub = 1) {
  const int R = 32 / sub;
  int64_t tot = 0;
  for (int64_t s0 = 0; s0 < A.nrows; s0 += R) {
    int32_t w = 0;
    for (int64_t k = s0; k < std::min<int64_t>(A.nrows, s0 + R); ++k) w = std::max(w, A.rp[ord[k] + 1] - A.rp[ord[k]]);
    tot += 32 * (int64_t)((w + sub - 1) / sub);
  }
  return tot;
}

// Column indices of a layout (SELL slices or CSR-vector rows, "groups"): col = the 32-bit
// indices, base[g] = the smallest column of group g when it spans < 2^16 columns, else -1.
// Mostly narrow (at least half the nonzeros in narrow groups): 16-bit offsets, plus the
// 32-bit array when some group is wide; mostly wide: 32-bit indices only.
template <typename T, typename Each>
void set_indices(SellMat<T>& S, DevMem& mem, const std::vector<int32_t>& col, std::vector<int32_t>& base,
                 int64_t narrow_nnz, Each&& each) {
  const int64_t nnz = S.nnz;
  if (2 * narrow_nnz < nnz) {
    S.col = mem.upload(col);
    S.idx_bytes = 4.0 * (double)nnz;
    return;
  }
  std::vector<uint16_t> c16(col.size(), 0);
  bool any_wide = false;
  for (size_t g = 0; g < base.size(); ++g) {
    if (base[g] < 0) {
      any_wide = true;
      continue;
    }
    const int32_t b = base[g];
    each((int64_t)g, [&](int64_t k) { c16[k] = (uint16_t)(col[k] - b); });
  }
  S.col16 = mem.upload(c16);
  S.cbase = mem.upload(base);
  if (any_wide) S.col = mem.upload(col);
  S.idx_bytes = 2.0 * (double)narrow_nnz + 4.0 * (double)(nnz - narrow_nnz);
}

// Host CSR -> device SELL (values converted to T), slots in the order of sell_order. With
// sub lanes per row a slice holds 32/sub rows and entry j of its row r sits at step j/sub,
// lane r*sub + j%sub; padding has value 0 and the slice's smallest column.
template <typename T>
SellMat<T> make_sell(const Csr& A, DevMem& mem, int sigma = 1, int sub = 1, bool wide_only = false) {
  SellMat<T> S;
  const int R = 32 / sub;
  S.nrows = (int32_t)A.nrows;
  S.ncols = (int32_t)A.ncols;
  S.nnz = A.nnz();
  S.sigma = std::max(1, sigma);
  S.sub = sub;
  S.nslices = (int32_t)((A.nrows + R - 1) / R);
  std::vector<int32_t> ord = sell_order(A, sigma);
  std::vector<int64_t> off(S.nslices + 1, 0);
  std::vector<int32_t> smin(S.nslices, 0);
  for (int32_t s = 0; s < S.nslices; ++s) {
    int32_t w = 0, mn = INT32_MAX;
    for (int64_t k = (int64_t)s * R; k < std::min<int64_t>(A.nrows, (int64_t)s * R + R); ++k) {
      const int32_t r = ord[k], len = A.rp[r + 1] - A.rp[r];
      w = std::max(w, len);
      if (len > 0) mn = std::min(mn, A.ci[A.rp[r]]);
    }
    smin[s] = mn == INT32_MAX ? 0 : mn;
    off[s + 1] = off[s] + 32 * (int64_t)((w + sub - 1) / sub);
  }
  S.padded = off[S.nslices];
  std::vector<int32_t> col(S.padded, 0);
  std::vector<T> val(S.padded, T(0));
  parallel_for(S.nslices, [&](int64_t lo, int64_t hi) {
    for (int64_t s = lo; s < hi; ++s) {
      for (int64_t o = off[s]; o < off[s + 1]; ++o) col[o] = smin[s];
      for (int r = 0; r < R; ++r) {
        const int64_t k = s * R + r;
        if (k >= A.nrows) break;
        const int32_t row = ord[k], len = A.rp[row + 1] - A.rp[row];
        for (int32_t j = 0; j < len; ++j) {
          const int64_t o = off[s] + (int64_t)(j / sub) * 32 + r * sub + j % sub;
          col[o] = A.ci[A.rp[row] + j];
          val[o] = (T)A.v[A.rp[row] + j];
        }
      }
    }
  });
  S.off = mem.upload(off);
  S.val = mem.upload(val);
  // 16-bit column offsets from the slice's smallest column for every slice that spans
  // < 2^16 columns; the others keep 32-bit indices (cbase = -1)
  std::vector<int32_t> base(S.nslices, 0);
  std::vector<int64_t> snnz(S.nslices, 0);
  int64_t narrow_nnz = 0;
  for (int32_t sl = 0; sl < S.nslices; ++sl) {
    for (int64_t k = (int64_t)sl * R; k < std::min<int64_t>(A.nrows, (int64_t)sl * R + R); ++k)
      snnz[sl] += A.rp[ord[k] + 1] - A.rp[ord[k]];
    if (off[sl + 1] == off[sl]) continue;
    int32_t mn = INT32_MAX, mx = INT32_MIN;
    for (int64_t k = off[sl]; k < off[sl + 1]; ++k) mn = std::min(mn, col[k]), mx = std::max(mx, col[k]);
    base[sl] = (int64_t)mx - mn <= 65535 ? mn : -1;
    if (base[sl] >= 0) narrow_nnz += snnz[sl];
  }
  if (wide_only) narrow_nnz = 0;  // 32-bit indices only
  set_indices(S, mem, col, base, narrow_nnz, [&](int32_t sl, auto&& f) {
    for (int64_t k = off[sl]; k < off[sl + 1]; ++k) f(k);
  });
  if (sigma > 1) S.perm = mem.upload(ord);
  // chunks of whole slices for the TMA-staged kernel (one lane per row, 32-bit indices, every
  // slice within one shared-memory stage)
  const int64_t E = tma_stage_entries<T>();
  bool fits = sub == 1 && S.col16 == nullptr && S.nslices > 0;
  for (int32_t sl = 0; fits && sl < S.nslices; ++sl) fits = off[sl + 1] - off[sl] <= E;
  if (fits) {
    std::vector<int32_t> ch(1, 0);
    int64_t acc = 0;
    for (int32_t sl = 0; sl < S.nslices; ++sl) {
      const int64_t n = off[sl + 1] - off[sl];
      if (acc + n > E) ch.push_back(sl), acc = 0;
      acc += n;
    }
    ch.push_back(S.nslices);
    S.nchunks = (int32_t)ch.size() - 1;
    S.chunks = mem.upload(ch);
  }
  return S;
}

// Host CSR -> device CSR-vector layout (G lanes per row; values converted to T).
template <typename T>
SellMat<T> make_csrv(const Csr& A, DevMem& mem, int lanes) {
  SellMat<T> S;
  S.nrows = (int32_t)A.nrows;
  S.ncols = (int32_t)A.ncols;
  S.nnz = A.nnz();
  S.padded = A.nnz();
  S.lanes = lanes;
  std::vector<T> val(A.v.begin(), A.v.end());
  S.rp = mem.upload(A.rp);
  S.val = mem.upload(val);
  // 16-bit column offsets from each row's first (smallest) column for rows spanning
  // < 2^16 columns; the others keep 32-bit indices (cbase = -1)
  std::vector<int32_t> base(A.nrows, 0);
  int64_t narrow_nnz = 0;
  for (int64_t i = 0; i < A.nrows; ++i)
    if (A.rp[i + 1] > A.rp[i]) {
      base[i] = (int64_t)A.ci[A.rp[i + 1] - 1] - A.ci[A.rp[i]] <= 65535 ? A.ci[A.rp[i]] : -1;
      if (base[i] >= 0) narrow_nnz += A.rp[i + 1] - A.rp[i];
    }
  set_indices(S, mem, A.ci, base, narrow_nnz, [&](int64_t i, auto&& f) {
    for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) f(k);
  });
  return S;
}

struct Layout {
  int lanes, sigma, unroll, sub, pf;
};

template <typename T>
SellMat<T> make_layout(const Csr& A, DevMem& mem, Layout L) {
  // the TMA-staged kernel (unroll 5) streams 32-bit indices
  SellMat<T> S = L.lanes > 1 ? make_csrv<T>(A, mem, L.lanes) : make_sell<T>(A, mem, L.sigma, L.sub, L.unroll == 5);
  S.unroll = L.unroll;
  S.pf = L.lanes > 1 ? 0 : L.pf;
  S.tma = L.lanes == 1 && L.unroll == 5 && S.chunks != nullptr;
  return S;
}

std::string layout_name(const Layout& c) {
  if (c.lanes > 1) return "v" + std::to_string(c.lanes);
  const char* loop = c.unroll == 2 ? "p" : (c.unroll == 3 ? "q" : (c.unroll == 5 ? "t" : ""));
  return "s" + std::to_string(c.sigma) + (c.sub > 1 ? "x" + std::to_string(c.sub) : "") + loop +
         (c.pf > 0 ? "f" + std::to_string(c.pf) : "");
}

// Tuning cache (environment variable NNMG_TUNE_CACHE = a file path): the autotuner's choice
// per operator, keyed by value type, shape, nonzeros and a checksum of the pattern, so that
// another run on the same operators (a profiler run, whose own timings are distorted) uses
// the same layouts. Lines: key lanes sigma unroll sub.
std::mutex g_tune_mu;
std::map<std::string, Layout>* g_tune = nullptr;

std::string tune_key(const Csr& A, int vbytes) {
  uint64_t h = 1469598103934665603ull;
  for (int32_t c : A.ci) h = (h ^ (uint32_t)c) * 1099511628211ull;
  for (int32_t r : A.rp) h = (h ^ (uint32_t)r) * 1099511628211ull;
  char buf[128];
  std::snprintf(buf, sizeof(buf), "%d:%lld:%lld:%lld:%016llx", vbytes, (long long)A.nrows, (long long)A.ncols,
                (long long)A.nnz(), (unsigned long long)h);
  return buf;
}

bool tune_lookup(const std::string& key, Layout* out) {
  const char* path = std::getenv("NNMG_TUNE_CACHE");
  if (!path || !*path) return false;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (!g_tune) {
    g_tune = new std::map<std::string, Layout>();
    if (FILE* f = std::fopen(path, "r")) {
      char k[128];
      Layout L{};
      while (std::fscanf(f, "%127s %d %d %d %d %d", k, &L.lanes, &L.sigma, &L.unroll, &L.sub, &L.pf) == 6)
        (*g_tune)[k] = L;
      std::fclose(f);
    }
  }
  auto it = g_tune->find(key);
  if (it == g_tune->end()) return false;
  *out = it->second;
  return true;
}

void tune_store(const std::string& key, const Layout& L) {
  const char* path = std::getenv("NNMG_TUNE_CACHE");
  if (!path || !*path) return;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (g_tune) (*g_tune)[key] = L;
  if (FILE* f = std::fopen(path, "a")) {
    std::fprintf(f, "%s %d %d %d %d %d\n", key.c_str(), L.lanes, L.sigma, L.unroll, L.sub, L.pf);
    std::fclose(f);
  }
}

// Layout of an operator too small for timing to separate the candidates: CSR vector with G
// lanes per row, G the smallest power of two >= half the mean row length, within [4, 32], so
// that a row takes about two dependent load steps, but with no more threads than one wave of
// the device (152 SMs x 2048); an operator with rows enough for two waves at four lanes takes
// SELL with one lane per row (predicated steps of eight) instead.
Layout rule_layout(const Csr& A) {
  constexpr int64_t kWave = 152 * 2048;
  const double mean = A.nrows > 0 ? (double)A.nnz() / (double)A.nrows : 0.0;
  if (A.nrows * 4 > 2 * kWave) return Layout{1, 1, 3, 1, 0};
  int g = 4;
  while (g < 32 && 2.0 * g < mean && A.nrows * 2 * g <= kWave) g *= 2;
  return Layout{g, 1, 1, 1, 0};
}

// Layout from its name (the inverse of layout_name): "v<G>" = CSR vector with G in {4, 8,
// 16, 32} lanes per row; "s<sigma>[x<S>][p|q|t][f<pf>]" = SELL with rows sorted in windows of
// sigma, S in {2, 4} lanes per row, row loop p = predicated steps of four, q = predicated
// steps of eight, t = the TMA-staged kernel (default: steps of four with a scalar tail), and
// an L2 prefetch distance of pf slices; "tma" = "s1t".
bool parse_layout(const std::string& name, Layout* out) {
  Layout L{1, 1, 1, 1, 0};
  if (name == "tma") {
    *out = {1, 1, 5, 1, 0};
    return true;
  }
  size_t i = 0;
  auto num = [&](int* v) {
    size_t j = i;
    while (j < name.size() && std::isdigit((unsigned char)name[j])) ++j;
    if (j == i || j - i > 7) return false;
    *v = std::atoi(name.substr(i, j - i).c_str());
    i = j;
    return true;
  };
  if (name.empty()) return false;
  if (name[0] == 'v') {
    ++i;
    if (!num(&L.lanes) || i != name.size()) return false;
    if (L.lanes != 4 && L.lanes != 8 && L.lanes != 16 && L.lanes != 32) return false;
    *out = L;
    return true;
  }
  if (name[0] != 's') return false;
  ++i;
  if (!num(&L.sigma) || L.sigma < 1) return false;
  if (i < name.size() && name[i] == 'x') {
    ++i;
    if (!num(&L.sub) || (L.sub != 2 && L.sub != 4)) return false;
    L.unroll = 2;
  }
  if (i < name.size() && (name[i] == 'p' || name[i] == 'q' || name[i] == 't')) {
    L.unroll = name[i] == 'p' ? 2 : (name[i] == 'q' ? 3 : 5);
    ++i;
  }
  if (L.unroll == 5 && L.sub != 1) return false;
  if (i < name.size() && name[i] == 'f') {
    ++i;
    if (!num(&L.pf) || L.pf < 1) return false;
  }
  if (i != name.size()) return false;
  *out = L;
  return true;
}

// Autotuner (sigma option 0): time y = A x on the device for each candidate layout and keep
// the fastest. Candidates: SELL with one lane per row and windows 1, 256, 2048 (when sorting
// removes padding), each with steps of four and a scalar or a predicated row remainder and
// with predicated steps of eight; SELL with 2 and 4 lanes per row at the best window; CSR
// vector with 4, 8, 16, 32 lanes per row up to twice the longest row; then, on large
// operators whose best layout is SELL, bulk L2 prefetch distances of half, one and two
// waves of slices. Timing: one warm-up launch, then the mean of 5 launches between CUDA
// events, the best of three rounds.
// The environment variable NNMG_FORCE_LAYOUT=<layout name> (parse_layout) skips the timing
// and gives every operator that layout, so that tests can run each candidate's kernels; the
// TMA-staged kernel ("tma", "s1t") exists only behind this switch and applies to the level
// operators whose slices fit its shared-memory stages (allow_tma), the others are tuned.
template <typename T>
SellMat<T> tuned_sell(const Csr& A, DevMem& mem, int sigma, int64_t rule_below, std::string* log,
                      bool allow_tma = false) {
  if (sigma != 0 || A.nrows == 0) return make_sell<T>(A, mem, std::max(sigma, 1));
  const char* force = std::getenv("NNMG_FORCE_LAYOUT");
  if (force && *force) {
    Layout F{};
    if (!parse_layout(force, &F)) throw Error(MG_ERR_INVALID_ARG, std::string("NNMG_FORCE_LAYOUT: unknown layout ") + force);
    bool use = true;
    if (F.unroll == 5) {  // the TMA-staged kernel where its chunk table exists
      use = false;
      if (allow_tma) {
        DevMem trial;
        trial.stream = mem.stream;
        use = make_layout<T>(A, trial, F).tma != 0;
        trial.release();
      }
    }
    if (use) {
      if (log) *log += " forced " + layout_name(F);
      return make_layout<T>(A, mem, F);
    }
  }
  if (A.nnz() < rule_below) {
    const Layout R = rule_layout(A);
    if (log) *log += " rule " + layout_name(R);
    return make_layout<T>(A, mem, R);
  }
  const std::string key = tune_key(A, (int)sizeof(T));
  Layout cached{};
  if (tune_lookup(key, &cached)) {
    if (log) *log += " cached " + layout_name(cached);
    return make_layout<T>(A, mem, cached);
  }
  int maxlen = 0;
  for (int64_t i = 0; i < A.nrows; ++i) maxlen = std::max(maxlen, A.rp[i + 1] - A.rp[i]);
  std::vector<Layout> cand;
  int64_t last_pad = -1;
  for (int c : {1, 256, 2048}) {
    int64_t pad = sell_padded(A, sell_order(A, c));
    if (last_pad >= 0 && pad >= (int64_t)(0.995 * (double)last_pad)) continue;  // sorting gains nothing more
    last_pad = pad;
    cand.push_back({1, c, 1, 1, 0});
    cand.push_back({1, c, 2, 1, 0});
    cand.push_back({1, c, 3, 1, 0});
  }
  DevMem scratch;
  scratch.stream = mem.stream;
  const cudaStream_t st = mem.stream;
  T* x = scratch.alloc<T>(std::max<int64_t>(A.ncols, 1));
  T* y = scratch.alloc<T>(std::max<int64_t>(A.nrows, 1));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  Layout best = cand[0];
  float best_ms = -1.f;
  // Candidates that share a storage (lanes, window, lanes per row) are built once and timed
  // in three interleaved rounds; each keeps its fastest round, so that a slow moment of the
  // device does not decide between layouts that differ only in the row loop.
  auto try_layouts = [&](const std::vector<Layout>& cs) {
    DevMem trial;
    trial.stream = st;
    for (size_t g0 = 0; g0 < cs.size();) {
      size_t g1 = g0 + 1;
      while (g1 < cs.size() && cs[g1].lanes == cs[g0].lanes && cs[g1].sigma == cs[g0].sigma && cs[g1].sub == cs[g0].sub &&
             (cs[g1].unroll == 5) == (cs[g0].unroll == 5))
        ++g1;
      trial.release();
      SellMat<T> S = make_layout<T>(A, trial, cs[g0]);
      std::vector<float> tbest(g1 - g0, -1.f);
      std::vector<char> bad(g1 - g0, 0);
      for (int round = 0; round < 3; ++round)
        for (size_t i = g0; i < g1; ++i) {
          const Layout& c = cs[i];
          S.unroll = c.unroll;
          S.pf = c.lanes > 1 ? 0 : c.pf;
          S.tma = c.lanes == 1 && c.unroll == 5 && S.chunks != nullptr;
          if ((c.unroll == 5 && !S.tma) || bad[i - g0]) {
            bad[i - g0] = 1;  // no chunk table for this storage, or a bounded wait gave up
            continue;
          }
          sell_spmv<T>(S, x, y, st);
          CK(cudaEventRecord(e0, st));
          for (int rep = 0; rep < 5; ++rep) sell_spmv<T>(S, x, y, st);
          CK(cudaEventRecord(e1, st));
          CK(cudaEventSynchronize(e1));
          float ms = 0.f;
          CK(cudaEventElapsedTime(&ms, e0, e1));
          if (S.tma && take_wait_timeout(st)) bad[i - g0] = 1;
          if (tbest[i - g0] < 0 || ms < tbest[i - g0]) tbest[i - g0] = ms;
        }
      for (size_t i = g0; i < g1; ++i) {
        if (bad[i - g0]) continue;
        const float ms = tbest[i - g0];
        if (log) *log += " " + layout_name(cs[i]) + ":" + std::to_string((int)(ms / 5 * 1e3)) + "us";
        if (best_ms < 0 || ms < best_ms) {
          best_ms = ms;
          best = cs[i];
        }
      }
      g0 = g1;
    }
    trial.release();
  };
  try_layouts(cand);
  std::vector<Layout> more;
  for (int sub : {2, 4}) more.push_back({1, best.sigma, 2, sub, 0});
  for (int g : {4, 8, 16, 32})
    if (g <= 2 * std::max(maxlen, 2)) more.push_back({g, 1, 1, 1, 0});
  try_layouts(more);
  // bulk L2 prefetch of the slices about half a wave, one wave or two waves ahead (a wave:
  // 152 SMs x 64 resident warps, one slice per warp), on the best SELL layout
  if (best.lanes == 1 && A.nrows >= 8 * 9728 * 32 / best.sub) {
    std::vector<Layout> pfc;
    for (int pf : {4864, 9728, 19456}) pfc.push_back({1, best.sigma, best.unroll, best.sub, pf});
    try_layouts(pfc);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  scratch.release();
  tune_store(key, best);
  return make_layout<T>(A, mem, best);
}

template <typename T>
struct DevLevel {
  int n = 0;
  int32_t* perm = nullptr;  // internal index -> library index (null: same numbering)
  SellMat<T> A, P, R;
  T *dinv = nullptr, *b = nullptr, *x = nullptr, *xt = nullptr, *d = nullptr, *res = nullptr;
  std::vector<double> cd, cr;
  // local correction
  int np = 0, nt = 0, nitems = 0, max_patch = 0, pw = 0;
  int32_t *pdofs = nullptr, *pci = nullptr;   // patch rows of A, ELL with pw slots per row
  int32_t* plen = nullptr;                     // entries of each patch row
  double* pv = nullptr;
  double *inv = nullptr, *rbuf = nullptr;
  float* inv32 = nullptr;            // FP32 arena of the well-conditioned patches' inverses
  std::vector<int32_t> pfp32;        // per patch: 1 if applied in FP32
  PatchItem* items = nullptr;
  // rows (A P)_{i,:} of the patch rows, ELL with apw slots each and aplen entries (the S_c
  // after prolongation)
  int apw = 0;
  int32_t *apci = nullptr, *aplen = nullptr;
  double* apv = nullptr;
  // rows coupled to patch DoFs, with their entries of A (first Chebyshev step after S_c)
  int nh = 0;
  int32_t *hrow = nullptr, *hrp = nullptr, *hci = nullptr;
  T* hv = nullptr;
  // multicolour SGS: per colour, its rows of A without the diagonal and without couplings
  // inside the colour, and the level rows they update
  std::vector<SellMat<T>> gs;
  std::vector<int32_t*> gs_rows;
  // levels run inside the persistent launch: A, P, R as CSR (0, 1, 2) with G lanes per row,
  // and one descriptor per patch row
  int32_t *crp[3] = {nullptr, nullptr, nullptr}, *cci[3] = {nullptr, nullptr, nullptr};
  T* cval[3] = {nullptr, nullptr, nullptr};
  int cG[3] = {4, 4, 4};
  PRow* prow = nullptr;
};

}  // namespace

// The V-cycle in one arithmetic type T (double or float).
template <typename T>
struct Engine {
  std::vector<DevLevel<T>> lv;
  int cheb_k = 2, nu = 1, order = MG_SMOOTHER_SANDWICH;
  bool sgs = false;   // global smoother: multicolour SGS instead of Chebyshev
  uint32_t local_mask = 0xffffffffu;
  // coarsest level
  int nc = 0, kchunk = 256;
  double *Xc = nullptr, *cpart = nullptr;
  int launches = 0;
  // persistent launch of the cycle from level pers_from down (-1: none), its program
  int pers_from = -1, pers_phases = 0;
  PPhase* d_phases = nullptr;
  PTask* d_tasks = nullptr;
  PBarrier* bar = nullptr;
  double* cb64 = nullptr;   // FP64 copy of the coarsest right-hand side (persistent launch)
  // the FP64 level-0 operator as CSR for the CG product of a persistent solve (pers_from == 0)
  int32_t *a0rp = nullptr, *a0ci = nullptr;
  double* a0v = nullptr;
  int a0G = 4;
  std::vector<PTask> htasks;
  std::vector<PPhase> hphases;

  bool local_on(int l) const {
    return lv[l].np > 0 && order != MG_SMOOTHER_GLOBAL && ((local_mask >> std::min(l, 31)) & 1u);
  }
  // zero: 0 = general iterate, 1 = x is zero, 2 = x is zero outside the patch DoFs, 3 = x is
  // zero and the S_c from zero that precedes the first step runs in the same launch
  void cheb(int l, cudaStream_t s, int zero = 0) {
    DevLevel<T>& L = lv[l];
    T *xa = L.x, *xb = L.xt;
    for (int j = 0; j < cheb_k; ++j) {
      if (j == 0 && zero == 3) {
        cheb_entry_local<T>(L.nitems, L.items, L.pdofs, L.inv, L.inv32, L.max_patch, L.n, L.b, L.dinv, xa, L.d, xb,
                            L.cr[0], L.nh, L.hrow, L.hrp, L.hci, L.hv, s);
        launches += L.nh > 0 ? 2 : 1;
      } else if (j == 0 && zero) {
        const int nh = zero == 2 ? L.nh : 0;
        cheb_first_from_zero<T>(L.n, L.b, L.dinv, xa, L.d, xb, L.cr[0], nh, L.hrow, L.hrp, L.hci, L.hv, s);
        launches += nh > 0 ? 2 : 1;
      } else {
        sell_cheb<T>(L.A, xa, L.b, L.dinv, L.d, xb, L.cd[j], L.cr[j], j == 0, s);
        ++launches;
      }
      std::swap(xa, xb);
    }
    if (xa != L.x) {
      CK(cudaMemcpyAsync(L.x, xa, sizeof(T) * L.n, cudaMemcpyDeviceToDevice, s));
      ++launches;
    }
  }
  // One symmetric sweep: colours 0..C-1, then C-1..0.
  void sgs_sweep(int l, cudaStream_t s) {
    DevLevel<T>& L = lv[l];
    const int C = (int)L.gs.size();
    for (int j = 0; j < 2 * C; ++j) {
      const int c = j < C ? j : 2 * C - 1 - j;
      sell_gs<T>(L.gs[c], L.gs_rows[c], L.b, L.dinv, L.x, s);
    }
    launches += 2 * C;
  }
  // S_g; zero as in cheb (the SGS sweep has no zero-iterate shortcut)
  void global(int l, cudaStream_t s, int zero = 0) {
    if (sgs) sgs_sweep(l, s);
    else cheb(l, s, zero);
  }
  // zero: the iterate is zero (residual b); rready: the patch residual is already in rbuf
  void local(int l, cudaStream_t s, bool zero = false, bool rready = false) {
    DevLevel<T>& L = lv[l];
    if (!zero && !rready) {
      patch_residual<T>(L.nt, L.pw, L.pdofs, L.plen, L.pci, L.pv, L.b, L.x, L.rbuf, s);
      ++launches;
    }
    patch_solve<T>(L.nitems, L.items, L.pdofs, L.inv, L.inv32, zero ? nullptr : L.rbuf, L.b, L.x, L.max_patch, s);
    ++launches;
  }
  // zero: the iterate is zero on entry (first pre-smoothing on every level of a cycle);
  // rready: the residual of a leading S_c is already in rbuf (first post-smoothing)
  void smooth(int l, bool post, cudaStream_t s, bool zero = false, bool rready = false) {
    if (!local_on(l)) {
      global(l, s, zero ? 1 : 0);
      return;
    }
    if (order == MG_SMOOTHER_SANDWICH) {
      if (zero && !sgs) {
        cheb(l, s, 3);  // S_c from zero and the first Chebyshev step share a launch
      } else {
        local(l, s, zero, rready);
        global(l, s, zero ? 2 : 0);
      }
      local(l, s);
    } else if (!post) {
      global(l, s, zero ? 1 : 0);
      local(l, s);
    } else {
      local(l, s, false, rready);
      global(l, s);
    }
  }
  void coarse(cudaStream_t s) {
    DevLevel<T>& L = lv.back();
    dense_solve<T>(nc, Xc, L.b, L.x, cpart, kchunk, s);
    launches += 2;
  }
  void residual_restrict(int l, cudaStream_t s) {
    DevLevel<T>& L = lv[l];
    DevLevel<T>& C = lv[l + 1];
    sell_resid<T>(L.A, L.x, L.b, L.res, s);
    sell_restrict<T>(L.R, L.res, C.b, C.x, s);
    launches += 2;
  }
  void prolong(int l, cudaStream_t s) {
    sell_prolong<T>(lv[l].P, lv[l + 1].x, lv[l].x, s);
    ++launches;
  }
  // Prolongation and, in the same launch, the residual of the first post-smoothing S_c
  // (every post-smoothing order starts with S_c), from the residual kept by the restriction.
  bool prolong_with_patch_residual(int l) const { return local_on(l) && lv[l].apw > 0; }
  void prolong_pr(int l, cudaStream_t s) {
    DevLevel<T>& L = lv[l];
    sell_prolong_pr<T>(L.P, lv[l + 1].x, L.x, L.nt, L.apw, L.pdofs, L.aplen, L.apci, L.apv, L.res, L.rbuf, s);
    ++launches;
  }
  void cycle(int l, cudaStream_t s) {
    if (l == pers_from) {
      CK(persistent_launch<T>(d_phases, pers_phases, d_tasks, bar, s));
      ++launches;
      return;
    }
    if (l == (int)lv.size() - 1) {
      coarse(s);
      return;
    }
    for (int k = 0; k < nu; ++k) smooth(l, false, s, k == 0);
    residual_restrict(l, s);
    cycle(l + 1, s);
    const bool pr = prolong_with_patch_residual(l);
    if (pr) prolong_pr(l, s);
    else prolong(l, s);
    for (int k = 0; k < nu; ++k) smooth(l, true, s, false, pr && k == 0);
  }

  // ---- persistent launch of the small levels: set-up ----
  // Lanes per row of a CSR operator in the persistent kernel: about eight entries per lane
  // (two steps of four loads), at least 4 and at most 32 lanes.
  static int csr_lanes(const Csr& A) {
    const double avg = A.nrows > 0 ? (double)A.nnz() / (double)A.nrows : 0.0;
    int G = 4;
    while (G < 32 && 8.0 * G < avg) G *= 2;
    return G;
  }
  // The first level with at most thr DoFs such that every level below is smaller still (-1
  // when none, or thr = 0, or the global smoother is SGS); its CSR operators and patch rows
  // are uploaded and the cycle from it down is recorded and uploaded.
  void build_persistent(const std::vector<LevelH>& dl, const std::vector<std::vector<int64_t>>& inv_off, int thr,
                        DevMem& mem) {
    pers_from = -1;
    const int L = (int)lv.size();
    if (thr <= 0 || sgs) return;
    for (int l = L - 1; l >= 0 && lv[l].n <= thr; --l) pers_from = l;
    if (pers_from < 0) return;
    for (int l = pers_from; l + 1 < L; ++l) {
      DevLevel<T>& D = lv[l];
      const Csr* ops[3] = {&dl[l].A, &dl[l].P, &dl[l].R};
      for (int k = 0; k < 3; ++k) {
        const Csr& M = *ops[k];
        D.crp[k] = mem.upload(M.rp);
        D.cci[k] = mem.upload(M.ci);
        std::vector<T> v(M.v.begin(), M.v.end());
        D.cval[k] = mem.upload(v);
        D.cG[k] = csr_lanes(M);
      }
      if (D.np > 0) {
        const std::vector<int32_t>& ptr = dl[l].patch_ptr;
        std::vector<PRow> rows;
        rows.reserve(D.nt);
        for (int p = 0; p + 1 < (int)ptr.size(); ++p) {
          const int32_t m = ptr[p + 1] - ptr[p];
          for (int32_t i = 0; i < m; ++i) rows.push_back(PRow{ptr[p], m, i, 0, inv_off[l][p] + (int64_t)i * m});
        }
        D.prow = mem.upload(rows);
      }
    }
    if (pers_from == 0) {
      a0rp = mem.upload(dl[0].A.rp);
      a0ci = mem.upload(dl[0].A.ci);
      a0v = mem.upload(dl[0].A.v);
      a0G = csr_lanes(dl[0].A);
    }
    cb64 = mem.alloc<double>(nc);
    htasks.clear();
    hphases.clear();
    rec_cycle(pers_from);
    pers_phases = (int)hphases.size();
    d_tasks = mem.upload(htasks);
    d_phases = mem.upload(hphases);
    bar = mem.alloc<PBarrier>(1);
  }

  // ---- the cycle from a level down, recorded as a persistent program ----
  // Same schedule as cycle() and the functions it calls, step for step: every launch there is
  // a phase here (rec_* mirrors the function of the same name), and the two launches that
  // write disjoint arrays (S_c from zero with the first Chebyshev step; the prolongation with
  // the patch residual of the next S_c) each share a phase.
  void ph_open() { hphases.push_back(PPhase{(int)htasks.size(), (int)htasks.size(), 0, 0}); }
  void ph_task(PTask t) {
    if (t.n <= 0) return;
    PPhase& ph = hphases.back();
    t.u0 = ph.units;
    ph.units += ptask_units(t);
    htasks.push_back(t);
    ph.t1 = (int)htasks.size();
  }
  void ph_close() {
    if (hphases.back().units == 0) hphases.pop_back();
  }
  static PTask task(int kind, int n) {
    PTask t;
    std::memset(&t, 0, sizeof(t));
    t.kind = kind;
    t.n = n;
    t.G = 4;
    return t;
  }
  // A CSR task over operator op (0 = A, 1 = P, 2 = R) of level l.
  PTask csr_task(int kind, int l, int op) {
    DevLevel<T>& L = lv[l];
    PTask t = task(kind, op == 2 ? lv[l + 1].n : L.n);
    t.rp = L.crp[op];
    t.ci = L.cci[op];
    t.val = L.cval[op];
    t.G = L.cG[op];
    return t;
  }
  PTask halo_task(int l, const T* x, T* xout, double cr) {
    DevLevel<T>& L = lv[l];
    PTask t = task(PK_CHEB_FIRST, L.nh);
    t.rows = L.hrow;
    t.rp = L.hrp;
    t.ci = L.hci;
    t.val = L.hv;
    t.G = 8;
    t.x = x;
    t.b = L.b;
    t.dinv = L.dinv;
    t.d = L.d;
    t.y = xout;
    t.c2 = cr;
    return t;
  }
  PTask patch_solve_task(int l, bool zero) {
    DevLevel<T>& L = lv[l];
    PTask t = task(PK_PATCH_SOLVE, L.nt);
    t.prow = L.prow;
    t.inv = L.inv;
    t.pdofs = L.pdofs;
    t.rbuf = zero ? nullptr : L.rbuf;
    t.b = L.b;
    t.y = L.x;
    return t;
  }
  void rec_cheb(int l, int zero) {
    DevLevel<T>& L = lv[l];
    T *xa = L.x, *xb = L.xt;
    for (int j = 0; j < cheb_k; ++j) {
      if (j == 0 && zero) {
        ph_open();
        if (zero == 3) ph_task(patch_solve_task(l, true));
        PTask c = task(PK_CHEB0, L.n);
        c.x = zero == 3 ? nullptr : xa;
        c.b = L.b;
        c.dinv = L.dinv;
        c.d = L.d;
        c.y = xb;
        c.c2 = L.cr[0];
        ph_task(c);
        ph_close();
        if ((zero == 3 || zero == 2) && L.nh > 0) {
          ph_open();
          ph_task(halo_task(l, xa, xb, L.cr[0]));
          ph_close();
        }
      } else {
        PTask c = csr_task(j == 0 ? PK_CHEB_FIRST : PK_CHEB, l, 0);
        c.x = xa;
        c.b = L.b;
        c.dinv = L.dinv;
        c.d = L.d;
        c.y = xb;
        c.c1 = L.cd[j];
        c.c2 = L.cr[j];
        ph_open();
        ph_task(c);
        ph_close();
      }
      std::swap(xa, xb);
    }
    if (xa != L.x) {
      PTask c = task(PK_COPY, L.n);
      c.x = xa;
      c.y = L.x;
      ph_open();
      ph_task(c);
      ph_close();
    }
  }
  void rec_local(int l, bool zero = false, bool rready = false) {
    DevLevel<T>& L = lv[l];
    if (!zero && !rready) {
      PTask r = task(PK_PATCH_RES, L.nt);
      r.w = L.pw;
      r.pdofs = L.pdofs;
      r.plen = L.plen;
      r.pci = L.pci;
      r.pv = L.pv;
      r.b = L.b;
      r.x = L.x;
      r.rbuf = L.rbuf;
      ph_open();
      ph_task(r);
      ph_close();
    }
    ph_open();
    ph_task(patch_solve_task(l, zero));
    ph_close();
  }
  void rec_smooth(int l, bool post, bool zero = false, bool rready = false) {
    if (!local_on(l)) {
      rec_cheb(l, zero ? 1 : 0);
      return;
    }
    if (order == MG_SMOOTHER_SANDWICH) {
      if (zero) rec_cheb(l, 3);
      else {
        rec_local(l, false, rready);
        rec_cheb(l, 0);
      }
      rec_local(l);
    } else if (!post) {
      rec_cheb(l, zero ? 1 : 0);
      rec_local(l);
    } else {
      rec_local(l, false, rready);
      rec_cheb(l, 0);
    }
  }
  void rec_cycle(int l) {
    if (l == (int)lv.size() - 1) {
      DevLevel<T>& C = lv.back();
      PTask t = task(PK_DENSE, nc);
      t.inv = Xc;
      t.b = C.b;
      t.y = C.x;
      if (l > pers_from) t.y64 = cb64;   // filled by the restriction in this launch
      ph_open();
      ph_task(t);
      ph_close();
      return;
    }
    DevLevel<T>& L = lv[l];
    DevLevel<T>& C = lv[l + 1];
    for (int k = 0; k < nu; ++k) rec_smooth(l, false, k == 0);
    PTask r = csr_task(PK_RESID, l, 0);
    r.x = L.x;
    r.b = L.b;
    r.y = L.res;
    ph_open();
    ph_task(r);
    ph_close();
    PTask q = csr_task(PK_RESTRICT, l, 2);
    q.x = L.res;
    q.y = C.b;
    q.z = C.x;
    if (l + 2 == (int)lv.size()) q.y64 = cb64;
    ph_open();
    ph_task(q);
    ph_close();
    rec_cycle(l + 1);
    const bool pr = prolong_with_patch_residual(l);
    PTask p = csr_task(PK_PROLONG, l, 1);
    p.x = C.x;
    p.y = L.x;
    ph_open();
    ph_task(p);
    if (pr) {
      PTask a = task(PK_PATCH_RES_AP, L.nt);
      a.w = L.apw;
      a.pdofs = L.pdofs;
      a.plen = L.aplen;
      a.pci = L.apci;
      a.pv = L.apv;
      a.b = L.res;
      a.x = C.x;
      a.rbuf = L.rbuf;
      ph_task(a);
    }
    ph_close();
    for (int k = 0; k < nu; ++k) rec_smooth(l, true, false, pr && k == 0);
  }
};

}  // namespace nnmg

using namespace nnmg;

struct mg_hierarchy {
  mg_options_t opt{};
  int L = 0, degree = 0;
  bool geometric = false, device = false;
  std::vector<LevelH> host;
  std::vector<double> fine_load_unit;  // b for f = 1 (geometric Poisson only)
  BoundaryFaces fine_faces;            // level-0 boundary facets (geometric elasticity only)
  std::vector<int64_t> ncells;
  std::string err;
  // device
  DevMem mem;
  std::unique_ptr<Engine<double>> e64;
  std::unique_ptr<Engine<float>> e32;
  SellMat<double> A0;  // fine operator in FP64 for the CG recurrence
  int n0 = 0;
  double *cb = nullptr, *cx = nullptr, *cr = nullptr, *cp = nullptr, *cq = nullptr, *cz = nullptr, *part = nullptr;
  int32_t* perm0 = nullptr;  // level-0 internal order (see build_device), null = library order
  CgState* st = nullptr;
  unsigned* ticket = nullptr;  // arrival counter of the fused reductions (see Reduce)
  CgState* hst = nullptr;  // pinned
  int nparts = 1, ap_parts = 1;
  cudaGraphExec_t graph = nullptr;
  cudaStream_t own_stream = nullptr;
  int launches_vcycle = 0, launches_iter = 0;
  int64_t dropped_dofs = 0;  // DoFs excluded as dependent by the dense direct solves
  bool uses_tma = false;     // some operator runs the TMA-staged kernel (bounded waits)
  // the whole MG-PCG solve as one persistent launch (hierarchies whose whole cycle runs
  // persistently, small_level_dofs >= n_0); empty otherwise
  struct Solo {
    PPhase* phases = nullptr;
    PTask* tasks = nullptr;
    CgState** states = nullptr;
    PBarrier* bar = nullptr;
    int nhead = 0, nbody = 0;
  } solo;

  bool mixed() const { return opt.precision == MG_PREC_MIXED; }
  template <typename F>
  void with_engine(F&& f) {
    if (e64) f(*e64);
    else f(*e32);
  }
  ~mg_hierarchy() {
    if (own_stream) cudaStreamSynchronize(own_stream);
    if (graph) cudaGraphExecDestroy(graph);
    mem.release();
    if (own_stream) {
      cudaStreamSynchronize(own_stream);
      cudaStreamDestroy(own_stream);
    }
    if (hst) pinned_release(reinterpret_cast<double*>(hst));
  }
};

namespace nnmg {
namespace {

void validate_options(const mg_options_t& o) {
  if (o.cheb_degree < 1 || o.cheb_degree > 16) throw Error(MG_ERR_INVALID_ARG, "cheb_degree must be in [1, 16]");
  if (o.nu < 1 || o.nu > 16) throw Error(MG_ERR_INVALID_ARG, "nu must be in [1, 16]");
  if (o.patch_layers < 0 || o.patch_layers > 8) throw Error(MG_ERR_INVALID_ARG, "patch_layers must be in [0, 8]");
  if (o.smoother < 0 || o.smoother > 2) throw Error(MG_ERR_INVALID_ARG, "unknown smoother order");
  if (o.precision < 0 || o.precision > 1) throw Error(MG_ERR_INVALID_ARG, "unknown precision");
  if (!(o.lmin_ratio > 0 && o.lmin_ratio < 1)) throw Error(MG_ERR_INVALID_ARG, "lmin_ratio must be in (0, 1)");
  if (!(o.lmax_safety > 0)) throw Error(MG_ERR_INVALID_ARG, "lmax_safety must be positive");
  if (o.sell_sigma < 0 || o.sell_sigma > (1 << 20)) throw Error(MG_ERR_INVALID_ARG, "sell_sigma must be in [0, 2^20]");
  if (o.global_smoother < 0 || o.global_smoother > 1) throw Error(MG_ERR_INVALID_ARG, "unknown global smoother");
  if (o.reorder < 0 || o.reorder > 3) throw Error(MG_ERR_INVALID_ARG, "unknown reorder mode");
  if (o.pde < 0 || o.pde > 1) throw Error(MG_ERR_INVALID_ARG, "unknown pde");
  if (o.small_level_dofs < 0) throw Error(MG_ERR_INVALID_ARG, "small_level_dofs must be >= 0");
  if (o.fp32_patch_kappa < 0) throw Error(MG_ERR_INVALID_ARG, "fp32_patch_kappa must be >= 0");
  if (o.tune_min_nnz < 0) throw Error(MG_ERR_INVALID_ARG, "tune_min_nnz must be >= 0");
  if (o.pde == MG_PDE_ELASTICITY && !(o.young > 0 && o.poisson_ratio > -1.0 && o.poisson_ratio < 0.5))
    throw Error(MG_ERR_INVALID_ARG, "elasticity needs E > 0 and -1 < nu < 1/2");
}

// Chebyshev coefficients per step: d = cd d + cr D^{-1} r (Sec. 3.2 three-term recurrence).
void cheb_coefficients(double lmax, double lmin, int k, std::vector<double>& cd, std::vector<double>& cr) {
  double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta, rho = 1.0 / sigma;
  cd.assign(1, 0.0);
  cr.assign(1, 1.0 / theta);
  for (int j = 1; j < k; ++j) {
    double rn = 1.0 / (2.0 * sigma - rho);
    cd.push_back(rn * rho);
    cr.push_back(2.0 * rn / delta);
    rho = rn;
  }
}

// Multicolour SGS operators of one level. The colouring (Hl.colour, library numbering) is
// carried to the internal order (perm: internal -> library). Per colour: its rows of the
// internal-order operator Hd.A without the diagonal and without couplings to rows of the
// same colour (all below 1e-12 sqrt(a_ii a_jj) by the colouring's construction), so that
// one launch can update the whole colour in place.
template <typename T>
void build_sgs_ops(const LevelH& Hl, const LevelH& Hd, const std::vector<int32_t>& perm, DevLevel<T>& D, DevMem& mem,
                   int sigma, int64_t rule_below) {
  const int64_t n = Hd.A.nrows;
  std::vector<int32_t> col(n);
  for (int64_t i = 0; i < n; ++i) col[i] = Hl.colour[perm.empty() ? i : perm[i]];
  std::vector<std::vector<int32_t>> rows(Hl.ncolours);
  for (int64_t i = 0; i < n; ++i) rows[col[i]].push_back((int32_t)i);
  for (int c = 0; c < Hl.ncolours; ++c) {
    Csr M;
    M.nrows = (int64_t)rows[c].size();
    M.ncols = n;
    M.rp.assign(M.nrows + 1, 0);
    for (int64_t r = 0; r < M.nrows; ++r) {
      const int32_t i = rows[c][r];
      for (int32_t k = Hd.A.rp[i]; k < Hd.A.rp[i + 1]; ++k) {
        const int32_t j = Hd.A.ci[k];
        if (j == i || col[j] == c) continue;
        M.ci.push_back(j);
        M.v.push_back(Hd.A.v[k]);
      }
      M.rp[r + 1] = (int32_t)M.ci.size();
    }
    D.gs.push_back(tuned_sell<T>(M, mem, sigma, rule_below, nullptr));
    D.gs_rows.push_back(mem.upload(rows[c]));
  }
}

// Everything after the operators are known: diagonals, patch inverses, eigenvalues,
// coarsest inverse, then (unless host_only) the device upload and the solve graph.
// lambda_max of D^{-1/2} A D^{-1/2}, and of its restriction to the rows and columns keep
// marks, by Lanczos on the device. The scaled operator (all rows, entries s_i a_ij s_j in CSR
// order) is built once per level and uploaded as a SELL-32 FP64 matrix; both runs use it. The
// restricted run starts from a vector that is zero outside keep and zeroes w outside keep in
// every update, so its SpMV adds only exact zeros for the dropped columns and it computes the
// same numbers as a run on the restricted operator. Every step is an SpMV and two fixed-order
// reductions; the host solves the tridiagonal Ritz problem. Same start vector and stopping
// rule as lanczos_lmax (residual |beta s_last| <= tol theta).
struct DeviceLanczos {
  int64_t n = 0;
  std::vector<double> sc;   // s_i = a_ii^{-1/2}
  DevMem mem;
  SellMat<double> M;
  cudaStream_t s = nullptr;

  DeviceLanczos(const Csr& A, cudaStream_t stream) : n(A.nrows), s(stream) {
    sc = lanczos_scaling(A, nullptr);
    Csr S;
    S.nrows = S.ncols = n;
    S.rp = A.rp;
    S.ci = A.ci;
    S.v.resize(A.v.size());
    parallel_for(n, [&](int64_t lo, int64_t hi) {
      for (int64_t i = lo; i < hi; ++i)
        for (int32_t k = A.rp[i]; k < A.rp[i + 1]; ++k) S.v[k] = sc[i] * A.v[k] * sc[A.ci[k]];
    });
    mem.stream = s;
    M = make_sell<double>(S, mem, 1);
  }
  ~DeviceLanczos() { mem.release(); }

  // lambda_max of each of nv <= 2 runs (run r restricted to the rows keeps[r] marks, null: all),
  // advanced together through the same launches; iters[r] and the result theta[r] are those of
  // run r alone.
  void run(int nv, const uint8_t* const* keeps, double tol, int maxit, int* iters, double* theta) {
    // step k of run r leaves alpha_k in hist[r][2k] and beta_{k+1}^2 in hist[r][2k+1]; the host
    // reads them back every kLanczosBatch steps and replays each run's stopping rule step by
    // step, so every result (theta and the step count) is that of a loop which tested after
    // every step; the steps queued past a run's stopping point are discarded
    constexpr int kLanczosBatch = 16;
    DevMem run;
    run.stream = s;
    double* hh[2] = {nullptr, nullptr};
    struct Release {   // the runs' buffers also on an error path (stream-ordered frees)
      DevMem& m;
      double** h;
      ~Release() {
        m.release();
        if (h[0] || h[1]) cudaStreamSynchronize(m.stream);   // no copy into a staging buffer in flight
        for (int r = 0; r < 2; ++r)
          if (h[r]) pinned_release(h[r]);
      }
    } release{run, hh};
    double *v[2], *w[2], *vprev[2], *hist[2];
    const uint8_t* kd[2] = {nullptr, nullptr};
    int kmax[2] = {0, 0}, k[2] = {0, 0}, kall = 0;
    bool done[2] = {false, false};
    for (int r = 0; r < nv; ++r) {
      std::vector<double> sk = sc;
      int64_t nk = 0;
      for (int64_t i = 0; i < n; ++i) {
        if (keeps[r] && !keeps[r][i]) sk[i] = 0.0;
        nk += sk[i] != 0.0;
      }
      kmax[r] = (int)std::min<int64_t>(maxit, nk);
      kall = std::max(kall, kmax[r]);
      theta[r] = 0.0;
      if (iters) iters[r] = 0;
      done[r] = kmax[r] == 0;
      v[r] = run.upload(lanczos_start(sk));
      vprev[r] = run.alloc<double>(n);
      w[r] = run.alloc<double>(n);
      if (keeps[r]) kd[r] = run.upload(std::vector<uint8_t>(keeps[r], keeps[r] + n));
    }
    if (kall == 0) return;
    for (int r = 0; r < nv; ++r) {
      hist[r] = run.alloc<double>(2 * (size_t)kall);
      hh[r] = pinned_acquire(2 * (int64_t)kall);
    }
    // block partials of the reductions, per run (the SpMV's grid covers the 32-row slices)
    double* part = run.alloc<double>(2 * ((n + 31) / 32 * 32 / kBlock + 1));
    unsigned* ticket = run.alloc<unsigned>(1);
    std::vector<double> al[2], be[2];
    for (int r = 0; r < nv; ++r) be[r].assign(1, 0.0);
    int queued = 0;
    while (!(done[0] && (nv < 2 || done[1])) && queued < kall) {
      const int q1 = std::min(kall, queued + kLanczosBatch);
      for (int j = queued; j < q1; ++j) lanczos_step(M, nv, v, w, vprev, kd, hist, j, part, ticket, s);
      for (int r = 0; r < nv; ++r)
        CK(cudaMemcpyAsync(hh[r] + 2 * queued, hist[r] + 2 * queued, 2 * sizeof(double) * (q1 - queued),
                           cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (int r = 0; r < nv; ++r) {
        for (; !done[r] && k[r] < std::min(q1, kmax[r]); ++k[r]) {
          const double alpha = hh[r][2 * k[r]], beta = std::sqrt(hh[r][2 * k[r] + 1]);
          al[r].push_back(alpha);
          be[r].push_back(beta);
          double sl;
          tridiag_top(al[r], be[r], k[r] + 1, &theta[r], &sl);
          if (beta * sl <= tol * std::fabs(theta[r]) || beta <= 1e-14 * std::fabs(theta[r])) {
            ++k[r];
            done[r] = true;
            break;
          }
        }
        if (k[r] >= kmax[r]) done[r] = true;
      }
      queued = q1;
    }
    check_launch("device Lanczos");
    CK(cudaStreamSynchronize(s));
    if (iters)
      for (int r = 0; r < nv; ++r) iters[r] = k[r];
  }
};

// lambda_max (unadjusted and adjusted) of every smoothed level, on the host or the device.
void compute_eigenvalues(mg_hierarchy* h, bool on_device) {
  const mg_options_t& o = h->opt;
  PhaseTimer tm;
  for (int l = 0; l + 1 < h->L; ++l) {
    LevelH& lv = h->host[l];
    if (o.global_smoother == MG_GLOBAL_SGS) continue;   // SGS needs no spectral bounds
    if (o.lambda_override) {
      lv.lmax = o.lambda_override[l];
      if (!(lv.lmax > 0)) throw Error(MG_ERR_INVALID_ARG, "lambda_override must be positive");
    } else {
      // the unadjusted run and, with patches, the run restricted to the complement of the patch
      // DoFs (adjusted lambda, Sec. 5); on the device both advance through the same launches
      const bool adj = lv.patch_ptr.size() > 1;
      std::vector<uint8_t> keep;
      if (adj) {
        keep.assign(lv.A.nrows, 1);
        for (int32_t f : lv.patch_dofs) keep[f] = 0;
      }
      int it[2] = {0, 0};
      double th[2] = {0.0, 0.0};
      if (on_device) {
        DeviceLanczos dlz(lv.A, h->own_stream);
        const uint8_t* keeps[2] = {nullptr, adj ? keep.data() : nullptr};
        dlz.run(adj ? 2 : 1, keeps, o.eig_tol, o.eig_maxit, it, th);
      } else {
        th[0] = lanczos_lmax(lv.A, nullptr, o.eig_tol, o.eig_maxit, &it[0]);
        if (adj) th[1] = lanczos_lmax(lv.A, keep.data(), o.eig_tol, o.eig_maxit, &it[1]);
      }
      lv.lmax_unadj = th[0];
      lv.lmax_adj = adj ? th[1] : th[0];
      lv.lanczos_iters = it[0] + (adj ? it[1] : 0);
      lv.lmax = (o.adjusted_lambda ? lv.lmax_adj : lv.lmax_unadj) * o.lmax_safety;
      tm.mark(std::string(on_device ? "device" : "host") + " lanczos L" + std::to_string(l) + " (" +
              std::to_string(lv.lanczos_iters) + " it)");
    }
    lv.lmin = o.lmin_ratio * lv.lmax;
  }
}

void finish_setup_host(mg_hierarchy* h) {
  const mg_options_t& o = h->opt;
  const int L = h->L;
  for (int l = 0; l < L; ++l) {
    LevelH& lv = h->host[l];
    const int64_t n = lv.A.nrows;
    if (n == 0) throw Error(MG_ERR_INVALID_ARG, "level " + std::to_string(l) + " has no free DoFs");
    lv.dinv.resize(n);
    for (int64_t i = 0; i < n; ++i) {
      double dg = 0;
      for (int32_t k = lv.A.rp[i]; k < lv.A.rp[i + 1]; ++k)
        if (lv.A.ci[k] == i) dg = lv.A.v[k];
      if (!(dg > 0)) throw Error(MG_ERR_NOT_SPD, "level " + std::to_string(l) + ": non-positive diagonal at " + std::to_string(i));
      lv.dinv[i] = 1.0 / dg;
    }
  }
  if (o.global_smoother == MG_GLOBAL_SGS) {
    PhaseTimer tm;
    for (int l = 0; l + 1 < L; ++l) h->host[l].ncolours = greedy_colouring(h->host[l].A, h->host[l].colour);
    tm.mark("colouring");
  }
  const int64_t ncoarse = h->host[L - 1].A.nrows;
  if (ncoarse > 20000) throw Error(MG_ERR_INVALID_ARG, "coarsest level too large for the dense direct solve (> 20000 DoFs)");
  // eigenvalues (Sec. 3.2 / Sec. 5): on the host only for host-only hierarchies; otherwise
  // the device phase computes them on the GPU before the smoother coefficients are set
  if (o.host_only) compute_eigenvalues(h, false);
}

// Device phase of set-up: upload, batched dense inverses, autotuned layouts. All work is
// ordered on the hierarchy's own stream, which is synchronised before returning.
void build_device(mg_hierarchy* h) {
  const mg_options_t& o = h->opt;
  const int L = h->L;
  tma_prepare();
  PhaseTimer tm;
  const int64_t ncoarse = h->host[L - 1].A.nrows;

  // ---- device upload ----
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0) throw Error(MG_ERR_NO_DEVICE, "no CUDA device");
  if (!h->own_stream) CK(cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking));
  h->device = true;
  DevMem& mem = h->mem;
  mem.stream = h->own_stream;
  compute_eigenvalues(h, true);
  // Internal DoF order of each level (option reorder; the coarsest level keeps the library
  // numbering). The device holds the symmetrically permuted operators; vectors are
  // gathered/scattered at every boundary. Where a SELL slice (CSR row) spans < 2^16
  // columns its indices are stored as 16-bit offsets from a base.
  std::vector<std::vector<int32_t>> perm(L), iperm(L);
  std::vector<LevelH> dl(L);
  for (int l = 0; l < L; ++l) {
    if (l + 1 == L) continue;
    const LevelH& H = h->host[l];
    if (o.reorder == MG_REORDER_RCM) perm[l] = rcm_order(H.A);
    else if ((o.reorder == MG_REORDER_SPATIAL || (o.reorder == MG_REORDER_SPATIAL_COARSE && l > 0)) &&
             !H.dof_points.empty())
      perm[l] = morton_order(H.dof_points, H.dim);
    if (!perm[l].empty()) iperm[l] = inverse_perm(perm[l]);
  }
  for (int l = 0; l < L; ++l) {
    const LevelH& H = h->host[l];
    LevelH& D = dl[l];
    D.A = perm[l].empty() ? H.A : permute_csr(H.A, perm[l], iperm[l]);
    if (l + 1 < L) {
      D.P = (perm[l].empty() && iperm[l + 1].empty()) ? H.P : permute_csr(H.P, perm[l], iperm[l + 1]);
      D.R = transpose(D.P);
    }
    D.dinv.resize(H.dinv.size());
    for (size_t i = 0; i < H.dinv.size(); ++i) D.dinv[i] = H.dinv[perm[l].empty() ? i : perm[l][i]];
    D.patch_ptr = H.patch_ptr;
    D.patch_dofs = H.patch_dofs;
    if (!iperm[l].empty())
      for (int32_t& f : D.patch_dofs) f = iperm[l][f];
    D.lmax = H.lmax;
    D.lmin = H.lmin;
  }
  tm.mark("reorder");
  int max_patch = 0;
  // All dense blocks (every patch matrix A[B_d, B_d] of every level and the coarsest A)
  // are inverted together on the device by the batched Gauss-Jordan sweep.
  struct Blk {
    int level, patch;
    int32_t n;
  };
  std::vector<Blk> blks;
  for (int l = 0; l + 1 < L; ++l) {
    const LevelH& lv = h->host[l];
    for (int64_t p = 0; p + 1 < (int64_t)lv.patch_ptr.size(); ++p)
      blks.push_back({l, (int)p, lv.patch_ptr[p + 1] - lv.patch_ptr[p]});
  }
  blks.push_back({L - 1, -1, (int32_t)ncoarse});
  std::vector<int> order(blks.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return blks[a].n > blks[b].n; });
  GjBatch gj;
  std::vector<double> anorm;   // ||A_block||_1 by block id
  gj.nmat = (int)blks.size();
  std::vector<int64_t> boff(blks.size()), bvoff(blks.size());  // by block id
  std::vector<int64_t> soff, svoff;                              // by sorted position
  int64_t mtot = 0, vtot = 0;
  for (int id : order) {
    boff[id] = mtot;
    bvoff[id] = vtot;
    gj.hn.push_back(blks[id].n);
    soff.push_back(mtot);
    svoff.push_back(vtot);
    mtot += (int64_t)blks[id].n * blks[id].n;
    vtot += blks[id].n;
  }
  gj.max_n = gj.hn.empty() ? 0 : gj.hn[0];
  {
    std::vector<double> Mh(mtot), d0(vtot);
    anorm.assign(blks.size(), 0.0);
    parallel_for((int64_t)blks.size(), [&](int64_t lo, int64_t hi) {
      for (int64_t id = lo; id < hi; ++id) {
        const Blk& bk = blks[id];
        const LevelH& lv = h->host[bk.level];
        std::vector<int32_t> all;
        const int32_t* idx;
        if (bk.patch >= 0) {
          idx = &lv.patch_dofs[lv.patch_ptr[bk.patch]];
        } else {
          all.resize(bk.n);
          for (int32_t i = 0; i < bk.n; ++i) all[i] = i;
          idx = all.data();
        }
        std::vector<double> D = dense_submatrix(lv.A, idx, bk.n);
        std::copy(D.begin(), D.end(), Mh.begin() + boff[id]);
        for (int32_t i = 0; i < bk.n; ++i) d0[bvoff[id] + i] = D[(int64_t)i * bk.n + i];
        double nrm = 0.0;   // ||A[B,B]||_1 (symmetric: the largest row sum of |a_ij|)
        for (int32_t i = 0; i < bk.n; ++i) {
          double rs = 0.0;
          for (int32_t j = 0; j < bk.n; ++j) rs += std::fabs(D[(int64_t)i * bk.n + j]);
          nrm = std::max(nrm, rs);
        }
        anorm[id] = nrm;
      }
    });
    gj.M = mem.upload(Mh);
    gj.diag0 = mem.upload(d0);
  }
  gj.n = mem.upload(gj.hn);
  gj.off = mem.upload(soff);
  gj.voff = mem.upload(svoff);
  gj.rowk = mem.alloc<double>(vtot);
  gj.colk = mem.alloc<double>(vtot);
  gj.rowk2 = mem.alloc<double>(vtot);
  gj.colk2 = mem.alloc<double>(vtot);
  gj.piv = mem.alloc<double>(2 * (size_t)gj.nmat);
  gj.pdrop = mem.alloc<int32_t>(2 * (size_t)gj.nmat);
  gj.bad = mem.alloc<int32_t>(gj.nmat);
  gj.ndrop = mem.alloc<int32_t>(gj.nmat);
  if (tm.on) {
    CK(cudaStreamSynchronize(mem.stream));
    tm.mark("dense blocks (host + upload)");
  }
  batched_spsd_inverse(gj, mem.stream);
  check_launch("batched dense inverse");
  {
    std::vector<int32_t> bad(gj.nmat), nd(gj.nmat);
    CK(cudaMemcpyAsync(bad.data(), gj.bad, sizeof(int32_t) * gj.nmat, cudaMemcpyDeviceToHost, mem.stream));
    CK(cudaMemcpyAsync(nd.data(), gj.ndrop, sizeof(int32_t) * gj.nmat, cudaMemcpyDeviceToHost, mem.stream));
    CK(cudaStreamSynchronize(mem.stream));
    for (int sp = 0; sp < gj.nmat; ++sp) {
      const Blk& bk = blks[order[sp]];
      if (bad[sp])
        throw Error(MG_ERR_NOT_SPD, bk.patch >= 0 ? "level " + std::to_string(bk.level) + ": patch " +
                                                        std::to_string(bk.patch) + " is not positive semi-definite"
                                                  : std::string("coarsest operator is not positive semi-definite"));
      h->dropped_dofs += nd[sp];
    }
  }
  tm.mark("batched inverse (" + std::to_string(gj.nmat) + " blocks, max n " + std::to_string(gj.max_n) + ")");
  std::vector<std::vector<int64_t>> level_inv_off(L);
  for (size_t id = 0; id < blks.size(); ++id)
    if (blks[id].patch >= 0) level_inv_off[blks[id].level].push_back(boff[id]);
  const double* coarse_inv = gj.M + boff[blks.size() - 1];
  // Mixed precision: patches with kappa_1 = ||A_BB||_1 ||A_BB^-1||_1 <= fp32_patch_kappa apply an
  // FP32 copy of their inverse (an FP32 arena); the others, and the coarsest block, stay FP64.
  std::vector<std::vector<int32_t>> level_fp32(L);
  std::vector<std::vector<int64_t>> level_inv32_off(L);
  float* inv32 = nullptr;
  if (h->mixed() && o.fp32_patch_kappa > 0 && blks.size() > 1) {
    double* dn = mem.alloc<double>(gj.nmat);
    batched_norm1(gj, dn, mem.stream);
    std::vector<double> xn(gj.nmat);
    CK(cudaMemcpyAsync(xn.data(), dn, sizeof(double) * gj.nmat, cudaMemcpyDeviceToHost, mem.stream));
    CK(cudaStreamSynchronize(mem.stream));
    int64_t tot32 = 0;
    std::vector<int64_t> off32(blks.size(), -1);
    for (int sp = 0; sp < gj.nmat; ++sp) {
      const int id = order[sp];
      if (blks[id].patch < 0) continue;
      const double kappa = anorm[id] * xn[sp];
      if (kappa <= (double)o.fp32_patch_kappa && std::isfinite(kappa)) {
        off32[id] = tot32;
        tot32 += (int64_t)blks[id].n * blks[id].n;
      }
    }
    if (tot32 > 0) inv32 = mem.alloc<float>(tot32);
    for (size_t id = 0; id < blks.size(); ++id) {
      if (blks[id].patch < 0) continue;
      const int l = blks[id].level;
      level_fp32[l].push_back(off32[id] >= 0 ? 1 : 0);
      level_inv32_off[l].push_back(off32[id]);
      if (off32[id] >= 0)
        convert<double, float>(blks[id].n * blks[id].n, gj.M + boff[id], inv32 + off32[id], mem.stream);
    }
    check_launch("FP32 patch inverses");
  } else {
    for (size_t id = 0; id < blks.size(); ++id)
      if (blks[id].patch >= 0) {
        level_fp32[blks[id].level].push_back(0);
        level_inv32_off[blks[id].level].push_back(-1);
      }
  }
  auto upload_engine = [&](auto* eng, auto tag) {
    using T = decltype(tag);
    eng->cheb_k = o.cheb_degree;
    eng->nu = o.nu;
    eng->order = o.smoother;
    eng->local_mask = (uint32_t)o.local_levels_mask;
    eng->sgs = o.global_smoother == MG_GLOBAL_SGS;
    eng->lv.resize(L);
    for (int l = 0; l < L; ++l) {
      LevelH& H = dl[l];
      DevLevel<T>& D = eng->lv[l];
      if (!perm[l].empty()) D.perm = mem.upload(perm[l]);
      D.n = (int)H.A.nrows;
      std::string tlog;
      D.A = tuned_sell<T>(H.A, mem, o.sell_sigma, o.tune_min_nnz, &tlog, true);
      h->uses_tma |= D.A.tma != 0;
      if (l < L - 1) {
        D.P = tuned_sell<T>(H.P, mem, o.sell_sigma, o.tune_min_nnz, &tlog);
        D.R = tuned_sell<T>(H.R, mem, o.sell_sigma, o.tune_min_nnz, &tlog);
        std::vector<T> dv(H.dinv.begin(), H.dinv.end());
        D.dinv = mem.upload(dv);
        if (!eng->sgs) cheb_coefficients(H.lmax, H.lmin, o.cheb_degree, D.cd, D.cr);
        else build_sgs_ops(h->host[l], H, perm[l], D, mem, o.sell_sigma, o.tune_min_nnz);
        D.xt = mem.alloc<T>(D.n);
        D.d = mem.alloc<T>(D.n);
        D.res = mem.alloc<T>(D.n);
        // patches
        D.np = (int)H.patch_ptr.size() - 1;
        if (D.np > 0) {
          D.nt = (int)H.patch_dofs.size();
          D.pdofs = mem.upload(H.patch_dofs);
          // patch rows of A, ELL: pw entries per row, padded with value 0 at the row's own DoF
          int pw = 1;
          for (int t = 0; t < D.nt; ++t) {
            const int32_t r = H.patch_dofs[t];
            pw = std::max(pw, H.A.rp[r + 1] - H.A.rp[r]);
          }
          D.pw = pw;
          std::vector<int32_t> pci((size_t)D.nt * pw), plen(D.nt);
          std::vector<double> pv((size_t)D.nt * pw, 0.0);
          for (int t = 0; t < D.nt; ++t) {
            const int32_t r = H.patch_dofs[t];
            const int64_t o = (int64_t)t * pw;
            int j = 0;
            for (int32_t k = H.A.rp[r]; k < H.A.rp[r + 1]; ++k, ++j) pci[o + j] = H.A.ci[k], pv[o + j] = H.A.v[k];
            plen[t] = j;
            for (; j < pw; ++j) pci[o + j] = r;
          }
          D.plen = mem.upload(plen);
          // work list: the patches' row blocks, largest patches first
          std::vector<int> porder(D.np);
          for (int p = 0; p < D.np; ++p) porder[p] = p;
          std::stable_sort(porder.begin(), porder.end(), [&](int a, int b) {
            return H.patch_ptr[a + 1] - H.patch_ptr[a] > H.patch_ptr[b + 1] - H.patch_ptr[b];
          });
          std::vector<PatchItem> items;
          D.pfp32 = level_fp32[l];
          for (int p : porder) {
            const int32_t p0 = H.patch_ptr[p], m = H.patch_ptr[p + 1] - p0;
            D.max_patch = std::max(D.max_patch, m);
            const bool f32 = std::is_same<T, float>::value && level_fp32[l][p];
            const int64_t off = f32 ? level_inv32_off[l][p] : level_inv_off[l][p];
            // small patches: warp-per-row items (8 rows); larger: lane-per-row items (32 rows)
            const bool small = m <= kSmallPatch;
            const int mode = (f32 ? PI_FP32 : 0) | (small ? PI_WARP_ROWS : 0);
            const int step = small ? kPatchRowsPerWarpItem : kPatchRowsPerItem;
            for (int r0 = 0; r0 < m; r0 += step) items.push_back({p0, m, r0, mode, off});
          }
          if (D.max_patch > kMaxPatchDofs)
            throw Error(MG_ERR_INVALID_ARG, "patch larger than " + std::to_string(kMaxPatchDofs) + " DoFs");
          max_patch = std::max(max_patch, D.max_patch);
          D.nitems = (int)items.size();
          D.pci = mem.upload(pci);
          D.pv = mem.upload(pv);
          D.inv = gj.M;
          D.inv32 = inv32;
          D.rbuf = mem.alloc<double>(D.nt);
          D.items = mem.upload(items);
          // rows of A with an entry in a patch column (A is symmetric: patch DoFs and neighbours)
          std::vector<uint8_t> inpatch(D.n, 0), halo(D.n, 0);
          for (int32_t f : H.patch_dofs) inpatch[f] = 1;
          for (int64_t i = 0; i < D.n; ++i)
            for (int32_t k = H.A.rp[i]; k < H.A.rp[i + 1]; ++k)
              if (inpatch[H.A.ci[k]]) {
                halo[i] = 1;
                break;
              }
          // rows (A P)_{i,:} of the patch rows (columns sorted), ELL padded with (0, 0.0)
          {
            std::vector<std::vector<std::pair<int32_t, double>>> ap(D.nt);
            std::vector<double> acc(H.P.ncols, 0.0);
            std::vector<uint8_t> hit(H.P.ncols, 0);
            std::vector<int32_t> cols;
            int apw = 1;
            for (int t = 0; t < D.nt; ++t) {
              const int32_t i = H.patch_dofs[t];
              cols.clear();
              for (int32_t k = H.A.rp[i]; k < H.A.rp[i + 1]; ++k) {
                const int32_t j = H.A.ci[k];
                for (int32_t m = H.P.rp[j]; m < H.P.rp[j + 1]; ++m) {
                  const int32_t c = H.P.ci[m];
                  if (!hit[c]) hit[c] = 1, cols.push_back(c);
                  acc[c] += H.A.v[k] * H.P.v[m];
                }
              }
              std::sort(cols.begin(), cols.end());
              for (int32_t c : cols) ap[t].push_back({c, acc[c]}), acc[c] = 0.0, hit[c] = 0;
              apw = std::max(apw, (int)cols.size());
            }
            std::vector<int32_t> apci((size_t)D.nt * apw, 0), aplen(D.nt);
            std::vector<double> apv((size_t)D.nt * apw, 0.0);
            for (int t = 0; t < D.nt; ++t) {
              aplen[t] = (int32_t)ap[t].size();
              for (size_t k = 0; k < ap[t].size(); ++k)
                apci[(size_t)t * apw + k] = ap[t][k].first, apv[(size_t)t * apw + k] = ap[t][k].second;
            }
            D.apw = apw;
            D.apci = mem.upload(apci);
            D.aplen = mem.upload(aplen);
            D.apv = mem.upload(apv);
          }
          std::vector<int32_t> hrow, hrp(1, 0), hci;
          std::vector<T> hv;
          for (int64_t i = 0; i < D.n; ++i)
            if (halo[i]) {
              hrow.push_back((int32_t)i);
              for (int32_t k = H.A.rp[i]; k < H.A.rp[i + 1]; ++k) hci.push_back(H.A.ci[k]), hv.push_back((T)H.A.v[k]);
              hrp.push_back((int32_t)hci.size());
            }
          D.nh = (int)hrow.size();
          D.hrow = mem.upload(hrow);
          D.hrp = mem.upload(hrp);
          D.hci = mem.upload(hci);
          D.hv = mem.upload(hv);
        }
      }
      auto lay = [](const SellMat<T>& M) {
        return layout_name({M.lanes, M.sigma, M.unroll, M.sub, M.pf}) +
               (M.col16 ? (M.col ? "/16+32" : "/16") : "/32");
      };
      tm.mark("upload L" + std::to_string(l) + " A/P/R " + lay(D.A) + "/" + lay(D.P) + "/" + lay(D.R) + " |" + tlog);
      bool fine_shared = (l == 0) && std::is_same<T, double>::value;
      if (!fine_shared) {
        D.b = mem.alloc<T>(D.n);
        D.x = mem.alloc<T>(D.n);
      }
    }
    eng->nc = (int)ncoarse;
    eng->kchunk = 256;
    int rowblocks = (eng->nc + kBlock - 1) / kBlock;
    int want_chunks = std::max(1, (8 * 152 + rowblocks - 1) / rowblocks);  // about 8 blocks per SM
    eng->kchunk = std::max(32, std::min(1024, ((eng->nc + want_chunks - 1) / want_chunks + 31) / 32 * 32));
    eng->Xc = const_cast<double*>(coarse_inv);
    eng->cpart = mem.alloc<double>((size_t)dense_chunks(eng->nc, eng->kchunk) * eng->nc);
  };
  h->n0 = (int)h->host[0].A.nrows;
  const int n0 = h->n0;
  h->cb = mem.alloc<double>(n0);
  h->cx = mem.alloc<double>(n0);
  h->cr = mem.alloc<double>(n0);
  h->cp = mem.alloc<double>(n0);
  h->cq = mem.alloc<double>(n0);
  h->cz = mem.alloc<double>(n0);
  h->nparts = cg_parts(n0);
  h->ap_parts = sell_blocks(n0, 32);  // at least the block partials of k_ap for any layout
  h->part = mem.alloc<double>(std::max(h->nparts, h->ap_parts));
  h->ticket = mem.alloc<unsigned>(1);
  h->st = mem.alloc<CgState>(1);
  h->hst = reinterpret_cast<CgState*>(pinned_acquire((sizeof(CgState) + 7) / 8));
  std::memset(h->hst, 0, sizeof(CgState));
  if (h->mixed()) {
    h->e32.reset(new Engine<float>());
    upload_engine(h->e32.get(), float());
    std::string tlog;
    h->A0 = tuned_sell<double>(dl[0].A, mem, o.sell_sigma, o.tune_min_nnz, &tlog);
  } else {
    h->e64.reset(new Engine<double>());
    upload_engine(h->e64.get(), double());
    h->e64->lv[0].b = h->cr;  // the V-cycle of CG reads r and writes z in place
    h->e64->lv[0].x = h->cz;
    h->A0 = h->e64->lv[0].A;
  }
  {
    h->perm0 = h->e64 ? h->e64->lv[0].perm : h->e32->lv[0].perm;
  }
  // the small levels in one persistent launch per cycle (after the level-0 vectors are final)
  h->with_engine([&](auto& e) { e.build_persistent(dl, level_inv_off, o.small_level_dofs, mem); });
  if (max_patch > 0) patch_solve_setup(max_patch);
  CK(cudaStreamSynchronize(h->own_stream));
  tm.mark("device upload");
}

}  // namespace
}  // namespace nnmg

// ---- CG orchestration -------------------------------------------------------------------

namespace nnmg {
namespace {

template <typename T>
struct CgRunner {
  mg_hierarchy* h;
  Engine<T>& e;
  T* vb() { return e.lv[0].b; }
  T* vx() { return e.lv[0].x; }
  int launches = 0;

  Reduce red(int op, int use_cond = 0, unsigned long long cond = 0) {
    return Reduce{h->part, h->ticket, h->st, op, use_cond, cond};
  }
  void tail(cudaStream_t s, int use_cond, unsigned long long cond) {
    sell_ap(h->A0, h->cp, h->cq, red(FIN_PQ), s);
    cg_update<T>(h->n0, h->st, h->cp, h->cq, h->cx, h->cr, vb(), vx(), red(FIN_RR, use_cond, cond), s);
    launches += 2;
  }
  void head(cudaStream_t s, int use_cond, unsigned long long cond) {
    CK(cudaMemsetAsync(h->ticket, 0, sizeof(unsigned), s));
    cg_init<T>(h->n0, h->cb, h->cr, h->cx, vb(), vx(), red(FIN_BB), s);
    e.launches = 0;
    e.cycle(0, s);
    cg_dotz<T>(h->n0, h->cr, vx(), h->cp, true, red(FIN_RZ0), s);
    launches += 3 + e.launches;
    tail(s, use_cond, cond);
  }
  void body(cudaStream_t s, int use_cond, unsigned long long cond) {
    e.launches = 0;
    e.cycle(0, s);
    cg_dotz<T>(h->n0, h->cr, vx(), h->cp, false, red(FIN_RZ), s);
    cg_pupdate<T>(h->n0, h->st, vx(), h->cp, s);
    launches = 2 + e.launches;
    tail(s, use_cond, cond);
  }
};

template <typename F>
void dispatch(mg_hierarchy* h, F&& f) {
  if (h->e64) {
    CgRunner<double> r{h, *h->e64};
    f(r);
  } else {
    CgRunner<float> r{h, *h->e32};
    f(r);
  }
}

void build_graph(mg_hierarchy* h) {
  cudaStream_t s = h->own_stream;
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle handle;
  CK(cudaGraphConditionalHandleCreate(&handle, g, 1, cudaGraphCondAssignDefault));
  CK(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  dispatch(h, [&](auto& r) { r.head(s, 1, (unsigned long long)handle); });
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &deps, nullptr, &ndeps));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  CK(cudaGraphAddNode(&cnode, g, deps, nullptr, ndeps, &cp));
  cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
  CK(cudaStreamUpdateCaptureDependencies(s, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
  CK(cudaStreamEndCapture(s, &g));
  CK(cudaStreamBeginCaptureToGraph(s, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  dispatch(h, [&](auto& r) { r.body(s, 1, (unsigned long long)handle); });
  CK(cudaStreamEndCapture(s, &bodyg));
  CK(cudaGraphInstantiate(&h->graph, g, 0));
  CK(cudaGraphDestroy(g));
}

void count_launches(mg_hierarchy* h) {
  // a dry pass through the schedule on a capture stream counts launches without running
  dispatch(h, [&](auto& r) {
    cudaStream_t s = h->own_stream;
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    r.e.launches = 0;
    r.e.cycle(0, s);
    h->launches_vcycle = r.e.launches;
    r.body(s, 0, 0);
    h->launches_iter = r.launches;
    CK(cudaStreamEndCapture(s, &g));
    CK(cudaGraphDestroy(g));
  });
}

void enqueue_state(mg_hierarchy* h, double rtol, int maxit, cudaStream_t s) {
  if (!(rtol >= 0) || maxit < 1) throw Error(MG_ERR_INVALID_ARG, "rtol must be >= 0 and maxit >= 1");
  std::memset(h->hst, 0, sizeof(CgState));
  h->hst->rtol2 = rtol * rtol;
  h->hst->maxit = maxit;
  CK(cudaMemcpyAsync(h->st, h->hst, sizeof(CgState), cudaMemcpyHostToDevice, s));
}

// The FP64 residual b - A x of the final iterate, then the whole CG state to the host.
void enqueue_exit(mg_hierarchy* h, cudaStream_t s) {
  sell_resid<double>(h->A0, h->cx, h->cb, h->cq, s);
  dot_self(h->n0, h->cq, Reduce{h->part, h->ticket, h->st, FIN_TRUE, 0, 0}, s);
  CK(cudaMemcpyAsync(h->hst, h->st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
}

int collect_state(const mg_hierarchy* h, mg_solve_info_t* info) {
  const CgState st = *h->hst;
  if (info) {
    info->iterations = st.it;
    info->converged = st.status == 1 || st.bb == 0.0;
    info->rel_residual = st.bb > 0 ? std::sqrt(st.rr / st.bb) : 0.0;
    info->true_rel_residual = st.bb > 0 ? std::sqrt(st.rr_true / st.bb) : 0.0;
  }
  if (st.status == 3) return MG_ERR_BREAKDOWN;
  if (!(st.status == 1 || st.bb == 0.0)) return MG_ERR_NO_CONVERGENCE;
  return MG_OK;
}

// ---- MG-PCG of one or many hierarchies in one persistent launch ----
// The program: per problem the CG steps of CgRunner as tasks and the recorded V-cycle; the
// problems' phases are merged by index (phase k runs the k-th step of every problem), so one
// grid barrier serves every problem's step. The body repeats until every problem has
// stopped; a stopped problem's tasks do nothing (gated on its CG state). Each problem's
// arithmetic does not depend on the others (every unit computes the same values whichever
// warp runs it, and reductions sum per-unit partials in unit order), so a problem gives the
// same bits alone and in any batch.
struct PProgram {
  std::vector<PTask> tasks;
  std::vector<PPhase> phases;
  void phase(const std::vector<PTask>& ts, int check = 0) {
    PPhase ph{(int)tasks.size(), (int)tasks.size(), 0, check};
    for (PTask t : ts) {
      if (t.n <= 0) continue;
      t.u0 = ph.units;
      ph.units += ptask_units(t);
      tasks.push_back(t);
    }
    ph.t1 = (int)tasks.size();
    if (ph.units > 0 || check) phases.push_back(ph);
  }
};

template <typename T>
Engine<T>& engine_of(mg_hierarchy* h);
template <>
Engine<double>& engine_of<double>(mg_hierarchy* h) {
  return *h->e64;
}
template <>
Engine<float>& engine_of<float>(mg_hierarchy* h) {
  return *h->e32;
}

bool persistent_solve_ok(const mg_hierarchy* h) {
  return h->device && (h->e64 ? h->e64->pers_from == 0 : (h->e32 && h->e32->pers_from == 0));
}

// Records the program of the problems hs (same precision T, whole cycle persistent) into pg;
// part[i]: a partial-sum buffer of problem i with at least ceil(n_0 / 8) entries.
template <typename T>
void assemble_pcg(const std::vector<mg_hierarchy*>& hs, const std::vector<double*>& part, PProgram& pg, int* nhead) {
  const int K = (int)hs.size();
  auto base = [](int kind, int n) {
    PTask t;
    std::memset(&t, 0, sizeof(t));
    t.kind = kind;
    t.n = n;
    t.G = 4;
    return t;
  };
  auto units32 = [](int n) { return (n + 31) / 32; };
  auto per = [&](auto&& make) {
    std::vector<PTask> v;
    for (int i = 0; i < K; ++i) v.push_back(make(i, hs[i], engine_of<T>(hs[i])));
    return v;
  };
  auto fin = [&](int op, bool ap, bool gated) {
    return per([&, op, ap, gated](int i, mg_hierarchy* h, Engine<T>& e) {
      PTask t = base(PK_FINISH, 1);
      t.w = ap ? (h->n0 + 32 / e.a0G - 1) / (32 / e.a0G) : units32(h->n0);
      t.part = part[i];
      t.st = h->st;
      t.op = op;
      t.gate = gated ? h->st : nullptr;
      return t;
    });
  };
  auto vcycle = [&]() {
    size_t len = 0;
    for (mg_hierarchy* h : hs) len = std::max(len, engine_of<T>(h).hphases.size());
    for (size_t k = 0; k < len; ++k) {
      std::vector<PTask> ts;
      for (mg_hierarchy* h : hs) {
        Engine<T>& e = engine_of<T>(h);
        if (k >= e.hphases.size()) continue;
        for (int j = e.hphases[k].t0; j < e.hphases[k].t1; ++j) {
          PTask t = e.htasks[j];
          t.gate = h->st;
          ts.push_back(t);
        }
      }
      pg.phase(ts);
    }
  };
  auto vec = [&](int kind, bool gated, int first = 0) {
    return per([&, kind, gated, first](int i, mg_hierarchy* h, Engine<T>& e) {
      PTask t = base(kind, h->n0);
      t.cb = h->cb;
      t.cx = h->cx;
      t.cr = h->cr;
      t.cp = h->cp;
      t.cq = h->cq;
      t.vb = e.lv[0].b;
      t.vx = e.lv[0].x;
      t.st = h->st;
      t.part = part[i];
      t.w = first;
      t.gate = gated ? h->st : nullptr;
      return t;
    });
  };
  // head: r = b, x = 0; z = V r; p = z
  pg.phase(vec(PK_CG_INIT, false));
  pg.phase(fin(FIN_BB, false, false));
  vcycle();
  pg.phase(vec(PK_CG_DOTZ, true, 1));
  pg.phase(fin(FIN_RZ0, false, true));
  *nhead = (int)pg.phases.size();
  // body: q = A p, alpha; x, r updated, convergence (check); z = V r; beta; p = z + beta p
  pg.phase(per([&](int i, mg_hierarchy* h, Engine<T>& e) {
    PTask t = base(PK_CG_AP, h->n0);
    t.rp = e.a0rp;
    t.ci = e.a0ci;
    t.val = e.a0v;
    t.G = e.a0G;
    t.cp = h->cp;
    t.cq = h->cq;
    t.part = part[i];
    t.gate = h->st;
    return t;
  }));
  pg.phase(fin(FIN_PQ, true, true));
  pg.phase(vec(PK_CG_UPDATE, true));
  pg.phase(fin(FIN_RR, false, true), 1);
  vcycle();
  pg.phase(vec(PK_CG_DOTZ, true));
  pg.phase(fin(FIN_RZ, false, true));
  pg.phase(vec(PK_CG_PUPDATE, true));
}

// The program of one hierarchy, kept with it (device memory of the hierarchy).
// Partial sums of one problem's reductions: one per unit of its largest reduction task.
int64_t pcg_part_size(mg_hierarchy* h) {
  const int G = h->e64 ? h->e64->a0G : h->e32->a0G;
  return std::max<int64_t>((h->n0 + 31) / 32, ((int64_t)h->n0 * G + 31) / 32) + 1;
}

template <typename T>
void build_solo(mg_hierarchy* h) {
  std::vector<mg_hierarchy*> hs{h};
  std::vector<double*> part{h->mem.alloc<double>(pcg_part_size(h))};
  PProgram pg;
  int nhead = 0;
  assemble_pcg<T>(hs, part, pg, &nhead);
  h->solo.tasks = h->mem.upload(pg.tasks);
  h->solo.phases = h->mem.upload(pg.phases);
  std::vector<CgState*> st{h->st};
  h->solo.states = h->mem.upload(st);
  h->solo.bar = h->mem.alloc<PBarrier>(1);
  h->solo.nhead = nhead;
  h->solo.nbody = (int)pg.phases.size() - nhead;
}

int pcg_iteration_cap(int maxit) { return std::min(maxit, 100000) + 1; }

// The solve itself on s (state already enqueued): the persistent program, or the graph.
void enqueue_solo_or_graph(mg_hierarchy* h, int maxit, cudaStream_t s) {
  if (h->solo.tasks) {
    auto go = [&](auto tag) {
      using T = decltype(tag);
      CK(persistent_launch<T>(h->solo.phases, h->solo.nhead, h->solo.tasks, h->solo.bar, s, h->solo.nbody,
                              h->solo.states, 1, pcg_iteration_cap(maxit)));
    };
    if (h->e64) go(double());
    else go(float());
  } else {
    CK(cudaGraphLaunch(h->graph, s));
  }
}

int run_solve(mg_hierarchy* h, double rtol, int maxit, mg_solve_info_t* info, cudaStream_t s) {
  enqueue_state(h, rtol, maxit, s);
  if (h->solo.tasks) {
    enqueue_solo_or_graph(h, maxit, s);
  } else if (h->graph) {
    CK(cudaGraphLaunch(h->graph, s));
  } else {
    dispatch(h, [&](auto& r) { r.head(s, 0, 0); });
    check_launch("cg head");
    for (;;) {
      CK(cudaMemcpyAsync(h->hst, h->st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (!h->hst->cont) break;
      dispatch(h, [&](auto& r) { r.body(s, 0, 0); });
      check_launch("cg body");
    }
  }
  enqueue_exit(h, s);
  CK(cudaStreamSynchronize(s));
  return collect_state(h, info);
}

}  // namespace
}  // namespace nnmg

// ---- C ABI ------------------------------------------------------------------------------

#define API_BEGIN try {
#define API_END_H(h)                     \
  }                                      \
  catch (const nnmg::Error& e) {         \
    if (h) (h)->err = e.what();          \
    else nnmg::g_setup_error = e.what(); \
    return e.code;                       \
  }                                      \
  catch (const std::bad_alloc&) {        \
    if (h) (h)->err = "out of host memory"; \
    else nnmg::g_setup_error = "out of host memory"; \
    return MG_ERR_OOM;                   \
  }                                      \
  catch (const std::exception& e) {      \
    if (h) (h)->err = e.what();          \
    else nnmg::g_setup_error = e.what(); \
    return MG_ERR_INVALID_ARG;           \
  }

namespace {

mg_hierarchy* checked(mg_hierarchy* h, bool need_device = true) {
  if (!h) throw Error(MG_ERR_INVALID_ARG, "null hierarchy");
  if (need_device && !h->device) throw Error(MG_ERR_NO_DEVICE, "hierarchy was built with host_only = 1");
  return h;
}
void check_level(const mg_hierarchy* h, int l, bool below_coarsest = false) {
  if (l < 0 || l >= h->L || (below_coarsest && l >= h->L - 1))
    throw Error(MG_ERR_INVALID_ARG, "level index out of range");
}

// After the work enqueued on s, the bounded device-side waits of that work (synchronises s
// when the hierarchy has any): the grid barriers of the persistent small-level launch (the
// hierarchy's own error word, cleared with its barrier state) and, for hierarchies built with
// the TMA-staged SpMV forced (NNMG_FORCE_LAYOUT=tma), that kernel's device-wide flag, which
// concurrent forced-TMA work elsewhere can also set. Either expiry: MG_ERR_TIMEOUT.
bool take_persistent_error(mg_hierarchy* h, cudaStream_t s) {
  PBarrier* bars[2] = {h->e64 ? h->e64->bar : (h->e32 ? h->e32->bar : nullptr), h->solo.bar};
  bool any = false;
  for (PBarrier* bar : bars) {
    if (!bar) continue;
    int err = 0;
    CK(cudaMemcpyAsync(&err, &bar->error, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (err) {
      CK(cudaMemsetAsync(bar, 0, sizeof(PBarrier), s));
      CK(cudaStreamSynchronize(s));
      any = true;
    }
  }
  return any;
}
void check_device_waits(mg_hierarchy* h, cudaStream_t s) {
  if (take_persistent_error(h, s))
    throw Error(MG_ERR_TIMEOUT, "a grid barrier of the persistent small-level launch gave up; the result is not valid");
  if (h->uses_tma && take_wait_timeout(s))
    throw Error(MG_ERR_TIMEOUT, "a bounded wait in the TMA-staged SpMV gave up; the result is not valid");
}

// A library-numbered FP64 vector into a level's internal order and type (perm: internal
// index -> library index; null = same order), and back.
template <typename T>
void load(T* dst, const double* src, int n, const int32_t* perm, cudaStream_t s) {
  if (!src) throw Error(MG_ERR_INVALID_ARG, "null vector");
  if (std::is_same<T, double>::value && !perm) {
    if ((const void*)dst != (const void*)src)
      CK(cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  } else {
    gather<double, T>(n, perm, src, dst, s);
  }
}
template <typename T>
void store(double* dst, const T* src, int n, const int32_t* perm, cudaStream_t s) {
  if (!dst) throw Error(MG_ERR_INVALID_ARG, "null vector");
  if (std::is_same<T, double>::value && !perm) {
    if ((const void*)dst != (const void*)src)
      CK(cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  } else {
    scatter<T, double>(n, perm, src, dst, s);
  }
}

void device_phase(mg_hierarchy* h) {
  build_device(h);
  count_launches(h);
  if (persistent_solve_ok(h)) {  // the whole solve in one persistent launch; no graph needed
    if (h->e64) build_solo<double>(h);
    else build_solo<float>(h);
  } else if (h->opt.use_graph) {
    build_graph(h);
  }
  CK(cudaStreamSynchronize(h->own_stream));
}

void common_setup_tail(mg_hierarchy* h) {
  finish_setup_host(h);
  if (!h->opt.host_only) device_phase(h);
}

}  // namespace

namespace {
template <typename F>
int level_step(mg_hierarchy_t* h, int32_t l, const double* b, double* x, void* stream, F&& step) {
  checked(h);
  check_level(h, l, true);
  cudaStream_t s = (cudaStream_t)stream;
  h->with_engine([&](auto& e) {
    using T = typename std::remove_pointer<decltype(e.lv[0].b)>::type;
    auto& L = e.lv[l];
    load<T>(L.b, b, L.n, L.perm, s);
    load<T>(L.x, x, L.n, L.perm, s);
    step(e, s);
    store<T>(x, L.x, L.n, L.perm, s);
  });
  check_launch("level step");
  check_device_waits(h, s);
  return MG_OK;
}
}  // namespace

extern "C" {

void mg_default_options(mg_options_t* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->cheb_degree = 2;
  o->nu = 1;
  o->patch_layers = 1;
  o->smoother = MG_SMOOTHER_SANDWICH;
  o->adjusted_lambda = 1;
  o->precision = MG_PREC_FP64;
  o->host_only = 0;
  o->eig_maxit = 600;
  o->lmin_ratio = 0.1;
  o->lmax_safety = 1.0;
  o->eig_tol = 1e-8;
  o->lambda_override = nullptr;
  o->use_graph = 1;
  o->local_levels_mask = -1;
  o->quality_threshold = 0.1;
  o->sell_sigma = 0;
  o->reorder = MG_REORDER_NONE;
  o->pde = MG_PDE_POISSON;
  o->young = 6.9e10;
  o->poisson_ratio = 0.33;
  o->small_level_dofs = 0;
  o->fp32_patch_kappa = 10000;
  o->tune_min_nnz = 1 << 20;
}

}  // extern "C"

namespace nnmg {

// Everything mg_setup does on the host: DoF maps, assembly, quality, patches, transfer,
// Galerkin operators, diagonals and eigenvalues. The device phase is separate.
mg_hierarchy* build_host_hierarchy(const mg_mesh_t* levels, int32_t L, int32_t degree, double quality_threshold,
                                   const mg_options_t* opt) {
  if (!levels || L < 2 || L > 32) throw Error(MG_ERR_INVALID_ARG, "need 2 <= L <= 32 mesh levels");
  if (degree != 1 && degree != 2) throw Error(MG_ERR_INVALID_ARG, "degree must be 1 or 2");
  std::unique_ptr<mg_hierarchy> H(new mg_hierarchy());
  if (opt) H->opt = *opt;
  else mg_default_options(&H->opt);
  H->opt.quality_threshold = quality_threshold;
  validate_options(H->opt);
  H->L = L;
  H->degree = degree;
  H->geometric = true;
  const bool elastic = H->opt.pde == MG_PDE_ELASTICITY;
  std::vector<MeshH> meshes(L);
  std::vector<DofMapH> dms(L);
  H->host.resize(L);
  PhaseTimer tm;
  for (int l = 0; l < L; ++l) {
    const mg_mesh_t& m = levels[l];
    if ((m.dim != 2 && m.dim != 3) || m.nv < m.dim + 1 || m.nc < 1 || !m.coords || !m.cells)
      throw Error(MG_ERR_INVALID_ARG, "invalid mesh at level " + std::to_string(l));
    if (m.dim != levels[0].dim) throw Error(MG_ERR_INVALID_ARG, "all levels must have the same dimension");
    MeshH& M = meshes[l];
    M.dim = m.dim;
    M.nv = m.nv;
    M.nc = m.nc;
    M.x.assign(m.coords, m.coords + m.nv * m.dim);
    M.c.assign(m.cells, m.cells + m.nc * (m.dim + 1));
    for (int32_t v : M.c)
      if (v < 0 || v >= m.nv) throw Error(MG_ERR_INVALID_ARG, "cell vertex index out of range at level " + std::to_string(l));
    if (m.dirichlet_vertex_mask) M.mask.assign(m.dirichlet_vertex_mask, m.dirichlet_vertex_mask + m.nv);
    dms[l] = build_dofmap(M, degree);
    LevelH& lv = H->host[l];
    lv.dim = m.dim;
    lv.gamma = radius_ratio(M);
    for (int64_t c = 0; c < M.nc; ++c)
      if (!(lv.gamma[c] > 0)) throw Error(MG_ERR_DEGENERATE_CELL, "level " + std::to_string(l) + ": cell " + std::to_string(c) + " is degenerate");
    // vector problems: every free node carries ncomp consecutive DoFs (same point)
    const int ncomp = elastic ? m.dim : 1;
    lv.dof_points.resize(dms[l].nfree * ncomp * m.dim);
    for (int64_t i = 0; i < dms[l].nfree; ++i)
      for (int c = 0; c < ncomp; ++c)
        for (int r = 0; r < m.dim; ++r)
          lv.dof_points[(i * ncomp + c) * m.dim + r] = dms[l].points[dms[l].free_list[i] * m.dim + r];
    if ((H->opt.local_levels_mask >> std::min(l, 31)) & 1)
      local_patches(M, dms[l], lv.gamma, quality_threshold, H->opt.patch_layers, lv.patch_ptr, lv.patch_dofs);
    else
      lv.patch_ptr.assign(1, 0);
    if (ncomp > 1) {
      std::vector<int32_t> vdofs;
      vdofs.reserve(lv.patch_dofs.size() * ncomp);
      for (int32_t f : lv.patch_dofs)
        for (int c = 0; c < ncomp; ++c) vdofs.push_back(f * ncomp + c);
      lv.patch_dofs.swap(vdofs);
      for (int32_t& p : lv.patch_ptr) p *= ncomp;
    }
    H->ncells.push_back(M.nc);
    tm.mark("dofmap/gamma/patches L" + std::to_string(l));
  }
  if (elastic) {
    const double E = H->opt.young, nu = H->opt.poisson_ratio;
    H->host[0].A = assemble_elasticity(meshes[0], dms[0], E / (2.0 * (1.0 + nu)), E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)));
    H->fine_faces = boundary_faces(meshes[0], dms[0]);
    H->fine_load_unit = load_constant(meshes[0], dms[0], 1.0);  // per node: int phi_k
  } else {
    H->host[0].A = assemble_stiffness(meshes[0], dms[0]);
    H->fine_load_unit = load_constant(meshes[0], dms[0], 1.0);
  }
  tm.mark("assembly L0");
  for (int l = 1; l < L; ++l) {
    LevelH& f = H->host[l - 1];
    f.P = prolongation(dms[l - 1], meshes[l], dms[l]);
    if (elastic) f.P = kron_identity(f.P, meshes[0].dim);
    f.R = transpose(f.P);
    tm.mark("transfer L" + std::to_string(l));
    Csr AP = spgemm(f.A, f.P);
    tm.mark("A P L" + std::to_string(l));
    H->host[l].A = unit_diagonal_on_empty_rows(spgemm(f.R, AP));
    tm.mark("galerkin L" + std::to_string(l));
  }
  meshes.clear();
  dms.clear();
  finish_setup_host(H.get());
  return H.release();
}

void build_device_hierarchy(mg_hierarchy* h) { device_phase(h); }

void set_last_error(const std::string& msg) { g_setup_error = msg; }

int64_t estimate_device_bytes(const mg_hierarchy* h) {
  const int vbytes = h->opt.precision == MG_PREC_MIXED ? 4 : 8;
  int64_t tot = 0, largest = 0;
  auto op = [&](const Csr& A) {
    // SELL padding and the layout candidates of the autotuner: bound by 1.5 x CSR
    int64_t b = (int64_t)(1.5 * (double)A.nnz() * (vbytes + 4)) + 8 * (A.nrows + 1);
    largest = std::max(largest, b);
    tot += b;
  };
  for (int l = 0; l < h->L; ++l) {
    const LevelH& lv = h->host[l];
    op(lv.A);
    if (l + 1 < h->L) {
      op(lv.P);
      op(lv.R);
    }
    if (h->opt.global_smoother == MG_GLOBAL_SGS && l + 1 < h->L) op(lv.A);  // per-colour operators
    tot += 8 * vbytes * lv.A.nrows;  // level vectors
    const int64_t np = (int64_t)lv.patch_ptr.size() - 1;
    for (int64_t p = 0; p < np; ++p) {
      int64_t m = lv.patch_ptr[p + 1] - lv.patch_ptr[p];
      tot += (vbytes == 4 ? 12 : 8) * m * m + 64 * m;   // FP64 inverse (+ its FP32 copy, mixed)
    }
    if (np > 0) tot += 16 * (int64_t)lv.A.nnz() / std::max<int64_t>(lv.A.nrows, 1) * (int64_t)lv.patch_dofs.size() * 4;
    if (np > 0 && l + 1 < h->L)  // rows of A P on the patch rows
      tot += 12 * (int64_t)lv.patch_dofs.size() * (lv.A.nnz() / std::max<int64_t>(lv.A.nrows, 1) + 1) *
             (lv.P.nnz() / std::max<int64_t>(lv.P.nrows, 1) + 1);
  }
  const int64_t nc = h->host[h->L - 1].A.nrows;
  tot += 16 * nc * nc;  // coarse inverse and split-K partials
  const int64_t n0 = h->host[0].A.nrows;
  tot += 8 * 8 * n0;    // CG vectors
  if (h->opt.precision == MG_PREC_MIXED) tot += 12 * h->host[0].A.nnz() * 3 / 2;
  return tot + 2 * largest + (64 << 20);  // autotuner trial layouts + slack
}

int64_t hierarchy_device_bytes(const mg_hierarchy* h) { return h->mem.bytes; }
int64_t hierarchy_dofs(const mg_hierarchy* h) { return h->host[0].A.nrows; }
std::vector<double> hierarchy_unit_load(const mg_hierarchy* h) {
  if (h->opt.pde != MG_PDE_ELASTICITY) return h->fine_load_unit;
  const int d = h->fine_faces.dim;
  std::vector<double> b(h->fine_load_unit.size() * d);
  for (size_t k = 0; k < h->fine_load_unit.size(); ++k)
    for (int c = 0; c < d; ++c) b[k * d + c] = h->fine_load_unit[k];
  return b;
}

void enqueue_host_solve(mg_hierarchy* h, const double* b, double* x, double rtol, int maxit, cudaEvent_t done,
                        cudaEvent_t start) {
  if (!h->graph && !h->solo.tasks)
    throw Error(MG_ERR_INVALID_ARG, "the solve server needs hierarchies built with use_graph = 1");
  cudaStream_t s = h->own_stream;
  if (start) CK(cudaEventRecord(start, s));
  CK(cudaMemcpyAsync(h->cq, b, sizeof(double) * h->n0, cudaMemcpyHostToDevice, s));
  gather<double, double>(h->n0, h->perm0, h->cq, h->cb, s);
  enqueue_state(h, rtol, maxit, s);
  enqueue_solo_or_graph(h, maxit, s);
  enqueue_exit(h, s);
  scatter<double, double>(h->n0, h->perm0, h->cx, h->cq, s);
  CK(cudaMemcpyAsync(x, h->cq, sizeof(double) * h->n0, cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(done, s));
}

int collect_host_solve(mg_hierarchy* h, mg_solve_info_t* info) {
  const int rc = collect_state(h, info);
  if (take_persistent_error(h, h->own_stream)) return MG_ERR_TIMEOUT;
  if (h->uses_tma && take_wait_timeout(h->own_stream)) return MG_ERR_TIMEOUT;  // forced TMA-staged SpMV only
  return rc;
}

void destroy_hierarchy(mg_hierarchy* h) { delete h; }

namespace {
std::mutex g_pinned_mu;
std::multimap<int64_t, double*> g_pinned_free;   // capacity -> buffer
std::map<double*, int64_t> g_pinned_cap;
}  // namespace

double* pinned_acquire(int64_t n) {
  std::lock_guard<std::mutex> lk(g_pinned_mu);
  auto it = g_pinned_free.lower_bound(n);
  if (it != g_pinned_free.end()) {
    double* p = it->second;
    g_pinned_free.erase(it);
    return p;
  }
  int64_t cap = 1024;
  while (cap < n) cap *= 2;
  double* p = nullptr;
  CK(cudaMallocHost(&p, sizeof(double) * cap));
  g_pinned_cap[p] = cap;
  return p;
}

void pinned_release(double* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pinned_mu);
  g_pinned_free.emplace(g_pinned_cap[p], p);
}

}  // namespace nnmg

extern "C" {

int mg_setup(const mg_mesh_t* levels, int32_t L, int32_t degree, double quality_threshold, const mg_options_t* opt,
             mg_hierarchy_t** out) {
  mg_hierarchy* h = nullptr;
  API_BEGIN
  nnmg::g_setup_error.clear();
  if (!out) throw Error(MG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  std::unique_ptr<mg_hierarchy> H(build_host_hierarchy(levels, L, degree, quality_threshold, opt));
  if (!H->opt.host_only) device_phase(H.get());
  *out = H.release();
  return MG_OK;
  API_END_H(h)
}

int mg_setup_csr(const mg_csr_t* A, const mg_csr_t* P, int32_t L, const int32_t* const* patch_ptr,
                 const int32_t* const* patch_dofs, const int32_t* num_patches, const mg_options_t* opt,
                 mg_hierarchy_t** out) {
  mg_hierarchy* h = nullptr;
  API_BEGIN
  nnmg::g_setup_error.clear();
  if (!out) throw Error(MG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!A || !P || L < 2 || L > 32) throw Error(MG_ERR_INVALID_ARG, "need 2 <= L <= 32 levels and A, P arrays");
  std::unique_ptr<mg_hierarchy> H(new mg_hierarchy());
  if (opt) H->opt = *opt;
  else mg_default_options(&H->opt);
  validate_options(H->opt);
  if (!H->opt.lambda_override) throw Error(MG_ERR_INVALID_ARG, "mg_setup_csr needs opt->lambda_override");
  H->L = L;
  H->host.resize(L);
  auto copy_csr = [](const mg_csr_t& c, Csr& d) {
    if (c.nrows < 1 || c.ncols < 1 || !c.rowptr || c.nrows >= INT32_MAX || c.ncols >= INT32_MAX)
      throw Error(MG_ERR_INVALID_ARG, "invalid CSR matrix");
    d.nrows = c.nrows;
    d.ncols = c.ncols;
    d.rp.assign(c.rowptr, c.rowptr + c.nrows + 1);
    int64_t nnz = d.rp[c.nrows];
    if (d.rp[0] != 0 || nnz < 0) throw Error(MG_ERR_INVALID_ARG, "invalid CSR row pointer");
    for (int64_t i = 0; i < c.nrows; ++i)
      if (d.rp[i + 1] < d.rp[i]) throw Error(MG_ERR_INVALID_ARG, "CSR row pointer not monotone");
    if (nnz > 0 && (!c.colidx || !c.values)) throw Error(MG_ERR_INVALID_ARG, "null CSR arrays");
    d.ci.assign(c.colidx, c.colidx + nnz);
    d.v.assign(c.values, c.values + nnz);
    for (int32_t j : d.ci)
      if (j < 0 || j >= c.ncols) throw Error(MG_ERR_INVALID_ARG, "CSR column index out of range");
  };
  for (int l = 0; l < L; ++l) {
    copy_csr(A[l], H->host[l].A);
    if (A[l].nrows != A[l].ncols) throw Error(MG_ERR_INVALID_ARG, "A must be square");
    LevelH& lv = H->host[l];
    lv.patch_ptr.assign(1, 0);
    if (patch_ptr && patch_dofs && num_patches && patch_ptr[l] && num_patches[l] > 0) {
      int np = num_patches[l];
      lv.patch_ptr.assign(patch_ptr[l], patch_ptr[l] + np + 1);
      lv.patch_dofs.assign(patch_dofs[l], patch_dofs[l] + lv.patch_ptr[np]);
      std::vector<uint8_t> seen(A[l].nrows, 0);
      for (int32_t f : lv.patch_dofs) {
        if (f < 0 || f >= A[l].nrows || seen[f]) throw Error(MG_ERR_INVALID_ARG, "patch DoFs out of range or not disjoint");
        seen[f] = 1;
      }
    }
  }
  for (int l = 0; l + 1 < L; ++l) {
    copy_csr(P[l], H->host[l].P);
    if (P[l].nrows != A[l].nrows || P[l].ncols != A[l + 1].nrows) throw Error(MG_ERR_INVALID_ARG, "P shape mismatch");
    H->host[l].R = transpose(H->host[l].P);
  }
  common_setup_tail(H.get());
  *out = H.release();
  return MG_OK;
  API_END_H(h)
}

void mg_free(mg_hierarchy_t* h) { delete h; }

const char* mg_last_error(const mg_hierarchy_t* h) { return h ? h->err.c_str() : nnmg::g_setup_error.c_str(); }

int32_t mg_num_levels(const mg_hierarchy_t* h) { return h ? h->L : 0; }

int64_t mg_num_dofs(const mg_hierarchy_t* h, int32_t l) {
  if (!h || l < 0 || l >= h->L) return -1;
  return h->host[l].A.nrows;
}
int64_t mg_level_nnz(const mg_hierarchy_t* h, int32_t l) {
  if (!h || l < 0 || l >= h->L) return -1;
  return h->host[l].A.nnz();
}
int64_t mg_transfer_nnz(const mg_hierarchy_t* h, int32_t l) {
  if (!h || l < 0 || l >= h->L - 1) return -1;
  return h->host[l].P.nnz();
}

int mg_num_patches(const mg_hierarchy_t* hc, int32_t l, int32_t* num, int64_t* total) {
  mg_hierarchy* h = const_cast<mg_hierarchy*>(hc);
  API_BEGIN
  checked(h, false);
  check_level(h, l);
  if (num) *num = (int32_t)h->host[l].patch_ptr.size() - 1;
  if (total) *total = (int64_t)h->host[l].patch_dofs.size();
  return MG_OK;
  API_END_H(h)
}

int mg_export_level(const mg_hierarchy_t* hc, int32_t l, int32_t* rowptr, int32_t* colidx, double* values) {
  mg_hierarchy* h = const_cast<mg_hierarchy*>(hc);
  API_BEGIN
  checked(h, false);
  check_level(h, l);
  const Csr& A = h->host[l].A;
  if (rowptr) std::copy(A.rp.begin(), A.rp.end(), rowptr);
  if (colidx) std::copy(A.ci.begin(), A.ci.end(), colidx);
  if (values) std::copy(A.v.begin(), A.v.end(), values);
  return MG_OK;
  API_END_H(h)
}

int mg_export_transfer(const mg_hierarchy_t* hc, int32_t l, int32_t* rowptr, int32_t* colidx, double* values) {
  mg_hierarchy* h = const_cast<mg_hierarchy*>(hc);
  API_BEGIN
  checked(h, false);
  check_level(h, l, true);
  const Csr& P = h->host[l].P;
  if (rowptr) std::copy(P.rp.begin(), P.rp.end(), rowptr);
  if (colidx) std::copy(P.ci.begin(), P.ci.end(), colidx);
  if (values) std::copy(P.v.begin(), P.v.end(), values);
  return MG_OK;
  API_END_H(h)
}

int mg_export_patches(const mg_hierarchy_t* hc, int32_t l, int32_t* ptr, int32_t* dofs) {
  mg_hierarchy* h = const_cast<mg_hierarchy*>(hc);
  API_BEGIN
  checked(h, false);
  check_level(h, l);
  const LevelH& lv = h->host[l];
  if (ptr) std::copy(lv.patch_ptr.begin(), lv.patch_ptr.end(), ptr);
  if (dofs) std::copy(lv.patch_dofs.begin(), lv.patch_dofs.end(), dofs);
  return MG_OK;
  API_END_H(h)
}

int mg_export_patch_precision(const mg_hierarchy_t* hc, int32_t l, int32_t* flags) {
  mg_hierarchy* h = const_cast<mg_hierarchy*>(hc);
  API_BEGIN
  checked(h);
  check_level(h, l);
  const int64_t np = (int64_t)h->host[l].patch_ptr.size() - 1;
  if (np > 0 && !flags) throw Error(MG_ERR_INVALID_ARG, "null flags");
  h->with_engine([&](auto& e) {
    const auto& v = e.lv[l].pfp32;
    for (int64_t p = 0; p < np; ++p) flags[p] = (size_t)p < v.size() ? v[p] : 0;
  });
  return MG_OK;
  API_END_H(h)
}

int mg_export_colouring(const mg_hierarchy_t* hc, int32_t l, int32_t* ncolours, int32_t* colour) {
  mg_hierarchy* h = const_cast<mg_hierarchy*>(hc);
  API_BEGIN
  checked(h, false);
  check_level(h, l, true);
  if (h->opt.global_smoother != MG_GLOBAL_SGS)
    throw Error(MG_ERR_INVALID_ARG, "the hierarchy's global smoother is not SGS");
  const LevelH& lv = h->host[l];
  if (ncolours) *ncolours = lv.ncolours;
  if (colour) std::copy(lv.colour.begin(), lv.colour.end(), colour);
  return MG_OK;
  API_END_H(h)
}

int mg_eigs(const mg_hierarchy_t* hc, int32_t l, double* lmax, double* lmax_adj, double* lmax_used) {
  mg_hierarchy* h = const_cast<mg_hierarchy*>(hc);
  API_BEGIN
  checked(h, false);
  check_level(h, l, true);
  const LevelH& lv = h->host[l];
  if (lmax) *lmax = lv.lmax_unadj;
  if (lmax_adj) *lmax_adj = lv.lmax_adj;
  if (lmax_used) *lmax_used = lv.lmax;
  return MG_OK;
  API_END_H(h)
}

int mg_dof_coords(const mg_hierarchy_t* hc, int32_t l, double* out) {
  mg_hierarchy* h = const_cast<mg_hierarchy*>(hc);
  API_BEGIN
  checked(h, false);
  check_level(h, l);
  if (!h->geometric) throw Error(MG_ERR_INVALID_ARG, "not a geometric hierarchy");
  if (!out) throw Error(MG_ERR_INVALID_ARG, "null output");
  std::copy(h->host[l].dof_points.begin(), h->host[l].dof_points.end(), out);
  return MG_OK;
  API_END_H(h)
}

int mg_cell_quality(const mg_hierarchy_t* hc, int32_t l, double* out) {
  mg_hierarchy* h = const_cast<mg_hierarchy*>(hc);
  API_BEGIN
  checked(h, false);
  check_level(h, l);
  if (!h->geometric) throw Error(MG_ERR_INVALID_ARG, "not a geometric hierarchy");
  if (!out) throw Error(MG_ERR_INVALID_ARG, "null output");
  std::copy(h->host[l].gamma.begin(), h->host[l].gamma.end(), out);
  return MG_OK;
  API_END_H(h)
}

int mg_load_constant(const mg_hierarchy_t* hc, double f, double* out) {
  mg_hierarchy* h = const_cast<mg_hierarchy*>(hc);
  API_BEGIN
  checked(h, false);
  if (!h->geometric || h->opt.pde != MG_PDE_POISSON)
    throw Error(MG_ERR_INVALID_ARG, "not a geometric Poisson hierarchy");
  if (!out) throw Error(MG_ERR_INVALID_ARG, "null output");
  for (size_t i = 0; i < h->fine_load_unit.size(); ++i) out[i] = f * h->fine_load_unit[i];
  return MG_OK;
  API_END_H(h)
}

int mg_load_body(const mg_hierarchy_t* hc, const double* f, double* out) {
  mg_hierarchy* h = const_cast<mg_hierarchy*>(hc);
  API_BEGIN
  checked(h, false);
  if (!h->geometric || h->opt.pde != MG_PDE_ELASTICITY)
    throw Error(MG_ERR_INVALID_ARG, "not a geometric elasticity hierarchy");
  if (!f || !out) throw Error(MG_ERR_INVALID_ARG, "null pointer");
  const int d = h->fine_faces.dim;
  for (size_t k = 0; k < h->fine_load_unit.size(); ++k)
    for (int c = 0; c < d; ++c) out[k * d + c] = f[c] * h->fine_load_unit[k];
  return MG_OK;
  API_END_H(h)
}

int mg_load_traction(const mg_hierarchy_t* hc, int32_t axis, double value, const double* t, double* out) {
  mg_hierarchy* h = const_cast<mg_hierarchy*>(hc);
  API_BEGIN
  checked(h, false);
  if (!h->geometric || h->opt.pde != MG_PDE_ELASTICITY)
    throw Error(MG_ERR_INVALID_ARG, "not a geometric elasticity hierarchy");
  if (!t || !out) throw Error(MG_ERR_INVALID_ARG, "null pointer");
  const int d = h->fine_faces.dim;
  if (axis < 0 || axis >= d) throw Error(MG_ERR_INVALID_ARG, "axis out of range");
  const int64_t n = h->host[0].A.nrows;
  std::vector<double> b = traction_load(h->fine_faces, axis, value, 1e-12, t, n / d);
  std::copy(b.begin(), b.end(), out);
  return MG_OK;
  API_END_H(h)
}

int mg_vcycle(mg_hierarchy_t* h, const double* b, double* x, void* stream) {
  API_BEGIN
  checked(h);
  if (!b || !x) throw Error(MG_ERR_INVALID_ARG, "null vector");
  cudaStream_t s = (cudaStream_t)stream;
  const int n = h->n0;
  // x += V(b - A x) in the internal order: x and b gathered into p and q, r into the CG
  // residual buffer, the cycle from a zero guess, then x scattered back
  gather<double, double>(n, h->perm0, x, h->cp, s);
  gather<double, double>(n, h->perm0, b, h->cq, s);
  sell_resid<double>(h->A0, h->cp, h->cq, h->cr, s);
  h->with_engine([&](auto& e) {
    using T = typename std::remove_pointer<decltype(e.lv[0].b)>::type;
    load<T>(e.lv[0].b, h->cr, n, nullptr, s);
    CK(cudaMemsetAsync(e.lv[0].x, 0, sizeof(T) * n, s));
    e.cycle(0, s);
    axpy_from<T>(n, e.lv[0].x, h->cp, s);
  });
  scatter<double, double>(n, h->perm0, h->cp, x, s);
  check_launch("mg_vcycle");
  check_device_waits(h, s);
  return MG_OK;
  API_END_H(h)
}

int mg_solve(mg_hierarchy_t* h, const double* b, double* x, double rtol, int32_t maxit, mg_solve_info_t* info,
             void* stream) {
  API_BEGIN
  checked(h);
  if (!b || !x) throw Error(MG_ERR_INVALID_ARG, "null vector");
  cudaStream_t s = (cudaStream_t)stream;
  gather<double, double>(h->n0, h->perm0, b, h->cb, s);
  int rc = run_solve(h, rtol, maxit, info, s);
  scatter<double, double>(h->n0, h->perm0, h->cx, x, s);
  CK(cudaStreamSynchronize(s));
  check_device_waits(h, s);
  if (rc != MG_OK) h->err = rc == MG_ERR_BREAKDOWN ? "CG breakdown" : "no convergence within maxit";
  return rc;
  API_END_H(h)
}

int mg_solve_host(mg_hierarchy_t* h, const double* b, double* x, double rtol, int32_t maxit, mg_solve_info_t* info,
                  void* stream) {
  API_BEGIN
  checked(h);
  if (!b || !x) throw Error(MG_ERR_INVALID_ARG, "null vector");
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(h->cp, b, sizeof(double) * h->n0, cudaMemcpyHostToDevice, s));
  gather<double, double>(h->n0, h->perm0, h->cp, h->cb, s);
  int rc = run_solve(h, rtol, maxit, info, s);
  scatter<double, double>(h->n0, h->perm0, h->cx, h->cp, s);
  CK(cudaMemcpyAsync(x, h->cp, sizeof(double) * h->n0, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  check_device_waits(h, s);
  if (rc != MG_OK) h->err = rc == MG_ERR_BREAKDOWN ? "CG breakdown" : "no convergence within maxit";
  return rc;
  API_END_H(h)
}

int mg_solve_stationary(mg_hierarchy_t* h, const double* b, double* x, double rtol, int32_t maxit,
                        mg_solve_info_t* info, void* stream) {
  API_BEGIN
  checked(h);
  if (!b || !x) throw Error(MG_ERR_INVALID_ARG, "null vector");
  if (!(rtol >= 0) || maxit < 1) throw Error(MG_ERR_INVALID_ARG, "rtol must be >= 0 and maxit >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  auto norm2 = [&](const double* v) {
    CK(cudaMemsetAsync(h->ticket, 0, sizeof(unsigned), s));
    dot_self(h->n0, v, Reduce{h->part, h->ticket, h->st, FIN_NORM, 0, 0}, s);
    CK(cudaMemcpyAsync(h->hst, h->st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return h->hst->rr;
  };
  double bb = norm2(b);
  int it = 0;
  double rr = 0;
  for (;;) {
    gather<double, double>(h->n0, h->perm0, x, h->cp, s);
    gather<double, double>(h->n0, h->perm0, b, h->cz, s);
    sell_resid<double>(h->A0, h->cp, h->cz, h->cq, s);
    rr = norm2(h->cq);
    if (bb == 0.0 || rr <= rtol * rtol * bb || it >= maxit) break;
    int rc = mg_vcycle(h, b, x, stream);
    if (rc != MG_OK) return rc;
    ++it;
  }
  bool conv = bb == 0.0 || rr <= rtol * rtol * bb;
  if (info) {
    info->iterations = it;
    info->converged = conv;
    info->rel_residual = bb > 0 ? std::sqrt(rr / bb) : 0.0;
    info->true_rel_residual = info->rel_residual;
  }
  return conv ? MG_OK : MG_ERR_NO_CONVERGENCE;
  API_END_H(h)
}

int mg_solve_batch(mg_hierarchy_t* const* hs, const double* const* b, double* const* x, int32_t n, double rtol,
                   int32_t maxit, mg_solve_info_t* info, void* stream) {
  mg_hierarchy* h = nullptr;
  API_BEGIN
  if (n < 0 || (n > 0 && (!hs || !b || !x))) throw Error(MG_ERR_INVALID_ARG, "invalid batch arrays");
  if (!(rtol >= 0) || maxit < 1) throw Error(MG_ERR_INVALID_ARG, "rtol must be >= 0 and maxit >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  // problems whose whole solve runs persistently: one launch per precision for all of them;
  // the others: their graphs on their own streams, overlapping on the device
  std::vector<int> g64, g32, rest;
  for (int i = 0; i < n; ++i) {
    mg_hierarchy* hi = checked(hs[i]);
    if (persistent_solve_ok(hi)) (hi->e64 ? g64 : g32).push_back(i);
    else rest.push_back(i);
  }
  cudaEvent_t start;
  CK(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  CK(cudaEventRecord(start, s));
  for (int i : rest) {
    mg_hierarchy* hi = hs[i];
    if (!hi->graph) throw Error(MG_ERR_INVALID_ARG, "mg_solve_batch needs hierarchies built with use_graph = 1");
    CK(cudaStreamWaitEvent(hi->own_stream, start, 0));
    gather<double, double>(hi->n0, hi->perm0, b[i], hi->cb, hi->own_stream);
    enqueue_state(hi, rtol, maxit, hi->own_stream);
    CK(cudaGraphLaunch(hi->graph, hi->own_stream));
    enqueue_exit(hi, hi->own_stream);
    scatter<double, double>(hi->n0, hi->perm0, hi->cx, x[i], hi->own_stream);
  }
  DevMem tmp;
  tmp.stream = s;
  auto group = [&](const std::vector<int>& idx, auto tag) {
    using T = decltype(tag);
    if (idx.empty()) return;
    std::vector<mg_hierarchy*> gh;
    std::vector<double*> part;
    std::vector<CgState*> states;
    for (int i : idx) {
      mg_hierarchy* hi = hs[i];
      gh.push_back(hi);
      part.push_back(tmp.alloc<double>(pcg_part_size(hi)));
      states.push_back(hi->st);
      gather<double, double>(hi->n0, hi->perm0, b[i], hi->cb, s);
      enqueue_state(hi, rtol, maxit, s);
    }
    PProgram pg;
    int nhead = 0;
    assemble_pcg<T>(gh, part, pg, &nhead);
    PTask* dt = tmp.upload(pg.tasks);
    PPhase* dp = tmp.upload(pg.phases);
    CgState** ds = tmp.upload(states);
    PBarrier* bar = tmp.alloc<PBarrier>(1);
    CK(persistent_launch<T>(dp, nhead, dt, bar, s, (int)pg.phases.size() - nhead, ds, (int)gh.size(),
                            pcg_iteration_cap(maxit)));
    for (int i : idx) {
      enqueue_exit(hs[i], s);
      scatter<double, double>(hs[i]->n0, hs[i]->perm0, hs[i]->cx, x[i], s);
    }
    int err = 0;
    CK(cudaMemcpyAsync(&err, &bar->error, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (err) throw Error(MG_ERR_TIMEOUT, "a grid barrier of the batched persistent solve gave up; results not valid");
  };
  group(g64, double());
  group(g32, float());
  CK(cudaStreamSynchronize(s));
  tmp.release();
  int rc_all = MG_OK;
  for (int i = 0; i < n; ++i) {
    mg_hierarchy* hi = hs[i];
    if (std::find(rest.begin(), rest.end(), i) != rest.end()) {
      CK(cudaStreamSynchronize(hi->own_stream));
      check_device_waits(hi, hi->own_stream);
    }
    int rc = collect_state(hi, info ? &info[i] : nullptr);
    if (rc_all == MG_OK) rc_all = rc;
  }
  cudaEventDestroy(start);
  return rc_all;
  API_END_H(h)
}

int mg_apply_A(mg_hierarchy_t* h, int32_t l, const double* x, double* y, void* stream) {
  API_BEGIN
  checked(h);
  check_level(h, l);
  cudaStream_t s = (cudaStream_t)stream;
  if (!x || !y) throw Error(MG_ERR_INVALID_ARG, "null vector");
  if (l == 0) {
    gather<double, double>(h->n0, h->perm0, x, h->cp, s);
    sell_spmv<double>(h->A0, h->cp, h->cq, s);
    scatter<double, double>(h->n0, h->perm0, h->cq, y, s);
  } else {
    h->with_engine([&](auto& e) {
      using T = typename std::remove_pointer<decltype(e.lv[0].b)>::type;
      auto& L = e.lv[l];
      load<T>(L.x, x, L.n, L.perm, s);
      sell_spmv<T>(L.A, L.x, L.b, s);
      store<T>(y, L.b, L.n, L.perm, s);
    });
  }
  check_launch("mg_apply_A");
  check_device_waits(h, s);
  return MG_OK;
  API_END_H(h)
}


int mg_chebyshev(mg_hierarchy_t* h, int32_t l, const double* b, double* x, void* stream) {
  API_BEGIN
  if (h && h->opt.global_smoother != MG_GLOBAL_CHEBYSHEV)
    throw Error(MG_ERR_INVALID_ARG, "the hierarchy's global smoother is not Chebyshev");
  return level_step(h, l, b, x, stream, [&](auto& e, cudaStream_t s) { e.cheb(l, s); });
  API_END_H(h)
}

int mg_sgs(mg_hierarchy_t* h, int32_t l, const double* b, double* x, void* stream) {
  API_BEGIN
  if (h && h->opt.global_smoother != MG_GLOBAL_SGS)
    throw Error(MG_ERR_INVALID_ARG, "the hierarchy's global smoother is not SGS");
  return level_step(h, l, b, x, stream, [&](auto& e, cudaStream_t s) { e.sgs_sweep(l, s); });
  API_END_H(h)
}

int mg_local_correction(mg_hierarchy_t* h, int32_t l, const double* b, double* x, void* stream) {
  API_BEGIN
  return level_step(h, l, b, x, stream, [&](auto& e, cudaStream_t s) {
    if (e.lv[l].np > 0) e.local(l, s);
  });
  API_END_H(h)
}

int mg_smooth(mg_hierarchy_t* h, int32_t l, int32_t post, const double* b, double* x, void* stream) {
  API_BEGIN
  return level_step(h, l, b, x, stream, [&](auto& e, cudaStream_t s) { e.smooth(l, post != 0, s); });
  API_END_H(h)
}

int mg_residual_restrict(mg_hierarchy_t* h, int32_t l, const double* b, const double* x, double* r, double* bc,
                         void* stream) {
  API_BEGIN
  checked(h);
  check_level(h, l, true);
  if (!b || !x || !r || !bc) throw Error(MG_ERR_INVALID_ARG, "null vector");
  cudaStream_t s = (cudaStream_t)stream;
  h->with_engine([&](auto& e) {
    using T = typename std::remove_pointer<decltype(e.lv[0].b)>::type;
    auto& L = e.lv[l];
    auto& C = e.lv[l + 1];
    load<T>(L.b, b, L.n, L.perm, s);
    load<T>(L.x, x, L.n, L.perm, s);
    e.residual_restrict(l, s);
    store<T>(r, L.res, L.n, L.perm, s);
    store<T>(bc, C.b, C.n, C.perm, s);
  });
  check_launch("mg_residual_restrict");
  check_device_waits(h, s);
  return MG_OK;
  API_END_H(h)
}

int mg_prolong_correct(mg_hierarchy_t* h, int32_t l, const double* xc, double* x, void* stream) {
  API_BEGIN
  checked(h);
  check_level(h, l, true);
  if (!xc || !x) throw Error(MG_ERR_INVALID_ARG, "null vector");
  cudaStream_t s = (cudaStream_t)stream;
  h->with_engine([&](auto& e) {
    using T = typename std::remove_pointer<decltype(e.lv[0].b)>::type;
    auto& L = e.lv[l];
    auto& C = e.lv[l + 1];
    load<T>(C.x, xc, C.n, C.perm, s);
    load<T>(L.x, x, L.n, L.perm, s);
    e.prolong(l, s);
    store<T>(x, L.x, L.n, L.perm, s);
  });
  check_launch("mg_prolong_correct");
  return MG_OK;
  API_END_H(h)
}

int mg_coarse_solve(mg_hierarchy_t* h, const double* b, double* x, void* stream) {
  API_BEGIN
  checked(h);
  if (!b || !x) throw Error(MG_ERR_INVALID_ARG, "null vector");
  cudaStream_t s = (cudaStream_t)stream;
  h->with_engine([&](auto& e) {
    using T = typename std::remove_pointer<decltype(e.lv[0].b)>::type;
    auto& C = e.lv.back();
    load<T>(C.b, b, C.n, C.perm, s);
    e.coarse(s);
    store<T>(x, C.x, C.n, C.perm, s);
  });
  check_launch("mg_coarse_solve");
  return MG_OK;
  API_END_H(h)
}

int mg_time_vcycle(mg_hierarchy_t* h, int32_t level, int32_t reps, void* stream, double* ms) {
  API_BEGIN
  checked(h);
  check_level(h, level);
  if (reps < 1) throw Error(MG_ERR_INVALID_ARG, "reps must be >= 1");
  cudaStream_t s = h->own_stream;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  h->with_engine([&](auto& e) {
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    e.cycle(level, s);
    CK(cudaStreamEndCapture(s, &g));
  });
  CK(cudaGraphInstantiate(&ge, g, 0));
  cudaStream_t us = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaGraphLaunch(ge, us));  // warm-up
  CK(cudaEventRecord(e0, us));
  for (int i = 0; i < reps; ++i) CK(cudaGraphLaunch(ge, us));
  CK(cudaEventRecord(e1, us));
  CK(cudaEventSynchronize(e1));
  float t = 0;
  CK(cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGraphExecDestroy(ge);
  cudaGraphDestroy(g);
  if (ms) *ms = (double)t / reps;
  return MG_OK;
  API_END_H(h)
}

int mg_time_smoother_kernel(mg_hierarchy_t* h, int32_t reps, void* stream, double* ms, double* bytes) {
  API_BEGIN
  checked(h);
  if (reps < 1) throw Error(MG_ERR_INVALID_ARG, "reps must be >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  double nbytes = 0;
  h->with_engine([&](auto& e) {
    using T = typename std::remove_pointer<decltype(e.lv[0].b)>::type;
    auto& L = e.lv[0];
    const double sz = sizeof(T);
    auto meta_bytes = [&](const SellMat<T>& M) {
      return M.lanes > 1 ? 4.0 * (M.nrows + 1) + (M.col16 ? 4.0 * M.nrows : 0.0)
                         : 8.0 * (M.nslices + 1) + (M.col16 ? 4.0 * M.nslices : 0.0) + (M.perm ? 4.0 * M.nrows : 0.0);
    };
    if (e.sgs) {
      // one multicolour SGS application on the fine level (2C launches); per colour and
      // sweep: its nonzeros once, rows[], b, dinv read and x written for its rows
      e.sgs_sweep(0, s);  // warm-up
      CK(cudaEventRecord(e0, s));
      for (int i = 0; i < reps; ++i) e.sgs_sweep(0, s);
      CK(cudaEventRecord(e1, s));
      for (const SellMat<T>& M : L.gs)
        nbytes += 2.0 * ((double)M.nnz * sz + M.idx_bytes + (double)M.nrows * (4.0 + 3.0 * sz) + meta_bytes(M));
      return;
    }
    double cd = L.cd.size() > 1 ? L.cd[1] : 0.0, cr = L.cr.size() > 1 ? L.cr[1] : L.cr[0];
    sell_cheb<T>(L.A, L.x, L.b, L.dinv, L.d, L.xt, cd, cr, false, s);  // warm-up
    CK(cudaEventRecord(e0, s));
    for (int i = 0; i < reps; ++i) sell_cheb<T>(L.A, L.x, L.b, L.dinv, L.d, L.xt, cd, cr, false, s);
    CK(cudaEventRecord(e1, s));
    // algorithmic bytes: each nonzero's value and index once, six vectors, slice/row metadata
    nbytes = (double)L.A.nnz * sz + L.A.idx_bytes + (double)L.n * 6.0 * sz + meta_bytes(L.A);
  });
  check_launch("mg_time_smoother_kernel");
  CK(cudaEventSynchronize(e1));
  float t = 0;
  CK(cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ms) *ms = (double)t / reps;
  if (bytes) *bytes = nbytes;
  return MG_OK;
  API_END_H(h)
}

int mg_time_cg_product(mg_hierarchy_t* h, int32_t reps, void* stream, double* ms, double* bytes) {
  API_BEGIN
  checked(h);
  if (reps < 1) throw Error(MG_ERR_INVALID_ARG, "reps must be >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // q = A p with the p.q reduction (into the CG state, which the next solve re-initialises)
  CgState* st = h->st;
  const Reduce rd{h->part, h->ticket, st, FIN_NORM, 0, 0};
  sell_ap(h->A0, h->cp, h->cq, rd, s);  // warm-up
  CK(cudaEventRecord(e0, s));
  for (int i = 0; i < reps; ++i) sell_ap(h->A0, h->cp, h->cq, rd, s);
  CK(cudaEventRecord(e1, s));
  check_launch("mg_time_cg_product");
  CK(cudaEventSynchronize(e1));
  float t = 0;
  CK(cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const SellMat<double>& M = h->A0;
  const double meta = M.lanes > 1 ? 4.0 * (M.nrows + 1) + (M.col16 ? 4.0 * M.nrows : 0.0)
                                  : 8.0 * (M.nslices + 1) + (M.col16 ? 4.0 * M.nslices : 0.0) +
                                        (M.perm ? 4.0 * M.nrows : 0.0);
  if (ms) *ms = (double)t / reps;
  // algorithmic bytes: each nonzero's value and index once, p read (gathered) and q written
  // once, the slice/row metadata
  if (bytes) *bytes = 8.0 * (double)M.nnz + M.idx_bytes + 16.0 * (double)M.nrows + meta;
  return MG_OK;
  API_END_H(h)
}

int mg_time_patch_solve(mg_hierarchy_t* h, int32_t l, int32_t reps, void* stream, double* ms, double* fma64,
                        double* fma32, double* bytes) {
  API_BEGIN
  checked(h);
  check_level(h, l, true);
  if (reps < 1) throw Error(MG_ERR_INVALID_ARG, "reps must be >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  double f64 = 0.0, f32 = 0.0;
  float t = 0.f;
  h->with_engine([&](auto& e) {
    using T = typename std::remove_pointer<decltype(e.lv[0].b)>::type;
    auto& L = e.lv[l];
    const LevelH& H = h->host[l];
    for (size_t p = 0; p + 1 < H.patch_ptr.size(); ++p) {
      const double m = (double)(H.patch_ptr[p + 1] - H.patch_ptr[p]);
      const bool lo = std::is_same<T, float>::value && p < L.pfp32.size() && L.pfp32[p];
      (lo ? f32 : f64) += m * m;
    }
    if (L.nitems == 0) return;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    patch_solve<T>(L.nitems, L.items, L.pdofs, L.inv, L.inv32, L.rbuf, L.b, L.x, L.max_patch, s);  // warm-up
    CK(cudaEventRecord(e0, s));
    for (int i = 0; i < reps; ++i) patch_solve<T>(L.nitems, L.items, L.pdofs, L.inv, L.inv32, L.rbuf, L.b, L.x, L.max_patch, s);
    CK(cudaEventRecord(e1, s));
    check_launch("mg_time_patch_solve");
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&t, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  });
  if (ms) *ms = (double)t / reps;
  if (fma64) *fma64 = f64;
  if (fma32) *fma32 = f32;
  if (bytes) *bytes = 8.0 * f64 + 4.0 * f32;
  return MG_OK;
  API_END_H(h)
}

int mg_measure_fp64_fma(void* stream, double* fma_per_s) {
  mg_hierarchy* h = nullptr;
  API_BEGIN
  if (!fma_per_s) throw Error(MG_ERR_INVALID_ARG, "null output");
  cudaStream_t s = (cudaStream_t)stream;
  *fma_per_s = measure_fp64_fma(s);
  return MG_OK;
  API_END_H(h)
}

int64_t mg_device_bytes(const mg_hierarchy_t* h) { return h ? h->mem.bytes : 0; }

int mg_launch_counts(const mg_hierarchy_t* h, int32_t* per_vcycle, int32_t* per_iter) {
  if (!h) return MG_ERR_INVALID_ARG;
  if (per_vcycle) *per_vcycle = h->launches_vcycle;
  if (per_iter) *per_iter = h->launches_iter;
  return MG_OK;
}

}  // extern "C"
