// Allocation-free dense symmetric matrix-vector product (the coarsest-level direct solve).
//
// Some callers cannot allocate device memory at the point where they need this product:
// code that runs while all device memory has been handed to another allocator up front
// (a framework's pre-reserved pool, a multi-tenant service that forbids allocation after
// start-up), or code on a latency-critical path where a cudaMalloc/cudaFree would stall
// or implicitly synchronise the device. mg_dense_symv_static computes x = X b with the
// same split-K kernel as the coarsest-level solve, but keeps the kernel's partial sums in
// a file-scope device array instead of memory the library or the caller allocates.
//
// The array (kStaticPartials doubles, 8 MiB) lives in every device that loads this library
// until the process exits. Its device address is looked up once per device, with that
// device current, on the first call made there; that first call should therefore come
// before any stream capture. Every call shares the array: the kernel writes each partial
// before reading it, so nothing needs clearing, but two calls whose kernels overlap on the
// GPU (different streams, or different host threads) race on it.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "internal.hpp"
#include "kernels.cuh"

namespace nnmg {
namespace {

constexpr int64_t kStaticPartials = int64_t(1) << 20;   // doubles (8 MiB)
constexpr int kStaticMaxChunk = 4096;                   // columns per split-K chunk (32 KiB of shared memory)
constexpr int64_t kStaticMaxN = int64_t(1) << 16;       // largest n: 16 chunks of 4096 columns
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_static_partials[kStaticPartials];

std::mutex g_static_mu;
double* g_static_addr[kMaxDevices] = {};

// Device address of the static array on the current device (looked up once per device).
double* static_partials(int* code) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    *code = MG_ERR_CUDA;
    set_last_error("mg_dense_symv_static: no current CUDA device");
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_partials);
    if (e != cudaSuccess) {
      *code = MG_ERR_CUDA;
      set_last_error(std::string("mg_dense_symv_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return nullptr;
    }
    g_static_addr[dev] = static_cast<double*>(p);
  }
  *code = MG_OK;
  return g_static_addr[dev];
}

}  // namespace
}  // namespace nnmg

extern "C" {

int mg_dense_symv_static(const double* X, int64_t n, const double* b, double* x, void* stream) {
  using namespace nnmg;
  if (!X || !b || !x || n < 1) {
    set_last_error("mg_dense_symv_static: null pointer or n < 1");
    return MG_ERR_INVALID_ARG;
  }
  if (n > kStaticMaxN) {
    set_last_error("mg_dense_symv_static: n = " + std::to_string(n) + " exceeds the limit n <= " +
                   std::to_string(kStaticMaxN) + " of the static scratch (2^20 partial sums)");
    return MG_ERR_INVALID_ARG;
  }
  // split-K: about four blocks per SM (152 SMs) from the row blocks times the chunks, then
  // at least ceil(n / kStaticMaxChunk) chunks so that no chunk exceeds kStaticMaxChunk
  // columns; nchunks partial vectors of length n must fit the static array. For
  // n <= kStaticMaxN = 2^16 the second rule gives at most 16 chunks, so n * nchunks <= 2^20.
  const int64_t rowblocks = (n + kBlock - 1) / kBlock;
  int64_t nchunks = std::max<int64_t>(1, (4 * 152 + rowblocks - 1) / rowblocks);
  nchunks = std::min<int64_t>(nchunks, kStaticPartials / n);
  nchunks = std::max<int64_t>(nchunks, (n + kStaticMaxChunk - 1) / kStaticMaxChunk);
  const int64_t kchunk = ((n + nchunks - 1) / nchunks + 31) / 32 * 32;
  const int64_t used = n * dense_chunks((int)n, (int)kchunk);
  if (used > kStaticPartials || kchunk > kStaticMaxChunk) {  // unreachable for n <= kStaticMaxN
    set_last_error("mg_dense_symv_static: internal chunking error for n = " + std::to_string(n));
    return MG_ERR_INVALID_ARG;
  }
  int code = MG_OK;
  double* part = static_partials(&code);
  if (!part) return code;
  // the status of this call's own launches (not a sticky error left by an earlier call)
  cudaError_t e = dense_solve<double>((int)n, X, b, x, part, (int)kchunk, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    set_last_error(std::string("mg_dense_symv_static: ") + cudaGetErrorString(e));
    return MG_ERR_CUDA;
  }
  return MG_OK;
}

}  // extern "C"
