// Allocation-free residual and norms for callers that cannot allocate device
// memory: code running inside another framework's memory pool, or under a
// custom allocator that forbids cudaMalloc, or where an allocation would
// synchronise the device.  It is the FP64 residual-with-norm of the outer
// iteration (r = b - A x plus a fixed-order reduction of squares) in a
// stand-alone form on caller-owned CSR data; the block partial sums live in a
// file-scope device array instead of a library allocation.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "gmg_internal.cuh"

namespace gmg {

constexpr int kNoAllocBlock = 256;                 // rows per block
constexpr int64_t kNoAllocMaxBlocks = 65536;       // partials capacity
constexpr int64_t kNoAllocMaxRows = kNoAllocMaxBlocks * kNoAllocBlock;  // 16,777,216

// Two partial sums (r^2, b^2) per block: 1 MiB, held by every device that
// loads the library until the process exits.
static __device__ __align__(256) double g_noalloc_partials[2 * kNoAllocMaxBlocks];

// r = b - A x row by row, and per-block sums of r^2 and b^2 (fixed tree).
__global__ void __launch_bounds__(kNoAllocBlock)
    k_noalloc_residual(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                       const double* __restrict__ val, const double* __restrict__ x, const double* __restrict__ b,
                       double* __restrict__ r, double* __restrict__ partials) {
  __shared__ double sr[kNoAllocBlock], sb[kNoAllocBlock];
  const int64_t i = (int64_t)blockIdx.x * kNoAllocBlock + threadIdx.x;
  double rr = 0.0, bb = 0.0;
  if (i < n) {
    double acc = 0.0;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) acc += val[k] * x[col[k]];
    const double bi = b[i];
    const double ri = bi - acc;
    r[i] = ri;
    rr = ri * ri;
    bb = bi * bi;
  }
  sr[threadIdx.x] = rr;
  sb[threadIdx.x] = bb;
  __syncthreads();
  for (int o = kNoAllocBlock / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sr[threadIdx.x] += sr[threadIdx.x + o];
      sb[threadIdx.x] += sb[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = sr[0];
    partials[2 * blockIdx.x + 1] = sb[0];
  }
}

// norms = (||r||_2, ||b||_2) from the block partials, summed in a fixed order.
__global__ void __launch_bounds__(256) k_noalloc_finish(int nblocks, const double* __restrict__ partials,
                                                        double* __restrict__ norms) {
  __shared__ double sr[256], sb[256];
  double rr = 0.0, bb = 0.0;
  for (int k = threadIdx.x; k < nblocks; k += 256) {
    rr += partials[2 * k];
    bb += partials[2 * k + 1];
  }
  sr[threadIdx.x] = rr;
  sb[threadIdx.x] = bb;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sr[threadIdx.x] += sr[threadIdx.x + o];
      sb[threadIdx.x] += sb[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    norms[0] = sqrt(sr[0]);
    norms[1] = sqrt(sb[0]);
  }
}

// Device address of the partials array, looked up once per device context
// (with that device current) and cached.  The cache is keyed on the CUDA
// context current at the call as well as the device index: after
// cudaDeviceReset the device gets a new primary context in which the
// library's module (and the array) is loaded again at a new address, so the
// first call in the new context looks the address up afresh.
constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[kMaxDevices] = {};
static void* g_noalloc_ctx[kMaxDevices] = {};

// The current context through the driver's cuCtxGetCurrent, reached via the
// runtime (the library does not link the driver library directly); NULL when
// no context is current on the calling thread or the query is unavailable.
static void* current_context() {
  typedef int (*ctx_get_fn)(void**);
  static ctx_get_fn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    const bool ok = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                        cudaSuccess &&
                    q == cudaDriverEntryPointSuccess;
    cudaGetLastError();
    return ok ? (ctx_get_fn)f : (ctx_get_fn) nullptr;
  }();
  void* ctx = nullptr;
  if (!fn || fn(&ctx) != 0) return nullptr;
  return ctx;
}

static gmg_status noalloc_scratch(double** out) {
  int dev = 0;
  GMG_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("gmg_residual_norm_noalloc: device index beyond " + std::to_string(kMaxDevices));
    return GMG_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  void* ctx = current_context();
  // Without a known context (none current yet, or the query is unavailable)
  // the address is looked up on every call: still correct, only slower.
  if (!ctx || !g_noalloc_ptr[dev] || g_noalloc_ctx[dev] != ctx) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);  // makes the primary context current
    if (e != cudaSuccess || !p) {
      set_error(std::string("gmg_residual_norm_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return GMG_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = (double*)p;
    g_noalloc_ctx[dev] = current_context();
  }
  *out = g_noalloc_ptr[dev];
  return GMG_OK;
}

}  // namespace gmg

using namespace gmg;

extern "C" gmg_status gmg_residual_norm_noalloc(int64_t n, const int64_t* rowptr, const int32_t* col,
                                                const double* val, const double* x, const double* b, double* r,
                                                double* norms, void* stream) {
  if (n < 0 || (n > 0 && (!rowptr || !col || !val || !x || !b || !r)) || !norms) {
    set_error("gmg_residual_norm_noalloc: negative size or null pointer");
    return GMG_ERR_INVALID_ARG;
  }
  if (n > kNoAllocMaxRows) {
    set_error("gmg_residual_norm_noalloc: n = " + std::to_string(n) + " exceeds the limit of " +
              std::to_string(kNoAllocMaxRows) + " rows of the static scratch array");
    return GMG_ERR_TOO_LARGE;
  }
  double* partials = nullptr;
  GMG_TRY(noalloc_scratch(&partials));
  cudaStream_t s = (cudaStream_t)stream;
  const int nblocks = (int)((n + kNoAllocBlock - 1) / kNoAllocBlock);
  if (nblocks > 0) {
    k_noalloc_residual<<<nblocks, kNoAllocBlock, 0, s>>>(n, rowptr, col, val, x, b, r, partials);
    GMG_LAUNCHED();
  }
  k_noalloc_finish<<<1, 256, 0, s>>>(nblocks, partials, norms);
  GMG_LAUNCHED();
  return GMG_OK;
}
