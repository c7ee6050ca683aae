// Internal structures of libgmg (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "gmg.h"

namespace gmg {

constexpr int kSlice = 32;          // rows per sliced-ELL slice (one warp)
constexpr int kHashSlots = 1024;    // per-warp hash table of the Galerkin product
constexpr int kMaxRowEntries = 768; // Galerkin row limit (3/4 of the table)
constexpr int64_t kMaxCoarse = 8192;
constexpr int kRedBlocks = 608;     // fixed grid of the deterministic reductions (4 x 152 SMs)
constexpr int kMaxRhs = 16;

void set_error(const std::string& msg);

// Kernels launched by this library on the calling thread (graph replays add
// the number of kernel nodes captured in the graph).
extern thread_local uint64_t g_launches;

#define GMG_LAUNCHED()                                                                    \
  do {                                                                                    \
    ++::gmg::g_launches;                                                                  \
    cudaError_t e_ = cudaGetLastError();                                                  \
    if (e_ != cudaSuccess) {                                                              \
      ::gmg::set_error(std::string("kernel launch: ") + cudaGetErrorString(e_));          \
      return GMG_ERR_CUDA;                                                                \
    }                                                                                     \
  } while (0)

#define GMG_CK(call)                                                                      \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      ::gmg::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));               \
      return e_ == cudaErrorMemoryAllocation ? GMG_ERR_OOM : GMG_ERR_CUDA;                \
    }                                                                                     \
  } while (0)

#define GMG_TRY(call)                     \
  do {                                    \
    gmg_status s_ = (call);               \
    if (s_ != GMG_OK) return s_;          \
  } while (0)

// Device allocation registry of a handle: everything is freed by gmg_destroy.
struct Arena {
  std::vector<void*> ptrs;
  template <class T>
  gmg_status alloc(T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e != cudaSuccess) {
      set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
      return GMG_ERR_OOM;
    }
    ptrs.push_back(*p);
    return GMG_OK;
  }
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
  }
};

// A sliced-ELL matrix: rows grouped in slices of 32 consecutive rows; slice s
// stores width_s columns as [k][lane] (entry (row0_s + lane, k) at
// ptr[s] + k * 32 + lane), so a warp's loads of one k are contiguous.
// Padding entries carry weight 0 and a valid column.
struct Ell {
  int64_t nslice = 0, entries = 0;
  int64_t* ptr = nullptr;     // nslice + 1 entry offsets
  int32_t* row0 = nullptr;    // first row of each slice
  int32_t* nrow = nullptr;    // rows in each slice (<= 32)
  int32_t* col = nullptr;
  double* v64 = nullptr;
  float* v32 = nullptr;
};

struct Level {
  int64_t n = 0, nnz = 0;
  int ncolor = 0;
  int lanes = 1;  // warps sharing one row in Gauss-Seidel / residual (1, 2, 4, 8)
  std::vector<int64_t> color_off;        // host: first permuted row of each colour (+ end)
  std::vector<int64_t> color_slice_off;  // host: first slice of each colour (+ end)
  std::vector<int32_t> h_color;          // host: colour of every row (caller numbering)
  // numbering: perm[new] = old, iperm[old] = new
  int32_t* perm = nullptr;
  int32_t* iperm = nullptr;
  // Galerkin operator in caller numbering (CSR, FP64): source of all values
  int64_t* csr_rowptr = nullptr;
  int32_t* csr_col = nullptr;
  double* csr_val = nullptr;
  int64_t* csr2ell = nullptr;  // ELL slot of each CSR entry, or -1 - row for the diagonal
  // Galerkin plan of this level (l > 0): terms of entry e are
  // plan_edge/plan_coef[plan_ptr[e] .. plan_ptr[e+1]) (CSR positions in level
  // l-1 and P_iJ P_jK), in canonical order; empty below the diagonal
  int64_t* plan_ptr = nullptr;
  int32_t* plan_edge = nullptr;
  double* plan_coef = nullptr;
  int64_t plan_terms = 0;
  // off-diagonal part of A_l in the permuted numbering
  Ell A;
  double* diag64 = nullptr;
  double* dinv64 = nullptr;
  float* diag32 = nullptr;
  float* dinv32 = nullptr;
  // prolongation P_l to the next level, caller numbering (Galerkin product input)
  int64_t nc = 0;
  int32_t* p_idx_o = nullptr;
  double* p_w_o = nullptr;
  int64_t* pt_rowptr_o = nullptr;  // columns of P_l (caller numbering)
  int32_t* pt_col_o = nullptr;
  double* pt_w_o = nullptr;
  // prolongation in the permuted numbering of both levels
  int32_t* p_idx = nullptr;
  double* p_w64 = nullptr;
  float* p_w32 = nullptr;
  // restriction P_l^T as sliced ELL over the next level's permuted rows
  Ell R;
  // work vectors (permuted numbering); batched forms use nrhs columns
  double *x64 = nullptr, *b64 = nullptr, *r64 = nullptr;
  float *x32 = nullptr, *b32 = nullptr, *r32 = nullptr;
  float *X32 = nullptr, *B32 = nullptr, *R32 = nullptr;  // [n x kMaxRhs]
};

// Device-side descriptor of a level for the persistent small-level kernel.
constexpr int kClusterCTAs = 8;              // CTAs of the small-level cluster
constexpr int64_t kClusterMaxRows = 65536;   // levels this small run inside it
struct DevLevel {
  int64_t n;
  int ncolor, lanes;
  const int64_t* cso;  // first slice of every colour (+ end)
  int64_t nslice;
  const int64_t* a_ptr;
  const int32_t *a_row0, *a_nrow, *a_col;
  const float* a_v32;
  const double* a_v64;
  const float *dinv32, *diag32;
  const double *dinv64, *diag64;
  int64_t r_nslice;
  const int64_t* r_ptr;
  const int32_t *r_row0, *r_nrow, *r_col;
  const float* r_v32;
  const double* r_v64;
  const int32_t* p_idx;
  const float* p_w32;
  const double* p_w64;
  float *x32, *b32, *r32;
  double *x64, *b64, *r64;
};

}  // namespace gmg

struct gmg_ctx {
  gmg_options opt{};
  int device = 0;
  int nlev = 0;
  std::vector<gmg::Level> L;
  gmg::Arena arena;
  // coarsest level
  int64_t nco = 0;
  double* dense = nullptr;  // n x n work / Cholesky factor
  double* Winv = nullptr;   // L^-1
  double* Ainv = nullptr;   // A_lambda^-1 (symmetric, full)
  double* dbuf = nullptr;   // diagonal factor blocks, then 1 / L_ii
  // A(t) = M + t L kept split (gmg_setup_ML): lumped mass, L values (caller
  // CSR order), position of every row's diagonal entry
  double* ml_M = nullptr;
  double* ml_L = nullptr;
  int64_t* ml_dpos = nullptr;
  double ml_t = 0.0;
  // small levels l >= cluster_l0 run in one cluster kernel (0 = disabled)
  int cluster_l0 = 0;
  gmg::DevLevel* dlv = nullptr;
  int* dstatus = nullptr;   // device status words
  // outer iteration (finest level, permuted numbering, FP64)
  double *xs = nullptr, *bs = nullptr, *rs = nullptr, *zs = nullptr, *ps = nullptr, *qs = nullptr, *ros = nullptr;
  double* io = nullptr;    // n x kMaxRhs staging for caller-numbered vectors
  double* io2 = nullptr;
  double* XS = nullptr;    // batched FP64 iterate [n x kMaxRhs]
  double* RS = nullptr;    // batched FP64 residual
  double* BS = nullptr;
  double* red = nullptr;   // reduction partials
  double* scal = nullptr;  // device scalars (norms, dots)
  double* h_scal = nullptr;  // pinned host mirror
  // captured iteration bodies, indexed by mode * 2 + segment
  cudaGraphExec_t graphs[8] = {};
  uint64_t graph_kernels[8] = {};  // kernel nodes of each captured graph
  cudaStream_t g_stream = nullptr;
  bool values_ready = false;
  // kernel timing: events bracket the finest level's smoothing blocks
  // (0-1 pre, 2-3 post) and the whole cycle (4-5)
  bool prof = false;
  bool prof_pending = false;
  cudaEvent_t ev[6] = {};
  double prof_acc[4] = {0, 0, 0, 0};  // smoothing ms, GS launches, cycle ms, cycles
};
