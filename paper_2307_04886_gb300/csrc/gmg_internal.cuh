// Internal structures of libgmg (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdint>
#include <cstdlib>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gmg.h"
#include "gmg_fpbits.cuh"

namespace gmg {

constexpr int kSlice = 32;          // rows per sliced-ELL slice (one warp)
constexpr int kHashSlots = 1024;    // per-warp hash table of the Galerkin product
constexpr int kMaxRowEntries = 768; // Galerkin row limit (3/4 of the table)
constexpr int64_t kMaxCoarse = 8192;
constexpr int kRedBlocks = 608;     // fixed grid of the deterministic reductions (4 x 152 SMs)
constexpr int kMaxRhs = 16;
// Index of a multi-right-hand-side block width NR (1, 2, 4, 8, 16) in per-width tables.
constexpr int nr_index(int NR) { return NR == 1 ? 0 : NR == 2 ? 1 : NR == 4 ? 2 : NR == 8 ? 3 : 4; }

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

// Programmatic dependent launch: a kernel may start while its predecessor
// drains; `pdl_wait` blocks until the predecessor grid has completed and its
// writes are visible, `pdl_trigger` lets the successor start launching.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// GMG_NO_PDL=1 turns programmatic dependent launch off (plain stream order);
// g_pdl_suspended turns it off for the launches of the calling thread.
extern thread_local bool g_pdl_suspended;
inline bool use_pdl() {
  static const bool on = [] {
    const char* e = std::getenv("GMG_NO_PDL");
    return !(e && e[0] == '1');
  }();
  return on && !g_pdl_suspended;
}

// Launches `k` on `s` with programmatic stream serialisation.
template <typename... P, typename... A>
inline gmg_status launch(void (*k)(P...), int64_t grid, int block, cudaStream_t s, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)std::max<int64_t>(1, grid));
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = use_pdl() ? 1 : 0;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
  ++g_launches;
  if (e != cudaSuccess) {
    set_error(std::string("kernel launch: ") + cudaGetErrorString(e));
    return GMG_ERR_CUDA;
  }
  return GMG_OK;
}

// Device allocation registry of a handle: everything is freed by gmg_destroy.
// A named range on the host timeline of a profiler (NVTX; next to no cost
// when no tool is attached).  next() ends the current range and opens another.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  void next(const char* name) {
    nvtxRangePop();
    nvtxRangePushA(name);
  }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct Arena {
  std::vector<void*> ptrs;
  double ms_alloc = 0.0, ms_copy = 0.0;  // host time in cudaMalloc and in uploads (GMG_VERBOSE=1 reports it)
  int64_t n_alloc = 0;
  template <class T>
  gmg_status alloc(T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    const auto t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    ms_alloc += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    ++n_alloc;
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
  void release_one(void* p) {
    for (auto& q : ptrs)
      if (q == p) {
        cudaFree(q);
        q = ptrs.back();
        ptrs.pop_back();
        return;
      }
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
  int lanes = 1;   // warps sharing one row in Gauss-Seidel (1, 2, 4, 8)
  int mlanes[5] = {0, 0, 0, 0, 0};  // the same for the multi-right-hand-side kernels, by block width
                                    // NR = 1, 2, 4, 8, 16 (0: default by mean row length)
  int rlanes = 1;  // the same for the residual (all rows at once, so more parallel)
  std::vector<int64_t> color_off;        // host: first permuted row of each colour (+ end)
  std::vector<int64_t> color_slice_off;  // host: first slice of each colour (+ end)
  std::vector<int32_t> h_color;          // host: colour of every row (caller numbering)
  std::vector<int32_t> h_key;            // host: locality rank of every row (caller numbering)
  // numbering: perm[new] = old, iperm[old] = new
  int32_t* perm = nullptr;
  int32_t* iperm = nullptr;
  // Galerkin operator in caller numbering (CSR, FP64): source of all values
  int64_t* csr_rowptr = nullptr;
  int32_t* csr_col = nullptr;
  double* csr_val = nullptr;
  int64_t* csr2ell = nullptr;  // ELL slot of each CSR entry, or -1 - row for the diagonal (levels > 0)
  // Galerkin plan of this level (l > 0): terms of entry e are
  // plan_edge/plan_coef[plan_ptr[e] .. plan_ptr[e+1]) (CSR positions in level
  // l-1 and P_iJ P_jK), in canonical order; empty below the diagonal
  int64_t* plan_ptr = nullptr;
  int32_t* plan_edge = nullptr;
  double* plan_coef = nullptr;
  int64_t plan_terms = 0;
  // the same plan sliced for the numeric pass (entries with terms, sorted by
  // term count, 32 per slice, terms stored [k][lane], zero-padded)
  int64_t plan_nup = 0;
  int64_t plan_long_slices = 0;  // leading slices whose width exceeds 32 terms
  int32_t* plan_up = nullptr;
  int32_t* plan_mirror = nullptr;  // CSR position of each entry's mirror, -1 on the diagonal
  int64_t* plan_sptr = nullptr;
  int32_t* plan_sedge = nullptr;
  double* plan_scoef = nullptr;
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

// The tail of an FP32 V-cycle (the smoothed levels l0 .. lambda-1 and the
// coarsest level) runs as one launch on one thread-block cluster; these are
// its descriptors (passed by value).  Offsets are bytes into the dynamic
// shared memory of every CTA (the same layout in each).
constexpr int kMaxTail = 4;            // smoothed levels in the tail
constexpr int kTailSmemLimit = 227 * 1024;  // the largest dynamic shared memory of a CTA (no static shared memory)
struct TailLevel {
  int n, ncolor, nslice, r_nslice;
  int nc0;  // rows of colour 0 (the first rows in the colour-major numbering)
  // shared-memory copies: x, r, b, 1/a_ii, a_ii (all rows); per slice: first
  // row, rows, width, offset of its entries in the owner's arrays; colour
  // slice offsets; the owned slices' values and columns
  int o_x, o_r, o_b, o_dinv, o_diag, o_row0, o_nrow, o_width, o_soff, o_cso, o_own, o_val, o_col, o_ocs, o_mask;
  int maxown;             // owned slices per CTA (list padded with -1)
  const int32_t* own;     // ncta x maxown: each CTA's slices, colour by colour
  const int32_t* ocs;     // ncta x (ncolor + 1): where each colour starts in a CTA's list
  const uint16_t* mask;   // per row: the other CTAs that read its x (bit per CTA)
  const int64_t* a_ptr;
  const int32_t *a_row0, *a_nrow, *a_col;
  const float *a_v32, *dinv32, *diag32;
  const int32_t* soff;  // offset of each slice's entries in its owner CTA's arrays
  const int32_t* cso;   // first slice of every colour (+ end)
  // restriction into the next level (sliced ELL over its rows) and
  // prolongation from it (three slots per row of this level)
  const int64_t* r_ptr;
  const int32_t *r_row0, *r_nrow, *r_col;
  const float* r_v32;
  const int32_t* p_idx;
  const float* p_w32;
  float *x32, *b32;  // global vectors of this level (the first tail level reads x, b and writes x)
};
struct TailDesc {
  int ntail, nc, ncta;
  int nu_pre, nu_post, post_forward;
  int c0_first;          // colour 0 of the first pre-smoothing sweep is done by the restriction
  int o_xc, o_bc;        // shared-memory copies of the coarsest x and b
  const float* ainv32;   // coarsest inverse, FP32, nc x nc
  TailLevel lv[kMaxTail];
};

// A smoothed level whose FP32 sweeps, residual, restriction (one launch) and
// prolongation, sweeps (another) run on one thread-block cluster: the rows
// are split into ncta contiguous ranges of the caller's numbering (one per
// CTA, every colour balanced), each CTA keeps x of its rows and of their
// neighbours owned by other CTAs (the halo) in shared memory, an updated row
// is stored into the halo copies of the CTAs that read it, and the entries of
// the next phases' rows stream from L2 into shared memory while the current
// phase computes.  Per-CTA arrays are concatenated; *_off[cta] is a CTA's
// start in them.
constexpr int kClusterStagesMax = 4;  // entry buffers (the current phase and up to three ahead)
struct ClusterLevel {
  int l = 0, ncta = 0, threads = 0, ncolor = 0;
  int nu_pre = 0, nu_post = 0, post_forward = 0, c0_first = 0;
  int n_loc_max = 0, n_own_max = 0, nsl_max = 0, blk_max = 0;
  int nstage = 0, push_max = 0;
  // shared memory: x (own and halo rows), b (own rows), then the set-up image
  // [o_st, o_st + st_bytes) holding 1/a_ii, a_ii, the slice and colour
  // tables, the local-to-global rows and the halo stores (copied whole from
  // img + cta * st_bytes), then the barriers of the copies and the entry stages
  int o_x = 0, o_b = 0, o_st = 0, st_bytes = 0, o_dinv = 0, o_diag = 0, o_sl = 0, o_csl = 0, o_l2g = 0, o_pp = 0,
      o_pd = 0, o_mbar = 0, o_buf = 0, smem = 0;
  const char* img = nullptr;
  int* err = nullptr;  // set when a bounded wait for an entry block gave up
  const int32_t *n_own = nullptr, *n_loc = nullptr, *loc_off = nullptr, *loc2glob = nullptr;
  // slices of each CTA, colour by colour: first local row, rows, width, first
  // entry (relative to the CTA's entries); csl: first slice of every colour
  // (+ end), relative to the CTA's slices
  const int32_t *sl_off = nullptr, *sl_row0 = nullptr, *sl_nrow = nullptr, *sl_w = nullptr, *sl_eoff = nullptr;
  const int32_t* csl = nullptr;  // ncta x (ncolor + 1)
  const int64_t* ent_off = nullptr;
  const float* ent_val = nullptr;  // [k][lane] per slice; refreshed with the level's values
  const int32_t* ent_col = nullptr;  // local column
  // halo stores: for each own row, the (CTA << 16 | local index) copies to update
  const int32_t *push_off = nullptr, *push_ptr = nullptr, *push_dst = nullptr;
  // the level's global vectors and transfers
  float *x32 = nullptr, *b32 = nullptr, *r32 = nullptr;
  const float *dinv32 = nullptr, *diag32 = nullptr;
  const int32_t* p_idx = nullptr;
  const float* p_w32 = nullptr;
  const int64_t* r_ptr = nullptr;
  const int32_t *r_row0 = nullptr, *r_nrow = nullptr, *r_col = nullptr;
  const float* r_v32 = nullptr;
  int64_t r_nslice = 0;
  float *xc32 = nullptr, *bc32 = nullptr;  // next level's x and b
  const float* dinvc32 = nullptr;
  int64_t nc0 = 0;  // next level's colour-0 rows (their first update done by the restriction)
};

}  // namespace gmg

struct gmg_ctx {
  gmg_options opt{};
  int device = 0;
  int nlev = 0;
  double p_unity_dev = 0.0;  // largest |sum_k w_ik - 1| over the rows of every P_l
  std::vector<gmg::Level> L;
  gmg::Arena arena;
  // coarsest level
  int64_t nco = 0;
  double* dense = nullptr;  // npad x npad sweep work matrix (npad = n rounded up to 32)
  double* Ainv = nullptr;   // A_lambda^-1 (symmetric, full, n x n)
  double* dbuf = nullptr;   // two 32 x 32 pivot inverses, panel U and U D^-1 (npad x 32 each)
  int* gj_cnt = nullptr;    // per sweep: arrival counter of the next pivot tile, then work counter
  int nsm = 1;              // SMs of the device (persistent grids)
  // A(t) = M + t L kept split (gmg_setup_ML): lumped mass, L values (caller
  // CSR order), position of every row's diagonal entry
  double* ml_M = nullptr;
  double* ml_L = nullptr;
  int64_t* ml_dpos = nullptr;
  double ml_t = 0.0;
  // FP32 cycles run levels >= tail_l0 as one cluster launch (0 = off)
  int tail_l0 = 0;
  int tail_smem = 0;
  int tail_threads = 1024;
  gmg::TailDesc tail{};
  // FP32 cycles run level clev.l (0 = none) as two cluster launches
  gmg::ClusterLevel clev{};
  int64_t* clev_src = nullptr;  // ELL slot of every cluster-level entry (-1: padding)
  int64_t clev_nent = 0;
  float* Ainv32 = nullptr;  // coarsest inverse in FP32 for the tail launch
  int* dstatus = nullptr;   // device status words
  // outer iteration (finest level, permuted numbering, FP64)
  double *xs = nullptr, *bs = nullptr, *rs = nullptr, *zs = nullptr, *ps = nullptr, *qs = nullptr, *ros = nullptr;
  double* io = nullptr;    // n x kMaxRhs staging for caller-numbered vectors
  double* io2 = nullptr;
  double* XS = nullptr;    // batched FP64 iterate [n x kMaxRhs]
  double* RS = nullptr;    // batched FP64 residual
  double* BS = nullptr;
  double* red = nullptr;   // reduction partials
  int64_t red_cap = 0;     // capacity of `red` in doubles
  int* red_cnt = nullptr;  // arrival counters of the fused last-block reductions (zero between launches)
  double* scal = nullptr;  // device scalars (norms, dots)
  double* h_scal = nullptr;  // pinned host mirror
  // captured iteration bodies, indexed by mode * 2 + segment
  cudaGraphExec_t graphs[8] = {};
  uint64_t graph_kernels[8] = {};  // kernel nodes of each captured graph
  // device-side outer loop per mode: a graph whose conditional WHILE node
  // repeats the iteration until the convergence test fails on the device
  cudaGraphExec_t loops[4] = {};
  uint64_t loop_kernels[4] = {};  // kernel nodes of one loop iteration
  bool loop_refused[4] = {};      // instantiation failed: the host loop serves the mode
  bool loop_pdl[4] = {};          // the loop body kept its programmatic launch edges
  int* dloop = nullptr;           // device iteration counter, iteration limit
  double* dhist = nullptr;        // relative residual per iteration (max_iter + 1)
  cudaStream_t g_stream = nullptr;
  bool values_ready = false;
  // the coarsest inverse of a numeric refresh runs on its own stream while the
  // caller's next work starts; ev_inv marks its end, and until a call joins it
  // (inv_pending) nothing may read the inverse; its pivot check is read at the
  // join (inv_check)
  cudaStream_t inv_stream = nullptr;
  cudaEvent_t ev_gal = nullptr, ev_inv = nullptr;
  bool inv_pending = false, inv_check = false;
  // kernel timing: events bracket the finest level's smoothing blocks
  // (0-1 pre, 2-3 post) and the whole cycle (4-5)
  bool prof = false;
  bool prof_pending = false;
  cudaEvent_t ev[6] = {};
  double prof_acc[4] = {0, 0, 0, 0};  // smoothing ms, GS launches, cycle ms, cycles
  int prof_gs = 0;                    // finest-level GS launches of the last timed cycle
  // per-level timing of the same cycles: six events per level (before and
  // after pre-smoothing, after the restriction, after the coarser levels,
  // after the prolongation, after post-smoothing); levels run inside the
  // cluster tail or as the coarsest solve record only the first and last
  std::vector<cudaEvent_t> lev_ev;
  std::vector<int> lev_kind;    // per level: 0 not recorded, 1 all six events, 2 first and last only
  std::vector<int> lev_gs;      // GS launches of the level in the last timed cycle
  std::vector<double> lev_acc;  // per level: smoothing ms, GS launches, transfer ms, whole-level ms
};

namespace gmg {
// Makes `s` wait for a coarsest inverse still running on its own stream; with
// `check` also reads its pivot check (host synchronisation).
gmg_status join_inverse(gmg_ctx* c, cudaStream_t s, bool check);
// Reads the pivot check of a joined inverse once (GMG_ERR_CHOLESKY on failure).
gmg_status inverse_status(gmg_ctx* c, cudaStream_t s);
// Whether a tail cluster of ncta CTAs with `smem` bytes of shared memory each
// can be scheduled on the device (sets the kernel's attributes).
gmg_status tail_configure(gmg_ctx* c, int ncta, int threads, int smem, bool* ok);
// Cluster form of one smoothed level of the FP32 cycle (gmg_clevel.cu): the
// tables from the level's pattern and numberings (host), the entry values
// after a numeric set-up, and the two launches (mode 0: pre-smoothing,
// residual, restriction; mode 1: prolongation, post-smoothing).
gmg_status build_cluster_level(gmg_ctx* c, int l, const int64_t* rp, const int32_t* ci,
                               const std::vector<int32_t>& perm, const std::vector<int32_t>& iperm);
gmg_status refresh_cluster_values(gmg_ctx* c, cudaStream_t s);
gmg_status launch_cluster_level(gmg_ctx* c, int mode, cudaStream_t s);
gmg_status cluster_level_status(gmg_ctx* c, cudaStream_t s);
}  // namespace gmg
