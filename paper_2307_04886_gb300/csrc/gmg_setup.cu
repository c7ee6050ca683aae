// Setup of the multigrid hierarchy (the level-matrix steps of Alg. 1):
//  * validation of A and P_l (host);
//  * Galerkin product A_{l+1} = P_l^T A_l P_l on the GPU: a symbolic pass
//    (per-row hash sets in shared memory: count, scan, sorted fill) and a
//    numeric pass with a fixed accumulation order, then mirrored to exact
//    symmetry (the entry below the diagonal takes the value above it);
//  * colouring (two greedy colourings improved by iterated greedy, the one
//    with fewer colours kept) and colour-major renumbering (host, integer work);
//  * sliced-ELL layout of every level and of every restriction P_l^T;
//  * explicit FP64 inverse of the coarsest level (the direct solve of
//    Alg. 2 at the coarsest level) by block sweeps.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "gmg_internal.cuh"

namespace gmg {

thread_local std::string g_last_error;
thread_local uint64_t g_launches = 0;
thread_local bool g_pdl_suspended = false;
void set_error(const std::string& msg) { g_last_error = msg; }

// ------------------------------------------------------------------ device

__device__ __forceinline__ unsigned slot_of(int32_t key) {
  return ((unsigned)key * 2654435761u) >> (32 - 10);  // kHashSlots = 1024
}
static_assert(kHashSlots == 1024, "slot_of assumes 1024 slots");

// Returns 1 when `key` was added, 0 when present, -1 when the table is full.
__device__ __forceinline__ int hash_insert(int32_t* tab, int32_t key) {
  unsigned h = slot_of(key);
  for (int probe = 0; probe < kHashSlots; ++probe) {
    int32_t prev = atomicCAS(&tab[h], -1, key);
    if (prev == -1) return 1;
    if (prev == key) return 0;
    h = (h + 1) & (kHashSlots - 1);
  }
  return -1;
}

__device__ __forceinline__ int hash_find(const int32_t* tab, int32_t key) {
  unsigned h = slot_of(key);
  for (int probe = 0; probe < kHashSlots; ++probe) {
    int32_t v = tab[h];
    if (v == key) return (int)h;
    if (v == -1) return -1;
    h = (h + 1) & (kHashSlots - 1);
  }
  return -1;
}

__device__ __forceinline__ int warp_sum_i(int v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Inserts every coarse column K reachable from coarse row J: the slots of
// P row j for every entry j of A row i, for every fine row i of column J of P.
// Returns the number of keys this lane added; sets *full when the table
// overflowed.
__device__ int insert_row_keys(int32_t* tab, int64_t J, const int64_t* __restrict__ pt_rp,
                               const int32_t* __restrict__ pt_col, const int64_t* __restrict__ a_rp,
                               const int32_t* __restrict__ a_col, const int32_t* __restrict__ p_idx,
                               const double* __restrict__ p_w, bool* full) {
  const int lane = threadIdx.x & 31;
  int cnt = 0;
  for (int64_t q = pt_rp[J]; q < pt_rp[J + 1]; ++q) {
    const int32_t i = pt_col[q];
    for (int64_t k = a_rp[i] + lane; k < a_rp[i + 1]; k += 32) {
      const int64_t j = a_col[k];
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        if (p_w[3 * j + m] != 0.0) {
          int r = hash_insert(tab, p_idx[3 * j + m]);
          if (r > 0) ++cnt;
          else if (r < 0) *full = true;
        }
      }
    }
  }
  return cnt;
}

constexpr int kCountWarps = 8;
__global__ void k_gal_count(int64_t nc, const int64_t* __restrict__ pt_rp, const int32_t* __restrict__ pt_col,
                            const int64_t* __restrict__ a_rp, const int32_t* __restrict__ a_col,
                            const int32_t* __restrict__ p_idx, const double* __restrict__ p_w,
                            int64_t* __restrict__ counts, int* __restrict__ err) {
  __shared__ int32_t tab_all[kCountWarps][kHashSlots];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* tab = tab_all[warp];
  for (int64_t J = (int64_t)blockIdx.x * kCountWarps + warp; J < nc; J += (int64_t)gridDim.x * kCountWarps) {
    for (int s = lane; s < kHashSlots; s += 32) tab[s] = -1;
    __syncwarp();
    bool full = false;
    int cnt = insert_row_keys(tab, J, pt_rp, pt_col, a_rp, a_col, p_idx, p_w, &full);
    cnt = warp_sum_i(cnt);
    full = __any_sync(0xffffffffu, full);
    if (lane == 0) {
      counts[J] = cnt;
      if (full || cnt > kMaxRowEntries) atomicOr(err, 1);
    }
    __syncwarp();
  }
}

// Exclusive scan of n counts into rp[0..n] (one block of 1024 threads).
__global__ void k_scan_counts(int64_t n, const int64_t* __restrict__ cnt, int64_t* __restrict__ rp) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x;
  const int64_t chunk = (n + 1023) / 1024;
  const int64_t b = t * chunk, e = b + chunk < n ? b + chunk : n;
  int64_t s = 0;
  for (int64_t i = b; i < e; ++i) s += cnt[i];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int64_t acc = 0;
    for (int k = 0; k < 1024; ++k) {
      int64_t v = part[k];
      part[k] = acc;
      acc += v;
    }
    rp[n] = acc;
  }
  __syncthreads();
  int64_t acc = part[t];
  for (int64_t i = b; i < e; ++i) {
    rp[i] = acc;
    acc += cnt[i];
  }
}

constexpr int kFillWarps = 4;
__global__ void k_gal_fill(int64_t nc, const int64_t* __restrict__ pt_rp, const int32_t* __restrict__ pt_col,
                           const int64_t* __restrict__ a_rp, const int32_t* __restrict__ a_col,
                           const int32_t* __restrict__ p_idx, const double* __restrict__ p_w,
                           const int64_t* __restrict__ c_rp, int32_t* __restrict__ c_col) {
  __shared__ int32_t tab_all[kFillWarps][kHashSlots];
  __shared__ int32_t lst_all[kFillWarps][kMaxRowEntries];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* tab = tab_all[warp];
  int32_t* lst = lst_all[warp];
  for (int64_t J = (int64_t)blockIdx.x * kFillWarps + warp; J < nc; J += (int64_t)gridDim.x * kFillWarps) {
    for (int s = lane; s < kHashSlots; s += 32) tab[s] = -1;
    __syncwarp();
    bool full = false;
    insert_row_keys(tab, J, pt_rp, pt_col, a_rp, a_col, p_idx, p_w, &full);
    __syncwarp();
    int base = 0;
    for (int s0 = 0; s0 < kHashSlots; s0 += 32) {
      const int32_t key = tab[s0 + lane];
      const unsigned m = __ballot_sync(0xffffffffu, key != -1);
      const int pos = base + __popc(m & ((1u << lane) - 1u));
      if (key != -1 && pos < kMaxRowEntries) lst[pos] = key;
      base += __popc(m);
    }
    if (base > kMaxRowEntries) base = kMaxRowEntries;  // flagged by the count pass
    __syncwarp();
    const int64_t out = c_rp[J];
    const int64_t len = c_rp[J + 1] - out;
    for (int a = lane; a < base; a += 32) {
      const int32_t key = lst[a];
      int rank = 0;
      for (int b2 = 0; b2 < base; ++b2) rank += lst[b2] < key;
      if (rank < len) c_col[out + rank] = key;
    }
    __syncwarp();
  }
}

// Galerkin product plan.  For coarse row J the terms (P_iJ P_jK) A_ij of
// A_{l+1} = P_l^T A_l P_l are enumerated in a canonical order: i ascending in
// column J of P, j ascending in row i of A, slot order of row j of P.  The
// symbolic pass records, for every entry (J, K) with K >= J, its terms in
// that order as (position of A_ij in A_l's CSR, coefficient P_iJ P_jK);
// entries below the diagonal take the mirrored value.  The numeric pass is
// then one FP64 gather-dot per entry, summed in plan order.
constexpr int kPlanWarps = 4;
constexpr int kPlanChunk = 510;  // terms staged per pass (3 per (i, j) pair)
constexpr int kSegQ = 256;       // entries of column J of P handled per segment
struct alignas(16) PlanSmem {
  double fw[kSegQ];
  int64_t fk[kSegQ];
  double pc[kPlanChunk];
  int32_t pe[kPlanChunk];
  int32_t tab[kHashSlots];
  int32_t off[kSegQ + 1];
  int32_t fill[kMaxRowEntries];
  int32_t cnt[32];
  int16_t tpos[kHashSlots];
  int16_t ps[kPlanChunk];
  int16_t list[kPlanChunk];
};

// Loads row J's sorted columns into the hash table (slot -> position).
__device__ void plan_row_table(PlanSmem& S, int64_t r0, int64_t r1, const int32_t* __restrict__ c_col) {
  const int lane = threadIdx.x & 31;
  for (int s = lane; s < kHashSlots; s += 32) S.tab[s] = -1;
  __syncwarp();
  for (int64_t a = r0 + lane; a < r1; a += 32) {
    const int32_t K = c_col[a];
    hash_insert(S.tab, K);
  }
  __syncwarp();
  for (int64_t a = r0 + lane; a < r1; a += 32) S.tpos[hash_find(S.tab, c_col[a])] = (int16_t)(a - r0);
  __syncwarp();
}

// Fine rows, weights, row starts and pair offsets of one segment of column J
// of P; returns the number of (i, j) pairs.
__device__ int plan_segment(PlanSmem& S, int64_t seg, int nq, const int32_t* __restrict__ pt_col,
                            const double* __restrict__ pt_w, const int64_t* __restrict__ a_rp) {
  const int lane = threadIdx.x & 31;
  int carry = 0;
  for (int q0 = 0; q0 < nq; q0 += 32) {
    const int q = q0 + lane;
    int len = 0;
    if (q < nq) {
      const int32_t i = pt_col[seg + q];
      S.fw[q] = pt_w[seg + q];
      S.fk[q] = a_rp[i];
      len = (int)(a_rp[i + 1] - a_rp[i]);
    }
    int incl = len;
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (q < nq) S.off[q + 1] = carry + incl;
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) S.off[0] = 0;
  __syncwarp();
  return carry;
}

// Terms of pairs [t0, t0 + np) of the segment: position of (J, K) in row J
// (-1 when P_jK = 0 or K < J), CSR position of A_ij and P_iJ P_jK.
__device__ void plan_stage(PlanSmem& S, int64_t J, int nq, int t0, int np, const int32_t* __restrict__ a_col,
                           const int32_t* __restrict__ p_idx, const double* __restrict__ p_w) {
  const int lane = threadIdx.x & 31;
  for (int tt = lane; tt < np; tt += 32) {
    const int t = t0 + tt;
    int lo = 0, hi = nq - 1;  // last q with off[q] <= t
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (S.off[mid] <= t) lo = mid;
      else hi = mid - 1;
    }
    const int64_t k = S.fk[lo] + (t - S.off[lo]);
    const int64_t j = a_col[k];
    const double wi = S.fw[lo];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const double w = p_w[3 * j + m];
      const int32_t K = p_idx[3 * j + m];
      int pos = -1;
      if (w != 0.0 && K >= J) pos = S.tpos[hash_find(S.tab, K)];
      S.ps[3 * tt + m] = (int16_t)pos;
      S.pe[3 * tt + m] = (int32_t)k;
      S.pc[3 * tt + m] = __dmul_rn(wi, w);
    }
  }
  __syncwarp();
}

// Symbolic pass 1: number of terms of every entry (J, K), K >= J.
__global__ void __launch_bounds__(kPlanWarps * 32)
    k_gal_plan_count(int64_t nc, const int64_t* __restrict__ pt_rp, const int32_t* __restrict__ pt_col,
                     const double* __restrict__ pt_w, const int64_t* __restrict__ a_rp,
                     const int32_t* __restrict__ a_col, const int32_t* __restrict__ p_idx,
                     const double* __restrict__ p_w, const int64_t* __restrict__ c_rp,
                     const int32_t* __restrict__ c_col, int64_t* __restrict__ terms) {
  extern __shared__ unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  PlanSmem& S = reinterpret_cast<PlanSmem*>(smem_raw)[warp];
  for (int64_t J = (int64_t)blockIdx.x * kPlanWarps + warp; J < nc; J += (int64_t)gridDim.x * kPlanWarps) {
    const int64_t r0 = c_rp[J], r1 = c_rp[J + 1];
    const int len = (int)(r1 - r0);
    plan_row_table(S, r0, r1, c_col);
    for (int a = lane; a < len; a += 32) S.fill[a] = 0;
    __syncwarp();
    for (int64_t seg = pt_rp[J]; seg < pt_rp[J + 1]; seg += kSegQ) {
      const int64_t left = pt_rp[J + 1] - seg;
      const int nq = left < kSegQ ? (int)left : kSegQ;
      const int pairs = plan_segment(S, seg, nq, pt_col, pt_w, a_rp);
      for (int t0 = 0; t0 < pairs; t0 += kPlanChunk / 3) {
        const int np = min(kPlanChunk / 3, pairs - t0);
        plan_stage(S, J, nq, t0, np, a_col, p_idx, p_w);
        for (int p = lane; p < 3 * np; p += 32)
          if (S.ps[p] >= 0) atomicAdd(&S.fill[S.ps[p]], 1);
        __syncwarp();
      }
    }
    for (int a = lane; a < len; a += 32) terms[r0 + a] = S.fill[a];
    __syncwarp();
  }
}

// Symbolic pass 2: writes every entry's terms in canonical order.  The lane
// owning a position (pos & 31) appends that position's terms; products of a
// chunk are grouped by owner first so all lanes append in parallel.
__global__ void __launch_bounds__(kPlanWarps * 32)
    k_gal_plan_fill(int64_t nc, const int64_t* __restrict__ pt_rp, const int32_t* __restrict__ pt_col,
                    const double* __restrict__ pt_w, const int64_t* __restrict__ a_rp,
                    const int32_t* __restrict__ a_col, const int32_t* __restrict__ p_idx,
                    const double* __restrict__ p_w, const int64_t* __restrict__ c_rp,
                    const int32_t* __restrict__ c_col, const int64_t* __restrict__ plan_ptr,
                    int32_t* __restrict__ plan_edge, double* __restrict__ plan_coef) {
  extern __shared__ unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  PlanSmem& S = reinterpret_cast<PlanSmem*>(smem_raw)[warp];
  for (int64_t J = (int64_t)blockIdx.x * kPlanWarps + warp; J < nc; J += (int64_t)gridDim.x * kPlanWarps) {
    const int64_t r0 = c_rp[J], r1 = c_rp[J + 1];
    const int len = (int)(r1 - r0);
    plan_row_table(S, r0, r1, c_col);
    for (int a = lane; a < len; a += 32) S.fill[a] = 0;
    __syncwarp();
    for (int64_t seg = pt_rp[J]; seg < pt_rp[J + 1]; seg += kSegQ) {
      const int64_t left = pt_rp[J + 1] - seg;
      const int nq = left < kSegQ ? (int)left : kSegQ;
      const int pairs = plan_segment(S, seg, nq, pt_col, pt_w, a_rp);
      for (int t0 = 0; t0 < pairs; t0 += kPlanChunk / 3) {
        const int np = min(kPlanChunk / 3, pairs - t0);
        plan_stage(S, J, nq, t0, np, a_col, p_idx, p_w);
        const int nprod = 3 * np;
        S.cnt[lane] = 0;
        __syncwarp();
        for (int g0 = 0; g0 < nprod; g0 += 32) {
          const int p = g0 + lane;
          const int ps = p < nprod ? S.ps[p] : -1;
          const int own = ps >= 0 ? (ps & 31) : 32;
          const unsigned peers = __match_any_sync(0xffffffffu, own);
          if (own < 32 && lane == __ffs(peers) - 1) S.cnt[own] += __popc(peers);
          __syncwarp();
        }
        const int mine = S.cnt[lane];
        int start = mine;
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, start, o);
          if (lane >= o) start += v;
        }
        start -= mine;
        __syncwarp();
        S.cnt[lane] = start;
        __syncwarp();
        for (int g0 = 0; g0 < nprod; g0 += 32) {
          const int p = g0 + lane;
          const int ps = p < nprod ? S.ps[p] : -1;
          const int own = ps >= 0 ? (ps & 31) : 32;
          const unsigned peers = __match_any_sync(0xffffffffu, own);
          if (own < 32) S.list[S.cnt[own] + __popc(peers & ((1u << lane) - 1u))] = (int16_t)p;
          __syncwarp();
          if (own < 32 && lane == __ffs(peers) - 1) S.cnt[own] += __popc(peers);
          __syncwarp();
        }
        for (int q = start; q < start + mine; ++q) {
          const int p = S.list[q];
          const int pos = S.ps[p];
          const int64_t dst = plan_ptr[r0 + pos] + S.fill[pos]++;
          plan_edge[dst] = S.pe[p];
          plan_coef[dst] = S.pc[p];
        }
        __syncwarp();
      }
    }
  }
}

// The plan re-laid for the numeric pass: the entries on or above the
// diagonal, sorted by their number of terms (descending), in slices of 32;
// slice g stores its terms [k][lane] (term k of the slice's lane-th entry at
// sptr[g] + 32 k + lane), padded with zero coefficients.  A thread per entry
// then reads its terms with the warp's loads contiguous, and still adds them
// in the entry's canonical order.
__global__ void k_plan_slice(int64_t nup, const int32_t* __restrict__ up_entry, const int64_t* __restrict__ plan_ptr,
                             const int32_t* __restrict__ plan_edge, const double* __restrict__ plan_coef,
                             const int64_t* __restrict__ sptr, int32_t* __restrict__ sedge,
                             double* __restrict__ scoef) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nup; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = i >> 5, lane = i & 31;
    const int64_t e = up_entry[i];
    const int64_t t0 = plan_ptr[e], nt = plan_ptr[e + 1] - t0;
    const int64_t width = (sptr[g + 1] - sptr[g]) >> 5;
    for (int64_t k = 0; k < width; ++k) {
      const int64_t dst = sptr[g] + k * 32 + lane;
      sedge[dst] = k < nt ? plan_edge[t0 + k] : 0;
      scoef[dst] = k < nt ? plan_coef[t0 + k] : 0.0;
    }
  }
}

// Writes the value x of Galerkin entry e (on or above the diagonal) and of
// its mirror m (below it; m < 0 on the diagonal) into the level's CSR and
// solve layout: sliced-ELL slot (FP64 and FP32) or diagonal with its
// reciprocal.  err bit 0: a diagonal entry <= 0; bit 1: a non-finite value.
__device__ __forceinline__ void emit_entry(int64_t e, int64_t m, double x, double* __restrict__ c_val,
                                           const int64_t* __restrict__ csr2ell, double* __restrict__ e64,
                                           float* __restrict__ e32, double* __restrict__ d64,
                                           float* __restrict__ d32, double* __restrict__ di64,
                                           float* __restrict__ di32, int* __restrict__ err) {
  if (!finite_bits(x)) atomicOr(err, 2);
  c_val[e] = x;
  const int64_t se = csr2ell[e];
  const float x32 = f32_rn(x);
  if (se >= 0) {
    e64[se] = x;
    e32[se] = x32;
  } else {
    const int64_t r = -1 - se;
    if (!positive_bits(x)) atomicOr(err, 1);
    const double xi = recip_newton(x);
    d64[r] = x;
    d32[r] = x32;
    di64[r] = xi;
    di32[r] = f32_rn(xi);
  }
  if (m >= 0) {
    c_val[m] = x;
    const int64_t sm = csr2ell[m];
    e64[sm] = x;
    e32[sm] = x32;
  }
}

// Numeric pass of one Galerkin level, one thread per entry on or above the
// diagonal (sliced plan order, slices [g0, g1)): value = sum over its terms
// of coef * A_l value, each term added with one fused multiply-add in the
// plan's order (zero padding adds +0), then written with its mirror (exact
// symmetry) into the CSR and the solve layout.  Terms are loaded B at a time
// before they are added, so a long term list is not a chain of dependent
// loads, and the plan of batch k + 1 is loaded while the gathered values of
// batch k arrive: B = 16 for the slices of long entries (hundreds of terms
// on coarse levels; B = 32 took 226 registers and halved the warps in
// flight), B = 8 elsewhere (fewer registers, more warps in flight).  The
// plan is read once, with the evict-first (streaming) hint, so that it does
// not push the finer level's gathered values out of L2.
constexpr int kGalThreads = 64;  // small blocks: coarse levels have few entries, and each SM's FP64 pipe counts
constexpr int kGalLongWidth = 32;  // slices wider than this take the B = 16 kernel
template <int B>
__global__ void __launch_bounds__(kGalThreads)
    k_gal_level(int64_t g0, int64_t g1, const int32_t* __restrict__ up_entry, const int32_t* __restrict__ mirror,
                const int64_t* __restrict__ sptr, const int32_t* __restrict__ sedge,
                const double* __restrict__ scoef, const double* __restrict__ a_val, double* __restrict__ c_val,
                const int64_t* __restrict__ csr2ell, double* __restrict__ e64, float* __restrict__ e32,
                double* __restrict__ d64, float* __restrict__ d32, double* __restrict__ di64,
                float* __restrict__ di32, int* __restrict__ err) {
  const int64_t i1 = g1 * 32;
  for (int64_t i = g0 * 32 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < i1;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = i >> 5, lane = i & 31;
    const int64_t base = sptr[g] + lane, width = (sptr[g + 1] - sptr[g]) >> 5;
    double acc = 0.0;
    int ed[B];
    double cf[B];
#pragma unroll
    for (int j = 0; j < B; ++j)
      if (j < width) {
        ed[j] = __ldcs(sedge + base + (int64_t)j * 32);
        cf[j] = __ldcs(scoef + base + (int64_t)j * 32);
      }
    for (int64_t k0 = 0; k0 < width; k0 += B) {
      // gathers of this batch, then the plan of the next one, then the adds:
      // one memory round trip per batch instead of two
      double av[B];
#pragma unroll
      for (int j = 0; j < B; ++j)
        if (k0 + j < width) av[j] = a_val[ed[j]];
      int edn[B];
      double cfn[B];
#pragma unroll
      for (int j = 0; j < B; ++j)
        if (k0 + B + j < width) {
          edn[j] = __ldcs(sedge + base + (k0 + B + j) * 32);
          cfn[j] = __ldcs(scoef + base + (k0 + B + j) * 32);
        }
#pragma unroll
      for (int j = 0; j < B; ++j)
        if (k0 + j < width) acc = __fma_rn(cf[j], av[j], acc);
#pragma unroll
      for (int j = 0; j < B; ++j) {
        ed[j] = edn[j];
        cf[j] = cfn[j];
      }
    }
    emit_entry(up_entry[i], mirror[i], acc, c_val, csr2ell, e64, e32, d64, d32, di64, di32, err);
  }
}

// CSR values -> sliced-ELL values, diagonal and inverse diagonal (both
// precisions), one thread per row of the permuted numbering: the thread of
// (slice s, lane) walks the CSR row of row0[s] + lane in order and puts its
// k-th off-diagonal value in slot ptr[s] + 32 k + lane (the slot the layout
// gives that entry), so a warp stores each slot column as 32 contiguous
// values and each thread reads one contiguous CSR row.  Padding slots keep
// their zeros.  err bit 0: diagonal <= 0; bit 1: non-finite value.
__global__ void k_scatter_rows(int64_t nslice, const int64_t* __restrict__ ptr, const int32_t* __restrict__ row0,
                               const int32_t* __restrict__ nrow, const int32_t* __restrict__ perm,
                               const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                               const double* __restrict__ v, double* __restrict__ e64, float* __restrict__ e32,
                               double* __restrict__ d64, float* __restrict__ d32, double* __restrict__ di64,
                               float* __restrict__ di32, int* __restrict__ err) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nslice * 32;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sl = t >> 5;
    const int lane = (int)(t & 31);
    if (lane >= nrow[sl]) continue;
    const int64_t r = (int64_t)row0[sl] + lane;
    const int32_t old = perm[r];
    int64_t slot = ptr[sl] + lane;
    for (int64_t e = rp[old], e1 = rp[old + 1]; e < e1; ++e) {
      const double x = v[e];
      if (!finite_bits(x)) atomicOr(err, 2);
      if (ci[e] == old) {
        if (!positive_bits(x)) atomicOr(err, 1);
        const double xi = recip_newton(x);
        d64[r] = x;
        d32[r] = f32_rn(x);
        di64[r] = xi;
        di32[r] = f32_rn(xi);
      } else {
        e64[slot] = x;
        e32[slot] = f32_rn(x);
        slot += 32;
      }
    }
  }
}

// Dense coarsest operator in the level's colour-permuted numbering (the
// numbering of the vectors the cycle hands to the coarse solve).
__global__ void k_csr_to_dense(int64_t n, int64_t ld, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                               const double* __restrict__ val, const int32_t* __restrict__ iperm,
                               double* __restrict__ D) {
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const int64_t pi = iperm[i];
    for (int64_t k = rp[i] + threadIdx.x; k < rp[i + 1]; k += blockDim.x) D[pi * ld + iperm[col[k]]] = val[k];
  }
}

// ---- explicit inverse of the coarsest operator by block sweeps ----
// The coarse solve applies A_lambda^-1 as a GEMV; the inverse is formed by
// the symmetric sweep operator (Gauss-Jordan elimination without pivoting,
// stable on SPD matrices), 32 x 32 blocks.  S is the operator padded to
// npad = 32 nbk rows (identity on the padded diagonal), row-major with
// leading dimension npad; only its lower triangle (S_ij, i >= j) is stored.
// Sweeping pivot block P replaces
//   S_PP by -S_PP^-1,   S_IP by S_IP S_PP^-1   (I != P),
//   S_IJ by S_IJ - S_IP S_PP^-1 S_PJ          (I, J != P),
// with S_PJ = S_JP^T; after every block has been swept S = -A^-1.  Each pivot
// is a Schur complement of A, hence SPD when A is (status bit 0 otherwise).
// One sweep is two launches: the panel (the pivot column before the sweep,
// U = S_:P, and U S_PP^-1) and the update of every lower tile; the last CTA
// to finish the next pivot tile inverts it for the following sweep.

__device__ __forceinline__ double sym_at(const double* S, int ld, int i, int j) {
  return i >= j ? S[(int64_t)i * ld + j] : S[(int64_t)j * ld + i];
}

// m <- m^-1 for a 32 x 32 SPD block held in both triangles, by 32 scalar
// sweeps of its lower triangle, software-pipelined: during step k, warp 0
// updates column k+1 itself and from it forms step k+1's pivot reciprocal
// and scaled column, while six other warps (on the other three SM
// sub-partitions) update the remaining entries; one block barrier per step.
// Every entry is updated as v - c_i (c_j / d) with one fused multiply-add.  A
// pivot that is not positive sets *bad and is replaced by 1.  blockDim.x ==
// 256; all threads must call it.
__device__ void sweep_inverse32(double (&m)[32][33], int* bad) {
  __shared__ double ck[2][32], cs[2][32], sdk[2];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // workers: warps 1, 2, 3, 5, 6, 7; entry e of the packed lower triangle
  const int wk = warp == 0 || warp == 4 ? -1 : (warp < 4 ? warp - 1 : warp - 2) * 32 + lane;
  int ei[3], ej[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int e = wk + 192 * q;
    int i = wk < 0 ? 0 : (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= e) ++i;
    while (i > 0 && i * (i + 1) / 2 > e) --i;
    ei[q] = (wk >= 0 && e < 528) ? i : -1;
    ej[q] = e - i * (i + 1) / 2;
  }
  // step 0's pivot and column
  if (warp == 0) {
    double d = m[0][0];
    if (!positive_bits(d)) {
      if (lane == 0) *bad = 1;
      d = 1.0;
    }
    const double dk = recip_newton(d);
    const double c = m[lane][0];
    ck[0][lane] = c;
    cs[0][lane] = c * dk;
    if (lane == 0) sdk[0] = dk;
  }
  __syncthreads();
  for (int k = 0; k < 32; ++k) {
    const int cur = k & 1, nxt = cur ^ 1;
    if (warp == 0) {
      if (k + 1 < 32) {
        // entry (a, b) of column k+1 (lower storage) after step k
        const int kp = k + 1, a = lane > kp ? lane : kp, bb = lane > kp ? kp : lane;
        double v;
        if (bb == k)
          v = cs[cur][a];
        else
          v = __fma_rn(-ck[cur][a], cs[cur][bb], m[a][bb]);
        m[a][bb] = v;
        double d = __shfl_sync(0xffffffffu, v, kp);
        if (!positive_bits(d)) {
          if (lane == 0) *bad = 1;
          d = 1.0;
        }
        const double dk = recip_newton(d);
        ck[nxt][lane] = v;
        cs[nxt][lane] = v * dk;
        if (lane == 0) sdk[nxt] = dk;
      }
    } else if (wk >= 0) {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int i = ei[q], j = ej[q];
        if (i < 0 || i == k + 1 || j == k + 1) continue;
        double v;
        if (i == k && j == k)
          v = -sdk[cur];
        else if (i == k)
          v = cs[cur][j];
        else if (j == k)
          v = cs[cur][i];
        else
          v = __fma_rn(-ck[cur][i], cs[cur][j], m[i][j]);
        m[i][j] = v;
      }
    }
    __syncthreads();
  }
  // the lower triangle holds -m^-1: negate, then mirror
  for (int e = tid; e < 1024; e += 256) {
    const int i = e >> 5, j = e & 31;
    if (i >= j) m[i][j] = -m[i][j];
  }
  __syncthreads();
  for (int e = tid; e < 1024; e += 256) {
    const int i = e >> 5, j = e & 31;
    if (i < j) m[i][j] = m[j][i];
  }
  __syncthreads();
}

// S = 0 with ones on the padded diagonal (rows n .. npad-1).
__global__ void k_gj_pad(int npad, int n, double* __restrict__ S) {
  const int64_t total = (int64_t)npad * npad;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / npad, j = e % npad;
    S[e] = (i == j && i >= n) ? 1.0 : 0.0;
  }
}

// Dinv = S_00^-1 (the first pivot).
__global__ void __launch_bounds__(256) k_gj_first(int npad, const double* __restrict__ S, double* __restrict__ Dinv,
                                                  int* __restrict__ status) {
  __shared__ double m[32][33];
  __shared__ int bad;
  pdl_wait();
  pdl_trigger();
  if (threadIdx.x == 0) bad = 0;
  for (int e = threadIdx.x; e < 1024; e += 256) m[e >> 5][e & 31] = sym_at(S, npad, e >> 5, e & 31);
  __syncthreads();
  sweep_inverse32(m, &bad);
  for (int e = threadIdx.x; e < 1024; e += 256) Dinv[e] = m[e >> 5][e & 31];
  if (threadIdx.x == 0 && bad) atomicOr(status, 1);
}

// Panel of sweep P, 8 rows per CTA: Uo[r][k] = S_{r, 32P+k} (before the
// sweep), Uh[r][k] = sum_j Uo[r][j] Dinv[j][k].
__global__ void __launch_bounds__(256) k_gj_panel(int npad, int P, const double* __restrict__ S,
                                                  const double* __restrict__ Dinv, double* __restrict__ Uo,
                                                  double* __restrict__ Uh) {
  __shared__ double D[32][33], u[8][32];
  pdl_wait();
  pdl_trigger();
  const int tid = threadIdx.x, rr = tid >> 5, k = tid & 31;
  const int r = blockIdx.x * 8 + rr;
  for (int e = tid; e < 1024; e += 256) D[e >> 5][e & 31] = Dinv[e];
  const double v = sym_at(S, npad, r, P * 32 + k);
  u[rr][k] = v;
  Uo[(int64_t)r * 32 + k] = v;
  __syncthreads();
  double acc = 0.0;
#pragma unroll 8
  for (int j = 0; j < 32; ++j) acc += u[rr][j] * D[j][k];
  Uh[(int64_t)r * 32 + k] = acc;
}

// Maps a linear tile index to (I, J), J in [first, nbk), I in [J, nbk).
__device__ __forceinline__ void lower_tile(int t, int first, int nbk, int* I, int* J) {
  int j = first;
  while (t >= nbk - j) {
    t -= nbk - j;
    ++j;
  }
  *J = j;
  *I = j + t;
}

// Quarter `it` of the work list of sweep P: tile (I, J) (the next pivot tile
// first, then lower_tile order) and its quarter q.
__device__ __forceinline__ void gj_item(int it, int P, int nbk, int* I, int* J, int* q) {
  *q = it & 3;
  const int tt = it >> 2;
  int t = tt;
  if (P + 1 < nbk) {
    const int tD = (P + 1) * nbk - P * (P + 1) / 2;  // lower_tile index of (P+1, P+1)
    t = tt == 0 ? tD : (tt <= tD ? tt - 1 : tt);
  }
  lower_tile(t, 0, nbk, I, J);
}

// Update of sweep P over the 8-row quarters of every lower tile, taken from a
// work counter (work[P]) by a persistent grid of about one CTA per SM; each
// CTA claims its next quarter and loads that quarter's operands into
// registers while it computes the current one.  The four quarters of the
// next pivot tile (P+1, P+1) come first; the CTA that finishes the last of
// them (arrival counter cnt[P]) inverts that tile into DinvNext and takes no
// more quarters, so the 32 dependent pivot steps of the inversion run on an
// SM of their own: an SM's FP64 pipe is shared by its warps (a warp's FP64
// instruction occupies its sub-partition's pipe for 64 cycles), and with the
// whole update resident at once the inversion used to wait behind the
// quarters placed on its SM.
__global__ void __launch_bounds__(256) k_gj_update(int npad, int P, double* __restrict__ S,
                                                   const double* __restrict__ Dinv, const double* __restrict__ Uo,
                                                   const double* __restrict__ Uh, int* __restrict__ cnt,
                                                   int* __restrict__ work, double* __restrict__ DinvNext,
                                                   int* __restrict__ status) {
  __shared__ double uo[32][33], uh[8][33];
  __shared__ double m[32][33];
  __shared__ int last, bad, item;
  pdl_wait();
  pdl_trigger();
  const int nbk = npad / 32;
  const int nitems = 4 * nbk * (nbk + 1) / 2;
  const int tid = threadIdx.x, rr = tid >> 5, cc = tid & 31;
  const bool has_next = P + 1 < nbk;
  double ruo[4], ruh = 0.0, rs = 0.0;
  // operands of a bulk quarter (neither index on the pivot block P) into
  // registers, with the entry of S it updates
  auto fetch = [&](int it) {
    if (it >= nitems) return;
    int I, J, q;
    gj_item(it, P, nbk, &I, &J, &q);
    if (I == P || J == P) return;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + 256 * u;
      ruo[u] = Uo[(int64_t)(J * 32 + (e >> 5)) * 32 + (e & 31)];
    }
    const int r = I * 32 + q * 8 + rr;
    ruh = Uh[(int64_t)r * 32 + cc];
    rs = S[(int64_t)r * npad + J * 32 + cc];
  };
  if (tid == 0) item = atomicAdd(work + P, 1);
  __syncthreads();
  int cur = item;
  __syncthreads();
  fetch(cur);
  while (cur < nitems) {
    int I, J, q;
    gj_item(cur, P, nbk, &I, &J, &q);
    // a quarter of the next pivot tile may end with this CTA inverting it:
    // its successor is claimed only after the arrival test
    const bool pivq = has_next && I == P + 1 && J == P + 1;
    const bool bulk = I != P && J != P;
    if (!pivq && tid == 0) item = atomicAdd(work + P, 1);
    const double s_old = rs;
    if (bulk) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = tid + 256 * u;
        uo[e >> 5][e & 31] = ruo[u];
      }
      uh[rr][cc] = ruh;
    }
    __syncthreads();
    int nxt = pivq ? nitems : item;
    if (!pivq) fetch(nxt);
    const int r = I * 32 + q * 8 + rr, c = J * 32 + cc;
    double* out = S + (int64_t)r * npad + c;
    if (I == P && J == P) {
      *out = -Dinv[(r - P * 32) * 32 + cc];
    } else if (J == P) {
      *out = Uh[(int64_t)r * 32 + cc];
    } else if (I == P) {
      *out = Uh[(int64_t)c * 32 + (r - P * 32)];
    } else {
      double acc = 0.0;
#pragma unroll 8
      for (int k = 0; k < 32; ++k) acc += uh[rr][k] * uo[cc][k];
      *out = s_old - acc;
    }
    if (pivq) {
      __threadfence();
      __syncthreads();
      if (tid == 0) {
        last = atomicAdd(cnt + P, 1) == 3;
        bad = 0;
      }
      __syncthreads();
      if (last) {
        __threadfence();
        const double* T = S + (int64_t)(P + 1) * 32 * npad + (P + 1) * 32;
        for (int e = tid; e < 1024; e += 256) {
          const int i = e >> 5, j = e & 31;
          m[i][j] = __ldcg(T + (int64_t)(i >= j ? i : j) * npad + (i >= j ? j : i));
        }
        __syncthreads();
        sweep_inverse32(m, &bad);
        for (int e = tid; e < 1024; e += 256) DinvNext[e] = m[e >> 5][e & 31];
        if (tid == 0 && bad) atomicOr(status, 1);
        return;
      }
      if (tid == 0) item = atomicAdd(work + P, 1);
      __syncthreads();
      nxt = item;
      fetch(nxt);
    }
    __syncthreads();  // the tile in shared memory and `item` are reused
    cur = nxt;
  }
}

// Ainv = -S (both triangles, leading dimension n), and its FP32 copy.
__global__ void k_gj_finish(int n, int npad, const double* __restrict__ S, double* __restrict__ Ainv,
                            float* __restrict__ Ainv32) {
  pdl_wait();
  pdl_trigger();
  const int64_t total = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    const double v = -sym_at(S, npad, i, j);
    Ainv[e] = v;
    Ainv32[e] = (float)v;
  }
}

// ------------------------------------------------------------------ host

static int grid_for(int64_t work, int threads, int cap = 152 * 32) {
  int64_t g = (work + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

template <class T>
static gmg_status upload(Arena& a, T** d, const T* h, size_t n) {
  GMG_TRY(a.alloc(d, n));
  const auto t0 = std::chrono::steady_clock::now();
  if (n) GMG_CK(cudaMemcpy(*d, h, n * sizeof(T), cudaMemcpyHostToDevice));
  a.ms_copy += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return GMG_OK;
}

// ---- colouring of a level's pattern (host).  Two greedy colourings are
// built and the one with fewer colours kept (the first on a tie): first fit
// in increasing row index, and first fit in smallest-last order (Matula and
// Beck); each is then improved by kColourPasses passes of iterated greedy
// (Culberson), which recolour by first fit visiting the colour classes from
// the highest colour down, rows ascending within a class, and never add a
// colour.  Every rule is deterministic, so the oracle, which implements the
// same steps on its own, produces the same colouring.

constexpr int kColourPasses = 8;

// First fit of the rows rows[0 .. cnt) in that order against the colours
// already in `color` (-1 = not coloured).  `mark` holds one stamp per colour
// (at least the longest row + 2 entries); `stamp` increases by one per row.
// The visiting order jumps across the pattern (a class of the previous pass
// is spread over the whole level), so the pattern entries of the rows a few
// places ahead are prefetched.
static int fit_rows(const int32_t* rows, int64_t cnt, const int64_t* rp, const int32_t* ci, int32_t* color,
                    std::vector<int64_t>& mark, int64_t& stamp) {
  constexpr int64_t kAhead = 8;
  int ncol = 0;
  for (int64_t t = 0; t < cnt; ++t) {
    if (t + 2 * kAhead < cnt) __builtin_prefetch(&rp[rows[t + 2 * kAhead]]);
    if (t + kAhead < cnt) {
      const int64_t k0 = rp[rows[t + kAhead]], k1 = rp[rows[t + kAhead] + 1];
      for (int64_t k = k0; k < k1; k += 16) __builtin_prefetch(&ci[k]);
      if (k1 > k0) __builtin_prefetch(&ci[k1 - 1]);
    }
    const int32_t i = rows[t];
    ++stamp;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      const int32_t cj = color[ci[k]];  // the row itself is not coloured yet
      if (cj >= 0) mark[cj] = stamp;
    }
    int32_t c = 0;
    while (mark[c] == stamp) ++c;
    color[i] = c;
    ncol = std::max(ncol, c + 1);
  }
  return ncol;
}

// First fit in the given visiting order: each row takes the smallest colour
// not used by a neighbour coloured earlier in this pass.
static int first_fit(int64_t n, const int64_t* rp, const int32_t* ci, const std::vector<int32_t>& order,
                     std::vector<int32_t>& color, int64_t maxlen) {
  color.assign(n, -1);
  std::vector<int64_t> mark(maxlen + 2, -1);
  int64_t stamp = 0;
  return fit_rows(order.data(), n, rp, ci, color.data(), mark, stamp);
}

// Barrier of a team of threads that wait by yielding.
struct YieldBarrier {
  std::atomic<int> count{0}, gen{0};
  int n = 1;
  void wait() {
    const int g = gen.load(std::memory_order_acquire);
    if (count.fetch_add(1, std::memory_order_acq_rel) == n - 1) {
      count.store(0, std::memory_order_relaxed);
      gen.store(g + 1, std::memory_order_release);
    } else {
      while (gen.load(std::memory_order_acquire) == g) std::this_thread::yield();
    }
  }
};

// One iterated-greedy pass: first fit over the classes of `color` from the
// highest colour down, rows ascending within a class.  The rows of one class
// are pairwise non-adjacent, so each row's choice depends only on the
// classes visited before its own: a class is split into contiguous parts
// coloured by up to `nthreads` threads, with a barrier between classes, and
// the result is that of the sequential pass.
static int iterated_pass(int64_t n, const int64_t* rp, const int32_t* ci, int ncol, std::vector<int32_t>& color,
                         int nthreads, int64_t maxlen) {
  std::vector<int64_t> start(ncol + 1, 0);
  for (int64_t i = 0; i < n; ++i) start[ncol - color[i]]++;  // class of colour c goes to slot ncol - 1 - c
  for (int c = 0; c < ncol; ++c) start[c + 1] += start[c];
  const std::vector<int64_t> cs(start);  // first position of each class
  std::vector<int32_t> order(n);
  for (int64_t i = 0; i < n; ++i) order[start[ncol - 1 - color[i]]++] = (int32_t)i;
  color.assign(n, -1);
  YieldBarrier bar;
  std::atomic<int> team{0};  // team size once every helper thread is started
  std::vector<int> nc(std::max(1, nthreads), 0);
  auto work = [&](int t) {
    int m;
    while ((m = team.load(std::memory_order_acquire)) == 0) std::this_thread::yield();
    if (t >= m) return;
    std::vector<int64_t> mark(maxlen + 2, -1);
    int64_t stamp = 0;
    for (int k = 0; k < ncol; ++k) {
      const int64_t len = cs[k + 1] - cs[k];
      const int64_t lo = cs[k] + len * t / m, hi = cs[k] + len * (t + 1) / m;
      nc[t] = std::max(nc[t], fit_rows(order.data() + lo, hi - lo, rp, ci, color.data(), mark, stamp));
      if (m > 1) bar.wait();
    }
  };
  std::vector<std::thread> helpers;
  for (int t = 1; t < nthreads; ++t) {
    try {
      helpers.emplace_back(work, t);
    } catch (...) {  // fewer threads: the team is the ones started
      break;
    }
  }
  bar.n = 1 + (int)helpers.size();
  team.store(bar.n, std::memory_order_release);
  work(0);
  for (auto& h : helpers) h.join();
  return *std::max_element(nc.begin(), nc.end());
}

// Smallest-last order: rows sit in buckets by their number of neighbours not
// yet removed, each bucket a stack (initially filled from the highest row
// index down, so the smallest index is on top); the next row removed is the
// top of the lowest non-empty bucket, and each of its remaining neighbours
// (in pattern order) moves to the top of the bucket one lower.  The order is
// the reverse of the removal order.
static void smallest_last(int64_t n, const int64_t* rp, const int32_t* ci, std::vector<int32_t>& order) {
  std::vector<int32_t> deg(n), next(n), prev(n);
  int maxd = 0;
  for (int64_t i = 0; i < n; ++i) {
    int d = 0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) d += ci[k] != i;
    deg[i] = d;
    maxd = std::max(maxd, d);
  }
  std::vector<int32_t> head(maxd + 1, -1);
  std::vector<char> gone(n, 0);
  auto push = [&](int32_t v, int d) {
    next[v] = head[d];
    prev[v] = -1;
    if (head[d] >= 0) prev[head[d]] = v;
    head[d] = v;
  };
  auto unlink = [&](int32_t v, int d) {
    if (prev[v] >= 0) next[prev[v]] = next[v];
    else head[d] = next[v];
    if (next[v] >= 0) prev[next[v]] = prev[v];
  };
  for (int64_t i = n - 1; i >= 0; --i) push((int32_t)i, deg[i]);
  order.assign(n, 0);
  int cur = 0;
  for (int64_t t = n - 1; t >= 0; --t) {
    cur = std::max(cur - 1, 0);
    while (head[cur] < 0) ++cur;
    const int32_t v = head[cur];
    unlink(v, cur);
    gone[v] = 1;
    order[t] = v;
    for (int64_t k = rp[v]; k < rp[v + 1]; ++k) {
      const int32_t u = ci[k];
      if (u == v || gone[u]) continue;
      unlink(u, deg[u]);
      --deg[u];
      push(u, deg[u]);
    }
  }
}

// One candidate: first fit in increasing row index (sl = false) or in
// smallest-last order (sl = true), then kColourPasses iterated-greedy passes.
// A pass is a function of the colouring alone, so once the colouring after a
// pass equals the one two passes earlier the passes alternate between the
// last two colourings, and the result after all passes is known without
// running the rest (the same colouring as running them).
static int colour_candidate(int64_t n, const int64_t* rp, const int32_t* ci, bool sl, std::vector<int32_t>& color) {
  int64_t maxlen = 0;
  for (int64_t i = 0; i < n; ++i) maxlen = std::max(maxlen, rp[i + 1] - rp[i]);
  const unsigned hw = std::thread::hardware_concurrency();
  const int nthreads = n >= (1 << 16) ? (int)std::min(4u, std::max(1u, hw / 4)) : 1;
  std::vector<int32_t> order(n);
  if (sl) {
    smallest_last(n, rp, ci, order);
  } else {
    for (int64_t i = 0; i < n; ++i) order[i] = (int32_t)i;
  }
  int nc = first_fit(n, rp, ci, order, color, maxlen);
  std::vector<int32_t> prev1, prev2;  // colourings after the previous pass and the one before
  int nc1 = 0;
  for (int p = 0; p < kColourPasses; ++p) {
    prev2.swap(prev1);
    prev1 = color;
    nc1 = nc;
    nc = iterated_pass(n, rp, ci, nc, color, nthreads, maxlen);
    if (p >= 1 && color == prev2) {
      if ((kColourPasses - 1 - p) % 2 == 1) {
        color.swap(prev1);
        nc = nc1;
      }
      break;
    }
  }
  return nc;
}

// The two candidates of a level, computed on two host threads; the one with
// fewer colours is kept, the index-order one on a tie.  The threads start as
// soon as the level's pattern is on the host (while the device computes the
// next level's pattern) and are joined before the level's layout is built.
struct ColourJob {
  int64_t n = 0;
  const int64_t* rp = nullptr;
  const int32_t* ci = nullptr;
  std::vector<int32_t> ca, cb;
  int na = 0, nb = 0;
  std::thread ta, tb;
  void start(int64_t n_, const int64_t* rp_, const int32_t* ci_) {
    n = n_;
    rp = rp_;
    ci = ci_;
    try {
      ta = std::thread([this] { na = colour_candidate(n, rp, ci, false, ca); });
      tb = std::thread([this] { nb = colour_candidate(n, rp, ci, true, cb); });
    } catch (...) {  // no thread available: the candidates are computed in finish()
    }
  }
  // Joins the threads (or computes what they did not) and returns the number
  // of colours of the kept candidate, moved into `color`.
  int finish(std::vector<int32_t>& color) {
    join();
    if (!started_a) na = colour_candidate(n, rp, ci, false, ca);
    if (!started_b) nb = colour_candidate(n, rp, ci, true, cb);
    if (nb < na) {
      color.swap(cb);
      return nb;
    }
    color.swap(ca);
    return na;
  }
  void join() {
    if (ta.joinable()) {
      ta.join();
      started_a = true;
    }
    if (tb.joinable()) {
      tb.join();
      started_b = true;
    }
  }
  bool started_a = false, started_b = false;
  ~ColourJob() { join(); }
};

// Sliced-ELL structure for `nrows` rows given the rows' entry lists; slices
// start at every `seg` boundary (colour starts), 32 rows per slice.
struct EllPlan {
  std::vector<int64_t> ptr;
  std::vector<int32_t> row0, nrow;
};

static void plan_slices(const std::vector<int64_t>& seg, const std::vector<int64_t>& rowlen, EllPlan& P,
                        std::vector<int64_t>* seg_slice) {
  P.ptr.assign(1, 0);
  P.row0.clear();
  P.nrow.clear();
  if (seg_slice) seg_slice->assign(1, 0);
  for (size_t s = 0; s + 1 < seg.size(); ++s) {
    for (int64_t r0 = seg[s]; r0 < seg[s + 1]; r0 += kSlice) {
      const int64_t r1 = std::min(seg[s + 1], r0 + kSlice);
      int64_t w = 0;
      for (int64_t r = r0; r < r1; ++r) w = std::max(w, rowlen[r]);
      P.row0.push_back((int32_t)r0);
      P.nrow.push_back((int32_t)(r1 - r0));
      P.ptr.push_back(P.ptr.back() + w * kSlice);
    }
    if (seg_slice) seg_slice->push_back((int64_t)P.row0.size());
  }
}

static gmg_status upload_ell(Arena& a, Ell& E, const EllPlan& P, const std::vector<int32_t>& col) {
  E.nslice = (int64_t)P.row0.size();
  E.entries = P.ptr.back();
  GMG_TRY(upload(a, &E.ptr, P.ptr.data(), P.ptr.size()));
  GMG_TRY(upload(a, &E.row0, P.row0.data(), P.row0.size()));
  GMG_TRY(upload(a, &E.nrow, P.nrow.data(), P.nrow.size()));
  GMG_TRY(upload(a, &E.col, col.data(), col.size()));
  GMG_TRY(a.alloc(&E.v64, (size_t)E.entries));
  GMG_TRY(a.alloc(&E.v32, (size_t)E.entries));
  GMG_CK(cudaMemset(E.v64, 0, sizeof(double) * (size_t)std::max<int64_t>(1, E.entries)));
  GMG_CK(cudaMemset(E.v32, 0, sizeof(float) * (size_t)std::max<int64_t>(1, E.entries)));
  return GMG_OK;
}

// Checks a caller's colouring of a level with pattern (rp, ci): every colour in
// [0, n) and no two adjacent rows of the same colour (rows of one colour must
// be independent for the in-place Gauss-Seidel update).  Returns the number
// of colours (largest + 1) or -1 after setting the error message.
static int check_colouring(int l, int64_t n, const int64_t* rp, const int32_t* ci, const int32_t* color) {
  int nc = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (color[i] < 0 || color[i] >= n) {
      set_error("coloring[" + std::to_string(l) + "]: colour of row " + std::to_string(i) + " outside [0, n)");
      return -1;
    }
    nc = std::max(nc, color[i] + 1);
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] != i && color[ci[k]] == color[i]) {
        set_error("coloring[" + std::to_string(l) + "]: adjacent rows " + std::to_string(i) + " and " +
                  std::to_string(ci[k]) + " share colour " + std::to_string(color[i]));
        return -1;
      }
  return nc;
}

// Locality rank of every row of every level (a permutation of 0 .. n_l - 1):
// the order of rows within a colour, and the ranges that the cluster kernels
// give their CTAs.  Rows of one colour are independent, so this order changes
// no result of a Gauss-Seidel sweep; it decides which values a warp's gathers
// touch together and which rows share a CTA.  It is the caller's index where
// the caller's numbering is local (at most a fifth of the off-diagonal
// entries join rows more than max(32, n/32) indices apart, e.g. a structured
// mesh).  Otherwise the coarsest level takes breadth-first order (from the
// smallest unvisited row, neighbours in pattern order) and the finer levels
// the order of the hierarchy's tree: rows sorted by the rank of their
// heaviest coarse parent (the first of equal weights), then by caller index,
// so that the rows under one coarse row, and under one coarser ancestor, are
// consecutive (a point cloud in random order).
static void locality_ranks(gmg_ctx* c, const std::vector<std::vector<int64_t>>& hrp,
                           const std::vector<std::vector<int32_t>>& hcol, const gmg_prolong* P) {
  const int nlev = c->nlev;
  const char* env = std::getenv("GMG_CALLER_ORDER");
  const bool caller_only = env && env[0] == '1';
  for (int l = nlev - 1; l >= 0; --l) {
    Level& L = c->L[l];
    const int64_t n = L.n;
    const int64_t* rp = hrp[l].data();
    const int32_t* ci = hcol[l].data();
    L.h_key.resize(n);
    const int64_t span = std::max<int64_t>(32, n / 32);
    int64_t off = 0, far = 0;
    for (int64_t i = 0; i < n; ++i)
      for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
        const int64_t d = (int64_t)ci[k] - i;
        off += d != 0;
        far += d > span || d < -span;
      }
    if (caller_only || 5 * far <= off) {
      for (int64_t i = 0; i < n; ++i) L.h_key[i] = (int32_t)i;
      continue;
    }
    if (l == nlev - 1) {
      std::vector<int32_t> queue(n);
      std::vector<char> seen(n, 0);
      int64_t head = 0, tail = 0;
      for (int64_t s0 = 0; s0 < n; ++s0) {
        if (seen[s0]) continue;
        seen[s0] = 1;
        queue[tail++] = (int32_t)s0;
        while (head < tail) {
          const int32_t u = queue[head];
          L.h_key[u] = (int32_t)head++;
          for (int64_t k = rp[u]; k < rp[u + 1]; ++k)
            if (!seen[ci[k]]) {
              seen[ci[k]] = 1;
              queue[tail++] = ci[k];
            }
        }
      }
      continue;
    }
    const gmg_prolong& p = P[l];
    const std::vector<int32_t>& kc = c->L[l + 1].h_key;
    std::vector<int32_t> pk(n);
    for (int64_t i = 0; i < n; ++i) {
      int q = 0;
      for (int s = 1; s < 3; ++s)
        if (p.w[3 * i + s] > p.w[3 * i + q]) q = s;
      pk[i] = kc[p.idx[3 * i + q]];
    }
    // stable counting sort by parent rank
    std::vector<int64_t> start(p.n_coarse + 1, 0);
    for (int64_t i = 0; i < n; ++i) start[pk[i] + 1]++;
    for (int64_t J = 0; J < p.n_coarse; ++J) start[J + 1] += start[J];
    for (int64_t i = 0; i < n; ++i) L.h_key[i] = (int32_t)start[pk[i]]++;
  }
}

// Colours level l (the caller's colouring when given, else the greedy one of `job`),
// renumbers it colour by colour (ascending locality rank within a colour), and
// builds the sliced-ELL layout of its off-diagonal part.
static gmg_status build_level_structure(gmg_ctx* c, int l, const int64_t* rp, const int32_t* ci,
                                        const int32_t* given, ColourJob& job, std::vector<int32_t>& perm,
                                        std::vector<int32_t>& iperm) {
  Level& L = c->L[l];
  const int64_t n = L.n;
  std::vector<int32_t> color;
  if (given) {
    L.ncolor = check_colouring(l, n, rp, ci, given);
    if (L.ncolor < 0) return GMG_ERR_INVALID_ARG;
    color.assign(given, given + n);
  } else {
    L.ncolor = job.finish(color);
  }
  L.h_color = color;
  L.color_off.assign(L.ncolor + 1, 0);
  for (int64_t i = 0; i < n; ++i) L.color_off[color[i] + 1]++;
  for (int k = 0; k < L.ncolor; ++k) L.color_off[k + 1] += L.color_off[k];
  perm.assign(n, 0);
  iperm.assign(n, 0);
  {
    std::vector<int32_t> byrank(n);
    for (int64_t i = 0; i < n; ++i) byrank[L.h_key[i]] = (int32_t)i;
    std::vector<int64_t> fill(L.color_off.begin(), L.color_off.end() - 1);
    for (int64_t t = 0; t < n; ++t) {
      const int32_t i = byrank[t];
      const int64_t r = fill[color[i]]++;
      perm[r] = i;
      iperm[i] = (int32_t)r;
    }
  }
  std::vector<int64_t> rowlen(n);
  for (int64_t r = 0; r < n; ++r) rowlen[r] = rp[perm[r] + 1] - rp[perm[r]] - 1;
  EllPlan P;
  plan_slices(L.color_off, rowlen, P, &L.color_slice_off);
  std::vector<int32_t> ecol(P.ptr.back());
  std::vector<int64_t> c2e(l > 0 ? rp[n] : 0);  // level 0 scatters row by row
  for (size_t s = 0; s < P.row0.size(); ++s) {
    const int64_t w = (P.ptr[s + 1] - P.ptr[s]) / kSlice;
    for (int lane = 0; lane < kSlice; ++lane) {
      const int64_t r = P.row0[s] + lane;
      int64_t k = 0;
      if (lane < P.nrow[s]) {
        const int64_t old = perm[r];
        for (int64_t e = rp[old]; e < rp[old + 1]; ++e) {
          if (ci[e] == old) {
            if (l > 0) c2e[e] = -1 - r;
          } else {
            const int64_t slot = P.ptr[s] + k * kSlice + lane;
            ecol[slot] = iperm[ci[e]];
            if (l > 0) c2e[e] = slot;
            ++k;
          }
        }
      }
      const int32_t pad = (int32_t)(lane < P.nrow[s] ? r : P.row0[s]);
      for (; k < w; ++k) ecol[P.ptr[s] + k * kSlice + lane] = pad;
    }
  }
  Arena& a = c->arena;
  GMG_TRY(upload_ell(a, L.A, P, ecol));
  // Rows longer than a few entries are split over several warps so that the
  // chain of dependent loads per row stays short (coarse levels carry 15-40
  // entries per row; the finest mesh level about 6).
  {
    const double wavg = P.row0.empty() ? 0.0 : (double)P.ptr.back() / (32.0 * (double)P.row0.size());
    L.lanes = wavg <= 8.0 ? 1 : wavg <= 16.0 ? 2 : wavg <= 32.0 ? 4 : 8;
    if (const char* e = std::getenv("GMG_LANES")) L.lanes = std::atoi(e);
    if (L.lanes != 1 && L.lanes != 2 && L.lanes != 4 && L.lanes != 8) L.lanes = 1;
    L.rlanes = L.lanes;
  }
  if (l > 0) GMG_TRY(upload(a, &L.csr2ell, c2e.data(), c2e.size()));  // level 0 scatters row by row
  GMG_TRY(upload(a, &L.perm, perm.data(), perm.size()));
  GMG_TRY(upload(a, &L.iperm, iperm.data(), iperm.size()));
  GMG_TRY(a.alloc(&L.diag64, n));
  GMG_TRY(a.alloc(&L.dinv64, n));
  GMG_TRY(a.alloc(&L.diag32, n));
  GMG_TRY(a.alloc(&L.dinv32, n));
  GMG_TRY(a.alloc(&L.x64, n));
  GMG_TRY(a.alloc(&L.b64, n));
  GMG_TRY(a.alloc(&L.r64, n));
  GMG_TRY(a.alloc(&L.x32, n));
  GMG_TRY(a.alloc(&L.b32, n));
  GMG_TRY(a.alloc(&L.r32, n));
  return GMG_OK;
}

// Prolongation of level l in permuted numbering, and its transpose as sliced
// ELL over the next level's permuted rows (fine rows ascending).
static gmg_status build_transfer_structure(gmg_ctx* c, int l, const gmg_prolong& P,
                                           const std::vector<int32_t>& perm_f, const std::vector<int32_t>& iperm_f,
                                           const std::vector<int32_t>& perm_c, const std::vector<int32_t>& iperm_c) {
  Level& L = c->L[l];
  const int64_t nf = P.n_fine, nc = P.n_coarse;
  std::vector<int32_t> idx(3 * nf);
  std::vector<double> w64(3 * nf);
  std::vector<float> w32(3 * nf);
  for (int64_t r = 0; r < nf; ++r) {
    const int64_t old = perm_f[r];
    for (int s = 0; s < 3; ++s) {
      idx[3 * r + s] = iperm_c[P.idx[3 * old + s]];
      w64[3 * r + s] = P.w[3 * old + s];
      w32[3 * r + s] = (float)P.w[3 * old + s];
    }
  }
  Arena& a = c->arena;
  GMG_TRY(upload(a, &L.p_idx, idx.data(), idx.size()));
  GMG_TRY(upload(a, &L.p_w64, w64.data(), w64.size()));
  GMG_TRY(upload(a, &L.p_w32, w32.data(), w32.size()));
  // transpose in permuted numbering: coarse row J' -> (fine row i', w)
  std::vector<int64_t> cnt(nc + 1, 0);
  for (int64_t r = 0; r < nf; ++r)
    for (int s = 0; s < 3; ++s)
      if (w64[3 * r + s] != 0.0) cnt[idx[3 * r + s] + 1]++;
  for (int64_t J = 0; J < nc; ++J) cnt[J + 1] += cnt[J];
  std::vector<int32_t> tcol(cnt[nc]);
  std::vector<double> tw(cnt[nc]);
  {
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t r = 0; r < nf; ++r)  // ascending fine row -> sorted lists
      for (int s = 0; s < 3; ++s)
        if (w64[3 * r + s] != 0.0) {
          const int64_t q = fill[idx[3 * r + s]]++;
          tcol[q] = (int32_t)r;
          tw[q] = w64[3 * r + s];
        }
  }
  std::vector<int64_t> seg = {0, nc}, rowlen(nc);
  for (int64_t J = 0; J < nc; ++J) rowlen[J] = cnt[J + 1] - cnt[J];
  EllPlan EP;
  plan_slices(seg, rowlen, EP, nullptr);
  std::vector<int32_t> ecol(EP.ptr.back());
  std::vector<double> ew(EP.ptr.back(), 0.0);
  for (size_t s = 0; s < EP.row0.size(); ++s) {
    const int64_t wd = (EP.ptr[s + 1] - EP.ptr[s]) / kSlice;
    for (int lane = 0; lane < kSlice; ++lane) {
      const int64_t J = EP.row0[s] + lane;
      int64_t k = 0;
      if (lane < EP.nrow[s])
        for (int64_t q = cnt[J]; q < cnt[J + 1]; ++q, ++k) {
          ecol[EP.ptr[s] + k * kSlice + lane] = tcol[q];
          ew[EP.ptr[s] + k * kSlice + lane] = tw[q];
        }
      const int32_t pad = lane < EP.nrow[s] && cnt[J + 1] > cnt[J] ? tcol[cnt[J]] : 0;
      for (; k < wd; ++k) ecol[EP.ptr[s] + k * kSlice + lane] = pad;
    }
  }
  GMG_TRY(upload_ell(a, L.R, EP, ecol));
  std::vector<float> ew32(ew.size());
  for (size_t q = 0; q < ew.size(); ++q) ew32[q] = (float)ew[q];
  GMG_CK(cudaMemcpy(L.R.v64, ew.data(), ew.size() * sizeof(double), cudaMemcpyHostToDevice));
  GMG_CK(cudaMemcpy(L.R.v32, ew32.data(), ew32.size() * sizeof(float), cudaMemcpyHostToDevice));
  (void)iperm_f;
  (void)perm_c;
  return GMG_OK;
}

static gmg_status check_err_word(int* d, cudaStream_t s, int* h) {
  GMG_CK(cudaMemcpyAsync(h, d, sizeof(int), cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaStreamSynchronize(s));
  return GMG_OK;
}

// Galerkin product of level l into level l+1: symbolic part (pattern).
// The entries with at least one product term (plan pointer hp), ordered by
// term count, most terms first, ascending position among equal counts: a
// stable counting sort.
static void plan_order(int64_t nnz, const std::vector<int64_t>& hp, std::vector<int32_t>& up) {
  int64_t wmax = 0;
  for (int64_t e = 0; e < nnz; ++e) wmax = std::max(wmax, hp[e + 1] - hp[e]);
  std::vector<int64_t> start(wmax + 2, 0);  // bucket of count w at slot wmax - w
  for (int64_t e = 0; e < nnz; ++e) {
    const int64_t w = hp[e + 1] - hp[e];
    if (w > 0) start[wmax - w + 1]++;
  }
  for (int64_t b = 0; b <= wmax; ++b) start[b + 1] += start[b];
  up.resize(start[wmax + 1]);
  for (int64_t e = 0; e < nnz; ++e) {
    const int64_t w = hp[e + 1] - hp[e];
    if (w > 0) up[start[wmax - w]++] = (int32_t)e;
  }
}

// For every entry (J, K) of a pattern with sorted rows, the position of
// (K, J), -1 for a diagonal entry.  Walking the rows K in increasing order
// visits the entries (K, J) of each column J in increasing K, i.e. in the
// order of row J's sorted entries, so a cursor per row pairs them.  Returns
// false if the pattern is not symmetric.
static bool mirror_positions(int64_t n, const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                             std::vector<int32_t>& m) {
  m.assign(rp[n], -1);
  std::vector<int64_t> cur(rp.begin(), rp.end() - 1);
  for (int64_t K = 0; K < n; ++K)
    for (int64_t f = rp[K]; f < rp[K + 1]; ++f) {
      const int64_t J = ci[f];
      if (J < 0 || J >= n || cur[J] >= rp[J + 1] || ci[cur[J]] != K) return false;
      m[cur[J]++] = J == K ? -1 : (int32_t)f;
    }
  for (int64_t J = 0; J < n; ++J)
    if (cur[J] != rp[J + 1]) return false;
  return true;
}

static gmg_status galerkin_symbolic(gmg_ctx* c, int l, cudaStream_t s, std::vector<int64_t>& hrp,
                                    std::vector<int32_t>& hcol) {
  Level& F = c->L[l];
  Level& C = c->L[l + 1];
  const int64_t nc = F.nc;
  int64_t* counts;
  GMG_TRY(c->arena.alloc(&counts, nc));
  GMG_CK(cudaMemsetAsync(c->dstatus, 0, sizeof(int), s));
  const int g1 = grid_for(nc, kCountWarps, 152 * 16);
  k_gal_count<<<g1, kCountWarps * 32, 0, s>>>(nc, F.pt_rowptr_o, F.pt_col_o, F.csr_rowptr, F.csr_col, F.p_idx_o,
                                             F.p_w_o, counts, c->dstatus);
  GMG_LAUNCHED();
  int herr = 0;
  GMG_TRY(check_err_word(c->dstatus, s, &herr));
  if (herr) {
    set_error("Galerkin row of level " + std::to_string(l + 1) + " exceeds " + std::to_string(kMaxRowEntries) +
              " entries");
    return GMG_ERR_TOO_LARGE;
  }
  GMG_TRY(c->arena.alloc(&C.csr_rowptr, nc + 1));
  k_scan_counts<<<1, 1024, 0, s>>>(nc, counts, C.csr_rowptr);
  GMG_LAUNCHED();
  hrp.resize(nc + 1);
  GMG_CK(cudaMemcpyAsync(hrp.data(), C.csr_rowptr, (nc + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaStreamSynchronize(s));
  C.nnz = hrp[nc];
  if (C.nnz >= INT32_MAX || F.nnz >= INT32_MAX) {
    set_error("Galerkin level " + std::to_string(l + 1) + ": more than 2^31 stored entries");
    return GMG_ERR_TOO_LARGE;
  }
  GMG_TRY(c->arena.alloc(&C.csr_col, C.nnz));
  GMG_TRY(c->arena.alloc(&C.csr_val, C.nnz));
  const int g2 = grid_for(nc, kFillWarps, 152 * 32);
  k_gal_fill<<<g2, kFillWarps * 32, 0, s>>>(nc, F.pt_rowptr_o, F.pt_col_o, F.csr_rowptr, F.csr_col, F.p_idx_o,
                                           F.p_w_o, C.csr_rowptr, C.csr_col);
  GMG_LAUNCHED();
  hcol.resize(C.nnz);
  GMG_CK(cudaMemcpyAsync(hcol.data(), C.csr_col, C.nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaStreamSynchronize(s));
  // product plan of the numeric pass
  const size_t psm = sizeof(PlanSmem) * kPlanWarps;
  GMG_CK(cudaFuncSetAttribute(k_gal_plan_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm));
  GMG_CK(cudaFuncSetAttribute(k_gal_plan_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm));
  int64_t* terms;
  GMG_TRY(c->arena.alloc(&terms, (size_t)C.nnz));
  const int gp = grid_for(nc, kPlanWarps, 152 * 16);
  k_gal_plan_count<<<gp, kPlanWarps * 32, psm, s>>>(nc, F.pt_rowptr_o, F.pt_col_o, F.pt_w_o, F.csr_rowptr, F.csr_col,
                                                    F.p_idx_o, F.p_w_o, C.csr_rowptr, C.csr_col, terms);
  GMG_LAUNCHED();
  GMG_TRY(c->arena.alloc(&C.plan_ptr, (size_t)C.nnz + 1));
  k_scan_counts<<<1, 1024, 0, s>>>(C.nnz, terms, C.plan_ptr);
  GMG_LAUNCHED();
  int64_t total = 0;
  GMG_CK(cudaMemcpyAsync(&total, C.plan_ptr + C.nnz, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaStreamSynchronize(s));
  C.plan_terms = total;
  GMG_TRY(c->arena.alloc(&C.plan_edge, (size_t)total));
  GMG_TRY(c->arena.alloc(&C.plan_coef, (size_t)total));
  k_gal_plan_fill<<<gp, kPlanWarps * 32, psm, s>>>(nc, F.pt_rowptr_o, F.pt_col_o, F.pt_w_o, F.csr_rowptr, F.csr_col,
                                                   F.p_idx_o, F.p_w_o, C.csr_rowptr, C.csr_col, C.plan_ptr,
                                                   C.plan_edge, C.plan_coef);
  GMG_LAUNCHED();
  // sliced layout of the plan (entries with terms, sorted by term count)
  std::vector<int64_t> hp(C.nnz + 1);
  GMG_CK(cudaMemcpyAsync(hp.data(), C.plan_ptr, (C.nnz + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaStreamSynchronize(s));
  std::vector<int32_t> up;
  plan_order(C.nnz, hp, up);
  const int64_t nup = (int64_t)up.size();
  if (nup == 0) {
    set_error("Galerkin level " + std::to_string(l + 1) + ": empty product");
    return GMG_ERR_INVALID_ARG;
  }
  const int64_t nsl = (nup + 31) / 32;
  std::vector<int64_t> sptr(nsl + 1, 0);
  C.plan_long_slices = 0;
  for (int64_t g = 0; g < nsl; ++g) {
    const int64_t width = hp[up[32 * g] + 1] - hp[up[32 * g]];
    sptr[g + 1] = sptr[g] + 32 * width;
    if (width > kGalLongWidth) C.plan_long_slices = g + 1;  // widths are non-increasing
  }
  while ((int64_t)up.size() < 32 * nsl) up.push_back(up.back());  // pad the last slice with a repeated entry
  C.plan_nup = 32 * nsl;
  // CSR position of every entry's mirror (K, J), -1 on the diagonal
  std::vector<int32_t> mfull;
  if (!mirror_positions(nc, hrp, hcol, mfull)) {
    set_error("Galerkin level " + std::to_string(l + 1) + ": pattern not symmetric");
    return GMG_ERR_INVALID_ARG;
  }
  std::vector<int32_t> mir(up.size());
  for (size_t i = 0; i < up.size(); ++i) mir[i] = mfull[up[i]];
  GMG_TRY(upload(c->arena, &C.plan_mirror, mir.data(), mir.size()));
  GMG_TRY(upload(c->arena, &C.plan_up, up.data(), up.size()));
  GMG_TRY(upload(c->arena, &C.plan_sptr, sptr.data(), sptr.size()));
  GMG_TRY(c->arena.alloc(&C.plan_sedge, (size_t)sptr.back()));
  GMG_TRY(c->arena.alloc(&C.plan_scoef, (size_t)sptr.back()));
  k_plan_slice<<<grid_for(C.plan_nup, 256), 256, 0, s>>>(C.plan_nup, C.plan_up, C.plan_ptr, C.plan_edge, C.plan_coef,
                                                          C.plan_sptr, C.plan_sedge, C.plan_scoef);
  GMG_LAUNCHED();
  GMG_CK(cudaStreamSynchronize(s));
  c->arena.release_one(C.plan_edge);
  c->arena.release_one(C.plan_coef);
  c->arena.release_one(C.plan_ptr);
  c->arena.release_one(terms);
  C.plan_edge = nullptr;
  C.plan_coef = nullptr;
  C.plan_ptr = nullptr;
  return GMG_OK;
}

// Numeric part of every Galerkin level, value scatter into the solve layout,
// and the coarsest factorisation.  Runs entirely on the GPU.
gmg_status join_inverse(gmg_ctx* c, cudaStream_t s, bool check) {
  if (c->inv_pending) {
    GMG_CK(cudaStreamWaitEvent(s, c->ev_inv, 0));
    c->inv_pending = false;
    c->inv_check = true;
  }
  return check ? inverse_status(c, s) : GMG_OK;
}

gmg_status inverse_status(gmg_ctx* c, cudaStream_t s) {
  if (!c->inv_check) return GMG_OK;
  int h = 0;
  GMG_CK(cudaMemcpyAsync(&h, c->dstatus + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaStreamSynchronize(s));
  c->inv_check = false;
  if (h) {
    set_error("coarsest operator not positive definite (sweep pivot <= 0)");
    return GMG_ERR_CHOLESKY;
  }
  return GMG_OK;
}

gmg_status numeric_setup(gmg_ctx* c, cudaStream_t s, bool defer) {
  GMG_TRY(join_inverse(c, s, false));  // the previous inverse still reads the dense work matrix
  c->inv_check = false;
  GMG_CK(cudaMemsetAsync(c->dstatus, 0, 2 * sizeof(int), s));
  // level 1's product first: it gathers level 0's CSR values, which the copy
  // that brought them has just left in L2 (the finest scatter streams far
  // more than L2 holds and would push them out)
  std::vector<int> order;
  if (c->nlev > 1) order.push_back(1);
  order.push_back(0);
  for (int l = 2; l < c->nlev; ++l) order.push_back(l);
  for (int l : order) {
    Level& F = c->L[l];
    if (l > 0) {
      Level& P = c->L[l - 1];
      const int64_t nsl = F.plan_nup / 32, nlong = F.plan_long_slices;
      if (nlong > 0) {
        k_gal_level<16><<<grid_for(nlong * 32, kGalThreads, 152 * 128), kGalThreads, 0, s>>>(
            0, nlong, F.plan_up, F.plan_mirror, F.plan_sptr, F.plan_sedge, F.plan_scoef, P.csr_val, F.csr_val,
            F.csr2ell, F.A.v64, F.A.v32, F.diag64, F.diag32, F.dinv64, F.dinv32, c->dstatus);
        GMG_LAUNCHED();
      }
      if (nsl > nlong) {
        k_gal_level<8><<<grid_for((nsl - nlong) * 32, kGalThreads, 152 * 128), kGalThreads, 0, s>>>(
            nlong, nsl, F.plan_up, F.plan_mirror, F.plan_sptr, F.plan_sedge, F.plan_scoef, P.csr_val, F.csr_val,
            F.csr2ell, F.A.v64, F.A.v32, F.diag64, F.diag32, F.dinv64, F.dinv32, c->dstatus);
        GMG_LAUNCHED();
      }
    } else {
      k_scatter_rows<<<grid_for(F.A.nslice * 32, 256), 256, 0, s>>>(
          F.A.nslice, F.A.ptr, F.A.row0, F.A.nrow, F.perm, F.csr_rowptr, F.csr_col, F.csr_val, F.A.v64, F.A.v32,
          F.diag64, F.diag32, F.dinv64, F.dinv32, c->dstatus);
      GMG_LAUNCHED();
    }
  }
  GMG_TRY(refresh_cluster_values(c, s));
  // coarsest: explicit inverse by block sweeps (on the handle's own stream when deferred)
  const cudaStream_t s_main = s;
  if (defer) {
    if (!c->inv_stream) GMG_CK(cudaStreamCreateWithFlags(&c->inv_stream, cudaStreamNonBlocking));
    if (!c->ev_gal) GMG_CK(cudaEventCreateWithFlags(&c->ev_gal, cudaEventDisableTiming));
    if (!c->ev_inv) GMG_CK(cudaEventCreateWithFlags(&c->ev_inv, cudaEventDisableTiming));
    GMG_CK(cudaEventRecord(c->ev_gal, s));
    GMG_CK(cudaStreamWaitEvent(c->inv_stream, c->ev_gal, 0));
    s = c->inv_stream;
  }
  Level& C = c->L[c->nlev - 1];
  const int n = (int)c->nco;
  const int nbk = (n + 31) / 32, npad = nbk * 32;
  double* Dinv[2] = {c->dbuf, c->dbuf + 1024};
  double* Uo = c->dbuf + 2048;
  double* Uh = Uo + (size_t)npad * 32;
  GMG_CK(cudaMemsetAsync(c->gj_cnt, 0, sizeof(int) * (size_t)(2 * nbk), s));  // arrival and work counters
  k_gj_pad<<<grid_for((int64_t)npad * npad, 256), 256, 0, s>>>(npad, n, c->dense);
  GMG_LAUNCHED();
  k_csr_to_dense<<<std::min(n, 4096), 128, 0, s>>>(n, npad, C.csr_rowptr, C.csr_col, C.csr_val, C.iperm, c->dense);
  GMG_LAUNCHED();
  GMG_TRY(launch(k_gj_first, 1, 256, s, npad, (const double*)c->dense, Dinv[0], c->dstatus + 1));
  for (int p = 0; p < nbk; ++p) {
    GMG_TRY(launch(k_gj_panel, npad / 8, 256, s, npad, p, (const double*)c->dense, (const double*)Dinv[p & 1], Uo,
                   Uh));
    GMG_TRY(launch(k_gj_update, std::min<int64_t>(c->nsm, (int64_t)4 * nbk * (nbk + 1) / 2), 256, s, npad, p,
                   c->dense, (const double*)Dinv[p & 1], (const double*)Uo, (const double*)Uh, c->gj_cnt,
                   c->gj_cnt + nbk, Dinv[(p + 1) & 1], c->dstatus + 1));
  }
  GMG_TRY(launch(k_gj_finish, grid_for((int64_t)n * n, 256), 256, s, n, npad, (const double*)c->dense, c->Ainv,
                 c->Ainv32));
  int h[2] = {0, 0};
  if (defer) {
    // the Galerkin values are checked now; the inverse's pivot check at the join
    GMG_CK(cudaEventRecord(c->ev_inv, s));
    c->inv_pending = true;
    s = s_main;
    GMG_CK(cudaMemcpyAsync(h, c->dstatus, sizeof(int), cudaMemcpyDeviceToHost, s));
  } else {
    GMG_CK(cudaMemcpyAsync(h, c->dstatus, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  }
  GMG_CK(cudaStreamSynchronize(s));
  if (h[0] & 2) {
    set_error("non-finite value in a level operator");
    return GMG_ERR_NONFINITE;
  }
  if (h[0] & 1) {
    set_error("non-positive diagonal in a level operator");
    return GMG_ERR_NOT_SPD;
  }
  if (h[1]) {
    set_error("coarsest operator not positive definite (sweep pivot <= 0)");
    return GMG_ERR_CHOLESKY;
  }
  c->values_ready = true;
  return GMG_OK;
}

// ---- validation (host) ----
static gmg_status validate(const gmg_csr* A, int nP, const gmg_prolong* P, const int32_t* const* coloring,
                           double* unity_dev) {
  if (!A || A->n <= 0 || !A->rowptr || !A->col || !A->val) {
    set_error("A: null pointer or n <= 0");
    return GMG_ERR_INVALID_ARG;
  }
  const int64_t n = A->n;
  if (n > INT32_MAX) {
    set_error("A: n exceeds the 32-bit column index range");
    return GMG_ERR_TOO_LARGE;
  }
  if (A->rowptr[0] != 0) {
    set_error("A: rowptr[0] != 0");
    return GMG_ERR_INVALID_ARG;
  }
  for (int64_t i = 0; i < n; ++i) {
    if (A->rowptr[i + 1] < A->rowptr[i]) {
      set_error("A: rowptr not monotone");
      return GMG_ERR_INVALID_ARG;
    }
    bool diag = false;
    for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) {
      const int32_t j = A->col[k];
      if (j < 0 || j >= n || (k > A->rowptr[i] && j <= A->col[k - 1])) {
        set_error("A: column indices out of range, unsorted or repeated in row " + std::to_string(i));
        return GMG_ERR_INVALID_ARG;
      }
      if (!std::isfinite(A->val[k])) {
        set_error("A: non-finite value in row " + std::to_string(i));
        return GMG_ERR_NONFINITE;
      }
      if (j == i) {
        diag = true;
        if (!(A->val[k] > 0.0)) {
          set_error("A: diagonal entry <= 0 in row " + std::to_string(i));
          return GMG_ERR_NOT_SPD;
        }
      }
    }
    if (!diag) {
      set_error("A: missing diagonal in row " + std::to_string(i));
      return GMG_ERR_NOT_SPD;
    }
  }
  // symmetry: every (i, j) has a matching (j, i) with the same value.  Rows
  // i in increasing order meet the entries (j, i) of each row j in the order
  // they are stored (sorted columns), so one cursor per row pairs them.
  {
    std::vector<int64_t> cur(A->rowptr, A->rowptr + n);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) {
        const int32_t j = A->col[k];
        const int64_t q = cur[j]++;
        if (q >= A->rowptr[j + 1] || A->col[q] != i || A->val[q] != A->val[k]) {
          set_error("A: not symmetric at (" + std::to_string(i) + ", " + std::to_string(j) + ")");
          return GMG_ERR_NOT_SPD;
        }
      }
    for (int64_t j = 0; j < n; ++j)
      if (cur[j] != A->rowptr[j + 1]) {
        set_error("A: not symmetric in row " + std::to_string(j));
        return GMG_ERR_NOT_SPD;
      }
  }
  int64_t nf = n;
  for (int l = 0; l < nP; ++l) {
    const gmg_prolong& p = P[l];
    if (p.n_fine != nf || p.n_coarse <= 0 || p.n_coarse >= INT32_MAX || !p.idx || !p.w) {
      set_error("P[" + std::to_string(l) + "]: sizes do not chain or null pointer");
      return GMG_ERR_INVALID_ARG;
    }
    std::vector<char> used(p.n_coarse, 0);
    for (int64_t i = 0; i < nf; ++i) {
      const double wsum = p.w[3 * i] + p.w[3 * i + 1] + p.w[3 * i + 2];
      if (std::isfinite(wsum)) *unity_dev = std::max(*unity_dev, std::fabs(wsum - 1.0));
      for (int s = 0; s < 3; ++s) {
        const int32_t k = p.idx[3 * i + s];
        const double w = p.w[3 * i + s];
        if (k < 0 || k >= p.n_coarse) {
          set_error("P[" + std::to_string(l) + "]: index out of range in row " + std::to_string(i));
          return GMG_ERR_INVALID_ARG;
        }
        if (!std::isfinite(w)) {
          set_error("P[" + std::to_string(l) + "]: non-finite weight in row " + std::to_string(i));
          return GMG_ERR_NONFINITE;
        }
        if (w != 0.0) {
          for (int s2 = 0; s2 < s; ++s2)
            if (p.w[3 * i + s2] != 0.0 && p.idx[3 * i + s2] == k) {
              set_error("P[" + std::to_string(l) + "]: repeated coarse index in row " + std::to_string(i));
              return GMG_ERR_INVALID_ARG;
            }
          used[k] = 1;
        }
      }
    }
    for (int64_t k = 0; k < p.n_coarse; ++k)
      if (!used[k]) {
        set_error("P[" + std::to_string(l) + "]: coarse point " + std::to_string(k) + " has no fine row");
        return GMG_ERR_EMPTY_P_COLUMN;
      }
    nf = p.n_coarse;
  }
  if (nf > kMaxCoarse) {
    set_error("coarsest level has " + std::to_string(nf) + " rows (limit " + std::to_string(kMaxCoarse) + ")");
    return GMG_ERR_TOO_LARGE;
  }
  // a caller colouring of level 0 is checked here, before any device work
  // (the coarse levels' patterns are known only after the symbolic product)
  if (coloring && coloring[0] && check_colouring(0, n, A->rowptr, A->col, coloring[0]) < 0)
    return GMG_ERR_INVALID_ARG;
  return GMG_OK;
}

// Tail of the FP32 cycle: the smoothed levels l0 .. lambda-1 (at most
// kMaxTail, l0 >= 1) and the coarsest level run as one cluster launch when
// their shared-memory copies fit in kTailSmemLimit bytes per CTA; l0 is the
// smallest level index that fits.  16 CTAs per cluster if the device can
// schedule them, else 8; off if neither fits or GMG_NO_TAIL=1.
static gmg_status build_tail(gmg_ctx* c, const std::vector<std::vector<int64_t>>& hrp,
                             const std::vector<std::vector<int32_t>>& hcol,
                             const std::vector<std::vector<int32_t>>& perm,
                             const std::vector<std::vector<int32_t>>& iperm, const gmg_prolong* P) {
  c->tail_l0 = 0;
  const int lam = c->nlev - 1;
  if (const char* e = std::getenv("GMG_NO_TAIL"))
    if (e[0] == '1') return GMG_OK;
  if (lam < 2) return GMG_OK;
  auto al = [](int64_t v) { return (v + 15) & ~(int64_t)15; };
  // slice tables of every candidate level (host)
  std::vector<std::vector<int64_t>> ptr(c->nlev);
  std::vector<std::vector<int32_t>> row0(c->nlev), nrow(c->nlev);
  for (int l = std::max(1, lam - kMaxTail); l < lam; ++l) {
    const int64_t ns = c->L[l].A.nslice;
    ptr[l].resize(ns + 1);
    row0[l].resize(ns);
    nrow[l].resize(ns);
    GMG_CK(cudaMemcpy(ptr[l].data(), c->L[l].A.ptr, ptr[l].size() * sizeof(int64_t), cudaMemcpyDeviceToHost));
    GMG_CK(cudaMemcpy(row0[l].data(), c->L[l].A.row0, ns * sizeof(int32_t), cudaMemcpyDeviceToHost));
    GMG_CK(cudaMemcpy(nrow[l].data(), c->L[l].A.nrow, ns * sizeof(int32_t), cudaMemcpyDeviceToHost));
  }
  // cluster size and threads per CTA (GMG_TAIL_CTAS, GMG_TAIL_THREADS override)
  std::vector<int> sizes = {16, 8};
  int threads = 1024;
  if (const char* e = std::getenv("GMG_TAIL_CTAS")) sizes = {std::atoi(e)};
  if (const char* e = std::getenv("GMG_TAIL_THREADS")) threads = std::atoi(e);
  if (threads < 32 || threads > 1024 || threads % 32 != 0) threads = 1024;
  for (int ncta : sizes) {
    if (ncta < 1 || ncta > 16) continue;
    for (int l0 = std::max(1, lam - kMaxTail); l0 < lam; ++l0) {
      TailDesc D{};
      std::vector<std::vector<int32_t>> soff(lam), own(lam), ocs(lam), owner(lam);
      std::vector<std::vector<uint16_t>> mask(lam);
      int64_t cur = 0;
      for (int l = l0; l < lam; ++l) {
        Level& L = c->L[l];
        TailLevel& T = D.lv[l - l0];
        const int64_t ns = L.A.nslice, n = L.n;
        soff[l].assign(ns, 0);
        // a slice belongs to the CTA of its first row's range of the caller's
        // numbering, so that a row's neighbours mostly share its CTA
        std::vector<int32_t> slice_cta(ns);
        owner[l].assign(n, 0);
        for (int64_t sl = 0; sl < ns; ++sl) {
          slice_cta[sl] = (int32_t)((int64_t)c->L[l].h_key[perm[l][row0[l][sl]]] * ncta / n);
          for (int q = 0; q < nrow[l][sl]; ++q) owner[l][row0[l][sl] + q] = slice_cta[sl];
        }
        int64_t emax = 0, maxown = 0;
        std::vector<std::vector<int32_t>> ownl(ncta);
        ocs[l].assign((size_t)ncta * (L.ncolor + 1), 0);
        for (int cta = 0; cta < ncta; ++cta) {
          int64_t off = 0;
          for (int k = 0; k < L.ncolor; ++k) {
            ocs[l][(size_t)cta * (L.ncolor + 1) + k] = (int32_t)ownl[cta].size();
            for (int64_t sl = L.color_slice_off[k]; sl < L.color_slice_off[k + 1]; ++sl)
              if (slice_cta[sl] == cta) {
                soff[l][sl] = (int32_t)off;
                off += ptr[l][sl + 1] - ptr[l][sl];
                ownl[cta].push_back((int32_t)sl);
              }
          }
          ocs[l][(size_t)cta * (L.ncolor + 1) + L.ncolor] = (int32_t)ownl[cta].size();
          emax = std::max(emax, off);
          maxown = std::max<int64_t>(maxown, (int64_t)ownl[cta].size());
        }
        maxown = std::max<int64_t>(maxown, 1);
        own[l].assign(ncta * maxown, -1);
        for (int cta = 0; cta < ncta; ++cta)
          std::copy(ownl[cta].begin(), ownl[cta].end(), own[l].begin() + cta * maxown);
        // the CTAs other than its owner that read a row's x: owners of its
        // neighbours, and (below) owners of the finer tail level's rows that
        // prolongate from it
        mask[l].assign(n, 0);
        for (int64_t r = 0; r < n; ++r) {
          const int32_t old = perm[l][r];
          for (int64_t e = hrp[l][old]; e < hrp[l][old + 1]; ++e)
            mask[l][r] |= (uint16_t)(1u << owner[l][iperm[l][hcol[l][e]]]);
        }
        if (l > l0) {
          const gmg_prolong& Pf = P[l - 1];
          for (int64_t i = 0; i < Pf.n_fine; ++i)
            for (int q = 0; q < 3; ++q)
              if (Pf.w[3 * i + q] != 0.0)
                mask[l][iperm[l][Pf.idx[3 * i + q]]] |= (uint16_t)(1u << owner[l - 1][iperm[l - 1][i]]);
        }
        for (int64_t r = 0; r < n; ++r) mask[l][r] &= (uint16_t)~(1u << owner[l][r]);
        T.maxown = (int)maxown;
        T.n = (int)L.n;
        T.nc0 = (int)L.color_off[1];
        T.ncolor = L.ncolor;
        T.nslice = (int)ns;
        T.r_nslice = (int)L.R.nslice;
        T.o_x = (int)cur; cur = al(cur + 4 * L.n);
        T.o_r = (int)cur; cur = al(cur + 4 * L.n);
        T.o_b = (int)cur; cur = al(cur + 4 * L.n);
        T.o_dinv = (int)cur; cur = al(cur + 4 * L.n);
        T.o_diag = (int)cur; cur = al(cur + 4 * L.n);
        T.o_row0 = (int)cur; cur = al(cur + 4 * ns);
        T.o_nrow = (int)cur; cur = al(cur + 4 * ns);
        T.o_width = (int)cur; cur = al(cur + 4 * ns);
        T.o_soff = (int)cur; cur = al(cur + 4 * ns);
        T.o_cso = (int)cur; cur = al(cur + 4 * (L.ncolor + 1));
        T.o_own = (int)cur; cur = al(cur + 4 * T.maxown);
        T.o_ocs = (int)cur; cur = al(cur + 4 * (L.ncolor + 1));
        T.o_mask = (int)cur; cur = al(cur + 2 * L.n);
        T.o_val = (int)cur; cur = al(cur + 4 * emax);
        T.o_col = (int)cur; cur = al(cur + 4 * emax);
      }
      D.nc = (int)c->L[lam].n;
      D.o_xc = (int)cur; cur = al(cur + 4 * D.nc);
      D.o_bc = (int)cur; cur = al(cur + 4 * D.nc);
      if (cur > kTailSmemLimit) continue;
      bool ok = false;
      GMG_TRY(tail_configure(c, ncta, threads, (int)cur, &ok));
      if (!ok) break;  // this cluster size cannot be scheduled: try the next
      // fill the global pointers and upload the per-slice tables
      for (int l = l0; l < lam; ++l) {
        Level& L = c->L[l];
        TailLevel& T = D.lv[l - l0];
        int32_t *so, *cs, *ow;
        GMG_TRY(upload(c->arena, &so, soff[l].data(), soff[l].size()));
        GMG_TRY(upload(c->arena, &ow, own[l].data(), own[l].size()));
        T.own = ow;
        int32_t* oc;
        uint16_t* mk;
        GMG_TRY(upload(c->arena, &oc, ocs[l].data(), ocs[l].size()));
        GMG_TRY(upload(c->arena, &mk, mask[l].data(), mask[l].size()));
        T.ocs = oc;
        T.mask = mk;
        std::vector<int32_t> cso32(L.color_slice_off.begin(), L.color_slice_off.end());
        GMG_TRY(upload(c->arena, &cs, cso32.data(), cso32.size()));
        T.soff = so;
        T.cso = cs;
        T.a_ptr = L.A.ptr;
        T.a_row0 = L.A.row0;
        T.a_nrow = L.A.nrow;
        T.a_col = L.A.col;
        T.a_v32 = L.A.v32;
        T.dinv32 = L.dinv32;
        T.diag32 = L.diag32;
        T.r_ptr = L.R.ptr;
        T.r_row0 = L.R.row0;
        T.r_nrow = L.R.nrow;
        T.r_col = L.R.col;
        T.r_v32 = L.R.v32;
        T.p_idx = L.p_idx;
        T.p_w32 = L.p_w32;
        T.x32 = L.x32;
        T.b32 = L.b32;
      }
      D.ntail = lam - l0;
      D.ncta = ncta;
      D.nu_pre = c->opt.nu_pre;
      D.nu_post = c->opt.nu_post;
      D.post_forward = c->opt.post_forward;
      D.c0_first = c->opt.nu_pre > 0 ? 1 : 0;
      D.ainv32 = c->Ainv32;
      c->tail = D;
      c->tail_smem = (int)cur;
      c->tail_threads = threads;
      c->tail_l0 = l0;
      return GMG_OK;
    }
  }
  return GMG_OK;
}

gmg_status setup_impl(gmg_ctx* c, const gmg_csr* A, int nP, const gmg_prolong* P, const int32_t* const* coloring,
                      cudaStream_t s) {
  // wall time of the set-up's parts, printed with GMG_VERBOSE=1
  using clk = std::chrono::steady_clock;
  const clk::time_point t_start = clk::now();
  double t_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  clk::time_point t_last = t_start;
  NvtxRange nv("gmg_setup: validation and uploads");
  auto lap = [&](int k, const char* next = nullptr) {
    const clk::time_point t = clk::now();
    t_ms[k] += std::chrono::duration<double, std::milli>(t - t_last).count();
    t_last = t;
    if (next) nv.next(next);
  };
  c->p_unity_dev = 0.0;
  GMG_TRY(validate(A, nP, P, coloring, &c->p_unity_dev));
  GMG_CK(cudaGetDevice(&c->device));
  GMG_CK(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device));
  Arena& a = c->arena;
  c->nlev = nP + 1;
  c->L.resize(c->nlev);
  GMG_TRY(a.alloc(&c->dstatus, 4));
  // level 0 CSR (caller numbering)
  Level& L0 = c->L[0];
  L0.n = A->n;
  L0.nnz = A->rowptr[A->n];
  GMG_TRY(upload(a, &L0.csr_rowptr, A->rowptr, L0.n + 1));
  GMG_TRY(upload(a, &L0.csr_col, A->col, L0.nnz));
  GMG_TRY(upload(a, &L0.csr_val, A->val, L0.nnz));
  // prolongations and their transposes in caller numbering
  for (int l = 0; l < nP; ++l) {
    Level& F = c->L[l];
    const gmg_prolong& p = P[l];
    F.nc = p.n_coarse;
    c->L[l + 1].n = p.n_coarse;
    GMG_TRY(upload(a, &F.p_idx_o, p.idx, 3 * p.n_fine));
    GMG_TRY(upload(a, &F.p_w_o, p.w, 3 * p.n_fine));
    std::vector<int64_t> cnt(p.n_coarse + 1, 0);
    for (int64_t i = 0; i < p.n_fine; ++i)
      for (int q = 0; q < 3; ++q)
        if (p.w[3 * i + q] != 0.0) cnt[p.idx[3 * i + q] + 1]++;
    for (int64_t J = 0; J < p.n_coarse; ++J) cnt[J + 1] += cnt[J];
    std::vector<int32_t> tc(cnt.back());
    std::vector<double> tw(cnt.back());
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t i = 0; i < p.n_fine; ++i)
      for (int q = 0; q < 3; ++q)
        if (p.w[3 * i + q] != 0.0) {
          const int64_t pos = fill[p.idx[3 * i + q]]++;
          tc[pos] = (int32_t)i;
          tw[pos] = p.w[3 * i + q];
        }
    GMG_TRY(upload(a, &F.pt_rowptr_o, cnt.data(), cnt.size()));
    GMG_TRY(upload(a, &F.pt_col_o, tc.data(), tc.size()));
    GMG_TRY(upload(a, &F.pt_w_o, tw.data(), tw.size()));
  }
  // symbolic Galerkin levels (patterns come back to the host for colouring)
  std::vector<std::vector<int64_t>> hrp(c->nlev);
  std::vector<std::vector<int32_t>> hcol(c->nlev);
  hrp[0].assign(A->rowptr, A->rowptr + A->n + 1);
  hcol[0].assign(A->col, A->col + L0.nnz);
  // each level's greedy colouring starts on host threads once its pattern is
  // here, overlapping the device's symbolic pass of the next level
  std::vector<std::unique_ptr<ColourJob>> jobs(c->nlev);
  for (auto& j : jobs) j.reset(new ColourJob);
  auto start_colouring = [&](int l) {
    if (!(coloring && coloring[l])) jobs[l]->start(c->L[l].n, hrp[l].data(), hcol[l].data());
  };
  lap(0, "gmg_setup: symbolic Galerkin product");
  start_colouring(0);
  for (int l = 0; l + 1 < c->nlev; ++l) {
    GMG_TRY(galerkin_symbolic(c, l, s, hrp[l + 1], hcol[l + 1]));
    start_colouring(l + 1);
  }
  locality_ranks(c, hrp, hcol, P);
  lap(1, "gmg_setup: colouring wait");
  for (auto& j : jobs) j->join();
  lap(2, "gmg_setup: level layouts");
  // colouring, renumbering, layouts
  std::vector<std::vector<int32_t>> perm(c->nlev), iperm(c->nlev);
  for (int l = 0; l < c->nlev; ++l)
    GMG_TRY(build_level_structure(c, l, hrp[l].data(), hcol[l].data(), coloring ? coloring[l] : nullptr, *jobs[l],
                                  perm[l], iperm[l]));
  lap(6, "gmg_setup: transfer layouts");
  for (int l = 0; l + 1 < c->nlev; ++l)
    GMG_TRY(build_transfer_structure(c, l, P[l], perm[l], iperm[l], perm[l + 1], iperm[l + 1]));
  lap(7, "gmg_setup: vectors");
  // coarsest dense buffers
  c->nco = c->L[c->nlev - 1].n;
  {
    const int64_t nbk = (c->nco + 31) / 32, npad = 32 * nbk;
    GMG_TRY(a.alloc(&c->dense, (size_t)(npad * npad)));
    GMG_TRY(a.alloc(&c->Ainv, (size_t)(c->nco * c->nco)));
    GMG_TRY(a.alloc(&c->Ainv32, (size_t)(c->nco * c->nco)));
    GMG_TRY(a.alloc(&c->dbuf, (size_t)(2048 + 64 * npad)));  // two pivot inverses, panel U and U D^-1
    GMG_TRY(a.alloc(&c->gj_cnt, (size_t)(2 * nbk)));
  }
  // outer-iteration vectors
  const int64_t n = L0.n;
  c->xs = L0.x64;  // the FP64 cycle runs directly on the outer iterate
  c->bs = L0.b64;
  GMG_TRY(a.alloc(&c->rs, n));
  GMG_TRY(a.alloc(&c->zs, n));
  GMG_TRY(a.alloc(&c->ps, n));
  GMG_TRY(a.alloc(&c->qs, n));
  GMG_TRY(a.alloc(&c->ros, n));
  GMG_TRY(a.alloc(&c->io, n));
  GMG_TRY(a.alloc(&c->io2, n));
  // one partial per residual block: with rows split over G warps a block covers 8 / G slices,
  // so up to one block per slice (G = 8)
  c->red_cap = std::max<int64_t>(4 * kRedBlocks, L0.A.nslice + 64);
  GMG_TRY(a.alloc(&c->red, (size_t)c->red_cap));
  GMG_TRY(a.alloc(&c->scal, 64));
  GMG_TRY(a.alloc(&c->dloop, 2));
  GMG_TRY(a.alloc(&c->red_cnt, 4));
  GMG_CK(cudaMemset(c->red_cnt, 0, 4 * sizeof(int)));
  GMG_TRY(a.alloc(&c->dhist, (size_t)c->opt.max_iter + 2));
  GMG_CK(cudaMallocHost((void**)&c->h_scal, 64 * sizeof(double)));
  lap(3, "gmg_setup: tail and cluster level");
  GMG_TRY(build_tail(c, hrp, hcol, perm, iperm, P));
  if (c->tail_l0 >= 2) {
    const int l = c->tail_l0 - 1;
    GMG_TRY(build_cluster_level(c, l, hrp[l].data(), hcol[l].data(), perm[l], iperm[l]));
  }
  lap(4, "gmg_setup: numeric set-up");
  const gmg_status st = numeric_setup(c, s, false);
  if (const char* e = std::getenv("GMG_VERBOSE"))
    if (e[0] == '1' && st == GMG_OK) {
      cudaStreamSynchronize(s);
      lap(5);
      std::fprintf(stderr,
                   "gmg: set-up %.1f ms: validation and uploads %.1f, symbolic Galerkin %.1f, colouring wait %.1f, "
                   "level layouts %.1f, transfer layouts %.1f, vectors %.1f, tail and cluster level %.1f, "
                   "numeric set-up %.1f; in all: %lld cudaMalloc %.1f, uploads %.1f\n",
                   std::chrono::duration<double, std::milli>(t_last - t_start).count(), t_ms[0], t_ms[1], t_ms[2],
                   t_ms[6], t_ms[7], t_ms[3], t_ms[4], t_ms[5], (long long)c->arena.n_alloc, c->arena.ms_alloc,
                   c->arena.ms_copy);
    }
  return st;
}

}  // namespace gmg

namespace gmg {
__global__ void k_pivot_reciprocal(int64_t n, const double* __restrict__ d, double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = recip_newton(d[i]);
}
__global__ void k_convert(int64_t n, int dir, const void* __restrict__ in, void* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (dir == 0)
      static_cast<float*>(out)[i] = f32_rn(static_cast<const double*>(in)[i]);
    else
      static_cast<double*>(out)[i] = f64_of(static_cast<const float*>(in)[i]);
  }
}
}  // namespace gmg

// The library's colouring of a symmetric pattern, on the host.
extern "C" gmg_status gmg_colour(int64_t n, const int64_t* rowptr, const int32_t* col, int32_t* color,
                                 int32_t* ncolor) {
  using namespace gmg;
  if (n < 0 || !rowptr || !ncolor || (n > 0 && (!col || !color))) {
    set_error("gmg_colour: negative size or null pointer");
    return GMG_ERR_INVALID_ARG;
  }
  if (n > INT32_MAX || rowptr[0] != 0) {
    set_error("gmg_colour: n exceeds the 32-bit index range or rowptr[0] != 0");
    return GMG_ERR_INVALID_ARG;
  }
  for (int64_t i = 0; i < n; ++i) {
    if (rowptr[i + 1] < rowptr[i]) {
      set_error("gmg_colour: rowptr not monotone");
      return GMG_ERR_INVALID_ARG;
    }
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
      if (col[k] < 0 || col[k] >= n || (k > rowptr[i] && col[k] <= col[k - 1])) {
        set_error("gmg_colour: column out of range, unsorted or repeated in row " + std::to_string(i));
        return GMG_ERR_INVALID_ARG;
      }
  }
  const std::vector<int64_t> rp(rowptr, rowptr + n + 1);
  const std::vector<int32_t> ci(col, col + rowptr[n]);
  std::vector<int32_t> mirror;
  if (!mirror_positions(n, rp, ci, mirror)) {
    set_error("gmg_colour: pattern not symmetric");
    return GMG_ERR_INVALID_ARG;
  }
  if (n == 0) {
    *ncolor = 0;
    return GMG_OK;
  }
  ColourJob job;
  job.start(n, rp.data(), ci.data());
  std::vector<int32_t> c;
  *ncolor = job.finish(c);
  std::copy(c.begin(), c.end(), color);
  return GMG_OK;
}

// The reciprocal the coarsest inverse takes of every pivot, applied to n
// device values (exposed so that its accuracy can be checked against the
// correctly rounded FP64 division).
extern "C" gmg_status gmg_pivot_reciprocal(int64_t n, const double* d, double* out, void* stream) {
  using namespace gmg;
  if (n < 0 || (n > 0 && (!d || !out))) {
    set_error("gmg_pivot_reciprocal: negative size or null pointer");
    return GMG_ERR_INVALID_ARG;
  }
  if (n == 0) return GMG_OK;
  const int64_t grid = std::min<int64_t>((n + 255) / 256, 152 * 16);
  k_pivot_reciprocal<<<(unsigned)grid, 256, 0, (cudaStream_t)stream>>>(n, d, out);
  GMG_LAUNCHED();
  return GMG_OK;
}

// The precision conversions of the solver's kernels (done on the bits),
// applied to n device values (exposed so that they can be checked against
// the IEEE 754 conversions).
extern "C" gmg_status gmg_convert(int64_t n, int dir, const void* in, void* out, void* stream) {
  using namespace gmg;
  if (n < 0 || (dir != 0 && dir != 1) || (n > 0 && (!in || !out))) {
    set_error("gmg_convert: negative size, direction not 0 or 1, or null pointer");
    return GMG_ERR_INVALID_ARG;
  }
  if (n == 0) return GMG_OK;
  const int64_t grid = std::min<int64_t>((n + 255) / 256, 152 * 16);
  k_convert<<<(unsigned)grid, 256, 0, (cudaStream_t)stream>>>(n, dir, in, out);
  GMG_LAUNCHED();
  return GMG_OK;
}
