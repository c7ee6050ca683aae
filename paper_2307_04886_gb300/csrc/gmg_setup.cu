// Setup of the multigrid hierarchy (Alg. 1, lines "build level matrix"):
//  * validation of A and P_l (host);
//  * Galerkin product A_{l+1} = P_l^T A_l P_l on the GPU: a symbolic pass
//    (per-row hash sets in shared memory: count, scan, sorted fill) and a
//    numeric pass with a fixed accumulation order, then mirrored to exact
//    symmetry (the entry below the diagonal takes the value above it);
//  * greedy colouring and colour-major renumbering (host, integer work);
//  * sliced-ELL layout of every level and of every restriction P_l^T;
//  * dense FP64 Cholesky of the coarsest level and its explicit inverse.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "gmg_internal.cuh"

namespace gmg {

thread_local std::string g_last_error;
thread_local uint64_t g_launches = 0;
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

// Numeric pass: value of every entry = sum over its plan of coef * A_l value,
// multiplied and added with separate roundings in plan order.
__global__ void __launch_bounds__(256)
    k_gal_apply(int64_t nnz, const int64_t* __restrict__ plan_ptr, const int32_t* __restrict__ plan_edge,
                const double* __restrict__ plan_coef, const double* __restrict__ a_val, double* __restrict__ c_val) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int64_t t = plan_ptr[e]; t < plan_ptr[e + 1]; ++t)
      acc = __dadd_rn(acc, __dmul_rn(plan_coef[t], a_val[plan_edge[t]]));
    c_val[e] = acc;
  }
}

// Exact symmetry: entry (J, K) with K < J takes the value of (K, J).
__global__ void k_gal_mirror(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                             double* __restrict__ val) {
  for (int64_t J = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; J < n; J += (int64_t)gridDim.x * blockDim.x) {
    for (int64_t k = rp[J]; k < rp[J + 1]; ++k) {
      const int32_t K = col[k];
      if (K >= J) break;
      int64_t lo = rp[K], hi = rp[K + 1] - 1;
      while (lo <= hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int32_t cm = col[mid];
        if (cm < J) lo = mid + 1;
        else if (cm > J) hi = mid - 1;
        else {
          val[k] = val[mid];
          break;
        }
      }
    }
  }
}

// CSR values -> sliced-ELL values, diagonal and inverse diagonal (both
// precisions).  err bit 1: diagonal <= 0; bit 2: non-finite value.
__global__ void k_scatter_values(int64_t nnz, const int64_t* __restrict__ csr2ell, const double* __restrict__ v,
                                 double* __restrict__ e64, float* __restrict__ e32, double* __restrict__ d64,
                                 float* __restrict__ d32, double* __restrict__ di64, float* __restrict__ di32,
                                 int* __restrict__ err) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = csr2ell[e];
    const double x = v[e];
    if (!isfinite(x)) atomicOr(err, 2);
    if (m >= 0) {
      e64[m] = x;
      e32[m] = (float)x;
    } else {
      const int64_t r = -1 - m;
      if (!(x > 0.0)) atomicOr(err, 1);
      d64[r] = x;
      d32[r] = (float)x;
      di64[r] = 1.0 / x;
      di32[r] = (float)(1.0 / x);
    }
  }
}

// Dense coarsest operator in the level's colour-permuted numbering (the
// numbering of the vectors the cycle hands to the coarse solve).
__global__ void k_csr_to_dense(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                               const double* __restrict__ val, const int32_t* __restrict__ iperm,
                               double* __restrict__ D) {
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const int64_t pi = iperm[i];
    for (int64_t k = rp[i] + threadIdx.x; k < rp[i + 1]; k += blockDim.x) D[pi * n + iperm[col[k]]] = val[k];
  }
}

// ---- dense FP64 Cholesky, right-looking, 32 x 32 blocks ----
// k_chol_panel factors the diagonal block p in every CTA's shared memory
// (identical arithmetic in every CTA), CTA 0 stores the factor L_pp in Dbuf,
// and every CTA solves its rows below the block: L_ip = A_ip L_pp^-T.
// k_chol_update then applies the trailing update; k_chol_store_diag writes
// the stored diagonal factors into A once all steps are done (block p of A is
// not read again after step p).  status bit 0: a pivot <= 0.
__device__ void chol_factor_block(double (&D)[32][33], double (&rdiag)[32], int nb, int* bad) {
  for (int k = 0; k < nb; ++k) {
    if (threadIdx.x == 0) {
      double d = D[k][k];
      if (!(d > 0.0)) {
        *bad = 1;
        d = 1.0;
      }
      const double l = sqrt(d);
      D[k][k] = l;
      rdiag[k] = 1.0 / l;
    }
    __syncthreads();
    for (int r = k + 1 + threadIdx.x; r < nb; r += blockDim.x) D[r][k] *= rdiag[k];
    __syncthreads();
    for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) {
      const int r = idx >> 5, c = idx & 31;
      if (c > k && r >= c && r < nb) D[r][c] -= D[r][k] * D[c][k];
    }
    __syncthreads();
  }
}

__global__ void k_chol_panel(int n, int p, double* __restrict__ A, double* __restrict__ Dbuf,
                             int* __restrict__ status) {
  __shared__ double D[32][33];
  __shared__ double rdiag[32];
  __shared__ int bad;
  const int j0 = p * 32;
  const int nb = min(32, n - j0);
  if (threadIdx.x == 0) bad = 0;
  for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) {
    const int r = idx >> 5, c = idx & 31;
    D[r][c] = (r < nb && c < nb) ? A[(int64_t)(j0 + r) * n + j0 + c] : (r == c ? 1.0 : 0.0);
  }
  __syncthreads();
  chol_factor_block(D, rdiag, nb, &bad);
  if (blockIdx.x == 0) {
    if (bad && threadIdx.x == 0) atomicOr(status, 1);
    for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) {
      const int r = idx >> 5, c = idx & 31;
      Dbuf[(int64_t)p * 1024 + idx] = (c <= r) ? D[r][c] : 0.0;
    }
  }
  const int i = j0 + nb + blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    double v[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) v[c] = c < nb ? A[(int64_t)i * n + j0 + c] : 0.0;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      if (c < nb) {
        double s = v[c];
#pragma unroll
        for (int k = 0; k < c; ++k) s -= v[k] * D[c][k];
        v[c] = s * rdiag[c];
      }
    }
#pragma unroll
    for (int c = 0; c < 32; ++c)
      if (c < nb) A[(int64_t)i * n + j0 + c] = v[c];
  }
}

__global__ void k_chol_store_diag(int n, const double* __restrict__ Dbuf, double* __restrict__ A) {
  const int p = blockIdx.x;
  const int j0 = p * 32;
  const int nb = min(32, n - j0);
  for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) {
    const int r = idx >> 5, c = idx & 31;
    if (r < nb && c < nb) A[(int64_t)(j0 + r) * n + j0 + c] = Dbuf[(int64_t)p * 1024 + idx];
  }
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

// Trailing update A_IJ -= L_Ip L_Jp^T for the lower tiles right of block p.
__global__ void k_chol_update(int n, int p, double* __restrict__ A) {
  __shared__ double Li[32][33], Lj[32][33];
  const int nbk = (n + 31) / 32;
  int I, J;
  lower_tile(blockIdx.x, p + 1, nbk, &I, &J);
  const int j0 = p * 32;
  for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) {
    const int r = idx >> 5, k = idx & 31;
    const int gi = I * 32 + r, gj = J * 32 + r, gk = j0 + k;
    Li[r][k] = (gi < n && gk < n) ? A[(int64_t)gi * n + gk] : 0.0;
    Lj[r][k] = (gj < n && gk < n) ? A[(int64_t)gj * n + gk] : 0.0;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) {
    const int r = idx >> 5, c = idx & 31;
    const int gi = I * 32 + r, gj = J * 32 + c;
    if (gi < n && gj < n && gj <= gi) {
      double s = 0.0;
#pragma unroll 8
      for (int k = 0; k < 32; ++k) s += Li[r][k] * Lj[c][k];
      A[(int64_t)gi * n + gj] -= s;
    }
  }
}

// rdiag[i] = 1 / L_ii
__global__ void k_recip_diag(int n, const double* __restrict__ Lf, double* __restrict__ rdiag) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    rdiag[i] = 1.0 / Lf[(int64_t)i * n + i];
}

// Wt = (L^-1)^T: row k of Wt is column k of L^-1, by forward substitution
// (one warp per column; Wt must be zero-initialised).
__global__ void k_tri_inverse(int n, const double* __restrict__ Lf, const double* __restrict__ rdiag,
                              double* __restrict__ Wt) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  const int k = warp;
  double* w = Wt + (int64_t)k * n;
  if (lane == 0) w[k] = rdiag[k];
  __syncwarp();
  for (int i = k + 1; i < n; ++i) {
    const double* Li = Lf + (int64_t)i * n;
    double s = 0.0;
    for (int m = k + lane; m < i; m += 32) s += Li[m] * w[m];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) w[i] = -s * rdiag[i];
    __syncwarp();
  }
}

// Ainv = L^-T L^-1: Ainv_ij = sum_k Wt[i][k] Wt[j][k]; lower tiles computed,
// both halves written.
__global__ void k_inv_gram(int n, const double* __restrict__ Wt, double* __restrict__ Ainv) {
  __shared__ double Ti[32][33], Tj[32][33];
  const int nbk = (n + 31) / 32;
  int I, J;
  lower_tile(blockIdx.x, 0, nbk, &I, &J);
  double acc[4] = {0, 0, 0, 0};
  for (int kb = I; kb < nbk; ++kb) {  // Wt[i][k] = 0 for k < i
    __syncthreads();
    for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) {
      const int r = idx >> 5, k = idx & 31;
      const int gi = I * 32 + r, gj = J * 32 + r, gk = kb * 32 + k;
      Ti[r][k] = (gi < n && gk < n) ? Wt[(int64_t)gi * n + gk] : 0.0;
      Tj[r][k] = (gj < n && gk < n) ? Wt[(int64_t)gj * n + gk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = threadIdx.x + q * 256;
      const int r = idx >> 5, c = idx & 31;
      double s = 0.0;
#pragma unroll 8
      for (int k = 0; k < 32; ++k) s += Ti[r][k] * Tj[c][k];
      acc[q] += s;
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int idx = threadIdx.x + q * 256;
    const int r = idx >> 5, c = idx & 31;
    const int gi = I * 32 + r, gj = J * 32 + c;
    if (gi < n && gj < n) {
      Ainv[(int64_t)gi * n + gj] = acc[q];
      Ainv[(int64_t)gj * n + gi] = acc[q];
    }
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
  if (n) GMG_CK(cudaMemcpy(*d, h, n * sizeof(T), cudaMemcpyHostToDevice));
  return GMG_OK;
}

// Greedy first-fit colouring in increasing row index over the pattern.
static int greedy_colour(int64_t n, const int64_t* rp, const int32_t* ci, std::vector<int32_t>& color) {
  color.assign(n, 0);
  std::vector<int64_t> mark(n + 1, -1);
  int ncol = 0;
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] < i) mark[color[ci[k]]] = i;
    int32_t c = 0;
    while (mark[c] == i) ++c;
    color[i] = c;
    ncol = std::max(ncol, c + 1);
  }
  return ncol;
}

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

// Colours level l, renumbers it colour by colour (ascending caller index within
// a colour), and builds the sliced-ELL layout of its off-diagonal part.
static gmg_status build_level_structure(gmg_ctx* c, int l, const int64_t* rp, const int32_t* ci,
                                        std::vector<int32_t>& perm, std::vector<int32_t>& iperm) {
  Level& L = c->L[l];
  const int64_t n = L.n;
  std::vector<int32_t> color;
  L.ncolor = greedy_colour(n, rp, ci, color);
  L.h_color = color;
  L.color_off.assign(L.ncolor + 1, 0);
  for (int64_t i = 0; i < n; ++i) L.color_off[color[i] + 1]++;
  for (int k = 0; k < L.ncolor; ++k) L.color_off[k + 1] += L.color_off[k];
  perm.assign(n, 0);
  iperm.assign(n, 0);
  {
    std::vector<int64_t> fill(L.color_off.begin(), L.color_off.end() - 1);
    for (int64_t i = 0; i < n; ++i) {
      const int64_t r = fill[color[i]]++;
      perm[r] = (int32_t)i;
      iperm[i] = (int32_t)r;
    }
  }
  std::vector<int64_t> rowlen(n);
  for (int64_t r = 0; r < n; ++r) rowlen[r] = rp[perm[r] + 1] - rp[perm[r]] - 1;
  EllPlan P;
  plan_slices(L.color_off, rowlen, P, &L.color_slice_off);
  std::vector<int32_t> ecol(P.ptr.back());
  std::vector<int64_t> c2e(rp[n]);
  for (size_t s = 0; s < P.row0.size(); ++s) {
    const int64_t w = (P.ptr[s + 1] - P.ptr[s]) / kSlice;
    for (int lane = 0; lane < kSlice; ++lane) {
      const int64_t r = P.row0[s] + lane;
      int64_t k = 0;
      if (lane < P.nrow[s]) {
        const int64_t old = perm[r];
        for (int64_t e = rp[old]; e < rp[old + 1]; ++e) {
          if (ci[e] == old) {
            c2e[e] = -1 - r;
          } else {
            const int64_t slot = P.ptr[s] + k * kSlice + lane;
            ecol[slot] = iperm[ci[e]];
            c2e[e] = slot;
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
  }
  GMG_TRY(upload(a, &L.csr2ell, c2e.data(), c2e.size()));
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
  GMG_CK(cudaStreamSynchronize(s));
  return GMG_OK;
}

// Numeric part of every Galerkin level, value scatter into the solve layout,
// and the coarsest factorisation.  Runs entirely on the GPU.
gmg_status numeric_setup(gmg_ctx* c, cudaStream_t s) {
  GMG_CK(cudaMemsetAsync(c->dstatus, 0, 2 * sizeof(int), s));
  for (int l = 0; l < c->nlev; ++l) {
    Level& F = c->L[l];
    if (l > 0) {
      Level& P = c->L[l - 1];
      k_gal_apply<<<grid_for(F.nnz, 256), 256, 0, s>>>(F.nnz, F.plan_ptr, F.plan_edge, F.plan_coef, P.csr_val,
                                                      F.csr_val);
      GMG_LAUNCHED();
      k_gal_mirror<<<grid_for(F.n, 256), 256, 0, s>>>(F.n, F.csr_rowptr, F.csr_col, F.csr_val);
      GMG_LAUNCHED();
    }
    k_scatter_values<<<grid_for(F.nnz, 256), 256, 0, s>>>(F.nnz, F.csr2ell, F.csr_val, F.A.v64, F.A.v32, F.diag64,
                                                         F.diag32, F.dinv64, F.dinv32, c->dstatus);
    GMG_LAUNCHED();
  }
  // coarsest: dense Cholesky and explicit inverse
  Level& C = c->L[c->nlev - 1];
  const int n = (int)c->nco;
  GMG_CK(cudaMemsetAsync(c->dense, 0, sizeof(double) * (size_t)n * n, s));
  k_csr_to_dense<<<std::min(n, 4096), 128, 0, s>>>(n, C.csr_rowptr, C.csr_col, C.csr_val, C.iperm, c->dense);
  GMG_LAUNCHED();
  const int nbk = (n + 31) / 32;
  for (int p = 0; p < nbk; ++p) {
    const int below = n - std::min(n, (p + 1) * 32);
    k_chol_panel<<<std::max(1, (below + 127) / 128), 128, 0, s>>>(n, p, c->dense, c->dbuf, c->dstatus + 1);
    GMG_LAUNCHED();
    const int T = nbk - p - 1;
    if (T > 0) {
      k_chol_update<<<T * (T + 1) / 2, 256, 0, s>>>(n, p, c->dense);
      GMG_LAUNCHED();
    }
  }
  k_chol_store_diag<<<nbk, 256, 0, s>>>(n, c->dbuf, c->dense);
  GMG_LAUNCHED();
  k_recip_diag<<<(n + 255) / 256, 256, 0, s>>>(n, c->dense, c->dbuf);
  GMG_LAUNCHED();
  GMG_CK(cudaMemsetAsync(c->Winv, 0, sizeof(double) * (size_t)n * n, s));
  k_tri_inverse<<<(n + 3) / 4, 128, 0, s>>>(n, c->dense, c->dbuf, c->Winv);
  GMG_LAUNCHED();
  k_inv_gram<<<nbk * (nbk + 1) / 2, 256, 0, s>>>(n, c->Winv, c->Ainv);
  GMG_LAUNCHED();
  int h[2] = {0, 0};
  GMG_CK(cudaMemcpyAsync(h, c->dstatus, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
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
    set_error("Cholesky pivot <= 0 on the coarsest level");
    return GMG_ERR_CHOLESKY;
  }
  c->values_ready = true;
  return GMG_OK;
}

// ---- validation (host) ----
static gmg_status validate(const gmg_csr* A, int nP, const gmg_prolong* P) {
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
  // symmetry: every (i, j) has a matching (j, i) with the same value
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) {
      const int32_t j = A->col[k];
      if (j <= i) continue;
      const int32_t* b = A->col + A->rowptr[j];
      const int32_t* e = A->col + A->rowptr[j + 1];
      const int32_t* f = std::lower_bound(b, e, (int32_t)i);
      if (f == e || *f != i || A->val[A->rowptr[j] + (f - b)] != A->val[k]) {
        set_error("A: not symmetric at (" + std::to_string(i) + ", " + std::to_string(j) + ")");
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
    for (int64_t i = 0; i < nf; ++i)
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
  return GMG_OK;
}

// Descriptors of every level for the persistent small-level kernel; the
// first level with at most kClusterMaxRows rows (below the finest) starts it.
static gmg_status build_small_level_descriptors(gmg_ctx* c) {
  // Off by default: measured on GB300 (1M-vertex torus) a cluster phase costs
  // 3-4 us against about 2 us for a PDL-chained launch.  GMG_CLUSTER_L0=l
  // starts the cluster kernel at level l.
  c->cluster_l0 = 0;
  if (const char* e = std::getenv("GMG_CLUSTER_L0")) c->cluster_l0 = std::atoi(e);
  if (c->cluster_l0 < 0 || c->cluster_l0 >= c->nlev) c->cluster_l0 = 0;
  std::vector<DevLevel> d(c->nlev);
  for (int l = 0; l < c->nlev; ++l) {
    Level& L = c->L[l];
    DevLevel& v = d[l];
    std::memset(&v, 0, sizeof(v));
    v.n = L.n;
    v.ncolor = L.ncolor;
    v.lanes = L.lanes;
    int64_t* cso;
    GMG_TRY(upload(c->arena, &cso, L.color_slice_off.data(), L.color_slice_off.size()));
    v.cso = cso;
    v.nslice = L.A.nslice;
    v.a_ptr = L.A.ptr;
    v.a_row0 = L.A.row0;
    v.a_nrow = L.A.nrow;
    v.a_col = L.A.col;
    v.a_v32 = L.A.v32;
    v.a_v64 = L.A.v64;
    v.dinv32 = L.dinv32;
    v.diag32 = L.diag32;
    v.dinv64 = L.dinv64;
    v.diag64 = L.diag64;
    v.r_nslice = L.R.nslice;
    v.r_ptr = L.R.ptr;
    v.r_row0 = L.R.row0;
    v.r_nrow = L.R.nrow;
    v.r_col = L.R.col;
    v.r_v32 = L.R.v32;
    v.r_v64 = L.R.v64;
    v.p_idx = L.p_idx;
    v.p_w32 = L.p_w32;
    v.p_w64 = L.p_w64;
    v.x32 = L.x32;
    v.b32 = L.b32;
    v.r32 = L.r32;
    v.x64 = L.x64;
    v.b64 = L.b64;
    v.r64 = L.r64;
  }
  return upload(c->arena, &c->dlv, d.data(), d.size());
}

gmg_status setup_impl(gmg_ctx* c, const gmg_csr* A, int nP, const gmg_prolong* P, cudaStream_t s) {
  GMG_TRY(validate(A, nP, P));
  GMG_CK(cudaGetDevice(&c->device));
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
  for (int l = 0; l + 1 < c->nlev; ++l) GMG_TRY(galerkin_symbolic(c, l, s, hrp[l + 1], hcol[l + 1]));
  // colouring, renumbering, layouts
  std::vector<std::vector<int32_t>> perm(c->nlev), iperm(c->nlev);
  for (int l = 0; l < c->nlev; ++l)
    GMG_TRY(build_level_structure(c, l, hrp[l].data(), hcol[l].data(), perm[l], iperm[l]));
  for (int l = 0; l + 1 < c->nlev; ++l)
    GMG_TRY(build_transfer_structure(c, l, P[l], perm[l], iperm[l], perm[l + 1], iperm[l + 1]));
  // coarsest dense buffers
  c->nco = c->L[c->nlev - 1].n;
  GMG_TRY(a.alloc(&c->dense, (size_t)(c->nco * c->nco)));
  GMG_TRY(a.alloc(&c->Winv, (size_t)(c->nco * c->nco)));
  GMG_TRY(a.alloc(&c->Ainv, (size_t)(c->nco * c->nco)));
  GMG_TRY(a.alloc(&c->dbuf, (size_t)(((c->nco + 31) / 32) * 1024 + c->nco)));
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
  GMG_TRY(a.alloc(&c->red, (size_t)std::max<int64_t>(4 * kRedBlocks, L0.A.nslice / 8 + 64)));
  GMG_TRY(a.alloc(&c->scal, 64));
  GMG_CK(cudaMallocHost((void**)&c->h_scal, 64 * sizeof(double)));
  GMG_TRY(build_small_level_descriptors(c));
  return numeric_setup(c, s);
}

}  // namespace gmg
