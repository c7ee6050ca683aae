// Many right-hand sides at once (SpMM-style V-cycle): every level's vectors
// are [n_l x NR] row-major in the permuted numbering, so each matrix entry is
// read once and applied to NR contiguous values (NR = 1, 2, 4, 8 or 16; the
// caller's nrhs is padded with zero columns).  The inner cycle runs in FP32
// (coarsest solve in FP64) inside FP64 iterative refinement, as in Alg. 1
// with the correction form x += MGI(0, b - A x).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <string>

#include "gmg_cycle.cuh"

namespace gmg {

template <int NR>
struct alignas(16) Row {
  float v[NR];
};

template <int NR>
__device__ __forceinline__ void load_row(const float* __restrict__ p, float (&o)[NR]) {
  if constexpr (NR % 4 == 0) {
#pragma unroll
    for (int c = 0; c < NR; c += 4) {
      const float4 q = __ldg(reinterpret_cast<const float4*>(p + c));
      o[c] = q.x;
      o[c + 1] = q.y;
      o[c + 2] = q.z;
      o[c + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int c = 0; c < NR; ++c) o[c] = __ldg(p + c);
  }
}

template <int NR>
__device__ __forceinline__ void store_row(float* __restrict__ p, const float (&o)[NR]) {
  if constexpr (NR % 4 == 0) {
#pragma unroll
    for (int c = 0; c < NR; c += 4) *reinterpret_cast<float4*>(p + c) = make_float4(o[c], o[c + 1], o[c + 2], o[c + 3]);
  } else {
#pragma unroll
    for (int c = 0; c < NR; ++c) p[c] = o[c];
  }
}

// One warp's share of a slice row for a launch that splits every row over G
// warps (warp `part` takes entries k = part, part + G, ...); 8 / G slices per
// block of 256 threads.
struct MRow {
  bool active;
  int nk;
  int64_t e, r;
};
template <int G>
__device__ __forceinline__ MRow m_row(int64_t s, int64_t s_end, const int64_t* __restrict__ ptr,
                                      const int32_t* __restrict__ row0, const int32_t* __restrict__ nrow, int part,
                                      int lane) {
  MRow m{false, 0, 0, 0};
  if (s < s_end) {
    m.active = lane < nrow[s];
    const int64_t e0 = ptr[s];
    const int w = (int)((ptr[s + 1] - e0) >> 5);
    m.nk = (m.active && part < w) ? (w - part + G - 1) / G : 0;
    m.e = e0 + (int64_t)part * 32 + lane;
    m.r = row0[s] + lane;
  }
  return m;
}

// acc[c] += sum over this warp's entries of a_rk X[k][c], entries in order.
template <int NR, int G>
__device__ __forceinline__ void m_dot(const MRow& m, const int32_t* __restrict__ col, const float* __restrict__ val,
                                      const float* X, float (&acc)[NR]) {
  int64_t e = m.e;
  for (int q = 0; q < m.nk; ++q, e += (int64_t)G * 32) {
    const float a = val[e];
    float xv[NR];
    load_row<NR>(X + (int64_t)col[e] * NR, xv);
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[c] += a * xv[c];
  }
}

// Adds the other G - 1 warps' partial sums to row part 0's, in warp order.
template <int NR, int G>
__device__ __forceinline__ void m_combine(float (&acc)[NR], int warp, int lane) {
  if constexpr (G > 1) {
    __shared__ float red[8][NR][32];
#pragma unroll
    for (int c = 0; c < NR; ++c) red[warp][c][lane] = acc[c];
    __syncthreads();
    if (warp % G == 0)
      for (int g = 1; g < G; ++g)
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[c] += red[warp + g][c][lane];
  }
}

// One colour of a multi-right-hand-side Gauss-Seidel sweep, rows split over G warps.
template <int NR, int G>
__global__ void __launch_bounds__(256) k_gs_m(int64_t s0, int64_t s1, const int64_t* __restrict__ ptr,
                                              const int32_t* __restrict__ row0, const int32_t* __restrict__ nrow,
                                              const int32_t* __restrict__ col, const float* __restrict__ val,
                                              const float* __restrict__ dinv, const float* __restrict__ B, float* X) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, part = warp % G;
  const int64_t s = s0 + (int64_t)blockIdx.x * (8 / G) + warp / G;
  const MRow m = m_row<G>(s, s1, ptr, row0, nrow, part, lane);
  float acc[NR], bv[NR];
#pragma unroll
  for (int c = 0; c < NR; ++c) acc[c] = bv[c] = 0.f;
  float d = 0.f;
  if (part == 0 && m.active) {  // issued with the gathers, not after the combining barrier
    load_row<NR>(B + m.r * NR, bv);
    d = dinv[m.r];
  }
  m_dot<NR, G>(m, col, val, X, acc);  // other colours: not written by this launch
  m_combine<NR, G>(acc, warp, lane);
  if (part == 0 && m.active) {
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[c] = (bv[c] - acc[c]) * d;
    store_row<NR>(X + m.r * NR, acc);
  }
}

// R = B - A X over all slices, rows split over G warps.
template <int NR, int G>
__global__ void __launch_bounds__(256) k_residual_m(int64_t nslice, const int64_t* __restrict__ ptr,
                                                    const int32_t* __restrict__ row0, const int32_t* __restrict__ nrow,
                                                    const int32_t* __restrict__ col, const float* __restrict__ val,
                                                    const float* __restrict__ diag, const float* __restrict__ X,
                                                    const float* __restrict__ B, float* __restrict__ R) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, part = warp % G;
  const int64_t s = (int64_t)blockIdx.x * (8 / G) + warp / G;
  const MRow m = m_row<G>(s, nslice, ptr, row0, nrow, part, lane);
  float acc[NR], bv[NR];
#pragma unroll
  for (int c = 0; c < NR; ++c) acc[c] = bv[c] = 0.f;
  if (part == 0 && m.active) {
    float xv[NR];
    load_row<NR>(X + m.r * NR, xv);
    load_row<NR>(B + m.r * NR, bv);  // issued with the gathers, not after the combining barrier
    const float d = diag[m.r];
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[c] = d * xv[c];
  }
  m_dot<NR, G>(m, col, val, X, acc);
  m_combine<NR, G>(acc, warp, lane);
  if (part == 0 && m.active) {
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[c] = bv[c] - acc[c];
    store_row<NR>(R + m.r * NR, acc);
  }
}

template <int NR>
__global__ void __launch_bounds__(256) k_restrict_m(int64_t nslice, const int64_t* __restrict__ ptr,
                                                    const int32_t* __restrict__ row0, const int32_t* __restrict__ nrow,
                                                    const int32_t* __restrict__ col, const float* __restrict__ w,
                                                    const float* __restrict__ R, float* __restrict__ Bc) {
  const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= nslice || lane >= nrow[s]) return;
  const int64_t e0 = ptr[s];
  const int wd = (int)((ptr[s + 1] - e0) >> 5);
  float acc[NR], rv[NR];
#pragma unroll
  for (int c = 0; c < NR; ++c) acc[c] = 0.f;
  int64_t e = e0 + lane;
  for (int k = 0; k < wd; ++k, e += 32) {
    const float a = w[e];
    load_row<NR>(R + (int64_t)col[e] * NR, rv);
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[c] += a * rv[c];
  }
  store_row<NR>(Bc + (int64_t)(row0[s] + lane) * NR, acc);
}

template <int NR>
__global__ void __launch_bounds__(256) k_prolong_m(int64_t n, const int32_t* __restrict__ idx,
                                                   const float* __restrict__ w, const float* __restrict__ U,
                                                   float* __restrict__ X) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float xv[NR], u[NR];
    load_row<NR>(X + i * NR, xv);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const float a = w[3 * i + m];
      load_row<NR>(U + (int64_t)idx[3 * i + m] * NR, u);
#pragma unroll
      for (int c = 0; c < NR; ++c) xv[c] += a * u[c];
    }
    store_row<NR>(X + i * NR, xv);
  }
}

// X = Ainv B on the coarsest level (FP64 accumulation), one warp per row.
template <int NR>
__global__ void __launch_bounds__(256) k_coarse_m(int n, const double* __restrict__ Ainv, const float* __restrict__ B,
                                                  float* __restrict__ X) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  double s[NR];
#pragma unroll
  for (int c = 0; c < NR; ++c) s[c] = 0.0;
  const double* a = Ainv + (int64_t)row * n;
  for (int j = lane; j < n; j += 32) {
    const double aj = a[j];
#pragma unroll
    for (int c = 0; c < NR; ++c) s[c] += aj * f64_of(B[(int64_t)j * NR + c]);
  }
#pragma unroll
  for (int c = 0; c < NR; ++c)
    for (int o = 16; o > 0; o >>= 1) s[c] += __shfl_xor_sync(0xffffffffu, s[c], o);
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < NR; ++c) X[(int64_t)row * NR + c] = f32_rn(s[c]);
}

// FP64 outer residual R = B - A X with per-block, per-column partial sums of
// R^2 (fixed-shape reduction), and the correction cast R32 = (float) R.
template <int NR>
__global__ void __launch_bounds__(256) k_outer_residual_m(int64_t nslice, const int64_t* __restrict__ ptr,
                                                          const int32_t* __restrict__ row0,
                                                          const int32_t* __restrict__ nrow,
                                                          const int32_t* __restrict__ col,
                                                          const double* __restrict__ val,
                                                          const double* __restrict__ diag,
                                                          const double* __restrict__ X, const double* __restrict__ B,
                                                          float* __restrict__ R32, double* __restrict__ partial) {
  const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  double sq[NR];
#pragma unroll
  for (int c = 0; c < NR; ++c) sq[c] = 0.0;
  if (s < nslice && lane < nrow[s]) {
    const int64_t r = row0[s] + lane;
    const int64_t e0 = ptr[s];
    const int w = (int)((ptr[s + 1] - e0) >> 5);
    double acc[NR];
    const double d = diag[r];
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[c] = d * X[r * NR + c];
    int64_t e = e0 + lane;
    for (int k = 0; k < w; ++k, e += 32) {
      const double a = val[e];
      const double* xj = X + (int64_t)col[e] * NR;
#pragma unroll
      for (int c = 0; c < NR; ++c) acc[c] += a * xj[c];
    }
#pragma unroll
    for (int c = 0; c < NR; ++c) {
      const double rv = B[r * NR + c] - acc[c];
      R32[r * NR + c] = f32_rn(rv);
      sq[c] = rv * rv;
    }
  }
  __shared__ double red[NR][256];
#pragma unroll
  for (int c = 0; c < NR; ++c) red[c][threadIdx.x] = sq[c];
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o)
#pragma unroll
      for (int c = 0; c < NR; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < NR) partial[(int64_t)blockIdx.x * NR + threadIdx.x] = red[threadIdx.x][0];
}

// out[c] = sum over blocks of partial[b * NR + c] (fixed order).
__global__ void k_reduce_cols(int nblocks, int nr, const double* __restrict__ partial, double* __restrict__ out) {
  __shared__ double red[256];
  for (int c = 0; c < nr; ++c) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 256) s += partial[(int64_t)b * nr + c];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = red[0];
    __syncthreads();
  }
}

// Caller [n x nrhs] (double) -> permuted [n x NR] with zero padding, and back.
__global__ void k_gather_m(int64_t n, int nrhs, int NR, const int32_t* __restrict__ perm, const double* __restrict__ src,
                           double* __restrict__ dst) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * NR; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / NR;
    const int c = (int)(t % NR);
    dst[t] = c < nrhs ? src[(int64_t)perm[i] * nrhs + c] : 0.0;
  }
}
__global__ void k_scatter_m(int64_t n, int nrhs, int NR, const int32_t* __restrict__ perm,
                            const double* __restrict__ src, double* __restrict__ dst) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * nrhs;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / nrhs;
    const int c = (int)(t % nrhs);
    dst[(int64_t)perm[i] * nrhs + c] = src[i * NR + c];
  }
}
__global__ void k_zero_cols(int64_t n, int NR, int mask, double* __restrict__ X) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * NR; t += (int64_t)gridDim.x * blockDim.x)
    if ((mask >> (int)(t % NR)) & 1) X[t] = 0.0;
}
__global__ void k_add_f2d_m(int64_t m, const float* __restrict__ e, double* __restrict__ x) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += f64_of(e[i]);
}

static inline int nblk(int64_t threads) { return (int)std::max<int64_t>(1, (threads + 255) / 256); }
static inline int gblk(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 64)); }

#define LCK() GMG_LAUNCHED()

// The warps-per-row split of a level's multi-right-hand-side sweeps and
// residual for NR columns: the autotuned or set choice, else a default by the
// level's mean row length (about 8 entries per warp).
template <int NR>
static int m_lanes(const Level& L) {
  const int v = L.mlanes[nr_index(NR)];
  if (v > 0) return v;
  const double mean = L.n > 0 ? (double)L.nnz / (double)L.n : 1.0;
  return mean <= 12 ? 1 : mean <= 24 ? 2 : mean <= 48 ? 4 : 8;
}

template <int NR>
static gmg_status sweep_m(Level& L, int k, cudaStream_t s, int G = 0) {
  const int64_t s0 = L.color_slice_off[k], s1 = L.color_slice_off[k + 1];
  if (s1 <= s0) return GMG_OK;
  if (G == 0) G = m_lanes<NR>(L);
  const int64_t grid = (s1 - s0 + 8 / G - 1) / (8 / G);
  const Ell& A = L.A;
  switch (G) {
    case 1: k_gs_m<NR, 1><<<(unsigned)grid, 256, 0, s>>>(s0, s1, A.ptr, A.row0, A.nrow, A.col, A.v32, L.dinv32, L.B32, L.X32); break;
    case 2: k_gs_m<NR, 2><<<(unsigned)grid, 256, 0, s>>>(s0, s1, A.ptr, A.row0, A.nrow, A.col, A.v32, L.dinv32, L.B32, L.X32); break;
    case 4: k_gs_m<NR, 4><<<(unsigned)grid, 256, 0, s>>>(s0, s1, A.ptr, A.row0, A.nrow, A.col, A.v32, L.dinv32, L.B32, L.X32); break;
    default: k_gs_m<NR, 8><<<(unsigned)grid, 256, 0, s>>>(s0, s1, A.ptr, A.row0, A.nrow, A.col, A.v32, L.dinv32, L.B32, L.X32);
  }
  LCK();
  return GMG_OK;
}

template <int NR>
static gmg_status residual_m(Level& L, cudaStream_t s, int G = 0) {
  if (G == 0) G = m_lanes<NR>(L);
  const Ell& A = L.A;
  const int64_t grid = std::max<int64_t>(1, (A.nslice + 8 / G - 1) / (8 / G));
  switch (G) {
    case 1: k_residual_m<NR, 1><<<(unsigned)grid, 256, 0, s>>>(A.nslice, A.ptr, A.row0, A.nrow, A.col, A.v32, L.diag32, L.X32, L.B32, L.R32); break;
    case 2: k_residual_m<NR, 2><<<(unsigned)grid, 256, 0, s>>>(A.nslice, A.ptr, A.row0, A.nrow, A.col, A.v32, L.diag32, L.X32, L.B32, L.R32); break;
    case 4: k_residual_m<NR, 4><<<(unsigned)grid, 256, 0, s>>>(A.nslice, A.ptr, A.row0, A.nrow, A.col, A.v32, L.diag32, L.X32, L.B32, L.R32); break;
    default: k_residual_m<NR, 8><<<(unsigned)grid, 256, 0, s>>>(A.nslice, A.ptr, A.row0, A.nrow, A.col, A.v32, L.diag32, L.X32, L.B32, L.R32);
  }
  LCK();
  return GMG_OK;
}

// MGI(X_l, B_l, l) on [n_l x NR] blocks.  Every level starts from X_l = 0
// (the recursive calls of Alg. 2, and the correction cycle of the outer
// refinement on the finest level) unless keep_x, which keeps the caller's
// initial iterate in the finest level's X32.
template <int NR>
static gmg_status vcycle_m(gmg_ctx* c, int l, cudaStream_t s, bool keep_x = false) {
  Level& L = c->L[l];
  if (l == c->nlev - 1) {
    k_coarse_m<NR><<<(int)((L.n * 32 + 255) / 256), 256, 0, s>>>((int)L.n, c->Ainv, L.B32, L.X32);
    LCK();
    return GMG_OK;
  }
  Level& C = c->L[l + 1];
  if (!keep_x) GMG_CK(cudaMemsetAsync(L.X32, 0, sizeof(float) * (size_t)(L.n * NR), s));
  for (int it = 0; it < c->opt.nu_pre; ++it)
    for (int k = 0; k < L.ncolor; ++k) GMG_TRY(sweep_m<NR>(L, k, s));
  GMG_TRY(residual_m<NR>(L, s));
  k_restrict_m<NR><<<nblk(L.R.nslice * 32), 256, 0, s>>>(L.R.nslice, L.R.ptr, L.R.row0, L.R.nrow, L.R.col, L.R.v32,
                                                        L.R32, C.B32);
  LCK();
  GMG_TRY(vcycle_m<NR>(c, l + 1, s));
  k_prolong_m<NR><<<gblk(L.n), 256, 0, s>>>(L.n, L.p_idx, L.p_w32, C.X32, L.X32);
  LCK();
  for (int it = 0; it < c->opt.nu_post; ++it)
    for (int q = 0; q < L.ncolor; ++q) GMG_TRY(sweep_m<NR>(L, c->opt.post_forward ? q : L.ncolor - 1 - q, s));
  return GMG_OK;
}

// R = B - A X (FP64) -> level-0 B32 and per-column ||R||^2 into scal[8 + c].
template <int NR>
static gmg_status outer_m(gmg_ctx* c, cudaStream_t s) {
  Level& L = c->L[0];
  const int nb = nblk(L.A.nslice * 32);
  k_outer_residual_m<NR><<<nb, 256, 0, s>>>(L.A.nslice, L.A.ptr, L.A.row0, L.A.nrow, L.A.col, L.A.v64, L.diag64,
                                           c->XS, c->BS, L.B32, c->red);
  LCK();
  k_reduce_cols<<<1, 256, 0, s>>>(nb, NR, c->red, c->scal + 8);
  LCK();
  return GMG_OK;
}

template <int NR>
static gmg_status iteration_m(gmg_ctx* c, cudaStream_t s) {
  Level& L = c->L[0];
  GMG_TRY(vcycle_m<NR>(c, 0, s));
  k_add_f2d_m<<<gblk(L.n * NR), 256, 0, s>>>(L.n * NR, L.X32, c->XS);
  LCK();
  return outer_m<NR>(c, s);
}

static gmg_status ensure_batched(gmg_ctx* c) {
  if (c->XS) return GMG_OK;
  for (auto& L : c->L) {
    GMG_TRY(c->arena.alloc(&L.X32, (size_t)L.n * kMaxRhs));
    GMG_TRY(c->arena.alloc(&L.B32, (size_t)L.n * kMaxRhs));
    GMG_TRY(c->arena.alloc(&L.R32, (size_t)L.n * kMaxRhs));
  }
  const int64_t n = c->L[0].n;
  GMG_TRY(c->arena.alloc(&c->XS, (size_t)n * kMaxRhs));
  GMG_TRY(c->arena.alloc(&c->BS, (size_t)n * kMaxRhs));
  GMG_TRY(c->arena.alloc(&c->RS, (size_t)n * kMaxRhs));
  // per-column partials of the batched residual, and never smaller than the
  // single-vector partials the buffer already serves
  const int64_t need = std::max<int64_t>((int64_t)nblk(c->L[0].A.nslice * 32) * kMaxRhs + 64, c->red_cap);
  double* red2;
  GMG_TRY(c->arena.alloc(&red2, (size_t)need));
  c->red = red2;
  c->red_cap = need;
  return GMG_OK;
}

template <int NR>
static gmg_status solve_m(gmg_ctx* c, int nrhs, const double* B, double* X, double tol, int mem,
                          gmg_solve_info* info, cudaStream_t s) {
  Level& L0 = c->L[0];
  const int64_t n = L0.n;
  const size_t bytes = sizeof(double) * (size_t)(n * nrhs);
  const double* bsrc = B;
  const double* xsrc = X;
  if (mem == GMG_MEM_HOST) {
    GMG_CK(cudaMemcpyAsync(c->RS, B, bytes, cudaMemcpyHostToDevice, s));
    bsrc = c->RS;
  }
  k_gather_m<<<gblk(n * NR), 256, 0, s>>>(n, nrhs, NR, L0.perm, bsrc, c->BS);
  LCK();
  if (mem == GMG_MEM_HOST) {
    GMG_CK(cudaMemcpyAsync(c->RS, X, bytes, cudaMemcpyHostToDevice, s));
    xsrc = c->RS;
  }
  k_gather_m<<<gblk(n * NR), 256, 0, s>>>(n, nrhs, NR, L0.perm, xsrc, c->XS);
  LCK();
  // column norms of B: the outer residual with X = 0 (RS as a zero iterate)
  GMG_CK(cudaMemsetAsync(c->scal, 0, 64 * sizeof(double), s));
  double nb[kMaxRhs];
  bool all_zero = true;
  {
    double* keep = c->XS;
    c->XS = c->RS;
    GMG_CK(cudaMemsetAsync(c->RS, 0, sizeof(double) * (size_t)(n * NR), s));
    GMG_TRY(outer_m<NR>(c, s));
    c->XS = keep;
    GMG_CK(cudaMemcpyAsync(c->h_scal + 8, c->scal + 8, NR * sizeof(double), cudaMemcpyDeviceToHost, s));
    GMG_CK(cudaStreamSynchronize(s));
    int zmask = 0;
    for (int q = 0; q < nrhs; ++q) {
      nb[q] = std::sqrt(c->h_scal[8 + q]);
      if (nb[q] == 0.0) zmask |= 1 << q;
      else all_zero = false;
    }
    if (zmask) {  // a zero right-hand side has the solution 0
      k_zero_cols<<<gblk(n * NR), 256, 0, s>>>(n, NR, zmask, c->XS);
      LCK();
    }
  }
  auto worst = [&]() {
    double w = 0.0;
    for (int q = 0; q < nrhs; ++q) {
      const double r = nb[q] > 0 ? std::sqrt(c->h_scal[8 + q]) / nb[q] : 0.0;
      if (!std::isfinite(r)) return r;
      w = std::max(w, r);
    }
    return w;
  };
  GMG_TRY(outer_m<NR>(c, s));
  GMG_CK(cudaMemcpyAsync(c->h_scal + 8, c->scal + 8, NR * sizeof(double), cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaStreamSynchronize(s));
  double rel = worst();
  if (info && info->history && info->history_cap > 0) info->history[0] = rel;
  gmg_status st = GMG_ERR_NOT_CONVERGED;
  int k = 0;
  if (!std::isfinite(rel)) {
    st = GMG_ERR_NONFINITE;
  } else if (all_zero) {
    st = GMG_OK;
  } else {
    while (k < c->opt.max_iter) {
      GMG_TRY(iteration_m<NR>(c, s));
      GMG_CK(cudaMemcpyAsync(c->h_scal + 8, c->scal + 8, NR * sizeof(double), cudaMemcpyDeviceToHost, s));
      GMG_CK(cudaStreamSynchronize(s));
      ++k;
      rel = worst();
      if (info && info->history && k < info->history_cap) info->history[k] = rel;
      if (!std::isfinite(rel)) {
        st = GMG_ERR_NONFINITE;
        break;
      }
      if (rel <= tol) {
        st = GMG_OK;
        break;
      }
    }
  }
  double* dst = mem == GMG_MEM_HOST ? c->RS : X;
  k_scatter_m<<<gblk(n * nrhs), 256, 0, s>>>(n, nrhs, NR, L0.perm, c->XS, dst);
  LCK();
  if (mem == GMG_MEM_HOST) {
    GMG_CK(cudaMemcpyAsync(X, c->RS, bytes, cudaMemcpyDeviceToHost, s));
    GMG_CK(cudaStreamSynchronize(s));
  }
  if (info) {
    info->iters = k;
    info->rel_res = rel;
  }
  if (st == GMG_ERR_NOT_CONVERGED) set_error("gmg_solve_batched: max_iter reached");
  if (st == GMG_ERR_NONFINITE) set_error("gmg_solve_batched: non-finite residual");
  return st;
}

}  // namespace gmg

using namespace gmg;

extern "C" gmg_status gmg_solve_batched(gmg_handle h, int nrhs, const double* B, double* X, double tol, int mem,
                                        gmg_solve_info* info, void* stream) {
  gmg::NvtxRange nv("gmg_solve_batched");
  if (!h || !B || !X || nrhs < 1 || nrhs > kMaxRhs || !(tol >= 0.0) ||
      (mem != GMG_MEM_HOST && mem != GMG_MEM_DEVICE)) {
    set_error("gmg_solve_batched: bad handle, vector, nrhs (1..16), tolerance or memory kind");
    return GMG_ERR_INVALID_ARG;
  }
  GMG_CK(cudaSetDevice(h->device));
  GMG_TRY(ensure_batched(h));
  cudaStream_t s = (cudaStream_t)stream;
  GMG_TRY(join_inverse(h, s, true));
  if (nrhs == 1) return solve_m<1>(h, nrhs, B, X, tol, mem, info, s);
  if (nrhs == 2) return solve_m<2>(h, nrhs, B, X, tol, mem, info, s);
  if (nrhs <= 4) return solve_m<4>(h, nrhs, B, X, tol, mem, info, s);
  if (nrhs <= 8) return solve_m<8>(h, nrhs, B, X, tol, mem, info, s);
  return solve_m<16>(h, nrhs, B, X, tol, mem, info, s);
}

namespace gmg {
// One FP32 multi-right-hand-side V-cycle on the finest level, X <- MGI32(X, B):
// caller-numbered FP64 blocks in, rounded to FP32, the cycle, widened back.
template <int NR>
static gmg_status vcycle_step_m(gmg_ctx* c, int nrhs, const double* B, double* X, cudaStream_t s) {
  Level& L0 = c->L[0];
  const int64_t n = L0.n;
  k_gather_m<<<gblk(n * NR), 256, 0, s>>>(n, nrhs, NR, L0.perm, B, c->BS);
  LCK();
  k_gather_m<<<gblk(n * NR), 256, 0, s>>>(n, nrhs, NR, L0.perm, X, c->XS);
  LCK();
  GMG_TRY(launch_d2f(n * NR, c->BS, L0.B32, s));
  GMG_TRY(launch_d2f(n * NR, c->XS, L0.X32, s));
  GMG_TRY(vcycle_m<NR>(c, 0, s, true));
  GMG_TRY(launch_f2d(n * NR, L0.X32, c->XS, s));
  k_scatter_m<<<gblk(n * nrhs), 256, 0, s>>>(n, nrhs, NR, L0.perm, c->XS, X);
  LCK();
  return GMG_OK;
}
}  // namespace gmg

extern "C" gmg_status gmg_vcycle_batched(gmg_handle h, int nrhs, const double* B, double* X, void* stream) {
  if (!h || !B || !X || nrhs < 1 || nrhs > kMaxRhs) {
    set_error("gmg_vcycle_batched: bad handle, block or nrhs (1..16)");
    return GMG_ERR_INVALID_ARG;
  }
  GMG_CK(cudaSetDevice(h->device));
  GMG_TRY(ensure_batched(h));
  cudaStream_t s = (cudaStream_t)stream;
  GMG_TRY(join_inverse(h, s, true));
  if (nrhs == 1) return vcycle_step_m<1>(h, nrhs, B, X, s);
  if (nrhs == 2) return vcycle_step_m<2>(h, nrhs, B, X, s);
  if (nrhs <= 4) return vcycle_step_m<4>(h, nrhs, B, X, s);
  if (nrhs <= 8) return vcycle_step_m<8>(h, nrhs, B, X, s);
  return vcycle_step_m<16>(h, nrhs, B, X, s);
}

namespace gmg {
// Times every smoothed level's multi-right-hand-side sweeps (all colours, four
// sweeps) and residual for NR columns with each warps-per-row split G, as
// captured CUDA graphs (the way a solve runs them), and keeps the fastest G.
template <int NR>
static gmg_status autotune_m(gmg_ctx* c, int* lanes_out, cudaStream_t stream) {
  GMG_CK(cudaStreamSynchronize(stream));
  if (!c->g_stream) GMG_CK(cudaStreamCreateWithFlags(&c->g_stream, cudaStreamNonBlocking));
  cudaStream_t cs = c->g_stream;
  cudaEvent_t e0, e1;
  GMG_CK(cudaEventCreate(&e0));
  GMG_CK(cudaEventCreate(&e1));
  const uint64_t launches_before = g_launches;
  gmg_status st = GMG_OK;
  for (int l = 0; l + 1 < c->nlev && st == GMG_OK; ++l) {
    Level& L = c->L[l];
    if (cudaMemsetAsync(L.X32, 0, sizeof(float) * (size_t)(L.n * NR), cs) != cudaSuccess ||
        cudaMemsetAsync(L.B32, 0, sizeof(float) * (size_t)(L.n * NR), cs) != cudaSuccess) {
      st = GMG_ERR_CUDA;
      break;
    }
    float best_ms = 1e30f;
    int best = m_lanes<NR>(L);
    for (int G : {1, 2, 4, 8}) {
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        st = GMG_ERR_CUDA;
        break;
      }
      for (int sweep = 0; sweep < 4 && st == GMG_OK; ++sweep)
        for (int k = 0; k < L.ncolor && st == GMG_OK; ++k) st = sweep_m<NR>(L, k, cs, G);
      if (st == GMG_OK) st = residual_m<NR>(L, cs, G);
      const cudaError_t ec = cudaStreamEndCapture(cs, &g);
      if (st == GMG_OK && ec == cudaSuccess && cudaGraphInstantiate(&ge, g, 0) == cudaSuccess) {
        float ms = 0.f;
        cudaGraphLaunch(ge, cs);  // warm-up
        cudaEventRecord(e0, cs);
        for (int rep = 0; rep < 3; ++rep) cudaGraphLaunch(ge, cs);
        cudaEventRecord(e1, cs);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = GMG_ERR_CUDA;
        cudaEventElapsedTime(&ms, e0, e1);
        if (st == GMG_OK && ms < best_ms) {
          best_ms = ms;
          best = G;
        }
      } else if (st == GMG_OK) {
        set_error("gmg_autotune_batched: graph capture of the sweeps failed");
        st = GMG_ERR_CUDA;
      }
      if (ge) cudaGraphExecDestroy(ge);
      if (g) cudaGraphDestroy(g);
    }
    if (st == GMG_OK) L.mlanes[nr_index(NR)] = best;
    if (lanes_out) lanes_out[l] = L.mlanes[nr_index(NR)];
  }
  g_launches = launches_before;  // timing launches are not the caller's work
  cudaStreamSynchronize(cs);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

static int block_width(int nrhs) { return nrhs <= 1 ? 1 : nrhs <= 2 ? 2 : nrhs <= 4 ? 4 : nrhs <= 8 ? 8 : 16; }

static gmg_status autotune_batched(gmg_ctx* c, int nrhs, int* lanes_out, cudaStream_t s) {
  GMG_CK(cudaSetDevice(c->device));
  GMG_TRY(ensure_batched(c));
  switch (block_width(nrhs)) {
    case 1: return autotune_m<1>(c, lanes_out, s);
    case 2: return autotune_m<2>(c, lanes_out, s);
    case 4: return autotune_m<4>(c, lanes_out, s);
    case 8: return autotune_m<8>(c, lanes_out, s);
    default: return autotune_m<16>(c, lanes_out, s);
  }
}
}  // namespace gmg

extern "C" gmg_status gmg_autotune_batched(gmg_handle h, int nrhs, int* lanes_out, void* stream) {
  if (!h || nrhs < 1 || nrhs > kMaxRhs) {
    set_error("gmg_autotune_batched: bad handle or nrhs (1..16)");
    return GMG_ERR_INVALID_ARG;
  }
  return autotune_batched(h, nrhs, lanes_out, (cudaStream_t)stream);
}

extern "C" gmg_status gmg_set_lanes_batched(gmg_handle h, int nrhs, const int* lanes) {
  if (!h || nrhs < 1 || nrhs > kMaxRhs || !lanes) {
    set_error("gmg_set_lanes_batched: bad handle, nrhs (1..16) or null lanes");
    return GMG_ERR_INVALID_ARG;
  }
  for (int l = 0; l + 1 < h->nlev; ++l)
    if (lanes[l] != 1 && lanes[l] != 2 && lanes[l] != 4 && lanes[l] != 8) {
      set_error("gmg_set_lanes_batched: level " + std::to_string(l) + " split " + std::to_string(lanes[l]) +
                " is not 1, 2, 4 or 8");
      return GMG_ERR_INVALID_ARG;
    }
  const int slot = nr_index(block_width(nrhs));
  for (int l = 0; l + 1 < h->nlev; ++l) h->L[l].mlanes[slot] = lanes[l];
  return GMG_OK;
}

// ------------------------------------------------------------------ many meshes
// A batch of independent systems (meshes of uneven size), each with its own
// hierarchy and nrhs right-hand sides.  The whole solve is ONE graph launch:
// a conditional WHILE node repeats an iteration in which a gate kernel opens
// one conditional IF node per mesh that has not converged yet; the IF bodies
// (each mesh's multi-right-hand-side FP32 V-cycle, FP64 correction and FP64
// residual with column norms) run concurrently, and a check kernel then
// updates every mesh's relative residual, iteration count and done flag and
// decides whether the loop goes on.  The host reads the per-mesh results once
// at the end.  Where the CUDA driver refuses the conditional graph, one graph
// per iteration with every mesh's branch and a host-side test is used instead.

struct gmg_many_ctx {
  std::vector<gmg_handle> h;
  cudaStream_t cap = nullptr;
  std::vector<cudaStream_t> br;
  std::vector<cudaEvent_t> ev;
  cudaGraphExec_t graph[5] = {};  // host-driven form, by NR = 1, 2, 4, 8, 16
  uint64_t graph_kernels[5] = {};
  cudaGraphExec_t loop[5] = {};  // device-side loop, by NR
  uint64_t loop_kernels[5] = {};  // kernel nodes of one loop iteration (all meshes open)
  bool loop_refused[5] = {};
  // device state of the device-side loop
  int* d_state = nullptr;        // [0] iterations done, [1] limit, [2] non-finite seen; then per mesh: done, iters
  double* d_nb = nullptr;        // per mesh kMaxRhs column norms of B (0: column unused or zero)
  double* d_rel = nullptr;       // per mesh worst relative residual
  double* d_tol = nullptr;
  double** d_rr = nullptr;       // per mesh: its squared column norms of R (the handle's scal + 8)
  cudaGraphConditionalHandle* d_if = nullptr;  // per mesh IF handle (for the current NR's loop)
  std::vector<cudaGraphConditionalHandle> h_if[5];
};

namespace gmg {

static int nr_slot(int NR) { return NR == 1 ? 0 : NR == 2 ? 1 : NR == 4 ? 2 : NR == 8 ? 3 : 4; }

// Opens the IF node of every mesh that is not done.
__global__ void k_many_gate(int K, const int* __restrict__ state, const cudaGraphConditionalHandle* __restrict__ hif) {
  for (int k = threadIdx.x; k < K; k += blockDim.x) cudaGraphSetConditional(hif[k], state[3 + 2 * k] ? 0u : 1u);
}

// After an iteration: every mesh that ran gets its worst column's relative
// residual and one more iteration, and is done once that is <= tol (a
// non-finite residual ends the whole loop).  The loop continues while a mesh
// is not done and the iteration limit is not reached.  One block.
__global__ void k_many_check(int K, int nrhs, int* state, const double* __restrict__ nb, double* rel,
                             const double* tol, double* const* rr, cudaGraphConditionalHandle hw) {
  __shared__ int open, bad;
  if (threadIdx.x == 0) {
    open = 0;
    bad = 0;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    int* st = state + 3 + 2 * k;
    if (st[0]) continue;
    double w = 0.0;
    bool fin = true;
    for (int q = 0; q < nrhs; ++q) {
      const double b = nb[k * kMaxRhs + q];
      const double r = b > 0.0 ? sqrt(rr[k][q]) / b : 0.0;
      if (!isfinite(r)) fin = false;
      w = fmax(w, r);
    }
    st[1] += 1;
    rel[k] = fin ? w : (double)NAN;
    if (!fin) atomicOr(&bad, 1);
    if (fin && w <= *tol) st[0] = 1;
    else atomicOr(&open, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int it = ++state[0];
    if (bad) state[2] = 1;
    cudaGraphSetConditional(hw, (open && !bad && it < state[1]) ? 1u : 0u);
  }
}

// The host-driven form: one graph per iteration with every mesh's branch.
template <int NR>
static gmg_status many_graph(gmg_many_ctx* m, cudaGraphExec_t* out, uint64_t* kernels) {
  const int K = (int)m->h.size();
  const uint64_t before = g_launches;
  GMG_CK(cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeThreadLocal));
  gmg_status st = GMG_OK;
  cudaError_t e = cudaEventRecord(m->ev[K], m->cap);
  for (int k = 0; k < K && st == GMG_OK && e == cudaSuccess; ++k) {
    e = cudaStreamWaitEvent(m->br[k], m->ev[K], 0);
    if (e == cudaSuccess) st = iteration_m<NR>(m->h[k], m->br[k]);
    if (st == GMG_OK && e == cudaSuccess) e = cudaEventRecord(m->ev[k], m->br[k]);
    if (st == GMG_OK && e == cudaSuccess) e = cudaStreamWaitEvent(m->cap, m->ev[k], 0);
  }
  cudaGraph_t g = nullptr;
  cudaError_t ee = cudaStreamEndCapture(m->cap, &g);
  *kernels = g_launches - before;
  g_launches = before;
  if (st != GMG_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  GMG_CK(e);
  GMG_CK(ee);
  cudaError_t ei = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  GMG_CK(ei);
  return GMG_OK;
}

// The device-side loop: WHILE { gate -> IF_k { iteration of mesh k } for all k -> check }.
template <int NR>
static gmg_status many_loop(gmg_many_ctx* m, int slot, int nrhs) {
  const int K = (int)m->h.size();
  cudaGraph_t g = nullptr;
  GMG_CK(cudaGraphCreate(&g, 0));
  cudaError_t e = cudaSuccess;
  gmg_status st = GMG_OK;
  const uint64_t before = g_launches;
  cudaGraphConditionalHandle hw = 0;
  cudaGraphNodeParams wp = {};
  cudaGraphNode_t wnode;
  e = cudaGraphConditionalHandleCreate(&hw, g, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = hw;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    e = cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &wp);
  }
  cudaGraph_t body = e == cudaSuccess ? wp.conditional.phGraph_out[0] : nullptr;
  std::vector<cudaGraphConditionalHandle>& hif = m->h_if[slot];
  hif.assign(K, 0);
  std::vector<cudaGraphNode_t> ifn(K);
  cudaGraphNode_t gate = nullptr, check = nullptr;
  // gate kernel node (handles are filled into d_if before every launch of this loop)
  if (e == cudaSuccess) {
    cudaKernelNodeParams kp = {};
    void* args[] = {(void*)&K, (void*)&m->d_state, (void*)&m->d_if};
    kp.func = (void*)k_many_gate;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(256);
    kp.kernelParams = args;
    e = cudaGraphAddKernelNode(&gate, body, nullptr, 0, &kp);
  }
  for (int k = 0; k < K && e == cudaSuccess && st == GMG_OK; ++k) {
    e = cudaGraphConditionalHandleCreate(&hif[k], body, 0, 0);
    if (e != cudaSuccess) break;
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = hif[k];
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    e = cudaGraphAddNode(&ifn[k], body, &gate, nullptr, 1, &ip);
    if (e != cudaSuccess) break;
    e = cudaStreamBeginCaptureToGraph(m->br[k], ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) break;
    st = iteration_m<NR>(m->h[k], m->br[k]);
    cudaGraph_t cg = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(m->br[k], &cg);
    if (e == cudaSuccess) e = ec;
  }
  if (e == cudaSuccess && st == GMG_OK) {
    cudaKernelNodeParams kp = {};
    void* args[] = {(void*)&K, (void*)&nrhs, (void*)&m->d_state, (void*)&m->d_nb, (void*)&m->d_rel,
                    (void*)&m->d_tol, (void*)&m->d_rr, (void*)&hw};
    kp.func = (void*)k_many_check;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(256);
    kp.kernelParams = args;
    e = cudaGraphAddKernelNode(&check, body, ifn.data(), (size_t)K, &kp);
  }
  m->loop_kernels[slot] = g_launches - before + 2;
  g_launches = before;
  if (st == GMG_OK && e == cudaSuccess) e = cudaGraphInstantiate(&m->loop[slot], g, 0);
  cudaGraphDestroy(g);
  if (st != GMG_OK) return st;
  if (e != cudaSuccess) {
    cudaGetLastError();
    m->loop[slot] = nullptr;
    m->loop_refused[slot] = true;
    if (const char* v = std::getenv("GMG_VERBOSE"))
      if (v[0] == '1') std::fprintf(stderr, "gmg: many-mesh device loop refused (%s), host loop\n", cudaGetErrorString(e));
  }
  return GMG_OK;
}

template <int NR>
static gmg_status many_solve(gmg_many_ctx* m, int nrhs, const double* const* B, double* const* X, double tol,
                             int mem, gmg_solve_info* info, cudaStream_t s) {
  const int K = (int)m->h.size();
  std::vector<double> nb((size_t)K * kMaxRhs, 0.0);
  std::vector<double> rel(K, 0.0);
  std::vector<int> iters(K, 0), done(K, 0);
  // right-hand sides and initial guesses into every hierarchy's permuted layout
  for (int k = 0; k < K; ++k) {
    gmg_ctx* c = m->h[k];
    Level& L0 = c->L[0];
    const int64_t n = L0.n;
    const size_t bytes = sizeof(double) * (size_t)(n * nrhs);
    const double* bsrc = B[k];
    if (mem == GMG_MEM_HOST) {
      GMG_CK(cudaMemcpyAsync(c->RS, B[k], bytes, cudaMemcpyHostToDevice, s));
      bsrc = c->RS;
    }
    k_gather_m<<<gblk(n * NR), 256, 0, s>>>(n, nrhs, NR, L0.perm, bsrc, c->BS);
    LCK();
    const double* xsrc = X[k];
    if (mem == GMG_MEM_HOST) {
      GMG_CK(cudaMemcpyAsync(c->RS, X[k], bytes, cudaMemcpyHostToDevice, s));
      xsrc = c->RS;
    }
    k_gather_m<<<gblk(n * NR), 256, 0, s>>>(n, nrhs, NR, L0.perm, xsrc, c->XS);
    LCK();
    // ||B_c||: the outer residual of a zero iterate
    double* keep = c->XS;
    c->XS = c->RS;
    GMG_CK(cudaMemsetAsync(c->RS, 0, sizeof(double) * (size_t)(n * NR), s));
    gmg_status st = outer_m<NR>(c, s);
    c->XS = keep;
    GMG_TRY(st);
    GMG_CK(cudaMemcpyAsync(c->h_scal + 8, c->scal + 8, NR * sizeof(double), cudaMemcpyDeviceToHost, s));
    GMG_CK(cudaStreamSynchronize(s));
    int zmask = 0;
    for (int q = 0; q < nrhs; ++q) {
      nb[(size_t)k * kMaxRhs + q] = std::sqrt(c->h_scal[8 + q]);
      if (nb[(size_t)k * kMaxRhs + q] == 0.0) zmask |= 1 << q;
    }
    if (zmask) {
      k_zero_cols<<<gblk(n * NR), 256, 0, s>>>(n, NR, zmask, c->XS);
      LCK();
    }
    GMG_TRY(outer_m<NR>(c, s));
  }
  // host-side residuals of every mesh not yet done (a done mesh keeps the
  // residual it converged with)
  auto fetch = [&]() -> gmg_status {
    for (int k = 0; k < K; ++k) {
      gmg_ctx* c = m->h[k];
      GMG_CK(cudaMemcpyAsync(c->h_scal + 8, c->scal + 8, NR * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    GMG_CK(cudaStreamSynchronize(s));
    for (int k = 0; k < K; ++k) {
      if (done[k]) continue;
      double w = 0.0;
      for (int q = 0; q < nrhs; ++q) {
        const double b = nb[(size_t)k * kMaxRhs + q];
        const double r = b > 0 ? std::sqrt(m->h[k]->h_scal[8 + q]) / b : 0.0;
        w = std::isfinite(r) ? std::max(w, r) : r;
        if (!std::isfinite(r)) break;
      }
      rel[k] = w;
    }
    return GMG_OK;
  };
  GMG_TRY(fetch());
  const int slot = nr_slot(NR);
  int max_iter = 0;
  for (auto* c : m->h) max_iter = std::max(max_iter, c->opt.max_iter);
  gmg_status st = GMG_ERR_NOT_CONVERGED;
  bool bad = false, open = false;
  for (int k = 0; k < K; ++k) {
    if (!std::isfinite(rel[k])) bad = true;
    done[k] = rel[k] <= tol;
    if (!done[k]) open = true;
  }
  if (bad) st = GMG_ERR_NONFINITE;
  else if (!open) st = GMG_OK;
  static const bool no_loop = [] {
    const char* v = std::getenv("GMG_NO_DEVICE_LOOP");
    return v && v[0] == '1';
  }();
  if (st == GMG_ERR_NOT_CONVERGED && max_iter > 0 && !no_loop && !m->loop_refused[slot] && !m->loop[slot])
    GMG_TRY(many_loop<NR>(m, slot, nrhs));
  if (st == GMG_ERR_NOT_CONVERGED && max_iter > 0 && m->loop[slot]) {
    // device-side loop: state, norms and the IF handles of this loop, one launch
    std::vector<int> hs(3 + 2 * K, 0);
    hs[1] = max_iter;
    for (int k = 0; k < K; ++k) hs[3 + 2 * k] = done[k];
    GMG_CK(cudaMemcpyAsync(m->d_state, hs.data(), sizeof(int) * hs.size(), cudaMemcpyHostToDevice, s));
    GMG_CK(cudaMemcpyAsync(m->d_nb, nb.data(), sizeof(double) * nb.size(), cudaMemcpyHostToDevice, s));
    GMG_CK(cudaMemcpyAsync(m->d_tol, &tol, sizeof(double), cudaMemcpyHostToDevice, s));
    GMG_CK(cudaMemcpyAsync(m->d_rel, rel.data(), sizeof(double) * K, cudaMemcpyHostToDevice, s));
    GMG_CK(cudaMemcpyAsync(m->d_if, m->h_if[slot].data(), sizeof(cudaGraphConditionalHandle) * K,
                           cudaMemcpyHostToDevice, s));
    GMG_CK(cudaGraphLaunch(m->loop[slot], s));
    GMG_CK(cudaMemcpyAsync(hs.data(), m->d_state, sizeof(int) * hs.size(), cudaMemcpyDeviceToHost, s));
    GMG_CK(cudaMemcpyAsync(rel.data(), m->d_rel, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
    GMG_CK(cudaStreamSynchronize(s));
    uint64_t ran = 0;
    for (int k = 0; k < K; ++k) {
      iters[k] = hs[4 + 2 * k];
      done[k] = hs[3 + 2 * k];
      ran += (uint64_t)iters[k];
    }
    // kernels run: per mesh-iteration its share of the body, plus gate and check per iteration
    g_launches += (uint64_t)hs[0] * 2 + (K > 0 ? ran * ((m->loop_kernels[slot] - 2) / (uint64_t)K) : 0);
    bool all = true;
    for (int k = 0; k < K; ++k) all = all && done[k];
    st = hs[2] ? GMG_ERR_NONFINITE : all ? GMG_OK : GMG_ERR_NOT_CONVERGED;
  } else if (st == GMG_ERR_NOT_CONVERGED) {
    // host-driven form: every mesh iterates until all have converged; a
    // mesh's count is the iteration at which it first met the tolerance
    int it = 0;
    while (st == GMG_ERR_NOT_CONVERGED && it < max_iter) {
      if (!m->graph[slot]) GMG_TRY(many_graph<NR>(m, &m->graph[slot], &m->graph_kernels[slot]));
      GMG_CK(cudaGraphLaunch(m->graph[slot], s));
      g_launches += m->graph_kernels[slot];
      ++it;
      GMG_TRY(fetch());
      bool all = true;
      for (int k = 0; k < K; ++k) {
        if (!std::isfinite(rel[k])) bad = true;
        if (!done[k]) {
          iters[k] = it;
          done[k] = rel[k] <= tol;
        }
        all = all && done[k];
      }
      if (bad) st = GMG_ERR_NONFINITE;
      else if (all) st = GMG_OK;
    }
  }
  for (int k = 0; k < K; ++k) {
    gmg_ctx* c = m->h[k];
    const int64_t n = c->L[0].n;
    double* dst = mem == GMG_MEM_HOST ? c->RS : X[k];
    k_scatter_m<<<gblk(n * nrhs), 256, 0, s>>>(n, nrhs, NR, c->L[0].perm, c->XS, dst);
    LCK();
    if (mem == GMG_MEM_HOST)
      GMG_CK(cudaMemcpyAsync(X[k], c->RS, sizeof(double) * (size_t)(n * nrhs), cudaMemcpyDeviceToHost, s));
    if (info) {
      info[k].iters = iters[k];
      info[k].rel_res = rel[k];
    }
  }
  GMG_CK(cudaStreamSynchronize(s));
  if (st == GMG_ERR_NOT_CONVERGED) set_error("gmg_solve_many: max_iter reached");
  if (st == GMG_ERR_NONFINITE) set_error("gmg_solve_many: non-finite residual");
  return st;
}

}  // namespace gmg

extern "C" gmg_status gmg_destroy_many(gmg_many m) {
  if (!m) return GMG_OK;
  for (auto& g : m->graph)
    if (g) cudaGraphExecDestroy(g);
  for (auto& g : m->loop)
    if (g) cudaGraphExecDestroy(g);
  for (void* p : {(void*)m->d_state, (void*)m->d_nb, (void*)m->d_rel, (void*)m->d_tol, (void*)m->d_rr,
                  (void*)m->d_if})
    if (p) cudaFree(p);
  for (auto e : m->ev)
    if (e) cudaEventDestroy(e);
  for (auto s : m->br)
    if (s) cudaStreamDestroy(s);
  if (m->cap) cudaStreamDestroy(m->cap);
  for (auto h : m->h) gmg_destroy(h);
  delete m;
  return GMG_OK;
}

extern "C" gmg_status gmg_setup_many(gmg_many* out, int nmesh, const gmg_csr* A, const int* n_prolong,
                                     const gmg_prolong* const* P, const gmg_options* opt, void* stream) {
  if (!out || nmesh < 1 || !A || !n_prolong || !P) {
    set_error("gmg_setup_many: null argument or nmesh < 1");
    return GMG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  gmg_many_ctx* m = new gmg_many_ctx();
  for (int k = 0; k < nmesh; ++k) {
    gmg_handle h = nullptr;
    gmg_status st = gmg_setup(&h, &A[k], n_prolong[k], P[k], nullptr, opt, stream);
    if (st == GMG_OK) st = ensure_batched(h);
    if (st != GMG_OK) {
      std::string keep = gmg_last_error();
      if (h) gmg_destroy(h);
      gmg_destroy_many(m);
      set_error("mesh " + std::to_string(k) + ": " + keep);
      return st;
    }
    m->h.push_back(h);
  }
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess) set_error(std::string("gmg_setup_many: ") + cudaGetErrorString(e));
    return e == cudaSuccess;
  };
  bool ok = ck(cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking));
  m->br.assign(nmesh, nullptr);
  m->ev.assign(nmesh + 1, nullptr);
  for (int k = 0; ok && k < nmesh; ++k) ok = ck(cudaStreamCreateWithFlags(&m->br[k], cudaStreamNonBlocking));
  for (int k = 0; ok && k <= nmesh; ++k) ok = ck(cudaEventCreateWithFlags(&m->ev[k], cudaEventDisableTiming));
  // device state of the device-side loop
  if (ok) ok = ck(cudaMalloc(&m->d_state, sizeof(int) * (size_t)(3 + 2 * nmesh)));
  if (ok) ok = ck(cudaMalloc(&m->d_nb, sizeof(double) * (size_t)nmesh * kMaxRhs));
  if (ok) ok = ck(cudaMalloc(&m->d_rel, sizeof(double) * (size_t)nmesh));
  if (ok) ok = ck(cudaMalloc(&m->d_tol, sizeof(double)));
  if (ok) ok = ck(cudaMalloc(&m->d_rr, sizeof(double*) * (size_t)nmesh));
  if (ok) ok = ck(cudaMalloc(&m->d_if, sizeof(cudaGraphConditionalHandle) * (size_t)nmesh));
  if (ok) {
    std::vector<double*> rr(nmesh);
    for (int k = 0; k < nmesh; ++k) rr[k] = m->h[k]->scal + 8;
    ok = ck(cudaMemcpy(m->d_rr, rr.data(), sizeof(double*) * (size_t)nmesh, cudaMemcpyHostToDevice));
  }
  if (!ok) {
    gmg_destroy_many(m);
    return GMG_ERR_CUDA;
  }
  *out = m;
  return GMG_OK;
}

extern "C" gmg_status gmg_solve_many(gmg_many m, int nrhs, const double* const* B, double* const* X, double tol,
                                     int mem, gmg_solve_info* info, void* stream) {
  gmg::NvtxRange nv("gmg_solve_many");
  if (!m || !B || !X || nrhs < 1 || nrhs > kMaxRhs || !(tol >= 0.0) ||
      (mem != GMG_MEM_HOST && mem != GMG_MEM_DEVICE)) {
    set_error("gmg_solve_many: bad handle, vector list, nrhs (1..16), tolerance or memory kind");
    return GMG_ERR_INVALID_ARG;
  }
  for (size_t k = 0; k < m->h.size(); ++k)
    if (!B[k] || !X[k]) {
      set_error("gmg_solve_many: null vector for mesh " + std::to_string(k));
      return GMG_ERR_INVALID_ARG;
    }
  GMG_CK(cudaSetDevice(m->h[0]->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (nrhs == 1) return many_solve<1>(m, nrhs, B, X, tol, mem, info, s);
  if (nrhs == 2) return many_solve<2>(m, nrhs, B, X, tol, mem, info, s);
  if (nrhs <= 4) return many_solve<4>(m, nrhs, B, X, tol, mem, info, s);
  if (nrhs <= 8) return many_solve<8>(m, nrhs, B, X, tol, mem, info, s);
  return many_solve<16>(m, nrhs, B, X, tol, mem, info, s);
}

extern "C" gmg_status gmg_autotune_many(gmg_many m, int nrhs, void* stream) {
  if (!m || nrhs < 1 || nrhs > kMaxRhs) {
    set_error("gmg_autotune_many: bad batch or nrhs (1..16)");
    return GMG_ERR_INVALID_ARG;
  }
  for (size_t k = 0; k < m->h.size(); ++k) {
    gmg_status st = autotune_batched(m->h[k], nrhs, nullptr, (cudaStream_t)stream);
    if (st != GMG_OK) {
      std::string keep = gmg_last_error();
      set_error("mesh " + std::to_string(k) + ": " + keep);
      return st;
    }
  }
  // the captured iterations hold the old launch shapes
  const int slot = nr_index(block_width(nrhs));
  if (m->loop[slot]) cudaGraphExecDestroy(m->loop[slot]);
  if (m->graph[slot]) cudaGraphExecDestroy(m->graph[slot]);
  m->loop[slot] = nullptr;
  m->graph[slot] = nullptr;
  m->loop_refused[slot] = false;
  return GMG_OK;
}
