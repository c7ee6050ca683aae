// V-cycle of Alg. 2 on the GPU and the outer iterations of Alg. 1.
//
// Layout: every level is renumbered colour by colour; the off-diagonal part
// of A_l is a sliced ELL with 32-row slices stored [k][lane], so the 32 lanes
// of a warp read 32 consecutive values and column indices per k.  A
// Gauss-Seidel colour is one launch over that colour's slices: rows of a
// colour are never adjacent, so every row reads only other colours' entries of
// x and the in-place update equals sequential Gauss-Seidel in colour order.
// Levels with long rows split each row over G warps (G = 1, 2, 4 or 8; warp
// `part` takes k = part, part + G, ...), combining the G partial sums in a
// fixed order, so the dependent-load chain per row is G times shorter.
// The restriction P_l^T is a sliced ELL over the coarse rows (a gather: no
// atomics, a fixed summation order); it also clears the coarse iterate (the
// recursive call of Alg. 2 starts from zero).  The prolongation reads three
// packed (index, weight) slots per fine row.  The coarsest level applies the
// explicit inverse of its FP64 Cholesky factor as a warp-per-row GEMV.
//
// Launches use programmatic dependent launch: a kernel may start while its
// predecessor drains; it loads only setup-time data (matrix values, column
// indices, inverse diagonal) before `griddepcontrol.wait`, and everything the
// previous kernel may write after it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <string>
#include <utility>

#include "gmg_cycle.cuh"

namespace gmg {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ------------------------------------------------------------------ kernels

constexpr int kPrefetch = 8;  // matrix entries per lane loaded before the dependency wait

// Per-lane view of a sliced-ELL row split over G warps.
struct RowPart {
  bool active;
  int nk;        // entries of this row handled by this warp
  int64_t e;     // first entry
  int64_t row;
};

template <int G>
__device__ __forceinline__ RowPart row_part(int64_t s, int64_t s_end, const int64_t* __restrict__ ptr,
                                            const int32_t* __restrict__ row0, const int32_t* __restrict__ nrow,
                                            int part, int lane) {
  RowPart p{false, 0, 0, 0};
  if (s < s_end) {
    p.active = lane < nrow[s];
    const int64_t e0 = ptr[s];
    const int w = (int)((ptr[s + 1] - e0) >> 5);
    p.nk = (p.active && part < w) ? (w - part + G - 1) / G : 0;
    p.e = e0 + (int64_t)part * 32 + lane;
    p.row = row0[s] + lane;
  }
  return p;
}

// sum_k a_rk x_{c_rk} over this warp's share of row r; the first kPrefetch
// values and columns were loaded before the wait.
template <class T, int G>
__device__ __forceinline__ T row_dot(const RowPart& p, const T (&pv)[kPrefetch], const int (&pc)[kPrefetch],
                                     const int32_t* __restrict__ col, const T* __restrict__ val, const T* x) {
  T acc = 0;
#pragma unroll
  for (int q = 0; q < kPrefetch; ++q)
    if (q < p.nk) acc += pv[q] * x[pc[q]];
  for (int q = kPrefetch; q < p.nk; ++q) {
    const int64_t e = p.e + (int64_t)q * G * 32;
    acc += val[e] * x[col[e]];
  }
  return acc;
}

template <class T, int G>
__device__ __forceinline__ void prefetch_row(const RowPart& p, const int32_t* __restrict__ col,
                                             const T* __restrict__ val, T (&pv)[kPrefetch], int (&pc)[kPrefetch]) {
#pragma unroll
  for (int q = 0; q < kPrefetch; ++q) {
    if (q < p.nk) {
      const int64_t e = p.e + (int64_t)q * G * 32;
      pv[q] = val[e];
      pc[q] = col[e];
    } else {
      pv[q] = 0;
      pc[q] = 0;
    }
  }
}

// Combines the G partial sums of a row in warp order (part 0 first).
template <class T, int G>
__device__ __forceinline__ T combine_parts(T acc, int warp, int lane) {
  if constexpr (G > 1) {
    __shared__ T red[8][32];
    red[warp][lane] = acc;
    __syncthreads();
    if (warp % G == 0) {
#pragma unroll
      for (int g = 1; g < G; ++g) acc += red[warp + g][lane];
    }
  }
  return acc;
}

// One colour of a Gauss-Seidel sweep: x_r = (b_r - sum_{k != r} a_rk x_k) / a_rr
// for the rows of slices [s0, s1).
template <class T, int G>
__global__ void __launch_bounds__(256) k_gs(int64_t s0, int64_t s1, const int64_t* __restrict__ ptr,
                                            const int32_t* __restrict__ row0, const int32_t* __restrict__ nrow,
                                            const int32_t* __restrict__ col, const T* __restrict__ val,
                                            const T* __restrict__ dinv, const T* b, T* x) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, part = warp % G;
  const int64_t s = s0 + (int64_t)blockIdx.x * (8 / G) + warp / G;
  const RowPart p = row_part<G>(s, s1, ptr, row0, nrow, part, lane);
  T pv[kPrefetch];
  int pc[kPrefetch];
  prefetch_row<T, G>(p, col, val, pv, pc);
  const T di = (part == 0 && p.active) ? dinv[p.row] : T(0);
  pdl_wait();
  pdl_trigger();
  T acc = row_dot<T, G>(p, pv, pc, col, val, x);
  acc = combine_parts<T, G>(acc, warp, lane);
  if (part == 0 && p.active) x[p.row] = (b[p.row] - acc) * di;
}

// r = b - A x over all slices; with `partial`, per-block sums of r^2.
template <class T, int G>
__global__ void __launch_bounds__(256) k_residual(int64_t nslice, const int64_t* __restrict__ ptr,
                                                  const int32_t* __restrict__ row0, const int32_t* __restrict__ nrow,
                                                  const int32_t* __restrict__ col, const T* __restrict__ val,
                                                  const T* __restrict__ diag, const T* x, const T* b, T* r,
                                                  double* __restrict__ partial) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, part = warp % G;
  const int64_t s = (int64_t)blockIdx.x * (8 / G) + warp / G;
  const RowPart p = row_part<G>(s, nslice, ptr, row0, nrow, part, lane);
  T pv[kPrefetch];
  int pc[kPrefetch];
  prefetch_row<T, G>(p, col, val, pv, pc);
  const T d = (part == 0 && p.active) ? diag[p.row] : T(0);
  pdl_wait();
  pdl_trigger();
  T acc = row_dot<T, G>(p, pv, pc, col, val, x);
  acc = combine_parts<T, G>(acc, warp, lane);
  double sq = 0.0;
  if (part == 0 && p.active) {
    const T rv = b[p.row] - (acc + d * x[p.row]);
    r[p.row] = rv;
    sq = (double)rv * (double)rv;
  }
  if (partial) {  // fixed-shape block reduction of r^2
    __shared__ double red[256];
    red[threadIdx.x] = sq;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
  }
}

// q = A p (FP64) with per-block partials of p.q (fixed-shape reduction).
__global__ void __launch_bounds__(256) k_spmv_dot(int64_t nslice, const int64_t* __restrict__ ptr,
                                                  const int32_t* __restrict__ row0, const int32_t* __restrict__ nrow,
                                                  const int32_t* __restrict__ col, const double* __restrict__ val,
                                                  const double* __restrict__ diag, const double* p,
                                                  double* q, double* __restrict__ partial) {
  const int lane = threadIdx.x & 31;
  const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const RowPart rp = row_part<1>(s, nslice, ptr, row0, nrow, 0, lane);
  double pv[kPrefetch];
  int pc[kPrefetch];
  prefetch_row<double, 1>(rp, col, val, pv, pc);
  pdl_wait();
  pdl_trigger();
  double pq = 0.0;
  if (rp.active) {
    const double acc = row_dot<double, 1>(rp, pv, pc, col, val, p) + diag[rp.row] * p[rp.row];
    q[rp.row] = acc;
    pq = p[rp.row] * acc;
  }
  __shared__ double red[256];
  red[threadIdx.x] = pq;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// bc = P^T r (gather over the transpose) and xc = 0 (the coarse iterate of the
// recursive call starts from zero).
template <class T>
__global__ void __launch_bounds__(256) k_restrict(int64_t nslice, const int64_t* __restrict__ ptr,
                                                  const int32_t* __restrict__ row0, const int32_t* __restrict__ nrow,
                                                  const int32_t* __restrict__ col, const T* __restrict__ w,
                                                  const T* r, T* bc, T* xc) {
  const int lane = threadIdx.x & 31;
  const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const RowPart p = row_part<1>(s, nslice, ptr, row0, nrow, 0, lane);
  T pv[kPrefetch];
  int pc[kPrefetch];
  prefetch_row<T, 1>(p, col, w, pv, pc);
  pdl_wait();
  pdl_trigger();
  if (!p.active) return;
  const T acc = row_dot<T, 1>(p, pv, pc, col, w, r);
  bc[p.row] = acc;
  xc[p.row] = T(0);
}

// x += P u (three packed slots per fine row).
template <class T>
__global__ void __launch_bounds__(256) k_prolong(int64_t n, const int32_t* __restrict__ idx, const T* __restrict__ w,
                                                 const T* u, T* x) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int i0 = 0, i1 = 0, i2 = 0;
  T w0 = 0, w1 = 0, w2 = 0;
  if (i < n) {
    i0 = idx[3 * i];
    i1 = idx[3 * i + 1];
    i2 = idx[3 * i + 2];
    w0 = w[3 * i];
    w1 = w[3 * i + 1];
    w2 = w[3 * i + 2];
  }
  pdl_wait();
  pdl_trigger();
  if (i < n) x[i] += w0 * u[i0] + w1 * u[i1] + w2 * u[i2];
}

// x = Ainv b, one warp per row, FP64 accumulation in both precisions.
template <class T>
__global__ void __launch_bounds__(256) k_coarse(int n, const double* __restrict__ Ainv, const T* b, T* x) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  pdl_wait();
  pdl_trigger();
  if (row >= n) return;
  const double* a = Ainv + (int64_t)row * n;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s += a[j] * (double)b[j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) x[row] = (T)s;
}

#define GRID_LOOP(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

__global__ void k_gather(int64_t n, const int32_t* __restrict__ perm, const double* src, double* dst) {
  pdl_wait();
  pdl_trigger();
  GRID_LOOP(i, n) dst[i] = src[perm[i]];
}
__global__ void k_scatter_vec(int64_t n, const int32_t* __restrict__ perm, const double* src, double* dst) {
  pdl_wait();
  pdl_trigger();
  GRID_LOOP(i, n) dst[perm[i]] = src[i];
}
__global__ void k_d2f(int64_t n, const double* a, float* b) {
  pdl_wait();
  pdl_trigger();
  GRID_LOOP(i, n) b[i] = (float)a[i];
}
// b32 = (float) r and x32 = 0: the right-hand side and zero initial guess of
// a correction cycle MGI(0, r).
__global__ void k_d2f_zero(int64_t n, const double* r, float* b32, float* x32) {
  pdl_wait();
  pdl_trigger();
  GRID_LOOP(i, n) {
    b32[i] = (float)r[i];
    x32[i] = 0.f;
  }
}
__global__ void k_f2d(int64_t n, const float* a, double* b) {
  pdl_wait();
  pdl_trigger();
  GRID_LOOP(i, n) b[i] = (double)a[i];
}
// x += (double) e
__global__ void k_add_f2d(int64_t n, const float* e, double* x) {
  pdl_wait();
  pdl_trigger();
  GRID_LOOP(i, n) x[i] += (double)e[i];
}

// Deterministic dot product: fixed grid, fixed per-thread ranges, fixed tree.
__global__ void __launch_bounds__(256) k_dot_partial(int64_t n, const double* a, const double* b, double* partial) {
  __shared__ double red[256];
  pdl_wait();
  pdl_trigger();
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) s += a[i] * b[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// out = sum of `count` partials (one block of 256, fixed order).
__global__ void k_reduce_final(int count, const double* partial, double* out) {
  __shared__ double red[256];
  pdl_wait();
  pdl_trigger();
  double s = 0.0;
  for (int i = threadIdx.x; i < count; i += 256) s += partial[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// PCG scalars live on the device: sc[2] = r.z, sc[3] = p.Ap, sc[4] = Polak-
// Ribiere numerator z.(r - r_old).
__global__ void k_pcg_axpy(int64_t n, const double* sc, const double* p, const double* q, double* x, double* r,
                           double* rold) {
  pdl_wait();
  pdl_trigger();
  const double alpha = sc[2] / sc[3];
  GRID_LOOP(i, n) {
    const double ri = r[i];
    rold[i] = ri;
    x[i] += alpha * p[i];
    r[i] = ri - alpha * q[i];
  }
}
__global__ void k_pcg_dir(int64_t n, const double* sc, const double* z, double* p) {
  pdl_wait();
  pdl_trigger();
  const double beta = sc[4] / sc[2];
  GRID_LOOP(i, n) p[i] = z[i] + beta * p[i];
}
__global__ void k_copy_scalar(const double* src, double* dst) {
  pdl_wait();
  pdl_trigger();
  *dst = *src;
}
// d = r - rold (for the Polak-Ribiere numerator)
__global__ void k_sub(int64_t n, const double* a, const double* b, double* d) {
  pdl_wait();
  pdl_trigger();
  GRID_LOOP(i, n) d[i] = a[i] - b[i];
}
__global__ void k_copy(int64_t n, const double* a, double* b) {
  pdl_wait();
  pdl_trigger();
  GRID_LOOP(i, n) b[i] = a[i];
}

// ------------------------------------------------------------------ small levels
// The levels at and below `l0` (all small) run as one persistent kernel per
// V-cycle on a single thread-block cluster: every colour phase, residual,
// restriction, coarse solve and prolongation of those levels is separated
// by a hardware cluster barrier instead of a kernel boundary.  Vectors are
// read through L2 (ld.global.cg): they are written by other CTAs of the
// cluster between barriers.  Matrix data is setup-time data.

template <class T> struct DV;
template <> struct DV<float> {
  __device__ static const float* av(const DevLevel& L) { return L.a_v32; }
  __device__ static const float* dinv(const DevLevel& L) { return L.dinv32; }
  __device__ static const float* diag(const DevLevel& L) { return L.diag32; }
  __device__ static const float* rv(const DevLevel& L) { return L.r_v32; }
  __device__ static const float* pw(const DevLevel& L) { return L.p_w32; }
  __device__ static float* x(const DevLevel& L) { return L.x32; }
  __device__ static float* b(const DevLevel& L) { return L.b32; }
  __device__ static float* r(const DevLevel& L) { return L.r32; }
};
template <> struct DV<double> {
  __device__ static const double* av(const DevLevel& L) { return L.a_v64; }
  __device__ static const double* dinv(const DevLevel& L) { return L.dinv64; }
  __device__ static const double* diag(const DevLevel& L) { return L.diag64; }
  __device__ static const double* rv(const DevLevel& L) { return L.r_v64; }
  __device__ static const double* pw(const DevLevel& L) { return L.p_w64; }
  __device__ static double* x(const DevLevel& L) { return L.x64; }
  __device__ static double* b(const DevLevel& L) { return L.b64; }
  __device__ static double* r(const DevLevel& L) { return L.r64; }
};

__device__ __forceinline__ void cluster_sync() {
  __syncwarp();
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// One Gauss-Seidel colour (mode 0) or the residual over all slices (mode 1)
// of level L, split over the cluster: G warps of one CTA share a slice.
template <class T, int G>
__device__ void cl_rows(const DevLevel& L, int64_t s0, int64_t s1, int mode, int cta, T (&red)[32][33]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, part = warp % G;
  constexpr int SPC = 32 / G;                 // slices per CTA per round
  constexpr int SPR = SPC * kClusterCTAs;     // slices per round
  const int64_t rounds = (s1 - s0 + SPR - 1) / SPR;
  const T* val = DV<T>::av(L);
  T* x = DV<T>::x(L);
  const T* b = DV<T>::b(L);
  for (int64_t rd = 0; rd < rounds; ++rd) {
    const int64_t s = s0 + rd * SPR + (int64_t)cta * SPC + warp / G;
    const RowPart p = row_part<G>(s, s1, L.a_ptr, L.a_row0, L.a_nrow, part, lane);
    // all matrix loads first, then all gathers: two dependent round trips per row
    T pv[kPrefetch];
    int pc[kPrefetch];
    prefetch_row<T, G>(p, L.a_col, val, pv, pc);
    T xv[kPrefetch];
#pragma unroll
    for (int q = 0; q < kPrefetch; ++q) xv[q] = q < p.nk ? __ldcg(x + pc[q]) : T(0);
    T acc = 0;
#pragma unroll
    for (int q = 0; q < kPrefetch; ++q) acc += pv[q] * xv[q];
    for (int q = kPrefetch; q < p.nk; ++q) {
      const int64_t e = p.e + (int64_t)q * G * 32;
      acc += val[e] * __ldcg(x + L.a_col[e]);
    }
    if constexpr (G > 1) {
      red[warp][lane] = acc;
      __syncthreads();
      if (part == 0) {
#pragma unroll
        for (int g = 1; g < G; ++g) acc += red[warp + g][lane];
      }
    }
    if (part == 0 && p.active) {
      if (mode == 0) {
        x[p.row] = (__ldcg(b + p.row) - acc) * DV<T>::dinv(L)[p.row];
      } else {
        DV<T>::r(L)[p.row] = __ldcg(b + p.row) - (acc + DV<T>::diag(L)[p.row] * __ldcg(x + p.row));
      }
    }
    if constexpr (G > 1) __syncthreads();
  }
}

template <class T>
__device__ void cl_rows_any(const DevLevel& L, int64_t s0, int64_t s1, int mode, int cta, T (&red)[32][33]) {
  switch (L.lanes) {
    case 1: cl_rows<T, 1>(L, s0, s1, mode, cta, red); break;
    case 2: cl_rows<T, 2>(L, s0, s1, mode, cta, red); break;
    case 4: cl_rows<T, 4>(L, s0, s1, mode, cta, red); break;
    default: cl_rows<T, 8>(L, s0, s1, mode, cta, red); break;
  }
}

// half 0: pre-smoothing, residual and restriction of levels l0 .. lambda-1
// (down to the coarsest right-hand side); half 1: prolongation and
// post-smoothing from lambda-1 back up to l0.  The coarsest solve between
// the halves runs on the whole GPU (its FP64 GEMV needs every SM's FP64 pipe).
template <class T>
__global__ void __launch_bounds__(1024) k_cluster_cycle(const DevLevel* __restrict__ lv, int l0, int nlev, int half,
                                                        int nu_pre, int nu_post, int post_forward) {
  __shared__ T red[32][33];
  const int cta = (int)cluster_rank();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gwarp = cta * 32 + warp;                         // warp index in the cluster
  const int64_t gthread = (int64_t)cta * 1024 + threadIdx.x;  // thread index in the cluster
  constexpr int kWarps = 32 * kClusterCTAs;
  constexpr int kThreads = 1024 * kClusterCTAs;
  pdl_wait();
  pdl_trigger();
  if (half == 0) {
    for (int l = l0; l < nlev - 1; ++l) {
      const DevLevel& L = lv[l];
      for (int it = 0; it < nu_pre; ++it)
        for (int k = 0; k < L.ncolor; ++k) {
          cl_rows_any<T>(L, L.cso[k], L.cso[k + 1], 0, cta, red);
          cluster_sync();
        }
      cl_rows_any<T>(L, 0, L.nslice, 1, cta, red);
      cluster_sync();
      // restriction into level l+1 (clears its iterate)
      const DevLevel& C = lv[l + 1];
      const T* r = DV<T>::r(L);
      const T* rw = DV<T>::rv(L);
      for (int64_t s = gwarp; s < L.r_nslice; s += kWarps) {
        if (lane >= L.r_nrow[s]) continue;
        const int64_t e0 = L.r_ptr[s] + lane;
        const int wd = (int)((L.r_ptr[s + 1] - L.r_ptr[s]) >> 5);
        T acc = 0;
#pragma unroll 8
        for (int k = 0; k < wd; ++k) {
          const int64_t e = e0 + (int64_t)k * 32;
          acc += rw[e] * __ldcg(r + L.r_col[e]);
        }
        const int64_t row = L.r_row0[s] + lane;
        DV<T>::b(C)[row] = acc;
        DV<T>::x(C)[row] = T(0);
      }
      if (l + 1 < nlev - 1) cluster_sync();
    }
    return;
  }
  for (int l = nlev - 2; l >= l0; --l) {
    const DevLevel& L = lv[l];
    const DevLevel& C = lv[l + 1];
    T* x = DV<T>::x(L);
    const T* u = DV<T>::x(C);
    const T* w = DV<T>::pw(L);
    for (int64_t i = gthread; i < L.n; i += kThreads) {
      const int64_t q = 3 * i;
      x[i] = __ldcg(x + i) + (w[q] * __ldcg(u + L.p_idx[q]) + w[q + 1] * __ldcg(u + L.p_idx[q + 1]) +
                              w[q + 2] * __ldcg(u + L.p_idx[q + 2]));
    }
    cluster_sync();
    for (int it = 0; it < nu_post; ++it)
      for (int q = 0; q < L.ncolor; ++q) {
        const int k = post_forward ? q : L.ncolor - 1 - q;
        cl_rows_any<T>(L, L.cso[k], L.cso[k + 1], 0, cta, red);
        if (!(l == l0 && it == nu_post - 1 && q == L.ncolor - 1)) cluster_sync();
      }
  }
}

// ------------------------------------------------------------------ launchers

// Timing events: inside a stream capture they become external event nodes
// of the graph; outside, plain records.
static cudaError_t record_timing_event(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t err = cudaStreamIsCapturing(s, &cs);
  if (err != cudaSuccess) return err;
  return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                                             : cudaEventRecord(e, s);
}

static bool use_pdl() {
  static const bool on = [] {
    const char* e = std::getenv("GMG_NO_PDL");
    return !(e && e[0] == '1');
  }();
  return on;
}

// Launches `k` on `s` with programmatic stream serialisation.
template <typename... P, typename... A>
static gmg_status launch(void (*k)(P...), int64_t grid, int block, cudaStream_t s, A&&... args) {
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

static inline int64_t blocks_for(int64_t threads, int per = 256, int64_t cap = 152 * 64) {
  const int64_t g = (threads + per - 1) / per;
  return std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

template <class T>
gmg_status launch_gs_colour(Level& L, int colour, const T* b, T* x, cudaStream_t s) {
  const int64_t s0 = L.color_slice_off[colour], s1 = L.color_slice_off[colour + 1];
  if (s1 <= s0) return GMG_OK;
  const int G = L.lanes;
  const int64_t grid = (s1 - s0 + (8 / G) - 1) / (8 / G);
  const Ell& A = L.A;
  switch (G) {
    case 1: return launch(k_gs<T, 1>, grid, 256, s, s0, s1, A.ptr, A.row0, A.nrow, A.col, Vec<T>::v(A), Vec<T>::dinv(L), b, x);
    case 2: return launch(k_gs<T, 2>, grid, 256, s, s0, s1, A.ptr, A.row0, A.nrow, A.col, Vec<T>::v(A), Vec<T>::dinv(L), b, x);
    case 4: return launch(k_gs<T, 4>, grid, 256, s, s0, s1, A.ptr, A.row0, A.nrow, A.col, Vec<T>::v(A), Vec<T>::dinv(L), b, x);
    default: return launch(k_gs<T, 8>, grid, 256, s, s0, s1, A.ptr, A.row0, A.nrow, A.col, Vec<T>::v(A), Vec<T>::dinv(L), b, x);
  }
}

template <class T>
static gmg_status launch_residual_p(Level& L, const T* x, const T* b, T* r, double* partial, cudaStream_t s,
                                    int64_t* nblocks = nullptr) {
  const int G = L.lanes;
  const int64_t grid = (L.A.nslice + (8 / G) - 1) / (8 / G);
  if (nblocks) *nblocks = grid;
  const Ell& A = L.A;
  switch (G) {
    case 1: return launch(k_residual<T, 1>, grid, 256, s, A.nslice, A.ptr, A.row0, A.nrow, A.col, Vec<T>::v(A), Vec<T>::diag(L), x, b, r, partial);
    case 2: return launch(k_residual<T, 2>, grid, 256, s, A.nslice, A.ptr, A.row0, A.nrow, A.col, Vec<T>::v(A), Vec<T>::diag(L), x, b, r, partial);
    case 4: return launch(k_residual<T, 4>, grid, 256, s, A.nslice, A.ptr, A.row0, A.nrow, A.col, Vec<T>::v(A), Vec<T>::diag(L), x, b, r, partial);
    default: return launch(k_residual<T, 8>, grid, 256, s, A.nslice, A.ptr, A.row0, A.nrow, A.col, Vec<T>::v(A), Vec<T>::diag(L), x, b, r, partial);
  }
}

template <class T>
gmg_status launch_residual(Level& L, const T* x, const T* b, T* r, cudaStream_t s) {
  return launch_residual_p<T>(L, x, b, r, nullptr, s);
}

template <class T>
gmg_status launch_restrict(Level& L, const T* r, T* bc, T* xc, cudaStream_t s) {
  const Ell& R = L.R;
  return launch(k_restrict<T>, blocks_for(R.nslice * 32, 256, INT32_MAX), 256, s, R.nslice, R.ptr, R.row0, R.nrow,
                R.col, Vec<T>::v(R), r, bc, xc);
}

template <class T>
gmg_status launch_prolong(Level& L, const T* u, T* x, cudaStream_t s) {
  return launch(k_prolong<T>, blocks_for(L.n, 256, INT32_MAX), 256, s, L.n, L.p_idx, Vec<T>::pw(L), u, x);
}

template <class T>
gmg_status launch_coarse(gmg_ctx* c, const T* b, T* x, cudaStream_t s) {
  const int n = (int)c->nco;
  return launch(k_coarse<T>, (n * 32 + 255) / 256, 256, s, n, (const double*)c->Ainv, b, x);
}

// The V-cycle below and including level l0: the descending half on one
// cluster, the coarsest solve on the whole GPU, the ascending half on one
// cluster.
template <class T>
static gmg_status launch_cluster_half(gmg_ctx* c, int l0, int half, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kClusterCTAs);
  cfg.blockDim = dim3(1024);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kClusterCTAs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = use_pdl() ? 2 : 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_cluster_cycle<T>, (const DevLevel*)c->dlv, l0, c->nlev, half,
                                     c->opt.nu_pre, c->opt.nu_post, c->opt.post_forward);
  ++g_launches;
  if (e != cudaSuccess) {
    set_error(std::string("cluster launch: ") + cudaGetErrorString(e));
    return GMG_ERR_CUDA;
  }
  return GMG_OK;
}

template <class T>
static gmg_status launch_cluster(gmg_ctx* c, int l0, cudaStream_t s) {
  GMG_TRY(launch_cluster_half<T>(c, l0, 0, s));
  Level& C = c->L[c->nlev - 1];
  GMG_TRY(launch_coarse<T>(c, Vec<T>::b(C), Vec<T>::x(C), s));
  return launch_cluster_half<T>(c, l0, 1, s);
}

// MGI(x_l, b_l, l) of Alg. 2 on the level's own vectors.  x_l holds the
// initial iterate (zero for every l > 0: the restriction clears it).
template <class T>
gmg_status vcycle(gmg_ctx* c, int l, cudaStream_t s) {
  Level& L = c->L[l];
  T* x = Vec<T>::x(L);
  T* b = Vec<T>::b(L);
  if (l == c->nlev - 1) return launch_coarse<T>(c, b, x, s);
  if (c->cluster_l0 > 0 && l == c->cluster_l0) return launch_cluster<T>(c, l, s);
  Level& C = c->L[l + 1];
  const bool prof = c->prof && l == 0;
  if (prof) GMG_CK(record_timing_event(c->ev[0], s));
  for (int it = 0; it < c->opt.nu_pre; ++it)
    for (int k = 0; k < L.ncolor; ++k) GMG_TRY(launch_gs_colour<T>(L, k, b, x, s));
  if (prof) GMG_CK(record_timing_event(c->ev[1], s));
  GMG_TRY(launch_residual<T>(L, x, b, Vec<T>::r(L), s));
  GMG_TRY(launch_restrict<T>(L, Vec<T>::r(L), Vec<T>::b(C), Vec<T>::x(C), s));
  GMG_TRY(vcycle<T>(c, l + 1, s));
  GMG_TRY(launch_prolong<T>(L, Vec<T>::x(C), x, s));
  if (prof) GMG_CK(record_timing_event(c->ev[2], s));
  for (int it = 0; it < c->opt.nu_post; ++it)
    for (int q = 0; q < L.ncolor; ++q) {
      const int k = c->opt.post_forward ? q : L.ncolor - 1 - q;
      GMG_TRY(launch_gs_colour<T>(L, k, b, x, s));
    }
  if (prof) GMG_CK(record_timing_event(c->ev[3], s));
  return GMG_OK;
}

template gmg_status launch_gs_colour<double>(Level&, int, const double*, double*, cudaStream_t);
template gmg_status launch_gs_colour<float>(Level&, int, const float*, float*, cudaStream_t);
template gmg_status launch_residual<double>(Level&, const double*, const double*, double*, cudaStream_t);
template gmg_status launch_residual<float>(Level&, const float*, const float*, float*, cudaStream_t);
template gmg_status launch_restrict<double>(Level&, const double*, double*, double*, cudaStream_t);
template gmg_status launch_restrict<float>(Level&, const float*, float*, float*, cudaStream_t);
template gmg_status launch_prolong<double>(Level&, const double*, double*, cudaStream_t);
template gmg_status launch_prolong<float>(Level&, const float*, float*, cudaStream_t);
template gmg_status launch_coarse<double>(gmg_ctx*, const double*, double*, cudaStream_t);
template gmg_status launch_coarse<float>(gmg_ctx*, const float*, float*, cudaStream_t);
template gmg_status vcycle<double>(gmg_ctx*, int, cudaStream_t);
template gmg_status vcycle<float>(gmg_ctx*, int, cudaStream_t);

gmg_status launch_gather(int64_t n, const int32_t* perm, const double* src, double* dst, cudaStream_t s) {
  return launch(k_gather, blocks_for(n), 256, s, n, perm, src, dst);
}
gmg_status launch_scatter(int64_t n, const int32_t* perm, const double* src, double* dst, cudaStream_t s) {
  return launch(k_scatter_vec, blocks_for(n), 256, s, n, perm, src, dst);
}
gmg_status launch_d2f(int64_t n, const double* a, float* b, cudaStream_t s) {
  return launch(k_d2f, blocks_for(n), 256, s, n, a, b);
}
gmg_status launch_f2d(int64_t n, const float* a, double* b, cudaStream_t s) {
  return launch(k_f2d, blocks_for(n), 256, s, n, a, b);
}

// ------------------------------------------------------------------ outer iteration

// rs = bs - A xs (FP64, finest level) and scal[slot] = ||rs||^2.
static gmg_status outer_residual(gmg_ctx* c, int slot, cudaStream_t s) {
  Level& L = c->L[0];
  int64_t nb = 0;
  GMG_TRY(launch_residual_p<double>(L, c->xs, c->bs, c->rs, c->red, s, &nb));
  return launch(k_reduce_final, 1, 256, s, (int)nb, (const double*)c->red, c->scal + slot);
}

static gmg_status dot(gmg_ctx* c, int64_t n, const double* a, const double* b, int slot, cudaStream_t s) {
  GMG_TRY(launch(k_dot_partial, kRedBlocks, 256, s, n, a, b, c->red));
  return launch(k_reduce_final, 1, 256, s, kRedBlocks, (const double*)c->red, c->scal + slot);
}

// A finest-level V-cycle, bracketed by timing events when profiling is on.
template <class T>
static gmg_status timed_vcycle(gmg_ctx* c, cudaStream_t s) {
  if (c->prof) GMG_CK(record_timing_event(c->ev[4], s));
  GMG_TRY(vcycle<T>(c, 0, s));
  if (c->prof) GMG_CK(record_timing_event(c->ev[5], s));
  return GMG_OK;
}

// z = MGI32(0, r), widened to FP64.
static gmg_status precond32(gmg_ctx* c, const double* r, double* z, cudaStream_t s) {
  Level& L = c->L[0];
  GMG_TRY(launch(k_d2f_zero, blocks_for(L.n), 256, s, L.n, r, L.b32, L.x32));
  GMG_TRY(timed_vcycle<float>(c, s));
  return launch_f2d(L.n, L.x32, z, s);
}

// One outer iteration (captured as a graph when enabled).
//  FP64         : x <- MGI(x, b) (FP64 cycle on the iterate), r = b - A x, rr
//  FP32_REFINE  : e = MGI32(0, r), x += e, r = b - A x, rr
//  FP32_PCG seg 0: q = A p, pq, alpha = rz/pq, x += alpha p, r -= alpha q, rr
//  FP32_PCG seg 1: z = MGI32(0, r), num = z.(r - r_old), rz' = r.z,
//                  p = z + (num/rz) p, rz = rz'
gmg_status iteration_body(gmg_ctx* c, int mode, int seg, cudaStream_t s) {
  Level& L = c->L[0];
  const int64_t n = L.n;
  if (mode == GMG_FP64) {
    GMG_TRY(timed_vcycle<double>(c, s));  // level-0 x64/b64 alias xs/bs
    return outer_residual(c, S_RR, s);
  }
  if (mode == GMG_FP32_REFINE) {
    GMG_TRY(launch(k_d2f_zero, blocks_for(n), 256, s, n, (const double*)c->rs, L.b32, L.x32));
    GMG_TRY(timed_vcycle<float>(c, s));
    GMG_TRY(launch(k_add_f2d, blocks_for(n), 256, s, n, (const float*)L.x32, c->xs));
    return outer_residual(c, S_RR, s);
  }
  if (seg == 0) {
    const int64_t nb = (L.A.nslice * 32 + 255) / 256;
    GMG_TRY(launch(k_spmv_dot, nb, 256, s, L.A.nslice, L.A.ptr, L.A.row0, L.A.nrow, L.A.col, L.A.v64, L.diag64,
                   (const double*)c->ps, c->qs, c->red));
    GMG_TRY(launch(k_reduce_final, 1, 256, s, (int)nb, (const double*)c->red, c->scal + S_PQ));
    GMG_TRY(launch(k_pcg_axpy, blocks_for(n), 256, s, n, (const double*)c->scal, (const double*)c->ps,
                   (const double*)c->qs, c->xs, c->rs, c->ros));
    return dot(c, n, c->rs, c->rs, S_RR, s);
  }
  GMG_TRY(precond32(c, c->rs, c->zs, s));
  GMG_TRY(launch(k_sub, blocks_for(n), 256, s, n, (const double*)c->rs, (const double*)c->ros, c->qs));
  GMG_TRY(dot(c, n, c->zs, c->qs, S_NUM, s));
  GMG_TRY(dot(c, n, c->rs, c->zs, S_RZN, s));
  GMG_TRY(launch(k_pcg_dir, blocks_for(n), 256, s, n, (const double*)c->scal, (const double*)c->zs, c->ps));
  return launch(k_copy_scalar, 1, 1, s, (const double*)(c->scal + S_RZN), c->scal + S_RZ);
}

// PCG start: z = MGI32(0, r), rz = r.z, p = z (r must be current).
gmg_status pcg_start(gmg_ctx* c, cudaStream_t s) {
  const int64_t n = c->L[0].n;
  GMG_TRY(precond32(c, c->rs, c->zs, s));
  GMG_TRY(dot(c, n, c->rs, c->zs, S_RZ, s));
  return launch(k_copy, blocks_for(n), 256, s, n, (const double*)c->zs, c->ps);
}

gmg_status outer_residual_norm(gmg_ctx* c, cudaStream_t s) { return outer_residual(c, S_RR, s); }
gmg_status norm_b(gmg_ctx* c, cudaStream_t s) { return dot(c, c->L[0].n, c->bs, c->bs, S_NB2, s); }

}  // namespace gmg
