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
// explicit FP64 inverse of its operator as a warp-per-row GEMV.
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
#include <type_traits>
#include <utility>

#include "gmg_cycle.cuh"

namespace gmg {


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

// Sum of partial[0 .. count) by one block of 256 threads in a fixed order
// (strided per-thread sums, then a tree); every thread gets the result.
// Partials written by other blocks of the same grid are read through L2.
__device__ double block_final_sum(int count, const double* partial, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < count; i += 256) s += __ldcg(partial + i);
  __syncthreads();
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double v = red[0];
  __syncthreads();
  return v;
}

// True in the one block of the grid that arrives last (after every block has
// written its partial sums); that block then finishes the reduction, so no
// separate single-block kernel is launched.  `counter` returns to 0.
__device__ bool last_block(int* counter) {
  __shared__ int is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    is_last = atomicAdd(counter, 1) == (int)gridDim.x - 1;
    if (is_last) *counter = 0;
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last != 0;
}

// One colour of a Gauss-Seidel sweep: x_r = (b_r - sum_{k != r} a_rk x_k) / a_rr
// for the rows of slices [s0, s1).  The FP32 one-warp-per-slice form (the
// finest level) is held to 32 registers so that 8 CTAs fit per SM and a whole
// colour of the finest level is resident in one wave (measured: 5.9 -> 5.6 us
// per colour on the 1M-vertex torus).
template <class T, int G>
__global__ void __launch_bounds__(256, (G == 1 && sizeof(T) == 4) ? 8 : 1) k_gs(int64_t s0, int64_t s1, const int64_t* __restrict__ ptr,
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
  // b is issued with the gathers: after the barrier of combine_parts its load
  // would be one more dependent round trip to L2
  const T bv = (part == 0 && p.active) ? b[p.row] : T(0);
  T acc = row_dot<T, G>(p, pv, pc, col, val, x);
  acc = combine_parts<T, G>(acc, warp, lane);
  if (part == 0 && p.active) x[p.row] = (bv - acc) * di;
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
  const bool own = part == 0 && p.active;
  const T bv = own ? b[p.row] : T(0), xv = own ? x[p.row] : T(0);  // issued with the gathers
  T acc = row_dot<T, G>(p, pv, pc, col, val, x);
  acc = combine_parts<T, G>(acc, warp, lane);
  double sq = 0.0;
  if (own) {
    const T rv = bv - (acc + d * xv);
    r[p.row] = rv;
    sq = to_f64(rv) * to_f64(rv);
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
                                                  double* q, double* __restrict__ partial, int* counter,
                                                  double* out) {
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
  if (last_block(counter)) {
    const double v = block_final_sum(gridDim.x, partial, red);
    if (threadIdx.x == 0) *out = v;
  }
}

// bc = P^T r (gather over the transpose) and xc = 0 (the coarse iterate of the
// recursive call starts from zero).
template <class T>
__global__ void __launch_bounds__(256) k_restrict(int64_t nslice, const int64_t* __restrict__ ptr,
                                                  const int32_t* __restrict__ row0, const int32_t* __restrict__ nrow,
                                                  const int32_t* __restrict__ col, const T* __restrict__ w,
                                                  const T* r, T* bc, T* xc, const T* __restrict__ dinvc,
                                                  int64_t nc0) {
  const int lane = threadIdx.x & 31;
  const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const RowPart p = row_part<1>(s, nslice, ptr, row0, nrow, 0, lane);
  T pv[kPrefetch];
  int pc[kPrefetch];
  prefetch_row<T, 1>(p, col, w, pv, pc);
  const bool c0 = p.active && p.row < nc0;
  const T dc = c0 ? dinvc[p.row] : T(0);
  pdl_wait();
  pdl_trigger();
  if (!p.active) return;
  const T acc = row_dot<T, 1>(p, pv, pc, col, w, r);
  bc[p.row] = acc;
  // the first Gauss-Seidel colour of the coarse pre-smoothing from x = 0:
  // (b - 0) / a_ii for the rows of colour 0 (the first nc0 rows)
  xc[p.row] = c0 ? (acc - T(0)) * dc : T(0);
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
  for (int j = lane; j < n; j += 32) s += a[j] * to_f64(b[j]);
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
  GRID_LOOP(i, n) b[i] = f32_rn(a[i]);
}
// b32 = (float) r and x32 = 0: the right-hand side and zero initial guess of
// a correction cycle MGI(0, r); the rows of colour 0 (the first n0) take
// their first Gauss-Seidel update from x = 0 right away, (b - 0) / a_ii.
__global__ void k_d2f_zero(int64_t n, const double* r, float* b32, float* x32, const float* __restrict__ dinv32,
                           int64_t n0) {
  pdl_wait();
  pdl_trigger();
  GRID_LOOP(i, n) {
    const float bi = f32_rn(r[i]);
    b32[i] = bi;
    x32[i] = i < n0 ? (bi - 0.f) * dinv32[i] : 0.f;
  }
}
__global__ void k_f2d(int64_t n, const float* a, double* b) {
  pdl_wait();
  pdl_trigger();
  GRID_LOOP(i, n) b[i] = f64_of(a[i]);
}
// x += (double) e
__global__ void k_add_f2d(int64_t n, const float* e, double* x) {
  pdl_wait();
  pdl_trigger();
  GRID_LOOP(i, n) x[i] += f64_of(e[i]);
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
  const double v = block_final_sum(count, partial, red);
  if (threadIdx.x == 0) *out = v;
}

// PCG scalars live on the device (slots S_*): r.z, p.Ap, the Polak-Ribiere
// numerator z.(r - r_old), beta.
//
// Block sums in the fixed order of k_dot_partial (same grid, same per-thread
// ranges, same tree), so the fused kernels below give the same bits as a
// separate dot product.
__device__ __forceinline__ void block_sum_store(double v, double* red, double* out) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// The convergence test of the device-side loop (one thread): advances the
// iteration counter it[0], records rel = ||r|| / ||b|| (same arithmetic as the
// host test) and keeps the loop going while rel is finite, above the
// tolerance and the counter below it[1].
__device__ void iter_check(const double* sc, int* it, double* hist, cudaGraphConditionalHandle h) {
  const int k = ++it[0];
  const double rel = sqrt(sc[S_RR]) / sqrt(sc[S_NB2]);
  hist[k] = rel;
  const bool go = isfinite(rel) && !(rel <= sc[S_TOL]) && k < it[1];
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

// alpha = rz / pq; r_old = r; x += alpha p; r -= alpha q; rr = r.r into
// sc[S_RR] (partials, finished by the last block); and the initial iterate of
// the next preconditioning cycle MGI(0, r): with an FP32 cycle its right-hand
// side b32 = (float) r and x32 (as k_d2f_zero), with an FP64 cycle (which
// reads r itself as its right-hand side) z64.  The rows of colour 0 (the
// first n0) take their first Gauss-Seidel update from zero, (r - 0) / a_ii.
// With `check` the last block also runs the convergence test of the
// device-side loop.  Grid: kRedBlocks x 256.
template <class Z>
__global__ void __launch_bounds__(256) k_pcg_axpy(int64_t n, double* sc, const double* __restrict__ p,
                                                  const double* __restrict__ q, double* __restrict__ x,
                                                  double* __restrict__ r, double* __restrict__ rold,
                                                  float* __restrict__ b32, Z* __restrict__ z0,
                                                  const Z* __restrict__ dinv, int64_t n0,
                                                  double* __restrict__ partial, int* counter, int check, int* it,
                                                  double* hist, cudaGraphConditionalHandle h) {
  __shared__ double red[256];
  pdl_wait();
  pdl_trigger();
  const double alpha = sc[S_RZ] / sc[S_PQ];
  double rr = 0.0;
#pragma unroll 4
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    const double ri = r[i];
    rold[i] = ri;
    x[i] += alpha * p[i];
    const double rn = ri - alpha * q[i];
    r[i] = rn;
    if constexpr (sizeof(Z) == 4) {
      const float bi = f32_rn(rn);
      b32[i] = bi;
      z0[i] = i < n0 ? (bi - 0.f) * dinv[i] : 0.f;
    } else {
      z0[i] = i < n0 ? (rn - 0.0) * dinv[i] : 0.0;
    }
    rr += rn * rn;
  }
  block_sum_store(rr, red, partial + blockIdx.x);
  if (last_block(counter)) {
    const double v = block_final_sum(gridDim.x, partial, red);
    if (threadIdx.x == 0) {
      sc[S_RR] = v;
      if (check) iter_check(sc, it, hist, h);
    }
  }
}

// z = the preconditioned residual (the cycle's output, FP32 or FP64); the
// Polak-Ribiere numerator z.(r - r_old) and r.z, partial sums finished by the
// last block, which sets beta = num / rz_old and rz = r.z for the next
// iteration.  Grid: kRedBlocks x 256.
template <class Z>
__global__ void __launch_bounds__(256) k_pcg_zdots(int64_t n, const Z* __restrict__ z, const double* __restrict__ r,
                                                   const double* __restrict__ rold, double* __restrict__ partial,
                                                   int* counter, double* sc) {
  __shared__ double red[256];
  pdl_wait();
  pdl_trigger();
  double num = 0.0, rz = 0.0;
#pragma unroll 4
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    const double zi = to_f64(z[i]), ri = r[i];
    num += zi * (ri - rold[i]);
    rz += ri * zi;
  }
  block_sum_store(num, red, partial + blockIdx.x);
  __syncthreads();
  block_sum_store(rz, red, partial + gridDim.x + blockIdx.x);
  if (last_block(counter)) {
    const double a = block_final_sum(gridDim.x, partial, red);
    const double rzn = block_final_sum(gridDim.x, partial + gridDim.x, red);
    if (threadIdx.x == 0) {
      sc[S_NUM] = a;
      sc[S_BETA] = a / sc[S_RZ];
      sc[S_RZN] = rzn;
      sc[S_RZ] = rzn;
    }
  }
}

// p = z + beta p.
template <class Z>
__global__ void k_pcg_dir(int64_t n, const double* sc, const Z* __restrict__ z, double* __restrict__ p) {
  pdl_wait();
  pdl_trigger();
  const double beta = sc[S_BETA];
  GRID_LOOP(i, n) p[i] = to_f64(z[i]) + beta * p[i];
}
// z = 0 with the rows of colour 0 (the first n0) at their first Gauss-Seidel
// update from zero, (r - 0) / a_ii: the start of an FP64 correction cycle
// MGI(0, r) that reads r as its right-hand side.
__global__ void k_zero_c0(int64_t n, const double* r, double* z, const double* __restrict__ dinv, int64_t n0) {
  pdl_wait();
  pdl_trigger();
  GRID_LOOP(i, n) z[i] = i < n0 ? (r[i] - 0.0) * dinv[i] : 0.0;
}
__global__ void k_copy(int64_t n, const double* a, double* b) {
  pdl_wait();
  pdl_trigger();
  GRID_LOOP(i, n) b[i] = a[i];
}

// ------------------------------------------------------------------ tail of the FP32 cycle
// The smoothed levels l0 .. lambda-1 whose vectors fit in shared memory and
// the coarsest level run in one launch on one thread-block cluster of ncta
// CTAs.  Every CTA keeps full copies of x, r, b, 1/a_ii and a_ii of each tail
// level (and x, b of the coarsest level) in its shared memory, plus the
// sliced-ELL entries of the slices it owns: a slice belongs to the CTA of
// its first row's range of the caller's numbering (ncta contiguous ranges),
// so that most neighbours of a row share its CTA.  A phase (one Gauss-Seidel
// colour, the residual, the restriction, the coarsest GEMV, the
// prolongation) updates the rows the CTA owns and stores every new value
// through distributed shared memory into the copies that read it: x of a row
// into the CTAs owning its neighbours or the finer tail level's rows
// prolongated from it (a per-row mask), the residual, the restricted
// right-hand side and the coarsest solution into every CTA; a cluster
// barrier (release / acquire) ends the phase.  So a phase costs a hardware barrier
// rather than a kernel boundary, and reads global memory only for the
// restriction and prolongation weights and the coarsest inverse.  Rows of one
// colour are never adjacent, so a colour phase reads only values that no CTA
// writes during it.  All CTAs run the same sequence of barriers.

__device__ __forceinline__ void tail_sync() {
  __syncwarp();
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Stores v at the same shared-memory location in every CTA of the cluster.
__device__ __forceinline__ void tail_bcast(float* p, float v, int ncta) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  for (int r = 0; r < ncta; ++r) {
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(r));
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(ra), "f"(v) : "memory");
  }
}

// Stores v at p in this CTA and at the same location in every CTA whose bit
// is set in `mask` (the CTAs that read it).
__device__ __forceinline__ void tail_push(float* p, float v, unsigned mask) {
  *p = v;
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  while (mask) {
    const int r = __ffs(mask) - 1;
    mask &= mask - 1;
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(r));
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(ra), "f"(v) : "memory");
  }
}

template <class U>
__device__ __forceinline__ U* sm_at(char* sm, int off) {
  return reinterpret_cast<U*>(sm + off);
}

// acc = sum over the slice row's entries of a_ij x_j (shared-memory copies),
// in entry order, loads issued eight entries ahead of the adds.
__device__ __forceinline__ float tail_row_dot(const float* val, const int* col, const float* x, int off, int w) {
  float acc = 0.f;
  int q = 0;
  for (; q + 8 <= w; q += 8) {
    int c[8];
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      c[j] = col[off + (q + j) * 32];
      v[j] = val[off + (q + j) * 32];
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) acc += v[j] * x[c[j]];
  }
  for (; q < w; ++q) acc += val[off + q * 32] * x[col[off + q * 32]];
  return acc;
}

// One Gauss-Seidel colour k over the owned slices of that colour; each new
// value goes to this CTA's copy and to the copies of the CTAs that read it.
__device__ void tail_colour(const TailLevel& L, char* sm, int k) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int* own = sm_at<int>(sm, L.o_own);
  const int* ocs = sm_at<int>(sm, L.o_ocs);
  const uint16_t* mask = sm_at<uint16_t>(sm, L.o_mask);
  float* x = sm_at<float>(sm, L.o_x);
  for (int j = ocs[k] + warp; j < ocs[k + 1]; j += nw) {
    const int s = own[j];
    const float acc = tail_row_dot(sm_at<float>(sm, L.o_val), sm_at<int>(sm, L.o_col), x,
                                   sm_at<int>(sm, L.o_soff)[s] + lane, sm_at<int>(sm, L.o_width)[s]);
    if (lane < sm_at<int>(sm, L.o_nrow)[s]) {
      const int row = sm_at<int>(sm, L.o_row0)[s] + lane;
      tail_push(x + row, (sm_at<float>(sm, L.o_b)[row] - acc) * sm_at<float>(sm, L.o_dinv)[row], mask[row]);
    }
  }
}

// Over all owned slices (every colour): the residual (mode 1), the
// prolongation from the next level's x in xn (mode 2), or the copy of the
// owned rows of x back to global memory (mode 3).
__device__ void tail_owned(const TailLevel& L, char* sm, int mode, const float* xn, int ncta) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int* own = sm_at<int>(sm, L.o_own);
  float* x = sm_at<float>(sm, L.o_x);
  for (int j = warp; j < L.maxown; j += nw) {
    const int s = own[j];
    if (s < 0) continue;
    const bool active = lane < sm_at<int>(sm, L.o_nrow)[s];
    const int row = sm_at<int>(sm, L.o_row0)[s] + lane;
    if (mode == 1) {
      const float acc = tail_row_dot(sm_at<float>(sm, L.o_val), sm_at<int>(sm, L.o_col), x,
                                     sm_at<int>(sm, L.o_soff)[s] + lane, sm_at<int>(sm, L.o_width)[s]);
      if (active)
        tail_bcast(sm_at<float>(sm, L.o_r) + row,
                   sm_at<float>(sm, L.o_b)[row] - (acc + sm_at<float>(sm, L.o_diag)[row] * x[row]), ncta);
    } else if (mode == 2) {
      if (active) {
        const int q = 3 * row;
        const float v = x[row] + (L.p_w32[q] * xn[L.p_idx[q]] + L.p_w32[q + 1] * xn[L.p_idx[q + 1]] +
                                  L.p_w32[q + 2] * xn[L.p_idx[q + 2]]);
        tail_push(x + row, v, sm_at<uint16_t>(sm, L.o_mask)[row]);
      }
    } else if (active) {
      L.x32[row] = x[row];
    }
  }
}

__global__ void __launch_bounds__(1024, 1) k_tail_cycle(const __grid_constant__ TailDesc D) {
  extern __shared__ __align__(16) char sm[];
  const int cta = (int)cluster_rank(), ncta = D.ncta;
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  // load everything of the tail that is read during the phases
  for (int t = 0; t < D.ntail; ++t) {
    const TailLevel& L = D.lv[t];
    for (int i = tid; i < L.n; i += nt) {
      sm_at<float>(sm, L.o_dinv)[i] = L.dinv32[i];
      sm_at<float>(sm, L.o_diag)[i] = L.diag32[i];
    }
    for (int s = tid; s < L.nslice; s += nt) {
      sm_at<int>(sm, L.o_row0)[s] = L.a_row0[s];
      sm_at<int>(sm, L.o_nrow)[s] = L.a_nrow[s];
      sm_at<int>(sm, L.o_width)[s] = (int)((L.a_ptr[s + 1] - L.a_ptr[s]) >> 5);
      sm_at<int>(sm, L.o_soff)[s] = L.soff[s];
    }
    for (int k = tid; k <= L.ncolor; k += nt) sm_at<int>(sm, L.o_cso)[k] = L.cso[k];
    const int32_t* own = L.own + (int64_t)cta * L.maxown;
    for (int j = tid; j < L.maxown; j += nt) sm_at<int>(sm, L.o_own)[j] = own[j];
    for (int k = tid; k <= L.ncolor; k += nt) sm_at<int>(sm, L.o_ocs)[k] = L.ocs[(int64_t)cta * (L.ncolor + 1) + k];
    for (int i = tid; i < L.n; i += nt) sm_at<uint16_t>(sm, L.o_mask)[i] = L.mask[i];
    // owned slices' entries, one warp per slice
    for (int j = warp; j < L.maxown; j += nw) {
      const int s = own[j];
      if (s < 0) continue;
      const int64_t e0 = L.a_ptr[s], ne = L.a_ptr[s + 1] - e0;
      const int o = L.soff[s];
      for (int64_t e = lane; e < ne; e += 32) {
        sm_at<float>(sm, L.o_val)[o + e] = L.a_v32[e0 + e];
        sm_at<int>(sm, L.o_col)[o + e] = L.a_col[e0 + e];
      }
    }
  }
  pdl_wait();  // the vectors below are written by the previous kernel
  pdl_trigger();
  {
    const TailLevel& L = D.lv[0];
    for (int i = tid; i < L.n; i += nt) {
      sm_at<float>(sm, L.o_x)[i] = L.x32[i];
      sm_at<float>(sm, L.o_b)[i] = L.b32[i];
    }
  }
  __syncthreads();
  tail_sync();
  // down: smoothing (colour 0 of the first sweep was applied from x = 0 by the
  // restriction that produced b when c0_first), residual, restriction
  for (int t = 0; t < D.ntail; ++t) {
    const TailLevel& L = D.lv[t];
    for (int it = 0; it < D.nu_pre; ++it)
      for (int k = (it == 0 && D.c0_first) ? 1 : 0; k < L.ncolor; ++k) {
        tail_colour(L, sm, k);
        tail_sync();
      }
    tail_owned(L, sm, 1, nullptr, ncta);
    tail_sync();
    // restriction: b_next = P^T r over the owned slices of the transpose; the
    // next iterate starts from zero (each CTA clears its own copy), except
    // that a smoothed next level gets its colour-0 rows' first Gauss-Seidel
    // update (b - 0) / a_ii right away, stored by their owner into every copy
    const bool last = t + 1 == D.ntail;
    float* bn = last ? sm_at<float>(sm, D.o_bc) : sm_at<float>(sm, D.lv[t + 1].o_b);
    float* xn = last ? sm_at<float>(sm, D.o_xc) : sm_at<float>(sm, D.lv[t + 1].o_x);
    const float* dn = last ? nullptr : sm_at<float>(sm, D.lv[t + 1].o_dinv);
    const int nn = last ? D.nc : D.lv[t + 1].n;
    const int n0 = (last || !D.c0_first) ? 0 : D.lv[t + 1].nc0;
    for (int i = n0 + tid; i < nn; i += nt) xn[i] = 0.f;
    const float* r = sm_at<float>(sm, L.o_r);
    for (int s = cta + warp * ncta; s < L.r_nslice; s += nw * ncta) {
      if (lane >= L.r_nrow[s]) continue;
      const int64_t e0 = L.r_ptr[s] + lane;
      const int wd = (int)((L.r_ptr[s + 1] - L.r_ptr[s]) >> 5);
      float acc = 0.f;
      for (int q = 0; q < wd; ++q) acc += L.r_v32[e0 + (int64_t)q * 32] * r[L.r_col[e0 + (int64_t)q * 32]];
      const int row = L.r_row0[s] + lane;
      tail_bcast(bn + row, acc, ncta);
      if (row < n0) tail_bcast(xn + row, (acc - 0.f) * dn[row], ncta);
    }
    tail_sync();
  }
  // coarsest: x_c = A^-1 b_c, one warp per row
  {
    const float* bc = sm_at<float>(sm, D.o_bc);
    float* xc = sm_at<float>(sm, D.o_xc);
    for (int J = cta + warp * ncta; J < D.nc; J += nw * ncta) {
      const float* a = D.ainv32 + (int64_t)J * D.nc;
      float acc = 0.f;
      for (int K = lane; K < D.nc; K += 32) acc += a[K] * bc[K];
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) tail_bcast(xc + J, acc, ncta);
    }
    tail_sync();
  }
  // up: prolongation and post-smoothing
  for (int t = D.ntail - 1; t >= 0; --t) {
    const TailLevel& L = D.lv[t];
    const float* xn = t + 1 == D.ntail ? sm_at<float>(sm, D.o_xc) : sm_at<float>(sm, D.lv[t + 1].o_x);
    tail_owned(L, sm, 2, xn, ncta);
    tail_sync();
    for (int it = 0; it < D.nu_post; ++it)
      for (int q = 0; q < L.ncolor; ++q) {
        tail_colour(L, sm, D.post_forward ? q : L.ncolor - 1 - q);
        tail_sync();
      }
  }
  // the owned rows of the first tail level back to global memory
  tail_owned(D.lv[0], sm, 3, nullptr, ncta);
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
  const int G = L.rlanes;
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
gmg_status launch_restrict(Level& L, const T* r, T* bc, T* xc, cudaStream_t s, const T* dinvc, int64_t nc0) {
  const Ell& R = L.R;
  return launch(k_restrict<T>, blocks_for(R.nslice * 32, 256, INT32_MAX), 256, s, R.nslice, R.ptr, R.row0, R.nrow,
                R.col, Vec<T>::v(R), r, bc, xc, dinvc, nc0);
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

// The tail of an FP32 cycle (levels tail_l0 .. lambda) as one cluster launch.
static gmg_status launch_tail(gmg_ctx* c, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(c->tail.ncta);
  cfg.blockDim = dim3(c->tail_threads);
  cfg.dynamicSmemBytes = (size_t)c->tail_smem;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = c->tail.ncta;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = use_pdl() ? 2 : 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_tail_cycle, c->tail);
  ++g_launches;
  if (e != cudaSuccess) {
    set_error(std::string("tail cluster launch: ") + cudaGetErrorString(e));
    return GMG_ERR_CUDA;
  }
  return GMG_OK;
}

gmg_status tail_configure(gmg_ctx* c, int ncta, int threads, int smem, bool* ok) {
  *ok = false;
  if (cudaFuncSetAttribute(k_tail_cycle, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
      cudaFuncSetAttribute(k_tail_cycle, cudaFuncAttributeMaxDynamicSharedMemorySize, kTailSmemLimit) != cudaSuccess) {
    cudaGetLastError();
    return GMG_OK;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ncta);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = (size_t)smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = ncta;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, k_tail_cycle, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return GMG_OK;
  }
  *ok = nclusters >= 1;
  return GMG_OK;
}

// MGI(x_l, b_l, l) of Alg. 2 on the level's own vectors.  x_l holds the
// initial iterate (zero for every l > 0: the restriction clears it).  With
// c0_done the kernel that produced b_l has already applied the first
// Gauss-Seidel colour to x_l = 0 (the restriction does so for every level it
// feeds that is smoothed), and the first sweep starts at colour 1.
template <class T>
gmg_status vcycle(gmg_ctx* c, int l, cudaStream_t s, bool c0_done, T* x_in, const T* b_in) {
  Level& L = c->L[l];
  T* x = x_in ? x_in : Vec<T>::x(L);
  const T* b = b_in ? b_in : Vec<T>::b(L);
  const bool lp = c->prof && (int)c->lev_ev.size() >= 6 * c->nlev;  // per-level events
  cudaEvent_t* E = lp ? &c->lev_ev[6 * l] : nullptr;
  bool whole = l == c->nlev - 1;
  if constexpr (std::is_same<T, float>::value) whole = whole || (c->tail_l0 > 0 && l == c->tail_l0);
  if (whole) {  // the coarsest solve, or the cluster tail from this level down
    if (c->inv_pending) {  // a refresh's coarsest inverse may still be running: wait for it here
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      GMG_CK(cudaStreamIsCapturing(s, &cs));
      if (cs != cudaStreamCaptureStatusNone) {
        set_error("internal: coarsest inverse pending during a graph capture");
        return GMG_ERR_CUDA;
      }
      GMG_TRY(join_inverse(c, s, false));
    }
    if (lp) {
      GMG_CK(record_timing_event(E[0], s));
      c->lev_kind[l] = 2;
      c->lev_gs[l] = 0;
    }
    if (l == c->nlev - 1) GMG_TRY(launch_coarse<T>(c, b, x, s));
    else GMG_TRY(launch_tail(c, s));
    if (lp) {
      GMG_CK(record_timing_event(E[5], s));
      for (int k = l + 1; k < c->nlev; ++k) c->lev_kind[k] = 0;
    }
    return GMG_OK;
  }
  Level& C = c->L[l + 1];
  if constexpr (std::is_same<T, float>::value) {
    if (c->clev.l == l && l > 0 && c0_done && !x_in && !b_in) {  // this level on a thread-block cluster
      if (lp) GMG_CK(record_timing_event(E[0], s));
      GMG_TRY(launch_cluster_level(c, 0, s));
      if (lp) GMG_CK(record_timing_event(E[1], s));
      GMG_TRY(vcycle<T>(c, l + 1, s, true));
      if (lp) GMG_CK(record_timing_event(E[3], s));
      GMG_TRY(launch_cluster_level(c, 1, s));
      if (lp) {
        GMG_CK(record_timing_event(E[5], s));
        c->lev_kind[l] = 3;
        c->lev_gs[l] = c->opt.nu_pre * L.ncolor - 1 + c->opt.nu_post * L.ncolor;
      }
      return GMG_OK;
    }
  }
  const bool prof = c->prof && l == 0;
  if (prof) GMG_CK(record_timing_event(c->ev[0], s));
  if (lp) GMG_CK(record_timing_event(E[0], s));
  int gs = 0;
  for (int it = 0; it < c->opt.nu_pre; ++it)
    for (int k = (it == 0 && c0_done) ? 1 : 0; k < L.ncolor; ++k, ++gs) GMG_TRY(launch_gs_colour<T>(L, k, b, x, s));
  if (prof) GMG_CK(record_timing_event(c->ev[1], s));
  if (lp) GMG_CK(record_timing_event(E[1], s));
  GMG_TRY(launch_residual<T>(L, x, b, Vec<T>::r(L), s));
  const bool next_c0 = c->opt.nu_pre > 0 && l + 1 < c->nlev - 1;
  GMG_TRY(launch_restrict<T>(L, Vec<T>::r(L), Vec<T>::b(C), Vec<T>::x(C), s, next_c0 ? Vec<T>::dinv(C) : nullptr,
                             next_c0 ? C.color_off[1] : 0));
  if (lp) GMG_CK(record_timing_event(E[2], s));
  GMG_TRY(vcycle<T>(c, l + 1, s, next_c0));
  if (lp) GMG_CK(record_timing_event(E[3], s));
  GMG_TRY(launch_prolong<T>(L, Vec<T>::x(C), x, s));
  if (prof) GMG_CK(record_timing_event(c->ev[2], s));
  if (lp) GMG_CK(record_timing_event(E[4], s));
  for (int it = 0; it < c->opt.nu_post; ++it)
    for (int q = 0; q < L.ncolor; ++q, ++gs) {
      const int k = c->opt.post_forward ? q : L.ncolor - 1 - q;
      GMG_TRY(launch_gs_colour<T>(L, k, b, x, s));
    }
  if (prof) {
    GMG_CK(record_timing_event(c->ev[3], s));
    c->prof_gs = gs;
  }
  if (lp) {
    GMG_CK(record_timing_event(E[5], s));
    c->lev_kind[l] = 1;
    c->lev_gs[l] = gs;
  }
  return GMG_OK;
}

template gmg_status launch_gs_colour<double>(Level&, int, const double*, double*, cudaStream_t);
template gmg_status launch_gs_colour<float>(Level&, int, const float*, float*, cudaStream_t);
template gmg_status launch_residual<double>(Level&, const double*, const double*, double*, cudaStream_t);
template gmg_status launch_residual<float>(Level&, const float*, const float*, float*, cudaStream_t);
template gmg_status launch_restrict<double>(Level&, const double*, double*, double*, cudaStream_t, const double*,
                                           int64_t);
template gmg_status launch_restrict<float>(Level&, const float*, float*, float*, cudaStream_t, const float*, int64_t);
template gmg_status launch_prolong<double>(Level&, const double*, double*, cudaStream_t);
template gmg_status launch_prolong<float>(Level&, const float*, float*, cudaStream_t);
template gmg_status launch_coarse<double>(gmg_ctx*, const double*, double*, cudaStream_t);
template gmg_status launch_coarse<float>(gmg_ctx*, const float*, float*, cudaStream_t);
template gmg_status vcycle<double>(gmg_ctx*, int, cudaStream_t, bool, double*, const double*);
template gmg_status vcycle<float>(gmg_ctx*, int, cudaStream_t, bool, float*, const float*);

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
  const int64_t blocks = (L.A.nslice + (8 / L.rlanes) - 1) / (8 / L.rlanes);
  if (blocks > c->red_cap) {
    set_error("outer residual: more blocks than reduction partials");
    return GMG_ERR_TOO_LARGE;
  }
  int64_t nb = 0;
  GMG_TRY(launch_residual_p<double>(L, c->xs, c->bs, c->rs, c->red, s, &nb));
  return launch(k_reduce_final, 1, 256, s, (int)nb, (const double*)c->red, c->scal + slot);
}

static gmg_status dot(gmg_ctx* c, int64_t n, const double* a, const double* b, int slot, cudaStream_t s) {
  GMG_TRY(launch(k_dot_partial, kRedBlocks, 256, s, n, a, b, c->red));
  return launch(k_reduce_final, 1, 256, s, kRedBlocks, (const double*)c->red, c->scal + slot);
}

// A finest-level V-cycle, bracketed by timing events when profiling is on;
// x and b replace the finest level's own vectors when given.
template <class T>
static gmg_status timed_vcycle(gmg_ctx* c, cudaStream_t s, bool c0_done, T* x = nullptr, const T* b = nullptr) {
  if (c->prof) GMG_CK(record_timing_event(c->ev[4], s));
  GMG_TRY(vcycle<T>(c, 0, s, c0_done, x, b));
  if (c->prof) GMG_CK(record_timing_event(c->ev[5], s));
  return GMG_OK;
}

static bool pcg_mode(int mode) { return mode == GMG_FP32_PCG || mode == GMG_FP64_PCG; }

// z = MGI(0, r) in the mode's cycle precision (FP64: z itself is the cycle's
// iterate; FP32: widened from the finest level's x32).
static gmg_status precond(gmg_ctx* c, int mode, const double* r, double* z, cudaStream_t s) {
  Level& L = c->L[0];
  const int64_t n0 = c->opt.nu_pre > 0 ? L.color_off[1] : 0;
  if (mode == GMG_FP64_PCG) {
    GMG_TRY(launch(k_zero_c0, blocks_for(L.n), 256, s, L.n, r, z, (const double*)L.dinv64, n0));
    return timed_vcycle<double>(c, s, n0 > 0, z, r);
  }
  GMG_TRY(launch(k_d2f_zero, blocks_for(L.n), 256, s, L.n, r, L.b32, L.x32, (const float*)L.dinv32, n0));
  GMG_TRY(timed_vcycle<float>(c, s, n0 > 0));
  return launch_f2d(L.n, L.x32, z, s);
}

// One outer iteration (captured as a graph when enabled).
//  FP64         : x <- MGI(x, b) (FP64 cycle on the iterate), r = b - A x, rr
//  FP32_REFINE  : e = MGI32(0, r), x += e, r = b - A x, rr
//  *_PCG seg 0  : q = A p, pq, alpha = rz/pq, x += alpha p, r -= alpha q, rr
//  *_PCG seg 1  : z = MGI(0, r) (FP32 or FP64 cycle), num = z.(r - r_old),
//                 rz' = r.z, p = z + (num/rz) p, rz = rz'
gmg_status iteration_body(gmg_ctx* c, int mode, int seg, cudaStream_t s, cudaGraphConditionalHandle h, bool check) {
  Level& L = c->L[0];
  const int64_t n = L.n;
  const int64_t n0 = c->opt.nu_pre > 0 ? L.color_off[1] : 0;
  if (mode == GMG_FP64) {
    GMG_TRY(timed_vcycle<double>(c, s, false));  // level-0 x64/b64 alias xs/bs
    return outer_residual(c, S_RR, s);
  }
  if (mode == GMG_FP32_REFINE) {
    GMG_TRY(launch(k_d2f_zero, blocks_for(n), 256, s, n, (const double*)c->rs, L.b32, L.x32, (const float*)L.dinv32,
                   n0));
    GMG_TRY(timed_vcycle<float>(c, s, n0 > 0));
    GMG_TRY(launch(k_add_f2d, blocks_for(n), 256, s, n, (const float*)L.x32, c->xs));
    return outer_residual(c, S_RR, s);
  }
  const bool f64 = mode == GMG_FP64_PCG;
  if (seg == 0) {
    const int64_t nb = (L.A.nslice * 32 + 255) / 256;
    if (nb > c->red_cap) {
      set_error("PCG: more blocks than reduction partials");
      return GMG_ERR_TOO_LARGE;
    }
    GMG_TRY(launch(k_spmv_dot, nb, 256, s, L.A.nslice, L.A.ptr, L.A.row0, L.A.nrow, L.A.col, L.A.v64, L.diag64,
                   (const double*)c->ps, c->qs, c->red, c->red_cnt, c->scal + S_PQ));
    if (f64)
      return launch(k_pcg_axpy<double>, kRedBlocks, 256, s, n, c->scal, (const double*)c->ps, (const double*)c->qs,
                    c->xs, c->rs, c->ros, (float*)nullptr, c->zs, (const double*)L.dinv64, n0, c->red,
                    c->red_cnt + 1, check ? 1 : 0, c->dloop, c->dhist, h);
    return launch(k_pcg_axpy<float>, kRedBlocks, 256, s, n, c->scal, (const double*)c->ps, (const double*)c->qs,
                  c->xs, c->rs, c->ros, L.b32, L.x32, (const float*)L.dinv32, n0, c->red, c->red_cnt + 1,
                  check ? 1 : 0, c->dloop, c->dhist, h);
  }
  // the cycle's right-hand side and initial iterate (colour 0 already
  // smoothed from zero) were set by segment 0
  if (f64) {
    GMG_TRY(timed_vcycle<double>(c, s, n0 > 0, c->zs, (const double*)c->rs));
    GMG_TRY(launch(k_pcg_zdots<double>, kRedBlocks, 256, s, n, (const double*)c->zs, (const double*)c->rs,
                   (const double*)c->ros, c->red, c->red_cnt + 2, c->scal));
    return launch(k_pcg_dir<double>, blocks_for(n), 256, s, n, (const double*)c->scal, (const double*)c->zs, c->ps);
  }
  GMG_TRY(timed_vcycle<float>(c, s, n0 > 0));
  GMG_TRY(launch(k_pcg_zdots<float>, kRedBlocks, 256, s, n, (const float*)L.x32, (const double*)c->rs,
                 (const double*)c->ros, c->red, c->red_cnt + 2, c->scal));
  return launch(k_pcg_dir<float>, blocks_for(n), 256, s, n, (const double*)c->scal, (const float*)L.x32, c->ps);
}

// PCG start: z = MGI(0, r), rz = r.z, p = z (r must be current).
gmg_status pcg_start(gmg_ctx* c, int mode, cudaStream_t s) {
  const int64_t n = c->L[0].n;
  GMG_TRY(precond(c, mode, c->rs, c->zs, s));
  GMG_TRY(dot(c, n, c->rs, c->zs, S_RZ, s));
  return launch(k_copy, blocks_for(n), 256, s, n, (const double*)c->zs, c->ps);
}

// Convergence test of the device-side loop as its own one-thread kernel (the
// CG form runs it inside the last block of k_pcg_axpy instead).
__global__ void k_iter_check(double* sc, int* it, double* hist, cudaGraphConditionalHandle h) {
  pdl_wait();
  pdl_trigger();
  iter_check(sc, it, hist, h);
}

gmg_status loop_body(gmg_ctx* c, int mode, cudaGraphConditionalHandle h, cudaStream_t s) {
  if (pcg_mode(mode)) {
    GMG_TRY(iteration_body(c, mode, 1, s));
    return iteration_body(c, mode, 0, s, h, true);
  }
  GMG_TRY(iteration_body(c, mode, 0, s));
  return launch(k_iter_check, 1, 1, s, c->scal, c->dloop, c->dhist, h);
}

gmg_status outer_residual_norm(gmg_ctx* c, cudaStream_t s) { return outer_residual(c, S_RR, s); }
gmg_status norm_b(gmg_ctx* c, cudaStream_t s) { return dot(c, c->L[0].n, c->bs, c->bs, S_NB2, s); }

}  // namespace gmg
