// V-cycle of Alg. 2 on the GPU and the outer iterations of Alg. 1.
//
// Layout: every level is renumbered colour by colour; the off-diagonal part
// of A_l is a sliced ELL with 32-row slices stored [k][lane], so the 32 lanes
// of a warp (one slice) read 32 consecutive values and column indices per k.
// A Gauss-Seidel colour is one launch over that colour's slices: rows of a
// colour are never adjacent, so every row reads only other colours' entries
// of x and the in-place update equals sequential Gauss-Seidel in colour order.
// The restriction P_l^T is a sliced ELL over the coarse rows (a gather: no
// atomics, a fixed summation order).  The prolongation reads three packed
// (index, weight) slots per fine row.  The coarsest level applies the
// explicit inverse of its FP64 Cholesky factor as a warp-per-row GEMV.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "gmg_cycle.cuh"

namespace gmg {

// ------------------------------------------------------------------ kernels

template <class T>
__global__ void __launch_bounds__(256) k_gs(int64_t s0, int64_t s1, const int64_t* __restrict__ ptr,
                                            const int32_t* __restrict__ row0, const int32_t* __restrict__ nrow,
                                            const int32_t* __restrict__ col, const T* __restrict__ val,
                                            const T* __restrict__ dinv, const T* __restrict__ b, T* x) {
  const int64_t s = s0 + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= s1 || lane >= nrow[s]) return;
  const int64_t r = row0[s] + lane;
  const int64_t e0 = ptr[s];
  const int w = (int)((ptr[s + 1] - e0) >> 5);
  const T* xr = x;  // entries of other colours: not written by this launch
  T acc = 0;
  int64_t e = e0 + lane;
#pragma unroll 4
  for (int k = 0; k < w; ++k, e += 32) acc += val[e] * __ldg(xr + col[e]);
  x[r] = (b[r] - acc) * dinv[r];
}

template <class T>
__global__ void __launch_bounds__(256) k_residual(int64_t nslice, const int64_t* __restrict__ ptr,
                                                  const int32_t* __restrict__ row0, const int32_t* __restrict__ nrow,
                                                  const int32_t* __restrict__ col, const T* __restrict__ val,
                                                  const T* __restrict__ diag, const T* __restrict__ x,
                                                  const T* __restrict__ b, T* __restrict__ r,
                                                  double* __restrict__ partial) {
  const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  double sq = 0.0;
  if (s < nslice && lane < nrow[s]) {
    const int64_t row = row0[s] + lane;
    const int64_t e0 = ptr[s];
    const int w = (int)((ptr[s + 1] - e0) >> 5);
    T acc = diag[row] * x[row];
    int64_t e = e0 + lane;
#pragma unroll 4
    for (int k = 0; k < w; ++k, e += 32) acc += val[e] * x[col[e]];
    const T rv = b[row] - acc;
    r[row] = rv;
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
                                                  const double* __restrict__ diag, const double* __restrict__ p,
                                                  double* __restrict__ q, double* __restrict__ partial) {
  const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  double pq = 0.0;
  if (s < nslice && lane < nrow[s]) {
    const int64_t row = row0[s] + lane;
    const int64_t e0 = ptr[s];
    const int w = (int)((ptr[s + 1] - e0) >> 5);
    double acc = diag[row] * p[row];
    int64_t e = e0 + lane;
#pragma unroll 4
    for (int k = 0; k < w; ++k, e += 32) acc += val[e] * p[col[e]];
    q[row] = acc;
    pq = p[row] * acc;
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

template <class T>
__global__ void __launch_bounds__(256) k_restrict(int64_t nslice, const int64_t* __restrict__ ptr,
                                                  const int32_t* __restrict__ row0, const int32_t* __restrict__ nrow,
                                                  const int32_t* __restrict__ col, const T* __restrict__ w,
                                                  const T* __restrict__ r, T* __restrict__ bc) {
  const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= nslice || lane >= nrow[s]) return;
  const int64_t e0 = ptr[s];
  const int wd = (int)((ptr[s + 1] - e0) >> 5);
  T acc = 0;
  int64_t e = e0 + lane;
  for (int k = 0; k < wd; ++k, e += 32) acc += w[e] * r[col[e]];
  bc[row0[s] + lane] = acc;
}

template <class T>
__global__ void __launch_bounds__(256) k_prolong(int64_t n, const int32_t* __restrict__ idx, const T* __restrict__ w,
                                                 const T* __restrict__ u, T* __restrict__ x) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = 3 * i;
    x[i] += w[q] * u[idx[q]] + w[q + 1] * u[idx[q + 1]] + w[q + 2] * u[idx[q + 2]];
  }
}

// x = Ainv b, one warp per row, FP64 accumulation in both precisions.
template <class T>
__global__ void __launch_bounds__(256) k_coarse(int n, const double* __restrict__ Ainv, const T* __restrict__ b,
                                                T* __restrict__ x) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const double* a = Ainv + (int64_t)row * n;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s += a[j] * (double)b[j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) x[row] = (T)s;
}

__global__ void k_gather(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ src,
                         double* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[perm[i]];
}
__global__ void k_scatter_vec(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ src,
                              double* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[perm[i]] = src[i];
}
__global__ void k_d2f(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void k_f2d(int64_t n, const float* __restrict__ a, double* __restrict__ b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}
// x += (double) e
__global__ void k_add_f2d(int64_t n, const float* __restrict__ e, double* __restrict__ x) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += (double)e[i];
}

// Deterministic dot product: fixed grid, fixed per-thread ranges, fixed tree.
__global__ void __launch_bounds__(256) k_dot_partial(int64_t n, const double* __restrict__ a,
                                                     const double* __restrict__ b, double* __restrict__ partial) {
  __shared__ double red[256];
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
__global__ void k_reduce_final(int count, const double* __restrict__ partial, double* __restrict__ out) {
  __shared__ double red[256];
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
__global__ void k_pcg_axpy(int64_t n, const double* __restrict__ sc, const double* __restrict__ p,
                           const double* __restrict__ q, double* __restrict__ x, double* __restrict__ r,
                           double* __restrict__ rold) {
  const double alpha = sc[2] / sc[3];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = r[i];
    rold[i] = ri;
    x[i] += alpha * p[i];
    r[i] = ri - alpha * q[i];
  }
}
__global__ void k_pcg_dir(int64_t n, const double* __restrict__ sc, const double* __restrict__ z,
                          double* __restrict__ p) {
  const double beta = sc[4] / sc[2];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}
__global__ void k_copy_scalar(const double* __restrict__ src, double* __restrict__ dst) { *dst = *src; }
// d = r - rold (for the Polak-Ribiere numerator)
__global__ void k_sub(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ d) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = a[i] - b[i];
}

// ------------------------------------------------------------------ launchers

static inline int blocks_for(int64_t threads, int per = 256, int cap = 152 * 64) {
  int64_t g = (threads + per - 1) / per;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

#define LAUNCH_CK() GMG_LAUNCHED()

template <class T>
gmg_status launch_gs_colour(Level& L, int colour, const T* b, T* x, cudaStream_t s) {
  const int64_t s0 = L.color_slice_off[colour], s1 = L.color_slice_off[colour + 1];
  if (s1 <= s0) return GMG_OK;
  const int64_t threads = (s1 - s0) * 32;
  k_gs<T><<<(int)((threads + 255) / 256), 256, 0, s>>>(s0, s1, L.A.ptr, L.A.row0, L.A.nrow, L.A.col,
                                                      Vec<T>::v(L.A), Vec<T>::dinv(L), b, x);
  LAUNCH_CK();
  return GMG_OK;
}

template <class T>
gmg_status launch_residual(Level& L, const T* x, const T* b, T* r, cudaStream_t s) {
  const int64_t threads = L.A.nslice * 32;
  k_residual<T><<<(int)((threads + 255) / 256), 256, 0, s>>>(L.A.nslice, L.A.ptr, L.A.row0, L.A.nrow, L.A.col,
                                                            Vec<T>::v(L.A), Vec<T>::diag(L), x, b, r, nullptr);
  LAUNCH_CK();
  return GMG_OK;
}

template <class T>
gmg_status launch_restrict(Level& L, const T* r, T* bc, cudaStream_t s) {
  const int64_t threads = L.R.nslice * 32;
  k_restrict<T><<<(int)((threads + 255) / 256), 256, 0, s>>>(L.R.nslice, L.R.ptr, L.R.row0, L.R.nrow, L.R.col,
                                                            Vec<T>::v(L.R), r, bc);
  LAUNCH_CK();
  return GMG_OK;
}

template <class T>
gmg_status launch_prolong(Level& L, const T* u, T* x, cudaStream_t s) {
  k_prolong<T><<<blocks_for(L.n), 256, 0, s>>>(L.n, L.p_idx, Vec<T>::pw(L), u, x);
  LAUNCH_CK();
  return GMG_OK;
}

template <class T>
gmg_status launch_coarse(gmg_ctx* c, const T* b, T* x, cudaStream_t s) {
  const int n = (int)c->nco;
  k_coarse<T><<<(n * 32 + 255) / 256, 256, 0, s>>>(n, c->Ainv, b, x);
  LAUNCH_CK();
  return GMG_OK;
}

// MGI(x_l, b_l, l) of Alg. 2 on the level's own vectors.
template <class T>
gmg_status vcycle(gmg_ctx* c, int l, bool zero_x, cudaStream_t s) {
  Level& L = c->L[l];
  T* x = Vec<T>::x(L);
  T* b = Vec<T>::b(L);
  if (l == c->nlev - 1) return launch_coarse<T>(c, b, x, s);
  Level& C = c->L[l + 1];
  const bool prof = c->prof && l == 0;
  if (zero_x) GMG_CK(cudaMemsetAsync(x, 0, sizeof(T) * (size_t)L.n, s));
  if (prof) GMG_CK(cudaEventRecordWithFlags(c->ev[0], s, cudaEventRecordExternal));
  for (int it = 0; it < c->opt.nu_pre; ++it)
    for (int k = 0; k < L.ncolor; ++k) GMG_TRY(launch_gs_colour<T>(L, k, b, x, s));
  if (prof) GMG_CK(cudaEventRecordWithFlags(c->ev[1], s, cudaEventRecordExternal));
  GMG_TRY(launch_residual<T>(L, x, b, Vec<T>::r(L), s));
  GMG_TRY(launch_restrict<T>(L, Vec<T>::r(L), Vec<T>::b(C), s));
  GMG_TRY(vcycle<T>(c, l + 1, true, s));
  GMG_TRY(launch_prolong<T>(L, Vec<T>::x(C), x, s));
  if (prof) GMG_CK(cudaEventRecordWithFlags(c->ev[2], s, cudaEventRecordExternal));
  for (int it = 0; it < c->opt.nu_post; ++it)
    for (int q = 0; q < L.ncolor; ++q) {
      const int k = c->opt.post_forward ? q : L.ncolor - 1 - q;
      GMG_TRY(launch_gs_colour<T>(L, k, b, x, s));
    }
  if (prof) GMG_CK(cudaEventRecordWithFlags(c->ev[3], s, cudaEventRecordExternal));
  return GMG_OK;
}

template gmg_status launch_gs_colour<double>(Level&, int, const double*, double*, cudaStream_t);
template gmg_status launch_gs_colour<float>(Level&, int, const float*, float*, cudaStream_t);
template gmg_status launch_residual<double>(Level&, const double*, const double*, double*, cudaStream_t);
template gmg_status launch_residual<float>(Level&, const float*, const float*, float*, cudaStream_t);
template gmg_status launch_restrict<double>(Level&, const double*, double*, cudaStream_t);
template gmg_status launch_restrict<float>(Level&, const float*, float*, cudaStream_t);
template gmg_status launch_prolong<double>(Level&, const double*, double*, cudaStream_t);
template gmg_status launch_prolong<float>(Level&, const float*, float*, cudaStream_t);
template gmg_status launch_coarse<double>(gmg_ctx*, const double*, double*, cudaStream_t);
template gmg_status launch_coarse<float>(gmg_ctx*, const float*, float*, cudaStream_t);
template gmg_status vcycle<double>(gmg_ctx*, int, bool, cudaStream_t);
template gmg_status vcycle<float>(gmg_ctx*, int, bool, cudaStream_t);

gmg_status launch_gather(int64_t n, const int32_t* perm, const double* src, double* dst, cudaStream_t s) {
  k_gather<<<blocks_for(n), 256, 0, s>>>(n, perm, src, dst);
  LAUNCH_CK();
  return GMG_OK;
}
gmg_status launch_scatter(int64_t n, const int32_t* perm, const double* src, double* dst, cudaStream_t s) {
  k_scatter_vec<<<blocks_for(n), 256, 0, s>>>(n, perm, src, dst);
  LAUNCH_CK();
  return GMG_OK;
}
gmg_status launch_d2f(int64_t n, const double* a, float* b, cudaStream_t s) {
  k_d2f<<<blocks_for(n), 256, 0, s>>>(n, a, b);
  LAUNCH_CK();
  return GMG_OK;
}
gmg_status launch_f2d(int64_t n, const float* a, double* b, cudaStream_t s) {
  k_f2d<<<blocks_for(n), 256, 0, s>>>(n, a, b);
  LAUNCH_CK();
  return GMG_OK;
}

// ------------------------------------------------------------------ outer iteration


// rs = bs - A xs (FP64, finest level) and scal[slot] = ||rs||^2.
static gmg_status outer_residual(gmg_ctx* c, int slot, cudaStream_t s) {
  Level& L = c->L[0];
  const int64_t threads = L.A.nslice * 32;
  const int nb = (int)((threads + 255) / 256);
  k_residual<double><<<nb, 256, 0, s>>>(L.A.nslice, L.A.ptr, L.A.row0, L.A.nrow, L.A.col, L.A.v64, L.diag64, c->xs,
                                        c->bs, c->rs, c->red);
  LAUNCH_CK();
  k_reduce_final<<<1, 256, 0, s>>>(nb, c->red, c->scal + slot);
  LAUNCH_CK();
  return GMG_OK;
}

static gmg_status dot(gmg_ctx* c, int64_t n, const double* a, const double* b, int slot, cudaStream_t s) {
  k_dot_partial<<<kRedBlocks, 256, 0, s>>>(n, a, b, c->red);
  LAUNCH_CK();
  k_reduce_final<<<1, 256, 0, s>>>(kRedBlocks, c->red, c->scal + slot);
  LAUNCH_CK();
  return GMG_OK;
}

// A finest-level V-cycle, bracketed by timing events when profiling is on.
template <class T>
static gmg_status timed_vcycle(gmg_ctx* c, bool zero_x, cudaStream_t s) {
  if (c->prof) GMG_CK(cudaEventRecordWithFlags(c->ev[4], s, cudaEventRecordExternal));
  GMG_TRY(vcycle<T>(c, 0, zero_x, s));
  if (c->prof) GMG_CK(cudaEventRecordWithFlags(c->ev[5], s, cudaEventRecordExternal));
  return GMG_OK;
}

// z = V(r) with one FP32 V-cycle (zero initial guess), widened to FP64.
static gmg_status precond32(gmg_ctx* c, const double* r, double* z, cudaStream_t s) {
  Level& L = c->L[0];
  GMG_TRY(launch_d2f(L.n, r, L.b32, s));
  GMG_TRY(timed_vcycle<float>(c, true, s));
  GMG_TRY(launch_f2d(L.n, L.x32, z, s));
  return GMG_OK;
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
    GMG_TRY(timed_vcycle<double>(c, false, s));  // level-0 x64/b64 alias xs/bs
    return outer_residual(c, S_RR, s);
  }
  if (mode == GMG_FP32_REFINE) {
    GMG_TRY(launch_d2f(n, c->rs, L.b32, s));
    GMG_TRY(timed_vcycle<float>(c, true, s));
    k_add_f2d<<<blocks_for(n), 256, 0, s>>>(n, L.x32, c->xs);
    LAUNCH_CK();
    return outer_residual(c, S_RR, s);
  }
  if (seg == 0) {
    const int64_t threads = L.A.nslice * 32;
    const int nb = (int)((threads + 255) / 256);
    k_spmv_dot<<<nb, 256, 0, s>>>(L.A.nslice, L.A.ptr, L.A.row0, L.A.nrow, L.A.col, L.A.v64, L.diag64, c->ps,
                                  c->qs, c->red);
    LAUNCH_CK();
    k_reduce_final<<<1, 256, 0, s>>>(nb, c->red, c->scal + S_PQ);
    LAUNCH_CK();
    k_pcg_axpy<<<blocks_for(n), 256, 0, s>>>(n, c->scal, c->ps, c->qs, c->xs, c->rs, c->ros);
    LAUNCH_CK();
    return dot(c, n, c->rs, c->rs, S_RR, s);
  }
  GMG_TRY(precond32(c, c->rs, c->zs, s));
  k_sub<<<blocks_for(n), 256, 0, s>>>(n, c->rs, c->ros, c->qs);
  LAUNCH_CK();
  GMG_TRY(dot(c, n, c->zs, c->qs, S_NUM, s));
  GMG_TRY(dot(c, n, c->rs, c->zs, S_RZN, s));
  k_pcg_dir<<<blocks_for(n), 256, 0, s>>>(n, c->scal, c->zs, c->ps);
  LAUNCH_CK();
  k_copy_scalar<<<1, 1, 0, s>>>(c->scal + S_RZN, c->scal + S_RZ);
  LAUNCH_CK();
  return GMG_OK;
}

// PCG start: z = MGI32(0, r), rz = r.z, p = z (r must be current).
gmg_status pcg_start(gmg_ctx* c, cudaStream_t s) {
  const int64_t n = c->L[0].n;
  GMG_TRY(precond32(c, c->rs, c->zs, s));
  GMG_TRY(dot(c, n, c->rs, c->zs, S_RZ, s));
  GMG_CK(cudaMemcpyAsync(c->ps, c->zs, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, s));
  return GMG_OK;
}

gmg_status outer_residual_norm(gmg_ctx* c, cudaStream_t s) { return outer_residual(c, S_RR, s); }
gmg_status norm_b(gmg_ctx* c, cudaStream_t s) { return dot(c, c->L[0].n, c->bs, c->bs, S_NB2, s); }

}  // namespace gmg
