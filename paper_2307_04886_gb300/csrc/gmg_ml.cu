// Systems of the form A(t) = M + t L (Eq. (smoothing), M the lumped mass,
// L the Laplacian) kept split, and the adjoint gradient of a loss of the
// solution of A(t) x = M u0:
//   lambda = A^-1 dloss/dx   (same hierarchy: A is symmetric),
//   dloss/du0 = M lambda,    dloss/dt = -lambda^T L x,
//   dloss/dA_ij = -lambda_i x_j on the pattern of A.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "gmg_cycle.cuh"

namespace gmg {

// A_1 values = t L + M (M on the diagonal positions), one thread per row.
__global__ void k_ml_values(int64_t n, const int64_t* __restrict__ rp, const int64_t* __restrict__ dpos, double t,
                            const double* __restrict__ Lval, const double* __restrict__ M, double* __restrict__ A) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = dpos[i];
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      const double tl = __dmul_rn(t, Lval[k]);  // rounded product, then the sum (no fused multiply-add)
      A[k] = k == d ? __dadd_rn(tl, M[i]) : tl;
    }
  }
}

// out = M u (elementwise with the lumped mass)
__global__ void k_mass(int64_t n, const double* __restrict__ M, const double* __restrict__ u, double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = M[i] * u[i];
}

// Row i of the pattern: G_ij = -lambda_i x_j; per-block sums of
// -lambda_i (L x)_i (fixed tree), one thread per row.
__global__ void __launch_bounds__(256)
    k_grad_rows(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                const double* __restrict__ Lval, const double* __restrict__ lam, const double* __restrict__ x,
                double* __restrict__ G, double* __restrict__ partial) {
  __shared__ double red[256];
  const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
  double v = 0.0;
  if (i < n) {
    const double li = lam[i];
    double lx = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      const double xj = x[col[k]];
      lx += Lval[k] * xj;
      if (G) G[k] = -li * xj;
    }
    v = -li * lx;
  }
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_grad_finish(int nblocks, const double* __restrict__ partial, double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int k = threadIdx.x; k < nblocks; k += 256) s += partial[k];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

static int grid_of(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 64)); }

}  // namespace gmg

using namespace gmg;

extern "C" {

gmg_status gmg_setup_ML(gmg_handle* h, const double* M_diag, const gmg_csr* L, double t, int n_prolong,
                        const gmg_prolong* P, const int32_t* const* coloring, const gmg_options* opt,
                        void* stream) {
  if (!h || !M_diag || !L || !L->rowptr || !L->col || !L->val || L->n <= 0 || !(t >= 0.0)) {
    set_error("gmg_setup_ML: null pointer, n <= 0 or t < 0");
    return GMG_ERR_INVALID_ARG;
  }
  const int64_t n = L->n, nnz = L->rowptr[n];
  std::vector<double> Aval(nnz);
  std::vector<int64_t> dpos(n, -1);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = L->rowptr[i]; k < L->rowptr[i + 1]; ++k) {
      Aval[k] = t * L->val[k];
      if (L->col[k] == i) {
        Aval[k] = t * L->val[k] + M_diag[i];
        dpos[i] = k;
      }
    }
  for (int64_t i = 0; i < n; ++i)
    if (dpos[i] < 0) {
      set_error("gmg_setup_ML: L has no diagonal entry in row " + std::to_string(i));
      return GMG_ERR_INVALID_ARG;
    }
  gmg_csr A = {n, L->rowptr, L->col, Aval.data()};
  GMG_TRY(gmg_setup(h, &A, n_prolong, P, coloring, opt, stream));
  gmg_ctx* c = *h;
  auto fail = [&](gmg_status st) {
    std::string keep = gmg_last_error();
    gmg_destroy(c);
    *h = nullptr;
    set_error(keep);
    return st;
  };
  gmg_status st;
  if ((st = c->arena.alloc(&c->ml_M, n)) != GMG_OK) return fail(st);
  if ((st = c->arena.alloc(&c->ml_L, nnz)) != GMG_OK) return fail(st);
  if ((st = c->arena.alloc(&c->ml_dpos, n)) != GMG_OK) return fail(st);
  if (cudaMemcpy(c->ml_M, M_diag, n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->ml_L, L->val, nnz * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->ml_dpos, dpos.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice) != cudaSuccess) {
    set_error("gmg_setup_ML: upload failed");
    return fail(GMG_ERR_CUDA);
  }
  c->ml_t = t;
  return GMG_OK;
}

gmg_status gmg_set_t(gmg_handle h, double t, void* stream) {
  if (!h || !h->ml_L || !(t >= 0.0)) {
    set_error("gmg_set_t: handle not made by gmg_setup_ML, or t < 0");
    return GMG_ERR_INVALID_ARG;
  }
  GMG_CK(cudaSetDevice(h->device));
  cudaStream_t s = (cudaStream_t)stream;
  Level& L0 = h->L[0];
  GMG_TRY(join_inverse(h, s, false));  // a previous refresh's inverse still reads the level values
  k_ml_values<<<grid_of(L0.n), 256, 0, s>>>(L0.n, L0.csr_rowptr, h->ml_dpos, t, h->ml_L, h->ml_M, L0.csr_val);
  GMG_LAUNCHED();
  h->ml_t = t;
  return numeric_setup(h, s, true);
}

gmg_status gmg_mass(gmg_handle h, const double* u, double* out, void* stream) {
  if (!h || !h->ml_M || !u || !out) {
    set_error("gmg_mass: handle not made by gmg_setup_ML, or null vector");
    return GMG_ERR_INVALID_ARG;
  }
  GMG_CK(cudaSetDevice(h->device));
  const int64_t n = h->L[0].n;
  k_mass<<<grid_of(n), 256, 0, (cudaStream_t)stream>>>(n, h->ml_M, u, out);
  GMG_LAUNCHED();
  return GMG_OK;
}

gmg_status gmg_grad(gmg_handle h, const double* lambda, const double* x, double* grad_u0, double* dLdt,
                    double* G_vals, void* stream) {
  if (!h || !h->ml_L || !lambda || !x) {
    set_error("gmg_grad: handle not made by gmg_setup_ML, or null vector");
    return GMG_ERR_INVALID_ARG;
  }
  GMG_CK(cudaSetDevice(h->device));
  cudaStream_t s = (cudaStream_t)stream;
  Level& L0 = h->L[0];
  const int64_t n = L0.n;
  if (grad_u0) {
    k_mass<<<grid_of(n), 256, 0, s>>>(n, h->ml_M, lambda, grad_u0);
    GMG_LAUNCHED();
  }
  if (dLdt || G_vals) {
    const int nb = (int)((n + 255) / 256);
    if (nb > h->red_cap) {
      set_error("gmg_grad: reduction scratch too small");
      return GMG_ERR_TOO_LARGE;
    }
    k_grad_rows<<<nb, 256, 0, s>>>(n, L0.csr_rowptr, L0.csr_col, h->ml_L, lambda, x, G_vals, h->red);
    GMG_LAUNCHED();
    if (dLdt) {
      k_grad_finish<<<1, 256, 0, s>>>(nb, h->red, dLdt);
      GMG_LAUNCHED();
    }
  }
  return GMG_OK;
}

}  // extern "C"

// The pattern gradient under the name of the interface it belongs to:
// G_vals[k] = -lambda_i x_j on L's stored entries and dLdt = -lambda^T L x.
extern "C" gmg_status gmg_grad_pattern(gmg_handle h, const double* lambda, const double* x, double* G_vals, double* dLdt,
                            void* stream) {
  return gmg_grad(h, lambda, x, nullptr, dLdt, G_vals, stream);
}
