// One smoothed level of the FP32 V-cycle (Alg. 2) on a thread-block cluster.
//
// The level above the cluster tail is too large for every CTA to hold all of
// it (torus1m level 2: 28,697 rows, 607k entries), yet its colour phases are
// too small for a grid launch each to pay off (≈ 2 µs per phase, mostly the
// kernel boundary and one dependent L2 round trip).  Here its rows are split
// into `ncta` contiguous ranges of the caller's numbering, one per CTA of a
// cluster; every range holds about 1/ncta of each colour.  A CTA keeps in
// shared memory x of its own rows and of the neighbours of its rows that
// other CTAs own (its halo), and b, 1/a_ii, a_ii of its own rows.  A colour
// phase updates the CTA's rows of that colour, stores each new value into
// the halo copies of the CTAs that read it (distributed shared memory), and
// ends with a cluster barrier; the matrix entries of the rows of each phase
// stream from L2 into shared memory three phases ahead (bulk copies by the
// TMA engine, which keeps far more bytes in flight per SM than per-thread
// loads; measured: per-thread 16-byte asynchronous copies left a phase at
// ≈ 3.6 µs, bound by the SM's outstanding requests), so a phase costs the
// barrier and its arithmetic rather than a kernel boundary.
//
// Launch 0 (pre): the pre-smoothing sweeps, the residual, and the restriction
// b_{l+1} = P^T r with x_{l+1} = 0 except that the next level's colour-0 rows
// get their first Gauss-Seidel update, exactly as k_restrict does.  Launch 1
// (post): the prolongation x += P x_{l+1} (each CTA for its own and halo
// rows, the same arithmetic for the same row in every CTA) and the
// post-smoothing sweeps.  Each row's sums run over its entries in the order
// of the level's sliced ELL, so the results are those of the per-colour
// kernels with one warp per row.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <string>
#include <vector>

#include "gmg_cycle.cuh"

namespace gmg {

namespace {

__device__ __forceinline__ unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cl_sync() {
  __syncwarp();
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// v into the same shared-memory location of CTA `rank` of the cluster.
__device__ __forceinline__ void cl_store(float* p, unsigned rank, float v) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(ra), "f"(v) : "memory");
}
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* m, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count) : "memory");
}
// One arrival that also expects `bytes` of bulk copies to complete on m.
__device__ __forceinline__ void mbar_expect(uint64_t* m, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)), "r"(bytes) : "memory");
}
// Bulk copy (TMA engine) of `bytes` (a multiple of 16, both addresses 16-byte
// aligned) from global to this CTA's shared memory, completing on m.
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, uint64_t* m) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(m))
               : "memory");
}
// Waits for the phase of m with the given parity to complete; gives up after
// `polls` polls (sets *err) so that a lost copy cannot hang the GPU.  A
// failing poll suspends the warp for about 3.8 us on GB300 (measured with
// gmg_wait_selftest), so the limit gives up after about one second; a poll
// does not advance while the context is switched out.
constexpr int kWaitPolls = 1 << 18;
__device__ __forceinline__ void mbar_wait(uint64_t* m, unsigned parity, int* err, int polls = kWaitPolls) {
  for (int it = 0; it < polls; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(m)), "r"(parity)
        : "memory");
    if (done) return;
  }
  atomicOr(err, 1);
}

// sum over the slice row's entries of a_ij x_j (shared-memory copies), in
// entry order; the next eight entries' values and columns are loaded while
// the current eight gather x and are added
__device__ __forceinline__ float local_row_dot(const float* val, const int* col, const float* x, int off, int w) {
  float acc = 0.f;
  int c[8];
  float v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    c[k] = k < w ? col[off + k * 32] : 0;
    v[k] = k < w ? val[off + k * 32] : 0.f;
  }
  for (int q = 0; q < w; q += 8) {
    int cn[8];
    float vn[8], xv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      cn[k] = q + 8 + k < w ? col[off + (q + 8 + k) * 32] : 0;
      vn[k] = q + 8 + k < w ? val[off + (q + 8 + k) * 32] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) xv[k] = x[c[k]];
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (q + k < w) acc += v[k] * xv[k];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      c[k] = cn[k];
      v[k] = vn[k];
    }
  }
  return acc;
}

// Colour of stream step j: the Gauss-Seidel phases (pre-smoothing ascending,
// colour 0 of the first sweep skipped when the restriction did it;
// post-smoothing descending unless post_forward), then, before the
// restriction, one residual step per colour.
__device__ __forceinline__ int step_colour(const ClusterLevel& D, int mode, int j, int P) {
  if (j >= P) return j - P;
  if (mode == 0) return (j + (D.c0_first ? 1 : 0)) % D.ncolor;
  const int q = j % D.ncolor;
  return D.post_forward ? q : D.ncolor - 1 - q;
}

}  // namespace

// 1/a_ii and a_ii of every CTA's own rows into its set-up image.
__global__ void k_clevel_diag(const __grid_constant__ ClusterLevel D, char* __restrict__ img) {
  const int t = blockIdx.y;
  float* di = reinterpret_cast<float*>(img + (int64_t)t * D.st_bytes + (D.o_dinv - D.o_st));
  float* dg = reinterpret_cast<float*>(img + (int64_t)t * D.st_bytes + (D.o_diag - D.o_st));
  const int* l2g = D.loc2glob + D.loc_off[t];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < D.n_own[t]; i += gridDim.x * blockDim.x) {
    di[i] = D.dinv32[l2g[i]];
    dg[i] = D.diag32[l2g[i]];
  }
}

// ent_val[e] = the level's FP32 value in ELL slot src[e] (0 for padding).
__global__ void k_clevel_values(int64_t n, const int64_t* __restrict__ src, const float* __restrict__ v32,
                                float* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = src[e];
    out[e] = s >= 0 ? v32[s] : 0.f;
  }
}

__global__ void __launch_bounds__(256, 1) k_level_cluster(const __grid_constant__ ClusterLevel D, int mode) {
  extern __shared__ __align__(16) char sm[];
  const int cta = (int)cl_rank();
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  float* xl = reinterpret_cast<float*>(sm + D.o_x);
  float* bo = reinterpret_cast<float*>(sm + D.o_b);
  float* dio = reinterpret_cast<float*>(sm + D.o_dinv);
  float* dgo = reinterpret_cast<float*>(sm + D.o_diag);
  int* slrow0 = reinterpret_cast<int*>(sm + D.o_sl);
  int* slnrow = slrow0 + (D.nsl_max + 1);
  int* slw = slnrow + (D.nsl_max + 1);
  int* sleoff = slw + (D.nsl_max + 1);
  int* csl = reinterpret_cast<int*>(sm + D.o_csl);
  char* bufs = sm + D.o_buf;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + D.o_mbar);
  int* l2g = reinterpret_cast<int*>(sm + D.o_l2g);
  int* pp = reinterpret_cast<int*>(sm + D.o_pp);
  int* pd = reinterpret_cast<int*>(sm + D.o_pd);
  const int NS = D.nstage;
  const int stage_bytes = 8 * D.blk_max;
  const int nown = D.n_own[cta], nloc = D.n_loc[cta];
  const float* gval = D.ent_val + D.ent_off[cta];
  const int* gcol = D.ent_col + D.ent_off[cta];
  const int P = mode == 0 ? D.nu_pre * D.ncolor - (D.c0_first ? 1 : 0) : D.nu_post * D.ncolor;
  const int S = P + (mode == 0 ? D.ncolor : 0);

  // the CTA's set-up tables (slices, colours, local-to-global rows, halo
  // stores, 1/a_ii, a_ii): one bulk copy of its image, before the wait for
  // the previous kernel
  if (tid == 0) {
    for (int q = 0; q <= NS; ++q) mbar_init(mbar + q, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    mbar_expect(mbar + NS, (unsigned)D.st_bytes);
    bulk_copy(sm + D.o_st, D.img + (int64_t)cta * D.st_bytes, (unsigned)D.st_bytes, mbar + NS);
  }
  mbar_wait(mbar + NS, 0u, D.err);
  // step j's entry block (values, then columns) into stage j % NS by one
  // thread of the last warp: an arrival expecting the bytes, then two bulk
  // copies; the other warps take the rows
  auto issue = [&](int j) {
    if (tid != nt - 32 || j >= S) return;  // lane 0 of the last warp, which computes no rows
    const int c = step_colour(D, mode, j, P);
    const int e0 = sleoff[csl[c]], e1 = sleoff[csl[c + 1]];
    float* bv = reinterpret_cast<float*>(bufs + (j % NS) * stage_bytes);
    int* bc = reinterpret_cast<int*>(bv + D.blk_max);
    uint64_t* m = mbar + j % NS;
    const unsigned bytes = 4u * (unsigned)(e1 - e0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the stage's earlier reads come first
    mbar_expect(m, 2 * bytes);
    if (bytes) {
      bulk_copy(bv, gval + e0, bytes, m);
      bulk_copy(bc, gcol + e0, bytes, m);
    }
  };
  for (int j = 0; j < NS - 1; ++j) issue(j);
  pdl_wait();  // x and b were written by the previous kernels
  pdl_trigger();
  // gathers of x (own and halo rows) and b (own rows), eight loads in flight per thread
  for (int i0 = tid; i0 < nloc; i0 += 8 * nt) {
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = i0 + k * nt < nloc ? D.x32[l2g[i0 + k * nt]] : 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (i0 + k * nt < nloc) xl[i0 + k * nt] = v[k];
  }
  for (int i0 = tid; i0 < nown; i0 += 8 * nt) {
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = i0 + k * nt < nown ? D.b32[l2g[i0 + k * nt]] : 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (i0 + k * nt < nown) bo[i0 + k * nt] = v[k];
  }
  if (mode == 1) {
    __syncthreads();
    // x += P x_{l+1} on every local row (k_prolong's arithmetic), eight rows
    // per thread at a time so that their loads overlap
    const float* u = D.xc32;
    for (int i0 = tid; i0 < nloc; i0 += 8 * nt) {
      int id[8][3];
      float w[8][3], uv[8][3];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int64_t q = i0 + k * nt < nloc ? 3 * (int64_t)l2g[i0 + k * nt] : 0;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          id[k][m] = D.p_idx[q + m];
          w[k][m] = D.p_w32[q + m];
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k)
#pragma unroll
        for (int m = 0; m < 3; ++m) uv[k][m] = u[id[k][m]];
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (i0 + k * nt < nloc)
          xl[i0 + k * nt] += w[k][0] * uv[k][0] + w[k][1] * uv[k][1] + w[k][2] * uv[k][2];
    }
  }
  __syncthreads();
  cl_sync();  // every CTA's copies are set before any halo store arrives

  for (int j = 0; j < S; ++j) {
    issue(j + NS - 1);
    mbar_wait(mbar + j % NS, (unsigned)(j / NS) & 1u, D.err);
    const int c = step_colour(D, mode, j, P);
    const float* bv = reinterpret_cast<const float*>(bufs + (j % NS) * stage_bytes);
    const int* bc = reinterpret_cast<const int*>(bv + D.blk_max);
    const int s0 = csl[c], s1 = warp < nw - 1 ? csl[c + 1] : s0, ebase = sleoff[s0];
    if (j < P) {
      for (int s = s0 + warp; s < s1; s += nw - 1) {
        const float acc = local_row_dot(bv, bc, xl, sleoff[s] - ebase + lane, slw[s]);
        if (lane < slnrow[s]) {
          const int li = slrow0[s] + lane;
          const float xn = (bo[li] - acc) * dio[li];
          xl[li] = xn;
          for (int q = pp[li]; q < pp[li + 1]; ++q) {
            const int d = pd[q];
            cl_store(xl + (d & 0xFFFF), (unsigned)d >> 16, xn);
          }
        }
      }
      cl_sync();
    } else {
      // residual of the CTA's rows of colour c (k_residual's arithmetic)
      for (int s = s0 + warp; s < s1; s += nw - 1) {
        const float acc = local_row_dot(bv, bc, xl, sleoff[s] - ebase + lane, slw[s]);
        if (lane < slnrow[s]) {
          const int li = slrow0[s] + lane;
          D.r32[l2g[li]] = bo[li] - (acc + dgo[li] * xl[li]);
        }
      }
      __syncthreads();
    }
  }
  for (int i = tid; i < nown; i += nt) D.x32[l2g[i]] = xl[i];
  if (mode == 1) return;
  // b_{l+1} = P^T r over the transpose's slices, one warp per slice across
  // the cluster (k_restrict's arithmetic, terms added in order); x_{l+1} = 0,
  // or b / a_ii on its colour-0 rows.  The first sixteen terms' weights and
  // columns are loaded before the barrier that publishes r, the next sixteen
  // while the current ones gather r.
  const int gw = cta * nw + warp, ngw = D.ncta * nw;
  int64_t sr = gw;
  int wd = 0;
  int64_t e0 = 0;
  int ci[16];
  float wv[16];
  auto load_terms = [&](int q0) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const bool in = q0 + k < wd;
      ci[k] = in ? D.r_col[e0 + (int64_t)(q0 + k) * 32] : 0;
      wv[k] = in ? D.r_v32[e0 + (int64_t)(q0 + k) * 32] : 0.f;
    }
  };
  auto start_slice = [&]() {
    wd = 0;
    if (sr < D.r_nslice && lane < D.r_nrow[sr]) {
      e0 = D.r_ptr[sr] + lane;
      wd = (int)((D.r_ptr[sr + 1] - D.r_ptr[sr]) >> 5);
    }
    load_terms(0);
  };
  start_slice();
  cl_sync();  // the residual of every CTA is in global memory
  for (; sr < D.r_nslice; sr += ngw) {
    float acc = 0.f;
    for (int q0 = 0; q0 < wd; q0 += 16) {
      float rv[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) rv[k] = __ldcg(D.r32 + ci[k]);
      float wc[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) wc[k] = wv[k];
      load_terms(q0 + 16);
#pragma unroll
      for (int k = 0; k < 16; ++k)
        if (q0 + k < wd) acc += wc[k] * rv[k];
    }
    if (wd > 0) {
      const int row = D.r_row0[sr] + lane;
      D.bc32[row] = acc;
      D.xc32[row] = row < D.nc0 ? (acc - 0.f) * D.dinvc32[row] : 0.f;
    }
    const int64_t cur = sr;
    sr += ngw;
    start_slice();
    sr = cur;
  }
}

// ------------------------------------------------------------------ host

static bool cluster_level_fits(const ClusterLevel& D) {
  if (cudaFuncSetAttribute(k_level_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
      cudaFuncSetAttribute(k_level_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, kTailSmemLimit) !=
          cudaSuccess) {  // the limit every handle's layout stays within
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(D.ncta);
  cfg.blockDim = dim3(D.threads);
  cfg.dynamicSmemBytes = (size_t)D.smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = D.ncta;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, k_level_cluster, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return nclusters >= 1;
}

// Builds the tables of the cluster form of level l (the smoothed level just
// above the tail) from its pattern in the caller's numbering (rp, ci), its
// colour-major numbering (perm: new -> old, iperm: old -> new) and its sliced
// ELL, checks every index on the host, and uploads them.  Leaves c->clev.l =
// 0 when the level does not qualify or its tables do not fit.
gmg_status build_cluster_level(gmg_ctx* c, int l, const int64_t* rp, const int32_t* ci,
                               const std::vector<int32_t>& perm, const std::vector<int32_t>& iperm) {
  c->clev = ClusterLevel{};
  if (const char* e = std::getenv("GMG_NO_CLUSTER_LEVEL"))
    if (e[0] == '1') return GMG_OK;
  if (l < 1 || c->tail_l0 != l + 1 || c->opt.nu_pre < 1 || c->opt.nu_post < 0) return GMG_OK;
  Level& L = c->L[l];
  Level& C = c->L[l + 1];
  const int64_t n = L.n;
  const int ncta = 16, threads = 256;
  if (n < 32 * ncta) return GMG_OK;
  // the level's sliced ELL on the host
  const int64_t ns = L.A.nslice;
  std::vector<int64_t> ptr(ns + 1);
  std::vector<int32_t> row0(ns), nrow(ns);
  GMG_CK(cudaMemcpy(ptr.data(), L.A.ptr, (ns + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
  GMG_CK(cudaMemcpy(row0.data(), L.A.row0, ns * sizeof(int32_t), cudaMemcpyDeviceToHost));
  GMG_CK(cudaMemcpy(nrow.data(), L.A.nrow, ns * sizeof(int32_t), cudaMemcpyDeviceToHost));
  std::vector<int32_t> slice_of(n, -1), lane_of(n, -1);
  for (int64_t s = 0; s < ns; ++s)
    for (int q = 0; q < nrow[s]; ++q) {
      slice_of[row0[s] + q] = (int32_t)s;
      lane_of[row0[s] + q] = q;
    }
  std::vector<int32_t> colour(n);
  for (int k = 0; k < L.ncolor; ++k)
    for (int64_t r = L.color_off[k]; r < L.color_off[k + 1]; ++r) colour[r] = k;
  // owner of every row: contiguous ranges of the locality rank (the caller's
  // numbering where that is local)
  std::vector<int32_t> owner(n);
  for (int64_t r = 0; r < n; ++r) owner[r] = (int32_t)((int64_t)L.h_key[perm[r]] * ncta / n);
  // off-diagonal neighbours of a row in ELL entry order
  auto neighbours = [&](int64_t r, std::vector<int32_t>& out) {
    out.clear();
    const int64_t old = perm[r];
    for (int64_t e = rp[old]; e < rp[old + 1]; ++e)
      if (ci[e] != old) out.push_back(iperm[ci[e]]);
  };
  std::vector<std::vector<int32_t>> own(ncta), halo(ncta);
  for (int64_t r = 0; r < n; ++r) own[owner[r]].push_back((int32_t)r);  // ascending: colour by colour
  std::vector<int32_t> local(n, -1);  // local index of a row in its owner
  for (int t = 0; t < ncta; ++t)
    for (size_t i = 0; i < own[t].size(); ++i) local[own[t][i]] = (int32_t)i;
  std::vector<int32_t> nb;
  std::vector<int32_t> n_own(ncta), n_loc(ncta), loc_off(ncta + 1, 0), loc2glob;
  std::vector<int32_t> sl_off(ncta + 1, 0), sl_row0, sl_nrow, sl_w, sl_eoff, csl;
  std::vector<int64_t> ent_off(ncta + 1, 0), src;
  std::vector<int32_t> ecol;
  int n_loc_max = 0, n_own_max = 0, nsl_max = 0, blk_max = 0;
  for (int t = 0; t < ncta; ++t) {
    // halo: neighbours of own rows owned elsewhere, ascending
    std::vector<int32_t>& h = halo[t];
    for (int32_t r : own[t]) {
      neighbours(r, nb);
      for (int32_t j : nb)
        if (owner[j] != t) h.push_back(j);
    }
    std::sort(h.begin(), h.end());
    h.erase(std::unique(h.begin(), h.end()), h.end());
    n_own[t] = (int32_t)own[t].size();
    n_loc[t] = n_own[t] + (int32_t)h.size();
    if (n_loc[t] > 65535) return GMG_OK;  // halo stores pack the local index in 16 bits
    loc_off[t + 1] = loc_off[t] + n_loc[t];
    for (int32_t r : own[t]) loc2glob.push_back(r);
    for (int32_t r : h) loc2glob.push_back(r);
    auto loc_of = [&](int32_t j) -> int32_t {
      if (owner[j] == t) return local[j];
      const auto it = std::lower_bound(h.begin(), h.end(), j);
      return n_own[t] + (int32_t)(it - h.begin());
    };
    // slices: own rows of each colour in chunks of 32, entries [k][lane]
    int nsl = 0;
    int64_t e = 0;
    size_t i = 0;
    for (int k = 0; k < L.ncolor; ++k) {
      csl.push_back(nsl);
      const int64_t blk0 = e;
      while (i < own[t].size() && colour[own[t][i]] == k) {
        const size_t i0 = i;
        int w = 0;
        while (i < own[t].size() && colour[own[t][i]] == k && i - i0 < 32) {
          const int64_t r = own[t][i];
          w = std::max<int>(w, (int)(rp[perm[r] + 1] - rp[perm[r]] - 1));
          ++i;
        }
        const int nr = (int)(i - i0);
        sl_row0.push_back((int32_t)i0);
        sl_nrow.push_back(nr);
        sl_w.push_back(w);
        sl_eoff.push_back((int32_t)e);
        const size_t base = src.size();
        src.resize(base + (size_t)32 * w, -1);
        ecol.resize(base + (size_t)32 * w, 0);
        for (int q = 0; q < nr; ++q) {
          const int64_t r = own[t][i0 + q];
          neighbours(r, nb);
          const int64_t gs = slice_of[r], gl = lane_of[r];
          for (size_t kk = 0; kk < nb.size(); ++kk) {
            src[base + kk * 32 + q] = ptr[gs] + (int64_t)kk * 32 + gl;
            ecol[base + kk * 32 + q] = loc_of(nb[kk]);
          }
        }
        e += (int64_t)32 * w;
        ++nsl;
      }
      blk_max = std::max<int>(blk_max, (int)(e - blk0));
    }
    csl.push_back(nsl);
    if (i != own[t].size()) {
      set_error("internal: cluster level rows of a CTA are not colour by colour");
      return GMG_ERR_INVALID_ARG;
    }
    sl_row0.push_back(n_own[t]);  // sentinel slice: the end of the entries
    sl_nrow.push_back(0);
    sl_w.push_back(0);
    sl_eoff.push_back((int32_t)e);
    sl_off[t + 1] = sl_off[t] + nsl + 1;
    ent_off[t + 1] = ent_off[t] + e;
    n_loc_max = std::max(n_loc_max, n_loc[t]);
    n_own_max = std::max(n_own_max, n_own[t]);
    nsl_max = std::max(nsl_max, nsl);
    if (e > INT32_MAX) return GMG_OK;
  }
  // halo stores: each CTA's halo row is written by its owner in the row's phase
  std::vector<std::vector<std::pair<int32_t, int32_t>>> pushes(n);  // per row: (CTA, local index)
  for (int t = 0; t < ncta; ++t)
    for (size_t q = 0; q < halo[t].size(); ++q) pushes[halo[t][q]].push_back({t, n_own[t] + (int32_t)q});
  std::vector<int32_t> push_off(ncta + 1, 0), push_ptr, push_dst;
  for (int t = 0; t < ncta; ++t) {
    push_off[t] = (int32_t)push_ptr.size();
    for (int32_t r : own[t]) {
      push_ptr.push_back((int32_t)push_dst.size());
      for (const auto& d : pushes[r]) push_dst.push_back((d.first << 16) | d.second);
    }
    push_ptr.push_back((int32_t)push_dst.size());
  }
  // With little locality in the caller's numbering (a point cloud in random
  // order: measured 11-13 halo stores per row on a kNN cloud against 0.3-0.8
  // on the meshes) a phase would store nearly every row into every CTA, and the
  // per-colour launches are kept.
  if ((int64_t)push_dst.size() > 2 * n) return GMG_OK;
  // host check of every index the kernel uses
  {
    bool ok = true;
    std::vector<int> halo_writes(loc_off[ncta], 0);
    for (int t = 0; t < ncta && ok; ++t) {
      for (int i = 0; i < n_own[t] && ok; ++i) {
        ok = owner[loc2glob[loc_off[t] + i]] == t;
        for (int q = push_ptr[push_off[t] + i]; q < push_ptr[push_off[t] + i + 1] && ok; ++q) {
          const int d = push_dst[q], tt = d >> 16, li = d & 0xFFFF;
          ok = tt >= 0 && tt < ncta && tt != t && li >= n_own[tt] && li < n_loc[tt] &&
               loc2glob[loc_off[tt] + li] == loc2glob[loc_off[t] + i];
          if (ok) ++halo_writes[loc_off[tt] + li];
        }
      }
      const int nsl = csl[(size_t)t * (L.ncolor + 1) + L.ncolor];
      int covered = 0;
      for (int s = 0; s < nsl && ok; ++s) {
        const int g = sl_off[t] + s;
        ok = sl_row0[g] == covered && sl_nrow[g] >= 1 && sl_nrow[g] <= 32 && sl_eoff[g + 1] - sl_eoff[g] == 32 * sl_w[g];
        covered += sl_nrow[g];
        for (int64_t e = ent_off[t] + sl_eoff[g]; e < ent_off[t] + sl_eoff[g + 1] && ok; ++e)
          ok = ecol[e] >= 0 && ecol[e] < n_loc[t] && src[e] < ptr[ns];
      }
      ok = ok && covered == n_own[t];
    }
    for (int t = 0; t < ncta && ok; ++t)
      for (int li = n_own[t]; li < n_loc[t] && ok; ++li) ok = halo_writes[loc_off[t] + li] == 1;
    if (!ok) {
      set_error("internal: cluster level tables failed their host check");
      return GMG_ERR_INVALID_ARG;
    }
  }
  // shared-memory layout
  ClusterLevel D{};
  auto al = [](int64_t v) { return (int)((v + 15) & ~(int64_t)15); };
  D.o_x = 0;
  D.o_b = al(D.o_x + 4 * (int64_t)n_loc_max);
  D.o_st = al(D.o_b + 4 * (int64_t)n_own_max);
  D.o_dinv = D.o_st;
  D.o_diag = al(D.o_dinv + 4 * (int64_t)n_own_max);
  D.o_sl = al(D.o_diag + 4 * (int64_t)n_own_max);
  D.o_csl = al(D.o_sl + 16 * (int64_t)(nsl_max + 1));
  int push_max = 0;
  for (int t = 0; t < ncta; ++t)
    push_max = std::max(push_max, push_ptr[push_off[t] + n_own[t]] - push_ptr[push_off[t]]);
  D.o_l2g = al(D.o_csl + 4 * (int64_t)(L.ncolor + 1));
  D.o_pp = al(D.o_l2g + 4 * (int64_t)n_loc_max);
  D.o_pd = al(D.o_pp + 4 * (int64_t)(n_own_max + 1));
  D.st_bytes = al(D.o_pd + 4 * (int64_t)std::max(push_max, 1)) - D.o_st;
  D.o_mbar = D.o_st + D.st_bytes;
  D.o_buf = al(D.o_mbar + 8 * (int64_t)(kClusterStagesMax + 1));
  // as many entry stages (up to four: the current phase and three ahead) as fit
  D.nstage = 0;
  for (int ns_try = kClusterStagesMax; ns_try >= 2 && D.nstage == 0; --ns_try)
    if ((int64_t)D.o_buf + (int64_t)ns_try * 8 * blk_max <= kTailSmemLimit) D.nstage = ns_try;
  if (D.nstage == 0) return GMG_OK;
  D.smem = (int)((int64_t)D.o_buf + (int64_t)D.nstage * 8 * blk_max);
  D.push_max = push_max;
  D.l = l;
  D.ncta = ncta;
  D.threads = threads;
  D.ncolor = L.ncolor;
  D.nu_pre = c->opt.nu_pre;
  D.nu_post = c->opt.nu_post;
  D.post_forward = c->opt.post_forward;
  D.c0_first = 1;  // the restriction from level l - 1 applies colour 0 of the first sweep
  D.n_loc_max = n_loc_max;
  D.n_own_max = n_own_max;
  D.nsl_max = nsl_max;
  D.blk_max = blk_max;
  if (!cluster_level_fits(D)) return GMG_OK;
  Arena& a = c->arena;
  int32_t *d_n_own, *d_n_loc, *d_loc_off, *d_l2g, *d_sl_off, *d_row0, *d_nrow, *d_w, *d_eoff, *d_csl, *d_ecol,
      *d_push_off, *d_push_ptr, *d_push_dst;
  int64_t* d_ent_off;
  float* d_val;
  auto up32 = [&](int32_t** d, const std::vector<int32_t>& h) -> gmg_status {
    GMG_TRY(a.alloc(d, std::max<size_t>(h.size(), 1)));
    if (!h.empty()) GMG_CK(cudaMemcpy(*d, h.data(), h.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    return GMG_OK;
  };
  GMG_TRY(up32(&d_n_own, n_own));
  GMG_TRY(up32(&d_n_loc, n_loc));
  GMG_TRY(up32(&d_loc_off, loc_off));
  GMG_TRY(up32(&d_l2g, loc2glob));
  GMG_TRY(up32(&d_sl_off, sl_off));
  GMG_TRY(up32(&d_row0, sl_row0));
  GMG_TRY(up32(&d_nrow, sl_nrow));
  GMG_TRY(up32(&d_w, sl_w));
  GMG_TRY(up32(&d_eoff, sl_eoff));
  GMG_TRY(up32(&d_csl, csl));
  GMG_TRY(up32(&d_ecol, ecol));
  GMG_TRY(up32(&d_push_off, push_off));
  GMG_TRY(up32(&d_push_ptr, push_ptr));
  GMG_TRY(up32(&d_push_dst, push_dst));
  GMG_TRY(a.alloc(&d_ent_off, ent_off.size()));
  GMG_CK(cudaMemcpy(d_ent_off, ent_off.data(), ent_off.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  // each CTA's set-up image, laid out as its shared-memory copy (1/a_ii and
  // a_ii are filled after every numeric set-up)
  {
    std::vector<char> img((size_t)ncta * D.st_bytes, 0);
    for (int t = 0; t < ncta; ++t) {
      char* base = img.data() + (size_t)t * D.st_bytes;
      int32_t* i_sl = reinterpret_cast<int32_t*>(base + (D.o_sl - D.o_st));
      const int nsl = csl[(size_t)t * (L.ncolor + 1) + L.ncolor];
      for (int q = 0; q <= nsl; ++q) {
        i_sl[q] = sl_row0[sl_off[t] + q];
        i_sl[(nsl_max + 1) + q] = sl_nrow[sl_off[t] + q];
        i_sl[2 * (nsl_max + 1) + q] = sl_w[sl_off[t] + q];
        i_sl[3 * (nsl_max + 1) + q] = sl_eoff[sl_off[t] + q];
      }
      int32_t* i_csl = reinterpret_cast<int32_t*>(base + (D.o_csl - D.o_st));
      for (int k = 0; k <= L.ncolor; ++k) i_csl[k] = csl[(size_t)t * (L.ncolor + 1) + k];
      int32_t* i_l2g = reinterpret_cast<int32_t*>(base + (D.o_l2g - D.o_st));
      for (int q = 0; q < n_loc[t]; ++q) i_l2g[q] = loc2glob[loc_off[t] + q];
      int32_t* i_pp = reinterpret_cast<int32_t*>(base + (D.o_pp - D.o_st));
      int32_t* i_pd = reinterpret_cast<int32_t*>(base + (D.o_pd - D.o_st));
      const int32_t p0 = push_ptr[push_off[t]];
      for (int q = 0; q <= n_own[t]; ++q) i_pp[q] = push_ptr[push_off[t] + q] - p0;
      for (int32_t q = p0; q < push_ptr[push_off[t] + n_own[t]]; ++q) i_pd[q - p0] = push_dst[q];
    }
    char* d_img;
    GMG_TRY(a.alloc(&d_img, img.size()));
    GMG_CK(cudaMemcpy(d_img, img.data(), img.size(), cudaMemcpyHostToDevice));
    D.img = d_img;
  }
  GMG_TRY(a.alloc(&d_val, std::max<size_t>(src.size(), 1)));
  GMG_TRY(a.alloc(&c->clev_src, std::max<size_t>(src.size(), 1)));
  if (!src.empty())
    GMG_CK(cudaMemcpy(c->clev_src, src.data(), src.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  c->clev_nent = (int64_t)src.size();
  D.n_own = d_n_own;
  D.n_loc = d_n_loc;
  D.loc_off = d_loc_off;
  D.loc2glob = d_l2g;
  D.sl_off = d_sl_off;
  D.sl_row0 = d_row0;
  D.sl_nrow = d_nrow;
  D.sl_w = d_w;
  D.sl_eoff = d_eoff;
  D.csl = d_csl;
  D.ent_off = d_ent_off;
  D.ent_val = d_val;
  D.ent_col = d_ecol;
  D.push_off = d_push_off;
  D.push_ptr = d_push_ptr;
  D.push_dst = d_push_dst;
  D.x32 = L.x32;
  D.b32 = L.b32;
  D.r32 = L.r32;
  D.dinv32 = L.dinv32;
  D.diag32 = L.diag32;
  D.p_idx = L.p_idx;
  D.p_w32 = L.p_w32;
  D.r_ptr = L.R.ptr;
  D.r_row0 = L.R.row0;
  D.r_nrow = L.R.nrow;
  D.r_col = L.R.col;
  D.r_v32 = L.R.v32;
  D.r_nslice = L.R.nslice;
  D.err = c->dstatus + 3;
  D.xc32 = C.x32;
  D.bc32 = C.b32;
  D.dinvc32 = C.dinv32;
  D.nc0 = C.color_off[1];
  GMG_CK(cudaMemset(D.err, 0, sizeof(int)));
  c->clev = D;
  return GMG_OK;
}

// The cluster level's entry values from its level's FP32 ELL values (after
// every numeric set-up).
gmg_status refresh_cluster_values(gmg_ctx* c, cudaStream_t s) {
  if (c->clev.l == 0 || c->clev_nent == 0) return GMG_OK;
  const int64_t grid = std::min<int64_t>((c->clev_nent + 255) / 256, 152 * 8);
  k_clevel_values<<<(unsigned)grid, 256, 0, s>>>(c->clev_nent, c->clev_src, c->L[c->clev.l].A.v32,
                                                  const_cast<float*>(c->clev.ent_val));
  GMG_LAUNCHED();
  k_clevel_diag<<<dim3(8, (unsigned)c->clev.ncta), 256, 0, s>>>(c->clev, const_cast<char*>(c->clev.img));
  GMG_LAUNCHED();
  return GMG_OK;
}

// Self-test of the bounded wait: one warp waits on an mbarrier that nothing
// arrives on, so every poll fails and the wait gives up; elapsed device time
// in *ns.
__global__ void k_wait_selftest(int polls, int* err, unsigned long long* ns) {
  __shared__ uint64_t m;
  if (threadIdx.x == 0) mbar_init(&m, 1);
  __syncthreads();
  unsigned long long t0, t1;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  mbar_wait(&m, 0u, err, polls);
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
  if (threadIdx.x == 0) *ns = t1 - t0;
}

// GMG_ERR_TIMEOUT once if a cluster-level launch gave up waiting for an
// entry block (its results are then not to be trusted); clears the flag.
gmg_status cluster_level_status(gmg_ctx* c, cudaStream_t s) {
  if (c->clev.l == 0) return GMG_OK;
  int h = 0;
  GMG_CK(cudaMemcpyAsync(&h, c->clev.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaStreamSynchronize(s));
  if (h) {
    GMG_CK(cudaMemsetAsync(c->clev.err, 0, sizeof(int), s));
    set_error("cluster level: a wait for streamed matrix entries timed out");
    return GMG_ERR_TIMEOUT;
  }
  return GMG_OK;
}

gmg_status launch_cluster_level(gmg_ctx* c, int mode, cudaStream_t s) {
  const ClusterLevel& D = c->clev;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(D.ncta);
  cfg.blockDim = dim3(D.threads);
  cfg.dynamicSmemBytes = (size_t)D.smem;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = D.ncta;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = use_pdl() ? 2 : 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_level_cluster, D, mode);
  if (e != cudaSuccess) {
    set_error(std::string("cluster level launch: ") + cudaGetErrorString(e));
    return GMG_ERR_CUDA;
  }
  GMG_LAUNCHED();
  return GMG_OK;
}

}  // namespace gmg

// The cluster level's bounded wait run on a barrier that never completes
// (polls <= 0: the limit the solve kernels use).
extern "C" gmg_status gmg_wait_selftest(int polls, int* timed_out, double* ms, void* stream) {
  using namespace gmg;
  if (!timed_out) {
    set_error("gmg_wait_selftest: null pointer");
    return GMG_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int* err = nullptr;
  unsigned long long* ns = nullptr;
  GMG_CK(cudaMalloc((void**)&err, sizeof(int)));
  if (cudaMalloc((void**)&ns, sizeof(unsigned long long)) != cudaSuccess) {
    cudaFree(err);
    set_error("gmg_wait_selftest: cudaMalloc failed");
    return GMG_ERR_OOM;
  }
  int h = 0;
  unsigned long long hns = 0;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 32, 0, s>>>(polls > 0 ? polls : kWaitPolls, err, ns);
    ++g_launches;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hns, ns, sizeof(hns), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(err);
  cudaFree(ns);
  if (e != cudaSuccess) {
    set_error(std::string("gmg_wait_selftest: ") + cudaGetErrorString(e));
    return GMG_ERR_CUDA;
  }
  *timed_out = h;
  if (ms) *ms = 1e-6 * (double)hns;
  return GMG_OK;
}
