// Hierarchy construction of Sec. 4 on the GPU: from a level's points X_l and
// neighbour graph E_l to the coarse level {X_{l+1}, E_{l+1}} and the
// prolongation P_l with at most three entries per row, level after level.
//
//  * sampling (Sec. 4.2): the points are swept in index order and a point
//    that is still eligible becomes a sample and makes every point within
//    distance r ineligible, the distance being Dijkstra's with Euclidean edge
//    lengths inside the point's 2-ring and r = phi^(-1/3) times the mean edge
//    length.  The sweep is the lexicographically first maximal independent
//    set of the relation "t < s and s lies within r of t"; on the GPU every
//    point first finds the later points within r of it, then the decisions
//    propagate from the points with no earlier point within r: a point taken
//    as a sample rules out the later points within r of it, and a point
//    whose earlier neighbours in that relation have all been ruled out
//    becomes a sample.  The rounds of this propagation run inside one graph
//    launch (a conditional WHILE node) and give exactly the sweep's samples;
//  * graph Voronoi cells (Sec. 4.3): multi-source shortest paths from the
//    samples with ties to the smaller sample index, by Jacobi rounds of
//    lexicographic (distance, sample) minimisation until nothing changes;
//  * coarse neighbour graph: cells that share an edge of E_l;
//  * coarse points: the cell means ("Reducing single-entry rows", Sec. 4.4);
//  * prolongation (Sec. 4.4): for each point the closest point on the
//    candidate triangles (3-cliques of the coarse graph with positive area)
//    around its own cell's sample, barycentric weights of that closest point,
//    ties to the lexicographically smallest triangle; inverse-distance
//    weights over the three closest of the sample and its coarse neighbours
//    when the sample has no candidate triangle; a coarse column left empty
//    makes its sample's own row the identity.
//
// Every geometric quantity is computed with the same IEEE operations in the
// same order as the host builder that produces this project's reference
// hierarchies (explicitly rounded multiplies and adds, no fused
// multiply-add), so the GPU hierarchy is bit-identical to it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <string>
#include <vector>

#include "gmg_internal.cuh"

namespace gmg {
namespace build {

constexpr int kRing = 96;      // points of a 2-ring handled per sampling search
constexpr int kCand = 512;     // coarse-neighbour candidates gathered per cell
constexpr int kFallback = 64;  // candidates of the inverse-distance fallback
constexpr int kBlockRows = 1024;

// ---- explicitly rounded double arithmetic (never contracted into an FMA)
__device__ __forceinline__ double ad(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sb(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double ml(double a, double b) { return __dmul_rn(a, b); }

struct V3 {
  double x, y, z;
};
__device__ __forceinline__ V3 at(const double* X, int64_t i) { return V3{X[3 * i], X[3 * i + 1], X[3 * i + 2]}; }
__device__ __forceinline__ V3 vsub(V3 a, V3 b) { return V3{sb(a.x, b.x), sb(a.y, b.y), sb(a.z, b.z)}; }
__device__ __forceinline__ double vdot(V3 a, V3 b) { return ad(ad(ml(a.x, b.x), ml(a.y, b.y)), ml(a.z, b.z)); }
__device__ __forceinline__ V3 vcross(V3 a, V3 b) {
  return V3{sb(ml(a.y, b.z), ml(a.z, b.y)), sb(ml(a.z, b.x), ml(a.x, b.z)), sb(ml(a.x, b.y), ml(a.y, b.x))};
}
__device__ __forceinline__ double vnorm(V3 a) { return __dsqrt_rn(vdot(a, a)); }
__device__ __forceinline__ double edge_len(const double* X, int64_t u, int64_t v) {
  return vnorm(vsub(at(X, u), at(X, v)));
}

// ---- mean edge length: row sums, block sums, then the block sums in order
__global__ void k_row_lengths(int64_t n, const double* __restrict__ X, const int64_t* __restrict__ rp,
                              const int32_t* __restrict__ ci, double* __restrict__ rsum, int* __restrict__ rcnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    int c = 0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] > i) {
        s = ad(s, edge_len(X, i, ci[k]));
        ++c;
      }
    rsum[i] = s;
    rcnt[i] = c;
  }
}
__global__ void k_block_lengths(int64_t n, const double* __restrict__ rsum, const int* __restrict__ rcnt,
                                double* __restrict__ bsum, int64_t* __restrict__ bcnt) {
  const int64_t nb = (n + kBlockRows - 1) / kBlockRows;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    int64_t c = 0;
    for (int64_t i = b * kBlockRows; i < n && i < (b + 1) * kBlockRows; ++i) {
      s = ad(s, rsum[i]);
      c += rcnt[i];
    }
    bsum[b] = s;
    bcnt[b] = c;
  }
}
// geo[0] = mean edge length, geo[1] = sampling radius f * mean, geo[2] =
// smallest candidate-triangle area 1e-12 * mean^2
__global__ void k_mean_length(int64_t nb, const double* __restrict__ bsum, const int64_t* __restrict__ bcnt,
                              double f, double* __restrict__ geo) {
  double s = 0.0;
  int64_t c = 0;
  for (int64_t b = 0; b < nb; ++b) {
    s = ad(s, bsum[b]);
    c += bcnt[b];
  }
  const double e = c ? s / (double)c : 1.0;
  geo[0] = e;
  geo[1] = ml(f, e);
  geo[2] = ml(ml(1e-12, e), e);
}

// ---- sampling: the later points within r of every point (2-ring Dijkstra)
// With fill == nullptr counts them (and counts every point's earlier points
// within r in `blockers`); else writes them at fill[off[t] ..].
__global__ void k_balls(int64_t n, const double* __restrict__ X, const int64_t* __restrict__ rp,
                        const int32_t* __restrict__ ci, const double* __restrict__ geo, int* __restrict__ nlater,
                        int* __restrict__ blockers, const int64_t* __restrict__ off, int32_t* __restrict__ fill,
                        int* __restrict__ err) {
  const double r = geo[1];
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    int32_t ring[kRing];
    double dist[kRing];
    bool done[kRing];
    int m = 0;
    auto has = [&](int32_t v) {
      for (int q = 0; q < m; ++q)
        if (ring[q] == v) return true;
      return false;
    };
    ring[m++] = (int32_t)s;
    bool over = false;
    for (int64_t k = rp[s]; k < rp[s + 1] && !over; ++k)
      if (!has(ci[k])) {
        if (m == kRing) over = true;
        else ring[m++] = ci[k];
      }
    const int n1 = m;
    for (int q = 1; q < n1 && !over; ++q)
      for (int64_t k = rp[ring[q]]; k < rp[ring[q] + 1] && !over; ++k)
        if (!has(ci[k])) {
          if (m == kRing) over = true;
          else ring[m++] = ci[k];
        }
    if (over) {
      atomicExch(err, 1);
      if (!fill) nlater[s] = 0;
      continue;
    }
    for (int q = 0; q < m; ++q) {
      dist[q] = INFINITY;
      done[q] = false;
    }
    dist[0] = 0.0;
    int out = 0;
    for (;;) {
      int best = -1;
      for (int q = 0; q < m; ++q)
        if (!done[q] && (best < 0 || dist[q] < dist[best])) best = q;
      if (best < 0 || !(dist[best] <= r)) break;
      done[best] = true;
      const int32_t u = ring[best];
      if (u > s) {
        if (fill) fill[off[s] + out] = u;
        else atomicAdd(&blockers[u], 1);
        ++out;
      }
      for (int64_t k = rp[u]; k < rp[u + 1]; ++k) {
        const int32_t v = ci[k];
        int q = 0;
        while (q < m && ring[q] != v) ++q;
        if (q == m || done[q]) continue;
        const double nd = ad(dist[best], edge_len(X, u, v));
        if (nd < dist[q]) dist[q] = nd;
      }
    }
    if (!fill) nlater[s] = out;
  }
}

// Exclusive scan of n int counts into off[0..n] (one block of 1024 threads).
__global__ void k_scan(int64_t n, const int* __restrict__ cnt, int64_t* __restrict__ off) {
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
      const int64_t v = part[k];
      part[k] = acc;
      acc += v;
    }
    off[n] = acc;
  }
  __syncthreads();
  int64_t acc = part[t];
  for (int64_t i = b; i < e; ++i) {
    off[i] = acc;
    acc += cnt[i];
  }
}

enum { UNDECIDED = 0, SAMPLE = 1, RULED_OUT = 2 };

// Points without an earlier point within r are samples: the first frontier.
__global__ void k_mis_start(int64_t n, const int* __restrict__ blockers, int* __restrict__ state,
                            int32_t* __restrict__ front, int* __restrict__ fsize) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    if (blockers[s] == 0) {
      state[s] = SAMPLE;
      front[atomicAdd(fsize, 1)] = (int32_t)s;
    } else {
      state[s] = UNDECIDED;
    }
  }
}

// One propagation round over the points decided in the previous round.
// A sample rules out its later points within r; a ruled-out point counts
// down its later points' undecided earlier points, and the one that reaches
// zero (no earlier point within r was a sample) becomes a sample.  ctl[0] is
// the round, ctl[1] and ctl[2] the sizes of the two frontier buffers (the
// round's input in buffer round & 1), ctl[3] the round limit.  The last block
// to finish starts the next round: it clears the consumed buffer's size and
// sets the loop condition (a new frontier, and the limit not reached).
__global__ void __launch_bounds__(256) k_mis_round(const int64_t* __restrict__ off, const int32_t* __restrict__ later,
                                                   int* __restrict__ state, int* __restrict__ blockers,
                                                   int32_t* __restrict__ fa, int32_t* __restrict__ fb, int* ctl,
                                                   int* counter, cudaGraphConditionalHandle h, int use_h) {
  const int round = ctl[0];
  const int32_t* fin = (round & 1) ? fb : fa;
  int32_t* fout = (round & 1) ? fa : fb;
  const int nin = ctl[1 + (round & 1)];
  int* nout = &ctl[1 + ((round + 1) & 1)];
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nin; q += gridDim.x * blockDim.x) {
    const int32_t t = fin[q];
    const bool sample = state[t] == SAMPLE;
    for (int64_t k = off[t]; k < off[t + 1]; ++k) {
      const int32_t u = later[k];
      if (sample) {
        if (atomicCAS(&state[u], UNDECIDED, RULED_OUT) == UNDECIDED) fout[atomicAdd(nout, 1)] = u;
      } else if (atomicSub(&blockers[u], 1) == 1) {
        state[u] = SAMPLE;
        fout[atomicAdd(nout, 1)] = u;
      }
    }
  }
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    last = atomicAdd(counter, 1) == (int)gridDim.x - 1;
    if (last) *counter = 0;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    ctl[1 + (round & 1)] = 0;
    ctl[0] = round + 1;
    const bool go = *(volatile int*)nout > 0 && round + 1 < ctl[3];
    if (use_h) cudaGraphSetConditional(h, go ? 1u : 0u);
  }
}

// ---- samples in index order: rank of every sample
__global__ void k_sample_flags(int64_t n, const int* __restrict__ state, int* __restrict__ flag) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
    flag[s] = state[s] == SAMPLE ? 1 : 0;
}
__global__ void k_sample_list(int64_t n, const int* __restrict__ flag, const int64_t* __restrict__ rank,
                              int32_t* __restrict__ samples, double* __restrict__ d, int32_t* __restrict__ cell) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    if (flag[s]) {
      samples[rank[s]] = (int32_t)s;
      d[s] = 0.0;
      cell[s] = (int32_t)rank[s];
    } else {
      d[s] = INFINITY;
      cell[s] = INT32_MAX;
    }
  }
}

// ---- graph Voronoi cells: one Jacobi round of lexicographic (distance, sample)
__global__ void k_voronoi(int64_t n, const double* __restrict__ X, const int64_t* __restrict__ rp,
                          const int32_t* __restrict__ ci, const double* __restrict__ d0, const int32_t* __restrict__ c0,
                          double* __restrict__ d1, int32_t* __restrict__ c1, int* __restrict__ changed) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    double bd = d0[v];
    int32_t bc = c0[v];
    for (int64_t k = rp[v]; k < rp[v + 1]; ++k) {
      const int32_t u = ci[k];
      if (c0[u] == INT32_MAX) continue;
      const double nd = ad(d0[u], edge_len(X, u, v));
      if (nd < bd || (nd == bd && c0[u] < bc)) {
        bd = nd;
        bc = c0[u];
      }
    }
    d1[v] = bd;
    c1[v] = bc;
    if (bd != d0[v] || bc != c0[v]) *changed = 1;
  }
}

// ---- cells as lists of their points (ascending)
// Every point lies in some cell (each connected part of the graph holds a
// sample: its smallest point has no earlier point within r); a point left
// without one would be reported through err rather than indexed.
__global__ void k_cell_count(int64_t n, int64_t nc, const int32_t* __restrict__ cell, int* __restrict__ cnt,
                             int* __restrict__ err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (cell[i] < 0 || cell[i] >= nc) {
      atomicExch(err, 4);
      continue;
    }
    atomicAdd(&cnt[cell[i]], 1);
  }
}
__global__ void k_cell_fill(int64_t n, const int32_t* __restrict__ cell, const int64_t* __restrict__ coff,
                            int* __restrict__ cur, int32_t* __restrict__ members) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = cell[i];
    members[coff[c] + atomicAdd(&cur[c], 1)] = (int32_t)i;
  }
}
template <class T>
__device__ void insertion_sort(T* a, int m) {
  for (int i = 1; i < m; ++i) {
    const T v = a[i];
    int j = i - 1;
    while (j >= 0 && v < a[j]) {
      a[j + 1] = a[j];
      --j;
    }
    a[j + 1] = v;
  }
}
// Sorts each cell's points and forms the coarse point: the mean of the
// cell's points summed in index order (shift) or the sample itself.
__global__ void k_cell_points(int64_t nc, const int64_t* __restrict__ coff, int32_t* __restrict__ members,
                              const double* __restrict__ X, const int32_t* __restrict__ samples, int shift,
                              double* __restrict__ Xc) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
    int32_t* m = members + coff[c];
    const int cnt = (int)(coff[c + 1] - coff[c]);
    insertion_sort(m, cnt);
    if (shift) {
      double sx = 0.0, sy = 0.0, sz = 0.0;
      for (int q = 0; q < cnt; ++q) {
        sx = ad(sx, X[3 * (int64_t)m[q]]);
        sy = ad(sy, X[3 * (int64_t)m[q] + 1]);
        sz = ad(sz, X[3 * (int64_t)m[q] + 2]);
      }
      Xc[3 * c] = sx / (double)cnt;
      Xc[3 * c + 1] = sy / (double)cnt;
      Xc[3 * c + 2] = sz / (double)cnt;
    } else {
      for (int d = 0; d < 3; ++d) Xc[3 * c + d] = X[3 * (int64_t)samples[c] + d];
    }
  }
}

// ---- coarse neighbour graph: the cells adjacent to each cell, ascending
__global__ void k_coarse_graph(int64_t nc, const int64_t* __restrict__ coff, const int32_t* __restrict__ members,
                               const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                               const int32_t* __restrict__ cell, int* __restrict__ cnt,
                               const int64_t* __restrict__ crp, int32_t* __restrict__ ccol, int* __restrict__ err) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < nc; a += (int64_t)gridDim.x * blockDim.x) {
    int32_t cand[kCand];
    int m = 0;
    bool over = false;
    for (int64_t q = coff[a]; q < coff[a + 1] && !over; ++q) {
      const int32_t i = members[q];
      for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
        const int32_t b = cell[ci[k]];
        if (b == a) continue;
        int z = 0;
        while (z < m && cand[z] != b) ++z;
        if (z < m) continue;
        if (m == kCand) {
          over = true;
          break;
        }
        cand[m++] = b;
      }
    }
    if (over) {
      atomicExch(err, 2);
      m = 0;
    }
    if (!ccol) {
      cnt[a] = m;
      continue;
    }
    insertion_sort(cand, m);
    for (int z = 0; z < m; ++z) ccol[crp[a] + z] = cand[z];
  }
}

// ---- candidate triangles (c, a, b): a < b adjacent neighbours of c in the
// order of c's row, with area above the threshold
__device__ __forceinline__ bool adjacent(const int64_t* crp, const int32_t* ccol, int32_t a, int32_t b) {
  int64_t lo = crp[a], hi = crp[a + 1];
  while (lo < hi) {
    const int64_t mid = (lo + hi) / 2;
    if (ccol[mid] < b) lo = mid + 1;
    else hi = mid;
  }
  return lo < crp[a + 1] && ccol[lo] == b;
}
__global__ void k_triangles(int64_t nc, const int64_t* __restrict__ crp, const int32_t* __restrict__ ccol,
                            const double* __restrict__ Xc, const double* __restrict__ geo, int* __restrict__ cnt,
                            const int64_t* __restrict__ toff, int32_t* __restrict__ tri) {
  const double min_area = geo[2];
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
    int m = 0;
    for (int64_t p = crp[c]; p < crp[c + 1]; ++p)
      for (int64_t q = p + 1; q < crp[c + 1]; ++q) {
        const int32_t a = ccol[p], b = ccol[q];
        if (!adjacent(crp, ccol, a, b)) continue;
        const V3 C = at(Xc, c);
        const double area = ml(0.5, vnorm(vcross(vsub(at(Xc, a), C), vsub(at(Xc, b), C))));
        if (!(area > min_area)) continue;
        if (tri) {
          tri[2 * (toff[c] + m)] = a;
          tri[2 * (toff[c] + m) + 1] = b;
        }
        ++m;
      }
    if (!tri) cnt[c] = m;
  }
}

// Barycentric coordinates on (a, b, c) of the point of triangle abc closest
// to p: the Voronoi-region classification published by Ericson (Real-Time
// Collision Detection, 2005, Sec. 5.1.5).
__device__ void closest_on_triangle(V3 p, V3 a, V3 b, V3 c, double bary[3]) {
  const V3 ab = vsub(b, a), ac = vsub(c, a), ap = vsub(p, a);
  const double d1 = vdot(ab, ap), d2 = vdot(ac, ap);
  if (d1 <= 0 && d2 <= 0) {
    bary[0] = 1; bary[1] = 0; bary[2] = 0;
    return;
  }
  const V3 bp = vsub(p, b);
  const double d3 = vdot(ab, bp), d4 = vdot(ac, bp);
  if (d3 >= 0 && d4 <= d3) {
    bary[0] = 0; bary[1] = 1; bary[2] = 0;
    return;
  }
  const double vc = sb(ml(d1, d4), ml(d3, d2));
  if (vc <= 0 && d1 >= 0 && d3 <= 0) {
    const double v = d1 / sb(d1, d3);
    bary[0] = sb(1.0, v); bary[1] = v; bary[2] = 0;
    return;
  }
  const V3 cp = vsub(p, c);
  const double d5 = vdot(ab, cp), d6 = vdot(ac, cp);
  if (d6 >= 0 && d5 <= d6) {
    bary[0] = 0; bary[1] = 0; bary[2] = 1;
    return;
  }
  const double vb = sb(ml(d5, d2), ml(d1, d6));
  if (vb <= 0 && d2 >= 0 && d6 <= 0) {
    const double w = d2 / sb(d2, d6);
    bary[0] = sb(1.0, w); bary[1] = 0; bary[2] = w;
    return;
  }
  const double va = sb(ml(d3, d6), ml(d5, d4));
  if (va <= 0 && sb(d4, d3) >= 0 && sb(d5, d6) >= 0) {
    const double w = sb(d4, d3) / ad(sb(d4, d3), sb(d5, d6));
    bary[0] = 0; bary[1] = sb(1.0, w); bary[2] = w;
    return;
  }
  const double den = 1.0 / ad(ad(va, vb), vc);
  const double v = ml(vb, den), w = ml(vc, den);
  bary[0] = sb(sb(1.0, v), w); bary[1] = v; bary[2] = w;
}

__device__ __forceinline__ void sort3(int32_t k[3]) {
  if (k[1] < k[0]) { const int32_t t = k[0]; k[0] = k[1]; k[1] = t; }
  if (k[2] < k[1]) { const int32_t t = k[1]; k[1] = k[2]; k[2] = t; }
  if (k[1] < k[0]) { const int32_t t = k[0]; k[0] = k[1]; k[1] = t; }
}
__device__ __forceinline__ bool lex_less(const int32_t a[3], const int32_t b[3]) {
  for (int s = 0; s < 3; ++s)
    if (a[s] != b[s]) return a[s] < b[s];
  return false;
}

struct DistId {
  double d;
  int32_t id;
  __device__ bool operator<(const DistId& o) const { return d < o.d || (d == o.d && id < o.id); }
};
struct IdW {
  int32_t id;
  double w;
  __device__ bool operator<(const IdW& o) const { return id < o.id || (id == o.id && w < o.w); }
};

// The prolongation row of every fine point (three slots; weight 0 = unused).
__global__ void k_prolong_rows(int64_t n, const double* __restrict__ X, const int32_t* __restrict__ cell,
                               const double* __restrict__ Xc, const int64_t* __restrict__ crp,
                               const int32_t* __restrict__ ccol, const int64_t* __restrict__ toff,
                               const int32_t* __restrict__ tri, int32_t* __restrict__ idx, double* __restrict__ w,
                               int* __restrict__ fallbacks, int* __restrict__ err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = cell[i];
    const V3 p = at(X, i);
    int32_t ent_i[3] = {0, 0, 0};
    double ent_w[3] = {0, 0, 0};
    int ne = 0;
    double best = INFINITY;
    int32_t bk[3] = {0, 0, 0};
    double bw[3] = {0, 0, 0};
    bool found = false;
    for (int64_t t = toff[c]; t < toff[c + 1]; ++t) {
      const int32_t a = tri[2 * t], b = tri[2 * t + 1];
      const V3 C = at(Xc, c), A = at(Xc, a), B = at(Xc, b);
      double bary[3];
      closest_on_triangle(p, C, A, B, bary);
      const V3 q = {ad(ad(ml(bary[0], C.x), ml(bary[1], A.x)), ml(bary[2], B.x)),
                    ad(ad(ml(bary[0], C.y), ml(bary[1], A.y)), ml(bary[2], B.y)),
                    ad(ad(ml(bary[0], C.z), ml(bary[1], A.z)), ml(bary[2], B.z))};
      const V3 pq = vsub(p, q);
      const double d2 = vdot(pq, pq);
      int32_t key[3] = {c, a, b};
      sort3(key);
      const bool better = d2 < best || (d2 == best && lex_less(key, bk));
      if (better) {
        best = d2;
        found = true;
        for (int s = 0; s < 3; ++s) bk[s] = key[s];
        const int32_t tv[3] = {c, a, b};
        for (int s = 0; s < 3; ++s)
          for (int u = 0; u < 3; ++u)
            if (tv[u] == key[s]) bw[s] = bary[u];
      }
    }
    if (found) {
      for (int s = 0; s < 3; ++s)
        if (bw[s] > 0) {
          ent_i[ne] = bk[s];
          ent_w[ne] = bw[s];
          ++ne;
        }
    } else {
      // inverse-distance weights over the three closest of {c} and c's coarse neighbours
      atomicAdd(fallbacks, 1);
      DistId cand[kFallback];
      int m = 0;
      cand[m++] = DistId{vnorm(vsub(p, at(Xc, c))), c};
      for (int64_t k = crp[c]; k < crp[c + 1]; ++k) {
        if (m == kFallback) {
          atomicExch(err, 3);
          break;
        }
        cand[m++] = DistId{vnorm(vsub(p, at(Xc, ccol[k]))), ccol[k]};
      }
      insertion_sort(cand, m);
      const int mm = m < 3 ? m : 3;
      if (cand[0].d == 0.0) {
        ent_i[0] = cand[0].id;
        ent_w[0] = 1.0;
        ne = 1;
      } else {
        double s = 0.0;
        for (int q = 0; q < mm; ++q) s = ad(s, 1.0 / cand[q].d);
        IdW e[3];
        for (int q = 0; q < mm; ++q) e[q] = IdW{cand[q].id, (1.0 / cand[q].d) / s};
        insertion_sort(e, mm);
        for (int q = 0; q < mm; ++q) {
          ent_i[ne] = e[q].id;
          ent_w[ne] = e[q].w;
          ++ne;
        }
      }
    }
    for (int s = 0; s < 3; ++s) {
      idx[3 * i + s] = s < ne ? ent_i[s] : ent_i[0];
      w[3 * i + s] = s < ne ? ent_w[s] : 0.0;
    }
  }
}

// Empty coarse columns (possible after the shift): the sample's own row
// becomes the identity on its column, repeated until every column is used
// (one thread; it happens rarely).  stats[1] = repaired columns, stats[2] =
// single-entry rows.
__global__ void k_repair(int64_t n, int64_t nc, const int32_t* __restrict__ samples, int32_t* __restrict__ idx,
                         double* __restrict__ w, int* __restrict__ colcount, int64_t* __restrict__ stats) {
  for (int64_t i = 0; i < n; ++i)
    for (int s = 0; s < 3; ++s)
      if (w[3 * i + s] != 0) colcount[idx[3 * i + s]]++;
  bool changed = true;
  int64_t repaired = 0;
  while (changed) {
    changed = false;
    for (int64_t c = 0; c < nc; ++c) {
      if (colcount[c] > 0) continue;
      const int64_t i = samples[c];
      for (int s = 0; s < 3; ++s)
        if (w[3 * i + s] != 0) colcount[idx[3 * i + s]]--;
      idx[3 * i] = idx[3 * i + 1] = idx[3 * i + 2] = (int32_t)c;
      w[3 * i] = 1.0;
      w[3 * i + 1] = w[3 * i + 2] = 0.0;
      colcount[c] = 1;
      ++repaired;
      changed = true;
    }
  }
  int64_t single = 0;
  for (int64_t i = 0; i < n; ++i) {
    int cnt = 0;
    for (int s = 0; s < 3; ++s) cnt += w[3 * i + s] != 0;
    single += cnt == 1;
  }
  stats[1] = repaired;
  stats[2] = single;
}

static inline unsigned grid_of(int64_t n, int per = 256) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + per - 1) / per, 152 * 32));
}

}  // namespace build
}  // namespace gmg

// One level of the built hierarchy, on the host.
struct gmg_hier_level {
  int64_t n_fine = 0, n_coarse = 0;
  std::vector<int32_t> idx, samples, cell;
  std::vector<double> w, Xc;
  std::vector<int64_t> crp;
  std::vector<int32_t> ccol;
  int64_t stats[4] = {0, 0, 0, 0};  // fallback rows, repaired columns, single-entry rows, samples
};
struct gmg_hier_ctx {
  std::vector<gmg_hier_level> levels;
  double build_ms = 0.0;
};

namespace gmg {
namespace build {

// Device buffers of one level's construction (freed at the end).
struct Buffers {
  std::vector<void*> ptrs;
  template <class T>
  gmg_status get(T** p, size_t n) {
    *p = nullptr;
    cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(1, n) * sizeof(T));
    if (e != cudaSuccess) {
      set_error(std::string("gmg_build_hierarchy: cudaMalloc: ") + cudaGetErrorString(e));
      return GMG_ERR_OOM;
    }
    ptrs.push_back(*p);
    return GMG_OK;
  }
  ~Buffers() {
    for (void* p : ptrs) cudaFree(p);
  }
};

// The sampling propagation rounds until no point is decided any more: in a
// graph holding a conditional WHILE node when the driver accepts it, else
// launched from the host in batches.
static gmg_status run_mis(int64_t n, const int64_t* off, const int32_t* later, int* state, int* blockers,
                          int32_t* fa, int32_t* fb, int* ctl, int* counter, cudaStream_t s) {
  const unsigned grid = 152 * 2;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
  cudaGraphConditionalHandle h = 0;
  cudaGraphNodeParams np = {};
  if (ok) ok = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
  if (ok) {
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) == cudaSuccess;
  }
  if (ok) {
    cudaKernelNodeParams kp = {};
    int use_h = 1;
    void* args[] = {(void*)&off, (void*)&later, (void*)&state, (void*)&blockers, (void*)&fa, (void*)&fb,
                    (void*)&ctl, (void*)&counter, (void*)&h, (void*)&use_h};
    kp.func = (void*)k_mis_round;
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(256);
    kp.kernelParams = args;
    cudaGraphNode_t kn;
    ok = cudaGraphAddKernelNode(&kn, np.conditional.phGraph_out[0], nullptr, 0, &kp) == cudaSuccess;
  }
  if (ok) ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (ok) {
    GMG_CK(cudaGraphLaunch(ge, s));
    g_launches += 1;
    cudaGraphExecDestroy(ge);
    return GMG_OK;
  }
  cudaGetLastError();
  if (ge) cudaGraphExecDestroy(ge);
  // host-driven rounds, 64 at a time between checks
  for (;;) {
    for (int k = 0; k < 64; ++k) {
      k_mis_round<<<grid, 256, 0, s>>>(off, later, state, blockers, fa, fb, ctl, counter, 0, 0);
      GMG_LAUNCHED();
    }
    int hc[3];
    GMG_CK(cudaMemcpyAsync(hc, ctl, sizeof(hc), cudaMemcpyDeviceToHost, s));
    GMG_CK(cudaStreamSynchronize(s));
    if ((hc[1] == 0 && hc[2] == 0) || hc[0] > n + 1) return GMG_OK;
  }
}

// One level: points X (device, 3n), neighbour graph (device CSR, symmetric,
// sorted, no self loops) -> the host record and the coarse level's device
// points and graph (allocated with cudaMalloc, owned by the caller).
static gmg_status build_one(int64_t n, const double* X, const int64_t* rp, const int32_t* ci, double phi, int shift,
                            gmg_hier_level& out, double** Xc_out, int64_t** crp_out, int32_t** ccol_out,
                            cudaStream_t s) {
  Buffers B;
  const unsigned G = grid_of(n);
  int* err;
  GMG_TRY(B.get(&err, 1));
  GMG_CK(cudaMemsetAsync(err, 0, sizeof(int), s));
  // mean edge length, radius, smallest triangle area
  const int64_t nb = (n + kBlockRows - 1) / kBlockRows;
  double *rsum, *bsum, *geo;
  int* rcnt;
  int64_t* bcnt;
  GMG_TRY(B.get(&rsum, n));
  GMG_TRY(B.get(&rcnt, n));
  GMG_TRY(B.get(&bsum, nb));
  GMG_TRY(B.get(&bcnt, nb));
  GMG_TRY(B.get(&geo, 3));
  k_row_lengths<<<G, 256, 0, s>>>(n, X, rp, ci, rsum, rcnt);
  GMG_LAUNCHED();
  k_block_lengths<<<grid_of(nb, 64), 64, 0, s>>>(n, rsum, rcnt, bsum, bcnt);
  GMG_LAUNCHED();
  k_mean_length<<<1, 1, 0, s>>>(nb, bsum, bcnt, std::pow(phi, -1.0 / 3.0), geo);
  GMG_LAUNCHED();
  // sampling: the later points within r of every point, then the propagation
  int *nlater, *blockers, *state, *ctl, *counter;
  int64_t* off;
  GMG_TRY(B.get(&nlater, n));
  GMG_TRY(B.get(&blockers, n));
  GMG_TRY(B.get(&state, n));
  GMG_TRY(B.get(&off, n + 1));
  GMG_CK(cudaMemsetAsync(blockers, 0, sizeof(int) * (size_t)n, s));
  k_balls<<<G, 128, 0, s>>>(n, X, rp, ci, geo, nlater, blockers, nullptr, nullptr, err);
  GMG_LAUNCHED();
  k_scan<<<1, 1024, 0, s>>>(n, nlater, off);
  GMG_LAUNCHED();
  int64_t nlat = 0;
  GMG_CK(cudaMemcpyAsync(&nlat, off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaStreamSynchronize(s));
  int32_t *later, *fa, *fb;
  GMG_TRY(B.get(&later, (size_t)nlat));
  GMG_TRY(B.get(&fa, n));
  GMG_TRY(B.get(&fb, n));
  GMG_TRY(B.get(&ctl, 4));
  GMG_TRY(B.get(&counter, 1));
  k_balls<<<G, 128, 0, s>>>(n, X, rp, ci, geo, nlater, blockers, off, later, err);
  GMG_LAUNCHED();
  const int ctl0[4] = {0, 0, 0, (int)std::min<int64_t>(n + 2, INT32_MAX)};
  GMG_CK(cudaMemcpyAsync(ctl, ctl0, sizeof(ctl0), cudaMemcpyHostToDevice, s));
  GMG_CK(cudaMemsetAsync(counter, 0, sizeof(int), s));
  k_mis_start<<<G, 256, 0, s>>>(n, blockers, state, fa, ctl + 1);
  GMG_LAUNCHED();
  GMG_TRY(run_mis(n, off, later, state, blockers, fa, fb, ctl, counter, s));
  // samples in index order
  int* flag;
  int64_t* rank;
  GMG_TRY(B.get(&flag, n));
  GMG_TRY(B.get(&rank, n + 1));
  k_sample_flags<<<G, 256, 0, s>>>(n, state, flag);
  GMG_LAUNCHED();
  k_scan<<<1, 1024, 0, s>>>(n, flag, rank);
  GMG_LAUNCHED();
  int64_t nc = 0;
  int herr = 0;
  GMG_CK(cudaMemcpyAsync(&nc, rank + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaStreamSynchronize(s));
  if (herr == 1) {
    set_error("gmg_build_hierarchy: a 2-ring has more than " + std::to_string(kRing) + " points");
    return GMG_ERR_TOO_LARGE;
  }
  out.n_fine = n;
  out.n_coarse = nc;
  if (nc == 0 || nc >= n) return GMG_OK;  // no coarsening: the caller stops
  int32_t *samples, *cell0, *cell1;
  double *d0, *d1;
  int* changed;
  GMG_TRY(B.get(&samples, nc));
  GMG_TRY(B.get(&cell0, n));
  GMG_TRY(B.get(&cell1, n));
  GMG_TRY(B.get(&d0, n));
  GMG_TRY(B.get(&d1, n));
  GMG_TRY(B.get(&changed, 1));
  k_sample_list<<<G, 256, 0, s>>>(n, flag, rank, samples, d0, cell0);
  GMG_LAUNCHED();
  // graph Voronoi cells
  for (int64_t round = 0;; ++round) {
    GMG_CK(cudaMemsetAsync(changed, 0, sizeof(int), s));
    k_voronoi<<<G, 256, 0, s>>>(n, X, rp, ci, d0, cell0, d1, cell1, changed);
    GMG_LAUNCHED();
    std::swap(d0, d1);
    std::swap(cell0, cell1);
    int hch = 0;
    GMG_CK(cudaMemcpyAsync(&hch, changed, sizeof(int), cudaMemcpyDeviceToHost, s));
    GMG_CK(cudaStreamSynchronize(s));
    if (!hch) break;
    if (round > n) {
      set_error("gmg_build_hierarchy: Voronoi rounds did not settle");
      return GMG_ERR_CUDA;
    }
  }
  const int32_t* cell = cell0;
  // cells as point lists, coarse points
  int *ccnt, *ccur;
  int64_t* coff;
  int32_t* members;
  GMG_TRY(B.get(&ccnt, nc));
  GMG_TRY(B.get(&ccur, nc));
  GMG_TRY(B.get(&coff, nc + 1));
  GMG_TRY(B.get(&members, n));
  GMG_CK(cudaMemsetAsync(ccnt, 0, sizeof(int) * (size_t)nc, s));
  GMG_CK(cudaMemsetAsync(ccur, 0, sizeof(int) * (size_t)nc, s));
  k_cell_count<<<G, 256, 0, s>>>(n, nc, cell, ccnt, err);
  GMG_LAUNCHED();
  GMG_CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaStreamSynchronize(s));
  if (herr == 4) {
    set_error("gmg_build_hierarchy: a point is in no Voronoi cell");
    return GMG_ERR_CUDA;
  }
  k_scan<<<1, 1024, 0, s>>>(nc, ccnt, coff);
  GMG_LAUNCHED();
  k_cell_fill<<<G, 256, 0, s>>>(n, cell, coff, ccur, members);
  GMG_LAUNCHED();
  double* Xc;
  GMG_CK(cudaMalloc(&Xc, sizeof(double) * 3 * (size_t)nc));
  *Xc_out = Xc;
  const unsigned GC = grid_of(nc, 128);
  k_cell_points<<<GC, 128, 0, s>>>(nc, coff, members, X, samples, shift, Xc);
  GMG_LAUNCHED();
  // coarse neighbour graph
  int* gcnt;
  GMG_TRY(B.get(&gcnt, nc));
  int64_t* crp;
  GMG_CK(cudaMalloc(&crp, sizeof(int64_t) * (size_t)(nc + 1)));
  *crp_out = crp;
  k_coarse_graph<<<GC, 64, 0, s>>>(nc, coff, members, rp, ci, cell, gcnt, nullptr, nullptr, err);
  GMG_LAUNCHED();
  k_scan<<<1, 1024, 0, s>>>(nc, gcnt, crp);
  GMG_LAUNCHED();
  int64_t cnnz = 0;
  GMG_CK(cudaMemcpyAsync(&cnnz, crp + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaStreamSynchronize(s));
  int32_t* ccol;
  GMG_CK(cudaMalloc(&ccol, sizeof(int32_t) * (size_t)std::max<int64_t>(1, cnnz)));
  *ccol_out = ccol;
  k_coarse_graph<<<GC, 64, 0, s>>>(nc, coff, members, rp, ci, cell, gcnt, crp, ccol, err);
  GMG_LAUNCHED();
  // candidate triangles
  int* tcnt;
  int64_t* toff;
  GMG_TRY(B.get(&tcnt, nc));
  GMG_TRY(B.get(&toff, nc + 1));
  k_triangles<<<GC, 128, 0, s>>>(nc, crp, ccol, Xc, geo, tcnt, nullptr, nullptr);
  GMG_LAUNCHED();
  k_scan<<<1, 1024, 0, s>>>(nc, tcnt, toff);
  GMG_LAUNCHED();
  int64_t ntri = 0;
  GMG_CK(cudaMemcpyAsync(&ntri, toff + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaStreamSynchronize(s));
  int32_t* tri;
  GMG_TRY(B.get(&tri, 2 * (size_t)ntri));
  k_triangles<<<GC, 128, 0, s>>>(nc, crp, ccol, Xc, geo, tcnt, toff, tri);
  GMG_LAUNCHED();
  // prolongation rows, repair, statistics
  int32_t* idx;
  double* w;
  int *fallbacks, *colcount;
  int64_t* stats;
  GMG_TRY(B.get(&idx, 3 * (size_t)n));
  GMG_TRY(B.get(&w, 3 * (size_t)n));
  GMG_TRY(B.get(&fallbacks, 1));
  GMG_TRY(B.get(&colcount, nc));
  GMG_TRY(B.get(&stats, 4));
  GMG_CK(cudaMemsetAsync(fallbacks, 0, sizeof(int), s));
  GMG_CK(cudaMemsetAsync(colcount, 0, sizeof(int) * (size_t)nc, s));
  k_prolong_rows<<<G, 128, 0, s>>>(n, X, cell, Xc, crp, ccol, toff, tri, idx, w, fallbacks, err);
  GMG_LAUNCHED();
  k_repair<<<1, 1, 0, s>>>(n, nc, samples, idx, w, colcount, stats);
  GMG_LAUNCHED();
  // to the host
  out.idx.resize(3 * (size_t)n);
  out.w.resize(3 * (size_t)n);
  out.samples.resize(nc);
  out.cell.resize(n);
  out.Xc.resize(3 * (size_t)nc);
  out.crp.resize(nc + 1);
  out.ccol.resize(cnnz);
  int hfb = 0;
  int64_t hst[4];
  GMG_CK(cudaMemcpyAsync(out.idx.data(), idx, sizeof(int32_t) * 3 * (size_t)n, cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaMemcpyAsync(out.w.data(), w, sizeof(double) * 3 * (size_t)n, cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaMemcpyAsync(out.samples.data(), samples, sizeof(int32_t) * (size_t)nc, cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaMemcpyAsync(out.cell.data(), cell, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaMemcpyAsync(out.Xc.data(), Xc, sizeof(double) * 3 * (size_t)nc, cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaMemcpyAsync(out.crp.data(), crp, sizeof(int64_t) * (size_t)(nc + 1), cudaMemcpyDeviceToHost, s));
  if (cnnz) GMG_CK(cudaMemcpyAsync(out.ccol.data(), ccol, sizeof(int32_t) * (size_t)cnnz, cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaMemcpyAsync(&hfb, fallbacks, sizeof(int), cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaMemcpyAsync(hst, stats, sizeof(hst), cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaStreamSynchronize(s));
  if (herr == 2) {
    set_error("gmg_build_hierarchy: a cell borders more than " + std::to_string(kCand) + " cells");
    return GMG_ERR_TOO_LARGE;
  }
  if (herr == 3) {
    set_error("gmg_build_hierarchy: a sample has more than " + std::to_string(kFallback - 1) + " coarse neighbours");
    return GMG_ERR_TOO_LARGE;
  }
  out.stats[0] = hfb;
  out.stats[1] = hst[1];
  out.stats[2] = hst[2];
  out.stats[3] = nc;
  return GMG_OK;
}

}  // namespace build
}  // namespace gmg

using namespace gmg;

extern "C" gmg_status gmg_build_hierarchy(gmg_hierarchy* out, int64_t n, const double* X, const int64_t* rowptr,
                                          const int32_t* col, double phi, int64_t stop, int max_levels,
                                          void* stream) {
  if (!out || n <= 0 || n > INT32_MAX || !X || !rowptr || !col || !(phi > 0.0 && phi < 1.0) || max_levels < 0) {
    set_error("gmg_build_hierarchy: null pointer, size outside [1, 2^31), phi outside (0, 1) or max_levels < 0");
    return GMG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  const int64_t nnz = rowptr[n];
  for (int64_t i = 0; i < n; ++i) {
    if (rowptr[i + 1] < rowptr[i]) {
      set_error("gmg_build_hierarchy: rowptr not monotone");
      return GMG_ERR_INVALID_ARG;
    }
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
      if (col[k] < 0 || col[k] >= n || col[k] == i || (k > rowptr[i] && col[k] <= col[k - 1])) {
        set_error("gmg_build_hierarchy: row " + std::to_string(i) +
                  " has a column out of range, a self loop, or unsorted columns");
        return GMG_ERR_INVALID_ARG;
      }
  }
  for (int64_t i = 0; i < 3 * n; ++i)
    if (!std::isfinite(X[i])) {
      set_error("gmg_build_hierarchy: non-finite point coordinate");
      return GMG_ERR_NONFINITE;
    }
  cudaStream_t s = (cudaStream_t)stream;
  gmg_hier_ctx* h = new gmg_hier_ctx();
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  double* dX = nullptr;
  int64_t* drp = nullptr;
  int32_t* dci = nullptr;
  auto release = [&]() {
    cudaFree(dX);
    cudaFree(drp);
    cudaFree(dci);
    dX = nullptr;
    drp = nullptr;
    dci = nullptr;
  };
  gmg_status st = GMG_OK;
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess && st == GMG_OK) {
      set_error(std::string("gmg_build_hierarchy: ") + cudaGetErrorString(e));
      st = e == cudaErrorMemoryAllocation ? GMG_ERR_OOM : GMG_ERR_CUDA;
    }
  };
  ck(cudaMalloc(&dX, sizeof(double) * 3 * (size_t)n));
  ck(cudaMalloc(&drp, sizeof(int64_t) * (size_t)(n + 1)));
  ck(cudaMalloc(&dci, sizeof(int32_t) * (size_t)std::max<int64_t>(1, nnz)));
  if (st == GMG_OK) ck(cudaMemcpyAsync(dX, X, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice, s));
  if (st == GMG_OK) ck(cudaMemcpyAsync(drp, rowptr, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyHostToDevice, s));
  if (st == GMG_OK && nnz)
    ck(cudaMemcpyAsync(dci, col, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, s));
  int64_t cur = n;
  while (st == GMG_OK && cur > stop && (int)h->levels.size() < max_levels) {
    gmg_hier_level lv;
    double* Xc = nullptr;
    int64_t* crp = nullptr;
    int32_t* ccol = nullptr;
    st = build::build_one(cur, dX, drp, dci, phi, 1, lv, &Xc, &crp, &ccol, s);
    const bool stop_here = st != GMG_OK || lv.n_coarse == 0 || lv.n_coarse >= cur;
    release();
    dX = Xc;
    drp = crp;
    dci = ccol;
    if (stop_here) break;
    cur = lv.n_coarse;
    h->levels.push_back(std::move(lv));
  }
  release();
  cudaEventRecord(e1, s);
  if (cudaEventSynchronize(e1) == cudaSuccess) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    h->build_ms = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != GMG_OK) {
    delete h;
    return st;
  }
  *out = h;
  return GMG_OK;
}

extern "C" gmg_status gmg_hierarchy_info(gmg_hierarchy h, int* n_prolong, double* build_ms) {
  if (!h) {
    set_error("gmg_hierarchy_info: null hierarchy");
    return GMG_ERR_INVALID_ARG;
  }
  if (n_prolong) *n_prolong = (int)h->levels.size();
  if (build_ms) *build_ms = h->build_ms;
  return GMG_OK;
}

extern "C" gmg_status gmg_hierarchy_level(gmg_hierarchy h, int l, int64_t* n_fine, int64_t* n_coarse,
                                          int64_t* graph_nnz, int32_t* idx, double* w, int32_t* samples,
                                          int32_t* cell, double* Xc, int64_t* graph_rowptr, int32_t* graph_col,
                                          int64_t* stats) {
  if (!h || l < 0 || l >= (int)h->levels.size()) {
    set_error("gmg_hierarchy_level: null hierarchy or level out of range");
    return GMG_ERR_INVALID_ARG;
  }
  const gmg_hier_level& L = h->levels[l];
  if (n_fine) *n_fine = L.n_fine;
  if (n_coarse) *n_coarse = L.n_coarse;
  if (graph_nnz) *graph_nnz = (int64_t)L.ccol.size();
  if (idx) std::copy(L.idx.begin(), L.idx.end(), idx);
  if (w) std::copy(L.w.begin(), L.w.end(), w);
  if (samples) std::copy(L.samples.begin(), L.samples.end(), samples);
  if (cell) std::copy(L.cell.begin(), L.cell.end(), cell);
  if (Xc) std::copy(L.Xc.begin(), L.Xc.end(), Xc);
  if (graph_rowptr) std::copy(L.crp.begin(), L.crp.end(), graph_rowptr);
  if (graph_col) std::copy(L.ccol.begin(), L.ccol.end(), graph_col);
  if (stats) std::copy(L.stats, L.stats + 4, stats);
  return GMG_OK;
}

extern "C" gmg_status gmg_destroy_hierarchy(gmg_hierarchy h) {
  delete h;
  return GMG_OK;
}
