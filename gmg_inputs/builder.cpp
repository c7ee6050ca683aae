// Host hierarchy builder: one coarsening level of the graph-Voronoi
// construction of Sec. 4 (sampling Sec. 4.2, neighbour graph Sec. 4.3,
// prolongation Sec. 4.4).  It turns a level {V_l, E_l} into the coarse level
// {V_{l+1}, E_{l+1}} and the prolongation P_l (at most three entries per row).
//
// The output is an INPUT of the multigrid solve: both the CPU oracle and the
// GPU library receive P_l as arrays and share none of this code's arithmetic
// with each other.
//
// Readings where the paper leaves details open:
//  * "geodesic distance r" during sampling = Dijkstra distance with Euclidean
//    edge lengths, explored only inside the 2-ring of the sample (Sec. 4.2);
//  * points are swept in index order (Sec. 4.2);
//  * graph Voronoi cells: multi-source Dijkstra with Euclidean edge lengths,
//    ties resolved towards the smaller seed id (Sec. 4.3);
//  * "coarse point closest to p" = p's own Voronoi seed (Sec. 4.4);
//  * the coarse points are moved to the mean of their cells before the
//    projection (Sec. 4.4, "Reducing single-entry rows"); the moved positions
//    are also the positions of level l+1;
//  * a triangle is a candidate when its three coarse edges exist and its area
//    exceeds 1e-12 * ehat^2; the fallback (inverse-distance weights over the
//    three closest points of the seed's neighbourhood) is taken only when the
//    seed has no candidate triangle (Sec. 4.4, "Edge-cases");
//  * closest point on a triangle: the Voronoi-region classification published
//    by Ericson (Real-Time Collision Detection, 2005, Sec. 5.1.5);
//  * a coarse column left empty (possible after the shift) is repaired by
//    making the seed's own fine row the identity on that column.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <queue>
#include <vector>

namespace {

struct V3 {
  double x, y, z;
};
inline V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }

// Barycentric coordinates (u, v, w) on (a, b, c) of the point of triangle abc
// closest to p.
void closest_on_triangle(V3 p, V3 a, V3 b, V3 c, double bary[3]) {
  V3 ab = sub(b, a), ac = sub(c, a), ap = sub(p, a);
  double d1 = dot(ab, ap), d2 = dot(ac, ap);
  if (d1 <= 0 && d2 <= 0) { bary[0] = 1; bary[1] = 0; bary[2] = 0; return; }
  V3 bp = sub(p, b);
  double d3 = dot(ab, bp), d4 = dot(ac, bp);
  if (d3 >= 0 && d4 <= d3) { bary[0] = 0; bary[1] = 1; bary[2] = 0; return; }
  double vc = d1 * d4 - d3 * d2;
  if (vc <= 0 && d1 >= 0 && d3 <= 0) {
    double v = d1 / (d1 - d3);
    bary[0] = 1 - v; bary[1] = v; bary[2] = 0; return;
  }
  V3 cp = sub(p, c);
  double d5 = dot(ab, cp), d6 = dot(ac, cp);
  if (d6 >= 0 && d5 <= d6) { bary[0] = 0; bary[1] = 0; bary[2] = 1; return; }
  double vb = d5 * d2 - d1 * d6;
  if (vb <= 0 && d2 >= 0 && d6 <= 0) {
    double w = d2 / (d2 - d6);
    bary[0] = 1 - w; bary[1] = 0; bary[2] = w; return;
  }
  double va = d3 * d6 - d5 * d4;
  if (va <= 0 && (d4 - d3) >= 0 && (d5 - d6) >= 0) {
    double w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
    bary[0] = 0; bary[1] = 1 - w; bary[2] = w; return;
  }
  double den = 1.0 / (va + vb + vc);
  double v = vb * den, w = vc * den;
  bary[0] = 1 - v - w; bary[1] = v; bary[2] = w;
}

struct Level {
  int64_t nc = 0;
  std::vector<int32_t> idx;  // 3 per fine row
  std::vector<double> w;     // 3 per fine row, 0 = padding
  std::vector<double> Xc;    // 3 per coarse point
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  int64_t stats[4] = {0, 0, 0, 0};  // fallback rows, repaired columns, single-entry rows, seeds
  std::vector<int32_t> samples;     // fine index of every coarse point
  std::vector<int32_t> seed;        // Voronoi cell (coarse index) of every fine point
};

struct HeapItem {
  double d;
  int32_t seed;
  int32_t node;
  bool operator>(const HeapItem& o) const {
    if (d != o.d) return d > o.d;
    if (seed != o.seed) return seed > o.seed;
    return node > o.node;
  }
};

Level* build_level(int64_t n, const double* Xp, const int64_t* rp, const int32_t* ci, double phi, int shift) {
  auto X = [&](int64_t i) { return V3{Xp[3 * i], Xp[3 * i + 1], Xp[3 * i + 2]}; };
  Level* L = new Level();

  // mean edge length over undirected edges (i < j).  Summation order: the
  // lengths of a row in pattern order, the rows of each block of 1024
  // consecutive rows in order, then the block sums in order (a fixed order that
  // a parallel builder reproduces exactly)
  double esum = 0;
  int64_t ecount = 0;
  for (int64_t b0 = 0; b0 < n; b0 += 1024) {
    double bsum = 0;
    for (int64_t i = b0; i < std::min<int64_t>(n, b0 + 1024); ++i) {
      double rsum = 0;
      for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
        if (ci[k] > i) { rsum += norm(sub(X(i), X(ci[k]))); ++ecount; }
      bsum += rsum;
    }
    esum += bsum;
  }
  const double ehat = ecount ? esum / ecount : 1.0;
  const double r = std::pow(phi, -1.0 / 3.0) * ehat;  // Eq. (sampling radius)

  // ---- sampling (Sec. 4.2): one sweep, 2-ring restricted Dijkstra ----
  std::vector<char> eligible(n, 1);
  std::vector<int32_t> samples;
  std::vector<int64_t> stamp(n, -1);
  std::vector<double> dist(n, 0.0);
  std::vector<int32_t> ring;
  for (int64_t s = 0; s < n; ++s) {
    if (!eligible[s]) continue;
    samples.push_back((int32_t)s);
    ring.clear();
    ring.push_back((int32_t)s);
    stamp[s] = s;
    for (int64_t k = rp[s]; k < rp[s + 1]; ++k) {
      int32_t a = ci[k];
      if (stamp[a] != s) { stamp[a] = s; ring.push_back(a); }
    }
    size_t n1 = ring.size();
    for (size_t q = 1; q < n1; ++q) {
      int32_t a = ring[q];
      for (int64_t k = rp[a]; k < rp[a + 1]; ++k) {
        int32_t b = ci[k];
        if (stamp[b] != s) { stamp[b] = s; ring.push_back(b); }
      }
    }
    for (int32_t v : ring) dist[v] = INFINITY;
    dist[s] = 0;
    std::priority_queue<std::pair<double, int32_t>, std::vector<std::pair<double, int32_t>>,
                        std::greater<std::pair<double, int32_t>>> pq;
    pq.push({0.0, (int32_t)s});
    while (!pq.empty()) {
      auto [d, u] = pq.top();
      pq.pop();
      if (d > dist[u]) continue;
      if (d > r) break;
      eligible[u] = 0;
      for (int64_t k = rp[u]; k < rp[u + 1]; ++k) {
        int32_t v = ci[k];
        if (stamp[v] != s) continue;  // outside the 2-ring
        double nd = d + norm(sub(X(u), X(v)));
        if (nd < dist[v]) { dist[v] = nd; pq.push({nd, v}); }
      }
    }
  }
  const int64_t nc = (int64_t)samples.size();
  L->nc = nc;
  L->stats[3] = nc;

  // ---- graph Voronoi cells (Sec. 4.3): multi-source Dijkstra ----
  std::vector<double> vd(n, INFINITY);
  std::vector<int32_t> seed(n, -1);
  std::priority_queue<HeapItem, std::vector<HeapItem>, std::greater<HeapItem>> pq;
  for (int64_t c = 0; c < nc; ++c) {
    vd[samples[c]] = 0;
    seed[samples[c]] = (int32_t)c;
    pq.push({0.0, (int32_t)c, samples[c]});
  }
  while (!pq.empty()) {
    HeapItem it = pq.top();
    pq.pop();
    if (it.d > vd[it.node] || (it.d == vd[it.node] && it.seed != seed[it.node])) continue;
    for (int64_t k = rp[it.node]; k < rp[it.node + 1]; ++k) {
      int32_t v = ci[k];
      double nd = it.d + norm(sub(X(it.node), X(v)));
      if (nd < vd[v] || (nd == vd[v] && it.seed < seed[v])) {
        vd[v] = nd;
        seed[v] = it.seed;
        pq.push({nd, it.seed, v});
      }
    }
  }

  // ---- coarse edges E_{l+1}: adjacent Voronoi cells ----
  std::vector<int64_t> keys;
  keys.reserve((size_t)rp[n]);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      int64_t a = seed[i], b = seed[ci[k]];
      if (a != b) keys.push_back(a * nc + b);
    }
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  L->rowptr.assign(nc + 1, 0);
  L->col.resize(keys.size());
  for (size_t q = 0; q < keys.size(); ++q) {
    L->rowptr[keys[q] / nc + 1]++;
    L->col[q] = (int32_t)(keys[q] % nc);
  }
  for (int64_t c = 0; c < nc; ++c) L->rowptr[c + 1] += L->rowptr[c];
  const int64_t* crp = L->rowptr.data();
  const int32_t* cci = L->col.data();
  auto adjacent = [&](int32_t a, int32_t b) {
    return std::binary_search(cci + crp[a], cci + crp[a + 1], b);
  };

  // ---- coarse positions: cell means (shift) or the samples themselves ----
  L->Xc.assign(3 * nc, 0.0);
  if (shift) {
    std::vector<int64_t> cnt(nc, 0);
    for (int64_t i = 0; i < n; ++i) {
      int32_t c = seed[i];
      L->Xc[3 * c] += Xp[3 * i];
      L->Xc[3 * c + 1] += Xp[3 * i + 1];
      L->Xc[3 * c + 2] += Xp[3 * i + 2];
      cnt[c]++;
    }
    for (int64_t c = 0; c < nc; ++c)
      for (int d = 0; d < 3; ++d) L->Xc[3 * c + d] /= (double)cnt[c];
  } else {
    for (int64_t c = 0; c < nc; ++c)
      for (int d = 0; d < 3; ++d) L->Xc[3 * c + d] = Xp[3 * samples[c] + d];
  }
  auto XC = [&](int64_t c) { return V3{L->Xc[3 * c], L->Xc[3 * c + 1], L->Xc[3 * c + 2]}; };

  // ---- candidate triangles per coarse point: 3-cliques of E_{l+1} ----
  const double min_area = 1e-12 * ehat * ehat;
  std::vector<int64_t> tptr(nc + 1, 0);
  std::vector<int32_t> tri;  // pairs (a, b), a < b, triangle (c, a, b)
  for (int64_t c = 0; c < nc; ++c) {
    for (int64_t p = crp[c]; p < crp[c + 1]; ++p)
      for (int64_t q = p + 1; q < crp[c + 1]; ++q) {
        int32_t a = cci[p], b = cci[q];
        if (!adjacent(a, b)) continue;
        double area = 0.5 * norm(cross(sub(XC(a), XC(c)), sub(XC(b), XC(c))));
        if (!(area > min_area)) continue;
        tri.push_back(a);
        tri.push_back(b);
      }
    tptr[c + 1] = (int64_t)tri.size() / 2;
  }

  // ---- prolongation rows (Sec. 4.4) ----
  L->idx.assign(3 * n, 0);
  L->w.assign(3 * n, 0.0);
  for (int64_t i = 0; i < n; ++i) {
    const int32_t c = seed[i];
    const V3 p = X(i);
    int32_t ent_i[3];
    double ent_w[3];
    int ne = 0;
    double best = INFINITY;
    int32_t bk[3] = {0, 0, 0};
    double bw[3] = {0, 0, 0};
    bool found = false;
    for (int64_t t = tptr[c]; t < tptr[c + 1]; ++t) {
      int32_t a = tri[2 * t], b = tri[2 * t + 1];
      double bary[3];
      closest_on_triangle(p, XC(c), XC(a), XC(b), bary);
      V3 q = {bary[0] * XC(c).x + bary[1] * XC(a).x + bary[2] * XC(b).x,
              bary[0] * XC(c).y + bary[1] * XC(a).y + bary[2] * XC(b).y,
              bary[0] * XC(c).z + bary[1] * XC(a).z + bary[2] * XC(b).z};
      double d2 = dot(sub(p, q), sub(p, q));
      int32_t key[3] = {c, a, b};
      std::sort(key, key + 3);
      bool better = d2 < best;
      if (!better && d2 == best) better = std::lexicographical_compare(key, key + 3, bk, bk + 3);
      if (better) {
        best = d2;
        found = true;
        std::memcpy(bk, key, sizeof(bk));
        // weights in sorted-key order
        int32_t tv[3] = {c, a, b};
        for (int s = 0; s < 3; ++s)
          for (int u = 0; u < 3; ++u)
            if (tv[u] == key[s]) bw[s] = bary[u];
      }
    }
    if (found) {
      for (int s = 0; s < 3; ++s)
        if (bw[s] > 0) { ent_i[ne] = bk[s]; ent_w[ne] = bw[s]; ++ne; }
    } else {
      // fallback: inverse-distance weights over the 3 closest of {c} u N(c)
      L->stats[0]++;
      std::vector<std::pair<double, int32_t>> cand;
      cand.push_back({norm(sub(p, XC(c))), c});
      for (int64_t k = crp[c]; k < crp[c + 1]; ++k) cand.push_back({norm(sub(p, XC(cci[k]))), cci[k]});
      std::sort(cand.begin(), cand.end());
      int m = (int)std::min<size_t>(3, cand.size());
      if (cand[0].first == 0.0) {
        ent_i[0] = cand[0].second; ent_w[0] = 1.0; ne = 1;
      } else {
        double s = 0;
        for (int q = 0; q < m; ++q) s += 1.0 / cand[q].first;
        std::vector<std::pair<int32_t, double>> e;
        for (int q = 0; q < m; ++q) e.push_back({cand[q].second, (1.0 / cand[q].first) / s});
        std::sort(e.begin(), e.end());
        for (auto& pr : e) { ent_i[ne] = pr.first; ent_w[ne] = pr.second; ++ne; }
      }
    }
    for (int s = 0; s < 3; ++s) {
      L->idx[3 * i + s] = s < ne ? ent_i[s] : ent_i[0];
      L->w[3 * i + s] = s < ne ? ent_w[s] : 0.0;
    }
  }

  // ---- repair empty coarse columns ----
  std::vector<int64_t> colcount(nc, 0);
  for (int64_t i = 0; i < n; ++i)
    for (int s = 0; s < 3; ++s)
      if (L->w[3 * i + s] != 0) colcount[L->idx[3 * i + s]]++;
  bool changed = true;
  while (changed) {
    changed = false;
    for (int64_t c = 0; c < nc; ++c) {
      if (colcount[c] > 0) continue;
      int64_t i = samples[c];
      for (int s = 0; s < 3; ++s)
        if (L->w[3 * i + s] != 0) colcount[L->idx[3 * i + s]]--;
      L->idx[3 * i] = L->idx[3 * i + 1] = L->idx[3 * i + 2] = (int32_t)c;
      L->w[3 * i] = 1.0;
      L->w[3 * i + 1] = L->w[3 * i + 2] = 0.0;
      colcount[c] = 1;
      L->stats[1]++;
      changed = true;
    }
  }
  for (int64_t i = 0; i < n; ++i) {
    int cnt = 0;
    for (int s = 0; s < 3; ++s) cnt += L->w[3 * i + s] != 0;
    if (cnt == 1) L->stats[2]++;
  }
  L->samples = samples;
  L->seed = seed;
  return L;
}

}  // namespace

extern "C" {

void* gb_build_level(int64_t n, const double* X, const int64_t* rowptr, const int32_t* col, double phi, int shift) {
  return build_level(n, X, rowptr, col, phi, shift);
}

void gb_level_sizes(void* h, int64_t* nc, int64_t* nnz_adj, int64_t* stats) {
  Level* L = (Level*)h;
  *nc = L->nc;
  *nnz_adj = (int64_t)L->col.size();
  for (int k = 0; k < 4; ++k) stats[k] = L->stats[k];
}

void gb_level_copy(void* h, int32_t* idx, double* w, double* Xc, int64_t* rowptr, int32_t* col) {
  Level* L = (Level*)h;
  std::memcpy(idx, L->idx.data(), L->idx.size() * sizeof(int32_t));
  std::memcpy(w, L->w.data(), L->w.size() * sizeof(double));
  std::memcpy(Xc, L->Xc.data(), L->Xc.size() * sizeof(double));
  std::memcpy(rowptr, L->rowptr.data(), L->rowptr.size() * sizeof(int64_t));
  std::memcpy(col, L->col.data(), L->col.size() * sizeof(int32_t));
}

// Sampled fine points (n_coarse) and the Voronoi cell of every fine point (n).
void gb_level_cells(void* h, int32_t* samples, int32_t* seed) {
  Level* L = (Level*)h;
  std::memcpy(samples, L->samples.data(), L->samples.size() * sizeof(int32_t));
  std::memcpy(seed, L->seed.data(), L->seed.size() * sizeof(int32_t));
}

void gb_level_free(void* h) { delete (Level*)h; }

}  // extern "C"
