// CPU oracle for index-based SCAN -- TEST INFRASTRUCTURE ONLY.
//
// Only the tests, the package smoke check and the benchmark's CPU-baseline leg
// may load this library. It shares no code with the CUDA path and is written to
// be checked against the paper by eye: plain loops, double precision, a library
// sort where the paper sorts. Every entry point is single-threaded.
//
// Paper: Tseng, Dhulipala, Shun, "Parallel Index-Based Structural Graph
// Clustering and Its Approximation", SIGMOD 2021.
//
// Conventions (readings of the paper, each one listed in the design notes):
//  * Graphs are simple and undirected, CSR with int64 offsets and id-sorted
//    adjacency (Section 2.2). Vertex ids are 0-based (the paper uses [1, n]).
//  * N̄(v) = N(v) ∪ {v} and degree d_v = |N(v)| (Section 2.2).
//  * Cosine similarity of closed neighbourhoods, Section 3.1:
//      sigma(u,v) = |N̄(u) ∩ N̄(v)| / (sqrt|N̄(u)| sqrt|N̄(v)|),
//    evaluated as c / sqrt((d_u+1)(d_v+1)) with ONE square root of the exact
//    integer product and one division, both IEEE round-to-nearest.
//    Jaccard (Section 2.1.1): c / |N̄(u) ∪ N̄(v)| = c / (d_u + 1 + d_v + 1 - c).
//  * Neighbour order NO[v] (Section 3.2; Algorithm 2): N(v) sorted by
//    non-increasing similarity; v itself is implicit at closed rank 1 (it has
//    similarity 1, the maximum); equal similarities keep ascending id.
//  * Core order CO[mu], mu = 2..maxdeg+1 (Section 3.2; Algorithm 2): vertices
//    with |N̄(v)| >= mu, sorted by non-increasing core threshold
//    sigma(v, NO[v][mu]) -- the mu-th largest similarity over N̄(v) counting
//    v itself first, i.e. open rank mu-2 (0-based); equal thresholds keep
//    ascending id.
//  * Query (mu, eps), Section 3.1 definitions: eps-similar means sigma >= eps;
//    core iff |N_eps(v)| >= mu where N_eps(v) includes v. Clusters are the
//    connected components of cores under eps-similar core-core edges; a
//    non-core eps-similar to some core is a border and joins the cluster of
//    the MOST similar such core, smallest id on ties (Section 7.3.4's
//    deterministic rule). Cluster label = smallest core id in the cluster.
//    Unclustered vertices are -1; with the hub flag, an unclustered vertex
//    whose neighbours (any edge) carry >= 2 distinct cluster labels is a hub
//    (-2), else an outlier (-1) (Section 4.3).
//  * mu > maxdeg+1 means no cores (Algorithm 3).
//  * Weighted cosine (Section 4.1.1, WeightedCosineSim of Section 2.1.1):
//    sum over N̄(u) ∩ N̄(v) of w(u,x) w(v,x), divided by the two norms
//    sqrt(sum over N̄ of w^2), with w(x,x) = 1; terms added in id order.
//  * Modularity (Section 7.2), unclustered vertices as singletons.
// No entry point is unpinned: each has pins in the tests.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <utility>
#include <vector>

namespace {

constexpr int COSINE = 0;
constexpr int JACCARD = 1;
constexpr int FLAG_HUBS = 1;

inline int64_t deg_of(const int64_t* off, int64_t v) { return off[v + 1] - off[v]; }

// Closed neighbourhood N̄(v) = N(v) ∪ {v}, ascending.
std::vector<int32_t> closed_list(const int64_t* off, const int32_t* adj, int32_t v) {
  std::vector<int32_t> s(adj + off[v], adj + off[v + 1]);
  s.insert(std::lower_bound(s.begin(), s.end(), v), v);
  return s;
}

// |A ∩ B| of two ascending lists by a two-pointer merge.
int64_t merge_count(const std::vector<int32_t>& a, const std::vector<int32_t>& b) {
  size_t i = 0, j = 0;
  int64_t c = 0;
  while (i < a.size() && j < b.size()) {
    if (a[i] < b[j]) ++i;
    else if (a[i] > b[j]) ++j;
    else { ++c; ++i; ++j; }
  }
  return c;
}

// Section 3.1 / Section 2.1.1 similarity from the count and the two degrees.
double similarity(int kind, int64_t c, int64_t du, int64_t dv) {
  if (kind == COSINE) {
    const int64_t prod = (du + 1) * (dv + 1);
    return (double)c / std::sqrt((double)prod);
  }
  return (double)c / (double)(du + 1 + dv + 1 - c);
}

// Sequential union-find whose root is always the smallest member.
struct MinDSU {
  std::vector<int32_t> p;
  explicit MinDSU(int64_t n) : p((size_t)n) { for (int64_t i = 0; i < n; ++i) p[i] = (int32_t)i; }
  int32_t find(int32_t x) {
    while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
    return x;
  }
  void unite(int32_t a, int32_t b) {
    a = find(a); b = find(b);
    if (a == b) return;
    if (a < b) p[b] = a; else p[a] = b;
  }
};

// Section 4.3: an unclustered vertex is a hub iff its neighbours carry at least
// two distinct cluster labels; labels[] holds final cluster labels (>= 0) or -1.
void mark_hubs(int64_t n, const int64_t* off, const int32_t* adj, int32_t* labels) {
  std::vector<int32_t> out(labels, labels + n);
  for (int64_t v = 0; v < n; ++v) {
    if (labels[v] >= 0) continue;
    int32_t first = -1;
    bool hub = false;
    for (int64_t i = off[v]; i < off[v + 1]; ++i) {
      int32_t l = labels[adj[i]];
      if (l < 0) continue;
      if (first < 0) first = l;
      else if (l != first) { hub = true; break; }
    }
    out[v] = hub ? -2 : -1;
  }
  std::memcpy(labels, out.data(), (size_t)n * sizeof(int32_t));
}

}  // namespace

extern "C" {

int orc_version() { return 1; }

// |N̄(u) ∩ N̄(v)| for every arc u->v (definition of sigma, Section 3.1).
// Each undirected edge is counted once, from its endpoint u with the larger
// (degree, id): N̄(u) is marked in a flag array and the members of N̄(v) that
// carry a flag are counted. The value is written to both arcs of the edge.
int orc_closed_counts(int64_t n, const int64_t* off, const int32_t* adj, int32_t* cnt) {
  std::vector<char> mark((size_t)n, 0);
  for (int64_t u = 0; u < n; ++u) {
    const std::vector<int32_t> cu = closed_list(off, adj, (int32_t)u);
    for (int32_t x : cu) mark[x] = 1;
    for (int64_t i = off[u]; i < off[u + 1]; ++i) {
      const int32_t v = adj[i];
      const int64_t du = deg_of(off, u), dv = deg_of(off, v);
      if (dv > du || (dv == du && v > u)) continue;  // counted from v
      int64_t c = mark[v];  // v itself is in N̄(v)
      for (int64_t j = off[v]; j < off[v + 1]; ++j) c += mark[adj[j]];
      cnt[i] = (int32_t)c;
      const int32_t* b = adj + off[v];
      const int32_t* e = adj + off[v + 1];
      const int32_t* t = std::lower_bound(b, e, (int32_t)u);
      if (t == e || *t != u) return -3;  // asymmetric adjacency
      cnt[off[v] + (t - b)] = (int32_t)c;
    }
    for (int32_t x : cu) mark[x] = 0;
  }
  return 0;
}

// Counts for an explicit list of adjacent or non-adjacent pairs (sampled checks).
int orc_count_pairs(int64_t n, const int64_t* off, const int32_t* adj, int64_t k,
                    const int32_t* us, const int32_t* vs, int32_t* out) {
  for (int64_t i = 0; i < k; ++i) {
    if (us[i] < 0 || us[i] >= n || vs[i] < 0 || vs[i] >= n) return -1;
    out[i] = (int32_t)merge_count(closed_list(off, adj, us[i]), closed_list(off, adj, vs[i]));
  }
  return 0;
}

// sigma for every arc from its closed count (cosine: Section 3.1; Jaccard: Section 2.1.1).
int orc_similarities(int kind, int64_t n, const int64_t* off, const int32_t* adj,
                     const int32_t* cnt, double* sim) {
  if (kind != COSINE && kind != JACCARD) return -1;
  for (int64_t u = 0; u < n; ++u)
    for (int64_t i = off[u]; i < off[u + 1]; ++i)
      sim[i] = similarity(kind, cnt[i], deg_of(off, u), deg_of(off, adj[i]));
  return 0;
}

// NO: each N(v) stably sorted by non-increasing sigma (Algorithm 2, MakeNeighborOrder).
int orc_neighbor_order(int64_t n, const int64_t* off, const int32_t* adj, const double* sim,
                       int32_t* no_id, double* no_sim) {
  std::vector<std::pair<double, int32_t>> row;
  for (int64_t v = 0; v < n; ++v) {
    row.clear();
    for (int64_t i = off[v]; i < off[v + 1]; ++i) row.emplace_back(sim[i], adj[i]);
    std::stable_sort(row.begin(), row.end(),
                     [](const std::pair<double, int32_t>& a, const std::pair<double, int32_t>& b) {
                       return a.first > b.first;
                     });
    for (size_t j = 0; j < row.size(); ++j) {
      no_id[off[v] + (int64_t)j] = row[j].second;
      no_sim[off[v] + (int64_t)j] = row[j].first;
    }
  }
  return 0;
}

// CO (Algorithm 2, MakeCoreOrder). co_off has maxdeg+1 entries:
// CO[mu] = co_id[co_off[mu-2] .. co_off[mu-1]), mu = 2..maxdeg+1.
// The members of CO[mu] are the vertices with d_v + 1 >= mu. They are kept in
// one ascending-id list that loses the vertices with d_v + 1 < mu as mu grows,
// so building every CO[mu] reads each member once (sum over mu of |CO[mu]| =
// the number of arcs) instead of scanning all n vertices for every mu.
int orc_core_order(int64_t n, const int64_t* off, const double* no_sim, int64_t maxdeg,
                   int64_t* co_off, int32_t* co_id, double* co_thr) {
  std::vector<std::pair<double, int32_t>> row;
  std::vector<int32_t> members;  // {v : d_v + 1 >= mu}, ascending id
  for (int64_t v = 0; v < n; ++v) members.push_back((int32_t)v);
  int64_t w = 0;
  co_off[0] = 0;
  for (int64_t mu = 2; mu <= maxdeg + 1; ++mu) {
    members.erase(std::remove_if(members.begin(), members.end(),
                                 [&](int32_t v) { return deg_of(off, v) + 1 < mu; }),
                  members.end());
    row.clear();
    for (int32_t v : members) row.emplace_back(no_sim[off[v] + mu - 2], v);
    std::stable_sort(row.begin(), row.end(),
                     [](const std::pair<double, int32_t>& a, const std::pair<double, int32_t>& b) {
                       return a.first > b.first;
                     });
    for (const auto& e : row) { co_id[w] = e.second; co_thr[w] = e.first; ++w; }
    co_off[mu - 1] = w;
  }
  return 0;
}

// Query from the index, the steps of Algorithms 3, 5 and 4 in order, run
// sequentially: GetCores (prefix of CO[mu] with threshold >= eps), the
// eps-prefix of NO[u] for each core, union of core-core eps-edges, then
// borders (first core in the eps-prefix of NO[v] = most similar, smallest id).
int orc_query_index(int64_t n, const int64_t* off, const int32_t* adj, const int32_t* no_id,
                    const double* no_sim, int64_t maxdeg, const int64_t* co_off,
                    const int32_t* co_id, const double* co_thr, int mu, double eps, int flags,
                    int32_t* labels) {
  if (mu < 2 || !(eps >= 0.0 && eps <= 1.0)) return -1;
  for (int64_t v = 0; v < n; ++v) labels[v] = -1;
  std::vector<char> core((size_t)n, 0);
  if (mu <= maxdeg + 1) {
    // Algorithm 3: cores are the prefix of CO[mu] whose threshold is >= eps
    for (int64_t i = co_off[mu - 2]; i < co_off[mu - 1] && co_thr[i] >= eps; ++i) core[co_id[i]] = 1;
  }
  MinDSU dsu(n);
  for (int64_t u = 0; u < n; ++u) {
    if (!core[u]) continue;
    for (int64_t i = off[u]; i < off[u + 1] && no_sim[i] >= eps; ++i)
      if (core[no_id[i]]) dsu.unite((int32_t)u, no_id[i]);
  }
  for (int64_t u = 0; u < n; ++u)
    if (core[u]) labels[u] = dsu.find((int32_t)u);
  for (int64_t v = 0; v < n; ++v) {
    if (core[v]) continue;
    for (int64_t i = off[v]; i < off[v + 1] && no_sim[i] >= eps; ++i)
      if (core[no_id[i]]) { labels[v] = dsu.find(no_id[i]); break; }
  }
  (void)adj;
  if (flags & FLAG_HUBS) mark_hubs(n, off, adj, labels);
  return 0;
}

// Query from the definitions only (Section 3.1), ignoring any index: count
// each vertex's eps-neighbourhood (itself included), breadth-first search over
// cores through eps-similar edges, label by the smallest core id, then attach
// each non-core to its most similar eps-similar core (smallest id on ties).
int orc_query_definition(int64_t n, const int64_t* off, const int32_t* adj, const double* sim,
                         int mu, double eps, int flags, int32_t* labels) {
  if (mu < 2 || !(eps >= 0.0 && eps <= 1.0)) return -1;
  std::vector<char> core((size_t)n, 0);
  for (int64_t v = 0; v < n; ++v) {
    int64_t ne = 1;  // v itself: sigma(v,v) = 1 >= eps
    for (int64_t i = off[v]; i < off[v + 1]; ++i) ne += sim[i] >= eps;
    core[v] = ne >= mu;
  }
  std::vector<int32_t> comp((size_t)n, -1);
  for (int64_t s = 0; s < n; ++s) {
    if (!core[s] || comp[s] >= 0) continue;
    // s is the smallest id of its (not yet seen) component: ids are visited in order
    std::deque<int32_t> q{(int32_t)s};
    comp[s] = (int32_t)s;
    while (!q.empty()) {
      int32_t x = q.front();
      q.pop_front();
      for (int64_t i = off[x]; i < off[x + 1]; ++i) {
        int32_t y = adj[i];
        if (core[y] && comp[y] < 0 && sim[i] >= eps) { comp[y] = (int32_t)s; q.push_back(y); }
      }
    }
  }
  for (int64_t v = 0; v < n; ++v) {
    if (core[v]) { labels[v] = comp[v]; continue; }
    int32_t best = -1;
    double bs = -1.0;
    for (int64_t i = off[v]; i < off[v + 1]; ++i) {
      const int32_t x = adj[i];
      if (!core[x] || sim[i] < eps) continue;
      if (sim[i] > bs || (sim[i] == bs && x < best)) { bs = sim[i]; best = x; }
    }
    labels[v] = best >= 0 ? comp[best] : -1;
  }
  if (flags & FLAG_HUBS) mark_hubs(n, off, adj, labels);
  return 0;
}

// Weighted cosine similarity of every arc (Section 4.1.1: WeightedCosineSim, Section 2.1.1, of
// the closed neighbourhoods with w(x, x) = 1 for every vertex x):
//   sigma(u,v) = sum_{x in N̄(u) ∩ N̄(v)} w(u,x) w(v,x)
//                / ( sqrt(sum_{x in N̄(u)} w(u,x)^2) * sqrt(sum_{x in N̄(v)} w(v,x)^2) ).
// w[i] is the weight of arc i (w(u, adj[i]) for i in u's row); the graph's
// weights must be symmetric. The numerator walks the two closed lists (each
// in id order, the vertex itself with weight 1) with two pointers; the
// norms and the final division are plain double arithmetic.
int orc_weighted_similarities(int64_t n, const int64_t* off, const int32_t* adj, const double* w,
                              double* sim) {
  // closed list of x with weights, in id order
  auto closed_w = [&](int64_t x, std::vector<int32_t>& ids, std::vector<double>& ws) {
    ids.clear();
    ws.clear();
    bool self_done = false;
    for (int64_t i = off[x]; i < off[x + 1]; ++i) {
      if (!self_done && adj[i] > x) {
        ids.push_back((int32_t)x);
        ws.push_back(1.0);
        self_done = true;
      }
      ids.push_back(adj[i]);
      ws.push_back(w[i]);
    }
    if (!self_done) {
      ids.push_back((int32_t)x);
      ws.push_back(1.0);
    }
  };
  std::vector<double> norm((size_t)n);
  std::vector<int32_t> ia, ib;
  std::vector<double> wa, wb;
  for (int64_t x = 0; x < n; ++x) {
    closed_w(x, ia, wa);
    double s2 = 0.0;
    for (double y : wa) s2 += y * y;
    norm[x] = std::sqrt(s2);
  }
  for (int64_t u = 0; u < n; ++u) {
    closed_w(u, ia, wa);
    for (int64_t i = off[u]; i < off[u + 1]; ++i) {
      const int64_t v = adj[i];
      closed_w(v, ib, wb);
      double num = 0.0;
      size_t a = 0, b = 0;
      while (a < ia.size() && b < ib.size()) {
        if (ia[a] < ib[b]) ++a;
        else if (ia[a] > ib[b]) ++b;
        else { num += wa[a] * wb[b]; ++a; ++b; }
      }
      sim[i] = num / (norm[u] * norm[v]);
    }
  }
  return 0;
}

// Weighted cosine similarities of the arcs of one vertex v (sampled checks on
// graphs too large for the all-arcs routine): out[j] = sigma(v, adj[off[v]+j])
// by the same definition (Section 4.1.1). w(v, .) is spread over a dense
// vector; each neighbour u's closed list is walked in id order, so the terms
// of a numerator are added in the same order as by the two-pointer walk of
// orc_weighted_similarities and the results are the same doubles.
int orc_weighted_vertex_similarities(int64_t n, const int64_t* off, const int32_t* adj,
                                     const double* w, int32_t v, double* out) {
  if (v < 0 || v >= n) return -1;
  std::vector<double> wv((size_t)n, 0.0);
  std::vector<char> in_v((size_t)n, 0);
  wv[v] = 1.0;
  in_v[v] = 1;
  for (int64_t i = off[v]; i < off[v + 1]; ++i) {
    wv[adj[i]] = w[i];
    in_v[adj[i]] = 1;
  }
  // sqrt of the sum of squares over the closed list of x, in id order
  auto norm_of = [&](int64_t x) {
    double s2 = 0.0;
    bool self_done = false;
    for (int64_t i = off[x]; i < off[x + 1]; ++i) {
      if (!self_done && adj[i] > x) {
        s2 += 1.0;
        self_done = true;
      }
      s2 += w[i] * w[i];
    }
    if (!self_done) s2 += 1.0;
    return std::sqrt(s2);
  };
  const double norm_v = norm_of(v);
  for (int64_t j = off[v]; j < off[v + 1]; ++j) {
    const int64_t u = adj[j];
    double num = 0.0;
    bool self_done = false;
    for (int64_t i = off[u]; i < off[u + 1]; ++i) {
      const int64_t x = adj[i];
      if (!self_done && x > u) {
        if (in_v[u]) num += 1.0 * wv[u];  // x = u, w(u,u) = 1
        self_done = true;
      }
      if (in_v[x]) num += w[i] * wv[x];
    }
    if (!self_done && in_v[u]) num += 1.0 * wv[u];
    out[j - off[v]] = num / (norm_of(u) * norm_v);
  }
  return 0;
}

// Similarities of all arcs of one vertex v (sampled checks on large graphs):
// out[j] = sigma(v, adj[off[v]+j]), counting members of each N̄(u) among the
// flagged N̄(v).
int orc_vertex_similarities(int kind, int64_t n, const int64_t* off, const int32_t* adj,
                            int32_t v, double* out) {
  if (v < 0 || v >= n) return -1;
  std::vector<char> mark((size_t)n, 0);
  for (int32_t x : closed_list(off, adj, v)) mark[x] = 1;
  for (int64_t i = off[v]; i < off[v + 1]; ++i) {
    const int32_t u = adj[i];
    int64_t c = mark[u];
    for (int64_t j = off[u]; j < off[u + 1]; ++j) c += mark[adj[j]];
    out[i - off[v]] = similarity(kind, c, deg_of(off, v), deg_of(off, u));
  }
  return 0;
}

// Adjusted Rand index (Section 7.2, Hubert and Arabie) of two labelings of n
// vertices; every negative label is its own singleton cluster.
double orc_ari(int64_t n, const int32_t* a, const int32_t* b) {
  auto key = [](int32_t l, int64_t v) -> int64_t { return l >= 0 ? (int64_t)l : -1 - v; };
  std::map<std::pair<int64_t, int64_t>, int64_t> nij;
  std::map<int64_t, int64_t> ni, nj;
  for (int64_t v = 0; v < n; ++v) {
    int64_t x = key(a[v], v), y = key(b[v], v);
    nij[{x, y}]++;
    ni[x]++;
    nj[y]++;
  }
  auto c2 = [](int64_t k) { return (double)k * (double)(k - 1) / 2.0; };
  double sij = 0, si = 0, sj = 0;
  for (const auto& e : nij) sij += c2(e.second);
  for (const auto& e : ni) si += c2(e.second);
  for (const auto& e : nj) sj += c2(e.second);
  const double expected = si * sj / c2(n);
  const double maxi = (si + sj) / 2.0;
  if (maxi == expected) return 1.0;  // both partitions trivial and identical in shape
  return (sij - expected) / (maxi - expected);
}

// Modularity (Section 7.2, Newman): (1/2m) sum_{u,v} (A_uv - d_u d_v / 2m) delta_uv,
// unclustered (negative-label) vertices each a singleton cluster.
double orc_modularity(int64_t n, const int64_t* off, const int32_t* adj, const int32_t* labels) {
  const double two_m = (double)off[n];
  if (two_m == 0) return 0.0;
  auto key = [&](int64_t v) -> int64_t { return labels[v] >= 0 ? (int64_t)labels[v] : -1 - v; };
  double inside = 0;
  std::map<int64_t, double> degsum;
  for (int64_t u = 0; u < n; ++u) {
    degsum[key(u)] += (double)deg_of(off, u);
    for (int64_t i = off[u]; i < off[u + 1]; ++i) inside += key(u) == key(adj[i]);
  }
  double expect = 0;
  for (const auto& e : degsum) expect += e.second * e.second;
  return inside / two_m - expect / (two_m * two_m);
}

}  // extern "C"
