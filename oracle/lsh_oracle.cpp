// CPU oracle for the LSH index mode -- TEST INFRASTRUCTURE ONLY.
//
// Same status as scan_oracle.cpp: loaded only by the tests, the smoke check and
// the benchmark's CPU-baseline leg; no code shared with the CUDA library.
//
// What it computes (Sections 2.1.2, 5 and 6.3 of the paper):
//  * Selection (Section 6.3 heuristic): with degree threshold T, an edge is
//    approximated iff both endpoints have degree > T; a vertex is sketched iff
//    its degree is > T and it has a neighbour of degree > T. row[v] numbers the
//    sketched vertices in ascending id order (-1 = not sketched).
//  * SimHash (Charikar; Section 2.1.2): k hyperplanes. For a sketched v,
//    s_j(v) = sum over x in N̄(v) of rho_j(x), and bit j of the sketch is
//    [s_j(v) >= 0]. The paper draws Gaussian coordinates; here rho_j(x) is a
//    Rademacher sign: +1 iff bit (j mod 64) of R(key_s, x*1024 + j/64) is set,
//    where R(key, c) is output number c of SplitMix64 started at state key
//    (Steele, Lea, Flood 2014) and key_s = mix(seed ^ 0x53494D48). Sums are
//    FP32; they are integers of magnitude <= d+1 < 2^24, so exact.
//    Estimate: h = Hamming distance of the two k-bit sketches, theta = pi h / k,
//    sigma~ = max(0, cos(theta)) (the clamp keeps the estimate inside the range
//    of the exact measure).
//  * Weighted SimHash: the same hyperplanes applied to the weighted closed
//    neighbourhood (w(v,v) = 1), double-precision sums in a fixed order.
//  * k-partition MinHash (one-permutation hashing, Li, Owen, Zhang 2012;
//    Section 6.3): k a power of two, L = log2 k, h(x) = low 32 bits of
//    R(key_m, x), key_m = mix(seed ^ 0x4D494E48). Bin = top L bits of h(x),
//    value = the remaining 32-L bits; sketch[b] = min value in bin b over
//    N̄(v), 0xFFFFFFFF when the bin is empty. Estimate: equal non-empty bins
//    divided by (k - bins empty in both).
//  * Standard MinHash (Section 2.1.2): k independent hashes h_j(x) = low 32 bits
//    of R(key_m ^ ((j+1) * 0x9E3779B97F4A7C15), x); sketch[j] = min over N̄(v);
//    estimate = equal coordinates / k.
//  * Approximate index (Section 5): approximated arcs take the estimate, every
//    other arc keeps its exact similarity; the orders are then built as usual.
#include <cmath>
#include <cstdint>
#include <vector>

namespace {

constexpr uint64_t GAMMA = 0x9E3779B97F4A7C15ULL;

uint64_t mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Output number c (0-based) of SplitMix64 whose state starts at key.
uint64_t R(uint64_t key, uint64_t c) { return mix(key + (c + 1) * GAMMA); }

uint64_t simhash_key(uint64_t seed) { return mix(seed ^ 0x53494D48ULL); }  // "SIMH"
uint64_t minhash_key(uint64_t seed) { return mix(seed ^ 0x4D494E48ULL); }  // "MINH"

int log2_exact(int k) {
  int L = 0;
  while ((1 << L) < k) ++L;
  return (1 << L) == k ? L : -1;
}

int popcount64(uint64_t x) {
  int c = 0;
  while (x) { x &= x - 1; ++c; }
  return c;
}

}  // namespace

extern "C" {

uint64_t orc_splitmix64(uint64_t key, uint64_t c) { return R(key, c); }

int64_t orc_lsh_select(int64_t n, const int64_t* off, const int32_t* adj, int64_t T, int32_t* row) {
  int64_t h = 0;
  for (int64_t v = 0; v < n; ++v) {
    row[v] = -1;
    if (off[v + 1] - off[v] <= T) continue;
    bool any = false;
    for (int64_t i = off[v]; i < off[v + 1]; ++i) {
      const int32_t u = adj[i];
      if (off[u + 1] - off[u] > T) { any = true; break; }
    }
    if (any) row[v] = (int32_t)h++;
  }
  return h;
}

// sig: nH rows of k/64 words; bit j of the sketch is bit (j % 64) of word j / 64.
int orc_simhash_sketch(int64_t n, const int64_t* off, const int32_t* adj, const int32_t* row,
                       int64_t nH, int k, uint64_t seed, uint64_t* sig) {
  if (k <= 0 || k % 64 != 0 || k > 65536) return -1;
  const uint64_t key = simhash_key(seed);
  const int W = k / 64;
  std::vector<float> s((size_t)k);
  for (int64_t v = 0; v < n; ++v) {
    if (row[v] < 0) continue;
    if (row[v] >= nH) return -1;
    for (int j = 0; j < k; ++j) s[j] = 0.0f;
    // N̄(v): v itself, then its neighbours
    for (int64_t i = off[v] - 1; i < off[v + 1]; ++i) {
      const int64_t x = i < off[v] ? v : adj[i];
      for (int j = 0; j < k; ++j) {
        const uint64_t bits = R(key, (uint64_t)x * 1024u + (uint64_t)(j / 64));
        const float rho = ((bits >> (j % 64)) & 1u) ? 1.0f : -1.0f;
        s[j] += rho;
      }
    }
    uint64_t* out = sig + (size_t)row[v] * W;
    for (int w = 0; w < W; ++w) out[w] = 0;
    for (int j = 0; j < k; ++j)
      if (s[j] >= 0.0f) out[j / 64] |= 1ULL << (j % 64);
  }
  return 0;
}

// SimHash of the weighted closed neighbourhood (Section 4.1.1 with w(v,v) = 1;
// the paper's LSH bound covers SimHash on weighted graphs, Section 5):
// s_j(v) = sum over x in N̄(v) of rho_j(x) w(v,x), bit j = [s_j(v) >= 0].
// rho_j(x) w(v,x) is +-w exactly; the sum is taken in double precision in the
// order v (weight 1), then N(v) in id order, so any implementation that adds
// the same terms in the same order takes every sign decision identically.
// w[i] is the weight of arc i.
int orc_simhash_sketch_weighted(int64_t n, const int64_t* off, const int32_t* adj,
                                const double* w, const int32_t* row, int64_t nH, int k,
                                uint64_t seed, uint64_t* sig) {
  if (k <= 0 || k % 64 != 0 || k > 65536) return -1;
  const uint64_t key = simhash_key(seed);
  const int W = k / 64;
  std::vector<double> s((size_t)k);
  for (int64_t v = 0; v < n; ++v) {
    if (row[v] < 0) continue;
    if (row[v] >= nH) return -1;
    for (int j = 0; j < k; ++j) s[j] = 0.0;
    for (int64_t i = off[v] - 1; i < off[v + 1]; ++i) {
      const int64_t x = i < off[v] ? v : adj[i];
      const double wx = i < off[v] ? 1.0 : w[i];
      for (int j = 0; j < k; ++j) {
        const uint64_t bits = R(key, (uint64_t)x * 1024u + (uint64_t)(j / 64));
        s[j] += ((bits >> (j % 64)) & 1u) ? wx : -wx;
      }
    }
    uint64_t* out = sig + (size_t)row[v] * W;
    for (int q = 0; q < W; ++q) out[q] = 0;
    for (int j = 0; j < k; ++j)
      if (s[j] >= 0.0) out[j / 64] |= 1ULL << (j % 64);
  }
  return 0;
}

// mh: nH rows of k uint32.
int orc_minhash_sketch(int64_t n, const int64_t* off, const int32_t* adj, const int32_t* row,
                       int64_t nH, int k, int kpartition, uint64_t seed, uint32_t* mh) {
  const int L = log2_exact(k);
  if (k <= 0 || k > 65536 || (kpartition && (L < 0 || L > 16))) return -1;
  const uint64_t key = minhash_key(seed);
  for (int64_t v = 0; v < n; ++v) {
    if (row[v] < 0) continue;
    if (row[v] >= nH) return -1;
    uint32_t* out = mh + (size_t)row[v] * k;
    for (int j = 0; j < k; ++j) out[j] = 0xFFFFFFFFu;
    for (int64_t i = off[v] - 1; i < off[v + 1]; ++i) {
      const int64_t x = i < off[v] ? v : adj[i];
      if (kpartition) {
        const uint32_t h = (uint32_t)R(key, (uint64_t)x);
        const uint32_t b = L == 0 ? 0u : h >> (32 - L);
        const uint32_t val = L == 0 ? h & 0x7FFFFFFFu : h & ((1u << (32 - L)) - 1u);
        if (val < out[b]) out[b] = val;
      } else {
        for (int j = 0; j < k; ++j) {
          const uint32_t h = (uint32_t)R(key ^ ((uint64_t)(j + 1) * GAMMA), (uint64_t)x);
          if (h < out[j]) out[j] = h;
        }
      }
    }
  }
  return 0;
}

// tab[h] = max(0, cos(pi * h / k)), h = 0..k.
int orc_simhash_table(int k, double* tab) {
  if (k <= 0) return -1;
  for (int h = 0; h <= k; ++h) {
    const double c = std::cos(M_PI * (double)h / (double)k);
    tab[h] = c > 0.0 ? c : 0.0;
  }
  return 0;
}

// scheme 0: SimHash (sketch = uint64 words), 1: MinHash (sketch = uint32).
// exact[] holds the exact similarity of every arc; approximated arcs are
// overwritten with the estimate in out[].
int orc_lsh_similarities(int scheme, int64_t n, const int64_t* off, const int32_t* adj,
                         const int32_t* row, const void* sketch, const double* exact, int k,
                         int kpartition, int unused, double* out) {
  (void)unused;
  std::vector<double> tab;
  if (scheme == 0) {
    if (k % 64 != 0) return -1;
    tab.resize((size_t)k + 1);
    orc_simhash_table(k, tab.data());
  }
  for (int64_t u = 0; u < n; ++u) {
    for (int64_t i = off[u]; i < off[u + 1]; ++i) {
      const int32_t v = adj[i];
      out[i] = exact[i];
      if (row[u] < 0 || row[v] < 0) continue;
      if (scheme == 0) {
        const uint64_t* a = (const uint64_t*)sketch + (size_t)row[u] * (k / 64);
        const uint64_t* b = (const uint64_t*)sketch + (size_t)row[v] * (k / 64);
        int h = 0;
        for (int w = 0; w < k / 64; ++w) h += popcount64(a[w] ^ b[w]);
        out[i] = tab[h];
      } else {
        const uint32_t* a = (const uint32_t*)sketch + (size_t)row[u] * k;
        const uint32_t* b = (const uint32_t*)sketch + (size_t)row[v] * k;
        int match = 0, both_empty = 0;
        for (int j = 0; j < k; ++j) {
          if (a[j] == 0xFFFFFFFFu && b[j] == 0xFFFFFFFFu) ++both_empty;
          else if (a[j] == b[j]) ++match;
        }
        const int denom = kpartition ? k - both_empty : k;
        out[i] = denom > 0 ? (double)match / (double)denom : 0.0;
      }
    }
  }
  return 0;
}

}  // extern "C"
