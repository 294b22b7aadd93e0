/*
 * graphgen.c -- seeded synthetic graph generators shared by the tests, the
 * benchmark and the oracle's test harness.
 *
 * This file holds no part of the subgraph-census arithmetic: it only draws
 * random graphs and normalises edge lists into a simple undirected CSR
 * (direction ignored, duplicates and self-loops dropped, neighbour lists
 * sorted by id), the input convention of the paper's experiments (Sec. 8).
 *
 * Every random number comes from a counter-based stream built on splitmix64
 * (Steele, Lea, Flood 2014), keyed by (seed, stream, counter), and all draws
 * are turned into decisions with integer arithmetic only, so a given call
 * produces the same graph on every platform.  The Chung-Lu weights are the
 * one place that uses floating point (pow); they are quantised to integers
 * before any sampling.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct {
  int64_t n;
  int64_t nnz;       /* = 2 * undirected edges */
  int64_t* row_ptr;  /* n + 1 */
  int32_t* col;      /* nnz, sorted within each row */
} gg_graph;

static uint64_t sm64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

/* Counter-based draw: stream key mixes (seed, stream); the counter indexes it. */
static uint64_t gg_key(uint64_t seed, uint64_t stream) {
  return sm64(sm64(seed) ^ (stream * 0xD1B54A32D192ED03ull));
}
static uint64_t gg_draw(uint64_t key, uint64_t ctr) {
  return sm64(key + ctr * 0x9E3779B97F4A7C15ull);
}
/* Uniform integer in [0, bound) by the 128-bit multiply-high reduction. */
static uint64_t gg_below(uint64_t r, uint64_t bound) {
  return (uint64_t)(((unsigned __int128)r * bound) >> 64);
}

uint64_t gg_splitmix64(uint64_t x) { return sm64(x); }
uint64_t gg_stream_draw(uint64_t seed, uint64_t stream, uint64_t ctr) {
  return gg_draw(gg_key(seed, stream), ctr);
}

/* ---------- LSD radix sort of 64-bit keys (11-bit digits) ---------- */
static int radix_sort_u64(uint64_t* keys, int64_t cnt, int key_bits) {
  if (cnt <= 1) return 0;
  uint64_t* tmp = (uint64_t*)malloc((size_t)cnt * sizeof(uint64_t));
  if (!tmp) return -1;
  const int B = 11, R = 1 << B;
  int64_t* hist = (int64_t*)malloc(sizeof(int64_t) * R);
  if (!hist) { free(tmp); return -1; }
  uint64_t* src = keys; uint64_t* dst = tmp;
  for (int shift = 0; shift < key_bits; shift += B) {
    memset(hist, 0, sizeof(int64_t) * R);
    for (int64_t i = 0; i < cnt; ++i) hist[(src[i] >> shift) & (R - 1)]++;
    int64_t s = 0;
    for (int d = 0; d < R; ++d) { int64_t c = hist[d]; hist[d] = s; s += c; }
    for (int64_t i = 0; i < cnt; ++i) dst[hist[(src[i] >> shift) & (R - 1)]++] = src[i];
    uint64_t* t = src; src = dst; dst = t;
  }
  if (src != keys) memcpy(keys, src, (size_t)cnt * sizeof(uint64_t));
  free(hist); free(tmp);
  return 0;
}

static int bits_for(int64_t n) { int b = 1; while (b < 62 && ((int64_t)1 << b) < n) ++b; return b; }

/* Build a simple symmetric CSR from `cnt` (u, v) pairs packed as u<<32|v,
 * already containing both directions.  Sorts, drops duplicates/self-loops. */
static gg_graph* csr_from_keys(int64_t n, uint64_t* keys, int64_t cnt) {
  int vb = bits_for(n);
  /* repack into a dense key u*2^vb + v for a shorter sort */
  for (int64_t i = 0; i < cnt; ++i) {
    uint64_t u = keys[i] >> 32, v = keys[i] & 0xffffffffull;
    keys[i] = (u << vb) | v;
  }
  if (radix_sort_u64(keys, cnt, 2 * vb) != 0) return NULL;
  gg_graph* g = (gg_graph*)calloc(1, sizeof(gg_graph));
  if (!g) return NULL;
  g->n = n;
  g->row_ptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t w = 0;
  uint64_t mask = (vb >= 64) ? ~0ull : ((1ull << vb) - 1);
  for (int64_t i = 0; i < cnt; ++i) {
    uint64_t u = keys[i] >> vb, v = keys[i] & mask;
    if (u == v) continue;
    if (w > 0 && keys[w - 1] == keys[i]) continue;
    keys[w++] = keys[i];
  }
  g->nnz = w;
  g->col = (int32_t*)malloc((size_t)(w > 0 ? w : 1) * sizeof(int32_t));
  if (!g->row_ptr || !g->col) return NULL;
  for (int64_t i = 0; i < w; ++i) {
    uint64_t u = keys[i] >> vb;
    g->col[i] = (int32_t)(keys[i] & mask);
    g->row_ptr[u + 1]++;
  }
  for (int64_t u = 0; u < n; ++u) g->row_ptr[u + 1] += g->row_ptr[u];
  return g;
}

/* Both directions of each input pair, optionally relabelled by perm. */
static gg_graph* csr_from_pairs(int64_t n, const int64_t* src, const int64_t* dst,
                                int64_t cnt, const int64_t* perm) {
  uint64_t* keys = (uint64_t*)malloc((size_t)(2 * cnt > 0 ? 2 * cnt : 1) * sizeof(uint64_t));
  if (!keys) return NULL;
  for (int64_t i = 0; i < cnt; ++i) {
    uint64_t u = (uint64_t)(perm ? perm[src[i]] : src[i]);
    uint64_t v = (uint64_t)(perm ? perm[dst[i]] : dst[i]);
    keys[2 * i] = (u << 32) | v;
    keys[2 * i + 1] = (v << 32) | u;
  }
  gg_graph* g = csr_from_keys(n, keys, 2 * cnt);
  free(keys);
  return g;
}

/* Seeded Fisher-Yates permutation of 0..n-1. */
static int64_t* random_perm(int64_t n, uint64_t seed) {
  int64_t* p = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  if (!p) return NULL;
  for (int64_t i = 0; i < n; ++i) p[i] = i;
  uint64_t key = gg_key(seed, 0x5045524dull /* "PERM" */);
  for (int64_t i = n - 1; i > 0; --i) {
    int64_t j = (int64_t)gg_below(gg_draw(key, (uint64_t)i), (uint64_t)i + 1);
    int64_t t = p[i]; p[i] = p[j]; p[j] = t;
  }
  return p;
}

/* ---------------------------- public API ---------------------------- */

gg_graph* gg_from_edges(int64_t n, int64_t cnt, const int64_t* src, const int64_t* dst) {
  for (int64_t i = 0; i < cnt; ++i)
    if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) return NULL;
  return csr_from_pairs(n, src, dst, cnt, NULL);
}

/* Erdos-Renyi G(n, p): one Bernoulli draw per unordered pair {i<j}; the edge
 * exists iff the pair's 64-bit draw is below `threshold` = p * 2^64. */
gg_graph* gg_erdos_renyi(int64_t n, uint64_t threshold, uint64_t seed) {
  uint64_t key = gg_key(seed, 0x4552ull /* "ER" */);
  int64_t cap = 1024, cnt = 0;
  int64_t* s = (int64_t*)malloc(sizeof(int64_t) * cap);
  int64_t* d = (int64_t*)malloc(sizeof(int64_t) * cap);
  uint64_t ctr = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j, ++ctr) {
      if (gg_draw(key, ctr) < threshold) {
        if (cnt == cap) {
          cap *= 2;
          s = (int64_t*)realloc(s, sizeof(int64_t) * cap);
          d = (int64_t*)realloc(d, sizeof(int64_t) * cap);
        }
        s[cnt] = i; d[cnt] = j; ++cnt;
      }
    }
  gg_graph* g = csr_from_pairs(n, s, d, cnt, NULL);
  free(s); free(d);
  return g;
}

/* Chung-Lu by edge sampling: weights w_i ~ (i+1)^(-1/(gamma-1)), rescaled to
 * mean `mean_deg` after clipping at `max_deg`; round(sum(w)/2) edges, both endpoints
 * drawn proportionally to w; ids relabelled by a seeded permutation. */
gg_graph* gg_chung_lu(int64_t n, double gamma, double mean_deg, double max_deg, uint64_t seed) {
  if (n <= 1) return csr_from_pairs(n > 0 ? n : 0, NULL, NULL, 0, NULL);
  double* w = (double*)malloc(sizeof(double) * n);
  double alpha = 1.0 / (gamma - 1.0), sum = 0.0;
  for (int64_t i = 0; i < n; ++i) { w[i] = pow((double)(i + 1), -alpha); sum += w[i]; }
  /* rescale to the target mean and clip, repeated so that the clipped
   * weights keep the target mean */
  for (int it = 0; it < 16; ++it) {
    double scale = mean_deg * (double)n / sum;
    sum = 0.0;
    for (int64_t i = 0; i < n; ++i) { w[i] *= scale; if (w[i] > max_deg) w[i] = max_deg; sum += w[i]; }
  }
  /* integer weights (2^20 fixed point) and their prefix sums */
  uint64_t* cum = (uint64_t*)malloc(sizeof(uint64_t) * n);
  uint64_t tot = 0;
  for (int64_t i = 0; i < n; ++i) { tot += (uint64_t)(w[i] * 1048576.0); cum[i] = tot; }
  int64_t m = (int64_t)(sum / 2.0 + 0.5);
  free(w);
  int64_t* s = (int64_t*)malloc(sizeof(int64_t) * (m > 0 ? m : 1));
  int64_t* d = (int64_t*)malloc(sizeof(int64_t) * (m > 0 ? m : 1));
  uint64_t key = gg_key(seed, 0x434cull /* "CL" */);
  for (int64_t e = 0; e < m; ++e) {
    for (int side = 0; side < 2; ++side) {
      uint64_t r = gg_below(gg_draw(key, 2 * (uint64_t)e + side), tot);
      int64_t lo = 0, hi = n - 1;           /* first index with cum > r */
      while (lo < hi) { int64_t mid = (lo + hi) >> 1; if (cum[mid] > r) hi = mid; else lo = mid + 1; }
      if (side == 0) s[e] = lo; else d[e] = lo;
    }
  }
  free(cum);
  int64_t* perm = random_perm(n, seed);
  gg_graph* g = csr_from_pairs(n, s, d, m, perm);
  free(s); free(d); free(perm);
  return g;
}

/* R-MAT (Chakrabarti, Zhan, Faloutsos 2004): 2^scale vertices, edge_factor *
 * 2^scale samples; each of the `scale` levels picks a quadrant with
 * probabilities (a, b, c, 1-a-b-c) quantised to 1/65536; Graph500-style seeded
 * vertex permutation; symmetrised, deduplicated, self-loops dropped. */
gg_graph* gg_rmat(int scale, int64_t edge_factor, double a, double b, double c, uint64_t seed) {
  int64_t n = (int64_t)1 << scale;
  int64_t m = edge_factor * n;
  uint32_t ta = (uint32_t)(a * 65536.0 + 0.5);
  uint32_t tb = (uint32_t)((a + b) * 65536.0 + 0.5);
  uint32_t tc = (uint32_t)((a + b + c) * 65536.0 + 0.5);
  int64_t* perm = random_perm(n, seed);
  uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * 2 * (m > 0 ? m : 1));
  if (!perm || !keys) return NULL;
  uint64_t key = gg_key(seed, 0x524d4154ull /* "RMAT" */);
  int words = (scale + 3) / 4;
  for (int64_t e = 0; e < m; ++e) {
    uint64_t u = 0, v = 0;
    for (int wi = 0; wi < words; ++wi) {
      uint64_t r = gg_draw(key, (uint64_t)e * (uint64_t)words + (uint64_t)wi);
      for (int k = 0; k < 4 && wi * 4 + k < scale; ++k) {
        uint32_t q = (uint32_t)(r >> (16 * k)) & 0xffffu;
        uint64_t bu = (q >= tb), bv = (q >= ta && q < tb) || (q >= tc);
        u = (u << 1) | bu; v = (v << 1) | bv;
      }
    }
    u = (uint64_t)perm[u]; v = (uint64_t)perm[v];
    keys[2 * e] = (u << 32) | v;
    keys[2 * e + 1] = (v << 32) | u;
  }
  free(perm);
  gg_graph* g = csr_from_keys(n, keys, 2 * m);
  free(keys);
  return g;
}

/* Barabasi-Albert: seed clique on m_attach+1 vertices, then each new vertex
 * attaches to m_attach distinct targets drawn uniformly from the endpoint
 * multiset (probability proportional to degree). */
gg_graph* gg_barabasi_albert(int64_t n, int64_t m_attach, uint64_t seed) {
  if (m_attach < 1) m_attach = 1;
  int64_t n0 = m_attach + 1 < n ? m_attach + 1 : n;
  int64_t cap = n0 * n0 + 2 * (n > n0 ? (n - n0) : 0) * m_attach + 2;
  int64_t* s = (int64_t*)malloc(sizeof(int64_t) * cap);
  int64_t* d = (int64_t*)malloc(sizeof(int64_t) * cap);
  int64_t* ends = (int64_t*)malloc(sizeof(int64_t) * 2 * cap);
  int64_t* pick = (int64_t*)malloc(sizeof(int64_t) * (m_attach + 1));
  int64_t cnt = 0, ne = 0;
  for (int64_t i = 0; i < n0; ++i)
    for (int64_t j = i + 1; j < n0; ++j) { s[cnt] = i; d[cnt] = j; ++cnt; ends[ne++] = i; ends[ne++] = j; }
  uint64_t key = gg_key(seed, 0x4241ull /* "BA" */);
  uint64_t ctr = 0;
  for (int64_t v = n0; v < n; ++v) {
    int64_t got = 0;
    while (got < m_attach) {
      int64_t t = ends[gg_below(gg_draw(key, ctr++), (uint64_t)ne)];
      int dup = 0;
      for (int64_t q = 0; q < got; ++q) dup |= (pick[q] == t);
      if (!dup) pick[got++] = t;
    }
    for (int64_t q = 0; q < got; ++q) {
      s[cnt] = v; d[cnt] = pick[q]; ++cnt; ends[ne++] = v; ends[ne++] = pick[q];
    }
  }
  gg_graph* g = csr_from_pairs(n, s, d, cnt, NULL);
  free(s); free(d); free(ends); free(pick);
  return g;
}

int64_t gg_n(const gg_graph* g) { return g ? g->n : -1; }
int64_t gg_nnz(const gg_graph* g) { return g ? g->nnz : -1; }
void gg_copy(const gg_graph* g, int64_t* row_ptr, int32_t* col) {
  memcpy(row_ptr, g->row_ptr, sizeof(int64_t) * (size_t)(g->n + 1));
  if (g->nnz) memcpy(col, g->col, sizeof(int32_t) * (size_t)g->nnz);
}
void gg_free(gg_graph* g) {
  if (!g) return;
  free(g->row_ptr); free(g->col); free(g);
}
