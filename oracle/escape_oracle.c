/*
 * escape_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU restatement of what the ESCAPE census
 * computes (Pinar, Seshadhri, Vishal, "ESCAPE: Efficiently Counting All
 * 5-Vertex Subgraphs", arXiv 1610.09411).  It exists to check the CUDA path
 * and is used only by the tests, the entry point's smoke check and the
 * benchmark's CPU-baseline leg.  It shares no code, table or header with the
 * CUDA library.
 *
 * Two tiers:
 *   O1  oracle_brute_census: the definition itself -- every k-subset
 *       (k = 3, 4, 5) is classified by canonical form (Sec. 3.1); only for
 *       small n.
 *   O2  oracle_census_sums: per-vertex / per-edge quantities computed from
 *       their plain definitions (common-neighbour lists by sorted merge,
 *       per-vertex two-hop pair counts), then the sums that the paper's
 *       closed forms (Thms 4, 8-11, 13, 14; App. A) are built from.  The
 *       closed forms themselves are assembled in exact Python integers in
 *       oracle/__init__.py.
 *
 * Input: simple undirected graph as CSR (row_ptr int64[n+1], col int32[nnz]),
 * neighbour lists sorted ascending, symmetric, no loops or duplicates.
 * Degree order (Sec. 3.2): i < j iff d(i) < d(j), or d(i) = d(j) and i < j.
 * All sums are unsigned 128-bit with overflow detection; any overflow makes
 * the call return ORACLE_EOVERFLOW.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads the census runs on: 1 in the default (serial) build; with
 * -fopenmp, the OpenMP thread count (OMP_NUM_THREADS). */
int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static int thread_id(void) {
#ifdef _OPENMP
  return omp_get_thread_num();
#else
  return 0;
#endif
}

typedef unsigned __int128 u128;

enum { ORACLE_OK = 0, ORACLE_EINVAL = 1, ORACLE_ENOMEM = 2, ORACLE_EOVERFLOW = 4 };

/* ------------------------------------------------------------------ */
/* Pattern catalogue.  5-vertex connected patterns 1..21 follow the    */
/* paper's figure of all connected 5-vertex patterns (tikz macros       */
/* \pone..\ptwentyone); 22..32 follow its figure of disconnected         */
/* 5-vertex patterns; 33 (P3 + K2) and 34 (K3 + K2) complete the 34     */
/* isomorphism classes (the paper's disconnected figure omits these two). */
/* Vertices are the paper's labels 1..5; edges written as two digits.    */
/* ------------------------------------------------------------------ */
static const char* const CAT5[34] = {
  "12 13 14 15",                     /* 1  4-star                       */
  "12 13 14 25",                     /* 2                               */
  "12 13 24 35",                     /* 3  path P5                      */
  "12 13 23 34 35",                  /* 4                               */
  "12 13 23 24 45",                  /* 5                               */
  "12 13 23 24 35",                  /* 6                               */
  "12 13 24 34 35",                  /* 7                               */
  "12 13 24 35 45",                  /* 8  5-cycle                      */
  "12 13 23 34 35 45",               /* 9  bowtie                       */
  "12 13 14 24 34 35",               /* 10                              */
  "12 13 23 24 34 35",               /* 11                              */
  "12 13 24 34 35 45",               /* 12 house                        */
  "12 13 14 25 35 45",               /* 13 K2,3                         */
  "12 13 14 15 25 35 45",            /* 14                              */
  "12 13 14 23 24 34 35",            /* 15 K4 + pendant                 */
  "12 13 23 24 34 35 45",            /* 16                              */
  "12 13 14 23 24 35 45",            /* 17                              */
  "12 13 14 15 23 24 35 45",         /* 18 wheel                        */
  "12 13 14 23 24 34 35 45",         /* 19                              */
  "13 14 15 23 24 25 34 35 45",      /* 20 K5 minus an edge             */
  "12 13 14 15 23 24 25 34 35 45",   /* 21 K5                           */
  "",                                /* 22 5K1                          */
  "12",                              /* 23 K2 + 3K1                     */
  "12 34",                           /* 24 2K2 + K1                     */
  "12 23",                           /* 25 P3 + 2K1                     */
  "12 13 23",                        /* 26 K3 + 2K1                     */
  "12 13 14",                        /* 27 3-star + K1                  */
  "12 13 24",                        /* 28 P4 + K1                      */
  "12 13 14 23",                     /* 29 tailed triangle + K1         */
  "12 13 24 34",                     /* 30 C4 + K1                      */
  "12 13 14 23 24",                  /* 31 diamond + K1                 */
  "12 13 14 23 24 34",               /* 32 K4 + K1                      */
  "12 23 45",                        /* 33 P3 + K2                      */
  "12 13 23 45",                     /* 34 K3 + K2                      */
};
/* 4-vertex: connected patterns of the paper's 4-vertex figure (3-star,
 * 3-path, tailed triangle, 4-cycle, diamond, 4-clique), then its
 * disconnected 4-vertex figure (independent set, edge, matching, wedge,
 * triangle). */
static const char* const CAT4[11] = {
  "12 13 14", "12 13 24", "12 13 14 23", "12 13 24 34", "12 13 14 23 24",
  "12 13 14 23 24 34", "", "12", "12 34", "12 23", "12 13 23",
};
/* 3-vertex: empty, edge, wedge, triangle. */
static const char* const CAT3[4] = { "", "12", "12 13", "12 13 23" };

static int pair_index(int k, int a, int b) { /* a < b, 0-based, bit of pair */
  int idx = 0;
  for (int x = 0; x < k; ++x)
    for (int y = x + 1; y < k; ++y, ++idx)
      if (x == a && y == b) return idx;
  return -1;
}

static int parse_mask(int k, const char* s) {
  int mask = 0;
  for (const char* p = s; *p; ++p) {
    if (*p >= '1' && *p <= '9' && p[1] >= '1' && p[1] <= '9') {
      int a = p[0] - '1', b = p[1] - '1';
      if (a > b) { int t = a; a = b; b = t; }
      mask |= 1 << pair_index(k, a, b);
      ++p;
    }
  }
  return mask;
}

static int permute_mask(int k, int mask, const int* perm) {
  int out = 0, idx = 0;
  for (int x = 0; x < k; ++x)
    for (int y = x + 1; y < k; ++y, ++idx)
      if (mask >> idx & 1) {
        int a = perm[x], b = perm[y];
        if (a > b) { int t = a; a = b; b = t; }
        out |= 1 << pair_index(k, a, b);
      }
  return out;
}

/* canonical form = smallest mask over all k! relabellings */
static int canon(int k, int mask) {
  int perm[5] = {0, 1, 2, 3, 4}, best = 1 << 30;
  /* iterate permutations (Heap's algorithm, iterative) */
  int c[5] = {0}, i = 0;
  int v = permute_mask(k, mask, perm);
  if (v < best) best = v;
  while (i < k) {
    if (c[i] < i) {
      int a = (i % 2 == 0) ? 0 : c[i];
      int t = perm[a]; perm[a] = perm[i]; perm[i] = t;
      v = permute_mask(k, mask, perm);
      if (v < best) best = v;
      ++c[i]; i = 0;
    } else { c[i] = 0; ++i; }
  }
  return best;
}

static int g_tables_ready = 0;
static signed char g_cls3[8], g_cls4[64], g_cls5[1024];
static int g_rep3[4], g_rep4[11], g_rep5[34];

static int build_tables(void) {
  if (g_tables_ready) return 0;
  const char* const* cats[3] = {CAT3, CAT4, CAT5};
  int ks[3] = {3, 4, 5}, ncls[3] = {4, 11, 34};
  signed char* tabs[3] = {g_cls3, g_cls4, g_cls5};
  int* reps[3] = {g_rep3, g_rep4, g_rep5};
  for (int t = 0; t < 3; ++t) {
    int k = ks[t], npairs = k * (k - 1) / 2;
    int cf[34];
    for (int c = 0; c < ncls[t]; ++c) {
      reps[t][c] = parse_mask(k, cats[t][c]);
      cf[c] = canon(k, reps[t][c]);
      for (int d = 0; d < c; ++d) if (cf[d] == cf[c]) return ORACLE_EINVAL; /* duplicate class */
    }
    for (int mask = 0; mask < (1 << npairs); ++mask) {
      int f = canon(k, mask), cls = -1;
      for (int c = 0; c < ncls[t]; ++c) if (cf[c] == f) cls = c;
      if (cls < 0) return ORACLE_EINVAL;                               /* catalogue incomplete */
      tabs[t][mask] = (signed char)cls;
    }
  }
  g_tables_ready = 1;
  return 0;
}

/* Class id (0-based) of a k-vertex graph given by its pair mask. */
int oracle_classify(int k, int mask) {
  if (build_tables()) return -1;
  if (k == 3) return g_cls3[mask & 7];
  if (k == 4) return g_cls4[mask & 63];
  if (k == 5) return g_cls5[mask & 1023];
  return -1;
}

/* A[i][j] = number of spanning subgraphs (all k vertices, a subset of the
 * edges) of class j's graph that are isomorphic to class i (App. B: N = A C).
 * Written row-major into A (ncls x ncls). */
int oracle_matrix(int k, int64_t* A) {
  if (build_tables()) return ORACLE_EINVAL;
  int ncls = k == 3 ? 4 : (k == 4 ? 11 : (k == 5 ? 34 : 0));
  if (!ncls) return ORACLE_EINVAL;
  const int* reps = k == 3 ? g_rep3 : (k == 4 ? g_rep4 : g_rep5);
  memset(A, 0, sizeof(int64_t) * ncls * ncls);
  for (int j = 0; j < ncls; ++j) {
    int e = reps[j];
    /* every subset of the edge set of class j */
    for (int sub = e;; sub = (sub - 1) & e) {
      A[oracle_classify(k, sub) * ncls + j] += 1;
      if (sub == 0) break;
    }
  }
  return ORACLE_OK;
}

/* ------------------------------------------------------------------ */
/* O1: brute force over every k-subset (the definition, Sec. 3.1).      */
/* ------------------------------------------------------------------ */
static int has_edge(const int64_t* rp, const int32_t* col, int64_t u, int64_t v) {
  int64_t lo = rp[u], hi = rp[u + 1];
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (col[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo < rp[u + 1] && col[lo] == v;
}

int oracle_brute_census(int64_t n, const int64_t* rp, const int32_t* col,
                        uint64_t* c3, uint64_t* c4, uint64_t* c5) {
  if (build_tables()) return ORACLE_EINVAL;
  if (n > 200) return ORACLE_EINVAL;
  memset(c3, 0, 4 * sizeof(uint64_t));
  memset(c4, 0, 11 * sizeof(uint64_t));
  memset(c5, 0, 34 * sizeof(uint64_t));
  unsigned char* adj = (unsigned char*)calloc((size_t)(n > 0 ? n * n : 1), 1);
  if (!adj) return ORACLE_ENOMEM;
  for (int64_t u = 0; u < n; ++u)
    for (int64_t p = rp[u]; p < rp[u + 1]; ++p) adj[u * n + col[p]] = 1;
  int64_t v[5];
  for (v[0] = 0; v[0] < n; ++v[0])
    for (v[1] = v[0] + 1; v[1] < n; ++v[1])
      for (v[2] = v[1] + 1; v[2] < n; ++v[2]) {
        int m3 = (adj[v[0] * n + v[1]]) | (adj[v[0] * n + v[2]] << 1) | (adj[v[1] * n + v[2]] << 2);
        c3[g_cls3[m3]]++;
        for (v[3] = v[2] + 1; v[3] < n; ++v[3]) {
          int m4 = 0, idx = 0;
          for (int x = 0; x < 4; ++x)
            for (int y = x + 1; y < 4; ++y, ++idx) m4 |= adj[v[x] * n + v[y]] << idx;
          c4[g_cls4[m4]]++;
          for (v[4] = v[3] + 1; v[4] < n; ++v[4]) {
            int m5 = 0; idx = 0;
            for (int x = 0; x < 5; ++x)
              for (int y = x + 1; y < 5; ++y, ++idx) m5 |= adj[v[x] * n + v[y]] << idx;
            c5[g_cls5[m5]]++;
          }
        }
      }
  free(adj);
  return ORACLE_OK;
}

/* ------------------------------------------------------------------ */
/* O2: the paper's method, written plainly.                            */
/* ------------------------------------------------------------------ */
static int g_ovf;
static void set_ovf(void) { __atomic_store_n(&g_ovf, 1, __ATOMIC_RELAXED); }
static u128 add(u128 a, u128 b) { u128 s = a + b; if (s < a) set_ovf(); return s; }
static u128 mul(u128 a, u128 b) {
  if (a != 0 && b > ((u128)0 - 1) / a) set_ovf();
  return a * b;
}
static u128 ch2(uint64_t x) { return x < 2 ? 0 : (u128)x * (x - 1) / 2; }
static u128 ch3(uint64_t x) { return x < 3 ? 0 : ch2(x) * (x - 2) / 3; }
static u128 ch4(uint64_t x) { return x < 4 ? 0 : ch3(x) * (x - 3) / 4; }

/* Indices of the sums returned by oracle_census_sums (each 2 x u64, lo/hi). */
enum {
  S_N, S_M, S_W, S_S3, S_S4, S_T, S_EDGE_DD /* sum_e (d_i-1)(d_j-1) */, S_TT,
  S_C4, S_D, S_K4, S_N2A, S_N3A, S_N4, S_N5A, S_N6A, S_N7A, S_N8M, S_N8Z, S_N9A,
  S_N10A, S_N11, S_N12A, S_N13, S_N14, S_N15, S_N16A, S_N17, S_N18X4, S_N19,
  S_N20, S_N21, S_WM /* W*m */, S_D2D /* sum_c C(d_c,2) d_c */,
  S_DNBR /* sum_c (d_c-1) sum_{a in N(c)} d_a */, S_TM /* T*m */, S_TD /* sum_i t_i d_i */,
  S_COUNT
};

int oracle_num_sums(void) { return S_COUNT; }

typedef struct {
  int64_t n;
  const int64_t* rp;
  const int32_t* col;
  int64_t* deg;
  /* common-neighbour list of every CSR slot p = (u -> v):
   * U[ubeg[p] .. ubeg[p] + ulen[p]) = N(u) cap N(v), sorted; the two slots
   * of an edge share one stored list */
  int64_t* ubeg;
  int64_t* ulen;
  int32_t* U;
  int64_t* rev;   /* rev[p] = slot of (v -> u) */
} G;

static int prec(const G* g, int64_t a, int64_t b) {  /* a precedes b in the degree order */
  return g->deg[a] < g->deg[b] || (g->deg[a] == g->deg[b] && a < b);
}

static int64_t slot_of(const G* g, int64_t u, int64_t v) {
  int64_t lo = g->rp[u], hi = g->rp[u + 1];
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (g->col[mid] < v) lo = mid + 1; else hi = mid;
  }
  return (lo < g->rp[u + 1] && g->col[lo] == v) ? lo : -1;
}

static int64_t merge_count(const int32_t* a, int64_t na, const int32_t* b, int64_t nb) {
  int64_t i = 0, j = 0, c = 0;
  while (i < na && j < nb) {
    if (a[i] < b[j]) ++i; else if (a[i] > b[j]) ++j; else { ++c; ++i; ++j; }
  }
  return c;
}

static int validate(int64_t n, const int64_t* rp, const int32_t* col) {
  if (n < 0 || rp[0] != 0) return ORACLE_EINVAL;
  for (int64_t u = 0; u < n; ++u)
    if (rp[u + 1] < rp[u]) return ORACLE_EINVAL;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(| : bad)
  for (int64_t u = 0; u < n; ++u)
    for (int64_t p = rp[u]; p < rp[u + 1]; ++p) {
      if (col[p] < 0 || col[p] >= n || col[p] == u) bad = 1;
      else if (p > rp[u] && col[p] <= col[p - 1]) bad = 1;
    }
  if (bad) return ORACLE_EINVAL;
#pragma omp parallel for schedule(dynamic, 256) reduction(| : bad)
  for (int64_t u = 0; u < n; ++u)
    for (int64_t p = rp[u]; p < rp[u + 1]; ++p)
      if (!has_edge(rp, col, col[p], u)) bad = 1;
  return bad ? ORACLE_EINVAL : ORACLE_OK;
}

static void free_g(G* g) { free(g->deg); free(g->ubeg); free(g->ulen); free(g->U); free(g->rev); }

static int setup(G* g, int64_t n, const int64_t* rp, const int32_t* col) {
  memset(g, 0, sizeof(*g));
  g->n = n; g->rp = rp; g->col = col;
  int64_t nnz = n > 0 ? rp[n] : 0;
  g->deg = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
  g->ubeg = (int64_t*)malloc(sizeof(int64_t) * (nnz + 1));
  g->ulen = (int64_t*)malloc(sizeof(int64_t) * (nnz + 1));
  g->rev = (int64_t*)malloc(sizeof(int64_t) * (nnz + 1));
  if (!g->deg || !g->ubeg || !g->ulen || !g->rev) return ORACLE_ENOMEM;
  for (int64_t u = 0; u < n; ++u) g->deg[u] = rp[u + 1] - rp[u];
  /* T(e) = |N(u) cap N(v)| for every slot; the list of an edge is stored
   * once, at the slot whose row has the smaller id, and the reverse slot
   * points at it */
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t u = 0; u < n; ++u)
    for (int64_t p = rp[u]; p < rp[u + 1]; ++p) {
      int64_t v = col[p];
      g->ulen[p] = merge_count(col + rp[u], g->deg[u], col + rp[v], g->deg[v]);
      g->rev[p] = slot_of(g, v, u);
    }
  int64_t total = 0;
  for (int64_t u = 0; u < n; ++u)
    for (int64_t p = rp[u]; p < rp[u + 1]; ++p)
      if (u < col[p]) { g->ubeg[p] = total; total += g->ulen[p]; }
  for (int64_t u = 0; u < n; ++u)
    for (int64_t p = rp[u]; p < rp[u + 1]; ++p)
      if (u > col[p]) g->ubeg[p] = g->ubeg[g->rev[p]];
  g->U = (int32_t*)malloc(sizeof(int32_t) * (total + 1));
  if (!g->U) return ORACLE_ENOMEM;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t u = 0; u < n; ++u)
    for (int64_t p = rp[u]; p < rp[u + 1]; ++p) {
      int64_t v = col[p], i = rp[u], j = rp[v], w = g->ubeg[p];
      if (v < u) continue;
      while (i < rp[u + 1] && j < rp[v + 1]) {
        if (col[i] < col[j]) ++i; else if (col[i] > col[j]) ++j;
        else { g->U[w++] = col[i]; ++i; ++j; }
      }
    }
  return ORACLE_OK;
}

#define TE(p) ((uint64_t)g.ulen[(p)])
#define UB(p) (g.ubeg[(p)])
#define UE(p) (g.ubeg[(p)] + g.ulen[(p)])

/* Scratch of one thread: marks and counters over the vertices, and the
 * thread's partial sums.  The serial build has exactly one. */
typedef struct {
  int64_t *cnt, *cc, *wp, *stamp, *stamp2, *stamp3, *touched, *pos;
  u128 S[S_COUNT];
} Work;

static void free_work(Work* w, int nw) {
  if (!w) return;
  for (int t = 0; t < nw; ++t) {
    free(w[t].cnt); free(w[t].cc); free(w[t].wp); free(w[t].stamp);
    free(w[t].stamp2); free(w[t].stamp3); free(w[t].touched); free(w[t].pos);
  }
  free(w);
}

static Work* alloc_work(int nw, int64_t n) {
  Work* w = (Work*)calloc((size_t)nw, sizeof(Work));
  if (!w) return NULL;
  for (int t = 0; t < nw; ++t) {
    w[t].cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));     /* W(i, .) */
    w[t].cc = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));      /* cc(i, .) */
    w[t].wp = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));      /* w'(i, .) */
    w[t].stamp = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
    w[t].stamp2 = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
    w[t].stamp3 = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
    w[t].touched = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
    w[t].pos = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
    if (!w[t].cnt || !w[t].cc || !w[t].wp || !w[t].stamp || !w[t].stamp2 || !w[t].stamp3 ||
        !w[t].touched || !w[t].pos) { free_work(w, nw); return NULL; }
    for (int64_t v = 0; v <= n; ++v) { w[t].stamp[v] = -1; w[t].stamp2[v] = -1; w[t].stamp3[v] = -1; }
  }
  return w;
}

/* Add every thread's partial sums to S, in thread order, and clear them. */
static void fold(u128* S, Work* w, int nw) {
  for (int t = 0; t < nw; ++t)
    for (int s = 0; s < S_COUNT; ++s) { S[s] = add(S[s], w[t].S[s]); w[t].S[s] = 0; }
}

static void reset_marks(Work* w, int nw, int64_t n) {
  for (int t = 0; t < nw; ++t)
    for (int64_t v = 0; v <= n; ++v) { w[t].stamp[v] = -1; w[t].stamp2[v] = -1; }
}

/*
 * Per-element outputs (any may be NULL), indexed like the input:
 *   Te[p], C4e[p], K4e[p] per CSR slot p (both slots of an edge agree);
 *   ti[v], C4i[v], K4i[v] per vertex.
 * sums: S_COUNT entries of two u64 words (lo, hi) each.
 *
 * Built with -fopenmp, each loop over a vertex (or over the rows of the
 * edges) runs its iterations on several threads: every iteration writes only
 * its own per-element entries and its thread's scratch and partial sums, and
 * the partial sums are added in thread order.  The arithmetic is the same as
 * in the serial build; only the order of the exact additions differs.
 */
int oracle_census_sums(int64_t n, const int64_t* rp, const int32_t* col, uint64_t* sums,
                       uint64_t* Te_out, uint64_t* ti_out, uint64_t* C4e_out, uint64_t* C4i_out,
                       uint64_t* K4e_out, uint64_t* K4i_out) {
  int rc = validate(n, rp, col);
  if (rc) return rc;
  G g;
  rc = setup(&g, n, rp, col);
  if (rc) { free_g(&g); return rc; }
  g_ovf = 0;
  int64_t nnz = n > 0 ? rp[n] : 0;
  u128 S[S_COUNT];
  memset(S, 0, sizeof(S));
  const int nw = oracle_num_threads();

  uint64_t* t = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
  uint64_t* C4e = (uint64_t*)calloc((size_t)nnz + 1, sizeof(uint64_t));
  uint64_t* C4i = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
  uint64_t* K4e = (uint64_t*)calloc((size_t)nnz + 1, sizeof(uint64_t));
  uint64_t* K4i = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
  Work* work = alloc_work(nw, n);
  int64_t* outp = NULL;
  int32_t* outc = NULL;
  if (!t || !C4e || !C4i || !K4e || !K4i || !work) { rc = ORACLE_ENOMEM; goto done; }

  /* ---- degrees, wedges, stars (Thm 4) ---- */
  S[S_N] = (u128)n;
  S[S_M] = (u128)(nnz / 2);
  for (int64_t i = 0; i < n; ++i) {
    S[S_W] = add(S[S_W], ch2(g.deg[i]));
    S[S_S3] = add(S[S_S3], ch3(g.deg[i]));
    S[S_S4] = add(S[S_S4], ch4(g.deg[i]));            /* N1 (Thm 8) */
  }

  /* ---- triangles per vertex: t(i) = (1/2) sum_{j in N(i)} T(i,j) ---- */
  for (int64_t i = 0; i < n; ++i) {
    uint64_t s = 0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s += TE(p);
    t[i] = s / 2;
  }
  for (int64_t i = 0; i < n; ++i) S[S_T] = add(S[S_T], t[i]);
  S[S_T] /= 3;
  for (int64_t i = 0; i < n; ++i)
    if (g.deg[i] >= 2) S[S_TT] = add(S[S_TT], mul(t[i], (uint64_t)(g.deg[i] - 2)));   /* tailed triangles */

  /* ---- per-edge sums over unordered edges e = {i, j} (Thms 4, 9) ---- */
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int64_t j = col[p];
      uint64_t te = TE(p), di = (uint64_t)g.deg[i], dj = (uint64_t)g.deg[j];
      /* ordered sums: every slot (i -> j) */
      S[S_N2A] = add(S[S_N2A], mul(ch2(di - 1), dj - 1));                 /* N2 first term */
      S[S_N5A] = add(S[S_N5A], mul(t[i] - te, dj - 1));                   /* N5 first term */
      if (te >= 2) S[S_N11] = add(S[S_N11], mul(ch2(te), di - 3));         /* N11 */
      if (i < j) {   /* unordered */
        S[S_EDGE_DD] = add(S[S_EDGE_DD], mul(di - 1, dj - 1));
        S[S_D] = add(S[S_D], ch2(te));                                     /* diamonds */
        if (te) S[S_N6A] = add(S[S_N6A], mul(mul(te, di - 2), dj - 2));    /* N6 first term */
        S[S_N14] = add(S[S_N14], ch3(te));                                 /* N14 */
      }
    }

  /* ---- N3 first term: sum_i sum_{j<k in N(i)} (d_j-1)(d_k-1) (Thm 8) ---- */
  for (int64_t i = 0; i < n; ++i) {
    u128 s1 = 0, s2 = 0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      uint64_t x = (uint64_t)g.deg[col[p]] - 1;
      s1 = add(s1, x);
      s2 = add(s2, mul(x, x));
    }
    S[S_N3A] = add(S[S_N3A], (mul(s1, s1) - s2) / 2);
  }
  /* N4 = sum_i t(i) C(d(i)-2, 2); N9 first term = sum_i C(t(i), 2) (Thm 8) */
  for (int64_t i = 0; i < n; ++i) {
    if (g.deg[i] >= 2) S[S_N4] = add(S[S_N4], mul(t[i], ch2((uint64_t)g.deg[i] - 2)));
    S[S_N9A] = add(S[S_N9A], ch2(t[i]));
  }

  /* ---- per-edge and per-triangle 4-clique counts.  For an edge u < v (by
   * id) and x in U(u,v), the triangle {u, v, x} lies in |U(u,v) cap U(u,x)|
   * 4-cliques (its common neighbours); K4(e) is half the sum over x (Thm 7).
   * U(u,v) is marked in `stamp` so each intersection is one scan of U(u,x). */
#pragma omp parallel
  {
    Work* w = &work[thread_id()];
    int64_t* stamp = w->stamp;
#pragma omp for schedule(dynamic, 16)
    for (int64_t u = 0; u < n; ++u)
      for (int64_t p = rp[u]; p < rp[u + 1]; ++p) {
        int64_t v = col[p];
        if (v < u) continue;
        for (int64_t q = UB(p); q < UE(p); ++q) stamp[g.U[q]] = p;
        uint64_t s = 0;
        for (int64_t q = UB(p); q < UE(p); ++q) {
          int64_t x = g.U[q];
          int64_t px = slot_of(&g, u, x);
          uint64_t k4t = 0;
          for (int64_t r = UB(px); r < UE(px); ++r) k4t += (stamp[g.U[r]] == p);
          s += k4t;
          if (v < x) w->S[S_N20] = add(w->S[S_N20], ch2(k4t));   /* each triangle once: N20 (Thm 10) */
        }
        K4e[p] = s / 2;
        K4e[g.rev[p]] = s / 2;
      }
  }
  fold(S, work, nw);
  reset_marks(work, nw, n);
  for (int64_t i = 0; i < n; ++i) {
    uint64_t s = 0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s += K4e[p];
    K4i[i] = s / 3;
    S[S_K4] = add(S[S_K4], K4i[i]);
  }
  S[S_K4] /= 4;

  /* ---- per-triangle sums N10, N16 (Thm 10) and the directed tailed-triangle
   * correction of the 5-cycle count: each triangle once (u < v < x by id) ---- */
#pragma omp parallel
  {
    Work* w = &work[thread_id()];
#pragma omp for schedule(dynamic, 16)
    for (int64_t u = 0; u < n; ++u)
      for (int64_t p = rp[u]; p < rp[u + 1]; ++p) {
        int64_t v = col[p];
        if (v <= u) continue;
        for (int64_t q = UB(p); q < UE(p); ++q) {
          int64_t x = g.U[q];
          if (x <= v) continue;
          int64_t vs[3] = {u, v, x};
          uint64_t T_uv = TE(p), T_ux = TE(slot_of(&g, u, x)), T_vx = TE(slot_of(&g, v, x));
          /* edge opposite vertex k: k = x -> (u,v), k = v -> (u,x), k = u -> (v,x) */
          uint64_t Topp[3] = {T_vx, T_ux, T_uv};
          for (int k = 0; k < 3; ++k) {
            uint64_t dk = (uint64_t)g.deg[vs[k]];
            w->S[S_N10A] = add(w->S[S_N10A], mul(Topp[k] - 1, dk - 2));
          }
          /* shared vertex i: the two triangle edges at i */
          w->S[S_N16A] = add(w->S[S_N16A], mul(T_uv - 1, T_ux - 1));   /* at u */
          w->S[S_N16A] = add(w->S[S_N16A], mul(T_uv - 1, T_vx - 1));   /* at v */
          w->S[S_N16A] = add(w->S[S_N16A], mul(T_ux - 1, T_vx - 1));   /* at x */
        }
      }
  }
  fold(S, work, nw);

  /* ---- 4-cycles per vertex and per edge from the pair counts
   * W(i, j) = |N(i) cap N(j)| (two-hop from each i):
   *   C4(i)      = sum_{j != i} C(W(i,j), 2)
   *   C4((i,k))  = sum_{j in N(k), j != i} (W(i,j) - 1)
   * and, on the same pass, N13 = sum_{i<j} C(W(i,j), 3) and
   * N17 = sum_{i<j} (W(i,j) - 2) cc(i,j) with cc(i,j) the number of edges
   * inside N(i) cap N(j) (Thm 11), gathered from the triangles at i. ---- */
#pragma omp parallel
  {
    Work* w = &work[thread_id()];
    int64_t *stamp = w->stamp, *cnt = w->cnt, *cc = w->cc, *touched = w->touched;
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
      int64_t nt = 0;
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
        int64_t c = col[p];
        for (int64_t q = rp[c]; q < rp[c + 1]; ++q) {
          int64_t j = col[q];
          if (j == i) continue;
          if (stamp[j] != i) { stamp[j] = i; cnt[j] = 0; cc[j] = 0; touched[nt++] = j; }
          cnt[j]++;
        }
      }
      /* diamonds with tip i: triangle (i, x, y), x < y, and j in N(x) cap N(y), j != i */
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
        int64_t x = col[p];
        for (int64_t q = UB(p); q < UE(p); ++q) {
          int64_t y = g.U[q];
          if (y <= x) continue;
          int64_t pxy = slot_of(&g, x, y);
          for (int64_t r = UB(pxy); r < UE(pxy); ++r) {
            int64_t j = g.U[r];
            if (j != i) cc[j]++;
          }
        }
      }
      u128 c4 = 0;
      for (int64_t a = 0; a < nt; ++a) {
        int64_t j = touched[a];
        c4 = add(c4, ch2((uint64_t)cnt[j]));
        if (j > i) {
          w->S[S_N13] = add(w->S[S_N13], ch3((uint64_t)cnt[j]));
          if (cc[j]) w->S[S_N17] = add(w->S[S_N17], mul((uint64_t)(cnt[j] - 2), (uint64_t)cc[j]));
        }
      }
      C4i[i] = (uint64_t)c4;
      if (c4 >> 64) set_ovf();
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
        int64_t k = col[p];
        uint64_t s = 0;
        for (int64_t q = rp[k]; q < rp[k + 1]; ++q) {
          int64_t j = col[q];
          if (j != i) s += (uint64_t)(cnt[j] - 1);
        }
        C4e[p] = s;
      }
    }
  }
  fold(S, work, nw);
  for (int64_t i = 0; i < n; ++i) S[S_C4] = add(S[S_C4], C4i[i]);
  S[S_C4] /= 4;

  /* ---- vertex- and edge-cut sums using C4 and K4 (Thms 8, 9) ---- */
  for (int64_t i = 0; i < n; ++i) {
    if (C4i[i]) S[S_N7A] = add(S[S_N7A], mul(C4i[i], (uint64_t)g.deg[i] - 2));
    if (K4i[i]) S[S_N15] = add(S[S_N15], mul(K4i[i], (uint64_t)g.deg[i] - 3));
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      if (col[p] <= i) continue;
      uint64_t te = TE(p);
      S[S_N12A] = add(S[S_N12A], mul(C4e[p], te));
      if (K4e[p]) S[S_N19] = add(S[S_N19], mul(K4e[p], te - 2));
    }

  /* ---- wheels (N18): the number of 4-cycles in the graph induced on N(c),
   * summed over centres c.  For u in N(c) the two-hop count inside G[N(c)]
   * reaches v through k in N(c) cap N(u) = U(c,u) and v in U(c,k); every
   * 4-cycle is reached from each of its 4 vertices, so the sum of C(., 2)
   * over ordered (u, v) is 4 x N18 (Thm 11). ---- */
#pragma omp parallel
  {
    Work* w = &work[thread_id()];
    int64_t *stamp2 = w->stamp2, *cnt = w->cnt, *touched = w->touched, *pos = w->pos;
#pragma omp for schedule(dynamic, 16)
    for (int64_t c = 0; c < n; ++c) {
      for (int64_t p = rp[c]; p < rp[c + 1]; ++p) pos[col[p]] = p;   /* slot of (c -> x) */
      for (int64_t p = rp[c]; p < rp[c + 1]; ++p) {
        int64_t u = col[p], nt = 0;
        for (int64_t q = UB(p); q < UE(p); ++q) {
          int64_t k = g.U[q];
          int64_t pk = pos[k];
          for (int64_t r = UB(pk); r < UE(pk); ++r) {
            int64_t v = g.U[r];
            if (v == u) continue;
            if (stamp2[v] != p) { stamp2[v] = p; cnt[v] = 0; touched[nt++] = v; }
            cnt[v]++;
          }
        }
        for (int64_t a = 0; a < nt; ++a) w->S[S_N18X4] = add(w->S[S_N18X4], ch2((uint64_t)cnt[touched[a]]));
      }
    }
  }
  fold(S, work, nw);

  /* ---- 5-cycles (Thm 13).  For every directed 3-path i <- a -> b -> j of the
   * degree-ordered DAG (a < i, a < b < j, b != i, j != i), count the vertices
   * c in N(i) cap N(j), c != a, b, with c < max(i, j) (out-wedges and in-out
   * wedges between i and j in either direction):
   *   sum over paths of w'(i, j)             (the product term)
   *   minus sum over paths of [a~j] + [b~i] (paths whose own vertex is
   *                                           counted by w': the directed
   *                                           tailed triangles Z).
   * The degree order has three acyclic 5-cycle types up to isomorphism; each
   * 5-cycle is met exactly once this way. ---- */
  /* out-lists of the degree-ordered DAG: N+(v) = {u in N(v) : v < u} */
  outp = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
  outc = (int32_t*)malloc(sizeof(int32_t) * (nnz / 2 + 1));
  if (!outp || !outc) { rc = ORACLE_ENOMEM; goto done; }
  outp[0] = 0;
  for (int64_t v = 0; v < n; ++v) {
    int64_t q = outp[v];
    for (int64_t p = rp[v]; p < rp[v + 1]; ++p)
      if (prec(&g, v, col[p])) outc[q++] = col[p];
    outp[v + 1] = q;
  }
#pragma omp parallel
  {
    Work* w = &work[thread_id()];
    int64_t *stamp = w->stamp, *stamp2 = w->stamp2, *stamp3 = w->stamp3;
    int64_t *wp = w->wp, *touched = w->touched;
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
      int64_t nt = 0;
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
        int64_t c = col[p];
        for (int64_t q = rp[c]; q < rp[c + 1]; ++q) {
          int64_t j = col[q];
          if (j == i) continue;
          int64_t top = prec(&g, i, j) ? j : i;
          if (!prec(&g, c, top)) continue;
          if (stamp[j] != -2 - i) { stamp[j] = -2 - i; wp[j] = 0; touched[nt++] = j; }
          wp[j]++;
        }
      }
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) stamp2[col[p]] = -2 - i;   /* N(i) marker */
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
        int64_t a = col[p];
        if (!prec(&g, a, i)) continue;
        for (int64_t q = rp[a]; q < rp[a + 1]; ++q) stamp3[col[q]] = p;       /* N(a) marker */
        for (int64_t q = outp[a]; q < outp[a + 1]; ++q) {
          int64_t b = outc[q];
          if (b == i) continue;
          uint64_t b_adj_i = (stamp2[b] == -2 - i);
          for (int64_t r = outp[b]; r < outp[b + 1]; ++r) {
            int64_t j = outc[r];
            if (j == i) continue;
            uint64_t wv = (stamp[j] == -2 - i) ? (uint64_t)wp[j] : 0;
            w->S[S_N8M] = add(w->S[S_N8M], wv);
            w->S[S_N8Z] = add(w->S[S_N8Z], (uint64_t)(stamp3[j] == p) + b_adj_i);
          }
        }
      }
    }
  }
  fold(S, work, nw);

  /* ---- 5-cliques (Thm 14): every K5 contains exactly one directed
   * bipyramid whose triangle (i < j < k) is its three lowest vertices; count
   * adjacent pairs inside L = N+(i) cap N+(j) cap N+(k). ---- */
  reset_marks(work, nw, n);
#pragma omp parallel
  {
    Work* w = &work[thread_id()];
    int64_t *stamp = w->stamp, *stamp2 = w->stamp2, *touched = w->touched;
    int64_t tag = 0;
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i)
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
        int64_t j = col[p];
        if (!prec(&g, i, j)) continue;
        for (int64_t q = UB(p); q < UE(p); ++q) {
          int64_t k = g.U[q];
          if (!prec(&g, j, k)) continue;
          ++tag;
          for (int64_t r = outp[k]; r < outp[k + 1]; ++r) stamp[outc[r]] = tag;   /* N+(k) */
          int64_t nl = 0;
          for (int64_t r = UB(p); r < UE(p); ++r) {
            int64_t l = g.U[r];
            if (stamp[l] == tag) { touched[nl++] = l; stamp2[l] = tag; }        /* l in L */
          }
          for (int64_t a2 = 0; a2 < nl; ++a2) {
            int64_t l = touched[a2];
            for (int64_t r = outp[l]; r < outp[l + 1]; ++r)
              if (stamp2[outc[r]] == tag) w->S[S_N21] = add(w->S[S_N21], 1);    /* l -> l' inside L */
          }
        }
      }
  }
  fold(S, work, nw);

  /* ---- terms of the disconnected patterns (Thm 3, App. A) ---- */
  S[S_WM] = mul(S[S_W], S[S_M]);
  S[S_TM] = mul(S[S_T], S[S_M]);
  for (int64_t c = 0; c < n; ++c) {
    uint64_t dc = (uint64_t)g.deg[c];
    S[S_D2D] = add(S[S_D2D], mul(ch2(dc), dc));
    u128 nb = 0;
    for (int64_t p = rp[c]; p < rp[c + 1]; ++p) nb = add(nb, (uint64_t)g.deg[col[p]]);
    if (dc) S[S_DNBR] = add(S[S_DNBR], mul(dc - 1, nb));
    S[S_TD] = add(S[S_TD], mul(t[c], dc));
  }

  for (int s = 0; s < S_COUNT; ++s) {
    sums[2 * s] = (uint64_t)S[s];
    sums[2 * s + 1] = (uint64_t)(S[s] >> 64);
  }
  for (int64_t p = 0; p < nnz; ++p) {
    if (Te_out) Te_out[p] = TE(p);
    if (C4e_out) C4e_out[p] = C4e[p];
    if (K4e_out) K4e_out[p] = K4e[p];
  }
  for (int64_t v = 0; v < n; ++v) {
    if (ti_out) ti_out[v] = t[v];
    if (C4i_out) C4i_out[v] = C4i[v];
    if (K4i_out) K4i_out[v] = K4i[v];
  }
  rc = g_ovf ? ORACLE_EOVERFLOW : ORACLE_OK;
done:
  free(t); free(C4e); free(C4i); free(K4e); free(K4i); free(outp); free(outc);
  free_work(work, nw);
  free_g(&g);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Single-element values from their definitions (for sampled checks of */
/* graphs too large for the whole census above):                      */
/*   T(u,v)   = |N(u) cap N(v)|                                        */
/*   K4(u,v)  = number of edges inside N(u) cap N(v)                   */
/*   C4(u,v)  = sum_{j in N(v), j != u} (|N(u) cap N(j)| - 1)          */
/*   t(i)     = (1/2) sum_{v in N(i)} T(i,v)                           */
/*   C4(i)    = sum_{j != i} C(|N(i) cap N(j)|, 2)                     */
/* ------------------------------------------------------------------ */
static int64_t* two_hop(int64_t n, const int64_t* rp, const int32_t* col, int64_t u,
                        int64_t* cnt, int64_t* touched) {
  int64_t nt = 0;
  for (int64_t p = rp[u]; p < rp[u + 1]; ++p) {
    int64_t c = col[p];
    for (int64_t q = rp[c]; q < rp[c + 1]; ++q) {
      int64_t j = col[q];
      if (j == u) continue;
      if (cnt[j] == 0) touched[nt++] = j;
      cnt[j]++;
    }
  }
  touched[n] = nt;   /* count kept in the spare last slot */
  return touched;
}

/* ------------------------------------------------------------------ */
/* Wedges, triangles and diamonds alone (the unit counts of the census's */
/* algorithmic-byte model, for graphs whose full census is out of reach): */
/*   W = sum_i C(d(i), 2), T = (1/3) sum over edges of T(e),             */
/*   D = sum over edges e of C(T(e), 2), T(e) = |N(u) cap N(v)| by merge. */
/* out: 3 entries of two u64 words (lo, hi): W, T, D.                    */
/* ------------------------------------------------------------------ */
int oracle_wedge_diamond_sums(int64_t n, const int64_t* rp, const int32_t* col, uint64_t* out) {
  int rc = validate(n, rp, col);
  if (rc) return rc;
  g_ovf = 0;
  u128 W = 0, T3 = 0, D = 0;
  for (int64_t u = 0; u < n; ++u) W = add(W, ch2((uint64_t)(rp[u + 1] - rp[u])));
  const int nw = oracle_num_threads();
  u128* part = (u128*)calloc((size_t)nw * 2, sizeof(u128));
  if (!part) return ORACLE_ENOMEM;
#pragma omp parallel
  {
    u128* mine = part + 2 * thread_id();
#pragma omp for schedule(dynamic, 64)
    for (int64_t u = 0; u < n; ++u)
      for (int64_t p = rp[u]; p < rp[u + 1]; ++p) {
        int64_t v = col[p];
        if (v <= u) continue;                   /* each edge once */
        uint64_t te = (uint64_t)merge_count(col + rp[u], rp[u + 1] - rp[u], col + rp[v], rp[v + 1] - rp[v]);
        mine[0] = add(mine[0], te);
        mine[1] = add(mine[1], ch2(te));
      }
  }
  for (int t = 0; t < nw; ++t) { T3 = add(T3, part[2 * t]); D = add(D, part[2 * t + 1]); }
  free(part);
  u128 vals[3] = {W, T3 / 3, D};
  for (int k = 0; k < 3; ++k) { out[2 * k] = (uint64_t)vals[k]; out[2 * k + 1] = (uint64_t)(vals[k] >> 64); }
  return g_ovf ? ORACLE_EOVERFLOW : ORACLE_OK;
}

/* ------------------------------------------------------------------ */
/* Pair sums alone (Thm 5 and the K2,3 term of Thm 11; for graphs whose */
/* full census is out of reach).  W(i,j) = |N(i) cap N(j)| is counted  */
/* by two-hop walks i - c - j from every i:                             */
/*   C4  = (1/4) sum_i sum_{j != i} C(W(i,j), 2)  (each 4-cycle has two  */
/*         opposite pairs, each seen from both ends),                    */
/*   N13 = sum_{i<j} C(W(i,j), 3)  (non-induced K2,3).                   */
/* out: 2 entries of two u64 words (lo, hi): C4, N13.                   */
/* ------------------------------------------------------------------ */
int oracle_pair_sums(int64_t n, const int64_t* rp, const int32_t* col, uint64_t* out) {
  int rc = validate(n, rp, col);
  if (rc) return rc;
  g_ovf = 0;
  const int nw = oracle_num_threads();
  u128* part = (u128*)calloc((size_t)nw * 2, sizeof(u128));
  int64_t* scratch = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)(n + 1) * (size_t)nw);
  if (!part || !scratch) { free(part); free(scratch); return ORACLE_ENOMEM; }
#pragma omp parallel
  {
    const int t = thread_id();
    int64_t* stamp = scratch + (size_t)t * 3 * (size_t)(n + 1);
    int64_t* cnt = stamp + (n + 1);
    int64_t* touched = cnt + (n + 1);
    for (int64_t v = 0; v <= n; ++v) stamp[v] = -1;
    u128* mine = part + 2 * t;
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
      int64_t nt = 0;
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
        int64_t c = col[p];
        for (int64_t q = rp[c]; q < rp[c + 1]; ++q) {
          int64_t j = col[q];
          if (j == i) continue;
          if (stamp[j] != i) { stamp[j] = i; cnt[j] = 0; touched[nt++] = j; }
          cnt[j]++;
        }
      }
      for (int64_t a = 0; a < nt; ++a) {
        int64_t j = touched[a];
        mine[0] = add(mine[0], ch2((uint64_t)cnt[j]));
        if (j > i) mine[1] = add(mine[1], ch3((uint64_t)cnt[j]));
      }
    }
  }
  u128 S4 = 0, N13 = 0;
  for (int t = 0; t < nw; ++t) { S4 = add(S4, part[2 * t]); N13 = add(N13, part[2 * t + 1]); }
  free(part);
  free(scratch);
  u128 vals[2] = {S4 / 4, N13};
  for (int k = 0; k < 2; ++k) { out[2 * k] = (uint64_t)vals[k]; out[2 * k + 1] = (uint64_t)(vals[k] >> 64); }
  return g_ovf ? ORACLE_EOVERFLOW : ORACLE_OK;
}

/* ------------------------------------------------------------------ */
/* 4-cliques alone (Thm 6; for graphs whose full census is out of      */
/* reach): every K4 once, at its lowest vertex x in the degree order    */
/* (Sec. 3.2, ties by id), as a triangle a < b < c of G[N+(x)]:         */
/*   K4 = sum_x #{(a, b, c) : a in N+(x), b in N+(a) cap N+(x),         */
/*                            c in N+(b) cap N+(a) cap N+(x)}.          */
/* out: two u64 words (lo, hi).                                         */
/* ------------------------------------------------------------------ */
int oracle_clique4_count(int64_t n, const int64_t* rp, const int32_t* col, uint64_t* out) {
  int rc = validate(n, rp, col);
  if (rc) return rc;
  g_ovf = 0;
  G g = {0};
  g.n = n;
  g.rp = rp;
  g.col = col;
  g.deg = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t* orp = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!g.deg || !orp) { free(g.deg); free(orp); return ORACLE_ENOMEM; }
  for (int64_t v = 0; v < n; ++v) g.deg[v] = rp[v + 1] - rp[v];
  /* out-neighbour lists N+(v) = {w in N(v) : v precedes w}, ascending ids */
  for (int64_t v = 0; v < n; ++v) {
    int64_t k = 0;
    for (int64_t p = rp[v]; p < rp[v + 1]; ++p) k += prec(&g, v, col[p]);
    orp[v + 1] = orp[v] + k;
  }
  int32_t* ocol = (int32_t*)malloc(sizeof(int32_t) * (size_t)(orp[n] + 1));
  const int nw = oracle_num_threads();
  u128* part = (u128*)calloc((size_t)nw, sizeof(u128));
  int64_t* marks = (int64_t*)malloc(sizeof(int64_t) * 2 * (size_t)(n + 1) * (size_t)nw);
  if (!ocol || !part || !marks) { free(g.deg); free(orp); free(ocol); free(part); free(marks); return ORACLE_ENOMEM; }
  for (int64_t v = 0; v < n; ++v) {
    int64_t k = orp[v];
    for (int64_t p = rp[v]; p < rp[v + 1]; ++p)
      if (prec(&g, v, col[p])) ocol[k++] = col[p];
  }
#pragma omp parallel
  {
    const int t = thread_id();
    int64_t* in_x = marks + (size_t)t * 2 * (size_t)(n + 1);   /* in_x[v] == x: v in N+(x) */
    int64_t* in_a = in_x + (n + 1);                              /* in_a[v] == a: v in N+(a) cap N+(x) */
    for (int64_t v = 0; v <= n; ++v) { in_x[v] = -1; in_a[v] = -1; }
    u128 mine = 0;
#pragma omp for schedule(dynamic, 64)
    for (int64_t x = 0; x < n; ++x) {
      for (int64_t p = orp[x]; p < orp[x + 1]; ++p) in_x[ocol[p]] = x;
      for (int64_t p = orp[x]; p < orp[x + 1]; ++p) {
        int64_t a = ocol[p];
        for (int64_t q = orp[a]; q < orp[a + 1]; ++q)
          if (in_x[ocol[q]] == x) in_a[ocol[q]] = a;
        for (int64_t q = orp[a]; q < orp[a + 1]; ++q) {
          int64_t b = ocol[q];
          if (in_x[b] != x) continue;
          uint64_t k = 0;
          for (int64_t r = orp[b]; r < orp[b + 1]; ++r) {
            int64_t c = ocol[r];
            if (in_x[c] == x && in_a[c] == a) ++k;
          }
          mine = add(mine, k);
        }
      }
    }
    part[t] = mine;
  }
  u128 K4 = 0;
  for (int t = 0; t < nw; ++t) K4 = add(K4, part[t]);
  free(g.deg); free(orp); free(ocol); free(part); free(marks);
  out[0] = (uint64_t)K4;
  out[1] = (uint64_t)(K4 >> 64);
  return g_ovf ? ORACLE_EOVERFLOW : ORACLE_OK;
}

/* ------------------------------------------------------------------ */
/* 5-cliques alone (Thm 14; for graphs whose full census is out of      */
/* reach): every K5 once, at its lowest vertex x in the degree order, as */
/* a 4-clique a < b < c < e of H = G[N+(x)] (indices in N+(x)):          */
/*   K5 = sum_x sum over edges (a, b), a < b, of H and c in             */
/*        NH(a) cap NH(b) above b of |NH(a) cap NH(b) cap NH(c) above c|, */
/* with the neighbourhoods NH as bit sets over N+(x) and the sizes by   */
/* popcount.  out: two u64 words (lo, hi).                              */
/* ------------------------------------------------------------------ */
int oracle_clique5_count(int64_t n, const int64_t* rp, const int32_t* col, uint64_t* out) {
  int rc = validate(n, rp, col);
  if (rc) return rc;
  g_ovf = 0;
  G g = {0};
  g.n = n;
  g.rp = rp;
  g.col = col;
  g.deg = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t* orp = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!g.deg || !orp) { free(g.deg); free(orp); return ORACLE_ENOMEM; }
  for (int64_t v = 0; v < n; ++v) g.deg[v] = rp[v + 1] - rp[v];
  int64_t dmax = 0;
  for (int64_t v = 0; v < n; ++v) {
    int64_t k = 0;
    for (int64_t p = rp[v]; p < rp[v + 1]; ++p) k += prec(&g, v, col[p]);
    orp[v + 1] = orp[v] + k;
    if (k > dmax) dmax = k;
  }
  const int64_t wmax = (dmax + 63) / 64;
  int32_t* ocol = (int32_t*)malloc(sizeof(int32_t) * (size_t)(orp[n] + 1));
  const int nw = oracle_num_threads();
  u128* part = (u128*)calloc((size_t)nw, sizeof(u128));
  int32_t* posa = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1) * (size_t)nw);
  uint64_t* bits = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(dmax * wmax + 1) * (size_t)nw);
  if (!ocol || !part || !posa || !bits) {
    free(g.deg); free(orp); free(ocol); free(part); free(posa); free(bits);
    return ORACLE_ENOMEM;
  }
  for (int64_t v = 0; v < n; ++v) {
    int64_t k = orp[v];
    for (int64_t p = rp[v]; p < rp[v + 1]; ++p)
      if (prec(&g, v, col[p])) ocol[k++] = col[p];
  }
#pragma omp parallel
  {
    const int t = thread_id();
    int32_t* pos = posa + (size_t)t * (size_t)(n + 1);          /* pos[v] = index of v in N+(x), or -1 */
    uint64_t* B = bits + (size_t)t * (size_t)(dmax * wmax + 1);  /* row a of H: NH(a) as a bit set */
    for (int64_t v = 0; v <= n; ++v) pos[v] = -1;
    u128 mine = 0;
#pragma omp for schedule(dynamic, 64)
    for (int64_t x = 0; x < n; ++x) {
      const int64_t d = orp[x + 1] - orp[x];
      if (d < 4) continue;
      const int64_t W = (d + 63) / 64;
      for (int64_t a = 0; a < d; ++a) pos[ocol[orp[x] + a]] = (int32_t)a;
      memset(B, 0, sizeof(uint64_t) * (size_t)(d * W));
      for (int64_t a = 0; a < d; ++a) {
        int64_t va = ocol[orp[x] + a];
        for (int64_t q = orp[va]; q < orp[va + 1]; ++q) {
          int64_t b = pos[ocol[q]];
          if (b < 0) continue;
          B[a * W + b / 64] |= 1ull << (b % 64);
          B[b * W + a / 64] |= 1ull << (a % 64);
        }
      }
      for (int64_t a = 0; a < d; ++a)
        for (int64_t b = a + 1; b < d; ++b) {
          if (!((B[a * W + b / 64] >> (b % 64)) & 1)) continue;
          /* c: the common neighbours of a and b above b, word by word */
          for (int64_t wc = (b + 1) / 64; wc < W; ++wc) {
            uint64_t cm = B[a * W + wc] & B[b * W + wc];
            if (wc == (b + 1) / 64) cm &= ~0ull << ((b + 1) % 64);
            while (cm) {
              const int64_t c = wc * 64 + __builtin_ctzll(cm);
              cm &= cm - 1;
              uint64_t k = 0;   /* e above c adjacent to a, b and c */
              for (int64_t w = (c + 1) / 64; w < W; ++w) {
                uint64_t m = B[a * W + w] & B[b * W + w] & B[c * W + w];
                if (w == (c + 1) / 64) m &= ~0ull << ((c + 1) % 64);
                k += (uint64_t)__builtin_popcountll(m);
              }
              mine = add(mine, k);
            }
          }
        }
      for (int64_t a = 0; a < d; ++a) pos[ocol[orp[x] + a]] = -1;
    }
    part[t] = mine;
  }
  u128 K5 = 0;
  for (int t = 0; t < nw; ++t) K5 = add(K5, part[t]);
  free(g.deg); free(orp); free(ocol); free(part); free(posa); free(bits);
  out[0] = (uint64_t)K5;
  out[1] = (uint64_t)(K5 >> 64);
  return g_ovf ? ORACLE_EOVERFLOW : ORACLE_OK;
}

int oracle_edge_elements(int64_t n, const int64_t* rp, const int32_t* col, int64_t count,
                         const int64_t* us, const int64_t* vs, uint64_t* T, uint64_t* K4, uint64_t* C4) {
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t* touched = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
  int64_t* mark = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
  if (!cnt || !touched || !mark) { free(cnt); free(touched); free(mark); return ORACLE_ENOMEM; }
  for (int64_t v = 0; v <= n; ++v) mark[v] = -1;
  for (int64_t s = 0; s < count; ++s) {
    int64_t u = us[s], v = vs[s];
    if (u < 0 || u >= n || v < 0 || v >= n || !has_edge(rp, col, u, v)) { free(cnt); free(touched); free(mark); return ORACLE_EINVAL; }
    /* common neighbours, marked */
    uint64_t t = 0;
    for (int64_t p = rp[u]; p < rp[u + 1]; ++p)
      if (has_edge(rp, col, v, col[p])) { mark[col[p]] = s; ++t; }
    T[s] = t;
    uint64_t k = 0;
    for (int64_t p = rp[u]; p < rp[u + 1]; ++p) {
      int64_t x = col[p];
      if (mark[x] != s) continue;
      for (int64_t q = rp[x]; q < rp[x + 1]; ++q) k += (mark[col[q]] == s);
    }
    K4[s] = k / 2;
    two_hop(n, rp, col, u, cnt, touched);
    uint64_t c = 0;
    for (int64_t q = rp[v]; q < rp[v + 1]; ++q) {
      int64_t j = col[q];
      if (j != u) c += (uint64_t)(cnt[j] - 1);
    }
    C4[s] = c;
    for (int64_t a = 0; a < touched[n]; ++a) cnt[touched[a]] = 0;
  }
  free(cnt); free(touched); free(mark);
  return ORACLE_OK;
}

int oracle_vertex_elements(int64_t n, const int64_t* rp, const int32_t* col, int64_t count,
                           const int64_t* vs, uint64_t* t_out, uint64_t* C4_out) {
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t* touched = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
  if (!cnt || !touched) { free(cnt); free(touched); return ORACLE_ENOMEM; }
  for (int64_t s = 0; s < count; ++s) {
    int64_t i = vs[s];
    if (i < 0 || i >= n) { free(cnt); free(touched); return ORACLE_EINVAL; }
    uint64_t tt = 0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int64_t v = col[p];
      tt += (uint64_t)merge_count(col + rp[i], rp[i + 1] - rp[i], col + rp[v], rp[v + 1] - rp[v]);
    }
    t_out[s] = tt / 2;
    two_hop(n, rp, col, i, cnt, touched);
    uint64_t c = 0;
    for (int64_t a = 0; a < touched[n]; ++a) {
      uint64_t w = (uint64_t)cnt[touched[a]];
      c += w * (w - 1) / 2;
      cnt[touched[a]] = 0;
    }
    C4_out[s] = c;
  }
  free(cnt); free(touched);
  return ORACLE_OK;
}
