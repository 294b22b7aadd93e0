// census.cu -- the enumeration and assembly kernels of the 5-vertex census.
//
// All vertices are ranks of the degree order (Sec. 3.2), so `a < b` is the
// order itself; N+(v) is the suffix of row v, N-(v) its prefix.  Counts are
// exact: per-element counters are 32/64-bit, global sums 128-bit.
//
// Kernel map (paper section -> kernel):
//   Thm 4, 8, 9 degree/edge closed forms ...... k_vertex_basic, k_edge_sums
//   Thm 7 triangles T(e), t(i) ................ k_tri_small / k_tri_large (pass A)
//   Thm 6/7 4-cliques K4(e), K4(t); Thm 10 N10,
//     N16, N20; Thm 14 5-cliques ............... k_clique_warp / k_clique_large (pass B)
//   Thm 13's directed tailed triangles ......... k_tri_small / k_tri_large (pass A)
//   Thm 5 4-cycles C4(e), C4(i) ................ k_cycles4
//   Thm 12 common-neighbour lists of edges ..... k_tri_lists
//   Thm 11/12 N13, N17 (pairs and diamonds) .... k_pairs
//   Thm 11 N18 (wheels) ........................ k_wheels_warp / k_wheels_cta
//   Thm 13 5-cycles ............................ k_cycles5
//   Thm 3 + App. B assembly .................... k_assemble
#include "common.cuh"
#include "internal.h"

#include <algorithm>
#include <initializer_list>
#if defined(__has_include)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>          // header-only: no library to link
#define ESC_HAVE_NVTX 1
#endif
#endif
#ifndef ESC_HAVE_NVTX
#define ESC_HAVE_NVTX 0
#endif
#include <map>
#include <mutex>
#include <cstdio>
#include <cstdlib>
#include <vector>

namespace esc {

// ----------------------------------------------------------------------------
// Small device hash set of vertex ranks -> position (open addressing).
// ----------------------------------------------------------------------------
struct PosHash {
  int32_t* keys;     // EMPTY = -1
  int32_t* vals;
  int mask;
  __device__ __forceinline__ uint32_t h(int32_t k) const { return ((uint32_t)k * 0x9E3779B1u) >> 7; }
  __device__ __forceinline__ void insert(int32_t k, int32_t v) {
    uint32_t s = h(k) & mask;
    while (true) {
      int32_t old = atomicCAS(&keys[s], -1, k);
      if (old == -1 || old == k) { vals[s] = v; return; }
      s = (s + 1) & mask;
    }
  }
  __device__ __forceinline__ int32_t find(int32_t k) const {
    uint32_t s = h(k) & mask;
    while (true) {
      int32_t kk = keys[s];
      if (kk == k) return vals[s];
      if (kk == -1) return -1;
      s = (s + 1) & mask;
    }
  }
};

static __host__ __device__ __forceinline__ int pow2_at_least(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// ============================================================================
// Degree sums (Thm 4, Thm 8 N1/N3, Thm 9 N2, App. A P3+K2 terms).
// One warp per vertex.
// ============================================================================
__global__ void k_vertex_basic(DevGraph g, AccSet acc) {
  __shared__ u128 sh[32];
  int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int ids[9] = {ACC_W, ACC_S3, ACC_S4, ACC_D2D, ACC_DNBR, ACC_N2A, ACC_N3A, ACC_P4A, ACC_DP};
  LocalAcc<9> la;
  la.zero();
  for (int64_t v = warp; v < g.n; v += nwarps) {
    unsigned long long dv = (unsigned long long)dg_deg(g, v);
    unsigned long long dpv = (unsigned long long)dg_outdeg(g, v);
    u128 s1 = 0, s2 = 0, nb = 0, n2a = 0, p4a = 0, dp = 0;
    for (int64_t p = g.R[v] + lane; p < g.R[v + 1]; p += 32) {
      int32_t a = g.C[p];
      unsigned long long da = (unsigned long long)dg_deg(g, a);
      s1 += da - 1;
      s2 += (u128)(da - 1) * (da - 1);
      nb += da;
      n2a += ch2(dv - 1) * (da - 1);
      if (a > v) {
        p4a += (u128)(dv - 1) * (da - 1);
        dp += (u128)(dpv - 1) * (unsigned long long)dg_outdeg(g, a);   // the path's middle edge v -> a
      }
    }
    s1 = warp_sum_u128(s1);
    s2 = warp_sum_u128(s2);
    nb = warp_sum_u128(nb);
    n2a = warp_sum_u128(n2a);
    p4a = warp_sum_u128(p4a);
    dp = warp_sum_u128(dp);
    if (lane == 0) {
      la.v[8] += dp;
      la.v[0] += ch2(dv);
      la.v[1] += ch3(dv);
      la.v[2] += ch4(dv);
      la.v[3] += ch2(dv) * dv;
      la.v[4] += dv ? (u128)(dv - 1) * nb : 0;
      la.v[5] += n2a;
      la.v[6] += (s1 * s1 - s2) / 2;
      la.v[7] += p4a;
    }
    warp_item_flush(la, ids, acc, v);
  }
  final_flush(la, ids, acc, sh);
}

// ============================================================================
// Pass A: triangles.  Every triangle x < v < w is found once from its lowest
// vertex x as v in N+(x), w in N+(v) cap N+(x) (Thm 7).  It adds one to the
// triangle counts of its three edges (canonical slots in the lower endpoint's
// out-list) and contributes d+(x) + d+(v) + d+(w) - 3 to the directed
// tailed-triangle term of the 5-cycle count (Thm 13).
// ============================================================================
static constexpr int SMALL_DPLUS = 32;    // warp-per-vertex path up to this out-degree

// Warp per vertex with d+ <= 32: N+(x) in a per-warp shared-memory list,
// membership by binary search.
__global__ void k_tri_small(DevGraph g, const int32_t* items, int64_t nitems, uint32_t* T, AccSet acc) {
  __shared__ u128 sh[32];
  __shared__ int32_t lst[8][SMALL_DPLUS];
  __shared__ uint32_t cnt[8][SMALL_DPLUS];
  int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int ids[2] = {ACC_T, ACC_N8Z};
  LocalAcc<2> la;
  la.zero();
  for (int64_t it = warp; it < nitems; it += nwarps) {
    int64_t x = items[it];
    int64_t o = g.op[x];
    int d = (int)(g.R[x + 1] - o);
    if (lane < d) lst[wl][lane] = g.C[o + lane];
    cnt[wl][lane] = 0;
    __syncwarp();
    unsigned long long dpx = (unsigned long long)d;
    for (int a = 0; a < d; ++a) {
      int32_t v = lst[wl][a];
      int64_t vo = g.op[v], ve = g.R[v + 1];
      unsigned long long dpv = (unsigned long long)(ve - vo);
      for (int64_t q = vo + lane; q < ve; q += 32) {
        int32_t w = g.C[q];
        int lo = a + 1, hi = d;                 // w > v, so only positions after a
        while (lo < hi) { int mid = (lo + hi) >> 1; if (lst[wl][mid] < w) lo = mid + 1; else hi = mid; }
        if (lo < d && lst[wl][lo] == w) {
          atomicAdd(&T[q], 1u);
          atomicAdd(&cnt[wl][a], 1u);
          atomicAdd(&cnt[wl][lo], 1u);
          la.v[0] += 1;
          la.v[1] += dpx + dpv + (unsigned long long)(g.R[w + 1] - g.op[w]) - 3;
        }
      }
    }
    __syncwarp();
    if (lane < d && cnt[wl][lane]) atomicAdd(&T[o + lane], cnt[wl][lane]);
    __syncwarp();
    warp_item_flush(la, ids, acc, x);
  }
  final_flush(la, ids, acc, sh);
}

// CTA per vertex with d+ > 32: N+(x) in a shared-memory hash.
__global__ void k_tri_large(DevGraph g, const int32_t* items, int64_t nitems, unsigned long long* qctr,
                            uint32_t* T, AccSet acc, int hash_cap) {
  extern __shared__ int32_t smem[];
  __shared__ u128 sh[32];
  __shared__ int64_t sh_item;
  int32_t* hk = smem;
  int32_t* hv = hk + hash_cap;
  uint32_t* cnt = (uint32_t*)(hv + hash_cap);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int ids[2] = {ACC_T, ACC_N8Z};
  LocalAcc<2> la;
  la.zero();
  while (true) {
    int64_t it = next_item(qctr, nitems, &sh_item);
    if (it < 0) break;
    int64_t x = items[it];
    int64_t o = g.op[x];
    int d = (int)(g.R[x + 1] - o);
    int hsz = pow2_at_least(2 * d);
    PosHash H{hk, hv, hsz - 1};
    for (int i = threadIdx.x; i < hsz; i += blockDim.x) hk[i] = -1;
    for (int i = threadIdx.x; i < d; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < d; i += blockDim.x) H.insert(g.C[o + i], i);
    __syncthreads();
    unsigned long long dpx = (unsigned long long)d;
    for (int a = wid; a < d; a += nw) {
      int32_t v = g.C[o + a];
      int64_t vo = g.op[v], ve = g.R[v + 1];
      unsigned long long dpv = (unsigned long long)(ve - vo);
      unsigned on_xv = 0;
      for (int64_t q = vo + lane; q < ve; q += 32) {
        int32_t w = g.C[q];
        int b = H.find(w);
        if (b >= 0) {
          atomicAdd(&T[q], 1u);
          atomicAdd(&cnt[b], 1u);
          on_xv += 1;
          la.v[0] += 1;
          la.v[1] += dpx + dpv + (unsigned long long)(g.R[w + 1] - g.op[w]) - 3;
        }
      }
      on_xv = (unsigned)warp_sum_u64(on_xv);
      if (lane == 0 && on_xv) atomicAdd(&cnt[a], on_xv);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < d; i += blockDim.x)
      if (cnt[i]) atomicAdd(&T[o + i], cnt[i]);
    block_item_flush(la, ids, acc, x, sh);
    __syncthreads();
  }
  final_flush(la, ids, acc, sh);
}

// Copy canonical per-edge values to the reverse slot; per-vertex sums.
__global__ void k_sym_T(DevGraph g, uint32_t* T, unsigned long long* tv) {
  int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < g.n; v += nwarps)
    for (int64_t p = g.op[v] + lane; p < g.R[v + 1]; p += 32) T[g.rev[p]] = T[p];
}

__global__ void k_vertex_from_edges_T(DevGraph g, const uint32_t* T, unsigned long long* tv) {
  int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < g.n; v += nwarps) {
    unsigned long long s = 0;
    for (int64_t p = g.R[v] + lane; p < g.R[v + 1]; p += 32) s += T[p];
    s = warp_sum_u64(s);
    if (lane == 0) tv[v] = s / 2;
  }
}

__global__ void k_sym_u64(DevGraph g, unsigned long long* E) {
  int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < g.n; v += nwarps)
    for (int64_t p = g.op[v] + lane; p < g.R[v + 1]; p += 32) E[g.rev[p]] = E[p];
}

// 4-cycle per-edge counts arrive in either slot of an edge: fold them.
__global__ void k_fold_u64(DevGraph g, unsigned long long* E) {
  int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < g.n; v += nwarps)
    for (int64_t p = g.op[v] + lane; p < g.R[v + 1]; p += 32) {
      int64_t r = g.rev[p];
      unsigned long long s = E[p] + E[r];
      E[p] = s;
      E[r] = s;
    }
}

__global__ void k_vertex_sum_div(DevGraph g, const unsigned long long* E, unsigned long long* V, unsigned div) {
  int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < g.n; v += nwarps) {
    unsigned long long s = 0;
    for (int64_t p = g.R[v] + lane; p < g.R[v + 1]; p += 32) s += E[p];
    s = warp_sum_u64(s);
    if (lane == 0) V[v] = s / div;
  }
}

// ============================================================================
// Pass B: 4-cliques, 5-cliques and the per-triangle sums.
//
// For the lowest vertex x, B holds the adjacency bit matrix of the graph
// induced on N+(x) (row a = the out-neighbours of N+(x)[a] that are also in
// N+(x)).  For an edge (a, b) of it -- the triangle {x, v_a, v_b} with x
// lowest --
//   alpha = |row_a & row_b|   apexes of the triangle above x (K4s x,a,b,c)
//   beta  = apexes below x: in-neighbours y of x adjacent to v_a and v_b.
//           With D_a = bit set over N-(x) of {y : v_a in N+(y)}, beta =
//           |D_a & D_b|.
// so K4(t) = alpha + beta (Thm 7), and
//   N20 += C(alpha + beta, 2)                                (Thm 10)
//   N10 += sum over the 3 vertices k of (T(opposite edge) - 1)(d_k - 2)
//   N16 += sum over the 3 vertices of (T(e1) - 1)(T(e2) - 1)  (Thm 10)
//   K4 total += alpha / 3; K4(v_a, v_b) += alpha; K4(x, v_a) += alpha / 2 summed
//   K5 += |row_a & row_b & row_c| above c for every c in row_a & row_b above b
//        (each 5-clique once, at its three lowest vertices: Thm 14)
// ============================================================================
struct CliqueScratch {
  uint64_t* D;         // per CTA: d+ x ceil(d-/64) words
  int64_t d_words;     // capacity per CTA in words
  uint64_t* G;         // per CTA: the bit matrix and its companions when they exceed shared memory
  int64_t g_words;     // capacity per CTA in words
};

// Bytes of the clique pass's work space for out-degree d (B, K4 accumulators,
// hash of 2 x pow2(2d) ints, T values).  B rows are clique_stride(d) words
// apart: an odd stride, so the lanes of a warp reading word w of 32 different
// rows hit different shared-memory banks (an even stride of 2^k words puts them
// on 32 / 2^k banks).
static inline __host__ __device__ int clique_stride(int d) { return ((d + 63) >> 6) | 1; }
static constexpr int CLQ_MAX_WARPS = 16;         // warps of a CTA of the clique pass (512 threads)
static inline size_t clique_space(int d) {
  int h = 1;
  while (h < 2 * d) h <<= 1;
  return sizeof(uint64_t) * ((size_t)d * clique_stride(d) + d) + sizeof(int32_t) * (2 * (size_t)h) +
         sizeof(uint32_t) * d;
}

// B rows are symmetric (row a = every neighbour of v_a inside N+(x)); W words
// per row, RS words apart.
// with_k5: count the candidates c above b (for DBP); lane_k5: also count the
// 5-cliques here, one lane per edge (else k5_warp does it for the warp).
__device__ __forceinline__ void clique_edge(const uint64_t* B, int W, int RS, int a, int b, const uint64_t* Da,
                                            const uint64_t* Db, int DW, bool with_k5, bool lane_k5,
                                            unsigned long long& alpha_out, unsigned long long& beta_out,
                                            unsigned long long& k5_out, unsigned long long& above_out) {
  const uint64_t* ra = B + (int64_t)a * RS;
  const uint64_t* rb = B + (int64_t)b * RS;
  unsigned long long alpha = 0, k5 = 0, above = 0;
#pragma unroll 4
  for (int w = 0; w < W; ++w) alpha += __popcll(ra[w] & rb[w]);
  // 5-cliques with lowest vertex x and next two v_a < v_b: every c in the
  // common neighbourhood above b, then every l adjacent to a, b, c above c
  int w0 = with_k5 ? (b + 1) >> 6 : W;
  for (int w = w0; w < W; ++w) {
    uint64_t cm = ra[w] & rb[w];
    if (w == w0) cm &= ~0ull << ((b + 1) & 63);
    above += __popcll(cm);
    while (lane_k5 && cm) {
      int c = w * 64 + __ffsll((long long)cm) - 1;
      cm &= cm - 1;
      const uint64_t* rc = B + (int64_t)c * RS;
      int u = (c + 1) >> 6;
      if (u < W) k5 += __popcll(ra[u] & rb[u] & rc[u] & (~0ull << ((c + 1) & 63)));
      // the remaining words four at a time (independent loads in flight)
      for (++u; u + 4 <= W; u += 4)
        k5 += __popcll(ra[u] & rb[u] & rc[u]) + __popcll(ra[u + 1] & rb[u + 1] & rc[u + 1]) +
              __popcll(ra[u + 2] & rb[u + 2] & rc[u + 2]) + __popcll(ra[u + 3] & rb[u + 3] & rc[u + 3]);
      for (; u < W; ++u) k5 += __popcll(ra[u] & rb[u] & rc[u]);
    }
  }
  unsigned long long beta = 0;
  if (Da) {
#pragma unroll 8
    for (int w = 0; w < DW; ++w) beta += __popcll(Da[w] & Db[w]);
  }
  alpha_out = alpha;
  beta_out = beta;
  k5_out = k5;
  above_out = above;
}

// Position of the k-th (0-based) set bit of m (k < popc(m)).
__device__ __forceinline__ int select32(unsigned m, int k) {
  int pos = 0, c = __popc(m & 0xffffu);
  if (k >= c) { k -= c; m >>= 16; pos += 16; }
  c = __popc(m & 0xffu);
  if (k >= c) { k -= c; m >>= 8; pos += 8; }
  c = __popc(m & 0xfu);
  if (k >= c) { k -= c; m >>= 4; pos += 4; }
  c = __popc(m & 0x3u);
  if (k >= c) { k -= c; m >>= 2; pos += 2; }
  if (k >= (int)(m & 1u)) pos += 1;
  return pos;
}
__device__ __forceinline__ int select64(uint64_t x, int k) {
  const int c = __popc((unsigned)x);
  return k < c ? select32((unsigned)x, k) : 32 + select32((unsigned)(x >> 32), k - c);
}

// 5-cliques (Thm 14) of the edges (a, b) of G[N+(x)] that the lanes hold
// (want: an edge with at least two candidates), one edge at a time for the
// whole warp: the candidates c (common neighbours of v_a and v_b above b) are
// taken 32 at a time, lane k the k-th, and each lane counts the common
// neighbours of v_a, v_b and v_c above c.  Consecutive candidates lie in the
// same or neighbouring words, so the lanes' word loops nearly coincide.  The
// common neighbourhood of a and b goes to the warp's buffer mb (W <= 32 words).
__device__ __forceinline__ unsigned long long k5_warp(const uint64_t* B, int W, int RS, int a, int b_l, bool want_l,
                                                      uint64_t* mb) {
  const int lane = threadIdx.x & 31;
  const uint64_t* ra = B + (int64_t)a * RS;
  unsigned long long k5 = 0;
  unsigned todo = __ballot_sync(0xffffffffu, want_l);
  while (todo) {
    const int k = __ffs(todo) - 1;
    todo &= todo - 1;
    const int b = __shfl_sync(0xffffffffu, b_l, k);
    const uint64_t* rb = B + (int64_t)b * RS;
    const int w0 = (b + 1) >> 6;
    uint64_t m = 0;
    if (lane >= w0 && lane < W) {
      m = ra[lane] & rb[lane];
      if (lane == w0) m &= ~0ull << ((b + 1) & 63);
    }
    if (lane < W) mb[lane] = m;
    __syncwarp();
    const int cnt = __popcll(m);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    for (int t0 = 0; t0 < total; t0 += 32) {
      const int kth = t0 + lane;
      int wq = w0;                              // the word of candidate kth: words whose candidates all precede it
      for (int u = w0; u < W; ++u) wq += __shfl_sync(0xffffffffu, incl, u) <= kth ? 1 : 0;
      wq = min(wq, W - 1);
      const int before = __shfl_sync(0xffffffffu, incl, wq) - __shfl_sync(0xffffffffu, cnt, wq);
      if (kth < total) {
        const int c = wq * 64 + select64(mb[wq], kth - before);
        const uint64_t* rc = B + (int64_t)c * RS;
        int u = (c + 1) >> 6;
        unsigned long long part = 0;
        if (u < W) part = __popcll(mb[u] & rc[u] & (~0ull << ((c + 1) & 63)));
        for (++u; u + 4 <= W; u += 4)
          part += __popcll(mb[u] & rc[u]) + __popcll(mb[u + 1] & rc[u + 1]) + __popcll(mb[u + 2] & rc[u + 2]) +
                  __popcll(mb[u + 3] & rc[u + 3]);
        for (; u < W; ++u) part += __popcll(mb[u] & rc[u]);
        k5 += part;
      }
    }
    __syncwarp();                               // the buffer is read before the next edge writes it
  }
  return k5;
}

// Work-space layout of the CTA path: B (d x W u64), K4 accumulators (d u64),
// hash (2 x hcap ints), T of x's out-edges (d u32), in shared memory; for
// out-degrees whose bit matrix does not fit there (GLOBAL_B), the same layout
// in a per-CTA region of global memory (cs.G, cs.g_words words per CTA).
// A launch takes the items with dlo < d+ <= dmax and skips the others.
template <bool GLOBAL_B>
__global__ void k_clique_large(DevGraph g, const int32_t* items, int64_t nitems, unsigned long long* qctr,
                               const uint32_t* T, unsigned long long* K4e, AccSet acc, CliqueScratch cs,
                               int hash_cap, int dlo, int dmax, unsigned* status, bool with_k5) {
  extern __shared__ uint64_t smem64[];
  __shared__ u128 sh[32];
  __shared__ int64_t sh_item;
  __shared__ uint64_t s_mb[CLQ_MAX_WARPS][32];   // k5_warp's buffers
  const int RS_cap = clique_stride(dmax);
  uint64_t* B = GLOBAL_B ? cs.G + (int64_t)blockIdx.x * cs.g_words : smem64;   // dmax * RS_cap
  unsigned long long* k4x = (unsigned long long*)(B + (int64_t)dmax * RS_cap);  // dmax
  int32_t* hk = (int32_t*)(k4x + dmax);                        // hash_cap
  int32_t* hv = hk + hash_cap;                                 // hash_cap
  uint32_t* Tx = (uint32_t*)(hv + hash_cap);                   // dmax
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint64_t* D = cs.D + (int64_t)blockIdx.x * cs.d_words;
  const int ids[6] = {ACC_K4, ACC_N20, ACC_N10A, ACC_N16A, ACC_N21, ACC_DBP};
  LocalAcc<6> la;
  la.zero();
  while (true) {
    int64_t it = next_item(qctr, nitems, &sh_item);
    if (it < 0) break;
    int64_t x = items[it];
    int64_t o = g.op[x], ib = g.R[x];
    int d = (int)(g.R[x + 1] - o);
    int din = (int)(o - ib);
    if (d <= dlo || d > dmax) continue;        // the other launch's item
    int W = (d + 63) >> 6;
    const int RS = clique_stride(d);
    int DW = (din + 63) >> 6;
    bool use_beta = din > 0 && (int64_t)d * DW <= cs.d_words;
    if (din > 0 && !use_beta && threadIdx.x == 0) set_err(status, DEVERR_SCRATCH);
    int hsz = pow2_at_least(2 * d);
    PosHash H{hk, hv, hsz - 1};
    for (int i = threadIdx.x; i < hsz; i += blockDim.x) hk[i] = -1;
    for (int64_t i = threadIdx.x; i < (int64_t)d * RS; i += blockDim.x) B[i] = 0;
    for (int i = threadIdx.x; i < d; i += blockDim.x) { k4x[i] = 0; Tx[i] = T[o + i]; }
    if (use_beta)
      for (int64_t i = threadIdx.x; i < (int64_t)d * DW; i += blockDim.x) D[i] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < d; i += blockDim.x) H.insert(g.C[o + i], i);
    __syncthreads();
    // build B
    for (int a = wid; a < d; a += nw) {
      int32_t v = g.C[o + a];
      for (int64_t q = g.op[v] + lane; q < g.R[v + 1]; q += 32) {
        int b = H.find(g.C[q]);
        if (b >= 0) {
          atomicOr((unsigned long long*)&B[(int64_t)a * RS + (b >> 6)], 1ull << (b & 63));
          atomicOr((unsigned long long*)&B[(int64_t)b * RS + (a >> 6)], 1ull << (a & 63));
        }
      }
    }
    // build D: in-neighbour y (index k) sets bit k of D_a for every v_a in N+(y)
    if (use_beta) {
      for (int k = wid; k < din; k += nw) {
        int32_t y = g.C[ib + k];
        for (int64_t q = g.op[y] + lane; q < g.R[y + 1]; q += 32) {
          int a = H.find(g.C[q]);
          if (a >= 0) atomicOr((unsigned long long*)&D[(int64_t)a * DW + (k >> 6)], 1ull << (k & 63));
        }
      }
    }
    __syncthreads();
    unsigned long long dx = (unsigned long long)(g.R[x + 1] - g.R[x]);
    // edges (a, b) of G[N+(x)]: scan N+(v_a) again to get the slot of (v_a, v_b);
    // the lanes step together so that k5_warp can take the 5-cliques
    const bool warp_k5 = with_k5 && !GLOBAL_B && W <= 32 && nw <= CLQ_MAX_WARPS;
    for (int a = wid; a < d; a += nw) {
      int32_t v = g.C[o + a];
      unsigned long long dva = (unsigned long long)(g.R[v + 1] - g.R[v]);
      unsigned long long k4a = 0;
      const int64_t qe = g.R[v + 1];
      for (int64_t qb = g.op[v]; qb < qe; qb += 32) {
        const int64_t q = qb + lane;
        int b = -1;
        int32_t w = 0;
        if (q < qe) {
          w = g.C[q];
          b = H.find(w);
        }
        unsigned long long above = 0;
        if (b >= 0) {
          unsigned long long alpha, beta, k5;
          clique_edge(B, W, RS, a, b, use_beta ? D + (int64_t)a * DW : nullptr,
                      use_beta ? D + (int64_t)b * DW : nullptr, DW, with_k5, with_k5 && !warp_k5, alpha, beta, k5,
                      above);
          la.v[5] += ch2(above);                                  // directed bipyramids on this triangle
          unsigned long long dvb = (unsigned long long)(g.R[w + 1] - g.R[w]);
          unsigned long long tab = T[q], txa = Tx[a], txb = Tx[b];
          la.v[0] += alpha;                                       // 3 x K4
          la.v[1] += ch2(alpha + beta);                           // N20
          la.v[2] += (u128)(tab - 1) * (dx - 2) + (u128)(txb - 1) * (dva - 2) + (u128)(txa - 1) * (dvb - 2);   // N10
          la.v[3] += (u128)(txa - 1) * (txb - 1) + (u128)(txa - 1) * (tab - 1) + (u128)(txb - 1) * (tab - 1);  // N16
          la.v[4] += k5;                                          // N21 (zero when k5_warp counts them)
          if (alpha) {
            atomicAdd(&K4e[q], alpha);
            atomicAdd(&k4x[b], alpha);
            k4a += alpha;
          }
        }
        if (warp_k5) la.v[4] += k5_warp(B, W, RS, a, b, b >= 0 && above >= 2, s_mb[wid]);
      }
      k4a = warp_sum_u64(k4a);
      if (lane == 0 && k4a) atomicAdd(&k4x[a], k4a);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < d; i += blockDim.x)
      if (k4x[i]) atomicAdd(&K4e[o + i], k4x[i] / 2);
    block_item_flush(la, ids, acc, x, sh);
    __syncthreads();
  }
  final_flush(la, ids, acc, sh);
}

// Small out-neighbourhoods (d+ <= 32 and d- <= CLQ_WARP_DIN): one warp per
// vertex x, everything in the warp's shared memory.  Lane a holds v_a, the
// a-th vertex of N+(x); row a of the bit matrix of G[N+(x)] is one 64-bit word
// and D_a (the in-neighbours of x adjacent to v_a) at most CLQ_WARP_DIN / 64.
// The sums and per-edge counts are those of k_clique_large.
static constexpr int CLQ_WARP_DIN = 512;
static constexpr int CLQ_WARPS = 8;            // warps per block
static constexpr int CLQ_ILP = 4;

__global__ void __launch_bounds__(CLQ_WARPS * 32, 4) k_clique_warp(DevGraph g, const int32_t* items, int64_t nitems,
                                                                unsigned long long* qctr, const uint32_t* T,
                                                                unsigned long long* K4e, AccSet acc, bool with_k5) {
  __shared__ u128 sh[32];
  __shared__ int32_t sL[CLQ_WARPS][32];
  __shared__ uint32_t sT[CLQ_WARPS][32];
  __shared__ unsigned long long sB[CLQ_WARPS][32], sK[CLQ_WARPS][32];
  __shared__ unsigned long long sD[CLQ_WARPS][32][CLQ_WARP_DIN / 64];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  int32_t* L = sL[wl];
  unsigned long long* Bw = sB[wl];
  unsigned long long* K = sK[wl];
  const int ids[6] = {ACC_K4, ACC_N20, ACC_N10A, ACC_N16A, ACC_N21, ACC_DBP};
  LocalAcc<6> la;
  la.zero();
  // position of vertex key in N+(x) (sorted, padded with INT32_MAX), or -1
  auto find = [&](int32_t key) -> int {
    int lo = 0;
#pragma unroll
    for (int st = 16; st > 0; st >>= 1)
      if (L[lo + st] <= key) lo += st;
    return L[lo] == key ? lo : -1;
  };
  while (true) {
    unsigned long long it_l = 0;
    if (lane == 0) it_l = atomicAdd(qctr, 1ull);
    int64_t it = (int64_t)__shfl_sync(0xffffffffu, it_l, 0);
    if (it >= nitems) break;
    int64_t x = items[it];
    int64_t o = g.op[x], ib = g.R[x];
    int d = (int)(g.R[x + 1] - o);
    int din = (int)(o - ib);
    int DW = (din + 63) >> 6;
    int32_t va = lane < d ? g.C[o + lane] : 0x7fffffff;
    L[lane] = va;
    sT[wl][lane] = lane < d ? T[o + lane] : 0u;
    Bw[lane] = 0;
    K[lane] = 0;
    for (int w = 0; w < DW; ++w) sD[wl][lane][w] = 0;
    __syncwarp();
    // rows of G[N+(x)]: lane a scans N+(v_a) (everything there is above v_a)
    int64_t qa0 = 0, qa1 = 0;
    if (lane < d) {
      qa0 = g.op[va];
      qa1 = g.R[va + 1];
    }
    for (int64_t q = qa0; q < qa1; q += CLQ_ILP) {
      int32_t ww[CLQ_ILP];
#pragma unroll
      for (int u = 0; u < CLQ_ILP; ++u) ww[u] = q + u < qa1 ? g.C[q + u] : 0x7fffffff;
#pragma unroll
      for (int u = 0; u < CLQ_ILP; ++u) {
        int b = ww[u] == 0x7fffffff ? -1 : find(ww[u]);
        if (b >= 0) {
          atomicOr(&Bw[lane], 1ull << b);
          atomicOr(&Bw[b], 1ull << lane);
        }
      }
    }
    // D: in-neighbour y (index k) marks bit k of D_a for every v_a in N+(y)
    for (int k = lane; k < din; k += 32) {
      int32_t y = g.C[ib + k];
      int64_t q1 = g.R[y + 1];
      for (int64_t q = g.op[y]; q < q1; q += CLQ_ILP) {
        int32_t ww[CLQ_ILP];
#pragma unroll
        for (int u = 0; u < CLQ_ILP; ++u) ww[u] = q + u < q1 ? g.C[q + u] : 0x7fffffff;
#pragma unroll
        for (int u = 0; u < CLQ_ILP; ++u) {
          int a = ww[u] == 0x7fffffff ? -1 : find(ww[u]);
          if (a >= 0) atomicOr(&sD[wl][a][k >> 6], 1ull << (k & 63));
        }
      }
    }
    __syncwarp();
    // edges (a, b) of G[N+(x)], a < b: lane a scans N+(v_a) again for the slot
    if (lane < d) {
      unsigned long long dx = (unsigned long long)(g.R[x + 1] - g.R[x]);
      unsigned long long dva = (unsigned long long)(g.R[va + 1] - g.R[va]);
      unsigned long long ra = Bw[lane], k4a = 0, txa = sT[wl][lane];
      for (int64_t q = qa0; q < qa1; ++q) {
        int32_t w = g.C[q];
        int b = find(w);
        if (b < 0) continue;
        unsigned long long cm = ra & Bw[b];
        unsigned long long alpha = (unsigned long long)__popcll(cm), beta = 0, k5 = 0;
        for (int t = 0; t < DW; ++t) beta += (unsigned long long)__popcll(sD[wl][lane][t] & sD[wl][b][t]);
        // 5-cliques at the three lowest vertices x, v_a, v_b: every c in the
        // common neighbourhood above b, then every l adjacent to a, b, c above c
        unsigned long long cm2 = with_k5 ? cm & (~0ull << (b + 1)) : 0ull;
        la.v[5] += ch2((unsigned long long)__popcll(cm2));        // directed bipyramids on this triangle
        while (cm2) {
          int c = __ffsll((long long)cm2) - 1;
          cm2 &= cm2 - 1;
          k5 += (unsigned long long)__popcll(cm & Bw[c] & (~0ull << (c + 1)));
        }
        unsigned long long dvb = (unsigned long long)(g.R[w + 1] - g.R[w]);
        unsigned long long tab = T[q], txb = sT[wl][b];
        la.v[0] += alpha;                                         // 3 x K4
        la.v[1] += ch2(alpha + beta);                             // N20
        la.v[2] += (u128)(tab - 1) * (dx - 2) + (u128)(txb - 1) * (dva - 2) + (u128)(txa - 1) * (dvb - 2);   // N10
        la.v[3] += (u128)(txa - 1) * (txb - 1) + (u128)(txa - 1) * (tab - 1) + (u128)(txb - 1) * (tab - 1);  // N16
        la.v[4] += k5;                                            // N21
        if (alpha) {
          atomicAdd(&K4e[q], alpha);
          atomicAdd(&K[b], alpha);
          k4a += alpha;
        }
      }
      if (k4a) atomicAdd(&K[lane], k4a);
    }
    __syncwarp();
    if (lane < d && K[lane]) atomicAdd(&K4e[o + lane], K[lane] / 2);
    warp_item_flush(la, ids, acc, x);
    __syncwarp();
  }
  final_flush(la, ids, acc, sh);
}

// Counters of the 4-cycle, pair and 5-cycle sweeps, tagged with the item they count
// for.  Before each increment a fire-and-forget atomicMax with the current tag
// turns an entry left by an earlier item into a zero count of the current one
// (a CTA's tags grow with the items it takes), so nothing is cleared between
// items and no list of touched entries is kept.  Every count at j (w(i,j),
// W(i,j) or w'(i,j)) is at most d(j), so the ranks below jbig, the first of degree
// >= 2^16, keep (tag << 16) | count in 32-bit words; the few ranks from jbig on
// keep (tag << 32) | count in a 64-bit side array.
struct TagScratch {
  uint32_t* w;              // per CTA: jbig words
  unsigned long long* wb;   // per CTA: n - jbig words
  int64_t jbig, n;
};

template <bool BIG>   // BIG: some rank has degree >= 2^16 (jbig < n)
struct TaggedCounters {
  static constexpr uint32_t TAG_MAX = 0xffffu;   // largest tag of the 32-bit words
  uint32_t* w;
  unsigned long long* wb;
  int32_t jbig;
  uint32_t tag;
  __device__ TaggedCounters(const TagScratch& ts) : TaggedCounters(ts, blockIdx.x) {}
  // the array of index `arr` (one per CTA, or one per cluster of CTAs)
  __device__ TaggedCounters(const TagScratch& ts, int64_t arr) {
    w = ts.w + arr * ts.jbig;
    wb = ts.wb + arr * (ts.n - ts.jbig);
    jbig = (int32_t)ts.jbig;
    tag = 0;
  }
  __device__ __forceinline__ uint32_t inc(int32_t j) const {
    if (!BIG || j < jbig) {
      atomicMax(&w[j], tag << 16);
      return atomicAdd(&w[j], 1u) & 0xffffu;
    }
    unsigned long long* p = &wb[j - jbig];
    atomicMax(p, (unsigned long long)tag << 32);
    return (uint32_t)atomicAdd(p, 1ull);
  }
  __device__ __forceinline__ void add(int32_t j) const {    // the same without the old value
    if (!BIG || j < jbig) {
      atomicMax(&w[j], tag << 16);
      atomicAdd(&w[j], 1u);
    } else {
      unsigned long long* p = &wb[j - jbig];
      atomicMax(p, (unsigned long long)tag << 32);
      atomicAdd(p, 1ull);
    }
  }
  __device__ __forceinline__ uint32_t get(int32_t j) const {
    if (!BIG || j < jbig) {
      uint32_t v = w[j];
      return (v >> 16) == tag ? (v & 0xffffu) : 0u;
    }
    unsigned long long v = wb[j - jbig];
    return (uint32_t)(v >> 32) == tag ? (uint32_t)v : 0u;
  }
  // get() for an array that CTAs of other SMs increment: read at L2 (the
  // increments are performed there; an L1 copy could be stale)
  __device__ __forceinline__ uint32_t get_l2(int32_t j) const {
    if (!BIG || j < jbig) {
      uint32_t v = __ldcg(&w[j]);
      return (v >> 16) == tag ? (v & 0xffffu) : 0u;
    }
    unsigned long long v = __ldcg(&wb[j - jbig]);
    return (uint32_t)(v >> 32) == tag ? (uint32_t)v : 0u;
  }
  // next item: a new tag, or zeroed counters once the tags are used up (all
  // threads of the CTA call it; returns true when it zeroed, and a barrier
  // must then publish the zeros before the next increment)
  __device__ __forceinline__ bool next(int64_t n) { return next_shared(n, 0, 1); }
  // the same for an array shared by the `parts` CTAs of a cluster: CTA
  // `part` zeroes its share, and a cluster barrier must follow a zeroing
  __device__ __forceinline__ bool next_shared(int64_t n, unsigned part, unsigned parts) {
    if (++tag <= TAG_MAX) return false;
    const int64_t t0 = (int64_t)part * blockDim.x + threadIdx.x, st = (int64_t)parts * blockDim.x;
    for (int64_t t = t0; t < jbig; t += st) w[t] = 0;
    if (BIG)
      for (int64_t t = t0; t < n - jbig; t += st) wb[t] = 0;
    tag = 1;
    return true;
  }
};

// ---------------------------------------------------------------- clusters
// Thread-block cluster helpers (PTX special registers and the hardware
// cluster barrier).  A kernel launched without a cluster dimension runs as
// clusters of one CTA, for which these reduce to the CTA itself.
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_index() {
  unsigned r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
// every thread of every CTA of the cluster; orders memory at cluster scope
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// 64-bit value at the address of `p` in the shared memory of cluster CTA `rank`
__device__ __forceinline__ long long ld_cluster_s64(const void* p, unsigned rank) {
  unsigned a = (unsigned)__cvta_generic_to_shared(p), ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  long long v;
  asm volatile("ld.shared::cluster.s64 %0, [%1];" : "=l"(v) : "r"(ra) : "memory");
  return v;
}

// ============================================================================
// Thm 5: 4-cycles.  For the highest vertex i and each j < i,
// w(i,j) = |{k in N(i) cap N(j) : k < i}| (out-wedges and in-out wedges);
// C4 = sum C(w,2).  Per element: every wedge i - k - j adds w-1 to edges
// (i,k), (k,j) and vertex k; every j adds C(w,2) to vertices i and j.
// CTA per i, dense per-CTA counters over j with a touched list.
// ============================================================================
#ifndef ESC_SWEEP_ILP
#define ESC_SWEEP_ILP 8
#endif
static constexpr int SWEEP_ILP = ESC_SWEEP_ILP;   // independent accesses in flight per lane (4- and 5-cycles)
// Independent accesses in flight per lane of the pair sweep (8 at 64 registers: R-MAT 22 pairs 14.4 -> 13.8 s).
#ifndef ESC_PAIR_ILP
#define ESC_PAIR_ILP 8
#endif
static constexpr int PAIR_ILP = ESC_PAIR_ILP;
static_assert(PAIR_ILP >= 1 && PAIR_ILP <= 8, "pair_range sums at most 8 values of C(old, 2) in 64 bits");

struct SweepScratch {
  uint32_t* cnt;       // per CTA: n counters (kept zero between items)
  int32_t* touched;    // per CTA: n entries
  uint32_t* cnt2;      // second counter array (5-cycles)
  int32_t* touched2;
  unsigned* ntouched;  // per CTA: 2 counters
  int64_t n;
};

template <bool BIG>
__global__ void k_cycles4(DevGraph g, unsigned long long* qctr, TagScratch ts, unsigned long long* C4raw,
                          unsigned long long* C4v, AccSet acc, Owner own) {
  __shared__ u128 sh[32];
  __shared__ int64_t sh_item;
  TaggedCounters<BIG> w(ts);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  u128 c4sum = 0;
  while (true) {
    int64_t it = next_item(qctr, own.count(g.n), &sh_item);
    if (it < 0) break;
    int64_t i = own.item(g.n, it);
    int64_t b0 = g.R[i], e0 = g.op[i];
    if (e0 == b0) continue;           // no lower neighbours
    if (w.next(g.n)) __syncthreads();
    // pass 1: wedge counts w(i, j).  C(w, 2) at j is the sum of the values the
    // increments of j return, so each increment adds its old value to C4(j)
    // at once and no second pass over the touched j's is needed.  The lists
    // N(k) below i are fetched 32 per warp (lane l the l-th), SWEEP_ILP
    // entries in flight per lane.
    u128 mine = 0;
    for (int64_t pbase = b0 + wid; pbase < e0; pbase += (int64_t)nw * 32) {
      int64_t p = pbase + (int64_t)lane * nw;
      int64_t kb_l = 0, ke_l = 0;
      if (p < e0) {
        kb_l = g.R[g.C[p]];
        ke_l = g.rev[p];                        // N(k) below i ends at the slot of i
      }
      int kmax = (int)min((int64_t)32, (e0 - pbase + nw - 1) / nw);
      for (int kk = 0; kk < kmax; ++kk) {
        int64_t kb = __shfl_sync(0xffffffffu, kb_l, kk), ke = __shfl_sync(0xffffffffu, ke_l, kk);
        for (int64_t q = kb + lane; q < ke; q += 32 * SWEEP_ILP) {
          int32_t jj[SWEEP_ILP];
          uint32_t oo[SWEEP_ILP];
#pragma unroll
          for (int u = 0; u < SWEEP_ILP; ++u) jj[u] = q + 32 * u < ke ? g.C[q + 32 * u] : -1;
#pragma unroll
          for (int u = 0; u < SWEEP_ILP; ++u) oo[u] = jj[u] >= 0 ? w.inc(jj[u]) : 0u;
#pragma unroll
          for (int u = 0; u < SWEEP_ILP; ++u)
            if (oo[u]) {
              atomicAdd(&C4v[jj[u]], (unsigned long long)oo[u]);
              mine += oo[u];
            }
        }
      }
    }
    u128 tot = block_sum_u128(mine, sh);        // its barriers also end pass 1
    if (threadIdx.x == 0) {
      if (tot) atomicAdd(&C4v[i], (unsigned long long)tot);
      if (acc.vg) acc_add(acc_of(acc, i), ACC_C4, tot);
      else c4sum += tot;
    }
    // pass 3: per-edge counts, the lists fetched as in pass 1
    for (int64_t pbase = b0 + wid; pbase < e0; pbase += (int64_t)nw * 32) {
      int64_t p_l = pbase + (int64_t)lane * nw;
      int64_t kb_l = 0, ke_l = 0;
      int32_t k_l = 0;
      if (p_l < e0) {
        k_l = g.C[p_l];
        kb_l = g.R[k_l];
        ke_l = g.rev[p_l];
      }
      int kmax = (int)min((int64_t)32, (e0 - pbase + nw - 1) / nw);
      for (int kk = 0; kk < kmax; ++kk) {
        int64_t kb = __shfl_sync(0xffffffffu, kb_l, kk), ke = __shfl_sync(0xffffffffu, ke_l, kk);
        unsigned long long sk = 0;
        for (int64_t q = kb + lane; q < ke; q += 32 * SWEEP_ILP) {
          int32_t jj[SWEEP_ILP];
#pragma unroll
          for (int u = 0; u < SWEEP_ILP; ++u) jj[u] = q + 32 * u < ke ? g.C[q + 32 * u] : -1;
#pragma unroll
          for (int u = 0; u < SWEEP_ILP; ++u) {
            if (jj[u] < 0) continue;
            unsigned long long c = w.get(jj[u]) - 1;
            if (c) { atomicAdd(&C4raw[q + 32 * u], c); sk += c; }
          }
        }
        sk = warp_sum_u64(sk);
        int32_t k = __shfl_sync(0xffffffffu, k_l, kk);
        if (lane == 0 && sk) {
          atomicAdd(&C4raw[pbase + (int64_t)kk * nw], sk);
          atomicAdd(&C4v[k], sk);
        }
      }
    }
    __syncthreads();                            // the next item's counts must not meet these reads
  }
  if (threadIdx.x == 0 && !acc.vg) acc_add(acc.base, ACC_C4, c4sum);
}

// Per-edge common-neighbour lists (built by the triangle-list pass).
struct TriLists {
  const int64_t* off;    // per slot: start of the edge's id list (both slots of an edge share it)
  const int32_t* U;      // sorted common-neighbour ids
  const int64_t* offp;   // per slot: start of the slot's position list
  const int32_t* P;      // per slot (u -> v): positions in row u of the common neighbours, ascending
};

// ============================================================================
// Thm 11/12: N13 = sum_{j<i} C(W(i,j), 3) and
// N17 = sum_{j<i} (W(i,j) - 2) cc(i,j), cc = edges inside N(i) cap N(j).
// W(i,.) from every wedge i - c - j (c in N(i), j in N(c), j < i); C(W,3) is
// accumulated on the fly as the sum of C(old, 2) over the increments.  The cc
// term is gathered per diamond: for each triangle {i, x, y} (x < y, y reached
// through the position list of (x, i), so its slot in row x is direct) and each
// j in N(x) cap N(y) below i, add W(i,j) - 2 (Thm 12's enumeration through the
// per-edge triangle lists).
// ============================================================================


// Items are split by their wedge count w_i = sum_{c in N(i)} |N(c) below i|
// (the number of W(i, .) increments, so also a bound on the distinct j):
//   light  (w_i <= PH_SMALL_W): one CTA, W(i, .) in a shared-memory hash table
//   medium (w_i <= PH_LARGE_W): one CTA, a larger shared-memory hash table
//   heavy:                      a cluster of CTAs shares one tagged counter
//                               array in global memory, and only as many
//                               clusters run as keep their arrays within L2
static constexpr int PH_SMALL_SLOTS = 4096, PH_SMALL_THREADS = 256;
static constexpr int PH_LARGE_SLOTS = 16384, PH_LARGE_THREADS = 512;
static constexpr int64_t PH_SMALL_W = PH_SMALL_SLOTS / 2;     // load factor <= 1/2
static constexpr int64_t PH_LARGE_W = PH_LARGE_SLOTS / 2;

// w_i of every vertex with degree >= 2, appended to the list of its class
// (roughly by decreasing rank, so the heaviest items come first)
// Also the largest common-neighbour list (triangles on one edge) into cnts[7].
__global__ void k_pair_classify(DevGraph g, const uint32_t* T, int32_t* lists, unsigned long long* cnts,
                                long long w_small, long long w_large, Owner own) {
  int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t k = warp; k < g.n; k += nwarps) {
    int64_t i = g.n - 1 - k;
    int64_t b0 = g.R[i], e0 = g.R[i + 1];
    unsigned tmax = 0;
    for (int64_t p = b0 + lane; p < e0; p += 32) tmax = max(tmax, T[p]);
    tmax = __reduce_max_sync(0xffffffffu, tmax);
    if (lane == 0 && tmax) atomicMax(&cnts[7], (unsigned long long)tmax);
    if (e0 - b0 < 2 || !own.owns(i)) continue;
    unsigned long long w = 0;
    for (int64_t p = b0 + lane; p < e0; p += 32) w += (unsigned long long)(g.rev[p] - g.R[g.C[p]]);
    w = warp_sum_u64(w);
    w = __shfl_sync(0xffffffffu, w, 0);
    if (w == 0) continue;
    int cls = (long long)w <= w_small ? 0 : ((long long)w <= w_large ? 1 : 2);
    if (lane == 0) {
      lists[(int64_t)cls * g.n + (int64_t)atomicAdd(&cnts[cls], 1ull)] = (int32_t)i;
      if (cls == 2) atomicMax(&cnts[6], w);    // the largest item, for the task buffers
    }
  }
}

// Open addressing in shared memory (keys -1 = empty), linear probing.  At most
// half the slots are ever used, so a probe sequence ends within the table.
template <int SLOTS>
__device__ __forceinline__ int ph_insert(int32_t* hk, int32_t j) {
  constexpr int LOG = __builtin_ctz(SLOTS);
  uint32_t sl = ((uint32_t)j * 0x9E3779B1u) >> (32 - LOG);
  volatile int32_t* vk = hk;
  for (int probe = 0; probe < SLOTS; ++probe) {
    int32_t k = vk[sl];
    if (k == j) return (int)sl;
    if (k == -1) {
      int32_t old = atomicCAS(&hk[sl], -1, j);
      if (old == -1 || old == j) return (int)sl;
    }
    sl = (sl + 1) & (SLOTS - 1);
  }
  return -1;
}
template <int SLOTS>
__device__ __forceinline__ int ph_find(const int32_t* hk, int32_t j) {
  constexpr int LOG = __builtin_ctz(SLOTS);
  uint32_t sl = ((uint32_t)j * 0x9E3779B1u) >> (32 - LOG);
  for (int probe = 0; probe < SLOTS; ++probe) {
    int32_t k = hk[sl];
    if (k == j) return (int)sl;
    if (k == -1) return -1;
    sl = (sl + 1) & (SLOTS - 1);
  }
  return -1;
}

// The two passes of one item i, shared by both forms of the sweep.  Warp
// `gw` of `gnw` (the warps of a CTA, or of a whole cluster) takes its share:
//   inc(j) counts the wedge i - c - j and returns W(i,j) before it;
//   get(j) returns W(i,j) after every increment.
// Pass 1: W(i,.) from every wedge i - c - j (c in N(i), j in N(c), j < i);
// C(W,3) is accumulated on the fly as the sum of C(old, 2).  The lists N(c) are
// fetched 32 per warp (lane k the k-th) and every lane keeps PAIR_ILP
// independent loads and counter operations in flight.
static constexpr int PAIR_TASK = 32 * 4 * 4;   // lists longer than this are shared as tasks of this size
#ifndef ESC_PAIR_SHORT
#define ESC_PAIR_SHORT 32
#endif
static constexpr int PAIR_SHORT = ESC_PAIR_SHORT;   // lists up to this long are walked by one lane (32: Chung-Lu pairs 40.8 -> 40.2 ms against 64)

// A 128-bit sum of 64-bit terms kept as a 64-bit word and a carry count:
// two 64-bit operations per term in the inner loops instead of a 128-bit add.
struct Sum128 {
  unsigned long long lo = 0;
  unsigned hi = 0;
  __device__ __forceinline__ void add(unsigned long long x) {
    lo += x;
    hi += lo < x ? 1u : 0u;
  }
  __device__ __forceinline__ u128 get() const { return ((u128)hi << 64) + lo; }
};

// C(old, 2) of a counter value below 2^32, exactly in 64 bits (zero for 0 and 1).
__device__ __forceinline__ unsigned long long pair_c2(uint32_t old) {
  return ((unsigned long long)old * (old - 1u)) >> 1;           // old = 0: 0 x (2^32 - 1)
}

// Increments for the entries C[cb .. ce) (one warp, PAIR_ILP loads per lane in
// flight).  Offsets within the list are 32-bit: a row has fewer than 2^31 entries.
template <class Inc>
__device__ __forceinline__ u128 pair_range(const DevGraph& g, int64_t cb, int64_t ce, Inc&& inc) {
  const int lane = threadIdx.x & 31;
  const int32_t* L = g.C + cb;
  const int len = (int)(ce - cb);
  Sum128 n13;
  for (int q = lane; q < len; q += 32 * PAIR_ILP) {
    int32_t jj[PAIR_ILP];
#pragma unroll
    for (int u = 0; u < PAIR_ILP; ++u) jj[u] = q + 32 * u < len ? __ldcs(L + q + 32 * u) : -1;
    unsigned long long blk = 0;                 // at most 8 terms below 2^61 (a count is below 2^31)
#pragma unroll
    for (int u = 0; u < PAIR_ILP; ++u)
      if (jj[u] >= 0) blk += pair_c2(inc(jj[u]));
    n13.add(blk);
  }
  return n13.get();
}

// defer(cb, ce) may take a long list off the warp (returning true) so that
// every warp shares it later; it is called by all 32 lanes with the same range.
template <class Inc, class Defer>
__device__ __forceinline__ u128 pair_wedges(const DevGraph& g, int64_t b0, int64_t e0, int64_t gw, int64_t gnw,
                                            Inc&& inc, Defer&& defer) {
  const int lane = threadIdx.x & 31;
  u128 n13 = 0;
  for (int64_t pbase = b0 + gw; pbase < e0; pbase += gnw * 32) {
    int64_t p = pbase + (int64_t)lane * gnw;
    int64_t cb_l = 0, ce_l = 0;
    if (p < e0) {
      int32_t c = g.C[p];
      cb_l = g.R[c];
      ce_l = g.rev[p];                          // N(c) below i ends at the slot of i
    }
    // short lists: each lane its own; the others one at a time by the warp
    if (ce_l - cb_l <= PAIR_SHORT) {
      const int32_t* L = g.C + cb_l;
      const int len = (int)(ce_l - cb_l);
      Sum128 sh13;
      for (int q = 0; q < len; q += 4) {
        int32_t jj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) jj[u] = q + u < len ? __ldcs(L + q + u) : -1;
        unsigned long long blk = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (jj[u] >= 0) blk += pair_c2(inc(jj[u]));
        sh13.add(blk);
      }
      n13 += sh13.get();
    }
    unsigned longm = __ballot_sync(0xffffffffu, ce_l - cb_l > PAIR_SHORT);
    while (longm) {
      const int k = __ffs(longm) - 1;
      longm &= longm - 1;
      int64_t cb = __shfl_sync(0xffffffffu, cb_l, k), ce = __shfl_sync(0xffffffffu, ce_l, k);
      if (ce - cb > PAIR_TASK && defer(cb, ce)) continue;
      n13 += pair_range(g, cb, ce, inc);
    }
  }
  return n13;
}

// Long lists split into tasks of PAIR_TASK entries, shared by all warps of a
// CTA or cluster: per work group a task array (entry ranges of C) and a count.
struct PairTasks {
  long long* q;             // per group: cap x (begin, end)
  unsigned long long* n;    // per group: number of tasks (zero between items)
  int64_t cap;              // tasks per group
};

// Appends the tasks of list [cb, ce) to group `grp`; false if they do not fit
// (the caller then counts the list itself).  All 32 lanes call it.
__device__ __forceinline__ bool pair_defer(const PairTasks& pt, int64_t grp, int64_t cb, int64_t ce) {
  const int lane = threadIdx.x & 31;
  const long long nt = (ce - cb + PAIR_TASK - 1) / PAIR_TASK;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(&pt.n[grp], (unsigned long long)nt);
  base = __shfl_sync(0xffffffffu, base, 0);
  if ((long long)base + nt > pt.cap) return false;   // never: sized by the largest item
  long long* q = pt.q + 2 * (grp * pt.cap + (long long)base);
  for (long long t = lane; t < nt; t += 32) {
    long long a = cb + t * PAIR_TASK;
    q[2 * t] = a;
    q[2 * t + 1] = min((long long)ce, a + PAIR_TASK);
  }
  return true;
}

// The tasks of group `grp`, task t taken by warp t mod gnw.
// nt: the group's task count, read after the barrier that ends the appends
template <class Inc>
__device__ __forceinline__ u128 pair_run_tasks(const DevGraph& g, const PairTasks& pt, int64_t grp,
                                               unsigned long long nt, int64_t gw, int64_t gnw, Inc&& inc) {
  nt = min(nt, (unsigned long long)pt.cap);
  const long long* q = pt.q + 2 * grp * pt.cap;
  u128 n13 = 0;
  for (unsigned long long t = (unsigned long long)gw; t < nt; t += (unsigned long long)gnw)
    n13 += pair_range(g, __ldcg(&q[2 * t]), __ldcg(&q[2 * t + 1]), inc);
  return n13;
}

// Pass 2: the cc term per diamond with tip i.  For each x in N(i), the
// triangles {i, x, y} with y above x are a suffix of the position list of
// slot (x -> i); the common-neighbour list of (x, y) is sorted, so the j
// below i are a prefix of it; each adds W(i,j) - 2 (Thm 12's enumeration
// through the per-edge triangle lists).
// The diamonds of one chunk of at most 32 triangles {i, x, y}: positions
// [r0, r1) of the position list of slot (x -> i), x = C[p] (lane k takes the
// k-th y; the whole warp then walks each y's common-neighbour list).
template <class Get>
__device__ __forceinline__ u128 pair_diamond_chunk(const DevGraph& g, const TriLists& tl3, const uint32_t* T,
                                                   int64_t i, int64_t xb, int64_t r0, int64_t r1, Get&& get) {
  const int lane = threadIdx.x & 31;
  const int32_t i32 = (int32_t)i;
  Sum128 n17;
  int64_t r = r0 + lane;
  int64_t vb_l = 0;
  uint32_t len_l = 0;
  if (r < r1) {
    int64_t sxy = xb + tl3.P[r];                // slot (x -> y)
    vb_l = tl3.off[sxy];
    len_l = T[sxy];
  }
  // short lists: each lane walks its own, a few entries in flight, until it
  // passes i (no entry loaded beyond the next few); long ones: the whole warp
  // on one list at a time.  Each term W(i,j) - 2 is below 2^32; a lane adds at
  // most 2^26 of them per list into 64 bits before the carry-counted sum.
  if (r < r1 && len_l <= PAIR_SHORT) {
    const int32_t* L = tl3.U + vb_l;
    const int len = (int)len_l;
    unsigned long long part = 0;
    for (int q = 0; q < len; q += 4) {
      int32_t jj[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) jj[u] = q + u < len ? __ldcs(L + q + u) : 0x7fffffff;
      bool past = false;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (jj[u] < i32) part += get(jj[u]) - 2u;
        else past = true;
      }
      if (past) break;
    }
    n17.add(part);
  }
  // long lists: each lane first finds how many entries of its list lie below
  // i (i is in the list: a binary search), then the warp reads exactly those,
  // one list at a time, in blocks of 32 x PAIR_ILP entries and then 4, 2, 1
  // and a last partial group of 32, so that no slot past the prefix is issued.
  const bool lng = r < r1 && len_l > PAIR_SHORT;
  int pre_l = 0;
  if (lng) {
    const int32_t* L = tl3.U + vb_l;
    int lo = 0, hi = (int)len_l;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(L + mid) < i32) lo = mid + 1;
      else hi = mid;
    }
    pre_l = lo;
  }
  unsigned longm = __ballot_sync(0xffffffffu, pre_l > 0);
  while (longm) {
    const int k = __ffs(longm) - 1;
    longm &= longm - 1;
    const int32_t* L = tl3.U + __shfl_sync(0xffffffffu, vb_l, k) + lane;
    const int pre = __shfl_sync(0xffffffffu, pre_l, k);
    unsigned long long part = 0;             // x, y are common neighbours of i and every j read here
    int sb = 0;
    for (; sb + 32 * PAIR_ILP <= pre; sb += 32 * PAIR_ILP) {
      int32_t jj[PAIR_ILP];
#pragma unroll
      for (int u = 0; u < PAIR_ILP; ++u) jj[u] = __ldcs(L + sb + 32 * u);
#pragma unroll
      for (int u = 0; u < PAIR_ILP; ++u) part += get(jj[u]) - 2u;
    }
#pragma unroll
    for (int gsz = PAIR_ILP / 2; gsz >= 1; gsz >>= 1) {
      if (sb + 32 * gsz <= pre) {
        int32_t jj[PAIR_ILP / 2];
#pragma unroll
        for (int u = 0; u < gsz; ++u) jj[u] = __ldcs(L + sb + 32 * u);
#pragma unroll
        for (int u = 0; u < gsz; ++u) part += get(jj[u]) - 2u;
        sb += 32 * gsz;
      }
    }
    if (sb + lane < pre) part += get(__ldcs(L + sb)) - 2u;
    n17.add(part);
  }
  return n17.get();
}

// The triangles {i, x, y} with y above x of slot p = (i -> x): positions
// [r0, r1) of the position list of slot (x -> i); r0 = r1 if there are none.
__device__ __forceinline__ void pair_tri_range(const DevGraph& g, const TriLists& tl3, const uint32_t* T, int64_t p,
                                               int64_t& xb, int64_t& r0, int64_t& r1) {
  int32_t x = g.C[p];
  xb = g.R[x];
  int32_t xo = (int32_t)(g.op[x] - xb);         // positions >= xo in row x are above x
  int64_t rp_ = g.rev[p];                       // slot (x -> i)
  int64_t yb = tl3.offp[rp_];
  r1 = yb + T[rp_];
  r0 = lower_bound_i32(tl3.P, yb, r1, xo);
}

template <class Get>
__device__ __forceinline__ u128 pair_diamonds(const DevGraph& g, const TriLists& tl3, const uint32_t* T, int64_t i,
                                              int64_t b0, int64_t e0, int64_t gw, int64_t gnw, Get&& get) {
  u128 n17 = 0;
  for (int64_t p = b0 + gw; p < e0; p += gnw) {
    if (T[p] == 0) continue;
    int64_t xb, r0, r1;
    pair_tri_range(g, tl3, T, p, xb, r0, r1);
    for (int64_t rb = r0; rb < r1; rb += 32) n17 += pair_diamond_chunk(g, tl3, T, i, xb, rb, min(rb + 32, r1), get);
  }
  return n17;
}

// Light and medium items: one CTA per item, W(i, .) in a shared-memory hash
// table (SLOTS keys and counts) that is cleared after every item.
template <int SLOTS>
__global__ void k_pairs_hash(DevGraph g, const int32_t* items, int64_t nitems, unsigned long long* qctr,
                             TriLists tl3, const uint32_t* T, AccSet acc, unsigned* status) {
  extern __shared__ int32_t ph_smem[];
  int32_t* hk = ph_smem;
  uint32_t* hv = (uint32_t*)(ph_smem + SLOTS);
  __shared__ u128 sh[32];
  __shared__ int64_t sh_item;
  const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int ids[2] = {ACC_N13, ACC_N17};
  LocalAcc<2> la;
  la.zero();
  for (int t = threadIdx.x; t < SLOTS; t += blockDim.x) { hk[t] = -1; hv[t] = 0u; }
  while (true) {
    int64_t it = next_item(qctr, nitems, &sh_item);     // its barriers publish the cleared table
    if (it < 0) break;
    const int64_t i = items[it];
    const int64_t b0 = g.R[i], e0 = g.R[i + 1];
    u128 n13 = pair_wedges(g, b0, e0, wid, nw, [&](int32_t j) -> uint32_t {
      int sl = ph_insert<SLOTS>(hk, j);
      if (sl < 0) { set_err(status, DEVERR_SCRATCH); return 0u; }
      return atomicAdd(&hv[sl], 1u);
    }, [](int64_t, int64_t) { return false; });
    __syncthreads();
    u128 n17 = pair_diamonds(g, tl3, T, i, b0, e0, wid, nw, [&](int32_t j) -> uint32_t {
      int sl = ph_find<SLOTS>(hk, j);
      if (sl < 0) { set_err(status, DEVERR_SCRATCH); return 2u; }
      return hv[sl];
    });
    __syncthreads();
    for (int t = threadIdx.x; t < SLOTS; t += blockDim.x) { hk[t] = -1; hv[t] = 0u; }
    la.v[0] += n13;
    la.v[1] += n17;
    block_item_flush(la, ids, acc, i, sh);
  }
  final_flush(la, ids, acc, sh);
}

// Heavy items: all CTAs of a cluster work on one item at a time, with one
// tagged counter array per cluster (index %clusterid.x).  CTA 0 of the
// cluster takes the next item from the queue and the others read it from its
// shared memory; two cluster barriers per item order the increments before
// the reads and the reads before the next item's increments.
// Lists longer than PAIR_TASK entries are cut into tasks that every warp of
// the cluster shares after a barrier, so one hub's list does not hold the
// cluster back.
//
// With clusters of one CTA, the counters of the ranks [wlo, jbig) -- the top
// ranks below the 64-bit side array, where nearly all the diamond reads and a
// good share of the increments land (measured: the top 16K ranks take 94% of
// the diamond reads on the Chung-Lu workload, the top 64K 98% on R-MAT scale
// 20) -- live in shared memory as 16-bit counts, two to a word, cleared for
// every item (a count there is at most the rank's degree, below 2^16).
template <bool BIG, int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) k_pairs_grp(DevGraph g, const int32_t* items,
                                                                         int64_t nitems, unsigned long long* qctr,
                                                                         TagScratch ts, TriLists tl3,
                                                                         const uint32_t* T, AccSet acc,
                                                                         PairTasks pt, int64_t wlo, int win_words) {
  extern __shared__ uint32_t win[];
  __shared__ u128 sh[32];
  __shared__ long long sh_item;
  const unsigned crank = cluster_rank(), csize = cluster_size();
  const int64_t grp = (int64_t)cluster_index();
  TaggedCounters<BIG> w(ts, grp);
  const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t gw = (int64_t)crank * nw + wid, gnw = (int64_t)csize * nw;
  const int ids[2] = {ACC_N13, ACC_N17};
  const int64_t whi = win_words > 0 ? min(ts.jbig, wlo + 2 * (int64_t)win_words) : wlo;   // window [wlo, whi)
  LocalAcc<2> la;
  la.zero();
  while (true) {
    if (crank == 0 && threadIdx.x == 0) {
      sh_item = (long long)atomicAdd(qctr, 1ull);
      pt.n[grp] = 0;                           // every CTA is past the last item's tasks
    }
    cluster_barrier();                         // also: the last item's reads are done
    const long long it = ld_cluster_s64(&sh_item, 0);
    if (it >= nitems) break;
    const int64_t i = items[it];
    const int64_t b0 = g.R[i], e0 = g.R[i + 1];
    if (w.next_shared(ts.n, crank, csize)) cluster_barrier();
    if (win_words > 0) {
      for (int t = threadIdx.x; t < win_words; t += blockDim.x) win[t] = 0u;
      cluster_barrier();
    }
    auto inc = [&](int32_t j) -> uint32_t {
      if (j >= wlo && j < whi) {
        const int64_t k = j - wlo;
        const unsigned sh16 = 16u * (unsigned)(k & 1);
        return (atomicAdd(&win[k >> 1], 1u << sh16) >> sh16) & 0xffffu;
      }
      return w.inc(j);
    };
    u128 n13 = pair_wedges(g, b0, e0, gw, gnw, inc,
                           [&](int64_t cb, int64_t ce) { return pair_defer(pt, grp, cb, ce); });
    cluster_barrier();
    // the task count is read before the next barrier, after which CTA 0 may
    // clear it for the next item
    const unsigned long long nt1 = __ldcg(&pt.n[grp]);
    n13 += pair_run_tasks(g, pt, grp, nt1, gw, gnw, inc);
    cluster_barrier();
    u128 n17 = pair_diamonds(g, tl3, T, i, b0, e0, gw, gnw, [&](int32_t j) -> uint32_t {
      if (j >= wlo && j < whi) {
        const int64_t k = j - wlo;
        return (win[k >> 1] >> (16u * (unsigned)(k & 1))) & 0xffffu;
      }
      return w.get_l2(j);
    });
    la.v[0] += n13;
    la.v[1] += n17;
    block_item_flush(la, ids, acc, i, sh);
  }
  cluster_barrier();                           // CTA 0's shared memory stays until every CTA has read it
  final_flush(la, ids, acc, sh);
}

// ---------------------------------------------------------------- windowed heavy items
// Heavy items, default form: one 1024-thread CTA per SM and item.  The ranks
// below jbig are cut into windows of S = 2 * win_words ranks on a grid
// anchored at jbig (window k = [jbig - (k+1) S, jbig - k S)).  An item i
// counts its wedges window by window, from the lowest window that can hold a
// neighbour of a neighbour up to the one holding rank min(i, jbig) - 1, every
// increment a 16-bit shared-memory atomic.  For every c in N(i) a cursor marks
// how far N(c) has been walked; a window takes the entries below its upper
// end.  A finished window below the top one is written whole to the CTA's
// dense 16-bit array; the top window stays in shared memory.  Ranks from jbig
// on (degree >= 2^16, so counts may need more than 16 bits) go to tagged
// 64-bit counters.  The diamond pass then reads W(i,j) from shared memory
// (the top window, where most diamond tips lie), the dense array or the 64-bit
// counters.
// A count below jbig is at most d_j < 2^16.  The dense array needs no clearing:
// a window is written whole, and the diamond pass reads only windows this item
// wrote (a diamond tip j shares two neighbours with i, so W(i,j) >= 2 and its
// window took increments).
struct PairWin {
  uint32_t* g16;              // per CTA: rank j at bits 16 ((j + par) & 1) of word ((j + par) >> 1) + woff
  int64_t g16_words;          // a multiple of 4, >= (n + 2) / 2 + 4
  int woff;                   // 0..3: puts the first word of every window on a 16-byte boundary
  longlong2* curs;            // per CTA: (cursor, end) of the list N(c) of every c in N(i)
  int64_t curs_cap;           // >= the largest degree
  unsigned long long* side;   // per CTA: n - jbig counters (tag << 32) | count
  int64_t jbig, n, n0;        // n0: the first rank of degree >= 1
  int win_words;              // a multiple of 4
};

// First position q in [a, b) with C[q] >= key (C ascending there), or b; one
// warp, 32 probes per round.
__device__ __forceinline__ int64_t warp_lower_bound(const int32_t* C, int64_t a, int64_t b, int32_t key) {
  const int lane = threadIdx.x & 31;
  // C[q] < key for q < a, C[q] >= key for q >= b
  while (b - a > 32) {
    const int64_t step = (b - a + 31) / 32;
    const int64_t q = a + (int64_t)lane * step;
    const unsigned m = __ballot_sync(0xffffffffu, q >= b || C[q] >= key);
    if (m == 0) {
      a += 31 * step + 1;
    } else {
      const int f = __ffs(m) - 1;
      b = min(b, a + (int64_t)f * step);
      if (f > 0) a += (int64_t)(f - 1) * step + 1;
    }
  }
  const int64_t q = a + lane;
  const unsigned m = __ballot_sync(0xffffffffu, q >= b || C[q] >= key);
  return m ? min(b, a + (int64_t)(__ffs(m) - 1)) : b;
}

// Pass 1 of one window: for every c in N(i) (this warp's share), the entries
// of N(c) from its cursor that lie below `hi` (all remaining ones when `last`).
// `first`: the cursors start at the heads of the lists; unless `last`, the new
// cursors are stored.
template <class Inc, class Defer>
__device__ __forceinline__ u128 pair_wedges_win(const DevGraph& g, longlong2* curs, int64_t b0, int64_t e0,
                                                int64_t gw, int64_t gnw, bool first, bool last, int32_t hi,
                                                Inc&& inc, Defer&& defer) {
  const int lane = threadIdx.x & 31;
  u128 n13 = 0;
  for (int64_t pbase = b0 + gw; pbase < e0; pbase += gnw * 32) {
    const int64_t p = pbase + (int64_t)lane * gnw;
    int64_t cb_l = 0, ce_l = 0;
    if (p < e0) {
      if (first) {
        cb_l = g.R[g.C[p]];
        ce_l = g.rev[p];                        // N(c) below i ends at the slot of i
      } else {
        const longlong2 cu = curs[p - b0];
        cb_l = cu.x;
        ce_l = cu.y;
      }
    }
    int64_t cn_l = ce_l;                        // the lane's new cursor
    if (ce_l - cb_l <= PAIR_SHORT) {            // short: each lane walks its own list up to hi
      const int32_t* L = g.C + cb_l;
      const int len = (int)(ce_l - cb_l);
      Sum128 sh13;
      int q = 0;
      while (q < len) {
        int32_t jj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) jj[u] = q + u < len ? __ldcs(L + q + u) : 0x7fffffff;
        int stop = 4;
#pragma unroll
        for (int u = 3; u >= 0; --u)
          if (jj[u] >= hi) stop = u;            // ascending: the first entry at or above hi
        unsigned long long blk = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (u < stop) blk += pair_c2(inc(jj[u]));
        sh13.add(blk);
        if (stop < 4) {
          q += stop;
          break;
        }
        q += 4;
      }
      n13 += sh13.get();
      cn_l = cb_l + min(q, len);
    }
    unsigned longm = __ballot_sync(0xffffffffu, ce_l - cb_l > PAIR_SHORT);
    while (longm) {                             // long: the warp takes them one at a time
      const int k = __ffs(longm) - 1;
      longm &= longm - 1;
      const int64_t cb = __shfl_sync(0xffffffffu, cb_l, k), ce = __shfl_sync(0xffffffffu, ce_l, k);
      const int64_t qe = last ? ce : warp_lower_bound(g.C, cb, ce, hi);
      if (lane == k) cn_l = qe;
      if (qe - cb > PAIR_TASK && defer(cb, qe)) continue;
      n13 += pair_range(g, cb, qe, inc);
    }
    if (!last && p < e0) curs[p - b0] = make_longlong2(cn_l, ce_l);
  }
  return n13;
}

template <bool BIG>
__global__ void __launch_bounds__(1024, 1) k_pairs_win(DevGraph g, const int32_t* items, int64_t nitems,
                                                        unsigned long long* qctr, PairWin pw, TriLists tl3,
                                                        const uint32_t* T, AccSet acc, PairTasks pt,
                                                        unsigned* status) {
  extern __shared__ uint32_t win[];
  __shared__ u128 sh[32];
  __shared__ int64_t sh_item;
  __shared__ int sh_flag[2];                   // a window took increments (windows alternate)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t grp = blockIdx.x;
  const int64_t S = 2 * (int64_t)pw.win_words;
  const int64_t par = pw.jbig & 1;
  uint32_t* g16 = pw.g16 + grp * pw.g16_words + pw.woff;
  uint4* const win4 = reinterpret_cast<uint4*>(win);
  const int nv = pw.win_words >> 2;
  longlong2* curs = pw.curs + grp * pw.curs_cap;
  unsigned long long* side = pw.side + grp * (pw.n - pw.jbig);
  uint32_t tag = 0;
  const int ids[2] = {ACC_N13, ACC_N17};
  LocalAcc<2> la;
  la.zero();
  for (int t = threadIdx.x; t < nv; t += blockDim.x) win4[t] = make_uint4(0u, 0u, 0u, 0u);
  if (threadIdx.x == 0) sh_flag[0] = sh_flag[1] = 0;
  while (true) {
    const int64_t it = next_item(qctr, nitems, &sh_item);   // its barriers publish the cleared window
    if (it < 0) break;
    const int64_t i = items[it];
    const int64_t b0 = g.R[i], e0 = g.R[i + 1];
    if (e0 - b0 > pw.curs_cap) {                // never: sized by the largest degree
      if (threadIdx.x == 0) set_err(status, DEVERR_SCRATCH);
      continue;
    }
    if (BIG && ++tag == 0xffffffffu) {          // tags used up: zero the 64-bit counters
      for (int64_t t = threadIdx.x; t < pw.n - pw.jbig; t += blockDim.x) side[t] = 0ull;
      tag = 1;
      __syncthreads();
    }
    const int64_t top = min(i, pw.jbig);        // ranks [0, top) are counted in windows
    const int64_t ktop = (pw.jbig - top) / S;   // the window of rank top - 1
    const int64_t kbot = max(ktop, (pw.jbig - 1 - pw.n0) / S);   // the window of rank n0
    u128 n13 = 0;
    bool top_touched = false;
    for (int64_t k = kbot; k >= ktop; --k) {
      const int64_t lo = pw.jbig - (k + 1) * S;
      const uint32_t lo32 = (uint32_t)lo;       // -S <= lo < 2^31: 32-bit differences below
      const bool last = k == ktop;
      const int32_t hi = last ? 0x7fffffff : (int32_t)(pw.jbig - k * S);
      bool tch = false;
      auto inc = [&](int32_t j) -> uint32_t {
        tch = true;
        if (BIG && j >= pw.jbig) {
          unsigned long long* q = &side[j - pw.jbig];
          atomicMax(q, (unsigned long long)tag << 32);
          return (uint32_t)atomicAdd(q, 1ull);
        }
        const uint32_t q = (uint32_t)j - lo32;  // in [0, S)
        const unsigned s16 = (q & 1u) << 4;
        return (atomicAdd(&win[q >> 1], 1u << s16) >> s16) & 0xffffu;
      };
      n13 += pair_wedges_win(g, curs, b0, e0, wid, nw, k == kbot, last, hi, inc,
                             [&](int64_t cb, int64_t ce) { return pair_defer(pt, grp, cb, ce); });
      __syncthreads();                          // the window's long lists are appended as tasks
      const unsigned long long nt = __ldcg(&pt.n[grp]);
      n13 += pair_run_tasks(g, pt, grp, nt, wid, nw, inc);
      if (__any_sync(0xffffffffu, tch) && lane == 0) sh_flag[k & 1] = 1;
      __syncthreads();                          // the window's counts are complete; every thread has read nt
      const bool touched = sh_flag[k & 1] != 0;
      if (threadIdx.x == 0) {
        pt.n[grp] = 0;                          // the next window appends after a later barrier
        sh_flag[(k - 1) & 1] = 0;               // the next window's flag (last read before the first barrier above)
      }
      if (last) {
        top_touched = touched;
      } else {
        if (touched) {                          // write the window whole and clear it, 4 words at a time
          const int64_t w0 = (lo + par) >> 1;   // lo + par is even; w0 + woff is a multiple of 4
          uint4* g4 = reinterpret_cast<uint4*>(g16 + w0);
          for (int t = threadIdx.x; t < nv; t += blockDim.x) {
            const uint4 v = win4[t];
            if (pw.woff + w0 + 4 * t >= 0) g4[t] = v;   // the lowest window may start below rank 0
            win4[t] = make_uint4(0u, 0u, 0u, 0u);
          }
        }
        __syncthreads();
      }
    }
    const uint32_t lo_top32 = (uint32_t)(pw.jbig - (ktop + 1) * S), S32 = (uint32_t)S;
    u128 n17 = pair_diamonds(g, tl3, T, i, b0, e0, wid, nw, [&](int32_t j) -> uint32_t {
      // j < min(i, jbig) lies in the top window exactly when j - lo_top (mod 2^32) is below S
      const uint32_t q = (uint32_t)j - lo_top32;
      if (q < S32) return (win[q >> 1] >> ((q & 1u) << 4)) & 0xffffu;
      if (BIG && j >= pw.jbig) {
        const unsigned long long v = __ldcg(&side[j - pw.jbig]);
        return (uint32_t)(v >> 32) == tag ? (uint32_t)v : 0u;
      }
      const uint32_t t = (uint32_t)j + (uint32_t)par;
      return (__ldcg(&g16[t >> 1]) >> ((t & 1u) << 4)) & 0xffffu;
    });
    la.v[0] += n13;
    la.v[1] += n17;
    __syncthreads();                            // the diamond reads of the window are done
    if (top_touched)
      for (int t = threadIdx.x; t < nv; t += blockDim.x) win4[t] = make_uint4(0u, 0u, 0u, 0u);
    if (threadIdx.x == 0) sh_flag[0] = sh_flag[1] = 0;
    block_item_flush(la, ids, acc, i, sh);
  }
  final_flush(la, ids, acc, sh);
}

// ============================================================================
// Thm 11: N18 (wheels) = sum over centres c of the 4-cycles of G[N(c)],
// counted by the 4-cycle rule inside the neighbourhood: for u in N(c) and
// v < u, C(w_c(u,v), 2) with w_c(u,v) = |{k in N(c) cap N(u) cap N(v): k < u}|.
// Everything happens in the position space of row c: the lists of the slots
// (c -> u) hold positions in row c, so k < u is pk < pu and the counters are
// indexed by position.  sum_v C(w, 2) is the sum of the values each increment
// returns.
// ============================================================================
static constexpr int WHEEL_WARP_MAX = 1024;     // centres up to this degree: warp items

// Walks, for one centre c and one position pu, every k in N(c) cap N(u) below
// u (a prefix of the list of slot c -> u) and every v in N(c) cap N(k) below u
// (a prefix of the list of slot c -> k), calling visit(pv) once per pair with
// pv the position of v in row c.  A warp takes the k's a0, a0 + astep, ...:
// it fetches 32 of them at a time (lane l the l-th) and scans each v list with
// WHEEL_ILP independent loads in flight per lane.
#ifndef ESC_WHEEL_ILP
#define ESC_WHEEL_ILP 8
#endif
static constexpr int WHEEL_ILP = ESC_WHEEL_ILP;

template <class Visit>
__device__ __forceinline__ void wheel_links(const TriLists& tl3, const uint32_t* T, int64_t base, const int32_t* Lu,
                                            uint32_t lenu, int pu, uint32_t a0, uint32_t astep, Visit&& visit) {
  const int lane = threadIdx.x & 31;
  for (uint32_t ab = a0; ab < lenu; ab += 32 * astep) {
    uint32_t a = ab + lane * astep;
    const int32_t* Lk_l = tl3.P;
    uint32_t lk_l = 0;
    bool live = a < lenu, in = false;
    if (live) {
      int32_t pk = Lu[a];
      if (pk < pu) {
        in = true;
        Lk_l = tl3.P + tl3.offp[base + pk];
        lk_l = T[base + pk];
      }
    }
    unsigned m = __ballot_sync(0xffffffffu, in);
    bool done = __any_sync(0xffffffffu, live && !in);   // the k list is sorted: later rounds are above u
    while (m) {
      int k = __ffs(m) - 1;
      m &= m - 1;
      const int32_t* Lk = reinterpret_cast<const int32_t*>(
          __shfl_sync(0xffffffffu, reinterpret_cast<uintptr_t>(Lk_l), k));
      uint32_t lk = __shfl_sync(0xffffffffu, lk_l, k);
      for (uint32_t tb = 0; tb < lk; tb += 32 * WHEEL_ILP) {
        int32_t pv[WHEEL_ILP];
        bool past = false;
#pragma unroll
        for (int u = 0; u < WHEEL_ILP; ++u) {
          uint32_t t = tb + lane + 32 * u;
          pv[u] = t < lk ? Lk[t] : 0x7fffffff;
          if (pv[u] >= pu) { pv[u] = -1; past = true; }
        }
#pragma unroll
        for (int u = 0; u < WHEEL_ILP; ++u)
          if (pv[u] >= 0) visit(pv[u]);
        if (__any_sync(0xffffffffu, past)) break;
      }
    }
    if (done) break;
  }
}

// Centres up to WHEEL_WARP_MAX: work items are (centre, block of WHEEL_WBLK
// positions u), pulled by whole warps from a queue, heaviest centres first.
// Each warp owns a counter array in shared memory whose entries are
// (tag << 16) | count for the u they were counted for; before each increment
// an atomicMax with the current u's tag turns an older entry into a zero
// count, so nothing is cleared between u's or items.
static constexpr int WHEEL_WBLK = 32;

// item_cnt[k] = number of items of centre c0 - 1 - k (position k in the queue)
__global__ void k_wheel_warp_counts(DevGraph g, int64_t c0, int64_t* item_cnt, Owner own) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < c0; k += (int64_t)gridDim.x * blockDim.x) {
    int64_t c = c0 - 1 - k;
    int64_t d = g.R[c + 1] - g.R[c];
    item_cnt[k] = d >= 4 && own.owns(c) ? (d + WHEEL_WBLK - 1) / WHEEL_WBLK : 0;
  }
}

__global__ void __launch_bounds__(256, 6) k_wheels_warp(DevGraph g, int64_t c0, const int64_t* item_off,
                                                        unsigned long long* qctr, TriLists tl3, const uint32_t* T,
                                                        AccSet acc) {
  __shared__ u128 sh[32];
  __shared__ uint32_t scr_all[8][WHEEL_WARP_MAX];
  int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  uint32_t* scr = scr_all[wl];
  const int ids[1] = {ACC_N18};
  LocalAcc<1> la;
  la.zero();
  for (int i = lane; i < WHEEL_WARP_MAX; i += 32) scr[i] = 0;
  __syncwarp();
  uint32_t tag = 0;
  const int64_t nitems = item_off[c0];
  while (true) {
    unsigned long long it_l = 0;
    if (lane == 0) it_l = atomicAdd(qctr, 1ull);
    int64_t it = (int64_t)__shfl_sync(0xffffffffu, it_l, 0);
    if (it >= nitems) break;
    // queue position of the centre: the last k with item_off[k] <= it
    int64_t lo = 0, hi = c0;
    while (hi - lo > 1) {
      int64_t mid = (lo + hi) >> 1;
      if (item_off[mid] <= it) lo = mid; else hi = mid;
    }
    int64_t c = c0 - 1 - lo;
    int64_t base = g.R[c];
    int d = (int)(g.R[c + 1] - base);
    int u0 = (int)(it - item_off[lo]) * WHEEL_WBLK;
    int u1 = min(d, u0 + WHEEL_WBLK);
    u128 n18 = 0;
    for (int pu = u0; pu < u1; ++pu) {
      uint32_t lenu = T[base + pu];
      if (lenu < 2) continue;
      if (++tag == 0x10000u) {                           // tags exhausted: start over from zeroed counters
        __syncwarp();
        for (int i = lane; i < WHEEL_WARP_MAX; i += 32) scr[i] = 0;
        __syncwarp();
        tag = 1;
      }
      const int32_t* Lu = tl3.P + tl3.offp[base + pu];
      unsigned long long part = 0;
      const uint32_t t16 = tag << 16;
      wheel_links(tl3, T, base, Lu, lenu, pu, 0u, 1u, [&](int32_t pv) {
        atomicMax(&scr[pv], t16);               // an older u's entry becomes a zero count of this one
        part += atomicAdd(&scr[pv], 1u) & 0xffffu;
      });
      __syncwarp();                             // this u's increments before the next u's tag
      n18 += part;
    }
    la.v[0] += n18;
    warp_item_flush(la, ids, acc, c);
  }
  final_flush(la, ids, acc, sh);
}

// Centres above WHEEL_WARP_MAX: work items (centre, block of WHEEL_CHUNK
// positions u); counters in shared memory when the degree fits, otherwise in a
// per-CTA global region.
static constexpr int WHEEL_CHUNK = 64;

// Counters are tagged with the u they count for, (tag << 16) | count in the
// 32-bit shared-memory words and (tag << 32) | count in the 64-bit global ones
// (counts there can pass 2^16); before each increment an atomicMax with the
// current tag turns an older entry into a zero count, so no clearing pass
// walks the lists a second time.  A CTA's tags grow with the u's it takes.
// win16: every count of the sweep stays below 2^16 (the largest common-
// neighbour list is shorter), so large centres keep a shared-memory window.
__global__ void k_wheels_cta(DevGraph g, int64_t c0, const int64_t* item_off, int64_t nitems,
                             unsigned long long* qctr, TriLists tl3, const uint32_t* T, unsigned long long* gscr,
                             int64_t gscr_stride, int smem_cap, AccSet acc, bool win16) {
  extern __shared__ uint32_t sscr[];
  __shared__ u128 sh[32];
  __shared__ int64_t sh_item;
  int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int ids[1] = {ACC_N18};
  LocalAcc<1> la;
  la.zero();
  unsigned long long* g64 = gscr + (int64_t)blockIdx.x * gscr_stride;
  for (int i = threadIdx.x; i < smem_cap; i += blockDim.x) sscr[i] = 0;
  __syncthreads();
  uint32_t tag = 0;                             // the same in every thread of the CTA
  while (true) {
    int64_t it = next_item(qctr, nitems, &sh_item);
    if (it < 0) break;
    it = nitems - 1 - it;                     // heaviest centres first
    // centre of item `it`: the last k with item_off[k] <= it (item_off over centres c0..n-1)
    int64_t lo = 0, hi = g.n - c0;
    while (hi - lo > 1) { int64_t mid = (lo + hi) >> 1; if (item_off[mid] <= it) lo = mid; else hi = mid; }
    int64_t c = c0 + lo;
    int64_t base = g.R[c];
    int d = (int)(g.R[c + 1] - base);
    int u0 = (int)(it - item_off[lo]) * WHEEL_CHUNK;
    int u1 = min(d, u0 + WHEEL_CHUNK);
    const bool in_smem = d <= smem_cap;
    for (int pu = u0; pu < u1; ++pu) {
      uint32_t lenu = T[base + pu];
      if (lenu < 2) continue;
      if (++tag > 0xffffu) {                    // tags used up: zero both counter sets, start over
        for (int i = threadIdx.x; i < smem_cap; i += blockDim.x) sscr[i] = 0;
        for (int64_t i = threadIdx.x; i < gscr_stride; i += blockDim.x) g64[i] = 0;
        __syncthreads();
        tag = 1;
      }
      const int32_t* Lu = tl3.P + tl3.offp[base + pu];
      unsigned long long part = 0;
      if (in_smem) {
        const uint32_t t16 = tag << 16;
        wheel_links(tl3, T, base, Lu, lenu, pu, (uint32_t)wid, (uint32_t)nw, [&](int32_t pv) {
          atomicMax(&sscr[pv], t16);
          part += atomicAdd(&sscr[pv], 1u) & 0xffffu;
        });
      } else {
        // a centre too large for shared memory: its last smem_cap positions
        // (the highest ranks, where the common neighbours concentrate) stay
        // there when every count fits 16 bits (win16), the rest in global memory
        const unsigned long long t32 = (unsigned long long)tag << 32;
        const uint32_t t16 = tag << 16;
        const int wstart = win16 ? d - smem_cap : d;
        wheel_links(tl3, T, base, Lu, lenu, pu, (uint32_t)wid, (uint32_t)nw, [&](int32_t pv) {
          if (pv >= wstart) {
            uint32_t* c = &sscr[pv - wstart];
            atomicMax(c, t16);
            part += atomicAdd(c, 1u) & 0xffffu;
          } else {
            atomicMax(&g64[pv], t32);
            part += (uint32_t)atomicAdd(&g64[pv], 1ull);
          }
        });
      }
      la.v[0] += part;
      __syncthreads();                          // the next u's tag must not meet this u's increments
    }
    block_item_flush(la, ids, acc, c, sh);
  }
  final_flush(la, ids, acc, sh);
}

// ============================================================================
// Thm 13: 5-cycles.  For every directed 3-path i <- a -> b -> j (a < i,
// a < b < j, b != i, j != i) add w'(i,j) = |{c in N(i) cap N(j) : c < max(i,j)}|.
// Grouped by the pair (i, b): sum_b P2(i,b) * sum_{j in N+(b)} w'(i,j) with
// P2(i,b) = |{a in N-(i) : b in N+(a)}| (each out-wedge pair visited once).
// The paths whose own a or b is counted by w' are the directed tailed
// triangles, subtracted through ACC_N8Z (pass A).
// ============================================================================
template <bool BIG>
__global__ void __launch_bounds__(512, 2) k_cycles5(DevGraph g, unsigned long long* qctr, TagScratch ts,
                                                   SweepScratch ss, AccSet acc, Owner own) {
  __shared__ u128 sh[32];
  __shared__ int64_t sh_item;
  TaggedCounters<BIG> wp(ts);                                                         // w'(i, .)
  uint32_t* p2 = ss.cnt2 + (int64_t)blockIdx.x * ss.n;                            // P2(i, .), with a list
  int32_t* tl2 = ss.touched2 + (int64_t)blockIdx.x * ss.n;
  unsigned* nt = ss.ntouched + 2 * blockIdx.x;
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int ids[1] = {ACC_N8M};
  LocalAcc<1> la;
  la.zero();
  while (true) {
    int64_t it = next_item(qctr, own.count(g.n), &sh_item);
    if (it < 0) break;
    int64_t i = own.item(g.n, it);
    int64_t b0 = g.R[i], o = g.op[i], e0 = g.R[i + 1];
    if (o == b0) continue;                      // needs an in-neighbour a
    wp.next(ts.n);
    if (threadIdx.x == 0) nt[1] = 0;
    __syncthreads();
    // w'(i, .): c < i -> every j in N(c); c > i -> j in N+(c).  Lists are
    // fetched 32 per warp (lane k the k-th), SWEEP_ILP entries in flight per lane.
    for (int64_t pbase = b0 + wid; pbase < e0; pbase += (int64_t)nw * 32) {
      int64_t p = pbase + (int64_t)lane * nw;
      int64_t cb_l = 0, ce_l = 0;
      if (p < e0) {
        int32_t c = g.C[p];
        cb_l = (p < o) ? g.R[c] : g.op[c];
        ce_l = g.R[c + 1];
      }
      int kmax = (int)min((int64_t)32, (e0 - pbase + nw - 1) / nw);
      for (int k = 0; k < kmax; ++k) {
        int64_t cb = __shfl_sync(0xffffffffu, cb_l, k), ce = __shfl_sync(0xffffffffu, ce_l, k);
        const int32_t* L = g.C + cb;            // 32-bit offsets: a row has fewer than 2^31 entries
        const int len = (int)(ce - cb);
        for (int q = lane; q < len; q += 32 * SWEEP_ILP) {
          int32_t jj[SWEEP_ILP];
#pragma unroll
          for (int u = 0; u < SWEEP_ILP; ++u) jj[u] = q + 32 * u < len ? L[q + 32 * u] : (int32_t)i;
#pragma unroll
          for (int u = 0; u < SWEEP_ILP; ++u)
            if (jj[u] != i) wp.add(jj[u]);
        }
      }
    }
    // P2(i, .): a in N-(i), b in N+(a)
    for (int64_t pbase = b0 + wid; pbase < o; pbase += (int64_t)nw * 32) {
      int64_t p = pbase + (int64_t)lane * nw;
      int64_t cb_l = 0, ce_l = 0;
      if (p < o) {
        int32_t a = g.C[p];
        cb_l = g.op[a];
        ce_l = g.R[a + 1];
      }
      int kmax = (int)min((int64_t)32, (o - pbase + nw - 1) / nw);
      for (int k = 0; k < kmax; ++k) {
        int64_t cb = __shfl_sync(0xffffffffu, cb_l, k), ce = __shfl_sync(0xffffffffu, ce_l, k);
        const int32_t* L = g.C + cb;
        const int len = (int)(ce - cb);
        for (int q = lane; q < len; q += 32 * SWEEP_ILP) {
          int32_t bb[SWEEP_ILP];
          uint32_t oo[SWEEP_ILP];
#pragma unroll
          for (int u = 0; u < SWEEP_ILP; ++u) bb[u] = q + 32 * u < len ? L[q + 32 * u] : (int32_t)i;
#pragma unroll
          for (int u = 0; u < SWEEP_ILP; ++u) oo[u] = bb[u] != i ? atomicAdd(&p2[bb[u]], 1u) : 1u;
#pragma unroll
          for (int u = 0; u < SWEEP_ILP; ++u) warp_append(tl2, &nt[1], oo[u] == 0, bb[u]);
        }
      }
    }
    __syncthreads();
    unsigned n2 = nt[1];
    // sum over the distinct b of P2(i, b) * sum_{j in N+(b)} w'(i, j); the
    // b's are fetched 32 per warp
    for (unsigned tb = (unsigned)wid * 32; tb < n2; tb += (unsigned)nw * 32) {
      unsigned t = tb + lane;
      int64_t cb_l = 0, ce_l = 0;
      uint32_t pk_l = 0;
      if (t < n2) {
        int32_t b = tl2[t];
        cb_l = g.op[b];
        ce_l = g.R[b + 1];
        pk_l = p2[b];
      }
      int kmax = (int)min(32u, n2 - tb);
      for (int k = 0; k < kmax; ++k) {
        int64_t cb = __shfl_sync(0xffffffffu, cb_l, k), ce = __shfl_sync(0xffffffffu, ce_l, k);
        uint32_t pk = __shfl_sync(0xffffffffu, pk_l, k);
        unsigned long long s_ = 0;
        const int32_t* L = g.C + cb;
        const int len = (int)(ce - cb);
        for (int q = lane; q < len; q += 32 * SWEEP_ILP) {
          int32_t jj[SWEEP_ILP];
#pragma unroll
          for (int u = 0; u < SWEEP_ILP; ++u) jj[u] = q + 32 * u < len ? L[q + 32 * u] : -1;
#pragma unroll
          for (int u = 0; u < SWEEP_ILP; ++u)
            if (jj[u] >= 0) s_ += wp.get(jj[u]);
        }
        la.v[0] += (u128)s_ * pk;
      }
    }
    __syncthreads();
    for (unsigned t = threadIdx.x; t < n2; t += blockDim.x) p2[tl2[t]] = 0;
    block_item_flush(la, ids, acc, i, sh);
    __syncthreads();
  }
  final_flush(la, ids, acc, sh);
}

// ============================================================================
// Per-edge common-neighbour lists (the per-edge triangle lists of Thm 7),
// stored sorted: the id list once per undirected edge (addressed from both
// slots), and for each slot (u -> v) the positions in row u of the same
// vertices.  Built per higher endpoint y: N(y) goes into a hash table (vertex
// -> position in row y), and for every lower neighbour x the row N(x) is
// filtered through it; a hit at index q of row x has position q - R[x] there.
// ============================================================================
__global__ void k_tri_lists(DevGraph g, unsigned long long* qctr, const int64_t* off, const int64_t* offp,
                            const uint32_t* T, int32_t* U, int32_t* P, int32_t* ghash, int64_t ghash_cap,
                            int hash_cap, unsigned* status) {
  extern __shared__ int32_t smem[];
  __shared__ int64_t sh_item;
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int32_t* gk = ghash + (int64_t)blockIdx.x * 2 * ghash_cap;
  while (true) {
    int64_t it = next_item(qctr, g.n, &sh_item);
    if (it < 0) break;
    int64_t y = g.n - 1 - it;
    int64_t yb = g.R[y], yo = g.op[y], ye = g.R[y + 1];
    if (yo == yb) continue;
    int dy = (int)(ye - yb);
    bool small = 2 * dy <= hash_cap;
    int hsz = pow2_at_least(2 * dy);
    if (!small && hsz > ghash_cap) {            // cannot happen: sized by the maximum degree
      if (threadIdx.x == 0) set_err(status, DEVERR_SCRATCH);
      continue;
    }
    PosHash H = small ? PosHash{smem, smem + hash_cap, hsz - 1} : PosHash{gk, gk + ghash_cap, hsz - 1};
    for (int i = threadIdx.x; i < hsz; i += blockDim.x) H.keys[i] = -1;
    __syncthreads();
    for (int i = threadIdx.x; i < dy; i += blockDim.x) H.insert(g.C[yb + i], i);
    __syncthreads();
    for (int64_t p = yb + wid; p < yo; p += nw) {   // x in N-(y); p = slot (y -> x)
      int32_t x = g.C[p];
      int64_t cs = g.rev[p];                        // canonical slot (x -> y)
      int64_t out = off[cs], outx = offp[cs], outy = offp[p];
      uint32_t expect = T[cs];
      uint32_t written = 0;
      int64_t xb = g.R[x];
      for (int64_t base = xb; base < g.R[x + 1]; base += 32) {
        int64_t q = base + lane;
        int32_t py = -1, z = -1;
        if (q < g.R[x + 1]) {
          z = g.C[q];
          py = H.find(z);
        }
        bool hit = py >= 0;
        unsigned hm = __ballot_sync(0xffffffffu, hit);
        if (hit) {
          unsigned k = written + __popc(hm & ((1u << lane) - 1u));
          if (k < expect) {
            U[out + k] = z;
            P[outx + k] = (int32_t)(q - xb);
            P[outy + k] = py;
          }
        }
        written += __popc(hm);
      }
      if (lane == 0 && written != expect) set_err(status, DEVERR_BOUNDS);
    }
    __syncthreads();
  }
}

// list offsets: off[p] for canonical slots = scan of T; reverse slots share it
__global__ void k_canon_counts(DevGraph g, const uint32_t* T, int64_t* cnt) {
  int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < g.n; v += nwarps) {
    for (int64_t p = g.R[v] + lane; p < g.op[v]; p += 32) cnt[p] = 0;
    for (int64_t p = g.op[v] + lane; p < g.R[v + 1]; p += 32) cnt[p] = T[p];
  }
}
__global__ void k_all_counts(const uint32_t* T, int64_t nnz, int64_t* cnt) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride) cnt[p] = T[p];
}
__global__ void k_share_offsets(DevGraph g, int64_t* off) {
  int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < g.n; v += nwarps)
    for (int64_t p = g.op[v] + lane; p < g.R[v + 1]; p += 32) off[g.rev[p]] = off[p];
}

// ============================================================================
// Per-edge and per-vertex closed-form sums (Thms 4, 8, 9): one warp per row,
// canonical slots only for unordered sums.
// ============================================================================
__global__ void k_edge_sums(DevGraph g, const uint32_t* T, const unsigned long long* C4e,
                            const unsigned long long* K4e, const unsigned long long* tv,
                            const unsigned long long* C4v, const unsigned long long* K4v, AccSet acc) {
  __shared__ u128 sh[32];
  int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int ids[13] = {ACC_N5A, ACC_N11, ACC_D, ACC_N14, ACC_N6A, ACC_N12A, ACC_N19,
                       ACC_TT, ACC_N4, ACC_N9A, ACC_N7A, ACC_N15, ACC_TD};
  LocalAcc<13> la;
  la.zero();
  for (int64_t v = warp; v < g.n; v += nwarps) {
    unsigned long long dv = (unsigned long long)dg_deg(g, v), tvv = tv[v];
    for (int64_t p = g.R[v] + lane; p < g.R[v + 1]; p += 32) {
      int32_t u = g.C[p];
      unsigned long long du = (unsigned long long)dg_deg(g, u), te = T[p];
      // ordered (v -> u)
      la.v[0] += (u128)(tvv - te) * (du - 1);                       // N5 first term
      if (te >= 2) la.v[1] += ch2(te) * (dv - 3);                   // N11
      if (u > v) {                                                  // unordered
        la.v[2] += ch2(te);                                         // D
        la.v[3] += ch3(te);                                         // N14
        if (te) la.v[4] += (u128)te * (dv - 2) * (du - 2);          // N6 first term
        la.v[5] += (u128)C4e[p] * te;                               // N12 first term
        if (K4e[p]) la.v[6] += (u128)K4e[p] * (te - 2);             // N19
      }
    }
    if (lane == 0) {
      if (dv >= 2) la.v[7] += (u128)tvv * (dv - 2);                 // TT
      if (dv >= 2) la.v[8] += (u128)tvv * ch2(dv - 2);              // N4
      la.v[9] += ch2(tvv);                                          // N9 first term
      if (C4v[v]) la.v[10] += (u128)C4v[v] * (dv - 2);              // N7 first term
      if (K4v[v]) la.v[11] += (u128)K4v[v] * (dv - 3);              // N15
      la.v[12] += (u128)tvv * dv;                                   // P3+K2 / K3+K2 terms
    }
    warp_item_flush(la, ids, acc, v);
  }
  final_flush(la, ids, acc, sh);
}

// ============================================================================
// Assembly (Thm 3, App. A; Thms 4, 8-14; App. B).  One thread; all arithmetic
// modulo 2^128, which is exact because every final count is below 2^127.
// out: induced c3[4], c4[11], c5[34], then non-induced n3, n4, n5 (u128 each).
// ============================================================================
struct ConvTables {
  long long a3[4 * 4];
  long long a4[11 * 11];
  long long a5[34 * 34];
};

__device__ __forceinline__ u128 cnk(u128 n, int k) {
  // C(n, k) for k <= 5 with n < 2^64: exact in 128-bit (product of k terms / k!)
  if (n < (u128)k) return 0;
  u128 r = 1;
  for (int i = 0; i < k; ++i) r = r * (n - i) / (i + 1);
  return r;
}

// One thread per graph: graph k reads accumulator row k and writes result k.
// basis_all (optional): per graph the four counts the runtime is linear in
// (Sec. 8's runtime fit): W, D, directed 3-paths, directed bipyramids.
__global__ void k_assemble(const Acc128* acc_all, const unsigned long long* n_arr, const unsigned long long* m_arr,
                           int num_graphs, ConvTables tabs, unsigned long long* out_all, u128* basis_all) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= num_graphs) return;
  const Acc128* acc = acc_all + (int64_t)k * ACC_COUNT;
  unsigned long long* out = out_all + (int64_t)k * 2 * 98;
  u128 A[ACC_COUNT];
  for (int i = 0; i < ACC_COUNT; ++i) A[i] = ((u128)acc[i].hi << 64) | acc[i].lo;
  if (basis_all) {
    u128* bo = basis_all + (int64_t)k * 4;
    bo[0] = A[ACC_W];
    bo[1] = A[ACC_D];
    bo[2] = A[ACC_DP];
    bo[3] = A[ACC_DBP];
  }
  u128 n = n_arr[k], m = m_arr[k];
  u128 W = A[ACC_W], T = A[ACC_T], TT = A[ACC_TT], C4 = A[ACC_C4], D = A[ACC_D];
  u128 K4 = A[ACC_K4] / 3, S3 = A[ACC_S3];
  u128 P4 = A[ACC_P4A] - 3 * T;
  u128 N[35];
  N[1] = A[ACC_S4];
  N[2] = A[ACC_N2A] - 2 * TT;
  N[3] = A[ACC_N3A] - 4 * C4 - 2 * TT - 3 * T;
  N[4] = A[ACC_N4];
  N[5] = A[ACC_N5A] - 4 * D;
  N[6] = A[ACC_N6A] - 2 * D;
  N[7] = A[ACC_N7A] - 2 * D;
  N[8] = A[ACC_N8M] - A[ACC_N8Z];
  N[9] = A[ACC_N9A] - 2 * D;
  N[10] = A[ACC_N10A] - 12 * K4;
  N[11] = A[ACC_N11];
  N[12] = A[ACC_N12A] - 4 * D;
  N[13] = A[ACC_N13];
  N[14] = A[ACC_N14];
  N[15] = A[ACC_N15];
  N[16] = A[ACC_N16A] - 12 * K4;
  N[17] = A[ACC_N17];
  N[18] = A[ACC_N18];
  N[19] = A[ACC_N19];
  N[20] = A[ACC_N20];
  N[21] = A[ACC_N21];
  N[22] = cnk(n, 5);
  N[23] = n >= 2 ? m * cnk(n - 2, 3) : 0;
  N[24] = n >= 4 ? (cnk(m, 2) - W) * (n - 4) : 0;
  N[25] = n >= 3 ? W * cnk(n - 3, 2) : 0;
  N[26] = n >= 3 ? T * cnk(n - 3, 2) : 0;
  N[27] = n >= 4 ? S3 * (n - 4) : 0;
  N[28] = n >= 4 ? P4 * (n - 4) : 0;
  N[29] = n >= 4 ? TT * (n - 4) : 0;
  N[30] = n >= 4 ? C4 * (n - 4) : 0;
  N[31] = n >= 4 ? D * (n - 4) : 0;
  N[32] = n >= 4 ? K4 * (n - 4) : 0;
  N[33] = W * m - A[ACC_D2D] - A[ACC_DNBR] + 2 * W + 3 * T;
  N[34] = T * m - A[ACC_TD] + 3 * T;
  u128 n4[11] = {S3, P4, TT, C4, D, K4, cnk(n, 4), n >= 2 ? m * cnk(n - 2, 2) : 0, cnk(m, 2) - W,
                 n >= 3 ? W * (n - 3) : 0, n >= 3 ? T * (n - 3) : 0};
  u128 n3[4] = {cnk(n, 3), n >= 2 ? m * (n - 2) : 0, W, T};
  // induced = A^-1 * non-induced (signed integer matrix, arithmetic mod 2^128)
  u128* o = (u128*)out;
  for (int i = 0; i < 4; ++i) {
    u128 s = 0;
    for (int j = 0; j < 4; ++j) s += (u128)(__int128)tabs.a3[i * 4 + j] * n3[j];
    o[i] = s;
    o[49 + i] = n3[i];
  }
  for (int i = 0; i < 11; ++i) {
    u128 s = 0;
    for (int j = 0; j < 11; ++j) s += (u128)(__int128)tabs.a4[i * 11 + j] * n4[j];
    o[4 + i] = s;
    o[49 + 4 + i] = n4[i];
  }
  for (int i = 0; i < 34; ++i) {
    u128 s = 0;
    for (int j = 0; j < 34; ++j) s += (u128)(__int128)tabs.a5[i * 34 + j] * N[j + 1];
    o[15 + i] = s;
    o[49 + 15 + i] = N[i + 1];
  }
}

// ============================================================================
// Host orchestration.
// ============================================================================
static unsigned grid_for(int64_t work, int threads, int sms) {
  int64_t b = (work + threads - 1) / threads;
  int64_t cap = (int64_t)sms * 8;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// batch bookkeeping: graph of every rank-space vertex; vertices and edges per graph
__global__ void k_graph_of_vertex(const int64_t* voff, int num_graphs, const int32_t* rank, int64_t n, int32_t* vg) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
    int lo = 0, hi = num_graphs;          // last k with voff[k] <= u
    while (hi - lo > 1) { int mid = (lo + hi) >> 1; if (voff[mid] <= u) lo = mid; else hi = mid; }
    vg[rank[u]] = lo;
  }
}
__global__ void k_graph_sizes(const int64_t* voff, const int64_t* rp, int num_graphs, unsigned long long* n_arr,
                              unsigned long long* m_arr) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= num_graphs) return;
  n_arr[k] = (unsigned long long)(voff[k + 1] - voff[k]);
  m_arr[k] = (unsigned long long)((rp[voff[k + 1]] - rp[voff[k]]) / 2);
}

// item lists of pass A/B: vertices by out-degree class
// small / large: d+ up to small_max or above (vertices with d+ >= 2); the
// small ones are also split by d- for the clique pass: up to warp_din in wsmall
// (one warp each), the rest in csmall (one CTA each).
// The clique pass takes only the owned vertices (wsmall, csmall, clarge);
// the triangle pass takes every vertex (small, large).
__global__ void k_split_items(DevGraph g, int32_t* small, int32_t* large, int32_t* wsmall, int32_t* csmall,
                              int32_t* clarge, unsigned long long* cnts, int small_max, int warp_din, Owner own) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < g.n; k += stride) {
    int64_t x = g.n - 1 - k;
    int64_t d = g.R[x + 1] - g.op[x];
    if (d < 2) continue;
    const bool mine = own.owns(x);
    if (d <= small_max) {
      small[atomicAdd(&cnts[0], 1ull)] = (int32_t)x;
      if (!mine) continue;
      if (g.op[x] - g.R[x] <= warp_din) wsmall[atomicAdd(&cnts[2], 1ull)] = (int32_t)x;
      else csmall[atomicAdd(&cnts[3], 1ull)] = (int32_t)x;
    } else {
      large[atomicAdd(&cnts[1], 1ull)] = (int32_t)x;
      if (mine) clarge[atomicAdd(&cnts[4], 1ull)] = (int32_t)x;
    }
  }
}

// max over vertices of d+ x ceil(d- / 64) (words of the D bit sets) and max d+
__global__ void k_clique_dims(DevGraph g, unsigned long long* out) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long mw = 0, md = 0;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < g.n; x += stride) {
    unsigned long long dp = (unsigned long long)(g.R[x + 1] - g.op[x]);
    unsigned long long dm = (unsigned long long)(g.op[x] - g.R[x]);
    if (dp >= 2) {
      unsigned long long wds = dp * ((dm + 63) / 64);
      if (wds > mw) mw = wds;
    }
    if (dp > md) md = dp;
  }
  atomicMax(&out[0], mw);
  atomicMax(&out[1], md);
}


// ---------------------------------------------------------------- buffers
// Device buffers of one census.  Repeated censuses would otherwise pay dozens
// of cudaMalloc / cudaFree calls each (cudaFree synchronises the device), so
// buffers released by a census are kept in a per-device cache, up to
// kCacheCap bytes, and handed to later ones: a request takes the smallest
// cached buffer that is large enough and at most twice the size.  Release
// happens only after the census's stream has drained (CacheScope), so a
// buffer never changes hands while kernels may still use it.  If cudaMalloc
// fails, the cache is emptied and the allocation tried once more.
static constexpr size_t kCacheCap = (size_t)8 << 30;

class BufCache {
 public:
  void* get(int dev, size_t b, size_t* got) {
    std::lock_guard<std::mutex> lk(mu_);
    auto& m = free_[dev & 63];
    auto it = m.lower_bound(b);
    if (it == m.end() || it->first > 2 * b) return nullptr;
    void* p = it->second;
    *got = it->first;
    bytes_[dev & 63] -= it->first;
    m.erase(it);
    return p;
  }
  void put(int dev, void* p, size_t b) {
    {
      std::lock_guard<std::mutex> lk(mu_);
      if (bytes_[dev & 63] + b <= kCacheCap) {
        free_[dev & 63].emplace(b, p);
        bytes_[dev & 63] += b;
        return;
      }
    }
    cudaFree(p);
  }
  void clear(int dev) {
    std::multimap<size_t, void*> m;
    {
      std::lock_guard<std::mutex> lk(mu_);
      m.swap(free_[dev & 63]);
      bytes_[dev & 63] = 0;
    }
    for (auto& kv : m) cudaFree(kv.second);
  }

 private:
  std::mutex mu_;
  std::multimap<size_t, void*> free_[64];
  size_t bytes_[64] = {};
};
static BufCache g_cache;

// Buffers released inside a scope wait until the scope ends, and the scope
// ends by draining its stream.
struct CacheScope;
static thread_local CacheScope* t_scope = nullptr;
struct CacheScope {
  cudaStream_t s;
  int dev = 0;
  CacheScope* prev;
  std::vector<std::pair<void*, size_t>> pending;
  explicit CacheScope(cudaStream_t st) : s(st), prev(t_scope) {
    cudaGetDevice(&dev);
    t_scope = this;
  }
  ~CacheScope() {
    cudaStreamSynchronize(s);
    for (auto& pb : pending) g_cache.put(dev, pb.first, pb.second);
    t_scope = prev;
  }
};

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  ~DevBuf() {
    if (!p) return;
    if (t_scope) t_scope->pending.emplace_back(p, bytes);
    else cudaFree(p);
  }
  cudaError_t alloc(size_t b) {
    b = ((b > 0 ? b : 16) + 255) & ~(size_t)255;
    int dev = 0;
    cudaGetDevice(&dev);
    size_t got = 0;
    if ((p = g_cache.get(dev, b, &got)) != nullptr) {
      bytes = got;
      return cudaSuccess;
    }
    cudaError_t e = cudaMalloc(&p, b);
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      g_cache.clear(dev);
      e = cudaMalloc(&p, b);
    }
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    bytes = b;
    return cudaSuccess;
  }
  template <class T> T* as() { return (T*)p; }
};

#define ESC_TRY(x) do { cudaError_t _e = (x); if (_e != cudaSuccess) return _e; } while (0)

// Side streams for the concurrent phases; events order them after / before
// the caller's stream.  Destroyed when the census returns, after each has
// drained: on an early error return the caller's stream may not have joined
// them, and the buffers their kernels use go back to the cache only after
// this destructor (they are declared before the StreamSet).
struct StreamSet {
  cudaStream_t st[4] = {nullptr, nullptr, nullptr, nullptr};
  int count = 0;
  ~StreamSet() {
    for (int i = 0; i < count; ++i) {
      cudaStreamSynchronize(st[i]);
      cudaStreamDestroy(st[i]);
    }
  }
  // prio[i] != 0: the device's greatest (most urgent) priority, else its least
  cudaError_t create(int k, const int* urgent) {
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    for (int i = 0; i < k; ++i) {
      cudaError_t e = cudaStreamCreateWithPriority(&st[i], cudaStreamNonBlocking, urgent[i] ? greatest : least);
      if (e != cudaSuccess) return e;
      count = i + 1;
    }
    return cudaSuccess;
  }
  // every stream in `to` waits for the work enqueued on `from` so far
  cudaError_t fork_from(cudaStream_t from, std::initializer_list<cudaStream_t> to) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (r != cudaSuccess) return r;
    r = cudaEventRecord(e, from);
    for (cudaStream_t t : to)
      if (r == cudaSuccess) r = cudaStreamWaitEvent(t, e, 0);
    cudaEventDestroy(e);
    return r;
  }
  // `into` waits for everything enqueued on the side streams
  cudaError_t join_into(cudaStream_t into) {
    for (int i = 0; i < count; ++i) {
      cudaEvent_t e;
      cudaError_t r = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
      if (r != cudaSuccess) return r;
      r = cudaEventRecord(e, st[i]);
      if (r == cudaSuccess) r = cudaStreamWaitEvent(into, e, 0);
      cudaEventDestroy(e);
      if (r != cudaSuccess) return r;
    }
    return cudaSuccess;
  }
};

// Lets kernel k use all of the device's opt-in shared memory (less its static
// shared memory) as dynamic shared memory.  Every call sets the same value, so
// censuses running on other host threads never lower the limit between this
// thread's setting and its launch.
static cudaError_t allow_max_smem(const void* k, int optin) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, k);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

// Launch shape of the heavy pair items: CTAs of `threads` threads grouped in
// clusters of `cs`, `nclusters` clusters (one counter array each), as many
// clusters as the SMs hold.  ESC_PAIR_SHAPE, ESC_PAIR_CLUSTER and
// ESC_PAIR_CLUSTERS override the choice (tuning only; results are the same).
struct PairPlan {
  int cs = 1, threads = 512, nclusters = 0;
  int shape = 1;                               // kernel instance, see ESC_PAIR_SHAPES
  int win_words = 0;                           // shared-memory window (clusters of one CTA)
  int64_t wlo = 0;                             // its first rank
  bool windowed = false;                       // k_pairs_win: every rank below jbig in successive windows
};

static int env_int(const char* name, int dflt) {
  const char* v = getenv(name);
  if (!v || !*v) return dflt;
  int x = atoi(v);
  return x > 0 ? x : dflt;
}

// Launch shapes of the heavy-item kernel: (threads, CTAs per SM) = (512, 3)
// at 40 registers, (512, 2) at 64, (1024, 1) at 64.
#define ESC_PAIR_SHAPES(X) X(0, 512, 3) X(1, 512, 2) X(2, 1024, 1)
static const void* pairs_grp_fn(bool big, int shape) {
#define ESC_PG(k, t, b) if (shape == k) return big ? (const void*)k_pairs_grp<true, t, b> : (const void*)k_pairs_grp<false, t, b>;
  ESC_PAIR_SHAPES(ESC_PG)
#undef ESC_PG
  return nullptr;
}

// The windowed form (k_pairs_win, the default): one 1024-thread CTA per SM,
// the window as wide as shared memory allows, but no wider than the ranks
// [n0, jbig) need.
static cudaError_t plan_pair_windows(bool big, int sms, int64_t n0, int64_t jbig, int smem_optin, PairPlan* plan) {
  const void* k = big ? (const void*)k_pairs_win<true> : (const void*)k_pairs_win<false>;
  cudaFuncAttributes fa;
  ESC_TRY(cudaFuncGetAttributes(&fa, k));
  ESC_TRY(allow_max_smem(k, smem_optin));     // the limit is the same for every graph
  const int bytes = (smem_optin - (int)fa.sharedSizeBytes - 1024) & ~15;
  const int64_t want = ((jbig - n0 + 2) / 2 + 3) & ~(int64_t)3;     // words covering [n0, jbig) in one window
  plan->windowed = true;
  plan->threads = 1024;
  plan->cs = 1;
  plan->shape = 0;
  plan->win_words = (int)std::min<int64_t>(bytes / 4, want);
  // ESC_PAIR_WIN_WORDS: narrower windows, so that small graphs take many (tests)
  plan->win_words = std::min(plan->win_words, env_int("ESC_PAIR_WIN_WORDS", plan->win_words));
  plan->win_words = std::max(4, plan->win_words & ~3);          // whole 16-byte vectors
  plan->wlo = jbig - 2 * (int64_t)plan->win_words;
  int per_sm = 0;
  ESC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, plan->threads, plan->win_words * 4));
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  plan->nclusters = sms * per_sm;
  return cudaSuccess;
}

static cudaError_t plan_pair_clusters(bool big, int sms, size_t arr_bytes, int64_t n0, int64_t jbig, int smem_optin,
                                      bool union_of_graphs, PairPlan* plan) {
  // ESC_PAIR_WINDOW: 3 every rank in successive windows (k_pairs_win, the
  // default for one graph); 2 one window over the top ranks and tagged global
  // counters below it (the default for a batch: in a block-diagonal union the
  // ranks of one member are spread over the whole rank range, so an item
  // would walk and write nearly every window for a few hundred wedges); 1 no
  // window.  The single window takes one 1024-thread CTA per SM (its window
  // is twice as wide as two 512-thread CTAs' each); without the window,
  // (512, 2).
  const int wmode = env_int("ESC_PAIR_WINDOW", union_of_graphs ? 2 : 3);
  if (wmode >= 3 && env_int("ESC_PAIR_CLUSTER", 1) == 1) return plan_pair_windows(big, sms, n0, jbig, smem_optin, plan);
  const bool window = env_int("ESC_PAIR_CLUSTER", 1) == 1 && wmode != 1;
  plan->shape = std::min(2, env_int("ESC_PAIR_SHAPE", window ? 3 : 2) - 1);
  plan->threads = plan->shape == 2 ? 1024 : 512;
  const void* k = pairs_grp_fn(big, plan->shape);
  int dev = 0, l2 = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
  ESC_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  const size_t budget = (size_t)std::max(l2, 1 << 20) / 2;
  const int64_t kmax = std::max<int64_t>(1, (int64_t)(budget / std::max<size_t>(arr_bytes, 1)));
  // the window: what shared memory leaves per CTA, for clusters of one CTA
  // (ESC_PAIR_WINDOW=1 turns it off)
  plan->win_words = 0;
  plan->wlo = jbig;
  if (window) {
    cudaFuncAttributes fa;
    ESC_TRY(cudaFuncGetAttributes(&fa, k));
    const int per_sm_target = plan->threads == 1024 ? 1 : 2;
    int bytes = (smem_optin / per_sm_target - (int)fa.sharedSizeBytes - 1024) & ~15;
    int64_t want = std::max<int64_t>(0, (jbig - n0 + 1) / 2);        // words covering every countable rank
    plan->win_words = (int)std::max<int64_t>(0, std::min<int64_t>(bytes / 4, want));
    plan->wlo = std::max<int64_t>(n0, jbig - 2 * (int64_t)plan->win_words);
    if (plan->win_words > 0) ESC_TRY(allow_max_smem(k, smem_optin));   // the limit is the same for every graph
  }
  int per_sm = 1;
  ESC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, plan->threads, plan->win_words * 4));
  const int64_t total = (int64_t)sms * std::max(1, per_sm);
  // clusters of one CTA with the shared-memory window by default; without
  // it, clusters of 4 CTAs were fastest on the Chung-Lu and R-MAT workloads,
  // ahead of the larger clusters whose fewer arrays stay in L2 (the items in
  // flight matter more than L2 hits); kmax, the cluster count that would fit
  // L2, is kept for the record of the plan
  int cs = env_int("ESC_PAIR_CLUSTER", plan->win_words > 0 ? 1 : 4);
  (void)kmax;
  plan->nclusters = (int)std::max<int64_t>(1, total / cs);
  // never more clusters than can be resident at once
  for (;; cs >>= 1) {
    cudaLaunchConfig_t lc = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.gridDim = dim3((unsigned)(plan->nclusters * cs));
    lc.blockDim = dim3((unsigned)plan->threads);
    lc.dynamicSmemBytes = (size_t)plan->win_words * 4;
    lc.attrs = at;
    lc.numAttrs = 1;
    int active = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&active, k, &lc);
    if (e == cudaSuccess && active > 0) {
      plan->nclusters = std::min(plan->nclusters, active);
      break;
    }
    cudaGetLastError();
    if (cs == 1) return e == cudaSuccess ? cudaErrorInvalidConfiguration : e;
    plan->nclusters *= 2;                       // the same CTAs in half-size clusters
  }
  plan->cs = cs;
  plan->nclusters = std::min(plan->nclusters, env_int("ESC_PAIR_CLUSTERS", plan->nclusters));
  return cudaSuccess;
}

static cudaError_t launch_pairs_grp(bool big, const PairPlan& plan, const DevGraph& g, const int32_t* items,
                                    int64_t nitems, unsigned long long* qctr, const TagScratch& ts,
                                    const TriLists& tl3, const uint32_t* T, const AccSet& accs,
                                    const PairTasks& pt, cudaStream_t s) {
  cudaLaunchConfig_t lc = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = plan.cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.gridDim = dim3((unsigned)(plan.nclusters * plan.cs));
  lc.blockDim = dim3((unsigned)plan.threads);
  lc.dynamicSmemBytes = (size_t)plan.win_words * 4;
  lc.stream = s;
  lc.attrs = at;
  lc.numAttrs = 1;
  cudaError_t e = cudaErrorInvalidValue;
#define ESC_PG(k, t, b)                                                                                   \
  if (plan.shape == k)                                                                                    \
    e = big ? cudaLaunchKernelEx(&lc, k_pairs_grp<true, t, b>, g, items, nitems, qctr, ts, tl3, T, accs, pt,     \
                                 plan.wlo, plan.win_words)                                                      \
            : cudaLaunchKernelEx(&lc, k_pairs_grp<false, t, b>, g, items, nitems, qctr, ts, tl3, T, accs, pt,    \
                                 plan.wlo, plan.win_words);
  ESC_PAIR_SHAPES(ESC_PG)
#undef ESC_PG
  note_launch();
  return e;
}

cudaError_t run_census(const int64_t* rp, const int32_t* col, int64_t n, int64_t nnz, const CensusConfig& cfg,
                       unsigned long long* d_out, unsigned* d_status, PerElement* pe_out, Oriented* or_out,
                       cudaStream_t s) {
  CacheScope cache_scope(s);                    // destroyed last: the buffers below return after the stream drains
  const int sms = cfg.sms > 0 ? cfg.sms : 1;
  int smem_optin = 0;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  }
  // phase k is timed by events 2k (begin) and 2k+1 (end) on the stream that runs it
  // Phase boundaries: CUDA events for the phase times, and NVTX ranges (a
  // profiler's timeline shows each phase's launches under its name).
  static const char* const kPhaseNames[9] = {"orient", "triangles", "cliques", "cycles4", "tri_lists",
                                             "pairs", "wheels", "cycles5", "assemble"};
  auto mark = [&](int k, int end, cudaStream_t st) {
    int i = 2 * k + end;
    if (cfg.phase_events && i < cfg.num_phase_events) cudaEventRecord(cfg.phase_events[i], st);
#if ESC_HAVE_NVTX
    if (!end) nvtxRangePushA(kPhaseNames[k]);
    else nvtxRangePop();
#else
    (void)kPhaseNames;
#endif
  };
  mark(0, 0, s);
  // ---------------- orientation (Sec. 3.2)
  DevBuf arena_buf;
  DeviceArena arena;
  int64_t nk = (n > nnz ? n : nnz) + 16;
  size_t arena_bytes = (size_t)nk * 8 * 2 + (size_t)(n + 16) * 8 + (size_t)(nk / 4096 + 2) * 256 * 8 * 2 + (1 << 22);
  ESC_TRY(arena_buf.alloc(arena_bytes));
  arena.base = arena_buf.as<char>();
  arena.cap = arena_bytes;

  DevBuf b_perm, b_rank, b_R, b_C, b_op, b_rev;
  ESC_TRY(b_perm.alloc(sizeof(int32_t) * (n + 1)));
  ESC_TRY(b_rank.alloc(sizeof(int32_t) * (n + 1)));
  ESC_TRY(b_R.alloc(sizeof(int64_t) * (n + 1)));
  ESC_TRY(b_C.alloc(sizeof(int32_t) * (nnz + 1)));
  ESC_TRY(b_op.alloc(sizeof(int64_t) * (n + 1)));
  ESC_TRY(b_rev.alloc(sizeof(int64_t) * (nnz + 1)));
  Oriented o;
  o.perm = b_perm.as<int32_t>();
  o.rank = b_rank.as<int32_t>();
  o.R = b_R.as<int64_t>();
  o.C = b_C.as<int32_t>();
  o.op = b_op.as<int64_t>();
  o.rev = b_rev.as<int64_t>();
  ESC_TRY(orient(rp, col, n, nnz, o, arena, s, sms));
  mark(0, 1, s);

  DevGraph g{n, nnz, o.R, o.C, o.op, o.rev};
  const int TPB = 256;
  // ---------------- per-element arrays and accumulators
  DevBuf b_T, b_K4e, b_C4e, b_tv, b_C4v, b_K4v, b_acc, b_ctr;
  ESC_TRY(b_T.alloc(sizeof(uint32_t) * (nnz + 1)));
  ESC_TRY(b_K4e.alloc(sizeof(unsigned long long) * (nnz + 1)));
  ESC_TRY(b_C4e.alloc(sizeof(unsigned long long) * (nnz + 1)));
  ESC_TRY(b_tv.alloc(sizeof(unsigned long long) * (n + 1)));
  ESC_TRY(b_C4v.alloc(sizeof(unsigned long long) * (n + 1)));
  ESC_TRY(b_K4v.alloc(sizeof(unsigned long long) * (n + 1)));
  const int G = cfg.num_graphs > 1 ? cfg.num_graphs : 1;
  ESC_TRY(b_acc.alloc(sizeof(Acc128) * ACC_COUNT * G));
  ESC_TRY(b_ctr.alloc(sizeof(unsigned long long) * 16));
  uint32_t* T = b_T.as<uint32_t>();
  unsigned long long *K4e = b_K4e.as<unsigned long long>(), *C4e = b_C4e.as<unsigned long long>();
  unsigned long long *tv = b_tv.as<unsigned long long>(), *C4v = b_C4v.as<unsigned long long>(),
                     *K4v = b_K4v.as<unsigned long long>();
  Acc128* acc = b_acc.as<Acc128>();
  unsigned long long* ctr = b_ctr.as<unsigned long long>();
  cudaMemsetAsync(T, 0, sizeof(uint32_t) * (nnz + 1), s);
  cudaMemsetAsync(K4e, 0, sizeof(unsigned long long) * (nnz + 1), s);
  cudaMemsetAsync(C4e, 0, sizeof(unsigned long long) * (nnz + 1), s);
  cudaMemsetAsync(C4v, 0, sizeof(unsigned long long) * (n + 1), s);
  cudaMemsetAsync(acc, 0, sizeof(Acc128) * ACC_COUNT * G, s);
  DevBuf b_vg, b_narr, b_marr;
  ESC_TRY(b_narr.alloc(sizeof(unsigned long long) * G));
  ESC_TRY(b_marr.alloc(sizeof(unsigned long long) * G));
  AccSet accs{acc, nullptr};
  if (G > 1) {
    ESC_TRY(b_vg.alloc(sizeof(int32_t) * (n + 1)));
    if (n > 0)
      (k_graph_of_vertex<<<grid_for(n, TPB, sms), TPB, 0, s>>>(cfg.d_vtx_offsets, G, o.rank, n, b_vg.as<int32_t>()),
       note_launch());
    (k_graph_sizes<<<(G + 127) / 128, 128, 0, s>>>(cfg.d_vtx_offsets, rp, G, b_narr.as<unsigned long long>(),
                                                   b_marr.as<unsigned long long>()), note_launch());
    accs.vg = b_vg.as<int32_t>();
  } else {
    unsigned long long nm[2] = {(unsigned long long)n, (unsigned long long)(nnz / 2)};
    cudaMemcpyAsync(b_narr.p, &nm[0], sizeof(unsigned long long), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(b_marr.p, &nm[1], sizeof(unsigned long long), cudaMemcpyHostToDevice, s);
    ESC_TRY(cudaStreamSynchronize(s));   // nm lives on this stack frame
  }
  cudaMemsetAsync(ctr, 0, sizeof(unsigned long long) * 16, s);
  // a census split over parts: the sweeps take the owned items only, and the
  // sums of the phases every part repeats (degree sums, triangles) count on
  // part 0 alone (the others add them to a discarded row)
  const Owner own{cfg.part, std::max(1, cfg.parts)};
  AccSet acc_rep = accs;
  DevBuf b_junk;
  if (own.part != 0) {
    ESC_TRY(b_junk.alloc(sizeof(Acc128) * ACC_COUNT * G));
    acc_rep.base = b_junk.as<Acc128>();
  }

  if (n > 0) (k_vertex_basic<<<grid_for(n * 32, TPB, sms), TPB, 0, s>>>(g, acc_rep), note_launch());

  // ---------------- item lists for the out-neighbourhood passes
  DevBuf b_small, b_large, b_wsmall, b_csmall, b_clarge, b_dims;
  ESC_TRY(b_small.alloc(sizeof(int32_t) * (n + 1)));
  ESC_TRY(b_large.alloc(sizeof(int32_t) * (n + 1)));
  ESC_TRY(b_wsmall.alloc(sizeof(int32_t) * (n + 1)));
  ESC_TRY(b_csmall.alloc(sizeof(int32_t) * (n + 1)));
  ESC_TRY(b_clarge.alloc(sizeof(int32_t) * (n + 1)));
  ESC_TRY(b_dims.alloc(sizeof(unsigned long long) * 2));
  cudaMemsetAsync(b_dims.p, 0, sizeof(unsigned long long) * 2, s);
  if (n > 0) {
    (k_split_items<<<grid_for(n, TPB, sms), TPB, 0, s>>>(g, b_small.as<int32_t>(), b_large.as<int32_t>(),
                                                          b_wsmall.as<int32_t>(), b_csmall.as<int32_t>(),
                                                          b_clarge.as<int32_t>(), ctr, SMALL_DPLUS,
                                                          std::min(CLQ_WARP_DIN, env_int("ESC_CLQ_WARP_DIN", CLQ_WARP_DIN)),
                                                          own), note_launch());
    (k_clique_dims<<<grid_for(n, TPB, sms), TPB, 0, s>>>(g, b_dims.as<unsigned long long>()), note_launch());
  }
  unsigned long long hcnt[16] = {0}, dims[2] = {0, 0};
  cudaMemcpyAsync(hcnt, ctr, sizeof(hcnt), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(dims, b_dims.p, sizeof(dims), cudaMemcpyDeviceToHost, s);
  ESC_TRY(cudaStreamSynchronize(s));
  int64_t nsmall = (int64_t)hcnt[0], nlarge = (int64_t)hcnt[1];
  int64_t nwsmall = (int64_t)hcnt[2], ncsmall = (int64_t)hcnt[3], nclarge = (int64_t)hcnt[4];
  int dmax = (int)dims[1];
  if (dmax < SMALL_DPLUS + 1) dmax = SMALL_DPLUS + 1;
  cudaMemsetAsync(ctr, 0, sizeof(unsigned long long) * 16, s);

  // ---------------- pass A: triangles
  mark(1, 0, s);
  int hcap_a = pow2_at_least(2 * dmax);
  size_t smem_a = sizeof(int32_t) * (2 * (size_t)hcap_a) + sizeof(uint32_t) * dmax;
  int grid_sweep = sms * (cfg.cta_per_sm > 0 ? cfg.cta_per_sm : 1);
  if (nsmall > 0)
    (k_tri_small<<<grid_for(nsmall * 32, TPB, sms), TPB, 0, s>>>(g, b_small.as<int32_t>(), nsmall, T, acc_rep),
     note_launch());
  if (nlarge > 0) {
    if (smem_a > 48 * 1024) ESC_TRY(allow_max_smem((const void*)k_tri_large, smem_optin));
    (k_tri_large<<<(unsigned)std::min<int64_t>(grid_sweep, nlarge), 512, smem_a, s>>>(
        g, b_large.as<int32_t>(), nlarge, ctr + 0, T, acc_rep, hcap_a), note_launch());
  }
  if (n > 0) {
    (k_sym_T<<<grid_for(n * 32, TPB, sms), TPB, 0, s>>>(g, T, tv), note_launch());
    (k_vertex_from_edges_T<<<grid_for(n * 32, TPB, sms), TPB, 0, s>>>(g, T, tv), note_launch());
  }
  mark(1, 1, s);

  // ---------------- everything the concurrent phases need is sized and
  // allocated here, so no branch below waits on the host
  int dev = 0;
  cudaGetDevice(&dev);
  // pass B inputs
  // CTA items: every large out-neighbourhood, then the small ones with many
  // in-neighbours; the other small ones go to the warp kernel
  int64_t nitems_b = nclarge + ncsmall;
  DevBuf b_items, b_D;
  ESC_TRY(b_items.alloc(sizeof(int32_t) * (nitems_b + 1)));
  if (nclarge) cudaMemcpyAsync(b_items.p, b_clarge.p, sizeof(int32_t) * nclarge, cudaMemcpyDeviceToDevice, s);
  if (ncsmall)
    cudaMemcpyAsync(b_items.as<int32_t>() + nclarge, b_csmall.p, sizeof(int32_t) * ncsmall, cudaMemcpyDeviceToDevice,
                    s);
  // out-degrees up to dsplit keep the bit matrix in shared memory; the few
  // larger ones (dense graphs) use a per-CTA region of global memory
  int dsplit = dmax;
  while (dsplit > SMALL_DPLUS + 1 &&
         clique_space(dsplit) + 1024 + sizeof(uint64_t) * 32 * CLQ_MAX_WARPS > (size_t)smem_optin)
    --dsplit;
  const int dmax_s = std::min(dmax, dsplit);
  int hcap_b = pow2_at_least(2 * dmax_s);
  size_t smem_b = clique_space(dmax_s);
  ESC_TRY(allow_max_smem((const void*)k_clique_large<false>, smem_optin));
  // as many 256-thread CTAs per SM as registers and the bit matrix allow;
  // one 512-thread CTA per SM when fewer than two fit (large bit matrices)
  int clq_threads = 256, clq_per_sm = 1;
  ESC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&clq_per_sm, k_clique_large<false>, clq_threads, smem_b));
  if (clq_per_sm < 2) {
    clq_threads = 512;
    clq_per_sm = 1;
  }
  const int blocks_b = sms * std::min(clq_per_sm, 4);
  unsigned long long dwords = dims[0] > 0 ? dims[0] : 1;
  ESC_TRY(b_D.alloc(sizeof(uint64_t) * dwords * blocks_b));
  DevBuf b_Gq;
  int blocks_g = 0;
  int64_t gwords = 0;
  if (dmax > dsplit) {
    gwords = (int64_t)((clique_space(dmax) + 7) / 8);
    // at most one CTA per SM, and at most 8 GiB of work space in all
    blocks_g = (int)std::max<int64_t>(1, std::min<int64_t>(sms, ((int64_t)8 << 30) / (8 * gwords)));
    ESC_TRY(b_Gq.alloc(sizeof(uint64_t) * (size_t)gwords * blocks_g));
  }
  CliqueScratch cs{b_D.as<uint64_t>(), (int64_t)dwords, b_Gq.as<uint64_t>(), gwords};

  // sweep scratch: one set per concurrent sweep (4-cycles; pairs and the
  // tagged 5-cycle counters are sized below, once the largest degree is known)
  // With four_only, only the 4-cycle sweep runs; the lists, pairs, wheels and
  // 5-cycles (and their work space) are skipped.
  const bool five = !cfg.four_only;
  DevBuf b_cntA, b_cntB, b_cntC, b_cntD, b_tlD, b_ntC;
  size_t sw = five ? sizeof(uint32_t) * (size_t)n * grid_sweep + 16 : 16;
  ESC_TRY(b_cntD.alloc(sw)); ESC_TRY(b_tlD.alloc(sw));
  ESC_TRY(b_ntC.alloc(sizeof(unsigned) * 2 * grid_sweep));
  cudaMemsetAsync(b_cntD.p, 0, sw, s);

  // common-neighbour list offsets and sizes
  DevBuf b_off, b_offp, b_U, b_P, b_gh;
  ESC_TRY(b_off.alloc(sizeof(int64_t) * (nnz + 2)));
  ESC_TRY(b_offp.alloc(sizeof(int64_t) * (nnz + 2)));
  int64_t* off = b_off.as<int64_t>();
  int64_t* offp = b_offp.as<int64_t>();
  int64_t ulen = 0, plen = 0;
  if (five) {
    if (n > 0) (k_canon_counts<<<grid_for(n * 32, TPB, sms), TPB, 0, s>>>(g, T, off), note_launch());
    ESC_TRY(exclusive_scan_i64(off, off, nnz, true, arena, s));
    if (n > 0) (k_all_counts<<<grid_for(nnz, TPB, sms), TPB, 0, s>>>(T, nnz, offp), note_launch());
    ESC_TRY(exclusive_scan_i64(offp, offp, nnz, true, arena, s));
    cudaMemcpyAsync(&ulen, off + nnz, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&plen, offp + nnz, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  }
  // pair-sweep items by wedge count (light / medium / heavy lists)
  DevBuf b_plist, b_pctr;
  ESC_TRY(b_plist.alloc(five ? sizeof(int32_t) * 3 * (size_t)(n + 1) : 16));
  ESC_TRY(b_pctr.alloc(sizeof(unsigned long long) * 8));
  cudaMemsetAsync(b_pctr.p, 0, sizeof(unsigned long long) * 8, s);
  unsigned long long pcnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (five && n > 0) {
    // item classes: hash capacities bound the light and medium classes
    // (ESC_PAIR_SMALL_W / ESC_PAIR_LARGE_W lower them for tuning)
    const long long w_small = std::min<long long>(PH_SMALL_W, env_int("ESC_PAIR_SMALL_W", PH_SMALL_W + 1) - 1);
    const long long w_large = std::min<long long>(PH_LARGE_W, env_int("ESC_PAIR_LARGE_W", PH_LARGE_W + 1) - 1);
    (k_pair_classify<<<grid_for(n * 32, TPB, sms), TPB, 0, s>>>(g, T, b_plist.as<int32_t>(),
                                                                b_pctr.as<unsigned long long>(), w_small,
                                                                std::max(w_small, w_large), own), note_launch());
    cudaMemcpyAsync(pcnt, b_pctr.p, sizeof(pcnt), cudaMemcpyDeviceToHost, s);
  }
  std::vector<int64_t> hR(n + 1, 0);
  if (n > 0) cudaMemcpyAsync(hR.data(), o.R, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, s);
  ESC_TRY(cudaStreamSynchronize(s));
  if (five && n > 0) (k_share_offsets<<<grid_for(n * 32, TPB, sms), TPB, 0, s>>>(g, off), note_launch());
  ESC_TRY(b_U.alloc(sizeof(int32_t) * (ulen + 1)));
  ESC_TRY(b_P.alloc(sizeof(int32_t) * (plen + 1)));
  int64_t maxdeg = n > 0 ? hR[n] - hR[n - 1] : 0;   // the highest rank has the largest degree
  // 4-cycle, pair and 5-cycle sweeps: tagged counters, 32-bit words below the first
  // rank of degree >= 2^16, 64-bit words from there on
  int64_t jbig = n;
  {
    int64_t lo = 0, hi = n;
    while (lo < hi) { int64_t mid = (lo + hi) >> 1; if (hR[mid + 1] - hR[mid] >= 65536) hi = mid; else lo = mid + 1; }
    jbig = lo;
  }
  // the heavy pair items: clusters sharing one counter array each
  PairPlan pplan;
  int64_t n0 = 0;                               // first rank of degree >= 1 (lower ranks are never counted)
  if (five && pcnt[2] > 0) {
    {
      int64_t lo = 0, hi = n;
      while (lo < hi) { int64_t mid = (lo + hi) >> 1; if (hR[mid + 1] - hR[mid] >= 1) hi = mid; else lo = mid + 1; }
      n0 = lo;
    }
    size_t arr_bytes = sizeof(uint32_t) * (size_t)std::max<int64_t>(jbig - n0, 0) +
                       sizeof(unsigned long long) * (size_t)(n - jbig);
    ESC_TRY(plan_pair_clusters(jbig < n, sms, arr_bytes, n0, jbig, smem_optin, cfg.num_graphs > 1, &pplan));
  }
  // task buffers of the heavy pair items: the largest item has at most
  // w_max / PAIR_TASK + d_max tasks
  DevBuf b_ptq, b_ptn;
  PairTasks ptasks{nullptr, nullptr, 0};
  if (five && pcnt[2] > 0) {
    ptasks.cap = (int64_t)(pcnt[6] / PAIR_TASK) + maxdeg + 1;
    ESC_TRY(b_ptq.alloc(sizeof(long long) * 2 * (size_t)ptasks.cap * pplan.nclusters));
    ESC_TRY(b_ptn.alloc(sizeof(unsigned long long) * (size_t)pplan.nclusters));
    cudaMemsetAsync(b_ptn.p, 0, sizeof(unsigned long long) * (size_t)pplan.nclusters, s);
    ptasks.q = b_ptq.as<long long>();
    ptasks.n = b_ptn.as<unsigned long long>();
  }
  size_t sw32 = sizeof(uint32_t) * (size_t)jbig * grid_sweep + 16;
  size_t sw64 = sizeof(unsigned long long) * (size_t)(n - jbig) * grid_sweep + 16;
  size_t sw32p = five && !pplan.windowed ? sizeof(uint32_t) * (size_t)jbig * pplan.nclusters + 16 : 16;
  size_t sw64p = five ? sizeof(unsigned long long) * (size_t)(n - jbig) * pplan.nclusters + 16 : 16;
  size_t sw32c = five ? sw32 : 16, sw64c = five ? sw64 : 16;
  DevBuf b_bigA, b_bigB, b_bigC;
  ESC_TRY(b_cntA.alloc(sw32)); ESC_TRY(b_bigA.alloc(sw64));
  ESC_TRY(b_cntB.alloc(sw32p)); ESC_TRY(b_bigB.alloc(sw64p));
  ESC_TRY(b_cntC.alloc(sw32c)); ESC_TRY(b_bigC.alloc(sw64c));
  cudaMemsetAsync(b_cntA.p, 0, sw32, s);
  cudaMemsetAsync(b_cntB.p, 0, sw32p, s);
  cudaMemsetAsync(b_cntC.p, 0, sw32c, s);
  cudaMemsetAsync(b_bigA.p, 0, sw64, s);
  cudaMemsetAsync(b_bigB.p, 0, sw64p, s);
  cudaMemsetAsync(b_bigC.p, 0, sw64c, s);
  TagScratch tsA{b_cntA.as<uint32_t>(), b_bigA.as<unsigned long long>(), jbig, n};
  TagScratch tsB{b_cntB.as<uint32_t>(), b_bigB.as<unsigned long long>(), jbig, n};
  // the windowed heavy items: per CTA the dense 16-bit counts and the list cursors
  DevBuf b_g16, b_curs;
  PairWin pwin{};
  if (five && pplan.windowed) {
    pwin.g16_words = ((n + 2) / 2 + 4 + 3) & ~(int64_t)3;
    pwin.curs_cap = std::max<int64_t>(maxdeg, 1);
    ESC_TRY(b_g16.alloc(sizeof(uint32_t) * (size_t)pwin.g16_words * pplan.nclusters));
    ESC_TRY(b_curs.alloc(sizeof(longlong2) * (size_t)pwin.curs_cap * pplan.nclusters));
    pwin.g16 = b_g16.as<uint32_t>();
    pwin.curs = b_curs.as<longlong2>();
    pwin.side = b_bigB.as<unsigned long long>();      // zeroed above
    pwin.jbig = jbig;
    pwin.n = n;
    pwin.n0 = n0;
    pwin.win_words = pplan.win_words;
    pwin.woff = (int)((4 - (((jbig + (jbig & 1)) >> 1) & 3)) & 3);
  }
  TagScratch tsC{b_cntC.as<uint32_t>(), b_bigC.as<unsigned long long>(), jbig, n};
  SweepScratch ssC{nullptr, nullptr, b_cntD.as<uint32_t>(), b_tlD.as<int32_t>(), b_ntC.as<unsigned>(), n};
  const int hcap_l = 8192;
  int64_t ghash_cap = pow2_at_least((int)std::max<int64_t>(2 * maxdeg, 2));
  if (2 * maxdeg <= hcap_l) ghash_cap = 2;
  ESC_TRY(b_gh.alloc(five ? sizeof(int32_t) * 2 * (size_t)ghash_cap * grid_sweep + 16 : 16));
  size_t smem_l = sizeof(int32_t) * 2 * (size_t)hcap_l;
  ESC_TRY(allow_max_smem((const void*)k_tri_lists, smem_optin));
  TriLists tl3{off, b_U.as<int32_t>(), offp, b_P.as<int32_t>()};

  // wheel work items: ranks are in degree order, so the large centres are a suffix
  int64_t c0 = n;
  {
    // first rank with degree > the warp items' limit (WHEEL_WARP_MAX, or lower
    // with ESC_WHEEL_WARP_MAX)
    const int64_t wmax = std::min(WHEEL_WARP_MAX, env_int("ESC_WHEEL_WARP_MAX", WHEEL_WARP_MAX));
    int64_t lo = 0, hi = n;
    while (lo < hi) { int64_t mid = (lo + hi) >> 1; if (hR[mid + 1] - hR[mid] > wmax) hi = mid; else lo = mid + 1; }
    c0 = lo;
  }
  DevBuf b_io, b_gs;
  int64_t nitems_w = 0;
  // counters in shared memory up to half the opt-in size: two CTAs per SM
  int smem_cap = std::max(0, (smem_optin / 2 - 4096) / 4);
  smem_cap = (int)std::min<int64_t>(smem_cap, maxdeg);
  int64_t gstride = maxdeg > smem_cap ? maxdeg : 1;
  size_t smem_w = sizeof(uint32_t) * (size_t)std::max(smem_cap, 1);
  std::vector<int64_t> item_off(n - c0 + 1, 0);
  if (five && c0 < n) {
    for (int64_t c = c0; c < n; ++c)
      item_off[c - c0 + 1] = item_off[c - c0] + (own.owns(c) ? (hR[c + 1] - hR[c] + WHEEL_CHUNK - 1) / WHEEL_CHUNK : 0);
    nitems_w = item_off[n - c0];
    ESC_TRY(b_io.alloc(sizeof(int64_t) * (n - c0 + 1)));
    cudaMemcpyAsync(b_io.p, item_off.data(), sizeof(int64_t) * (n - c0 + 1), cudaMemcpyHostToDevice, s);
    ESC_TRY(b_gs.alloc(sizeof(unsigned long long) * (size_t)gstride * 2 * sms + 16));
    cudaMemsetAsync(b_gs.p, 0, sizeof(unsigned long long) * (size_t)gstride * 2 * sms + 16, s);
    ESC_TRY(allow_max_smem((const void*)k_wheels_cta, smem_optin));
  }
  DevBuf b_wo;                                 // warp wheel items: offsets over centres c0-1 .. 0
  if (five && c0 > 0) {
    ESC_TRY(b_wo.alloc(sizeof(int64_t) * (size_t)(c0 + 1)));
    (k_wheel_warp_counts<<<grid_for(c0, TPB, sms), TPB, 0, s>>>(g, c0, b_wo.as<int64_t>(), own), note_launch());
    ESC_TRY(exclusive_scan_i64(b_wo.as<int64_t>(), b_wo.as<int64_t>(), c0, true, arena, s));
  }

  // ---------------- concurrent phases on forked streams
  // The common-neighbour lists come first (short when alone); then
  //   s3 (most urgent): wheels      s : pairs
  //   s1, s2, s4 (least urgent): cliques, 4-cycles, 5-cycles; s joins all.
  mark(4, 0, s);
  if (five && n > 0)
    (k_tri_lists<<<grid_sweep, 512, smem_l, s>>>(g, ctr + 3, off, offp, T, b_U.as<int32_t>(), b_P.as<int32_t>(),
                                                 b_gh.as<int32_t>(), ghash_cap, hcap_l, d_status), note_launch());
  mark(4, 1, s);
  StreamSet ss_all;
  cudaStream_t s1 = s, s2 = s, s3 = s, s4 = s;
  if (!cfg.serial_phases) {
    const int urgent[4] = {0, 0, 1, 0};
    ESC_TRY(ss_all.create(4, urgent));
    s1 = ss_all.st[0]; s2 = ss_all.st[1]; s3 = ss_all.st[2]; s4 = ss_all.st[3];
    ESC_TRY(ss_all.fork_from(s, {s1, s2, s3, s4}));
  }

  // wheels (Thm 11): the longest phase, started first
  mark(6, 0, s3);
  if (five && c0 < n)
    (k_wheels_cta<<<2 * sms, 512, smem_w, s3>>>(g, c0, b_io.as<int64_t>(), nitems_w, ctr + 5, tl3, T,
                                            b_gs.as<unsigned long long>(), gstride, smem_cap, accs,
                                            pcnt[7] < 65536 && env_int("ESC_WHEEL_WINDOW", 2) != 1), note_launch());
  if (five && c0 > 0) {
    int per_sm = 1;
    ESC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wheels_warp, 256, 0));
    (k_wheels_warp<<<(unsigned)std::max(1, per_sm) * sms, 256, 0, s3>>>(g, c0, b_wo.as<int64_t>(), ctr + 7, tl3, T,
                                                                          accs), note_launch());
  }
  mark(6, 1, s3);
  // pairs (Thms 11, 12); 16-bit counters when no degree reaches 2^16 (then no W(i,j) can)
  mark(5, 0, s);
  if (five && n > 0) {
    unsigned long long* pq = b_pctr.as<unsigned long long>() + 3;     // queue counters of the three lists
    const int32_t* pl = b_plist.as<int32_t>();
    if (pcnt[0] > 0) {
      const size_t sm0 = (sizeof(int32_t) + sizeof(uint32_t)) * PH_SMALL_SLOTS;
      int per_sm = 1;
      ESC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pairs_hash<PH_SMALL_SLOTS>, PH_SMALL_THREADS,
                                                            sm0));
      unsigned grid = (unsigned)std::min<int64_t>((int64_t)std::max(1, per_sm) * sms, (int64_t)pcnt[0]);
      (k_pairs_hash<PH_SMALL_SLOTS><<<grid, PH_SMALL_THREADS, sm0, s>>>(g, pl, (int64_t)pcnt[0], pq + 0, tl3, T, accs,
                                                                       d_status), note_launch());
    }
    if (pcnt[1] > 0) {
      const size_t sm1 = (sizeof(int32_t) + sizeof(uint32_t)) * PH_LARGE_SLOTS;
      ESC_TRY(allow_max_smem((const void*)k_pairs_hash<PH_LARGE_SLOTS>, smem_optin));
      int per_sm = 1;
      ESC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pairs_hash<PH_LARGE_SLOTS>, PH_LARGE_THREADS,
                                                            sm1));
      unsigned grid = (unsigned)std::min<int64_t>((int64_t)std::max(1, per_sm) * sms, (int64_t)pcnt[1]);
      (k_pairs_hash<PH_LARGE_SLOTS><<<grid, PH_LARGE_THREADS, sm1, s>>>(g, pl + n, (int64_t)pcnt[1], pq + 1, tl3, T,
                                                                       accs, d_status), note_launch());
    }
    if (pcnt[2] > 0 && pplan.windowed) {
      const size_t smw = sizeof(uint32_t) * (size_t)pplan.win_words;
      if (jbig < n)
        (k_pairs_win<true><<<pplan.nclusters, pplan.threads, smw, s>>>(g, pl + 2 * n, (int64_t)pcnt[2], pq + 2, pwin,
                                                                      tl3, T, accs, ptasks, d_status), note_launch());
      else
        (k_pairs_win<false><<<pplan.nclusters, pplan.threads, smw, s>>>(g, pl + 2 * n, (int64_t)pcnt[2], pq + 2, pwin,
                                                                       tl3, T, accs, ptasks, d_status), note_launch());
    } else if (pcnt[2] > 0) {
      ESC_TRY(launch_pairs_grp(jbig < n, pplan, g, pl + 2 * n, (int64_t)pcnt[2], pq + 2, tsB, tl3, T, accs, ptasks,
                               s));
    }
  }
  mark(5, 1, s);
  // cliques and per-triangle sums (Thms 6, 7, 10, 14)
  mark(2, 0, s1);
  if (nitems_b > 0)
    (k_clique_large<false><<<(unsigned)std::min<int64_t>(blocks_b, nitems_b), clq_threads, smem_b, s1>>>(
        g, b_items.as<int32_t>(), nitems_b, ctr + 1, T, K4e, accs, cs, hcap_b, -1, dmax_s, d_status, five),
     note_launch());
  if (nitems_b > 0 && blocks_g > 0)
    (k_clique_large<true><<<(unsigned)std::min<int64_t>(blocks_g, nitems_b), 512, 0, s1>>>(
        g, b_items.as<int32_t>(), nitems_b, ctr + 9, T, K4e, accs, cs, pow2_at_least(2 * dmax), dsplit, dmax,
        d_status, five), note_launch());
  if (nwsmall > 0) {
    int per_sm = 1;
    ESC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_clique_warp, CLQ_WARPS * 32, 0));
    unsigned grid_w = (unsigned)std::min<int64_t>((int64_t)std::max(1, per_sm) * sms, (nwsmall + CLQ_WARPS - 1) / CLQ_WARPS);
    (k_clique_warp<<<grid_w, CLQ_WARPS * 32, 0, s1>>>(g, b_wsmall.as<int32_t>(), nwsmall, ctr + 8, T, K4e, accs,
                                                      five), note_launch());
  }
  if (n > 0) {
    (k_sym_u64<<<grid_for(n * 32, TPB, sms), TPB, 0, s1>>>(g, K4e), note_launch());
    if (!cfg.partial)                          // a part's K4 sums are divided once every part's are in
      (k_vertex_sum_div<<<grid_for(n * 32, TPB, sms), TPB, 0, s1>>>(g, K4e, K4v, 3), note_launch());
  }
  mark(2, 1, s1);
  // 4-cycles (Thm 5)
  mark(3, 0, s2);
  if (n > 0) {
    if (jbig < n)
      (k_cycles4<true><<<grid_sweep, 512, 0, s2>>>(g, ctr + 2, tsA, C4e, C4v, accs, own), note_launch());
    else
      (k_cycles4<false><<<grid_sweep, 512, 0, s2>>>(g, ctr + 2, tsA, C4e, C4v, accs, own), note_launch());
    (k_fold_u64<<<grid_for(n * 32, TPB, sms), TPB, 0, s2>>>(g, C4e), note_launch());
  }
  mark(3, 1, s2);
  // 5-cycles (Thm 13)
  mark(7, 0, s4);
  if (five && n > 0) {
    if (jbig < n)
      (k_cycles5<true><<<grid_sweep, 512, 0, s4>>>(g, ctr + 6, tsC, ssC, accs, own), note_launch());
    else
      (k_cycles5<false><<<grid_sweep, 512, 0, s4>>>(g, ctr + 6, tsC, ssC, accs, own), note_launch());
  }
  mark(7, 1, s4);
  ESC_TRY(ss_all.join_into(s));

  // ---------------- closed forms over vertices and edges, then assembly
  mark(8, 0, s);
  if (cfg.partial) {
    // one part of a split census: its raw sums; the closed forms need every
    // part's per-element counts and run in run_census_finish
    ESC_TRY(cudaMemcpyAsync(cfg.d_acc_out, acc, sizeof(Acc128) * ACC_COUNT, cudaMemcpyDeviceToDevice, s));
  } else {
    if (n > 0)
      (k_edge_sums<<<grid_for(n * 32, TPB, sms), TPB, 0, s>>>(g, T, C4e, K4e, tv, C4v, K4v, accs), note_launch());
    ConvTables tabs;
    conversion_inverse(3, tabs.a3);
    conversion_inverse(4, tabs.a4);
    conversion_inverse(5, tabs.a5);
    (k_assemble<<<(G + 63) / 64, 64, 0, s>>>(acc, b_narr.as<unsigned long long>(), b_marr.as<unsigned long long>(),
                                            G, tabs, d_out, (u128*)cfg.d_basis), note_launch());
  }
  mark(8, 1, s);

  if (pe_out) {
    // hand the per-element arrays over to the caller (ownership moves)
    pe_out->Te = T; b_T.p = nullptr;
    pe_out->C4e = C4e; b_C4e.p = nullptr;
    pe_out->K4e = K4e; b_K4e.p = nullptr;
    pe_out->tv = tv; b_tv.p = nullptr;
    pe_out->C4v = C4v; b_C4v.p = nullptr;
    pe_out->K4v = K4v; b_K4v.p = nullptr;
  }
  if (or_out) {
    *or_out = o;
    b_perm.p = b_rank.p = b_R.p = b_C.p = b_op.p = b_rev.p = nullptr;
  }
  ESC_TRY(cudaStreamSynchronize(s));   // scratch buffers are freed on return
  return cudaGetLastError();
}

// The end of a split census: every part's sums added (d_acc, ACC_COUNT
// 128-bit words) and every part's per-element counts added into pe (K4e, C4e,
// C4v; T and tv are whole on every part).  K4 per vertex, the closed forms
// over vertices and edges, and the assembly.
cudaError_t run_census_finish(const Oriented& o, int64_t n, int64_t nnz, const PerElement& pe,
                              const unsigned long long* d_acc, unsigned long long* d_out, int sms, cudaStream_t s) {
  CacheScope cache_scope(s);
  const int TPB = 256;
  DevGraph g{n, nnz, o.R, o.C, o.op, o.rev};
  DevBuf b_acc, b_nm;
  ESC_TRY(b_acc.alloc(sizeof(Acc128) * ACC_COUNT));
  ESC_TRY(b_nm.alloc(sizeof(unsigned long long) * 2));
  ESC_TRY(cudaMemcpyAsync(b_acc.p, d_acc, sizeof(Acc128) * ACC_COUNT, cudaMemcpyDeviceToDevice, s));
  unsigned long long nm[2] = {(unsigned long long)n, (unsigned long long)(nnz / 2)};
  ESC_TRY(cudaMemcpyAsync(b_nm.p, nm, sizeof(nm), cudaMemcpyHostToDevice, s));
  AccSet accs{b_acc.as<Acc128>(), nullptr};
  if (n > 0) {
    (k_vertex_sum_div<<<grid_for(n * 32, TPB, sms), TPB, 0, s>>>(g, pe.K4e, pe.K4v, 3), note_launch());
    (k_edge_sums<<<grid_for(n * 32, TPB, sms), TPB, 0, s>>>(g, pe.Te, pe.C4e, pe.K4e, pe.tv, pe.C4v, pe.K4v, accs),
     note_launch());
  }
  ConvTables tabs;
  conversion_inverse(3, tabs.a3);
  conversion_inverse(4, tabs.a4);
  conversion_inverse(5, tabs.a5);
  (k_assemble<<<1, 64, 0, s>>>(b_acc.as<Acc128>(), b_nm.as<unsigned long long>(), b_nm.as<unsigned long long>() + 1,
                               1, tabs, d_out, nullptr), note_launch());
  ESC_TRY(cudaStreamSynchronize(s));   // nm lives on this stack frame
  return cudaGetLastError();
}

int census_sum_count() { return ACC_COUNT; }

}  // namespace esc
