// escape.cu -- the C ABI (include/escape.h): graph handles, the census entry
// points, per-element output and the induced/non-induced conversion tables.
#include "../../include/escape.h"
#include "common.cuh"
#include "internal.h"

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

struct escape_graph {
  int64_t n = 0, nnz = 0;
  int64_t* d_rp = nullptr;     // input CSR, original ids
  int32_t* d_col = nullptr;
  int device = 0, sms = 1;
  int keep_pe = 0, cta_per_sm = 2, serial = -1;   // serial: 1 on, 0 off, -1 by graph size
  bool has_pe = false;
  esc::PerElement pe;
  esc::Oriented ori;
  float phase_ms[9] = {0};
  int num_phases = 0;
  long long launches = 0;     // kernels launched by the last census call
  escape_u128 basis[4] = {};  // W, D, DP, DBP of the last census5 call
  bool has_basis = false;
  bool has_part = false;      // a part of a split census is held (pe, ori)
};

namespace esc {
static thread_local int t_last_cuda = 0;   // escape_last_cuda_error
void note_cuda_error(cudaError_t e) {
  if (e != cudaSuccess) t_last_cuda = (int)e;
}
}  // namespace esc

namespace {

escape_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return ESCAPE_OK;
  esc::note_cuda_error(e);
  if (e == cudaErrorMemoryAllocation) return ESCAPE_ENOMEM;
  if (e == cudaErrorInvalidConfiguration) return ESCAPE_EOVERFLOW;
  cudaGetLastError();   // clear a non-sticky error
  return ESCAPE_ECUDA;
}

void free_pe(escape_graph* g) {
  cudaFree(g->pe.Te); cudaFree(g->pe.C4e); cudaFree(g->pe.K4e);
  cudaFree(g->pe.tv); cudaFree(g->pe.C4v); cudaFree(g->pe.K4v);
  g->pe = esc::PerElement{};
  cudaFree(g->ori.perm); cudaFree(g->ori.rank); cudaFree(g->ori.R); cudaFree(g->ori.C);
  cudaFree(g->ori.op); cudaFree(g->ori.rev);
  g->ori = esc::Oriented{};
  g->has_pe = false;
}

// --------------------------------------------------------------------------
// Pattern catalogue for the conversion tables (App. B), 0-based vertex pairs:
// 5-vertex patterns 1-21 of the paper's connected-pattern figure, 22-32 of its
// disconnected-pattern figure, then wedge + edge and triangle + edge.
// --------------------------------------------------------------------------
struct Pat { int ne; unsigned char e[10][2]; };

const Pat kPat5[34] = {
  {4, {{0,1},{0,2},{0,3},{0,4}}},
  {4, {{0,1},{0,2},{0,3},{1,4}}},
  {4, {{0,1},{0,2},{1,3},{2,4}}},
  {5, {{0,1},{0,2},{1,2},{2,3},{2,4}}},
  {5, {{0,1},{0,2},{1,2},{1,3},{3,4}}},
  {5, {{0,1},{0,2},{1,2},{1,3},{2,4}}},
  {5, {{0,1},{0,2},{1,3},{2,3},{2,4}}},
  {5, {{0,1},{0,2},{1,3},{2,4},{3,4}}},
  {6, {{0,1},{0,2},{1,2},{2,3},{2,4},{3,4}}},
  {6, {{0,1},{0,2},{0,3},{1,3},{2,3},{2,4}}},
  {6, {{0,1},{0,2},{1,2},{1,3},{2,3},{2,4}}},
  {6, {{0,1},{0,2},{1,3},{2,3},{2,4},{3,4}}},
  {6, {{0,1},{0,2},{0,3},{1,4},{2,4},{3,4}}},
  {7, {{0,1},{0,2},{0,3},{0,4},{1,4},{2,4},{3,4}}},
  {7, {{0,1},{0,2},{0,3},{1,2},{1,3},{2,3},{2,4}}},
  {7, {{0,1},{0,2},{1,2},{1,3},{2,3},{2,4},{3,4}}},
  {7, {{0,1},{0,2},{0,3},{1,2},{1,3},{2,4},{3,4}}},
  {8, {{0,1},{0,2},{0,3},{0,4},{1,2},{1,3},{2,4},{3,4}}},
  {8, {{0,1},{0,2},{0,3},{1,2},{1,3},{2,3},{2,4},{3,4}}},
  {9, {{0,2},{0,3},{0,4},{1,2},{1,3},{1,4},{2,3},{2,4},{3,4}}},
  {10, {{0,1},{0,2},{0,3},{0,4},{1,2},{1,3},{1,4},{2,3},{2,4},{3,4}}},
  {0, {}},
  {1, {{0,1}}},
  {2, {{0,1},{2,3}}},
  {2, {{0,1},{1,2}}},
  {3, {{0,1},{0,2},{1,2}}},
  {3, {{0,1},{0,2},{0,3}}},
  {3, {{0,1},{0,2},{1,3}}},
  {4, {{0,1},{0,2},{0,3},{1,2}}},
  {4, {{0,1},{0,2},{1,3},{2,3}}},
  {5, {{0,1},{0,2},{0,3},{1,2},{1,3}}},
  {6, {{0,1},{0,2},{0,3},{1,2},{1,3},{2,3}}},
  {3, {{0,1},{1,2},{3,4}}},
  {4, {{0,1},{0,2},{1,2},{3,4}}},
};
const Pat kPat4[11] = {
  {3, {{0,1},{0,2},{0,3}}},
  {3, {{0,1},{0,2},{1,3}}},
  {4, {{0,1},{0,2},{0,3},{1,2}}},
  {4, {{0,1},{0,2},{1,3},{2,3}}},
  {5, {{0,1},{0,2},{0,3},{1,2},{1,3}}},
  {6, {{0,1},{0,2},{0,3},{1,2},{1,3},{2,3}}},
  {0, {}},
  {1, {{0,1}}},
  {2, {{0,1},{2,3}}},
  {2, {{0,1},{1,2}}},
  {3, {{0,1},{0,2},{1,2}}},
};
const Pat kPat3[4] = {
  {0, {}}, {1, {{0,1}}}, {2, {{0,1},{0,2}}}, {3, {{0,1},{0,2},{1,2}}},
};

// adjacency matrix of a pattern as a k x k bool table
void pat_adj(const Pat& p, int k, bool adj[5][5]) {
  for (int a = 0; a < 5; ++a) for (int b = 0; b < 5; ++b) adj[a][b] = false;
  for (int t = 0; t < p.ne; ++t) { adj[p.e[t][0]][p.e[t][1]] = true; adj[p.e[t][1]][p.e[t][0]] = true; }
  (void)k;
}

// number of bijections sigma of {0..k-1} with sigma(E_small) subset of E_big
long long embeddings(const Pat& small, const Pat& big, int k) {
  bool As[5][5], Ab[5][5];
  pat_adj(small, k, As);
  pat_adj(big, k, Ab);
  int perm[5] = {0, 1, 2, 3, 4};
  long long cnt = 0;
  // lexicographic permutations
  while (true) {
    bool ok = true;
    for (int a = 0; a < k && ok; ++a)
      for (int b = a + 1; b < k && ok; ++b)
        if (As[a][b] && !Ab[perm[a]][perm[b]]) ok = false;
    if (ok) ++cnt;
    int i = k - 2;
    while (i >= 0 && perm[i] > perm[i + 1]) --i;
    if (i < 0) break;
    int j = k - 1;
    while (perm[j] < perm[i]) --j;
    int t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    for (int l = i + 1, r = k - 1; l < r; ++l, --r) { t = perm[l]; perm[l] = perm[r]; perm[r] = t; }
  }
  return cnt;
}

}  // namespace

namespace esc {
static thread_local long long g_launches = 0;
void note_launch() { ++g_launches; }
long long launches_so_far() { return g_launches; }

// A[i][j] = (embeddings of pattern i into pattern j) / |Aut(pattern i)| = the
// number of spanning subgraphs of pattern j isomorphic to pattern i; its
// inverse by back-substitution (A is unit triangular when classes are ordered
// by edge count).
void conversion_inverse(int k, long long* Ainv) {
  const Pat* P = k == 3 ? kPat3 : (k == 4 ? kPat4 : kPat5);
  int c = k == 3 ? 4 : (k == 4 ? 11 : 34);
  std::vector<long long> A((size_t)c * c);
  for (int i = 0; i < c; ++i) {
    long long aut = embeddings(P[i], P[i], k);
    for (int j = 0; j < c; ++j) A[(size_t)i * c + j] = embeddings(P[i], P[j], k) / aut;
  }
  // X = A^-1: column by column, rows from most edges to fewest
  std::vector<int> order(c);
  for (int i = 0; i < c; ++i) order[i] = i;
  for (int a = 0; a < c; ++a)
    for (int b = a + 1; b < c; ++b)
      if (P[order[b]].ne > P[order[a]].ne) { int t = order[a]; order[a] = order[b]; order[b] = t; }
  for (int col = 0; col < c; ++col) {
    std::vector<long long> x(c, 0);
    for (int oi = 0; oi < c; ++oi) {
      int i = order[oi];
      long long s = (i == col) ? 1 : 0;
      for (int j = 0; j < c; ++j)
        if (j != i && A[(size_t)i * c + j]) s -= A[(size_t)i * c + j] * x[j];
      x[i] = s;    // A[i][i] == 1
    }
    for (int i = 0; i < c; ++i) Ainv[(size_t)i * c + col] = x[i];
  }
}
}  // namespace esc

namespace {

int device_sms(int dev) {
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

// batch: local ids of graph k's rows become union ids (add the graph's first
// vertex); an id outside its own graph is flagged and left in range
__global__ void k_globalize(const int64_t* voff, int num_graphs, const int64_t* rp, int64_t rows, int32_t* col,
                            unsigned* status) {
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int lane = threadIdx.x & 31;
  for (int64_t r = warp; r < rows; r += nwarps) {
    int lo = 0, hi = num_graphs;
    while (hi - lo > 1) { int mid = (lo + hi) >> 1; if (voff[mid] <= r) lo = mid; else hi = mid; }
    int64_t base = voff[lo], nk = voff[lo + 1] - base;
    for (int64_t p = rp[r] + lane; p < rp[r + 1]; p += 32) {
      int32_t v = col[p];
      if (v < 0 || v >= nk) { atomicOr(status, 1u); col[p] = (int32_t)r; continue; }   // later rejected
      col[p] = (int32_t)(base + v);
    }
  }
}

// input slot p (u -> v, original ids) -> value at the rank-space slot
__global__ void k_map_edges(const int64_t* rp, const int32_t* col, int64_t n, const int32_t* rank,
                            const int64_t* R, const int32_t* C, const uint32_t* Te, const unsigned long long* C4e,
                            const unsigned long long* K4e, unsigned long long* oT, unsigned long long* oC4,
                            unsigned long long* oK4) {
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int lane = threadIdx.x & 31;
  for (int64_t u = warp; u < n; u += nwarps) {
    int32_t ru = rank[u];
    for (int64_t p = rp[u] + lane; p < rp[u + 1]; p += 32) {
      int32_t rv = rank[col[p]];
      int64_t q = lower_bound_i32(C, R[ru], R[ru + 1], rv);
      oT[p] = Te[q];
      oC4[p] = C4e[q];
      oK4[p] = K4e[q];
    }
  }
}

__global__ void k_map_vertices(int64_t n, const int32_t* rank, const unsigned long long* tv,
                               const unsigned long long* C4v, const unsigned long long* K4v, unsigned long long* ot,
                               unsigned long long* oc, unsigned long long* ok) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
    int32_t r = rank[u];
    ot[u] = tv[r];
    oc[u] = C4v[r];
    ok[u] = K4v[r];
  }
}

// Every row offset of a CSR held in host memory: rp[0] = 0, non-decreasing,
// rp[rows] = nnz (nnz < 0: only rp[0] = 0 and monotone, nnz taken from the
// last entry).  Kernels index col through these offsets, so a CSR from device
// memory is copied here and checked before any kernel sees it.
bool row_ptr_ok(const int64_t* rp, int64_t rows, int64_t nnz) {
  if (rp[0] != 0) return false;
  for (int64_t i = 0; i < rows; ++i)
    if (rp[i + 1] < rp[i]) return false;
  return nnz < 0 || rp[rows] == nnz;
}

// The row offsets of a device-memory CSR, copied to the host (synchronises s).
cudaError_t fetch_row_ptr(const int64_t* d_rp, int64_t rows, std::vector<int64_t>& h, cudaStream_t s) {
  h.resize((size_t)rows + 1);
  cudaError_t e = cudaMemcpyAsync(h.data(), d_rp, sizeof(int64_t) * (rows + 1), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

escape_status census_one(escape_graph* g, const int64_t* d_rp, const int32_t* d_col, int64_t n, int64_t nnz,
                         escape_census* out, cudaStream_t s, bool keep, esc::PerElement* pe, esc::Oriented* ori,
                         float* phase_ms, int* nphase, bool four_only = false) {
  unsigned long long* d_out = nullptr;
  unsigned* d_status = nullptr;
  cudaError_t e = cudaMalloc(&d_out, sizeof(escape_census) + sizeof(escape_u128) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&d_status, sizeof(unsigned));
  if (e != cudaSuccess) { cudaFree(d_out); return from_cuda(e); }
  cudaMemsetAsync(d_status, 0, sizeof(unsigned), s);
  cudaEvent_t evs[18];
  int nev = phase_ms ? 18 : 0;
  for (int i = 0; i < nev; ++i) cudaEventCreate(&evs[i]);
  esc::CensusConfig cfg;
  cfg.sms = g->sms;
  cfg.cta_per_sm = g->cta_per_sm;
  cfg.keep_per_element = keep;
  // automatic: one phase after another once the graph is large enough that
  // every sweep fills the GPU alone (overlapping them then only adds contention)
  cfg.serial_phases = g->serial > 0 || (g->serial < 0 && nnz >= ((int64_t)1 << 24));
  cfg.phase_events = nev ? evs : nullptr;
  cfg.num_phase_events = nev;
  cfg.four_only = four_only;
  cfg.d_basis = d_out + sizeof(escape_census) / sizeof(unsigned long long);
  e = esc::run_census(d_rp, d_col, n, nnz, cfg, d_out, d_status, keep ? pe : nullptr,
                      keep ? ori : nullptr, s);
  escape_status st = from_cuda(e);
  unsigned hstat = 0;
  if (st == ESCAPE_OK) {
    escape_census tmp;
    escape_u128 basis[4];
    e = cudaMemcpyAsync(&tmp, d_out, sizeof(escape_census), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(basis, cfg.d_basis, sizeof(basis), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hstat, d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    st = from_cuda(e);
    if (st == ESCAPE_OK && hstat != 0) st = ESCAPE_EINTERNAL;
    if (st == ESCAPE_OK) {
      *out = tmp;
      for (int i = 0; i < 4; ++i) g->basis[i] = basis[i];
      g->has_basis = !four_only;
    }
  }
  if (nev) {
    int phases = 0;
    for (int i = 0; 2 * i + 1 < nev; ++i) {       // phase i: events 2i .. 2i+1
      float ms = 0;
      if (cudaEventElapsedTime(&ms, evs[2 * i], evs[2 * i + 1]) == cudaSuccess) { phase_ms[i] = ms; phases = i + 1; }
    }
    cudaGetLastError();
    *nphase = phases;
    for (int i = 0; i < nev; ++i) cudaEventDestroy(evs[i]);
  }
  cudaFree(d_out);
  cudaFree(d_status);
  return st;
}

}  // namespace

extern "C" {

int escape_last_cuda_error(const char** name) {
  const int e = esc::t_last_cuda;
  if (name) *name = e ? cudaGetErrorName((cudaError_t)e) : "";
  return e;
}

const char* escape_status_str(escape_status s) {
  switch (s) {
    case ESCAPE_OK: return "ok";
    case ESCAPE_EINVAL: return "invalid argument or malformed graph";
    case ESCAPE_ENOMEM: return "out of memory";
    case ESCAPE_ECUDA: return "CUDA error";
    case ESCAPE_EOVERFLOW: return "size beyond supported limits";
    case ESCAPE_ETIMEOUT: return "device wait timed out";
    case ESCAPE_EINTERNAL: return "device consistency check failed";
  }
  return "unknown status";
}

escape_status escape_load_csr(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col, uint32_t flags,
                              void* stream, escape_graph** out) {
  if (!out || n < 0 || n > 2147483647LL || nnz < 0 || (n > 0 && !row_ptr) || (nnz > 0 && !col))
    return ESCAPE_EINVAL;
  if (nnz > ((int64_t)1 << 40)) return ESCAPE_EOVERFLOW;
  cudaStream_t s = (cudaStream_t)stream;
  bool dev_ptrs = (flags & ESCAPE_DEVICE_PTRS) != 0;
  escape_graph* g = new (std::nothrow) escape_graph;
  if (!g) return ESCAPE_ENOMEM;
  cudaGetDevice(&g->device);
  g->sms = device_sms(g->device);
  // every row offset is checked on the host before any copy or kernel: host
  // input directly, device input after copying the offsets here
  if (n > 0) {
    std::vector<int64_t> hrp;
    const int64_t* h = row_ptr;
    if (dev_ptrs) {
      cudaError_t e0 = fetch_row_ptr(row_ptr, n, hrp, s);
      if (e0 != cudaSuccess) { delete g; return from_cuda(e0); }
      h = hrp.data();
    }
    if (!row_ptr_ok(h, n, nnz)) { delete g; return ESCAPE_EINVAL; }
  }
  int64_t* d_rp = nullptr;
  int32_t* d_col = nullptr;
  unsigned* d_status = nullptr;
  cudaError_t e = cudaMalloc(&d_rp, sizeof(int64_t) * (n + 1));
  if (e == cudaSuccess) e = cudaMalloc(&d_col, sizeof(int32_t) * (nnz > 0 ? nnz : 1));
  if (e == cudaSuccess) e = cudaMalloc(&d_status, sizeof(unsigned));
  if (e != cudaSuccess) { cudaFree(d_rp); cudaFree(d_col); delete g; return from_cuda(e); }
  cudaMemcpyKind kind = dev_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (n > 0) e = cudaMemcpyAsync(d_rp, row_ptr, sizeof(int64_t) * (n + 1), kind, s);
  else e = cudaMemsetAsync(d_rp, 0, sizeof(int64_t), s);
  if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(d_col, col, sizeof(int32_t) * nnz, kind, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(unsigned), s);
  escape_status st = from_cuda(e);
  if (st == ESCAPE_OK && (flags & ESCAPE_NORMALIZE)) {
    esc::DeviceArena arena;
    size_t ab = (size_t)(2 * nnz + 16) * 8 * 3 + (size_t)((2 * nnz) / 4096 + 2) * 256 * 8 * 2 + (1 << 22);
    e = cudaMalloc(&arena.base, ab);
    if (e == cudaSuccess) {
      arena.cap = ab;
      int64_t *nrp = nullptr;
      int32_t* ncol = nullptr;
      int64_t nnz2 = 0;
      e = esc::normalize_csr(n, nnz, d_rp, d_col, &nrp, &ncol, &nnz2, d_status, arena, s, g->sms);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      cudaFree(arena.base);
      if (e == cudaSuccess) {
        cudaFree(d_rp);
        cudaFree(d_col);
        d_rp = nrp;
        d_col = ncol;
        nnz = nnz2;
      }
    }
    st = from_cuda(e);
  } else if (st == ESCAPE_OK) {
    e = esc::validate_csr(n, d_rp, d_col, d_status, s, g->sms);
    st = from_cuda(e);
  }
  if (st == ESCAPE_OK) {
    unsigned h = 0;
    e = cudaMemcpyAsync(&h, d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    st = from_cuda(e);
    if (st == ESCAPE_OK && h) st = ESCAPE_EINVAL;
  }
  cudaFree(d_status);
  if (st != ESCAPE_OK) { cudaFree(d_rp); cudaFree(d_col); delete g; return st; }
  g->n = n;
  g->nnz = nnz;
  g->d_rp = d_rp;
  g->d_col = d_col;
  *out = g;
  return ESCAPE_OK;
}

escape_status escape_graph_info(const escape_graph* g, int64_t* n, int64_t* m) {
  if (!g) return ESCAPE_EINVAL;
  if (n) *n = g->n;
  if (m) *m = g->nnz / 2;
  return ESCAPE_OK;
}

escape_status escape_set_options(escape_graph* g, int keep_per_element, int cta_per_sm, int serial_phases) {
  if (!g || cta_per_sm < 0 || cta_per_sm > 8) return ESCAPE_EINVAL;
  g->keep_pe = keep_per_element ? 1 : 0;
  g->cta_per_sm = cta_per_sm ? cta_per_sm : 2;
  g->serial = serial_phases < 0 ? -1 : (serial_phases ? 1 : 0);
  return ESCAPE_OK;
}

escape_status escape_census5(escape_graph* g, escape_census* out, void* stream) {
  if (!g || !out) return ESCAPE_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  free_pe(g);
  g->has_basis = false;
  g->has_part = false;
  long long l0 = esc::launches_so_far();
  escape_status st = census_one(g, g->d_rp, g->d_col, g->n, g->nnz, out, s, g->keep_pe != 0, &g->pe, &g->ori,
                                g->phase_ms, &g->num_phases);
  g->launches = esc::launches_so_far() - l0;
  if (st == ESCAPE_OK && g->keep_pe) g->has_pe = true;
  else free_pe(g);
  return st;
}

escape_status escape_census4(escape_graph* g, escape_census34* out, void* stream) {
  if (!g || !out) return ESCAPE_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  free_pe(g);
  g->has_basis = false;
  g->has_part = false;
  long long l0 = esc::launches_so_far();
  escape_census full;
  escape_status st = census_one(g, g->d_rp, g->d_col, g->n, g->nnz, &full, s, g->keep_pe != 0, &g->pe, &g->ori,
                                g->phase_ms, &g->num_phases, true);
  g->launches = esc::launches_so_far() - l0;
  if (st == ESCAPE_OK) {
    for (int i = 0; i < 4; ++i) { out->c3[i] = full.c3[i]; out->n3[i] = full.n3[i]; }
    for (int i = 0; i < 11; ++i) { out->c4[i] = full.c4[i]; out->n4[i] = full.n4[i]; }
  }
  if (st == ESCAPE_OK && g->keep_pe) g->has_pe = true;
  else free_pe(g);
  return st;
}

// One chunk of a batch: G graphs whose vertex offsets voff (G + 1) and row
// pointer rp (rows + 1) are host arrays starting at 0, and whose entries are
// col[0 .. rp[rows]) (host or device memory).
static escape_status batch_chunk(int32_t num_graphs, const int64_t* voff_h, const int64_t* rp_h, const int32_t* col,
                                 bool dev_ptrs, uint32_t flags, escape_census* out, cudaStream_t s, int sms) {
  const int64_t rows = voff_h[num_graphs];
  int64_t nnz = rp_h[rows];
  cudaMemcpyKind kind = dev_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e = cudaSuccess;
  // device copies: offsets, rows, entries turned into union ids
  int64_t *d_voff = nullptr, *d_rp = nullptr;
  int32_t* d_col = nullptr;
  unsigned* d_status = nullptr;
  unsigned long long* d_out = nullptr;
  e = cudaMalloc(&d_voff, sizeof(int64_t) * (num_graphs + 1));
  if (e == cudaSuccess) e = cudaMalloc(&d_rp, sizeof(int64_t) * (rows + 1));
  if (e == cudaSuccess) e = cudaMalloc(&d_col, sizeof(int32_t) * (nnz > 0 ? nnz : 1));
  if (e == cudaSuccess) e = cudaMalloc(&d_status, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc(&d_out, sizeof(escape_census) * num_graphs);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_voff, voff_h, sizeof(int64_t) * (num_graphs + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_rp, rp_h, sizeof(int64_t) * (rows + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(d_col, col, sizeof(int32_t) * nnz, kind, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(unsigned), s);
  escape_status st = from_cuda(e);
  if (st == ESCAPE_OK && rows > 0) {
    (k_globalize<<<(unsigned)std::min<int64_t>((rows * 32 + 255) / 256, (int64_t)sms * 16), 256, 0, s>>>(
         d_voff, num_graphs, d_rp, rows, d_col, d_status), esc::note_launch());
    st = from_cuda(cudaGetLastError());
  }
  if (st == ESCAPE_OK && (flags & ESCAPE_NORMALIZE)) {
    esc::DeviceArena arena;
    size_t ab = (size_t)(2 * nnz + 16) * 8 * 3 + (size_t)((2 * nnz) / 4096 + 2) * 256 * 8 * 2 + (1 << 22);
    e = cudaMalloc(&arena.base, ab);
    if (e == cudaSuccess) {
      arena.cap = ab;
      int64_t* nrp = nullptr;
      int32_t* ncol = nullptr;
      int64_t nnz2 = 0;
      e = esc::normalize_csr(rows, nnz, d_rp, d_col, &nrp, &ncol, &nnz2, d_status, arena, s, sms);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      cudaFree(arena.base);
      if (e == cudaSuccess) { cudaFree(d_rp); cudaFree(d_col); d_rp = nrp; d_col = ncol; nnz = nnz2; }
    }
    st = from_cuda(e);
  } else if (st == ESCAPE_OK) {
    st = from_cuda(esc::validate_csr(rows, d_rp, d_col, d_status, s, sms));
  }
  if (st == ESCAPE_OK) {
    unsigned h = 0;
    e = cudaMemcpyAsync(&h, d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    st = from_cuda(e);
    if (st == ESCAPE_OK && h) st = ESCAPE_EINVAL;
  }
  if (st == ESCAPE_OK) {
    esc::CensusConfig cfg;
    cfg.sms = sms;
    cfg.cta_per_sm = 2;
    cfg.d_vtx_offsets = d_voff;
    cfg.num_graphs = num_graphs;
    e = esc::run_census(d_rp, d_col, rows, nnz, cfg, d_out, d_status, nullptr, nullptr, s);
    st = from_cuda(e);
    unsigned h = 0;
    if (st == ESCAPE_OK) {
      e = cudaMemcpyAsync(out, d_out, sizeof(escape_census) * num_graphs, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      st = from_cuda(e);
      if (st == ESCAPE_OK && h) st = ESCAPE_EINTERNAL;
    }
  }
  cudaFree(d_voff); cudaFree(d_rp); cudaFree(d_col); cudaFree(d_status); cudaFree(d_out);
  return st;
}


escape_status escape_census5_batch(int32_t num_graphs, const int64_t* vtx_offsets, const int64_t* row_ptr,
                                   const int32_t* col, uint32_t flags, escape_census* out, void* stream) {
  if (num_graphs < 0 || (num_graphs > 0 && (!vtx_offsets || !row_ptr || !out))) return ESCAPE_EINVAL;
  if (num_graphs == 0) return ESCAPE_OK;
  cudaStream_t s = (cudaStream_t)stream;
  bool dev_ptrs = (flags & ESCAPE_DEVICE_PTRS) != 0;
  int dev = 0;
  cudaGetDevice(&dev);
  int sms = device_sms(dev);
  // sizes on the host: the vertex offsets and the total entry count
  std::vector<int64_t> voff(num_graphs + 1);
  cudaError_t e = cudaSuccess;
  if (dev_ptrs) e = cudaMemcpyAsync(voff.data(), vtx_offsets, sizeof(int64_t) * (num_graphs + 1), cudaMemcpyDeviceToHost, s);
  else memcpy(voff.data(), vtx_offsets, sizeof(int64_t) * (num_graphs + 1));
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  if (voff[0] != 0) return ESCAPE_EINVAL;
  for (int k = 0; k < num_graphs; ++k)
    if (voff[k + 1] < voff[k] || voff[k + 1] - voff[k] > 2147483647LL) return ESCAPE_EINVAL;
  int64_t rows = voff[num_graphs];
  if (rows > 2147483647LL) return ESCAPE_EOVERFLOW;      // the union is one graph of int32 ids
  // every row offset is checked on the host before any kernel indexes col
  // through it (device input is copied here first)
  std::vector<int64_t> hrp;
  const int64_t* h = row_ptr;
  if (dev_ptrs) {
    e = fetch_row_ptr(row_ptr, rows, hrp, s);
    if (e != cudaSuccess) return from_cuda(e);
    h = hrp.data();
  }
  if (!row_ptr_ok(h, rows, -1)) return ESCAPE_EINVAL;
  int64_t nnz = h[rows];
  if (nnz > 0 && !col) return ESCAPE_EINVAL;
  // Chunks of consecutive graphs, each counted as one block-diagonal union,
  // sized so that a chunk's work space stays within about half of the free
  // device memory (at most 64 GiB): per graph the common-neighbour lists
  // (36 B per triangle, and 3T <= W), per-entry and per-vertex arrays, and per
  // union vertex the sweeps' per-CTA counters.
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  double budget = std::min((double)free_b * 0.5, (double)((size_t)64 << 30));
  if (const char* v = getenv("ESC_BATCH_CHUNK_MB"))          // a smaller chunk budget (tests, tuning)
    if (atof(v) > 0) budget = std::min(budget, atof(v) * (1 << 20));
  std::vector<int64_t> vrb, rrb;
  int32_t k0 = 0;
  while (k0 < num_graphs) {
    int32_t k1 = k0;
    double used = 0;
    while (k1 < num_graphs) {
      double wedges = 0;
      for (int64_t r = voff[k1]; r < voff[k1 + 1]; ++r) {
        double d = (double)(h[r + 1] - h[r]);
        wedges += d * (d - 1) / 2;
      }
      const double nk = (double)(voff[k1 + 1] - voff[k1]), ek = (double)(h[voff[k1 + 1]] - h[voff[k1]]);
      const double need = 12.0 * wedges + 160.0 * ek + 200.0 * nk + 32.0 * 4 * sms * nk;
      if (k1 > k0 && used + need > budget) break;
      used += need;
      ++k1;
    }
    // the chunk's offsets and rows, starting at 0
    const int64_t r0 = voff[k0], r1 = voff[k1], e0 = h[r0];
    vrb.resize((size_t)(k1 - k0) + 1);
    for (int32_t k = k0; k <= k1; ++k) vrb[k - k0] = voff[k] - r0;
    rrb.resize((size_t)(r1 - r0) + 1);
    for (int64_t r = r0; r <= r1; ++r) rrb[r - r0] = h[r] - e0;
    escape_status st = batch_chunk(k1 - k0, vrb.data(), rrb.data(), col ? col + e0 : nullptr, dev_ptrs, flags,
                                   out + k0, s, sms);
    if (st != ESCAPE_OK) return st;
    k0 = k1;
  }
  return ESCAPE_OK;
}
escape_status escape_per_element(escape_graph* g, uint64_t* tri_e, uint64_t* c4_e, uint64_t* k4_e, uint64_t* tri_v,
                                 uint64_t* c4_v, uint64_t* k4_v, void* stream) {
  if (!g || !g->has_pe) return ESCAPE_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long *dT = nullptr, *dC = nullptr, *dK = nullptr, *vt = nullptr, *vc = nullptr, *vk = nullptr;
  size_t eb = sizeof(unsigned long long) * (g->nnz + 1), vb = sizeof(unsigned long long) * (g->n + 1);
  cudaError_t e = cudaMalloc(&dT, eb);
  if (e == cudaSuccess) e = cudaMalloc(&dC, eb);
  if (e == cudaSuccess) e = cudaMalloc(&dK, eb);
  if (e == cudaSuccess) e = cudaMalloc(&vt, vb);
  if (e == cudaSuccess) e = cudaMalloc(&vc, vb);
  if (e == cudaSuccess) e = cudaMalloc(&vk, vb);
  if (e == cudaSuccess && g->n > 0) {
    (k_map_edges<<<(unsigned)std::min<int64_t>((g->n * 32 + 255) / 256, 65535), 256, 0, s>>>(
        g->d_rp, g->d_col, g->n, g->ori.rank, g->ori.R, g->ori.C, g->pe.Te, g->pe.C4e, g->pe.K4e, dT, dC, dK), esc::note_launch());
    (k_map_vertices<<<(unsigned)std::min<int64_t>((g->n + 255) / 256, 65535), 256, 0, s>>>(
        g->n, g->ori.rank, g->pe.tv, g->pe.C4v, g->pe.K4v, vt, vc, vk), esc::note_launch());
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && tri_e && g->nnz) e = cudaMemcpyAsync(tri_e, dT, sizeof(uint64_t) * g->nnz, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && c4_e && g->nnz) e = cudaMemcpyAsync(c4_e, dC, sizeof(uint64_t) * g->nnz, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && k4_e && g->nnz) e = cudaMemcpyAsync(k4_e, dK, sizeof(uint64_t) * g->nnz, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && tri_v && g->n) e = cudaMemcpyAsync(tri_v, vt, sizeof(uint64_t) * g->n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && c4_v && g->n) e = cudaMemcpyAsync(c4_v, vc, sizeof(uint64_t) * g->n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && k4_v && g->n) e = cudaMemcpyAsync(k4_v, vk, sizeof(uint64_t) * g->n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(dT); cudaFree(dC); cudaFree(dK); cudaFree(vt); cudaFree(vc); cudaFree(vk);
  return from_cuda(e);
}

int escape_last_phase_ms(const escape_graph* g, float* ms, int count) {
  if (!g) return 0;
  int k = g->num_phases < count ? g->num_phases : count;
  for (int i = 0; i < k && ms; ++i) ms[i] = g->phase_ms[i];
  return g->num_phases;
}

long long escape_last_kernel_launches(const escape_graph* g) { return g ? g->launches : 0; }

int escape_part_sum_count(void) { return esc::census_sum_count(); }

escape_status escape_census5_part(escape_graph* g, int32_t part, int32_t parts, escape_part* out, void* stream) {
  if (!g || !out || parts < 1 || part < 0 || part >= parts) return ESCAPE_EINVAL;
  if (esc::census_sum_count() > ESCAPE_PART_SUMS) return ESCAPE_EOVERFLOW;
  cudaStream_t s = (cudaStream_t)stream;
  free_pe(g);
  g->has_basis = false;
  g->has_part = false;
  long long l0 = esc::launches_so_far();
  unsigned long long *d_acc = nullptr, *d_out = nullptr;
  unsigned* d_status = nullptr;
  const int nsum = esc::census_sum_count();
  cudaError_t e = cudaMalloc(&d_acc, sizeof(escape_u128) * nsum);
  if (e == cudaSuccess) e = cudaMalloc(&d_out, sizeof(escape_census));
  if (e == cudaSuccess) e = cudaMalloc(&d_status, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(unsigned), s);
  escape_status st = from_cuda(e);
  if (st == ESCAPE_OK) {
    esc::CensusConfig cfg;
    cfg.sms = g->sms;
    cfg.cta_per_sm = g->cta_per_sm;
    cfg.keep_per_element = true;
    cfg.serial_phases = g->serial > 0 || (g->serial < 0 && g->nnz >= ((int64_t)1 << 24));
    cfg.part = part;
    cfg.parts = parts;
    cfg.partial = true;
    cfg.d_acc_out = d_acc;
    st = from_cuda(esc::run_census(g->d_rp, g->d_col, g->n, g->nnz, cfg, d_out, d_status, &g->pe, &g->ori, s));
  }
  if (st == ESCAPE_OK) {
    escape_part tmp;
    memset(&tmp, 0, sizeof(tmp));
    unsigned h = 0;
    e = cudaMemcpyAsync(tmp.sums, d_acc, sizeof(escape_u128) * nsum, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    st = from_cuda(e);
    if (st == ESCAPE_OK && h) st = ESCAPE_EINTERNAL;
    if (st == ESCAPE_OK) *out = tmp;
  }
  cudaFree(d_acc);
  cudaFree(d_out);
  cudaFree(d_status);
  g->launches = esc::launches_so_far() - l0;
  if (st == ESCAPE_OK) g->has_part = true;
  else free_pe(g);
  return st;
}

escape_status escape_part_counts(escape_graph* g, uint64_t* k4_e, uint64_t* c4_e, uint64_t* c4_v, uint32_t flags,
                                 void* stream) {
  if (!g || !g->has_part) return ESCAPE_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const bool dev = (flags & ESCAPE_DEVICE_PTRS) != 0, put = (flags & ESCAPE_PART_PUT) != 0;
  cudaMemcpyKind kind = put ? (dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice)
                            : (dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
  uint64_t* mine[3] = {(uint64_t*)g->pe.K4e, (uint64_t*)g->pe.C4e, (uint64_t*)g->pe.C4v};
  uint64_t* theirs[3] = {k4_e, c4_e, c4_v};
  const int64_t len[3] = {g->nnz, g->nnz, g->n};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
    if (!theirs[k] || len[k] == 0) continue;
    e = put ? cudaMemcpyAsync(mine[k], theirs[k], sizeof(uint64_t) * len[k], kind, s)
            : cudaMemcpyAsync(theirs[k], mine[k], sizeof(uint64_t) * len[k], kind, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return from_cuda(e);
}

escape_status escape_census5_finish(escape_graph* g, const escape_part* total, escape_census* out, void* stream) {
  if (!g || !total || !out || !g->has_part) return ESCAPE_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  long long l0 = esc::launches_so_far();
  unsigned long long *d_acc = nullptr, *d_out = nullptr;
  const int nsum = esc::census_sum_count();
  cudaError_t e = cudaMalloc(&d_acc, sizeof(escape_u128) * nsum);
  if (e == cudaSuccess) e = cudaMalloc(&d_out, sizeof(escape_census));
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_acc, total->sums, sizeof(escape_u128) * nsum, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = esc::run_census_finish(g->ori, g->n, g->nnz, g->pe, d_acc, d_out, g->sms, s);
  escape_census tmp;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&tmp, d_out, sizeof(escape_census), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  escape_status st = from_cuda(e);
  if (st == ESCAPE_OK) *out = tmp;
  cudaFree(d_acc);
  cudaFree(d_out);
  g->launches = esc::launches_so_far() - l0;
  free_pe(g);
  g->has_part = false;
  return st;
}

escape_status escape_last_basis_counts(const escape_graph* g, escape_u128* out) {
  if (!g || !out || !g->has_basis) return ESCAPE_EINVAL;
  for (int i = 0; i < 4; ++i) out[i] = g->basis[i];
  return ESCAPE_OK;
}

void escape_free(escape_graph* g) {
  if (!g) return;
  free_pe(g);
  cudaFree(g->d_rp);
  cudaFree(g->d_col);
  delete g;
}

}  // extern "C"
