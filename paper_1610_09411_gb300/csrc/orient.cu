// orient.cu -- input normalisation and the degree-ordered DAG (Sec. 3.2).
//
// * an LSD radix sort of 64-bit keys (8-bit digits, stable warp ranking with
//   __match_any_sync), used for the vertex ranking and for the edge list;
// * exclusive scans;
// * normalisation of an arbitrary CSR/edge list into a simple undirected
//   graph (direction ignored, duplicates and self-loops dropped, Sec. 8);
// * validation of an already-simple input;
// * orientation: rank vertices by (degree, id), rename them by rank, sort
//   every row, find the first out-neighbour of each row and the reverse slot
//   of every entry.
#include "common.cuh"
#include "internal.h"


namespace esc {

// ================================================================= scans
static constexpr int SCAN_BLOCK = 1024;
static constexpr int SCAN_ITEMS = 8;
static constexpr int64_t SCAN_CHUNK = (int64_t)SCAN_BLOCK * SCAN_ITEMS;

__device__ __forceinline__ int64_t block_excl_scan_i64(int64_t v, int64_t* sh, int64_t* total) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int nw = blockDim.x >> 5;
    int64_t s = lane < nw ? sh[lane] : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, s, off);
      if (lane >= off) s += y;
    }
    if (lane < nw) sh[lane] = s;
  }
  __syncthreads();
  int64_t warp_off = wid > 0 ? sh[wid - 1] : 0;
  if (total) *total = sh[(blockDim.x >> 5) - 1];
  int64_t incl = x + warp_off;
  __syncthreads();
  return incl - v;
}

__global__ void k_scan_reduce(const int64_t* in, int64_t n, int64_t* sums) {
  __shared__ int64_t sh[32];
  int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK;
  int64_t s = 0;
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + (int64_t)k * SCAN_BLOCK + threadIdx.x;
    if (i < n) s += in[i];
  }
  int64_t tot;
  block_excl_scan_i64(s, sh, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_chunks(const int64_t* in, int64_t* out, int64_t n, const int64_t* offs) {
  __shared__ int64_t sh[32];
  int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t v[SCAN_ITEMS];
  int64_t s = 0;
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + k;
    v[k] = i < n ? in[i] : 0;
    s += v[k];
  }
  int64_t ex = block_excl_scan_i64(s, sh, nullptr) + (offs ? offs[blockIdx.x] : 0);
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + k;
    if (i < n) out[i] = ex;
    ex += v[k];
  }
}

// out[i] = sum_{k<i} in[i] (in and out may alias); out[n] = total if with_total.
cudaError_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, bool with_total,
                               DeviceArena& arena, cudaStream_t s) {
  if (n <= 0) {
    if (with_total) return cudaMemsetAsync(out, 0, sizeof(int64_t), s);
    return cudaSuccess;
  }
  int64_t nb = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
  int64_t total_idx = n;
  if (nb == 1) {
    if (with_total) {
      // total = last exclusive + last input: computed by an extra reduce
      int64_t* sums = (int64_t*)arena.alloc(sizeof(int64_t));
      if (!sums) return cudaErrorMemoryAllocation;
      (k_scan_reduce<<<1, SCAN_BLOCK, 0, s>>>(in, n, sums), note_launch());
      (k_scan_chunks<<<1, SCAN_BLOCK, 0, s>>>(in, out, n, nullptr), note_launch());
      cudaMemcpyAsync(out + total_idx, sums, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    } else {
      (k_scan_chunks<<<1, SCAN_BLOCK, 0, s>>>(in, out, n, nullptr), note_launch());
    }
    return cudaGetLastError();
  }
  int64_t* sums = (int64_t*)arena.alloc(sizeof(int64_t) * (nb + 1));
  if (!sums) return cudaErrorMemoryAllocation;
  (k_scan_reduce<<<(unsigned)nb, SCAN_BLOCK, 0, s>>>(in, n, sums), note_launch());
  cudaError_t e = exclusive_scan_i64(sums, sums, nb, true, arena, s);
  if (e != cudaSuccess) return e;
  (k_scan_chunks<<<(unsigned)nb, SCAN_BLOCK, 0, s>>>(in, out, n, sums), note_launch());
  if (with_total) cudaMemcpyAsync(out + total_idx, sums + nb, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
  return cudaGetLastError();
}

// ================================================================= radix sort
static constexpr int RS_THREADS = 256;
static constexpr int RS_WARPS = RS_THREADS / 32;
static constexpr int RS_ROUNDS = 16;                        // per warp
static constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;      // 4096 keys per tile
static constexpr int RS_BINS = 256;

__global__ void k_rs_hist(const uint64_t* keys, int64_t n, int shift, int64_t ntiles, int64_t* counts) {
  __shared__ unsigned h[RS_BINS];
  for (int i = threadIdx.x; i < RS_BINS; i += blockDim.x) h[i] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int k = 0; k < RS_ROUNDS; ++k) {
    int64_t i = base + (int64_t)k * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xff], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < RS_BINS; d += blockDim.x) counts[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

__global__ void k_rs_scatter(const uint64_t* keys, const uint32_t* vals, uint64_t* okeys, uint32_t* ovals,
                             int64_t n, int shift, int64_t ntiles, const int64_t* offs) {
  __shared__ unsigned wh[RS_WARPS][RS_BINS];
  __shared__ int64_t wbase[RS_WARPS][RS_BINS];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += blockDim.x) (&wh[0][0])[i] = 0;
  __syncthreads();
  int64_t wstart = (int64_t)blockIdx.x * RS_TILE + (int64_t)w * (RS_ROUNDS * 32);
  for (int r = 0; r < RS_ROUNDS; ++r) {
    int64_t i = wstart + r * 32 + lane;
    if (i < n) atomicAdd(&wh[w][(keys[i] >> shift) & 0xff], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < RS_BINS; d += blockDim.x) {
    int64_t run = offs[(int64_t)d * ntiles + blockIdx.x];
    for (int ww = 0; ww < RS_WARPS; ++ww) { wbase[ww][d] = run; run += wh[ww][d]; }
  }
  __syncthreads();
  unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < RS_ROUNDS; ++r) {
    int64_t i = wstart + r * 32 + lane;
    bool valid = i < n;
    uint64_t key = valid ? keys[i] : 0;
    unsigned dig = valid ? (unsigned)((key >> shift) & 0xff) : 0x100u + lane;   // invalid lanes match nobody
    unsigned peers = __match_any_sync(0xffffffffu, dig);
    int rank = __popc(peers & lt);
    int64_t dst = 0;
    if (valid) dst = wbase[w][dig] + rank;
    __syncwarp();
    if (valid && rank == 0) wbase[w][dig] += __popc(peers);
    __syncwarp();
    if (valid) {
      okeys[dst] = key;
      if (vals) ovals[dst] = vals[i];
    }
  }
}

// Stable sort of (keys, vals) by the low `bits` bits of the key.  The result
// ends in `keys`/`vals`; `tk`/`tv` are scratch of the same size.
cudaError_t radix_sort(uint64_t* keys, uint32_t* vals, uint64_t* tk, uint32_t* tv, int64_t n, int bits,
                       DeviceArena& arena, cudaStream_t s) {
  if (n <= 1 || bits <= 0) return cudaSuccess;
  int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
  size_t mark = arena.mark();
  int64_t* counts = (int64_t*)arena.alloc(sizeof(int64_t) * (RS_BINS * ntiles + 1));
  if (!counts) return cudaErrorMemoryAllocation;
  uint64_t *ka = keys, *kb = tk;
  uint32_t *va = vals, *vb = tv;
  int passes = (bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    int shift = p * 8;
    (k_rs_hist<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(ka, n, shift, ntiles, counts), note_launch());
    cudaError_t e = exclusive_scan_i64(counts, counts, RS_BINS * ntiles, false, arena, s);
    if (e != cudaSuccess) return e;
    (k_rs_scatter<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(ka, va, kb, vb, n, shift, ntiles, counts), note_launch());
    uint64_t* t = ka; ka = kb; kb = t;
    uint32_t* t2 = va; va = vb; vb = t2;
  }
  if (ka != keys) {
    cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s);
    if (vals) cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
  }
  arena.release(mark);
  return cudaGetLastError();
}

int bits_for(int64_t n) {
  int b = 1;
  while (b < 62 && ((int64_t)1 << b) < n) ++b;
  return b;
}

// ================================================================= normalise / validate
// Keys (u << vb | v) for both directions of every input entry; loops and
// out-of-range ids get the sentinel 2^(2 vb), which sorts after every real key
// and is dropped.
__global__ void k_edge_keys_both(const int64_t* rp, const int32_t* col, int64_t n, int64_t nnz, int vb,
                                 uint64_t* keys, unsigned* st) {
  const uint64_t SENT = 1ull << (2 * vb);
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride) {
    // row of p by binary search over rp
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) { int64_t mid = (lo + hi) >> 1; if (rp[mid] <= p) lo = mid; else hi = mid; }
    uint64_t u = (uint64_t)lo, v = (uint64_t)(int64_t)col[p];
    if ((int64_t)v < 0 || (int64_t)v >= n) { set_err(st, DEVERR_BOUNDS); keys[2 * p] = keys[2 * p + 1] = SENT; continue; }
    if (u == v) { keys[2 * p] = keys[2 * p + 1] = SENT; continue; }
    keys[2 * p] = (u << vb) | v;
    keys[2 * p + 1] = (v << vb) | u;
  }
}

__global__ void k_mark_unique(const uint64_t* keys, int64_t cnt, int vb, int64_t* flag) {
  const uint64_t SENT = 1ull << (2 * vb);
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += stride)
    flag[i] = (keys[i] != SENT && (i == 0 || keys[i] != keys[i - 1])) ? 1 : 0;
}

__global__ void k_compact_csr(const uint64_t* keys, const int64_t* pos, int64_t cnt, int vb, int32_t* col,
                              int64_t* rowcnt) {
  const uint64_t SENT = 1ull << (2 * vb);
  uint64_t mask = (1ull << vb) - 1;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += stride) {
    bool keep = keys[i] != SENT && (i == 0 || keys[i] != keys[i - 1]);
    if (!keep) continue;
    col[pos[i]] = (int32_t)(keys[i] & mask);
    atomicAdd((unsigned long long*)&rowcnt[keys[i] >> vb], 1ull);
  }
}

// Input already simple?  Rows non-decreasing, ids in range, sorted strictly,
// no loops, symmetric.
__global__ void k_validate(const int64_t* rp, const int32_t* col, int64_t n, unsigned* st) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
    int64_t b = rp[u], e = rp[u + 1];
    if (e < b) { set_err(st, DEVERR_BOUNDS); continue; }
    for (int64_t p = b; p < e; ++p) {
      int32_t v = col[p];
      if (v < 0 || v >= n || v == u || (p > b && v <= col[p - 1])) { set_err(st, DEVERR_BOUNDS); break; }
      int64_t q = lower_bound_i32(col, rp[v], rp[v + 1], (int32_t)u);
      if (q >= rp[v + 1] || col[q] != (int32_t)u) { set_err(st, DEVERR_BOUNDS); break; }
    }
  }
}

// ================================================================= orientation
__global__ void k_degree_keys(const int64_t* rp, int64_t n, uint64_t* keys, uint32_t* vals) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    keys[v] = (uint64_t)(rp[v + 1] - rp[v]);
    vals[v] = (uint32_t)v;
  }
}

// perm[r] = original id of rank r (from the sorted vals); rank[perm[r]] = r;
// deg_r[r] = degree of rank r.
__global__ void k_ranks(const uint32_t* sorted_ids, const uint64_t* sorted_deg, int64_t n, int32_t* perm,
                        int32_t* rank, int64_t* deg_r) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    uint32_t v = sorted_ids[r];
    perm[r] = (int32_t)v;
    rank[v] = (int32_t)r;
    deg_r[r] = (int64_t)sorted_deg[r];
  }
}

__global__ void k_rank_edge_keys(const int64_t* rp, const int32_t* col, int64_t n, const int32_t* rank,
                                 int vb, uint64_t* keys) {
  // one warp per original row
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int lane = threadIdx.x & 31;
  for (int64_t u = warp; u < n; u += nwarps) {
    uint64_t ru = (uint64_t)rank[u];
    for (int64_t p = rp[u] + lane; p < rp[u + 1]; p += 32) keys[p] = (ru << vb) | (uint64_t)rank[col[p]];
  }
}

__global__ void k_keys_to_col(const uint64_t* keys, int64_t nnz, int vb, int32_t* C) {
  uint64_t mask = (1ull << vb) - 1;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride)
    C[p] = (int32_t)(keys[p] & mask);
}

__global__ void k_outptr(const int64_t* R, const int32_t* C, int64_t n, int64_t* op) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    op[v] = lower_bound_i32(C, R[v], R[v + 1], (int32_t)(v + 1));
}

__global__ void k_rev(const int64_t* R, const int32_t* C, int64_t n, int64_t* rev) {
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int lane = threadIdx.x & 31;
  for (int64_t v = warp; v < n; v += nwarps)
    for (int64_t p = R[v] + lane; p < R[v + 1]; p += 32) {
      int32_t w = C[p];
      rev[p] = lower_bound_i32(C, R[w], R[w + 1], (int32_t)v);
    }
}

static unsigned grid_for(int64_t n, int threads, int sms) {
  int64_t b = (n + threads - 1) / threads;
  int64_t cap = (int64_t)sms * 16;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// ---------------------------------------------------------------- public (internal) entry points
cudaError_t normalize_csr(int64_t n, int64_t nnz_in, const int64_t* rp_in, const int32_t* col_in,
                          int64_t** rp_out, int32_t** col_out, int64_t* nnz_out, unsigned* d_status,
                          DeviceArena& arena, cudaStream_t s, int sms) {
  int vb = bits_for(n > 1 ? n : 2);
  int64_t cnt = 2 * nnz_in;
  size_t mark = arena.mark();
  uint64_t* keys = (uint64_t*)arena.alloc(sizeof(uint64_t) * (cnt + 1));
  uint64_t* tk = (uint64_t*)arena.alloc(sizeof(uint64_t) * (cnt + 1));
  int64_t* flag = (int64_t*)arena.alloc(sizeof(int64_t) * (cnt + 1));
  if (!keys || !tk || !flag) return cudaErrorMemoryAllocation;
  if (cnt > 0) (k_edge_keys_both<<<grid_for(nnz_in, 256, sms), 256, 0, s>>>(rp_in, col_in, n, nnz_in, vb, keys, d_status), note_launch());
  // keys use 2 vb bits plus the sentinel bit above them
  cudaError_t e = radix_sort(keys, nullptr, tk, nullptr, cnt, 2 * vb + 1, arena, s);
  if (e != cudaSuccess) return e;
  if (cnt > 0) (k_mark_unique<<<grid_for(cnt, 256, sms), 256, 0, s>>>(keys, cnt, vb, flag), note_launch());
  e = exclusive_scan_i64(flag, flag, cnt, true, arena, s);
  if (e != cudaSuccess) return e;
  int64_t nnz = 0;
  cudaMemcpyAsync(&nnz, flag + cnt, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  int64_t* rp = nullptr;
  int32_t* col = nullptr;
  e = cudaMalloc(&rp, sizeof(int64_t) * (n + 1));
  if (e == cudaSuccess) e = cudaMalloc(&col, sizeof(int32_t) * (nnz > 0 ? nnz : 1));
  if (e != cudaSuccess) { cudaFree(rp); return e; }
  cudaMemsetAsync(rp, 0, sizeof(int64_t) * (n + 1), s);
  if (cnt > 0) (k_compact_csr<<<grid_for(cnt, 256, sms), 256, 0, s>>>(keys, flag, cnt, vb, col, rp), note_launch());
  e = exclusive_scan_i64(rp, rp, n, true, arena, s);
  if (e != cudaSuccess) { cudaFree(rp); cudaFree(col); return e; }
  arena.release(mark);
  *rp_out = rp;
  *col_out = col;
  *nnz_out = nnz;
  return cudaGetLastError();
}

cudaError_t validate_csr(int64_t n, const int64_t* rp, const int32_t* col, unsigned* d_status, cudaStream_t s,
                         int sms) {
  if (n > 0) (k_validate<<<grid_for(n, 128, sms), 128, 0, s>>>(rp, col, n, d_status), note_launch());
  return cudaGetLastError();
}

// Build the degree-ordered graph of an input CSR (original ids).
cudaError_t orient(const int64_t* rp, const int32_t* col, int64_t n, int64_t nnz, Oriented& o, DeviceArena& arena,
                   cudaStream_t s, int sms) {
  size_t mark = arena.mark();
  int64_t nk = n > nnz ? n : nnz;
  uint64_t* keys = (uint64_t*)arena.alloc(sizeof(uint64_t) * (nk + 1));
  uint64_t* tk = (uint64_t*)arena.alloc(sizeof(uint64_t) * (nk + 1));
  uint32_t* vals = (uint32_t*)arena.alloc(sizeof(uint32_t) * (n + 1));
  uint32_t* tv = (uint32_t*)arena.alloc(sizeof(uint32_t) * (n + 1));
  if (!keys || !tk || !vals || !tv) return cudaErrorMemoryAllocation;
  cudaError_t e;
  // 1. rank vertices by (degree, id): stable sort of degrees with ids as values
  if (n > 0) (k_degree_keys<<<grid_for(n, 256, sms), 256, 0, s>>>(rp, n, keys, vals), note_launch());
  int dbits = bits_for(nnz + 2);
  e = radix_sort(keys, vals, tk, tv, n, dbits, arena, s);
  if (e != cudaSuccess) return e;
  if (n > 0) (k_ranks<<<grid_for(n, 256, sms), 256, 0, s>>>(vals, keys, n, o.perm, o.rank, o.R), note_launch());
  // 2. row starts in rank order
  e = exclusive_scan_i64(o.R, o.R, n, true, arena, s);
  if (e != cudaSuccess) return e;
  // 3. renamed entries sorted by (row rank, neighbour rank)
  int vb = bits_for(n > 1 ? n : 2);
  if (nnz > 0) {
    (k_rank_edge_keys<<<grid_for(n * 32, 256, sms), 256, 0, s>>>(rp, col, n, o.rank, vb, keys), note_launch());
    e = radix_sort(keys, nullptr, tk, nullptr, nnz, 2 * vb, arena, s);
    if (e != cudaSuccess) return e;
    (k_keys_to_col<<<grid_for(nnz, 256, sms), 256, 0, s>>>(keys, nnz, vb, o.C), note_launch());
  }
  // 4. out-pointers and reverse slots
  if (n > 0) {
    (k_outptr<<<grid_for(n, 256, sms), 256, 0, s>>>(o.R, o.C, n, o.op), note_launch());
    (k_rev<<<grid_for(n * 32, 256, sms), 256, 0, s>>>(o.R, o.C, n, o.rev), note_launch());
  }
  arena.release(mark);
  return cudaGetLastError();
}

}  // namespace esc
