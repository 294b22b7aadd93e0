// common.cuh -- device helpers shared by the census kernels: exact 128-bit
// accumulation, warp/block reductions, the graph's device layout and the
// per-vertex work queue.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

typedef unsigned __int128 u128;

#define ESC_WARP 32

// ---------------------------------------------------------------- accumulators
// Every global sum the closed forms need (App. A / Thms 4-14).  Each is an
// unsigned 128-bit counter held as two 64-bit words; kernels add warp- or
// block-reduced partials with carry propagation, so the total is exact
// modulo 2^128 (every true value is < 2^127).
enum AccId {
  ACC_W = 0,      // sum C(d,2)                       wedges
  ACC_S3,         // sum C(d,3)                       3-stars
  ACC_S4,         // sum C(d,4)                       N1
  ACC_T,          // triangles
  ACC_P4A,        // sum_e (d_i-1)(d_j-1)              3-paths + 3T
  ACC_TT,         // sum t_i (d_i-2)                   tailed triangles
  ACC_C4,         // 4-cycles
  ACC_D,          // sum_e C(T_e,2)                    diamonds
  ACC_K4,         // 4-cliques (x3: sum of alpha over G+(x) edges)
  ACC_N2A, ACC_N3A, ACC_N4, ACC_N5A, ACC_N6A, ACC_N7A,
  ACC_N8M,        // 5-cycle product term
  ACC_N8Z,        // 5-cycle directed tailed-triangle term
  ACC_N9A, ACC_N10A, ACC_N11, ACC_N12A, ACC_N13, ACC_N14, ACC_N15, ACC_N16A,
  ACC_N17, ACC_N18, ACC_N19, ACC_N20, ACC_N21,
  ACC_D2D,        // sum_c C(d_c,2) d_c
  ACC_DNBR,       // sum_c (d_c-1) sum_{a in N(c)} d_a
  ACC_TD,         // sum_i t_i d_i
  ACC_DP,         // sum over out-edges a -> b of (d+(a) - 1) d+(b)   directed 3-paths i <- a -> b -> j
  ACC_DBP,        // sum over directed triangles of C(apexes above, 2)  directed bipyramids
  ACC_COUNT
};

struct Acc128 { unsigned long long lo, hi; };

__device__ __forceinline__ void acc_add(Acc128* acc, int id, u128 v) {
  if (v == 0) return;
  unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
  unsigned long long old = atomicAdd(&acc[id].lo, lo);
  if (old + lo < old) hi += 1;
  if (hi) atomicAdd(&acc[id].hi, hi);
}

__device__ __forceinline__ u128 shfl_down_u128(u128 v, int off) {
  unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
  lo = __shfl_down_sync(0xffffffffu, lo, off);
  hi = __shfl_down_sync(0xffffffffu, hi, off);
  return ((u128)hi << 64) | lo;
}

__device__ __forceinline__ u128 warp_sum_u128(u128 v) {
  for (int off = 16; off > 0; off >>= 1) v += shfl_down_u128(v, off);
  return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

// Block-wide sum of a u128 held by every thread; result valid in thread 0.
// `sh` must hold blockDim.x/32 entries.  All threads must call it.
__device__ __forceinline__ u128 block_sum_u128(u128 v, u128* sh) {
  v = warp_sum_u128(v);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  u128 r = 0;
  if (wid == 0) {
    int nw = (blockDim.x + 31) >> 5;
    r = lane < nw ? sh[lane] : 0;
    r = warp_sum_u128(r);
  }
  return r;
}

// Per-thread accumulation of several sums, flushed once per block.
template <int K>
struct LocalAcc {
  u128 v[K];
  __device__ void zero() {
#pragma unroll
    for (int i = 0; i < K; ++i) v[i] = 0;
  }
};

template <int K>
__device__ __forceinline__ void flush_acc(LocalAcc<K>& la, const int (&ids)[K], Acc128* acc, u128* sh) {
#pragma unroll
  for (int i = 0; i < K; ++i) {
    u128 s = block_sum_u128(la.v[i], sh);
    if (threadIdx.x == 0) acc_add(acc, ids[i], s);
  }
}

// Accumulator set: one row of ACC_COUNT counters per graph.  vg (graph id of
// every vertex) is null for a single graph; then every item adds to row 0 and
// partial sums are flushed once per block at the end.  In a batch, every work
// item belongs to one graph (no edge joins two graphs), so its partial sums are
// flushed to that graph's row when the item is done.
struct AccSet {
  Acc128* base;
  const int32_t* vg;
};

__device__ __forceinline__ Acc128* acc_of(const AccSet& A, int64_t v) {
  return A.vg ? A.base + (int64_t)A.vg[v] * ACC_COUNT : A.base;
}

// per-item flush for warp-per-item loops (all 32 lanes present)
template <int K>
__device__ __forceinline__ void warp_item_flush(LocalAcc<K>& la, const int (&ids)[K], const AccSet& A, int64_t v) {
  if (!A.vg) return;
  Acc128* a = acc_of(A, v);
#pragma unroll
  for (int i = 0; i < K; ++i) {
    u128 s = warp_sum_u128(la.v[i]);
    if ((threadIdx.x & 31) == 0) acc_add(a, ids[i], s);
    la.v[i] = 0;
  }
}

// per-item flush for CTA-per-item loops (all threads of the block present)
template <int K>
__device__ __forceinline__ void block_item_flush(LocalAcc<K>& la, const int (&ids)[K], const AccSet& A, int64_t v,
                                                 u128* sh) {
  if (!A.vg) return;
  Acc128* a = acc_of(A, v);
#pragma unroll
  for (int i = 0; i < K; ++i) {
    u128 s = block_sum_u128(la.v[i], sh);
    if (threadIdx.x == 0) acc_add(a, ids[i], s);
    la.v[i] = 0;
  }
}

template <int K>
__device__ __forceinline__ void final_flush(LocalAcc<K>& la, const int (&ids)[K], const AccSet& A, u128* sh) {
  if (A.vg) return;
  flush_acc(la, ids, A.base, sh);
}

__device__ __forceinline__ u128 ch2(unsigned long long x) { return x < 2 ? 0 : (u128)x * (x - 1) / 2; }
__device__ __forceinline__ u128 ch3(unsigned long long x) {
  if (x < 3) return 0;
  u128 a = (u128)x * (x - 1) * (x - 2);
  return a / 6;
}
__device__ __forceinline__ u128 ch4(unsigned long long x) {
  if (x < 4) return 0;
  u128 a = (u128)x * (x - 1) * (x - 2);
  a = a / 6 * (x - 3);       // C(x,3) * (x-3) = 4 C(x,4)
  return a / 4;
}

// ---------------------------------------------------------------- graph layout
// Device view of the degree-ordered graph.  Vertices are renamed by their rank
// in the degree order (Sec. 3.2: by degree, ties by original id), so u < v is
// the order itself.  Each row of the CSR is sorted; the out-list N+(v) of the
// DAG is the suffix C[op[v] .. R[v+1]) and the in-list N-(v) the prefix.
struct DevGraph {
  int64_t n;
  int64_t nnz;
  const int64_t* R;     // n+1 row starts
  const int32_t* C;     // nnz neighbours (ranks), sorted per row
  const int64_t* op;    // n: first out-neighbour position of each row
  const int64_t* rev;   // nnz: slot of the reverse entry
};

__device__ __forceinline__ int64_t dg_deg(const DevGraph& g, int64_t v) { return g.R[v + 1] - g.R[v]; }
__device__ __forceinline__ int64_t dg_outdeg(const DevGraph& g, int64_t v) { return g.R[v + 1] - g.op[v]; }

// lower_bound of key in sorted C[lo, hi)
__device__ __forceinline__ int64_t lower_bound_i32(const int32_t* a, int64_t lo, int64_t hi, int32_t key) {
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------- shared lists
// Append j to a block-shared list where `take` holds, with one atomic per warp
// instead of one per entry: the lanes executing together vote, the lowest
// voter reserves room for all of them and each voter writes its own slot.
// The order of entries inside the list is unspecified.
__device__ __forceinline__ void warp_append(int32_t* list, unsigned* n, bool take, int32_t j) {
  unsigned am = __activemask();
  unsigned b = __ballot_sync(am, take);
  if (!b) return;
  int lane = threadIdx.x & 31, leader = __ffs(b) - 1;
  unsigned base = 0;
  if (lane == leader) base = atomicAdd(n, (unsigned)__popc(b));
  base = __shfl_sync(am, base, leader);
  if (take) list[base + __popc(b & ((1u << lane) - 1u))] = j;
}

// ---------------------------------------------------------------- status word
// Device-side error flags (no traps): kernels record the first problem they
// meet here and skip the offending access; the host turns a non-zero word
// into an error status.
enum DevErr : unsigned {
  DEVERR_NONE = 0,
  DEVERR_SCRATCH = 1u << 0,   // a scratch capacity was exceeded
  DEVERR_BOUNDS = 1u << 1,    // an index fell outside its array
  DEVERR_OVERFLOW = 1u << 2,  // a per-element counter overflowed
};

__device__ __forceinline__ void set_err(unsigned* st, unsigned bit) { atomicOr(st, bit); }

// ---------------------------------------------------------------- ownership
// When one census is split over `parts` processes (each holding the whole
// graph), work item i -- a vertex rank -- belongs to part i mod parts.  Ranks
// are in degree order, so every part gets the same mix of heavy and light
// items.  Items are taken from the top rank down.
struct Owner {
  int part = 0, parts = 1;
  __host__ __device__ bool owns(int64_t i) const { return parts <= 1 || i % parts == part; }
  __host__ __device__ int64_t top(int64_t n) const {      // highest owned rank, or -1
    if (n <= 0) return -1;
    int64_t t = n - 1 - ((n - 1 - part) % parts + parts) % parts;
    return t >= part ? t : -1;
  }
  __host__ __device__ int64_t count(int64_t n) const {
    int64_t t = top(n);
    return t < 0 ? 0 : (t - part) / parts + 1;
  }
  __host__ __device__ int64_t item(int64_t n, int64_t it) const { return top(n) - it * parts; }
};

// ---------------------------------------------------------------- work queue
// Persistent CTAs pull vertex indices from `order` (vertices sorted by
// decreasing work estimate) through one global counter.
__device__ __forceinline__ int64_t next_item(unsigned long long* ctr, int64_t n, int64_t* sh_item) {
  if (threadIdx.x == 0) *sh_item = (int64_t)atomicAdd(ctr, 1ull);
  __syncthreads();
  int64_t it = *sh_item;
  __syncthreads();
  return it < n ? it : -1;
}
