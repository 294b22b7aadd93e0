// noalloc.cu -- per-vertex 4-cycle counts without any device allocation.
//
// Some callers cannot allocate device memory at the time they want a count:
// a serving loop that has handed all of the GPU's memory to its own pool, or
// a latency-critical path that must not let cudaMalloc/cudaFree synchronise
// the device behind other streams' backs.  escape_cycles4_noalloc serves them:
// the caller passes device inputs and outputs, and the only work space is the
// fixed array below, which lives as long as the library is loaded.
//
// The counting is the 4-cycle rule of the main library (for the highest
// vertex i of a 4-cycle and the opposite vertex j, the number of middles
// below i), run here directly on the caller's CSR with the degree order
// computed on the fly instead of renaming vertices.
#include "../../include/escape.h"
#include "common.cuh"
#include "internal.h"

#include <mutex>

namespace {

constexpr int NA_CTAS = 32;                         // persistent CTAs
constexpr int NA_THREADS = 512;
constexpr int64_t NA_MAX_N = ESCAPE_NOALLOC_MAX_N;  // vertices
// Work space shared by every call on this device: per CTA a counter array and
// a touched list of NA_MAX_N entries each (8 MiB in total), then a header of
// 64 words (work counter, status).
constexpr int64_t NA_WORDS = (int64_t)NA_CTAS * NA_MAX_N * 2 + 64;
static __device__ __align__(256) unsigned int g_noalloc_scratch[NA_WORDS];

std::mutex g_mu;
void* g_addr[64] = {nullptr};     // device address of g_noalloc_scratch, per device

__device__ __forceinline__ bool na_prec(const int64_t* rp, int64_t a, int64_t b) {
  int64_t da = rp[a + 1] - rp[a], db = rp[b + 1] - rp[b];
  return da < db || (da == db && a < b);
}

// Row v's entry range, clamped: an offset outside [0, rp[n]] or a row that
// ends before it starts sets the status word and reads as an empty row, so no
// access leaves col[0 .. rp[n]).
__device__ __forceinline__ void na_row(const int64_t* rp, int64_t n, int64_t v, int64_t& b, int64_t& e,
                                       unsigned int* status) {
  b = rp[v];
  e = rp[v + 1];
  int64_t lim = rp[n];
  if (b < 0 || e < b || e > lim) {
    atomicOr(status, 1u);
    b = e = 0;
  }
}

__global__ void k_cycles4_noalloc(const int64_t* rp, const int32_t* col, int64_t n, unsigned int* scratch,
                                  unsigned long long* c4v, unsigned long long* c4_total) {
  __shared__ u128 sh[32];
  __shared__ int64_t sh_item;
  unsigned int* w = scratch + (int64_t)blockIdx.x * NA_MAX_N;
  int32_t* tl = (int32_t*)(scratch + (int64_t)NA_CTAS * NA_MAX_N + (int64_t)blockIdx.x * NA_MAX_N);
  unsigned int* hdr = scratch + (int64_t)NA_CTAS * NA_MAX_N * 2;
  unsigned long long* ctr = (unsigned long long*)hdr;          // hdr[0..1]
  unsigned int* status = hdr + 2;
  __shared__ unsigned int nt;
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  u128 total = 0;
  while (true) {
    if (threadIdx.x == 0) sh_item = (int64_t)atomicAdd(ctr, 1ull);
    __syncthreads();
    int64_t i = sh_item;
    __syncthreads();
    if (i >= n) break;
    if (threadIdx.x == 0) nt = 0;
    __syncthreads();
    int64_t ib, ie;
    na_row(rp, n, i, ib, ie, status);
    // pass 1: wedges i - k - j with k, j below i in the degree order
    for (int64_t p = ib + wid; p < ie; p += nw) {
      int32_t k = col[p];
      if (k < 0 || k >= n) { if (lane == 0) atomicOr(status, 1u); continue; }
      if (!na_prec(rp, k, i)) continue;
      int64_t kb, ke;
      na_row(rp, n, k, kb, ke, status);
      for (int64_t q = kb + lane; q < ke; q += 32) {
        int32_t j = col[q];
        if (j < 0 || j >= n) { atomicOr(status, 1u); continue; }
        if (j == i || !na_prec(rp, j, i)) continue;
        if (atomicAdd(&w[j], 1u) == 0) tl[atomicAdd(&nt, 1u)] = j;
      }
    }
    __syncthreads();
    unsigned int ntc = nt;
    // pass 2: C(w, 2) to i and j
    u128 mine = 0;
    for (unsigned int t = threadIdx.x; t < ntc; t += blockDim.x) {
      int32_t j = tl[t];
      unsigned long long c = (unsigned long long)w[j] * (w[j] - 1) / 2;
      if (c) { atomicAdd(&c4v[j], c); mine += c; }
    }
    u128 s = block_sum_u128(mine, sh);
    if (threadIdx.x == 0) { if (s) atomicAdd(&c4v[i], (unsigned long long)s); total += s; }
    // pass 3: w - 1 to every middle k
    for (int64_t p = ib + wid; p < ie; p += nw) {
      int32_t k = col[p];
      if (k < 0 || k >= n || !na_prec(rp, k, i)) continue;
      unsigned long long sk = 0;
      int64_t kb, ke;
      na_row(rp, n, k, kb, ke, status);
      for (int64_t q = kb + lane; q < ke; q += 32) {
        int32_t j = col[q];
        if (j < 0 || j >= n || j == i || !na_prec(rp, j, i)) continue;
        sk += w[j] - 1;
      }
      sk = warp_sum_u64(sk);
      if (lane == 0 && sk) atomicAdd(&c4v[k], sk);
    }
    __syncthreads();
    for (unsigned int t = threadIdx.x; t < ntc; t += blockDim.x) w[tl[t]] = 0;
    __syncthreads();
  }
  // each 4-cycle is counted once, at its highest vertex
  if (threadIdx.x == 0 && total) atomicAdd(c4_total, (unsigned long long)total);
}

}  // namespace

extern "C" escape_status escape_cycles4_noalloc(int64_t n, const int64_t* row_ptr, const int32_t* col,
                                                uint64_t* c4_v, uint64_t* c4_total, void* stream) {
  if (n < 0 || (n > 0 && (!row_ptr || !col || !c4_v)) || !c4_total) return ESCAPE_EINVAL;
  if (n > NA_MAX_N) return ESCAPE_EOVERFLOW;     // beyond the fixed work space
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    esc::note_cuda_error(e);
    return ESCAPE_ECUDA;
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      e = cudaGetSymbolAddress(&g_addr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) { g_addr[dev] = nullptr; cudaGetLastError(); esc::note_cuda_error(e); return ESCAPE_ECUDA; }
    }
    base = g_addr[dev];
  }
  unsigned int* scratch = (unsigned int*)base;
  // everything the kernel expects to start at zero: counters, header, outputs
  e = cudaMemsetAsync(scratch, 0, sizeof(unsigned int) * (size_t)NA_WORDS, s);
  if (e == cudaSuccess && n > 0) e = cudaMemsetAsync(c4_v, 0, sizeof(uint64_t) * (size_t)n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c4_total, 0, sizeof(uint64_t), s);
  if (e != cudaSuccess) { cudaGetLastError(); esc::note_cuda_error(e); return ESCAPE_ECUDA; }
  if (n > 0) {
    k_cycles4_noalloc<<<NA_CTAS, NA_THREADS, 0, s>>>(row_ptr, col, n, scratch, (unsigned long long*)c4_v,
                                                     (unsigned long long*)c4_total);
  }
  unsigned int status = 0;
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&status, scratch + (int64_t)NA_CTAS * NA_MAX_N * 2 + 2, sizeof(unsigned int),
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { cudaGetLastError(); esc::note_cuda_error(e); return ESCAPE_ECUDA; }
  return status ? ESCAPE_EINVAL : ESCAPE_OK;
}
