// internal.h -- host-side declarations shared by the translation units of the
// CUDA library (not part of the public C ABI).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace esc {

// Bump allocator over one device buffer.  Kernels run in stream order on a
// single stream, so releasing a region (moving the mark back) while earlier
// kernels that used it are still queued is safe: later users are ordered
// after them.
struct DeviceArena {
  char* base = nullptr;
  size_t cap = 0;
  size_t top = 0;
  void* alloc(size_t bytes) {
    size_t a = (top + 255) & ~(size_t)255;
    if (a + bytes > cap) return nullptr;
    top = a + bytes;
    return base + a;
  }
  size_t mark() const { return top; }
  void release(size_t m) { top = m; }
};

// The degree-ordered graph in rank space (Sec. 3.2).
struct Oriented {
  int32_t* perm = nullptr;   // n: original id of each rank
  int32_t* rank = nullptr;   // n: rank of each original id
  int64_t* R = nullptr;      // n+1
  int32_t* C = nullptr;      // nnz
  int64_t* op = nullptr;     // n
  int64_t* rev = nullptr;    // nnz
};

// Counts kernel launches made by this thread (reported per census call).
void note_launch();
// Records a failing CUDA call of the calling thread (escape_last_cuda_error).
void note_cuda_error(cudaError_t e);
long long launches_so_far();

int bits_for(int64_t n);
cudaError_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, bool with_total, DeviceArena& arena,
                               cudaStream_t s);
cudaError_t radix_sort(uint64_t* keys, uint32_t* vals, uint64_t* tk, uint32_t* tv, int64_t n, int bits,
                       DeviceArena& arena, cudaStream_t s);
cudaError_t normalize_csr(int64_t n, int64_t nnz_in, const int64_t* rp_in, const int32_t* col_in, int64_t** rp_out,
                          int32_t** col_out, int64_t* nnz_out, unsigned* d_status, DeviceArena& arena,
                          cudaStream_t s, int sms);
cudaError_t validate_csr(int64_t n, const int64_t* rp, const int32_t* col, unsigned* d_status, cudaStream_t s,
                         int sms);
cudaError_t orient(const int64_t* rp, const int32_t* col, int64_t n, int64_t nnz, Oriented& o, DeviceArena& arena,
                   cudaStream_t s, int sms);

// Per-element results in rank space (canonical slots = the lower endpoint's
// out-list; both slots hold the value after symmetrisation).
struct PerElement {
  uint32_t* Te = nullptr;          // nnz: triangles on each edge
  unsigned long long* C4e = nullptr;  // nnz: 4-cycles on each edge
  unsigned long long* K4e = nullptr;  // nnz: 4-cliques on each edge
  unsigned long long* tv = nullptr;   // n: triangles at each vertex
  unsigned long long* C4v = nullptr;  // n
  unsigned long long* K4v = nullptr;  // n
};

struct CensusTimings {
  float ms[16];
  int count;
};

// Runs the whole census (orientation through conversion) for one graph held in
// device memory (original ids), writing 2 x 49 u128 counts (induced 4+11+34,
// then non-induced) to `d_out` (device) and, when `pe` is non-null, keeping the
// per-element arrays.  Work space comes from the library's device-buffer
// cache (allocated inside, sized from the graph).
struct CensusConfig {
  int sms = 0;                    // SM count of the device
  int cta_per_sm = 2;             // persistent CTAs per SM for the sweep kernels
  bool keep_per_element = false;
  bool serial_phases = false;     // run every phase on the caller's stream, one after another
  bool four_only = false;         // 3- and 4-vertex counts only: skip the lists, pairs, wheels and 5-cycles
  cudaEvent_t* phase_events = nullptr;   // optional: records an event after each phase
  int num_phase_events = 0;
  // batch: the graph is the block-diagonal union of num_graphs graphs whose
  // vertices are [d_vtx_offsets[k], d_vtx_offsets[k+1]) (device array); d_out
  // then receives num_graphs results
  const int64_t* d_vtx_offsets = nullptr;
  int num_graphs = 1;
  // optional device output: per graph W, D, directed 3-paths, directed
  // bipyramids (4 x u128, two little-endian words each)
  unsigned long long* d_basis = nullptr;
  // a census split over `parts` processes: this call counts the items of
  // `part` (vertex ranks i with i mod parts = part) and, with `partial`, stops
  // before the closed forms, writing its raw sums (census_sum_count() u128)
  // to d_acc_out and keeping the per-element arrays (pe_out, or_out required)
  int part = 0, parts = 1;
  bool partial = false;
  unsigned long long* d_acc_out = nullptr;
};

cudaError_t run_census(const int64_t* rp, const int32_t* col, int64_t n, int64_t nnz, const CensusConfig& cfg,
                       unsigned long long* d_out, unsigned* d_status, PerElement* pe_out, Oriented* or_out,
                       cudaStream_t s);

// The end of a split census (see CensusConfig::partial): d_acc holds every
// part's raw sums added, pe every part's per-element counts added.
cudaError_t run_census_finish(const Oriented& o, int64_t n, int64_t nnz, const PerElement& pe,
                              const unsigned long long* d_acc, unsigned long long* d_out, int sms, cudaStream_t s);

// Number of raw 128-bit sums of one part of a split census.
int census_sum_count();

// Conversion tables (App. B), built on the host by this library's own
// embedding count over the pattern catalogue.
void conversion_inverse(int k, long long* Ainv /* ncls x ncls */);

}  // namespace esc
