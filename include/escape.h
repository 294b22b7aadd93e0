/*
 * escape.h -- C ABI of the GB300 ESCAPE census library (libescape_gb300.so).
 *
 * The library computes the exact census of all 3-, 4- and 5-vertex patterns of
 * an undirected simple graph: for every isomorphism class H of k-vertex graphs
 * (k = 3, 4, 5) the induced count C_H = #{S : |S| = k, G[S] ~ H} and the
 * non-induced count N_H (Sec. 3.1 of Pinar, Seshadhri, Vishal, "ESCAPE:
 * Efficiently Counting All 5-Vertex Subgraphs", arXiv 1610.09411).  Every step
 * runs on the GPU: degree ordering (Sec. 3.2), per-vertex/per-edge triangle,
 * 4-cycle and 4-clique counts (Thms 5-7), the pattern-cutting closed forms
 * (Thms 4, 8-11), 5-cycles and 5-cliques (Thms 13-14), disconnected patterns
 * (Thm 3) and the induced/non-induced conversion (App. B).
 *
 * Class order.  3-vertex: empty, edge, wedge, triangle.  4-vertex: the six
 * connected patterns of the paper's 4-vertex figure (3-star, 3-path, tailed
 * triangle, 4-cycle, diamond, 4-clique), then independent set, edge + 2
 * isolated, 2 disjoint edges, wedge + isolated, triangle + isolated.
 * 5-vertex: patterns 1-21 of the paper's figure of connected 5-vertex patterns,
 * 22-32 of its figure of disconnected 5-vertex patterns (empty, edge, 2 edges,
 * wedge, triangle, 3-star, 3-path, tailed triangle, 4-cycle, diamond, 4-clique,
 * each plus isolated vertices), 33 = wedge + disjoint edge, 34 = triangle +
 * disjoint edge (the two classes the paper's figure leaves out).
 *
 * Counts are exact unsigned 128-bit integers (two little-endian 64-bit words).
 *
 * Threading: a handle may be used by one thread at a time; different handles
 * may be used from different threads at the same time, each on its own stream
 * (a serving loop with several workers does this).  All calls are
 * synchronous with respect to the host: they enqueue work on the given CUDA
 * stream (NULL = the legacy default stream) and wait for it before returning.
 * No C++ exception or exit() crosses this boundary.
 */
#ifndef ESCAPE_GB300_H
#define ESCAPE_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct escape_graph escape_graph;   /* opaque; owns a device copy of the CSR */

typedef struct { uint64_t lo, hi; } escape_u128;

typedef struct {
  escape_u128 c3[4], c4[11], c5[34];   /* induced counts, class order above       */
  escape_u128 n3[4], n4[11], n5[34];   /* non-induced counts (Sec. 3.1)             */
} escape_census;

typedef struct {                       /* the 3- and 4-vertex part of escape_census */
  escape_u128 c3[4], c4[11];
  escape_u128 n3[4], n4[11];
} escape_census34;

typedef enum {
  ESCAPE_OK = 0,
  ESCAPE_EINVAL = 1,     /* invalid argument or malformed graph                     */
  ESCAPE_ENOMEM = 2,     /* a host or device allocation failed                      */
  ESCAPE_ECUDA = 3,      /* a CUDA call failed (the context may be unusable)        */
  ESCAPE_EOVERFLOW = 4,  /* a size exceeds what the library supports                */
  ESCAPE_ETIMEOUT = 5,   /* a bounded device wait ran out                           */
  ESCAPE_EINTERNAL = 6   /* a device-side consistency check failed                  */
} escape_status;

/* flags for escape_load_csr / escape_census5_batch */
#define ESCAPE_HOST_PTRS   0u        /* row_ptr/col are host memory                    */
#define ESCAPE_DEVICE_PTRS 1u        /* row_ptr/col are device memory                  */
#define ESCAPE_NORMALIZE   2u        /* symmetrise, drop duplicates and self-loops (Sec. 8) */

/*
 * escape_load_csr -- copy a graph to the device and validate it.
 *   n        number of vertices, 0 <= n <= 2^31 - 1
 *   nnz      number of entries of col (= 2 x edges for a simple symmetric graph)
 *   row_ptr  int64[n + 1], row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz
 *   col      int32[nnz], neighbour ids in [0, n)
 *   flags    ESCAPE_HOST_PTRS or ESCAPE_DEVICE_PTRS, optionally | ESCAPE_NORMALIZE.
 *            Without NORMALIZE the input must already be simple: rows sorted
 *            strictly ascending, no self-loops, symmetric; otherwise EINVAL.
 *            With NORMALIZE any entries are accepted (direction ignored,
 *            duplicates and self-loops dropped); ids out of range give EINVAL.
 *   stream   cudaStream_t as void* (NULL = default stream)
 *   out      receives the new handle; untouched on error.
 * The caller keeps ownership of row_ptr/col (they are copied and may be freed
 * on return).  The handle is freed with escape_free.
 */
escape_status escape_load_csr(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col, uint32_t flags,
                              void* stream, escape_graph** out);

/* Vertices and undirected edges of a loaded graph (either pointer may be NULL). */
escape_status escape_graph_info(const escape_graph* g, int64_t* n, int64_t* m);

/*
 * escape_census5 -- the full census of a loaded graph (Thm 2: all connected
 * 5-vertex patterns; Thm 3: disconnected ones; App. B: induced counts),
 * together with the 3- and 4-vertex census (Thm 1).
 *   out      host memory; written only on success.
 * Device work space is allocated for the call and released before it returns;
 * released buffers (up to 8 GiB per device) are kept for later calls instead
 * of being freed, and the whole cache is freed whenever an allocation of a
 * later call would otherwise fail.
 * Graphs with n < 5, no edges, or no triangles are valid.
 */
escape_status escape_census5(escape_graph* g, escape_census* out, void* stream);

/*
 * escape_census4 -- the 3- and 4-vertex census alone (Thm 1; the paper's
 * section on counting 4-vertex patterns): the same counts as the c3, c4, n3,
 * n4 fields of escape_census5, computed from the degree sums, triangles,
 * 4-cycles and 4-cliques only, without the common-neighbour lists, pair,
 * wheel and 5-cycle sweeps that the 5-vertex counts need.
 *   out      host memory; written only on success.
 * Options, per-element arrays (escape_per_element: T, C4 and K4 are all
 * computed here), phase times and errors as for escape_census5; the skipped
 * phases report 0 ms.
 */
escape_status escape_census4(escape_graph* g, escape_census34* out, void* stream);

/*
 * escape_census5_batch -- census of many small graphs given as one block
 * diagonal CSR.
 *   num_graphs   G >= 0
 *   vtx_offsets  int64[G + 1]: graph k owns global rows vtx_offsets[k] ..
 *                vtx_offsets[k+1]-1; vtx_offsets[0] = 0
 *   row_ptr      int64[vtx_offsets[G] + 1] over all rows
 *   col          int32[row_ptr[last]]: neighbour ids LOCAL to each graph
 *                (0 .. n_k - 1)
 *   flags        as for escape_load_csr (pointers are host or device memory)
 *   out          host array of G results, written only on success.
 * Results are identical to calling escape_census5 on each graph alone.
 */
escape_status escape_census5_batch(int32_t num_graphs, const int64_t* vtx_offsets, const int64_t* row_ptr,
                                   const int32_t* col, uint32_t flags, escape_census* out, void* stream);

/*
 * escape_per_element -- per-vertex and per-edge counts of the last
 * escape_census5 call on this handle (Thm 7), in the layout of the loaded CSR:
 *   tri_e, c4_e, k4_e   uint64[nnz]: triangles / 4-cycles / 4-cliques through
 *                       the edge of each CSR entry (both entries of an edge agree)
 *   tri_v, c4_v, k4_v   uint64[n]: triangles / 4-cycles / 4-cliques at each vertex
 * Host memory; any pointer may be NULL.  EINVAL if no census has been run
 * with per-element output enabled (escape_set_options).
 */
escape_status escape_per_element(escape_graph* g, uint64_t* tri_e, uint64_t* c4_e, uint64_t* k4_e, uint64_t* tri_v,
                                 uint64_t* c4_v, uint64_t* k4_v, void* stream);

/* Options: keep_per_element (0/1) makes escape_census5 retain the arrays
 * read by escape_per_element; cta_per_sm sets the persistent-CTA count of the
 * sweep kernels (0 = default, 1..8); serial_phases 1 runs every phase on the
 * caller's stream one after another, 0 overlaps the independent sweeps on
 * side streams, and a negative value (the default) chooses by size: one after
 * another for graphs of at least 2^24 adjacency entries (2 x edges), where
 * each sweep fills the GPU alone, overlapped below.  The results are the
 * same either way; with the phases one after another, the times of
 * escape_last_phase_ms are each kernel's time alone. */
escape_status escape_set_options(escape_graph* g, int keep_per_element, int cta_per_sm, int serial_phases);

/*
 * escape_last_phase_ms -- device time (CUDA events) of each phase of the last
 * escape_census5 call on this handle: [0] orientation, [1] triangles,
 * [2] cliques and per-triangle sums, [3] 4-cycles, [4] common-neighbour lists,
 * [5] pair sweep (N13, N17), [6] wheels (N18), [7] 5-cycles, [8] assembly.
 * Writes min(count, 9) floats; returns the number of phases available.
 */
int escape_last_phase_ms(const escape_graph* g, float* ms, int count);

/* Number of CUDA kernels the last escape_census5 call on this handle launched. */
long long escape_last_kernel_launches(const escape_graph* g);

/*
 * escape_last_basis_counts -- the four counts the paper fits the census's run
 * time to (Sec. 8, the runtime-prediction figure; Thm 2's bound
 * O(W + D + DP + DBP + m + n)), from the last escape_census5 call on this
 * handle:
 *   out[0] W    wedges, sum_i C(d_i, 2)
 *   out[1] D    diamonds, sum over edges of C(T_e, 2)
 *   out[2] DP   directed 3-paths i <- a -> b -> j of the degree-ordered DAG,
 *               counted as sum over out-edges a -> b of (d+(a) - 1) d+(b)
 *   out[3] DBP  directed bipyramids: over directed triangles x < y < z,
 *               C(number of common out-neighbours of x, y, z above z, 2)
 *   out      host array of 4; written only on success.
 * EINVAL if the handle has no completed escape_census5 call (escape_census4
 * does not compute DP and DBP).
 */
escape_status escape_last_basis_counts(const escape_graph* g, escape_u128* out);

/*
 * escape_cycles4_noalloc -- per-vertex 4-cycle counts C4(i) and the total C4
 * of a graph, computed without allocating any memory.  (The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory when they need the count -- for example a serving loop whose
 * device memory is all handed to its own pool, or a latency-critical path that
 * must not let cudaMalloc/cudaFree synchronise the device.)
 *   n         number of vertices, 0 <= n <= ESCAPE_NOALLOC_MAX_N, else EOVERFLOW
 *   row_ptr   DEVICE int64[n + 1], col DEVICE int32[row_ptr[n]]: a simple graph
 *             as for escape_load_csr without NORMALIZE (sorted symmetric rows,
 *             no self-loops); ids outside [0, n), and row offsets outside
 *             [0, row_ptr[n]] or decreasing, are skipped and give EINVAL
 *   c4_v      DEVICE uint64[n] output: 4-cycles through each vertex
 *   c4_total  DEVICE uint64[1] output: number of 4-cycles
 * Work space is one fixed device array of ESCAPE_NOALLOC_MAX_N x 64 words
 * (8 MiB) inside the library, shared by every call: calls whose GPU work
 * overlaps (on different streams or threads) race and must be serialised by
 * the caller.  Each call clears the work space and the outputs before
 * counting.  The array takes its device memory when the library's device
 * code is loaded on a device -- with CUDA's lazy module loading, during the
 * first call on that device -- and keeps it until the process exits; so make
 * the first call on each device before the caller's own pool claims the
 * device's memory.  That first call also looks up the array's device address
 * (one-time set-up per device).  Every call reads a status word back and
 * waits for its stream before returning, so no call may be made while its
 * stream is being captured into a CUDA graph.
 * No cudaMalloc, cudaFree or allocating library routine is called.
 */
#define ESCAPE_NOALLOC_MAX_N 32768
escape_status escape_cycles4_noalloc(int64_t n, const int64_t* row_ptr, const int32_t* col, uint64_t* c4_v,
                                     uint64_t* c4_total, void* stream);

/*
 * A census split over several processes or GPUs, each holding the whole graph
 * (the graph is loaded by every part).  Every part runs
 *   escape_census5_part(g, part, parts, &p, s)
 * which orients the graph and counts its triangles in full, then counts the
 * enumeration sweeps (4-cliques, 5-cliques and the per-triangle sums; 4-cycles;
 * pair, wheel and 5-cycle sweeps; Thms 5-7, 10-14) for the work items it owns
 * only: vertex ranks r of the degree order (Sec. 3.2) with r mod parts = part.
 * Its result is
 *   p.sums       the part's raw 128-bit sums (the first escape_part_sum_count()
 *                entries; the rest zero); the sums of the phases every part
 *                repeats are counted by part 0 alone
 *   per-element  K4 per edge, C4 per edge, C4 per vertex (uint64 arrays of
 *                nnz, nnz and n entries in the library's internal order, the
 *                same on every part), read and written with escape_part_counts.
 * The parts then exchange: every sum added over the parts (exactly, modulo
 * 2^128), and every per-element array added element-wise over the parts (into
 * each part's copy with flags | ESCAPE_PART_PUT, or into one part's only).
 * One part (or each) then calls escape_census5_finish(g, &total, &out, s),
 * which applies the closed forms to the totals and writes the same census as
 * escape_census5 (Thm 2, Thm 3, App. B).  This is the one exchange step of the
 * census: no other data crosses between parts.
 *   part, parts  0 <= part < parts, else EINVAL
 *   out/total    host memory
 * escape_part_counts:
 *   k4_e, c4_e, c4_v   host (flags without ESCAPE_DEVICE_PTRS) or device
 *                      arrays of nnz, nnz, n uint64; any may be NULL
 *   flags              ESCAPE_HOST_PTRS / ESCAPE_DEVICE_PTRS, | ESCAPE_PART_PUT
 *                      to write the arrays into the handle instead of reading
 * EINVAL when the handle holds no part (no escape_census5_part since the last
 * census or finish).  escape_census5_finish releases the part's arrays.
 */
#define ESCAPE_PART_SUMS 64
#define ESCAPE_PART_PUT 4u
typedef struct { escape_u128 sums[ESCAPE_PART_SUMS]; } escape_part;
escape_status escape_census5_part(escape_graph* g, int32_t part, int32_t parts, escape_part* out, void* stream);
escape_status escape_part_counts(escape_graph* g, uint64_t* k4_e, uint64_t* c4_e, uint64_t* c4_v, uint32_t flags,
                                 void* stream);
escape_status escape_census5_finish(escape_graph* g, const escape_part* total, escape_census* out, void* stream);
/* Number of meaningful entries of escape_part.sums. */
int escape_part_sum_count(void);

void escape_free(escape_graph* g);

/* Static string for a status code. */
const char* escape_status_str(escape_status s);

/*
 * escape_last_cuda_error -- the CUDA runtime error (a cudaError_t value) of
 * the last failing CUDA call that a call of this library turned into a status
 * on the calling thread (always for ESCAPE_ECUDA; ESCAPE_ENOMEM and
 * ESCAPE_EOVERFLOW can also come from host-side checks, which leave it
 * unchanged), or 0 if there has been none.  If name is not NULL, *name
 * receives the error's symbolic name (static storage owned by the CUDA
 * runtime; "" for 0).  Diagnostic only: the value is per host thread.
 */
int escape_last_cuda_error(const char** name);

#ifdef __cplusplus
}
#endif
#endif /* ESCAPE_GB300_H */
