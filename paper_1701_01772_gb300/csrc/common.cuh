// Shared declarations of libgraphlet's CUDA sources (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "graphlet.h"

namespace gs {

// ---------------------------------------------------------------- errors

void set_error(const char* fmt, ...);
gs_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define GS_CUDA(call)                                                       \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess) return gs::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define GS_TRY(call)                      \
  do {                                    \
    gs_status s_ = (call);                \
    if (s_ != GS_OK) return s_;           \
  } while (0)

// Device-side error record: the first failing kernel stores a status code
// and the index of the offending element.
struct DevError {
  int32_t code;
  int32_t pad;
  int64_t index;
};

__device__ __forceinline__ void raise_error(DevError* err, int32_t code, int64_t index) {
  if (atomicCAS(&err->code, 0, code) == 0) err->index = index;
}

// ---------------------------------------------------------------- graph

// The hub-pair bit matrix covers at most this many vertices (32767 squared
// bits = 128 MiB, about the size of the 129 MB L2; its rows of the
// highest-degree vertices, which most tests touch, stay resident). On R-MAT
// scale 24 the 1% estimate took 3.69 s with 16384 vertices and 3.22 s with
// 32767 (more edges go dense, fewer single tests).
#ifndef GS_HUB_MATRIX_MAX
#define GS_HUB_MATRIX_MAX 32767
#endif
constexpr int64_t kHubMatrixMax = GS_HUB_MATRIX_MAX;
static_assert(kHubMatrixMax <= 32767, "matrix slots are stored in 16 bits");
// Default number of matrix slots (the highest-degree vertices) that take
// part in dense clique mode; the rest of the matrix answers single tests.
#ifndef GS_HUB_DENSE_SLOTS
#define GS_HUB_DENSE_SLOTS GS_HUB_MATRIX_MAX
#endif
constexpr int64_t kHubDenseSlots = GS_HUB_DENSE_SLOTS;

// Device view of a registered graph plus its hub index.
struct DevGraph {
  const int64_t* row_ptr;   // [n+1]
  const int32_t* col;       // [nnz], sorted per row
  const int64_t* up_ptr;    // [n] index in col of the first neighbour > v
  int64_t n;
  int64_t nnz;
  // adjacency bitmaps of the highest-degree vertices ("hubs")
  const int32_t* bm_slot;   // [n] bitmap slot of v, -1 if none (NULL if no bitmaps)
  const uint32_t* bm_bits;  // [bm_count][bm_words]
  int64_t bm_words;         // ceil(n / 32)
  int64_t bm_count;
  // co-degree table |N(x) cap N(y)| for the highest-degree vertices
  const int32_t* tb_slot;   // [n] table slot of v, -1 if none, <= -2 mid row (NULL if no table)
  const uint16_t* tb_codeg; // upper triangle, entry tb_index(lo, hi); 0xFFFF: see below
  int64_t tb_count;
  // pairs of "giant" table hubs (degree >= 65,536) have 32-bit co-degrees:
  // tb_giant_codeg[tb_giant[lo]][tb_giant[hi]] (tb_giant NULL if none)
  const int32_t* tb_giant;
  const uint32_t* tb_giant_codeg;
  int64_t tb_giants;
  // co-degrees between "mid" vertices (degree below the table's threshold,
  // tb_slot[a] = -2 - row) and the bg_count "big" table vertices
  // (bg_slot[b] >= 0): md_codeg[row][bg_slot[b]], 16-bit entries
  const int32_t* bg_slot;    // [n] column of v, -1 if none (NULL if absent)
  const uint16_t* md_codeg;  // [md_count][bg_count]
  int64_t md_count, bg_count;
  // adjacency among the top hm_count vertices as a bit matrix over their
  // own slots (hm_count^2 bits, small enough to stay in L2)
  const int32_t* hm_slot;   // [n] matrix slot of v, -1 if none
  const int16_t* col_hm;    // [nnz] matrix slot of col[p], -1 if none (NULL if no matrix)
  // adjacency bit matrices of small graphs (one block per graph of at most
  // kDenseGraphMax vertices; a batch holds one block per member graph):
  // row of v starts at word dm_row[v] (-1: no block), bit x - dm_first[v]
  const uint32_t* dm_bits;
  const int64_t* dm_row;
  const int32_t* dm_first;
  const uint32_t* hm_bits;  // [hm_count][hm_words]
  int64_t hm_words;         // ceil(hm_count / 128) * 4
  // dense clique mode uses the first hm_dense_words * 32 slots (a multiple
  // of 128, at most hm_words * 32; 0 = no dense mode); set per call
  int64_t hm_dense_words;
  // per vertex v, for the work of T's members without a dense slot in a
  // dense edge: the matrix slots of v's matrix neighbours (in adjacency
  // order) and v's neighbours above v without a matrix slot; hm_vertex =
  // vertex of each matrix slot (all NULL without a matrix)
  const int64_t* mn_ptr;   // [n+1]
  const int16_t* mn_slot;  // [mn_ptr[n]]
  const int64_t* nm_ptr;   // [n+1]
  const int32_t* nm_col;   // [nm_ptr[n]]
  const int32_t* hm_vertex;  // [hm_count]
  int64_t hm_count;
  // bucket directories of the adjacency lists of vertices that have no
  // bitmap (degree at least a threshold): the neighbours x of v with
  // x >> s_v == b sit at offsets [D[b], D[b + 1]) of N(v), D = dir +
  // dir_at[v], s_v = id_bits - dir_log2(deg v)
  const int64_t* dir_at;    // [n] first directory entry of v, -1 if none (NULL if absent)
  const uint32_t* dir;
  int32_t id_bits;          // vertex ids are below 2^id_bits
  int64_t dir_count;        // vertices with a directory
  // beside the adjacency (NULL if absent): tb_slot[col[p]]
  const int32_t* col_tb;
};

// Entry of the table pair (lo, hi), lo < hi < n, in the upper triangle
// stored row by row.
__host__ __device__ __forceinline__ int64_t tb_index(int64_t lo, int64_t hi, int64_t n) {
  return lo * (2 * n - lo - 1) / 2 + (hi - lo - 1);
}

// log2 of the number of directory buckets of a vertex of degree d >= 2:
// floor(log2 d) - 1, so a bucket holds 2 to 4 neighbours on average when
// ids are spread evenly; at most id_bits (one bucket per id).
__host__ __device__ __forceinline__ int dir_log2(int64_t d, int id_bits) {
#ifdef __CUDA_ARCH__
  const int f = 63 - __clzll((long long)d);
#else
  const int f = 63 - __builtin_clzll((unsigned long long)d);
#endif
  const int kb = f - 1;
  return kb < 0 ? 0 : (kb > id_bits ? id_bits : kb);
}

// Loads with an L2 eviction priority: keep (evict_last) for small, heavily
// reused structures, once (evict_first) for large randomly read tables.
__device__ __forceinline__ uint64_t l2_policy_keep() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_policy_once() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint32_t ld_keep(const uint32_t* a) {
  uint32_t v;
  asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(l2_policy_keep()));
  return v;
}
__device__ __forceinline__ uint4 ld_keep4(const uint4* a) {
  uint4 v;
  asm("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(a), "l"(l2_policy_keep()));
  return v;
}
__device__ __forceinline__ uint16_t ld_once16(const uint16_t* a) {
  uint16_t v;
  asm("ld.global.nc.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(v) : "l"(a), "l"(l2_policy_once()));
  return v;
}

// Membership of x in the sorted list a[0..len): branch-free halving search.
// Invariant: if x is present it lies in [base, base + len).
__device__ __forceinline__ bool sorted_contains(const int32_t* __restrict__ a, int64_t len,
                                                int32_t x) {
  if (len <= 0) return false;
  const int32_t* base = a;
  while (len > 1) {
    int64_t half = len >> 1;
    base = (__ldg(base + half) <= x) ? base + half : base;
    len -= half;
  }
  return __ldg(base) == x;
}

// Bitmap slot of v, or -1 (also when there are no bitmaps).
__device__ __forceinline__ int32_t bitmap_slot(const DevGraph& g, int32_t v) {
  return (g.bm_slot != nullptr && v >= 0) ? __ldg(g.bm_slot + v) : -1;
}

// Hub-pair matrix slot of v, or -1 (also when there is no matrix).
__device__ __forceinline__ int32_t table_slot(const DevGraph& g, int32_t v) {
  return (g.hm_bits != nullptr && v >= 0) ? __ldg(g.hm_slot + v) : -1;
}

// Membership of x in N(y): hub-pair bit matrix when both have matrix slots,
// bitmap test for bitmap hubs, halving search otherwise.
__device__ __forceinline__ bool adj_contains(const DevGraph& g, int32_t y, int64_t base_y,
                                             int64_t deg_y, int32_t x, int32_t xs_known = -2) {
  if (g.dm_row != nullptr) {
    const int64_t r = __ldg(g.dm_row + y);
    if (r >= 0) {
      const int32_t lx = x - __ldg(g.dm_first + y);
      return (__ldg(g.dm_bits + r + (lx >> 5)) >> (lx & 31)) & 1u;
    }
  }
  if (g.hm_bits != nullptr) {
    int32_t ys = __ldg(g.hm_slot + y);
    if (ys >= 0) {
      int32_t xs = xs_known != -2 ? xs_known : __ldg(g.hm_slot + x);
      if (xs >= 0) {
        uint32_t w = __ldg(g.hm_bits + (int64_t)ys * g.hm_words + (xs >> 5));
        return (w >> (xs & 31)) & 1u;
      }
    }
  }
  if (g.bm_slot != nullptr) {
    int32_t s = __ldg(g.bm_slot + y);
    if (s >= 0) {
      uint32_t w = __ldg(g.bm_bits + (int64_t)s * g.bm_words + (x >> 5));
      return (w >> (x & 31)) & 1u;
    }
  }
  if (g.dir_at != nullptr) {
    const int64_t at = __ldg(g.dir_at + y);
    if (at >= 0) {
      const uint32_t* d = g.dir + at + (x >> (g.id_bits - dir_log2(deg_y, g.id_bits)));
      const uint32_t lo = __ldg(d), hi = __ldg(d + 1);
      return sorted_contains(g.col + base_y + lo, (int64_t)(hi - lo), x);
    }
  }
  return sorted_contains(g.col + base_y, deg_y, x);
}

// Matrix slot value meaning "not known: look it up".
constexpr int32_t kNoSlotInfo = -2;

// ---------------------------------------------------------------- scan

// Exclusive prefix sum of in[0..count) into out[0..count], out[count] = total.
// `in` and `out` may alias. tmp must hold scan_tmp_elems(count) int64.
int64_t scan_tmp_elems(int64_t count);
gs_status exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t count, int64_t* tmp,
                             cudaStream_t stream);

// Grid size for grid-stride kernels: a multiple of the SM count.
int grid_for(int64_t work_items, int threads_per_block, int blocks_per_sm);
int sm_count();

}  // namespace gs

// ---------------------------------------------------------------- handles

struct gs_graph {
  gs::DevGraph dev;
  int64_t* nbr_degsum;  // [n] sum of the degrees of v's neighbours (cost model)
  int64_t m;            // undirected edges = nnz / 2
  int64_t max_degree;
  int64_t* up_ptr;      // [n]   index in col of the first neighbour > v
  int64_t* edge_off;    // [n+1] canonical (u < v) edge offsets per row
  int32_t* bm_slot;
  uint32_t* bm_bits;
  int32_t* tb_slot;
  uint16_t* tb_codeg;
  int32_t* hm_slot;
  uint32_t* hm_bits;
  int16_t* col_hm;
  int64_t* mn_ptr;
  int16_t* mn_slot;
  int64_t* nm_ptr;
  int32_t* nm_col;
  int32_t* hm_vertex;
  uint32_t* dm_bits;
  int64_t* dm_row;
  int32_t* dm_first;
  int32_t* bg_slot;
  uint16_t* md_codeg;
  int64_t* dir_at;
  uint32_t* dir;
  int32_t* col_tb;
  int32_t* tb_giant;
  uint32_t* tb_giant_codeg;
  // edges oriented from the lower to the higher (degree, id) endpoint, for
  // the exact 3-node pass (NULL when not built): out- and in-lists in
  // increasing id, in_pos = position of v in N+(u) for the in-edge u -> v,
  // orient_units = scanned work units per vertex
  int64_t* out_ptr;
  int32_t* out_col;
  int64_t* in_ptr;
  int32_t* in_col;
  uint32_t* in_pos;
  int64_t* orient_units;
  int64_t max_out_degree;
};

namespace gs {
// Launch-time choices of the counting kernels (the autotuner's knobs).
struct Tuning {
  int tri_blocks_per_sm;    // resident CTAs per SM of the triangle pass
  int quad_blocks_per_sm;   // resident CTAs per SM of the 4-node pass
  int64_t task_probes;      // membership tests per 4-node work unit
  int use_hubs;             // 0: ignore bitmaps / co-degree table / hub matrix
  int64_t dense_slots;      // hub-matrix slots that take part in dense mode
};
}  // namespace gs

struct gs_workspace {
  int has_tuning;
  gs::Tuning tuning;
  void* buf[5];
  size_t cap[5];
  cudaStream_t last_stream;
  int device;
  int timing;
  cudaEvent_t ev[12];   // start/stop pairs for the six gs_count phases
  gs_stats stats;       // last gs_count
  int64_t launches_total;
};

namespace gs {
// Graphs (or batch members) of at most this many vertices get an adjacency
// bit matrix (at most 32 MiB each).
constexpr int64_t kDenseGraphMax = 16384;
// Builds adjacency bit-matrix blocks for the vertex ranges [first[i],
// first[i+1]) of at most kDenseGraphMax vertices (ranges = member graphs of a
// disjoint union; a single range [0, n) for one graph). Skipped silently when
// the blocks would exceed max_bytes or cannot be allocated.
gs_status build_dense_blocks(gs_graph* g, const int64_t* h_first, int64_t ranges,
                             uint64_t max_bytes, cudaStream_t stream);
// Returns a device buffer of at least `bytes` in slot `slot` of the
// workspace, growing it (after synchronising the stream it was last used
// on) when needed. Previously held contents of that slot are lost on growth.
gs_status ws_reserve(gs_workspace* ws, int slot, size_t bytes, cudaStream_t stream, void** out);
gs_status sample_impl(const gs_graph* g, gs_workspace* ws, double fraction, uint64_t seed,
                      int32_t* d_pairs, int64_t max_k, int64_t* k_out, int32_t** pairs_out,
                      cudaStream_t stream);
// Samples canonical edges [e0, e0 + m) (hash index relative to e0).
// Edges of [e0, e0 + m) whose sampler key lies in [fraction_lo, fraction)
// x 2^53 (fraction_lo = 0: the Bernoulli(fraction) sample).
// Edges ranked [k_lo, k_hi) by their sampler key (ties by canonical index),
// in increasing canonical index; d_pairs NULL: into workspace slot 3.
gs_status sample_ranks(const gs_graph* g, gs_workspace* ws, int64_t k_lo, int64_t k_hi,
                       uint64_t seed, int32_t* d_pairs, int32_t** pairs_out,
                       cudaStream_t stream);
gs_status sample_range(const gs_graph* g, gs_workspace* ws, double fraction, uint64_t seed,
                       int64_t e0, int64_t m, int32_t* d_pairs, int64_t max_k, int64_t* k_out,
                       int32_t** pairs_out, cudaStream_t stream, double fraction_lo = 0.0);
}  // namespace gs

namespace gs {
// Device buffers of one counting run.
struct CountBufs {
  int64_t K = 0, P = 0, groups = 0, tsum = 0, dup_cap = 0, nseg = 0;
  int fold_blocks = 0;
  DevError* err = nullptr;
  unsigned long long* sums = nullptr;   // [32] single-segment result
  unsigned long long* stats = nullptr;  // [8]
  int32_t* pairs_all = nullptr;
  int2* uv = nullptr;
  int64_t* off = nullptr;
  int64_t* toff = nullptr;
  unsigned long long *t = nullptr, *k2 = nullptr, *q = nullptr;
  int64_t* tdeg = nullptr;
  int64_t* tmp0 = nullptr;
  unsigned long long* dup = nullptr;
  unsigned __int128* part = nullptr;
  unsigned long long* limbs = nullptr;     // [nseg][16][4]
  unsigned long long* seg_sums = nullptr;  // [nseg][16][2]
  uint32_t* tbits = nullptr;
  int32_t* tpre = nullptr;  // per chunk: T entries of its edge in earlier chunks
  uint32_t* cbits = nullptr;  // per chunk: lanes with tests, lanes answered by a table
  int64_t* task_off = nullptr;
  int64_t* tmp1 = nullptr;
  int32_t* T = nullptr;
  int16_t* T_hm = nullptr;  // matrix slots of T's entries (NULL without a matrix)
  // dense clique mode: per-edge mask index (-1 = sparse edge) and the
  // masks of T's dense-slot members ([ndense][hm_dense_words])
  int32_t* mask_idx = nullptr;
  uint32_t* tmask = nullptr;
  int64_t* dense_e = nullptr;  // edge of each mask ([ndense])
  int64_t* unit_off = nullptr;  // k_dense_pairs work units per mask, scanned ([ndense + 1])
  int64_t* unit_tmp = nullptr;
  int32_t* unit_idx = nullptr;  // dense edge (mask index) of each work unit
  int64_t ndense = 0;
};

Tuning default_tuning();
int quad_blocks_limit();
DevGraph graph_view(const gs_graph* gr, const Tuning& tu);
size_t count_front_bytes(int64_t K, bool all_edges, bool check_dup, int64_t nseg);
void carve_front(void* base, int64_t K, bool all_edges, bool check_dup, int64_t nseg,
                 CountBufs& b);
size_t count_mid_bytes(int64_t P);
void carve_mid(void* base, int64_t P, CountBufs& b);
int64_t launch_front(const gs_graph* gr, const DevGraph& g, const int32_t* pairs, bool four,
                     CountBufs& b, cudaStream_t stream);
int64_t launch_tri(const DevGraph& g, bool four, const Tuning& tu, CountBufs& b,
                   cudaStream_t stream);
int64_t launch_scan_t(CountBufs& b, cudaStream_t stream);
int64_t launch_compact(const DevGraph& g, CountBufs& b, cudaStream_t stream);
int64_t launch_tmask(const DevGraph& g, CountBufs& b, cudaStream_t stream);
int64_t launch_cost(const DevGraph& g, bool need_k, bool need_q, const Tuning& tu, CountBufs& b,
                    cudaStream_t stream);
int64_t launch_dense(const DevGraph& g, bool need_q, CountBufs& b, cudaStream_t stream);
int64_t launch_quad(const DevGraph& g, bool need_k, bool need_q, const Tuning& tu, CountBufs& b,
                    cudaStream_t stream);
int64_t launch_fold(const gs_graph* gr, const DevGraph& g, bool four, bool need_k, bool need_q,
                    int64_t* per_edge, CountBufs& b, cudaStream_t stream);
int64_t launch_fold_seg(const DevGraph& g, bool four, const int64_t* seg_off, CountBufs& b,
                        cudaStream_t stream);
gs_status fetch_error(DevError* d_err, cudaStream_t stream, const char* what);
void store_sums(const unsigned long long* h, uint32_t mask, gs_sums* out);
// tri_oriented.cu: oriented lists at registration and the exact 3-node pass
// over every edge through them (sums in gs_count's 32-word layout).
gs_status build_oriented(gs_graph* g, cudaStream_t stream);
gs_status count_tri_oriented(const gs_graph* g, gs_workspace* ws, unsigned long long* h_sums,
                             unsigned long long* h_stats, int64_t* launches, cudaStream_t stream);
gs_status count_run(const gs_graph* gr, gs_workspace* ws, const int32_t* d_pairs, int64_t K,
                    uint32_t mask, bool check_dup, int64_t* d_per_edge, const int64_t* seg_off,
                    int64_t nseg, const Tuning& tu, CountBufs& b, cudaStream_t stream,
                    const char* what);
}  // namespace gs

// Byte-offset bump allocator inside one workspace slot.
struct Carve {
  char* base;
  size_t used;
  template <class T>
  T* take(int64_t count) {
    size_t bytes = ((size_t)(count > 0 ? count : 1) * sizeof(T) + 255) & ~(size_t)255;
    T* p = reinterpret_cast<T*>(base + used);
    used += bytes;
    return p;
  }
  template <class T>
  static size_t bytes_for(int64_t count) {
    return ((size_t)(count > 0 ? count : 1) * sizeof(T) + 255) & ~(size_t)255;
  }
};
