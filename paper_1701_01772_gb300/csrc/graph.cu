// Graph registration (validation, upper-edge index, hub index) and the
// uniform edge sampler of Algorithm 1.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace gs {

// Vertices below this degree never get bitmaps, matrix or table rows.
constexpr int64_t kHubMinDegree = 64;
// Vertices of at least this degree (and no bitmap) get a bucket directory.
constexpr int64_t kDirMinDegree = 16;
// Mid rows of the mid x big co-degree table start at this degree, and their
// build adds at most kMidWorkMax wedge increments (higher-degree rows first).
// On R-MAT scale 24 the cap leaves the budget binding: 637,384 rows x
// 65,250 columns at 96 GiB (the 1% 4-node estimate in 1.02 s, against
// 2.08 s with 234,019 x 16,317 under a cap of 1.6e11 and 20 GiB).
constexpr int64_t kMidMinDegree = 2;
#ifndef GS_MID_WORK_MAX
#define GS_MID_WORK_MAX 640000000000ull
#endif
constexpr unsigned long long kMidWorkMax = GS_MID_WORK_MAX;

// ------------------------------------------------------------- validation
// One warp per row (grid-stride). Checks the simple-graph conditions of
// Sec. 2.1: ids in range, strictly increasing lists (sorted, no repeats),
// no self-loops, and symmetry (u lists v => v lists u, by halving search).
__global__ void k_validate(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                           int64_t n, int64_t nnz, DevError* err) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    int64_t s = row_ptr[v], e = row_ptr[v + 1];
    if (s < 0 || e < s || e > nnz) {
      if (lane == 0) raise_error(err, GS_EINVAL, v);
      continue;
    }
    for (int64_t p = s + lane; p < e; p += 32) {
      int32_t x = col[p];
      if (x < 0 || x >= n) { raise_error(err, GS_EINVAL, p); continue; }
      if (x == v) { raise_error(err, GS_ESELFLOOP, p); continue; }
      if (p > s) {
        int32_t prev = col[p - 1];
        if (prev == x) raise_error(err, GS_EDUP, p);
        else if (prev > x) raise_error(err, GS_ENOTSORTED, p);
      }
      int64_t xs = row_ptr[x], xe = row_ptr[x + 1];
      if (xs < 0 || xe < xs || xe > nnz || !sorted_contains(col + xs, xe - xs, (int32_t)v))
        raise_error(err, GS_EASYM, p);
    }
  }
}

// Per row: index of the first neighbour greater than v, the count of such
// neighbours (canonical edges u < v owned by row u) and the maximum degree.
__global__ void k_upper(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                        int64_t n, int64_t* __restrict__ up_ptr, int64_t* __restrict__ up_cnt,
                        unsigned long long* max_deg) {
  unsigned long long local_max = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    int64_t s = row_ptr[v], e = row_ptr[v + 1];
    int64_t lo = s, len = e - s;
    while (len > 0) {  // lower bound of v + 1
      int64_t half = len >> 1;
      if (col[lo + half] <= v) { lo += half + 1; len -= half + 1; }
      else len = half;
    }
    up_ptr[v] = lo;
    up_cnt[v] = e - lo;
    unsigned long long d = (unsigned long long)(e - s);
    local_max = d > local_max ? d : local_max;
  }
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long y = __shfl_down_sync(0xffffffffu, local_max, o);
    local_max = y > local_max ? y : local_max;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(max_deg, local_max);
}

// Sum of the degrees of each vertex's neighbours (one warp per vertex).
__global__ void k_nbr_degsum(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                             int64_t n, int64_t* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    long long s = 0;
    for (int64_t p = row_ptr[v] + lane; p < row_ptr[v + 1]; p += 32) {
      int32_t w = col[p];
      s += row_ptr[w + 1] - row_ptr[w];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[v] = s;
  }
}

// ------------------------------------------------------------- hub index
// "Hubs" are the vertices of highest degree. Two structures are built once
// per graph and reused by every request:
//   bitmaps  for the top bm_count vertices, a bit per vertex id marking the
//            neighbours, so "x in N(h)" is one load instead of a search;
//   table    for the top tb_count vertices, c(a, b) = |N(a) cap N(b)| for
//            every pair of table hubs (upper triangle a < b by slot);
//   mid x big  c(a, b) for the next md_count vertices a by degree (down to
//            kMidMinDegree) against the top bg_count table vertices b, which
//            answers most co-degree queries between a sampled edge's
//            high-degree end and a low-degree neighbour.
// Slots are assigned in increasing vertex id among vertices whose degree is
// at least a threshold, so the index is deterministic.

__global__ void k_count_deg_ge(const int64_t* __restrict__ row_ptr, int64_t n, int64_t d,
                               unsigned long long* cnt) {
  unsigned c = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    c += (row_ptr[v + 1] - row_ptr[v]) >= d;
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, (unsigned long long)c);
}

__global__ void k_flag_deg_ge(const int64_t* __restrict__ row_ptr, int64_t n, int64_t d,
                              int64_t* __restrict__ flag) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    flag[v] = (row_ptr[v + 1] - row_ptr[v]) >= d;
}

// slot[v] = rank of v among flagged vertices, -1 otherwise; hubs[slot] = v.
__global__ void k_assign_slots(const int64_t* __restrict__ flag_scan, const int64_t* __restrict__ row_ptr,
                               int64_t n, int64_t d, int32_t* __restrict__ slot,
                               int32_t* __restrict__ hubs) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    bool f = (row_ptr[v + 1] - row_ptr[v]) >= d;
    int64_t s = flag_scan[v];
    slot[v] = f ? (int32_t)s : -1;
    if (f) hubs[s] = (int32_t)v;
  }
}

// Bitmap rows: bit x of hub h's row is set iff x in N(h). One block per hub.
__global__ void k_hub_bitmaps(const int64_t* __restrict__ row_ptr,
                              const int32_t* __restrict__ col, const int32_t* __restrict__ hubs,
                              int64_t count, int64_t words, uint32_t* __restrict__ bits) {
  for (int64_t h = blockIdx.x; h < count; h += gridDim.x) {
    int32_t v = hubs[h];
    uint32_t* row = bits + h * words;
    for (int64_t p = row_ptr[v] + threadIdx.x; p < row_ptr[v + 1]; p += blockDim.x) {
      int32_t x = col[p];
      atomicOr(row + (x >> 5), 1u << (x & 31));
    }
  }
}

// Hub-pair bit matrix: bit s2 of row s1 set iff table hubs s1 and s2 are
// adjacent. One block per table hub.
__global__ void k_hub_matrix(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                             const int32_t* __restrict__ slot, const int32_t* __restrict__ hubs,
                             int64_t count, int64_t words, uint32_t* __restrict__ bits) {
  for (int64_t h = blockIdx.x; h < count; h += gridDim.x) {
    int32_t v = hubs[h];
    uint32_t* row = bits + h * words;
    for (int64_t p = row_ptr[v] + threadIdx.x; p < row_ptr[v + 1]; p += blockDim.x) {
      int32_t s = __ldg(slot + col[p]);
      if (s >= 0) atomicOr(row + (s >> 5), 1u << (s & 31));
    }
  }
}

// col_hm[p] = matrix slot of col[p] (-1 if none): stored beside the
// adjacency so a membership test gets the slot with the element.
__global__ void k_col_slots(const int32_t* __restrict__ col, int64_t nnz,
                            const int32_t* __restrict__ slot, int16_t* __restrict__ col_hm) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
       p += (int64_t)gridDim.x * blockDim.x)
    col_hm[p] = (int16_t)__ldg(slot + col[p]);
}

// Per vertex: matrix neighbours (mn) and neighbours above v without a
// matrix slot (nm). One warp per vertex; counts first, then the lists in
// adjacency order at the scanned offsets.
__global__ void k_rest_lists(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                             const int16_t* __restrict__ col_hm, int64_t n,
                             int64_t* __restrict__ mn_cnt, int64_t* __restrict__ nm_cnt,
                             const int64_t* __restrict__ mn_off, const int64_t* __restrict__ nm_off,
                             int16_t* __restrict__ mn_slot, int32_t* __restrict__ nm_col) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    int64_t am = mn_off != nullptr ? mn_off[v] : 0, an = nm_off != nullptr ? nm_off[v] : 0;
    unsigned cm = 0, cn = 0;
    for (int64_t p0 = row_ptr[v]; p0 < row_ptr[v + 1]; p0 += 32) {
      const int64_t p = p0 + lane;
      const bool in = p < row_ptr[v + 1];
      const int16_t s = in ? col_hm[p] : (int16_t)-1;
      const int32_t x = in ? col[p] : -1;
      const unsigned bm = __ballot_sync(0xffffffffu, in && s >= 0);
      const unsigned bn = __ballot_sync(0xffffffffu, in && s < 0 && x > (int32_t)v);
      const unsigned below = (1u << lane) - 1u;
      if (mn_off != nullptr) {
        if ((bm >> lane) & 1u) mn_slot[am + __popc(bm & below)] = s;
        if ((bn >> lane) & 1u) nm_col[an + __popc(bn & below)] = x;
      }
      am += __popc(bm);
      an += __popc(bn);
      cm += __popc(bm);
      cn += __popc(bn);
    }
    if (mn_off == nullptr && lane == 0) {
      mn_cnt[v] = cm;
      nm_cnt[v] = cn;
    }
  }
}

// col_tb[p] = table slot of col[p] (tb_slot encoding, mid rows included):
// stored beside the adjacency so the cost pass reads it with the element
// instead of gathering it per item before the table read.
__global__ void k_col_tb(const int32_t* __restrict__ col, int64_t nnz,
                         const int32_t* __restrict__ tb_slot, int32_t* __restrict__ col_tb) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
       p += (int64_t)gridDim.x * blockDim.x)
    col_tb[p] = __ldg(tb_slot + col[p]);
}

// Sets the adjacency bits of rows that have a dense block. One warp per row.
__global__ void k_dense_rows(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                             int64_t n, const int64_t* __restrict__ dm_row,
                             const int32_t* __restrict__ dm_first, uint32_t* __restrict__ bits) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    const int64_t r = dm_row[v];
    if (r < 0) continue;
    const int32_t f = dm_first[v];
    for (int64_t p = row_ptr[v] + lane; p < row_ptr[v + 1]; p += 32) {
      const int32_t lx = col[p] - f;
      atomicOr(bits + r + (lx >> 5), 1u << (lx & 31));
    }
  }
}

// Mid x big co-degrees, one table row at a time: c(w, b) for a mid vertex w
// (tb_slot[w] = -2 - row) and the bg_count big vertices b is the number of
// x in N(w) with b in N(x). A CTA holds the row's counters in shared memory
// (16 bits each, two per 32-bit word: a co-degree is below the mid vertex's
// degree < 65536, so no carry reaches the neighbouring counter), adds, for
// every x in N(w), one to the counter of each big neighbour of x (the
// 16-bit column slots of x's big neighbours, listed beforehand), and writes
// the finished row out. The whole CTA walks the concatenation of the
// big-neighbour lists of N(w) (kMidRowThreads entries at a time): warps
// take 32-position segments, one position per lane, so a hub in N(w) with
// thousands of big neighbours is spread over all warps.
#ifndef GS_BIG_MAX
#define GS_BIG_MAX 65536
#endif
constexpr int kBigMax = GS_BIG_MAX;
static_assert(kBigMax <= 65536, "column slots are stored in 16 bits");
constexpr int kBigMin = 1024;  // narrowest shape tried
constexpr int kMidRowThreads = 1024;

// Number of big neighbours of every vertex. One warp per vertex.
__global__ void k_big_count(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                            int64_t n, const int32_t* __restrict__ bg_slot,
                            int64_t* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += warps) {
    unsigned c = 0;
    for (int64_t p = row_ptr[x] + lane; p < row_ptr[x + 1]; p += 32) c += __ldg(bg_slot + col[p]) >= 0;
    c = __reduce_add_sync(0xffffffffu, c);
    if (lane == 0) cnt[x] = c;
  }
}

// Column slots of the big neighbours of every vertex, in adjacency order,
// at off[x]. One warp per vertex.
__global__ void k_big_fill(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                           int64_t n, const int32_t* __restrict__ bg_slot,
                           const int64_t* __restrict__ off, uint16_t* __restrict__ list) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += warps) {
    int64_t at = off[x];
    for (int64_t p0 = row_ptr[x]; p0 < row_ptr[x + 1]; p0 += 32) {
      const int64_t p = p0 + lane;
      const int32_t b = p < row_ptr[x + 1] ? __ldg(bg_slot + col[p]) : -1;
      const unsigned ball = __ballot_sync(0xffffffffu, b >= 0);
      if (b >= 0) list[at + __popc(ball & ((1u << lane) - 1u))] = (uint16_t)b;
      at += __popc(ball);
    }
  }
}

// Vertex of every mid row.
__global__ void k_mid_row_vertex(const int32_t* __restrict__ tb_slot, int64_t n,
                                 int32_t* __restrict__ rows_v) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = tb_slot[v];
    if (s < -1) rows_v[-2 - s] = (int32_t)v;
  }
}

__global__ void __launch_bounds__(kMidRowThreads, 1)
    k_mid_rows(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
               const int32_t* __restrict__ rows_v, int64_t rows,
               const int64_t* __restrict__ boff, const uint16_t* __restrict__ blist,
               int64_t bg_count, uint16_t* __restrict__ md,
               unsigned long long* __restrict__ counter) {
  extern __shared__ uint32_t acc[];  // (bg_count + 1) / 2 words
  // the current kMidRowThreads entries of N(w) that have big neighbours:
  // list offset and first position in the concatenation of their lists
  __shared__ int64_t sbo[kMidRowThreads];
  __shared__ int32_t sst[kMidRowThreads];
  __shared__ int32_t wn[kMidRowThreads / 32], wl[kMidRowThreads / 32];
  __shared__ int64_t cur;
  constexpr int kWarps = kMidRowThreads / 32;
  const int W = (int)((bg_count + 1) / 2);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) cur = (int64_t)atomicAdd(counter, 1ull);
    __syncthreads();  // the previous row has been written out
    const int64_t r = cur;
    if (r >= rows) break;
    for (int i = threadIdx.x; i < W; i += kMidRowThreads) acc[i] = 0u;
    const int32_t w = rows_v[r];
    const int64_t s = row_ptr[w], d = row_ptr[w + 1] - s;
    for (int64_t c0 = 0; c0 < d; c0 += kMidRowThreads) {
      int64_t bo = 0;
      int32_t len = 0;
      if (c0 + threadIdx.x < d) {
        const int32_t x = col[s + c0 + threadIdx.x];
        bo = boff[x];
        len = (int32_t)(boff[x + 1] - bo);
      }
      // block-wide exclusive scans of (len > 0) and len
      const unsigned nz = __ballot_sync(0xffffffffu, len > 0);
      int32_t incl = len;
#pragma unroll
      for (int k = 1; k < 32; k <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, incl, k);
        if (lane >= k) incl += y;
      }
      if (lane == 31) {
        wn[wid] = __popc(nz);
        wl[wid] = incl;
      }
      __syncthreads();
      int32_t bn = 0, bl = 0, cnt = 0, total = 0;
      for (int k = 0; k < kWarps; ++k) {
        if (k < wid) {
          bn += wn[k];
          bl += wl[k];
        }
        cnt += wn[k];
        total += wl[k];
      }
      if (len > 0) {
        const int at = bn + __popc(nz & ((1u << lane) - 1u));
        sbo[at] = bo;
        sst[at] = bl + incl - len;
      }
      __syncthreads();
      // 32-position segments of the concatenation, one per warp at a time;
      // a segment spans at most 32 entries (all non-empty)
      for (int32_t q0 = wid * 32; q0 < total; q0 += kMidRowThreads) {
        int k0 = 0;  // last entry starting at or before q0
        for (int step = kMidRowThreads / 2; step > 0; step >>= 1)
          if (k0 + step < cnt && sst[k0 + step] <= q0) k0 += step;
        const int32_t q = q0 + lane;
        int k = k0;  // last entry starting at or before q
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
          if (k + step < cnt && sst[k + step] <= q) k += step;
        if (q < total) {
          const uint32_t b = __ldg(blist + sbo[k] + (q - sst[k]));
          atomicAdd(acc + (b >> 1), 1u << (16 * (b & 1u)));
        }
      }
      __syncthreads();  // sbo, sst, wn and wl are reused by the next chunk
    }
    __syncthreads();
    const uint16_t* a16 = reinterpret_cast<const uint16_t*>(acc);
    uint16_t* out = md + r * bg_count;
    for (int64_t c = threadIdx.x; c < bg_count; c += kMidRowThreads) out[c] = a16[c];
  }
}

// Build work of the mid x big table for mid rows of degree [lo, hi) and big
// columns of degree >= big: sum over x of (mid neighbours) x (big
// neighbours). One warp per vertex.
__global__ void k_mid_big_work(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                               int64_t n, int64_t lo, int64_t hi, int64_t big,
                               unsigned long long* __restrict__ total) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  unsigned long long acc = 0;
  for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += warps) {
    unsigned m = 0, b = 0;
    for (int64_t p = row_ptr[x] + lane; p < row_ptr[x + 1]; p += 32) {
      const int32_t y = col[p];
      const int64_t d = __ldg(row_ptr + y + 1) - __ldg(row_ptr + y);
      m += d >= lo && d < hi;
      b += d >= big;
    }
    m = __reduce_add_sync(0xffffffffu, m);
    b = __reduce_add_sync(0xffffffffu, b);
    acc += (unsigned long long)m * b;
  }
  if (lane == 0 && acc) atomicAdd(total, acc);
}

// Pilot of the mid x big table's shape: for a deterministic spread of
// canonical edges (edge j * m / P for j < P), every 4-node item w of the
// edge (w in N(u) \ {v}, u the endpoint of smaller degree) queries the
// co-degree c(w, o), o = u for w in T, o = v otherwise, which costs
// min(d_w, d_o) membership tests unless a table answers it. Items with
// exactly one table vertex among (w, o) are recorded as (degree of the
// table vertex, degree of the other, cost); the cost of items with none
// is added to rest[0]. One warp per pilot edge.
struct PilotItem {
  int32_t d_tab, d_other, cost, pad;
};

__global__ void k_md_pilot(DevGraph g, const int32_t* __restrict__ tb_slot,
                           const int64_t* __restrict__ edge_off, int64_t P, int64_t cap,
                           PilotItem* __restrict__ items, unsigned long long* __restrict__ count,
                           unsigned long long* __restrict__ rest) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t m = g.nnz / 2;
  unsigned long long none = 0;
  for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < P; j += warps) {
    const int64_t i = (int64_t)((__int128)j * m / P);
    int64_t lo = 0, len = g.n;  // row owning canonical edge i
    while (len > 1) {
      const int64_t half = len >> 1;
      lo = (edge_off[lo + half] <= i) ? lo + half : lo;
      len -= half;
    }
    const int32_t x = (int32_t)lo, y = g.col[g.up_ptr[lo] + (i - edge_off[lo])];
    const int64_t dx = g.row_ptr[x + 1] - g.row_ptr[x], dy = g.row_ptr[y + 1] - g.row_ptr[y];
    const bool xs = dx < dy || (dx == dy && x < y);
    const int32_t u = xs ? x : y, v = xs ? y : x;
    const int64_t bu = g.row_ptr[u], du = xs ? dx : dy, bv = g.row_ptr[v], dv = xs ? dy : dx;
    for (int64_t p = lane; p < du; p += 32) {
      const int32_t w = g.col[bu + p];
      if (w == v) continue;
      const bool in_t = adj_contains(g, v, bv, dv, w);
      const int32_t o = in_t ? u : v;
      const int64_t dw = g.row_ptr[w + 1] - g.row_ptr[w], dob = in_t ? du : dv;
      const int64_t cost = dw < dob ? dw : dob;
      const bool tw = tb_slot[w] >= 0, to = tb_slot[o] >= 0;
      if (tw && to) continue;
      if (!tw && !to) {
        none += (unsigned long long)cost;
        continue;
      }
      const unsigned long long at = atomicAdd(count, 1ull);
      if ((int64_t)at < cap)
        items[at] = PilotItem{(int32_t)(tw ? dw : dob), (int32_t)(tw ? dob : dw),
                              (int32_t)(cost < INT32_MAX ? cost : INT32_MAX), 0};
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) none += __shfl_xor_sync(0xffffffffu, none, o);
  if (lane == 0 && none) atomicAdd(rest, none);
}

// Marks mid vertices (lo <= degree < hi, no table slot) and big vertices
// (table vertices of degree >= big).
__global__ void k_flag_mid(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ tb_slot,
                           int64_t n, int64_t lo, int64_t hi, int64_t* __restrict__ flag) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = row_ptr[v + 1] - row_ptr[v];
    flag[v] = d >= lo && d < hi && tb_slot[v] < 0;
  }
}

__global__ void k_set_mid_rows(const int64_t* __restrict__ flag_scan,
                               const int64_t* __restrict__ row_ptr, int64_t n, int64_t lo,
                               int64_t hi, int32_t* __restrict__ tb_slot) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = row_ptr[v + 1] - row_ptr[v];
    if (d >= lo && d < hi && tb_slot[v] < 0) tb_slot[v] = (int32_t)(-2 - flag_scan[v]);
  }
}

// Directory entries of v: 2^dir_log2(d) + 1 when v has degree >= d_min and no
// bitmap, else 0.
__device__ __forceinline__ int64_t dir_entries(const int64_t* __restrict__ row_ptr,
                                               const int32_t* __restrict__ bm_slot, int64_t v,
                                               int64_t d_min, int id_bits) {
  const int64_t d = row_ptr[v + 1] - row_ptr[v];
  if (d < d_min || d < 2) return 0;
  if (bm_slot != nullptr && bm_slot[v] >= 0) return 0;
  return ((int64_t)1 << dir_log2(d, id_bits)) + 1;
}

__global__ void k_dir_entries_total(const int64_t* __restrict__ row_ptr,
                                    const int32_t* __restrict__ bm_slot, int64_t n, int64_t d_min,
                                    int id_bits, unsigned long long* total) {
  unsigned long long c = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    c += (unsigned long long)dir_entries(row_ptr, bm_slot, v, d_min, id_bits);
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(total, c);
}

__global__ void k_dir_sizes(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ bm_slot,
                            int64_t n, int64_t d_min, int id_bits, int64_t* __restrict__ size) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    size[v] = dir_entries(row_ptr, bm_slot, v, d_min, id_bits);
}

__global__ void k_dir_at(const int64_t* __restrict__ size_scan, const int64_t* __restrict__ row_ptr,
                         const int32_t* __restrict__ bm_slot, int64_t n, int64_t d_min, int id_bits,
                         int64_t* __restrict__ dir_at) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    dir_at[v] = dir_entries(row_ptr, bm_slot, v, d_min, id_bits) > 0 ? size_scan[v] : -1;
}

// One warp per vertex with a directory: entry b is the offset in N(v) of the
// first neighbour whose bucket x >> s is at least b (entry 2^k is deg v).
// Entries b with bucket(N(v)[i-1]) < b <= bucket(N(v)[i]) are written by
// the lane holding i, so every entry is written exactly once.
__global__ void k_dir_fill(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                           const int64_t* __restrict__ dir_at, int64_t n, int id_bits,
                           uint32_t* __restrict__ dir) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    const int64_t at = dir_at[v];
    if (at < 0) continue;
    const int64_t s = row_ptr[v], d = row_ptr[v + 1] - s;
    const int kb = dir_log2(d, id_bits);
    const int sh = id_bits - kb;
    const int64_t nb = (int64_t)1 << kb;
    uint32_t* D = dir + at;
    for (int64_t i = lane; i < d; i += 32) {
      const int64_t b = col[s + i] >> sh;
      const int64_t bp = i > 0 ? (int64_t)(col[s + i - 1] >> sh) : -1;
      for (int64_t bb = bp + 1; bb <= b; ++bb) D[bb] = (uint32_t)i;
    }
    const int64_t last = col[s + d - 1] >> sh;
    for (int64_t bb = last + 1 + lane; bb <= nb; bb += 32) D[bb] = (uint32_t)d;
  }
}

__global__ void k_count_dirs(const int64_t* __restrict__ dir_at, int64_t n,
                             unsigned long long* cnt) {
  unsigned c = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    c += dir_at[v] >= 0;
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, (unsigned long long)c);
}

// Number of table hubs among the neighbours of each vertex.
__global__ void k_hub_nbr_count(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                const int32_t* __restrict__ slot, int64_t n,
                                int64_t* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += warps) {
    unsigned c = 0;
    for (int64_t p = row_ptr[x] + lane; p < row_ptr[x + 1]; p += 32) c += __ldg(slot + col[p]) >= 0;
    c = __reduce_add_sync(0xffffffffu, c);
    if (lane == 0) cnt[x] = c;
  }
}

// Compacted table-hub slots of each vertex's neighbours, in list order
// (hence increasing slot).
__global__ void k_hub_nbr_fill(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                               const int32_t* __restrict__ slot, int64_t n,
                               const int64_t* __restrict__ off, int32_t* __restrict__ lists) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += warps) {
    int64_t pos = off[x];
    for (int64_t p0 = row_ptr[x]; p0 < row_ptr[x + 1]; p0 += 32) {
      int64_t p = p0 + lane;
      int32_t s = p < row_ptr[x + 1] ? __ldg(slot + col[p]) : -1;
      unsigned b = __ballot_sync(0xffffffffu, s >= 0);
      if (s >= 0) {
        int64_t at = pos + __popc(b & ((1u << lane) - 1u));
        lists[at] = s;
      }
      pos += __popc(b);
    }
  }
}

// flag[s] = 1 when the table hub with slot s has degree >= 65,536.
__global__ void k_giant_flags(const int64_t* __restrict__ row_ptr,
                              const int32_t* __restrict__ tb_slot, int64_t n,
                              int64_t* __restrict__ flag) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t sl = tb_slot[v];
    if (sl >= 0) flag[sl] = (row_ptr[v + 1] - row_ptr[v]) >= 65536;
  }
}

// giant[s] = index of slot s among the giants (exclusive scan of the flags),
// or -1.
__global__ void k_giant_index(const int64_t* __restrict__ flag_scan, int64_t count,
                              int32_t* __restrict__ giant) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < count;
       s += (int64_t)gridDim.x * blockDim.x)
    giant[s] = flag_scan[s + 1] > flag_scan[s] ? (int32_t)flag_scan[s] : -1;
}

// Marks the 16-bit entries of giant pairs 0xFFFF (answered by the giant
// table). One thread per slot a; only giant rows do work.
// Co-degree table among the table vertices, one row at a time: row a holds
// c(a, b) for b > a (contiguous in tb_index order), the number of x in N(a)
// with b in N(x). A CTA accumulates the row in shared memory (16-bit
// counters, two per word) from the table-neighbour lists of a's neighbours
// -- each sorted by slot, so the part after a is a suffix found by a
// halving search -- walked as one concatenation in 32-position segments per
// warp, and writes the row once. Pairs of two giants (degree >= 65,536,
// whose co-degree may not fit 16 bits) go to the 32-bit giant table by
// global atomics instead (marked 0xFFFF afterwards by k_mark_giant_pairs).
__global__ void __launch_bounds__(kMidRowThreads, 1)
    k_table_rows(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                 const int32_t* __restrict__ tb_vertex, int64_t count,
                 const int64_t* __restrict__ loff, const int32_t* __restrict__ lists,
                 const int32_t* __restrict__ giant, int64_t giants,
                 uint32_t* __restrict__ giant_codeg, uint16_t* __restrict__ tb,
                 unsigned long long* __restrict__ counter) {
  extern __shared__ uint32_t acc[];  // count / 2 words (row 0 is the longest)
  __shared__ int64_t sbo[kMidRowThreads];
  __shared__ int32_t sst[kMidRowThreads];
  __shared__ int32_t wn[kMidRowThreads / 32], wl[kMidRowThreads / 32];
  __shared__ int64_t cur;
  constexpr int kWarps = kMidRowThreads / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) cur = (int64_t)atomicAdd(counter, 1ull);
    __syncthreads();  // the previous row has been written out
    const int64_t a = cur;
    if (a >= count - 1) break;  // the last row is empty
    const int64_t R = count - a - 1;
    const int W = (int)((R + 1) / 2);
    for (int i = threadIdx.x; i < W; i += kMidRowThreads) acc[i] = 0u;
    const int32_t va = tb_vertex[a];
    const int32_t ga = giant != nullptr ? giant[a] : -1;
    const int64_t s = row_ptr[va], d = row_ptr[va + 1] - s;
    for (int64_t c0 = 0; c0 < d; c0 += kMidRowThreads) {
      int64_t bo = 0;
      int32_t len = 0;
      if (c0 + threadIdx.x < d) {
        const int32_t x = col[s + c0 + threadIdx.x];
        int64_t lo = loff[x];
        const int64_t hi = loff[x + 1];
        int64_t n = hi - lo;  // first entry above a (a itself is in the list)
        while (n > 0) {
          const int64_t h = n >> 1;
          if (__ldg(lists + lo + h) <= a) {
            lo += h + 1;
            n -= h + 1;
          } else {
            n = h;
          }
        }
        bo = lo;
        len = (int32_t)(hi - lo);
      }
      const unsigned nz = __ballot_sync(0xffffffffu, len > 0);
      int32_t incl = len;
#pragma unroll
      for (int k = 1; k < 32; k <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, incl, k);
        if (lane >= k) incl += y;
      }
      if (lane == 31) {
        wn[wid] = __popc(nz);
        wl[wid] = incl;
      }
      __syncthreads();
      int32_t bn = 0, bl = 0, cnt = 0, total = 0;
      for (int k = 0; k < kWarps; ++k) {
        if (k < wid) {
          bn += wn[k];
          bl += wl[k];
        }
        cnt += wn[k];
        total += wl[k];
      }
      if (len > 0) {
        const int at = bn + __popc(nz & ((1u << lane) - 1u));
        sbo[at] = bo;
        sst[at] = bl + incl - len;
      }
      __syncthreads();
      for (int32_t q0 = wid * 32; q0 < total; q0 += kMidRowThreads) {
        int k0 = 0;
        for (int step = kMidRowThreads / 2; step > 0; step >>= 1)
          if (k0 + step < cnt && sst[k0 + step] <= q0) k0 += step;
        const int32_t q = q0 + lane;
        int k = k0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
          if (k + step < cnt && sst[k + step] <= q) k += step;
        if (q < total) {
          const int32_t b = __ldg(lists + sbo[k] + (q - sst[k]));
          const int32_t gb = ga >= 0 ? __ldg(giant + b) : -1;
          if (gb >= 0) {
            atomicAdd(giant_codeg + (int64_t)ga * giants + gb, 1u);
          } else {
            const uint32_t c = (uint32_t)(b - a - 1);
            atomicAdd(acc + (c >> 1), 1u << (16 * (c & 1u)));
          }
        }
      }
      __syncthreads();  // sbo, sst, wn and wl are reused by the next chunk
    }
    __syncthreads();
    const uint16_t* a16 = reinterpret_cast<const uint16_t*>(acc);
    uint16_t* out = tb + tb_index(a, a + 1, count);
    for (int64_t c = threadIdx.x; c < R; c += kMidRowThreads) out[c] = a16[c];
  }
}

__global__ void k_mark_giant_pairs(const int32_t* __restrict__ giant, int64_t count,
                                   uint32_t* __restrict__ words) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < count;
       a += (int64_t)gridDim.x * blockDim.x) {
    if (giant[a] < 0) continue;
    const int64_t base = a * (2 * count - a - 1) / 2 - a - 1;
    for (int64_t b = a + 1; b < count; ++b)
      if (giant[b] >= 0) {
        const int64_t at = base + b;
        atomicOr(words + (at >> 1), 0xFFFFu << (16 * (int)(at & 1)));
      }
  }
}

}  // namespace gs

// =================================================================== C ABI
using namespace gs;

static gs_status read_error(DevError* d_err, cudaStream_t stream, const char* what) {
  DevError h;
  GS_CUDA(cudaMemcpyAsync(&h, d_err, sizeof(h), cudaMemcpyDeviceToHost, stream));
  GS_CUDA(cudaStreamSynchronize(stream));
  if (h.code != 0) {
    const char* kind = "invalid argument";
    switch (h.code) {
      case GS_ENOTSORTED: kind = "adjacency list not sorted"; break;
      case GS_ESELFLOOP: kind = "self-loop"; break;
      case GS_EDUP: kind = "repeated neighbour"; break;
      case GS_EASYM: kind = "asymmetric adjacency"; break;
      case GS_EEDGE: kind = "sampled pair is not an edge"; break;
      case GS_EDUPSAMPLE: kind = "edge sampled twice"; break;
      default: break;
    }
    set_error("%s: %s (element %lld)", what, kind, (long long)h.index);
    return h.code;
  }
  return GS_OK;
}

// Smallest degree threshold d >= min_deg with at most `cap` vertices of
// degree >= d (binary search with a device count per probe).
static gs_status hub_threshold(const gs_graph* g, int64_t cap, int64_t min_deg,
                               unsigned long long* d_cnt, cudaStream_t stream, int64_t* d_out,
                               int64_t* count_out) {
  auto count_ge = [&](int64_t d, int64_t* c) -> gs_status {
    GS_CUDA(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), stream));
    k_count_deg_ge<<<grid_for(g->dev.n, 256, 8), 256, 0, stream>>>(g->dev.row_ptr, g->dev.n, d,
                                                                   d_cnt);
    unsigned long long h = 0;
    GS_CUDA(cudaMemcpyAsync(&h, d_cnt, sizeof(h), cudaMemcpyDeviceToHost, stream));
    GS_CUDA(cudaStreamSynchronize(stream));
    *c = (int64_t)h;
    return GS_OK;
  };
  int64_t lo = min_deg, hi = g->max_degree + 1;  // count(hi) = 0 <= cap
  int64_t c = 0;
  GS_TRY(count_ge(lo, &c));
  if (c <= cap) {
    *d_out = lo;
    *count_out = c;
    return GS_OK;
  }
  while (hi - lo > 1) {  // count(lo) > cap >= count(hi)
    int64_t mid = lo + (hi - lo) / 2;
    GS_TRY(count_ge(mid, &c));
    if (c <= cap) hi = mid; else lo = mid;
  }
  GS_TRY(count_ge(hi, &c));
  *d_out = hi;
  *count_out = c;
  return GS_OK;
}

// Builds, within `budget` bytes (0 = 96 GiB): bitmaps (up to 1/8 of the
// budget), the hub-pair matrix (up to 1/8, at most kHubMatrixMax vertices),
// bucket directories (up to 1/16), the 16-bit co-degree table (most of the
// rest, at most 65535 vertices), the mid x big table and, if room is left,
// the table slot of every adjacency entry.
static gs_status build_hub_index(gs_graph* g, uint64_t budget, cudaStream_t stream) {
  const int64_t n = g->dev.n;
  if (budget == 0) budget = (uint64_t)96 << 30;
  if (n == 0 || g->max_degree < kHubMinDegree) return GS_OK;
  const int64_t words = (n + 31) / 32;
  // bitmaps and the matrix get up to 1/8 of the budget each, the table the rest
  const double share = (double)budget / 8.0;
  const int64_t bm_cap = (int64_t)(share / ((double)words * 4.0));
  int64_t hm_cap = (int64_t)sqrt(share * 8.0);
  if (hm_cap > kHubMatrixMax) hm_cap = kHubMatrixMax;
  unsigned long long* d_cnt = nullptr;
  int64_t* flag = nullptr;
  int64_t* tmp = nullptr;
  GS_CUDA(cudaMalloc(&d_cnt, sizeof(unsigned long long)));
  struct Free {
    void* p[3];
    ~Free() { for (void* x : p) cudaFree(x); }
  } guard{{nullptr, nullptr, nullptr}};
  guard.p[0] = d_cnt;
  if (cudaMalloc(&flag, sizeof(int64_t) * (size_t)(n + 1)) != cudaSuccess ||
      cudaMalloc(&tmp, sizeof(int64_t) * (size_t)scan_tmp_elems(n)) != cudaSuccess) {
    cudaFree(flag);
    set_error("hub index: out of device memory");
    return GS_ENOMEM;
  }
  guard.p[1] = flag;
  guard.p[2] = tmp;
  auto assign = [&](int64_t d, int32_t** slot, int32_t** hubs, int64_t count) -> gs_status {
    GS_CUDA(cudaMalloc(slot, sizeof(int32_t) * (size_t)n));
    GS_CUDA(cudaMalloc(hubs, sizeof(int32_t) * (size_t)(count > 0 ? count : 1)));
    k_flag_deg_ge<<<grid_for(n, 256, 8), 256, 0, stream>>>(g->dev.row_ptr, n, d, flag);
    GS_TRY(exclusive_scan_i64(flag, flag, n, tmp, stream));
    k_assign_slots<<<grid_for(n, 256, 8), 256, 0, stream>>>(flag, g->dev.row_ptr, n, d, *slot,
                                                            *hubs);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
  };
  // ---- bitmaps
  int64_t d_bm = 0, n_bm = 0;
  if (bm_cap > 0) {
    GS_TRY(hub_threshold(g, bm_cap, kHubMinDegree, d_cnt, stream, &d_bm, &n_bm));
    if (n_bm > 0) {
      int32_t* hubs = nullptr;
      GS_TRY(assign(d_bm, &g->bm_slot, &hubs, n_bm));
      cudaError_t e = cudaMalloc(&g->bm_bits, sizeof(uint32_t) * (size_t)(words * n_bm));
      if (e != cudaSuccess) {
        cudaFree(hubs);
        return cuda_fail(e, "hub bitmaps", __FILE__, __LINE__);
      }
      GS_CUDA(cudaMemsetAsync(g->bm_bits, 0, sizeof(uint32_t) * (size_t)(words * n_bm), stream));
      k_hub_bitmaps<<<grid_for(n_bm * 256, 256, 8), 256, 0, stream>>>(
          g->dev.row_ptr, g->dev.col, hubs, n_bm, words, g->bm_bits);
      GS_CUDA(cudaStreamSynchronize(stream));
      cudaFree(hubs);
      g->dev.bm_slot = g->bm_slot;
      g->dev.bm_bits = g->bm_bits;
      g->dev.bm_words = words;
      g->dev.bm_count = n_bm;
    }
  }
  // ---- bucket directories for the vertices without bitmaps, highest degree
  // first, in up to 1/16 of the budget
  int id_bits = 0;
  while (((int64_t)1 << id_bits) < n) ++id_bits;
  g->dev.id_bits = id_bits;
  double dir_bytes = 0.0;
  {
    // entry offsets must fit 31 bits (a membership test carries them as int32)
    double dir_cap = (double)budget / 16.0;
    if (dir_cap > 4.0 * (double)INT32_MAX) dir_cap = 4.0 * (double)INT32_MAX;
    auto entries_ge = [&](int64_t d, int64_t* c) -> gs_status {
      GS_CUDA(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), stream));
      k_dir_entries_total<<<grid_for(n, 256, 8), 256, 0, stream>>>(g->dev.row_ptr, g->bm_slot, n,
                                                                   d, id_bits, d_cnt);
      unsigned long long h = 0;
      GS_CUDA(cudaMemcpyAsync(&h, d_cnt, sizeof(h), cudaMemcpyDeviceToHost, stream));
      GS_CUDA(cudaStreamSynchronize(stream));
      *c = (int64_t)h;
      return GS_OK;
    };
    // lowest threshold >= kDirMinDegree whose directories fit
    int64_t lo = kDirMinDegree, hi = g->max_degree + 1, c = 0;
    GS_TRY(entries_ge(lo, &c));
    if ((double)c * 4.0 > dir_cap) {
      while (hi - lo > 1) {  // entries(lo) too many, entries(hi) = 0 fits
        const int64_t mid = lo + (hi - lo) / 2;
        GS_TRY(entries_ge(mid, &c));
        if ((double)c * 4.0 <= dir_cap) hi = mid; else lo = mid;
      }
      lo = hi;
      GS_TRY(entries_ge(lo, &c));
    }
    if (c > 0) {
      GS_CUDA(cudaMalloc(&g->dir_at, sizeof(int64_t) * (size_t)n));
      k_dir_sizes<<<grid_for(n, 256, 8), 256, 0, stream>>>(g->dev.row_ptr, g->bm_slot, n, lo,
                                                           id_bits, flag);
      GS_TRY(exclusive_scan_i64(flag, flag, n, tmp, stream));
      k_dir_at<<<grid_for(n, 256, 8), 256, 0, stream>>>(flag, g->dev.row_ptr, g->bm_slot, n, lo,
                                                        id_bits, g->dir_at);
      cudaError_t de = cudaMalloc(&g->dir, sizeof(uint32_t) * (size_t)c);
      if (de != cudaSuccess) return cuda_fail(de, "adjacency directories", __FILE__, __LINE__);
      k_dir_fill<<<grid_for(n * 32, 256, 8), 256, 0, stream>>>(g->dev.row_ptr, g->dev.col,
                                                               g->dir_at, n, id_bits, g->dir);
      GS_CUDA(cudaStreamSynchronize(stream));
      g->dev.dir_at = g->dir_at;
      g->dev.dir = g->dir;
      GS_CUDA(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), stream));
      k_count_dirs<<<grid_for(n, 256, 8), 256, 0, stream>>>(g->dir_at, n, d_cnt);
      unsigned long long cnt = 0;
      GS_CUDA(cudaMemcpyAsync(&cnt, d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, stream));
      GS_CUDA(cudaStreamSynchronize(stream));
      g->dev.dir_count = (int64_t)cnt;
      dir_bytes = (double)c * 4.0;
    }
  }
  // ---- hub-pair bit matrix over the top vertices (kept small: it must stay
  // in L2 to pay off)
  int64_t d_hm = 0, n_hm = 0;
  double rest_bytes = 0.0;  // col_hm and the lists built with the matrix
  if (hm_cap > 1) GS_TRY(hub_threshold(g, hm_cap, kHubMinDegree, d_cnt, stream, &d_hm, &n_hm));
  if (n_hm > 1) {
    int32_t* hubs = nullptr;
    GS_TRY(assign(d_hm, &g->hm_slot, &hubs, n_hm));
    // rows padded to a multiple of 4 words (128 bits) so that dense clique
    // counting can read a row and a T mask with aligned 16-byte loads
    const int64_t hm_words = (n_hm + 127) / 128 * 4;
    cudaError_t he = cudaMalloc(&g->hm_bits, sizeof(uint32_t) * (size_t)(hm_words * n_hm));
    if (he != cudaSuccess) {
      cudaFree(hubs);
      return cuda_fail(he, "hub matrix", __FILE__, __LINE__);
    }
    GS_CUDA(cudaMemsetAsync(g->hm_bits, 0, sizeof(uint32_t) * (size_t)(hm_words * n_hm), stream));
    k_hub_matrix<<<grid_for(n_hm * 256, 256, 8), 256, 0, stream>>>(
        g->dev.row_ptr, g->dev.col, g->hm_slot, hubs, n_hm, hm_words, g->hm_bits);
    g->hm_vertex = hubs;  // slot -> vertex
    GS_CUDA(cudaMalloc(&g->col_hm, sizeof(int16_t) * (size_t)(g->dev.nnz > 0 ? g->dev.nnz : 1)));
    if (g->dev.nnz > 0)
      k_col_slots<<<grid_for(g->dev.nnz, 256, 8), 256, 0, stream>>>(g->dev.col, g->dev.nnz,
                                                                    g->hm_slot, g->col_hm);
    // matrix-neighbour and non-matrix-above lists (work of dense edges'
    // members without a dense slot)
    GS_CUDA(cudaMalloc(&g->mn_ptr, sizeof(int64_t) * (size_t)(n + 1)));
    GS_CUDA(cudaMalloc(&g->nm_ptr, sizeof(int64_t) * (size_t)(n + 1)));
    k_rest_lists<<<grid_for(n * 32, 256, 8), 256, 0, stream>>>(
        g->dev.row_ptr, g->dev.col, g->col_hm, n, g->mn_ptr, g->nm_ptr, nullptr, nullptr, nullptr,
        nullptr);
    GS_TRY(exclusive_scan_i64(g->mn_ptr, g->mn_ptr, n, tmp, stream));
    GS_TRY(exclusive_scan_i64(g->nm_ptr, g->nm_ptr, n, tmp, stream));
    int64_t tot[2] = {0, 0};
    GS_CUDA(cudaMemcpyAsync(tot, g->mn_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
    GS_CUDA(cudaMemcpyAsync(tot + 1, g->nm_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost,
                            stream));
    GS_CUDA(cudaStreamSynchronize(stream));
    GS_CUDA(cudaMalloc(&g->mn_slot, sizeof(int16_t) * (size_t)(tot[0] > 0 ? tot[0] : 1)));
    GS_CUDA(cudaMalloc(&g->nm_col, sizeof(int32_t) * (size_t)(tot[1] > 0 ? tot[1] : 1)));
    k_rest_lists<<<grid_for(n * 32, 256, 8), 256, 0, stream>>>(
        g->dev.row_ptr, g->dev.col, g->col_hm, n, nullptr, nullptr, g->mn_ptr, g->nm_ptr,
        g->mn_slot, g->nm_col);
    rest_bytes = 16.0 * (double)(n + 1) + 2.0 * (double)tot[0] + 4.0 * (double)tot[1] +
                 2.0 * (double)g->dev.nnz;
    GS_CUDA(cudaStreamSynchronize(stream));
    g->dev.mn_ptr = g->mn_ptr;
    g->dev.mn_slot = g->mn_slot;
    g->dev.nm_ptr = g->nm_ptr;
    g->dev.nm_col = g->nm_col;
    g->dev.hm_vertex = g->hm_vertex;
    g->dev.col_hm = g->col_hm;
    g->dev.hm_slot = g->hm_slot;
    g->dev.hm_bits = g->hm_bits;
    g->dev.hm_words = hm_words;
    g->dev.hm_count = n_hm;
  }
  // ---- co-degree table
  const double tb_bytes =
      (double)budget - share - (double)hm_cap * (double)hm_cap / 8.0 - dir_bytes;
  // n (n - 1) / 2 entries of 2 bytes
  int64_t tb_cap = tb_bytes > 0 ? (int64_t)sqrt(tb_bytes) : 0;
  if (tb_cap > 65535) tb_cap = 65535;
  int64_t d_tb = 0, n_tb = 0;
  if (tb_cap > 1) {
    GS_TRY(hub_threshold(g, tb_cap, kHubMinDegree, d_cnt, stream, &d_tb, &n_tb));
    if (n_tb > 1) {
      int32_t* hubs = nullptr;  // slot -> vertex, for the row build
      GS_TRY(assign(d_tb, &g->tb_slot, &hubs, n_tb));
      struct FreeHubs {
        int32_t* p;
        ~FreeHubs() { cudaFree(p); }
      } hubs_guard{hubs};
      const int64_t tb_words = (n_tb * (n_tb - 1) / 2 + 1) / 2;
      GS_CUDA(cudaMalloc(&g->tb_codeg, sizeof(uint32_t) * (size_t)tb_words));
      GS_CUDA(cudaMemsetAsync(g->tb_codeg, 0, sizeof(uint32_t) * (size_t)tb_words, stream));
      int64_t giants = 0;
      if (g->max_degree >= 65536) {
        // giant table hubs: slot -> index, and their 32-bit pair table
        GS_CUDA(cudaMemsetAsync(flag, 0, sizeof(int64_t) * (size_t)(n_tb + 1), stream));
        k_giant_flags<<<grid_for(n, 256, 8), 256, 0, stream>>>(g->dev.row_ptr, g->tb_slot, n,
                                                               flag);
        GS_TRY(exclusive_scan_i64(flag, flag, n_tb, tmp, stream));
        GS_CUDA(cudaMemcpyAsync(&giants, flag + n_tb, sizeof(int64_t), cudaMemcpyDeviceToHost,
                                stream));
        GS_CUDA(cudaStreamSynchronize(stream));
        if (giants > 0) {
          GS_CUDA(cudaMalloc(&g->tb_giant, sizeof(int32_t) * (size_t)n_tb));
          GS_CUDA(cudaMalloc(&g->tb_giant_codeg, sizeof(uint32_t) * (size_t)(giants * giants)));
          GS_CUDA(cudaMemsetAsync(g->tb_giant_codeg, 0,
                                  sizeof(uint32_t) * (size_t)(giants * giants), stream));
          k_giant_index<<<grid_for(n_tb, 256, 8), 256, 0, stream>>>(flag, n_tb, g->tb_giant);
        }
      }
      // per-vertex lists of table-hub neighbours
      k_hub_nbr_count<<<grid_for(n * 32, 256, 8), 256, 0, stream>>>(g->dev.row_ptr, g->dev.col,
                                                                    g->tb_slot, n, flag);
      GS_TRY(exclusive_scan_i64(flag, flag, n, tmp, stream));
      int64_t total = 0;
      GS_CUDA(cudaMemcpyAsync(&total, flag + n, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
      GS_CUDA(cudaStreamSynchronize(stream));
      int32_t* lists = nullptr;
      GS_CUDA(cudaMalloc(&lists, sizeof(int32_t) * (size_t)(total > 0 ? total : 1)));
      k_hub_nbr_fill<<<grid_for(n * 32, 256, 8), 256, 0, stream>>>(
          g->dev.row_ptr, g->dev.col, g->tb_slot, n, flag, lists);
      uint32_t* tb_w = reinterpret_cast<uint32_t*>(g->tb_codeg);
      const size_t row_smem = sizeof(uint32_t) * (size_t)(n_tb / 2 + 1);
      cudaError_t e = cudaFuncSetAttribute(k_table_rows,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)row_smem);
      if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), stream);
      if (e == cudaSuccess) {
        k_table_rows<<<sm_count(), kMidRowThreads, row_smem, stream>>>(
            g->dev.row_ptr, g->dev.col, hubs, n_tb, flag, lists, g->tb_giant, giants,
            g->tb_giant_codeg, g->tb_codeg, d_cnt);
        if (g->tb_giant != nullptr)
          k_mark_giant_pairs<<<grid_for(n_tb, 256, 8), 256, 0, stream>>>(g->tb_giant, n_tb, tb_w);
        e = cudaStreamSynchronize(stream);
      }
      cudaFree(lists);
      if (e != cudaSuccess) return cuda_fail(e, "co-degree table", __FILE__, __LINE__);
      g->dev.tb_slot = g->tb_slot;
      g->dev.tb_codeg = g->tb_codeg;
      g->dev.tb_count = n_tb;
      g->dev.tb_giant = g->tb_giant;
      g->dev.tb_giant_codeg = g->tb_giant_codeg;
      g->dev.tb_giants = giants;
    }
  }
  // ---- mid x big co-degrees: rows for the highest-degree vertices below
  // the table (degree >= kMidMinDegree), columns for the top 1024-65536
  // table vertices; whatever the budget has left
  double used = (double)n_bm * (double)words * 4.0 +
                (double)n_hm * (double)g->dev.hm_words * 4.0 + rest_bytes +
                (double)g->dev.tb_count * (double)g->dev.tb_count + dir_bytes;
  const int64_t d_hi = d_tb < 65536 ? d_tb : 65536;
  if (g->dev.tb_count > 1 && d_hi > kMidMinDegree && (double)budget > used) {
    // shape: columns = the top 1024 .. 65536 table vertices by degree, rows
    // = the highest-degree mid vertices that fit next to them in the budget
    // (and whose build stays within kMidWorkMax increments); the shape kept
    // leaves the fewest membership tests on a pilot of the graph's own edges
    // (measured miss cost of each shape)
    auto work_at = [&](int64_t lo, int64_t big, unsigned long long* w) -> gs_status {
      GS_CUDA(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), stream));
      k_mid_big_work<<<grid_for(n * 32, 256, 8), 256, 0, stream>>>(g->dev.row_ptr, g->dev.col, n,
                                                                   lo, d_hi, big, d_cnt);
      GS_CUDA(cudaMemcpyAsync(w, d_cnt, sizeof(*w), cudaMemcpyDeviceToHost, stream));
      GS_CUDA(cudaStreamSynchronize(stream));
      return GS_OK;
    };
    // pilot items
    constexpr int64_t kPilotEdges = 2048;
    constexpr int64_t kPilotCap = (int64_t)1 << 23;
    std::vector<PilotItem> pilot;
    {
      PilotItem* d_items = nullptr;
      unsigned long long* d_pc = nullptr;
      if (cudaMalloc(&d_items, sizeof(PilotItem) * (size_t)kPilotCap) == cudaSuccess &&
          cudaMalloc(&d_pc, 2 * sizeof(unsigned long long)) == cudaSuccess) {
        cudaMemsetAsync(d_pc, 0, 2 * sizeof(unsigned long long), stream);
        const int64_t P = g->m < kPilotEdges ? g->m : kPilotEdges;
        k_md_pilot<<<grid_for(P * 32, 256, 8), 256, 0, stream>>>(
            g->dev, g->tb_slot, g->edge_off, P, kPilotCap, d_items, d_pc, d_pc + 1);
        unsigned long long hc[2] = {0, 0};
        cudaMemcpyAsync(hc, d_pc, sizeof(hc), cudaMemcpyDeviceToHost, stream);
        cudaError_t pe = cudaStreamSynchronize(stream);
        if (pe == cudaSuccess) {
          const int64_t cnt = (int64_t)hc[0] < kPilotCap ? (int64_t)hc[0] : kPilotCap;
          pilot.resize((size_t)cnt);
          if (cnt > 0)
            pe = cudaMemcpy(pilot.data(), d_items, sizeof(PilotItem) * (size_t)cnt,
                            cudaMemcpyDeviceToHost);
        }
        if (pe != cudaSuccess) {
          cudaFree(d_items);
          cudaFree(d_pc);
          return cuda_fail(pe, "mid x big pilot", __FILE__, __LINE__);
        }
      }
      cudaFree(d_items);
      cudaFree(d_pc);
      cudaGetLastError();  // an allocation that failed only skips the pilot
    }
    int64_t d_bg = 0, n_bg = 0, d_md = d_hi;
    double best = -1.0;
    for (int64_t cols = kBigMin; cols <= kBigMax; cols *= 2) {
      const int64_t bg_cap = g->dev.tb_count < cols ? g->dev.tb_count : cols;
      int64_t dbg = 0, nbg = 0;
      GS_TRY(hub_threshold(g, bg_cap, d_tb, d_cnt, stream, &dbg, &nbg));
      if (nbg <= 0) continue;
      const int64_t md_cap = (int64_t)(((double)budget - used) / (2.0 * (double)nbg));
      if (md_cap <= 0) continue;
      // lowest degree d_md >= kMidMinDegree with at most md_cap mid vertices
      int64_t dmd = 0, n_ge = 0;
      GS_TRY(hub_threshold(g, md_cap + g->dev.tb_count, kMidMinDegree, d_cnt, stream, &dmd,
                           &n_ge));
      if (dmd >= d_hi) continue;
      // and, raising d_md if needed, at most kMidWorkMax build increments
      unsigned long long w = 0;
      GS_TRY(work_at(dmd, dbg, &w));
      if (w > kMidWorkMax) {
        int64_t lo = dmd, hi = d_hi;  // work(lo) too large, work(hi) = 0
        while (hi - lo > 1) {
          const int64_t mid = lo + (hi - lo) / 2;
          GS_TRY(work_at(mid, dbg, &w));
          if (w <= kMidWorkMax) hi = mid; else lo = mid;
        }
        dmd = hi;
      }
      if (dmd >= d_hi) continue;
      // pilot tests this shape answers
      double saved = 0.0;
      for (const PilotItem& it : pilot)
        if (it.d_tab >= dbg && it.d_other >= dmd && it.d_other >= kMidMinDegree &&
            it.d_other < d_hi)
          saved += (double)it.cost;
      if (saved > best) {  // ties keep the narrower shape
        best = saved;
        d_bg = dbg;
        n_bg = nbg;
        d_md = dmd;
      }
      if (bg_cap == g->dev.tb_count) break;
    }
    const int64_t md_cap = n_bg > 0 ? 1 : 0;
    if (md_cap > 0 && d_md < d_hi) {
      int32_t* hubs = nullptr;
      GS_TRY(assign(d_bg, &g->bg_slot, &hubs, n_bg));
      cudaFree(hubs);
      k_flag_mid<<<grid_for(n, 256, 8), 256, 0, stream>>>(g->dev.row_ptr, g->tb_slot, n, d_md,
                                                          d_hi, flag);
      GS_TRY(exclusive_scan_i64(flag, flag, n, tmp, stream));
      int64_t rows = 0;
      GS_CUDA(cudaMemcpyAsync(&rows, flag + n, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
      GS_CUDA(cudaStreamSynchronize(stream));
      if (rows > 0) {
        const int64_t nwords = (rows * n_bg + 1) / 2;
        cudaError_t me = cudaMalloc(&g->md_codeg, sizeof(uint32_t) * (size_t)nwords);
        if (me != cudaSuccess) return cuda_fail(me, "mid x big table", __FILE__, __LINE__);
        k_set_mid_rows<<<grid_for(n, 256, 8), 256, 0, stream>>>(flag, g->dev.row_ptr, n, d_md,
                                                                d_hi, g->tb_slot);
        // big-neighbour lists (flag is free again: offsets), row vertices
        k_big_count<<<grid_for(n * 32, 256, 8), 256, 0, stream>>>(g->dev.row_ptr, g->dev.col, n,
                                                                  g->bg_slot, flag);
        GS_TRY(exclusive_scan_i64(flag, flag, n, tmp, stream));
        int64_t nb = 0;
        GS_CUDA(cudaMemcpyAsync(&nb, flag + n, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
        GS_CUDA(cudaStreamSynchronize(stream));
        uint16_t* blist = nullptr;
        int32_t* rows_v = nullptr;
        cudaError_t le = cudaMalloc(&blist, sizeof(uint16_t) * (size_t)(nb > 0 ? nb : 1));
        if (le == cudaSuccess) le = cudaMalloc(&rows_v, sizeof(int32_t) * (size_t)rows);
        if (le != cudaSuccess) {
          cudaFree(blist);
          return cuda_fail(le, "mid x big table lists", __FILE__, __LINE__);
        }
        k_big_fill<<<grid_for(n * 32, 256, 8), 256, 0, stream>>>(g->dev.row_ptr, g->dev.col, n,
                                                                 g->bg_slot, flag, blist);
        k_mid_row_vertex<<<grid_for(n, 256, 8), 256, 0, stream>>>(g->tb_slot, n, rows_v);
        const size_t row_smem = sizeof(uint32_t) * (size_t)((n_bg + 1) / 2);
        cudaError_t e = cudaFuncSetAttribute(k_mid_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)row_smem);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), stream);
        if (e == cudaSuccess) {
          k_mid_rows<<<sm_count(), kMidRowThreads, row_smem, stream>>>(
              g->dev.row_ptr, g->dev.col, rows_v, rows, flag, blist, n_bg, g->md_codeg, d_cnt);
          e = cudaStreamSynchronize(stream);
        }
        cudaFree(blist);
        cudaFree(rows_v);
        if (e != cudaSuccess) return cuda_fail(e, "mid x big table", __FILE__, __LINE__);
        g->dev.bg_slot = g->bg_slot;
        g->dev.md_codeg = g->md_codeg;
        g->dev.md_count = rows;
        g->dev.bg_count = n_bg;
        used += (double)nwords * 4.0;
      }
    }
  }
  // ---- table slot of every adjacency entry (cost pass), if the budget has
  // room left after everything above
  const size_t tb_bytes_col = sizeof(int32_t) * (size_t)g->dev.nnz;
  if (g->dev.tb_count > 1 && g->dev.nnz > 0 && (double)budget >= used + (double)tb_bytes_col) {
    cudaError_t ae = cudaMalloc(&g->col_tb, tb_bytes_col);
    if (ae != cudaSuccess) return cuda_fail(ae, "adjacency table slots", __FILE__, __LINE__);
    k_col_tb<<<grid_for(g->dev.nnz, 256, 8), 256, 0, stream>>>(g->dev.col, g->dev.nnz,
                                                               g->tb_slot, g->col_tb);
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "adjacency table slots", __FILE__, __LINE__);
    g->dev.col_tb = g->col_tb;
  }
  return GS_OK;
}

namespace gs {
gs_status build_dense_blocks(gs_graph* g, const int64_t* h_first, int64_t ranges,
                             uint64_t max_bytes, cudaStream_t stream) {
  const int64_t n = g->dev.n;
  if (n == 0 || ranges <= 0) return GS_OK;
  std::vector<int64_t> row(n, -1);
  std::vector<int32_t> first(n, 0);
  int64_t words_total = 0;
  for (int64_t i = 0; i < ranges; ++i) {
    const int64_t f = h_first[i], len = h_first[i + 1] - h_first[i];
    if (len <= 0 || len > kDenseGraphMax) continue;
    const int64_t w = (len + 31) / 32;
    for (int64_t v = 0; v < len; ++v) {
      row[f + v] = words_total + v * w;
      first[f + v] = (int32_t)f;
    }
    words_total += len * w;
  }
  if (words_total == 0 || (uint64_t)words_total * 4 > max_bytes) return GS_OK;
  if (cudaMalloc(&g->dm_bits, sizeof(uint32_t) * (size_t)words_total) != cudaSuccess ||
      cudaMalloc(&g->dm_row, sizeof(int64_t) * (size_t)n) != cudaSuccess ||
      cudaMalloc(&g->dm_first, sizeof(int32_t) * (size_t)n) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(g->dm_bits);
    cudaFree(g->dm_row);
    cudaFree(g->dm_first);
    g->dm_bits = nullptr;
    g->dm_row = nullptr;
    g->dm_first = nullptr;
    return GS_OK;  // the matrices are an accelerator, not a requirement
  }
  GS_CUDA(cudaMemsetAsync(g->dm_bits, 0, sizeof(uint32_t) * (size_t)words_total, stream));
  GS_CUDA(cudaMemcpyAsync(g->dm_row, row.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice,
                          stream));
  GS_CUDA(cudaMemcpyAsync(g->dm_first, first.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice,
                          stream));
  k_dense_rows<<<grid_for(n * 32, 256, 8), 256, 0, stream>>>(g->dev.row_ptr, g->dev.col, n,
                                                             g->dm_row, g->dm_first, g->dm_bits);
  GS_CUDA(cudaStreamSynchronize(stream));
  g->dev.dm_bits = g->dm_bits;
  g->dev.dm_row = g->dm_row;
  g->dev.dm_first = g->dm_first;
  return GS_OK;
}
}  // namespace gs

extern "C" gs_status gs_graph_create(const int64_t* d_row_ptr, const int32_t* d_col, int64_t n,
                                     int64_t nnz, uint32_t flags, uint64_t hub_budget_bytes,
                                     void* stream_, gs_graph** out) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (out == nullptr || d_row_ptr == nullptr || n < 0 || nnz < 0 || (nnz > 0 && d_col == nullptr)) {
    set_error("gs_graph_create: invalid arguments");
    return GS_EINVAL;
  }
  if (n > INT32_MAX || (nnz & 1)) {
    set_error("gs_graph_create: n must fit int32 and nnz must be even (both orientations)");
    return GS_EINVAL;
  }
  int64_t ends[2] = {0, 0};
  GS_CUDA(cudaMemcpyAsync(&ends[0], d_row_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
  GS_CUDA(cudaMemcpyAsync(&ends[1], d_row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
  GS_CUDA(cudaStreamSynchronize(stream));
  if (ends[0] != 0 || ends[1] != nnz) {
    set_error("gs_graph_create: row_ptr[0] must be 0 and row_ptr[n] must equal nnz");
    return GS_EINVAL;
  }
  gs_graph* g = new gs_graph();
  memset(g, 0, sizeof(*g));
  g->dev.row_ptr = d_row_ptr;
  g->dev.col = d_col;
  g->dev.n = n;
  g->dev.nnz = nnz;
  g->m = nnz / 2;
  auto fail = [&](gs_status s) {
    gs_graph_destroy(g);
    return s;
  };
  DevError* d_err = nullptr;
  unsigned long long* d_max = nullptr;
  int64_t* tmp = nullptr;
  if (cudaMalloc(&d_err, sizeof(DevError) + sizeof(unsigned long long)) != cudaSuccess) {
    set_error("gs_graph_create: out of device memory");
    return fail(GS_ENOMEM);
  }
  d_max = reinterpret_cast<unsigned long long*>(d_err + 1);
  cudaMemsetAsync(d_err, 0, sizeof(DevError) + sizeof(unsigned long long), stream);
  if (flags & GS_VALIDATE) {
    k_validate<<<grid_for(n * 32, 256, 8), 256, 0, stream>>>(d_row_ptr, d_col, n, nnz, d_err);
    gs_status s = read_error(d_err, stream, "gs_graph_create");
    if (s != GS_OK) {
      cudaFree(d_err);
      return fail(s);
    }
  }
  int64_t tmp_elems = scan_tmp_elems(n);
  if (cudaMalloc(&g->up_ptr, sizeof(int64_t) * (size_t)(n > 0 ? n : 1)) != cudaSuccess ||
      cudaMalloc(&g->nbr_degsum, sizeof(int64_t) * (size_t)(n > 0 ? n : 1)) != cudaSuccess ||
      cudaMalloc(&g->edge_off, sizeof(int64_t) * (size_t)(n + 1)) != cudaSuccess ||
      cudaMalloc(&tmp, sizeof(int64_t) * (size_t)tmp_elems) != cudaSuccess) {
    cudaFree(d_err);
    cudaFree(tmp);
    set_error("gs_graph_create: out of device memory");
    return fail(GS_ENOMEM);
  }
  g->dev.up_ptr = g->up_ptr;
  if (n > 0) {
    k_nbr_degsum<<<grid_for(n * 32, 256, 8), 256, 0, stream>>>(d_row_ptr, d_col, n,
                                                               g->nbr_degsum);
    k_upper<<<grid_for(n, 256, 8), 256, 0, stream>>>(d_row_ptr, d_col, n, g->up_ptr, g->edge_off,
                                                     d_max);
  }
  gs_status s = exclusive_scan_i64(g->edge_off, g->edge_off, n, tmp, stream);
  unsigned long long hmax = 0;
  int64_t m_check = 0;
  cudaMemcpyAsync(&hmax, d_max, sizeof(hmax), cudaMemcpyDeviceToHost, stream);
  cudaMemcpyAsync(&m_check, g->edge_off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, stream);
  cudaError_t ce = cudaStreamSynchronize(stream);
  cudaFree(tmp);
  cudaFree(d_err);
  if (s != GS_OK) return fail(s);
  if (ce != cudaSuccess) return fail(cuda_fail(ce, "gs_graph_create", __FILE__, __LINE__));
  g->max_degree = (int64_t)hmax;
  if (m_check != g->m) {
    set_error("gs_graph_create: upper-triangle edge count %lld != nnz/2 = %lld (asymmetric CSR?)",
              (long long)m_check, (long long)g->m);
    return fail(GS_EASYM);
  }
  gs_status hs = build_hub_index(g, hub_budget_bytes, stream);
  if (hs != GS_OK) return fail(hs);
  hs = build_oriented(g, stream);
  if (hs != GS_OK) return fail(hs);
  if (n <= kDenseGraphMax && hub_budget_bytes != 1) {
    // a small graph gets its whole adjacency as a bit matrix (Sec. 2.6 notes
    // adjacency matrices for small graphs); a 1-byte budget turns every
    // index structure off
    const int64_t range[2] = {0, n};
    hs = build_dense_blocks(g, range, 1, (uint64_t)64 << 20, stream);
    if (hs != GS_OK) return fail(hs);
  }
  *out = g;
  return GS_OK;
}

extern "C" gs_status gs_graph_destroy(gs_graph* g) {
  if (g == nullptr) return GS_OK;
  cudaFree(g->up_ptr);
  cudaFree(g->nbr_degsum);
  cudaFree(g->edge_off);
  cudaFree(g->bm_slot);
  cudaFree(g->bm_bits);
  cudaFree(g->tb_slot);
  cudaFree(g->tb_codeg);
  cudaFree(g->hm_slot);
  cudaFree(g->hm_bits);
  cudaFree(g->col_hm);
  cudaFree(g->mn_ptr);
  cudaFree(g->mn_slot);
  cudaFree(g->nm_ptr);
  cudaFree(g->nm_col);
  cudaFree(g->hm_vertex);
  cudaFree(g->dm_bits);
  cudaFree(g->dm_row);
  cudaFree(g->dm_first);
  cudaFree(g->bg_slot);
  cudaFree(g->md_codeg);
  cudaFree(g->dir_at);
  cudaFree(g->dir);
  cudaFree(g->col_tb);
  cudaFree(g->tb_giant);
  cudaFree(g->tb_giant_codeg);
  cudaFree(g->out_ptr);
  cudaFree(g->out_col);
  cudaFree(g->in_ptr);
  cudaFree(g->in_col);
  cudaFree(g->in_pos);
  cudaFree(g->orient_units);
  delete g;
  return GS_OK;
}

extern "C" gs_status gs_graph_info(const gs_graph* g, int64_t* n, int64_t* m, int64_t* max_degree,
                                   int64_t* bitmap_hubs, int64_t* table_hubs) {
  if (g == nullptr) {
    set_error("gs_graph_info: null graph");
    return GS_EINVAL;
  }
  if (n) *n = g->dev.n;
  if (m) *m = g->m;
  if (max_degree) *max_degree = g->max_degree;
  if (bitmap_hubs) *bitmap_hubs = g->dev.bm_count;
  if (table_hubs) *table_hubs = g->dev.tb_count;
  return GS_OK;
}

extern "C" gs_status gs_graph_index_info(const gs_graph* g, int64_t* matrix_hubs,
                                         int64_t* mid_rows, int64_t* big_hubs,
                                         int64_t* dir_vertices) {
  if (g == nullptr) {
    set_error("gs_graph_index_info: null graph");
    return GS_EINVAL;
  }
  if (matrix_hubs) *matrix_hubs = g->dev.hm_count;
  if (mid_rows) *mid_rows = g->dev.md_count;
  if (big_hubs) *big_hubs = g->dev.bg_count;
  if (dir_vertices) *dir_vertices = g->dev.dir_count;
  return GS_OK;
}

// =================================================================== sampler
namespace gs {

// SplitMix64 output function (Steele, Lea, Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014) for generator state x.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Edge i is kept iff its 53-bit key lies in [lo, hi): lo = 0 is the plain
// Bernoulli(hi / 2^53) sample, and for lo > 0 the keys between two
// fractions give the edges one sample adds to a smaller one with the same
// seed (the samples are nested).
__device__ __forceinline__ bool edge_kept(uint64_t seed, uint64_t i, uint64_t lo, uint64_t hi) {
  const uint64_t key = splitmix64(seed ^ splitmix64(i)) >> 11;
  return key >= lo && key < hi;
}

constexpr int kSampThreads = 256;
constexpr int kSampItems = 16;
constexpr int64_t kSampTile = (int64_t)kSampThreads * kSampItems;

// Edges [e0, e0 + m) of the canonical order are sampled; the hash input is
// the index relative to e0 (so a graph inside a disjoint union samples
// exactly as it does on its own).
__global__ void k_sample_count(int64_t m, uint64_t seed, uint64_t lo, uint64_t threshold,
                               int64_t* __restrict__ tile_cnt) {
  int64_t base = (int64_t)blockIdx.x * kSampTile + (int64_t)threadIdx.x * kSampItems;
  int c = 0;
#pragma unroll
  for (int j = 0; j < kSampItems; ++j)
    if (base + j < m) c += edge_kept(seed, (uint64_t)(base + j), lo, threshold);
  c = __reduce_add_sync(0xffffffffu, c);
  __shared__ int wsum[kSampThreads / 32];
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t s = 0;
    for (int w = 0; w < kSampThreads / 32; ++w) s += wsum[w];
    tile_cnt[blockIdx.x] = s;
  }
}

__global__ void k_sample_write(const int32_t* __restrict__ col, const int64_t* __restrict__ up_ptr,
                               const int64_t* __restrict__ edge_off, int64_t n, int64_t e0,
                               int64_t m, uint64_t seed, uint64_t lo, uint64_t threshold,
                               const int64_t* __restrict__ tile_off, int32_t* __restrict__ pairs) {
  __shared__ int wsum[kSampThreads / 32];
  int64_t base = (int64_t)blockIdx.x * kSampTile + (int64_t)threadIdx.x * kSampItems;
  unsigned bits = 0;
#pragma unroll
  for (int j = 0; j < kSampItems; ++j)
    if (base + j < m && edge_kept(seed, (uint64_t)(base + j), lo, threshold)) bits |= 1u << j;
  int c = __popc(bits);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = c;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  int before = 0;
  for (int w = 0; w < warp; ++w) before += wsum[w];
  int64_t pos = tile_off[blockIdx.x] + before + x - c;
  while (bits) {
    int j = __ffs(bits) - 1;
    bits &= bits - 1;
    int64_t i = e0 + base + j;
    // row u owning canonical edge i: the last u with edge_off[u] <= i
    int64_t lo = 0, len = n;
    while (len > 1) {
      int64_t half = len >> 1;
      lo = (edge_off[lo + half] <= i) ? lo + half : lo;
      len -= half;
    }
    int32_t v = col[up_ptr[lo] + (i - edge_off[lo])];
    pairs[2 * pos] = (int32_t)lo;
    pairs[2 * pos + 1] = v;
    ++pos;
  }
}

}  // namespace gs

namespace gs {

// Samples into d_pairs (capacity max_k) or, when d_pairs is NULL, into
// workspace slot 3 sized to the number kept (*pairs_out receives it).
gs_status sample_impl(const gs_graph* g, gs_workspace* ws, double fraction, uint64_t seed,
                      int32_t* d_pairs, int64_t max_k, int64_t* k_out, int32_t** pairs_out,
                      cudaStream_t stream) {
  return sample_range(g, ws, fraction, seed, 0, g->m, d_pairs, max_k, k_out, pairs_out, stream);
}

gs_status sample_range(const gs_graph* g, gs_workspace* ws, double fraction, uint64_t seed,
                       int64_t e0, int64_t m, int32_t* d_pairs, int64_t max_k, int64_t* k_out,
                       int32_t** pairs_out, cudaStream_t stream, double fraction_lo) {
  *k_out = 0;
  if (pairs_out) *pairs_out = d_pairs;
  if (m == 0) return GS_OK;
  const uint64_t threshold = (uint64_t)floor(fraction * 9007199254740992.0);
  const uint64_t lo = (uint64_t)floor(fraction_lo * 9007199254740992.0);
  int64_t tiles = (m + kSampTile - 1) / kSampTile;
  size_t bytes = Carve::bytes_for<int64_t>(tiles + 1) * 2 +
                 Carve::bytes_for<int64_t>(scan_tmp_elems(tiles));
  void* base = nullptr;
  GS_TRY(ws_reserve(ws, 2, bytes, stream, &base));
  Carve c{(char*)base, 0};
  int64_t* cnt = c.take<int64_t>(tiles + 1);
  int64_t* off = c.take<int64_t>(tiles + 1);
  int64_t* tmp = c.take<int64_t>(scan_tmp_elems(tiles));
  k_sample_count<<<(unsigned)tiles, kSampThreads, 0, stream>>>(m, seed, lo, threshold, cnt);
  GS_TRY(exclusive_scan_i64(cnt, off, tiles, tmp, stream));
  ws->launches_total += 4;
  int64_t kept = 0;
  GS_CUDA(cudaMemcpyAsync(&kept, off + tiles, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
  GS_CUDA(cudaStreamSynchronize(stream));
  *k_out = kept;
  if (d_pairs == nullptr) {
    void* b3 = nullptr;
    GS_TRY(ws_reserve(ws, 3, Carve::bytes_for<int32_t>(2 * kept), stream, &b3));
    d_pairs = (int32_t*)b3;
    if (pairs_out) *pairs_out = d_pairs;
  } else if (kept > max_k) {
    set_error("gs_sample: %lld edges kept but the output holds %lld", (long long)kept,
              (long long)max_k);
    return GS_ECAPACITY;
  }
  if (kept > 0) {
    k_sample_write<<<(unsigned)tiles, kSampThreads, 0, stream>>>(
        g->dev.col, g->up_ptr, g->edge_off, g->dev.n, e0, m, seed, lo, threshold, off, d_pairs);
    ws->launches_total += 1;
  }
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

}  // namespace gs

extern "C" gs_status gs_sample(const gs_graph* g, gs_workspace* ws, double fraction, uint64_t seed,
                               int32_t* d_pairs, int64_t max_k, int64_t* k_out, void* stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (g == nullptr || ws == nullptr || k_out == nullptr || max_k < 0 || d_pairs == nullptr ||
      !(fraction >= 0.0 && fraction <= 1.0)) {
    set_error("gs_sample: invalid arguments (fraction must lie in [0, 1])");
    return GS_EINVAL;
  }
  GS_TRY(sample_impl(g, ws, fraction, seed, d_pairs, max_k, k_out, nullptr, stream));
  GS_CUDA(cudaStreamSynchronize(stream));
  return GS_OK;
}
