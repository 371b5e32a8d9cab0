// Exact triangle counts of every edge for the 3-node pass over all edges
// (gs_count with J = E, mask within G3 | G4, no per-edge output).
//
// Algorithm 2 gives every edge e its t = |N(u) cap N(v)|; over all edges
// the same integers follow from listing every triangle once. Edges are
// oriented from the lower to the higher (degree, id) endpoint, so out-lists
// N+(x) are short (at most about sqrt(2M) long; 1,761 on R-MAT scale 24).
// A triangle {u, v, x} with u < v < x in that order is found once: at the
// oriented edge u -> v as x in N+(u) cap N+(v). It adds one to t of its
// three edges:
//   (v, x): counted in shared memory per entry of N+(v), flushed once;
//   (u, v): summed over the warp that scans N+(u), one atomic per edge;
//   (u, x): one global atomic per triangle.
// Work is grouped by the middle vertex v: a CTA stages N+(v) in a
// shared-memory hash table and streams N+(u) (coalesced) for a chunk of v's
// in-neighbours u, so a membership test is a shared-memory probe instead of
// a random DRAM access. The per-edge t are folded in edge order of the
// out-lists (the sums do not depend on the order): N3 = t,
// N4 = d_u + d_v - 2 - 2t, their sums and sums of squares in 128 bits.
#include <string.h>

#include "common.cuh"

namespace gs {

// count.cu: fixed-order final pass over the 128-bit block partials.
__global__ void k_fold_final(const unsigned __int128* __restrict__ part, int blocks,
                             unsigned long long* __restrict__ out);

namespace {

constexpr int kThreads = 256;
constexpr unsigned kFull = 0xffffffffu;
constexpr int64_t kInChunk = 256;      // in-neighbours per work unit
constexpr int32_t kMaxOutDegree = 4096;  // larger out-lists: the general pass
// Resident CTAs per SM (shared memory allows 6-7 at R-MAT scale 24's
// 4096-slot tables, 8 for shorter out-lists). R-MAT 24 exact 3-node pass:
// 0.42 s at 4, 0.31 s at 6 and 8.
#ifndef GS_ORIENT_BLOCKS_PER_SM
#define GS_ORIENT_BLOCKS_PER_SM 8
#endif
constexpr int kOrientBlocksPerSm = GS_ORIENT_BLOCKS_PER_SM;
// Out-list entries a lane loads before it probes them (loads in flight;
// R-MAT 24 exact pass: 0.346 s at 2, 0.307 s at 4, 0.290 s at 8).
#ifndef GS_PROBE_BATCH
#define GS_PROBE_BATCH 8
#endif
constexpr int kProbeBatch = GS_PROBE_BATCH;

typedef unsigned __int128 u128;

__device__ __forceinline__ bool ranks_above(int64_t dx, int32_t x, int64_t dv, int32_t v) {
  return dx > dv || (dx == dv && x > v);
}

// Out- and in-degree of every vertex (one warp per vertex).
__global__ void k_orient_count(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                               int64_t n, int64_t* __restrict__ dplus, int64_t* __restrict__ dminus,
                               unsigned long long* __restrict__ maxd) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  unsigned long long mx = 0;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    const int64_t dv = row_ptr[v + 1] - row_ptr[v];
    unsigned up = 0;
    for (int64_t p = row_ptr[v] + lane; p < row_ptr[v + 1]; p += 32) {
      const int32_t x = col[p];
      up += ranks_above(__ldg(row_ptr + x + 1) - __ldg(row_ptr + x), x, dv, (int32_t)v);
    }
    up = __reduce_add_sync(kFull, up);
    if (lane == 0) {
      dplus[v] = up;
      dminus[v] = dv - up;
      mx = up > mx ? up : mx;
    }
  }
  if (lane == 0 && mx) atomicMax(maxd, mx);
}

// Out-list (higher-ranked neighbours) and in-list (lower-ranked ones) of
// every vertex, both in increasing id (one warp per vertex).
__global__ void k_orient_fill(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                              int64_t n, const int64_t* __restrict__ out_ptr,
                              const int64_t* __restrict__ in_ptr, int32_t* __restrict__ out_col,
                              int32_t* __restrict__ in_col) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    const int64_t dv = row_ptr[v + 1] - row_ptr[v];
    int64_t o = out_ptr[v], i = in_ptr[v];
    for (int64_t p0 = row_ptr[v]; p0 < row_ptr[v + 1]; p0 += 32) {
      const int64_t p = p0 + lane;
      const bool live = p < row_ptr[v + 1];
      int32_t x = 0;
      bool up = false;
      if (live) {
        x = col[p];
        up = ranks_above(__ldg(row_ptr + x + 1) - __ldg(row_ptr + x), x, dv, (int32_t)v);
      }
      const unsigned bu = __ballot_sync(kFull, live && up);
      const unsigned bd = __ballot_sync(kFull, live && !up);
      const unsigned below = (1u << lane) - 1u;
      if (live && up) out_col[o + __popc(bu & below)] = x;
      if (live && !up) in_col[i + __popc(bd & below)] = x;
      o += __popc(bu);
      i += __popc(bd);
    }
  }
}

// in_pos[j]: the out-list position of v in N+(u) for the in-edge u -> v
// stored at in_col[j] (halving search of the short out-list).
__global__ void k_orient_in_pos(const int64_t* __restrict__ out_ptr,
                                const int32_t* __restrict__ out_col,
                                const int64_t* __restrict__ in_ptr,
                                const int32_t* __restrict__ in_col, int64_t n,
                                uint32_t* __restrict__ in_pos) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    for (int64_t j = in_ptr[v] + lane; j < in_ptr[v + 1]; j += 32) {
      const int32_t u = in_col[j];
      int64_t lo = out_ptr[u], len = out_ptr[u + 1] - lo;
      while (len > 1) {
        const int64_t half = len >> 1;
        lo = (__ldg(out_col + lo + half) <= (int32_t)v) ? lo + half : lo;
        len -= half;
      }
      in_pos[j] = (uint32_t)lo;
    }
  }
}

// Work units: ceil(d-(v) / kInChunk) per vertex with a non-empty out-list.
__global__ void k_orient_units(const int64_t* __restrict__ out_ptr,
                               const int64_t* __restrict__ in_ptr, int64_t n,
                               int64_t* __restrict__ units) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t dp = out_ptr[v + 1] - out_ptr[v], dm = in_ptr[v + 1] - in_ptr[v];
    units[v] = dp > 0 ? (dm + kInChunk - 1) / kInChunk : 0;
  }
}

__device__ __forceinline__ uint32_t slot_hash(int32_t x, int bits) {
  return ((uint32_t)x * 2654435761u) >> (32 - bits);
}

// Triangles by middle vertex (see the file comment). Persistent CTAs take
// units from a counter; dynamic shared memory holds the hash table of
// N+(v): keys (int32, -1 empty) and one word per slot holding the out-list
// position of x (low 16 bits) and the count of (v, x) (high 16 bits: at
// most kInChunk per unit).
__global__ void __launch_bounds__(kThreads, kOrientBlocksPerSm)
    k_tri_oriented(const int64_t* __restrict__ out_ptr, const int32_t* __restrict__ out_col,
                   const int64_t* __restrict__ in_ptr, const int32_t* __restrict__ in_col,
                   const uint32_t* __restrict__ in_pos, const int64_t* __restrict__ unit_off,
                   int64_t n, int bits, unsigned int* __restrict__ tplus,
                   unsigned long long* __restrict__ counter,
                   unsigned long long* __restrict__ probes) {
  extern __shared__ int32_t smem[];
  const int S = 1 << bits;
  int32_t* keys = smem;
  uint32_t* slotw = reinterpret_cast<uint32_t*>(smem + S);
  __shared__ int64_t cur;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t U = __ldg(unit_off + n);
  unsigned long long my_probes = 0;
  for (;;) {
    if (threadIdx.x == 0) cur = (int64_t)atomicAdd(counter, 1ull);
    __syncthreads();
    const int64_t unit = cur;
    if (unit >= U) break;
    int64_t lo = 0, len = n;  // vertex owning the unit
    while (len > 1) {
      const int64_t half = len >> 1;
      lo = (__ldg(unit_off + lo + half) <= unit) ? lo + half : lo;
      len -= half;
    }
    const int32_t v = (int32_t)lo;
    const int64_t ob = out_ptr[v], od = out_ptr[v + 1] - ob;
    const int64_t j0 = in_ptr[v] + (unit - __ldg(unit_off + v)) * kInChunk;
    const int64_t j1 = min(in_ptr[v + 1], j0 + kInChunk);
    // this unit's table: the smallest power of two >= 2 |N+(v)| (at least
    // 64 slots), so short out-lists clear and flush only a few slots
    int ub_bits = 6;
    while ((1ll << ub_bits) < 2 * od) ++ub_bits;
    const int Su = 1 << ub_bits;
    for (int s = threadIdx.x; s < Su; s += kThreads) keys[s] = -1;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < od; i += kThreads) {
      const int32_t x = out_col[ob + i];
      uint32_t s = slot_hash(x, ub_bits);
      while (atomicCAS(keys + s, -1, x) != -1) s = (s + 1) & (uint32_t)(Su - 1);
      slotw[s] = (uint32_t)i;  // position, count 0
    }
    __syncthreads();
    for (int64_t j = j0 + wid; j < j1; j += kThreads / 32) {
      const int32_t u = in_col[j];
      const int64_t ub = out_ptr[u], ud = out_ptr[u + 1] - ub;
      unsigned hits = 0;
      for (int64_t i0 = lane; i0 < ud; i0 += 32 * kProbeBatch) {
        int32_t xb[kProbeBatch];
#pragma unroll
        for (int q = 0; q < kProbeBatch; ++q)
          xb[q] = i0 + 32 * q < ud ? __ldg(out_col + ub + i0 + 32 * q) : -1;
#pragma unroll
        for (int q = 0; q < kProbeBatch; ++q) {
          const int32_t x = xb[q];
          if (x < 0) continue;
          uint32_t s = slot_hash(x, ub_bits);
          int32_t k;
          while ((k = keys[s]) != -1 && k != x) s = (s + 1) & (uint32_t)(Su - 1);
          if (k == x) {
            ++hits;
            atomicAdd(slotw + s, 1u << 16);
            atomicAdd(tplus + ub + i0 + 32 * q, 1u);  // edge (u, x)
          }
        }
      }
      my_probes += (unsigned long long)(ud > lane ? (ud - lane + 31) / 32 : 0);
      hits = __reduce_add_sync(kFull, hits);
      if (lane == 0 && hits) atomicAdd(tplus + in_pos[j], hits);  // edge (u, v)
    }
    __syncthreads();
    for (int s = threadIdx.x; s < Su; s += kThreads) {
      const uint32_t w = slotw[s];
      if (keys[s] != -1 && (w >> 16) != 0) atomicAdd(tplus + ob + (w & 0xffffu), w >> 16);  // (v, x)
    }
    __syncthreads();  // the table and cur are reused for the next unit
  }
  my_probes = __reduce_add_sync(kFull, (unsigned)min(my_probes, 0xffffffffull));
  if (lane == 0 && my_probes) atomicAdd(probes, my_probes);
}

// N3 = t, N4 = d_u + d_v - 2 - 2t per oriented edge; 128-bit block sums in
// the layout of k_fold (order 3, 4, 7, ..., 12, then the squares).
__global__ void __launch_bounds__(kThreads)
    k_fold_oriented(const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ out_ptr,
                    const int32_t* __restrict__ out_col, const unsigned int* __restrict__ tplus,
                    int64_t n, u128* __restrict__ part, unsigned long long* __restrict__ stats) {
  u128 s3 = 0, s4 = 0, q3 = 0, q4 = 0;
  unsigned long long model = 0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
    const int64_t du = row_ptr[u + 1] - row_ptr[u];
    for (int64_t p = out_ptr[u] + lane; p < out_ptr[u + 1]; p += 32) {
      const int32_t v = out_col[p];
      const int64_t dv = __ldg(row_ptr + v + 1) - __ldg(row_ptr + v);
      const uint64_t t = tplus[p];
      const uint64_t n4 = (uint64_t)(du + dv - 2) - 2 * t;
      s3 += t;
      s4 += n4;
      q3 += (u128)t * t;
      q4 += (u128)n4 * n4;
      model += 24 + 4 * (unsigned long long)(du + dv);
    }
  }
  __shared__ u128 red[kThreads / 32][4];
  u128 v4[4] = {s3, s4, q3, q4};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    u128 x = v4[i];
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long lo = (unsigned long long)x, hi = (unsigned long long)(x >> 64);
      lo = __shfl_down_sync(kFull, lo, o);
      hi = __shfl_down_sync(kFull, hi, o);
      x += ((u128)hi << 64) | lo;
    }
    if (lane == 0) red[wid][i] = x;
  }
  for (int o = 16; o > 0; o >>= 1) model += __shfl_xor_sync(kFull, model, o);
  if (lane == 0 && model) atomicAdd(stats + 2, model);
  __syncthreads();
  if (threadIdx.x < 16) {
    u128 s = 0;
    const int k = threadIdx.x;
    const int src = k == 0 ? 0 : k == 1 ? 1 : k == 8 ? 2 : k == 9 ? 3 : -1;
    if (src >= 0)
      for (int w = 0; w < kThreads / 32; ++w) s += red[w][src];
    part[(int64_t)blockIdx.x * 16 + k] = s;
  }
}

}  // namespace

// Oriented out- and in-lists for the exact 3-node pass (registration).
// Skipped (the general pass serves) when the graph has 2^31 or more edges
// or an out-list longer than kMaxOutDegree.
gs_status build_oriented(gs_graph* g, cudaStream_t stream) {
  const int64_t n = g->dev.n, m = g->m;
  if (n == 0 || m == 0 || m >= ((int64_t)1 << 31)) return GS_OK;
  int64_t* dp = nullptr;
  int64_t* dm = nullptr;
  int64_t* tmp = nullptr;
  unsigned long long* d_max = nullptr;
  auto release = [&]() {
    cudaFree(dp);
    cudaFree(dm);
    cudaFree(tmp);
    cudaFree(d_max);
  };
  if (cudaMalloc(&dp, sizeof(int64_t) * (size_t)(n + 1)) != cudaSuccess ||
      cudaMalloc(&dm, sizeof(int64_t) * (size_t)(n + 1)) != cudaSuccess ||
      cudaMalloc(&tmp, sizeof(int64_t) * (size_t)scan_tmp_elems(n + 1)) != cudaSuccess ||
      cudaMalloc(&d_max, sizeof(unsigned long long)) != cudaSuccess) {
    release();
    cudaGetLastError();
    return GS_OK;  // no room: the general pass serves
  }
  cudaMemsetAsync(d_max, 0, sizeof(unsigned long long), stream);
  k_orient_count<<<grid_for(n * 32, kThreads, 8), kThreads, 0, stream>>>(
      g->dev.row_ptr, g->dev.col, n, dp, dm, d_max);
  unsigned long long hmax = 0;
  cudaMemcpyAsync(&hmax, d_max, sizeof(hmax), cudaMemcpyDeviceToHost, stream);
  cudaError_t e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    release();
    return cuda_fail(e, "oriented lists", __FILE__, __LINE__);
  }
  if ((int64_t)hmax > kMaxOutDegree) {
    release();
    return GS_OK;
  }
  bool ok = cudaMalloc(&g->out_ptr, sizeof(int64_t) * (size_t)(n + 1)) == cudaSuccess &&
            cudaMalloc(&g->in_ptr, sizeof(int64_t) * (size_t)(n + 1)) == cudaSuccess &&
            cudaMalloc(&g->out_col, sizeof(int32_t) * (size_t)m) == cudaSuccess &&
            cudaMalloc(&g->in_col, sizeof(int32_t) * (size_t)m) == cudaSuccess &&
            cudaMalloc(&g->in_pos, sizeof(uint32_t) * (size_t)m) == cudaSuccess &&
            cudaMalloc(&g->orient_units, sizeof(int64_t) * (size_t)(n + 1)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    release();
    cudaFree(g->out_ptr);
    cudaFree(g->in_ptr);
    cudaFree(g->out_col);
    cudaFree(g->in_col);
    cudaFree(g->in_pos);
    cudaFree(g->orient_units);
    g->out_ptr = g->in_ptr = g->orient_units = nullptr;
    g->out_col = g->in_col = nullptr;
    g->in_pos = nullptr;
    return GS_OK;
  }
  gs_status s = exclusive_scan_i64(dp, g->out_ptr, n, tmp, stream);
  if (s == GS_OK) s = exclusive_scan_i64(dm, g->in_ptr, n, tmp, stream);
  if (s == GS_OK) {
    k_orient_fill<<<grid_for(n * 32, kThreads, 8), kThreads, 0, stream>>>(
        g->dev.row_ptr, g->dev.col, n, g->out_ptr, g->in_ptr, g->out_col, g->in_col);
    k_orient_in_pos<<<grid_for(n * 32, kThreads, 8), kThreads, 0, stream>>>(
        g->out_ptr, g->out_col, g->in_ptr, g->in_col, n, g->in_pos);
    k_orient_units<<<grid_for(n, kThreads, 8), kThreads, 0, stream>>>(g->out_ptr, g->in_ptr, n,
                                                                       g->orient_units);
    s = exclusive_scan_i64(g->orient_units, g->orient_units, n, tmp, stream);
  }
  e = cudaStreamSynchronize(stream);
  release();
  if (s != GS_OK) return s;
  if (e != cudaSuccess) return cuda_fail(e, "oriented lists", __FILE__, __LINE__);
  g->max_out_degree = (int64_t)hmax;
  return GS_OK;
}

// The exact 3-node pass over every edge through the oriented lists: sums in
// the layout of gs_count's (32 words: 8 sums and 8 sums of squares, low and
// high) in d_sums, statistics in d_stats. Needs build_oriented's lists.
gs_status count_tri_oriented(const gs_graph* g, gs_workspace* ws, unsigned long long* h_sums,
                             unsigned long long* h_stats, int64_t* launches, cudaStream_t stream) {
  const int64_t n = g->dev.n, m = g->m;
  int bits = 6;
  while ((1 << bits) < 2 * g->max_out_degree) ++bits;
  const size_t smem = (size_t)(1 << bits) * 2 * sizeof(int32_t);
  const int fold_blocks = grid_for(n * 32, kThreads, 2);
  void* base = nullptr;
  GS_TRY(ws_reserve(ws, 0,
                    Carve::bytes_for<unsigned int>(m) + Carve::bytes_for<unsigned long long>(8) +
                        Carve::bytes_for<unsigned long long>(32) +
                        Carve::bytes_for<u128>((int64_t)fold_blocks * 16),
                    stream, &base));
  Carve c{(char*)base, 0};
  unsigned int* tplus = c.take<unsigned int>(m);
  unsigned long long* stats = c.take<unsigned long long>(8);
  unsigned long long* sums = c.take<unsigned long long>(32);
  u128* part = c.take<u128>((int64_t)fold_blocks * 16);
  if (ws->timing) cudaEventRecord(ws->ev[0], stream);
  GS_CUDA(cudaMemsetAsync(tplus, 0, sizeof(unsigned int) * (size_t)m, stream));
  GS_CUDA(cudaMemsetAsync(stats, 0, sizeof(unsigned long long) * 8, stream));
  if (ws->timing) cudaEventRecord(ws->ev[1], stream);
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    GS_CUDA(cudaFuncSetAttribute(k_tri_oriented, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)((size_t)(2 * kMaxOutDegree) * 2 * sizeof(int32_t))));
    attr_set[dev] = true;
  }
  if (ws->timing) cudaEventRecord(ws->ev[2], stream);
  k_tri_oriented<<<sm_count() * kOrientBlocksPerSm, kThreads, smem, stream>>>(
      g->out_ptr, g->out_col, g->in_ptr, g->in_col, g->in_pos, g->orient_units, n, bits, tplus,
      stats + 7, stats + 0);
  if (ws->timing)
    for (int ev = 3; ev <= 10; ++ev) cudaEventRecord(ws->ev[ev], stream);  // phases 2-4 empty
  GS_CUDA(cudaGetLastError());
  k_fold_oriented<<<fold_blocks, kThreads, 0, stream>>>(g->dev.row_ptr, g->out_ptr, g->out_col,
                                                        tplus, n, part, stats);
  k_fold_final<<<1, 32, 0, stream>>>(part, fold_blocks, sums);
  if (ws->timing) cudaEventRecord(ws->ev[11], stream);
  GS_CUDA(cudaGetLastError());
  GS_CUDA(cudaMemcpyAsync(h_sums, sums, sizeof(unsigned long long) * 32, cudaMemcpyDeviceToHost,
                          stream));
  GS_CUDA(cudaMemcpyAsync(h_stats, stats, sizeof(unsigned long long) * 8, cudaMemcpyDeviceToHost,
                          stream));
  GS_CUDA(cudaStreamSynchronize(stream));
  *launches = 5;
  return GS_OK;
}

}  // namespace gs
