// Disconnected 3- and 4-node graphlets (G5, G6, G13-G17): exact fold of
// their per-edge numerators from the per-edge (t, k, q) of gs_count. The
// numerators restate Sec. 2.3's estimators with the corrected terms listed
// in graphlet.h (R = vertices adjacent to neither end of the edge, C16 =
// edges touching neither end); every one is O(1) per edge.
#include <string.h>

#include "common.cuh"

namespace {

typedef unsigned __int128 u128;
typedef __int128 i128;

constexpr int kDiscThreads = 256;
constexpr int kDiscValues = 14;  // 7 sums (two's complement) + 7 sums of squares

__device__ __forceinline__ u128 shfl_down_128(u128 v, int o) {
  unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
  lo = __shfl_down_sync(0xffffffffu, lo, o);
  hi = __shfl_down_sync(0xffffffffu, hi, o);
  return ((u128)hi << 64) | lo;
}

// Per-edge numerators (order 5, 6, 13, 14, 15, 16, 17) and per-block sums:
// part[block][0..6] = sum N_i, part[block][7..13] = sum N_i^2. A sum of
// squares that wraps past 128 bits sets bit i of *ovf; a pair outside the
// graph sets *bad and is skipped.
__global__ void __launch_bounds__(kDiscThreads)
    k_fold_disc(const int64_t* __restrict__ row_ptr, int64_t n, int64_t m,
                const int32_t* __restrict__ pairs, int64_t K, const int64_t* __restrict__ per_edge,
                u128* __restrict__ part, unsigned* __restrict__ ovf, unsigned* __restrict__ bad) {
  u128 acc[kDiscValues];
#pragma unroll
  for (int i = 0; i < kDiscValues; ++i) acc[i] = 0;
  unsigned wrap = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < K;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = pairs[2 * e], y = pairs[2 * e + 1];
    if (x < 0 || y < 0 || x >= n || y >= n) {
      atomicOr(bad, 1u);
      continue;
    }
    const i128 du = row_ptr[x + 1] - row_ptr[x], dv = row_ptr[y + 1] - row_ptr[y];
    const i128 t = per_edge[3 * e], kk = per_edge[3 * e + 1], qq = per_edge[3 * e + 2];
    const i128 a = du - 1 - t, b = dv - 1 - t;
    const i128 n8 = t * (t - 1) / 2 - kk;
    const i128 n9 = t * (a + b) - 4 * n8;
    const i128 n11 = 2 * (a * (a - 1) / 2 + b * (b - 1) / 2) - t * (a + b) + 4 * n8;
    const i128 n12 = a * b - qq;
    const i128 R = (i128)n - 2 - t - a - b;
    const i128 c16 = (i128)m - du - dv + 1;
    i128 N[7];
    N[0] = R;
    N[1] = 2 * t + 3 * (a + b) + 6 * R;
    N[2] = 2 * t * R - n9;
    N[3] = (a + b) * R - 2 * n12;
    N[4] = c16 - kk - 4 * n8 - n9 - qq - 2 * n12;
    N[5] = R * (R - 1) / 2 - N[4];
    N[6] = 2 * kk + 12 * n8 + 6 * n9 + 3 * qq + 2 * n11 + 12 * n12 + 2 * N[2] + 6 * N[3] +
           6 * N[4] + 12 * N[5];
#pragma unroll
    for (int i = 0; i < 7; ++i) {
      acc[i] += (u128)N[i];
      const u128 mag = (u128)(N[i] < 0 ? -N[i] : N[i]);
      const u128 before = acc[7 + i];
      acc[7 + i] += mag * mag;
      if (acc[7 + i] < before) wrap |= 1u << i;
    }
  }
  __shared__ u128 red[kDiscThreads / 32][kDiscValues];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < kDiscValues; ++i) {
    u128 v = acc[i];
    for (int o = 16; o > 0; o >>= 1) {
      const u128 w = shfl_down_128(v, o);
      const u128 before = v;
      v += w;
      if (i >= 7 && lane + o < 32 && v < before) wrap |= 1u << (i - 7);
    }
    if (lane == 0) red[warp][i] = v;
  }
  if (wrap) atomicOr(ovf, wrap);
  __syncthreads();
  if (threadIdx.x < kDiscValues) {
    u128 s = 0;
    for (int w = 0; w < kDiscThreads / 32; ++w) {
      const u128 before = s;
      s += red[w][threadIdx.x];
      if (threadIdx.x >= 7 && s < before) atomicOr(ovf, 1u << (threadIdx.x - 7));
    }
    part[(int64_t)blockIdx.x * kDiscValues + threadIdx.x] = s;
  }
}

// Fixed-order sum of the block partials.
__global__ void k_fold_disc_final(const u128* __restrict__ part, int blocks,
                                  unsigned long long* __restrict__ out, unsigned* __restrict__ ovf) {
  if (threadIdx.x < kDiscValues) {
    u128 s = 0;
    for (int b = 0; b < blocks; ++b) {
      const u128 before = s;
      s += part[(int64_t)b * kDiscValues + threadIdx.x];
      if (threadIdx.x >= 7 && s < before) atomicOr(ovf, 1u << (threadIdx.x - 7));
    }
    out[2 * threadIdx.x] = (unsigned long long)s;
    out[2 * threadIdx.x + 1] = (unsigned long long)(s >> 64);
  }
}

}  // namespace

extern "C" gs_status gs_count_disconnected(const gs_graph* g, gs_workspace* ws, const int32_t* d_pairs,
                                           int64_t k, const int64_t* d_per_edge, gs_sums_disc* h_out,
                                           void* stream_) {
  using namespace gs;
  if (g == nullptr || ws == nullptr || h_out == nullptr || k < 0 || k > g->m ||
      (k > 0 && (d_pairs == nullptr || d_per_edge == nullptr))) {
    set_error("gs_count_disconnected: invalid arguments (need graph, workspace, output, "
              "0 <= k <= m, pairs and per-edge counts when k > 0)");
    return GS_EINVAL;
  }
  cudaStream_t stream = (cudaStream_t)stream_;
  memset(h_out, 0, sizeof(*h_out));
  h_out->k = k;
  h_out->m = g->m;
  h_out->n = g->dev.n;
  if (k == 0) return GS_OK;
  const int blocks = grid_for(k, kDiscThreads, 4);
  void* base = nullptr;
  GS_TRY(ws_reserve(ws, 0,
                    Carve::bytes_for<u128>((int64_t)blocks * kDiscValues) +
                        Carve::bytes_for<unsigned long long>(2 * kDiscValues) +
                        Carve::bytes_for<unsigned>(2),
                    stream, &base));
  Carve c{(char*)base, 0};
  u128* part = c.take<u128>((int64_t)blocks * kDiscValues);
  unsigned long long* out = c.take<unsigned long long>(2 * kDiscValues);
  unsigned* flags = c.take<unsigned>(2);  // [0] square overflow bits, [1] bad pair
  GS_CUDA(cudaMemsetAsync(flags, 0, 2 * sizeof(unsigned), stream));
  k_fold_disc<<<blocks, kDiscThreads, 0, stream>>>(g->dev.row_ptr, g->dev.n, g->m, d_pairs, k,
                                                   d_per_edge, part, flags, flags + 1);
  k_fold_disc_final<<<1, 32, 0, stream>>>(part, blocks, out, flags);
  GS_CUDA(cudaGetLastError());
  unsigned long long h[2 * kDiscValues];
  unsigned hf[2];
  GS_CUDA(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, stream));
  GS_CUDA(cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, stream));
  GS_CUDA(cudaStreamSynchronize(stream));
  if (hf[1] != 0) {
    set_error("gs_count_disconnected: a sampled pair names a vertex outside the graph");
    return GS_EINVAL;
  }
  for (int i = 0; i < 7; ++i) {
    h_out->sum[i][0] = h[2 * i];
    h_out->sum[i][1] = h[2 * i + 1];
    h_out->sumsq[i][0] = h[2 * (7 + i)];
    h_out->sumsq[i][1] = h[2 * (7 + i) + 1];
  }
  h_out->overflow = hf[0];
  return GS_OK;
}

// ------------------------------------------------- per-edge numerator matrix

namespace {

// Row e of out = (N3, N4, N7, N8, N9, N10, N11, N12) of sampled edge e.
__global__ void k_per_edge_numerators(const int64_t* __restrict__ row_ptr, int64_t n,
                                      const int32_t* __restrict__ pairs, int64_t K,
                                      const int64_t* __restrict__ per_edge,
                                      int64_t* __restrict__ out, unsigned* __restrict__ bad) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < K;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = pairs[2 * e], y = pairs[2 * e + 1];
    if (x < 0 || y < 0 || x >= n || y >= n) {
      atomicOr(bad, 1u);
      continue;
    }
    const int64_t du = row_ptr[x + 1] - row_ptr[x], dv = row_ptr[y + 1] - row_ptr[y];
    const int64_t t = per_edge[3 * e], kk = per_edge[3 * e + 1], qq = per_edge[3 * e + 2];
    const int64_t a = du - 1 - t, b = dv - 1 - t;
    const int64_t n8 = t * (t - 1) / 2 - kk;
    int64_t* o = out + 8 * e;
    o[0] = t;
    o[1] = a + b;
    o[2] = kk;
    o[3] = n8;
    o[4] = t * (a + b) - 4 * n8;
    o[5] = qq;
    o[6] = 2 * (a * (a - 1) / 2 + b * (b - 1) / 2) - t * (a + b) + 4 * n8;
    o[7] = a * b - qq;
  }
}

}  // namespace

extern "C" gs_status gs_per_edge_numerators(const gs_graph* g, gs_workspace* ws,
                                            const int32_t* d_pairs, int64_t k,
                                            const int64_t* d_per_edge, int64_t* d_out,
                                            void* stream_) {
  using namespace gs;
  if (g == nullptr || ws == nullptr || k < 0 ||
      (k > 0 && (d_pairs == nullptr || d_per_edge == nullptr || d_out == nullptr))) {
    set_error("gs_per_edge_numerators: invalid arguments");
    return GS_EINVAL;
  }
  if (k == 0) return GS_OK;
  cudaStream_t stream = (cudaStream_t)stream_;
  void* base = nullptr;
  GS_TRY(ws_reserve(ws, 0, Carve::bytes_for<unsigned>(1), stream, &base));
  unsigned* bad = (unsigned*)base;
  GS_CUDA(cudaMemsetAsync(bad, 0, sizeof(unsigned), stream));
  k_per_edge_numerators<<<grid_for(k, kDiscThreads, 8), kDiscThreads, 0, stream>>>(
      g->dev.row_ptr, g->dev.n, d_pairs, k, d_per_edge, d_out, bad);
  GS_CUDA(cudaGetLastError());
  unsigned hb = 0;
  GS_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(hb), cudaMemcpyDeviceToHost, stream));
  GS_CUDA(cudaStreamSynchronize(stream));
  if (hb != 0) {
    set_error("gs_per_edge_numerators: a sampled pair names a vertex outside the graph");
    return GS_EINVAL;
  }
  return GS_OK;
}
