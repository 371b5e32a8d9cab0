// Fixed-size uniform edge sampling (Algorithm 1 with a sample size K,
// without replacement: the K edges of smallest sampler key), weighted edge
// sampling (Algorithm 1 with a non-uniform distribution F,
// Sec. 3.1: edges drawn by k-core numbers, degrees or any vertex property),
// the k-core numbers it is usually weighted by (the extremal problem of
// Sec. 7 samples edges of large k-core number), and the estimators with a
// per-edge inverse inclusion probability (Sec. 2.3's sigma = 1/p applied
// edge by edge: Horvitz-Thompson).
//
// Edge weight w_e = min(w[u], w[v]) for a vertex weight w (with core
// numbers: the edge's own core number). Each canonical edge i (the i-th
// pair u < v in row-major CSR order) is kept independently with
// probability pi_e = min(1, s w_e), s = fraction M / W, W = sum_e w_e, by
// the uniform sampler's key: keep iff (sm(seed ^ sm(i)) >> 11) <
// floor(pi_e 2^53). The estimate of graphlet i is
//   X_i = sum_{e in J} N_i(e) / (D_i pi_e),
//   V_i = sum_{e in J} (1 - pi_e) N_i(e)^2 / (D_i^2 pi_e^2),
// with N_i the per-edge numerators of gs_count. pi_e depends only on the
// integer w_e, so the library folds exact 128-bit sums of N_i and N_i^2 per
// weight class on the device and the host evaluates the FP64 sums over the
// classes in increasing weight.
//
// k-core numbers by parallel peeling: level k starts with every remaining
// vertex of current degree <= k (core number k); removing a vertex
// decrements its remaining neighbours, and the one decrement that takes a
// neighbour from k + 1 to k adds it to the next frontier of the same level.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace gs {

namespace {

constexpr int kThreads = 256;
constexpr unsigned kFull = 0xffffffffu;
constexpr int64_t kMaxClasses = (int64_t)1 << 22;
constexpr int kSampItems = 16;
constexpr int64_t kSampTile = (int64_t)kThreads * kSampItems;

typedef unsigned __int128 u128;
typedef __int128 i128;

__device__ __forceinline__ uint64_t splitmix(uint64_t x) {
  uint64_t z = x + 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// ------------------------------------------------------------------ k-core

__global__ void k_core_init(const int64_t* __restrict__ row_ptr, int64_t n,
                            int32_t* __restrict__ deg, int32_t* __restrict__ core) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    deg[v] = (int32_t)(row_ptr[v + 1] - row_ptr[v]);
    core[v] = -1;
  }
}

// Level start: remaining vertices of current degree <= k get core k and
// join the frontier; the least degree above k is kept for the next level.
// ctr: [0] frontier size, [1] least remaining degree above k, [2] removed.
__global__ void k_core_scan(int64_t n, int32_t k, const int32_t* __restrict__ deg,
                            int32_t* __restrict__ core, int32_t* __restrict__ frontier,
                            unsigned long long* __restrict__ ctr) {
  unsigned long long least = ~0ull;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    if (core[v] != -1) continue;
    const int32_t d = deg[v];
    if (d <= k) {
      core[v] = k;
      frontier[atomicAdd(ctr, 1ull)] = (int32_t)v;
    } else if ((unsigned long long)d < least) {
      least = (unsigned long long)d;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(kFull, least, o);
    least = y < least ? y : least;
  }
  if ((threadIdx.x & 31) == 0 && least != ~0ull) atomicMin(ctr + 1, least);
}

// Removes the frontier (one warp per vertex): every remaining neighbour
// loses one; the neighbour whose degree falls from k + 1 to k gets core k
// and joins the next frontier.
__global__ void k_core_peel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                            int32_t k, const int32_t* __restrict__ frontier, int64_t fsize,
                            int32_t* __restrict__ deg, int32_t* __restrict__ core,
                            int32_t* __restrict__ next, unsigned long long* __restrict__ nsize) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t f = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; f < fsize; f += warps) {
    const int32_t v = frontier[f];
    for (int64_t p = row_ptr[v] + lane; p < row_ptr[v + 1]; p += 32) {
      const int32_t x = col[p];
      if (((volatile int32_t*)core)[x] != -1) continue;
      if (atomicSub(deg + x, 1) == k + 1) {
        core[x] = k;
        next[atomicAdd(nsize, 1ull)] = x;
      }
    }
  }
}

// ------------------------------------------------------------------ sampler

__device__ __forceinline__ int32_t edge_weight(const int32_t* __restrict__ vw, int32_t u,
                                               int32_t v) {
  const int32_t a = __ldg(vw + u), b = __ldg(vw + v);
  return a < b ? a : b;
}

// W = sum of edge weights, the largest vertex weight seen and whether any
// weight is negative. One warp per vertex over its upper neighbours.
__global__ void k_weight_sum(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                             const int64_t* __restrict__ up_ptr, const int32_t* __restrict__ vw,
                             int64_t n, unsigned long long* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  unsigned long long s = 0, neg = 0;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
    if (lane == 0 && __ldg(vw + u) < 0) neg = 1;
    for (int64_t p = up_ptr[u] + lane; p < row_ptr[u + 1]; p += 32) {
      const int32_t w = edge_weight(vw, (int32_t)u, col[p]);
      s += (unsigned long long)(w > 0 ? w : 0);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(kFull, s, o);
    neg |= __shfl_xor_sync(kFull, neg, o);
  }
  if (lane == 0) {
    if (s) atomicAdd(out, s);
    if (neg) atomicOr(out + 1, 1ull);
  }
}

__device__ __forceinline__ uint64_t keep_threshold(double scale, int32_t w) {
  double pi = scale * (double)w;
  if (pi > 1.0) pi = 1.0;
  return (uint64_t)floor(pi * 9007199254740992.0);
}

// keep[i] for every canonical edge (one warp per vertex).
__global__ void k_weighted_flags(const int64_t* __restrict__ row_ptr,
                                 const int32_t* __restrict__ col,
                                 const int64_t* __restrict__ up_ptr,
                                 const int64_t* __restrict__ edge_off,
                                 const int32_t* __restrict__ vw, int64_t n, double scale,
                                 uint64_t seed, uint8_t* __restrict__ keep) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
    const int64_t s = up_ptr[u], o = edge_off[u];
    for (int64_t p = s + lane; p < row_ptr[u + 1]; p += 32) {
      const uint64_t i = (uint64_t)(o + (p - s));
      const uint64_t key = splitmix(seed ^ splitmix(i)) >> 11;
      keep[i] = key < keep_threshold(scale, edge_weight(vw, (int32_t)u, col[p])) ? 1 : 0;
    }
  }
}

__global__ void k_flag_count(const uint8_t* __restrict__ keep, int64_t m,
                             int64_t* __restrict__ tile_cnt) {
  __shared__ int wsum[kThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kSampTile + (int64_t)threadIdx.x * kSampItems;
  int c = 0;
#pragma unroll
  for (int j = 0; j < kSampItems; ++j)
    if (base + j < m) c += keep[base + j];
  c = __reduce_add_sync(kFull, c);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t s = 0;
    for (int w = 0; w < kThreads / 32; ++w) s += wsum[w];
    tile_cnt[blockIdx.x] = s;
  }
}

// Kept edges in increasing canonical index: pairs (u, v), u < v, and w_e.
__global__ void k_flag_write(const int32_t* __restrict__ col, const int64_t* __restrict__ up_ptr,
                             const int64_t* __restrict__ edge_off, const int32_t* __restrict__ vw,
                             int64_t n, int64_t m, const uint8_t* __restrict__ keep,
                             const int64_t* __restrict__ tile_off, int32_t* __restrict__ pairs,
                             int32_t* __restrict__ pw) {
  __shared__ int wsum[kThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kSampTile + (int64_t)threadIdx.x * kSampItems;
  unsigned bits = 0;
#pragma unroll
  for (int j = 0; j < kSampItems; ++j)
    if (base + j < m && keep[base + j]) bits |= 1u << j;
  const int c = __popc(bits);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = c;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(kFull, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  int before = 0;
  for (int w = 0; w < warp; ++w) before += wsum[w];
  int64_t pos = tile_off[blockIdx.x] + before + x - c;
  while (bits) {
    const int j = __ffs(bits) - 1;
    bits &= bits - 1;
    const int64_t i = base + j;
    int64_t lo = 0, len = n;  // row owning canonical edge i
    while (len > 1) {
      const int64_t half = len >> 1;
      lo = (edge_off[lo + half] <= i) ? lo + half : lo;
      len -= half;
    }
    const int32_t v = col[up_ptr[lo] + (i - edge_off[lo])];
    pairs[2 * pos] = (int32_t)lo;
    pairs[2 * pos + 1] = v;
    if (pw != nullptr) pw[pos] = edge_weight(vw, (int32_t)lo, v);
    ++pos;
  }
}

// ------------------------------------------------------------------ fixed size

// Histogram of one radix digit of the 53-bit sampler keys, over the edges
// whose key agrees with `prefix` on the bits above `shift + bits`.
constexpr int kSelBins = 2048;

__global__ void k_key_hist(int64_t m, uint64_t seed, uint64_t prefix, int above, int shift,
                           int bits, unsigned long long* __restrict__ hist) {
  __shared__ unsigned int h[kSelBins];
  for (int b = threadIdx.x; b < kSelBins; b += blockDim.x) h[b] = 0;
  __syncthreads();
  const uint64_t dmask = ((uint64_t)1 << bits) - 1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t key = splitmix(seed ^ splitmix((uint64_t)i)) >> 11;
    if (above >= 53 || (key >> above) == prefix) atomicAdd(h + ((key >> shift) & dmask), 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < (1 << bits); b += blockDim.x)
    if (h[b]) atomicAdd(hist + b, (unsigned long long)h[b]);
}

// Indices of the edges whose key equals T (ties of the order statistic).
__global__ void k_key_ties(int64_t m, uint64_t seed, uint64_t T, int64_t cap,
                           int64_t* __restrict__ out, unsigned long long* __restrict__ cnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    if ((splitmix(seed ^ splitmix((uint64_t)i)) >> 11) == T) {
      const unsigned long long at = atomicAdd(cnt, 1ull);
      if ((int64_t)at < cap) out[at] = i;
    }
  }
}

// keep[i]: (key, i) among the k_hi smallest and not among the k_lo
// smallest; each set is {key < T} plus {key == T, i <= i_cut}.
__global__ void k_fixed_flags(int64_t m, uint64_t seed, uint64_t T_lo, int64_t cut_lo,
                              uint64_t T_hi, int64_t cut_hi, uint8_t* __restrict__ keep) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t key = splitmix(seed ^ splitmix((uint64_t)i)) >> 11;
    const bool in_hi = key < T_hi || (key == T_hi && i <= cut_hi);
    const bool in_lo = key < T_lo || (key == T_lo && i <= cut_lo);
    keep[i] = (in_hi && !in_lo) ? 1 : 0;
  }
}

// ------------------------------------------------------------------ HT fold

// Largest and smallest edge weight of a sampled list ([0] max, [1] min).
__global__ void k_pair_weight_range(const int2* __restrict__ uv, int64_t K,
                                    const int32_t* __restrict__ vw,
                                    unsigned long long* __restrict__ out) {
  unsigned long long mx = 0, mn = ~0ull;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < K;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int2 pr = uv[e];
    const int32_t w = edge_weight(vw, pr.x, pr.y);
    const unsigned long long ww = w < 0 ? 0ull : (unsigned long long)w;
    mx = ww > mx ? ww : mx;
    mn = ww < mn ? ww : mn;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long a = __shfl_xor_sync(kFull, mx, o);
    const unsigned long long b = __shfl_xor_sync(kFull, mn, o);
    mx = a > mx ? a : mx;
    mn = b < mn ? b : mn;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, mx);
    atomicMin(out + 1, mn);
  }
}

// Per-edge numerators (order 3, 4, 7, 8, 9, 10, 11, 12) and their squares
// added to the edge's weight class as four 32-bit limbs per 128-bit value
// (exact for fewer than 2^32 edges).
__global__ void __launch_bounds__(kThreads)
    k_fold_class(const int64_t* __restrict__ row_ptr, const int2* __restrict__ uv, int64_t K,
                 const unsigned long long* __restrict__ t, const unsigned long long* __restrict__ k2,
                 const unsigned long long* __restrict__ q, const int32_t* __restrict__ vw,
                 unsigned long long* __restrict__ limbs) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < K;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int2 pr = uv[e];
    const i128 du = __ldg(row_ptr + pr.x + 1) - __ldg(row_ptr + pr.x);
    const i128 dv = __ldg(row_ptr + pr.y + 1) - __ldg(row_ptr + pr.y);
    const i128 tt = (i128)t[e];
    const i128 kk = k2 != nullptr ? (i128)k2[e] : 0;
    const i128 qq = q != nullptr ? (i128)(long long)q[e] : 0;
    const i128 a = du - 1 - tt, b = dv - 1 - tt;
    const i128 n8 = tt * (tt - 1) / 2 - kk;
    i128 N[8];
    N[0] = tt;
    N[1] = a + b;
    N[2] = kk;
    N[3] = n8;
    N[4] = tt * (a + b) - 4 * n8;
    N[5] = qq;
    N[6] = 2 * (a * (a - 1) / 2 + b * (b - 1) / 2) - tt * (a + b) + 4 * n8;
    N[7] = a * b - qq;
    unsigned long long* dst = limbs + (int64_t)edge_weight(vw, pr.x, pr.y) * 64;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const u128 s = (u128)N[i];
      const u128 mg = (u128)(N[i] < 0 ? -N[i] : N[i]);
      const u128 sq = mg * mg;
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const unsigned long long a1 = (unsigned long long)((s >> (32 * l)) & 0xffffffffu);
        const unsigned long long a2 = (unsigned long long)((sq >> (32 * l)) & 0xffffffffu);
        if (a1) atomicAdd(dst + i * 4 + l, a1);
        if (a2) atomicAdd(dst + (8 + i) * 4 + l, a2);
      }
    }
  }
}

}  // namespace
}  // namespace gs

using namespace gs;

namespace {

u128 limb_value(const unsigned long long* l) {
  u128 s = 0;
  for (int j = 0; j < 4; ++j) s += (u128)l[j] << (32 * j);
  return s;
}

double i128_to_double(u128 v) {  // two's complement
  return (v >> 127) ? -(double)(u128)(-(i128)v) : (double)v;
}

}  // namespace

extern "C" gs_status gs_core_numbers(const gs_graph* gr, gs_workspace* ws, int32_t* d_core,
                                     int32_t* h_max_core, void* stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (gr == nullptr || ws == nullptr || (d_core == nullptr && gr->dev.n > 0)) {
    set_error("gs_core_numbers: invalid arguments");
    return GS_EINVAL;
  }
  const int64_t n = gr->dev.n;
  if (h_max_core) *h_max_core = 0;
  if (n == 0) return GS_OK;
  void* base = nullptr;
  GS_TRY(ws_reserve(ws, 0,
                    Carve::bytes_for<int32_t>(n) * 3 + Carve::bytes_for<unsigned long long>(8),
                    stream, &base));
  Carve c{(char*)base, 0};
  int32_t* deg = c.take<int32_t>(n);
  int32_t* fa = c.take<int32_t>(n);
  int32_t* fb = c.take<int32_t>(n);
  unsigned long long* ctr = c.take<unsigned long long>(8);
  k_core_init<<<grid_for(n, kThreads, 8), kThreads, 0, stream>>>(gr->dev.row_ptr, n, deg, d_core);
  int64_t removed = 0, launches = 1;
  int32_t k = 0, kmax = 0;
  while (removed < n) {
    const unsigned long long init[3] = {0ull, ~0ull, 0ull};
    GS_CUDA(cudaMemcpyAsync(ctr, init, sizeof(init), cudaMemcpyHostToDevice, stream));
    k_core_scan<<<grid_for(n, kThreads, 8), kThreads, 0, stream>>>(n, k, deg, d_core, fa, ctr);
    ++launches;
    unsigned long long h[2];
    GS_CUDA(cudaMemcpyAsync(h, ctr, sizeof(h), cudaMemcpyDeviceToHost, stream));
    GS_CUDA(cudaStreamSynchronize(stream));
    int64_t fsize = (int64_t)h[0];
    if (fsize == 0) {
      if (h[1] == ~0ull) break;  // nothing remains
      k = (int32_t)h[1];          // no vertex of degree <= k left: jump
      continue;
    }
    kmax = k;
    int32_t* cur = fa;
    int32_t* nxt = fb;
    while (fsize > 0) {
      removed += fsize;
      GS_CUDA(cudaMemsetAsync(ctr + 2, 0, sizeof(unsigned long long), stream));
      k_core_peel<<<grid_for(fsize * 32, kThreads, 8), kThreads, 0, stream>>>(
          gr->dev.row_ptr, gr->dev.col, k, cur, fsize, deg, d_core, nxt, ctr + 2);
      ++launches;
      unsigned long long ns = 0;
      GS_CUDA(cudaMemcpyAsync(&ns, ctr + 2, sizeof(ns), cudaMemcpyDeviceToHost, stream));
      GS_CUDA(cudaStreamSynchronize(stream));
      fsize = (int64_t)ns;
      int32_t* tsw = cur;
      cur = nxt;
      nxt = tsw;
    }
    ++k;
  }
  GS_CUDA(cudaGetLastError());
  ws->launches_total += launches;
  if (h_max_core) *h_max_core = kmax;
  return GS_OK;
}

extern "C" gs_status gs_sample_weighted(const gs_graph* gr, gs_workspace* ws,
                                        const int32_t* d_vertex_w, double fraction,
                                        uint64_t seed, int32_t* d_pairs, int32_t* d_pair_w,
                                        int64_t max_k, int64_t* k_out, double* scale_out,
                                        void* stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (gr == nullptr || ws == nullptr || d_vertex_w == nullptr || d_pairs == nullptr ||
      k_out == nullptr || max_k < 0 || !(fraction >= 0.0 && fraction <= 1.0)) {
    set_error("gs_sample_weighted: invalid arguments (fraction must lie in [0, 1])");
    return GS_EINVAL;
  }
  *k_out = 0;
  if (scale_out) *scale_out = 0.0;
  const int64_t n = gr->dev.n, m = gr->m;
  if (m == 0) return GS_OK;
  const int64_t tiles = (m + kSampTile - 1) / kSampTile;
  const size_t bytes = Carve::bytes_for<unsigned long long>(8) + Carve::bytes_for<uint8_t>(m) +
                       Carve::bytes_for<int64_t>(tiles + 1) * 2 +
                       Carve::bytes_for<int64_t>(scan_tmp_elems(tiles));
  void* base = nullptr;
  GS_TRY(ws_reserve(ws, 0, bytes, stream, &base));
  Carve c{(char*)base, 0};
  unsigned long long* acc = c.take<unsigned long long>(8);
  uint8_t* keep = c.take<uint8_t>(m);
  int64_t* cnt = c.take<int64_t>(tiles + 1);
  int64_t* off = c.take<int64_t>(tiles + 1);
  int64_t* tmp = c.take<int64_t>(scan_tmp_elems(tiles));
  GS_CUDA(cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 8, stream));
  k_weight_sum<<<grid_for(n * 32, kThreads, 8), kThreads, 0, stream>>>(
      gr->dev.row_ptr, gr->dev.col, gr->up_ptr, d_vertex_w, n, acc);
  unsigned long long h[2];
  GS_CUDA(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, stream));
  GS_CUDA(cudaStreamSynchronize(stream));
  if (h[1] != 0 || h[0] == 0) {
    set_error("gs_sample_weighted: vertex weights must be >= 0 and some edge weight > 0");
    return GS_EINVAL;
  }
  const double scale = fraction * (double)m / (double)h[0];
  if (scale_out) *scale_out = scale;
  k_weighted_flags<<<grid_for(n * 32, kThreads, 8), kThreads, 0, stream>>>(
      gr->dev.row_ptr, gr->dev.col, gr->up_ptr, gr->edge_off, d_vertex_w, n, scale, seed, keep);
  k_flag_count<<<(unsigned)tiles, kThreads, 0, stream>>>(keep, m, cnt);
  GS_TRY(exclusive_scan_i64(cnt, off, tiles, tmp, stream));
  int64_t kept = 0;
  GS_CUDA(cudaMemcpyAsync(&kept, off + tiles, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
  GS_CUDA(cudaStreamSynchronize(stream));
  *k_out = kept;
  ws->launches_total += 6;
  if (kept > max_k) {
    set_error("gs_sample_weighted: %lld edges kept but the output holds %lld", (long long)kept,
              (long long)max_k);
    return GS_ECAPACITY;
  }
  if (kept > 0) {
    k_flag_write<<<(unsigned)tiles, kThreads, 0, stream>>>(gr->dev.col, gr->up_ptr, gr->edge_off,
                                                           d_vertex_w, n, m, keep, off, d_pairs,
                                                           d_pair_w);
    ws->launches_total += 1;
  }
  GS_CUDA(cudaGetLastError());
  GS_CUDA(cudaStreamSynchronize(stream));
  return GS_OK;
}

extern "C" gs_status gs_count_weighted(const gs_graph* gr, gs_workspace* ws,
                                       const int32_t* d_pairs, int64_t K,
                                       const int32_t* d_vertex_w, double scale, uint32_t mask,
                                       double z, gs_result* out, void* stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (gr == nullptr || ws == nullptr || out == nullptr || d_vertex_w == nullptr || K < 0 ||
      (K > 0 && d_pairs == nullptr) || !(scale > 0.0) || !(z >= 0.0) || mask == 0 ||
      (mask & ~(uint32_t)GS_CONNECTED) != 0) {
    set_error("gs_count_weighted: invalid arguments (scale > 0, mask a non-empty subset of "
              "GS_CONNECTED)");
    return GS_EINVAL;
  }
  memset(out, 0, sizeof(*out));
  static const uint32_t bit[8] = {GS_G3, GS_G4, GS_G7, GS_G8, GS_G9, GS_G10, GS_G11, GS_G12};
  static const int D[8] = {3, 2, 6, 1, 2, 4, 6, 1};
  for (int i = 0; i < 8; ++i)
    if (mask & bit[i]) out->flags[i] = GS_F_COMPUTED;
  if (K == 0) return GS_OK;
  CountBufs b;
  const Tuning tu = ws->has_tuning ? ws->tuning : default_tuning();
  GS_TRY(count_run(gr, ws, d_pairs, K, mask, true, nullptr, nullptr, 0, tu, b, stream,
                   "gs_count_weighted"));
  // weight classes present
  void* base = nullptr;
  GS_TRY(ws_reserve(ws, 3, Carve::bytes_for<unsigned long long>(8), stream, &base));
  unsigned long long* range = (unsigned long long*)base;
  const unsigned long long init[2] = {0ull, ~0ull};
  GS_CUDA(cudaMemcpyAsync(range, init, sizeof(init), cudaMemcpyHostToDevice, stream));
  k_pair_weight_range<<<grid_for(K, kThreads, 4), kThreads, 0, stream>>>(b.uv, K, d_vertex_w,
                                                                          range);
  unsigned long long hr[2];
  GS_CUDA(cudaMemcpyAsync(hr, range, sizeof(hr), cudaMemcpyDeviceToHost, stream));
  GS_CUDA(cudaStreamSynchronize(stream));
  if (hr[1] == 0 || (int64_t)hr[0] >= kMaxClasses) {
    set_error("gs_count_weighted: every sampled edge needs a weight in [1, 2^22) (pi_e > 0)");
    return GS_EINVAL;
  }
  const int64_t classes = (int64_t)hr[0] + 1;
  GS_TRY(ws_reserve(ws, 3, Carve::bytes_for<unsigned long long>(classes * 64), stream, &base));
  unsigned long long* limbs = (unsigned long long*)base;
  GS_CUDA(cudaMemsetAsync(limbs, 0, sizeof(unsigned long long) * classes * 64, stream));
  const bool four = (mask & (GS_G7 | GS_G8 | GS_G9 | GS_G10 | GS_G11 | GS_G12)) != 0;
  k_fold_class<<<grid_for(K, kThreads, 4), kThreads, 0, stream>>>(
      gr->dev.row_ptr, b.uv, K, b.t, four ? b.k2 : nullptr, four ? b.q : nullptr, d_vertex_w,
      limbs);
  GS_CUDA(cudaGetLastError());
  ws->launches_total += 3;
  const int64_t lo = (int64_t)hr[1];
  // classes [lo, classes) back to the host
  unsigned long long* h = new unsigned long long[(size_t)(classes - lo) * 64];
  cudaError_t ce = cudaMemcpyAsync(h, limbs + lo * 64,
                                   sizeof(unsigned long long) * (size_t)(classes - lo) * 64,
                                   cudaMemcpyDeviceToHost, stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(stream);
  if (ce != cudaSuccess) {
    delete[] h;
    return cuda_fail(ce, "gs_count_weighted readback", __FILE__, __LINE__);
  }
  double X[8] = {0}, V[8] = {0};
  bool all_one = K == gr->m;
  for (int64_t c = lo; c < classes; ++c) {
    const unsigned long long* cl = h + (c - lo) * 64;
    bool any = false;
    for (int j = 0; j < 64 && !any; ++j) any = cl[j] != 0;
    if (!any) continue;
    double pi = scale * (double)c;
    if (pi > 1.0) pi = 1.0;
    if (pi < 1.0) all_one = false;
    for (int i = 0; i < 8; ++i) {
      const double s = i128_to_double(limb_value(cl + i * 4));
      const double s2 = (double)limb_value(cl + (8 + i) * 4);
      X[i] += s / pi;
      V[i] += (1.0 - pi) * s2 / (pi * pi);
    }
  }
  // exact integer totals when every edge was kept with pi = 1
  for (int i = 0; i < 8; ++i) {
    if (!(mask & bit[i])) continue;
    out->x[i] = X[i] / D[i];
    out->var[i] = V[i] / ((double)D[i] * D[i]);
    const double half = z * sqrt(out->var[i]);
    out->lb[i] = out->x[i] - half;
    out->ub[i] = out->x[i] + half;
    if (all_one) {
      u128 tot = 0;
      for (int64_t c = lo; c < classes; ++c) tot += limb_value(h + (c - lo) * 64 + i * 4);
      const i128 st = (i128)tot;
      if (st >= 0 && st % D[i] == 0 && st / D[i] <= (i128)UINT64_MAX) {
        out->exact[i] = (uint64_t)(st / D[i]);
        out->flags[i] |= GS_F_EXACT;
      }
    }
  }
  delete[] h;
  return GS_OK;
}

namespace gs {

// Boundary of the k smallest (key, i) of the sampler keys: the set is
// {key < T} plus {key == T, i <= i_cut}; k = 0 gives the empty set.
struct RankCut {
  uint64_t T;
  int64_t i_cut;
};

static gs_status rank_cut(const gs_graph* gr, int64_t k, uint64_t seed,
                          unsigned long long* hist, int64_t* ties, int64_t tie_cap,
                          int64_t* launches, RankCut* out, cudaStream_t stream) {
  const int64_t m = gr->m;
  if (k <= 0) {
    *out = RankCut{0, -1};
    return GS_OK;
  }
  // order statistic: the k-th smallest key T, five digits from the top
  uint64_t prefix = 0;
  int above = 53;
  int64_t rank = k - 1;  // 0-based rank of T among the keys with this prefix
  static const int kDigits[5] = {11, 11, 11, 10, 10};
  int64_t tie_count = 0;
  std::vector<unsigned long long> h(kSelBins);
  for (int d = 0; d < 5; ++d) {
    const int bits = kDigits[d], shift = above - bits;
    GS_CUDA(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * kSelBins, stream));
    k_key_hist<<<grid_for(m, kThreads, 4), kThreads, 0, stream>>>(m, seed, prefix, above, shift,
                                                                   bits, hist);
    ++*launches;
    GS_CUDA(cudaMemcpyAsync(h.data(), hist, sizeof(unsigned long long) << bits,
                            cudaMemcpyDeviceToHost, stream));
    GS_CUDA(cudaStreamSynchronize(stream));
    int64_t accum = 0;
    int b = 0;
    for (; b < (1 << bits); ++b) {
      if (accum + (int64_t)h[b] > rank) break;
      accum += (int64_t)h[b];
    }
    if (b == (1 << bits)) {
      set_error("sampler key selection lost its rank");
      return GS_ECUDA;
    }
    rank -= accum;
    prefix = (prefix << bits) | (uint64_t)b;
    above = shift;
    tie_count = (int64_t)h[b];
  }
  int64_t i_cut = m;  // every tie kept
  if (rank + 1 < tie_count) {
    if (tie_count > tie_cap) {
      set_error("%lld sampler keys tie at the cut", (long long)tie_count);
      return GS_ECAPACITY;
    }
    GS_CUDA(cudaMemsetAsync(hist + kSelBins, 0, sizeof(unsigned long long), stream));
    k_key_ties<<<grid_for(m, kThreads, 4), kThreads, 0, stream>>>(m, seed, prefix, tie_cap, ties,
                                                                   hist + kSelBins);
    ++*launches;
    std::vector<int64_t> ht((size_t)tie_count);
    GS_CUDA(cudaMemcpyAsync(ht.data(), ties, sizeof(int64_t) * (size_t)tie_count,
                            cudaMemcpyDeviceToHost, stream));
    GS_CUDA(cudaStreamSynchronize(stream));
    std::sort(ht.begin(), ht.end());
    i_cut = ht[(size_t)rank];
  }
  *out = RankCut{prefix, i_cut};
  return GS_OK;
}

// Edges ranked [k_lo, k_hi) by (key, i), in increasing canonical index,
// into d_pairs (device int32[2 (k_hi - k_lo)]) or, when d_pairs is NULL,
// into workspace slot 3 (*pairs_out).
gs_status sample_ranks(const gs_graph* gr, gs_workspace* ws, int64_t k_lo, int64_t k_hi,
                       uint64_t seed, int32_t* d_pairs, int32_t** pairs_out,
                       cudaStream_t stream) {
  const int64_t n = gr->dev.n, m = gr->m;
  if (pairs_out) *pairs_out = d_pairs;
  if (k_hi <= k_lo) return GS_OK;
  constexpr int64_t kTieCap = 1 << 16;
  const int64_t tiles = (m + kSampTile - 1) / kSampTile;
  const size_t bytes = Carve::bytes_for<unsigned long long>(kSelBins + 8) +
                       Carve::bytes_for<int64_t>(kTieCap) + Carve::bytes_for<uint8_t>(m) +
                       Carve::bytes_for<int64_t>(tiles + 1) * 2 +
                       Carve::bytes_for<int64_t>(scan_tmp_elems(tiles));
  void* base = nullptr;
  GS_TRY(ws_reserve(ws, 2, bytes, stream, &base));
  Carve c{(char*)base, 0};
  unsigned long long* hist = c.take<unsigned long long>(kSelBins + 8);
  int64_t* ties = c.take<int64_t>(kTieCap);
  uint8_t* keep = c.take<uint8_t>(m);
  int64_t* cnt = c.take<int64_t>(tiles + 1);
  int64_t* off = c.take<int64_t>(tiles + 1);
  int64_t* tmp = c.take<int64_t>(scan_tmp_elems(tiles));
  int64_t launches = 0;
  RankCut lo, hi;
  GS_TRY(rank_cut(gr, k_lo, seed, hist, ties, kTieCap, &launches, &lo, stream));
  GS_TRY(rank_cut(gr, k_hi, seed, hist, ties, kTieCap, &launches, &hi, stream));
  if (d_pairs == nullptr) {
    void* b3 = nullptr;
    GS_TRY(ws_reserve(ws, 3, Carve::bytes_for<int32_t>(2 * (k_hi - k_lo)), stream, &b3));
    d_pairs = (int32_t*)b3;
    if (pairs_out) *pairs_out = d_pairs;
  }
  k_fixed_flags<<<grid_for(m, kThreads, 8), kThreads, 0, stream>>>(m, seed, lo.T, lo.i_cut, hi.T,
                                                                    hi.i_cut, keep);
  k_flag_count<<<(unsigned)tiles, kThreads, 0, stream>>>(keep, m, cnt);
  GS_TRY(exclusive_scan_i64(cnt, off, tiles, tmp, stream));
  k_flag_write<<<(unsigned)tiles, kThreads, 0, stream>>>(gr->dev.col, gr->up_ptr, gr->edge_off,
                                                         nullptr, n, m, keep, off, d_pairs,
                                                         nullptr);
  launches += 6;
  int64_t kept = 0;
  GS_CUDA(cudaMemcpyAsync(&kept, off + tiles, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
  GS_CUDA(cudaStreamSynchronize(stream));
  ws->launches_total += launches;
  if (kept != k_hi - k_lo) {
    set_error("sampler: selected %lld edges instead of %lld", (long long)kept,
              (long long)(k_hi - k_lo));
    return GS_ECUDA;
  }
  return GS_OK;
}

}  // namespace gs

extern "C" gs_status gs_sample_fixed(const gs_graph* gr, gs_workspace* ws, int64_t k,
                                     uint64_t seed, int32_t* d_pairs, void* stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (gr == nullptr || ws == nullptr || k < 0 || k > gr->m || (k > 0 && d_pairs == nullptr)) {
    set_error("gs_sample_fixed: invalid arguments (need 0 <= k <= m and an output)");
    return GS_EINVAL;
  }
  return sample_ranks(gr, ws, 0, k, seed, d_pairs, nullptr, stream);
}

extern "C" gs_status gs_sample_ranks(const gs_graph* gr, gs_workspace* ws, int64_t k_lo,
                                     int64_t k_hi, uint64_t seed, int32_t* d_pairs,
                                     void* stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (gr == nullptr || ws == nullptr || k_lo < 0 || k_hi < k_lo || k_hi > gr->m ||
      (k_hi > k_lo && d_pairs == nullptr)) {
    set_error("gs_sample_ranks: invalid arguments (need 0 <= k_lo <= k_hi <= m and an output)");
    return GS_EINVAL;
  }
  return sample_ranks(gr, ws, k_lo, k_hi, seed, d_pairs, nullptr, stream);
}
