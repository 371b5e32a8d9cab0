// Algorithm 7 (micro-level estimation): per sampled edge e = (u, v) the
// vector x3..x17 of the paper's micro-level graphlet statistics, from
// ceil(d_w p_e) probes of N(w) for every w in the edge's neighbourhood.
//
// For e with d_u <= d_v (ties: smaller id is u), T = N(u) cap N(v),
// S_u = N(u) \ {v} \ T, S_v = N(v) \ {u} \ T. Each w of T, S_u and S_v
// reads a circular window of c_w = ceil(d_w p_e) consecutive entries of
// N(w) from the offset o_w = floor(h d_w / 2^64), h = sm(sm(seed ^ sm(key))
// ^ w), key = (min(u,v) << 32) | max(u,v), sm the SplitMix64 output
// function. A probe r counts, weighted d_w / c_w,
//   w in T:    r in T, r > w                    -> x7 (4-cliques)
//   w in S_u:  r in S_v                         -> x10 (4-cycles)
//              r in S_u, r > w                  -> x9 (tailed triangles)
//              r in T                           -> omega
//   w in S_v:  r in S_v, r > w                  -> x9
//              r in T                           -> omega
// ("r > w": each unordered pair inside a set counts once, from its smaller
// member, as the algorithm's label resets do). The remaining statistics
// follow from t, a = |S_u|, b = |S_v|, R = n - 2 - t - a - b:
//   x3 = t, x4 = a + b, x5 = R, x6 = C(n,3) - x3 - x4 - x5, x8 = C(t,2) - x7,
//   x11 = C(a,2) + C(b,2) - x9, x12 = a b - x10, x13 = t R, x14 = (a+b) R,
//   x15 = m - (t + d_u + d_v + 1) - omega, x16 = C(R,2),
//   x17 = C(n,4) - (x7 + ... + x16).
//
// GPU structure (same flattening as the 4-node pass of count.cu):
//   prep    k_prep of count.cu: orientation, edge check, duplicate check.
//   chunks  the two lists N(u), N(v) of every edge are cut into chunks of
//           32 positions (each list padded to 32); one warp per chunk
//           classifies its positions (T, S_u, S_v or none) with one
//           membership test each, counts t and the chunk's probes, and
//           turns them into tasks of kTaskProbes probes.
//   probe   tasks are split evenly over all warps; lanes take consecutive
//           probes of a task and find their item by a search over the
//           warp's scanned probe counts (item descriptors in shared
//           memory); a probe costs one or two membership tests (in N(u),
//           in N(v)).
//   final   one thread per edge writes the 15 statistics and keeps the
//           column maxima (the extremal statistics of Sec. 7).
// Weighted hits are accumulated exactly: weight d_w / c_w = q + f / 2^64
// with q = floor(d_w / c_w), f = floor((d_w mod c_w) 2^64 / c_w), per edge
// and statistic an integer part and a 128-bit fraction part, added with
// integer atomics (so the result does not depend on the order of the work)
// and converted to FP64 once. At p_e = 1 every weight is 1 and the
// statistics are exact integers.
#include <math.h>
#include <string.h>

#include "common.cuh"

namespace gs {

// count.cu: orientation (u = smaller degree), edge and duplicate checks,
// len[e] = d_u (pad = 0).
__global__ void k_prep(DevGraph g, const int32_t* __restrict__ pairs, int64_t K, int pad,
                       unsigned long long* __restrict__ dup_table, int64_t dup_mask,
                       int2* __restrict__ uv, int64_t* __restrict__ len, DevError* err);

namespace {

constexpr int kThreads = 256;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kProbeBlocksPerSm = 4;
constexpr int64_t kTaskProbes = 512;
constexpr int kCats = 4;   // x7, x9, x10, omega
constexpr int kCols = 15;  // x3 .. x17
constexpr int kNone = 0, kT = 1, kSu = 2, kSv = 3;

typedef unsigned __int128 u128;

__device__ __forceinline__ uint64_t splitmix(uint64_t x) {
  uint64_t z = x + 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ int64_t probes_of(int64_t d, double pe) {
  return (int64_t)ceil((double)d * pe);
}

__device__ __forceinline__ int64_t last_le64(const int64_t* __restrict__ off, int64_t count,
                                             int64_t p) {
  int64_t lo = 0, len = count;
  while (len > 1) {
    int64_t half = len >> 1;
    lo = (__ldg(off + lo + half) <= p) ? lo + half : lo;
    len -= half;
  }
  return lo;
}

// Per-edge set-up: chunk counts of the two lists.
__global__ void k_micro_chunks(const int64_t* __restrict__ row_ptr, const int2* __restrict__ uv,
                               int64_t K, int64_t* __restrict__ nch,
                               unsigned long long* __restrict__ t,
                               unsigned long long* __restrict__ acc) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < K;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int2 pr = uv[e];
    const int64_t du = __ldg(row_ptr + pr.x + 1) - __ldg(row_ptr + pr.x);
    const int64_t dv = __ldg(row_ptr + pr.y + 1) - __ldg(row_ptr + pr.y);
    nch[e] = ((du + 31) >> 5) + ((dv + 31) >> 5);
    t[e] = 0;
#pragma unroll
    for (int i = 0; i < 3 * kCats; ++i) acc[e * 3 * kCats + i] = 0;
  }
}

// Edge of every chunk. One warp per edge.
__global__ void k_micro_fill(const int64_t* __restrict__ choff, int64_t K,
                             int64_t* __restrict__ chunk_e) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < K; e += warps)
    for (int64_t c = choff[e] + lane; c < choff[e + 1]; c += 32) chunk_e[c] = e;
}

// Where chunk c of edge e lies: list owner (u side: N(u), else N(v)) and
// the first position.
struct ChunkAt {
  int32_t u, v, owner, other;
  int64_t bu, du, bv, dv, bo, dow, bx, dx;  // (bo, dow): owner list, (bx, dx): other's
  int64_t first;
  bool vside;
};

__device__ __forceinline__ ChunkAt chunk_at(const DevGraph& g, const int2* __restrict__ uv,
                                            const int64_t* __restrict__ choff, int64_t e,
                                            int64_t c) {
  ChunkAt a;
  const int2 pr = uv[e];
  a.u = pr.x;
  a.v = pr.y;
  a.bu = __ldg(g.row_ptr + a.u);
  a.du = __ldg(g.row_ptr + a.u + 1) - a.bu;
  a.bv = __ldg(g.row_ptr + a.v);
  a.dv = __ldg(g.row_ptr + a.v + 1) - a.bv;
  const int64_t lc = c - __ldg(choff + e), cu = (a.du + 31) >> 5;
  a.vside = lc >= cu;
  a.first = (a.vside ? lc - cu : lc) * 32;
  a.owner = a.vside ? a.v : a.u;
  a.other = a.vside ? a.u : a.v;
  a.bo = a.vside ? a.bv : a.bu;
  a.dow = a.vside ? a.dv : a.du;
  a.bx = a.vside ? a.bu : a.bv;
  a.dx = a.vside ? a.du : a.dv;
  return a;
}

// Class of position i of a chunk (one membership test in the other list).
__device__ __forceinline__ int classify(const DevGraph& g, const ChunkAt& a, int64_t i,
                                        int32_t* w_out) {
  if (i >= a.dow) return kNone;
  const int32_t w = __ldg(g.col + a.bo + i);
  *w_out = w;
  if (w == a.other) return kNone;
  const int32_t xs = g.col_hm != nullptr ? (int32_t)__ldg(g.col_hm + a.bo + i) : kNoSlotInfo;
  const bool both = adj_contains(g, a.other, a.bx, a.dx, w, xs);
  if (!a.vside) return both ? kT : kSu;
  return both ? kNone : kSv;  // T members are handled from the u side
}

// Classes, t and probe counts per chunk; tasks per chunk.
__global__ void __launch_bounds__(kThreads)
    k_micro_items(DevGraph g, const int2* __restrict__ uv, const int64_t* __restrict__ choff,
                  const int64_t* __restrict__ chunk_e, int64_t C, double pe,
                  unsigned long long* __restrict__ t, uint32_t* __restrict__ tmask,
                  int64_t* __restrict__ task_cnt, unsigned long long* __restrict__ stats) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  unsigned long long probes = 0;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < C; c += warps) {
    const int64_t e = chunk_e[c];
    const ChunkAt a = chunk_at(g, uv, choff, e, c);
    int32_t w = 0;
    const int cls = classify(g, a, a.first + lane, &w);
    int64_t cost = 0;
    if (cls != kNone) cost = probes_of(__ldg(g.row_ptr + w + 1) - __ldg(g.row_ptr + w), pe);
    const unsigned inT = __ballot_sync(kFull, cls == kT);
    const unsigned live = __ballot_sync(kFull, cls != kNone);
    int64_t total = cost;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(kFull, total, o);
    if (lane == 0) {
      tmask[2 * c] = inT;
      tmask[2 * c + 1] = live;
      task_cnt[c] = (total + kTaskProbes - 1) / kTaskProbes;
      if (inT) atomicAdd(t + e, (unsigned long long)__popc(inT));
      probes += (unsigned long long)total;
    }
  }
  if (lane == 0 && probes) atomicAdd(stats, probes);
}

struct ItemDesc {  // one lane's item, in shared memory for the probe loop
  int64_t bw, dw, o;
  uint64_t q, f;
  int32_t w, cls;
};

// Adds a 64-bit integer part and a 128-bit fraction to an edge's
// accumulator {I, F_lo, F_hi} with integer atomics (exact, order-free).
__device__ __forceinline__ void acc_add(unsigned long long* a, unsigned long long I, u128 F) {
  if (I) atomicAdd(a, I);
  const unsigned long long lo = (unsigned long long)F, hi = (unsigned long long)(F >> 64);
  if (lo) {
    const unsigned long long old = atomicAdd(a + 1, lo);
    if (old + lo < old) atomicAdd(a + 2, 1ull);
  }
  if (hi) atomicAdd(a + 2, hi);
}

__device__ __forceinline__ u128 shfl_xor_u128(u128 v, int o) {
  unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
  lo = __shfl_xor_sync(kFull, lo, o);
  hi = __shfl_xor_sync(kFull, hi, o);
  return ((u128)hi << 64) | lo;
}

struct Hits {
  unsigned long long I[kCats];
  u128 F[kCats];
};

__device__ __forceinline__ void flush_hits(Hits& h, unsigned long long* __restrict__ acc_e,
                                           int lane) {
#pragma unroll
  for (int k = 0; k < kCats; ++k) {
    unsigned long long I = h.I[k];
    u128 F = h.F[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      I += __shfl_xor_sync(kFull, I, o);
      F += shfl_xor_u128(F, o);
    }
    if (lane == 0 && (I || F)) acc_add(acc_e + 3 * k, I, F);
    h.I[k] = 0;
    h.F[k] = 0;
  }
}

__global__ void __launch_bounds__(kThreads, kProbeBlocksPerSm)
    k_micro_probe(const __grid_constant__ DevGraph g, const int2* __restrict__ uv,
                  const int64_t* __restrict__ choff, const int64_t* __restrict__ chunk_e,
                  const uint32_t* __restrict__ tmask, const int64_t* __restrict__ task_off,
                  int64_t C, double pe, uint64_t seed, unsigned long long* __restrict__ acc) {
  __shared__ ItemDesc items[kThreads / 32][32];
  const int lane = threadIdx.x & 31;
  ItemDesc* my = items[threadIdx.x >> 5];
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t NT = __ldg(task_off + C);
  const int64_t per = (NT + warps - 1) / warps;
  const int64_t t0 = warp * per, t1 = min(NT, t0 + per);
  if (t0 >= t1) return;
  int64_t c = last_le64(task_off, C, t0);
  int64_t cur = -1, cur_e = -1;
  int64_t start = 0, ctotal = 0;
  int32_t u = 0, v = 0;
  int64_t bu = 0, du = 0, bv = 0, dv = 0;
  Hits h;
#pragma unroll
  for (int k = 0; k < kCats; ++k) {
    h.I[k] = 0;
    h.F[k] = 0;
  }
  for (int64_t task = t0; task < t1; ++task) {
    while (c + 1 < C && __ldg(task_off + c + 1) <= task) ++c;
    if (c != cur) {
      const int64_t e = chunk_e[c];
      if (cur >= 0 && e != cur_e) flush_hits(h, acc + cur_e * 3 * kCats, lane);
      const ChunkAt a = chunk_at(g, uv, choff, e, c);
      u = a.u;
      v = a.v;
      bu = a.bu;
      du = a.du;
      bv = a.bv;
      dv = a.dv;
      const uint32_t inT = tmask[2 * c], live = tmask[2 * c + 1];
      int64_t mine = 0;
      __syncwarp();
      ItemDesc d;
      d.cls = kNone;
      d.w = 0;
      d.bw = 0;
      d.dw = 1;
      d.o = 0;
      d.q = 0;
      d.f = 0;
      const int64_t i = a.first + lane;
      if ((live >> lane) & 1u) {
        d.w = __ldg(g.col + a.bo + i);
        d.cls = a.vside ? kSv : (((inT >> lane) & 1u) ? kT : kSu);
        d.bw = __ldg(g.row_ptr + d.w);
        d.dw = __ldg(g.row_ptr + d.w + 1) - d.bw;
        mine = probes_of(d.dw, pe);
        const uint64_t key = ((uint64_t)(uint32_t)min(u, v) << 32) | (uint32_t)max(u, v);
        const uint64_t hh = splitmix(splitmix(seed ^ splitmix(key)) ^ (uint64_t)(uint32_t)d.w);
        d.o = (int64_t)__umul64hi(hh, (uint64_t)d.dw);
        d.q = (uint64_t)(d.dw / mine);
        d.f = (uint64_t)((((u128)(uint64_t)(d.dw % mine)) << 64) / (u128)(uint64_t)mine);
      }
      my[lane] = d;
      __syncwarp();
      int64_t incl = mine;
#pragma unroll
      for (int s = 1; s < 32; s <<= 1) {
        const int64_t y = __shfl_up_sync(kFull, incl, s);
        if (lane >= s) incl += y;
      }
      start = incl - mine;
      ctotal = __shfl_sync(kFull, incl, 31);
      cur = c;
      cur_e = e;
    }
    const int64_t lo = (task - __ldg(task_off + c)) * kTaskProbes;
    const int32_t len = (int32_t)min(ctotal - lo, kTaskProbes);
    // item starts relative to the task's first probe, clamped to 32 bits
    // (order kept; the item holding a probe of this task starts less than
    // one item's probes before lo)
    const int32_t srel = (int32_t)max(min(start - lo, kTaskProbes), (int64_t)INT32_MIN + 1);
    for (int32_t r = lane; r - lane < len; r += 32) {
      int j = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int32_t sv = __shfl_sync(kFull, srel, j + step);
        if (sv <= r) j += step;
      }
      const int32_t sj = __shfl_sync(kFull, srel, j);
      if (r >= len) continue;
      const ItemDesc& it = my[j];
      int64_t p = it.o + (int64_t)(r - sj);
      if (p >= it.dw) p -= it.dw;
      const int32_t x = __ldg(g.col + it.bw + p);
      const int32_t xs =
          g.col_hm != nullptr ? (int32_t)__ldg(g.col_hm + it.bw + p) : kNoSlotInfo;
      const bool in_u = adj_contains(g, u, bu, du, x, xs);
      int cat = -1;
      if (it.cls == kT) {
        if (in_u && x > it.w && adj_contains(g, v, bv, dv, x, xs)) cat = 0;
      } else if (x != u && x != v) {
        const bool in_v = adj_contains(g, v, bv, dv, x, xs);
        if (in_u && in_v) cat = 3;                                         // omega
        else if (it.cls == kSu && in_v) cat = 2;                           // 4-cycle
        else if (it.cls == kSu && in_u && x > it.w) cat = 1;               // S_u pair
        else if (it.cls == kSv && in_v && x > it.w) cat = 1;               // S_v pair
      }
      if (cat >= 0) {
#pragma unroll
        for (int k = 0; k < kCats; ++k)
          if (k == cat) {
            h.I[k] += it.q;
            h.F[k] += it.f;
          }
      }
    }
  }
  if (cur >= 0) flush_hits(h, acc + cur_e * 3 * kCats, lane);
}

__device__ __forceinline__ double acc_value(const unsigned long long* a) {
  // I + (F_hi 2^64 + F_lo) / 2^64
  return (double)(a[0] + a[2]) + (double)a[1] * 0x1p-64;
}

struct ColMax {
  double v;
  int64_t i;
};

__device__ __forceinline__ bool better(double v, int64_t i, const ColMax& m) {
  return v > m.v || (v == m.v && i < m.i);
}

// Rows x3..x17 and per-block column maxima (value, smallest edge index).
__global__ void __launch_bounds__(kThreads)
    k_micro_final(const int64_t* __restrict__ row_ptr, const int2* __restrict__ uv, int64_t K,
                  int64_t n, int64_t m, double cn3, double cn4,
                  const unsigned long long* __restrict__ t,
                  const unsigned long long* __restrict__ acc, double* __restrict__ x,
                  ColMax* __restrict__ part) {
  __shared__ ColMax red[kThreads / 32][kCols];
  ColMax best[kCols];
#pragma unroll
  for (int k = 0; k < kCols; ++k) best[k] = ColMax{-INFINITY, INT64_MAX};
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < K;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int2 pr = uv[e];
    const int64_t du = __ldg(row_ptr + pr.x + 1) - __ldg(row_ptr + pr.x);
    const int64_t dv = __ldg(row_ptr + pr.y + 1) - __ldg(row_ptr + pr.y);
    const int64_t tt = (int64_t)t[e], a = du - 1 - tt, b = dv - 1 - tt;
    const int64_t R = n - 2 - tt - a - b;
    const unsigned long long* ac = acc + e * 3 * kCats;
    const double x7 = acc_value(ac), x9 = acc_value(ac + 3), x10 = acc_value(ac + 6);
    const double om = acc_value(ac + 9);
    double r[kCols];
    r[0] = (double)tt;
    r[1] = (double)(a + b);
    r[2] = (double)R;
    r[3] = cn3;  // C(n,3) - t - (a+b) - R = C(n,3) - (n - 2), rounded on the host
    r[4] = x7;
    r[5] = (double)(tt * (tt - 1) / 2) - x7;
    r[6] = x9;
    r[7] = x10;
    r[8] = (double)(a * (a - 1) / 2 + b * (b - 1) / 2) - x9;
    r[9] = (double)(a * b) - x10;
    r[10] = (double)(tt * R);
    r[11] = (double)((a + b) * R);
    r[12] = (double)(m - (tt + du + dv + 1)) - om;
    r[13] = (double)(R * (R - 1) / 2);
    double s = 0.0;
#pragma unroll
    for (int k = 4; k <= 13; ++k) s += r[k];
    r[14] = cn4 - s;
#pragma unroll
    for (int k = 0; k < kCols; ++k) {
      x[e * kCols + k] = r[k];
      if (better(r[k], e, best[k])) best[k] = ColMax{r[k], e};
    }
  }
  if (part == nullptr) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kCols; ++k) {
    ColMax b = best[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(kFull, b.v, o);
      const long long oi = __shfl_xor_sync(kFull, (long long)b.i, o);
      if (better(ov, oi, b)) b = ColMax{ov, oi};
    }
    if (lane == 0) red[wid][k] = b;
  }
  __syncthreads();
  if (threadIdx.x < kCols) {
    ColMax b = red[0][threadIdx.x];
    for (int i = 1; i < kThreads / 32; ++i) {
      const ColMax& c = red[i][threadIdx.x];
      if (better(c.v, c.i, b)) b = c;
    }
    part[(int64_t)blockIdx.x * kCols + threadIdx.x] = b;
  }
}

__global__ void k_micro_max_final(const ColMax* __restrict__ part, int blocks,
                                  ColMax* __restrict__ out) {
  if (threadIdx.x < kCols) {
    ColMax b = part[threadIdx.x];
    for (int i = 1; i < blocks; ++i) {
      const ColMax& c = part[(int64_t)i * kCols + threadIdx.x];
      if (better(c.v, c.i, b)) b = c;
    }
    out[threadIdx.x] = b;
  }
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status gs_micro(const gs_graph* gr, gs_workspace* ws, const int32_t* d_pairs,
                              int64_t K, double p_e, uint64_t seed, double* d_x, double* h_max,
                              int64_t* h_argmax, void* stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (gr == nullptr || ws == nullptr || K < 0 || !(p_e > 0.0 && p_e <= 1.0) ||
      (K > 0 && (d_pairs == nullptr || d_x == nullptr))) {
    set_error("gs_micro: invalid arguments (need 0 < p_e <= 1, device pairs and output)");
    return GS_EINVAL;
  }
  memset(&ws->stats, 0, sizeof(ws->stats));
  ws->stats.k = K;
  if (h_max != nullptr)
    for (int k = 0; k < kCols; ++k) h_max[k] = NAN;
  if (h_argmax != nullptr)
    for (int k = 0; k < kCols; ++k) h_argmax[k] = -1;
  if (K == 0) return GS_OK;
  const DevGraph& g = gr->dev;
  const int64_t n = g.n, m = gr->m;
  // C(n,3) - (n - 2) and C(n,4), exact in 128 bits, rounded once
  const unsigned __int128 N = (unsigned __int128)n;
  const unsigned __int128 c3 = n >= 3 ? N * (N - 1) * (N - 2) / 6 : 0;
  const unsigned __int128 c4 = n >= 4 ? N * (N - 1) / 2 * (N - 2) * (N - 3) / 12 : 0;
  const double cn3 = (double)(c3 - (unsigned __int128)(n - 2));
  const double cn4 = (double)c4;

  int64_t dup_cap = 1;
  while (dup_cap < 2 * K) dup_cap <<= 1;
  const int final_blocks = grid_for(K, kThreads, 1);
  const size_t front = Carve::bytes_for<DevError>(1) + Carve::bytes_for<unsigned long long>(8) +
                       Carve::bytes_for<int2>(K) + Carve::bytes_for<int64_t>(K + 1) * 2 +
                       Carve::bytes_for<unsigned long long>(K) +
                       Carve::bytes_for<unsigned long long>(K * 3 * kCats) +
                       Carve::bytes_for<int64_t>(scan_tmp_elems(K + 1)) +
                       Carve::bytes_for<unsigned long long>(dup_cap) +
                       Carve::bytes_for<ColMax>((int64_t)final_blocks * kCols + kCols);
  void* base0 = nullptr;
  GS_TRY(ws_reserve(ws, 0, front, stream, &base0));
  Carve c0{(char*)base0, 0};
  DevError* err = c0.take<DevError>(1);
  unsigned long long* stats = c0.take<unsigned long long>(8);
  int2* uv = c0.take<int2>(K);
  int64_t* len = c0.take<int64_t>(K + 1);
  int64_t* choff = c0.take<int64_t>(K + 1);
  unsigned long long* t = c0.take<unsigned long long>(K);
  unsigned long long* acc = c0.take<unsigned long long>(K * 3 * kCats);
  int64_t* tmp0 = c0.take<int64_t>(scan_tmp_elems(K + 1));
  unsigned long long* dup = c0.take<unsigned long long>(dup_cap);
  ColMax* part = c0.take<ColMax>((int64_t)final_blocks * kCols);
  ColMax* best = c0.take<ColMax>(kCols);

  GS_CUDA(cudaMemsetAsync(err, 0, sizeof(DevError), stream));
  GS_CUDA(cudaMemsetAsync(stats, 0, sizeof(unsigned long long) * 8, stream));
  GS_CUDA(cudaMemsetAsync(dup, 0xff, sizeof(unsigned long long) * dup_cap, stream));
  k_prep<<<grid_for(K, kThreads, 8), kThreads, 0, stream>>>(g, d_pairs, K, 0, dup, dup_cap - 1,
                                                            uv, len, err);
  k_micro_chunks<<<grid_for(K, kThreads, 8), kThreads, 0, stream>>>(g.row_ptr, uv, K, choff, t,
                                                                     acc);
  GS_TRY(exclusive_scan_i64(choff, choff, K, tmp0, stream));
  DevError herr;
  int64_t C = 0;
  GS_CUDA(cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, stream));
  GS_CUDA(cudaMemcpyAsync(&C, choff + K, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
  GS_CUDA(cudaStreamSynchronize(stream));
  if (herr.code != 0) {
    set_error("gs_micro: %s (pair %lld)",
              herr.code == GS_EDUPSAMPLE ? "edge sampled twice"
                                         : "sampled pair is out of range or not an edge",
              (long long)herr.index);
    return herr.code;
  }
  int64_t launches = 5;
  if (C > 0) {
    const size_t mid = Carve::bytes_for<int64_t>(C) + Carve::bytes_for<uint32_t>(2 * C) +
                       Carve::bytes_for<int64_t>(C + 1) +
                       Carve::bytes_for<int64_t>(scan_tmp_elems(C + 1));
    void* base1 = nullptr;
    GS_TRY(ws_reserve(ws, 1, mid, stream, &base1));
    Carve c1{(char*)base1, 0};
    int64_t* chunk_e = c1.take<int64_t>(C);
    uint32_t* tmask = c1.take<uint32_t>(2 * C);
    int64_t* task_off = c1.take<int64_t>(C + 1);
    int64_t* tmp1 = c1.take<int64_t>(scan_tmp_elems(C + 1));
    k_micro_fill<<<grid_for(K * 32, kThreads, 8), kThreads, 0, stream>>>(choff, K, chunk_e);
    k_micro_items<<<grid_for(C * 32, kThreads, 8), kThreads, 0, stream>>>(
        g, uv, choff, chunk_e, C, p_e, t, tmask, task_off, stats);
    GS_TRY(exclusive_scan_i64(task_off, task_off, C, tmp1, stream));
    k_micro_probe<<<sm_count() * kProbeBlocksPerSm, kThreads, 0, stream>>>(
        g, uv, choff, chunk_e, tmask, task_off, C, p_e, seed, acc);
    launches += 8;
  }
  k_micro_final<<<final_blocks, kThreads, 0, stream>>>(
      g.row_ptr, uv, K, n, m, cn3, cn4, t, acc, d_x,
      (h_max != nullptr || h_argmax != nullptr) ? part : nullptr);
  ++launches;
  GS_CUDA(cudaGetLastError());
  unsigned long long hs[8];
  GS_CUDA(cudaMemcpyAsync(hs, stats, sizeof(hs), cudaMemcpyDeviceToHost, stream));
  if (h_max != nullptr || h_argmax != nullptr) {
    k_micro_max_final<<<1, 32, 0, stream>>>(part, final_blocks, best);
    ++launches;
    GS_CUDA(cudaGetLastError());
    ColMax hb[kCols];
    GS_CUDA(cudaMemcpyAsync(hb, best, sizeof(hb), cudaMemcpyDeviceToHost, stream));
    GS_CUDA(cudaStreamSynchronize(stream));
    for (int k = 0; k < kCols; ++k) {
      if (h_max != nullptr) h_max[k] = hb[k].v;
      if (h_argmax != nullptr) h_argmax[k] = hb[k].i;
    }
  }
  GS_CUDA(cudaStreamSynchronize(stream));
  ws->stats.micro_probes = (int64_t)hs[0];
  ws->stats.launches = launches;
  ws->launches_total += launches;
  return GS_OK;
}
