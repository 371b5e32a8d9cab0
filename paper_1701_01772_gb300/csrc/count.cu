// Edge-centric local counting over a sampled edge set J (Algorithms 2-4)
// and the exact fold of the per-edge numerators (Sec. 2.3).
//
// For an edge e = (u, v) with d_u <= d_v (ties: smaller id is u), let
// T = N(u) cap N(v), S_u = N(u) \ {v} \ T, S_v = N(v) \ {u} \ T. The paper's
// per-edge quantities are
//   t = |T|                                          (Algorithm 2)
//   k = adjacent pairs inside T                      (Algorithm 3)
//   q = pairs (w in S_u, r in S_v) with w ~ r        (Algorithm 4)
// For w in S_u the common neighbours of w and v are u, the members of T
// adjacent to w and the members of S_v adjacent to w, so with
// c(x, y) = |N(x) cap N(y)|:
//   q = sum_{w in S_u} (c(w, v) - 1) - sum_{r in T} (c(r, u) - 1) + 2k
// (sum_{w in S_u} |N(w) cap T| counted from the T side). Co-degrees of hub
// pairs, and of mid-degree x top-hub pairs, come from tables built at
// registration; the rest are computed by membership tests (see the item
// comment below).
//
// GPU structure (all work is flattened so that per-edge cost skew -- power
// law degrees -- does not serialise on one warp):
//   prep     one thread per pair: canonical orientation, edge check,
//            duplicate check, per-edge position count d_u (padded to 32
//            when 4-node work follows).
//   tri      positions of N(u) are split evenly over all warps; each lane
//            tests one x in N(u) for membership in N(v). Ballots give t and,
//            for 4-node work, one 32-bit word of "x in T" flags per chunk of
//            32 positions.
//   compact  T lists written in order with their hub-matrix slots (one warp
//            per edge); edges with at least kDenseMin matrix members in T
//            whose dense-mode work (row groups plus the other members'
//            neighbour lists) is below
//            their sparse-mode tests are marked dense and get a T mask over
//            matrix slots.
//   cost     per chunk of 32 positions (items w = N(u)[i]): membership-test
//            count of each item (iterate the shorter list, test in the
//            longer); constant terms (the -1s, table co-degrees) added
//            directly; two ballots per chunk (items with tests, items a table
//            answered) for the 4-node pass.
//   quad     chunks are cut into tasks of task_probes tests; warps take
//            runs of consecutive tasks from a counter; inside a task lanes
//            take consecutive tests (two per lane per iteration) and find
//            their item by a search over the warp's scanned costs
//            (load-balanced search).
//   dense    in a dense edge segment A is counted by k_dense_pairs, in work
//            units of kDenseUnit T entries: pairs of dense-slot members by
//            matrix rows ANDed with the T mask, 128 bits at a time; for the
//            other members w, w's matrix neighbours (a bit of the mask, or,
//            past the dense slots, a search of T when above w) and w's
//            neighbours above w without a matrix slot (a search of T).
//   fold     per edge numerators N_i in 128-bit, block partial sums, one
//            final fixed-order pass (or per-segment limb sums, k_fold_seg).
#include <string.h>

#include <algorithm>

#include "common.cuh"

namespace gs {

constexpr int kThreads = 256;
// k_chunk_cost: 6 CTAs per SM (at most 40 registers) hide more of its
// dependent loads than 4 do.
constexpr int kCostBlocksPerSm = 6;
#ifndef GS_QUAD_BLOCKS_PER_SM
#define GS_QUAD_BLOCKS_PER_SM 8
#endif
constexpr int kQuadBlocksPerSm = GS_QUAD_BLOCKS_PER_SM;
constexpr unsigned kFull = 0xffffffffu;
// An edge whose T has at least this many hub-matrix members, and whose
// dense-mode work is the smaller, counts the pairs among them with
// word-parallel AND + popcount over hub-matrix rows.
constexpr int kDenseMin = 64;
constexpr unsigned long long kEmpty = ~0ull;
// Device counters of one count (CountBufs::stats): 0 triangle-pass tests,
// 1 4-node tests, 2 / 3 model bytes (3-node / 4-node part), 4 dense groups,
// 5 k_quad task counter, 6 dense edges, 7 k_dense_pairs unit counter,
// 8 k_chunk_cost chunk counter, 9 tests of dense edges' members without a
// dense slot (k_dense_pairs).
constexpr int kStatSlots = 16;
// Chunks per run a k_chunk_cost warp takes from its counter.
constexpr int kCostGrab = 16;
// Filter of a dense edge's T members without a matrix slot in k_dense_pairs:
// 2^15 bits, built when T has at most kTFilterMaxT entries.
constexpr int kTFilterWords = 1024;
constexpr int64_t kTFilterMaxT = 16384;
__device__ __forceinline__ uint32_t tfilter_hash(int32_t x) {
  return ((uint32_t)x * 2654435761u) >> 17;
}

// Membership tests per run of consecutive tasks a k_quad warp takes from
// the task counter (at least one task).
#ifndef GS_QUAD_GRAB_TESTS
#define GS_QUAD_GRAB_TESTS 16384
#endif
constexpr int64_t kQuadGrabTests = GS_QUAD_GRAB_TESTS;
// Resident CTAs per SM of k_dense_pairs (at most 40 registers).
constexpr int kDenseBlocksPerSm = 6;
// T entries per k_dense_pairs work unit (a heavy dense edge is split into
// several units so that small samples still fill the GPU).
constexpr int64_t kDenseUnit = 4 * kThreads;
// Matrix rows are at most this many 128-bit groups.
constexpr int kHubMatrixMaxGroups = (int)((kHubMatrixMax + 127) / 128);
// 32-bit words of a bitmap over those groups.
constexpr int kGroupWords = (kHubMatrixMaxGroups + 31) / 32;
// Cost of one 128-bit dense group against one membership test, in quarters
// (the dense-mode choice compares kGroupCost * groups with 4 * tests).
#ifndef GS_DENSE_GROUP_COST
#define GS_DENSE_GROUP_COST 4
#endif
constexpr int kGroupCost = GS_DENSE_GROUP_COST;

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}


__device__ __forceinline__ int64_t deg_of(const int64_t* __restrict__ row_ptr, int32_t v,
                                          int64_t* base) {
  int64_t s = __ldg(row_ptr + v), e = __ldg(row_ptr + v + 1);
  *base = s;
  return e - s;
}

// Last index e in [0, count) with off[e] <= p (off[0] = 0 <= p).
__device__ __forceinline__ int64_t last_le(const int64_t* __restrict__ off, int64_t count,
                                           int64_t p) {
  int64_t lo = 0, len = count;
  while (len > 1) {
    int64_t half = len >> 1;
    lo = (__ldg(off + lo + half) <= p) ? lo + half : lo;
    len -= half;
  }
  return lo;
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// ---------------------------------------------------------------- prep

__global__ void k_all_pairs(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                            const int64_t* __restrict__ up_ptr,
                            const int64_t* __restrict__ edge_off, int64_t n,
                            int32_t* __restrict__ pairs) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
    int64_t s = up_ptr[u], e = row_ptr[u + 1], o = edge_off[u];
    for (int64_t p = s + lane; p < e; p += 32) {
      int64_t i = o + (p - s);
      pairs[2 * i] = (int32_t)u;
      pairs[2 * i + 1] = col[p];
    }
  }
}

__global__ void k_prep(DevGraph g, const int32_t* __restrict__ pairs, int64_t K, int pad,
                       unsigned long long* __restrict__ dup_table, int64_t dup_mask,
                       int2* __restrict__ uv, int64_t* __restrict__ len, DevError* err) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < K;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t x = pairs[2 * e], y = pairs[2 * e + 1];
    len[e] = 0;
    uv[e] = make_int2(0, 0);
    if (x < 0 || y < 0 || x >= g.n || y >= g.n || x == y) {
      raise_error(err, GS_EEDGE, e);
      continue;
    }
    int64_t bx, by;
    int64_t dx = deg_of(g.row_ptr, x, &bx), dy = deg_of(g.row_ptr, y, &by);
    bool x_small = dx < dy || (dx == dy && x < y);
    int32_t u = x_small ? x : y, v = x_small ? y : x;
    int64_t du = x_small ? dx : dy, bu = x_small ? bx : by;
    if (!sorted_contains(g.col + bu, du, v)) {
      raise_error(err, GS_EEDGE, e);
      continue;
    }
    if (dup_table != nullptr) {
      uint64_t key = ((uint64_t)(uint32_t)min(x, y) << 32) | (uint32_t)max(x, y);
      uint64_t h = mix64(key) & (uint64_t)dup_mask;
      for (int64_t probe = 0; probe <= dup_mask; ++probe) {
        unsigned long long prev = atomicCAS(dup_table + h, kEmpty, (unsigned long long)key);
        if (prev == kEmpty) break;
        if (prev == key) {
          raise_error(err, GS_EDUPSAMPLE, e);
          break;
        }
        h = (h + 1) & (uint64_t)dup_mask;
      }
    }
    uv[e] = make_int2(u, v);
    len[e] = pad ? ((du + 31) & ~(int64_t)31) : du;
  }
}

// ---------------------------------------------------------------- tri
// Positions [0, P) of the concatenated (padded) N(u) lists are split into
// equal contiguous ranges of 32-position groups, one range per warp.
template <bool kPad>
__global__ void __launch_bounds__(kThreads) k_tri(DevGraph g, const int2* __restrict__ uv,
                                                  const int64_t* __restrict__ off, int64_t K,
                                                  unsigned long long* __restrict__ t,
                                                  uint32_t* __restrict__ tbits) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t P = __ldg(off + K);
  const int64_t groups = (P + 31) >> 5;
  const int64_t per = (groups + warps - 1) / warps;
  const int64_t g0 = warp * per, g1 = min(groups, g0 + per);
  if (g0 >= g1) return;
  int64_t e = last_le(off, K, g0 * 32);
  for (int64_t gi = g0; gi < g1; ++gi) {
    const int64_t p = gi * 32 + lane;
    int64_t le = e;
    while (le + 1 < K && __ldg(off + le + 1) <= p) ++le;
    bool hit = false;
    if (p < P) {
      int2 pr = uv[le];
      int64_t bu, bv;
      int64_t du = deg_of(g.row_ptr, pr.x, &bu), dv = deg_of(g.row_ptr, pr.y, &bv);
      int64_t i = p - __ldg(off + le);
      if (i < du) {
        int32_t x = __ldg(g.col + bu + i);
        const int32_t xs = g.col_hm != nullptr ? (int32_t)__ldg(g.col_hm + bu + i) : -2;
        hit = x != pr.y && adj_contains(g, pr.y, bv, dv, x, xs);
      }
    }
    const unsigned ball = __ballot_sync(kFull, hit);
    if (kPad && lane == 0) tbits[gi] = ball;
    const unsigned grp = __match_any_sync(kFull, (unsigned long long)le);
    const int cnt = __popc(ball & grp);
    if (cnt && lane == __ffs(grp) - 1) atomicAdd(t + le, (unsigned long long)cnt);
    e = __shfl_sync(kFull, le, 31);
  }
}

// Host launcher of the unpadded triangle pass for count_static.cu (a
// kernel template can only be launched from the file that defines it).
void launch_tri_unpadded(const DevGraph& g, const int2* uv, const int64_t* off, int64_t K,
                         unsigned long long* t, int blocks, cudaStream_t stream) {
  k_tri<false><<<blocks, kThreads, 0, stream>>>(g, uv, off, K, t, nullptr);
}

// ---------------------------------------------------------------- compact T

// Writes T_e in order and tdeg[e] = sum of the degrees of T_e's members
// (the latter only feeds the cost model statistics).
__global__ void k_compact_T(DevGraph g, const int2* __restrict__ uv, const int64_t* __restrict__ off,
                            const int64_t* __restrict__ toff, int64_t K,
                            const uint32_t* __restrict__ tbits, int32_t* __restrict__ T,
                            int32_t* __restrict__ tpre, int16_t* __restrict__ T_hm,
                            int64_t* __restrict__ tdeg,
                            int32_t* __restrict__ mask_idx,
                            unsigned long long* __restrict__ dense_counter) {
  __shared__ uint32_t gbits[kThreads / 32][kGroupWords];  // member groups of a warp's edge
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < K; e += warps) {
    int2 pr = uv[e];
    int64_t bu;
    int64_t du = deg_of(g.row_ptr, pr.x, &bu);
    int64_t words = (du + 31) >> 5, w0 = off[e] >> 5, pos = toff[e];
    long long dsum = 0;
    int thm = 0;
    for (int64_t w = 0; w < words; ++w) {
      uint32_t word = __ldg(tbits + w0 + w);
      if (lane == 0) tpre[w0 + w] = (int32_t)(pos - toff[e]);
      bool hm_member = false;
      if ((word >> lane) & 1u) {
        int32_t x = __ldg(g.col + bu + w * 32 + lane);
        const int64_t at = pos + __popc(word & ((1u << lane) - 1u));
        T[at] = x;
        if (T_hm != nullptr) {
          const int16_t xs = __ldg(g.col_hm + bu + w * 32 + lane);
          T_hm[at] = xs;
          hm_member = xs >= 0 && xs < g.hm_dense_words * 32;
        }
        dsum += __ldg(g.row_ptr + x + 1) - __ldg(g.row_ptr + x);
      }
      thm += __popc(__ballot_sync(kFull, hm_member));
      pos += __popc(word);
    }
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(kFull, dsum, o);
    bool dense_mode = false;
    if (T_hm != nullptr && thm >= kDenseMin) {
      // segment-A work of this edge in either mode: sparse = tests over the
      // shorter of N(w) above w / T above w (estimated); dense = for each
      // dense-slot member, the 128-bit groups of the T mask that hold a
      // member and lie at or above its own (what k_dense_pairs reads), plus
      // the adjacency of the other members
      __syncwarp();  // this warp's T entries are visible to all its lanes
      const int64_t t0 = toff[e], te = pos - t0;
      const int D = (int)(g.hm_dense_words * 32);
      uint32_t* gb = gbits[threadIdx.x >> 5];
      for (int w = lane; w < kGroupWords; w += 32) gb[w] = 0u;
      __syncwarp();
      for (int64_t j = lane; j < te; j += 32) {
        const int xs = T_hm[t0 + j];
        if (xs >= 0 && xs < D) atomicOr(gb + (xs >> 12), 1u << ((xs >> 7) & 31));
      }
      __syncwarp();
      long long sparse = 0, dense = 0, groups = 0;
      for (int64_t j = lane; j < te; j += 32) {
        const int32_t x = T[t0 + j];
        const int xs = T_hm[t0 + j];
        const int64_t dx = __ldg(g.row_ptr + x + 1) - __ldg(g.row_ptr + x);
        sparse += min(dx / 2, te - j - 1);  // about half of N(x) lies above x
        if (xs >= 0 && xs < D) {
          const int g0 = xs >> 7;
          groups += __popc(gb[g0 >> 5] & (~0u << (g0 & 31)));
          for (int w = (g0 >> 5) + 1; w < kGroupWords; ++w) groups += __popc(gb[w]);
        } else {  // k_dense_pairs walks its matrix and non-matrix-above lists
          dense += g.mn_ptr != nullptr ? (__ldg(g.mn_ptr + x + 1) - __ldg(g.mn_ptr + x)) +
                                             (__ldg(g.nm_ptr + x + 1) - __ldg(g.nm_ptr + x))
                                       : dx;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        sparse += __shfl_xor_sync(kFull, sparse, o);
        dense += __shfl_xor_sync(kFull, dense, o);
        groups += __shfl_xor_sync(kFull, groups, o);
      }
      dense_mode = kGroupCost * groups + 4 * dense < 4 * sparse;
    }
    if (lane == 0) {
      tdeg[e] = dsum;
      if (mask_idx != nullptr)
        mask_idx[e] = dense_mode ? (int32_t)atomicAdd(dense_counter, 1ull) : -1;
    }
  }
}

// Masks of T's hub-matrix members for dense edges: bit s of the edge's
// mask is set iff the member with matrix slot s is in T. One warp per edge.
__global__ void k_build_tmask(const int64_t* __restrict__ toff, const unsigned long long* __restrict__ t,
                              const int16_t* __restrict__ T_hm, const int32_t* __restrict__ mask_idx,
                              int64_t K, int64_t words, uint32_t* __restrict__ tmask,
                              int64_t* __restrict__ dense_e, int64_t* __restrict__ units) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < K; e += warps) {
    const int32_t idx = mask_idx[e];
    if (idx < 0) continue;
    if (lane == 0) {
      dense_e[idx] = e;
      units[idx] = ((int64_t)t[e] + kDenseUnit - 1) / kDenseUnit;
    }
    uint32_t* m = tmask + (int64_t)idx * words;
    for (int64_t w = lane; w < words; w += 32) m[w] = 0u;
    __syncwarp();
    const int64_t b = toff[e], len = (int64_t)t[e];
    for (int64_t i = lane; i < len; i += 32) {
      const int32_t s = T_hm[b + i];
      if (s >= 0 && s < words * 32) atomicOr(m + (s >> 5), 1u << (s & 31));
    }
  }
}

// Dense edge of every k_dense_pairs work unit: unit_idx[u] = mask index.
// One warp per dense edge.
__global__ void k_unit_fill(const int64_t* __restrict__ unit_off, int64_t ndense,
                            int32_t* __restrict__ unit_idx) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t idx = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; idx < ndense;
       idx += warps)
    for (int64_t u = unit_off[idx] + lane; u < unit_off[idx + 1]; u += 32)
      unit_idx[u] = (int32_t)idx;
}

// Pairs of hub-matrix members of T in the dense edges: member w (slot s)
// contributes popcount(w's matrix row AND the edge's T mask) over the bits
// above s, so every adjacent pair of members counts once (k += 1, q += 2).
// Work units are kDenseUnit consecutive T entries of one dense edge
// (unit_off: exclusive scan of the units per dense edge, unit_idx: the
// dense edge of each unit); a CTA takes one unit at a time from a counter
// and stages the edge's mask (at most 2 KB) in shared memory; each warp
// takes 32 of the unit's entries at a time and walks the rows of the
// members among them with lanes over 128-bit groups (coalesced 512-byte
// reads of the L2-resident matrix).
__global__ void __launch_bounds__(kThreads, kDenseBlocksPerSm)
    k_dense_pairs(const __grid_constant__ DevGraph g, const int64_t* __restrict__ toff,
                  const unsigned long long* __restrict__ t, const int32_t* __restrict__ T,
                  const int16_t* __restrict__ T_hm, const uint32_t* __restrict__ tmask,
                  const int64_t* __restrict__ dense_e, const int64_t* __restrict__ unit_off,
                  const int32_t* __restrict__ unit_idx, int64_t ndense, int need_q,
                  unsigned long long* __restrict__ k_out, unsigned long long* __restrict__ q,
                  unsigned long long* __restrict__ counter,
                  unsigned long long* __restrict__ tests,
                  unsigned long long* __restrict__ rest_tests) {
  // the edge's T mask, whole (fmask) and compacted to its non-zero 128-bit
  // groups: smask[c] is group sgrp[c]; spos[g] = number of non-zero groups
  // below g
  __shared__ uint4 fmask[kHubMatrixMaxGroups];
  __shared__ uint4 smask[kHubMatrixMaxGroups];
  __shared__ uint16_t sgrp[kHubMatrixMaxGroups];
  __shared__ uint16_t spos[kHubMatrixMaxGroups + 1];
  __shared__ int wcnt[kThreads / 32], wlen[kThreads / 32];
  // members without a dense slot among kThreads T entries: vertex, list
  // offsets and lengths, first position in the concatenation of their lists
  __shared__ int64_t ra[kThreads], rb[kThreads];
  __shared__ int32_t rw[kThreads], rna[kThreads], rst[kThreads];
  // hashed filter of T's members without a matrix slot (what the
  // non-matrix lists search for): a clear bit means "not in T"
  __shared__ uint32_t tfilt[kTFilterWords];
  __shared__ unsigned long long part[kThreads / 32][3];
  __shared__ int64_t cur;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t dense_words = g.hm_dense_words;
  const int G = (int)(dense_words / 4);  // 128-bit groups of the dense slots
  const int D = (int)(dense_words * 32);
  const uint32_t* fmask32 = reinterpret_cast<const uint32_t*>(fmask);
  for (;;) {
    if (threadIdx.x == 0) cur = (int64_t)atomicAdd(counter, 1ull);
    __syncthreads();
    const int64_t unit = cur;
    if (unit >= __ldg(unit_off + ndense)) break;
    const int64_t idx = __ldg(unit_idx + unit);
    const int64_t e = dense_e[idx];
    const uint4* m = reinterpret_cast<const uint4*>(tmask + idx * dense_words);
    int L = 0;  // non-zero groups so far (the same in every thread)
    for (int i0 = 0; i0 < G; i0 += kThreads) {
      const int i = i0 + threadIdx.x;
      const uint4 mv = i < G ? m[i] : make_uint4(0u, 0u, 0u, 0u);
      if (i < G) fmask[i] = mv;
      const bool nz = (mv.x | mv.y | mv.z | mv.w) != 0u;
      const unsigned bal = __ballot_sync(kFull, nz);
      if (lane == 0) wcnt[wid] = __popc(bal);
      __syncthreads();
      int before = L, total = L;
      for (int w = 0; w < kThreads / 32; ++w) {
        before += w < wid ? wcnt[w] : 0;
        total += wcnt[w];
      }
      const int at = before + __popc(bal & ((1u << lane) - 1u));
      if (i < G) spos[i] = (uint16_t)at;
      if (nz) {
        smask[at] = mv;
        sgrp[at] = (uint16_t)i;
      }
      L = total;
      __syncthreads();  // wcnt is rewritten by the next round
    }
    if (threadIdx.x == 0) spos[G] = (uint16_t)L;
    __syncthreads();
    const int64_t b = toff[e];
    const int64_t r0 = (unit - __ldg(unit_off + idx)) * kDenseUnit;
    const int64_t len = min((int64_t)t[e], r0 + kDenseUnit);
    unsigned long long acc = 0, groups = 0;
    for (int64_t c0 = r0 + (int64_t)wid * 32; c0 < len; c0 += kThreads) {
      const int xs = c0 + lane < len ? (int)__ldg(T_hm + b + c0 + lane) : -1;
      unsigned members = __ballot_sync(kFull, xs >= 0 && xs < D);
      while (members) {
        const int src = __ffs(members) - 1;
        members &= members - 1;
        const int sl = __shfl_sync(kFull, xs, src);
        const int g0 = sl >> 7, b0 = sl & 127;
        const uint4* row = reinterpret_cast<const uint4*>(g.hm_bits + (int64_t)sl * g.hm_words);
        const int p0 = spos[g0];  // w's own group is non-zero (w is in T)
        groups += L - p0;
        for (int c = p0 + lane; c < L; c += 32) {
          const int gg = sgrp[c];
          const uint4 rw = ld_keep4(row + gg);
          const uint4 mk = smask[c];
          uint32_t wd[4] = {rw.x & mk.x, rw.y & mk.y, rw.z & mk.z, rw.w & mk.w};
          if (gg == g0) {  // only the bits above w's own
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) {
              const int lo_bit = 32 * q4;
              if (b0 >= lo_bit + 31) wd[q4] = 0u;
              else if (b0 >= lo_bit) wd[q4] &= ~0u << (b0 - lo_bit + 1);
            }
          }
          acc += __popc(wd[0]) + __popc(wd[1]) + __popc(wd[2]) + __popc(wd[3]);
        }
      }
    }
    // members without a dense slot: w's matrix neighbours x (a bit of the
    // mask below D; past D, x = hm_vertex[s] counts when above w and in T)
    // and w's neighbours above w without a matrix slot (counted when in T).
    // The block walks the concatenation of these lists, 32 positions per
    // warp at a time.
    unsigned long long rhits = 0, rtested = 0;
    const int64_t te = (int64_t)t[e];
    const int32_t* Te = T + b;
    const bool filt = te <= kTFilterMaxT;
    if (filt) {
      for (int i = threadIdx.x; i < kTFilterWords; i += kThreads) tfilt[i] = 0u;
      __syncthreads();
      for (int64_t i = threadIdx.x; i < te; i += kThreads)
        if (__ldg(T_hm + b + i) < 0) {
          const uint32_t h = tfilter_hash(__ldg(Te + i));
          atomicOr(tfilt + (h >> 5), 1u << (h & 31u));
        }
      __syncthreads();
    }
    for (int64_t c0 = r0; c0 < len; c0 += kThreads) {
      const int64_t j = c0 + threadIdx.x;
      int32_t w = -1, na = 0, nb = 0;
      int64_t a0 = 0, b0 = 0;
      if (j < len) {
        const int xs = __ldg(T_hm + b + j);
        if (!(xs >= 0 && xs < D)) {
          w = __ldg(Te + j);
          a0 = __ldg(g.mn_ptr + w);
          na = (int32_t)(__ldg(g.mn_ptr + w + 1) - a0);
          b0 = __ldg(g.nm_ptr + w);
          nb = (int32_t)(__ldg(g.nm_ptr + w + 1) - b0);
        }
      }
      const int32_t mine = na + nb;
      const unsigned nz = __ballot_sync(kFull, mine > 0);
      int32_t incl = mine;
#pragma unroll
      for (int k = 1; k < 32; k <<= 1) {
        const int32_t y = __shfl_up_sync(kFull, incl, k);
        if (lane >= k) incl += y;
      }
      if (lane == 31) {
        wcnt[wid] = __popc(nz);
        wlen[wid] = incl;
      }
      __syncthreads();
      int32_t bn = 0, bl = 0, cnt = 0, total = 0;
      for (int k = 0; k < kThreads / 32; ++k) {
        if (k < wid) {
          bn += wcnt[k];
          bl += wlen[k];
        }
        cnt += wcnt[k];
        total += wlen[k];
      }
      if (mine > 0) {
        const int at = bn + __popc(nz & ((1u << lane) - 1u));
        rw[at] = w;
        ra[at] = a0;
        rna[at] = na;
        rb[at] = b0;
        rst[at] = bl + incl - mine;
      }
      __syncthreads();
      for (int32_t q0 = wid * 32; q0 < total; q0 += kThreads) {
        int k0 = 0;  // last entry starting at or before q0
        for (int step = kThreads / 2; step > 0; step >>= 1)
          if (k0 + step < cnt && rst[k0 + step] <= q0) k0 += step;
        const int32_t qq = q0 + lane;
        int k = k0;  // last entry starting at or before qq (within 32)
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
          if (k + step < cnt && rst[k + step] <= qq) k += step;
        if (qq < total) {
          const int32_t o = qq - rst[k];
          bool hit;
          if (o < rna[k]) {
            const int sx = __ldg(g.mn_slot + ra[k] + o);
            if (sx < D) {
              hit = ((fmask32[sx >> 5] >> (sx & 31)) & 1u) != 0;
            } else {
              const int32_t x = __ldg(g.hm_vertex + sx);
              hit = x > rw[k] && sorted_contains(Te, te, x);
            }
          } else {
            const int32_t x = __ldg(g.nm_col + rb[k] + (o - rna[k]));
            const uint32_t h = tfilter_hash(x);
            hit = (!filt || ((tfilt[h >> 5] >> (h & 31u)) & 1u) != 0) && sorted_contains(Te, te, x);
          }
          rhits += hit ? 1 : 0;
          ++rtested;
        }
      }
      __syncthreads();  // rw, ra, rb, rna, rst, wcnt and wlen are reused
    }
    acc += rhits;
    acc = warp_sum<unsigned long long>(acc);
    rtested = warp_sum<unsigned long long>(rtested);
    if (lane == 0) {
      part[wid][0] = acc;
      part[wid][1] = groups;  // the same on every lane
      part[wid][2] = rtested;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long sk = 0, sg = 0, sr = 0;
      for (int w = 0; w < kThreads / 32; ++w) {
        sk += part[w][0];
        sg += part[w][1];
        sr += part[w][2];
      }
      if (sk) {
        atomicAdd(k_out + e, sk);
        if (need_q) atomicAdd(q + e, 2 * sk);
      }
      if (sg) atomicAdd(tests, sg);
      if (sr) atomicAdd(rest_tests, sr);
    }
    __syncthreads();  // the masks, part and cur are reused for the next unit
  }
}

// ---------------------------------------------------------------- items
// One item per position of a 32-position chunk: w = N(u)[i], w != v.
// With T = N(u) cap N(v) and c(x, y) = |N(x) cap N(y)|, the 4-node terms are
//   k = sum_{w in T} |N(w) cap T, above w|                 (each pair once)
//   q = sum_{w in S_u} (c(w, v) - 1) - sum_{r in T} (c(r, u) - 1) + 2k
// The second line is sum_{w in S_u} (|N(w) cap N(v)| - |N(w) cap T| - 1)
// with sum_{w in S_u} |N(w) cap T| = sum_{r in T} (c(r, u) - 1) - 2k
// (count the pairs (r in T, w in N(u) \ {v}) with r ~ w from the r side).
// Each item carries up to two segments of membership tests:
//   A (w in T):  x over the shorter of N(w) above w / T above w, tested in
//                the other; a hit is one 4-clique pair: k += 1, q += 2.
//   B (c(w, o)): o = u for w in T, o = v for w in S_u; x over the shorter
//                adjacency, tested in the longer; q -= 1 / q += 1 per hit.
//                Skipped (constant term instead) when the co-degree table
//                holds c(w, o).
// The searched side is a vertex y's adjacency (set_search) or a T list.
struct Seg {
  const int32_t* it;    // iterated list (its matrix slots lie beside it)
  const int32_t* sl;    // searched list
  int32_t sslot;        // matrix slot of y, or -1
  int32_t sbm;          // bitmap slot of y (>= 0), -2 - s when y has a
                        // bucket directory with shift s, else -1
  int32_t slen;         // length of sl, or (sbm < -1) the first entry of
                        // y's directory in g.dir
  int32_t cnt;          // number of tests
};

// Segment A of an item w in T (k_quad) counts the pairs above w. In a dense
// edge no item has a segment A: k_dense_pairs counts all of that edge's
// pairs.

struct EdgeCtx {
  int64_t e;
  int32_t u, v;
  int64_t bu, du, bv, dv;
  int64_t te, toff;
  const uint32_t* tmask;  // this edge's T mask (dense edges), else NULL
};

__device__ __forceinline__ void load_edge(const DevGraph& g, const int2* __restrict__ uv,
                                          const unsigned long long* __restrict__ t,
                                          const int64_t* __restrict__ toff,
                                          const int32_t* __restrict__ mask_idx,
                                          const uint32_t* __restrict__ tmask, int64_t e,
                                          EdgeCtx& c) {
  const int32_t mi = mask_idx != nullptr ? mask_idx[e] : -1;
  c.tmask = mi >= 0 ? tmask + (int64_t)mi * g.hm_dense_words : nullptr;
  int2 pr = uv[e];
  c.e = e;
  c.u = pr.x;
  c.v = pr.y;
  c.du = deg_of(g.row_ptr, pr.x, &c.bu);
  c.dv = deg_of(g.row_ptr, pr.y, &c.bv);
  c.te = (int64_t)t[e];
  c.toff = toff[e];
}

// c(a, b) + 1 from the co-degree table when both are table hubs or from the
// mid x big table when one is a mid vertex and the other a big hub; 0 when
// neither can answer (the +1 marks a present entry).
// sa is a's table slot (tb_slot[a], -1 without a table).
__device__ __forceinline__ uint32_t table_codeg_s(const DevGraph& g, int32_t a, int32_t sa,
                                                  int32_t b) {
  if (g.tb_slot == nullptr) return 0;
  const int32_t sb = __ldg(g.tb_slot + b);
  if (sa >= 0 && sb >= 0) {
    const int32_t lo = min(sa, sb), hi = max(sa, sb);
    const uint16_t c = ld_once16(g.tb_codeg + tb_index(lo, hi, g.tb_count));
    if (c != 0xFFFFu) return (uint32_t)c + 1u;
    if (g.tb_giant != nullptr) {  // a pair of giants
      const int32_t ga = __ldg(g.tb_giant + lo), gb = __ldg(g.tb_giant + hi);
      if (ga >= 0 && gb >= 0) return __ldg(g.tb_giant_codeg + (int64_t)ga * g.tb_giants + gb) + 1u;
    }
    return 0;  // a true co-degree of 65,535 is left to the tests
  }
  if (g.md_codeg != nullptr && (sa < -1 || sb < -1) && (sa >= 0 || sb >= 0)) {
    // one mid vertex (slot -2 - row), one table vertex that may be big
    const int32_t row = -2 - min(sa, sb);
    const int32_t col = __ldg(g.bg_slot + (sa >= 0 ? a : b));
    if (col >= 0) return (uint32_t)ld_once16(g.md_codeg + (int64_t)row * g.bg_count + col) + 1u;
  }
  return 0;
}

// What the cost pass learnt about an item, for the 4-node pass: it has
// tests, and a co-degree table answered its segment B (so the 4-node pass
// needs neither the table nor the item when it has no tests). The constant
// q terms are added by the cost pass alone.
constexpr int kHintLive = 1;
constexpr int kHintTabled = 2;

// sslot value marking a searched vertex whose adjacency is a dense bit-matrix
// row: sl then points at the row and sbm holds the first vertex of the block.
constexpr int32_t kDenseRow = -3;

// The searched side of a segment: vertex y's adjacency, answered by its
// dense row, the hub-pair matrix, its bitmap, or a halving search.
__device__ __forceinline__ void set_search(const DevGraph& g, int32_t y, int64_t by, int64_t dy,
                                           Seg& s) {
  s.sl = g.col + by;
  s.slen = (int32_t)dy;
  if (g.dm_row != nullptr) {
    const int64_t r = __ldg(g.dm_row + y);
    if (r >= 0) {
      s.sslot = kDenseRow;
      s.sl = reinterpret_cast<const int32_t*>(g.dm_bits + r);
      s.sbm = __ldg(g.dm_first + y);
      return;
    }
  }
  s.sslot = table_slot(g, y);
  s.sbm = bitmap_slot(g, y);
  if (s.sbm < 0 && g.dir_at != nullptr) {
    const int64_t at = __ldg(g.dir_at + y);
    if (at >= 0) {
      s.slen = (int32_t)at;
      s.sbm = -2 - (g.id_bits - dir_log2(dy, g.id_bits));
    }
  }
}

// Segment for c(w, o): iterate the shorter adjacency, test in the longer.
__device__ __forceinline__ void codeg_segment(const DevGraph& g, int32_t w, int64_t bw, int64_t dw,
                                              int32_t o, int64_t bo, int64_t dob, Seg& s) {
  if (dw <= dob) {
    s.it = g.col + bw;
    s.cnt = (int32_t)dw;
    set_search(g, o, bo, dob, s);
  } else {
    s.it = g.col + bo;
    s.cnt = (int32_t)dob;
    set_search(g, w, bw, dw, s);
  }
}

// Tests of item i of an edge (segment A + segment B) and its constant q
// term, for the cost pass (the 4-node pass re-derives the segments in
// setup_item). The table slot of w comes from beside the adjacency when
// the graph has it, so the table read does not wait for a gather.
struct ItemCost {
  int32_t a, b;    // tests of segments A and B
  int64_t qconst;  // constant q contribution
  bool tabled;     // a co-degree table answered segment B
};

__device__ __forceinline__ ItemCost item_cost(const DevGraph& g, const EdgeCtx& c, int64_t i,
                                              uint32_t tword, int32_t tbase, int lane,
                                              bool need_q) {
  ItemCost r{0, 0, 0, false};
  if (i >= c.du) return r;
  const int64_t p = c.bu + i;
  const int32_t w = __ldg(g.col + p);
  if (w == c.v) return r;
  const bool in_t = (tword >> lane) & 1u;
  const int64_t dw = __ldg(g.row_ptr + w + 1) - __ldg(g.row_ptr + w);
  if (in_t) {
    if (c.tmask != nullptr) {
      // dense edge: segment A is k_dense_pairs' work (pairs of dense-slot
      // members; the other members' matrix and non-matrix neighbours)
    } else {
      // |N(w) above w cap T above w|: the shorter side is iterated
      const int64_t iw = tbase + __popc(tword & ((1u << lane) - 1u));
      const int64_t tg = c.te - iw - 1;
      const int64_t dup = __ldg(g.row_ptr + w + 1) - __ldg(g.up_ptr + w);
      r.a = (int32_t)min(dup, tg);
    }
  }
  if (need_q) {
    // segment B: -(c(w, u) - 1) for w in T, c(w, v) - 1 for w in S_u
    const int32_t o = in_t ? c.u : c.v;
    const int32_t sw = g.col_tb != nullptr ? __ldg(g.col_tb + p)
                       : g.tb_slot != nullptr ? __ldg(g.tb_slot + w) : -1;
    const uint32_t tc = table_codeg_s(g, w, sw, o);
    r.tabled = tc != 0;
    if (tc != 0) {
      r.qconst = in_t ? 1 - (int64_t)(tc - 1u) : (int64_t)(tc - 1u) - 1;
    } else {
      r.qconst = in_t ? 1 : -1;
      r.b = (int32_t)min(dw, in_t ? c.du : c.dv);
    }
  }
  return r;
}


// Chunk costs: membership tests per chunk and the number of tasks it needs.
// Also adds the constant part of q. Same warp partition as k_tri.
__global__ void __launch_bounds__(kThreads, kCostBlocksPerSm)
    k_chunk_cost(DevGraph g, const int2* __restrict__ uv, const int64_t* __restrict__ off, int64_t K,
                 const unsigned long long* __restrict__ t, const int64_t* __restrict__ toff,
                 const uint32_t* __restrict__ tbits, const int32_t* __restrict__ tpre,
                 const int32_t* __restrict__ mask_idx, const uint32_t* __restrict__ tmask,
                 int need_q, int64_t task_probes, int64_t* __restrict__ task_cnt,
                 uint32_t* __restrict__ cbits, unsigned long long* __restrict__ q,
                 unsigned long long* __restrict__ stats) {
  unsigned long long tests = 0;
  const int lane = threadIdx.x & 31;
  const int64_t P = __ldg(off + K);
  const int64_t groups = P >> 5;  // padded: P is a multiple of 32
  int64_t e = 0;
  EdgeCtx c;
  c.e = -1;
  int64_t next = -1;  // the chunk after this warp's previous run
  // runs of kCostGrab consecutive chunks from a counter (chunks differ in
  // cost: table answers, hub edges)
  for (;;) {
    unsigned long long got = 0;
    if (lane == 0) got = atomicAdd(stats + 8, (unsigned long long)kCostGrab);
    const int64_t g0 = (int64_t)__shfl_sync(kFull, got, 0);
    if (g0 >= groups) break;
    const int64_t g1 = min(groups, g0 + (int64_t)kCostGrab);
    if (g0 != next) e = last_le(off, K, g0 * 32);
    next = g1;
    for (int64_t gi = g0; gi < g1; ++gi) {
      while (e + 1 < K && __ldg(off + e + 1) <= gi * 32) ++e;
      if (e != c.e) load_edge(g, uv, t, toff, mask_idx, tmask, e, c);
      const ItemCost it = item_cost(g, c, gi * 32 + lane - __ldg(off + e), __ldg(tbits + gi),
                                    __ldg(tpre + gi), lane, need_q);
      const unsigned live = __ballot_sync(kFull, it.a + it.b > 0);
      const unsigned tabled = __ballot_sync(kFull, it.tabled);
      if (lane == 0) reinterpret_cast<uint2*>(cbits)[gi] = make_uint2(live, tabled);
      int64_t cost = warp_sum<int64_t>((int64_t)it.a + it.b);
      int64_t qc = warp_sum<int64_t>(it.qconst);
      if (lane == 0) {
        task_cnt[gi] = (cost + task_probes - 1) / task_probes;
        if (qc != 0) atomicAdd(q + e, (unsigned long long)qc);
        tests += cost;
      }
    }
  }
  if (lane == 0 && tests) atomicAdd(stats + 1, (unsigned long long)tests);
}

// ---------------------------------------------------------------- quad

// Item descriptors of the chunk a warp is working on, in shared memory so a
// lane can read the item its test belongs to.
// Membership of x in a directory bucket p[0..len): short buckets (the usual
// case: 2 to 4 entries) are compared entry by entry with independent loads.
__device__ __forceinline__ bool bucket_contains(const int32_t* __restrict__ p, int32_t len,
                                                int32_t x) {
  if (len <= 4) {
    bool f = false;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < len) f |= __ldg(p + k) == x;
    return f;
  }
  return sorted_contains(p, len, x);
}

// Kept to 64 bytes: eight CTAs of 256 items then take 128 KB of shared
// memory, which leaves the rest of the SM's 256 KB to the L1 cache that the
// membership tests depend on. The matrix slots of an iterated list are found
// beside it (col_hm for adjacency lists, T_hm for T) and the segment-B sign
// is stored in one word.
struct SharedItem {
  const int32_t* it[2];
  const int32_t* sl[2];
  int32_t sbm[2];
  int32_t slen[2];
  int16_t sslot[2];
  int32_t ca;
  int32_t mode;  // (bsign + 1) << 8
};
static_assert(sizeof(SharedItem) == 64, "SharedItem size");

// Item set-up of k_quad, out of line: it runs once per chunk and its
// temporaries would otherwise raise the register count of the test loop.
// Derives the same segments as item_cost counts, with the cost pass's hint
// in place of the table reads, and stores each field to the lane's
// shared-memory descriptor as soon as it is known (only the segments that
// have tests are written; a segment with no tests is never read). Returns
// the item's test count.
__device__ __noinline__ int64_t setup_item(const DevGraph& g, const int2* __restrict__ uv,
                                           const unsigned long long* __restrict__ t,
                                           const int64_t* __restrict__ toff,
                                           const int32_t* __restrict__ mask_idx,
                                           const uint32_t* __restrict__ tmask, int64_t e,
                                           const int32_t* __restrict__ T, int64_t i,
                                           uint32_t tword, int32_t tbase, int lane, bool need_q,
                                           int hint, SharedItem* si) {
  EdgeCtx c;
  load_edge(g, uv, t, toff, mask_idx, tmask, e, c);
  int32_t ca = 0, cb = 0, bsign = 0;
  if (i < c.du && (hint & kHintLive)) {
    const int32_t w = __ldg(g.col + c.bu + i);
    if (w != c.v) {
      const bool in_t = (tword >> lane) & 1u;
      int64_t bw;
      const int64_t dw = deg_of(g.row_ptr, w, &bw);
      if (in_t && c.tmask != nullptr) {
        // dense edge: segment A is done by k_dense_pairs
      } else if (in_t) {
        const int64_t iw = tbase + __popc(tword & ((1u << lane) - 1u));
        const int64_t tg = c.te - iw - 1;
        const int64_t upw = __ldg(g.up_ptr + w);
        const int64_t dup = bw + dw - upw;
        if (dup <= tg) {
          si->it[0] = g.col + upw;
          si->sl[0] = T + c.toff + iw + 1;
          si->slen[0] = (int32_t)tg;
          si->sslot[0] = -1;
          si->sbm[0] = -1;
          ca = (int32_t)dup;
        } else {
          Seg sa;
          set_search(g, w, bw, dw, sa);
          si->it[0] = T + c.toff + iw + 1;
          si->sl[0] = sa.sl;
          si->slen[0] = sa.slen;
          si->sslot[0] = (int16_t)sa.sslot;
          si->sbm[0] = sa.sbm;
          ca = (int32_t)tg;
        }
      }
      if (need_q) {
        // segment B: c(w, u) for w in T (q -= 1 per hit), c(w, v) for w in
        // S_u (q += 1 per hit), unless a co-degree table answered it
        bsign = in_t ? -1 : 1;
        if (!(hint & kHintTabled)) {
          Seg sb;
          if (in_t) codeg_segment(g, w, bw, dw, c.u, c.bu, c.du, sb);
          else codeg_segment(g, w, bw, dw, c.v, c.bv, c.dv, sb);
          si->it[1] = sb.it;
          si->sl[1] = sb.sl;
          si->slen[1] = sb.slen;
          si->sslot[1] = (int16_t)sb.sslot;
          si->sbm[1] = sb.sbm;
          cb = sb.cnt;
        }
      }
    }
  }
  si->ca = ca;
  // per-hit weights: segment A adds one 4-clique pair (k += 1, q += 2 when q
  // is wanted); segment B adds bsign to q
  si->mode = (bsign + 1) << 8;
  return (int64_t)ca + cb;
}

__global__ void __launch_bounds__(kThreads, kQuadBlocksPerSm)
    k_quad(const __grid_constant__ DevGraph g, const int2* __restrict__ uv, const int64_t* __restrict__ off, int64_t K,
           const unsigned long long* __restrict__ t, const int64_t* __restrict__ toff,
           const uint32_t* __restrict__ tbits, const int32_t* __restrict__ tpre,
           const uint32_t* __restrict__ cbits,
           const int32_t* __restrict__ T, const int16_t* __restrict__ T_hm,
           const int32_t* __restrict__ mask_idx, const uint32_t* __restrict__ tmask,
           const int64_t* __restrict__ task_off,
           int64_t groups, int need_k, int need_q, int64_t task_probes,
           unsigned long long* __restrict__ k_out,
           unsigned long long* __restrict__ q,
           unsigned long long* __restrict__ task_counter) {
  __shared__ SharedItem items[kThreads / 32][32];
  const int lane = threadIdx.x & 31;
  SharedItem* my = items[threadIdx.x >> 5];
  const int64_t NT = __ldg(task_off + groups);
  // warps take runs of consecutive tasks from a counter: tasks differ in
  // cost (a chunk with few tests still pays a whole item set-up, tests
  // differ in latency), so fixed per-warp ranges left a long tail
  const int64_t grab = max((int64_t)1, kQuadGrabTests / task_probes);
  int64_t gi = 0, e = 0;
  int64_t cur = -1, cur_e = -1;
  int64_t start = 0, ctotal = 0;
  unsigned acc_k = 0;
  int acc_q = 0;
  int64_t next = -1;  // the task after this warp's previous run
  for (;;) {
    unsigned long long got = 0;
    if (lane == 0) got = atomicAdd(task_counter, (unsigned long long)grab);
    const int64_t t0 = (int64_t)__shfl_sync(kFull, got, 0);
    if (t0 >= NT) break;
    const int64_t t1 = min(NT, t0 + grab);
    if (t0 != next) {
      gi = last_le(task_off, groups, t0);
      e = last_le(off, K, gi * 32);
    }
    next = t1;
    for (int64_t task = t0; task < t1; ++task) {
      while (gi + 1 < groups && __ldg(task_off + gi + 1) <= task) ++gi;
      if (gi != cur) {
        // flush the previous chunk's counts to its edge
        const unsigned long long sk = warp_sum<unsigned long long>(acc_k);
        const long long sq = warp_sum<long long>(acc_q);
        if (lane == 0 && cur >= 0) {
          if (sk) atomicAdd(k_out + cur_e, sk);
          if (sq) atomicAdd(q + cur_e, (unsigned long long)sq);
        }
        acc_k = 0;
        acc_q = 0;
        while (e + 1 < K && __ldg(off + e + 1) <= gi * 32) ++e;
        __syncwarp();
        const uint2 cb = __ldg(reinterpret_cast<const uint2*>(cbits) + gi);
        const int hint = (int)((cb.x >> lane) & 1u) * kHintLive +
                         (int)((cb.y >> lane) & 1u) * kHintTabled;
        const int64_t mine =
            setup_item(g, uv, t, toff, mask_idx, tmask, e, T, gi * 32 + lane - __ldg(off + e),
                       __ldg(tbits + gi), __ldg(tpre + gi), lane, need_q, hint, my + lane);
        __syncwarp();
        int64_t incl = mine;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          int64_t y = __shfl_up_sync(kFull, incl, d);
          if (lane >= d) incl += y;
        }
        start = incl - mine;
        ctotal = __shfl_sync(kFull, incl, 31);
        cur = gi;
        cur_e = e;
      }
      const int64_t lo = (task - __ldg(task_off + gi)) * task_probes;
      const int32_t len = (int32_t)min(ctotal - lo, task_probes);
      // item starts relative to the task's first test, in 32 bits: clamping
      // keeps their order and never touches the item that holds a test of
      // this task (it starts less than one item's tests before lo)
      const int32_t srel = (int32_t)max(min(start - lo, task_probes), (int64_t)INT32_MIN + 1);
      // Two independent tests per lane per iteration (r and r + 32): their
      // loads are issued together so each warp keeps more requests in flight.
      for (int32_t r = lane; r - lane < len; r += 64) {
        int32_t x[2], xs[2], seg[2], o[2];
        const SharedItem* it[2];
        bool act[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int32_t rr = r + 32 * h;  // test index within the task
          int j = 0;  // item = last lane whose start <= rr
#pragma unroll
          for (int step = 16; step > 0; step >>= 1) {
            const int32_t sv = __shfl_sync(kFull, srel, j + step);
            if (sv <= rr) j += step;
          }
          const int32_t sj = __shfl_sync(kFull, srel, j);
          act[h] = rr < len;
          it[h] = &my[j];
          o[h] = rr - sj;
          seg[h] = o[h] < it[h]->ca ? 0 : 1;
          if (seg[h]) o[h] -= it[h]->ca;
          x[h] = 0;
          xs[h] = -1;
          if (act[h]) {
            const int32_t* ip = it[h]->it[seg[h]] + o[h];
            x[h] = __ldg(ip);
            xs[h] = kNoSlotInfo;
            if (T_hm != nullptr) {  // matrix slots stored beside the list
              const size_t pc = (size_t)(ip - g.col);
              xs[h] = pc < (size_t)g.nnz ? (int32_t)__ldg(g.col_hm + pc)
                                         : (int32_t)__ldg(T_hm + (ip - T));
            }
          }
        }
        // constant-time word for matrix / bitmap answers, or the bucket bounds
        // of a directory, issued for both
        uint32_t word[2], bitpos[2];
        bool direct[2], bucket[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          direct[h] = false;
          bucket[h] = false;
          word[h] = 0;
          bitpos[h] = 0;
          if (!act[h]) continue;
          const int sslot = it[h]->sslot[seg[h]];
          if (sslot == kDenseRow) {
            const int32_t lx = x[h] - it[h]->sbm[seg[h]];
            word[h] = __ldg(reinterpret_cast<const uint32_t*>(it[h]->sl[seg[h]]) + (lx >> 5));
            bitpos[h] = lx & 31;
            direct[h] = true;
            continue;
          }
          if (sslot >= 0) {
            if (xs[h] == kNoSlotInfo) xs[h] = __ldg(g.hm_slot + x[h]);
            if (xs[h] >= 0) {
              word[h] = ld_keep(g.hm_bits + (int64_t)sslot * g.hm_words + (xs[h] >> 5));
              bitpos[h] = xs[h] & 31;
              direct[h] = true;
              continue;
            }
          }
          const int sbm = it[h]->sbm[seg[h]];
          if (sbm >= 0) {
            word[h] = __ldg(g.bm_bits + (int64_t)sbm * g.bm_words + (x[h] >> 5));
            bitpos[h] = x[h] & 31;
            direct[h] = true;
          } else if (sbm < -1) {
            const uint32_t* d =
                g.dir + (uint32_t)it[h]->slen[seg[h]] + (uint32_t)(x[h] >> (-2 - sbm));
            word[h] = __ldg(d);
            bitpos[h] = __ldg(d + 1);
            bucket[h] = true;
          }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (!act[h]) continue;
          bool hit = direct[h]   ? ((word[h] >> bitpos[h]) & 1u) != 0
                     : bucket[h] ? bucket_contains(it[h]->sl[seg[h]] + word[h],
                                                   (int32_t)(bitpos[h] - word[h]), x[h])
                                 : sorted_contains(it[h]->sl[seg[h]], it[h]->slen[seg[h]], x[h]);
          if (hit) {
            if (seg[h] == 0) {
              ++acc_k;
              acc_q += need_q ? 2 : 0;
            } else {
              acc_q += (it[h]->mode >> 8) - 1;
            }
          }
        }
      }
    }
  }
  const unsigned long long sk = warp_sum<unsigned long long>(acc_k);
  const long long sq = warp_sum<long long>(acc_q);
  if (lane == 0 && cur >= 0) {
    if (sk) atomicAdd(k_out + cur_e, sk);
    if (sq) atomicAdd(q + cur_e, (unsigned long long)sq);
  }
}

// ---------------------------------------------------------------- fold

typedef unsigned __int128 u128;
typedef __int128 i128;

__device__ __forceinline__ u128 shfl_down_u128(u128 v, int o) {
  unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
  lo = __shfl_down_sync(kFull, lo, o);
  hi = __shfl_down_sync(kFull, hi, o);
  return ((u128)hi << 64) | lo;
}

// Per-edge numerators (order 3,4,7,8,9,10,11,12) and 128-bit block sums:
// part[block][0..7] = sum N_i (two's complement), part[block][8..15] = sum N_i^2.
__global__ void __launch_bounds__(kThreads)
    k_fold(DevGraph g, const int2* __restrict__ uv, int64_t K,
           const unsigned long long* __restrict__ t, const unsigned long long* __restrict__ k2,
           const unsigned long long* __restrict__ q, const int64_t* __restrict__ tdeg,
           const int64_t* __restrict__ nbr_degsum, int need_k, int need_q,
           int64_t* __restrict__ per_edge, u128* __restrict__ part,
           unsigned long long* __restrict__ stats) {
  u128 acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0;
  unsigned long long tri_tests = 0, model = 0, model4 = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < K;
       e += (int64_t)gridDim.x * blockDim.x) {
    int2 pr = uv[e];
    int64_t bu, bv;
    const i128 du = deg_of(g.row_ptr, pr.x, &bu), dv = deg_of(g.row_ptr, pr.y, &bv);
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
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      acc[i] += (u128)N[i];
      u128 m = (u128)(N[i] < 0 ? -N[i] : N[i]);
      acc[8 + i] += m * m;
    }
    // streaming cost model B(e) of Algorithms 2-4 (statistics only)
    tri_tests += (unsigned long long)du;
    model += 24 + 4 * (unsigned long long)(du + dv);
    if (tdeg != nullptr) {
      const long long td = tdeg[e];
      unsigned long long B4 = 0;
      if (need_k) B4 += 8 * (unsigned long long)tt + 4 * (unsigned long long)td;
      if (need_q) {
        long long su = (long long)(8 * a) + 4 * (nbr_degsum[pr.x] - (long long)dv - td);
        long long sv = (long long)(8 * b) + 4 * (nbr_degsum[pr.y] - (long long)du - td);
        B4 += (unsigned long long)(su < sv ? su : sv);
      }
      model4 += B4;
    }
    if (per_edge != nullptr) {
      per_edge[3 * e] = (int64_t)tt;
      per_edge[3 * e + 1] = (int64_t)kk;
      per_edge[3 * e + 2] = (int64_t)qq;
    }
  }
  __shared__ u128 red[kThreads / 32][16];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    u128 v = acc[i];
    for (int o = 16; o > 0; o >>= 1) v += shfl_down_u128(v, o);
    if (lane == 0) red[warp][i] = v;
  }
  tri_tests = warp_sum<unsigned long long>(tri_tests);
  model = warp_sum<unsigned long long>(model);
  model4 = warp_sum<unsigned long long>(model4);
  if (lane == 0) {
    atomicAdd(stats + 0, tri_tests);
    atomicAdd(stats + 2, model);
    if (model4) atomicAdd(stats + 3, model4);
  }
  __syncthreads();
  if (threadIdx.x < 16) {
    u128 s = 0;
    for (int w = 0; w < kThreads / 32; ++w) s += red[w][threadIdx.x];
    part[(int64_t)blockIdx.x * 16 + threadIdx.x] = s;
  }
}

__global__ void k_fold_final(const u128* __restrict__ part, int blocks,
                             unsigned long long* __restrict__ out) {
  if (threadIdx.x < 16) {
    u128 s = 0;
    for (int b = 0; b < blocks; ++b) s += part[(int64_t)b * 16 + threadIdx.x];
    out[2 * threadIdx.x] = (unsigned long long)s;
    out[2 * threadIdx.x + 1] = (unsigned long long)(s >> 64);
  }
}


// Per-segment exact sums. Edges [seg_off[s], seg_off[s+1]) form segment s
// (one graph of a batch, one request of a serving step). Each of the 16
// values (8 sums in two's complement, 8 sums of squares) is accumulated as
// four 32-bit limbs in 64-bit counters: a limb sum stays below 2^64 for
// fewer than 2^32 additions, so the 128-bit total is recovered exactly.
// Lanes of a warp are reduced per segment first (segmented shuffle scan).
__global__ void __launch_bounds__(kThreads)
    k_fold_seg(DevGraph g, const int2* __restrict__ uv, int64_t K,
               const unsigned long long* __restrict__ t, const unsigned long long* __restrict__ k2,
               const unsigned long long* __restrict__ q, const int64_t* __restrict__ seg_off,
               int64_t nseg, unsigned long long* __restrict__ limbs) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < K;
       base += stride) {
    const int64_t e = base + lane;
    int64_t seg = -1;
    u128 val[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) val[i] = 0;
    if (e < K) {
      seg = last_le(seg_off, nseg, e);
      int2 pr = uv[e];
      int64_t bu, bv;
      const i128 du = deg_of(g.row_ptr, pr.x, &bu), dv = deg_of(g.row_ptr, pr.y, &bv);
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
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        val[i] = (u128)N[i];
        u128 m = (u128)(N[i] < 0 ? -N[i] : N[i]);
        val[8 + i] = m * m;
      }
    }
    // segmented inclusive scan over the warp (segments are contiguous)
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int64_t sd = __shfl_up_sync(kFull, seg, d);
      const bool take = lane >= d && sd == seg;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        unsigned long long lo = __shfl_up_sync(kFull, (unsigned long long)val[i], d);
        unsigned long long hi = __shfl_up_sync(kFull, (unsigned long long)(val[i] >> 64), d);
        if (take) val[i] += ((u128)hi << 64) | lo;
      }
    }
    const int64_t next = __shfl_down_sync(kFull, seg, 1);
    const bool tail = seg >= 0 && (lane == 31 || next != seg);
    if (tail) {
      unsigned long long* dst = limbs + seg * 64;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          const unsigned long long limb = (unsigned long long)((val[i] >> (32 * l)) & 0xffffffffu);
          if (limb) atomicAdd(dst + i * 4 + l, limb);
        }
      }
    }
  }
}

// Recombines the limbs: sums[s][i] = sum_l limb_l << 32 l (mod 2^128), as
// (low, high) 64-bit words.
__global__ void k_fold_seg_final(const unsigned long long* __restrict__ limbs, int64_t nseg,
                                 unsigned long long* __restrict__ sums) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nseg * 16;
       x += (int64_t)gridDim.x * blockDim.x) {
    u128 s = 0;
#pragma unroll
    for (int l = 0; l < 4; ++l) s += (u128)limbs[x * 4 + l] << (32 * l);
    sums[2 * x] = (unsigned long long)s;
    sums[2 * x + 1] = (unsigned long long)(s >> 64);
  }
}

}  // namespace gs

// =================================================================== host side
namespace gs {

// 8 triangle-pass CTAs per SM (32 registers) and 512-test tasks: measured
// best on the 1M-vertex power-law graph (triangle pass 79 -> 47 ms exact).
Tuning default_tuning() { return Tuning{8, kQuadBlocksPerSm, 512, 1, kHubDenseSlots}; }

int quad_blocks_limit() { return kQuadBlocksPerSm; }

DevGraph graph_view(const gs_graph* gr, const Tuning& tu) {
  DevGraph g = gr->dev;
  g.hm_dense_words =
      g.hm_bits != nullptr ? std::min(g.hm_words, std::max<int64_t>(tu.dense_slots, 0) / 128 * 4)
                           : 0;
  if (!tu.use_hubs) {
    g.bm_slot = nullptr;
    g.bm_bits = nullptr;
    g.bm_count = 0;
    g.tb_slot = nullptr;
    g.tb_codeg = nullptr;
    g.tb_giant = nullptr;
    g.tb_count = 0;
    g.hm_slot = nullptr;
    g.hm_bits = nullptr;
    g.col_hm = nullptr;
    g.mn_ptr = nullptr;
    g.mn_slot = nullptr;
    g.nm_ptr = nullptr;
    g.nm_col = nullptr;
    g.hm_vertex = nullptr;
    g.bg_slot = nullptr;
    g.md_codeg = nullptr;
    g.dir_at = nullptr;
    g.dir = nullptr;
    g.col_tb = nullptr;
  }
  return g;
}

size_t count_front_bytes(int64_t K, bool all_edges, bool check_dup, int64_t nseg) {
  int64_t dup_cap = 1;
  while (dup_cap < 2 * K) dup_cap <<= 1;
  const int fold_blocks = grid_for(K, kThreads, 2);
  return Carve::bytes_for<DevError>(1) + Carve::bytes_for<unsigned long long>(32) +
         Carve::bytes_for<unsigned long long>(kStatSlots) +
         (all_edges ? Carve::bytes_for<int32_t>(2 * K) : 0) + Carve::bytes_for<int2>(K) +
         Carve::bytes_for<int64_t>(K + 1) * 2 + Carve::bytes_for<unsigned long long>(K) * 3 +
         Carve::bytes_for<int64_t>(K) + Carve::bytes_for<int32_t>(K) +
         Carve::bytes_for<int64_t>(scan_tmp_elems(K + 1)) +
         (check_dup ? Carve::bytes_for<unsigned long long>(dup_cap) : 0) +
         Carve::bytes_for<u128>((int64_t)fold_blocks * 16) +
         (nseg > 0 ? Carve::bytes_for<unsigned long long>(nseg * 64) +
                         Carve::bytes_for<unsigned long long>(nseg * 32)
                   : 0);
}

void carve_front(void* base, int64_t K, bool all_edges, bool check_dup, int64_t nseg,
                 CountBufs& b) {
  Carve c{(char*)base, 0};
  int64_t dup_cap = 1;
  while (dup_cap < 2 * K) dup_cap <<= 1;
  b.K = K;
  b.dup_cap = dup_cap;
  b.fold_blocks = grid_for(K, kThreads, 2);
  b.err = c.take<DevError>(1);
  b.sums = c.take<unsigned long long>(32);
  b.stats = c.take<unsigned long long>(kStatSlots);
  b.pairs_all = all_edges ? c.take<int32_t>(2 * K) : nullptr;
  b.uv = c.take<int2>(K);
  b.off = c.take<int64_t>(K + 1);
  b.toff = c.take<int64_t>(K + 1);
  b.t = c.take<unsigned long long>(K);
  b.k2 = c.take<unsigned long long>(K);
  b.q = c.take<unsigned long long>(K);
  b.tdeg = c.take<int64_t>(K);
  b.mask_idx = c.take<int32_t>(K);
  b.tmp0 = c.take<int64_t>(scan_tmp_elems(K + 1));
  b.dup = check_dup ? c.take<unsigned long long>(dup_cap) : nullptr;
  b.part = c.take<u128>((int64_t)b.fold_blocks * 16);
  b.nseg = nseg;
  b.limbs = nseg > 0 ? c.take<unsigned long long>(nseg * 64) : nullptr;
  b.seg_sums = nseg > 0 ? c.take<unsigned long long>(nseg * 32) : nullptr;
}

size_t count_mid_bytes(int64_t P) {
  const int64_t groups = (P + 31) / 32;
  return Carve::bytes_for<uint32_t>(groups) + Carve::bytes_for<int32_t>(groups) +
         Carve::bytes_for<uint32_t>(2 * groups) +
         Carve::bytes_for<int64_t>(groups + 1) +
         Carve::bytes_for<int64_t>(scan_tmp_elems(groups + 1));
}

void carve_mid(void* base, int64_t P, CountBufs& b) {
  Carve c{(char*)base, 0};
  b.P = P;
  b.groups = (P + 31) / 32;
  b.tbits = c.take<uint32_t>(b.groups);
  b.tpre = c.take<int32_t>(b.groups);
  b.cbits = c.take<uint32_t>(2 * b.groups);
  b.task_off = c.take<int64_t>(b.groups + 1);
  b.tmp1 = c.take<int64_t>(scan_tmp_elems(b.groups + 1));
}

// memsets + (all-pair enumeration) + prep + position scan. No host sync.
int64_t launch_front(const gs_graph* gr, const DevGraph& g, const int32_t* pairs, bool four,
                     CountBufs& b, cudaStream_t stream) {
  int64_t launches = 0;
  const int64_t K = b.K;
  cudaMemsetAsync(b.err, 0, sizeof(DevError), stream);
  cudaMemsetAsync(b.stats, 0, sizeof(unsigned long long) * kStatSlots, stream);
  cudaMemsetAsync(b.t, 0, sizeof(unsigned long long) * K, stream);
  if (four) {
    cudaMemsetAsync(b.k2, 0, sizeof(unsigned long long) * K, stream);
    cudaMemsetAsync(b.q, 0, sizeof(unsigned long long) * K, stream);
  }
  if (b.dup != nullptr) cudaMemsetAsync(b.dup, 0xff, sizeof(unsigned long long) * b.dup_cap, stream);
  if (pairs == nullptr) {
    k_all_pairs<<<grid_for(g.n * 32, kThreads, 8), kThreads, 0, stream>>>(
        g.row_ptr, g.col, gr->up_ptr, gr->edge_off, g.n, b.pairs_all);
    pairs = b.pairs_all;
    ++launches;
  }
  k_prep<<<grid_for(K, kThreads, 8), kThreads, 0, stream>>>(g, pairs, K, four ? 1 : 0, b.dup,
                                                            b.dup_cap - 1, b.uv, b.off, b.err);
  exclusive_scan_i64(b.off, b.off, K, b.tmp0, stream);
  return launches + 4;
}

int64_t launch_tri(const DevGraph& g, bool four, const Tuning& tu, CountBufs& b,
                   cudaStream_t stream) {
  const int grid = sm_count() * tu.tri_blocks_per_sm;
  if (four)
    k_tri<true><<<grid, kThreads, 0, stream>>>(g, b.uv, b.off, b.K, b.t, b.tbits);
  else
    k_tri<false><<<grid, kThreads, 0, stream>>>(g, b.uv, b.off, b.K, b.t, nullptr);
  return 1;
}

int64_t launch_scan_t(CountBufs& b, cudaStream_t stream) {
  exclusive_scan_i64((const int64_t*)b.t, b.toff, b.K, b.tmp0, stream);
  return 3;
}

// T lists (and their matrix slots) in order; marks dense edges (mask index
// from the counter stats[6]). T must hold b.toff[K] entries. No host sync.
int64_t launch_compact(const DevGraph& g, CountBufs& b, cudaStream_t stream) {
  int16_t* T_hm = g.col_hm != nullptr ? b.T_hm : nullptr;
  k_compact_T<<<grid_for(b.K * 32, kThreads, 8), kThreads, 0, stream>>>(
      g, b.uv, b.off, b.toff, b.K, b.tbits, b.T, b.tpre, T_hm, b.tdeg, b.mask_idx, b.stats + 6);
  return 1;
}

// T masks of the dense edges (b.ndense of them). No host sync.
int64_t launch_tmask(const DevGraph& g, CountBufs& b, cudaStream_t stream) {
  if (b.ndense <= 0 || g.col_hm == nullptr) return 0;
  k_build_tmask<<<grid_for(b.K * 32, kThreads, 8), kThreads, 0, stream>>>(
      b.toff, b.t, b.T_hm, b.mask_idx, b.K, g.hm_dense_words, b.tmask, b.dense_e, b.unit_off);
  exclusive_scan_i64(b.unit_off, b.unit_off, b.ndense, b.unit_tmp, stream);
  k_unit_fill<<<grid_for(b.ndense * 32, kThreads, 8), kThreads, 0, stream>>>(b.unit_off, b.ndense,
                                                                              b.unit_idx);
  return 5;
}

// Pairs among the matrix members of T in the dense edges (k_dense_pairs).
// No host sync.
int64_t launch_dense(const DevGraph& g, bool need_q, CountBufs& b, cudaStream_t stream) {
  if (b.ndense <= 0 || g.col_hm == nullptr) return 0;
  k_dense_pairs<<<sm_count() * kDenseBlocksPerSm, kThreads, 0, stream>>>(
      g, b.toff, b.t, b.T, b.T_hm, b.tmask, b.dense_e, b.unit_off, b.unit_idx, b.ndense,
      need_q ? 1 : 0, b.k2, b.q, b.stats + 7, b.stats + 4, b.stats + 9);
  return 1;
}

// Chunk costs and the task scan. No host sync.
int64_t launch_cost(const DevGraph& g, bool need_k, bool need_q, const Tuning& tu, CountBufs& b,
                    cudaStream_t stream) {
  (void)need_k;  // every item's segment A feeds both k and q
  const int32_t* mi = g.col_hm != nullptr ? b.mask_idx : nullptr;
  k_chunk_cost<<<sm_count() * kCostBlocksPerSm, kThreads, 0, stream>>>(
      g, b.uv, b.off, b.K, b.t, b.toff, b.tbits, b.tpre, mi, b.tmask, need_q, tu.task_probes,
      b.task_off, b.cbits, b.q, b.stats);
  exclusive_scan_i64(b.task_off, b.task_off, b.groups, b.tmp1, stream);
  return 4;
}

// The 4-node membership tests (k_quad). No host sync.
int64_t launch_quad(const DevGraph& g, bool need_k, bool need_q, const Tuning& tu, CountBufs& b,
                    cudaStream_t stream) {
  const int sms = sm_count();
  const int qb = tu.quad_blocks_per_sm < 1 ? 1
                 : tu.quad_blocks_per_sm > kQuadBlocksPerSm ? kQuadBlocksPerSm
                                                            : tu.quad_blocks_per_sm;
  k_quad<<<sms * qb, kThreads, 0, stream>>>(g, b.uv, b.off, b.K, b.t, b.toff, b.tbits, b.tpre,
                                            b.cbits, b.T,
                                            g.col_hm != nullptr ? b.T_hm : nullptr,
                                            g.col_hm != nullptr ? b.mask_idx : nullptr, b.tmask,
                                            b.task_off, b.groups, need_k, need_q,
                                            tu.task_probes, b.k2, b.q, b.stats + 5);
  return 1;
}

int64_t launch_fold(const gs_graph* gr, const DevGraph& g, bool four, bool need_k, bool need_q,
                    int64_t* per_edge, CountBufs& b, cudaStream_t stream) {
  k_fold<<<b.fold_blocks, kThreads, 0, stream>>>(g, b.uv, b.K, b.t, four ? b.k2 : nullptr,
                                                  four ? b.q : nullptr, four ? b.tdeg : nullptr,
                                                  gr->nbr_degsum, need_k, need_q, per_edge, b.part,
                                                  b.stats);
  k_fold_final<<<1, 32, 0, stream>>>(b.part, b.fold_blocks, b.sums);
  return 2;
}

int64_t launch_fold_seg(const DevGraph& g, bool four, const int64_t* seg_off, CountBufs& b,
                        cudaStream_t stream) {
  cudaMemsetAsync(b.limbs, 0, sizeof(unsigned long long) * b.nseg * 64, stream);
  k_fold_seg<<<grid_for(b.K, kThreads, 4), kThreads, 0, stream>>>(
      g, b.uv, b.K, b.t, four ? b.k2 : nullptr, four ? b.q : nullptr, seg_off, b.nseg, b.limbs);
  k_fold_seg_final<<<grid_for(b.nseg * 16, 256, 4), 256, 0, stream>>>(b.limbs, b.nseg,
                                                                       b.seg_sums);
  return 2;
}

gs_status fetch_error(DevError* d_err, cudaStream_t stream, const char* what) {
  DevError h;
  GS_CUDA(cudaMemcpyAsync(&h, d_err, sizeof(h), cudaMemcpyDeviceToHost, stream));
  GS_CUDA(cudaStreamSynchronize(stream));
  if (h.code != 0) {
    const char* kind = h.code == GS_EDUPSAMPLE ? "edge sampled twice"
                       : h.code == GS_EEDGE    ? "sampled pair is out of range or not an edge"
                                               : "invalid input";
    set_error("%s: %s (pair %lld)", what, kind, (long long)h.index);
    return h.code;
  }
  return GS_OK;
}

void store_sums(const unsigned long long* h, uint32_t mask, gs_sums* out) {
  static const uint32_t bit[8] = {GS_G3, GS_G4, GS_G7, GS_G8, GS_G9, GS_G10, GS_G11, GS_G12};
  for (int i = 0; i < 8; ++i) {
    if (!(mask & bit[i])) continue;
    out->sum[i][0] = h[2 * i];
    out->sum[i][1] = h[2 * i + 1];
    out->sumsq[i][0] = h[2 * (8 + i)];
    out->sumsq[i][1] = h[2 * (8 + i) + 1];
  }
}

// Full counting run with host synchronisation for sizing (gs_count and the
// sizing pass of the batched and served paths). seg_off != NULL selects the
// per-segment fold (results in b.seg_sums) instead of the single sum.
gs_status count_run(const gs_graph* gr, gs_workspace* ws, const int32_t* d_pairs, int64_t K,
                    uint32_t mask, bool check_dup, int64_t* d_per_edge, const int64_t* seg_off,
                    int64_t nseg, const Tuning& tu, CountBufs& b, cudaStream_t stream,
                    const char* what) {
  const bool need_k = (mask & (GS_G7 | GS_G8 | GS_G9 | GS_G11)) != 0;
  const bool need_q = (mask & (GS_G10 | GS_G12)) != 0;
  const bool four = need_k || need_q;
  const bool all_edges = d_pairs == nullptr;
  const DevGraph g = graph_view(gr, tu);
  int64_t launches = 0;
  struct Timer {
    gs_workspace* ws;
    cudaStream_t s;
    void start(int p) {
      if (ws->timing) cudaEventRecord(ws->ev[2 * p], s);
    }
    void stop(int p) {
      if (ws->timing) cudaEventRecord(ws->ev[2 * p + 1], s);
    }
  } timer{ws, stream};

  void* base0 = nullptr;
  GS_TRY(ws_reserve(ws, 0, count_front_bytes(K, all_edges, check_dup, seg_off ? nseg : 0), stream,
                    &base0));
  carve_front(base0, K, all_edges, check_dup, seg_off ? nseg : 0, b);
  timer.start(0);
  launches += launch_front(gr, g, d_pairs, four, b, stream);
  timer.stop(0);
  GS_CUDA(cudaGetLastError());
  int64_t P = 0;
  GS_CUDA(cudaMemcpyAsync(&P, b.off + K, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
  gs_status es = fetch_error(b.err, stream, what);
  ws->launches_total += launches;
  if (es != GS_OK) return es;

  void* base1 = nullptr;
  GS_TRY(ws_reserve(ws, 1, four ? count_mid_bytes(P) : 256, stream, &base1));
  if (four) {
    carve_mid(base1, P, b);
  } else {
    b.P = P;
    b.groups = (P + 31) / 32;
    b.tbits = nullptr;
  }
  int64_t more = 0;
  timer.start(1);
  more += launch_tri(g, four, tu, b, stream);
  timer.stop(1);
  GS_CUDA(cudaGetLastError());
  b.tsum = 0;
  if (four) {
    timer.start(2);
    more += launch_scan_t(b, stream);
    GS_CUDA(cudaMemcpyAsync(&b.tsum, b.toff + K, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
    GS_CUDA(cudaStreamSynchronize(stream));
    void* base2 = nullptr;
    GS_TRY(ws_reserve(ws, 2,
                      Carve::bytes_for<int32_t>(b.tsum) + Carve::bytes_for<int16_t>(b.tsum),
                      stream, &base2));
    Carve c2{(char*)base2, 0};
    b.T = c2.take<int32_t>(b.tsum);
    b.T_hm = c2.take<int16_t>(b.tsum);
    more += launch_compact(g, b, stream);
    unsigned long long nd = 0;
    GS_CUDA(cudaMemcpyAsync(&nd, b.stats + 6, sizeof(nd), cudaMemcpyDeviceToHost, stream));
    GS_CUDA(cudaStreamSynchronize(stream));
    b.ndense = (int64_t)nd;
    b.tmask = nullptr;
    b.dense_e = nullptr;
    if (b.ndense > 0) {
      void* base4 = nullptr;
      GS_TRY(ws_reserve(ws, 4,
                        Carve::bytes_for<uint32_t>(b.ndense * g.hm_dense_words) +
                            Carve::bytes_for<int64_t>(b.ndense) +
                            Carve::bytes_for<int64_t>(b.ndense + 1) +
                            Carve::bytes_for<int64_t>(scan_tmp_elems(b.ndense + 1)) +
                            Carve::bytes_for<int32_t>(b.tsum / kDenseUnit + b.ndense),
                        stream, &base4));
      Carve c4{(char*)base4, 0};
      b.tmask = c4.take<uint32_t>(b.ndense * g.hm_dense_words);
      b.dense_e = c4.take<int64_t>(b.ndense);
      b.unit_off = c4.take<int64_t>(b.ndense + 1);
      b.unit_tmp = c4.take<int64_t>(scan_tmp_elems(b.ndense + 1));
      // units of an edge: ceil(t / kDenseUnit) <= t / kDenseUnit + 1
      b.unit_idx = c4.take<int32_t>(b.tsum / kDenseUnit + b.ndense);
    }
    timer.stop(2);
    timer.start(3);
    more += launch_tmask(g, b, stream);
    more += launch_cost(g, need_k, need_q, tu, b, stream);
    timer.stop(3);
    timer.start(4);
    more += launch_quad(g, need_k, need_q, tu, b, stream);
    more += launch_dense(g, need_q, b, stream);
    timer.stop(4);
    GS_CUDA(cudaGetLastError());
  } else {
    for (int ph = 2; ph <= 4; ++ph) {
      timer.start(ph);
      timer.stop(ph);
    }
  }
  timer.start(5);
  if (seg_off != nullptr)
    more += launch_fold_seg(g, four, seg_off, b, stream);
  else
    more += launch_fold(gr, g, four, need_k, need_q, d_per_edge, b, stream);
  timer.stop(5);
  GS_CUDA(cudaGetLastError());
  ws->launches_total += more;
  ws->stats.launches = launches + more;
  return GS_OK;
}

}  // namespace gs

// =================================================================== C ABI
using namespace gs;

static const uint32_t kKnownMask = GS_CONNECTED;

extern "C" gs_status gs_count(const gs_graph* gr, gs_workspace* ws, const int32_t* d_pairs,
                              int64_t K, uint32_t mask, int64_t* d_per_edge, gs_sums* h_sums,
                              void* stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (gr == nullptr || ws == nullptr || h_sums == nullptr || K < 0 || mask == 0 ||
      (mask & ~kKnownMask) != 0) {
    set_error("gs_count: invalid arguments (mask must be a non-empty subset of GS_CONNECTED)");
    return GS_EINVAL;
  }
  memset(h_sums, 0, sizeof(*h_sums));
  h_sums->k = K;
  h_sums->m = gr->m;
  h_sums->mask = mask;
  memset(&ws->stats, 0, sizeof(ws->stats));
  ws->stats.k = K;
  if (K == 0) return GS_OK;  // empty sample (d_pairs is not read)
  if (d_pairs == nullptr && K != gr->m) {
    set_error("gs_count: with d_pairs = NULL, k must equal the edge count %lld", (long long)gr->m);
    return GS_EINVAL;
  }
  const Tuning tu = ws->has_tuning ? ws->tuning : default_tuning();
  if (d_pairs == nullptr && d_per_edge == nullptr && (mask & ~(uint32_t)GS_THREE_NODE) == 0 &&
      gr->out_col != nullptr && tu.use_hubs) {
    // every edge, triangles and 2-stars only: triangles listed once through
    // the oriented lists (same per-edge t, sums independent of the order)
    unsigned long long h[32], hs[8];
    int64_t nl = 0;
    GS_TRY(count_tri_oriented(gr, ws, h, hs, &nl, stream));
    store_sums(h, mask, h_sums);
    gs_stats& st = ws->stats;
    st.k = K;
    st.tri_tests = (int64_t)hs[0];
    st.model_bytes = hs[2];
    st.model_tri_bytes = hs[2];
    st.launches = nl;
    ws->launches_total += nl;
    st.timed = ws->timing;
    if (ws->timing) {
      float* ms[6] = {&st.ms_prep, &st.ms_tri, &st.ms_compact, &st.ms_cost, &st.ms_quad,
                      &st.ms_fold};
      for (int ph = 0; ph < 6; ++ph)
        cudaEventElapsedTime(ms[ph], ws->ev[2 * ph], ws->ev[2 * ph + 1]);
    }
    return GS_OK;
  }
  CountBufs b;
  GS_TRY(count_run(gr, ws, d_pairs, K, mask, d_pairs != nullptr, d_per_edge, nullptr, 0, tu, b,
                   stream, "gs_count"));
  const bool four = (mask & (GS_G7 | GS_G8 | GS_G9 | GS_G10 | GS_G11 | GS_G12)) != 0;
  unsigned long long h[32];
  unsigned long long hs[kStatSlots];
  int64_t ntasks = 0;
  GS_CUDA(cudaMemcpyAsync(h, b.sums, sizeof(h), cudaMemcpyDeviceToHost, stream));
  GS_CUDA(cudaMemcpyAsync(hs, b.stats, sizeof(hs), cudaMemcpyDeviceToHost, stream));
  if (four)
    GS_CUDA(cudaMemcpyAsync(&ntasks, b.task_off + b.groups, sizeof(int64_t),
                            cudaMemcpyDeviceToHost, stream));
  GS_CUDA(cudaStreamSynchronize(stream));
  store_sums(h, mask, h_sums);
  gs_stats& st = ws->stats;
  st.k = K;
  st.tri_tests = (int64_t)hs[0];
  st.dense_edges = (int64_t)hs[6];
  st.quad_tests = (int64_t)(hs[1] + hs[4] + hs[9]);
  st.dense_groups = (int64_t)hs[4];
  st.model_bytes = hs[2] + hs[3];
  st.model_tri_bytes = hs[2];
  st.model_quad_bytes = hs[3];
  st.t_sum = b.tsum;
  st.tasks = ntasks;
  st.timed = ws->timing;
  if (ws->timing) {
    float* ms[6] = {&st.ms_prep, &st.ms_tri, &st.ms_compact, &st.ms_cost, &st.ms_quad, &st.ms_fold};
    for (int ph = 0; ph < 6; ++ph) cudaEventElapsedTime(ms[ph], ws->ev[2 * ph], ws->ev[2 * ph + 1]);
  }
  return GS_OK;
}

extern "C" gs_status gs_workspace_set_tuning(gs_workspace* ws, int tri_blocks_per_sm,
                                             int quad_blocks_per_sm, int64_t task_probes,
                                             int use_hubs) {
  if (ws == nullptr || tri_blocks_per_sm < 1 || tri_blocks_per_sm > 8 || quad_blocks_per_sm < 1 ||
      quad_blocks_per_sm > kQuadBlocksPerSm || task_probes < 32 || task_probes > (1 << 20)) {
    set_error("gs_workspace_set_tuning: out-of-range parameter (tri 1..8, quad 1..%d, task "
              "32..2^20)",
              kQuadBlocksPerSm);
    return GS_EINVAL;
  }
  const int64_t ds = ws->has_tuning ? ws->tuning.dense_slots : kHubDenseSlots;
  ws->tuning = Tuning{tri_blocks_per_sm, quad_blocks_per_sm, task_probes, use_hubs ? 1 : 0, ds};
  ws->has_tuning = 1;
  return GS_OK;
}

extern "C" gs_status gs_workspace_set_dense_slots(gs_workspace* ws, int64_t slots) {
  if (ws == nullptr || slots < 0) {
    set_error("gs_workspace_set_dense_slots: null workspace or negative slot count");
    return GS_EINVAL;
  }
  if (!ws->has_tuning) ws->tuning = default_tuning();
  ws->tuning.dense_slots = slots;
  ws->has_tuning = 1;
  return GS_OK;
}
