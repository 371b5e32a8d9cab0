// Runtime pieces of libgraphlet: error reporting, device-wide prefix sums,
// grid sizing and the growable workspace.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "common.cuh"

namespace gs {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

gs_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  set_error("CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file, line);
  return e == cudaErrorMemoryAllocation ? GS_ENOMEM : GS_ECUDA;
}

int sm_count() {
  static int cached = 0;
  if (cached == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached = v > 0 ? v : 152;
  }
  return cached;
}

int grid_for(int64_t work_items, int threads_per_block, int blocks_per_sm) {
  int64_t cap = (int64_t)sm_count() * blocks_per_sm;
  int64_t need = (work_items + threads_per_block - 1) / threads_per_block;
  if (need < 1) need = 1;
  return (int)(need < cap ? need : cap);
}

// ---------------------------------------------------------------- scan
// Three passes: per-tile totals, a single-block scan of the tile totals,
// then a per-tile scan that adds the tile's carry. Tiles are 1024 threads x
// 8 elements.

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;
constexpr int64_t kScanTile = (int64_t)kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* total) {
  __shared__ int64_t warp_sums[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t s = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, s, d);
      if (lane >= d) s += y;
    }
    warp_sums[lane] = s;
  }
  __syncthreads();
  int64_t prefix = (warp > 0 ? warp_sums[warp - 1] : 0) + x - v;
  *total = warp_sums[(blockDim.x >> 5) - 1];
  __syncthreads();
  return prefix;
}

__global__ void scan_tile_totals(const int64_t* __restrict__ in, int64_t count,
                                 int64_t* __restrict__ totals) {
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < count) s += in[base + i];
  int64_t total;
  block_exclusive_scan(s, &total);
  if (threadIdx.x == 0) totals[blockIdx.x] = total;
}

__global__ void scan_totals_single(int64_t* totals, int64_t tiles) {
  int64_t carry = 0;
  for (int64_t start = 0; start < tiles; start += kScanThreads) {
    int64_t i = start + threadIdx.x;
    int64_t v = i < tiles ? totals[i] : 0;
    int64_t total;
    int64_t ex = block_exclusive_scan(v, &total);
    if (i < tiles) totals[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) totals[tiles] = carry;
}

__global__ void scan_tiles(const int64_t* in, int64_t* out, int64_t count,
                           const int64_t* __restrict__ carries) {
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t vals[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    vals[i] = base + i < count ? in[base + i] : 0;
    s += vals[i];
  }
  int64_t total;
  int64_t ex = block_exclusive_scan(s, &total) + carries[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < count) out[base + i] = ex;
    ex += vals[i];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[count] = carries[gridDim.x];
}

int64_t scan_tmp_elems(int64_t count) { return (count + kScanTile - 1) / kScanTile + 2; }

gs_status exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t count, int64_t* tmp,
                             cudaStream_t stream) {
  if (count <= 0) {
    GS_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), stream));
    return GS_OK;
  }
  int64_t tiles = (count + kScanTile - 1) / kScanTile;
  if (tiles > INT32_MAX) {
    set_error("scan of %lld elements exceeds the grid limit", (long long)count);
    return GS_EINVAL;
  }
  scan_tile_totals<<<(unsigned)tiles, kScanThreads, 0, stream>>>(in, count, tmp);
  scan_totals_single<<<1, kScanThreads, 0, stream>>>(tmp, tiles);
  scan_tiles<<<(unsigned)tiles, kScanThreads, 0, stream>>>(in, out, count, tmp);
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

// ---------------------------------------------------------------- workspace

gs_status ws_reserve(gs_workspace* ws, int slot, size_t bytes, cudaStream_t stream, void** out) {
  if (bytes == 0) bytes = 256;
  if (ws->cap[slot] < bytes) {
    if (ws->buf[slot] != nullptr) {
      GS_CUDA(cudaStreamSynchronize(ws->last_stream));
      GS_CUDA(cudaStreamSynchronize(stream));
      GS_CUDA(cudaFree(ws->buf[slot]));
      ws->buf[slot] = nullptr;
      ws->cap[slot] = 0;
    }
    size_t grow = bytes + bytes / 8;
    cudaError_t e = cudaMalloc(&ws->buf[slot], grow);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("workspace: cudaMalloc of %zu bytes failed (%s)", grow, cudaGetErrorString(e));
      return GS_ENOMEM;
    }
    ws->cap[slot] = grow;
  }
  ws->last_stream = stream;
  *out = ws->buf[slot];
  return GS_OK;
}

}  // namespace gs

extern "C" {

const char* gs_last_error(void) { return gs::g_err; }

const char* gs_version(void) { return "libgraphlet 0.1 (sm_103a)"; }

gs_status gs_workspace_create(gs_workspace** out) {
  if (out == nullptr) {
    gs::set_error("gs_workspace_create: null output pointer");
    return GS_EINVAL;
  }
  gs_workspace* ws = new gs_workspace();
  memset(ws, 0, sizeof(*ws));
  cudaGetDevice(&ws->device);
  *out = ws;
  return GS_OK;
}

gs_status gs_workspace_destroy(gs_workspace* ws) {
  if (ws == nullptr) return GS_OK;
  for (int i = 0; i < 5; ++i)
    if (ws->buf[i]) {
      cudaStreamSynchronize(ws->last_stream);
      cudaFree(ws->buf[i]);
    }
  if (ws->ev[0] != nullptr)
    for (int i = 0; i < 12; ++i) cudaEventDestroy(ws->ev[i]);
  delete ws;
  return GS_OK;
}

gs_status gs_workspace_set_timing(gs_workspace* ws, int enable) {
  if (ws == nullptr) {
    gs::set_error("gs_workspace_set_timing: null workspace");
    return GS_EINVAL;
  }
  if (enable && ws->ev[0] == nullptr)
    for (int i = 0; i < 12; ++i) GS_CUDA(cudaEventCreate(&ws->ev[i]));
  ws->timing = enable ? 1 : 0;
  return GS_OK;
}

gs_status gs_count_stats(const gs_workspace* ws, gs_stats* out) {
  if (ws == nullptr || out == nullptr) {
    gs::set_error("gs_count_stats: null argument");
    return GS_EINVAL;
  }
  *out = ws->stats;
  out->launches_total = ws->launches_total;
  return GS_OK;
}

gs_status gs_workspace_bytes(const gs_workspace* ws, uint64_t* bytes) {
  if (ws == nullptr || bytes == nullptr) {
    gs::set_error("gs_workspace_bytes: null argument");
    return GS_EINVAL;
  }
  *bytes = ws->cap[0] + ws->cap[1] + ws->cap[2] + ws->cap[3] + ws->cap[4];
  return GS_OK;
}

}  // extern "C"
