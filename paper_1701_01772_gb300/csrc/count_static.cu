// gs_count3_static: the triangle / 2-star count of gs_count for callers that
// cannot allocate device memory. Everything it needs beyond the caller's
// inputs and outputs lives in one file-scope device array whose size is
// fixed at compile time.
//
// Who needs this: hosts that hand the GPU a fixed memory pool when they
// start and forbid any later growth (embedded or real-time serving, where a
// failed allocation in the middle of a request is not an option), and
// latency paths where a cudaMalloc / cudaFree pair is too costly (both can
// wait for the whole device to become idle). The graph itself is still
// registered once with gs_graph_create at set-up time.
#include <mutex>
#include <string.h>

#include "common.cuh"

namespace gs {

// Kernels of the regular counting path (count.cu), launched here unchanged.
__global__ void k_prep(DevGraph g, const int32_t* __restrict__ pairs, int64_t K, int pad,
                       unsigned long long* __restrict__ dup_table, int64_t dup_mask,
                       int2* __restrict__ uv, int64_t* __restrict__ len, DevError* err);
void launch_tri_unpadded(const DevGraph& g, const int2* uv, const int64_t* off, int64_t K,
                         unsigned long long* t, int blocks, cudaStream_t stream);
__global__ void __launch_bounds__(256)
    k_fold(DevGraph g, const int2* __restrict__ uv, int64_t K, const unsigned long long* __restrict__ t,
                       const unsigned long long* __restrict__ k2,
                       const unsigned long long* __restrict__ q, const int64_t* __restrict__ tdeg,
                       const int64_t* __restrict__ nbr_degsum, int need_k, int need_q,
                       int64_t* __restrict__ per_edge, unsigned __int128* __restrict__ part,
                       unsigned long long* __restrict__ stats);
__global__ void k_fold_final(const unsigned __int128* __restrict__ part, int blocks,
                             unsigned long long* __restrict__ out);

namespace {

constexpr int kThreads = 256;
constexpr int kFoldBlocksMax = 1024;

// The scratch: GS_STATIC_SCRATCH_BYTES of device memory, reserved on every
// GPU that loads this library's code (possibly only at the first call, when
// the CUDA runtime loads modules lazily) for as long as the process runs.
static __device__ __align__(256) unsigned char g_static_scratch[GS_STATIC_SCRATCH_BYTES];

// Device address of g_static_scratch per device. In host code the symbol
// name is only a host-side handle, so the address must be looked up with
// cudaGetSymbolAddress while that device is current.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

gs_status scratch_address(void** out) {
  int dev = 0;
  GS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("gs_count3_static: device ordinal %d out of range", dev);
    return GS_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || p == nullptr) {
      set_error("gs_count3_static: cudaGetSymbolAddress failed on device %d (%s)", dev,
                cudaGetErrorString(e));
      return GS_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return GS_OK;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status gs_count3_static(const gs_graph* gr, const int32_t* d_pairs, int64_t K,
                                      uint32_t mask, gs_sums* h_sums, void* stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (gr == nullptr || h_sums == nullptr || K < 0 || mask == 0 ||
      (mask & ~(uint32_t)GS_THREE_NODE) != 0 || (K > 0 && d_pairs == nullptr)) {
    set_error("gs_count3_static: invalid arguments (mask must be a non-empty subset of "
              "GS_THREE_NODE and d_pairs must be given)");
    return GS_EINVAL;
  }
  if (K > GS_STATIC_MAX_PAIRS) {
    set_error("gs_count3_static: %lld sampled edges exceed the fixed scratch limit of %d; "
              "use gs_count for larger samples",
              (long long)K, (int)GS_STATIC_MAX_PAIRS);
    return GS_ECAPACITY;
  }
  void* base = nullptr;
  GS_TRY(scratch_address(&base));
  memset(h_sums, 0, sizeof(*h_sums));
  h_sums->k = K;
  h_sums->m = gr->m;
  h_sums->mask = mask;
  if (K == 0) return GS_OK;

  const DevGraph& g = gr->dev;
  int64_t dup_cap = 1;
  while (dup_cap < 2 * K) dup_cap <<= 1;
  int fold_blocks = grid_for(K, kThreads, 2);
  if (fold_blocks > kFoldBlocksMax) fold_blocks = kFoldBlocksMax;

  Carve c{(char*)base, 0};
  DevError* d_err = c.take<DevError>(1);
  unsigned long long* d_sums = c.take<unsigned long long>(32);
  unsigned long long* d_stats = c.take<unsigned long long>(8);
  int2* uv = c.take<int2>(K);
  int64_t* off = c.take<int64_t>(K + 1);
  unsigned long long* t = c.take<unsigned long long>(K);
  int64_t* tmp = c.take<int64_t>(scan_tmp_elems(K + 1));
  unsigned long long* dup = c.take<unsigned long long>(dup_cap);
  unsigned __int128* part = c.take<unsigned __int128>((int64_t)fold_blocks * 16);
  if (c.used > (size_t)GS_STATIC_SCRATCH_BYTES) {  // cannot happen for K <= the limit
    set_error("gs_count3_static: scratch layout exceeds GS_STATIC_SCRATCH_BYTES");
    return GS_ECAPACITY;
  }

  // The array keeps the previous call's contents: clear what accumulates.
  GS_CUDA(cudaMemsetAsync(d_err, 0, sizeof(DevError), stream));
  GS_CUDA(cudaMemsetAsync(d_stats, 0, sizeof(unsigned long long) * 8, stream));
  GS_CUDA(cudaMemsetAsync(t, 0, sizeof(unsigned long long) * K, stream));
  GS_CUDA(cudaMemsetAsync(dup, 0xff, sizeof(unsigned long long) * dup_cap, stream));
  k_prep<<<grid_for(K, kThreads, 8), kThreads, 0, stream>>>(g, d_pairs, K, 0, dup, dup_cap - 1,
                                                            uv, off, d_err);
  GS_TRY(exclusive_scan_i64(off, off, K, tmp, stream));
  DevError herr;
  GS_CUDA(cudaMemcpyAsync(&herr, d_err, sizeof(herr), cudaMemcpyDeviceToHost, stream));
  GS_CUDA(cudaStreamSynchronize(stream));
  if (herr.code != 0) {
    set_error("gs_count3_static: %s (pair %lld)",
              herr.code == GS_EDUPSAMPLE ? "edge sampled twice"
                                         : "sampled pair is out of range or not an edge",
              (long long)herr.index);
    return herr.code;
  }
  launch_tri_unpadded(g, uv, off, K, t, sm_count() * 4, stream);
  k_fold<<<fold_blocks, kThreads, 0, stream>>>(g, uv, K, t, nullptr, nullptr, nullptr,
                                                gr->nbr_degsum, 0, 0, nullptr, part, d_stats);
  k_fold_final<<<1, 32, 0, stream>>>(part, fold_blocks, d_sums);
  GS_CUDA(cudaGetLastError());
  unsigned long long h[32];
  GS_CUDA(cudaMemcpyAsync(h, d_sums, sizeof(h), cudaMemcpyDeviceToHost, stream));
  GS_CUDA(cudaStreamSynchronize(stream));
  static const uint32_t bit[2] = {GS_G3, GS_G4};
  for (int i = 0; i < 2; ++i) {
    if (!(mask & bit[i])) continue;
    h_sums->sum[i][0] = h[2 * i];
    h_sums->sum[i][1] = h[2 * i + 1];
    h_sums->sumsq[i][0] = h[2 * (8 + i)];
    h_sums->sumsq[i][1] = h[2 * (8 + i) + 1];
  }
  return GS_OK;
}
