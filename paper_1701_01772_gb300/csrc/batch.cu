// Batched exact counting over many small graphs in one CUDA-graph launch.
//
// The batch is registered as the disjoint union of its graphs (vertex ids
// shifted by each graph's vertex offset). A disjoint union has no edges
// between its parts, so every per-edge count (t, k, q of Algorithms 2-4) is
// the same as in the edge's own graph; the edges of graph g are a contiguous
// range of the union's canonical edge order, and the fold sums each range
// separately (one exact 128-bit sum set per graph).
//
// gs_batch_create sizes every buffer with one synchronised run, lets an
// autotuner time a small grid of launch choices (resident CTAs per SM of
// the two passes, 4-node work-unit size, hub index on/off) and captures the
// whole kernel sequence of the best one into a CUDA graph. gs_batch_count
// replays that graph: one host launch for all graphs of the batch.
#include <string.h>

#include <vector>

#include "common.cuh"

namespace gs {

// col_global[p] = col_local[p] + vtx_off[g] for the rows of graph g; local
// ids are checked against the graph's vertex count. One block per graph.
__global__ void k_batch_globalize(const int64_t* __restrict__ vtx_off,
                                  const int64_t* __restrict__ row_ptr,
                                  const int32_t* __restrict__ col_local, int64_t num_graphs,
                                  int32_t* __restrict__ col_global, DevError* err) {
  for (int64_t gi = blockIdx.x; gi < num_graphs; gi += gridDim.x) {
    const int64_t v0 = vtx_off[gi], v1 = vtx_off[gi + 1];
    const int64_t n = v1 - v0;
    for (int64_t p = row_ptr[v0] + threadIdx.x; p < row_ptr[v1]; p += blockDim.x) {
      const int32_t x = col_local[p];
      if (x < 0 || x >= n) {
        raise_error(err, GS_EINVAL, p);
        col_global[p] = (int32_t)v0;  // keeps later checks in range
      } else {
        col_global[p] = (int32_t)(v0 + x);
      }
    }
  }
}

// seg_off[g] = first canonical edge of graph g = edge_off[vtx_off[g]].
__global__ void k_batch_segments(const int64_t* __restrict__ vtx_off,
                                 const int64_t* __restrict__ edge_off, int64_t num_graphs,
                                 int64_t* __restrict__ seg_off) {
  for (int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gi <= num_graphs;
       gi += (int64_t)gridDim.x * blockDim.x)
    seg_off[gi] = edge_off[vtx_off[gi]];
}

}  // namespace gs

using namespace gs;

struct gs_batch {
  int64_t num_graphs;
  uint32_t mask;
  int32_t* col_global;
  int64_t* seg_off;
  int64_t* vtx_off_copy;
  DevError* err;
  gs_graph* graph;
  gs_workspace* ws;
  CountBufs bufs;
  Tuning tuning;
  cudaGraph_t cgraph;
  cudaGraphExec_t exec;
  std::vector<int64_t> edges;   // edges per graph
  std::vector<float> tune_ms;   // time of each autotuner candidate
  std::vector<Tuning> tune_cands;
  float best_ms;
  int64_t kernels;              // kernel nodes in the captured graph
};

namespace {

// The captured sequence: everything after sizing, no host synchronisation.
int64_t enqueue_batch(gs_batch* b, const Tuning& tu, cudaStream_t stream) {
  const bool need_k = (b->mask & (GS_G7 | GS_G8 | GS_G9 | GS_G11)) != 0;
  const bool need_q = (b->mask & (GS_G10 | GS_G12)) != 0;
  const bool four = need_k || need_q;
  const DevGraph g = graph_view(b->graph, tu);
  CountBufs& c = b->bufs;
  int64_t n = 0;
  n += launch_front(b->graph, g, c.pairs_all, four, c, stream);
  n += launch_tri(g, four, tu, c, stream);
  if (four) {
    n += launch_scan_t(c, stream);
    n += launch_compact(g, c, stream);
    n += launch_tmask(g, c, stream);
    n += launch_cost(g, need_k, need_q, tu, c, stream);
    n += launch_quad(g, need_k, need_q, tu, c, stream);
    n += launch_dense(g, need_q, c, stream);
  }
  n += launch_fold_seg(g, four, b->seg_off, c, stream);
  return n;
}

void destroy_batch(gs_batch* b) {
  if (b == nullptr) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cgraph) cudaGraphDestroy(b->cgraph);
  if (b->graph) gs_graph_destroy(b->graph);
  if (b->ws) gs_workspace_destroy(b->ws);
  cudaFree(b->col_global);
  cudaFree(b->seg_off);
  cudaFree(b->err);
  delete b;
}

}  // namespace

extern "C" gs_status gs_batch_create(const int64_t* d_vtx_off, const int64_t* d_row_ptr,
                                     const int32_t* d_col, int64_t num_graphs, int64_t total_n,
                                     int64_t total_nnz, uint32_t mask, uint32_t flags,
                                     uint64_t hub_budget_bytes, void* stream_, gs_batch** out) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (out == nullptr || d_vtx_off == nullptr || d_row_ptr == nullptr || num_graphs < 1 ||
      total_n < 0 || total_nnz < 0 || (total_nnz > 0 && d_col == nullptr) || mask == 0 ||
      (mask & ~(uint32_t)GS_CONNECTED) != 0) {
    set_error("gs_batch_create: invalid arguments");
    return GS_EINVAL;
  }
  gs_batch* b = new gs_batch();
  b->num_graphs = num_graphs;
  b->mask = mask;
  b->tuning = default_tuning();
  auto fail = [&](gs_status s) {
    destroy_batch(b);
    return s;
  };
  // host check of the graph offsets
  std::vector<int64_t> hv(num_graphs + 1);
  GS_CUDA(cudaMemcpyAsync(hv.data(), d_vtx_off, sizeof(int64_t) * (num_graphs + 1),
                          cudaMemcpyDeviceToHost, stream));
  GS_CUDA(cudaStreamSynchronize(stream));
  if (hv[0] != 0 || hv[num_graphs] != total_n) {
    set_error("gs_batch_create: vtx_off must start at 0 and end at total_n");
    return fail(GS_EINVAL);
  }
  for (int64_t i = 0; i < num_graphs; ++i)
    if (hv[i + 1] < hv[i]) {
      set_error("gs_batch_create: vtx_off must be non-decreasing");
      return fail(GS_EINVAL);
    }
  // union graph with global ids
  if (cudaMalloc(&b->col_global, sizeof(int32_t) * (size_t)(total_nnz > 0 ? total_nnz : 1)) !=
          cudaSuccess ||
      cudaMalloc(&b->seg_off, sizeof(int64_t) * (size_t)(num_graphs + 1)) != cudaSuccess ||
      cudaMalloc(&b->err, sizeof(DevError)) != cudaSuccess) {
    cudaGetLastError();
    set_error("gs_batch_create: out of device memory");
    return fail(GS_ENOMEM);
  }
  GS_CUDA(cudaMemsetAsync(b->err, 0, sizeof(DevError), stream));
  if (total_nnz > 0)
    k_batch_globalize<<<grid_for(num_graphs * 256, 256, 8), 256, 0, stream>>>(
        d_vtx_off, d_row_ptr, d_col, num_graphs, b->col_global, b->err);
  gs_status s = fetch_error(b->err, stream, "gs_batch_create (local vertex id out of range)");
  if (s != GS_OK) return fail(GS_EINVAL);
  s = gs_graph_create(d_row_ptr, b->col_global, total_n, total_nnz, flags,
                                hub_budget_bytes, stream, &b->graph);
  if (s != GS_OK) {
    b->graph = nullptr;
    return fail(s);
  }
  // adjacency bit matrices for the member graphs (all of them are small in
  // the intended use): every membership test becomes one word load
  s = build_dense_blocks(b->graph, hv.data(), num_graphs, (uint64_t)24 << 30, stream);
  if (s != GS_OK) return fail(s);
  k_batch_segments<<<grid_for(num_graphs + 1, 256, 4), 256, 0, stream>>>(
      d_vtx_off, b->graph->edge_off, num_graphs, b->seg_off);
  b->edges.resize(num_graphs + 1);
  GS_CUDA(cudaMemcpyAsync(b->edges.data(), b->seg_off, sizeof(int64_t) * (num_graphs + 1),
                          cudaMemcpyDeviceToHost, stream));
  GS_CUDA(cudaStreamSynchronize(stream));
  for (int64_t i = 0; i < num_graphs; ++i) b->edges[i] = b->edges[i + 1] - b->edges[i];
  b->edges.pop_back();
  s = gs_workspace_create(&b->ws);
  if (s != GS_OK) return fail(s);
  const int64_t M = b->graph->m;
  if (M == 0) {
    *out = b;
    return GS_OK;
  }
  // sizing run (allocates every buffer, materialises the edge list)
  s = count_run(b->graph, b->ws, nullptr, M, mask, false, nullptr, b->seg_off, num_graphs,
                b->tuning, b->bufs, stream, "gs_batch_create");
  if (s != GS_OK) return fail(s);
  GS_CUDA(cudaStreamSynchronize(stream));

  // autotuner: time each candidate on the real batch, keep the fastest
  if (flags & GS_BATCH_AUTOTUNE) {
    const int tri_opts[2] = {4, 8};
    const int quad_opts[2] = {4, quad_blocks_limit()};
    const int64_t task_opts[3] = {256, 1024, 4096};
    const int hub_opts[2] = {1, 0};
    cudaEvent_t e0, e1;
    GS_CUDA(cudaEventCreate(&e0));
    GS_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int h : hub_opts)
      for (int tq : tri_opts)
        for (int qq : quad_opts)
          for (int64_t tp : task_opts) {
            const Tuning tu{tq, qq, tp, h, kHubDenseSlots};
            enqueue_batch(b, tu, stream);  // warm
            cudaEventRecord(e0, stream);
            enqueue_batch(b, tu, stream);
            cudaEventRecord(e1, stream);
            cudaError_t ce = cudaEventSynchronize(e1);
            if (ce != cudaSuccess) {
              cudaEventDestroy(e0);
              cudaEventDestroy(e1);
              return fail(cuda_fail(ce, "gs_batch_create autotune", __FILE__, __LINE__));
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            b->tune_cands.push_back(tu);
            b->tune_ms.push_back(ms);
            if (ms < best) {
              best = ms;
              b->tuning = tu;
            }
          }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->best_ms = best;
  }
  // capture the chosen sequence into one CUDA graph
  cudaStream_t cap = nullptr;
  GS_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaError_t ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (ce == cudaSuccess) {
    b->kernels = enqueue_batch(b, b->tuning, cap);
    ce = cudaStreamEndCapture(cap, &b->cgraph);
  }
  if (ce == cudaSuccess) ce = cudaGraphInstantiate(&b->exec, b->cgraph, 0);
  cudaStreamDestroy(cap);
  if (ce != cudaSuccess) return fail(cuda_fail(ce, "gs_batch_create capture", __FILE__, __LINE__));
  *out = b;
  return GS_OK;
}

extern "C" gs_status gs_batch_count(gs_batch* b, gs_sums* h_sums, void* stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (b == nullptr || h_sums == nullptr) {
    set_error("gs_batch_count: invalid arguments");
    return GS_EINVAL;
  }
  const int64_t G = b->num_graphs;
  for (int64_t i = 0; i < G; ++i) {
    memset(&h_sums[i], 0, sizeof(gs_sums));
    h_sums[i].k = h_sums[i].m = b->edges[i];
    h_sums[i].mask = b->mask;
  }
  if (b->exec == nullptr) return GS_OK;  // no edges at all
  GS_CUDA(cudaGraphLaunch(b->exec, stream));
  std::vector<unsigned long long> h((size_t)G * 32);
  GS_CUDA(cudaMemcpyAsync(h.data(), b->bufs.seg_sums, sizeof(unsigned long long) * G * 32,
                          cudaMemcpyDeviceToHost, stream));
  GS_CUDA(cudaStreamSynchronize(stream));
  for (int64_t i = 0; i < G; ++i) store_sums(h.data() + 32 * i, b->mask, &h_sums[i]);
  b->ws->launches_total += b->kernels;
  return GS_OK;
}

extern "C" gs_status gs_batch_info(const gs_batch* b, gs_batch_stats* out) {
  if (b == nullptr || out == nullptr) {
    set_error("gs_batch_info: invalid arguments");
    return GS_EINVAL;
  }
  memset(out, 0, sizeof(*out));
  out->num_graphs = b->num_graphs;
  out->edges = b->graph ? b->graph->m : 0;
  out->tri_blocks_per_sm = b->tuning.tri_blocks_per_sm;
  out->quad_blocks_per_sm = b->tuning.quad_blocks_per_sm;
  out->task_probes = b->tuning.task_probes;
  out->use_hubs = b->tuning.use_hubs;
  out->graph_kernels = b->kernels;
  out->candidates = (int32_t)b->tune_ms.size();
  out->best_ms = b->best_ms;
  float worst = 0;
  for (float v : b->tune_ms) worst = v > worst ? v : worst;
  out->worst_ms = worst;
  out->workspace_bytes = 0;
  if (b->ws) gs_workspace_bytes(b->ws, &out->workspace_bytes);
  return GS_OK;
}

extern "C" gs_status gs_batch_destroy(gs_batch* b) {
  destroy_batch(b);
  return GS_OK;
}
