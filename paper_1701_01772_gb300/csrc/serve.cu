// Serving: continuous batching of estimation requests over resident graphs.
//
// Each resident graph keeps its own registration and hub index (sharing one
// index between graphs would hand the hub slots to the largest graph and
// slow every other one down). Worker lanes (host threads, each with its own
// CUDA stream and workspace) take queued requests in arrival order while the
// batch's estimated device memory fits the server budget next to what the
// other lanes hold (the estimate stays reserved until the batch finishes)
// and while the requests are of like estimated length (seconds per sampled
// edge of each graph and mask class, learnt from the groups counted so
// far), so that a short request is not held behind a long one.
// A batch is counted graph by graph: all its requests on one graph are
// sampled (the same sampler and seeds as gs_sample), concatenated and
// counted in one pass whose fold sums each request's edges separately.
// Per-edge counts do not depend on the other edges of a pass, so a result is
// identical alone and in any mix. Requests that arrive while a lane's batch
// is on the GPU are picked up by the next free lane, so batches overlap on
// the device.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace gs {

// Sum of roundup32(min(d_u, d_v)) over canonical edges u < v (4-node
// positions), for the memory estimate. One warp per vertex.
__global__ void k_positions(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                            const int64_t* __restrict__ up_ptr, int64_t n,
                            unsigned long long* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  unsigned long long s = 0;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
    const int64_t du = row_ptr[u + 1] - row_ptr[u];
    for (int64_t p = up_ptr[u] + lane; p < row_ptr[u + 1]; p += 32) {
      const int32_t v = col[p];
      const int64_t dv = row_ptr[v + 1] - row_ptr[v];
      const int64_t dm = du < dv ? du : dv;
      s += (unsigned long long)((dm + 31) & ~(int64_t)31);
    }
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0 && s) atomicAdd(out, s);
}

}  // namespace gs

using namespace gs;

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Source {
  const int64_t* row_ptr;
  const int32_t* col;
  int64_t n, nnz;
};

struct Req {
  gs_request r;
  uint64_t ticket;
  double t_submit, t_start, t_done;
  int64_t est_bytes;
  double est_s;  // estimated service time (admission)
  int64_t k;
  int64_t batch_size;
  gs_status status;
  int done;
  gs_result res;
};

}  // namespace

struct gs_server {
  int device = 0;
  uint64_t budget;
  int max_batch;
  int lanes;
  std::vector<Source> src;
  std::vector<gs_graph*> graphs;  // one registration (and hub index) per graph
  std::vector<int64_t> m;
  std::vector<double> bytes_per_edge;
  // running service time per sampled edge, per graph and mask class (3-node
  // only, or with 4-node graphlets), learnt from the groups counted so far
  std::vector<double> sec_per_edge[2];
  // queue
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> pending;
  std::unordered_map<uint64_t, Req*> reqs;
  uint64_t next_ticket = 1;
  bool started = false, stopping = false;
  uint64_t reserved = 0, peak_reserved = 0;
  int in_flight = 0, peak_in_flight = 0;
  int64_t batches = 0, batched_requests = 0, completed = 0;
  std::vector<std::thread> threads;
  gs_status first_error = GS_OK;
};

namespace {

double now_s();
// Batches of requests estimated shorter than this together are not split.
constexpr double kBatchFloorSeconds = 0.002;

// Marks a finished group's requests done (results are final) and wakes the
// waiters, so a group does not wait for the rest of its batch.
void release(gs_server* s, std::vector<Req*>& grp, gs_status st) {
  const double t = now_s();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    for (Req* q : grp) {
      if (st != GS_OK) q->status = st;
      q->t_done = t;
      q->done = 1;
      s->completed += 1;
    }
  }
  s->cv_done.notify_all();
}

// Samples and counts one graph's requests of a batch in one pass.
gs_status process_group(gs_server* s, gs_workspace* ws, cudaStream_t stream, size_t gi,
                        std::vector<Req*>& grp, int32_t** pair_buf, int64_t* pair_cap,
                        int64_t** seg_dev, int64_t* seg_cap) {
  gs_graph* gr = s->graphs[gi];
  const int64_t nb = (int64_t)grp.size();
  std::vector<int64_t> seg(nb + 1, 0);
  uint32_t mask = 0;
  for (int64_t i = 0; i < nb; ++i) {
    Req* q = grp[i];
    mask |= q->r.mask;
    int64_t k = 0;
    int32_t* dst = nullptr;  // sample into workspace slot 3, then append
    GS_TRY(sample_range(gr, ws, q->r.fraction, q->r.seed, 0, gr->m, nullptr, 0, &k, &dst,
                        stream));
    if (seg[i] + k > *pair_cap) {
      int64_t cap = std::max<int64_t>(2 * *pair_cap, seg[i] + k + 1024);
      int32_t* nbuf = nullptr;
      GS_CUDA(cudaMalloc(&nbuf, sizeof(int32_t) * 2 * cap));
      if (*pair_buf != nullptr) {
        GS_CUDA(cudaMemcpyAsync(nbuf, *pair_buf, sizeof(int32_t) * 2 * seg[i],
                                cudaMemcpyDeviceToDevice, stream));
        GS_CUDA(cudaStreamSynchronize(stream));
        cudaFree(*pair_buf);
      }
      *pair_buf = nbuf;
      *pair_cap = cap;
    }
    if (k > 0)
      GS_CUDA(cudaMemcpyAsync(*pair_buf + 2 * seg[i], dst, sizeof(int32_t) * 2 * k,
                              cudaMemcpyDeviceToDevice, stream));
    q->k = k;
    seg[i + 1] = seg[i] + k;
  }
  const int64_t K = seg[nb];
  if (nb + 1 > *seg_cap) {
    cudaFree(*seg_dev);
    GS_CUDA(cudaMalloc(seg_dev, sizeof(int64_t) * (nb + 1)));
    *seg_cap = nb + 1;
  }
  GS_CUDA(cudaMemcpyAsync(*seg_dev, seg.data(), sizeof(int64_t) * (nb + 1),
                          cudaMemcpyHostToDevice, stream));
  std::vector<unsigned long long> h((size_t)nb * 32, 0);
  if (K > 0) {
    CountBufs b;
    const Tuning tu = ws->has_tuning ? ws->tuning : default_tuning();
    if (nb == 1) {
      // a request alone: the plain fold (one sum, no per-request segments)
      GS_TRY(count_run(gr, ws, *pair_buf, K, mask, false, nullptr, nullptr, 0, tu, b, stream,
                       "gs_server"));
      GS_CUDA(cudaMemcpyAsync(h.data(), b.sums, sizeof(unsigned long long) * 32,
                              cudaMemcpyDeviceToHost, stream));
    } else {
      GS_TRY(count_run(gr, ws, *pair_buf, K, mask, false, nullptr, *seg_dev, nb, tu, b, stream,
                       "gs_server"));
      GS_CUDA(cudaMemcpyAsync(h.data(), b.seg_sums, sizeof(unsigned long long) * nb * 32,
                              cudaMemcpyDeviceToHost, stream));
    }
  }
  GS_CUDA(cudaStreamSynchronize(stream));
  for (int64_t i = 0; i < nb; ++i) {
    Req* q = grp[i];
    gs_sums sums;
    memset(&sums, 0, sizeof(sums));
    sums.k = q->k;
    sums.m = gr->m;
    sums.mask = q->r.mask;
    store_sums(h.data() + 32 * i, q->r.mask, &sums);
    q->status = gs_estimate(&sums, q->r.z, &q->res);
  }
  return GS_OK;
}

int mask_class(uint32_t mask) {
  return (mask & (GS_G7 | GS_G8 | GS_G9 | GS_G10 | GS_G11 | GS_G12)) != 0 ? 1 : 0;
}

// Runs a batch graph group by graph group (smallest estimated groups first)
// and releases each group's results as soon as it is counted. On return
// `batch` holds the requests that were not released (after an error).
gs_status run_batch(gs_server* s, gs_workspace* ws, cudaStream_t stream, std::vector<Req*>& batch,
                    int32_t** pair_buf, int64_t* pair_cap, int64_t** seg_dev, int64_t* seg_cap) {
  std::vector<std::vector<Req*>> groups(s->graphs.size());
  std::vector<double> est(s->graphs.size(), 0.0);
  for (Req* q : batch) {
    groups[q->r.graph].push_back(q);
    est[q->r.graph] += (double)q->est_bytes;
  }
  batch.clear();
  std::vector<size_t> order;
  for (size_t gi = 0; gi < groups.size(); ++gi)
    if (!groups[gi].empty()) order.push_back(gi);
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return est[a] < est[b]; });
  for (size_t k = 0; k < order.size(); ++k) {
    const double tg = now_s();
    gs_status st = process_group(s, ws, stream, order[k], groups[order[k]], pair_buf, pair_cap,
                                 seg_dev, seg_cap);
    if (st == GS_OK) {
      // learn the seconds per sampled edge of the classes in this group
      int64_t K = 0;
      bool c[2] = {false, false};
      for (Req* q : groups[order[k]]) {
        K += q->k;
        c[mask_class(q->r.mask)] = true;
      }
      if (K > 0) {
        const double r = (now_s() - tg) / (double)K;
        std::lock_guard<std::mutex> lock(s->mu);
        for (int ci = 0; ci < 2; ++ci) {
          if (!c[ci]) continue;
          double& x = s->sec_per_edge[ci][order[k]];
          x = x > 0.0 ? 0.7 * x + 0.3 * r : r;
        }
      }
    }
    if (st != GS_OK) {
      for (size_t r = k; r < order.size(); ++r)
        batch.insert(batch.end(), groups[order[r]].begin(), groups[order[r]].end());
      return st;
    }
    release(s, groups[order[k]], GS_OK);
  }
  return GS_OK;
}

void lane_main(gs_server* s) {
  cudaStream_t stream = nullptr;
  gs_workspace* ws = nullptr;
  int32_t* pair_buf = nullptr;
  int64_t pair_cap = 0;
  int64_t* seg_dev = nullptr;
  int64_t seg_cap = 0;
  cudaSetDevice(s->device);
  cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
  gs_workspace_create(&ws);
  for (;;) {
    std::vector<Req*> batch;
    int64_t est = 0;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      s->cv_work.wait(lock, [&] { return s->stopping || !s->pending.empty(); });
      if (s->stopping) break;
      // admit FIFO while the estimate fits the budget next to other lanes
      // and the requests are of like length: a request joins the batch only
      // while the batch's estimated time stays within twice the first
      // request's (or a few milliseconds), so a short request is not held
      // behind a long pass of the same batch
      double t_head = 0.0, t_batch = 0.0;
      while (!s->pending.empty() && (int)batch.size() < s->max_batch) {
        Req* q = s->pending.front();
        const bool alone = batch.empty() && s->reserved == 0;
        if (!alone && s->reserved + est + (uint64_t)q->est_bytes > s->budget) break;
        const double tq = s->sec_per_edge[mask_class(q->r.mask)][q->r.graph] *
                          q->r.fraction * (double)s->m[q->r.graph];
        if (!batch.empty() && t_batch + tq > std::max(2.0 * t_head, kBatchFloorSeconds)) break;
        if (batch.empty()) t_head = tq;
        t_batch += tq;
        q->est_s = tq;
        s->pending.pop_front();
        batch.push_back(q);
        est += q->est_bytes;
      }
      if (batch.empty()) {
        // the head request must wait for memory held by another lane
        s->cv_work.wait_for(lock, std::chrono::milliseconds(1));
        continue;
      }
      s->reserved += est;
      s->peak_reserved = std::max(s->peak_reserved, s->reserved);
      s->in_flight += 1;
      s->peak_in_flight = std::max(s->peak_in_flight, s->in_flight);
      s->batches += 1;
      s->batched_requests += (int64_t)batch.size();
    }
    const double t0 = now_s();
    for (Req* q : batch) {
      q->t_start = t0;
      q->batch_size = (int64_t)batch.size();
    }
    gs_status st = run_batch(s, ws, stream, batch, &pair_buf, &pair_cap, &seg_dev, &seg_cap);
    // requests of groups that did not finish (an error) are completed here;
    // released requests may already be gone, so only `batch` is touched
    if (!batch.empty()) release(s, batch, st != GS_OK ? st : GS_ECUDA);
    {
      std::lock_guard<std::mutex> lock(s->mu);
      if (st != GS_OK && s->first_error == GS_OK) s->first_error = st;
      s->reserved -= est;
      s->in_flight -= 1;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
  cudaStreamSynchronize(stream);
  cudaFree(pair_buf);
  cudaFree(seg_dev);
  gs_workspace_destroy(ws);
  cudaStreamDestroy(stream);
}

}  // namespace

extern "C" gs_status gs_server_create(uint64_t hbm_budget_bytes, int32_t max_batch, int32_t lanes,
                                      gs_server** out) {
  if (out == nullptr || hbm_budget_bytes == 0 || max_batch < 1 || lanes < 1 || lanes > 16) {
    set_error("gs_server_create: invalid arguments (budget > 0, max_batch >= 1, lanes 1..16)");
    return GS_EINVAL;
  }
  gs_server* s = new gs_server();
  s->budget = hbm_budget_bytes;
  s->max_batch = max_batch;
  s->lanes = lanes;
  *out = s;
  return GS_OK;
}

extern "C" gs_status gs_server_add_graph(gs_server* s, const int64_t* d_row_ptr,
                                         const int32_t* d_col, int64_t n, int64_t nnz,
                                         int32_t* graph_id) {
  if (s == nullptr || graph_id == nullptr || d_row_ptr == nullptr || n < 0 || nnz < 0 ||
      (nnz > 0 && d_col == nullptr)) {
    set_error("gs_server_add_graph: invalid arguments");
    return GS_EINVAL;
  }
  if (s->started) {
    set_error("gs_server_add_graph: graphs must be added before gs_server_start");
    return GS_EINVAL;
  }
  *graph_id = (int32_t)s->src.size();
  s->src.push_back(Source{d_row_ptr, d_col, n, nnz});
  return GS_OK;
}

extern "C" gs_status gs_server_start(gs_server* s, uint32_t flags, uint64_t hub_budget_bytes,
                                     void* stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (s == nullptr || s->started || s->src.empty()) {
    set_error("gs_server_start: no graphs added, or already started");
    return GS_EINVAL;
  }
  GS_CUDA(cudaGetDevice(&s->device));
  const size_t G = s->src.size();
  unsigned long long* d_pos = nullptr;
  GS_CUDA(cudaMalloc(&d_pos, sizeof(unsigned long long)));
  for (size_t g = 0; g < G; ++g) {
    const Source& c = s->src[g];
    gs_graph* gr = nullptr;
    gs_status st = gs_graph_create(c.row_ptr, c.col, c.n, c.nnz, flags, hub_budget_bytes, stream,
                                   &gr);
    if (st != GS_OK) {
      cudaFree(d_pos);
      return st;
    }
    s->graphs.push_back(gr);
    unsigned long long pos = 0;
    GS_CUDA(cudaMemsetAsync(d_pos, 0, sizeof(unsigned long long), stream));
    if (c.n > 0)
      k_positions<<<grid_for(c.n * 32, 256, 8), 256, 0, stream>>>(c.row_ptr, c.col, gr->up_ptr,
                                                                  c.n, d_pos);
    GS_CUDA(cudaMemcpyAsync(&pos, d_pos, sizeof(pos), cudaMemcpyDeviceToHost, stream));
    GS_CUDA(cudaStreamSynchronize(stream));
    s->m.push_back(gr->m);
    // per sampled edge: ~120 B of per-edge arrays plus, per 4-node position,
    // T-bit / cost / task words (20/32 B) and a T entry allowance (1 B)
    const double pp = gr->m > 0 ? (double)pos / (double)gr->m : 0.0;
    s->bytes_per_edge.push_back(120.0 + 1.625 * pp);
    s->sec_per_edge[0].push_back(0.0);  // learnt from the first groups counted
    s->sec_per_edge[1].push_back(0.0);
  }
  cudaFree(d_pos);
  s->started = true;
  for (int i = 0; i < s->lanes; ++i) s->threads.emplace_back(lane_main, s);
  return GS_OK;
}

extern "C" gs_status gs_server_submit(gs_server* s, const gs_request* r, uint64_t* ticket) {
  if (s == nullptr || r == nullptr || ticket == nullptr || !s->started) {
    set_error("gs_server_submit: invalid arguments or server not started");
    return GS_EINVAL;
  }
  if (r->graph < 0 || r->graph >= (int32_t)s->src.size() || r->mask == 0 ||
      (r->mask & ~(uint32_t)GS_CONNECTED) != 0 || !(r->fraction >= 0.0 && r->fraction <= 1.0) ||
      !(r->z >= 0.0)) {
    set_error("gs_server_submit: bad request (graph id, mask, fraction in [0,1], z >= 0)");
    return GS_EINVAL;
  }
  Req* q = new Req();
  memset(q, 0, sizeof(*q));
  q->r = *r;
  q->t_submit = now_s();
  const double kexp = r->fraction * (double)s->m[r->graph];
  const bool four = (r->mask & ~(uint32_t)GS_THREE_NODE) != 0;
  // 3-node requests need only the per-edge arrays
  const double bpe = four ? s->bytes_per_edge[r->graph] : 120.0;
  q->est_bytes = (int64_t)((kexp + 4.0 * sqrt(kexp + 1.0) + 64.0) * bpe);
  if ((uint64_t)q->est_bytes > s->budget) {
    delete q;
    set_error("gs_server_submit: the request's estimated memory exceeds the server budget");
    return GS_EBUDGET;
  }
  {
    std::lock_guard<std::mutex> lock(s->mu);
    q->ticket = s->next_ticket++;
    s->reqs[q->ticket] = q;
    s->pending.push_back(q);
    *ticket = q->ticket;
  }
  s->cv_work.notify_one();
  return GS_OK;
}

static void fill_req_stats(const Req* q, gs_request_stats* st) {
  if (st == nullptr) return;
  st->k = q->k;
  st->batch_size = q->batch_size;
  st->queue_s = q->t_start - q->t_submit;
  st->latency_s = q->t_done - q->t_submit;
  st->est_bytes = q->est_bytes;
}

extern "C" gs_status gs_server_wait(gs_server* s, uint64_t ticket, double timeout_s,
                                    gs_result* out, gs_request_stats* st) {
  if (s == nullptr || out == nullptr) {
    set_error("gs_server_wait: invalid arguments");
    return GS_EINVAL;
  }
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) {
    set_error("gs_server_wait: unknown ticket %llu", (unsigned long long)ticket);
    return GS_EINVAL;
  }
  Req* q = it->second;
  const auto until = std::chrono::steady_clock::now() +
                     std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                         std::chrono::duration<double>(timeout_s));
  if (!s->cv_done.wait_until(lock, until, [&] { return q->done != 0; })) {
    set_error("gs_server_wait: request %llu not finished within %.3f s",
              (unsigned long long)ticket, timeout_s);
    return GS_ETIMEOUT;
  }
  *out = q->res;
  fill_req_stats(q, st);
  gs_status status = q->status;
  s->reqs.erase(it);
  delete q;
  if (status != GS_OK) set_error("gs_server_wait: request %llu failed", (unsigned long long)ticket);
  return status;
}

extern "C" gs_status gs_server_info(gs_server* s, gs_server_stats* out) {
  if (s == nullptr || out == nullptr) {
    set_error("gs_server_info: invalid arguments");
    return GS_EINVAL;
  }
  std::lock_guard<std::mutex> lock(s->mu);
  memset(out, 0, sizeof(*out));
  out->graphs = (int64_t)s->src.size();
  out->batches = s->batches;
  out->completed = s->completed;
  out->pending = (int64_t)s->pending.size();
  out->mean_batch = s->batches ? (double)s->batched_requests / (double)s->batches : 0.0;
  out->peak_reserved_bytes = s->peak_reserved;
  out->peak_in_flight = s->peak_in_flight;
  out->budget_bytes = s->budget;
  return GS_OK;
}

extern "C" gs_status gs_server_destroy(gs_server* s) {
  if (s == nullptr) return GS_OK;
  {
    // queued requests that no worker has taken are cancelled; batches
    // already on the device finish first
    std::lock_guard<std::mutex> lock(s->mu);
    s->stopping = true;
    for (Req* q : s->pending) {
      q->status = GS_ECANCELLED;
      q->done = 1;
    }
    s->pending.clear();
  }
  s->cv_work.notify_all();
  s->cv_done.notify_all();
  for (auto& t : s->threads) t.join();
  for (auto& kv : s->reqs) delete kv.second;
  for (gs_graph* g : s->graphs) gs_graph_destroy(g);
  delete s;
  return GS_OK;
}
