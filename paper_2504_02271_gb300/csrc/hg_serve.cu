// hg_server: answers count, clustering-coefficient and sampled-estimate queries on
// hypergraphs kept resident on the device, with continuous batching.
//
// Queries are admitted in arrival order.  A worker that becomes free takes the oldest
// waiting query and everything that can share its launches:
//   * an exact query (counts, Def. 5.1 coefficient) takes every waiting exact query,
//     in order, whose hypergraph is already in the batch or still fits (member count,
//     device-memory budget); the batch is one hg_load_batch_members / build / count
//     over the distinct hypergraphs, each evaluated once however many queries ask;
//   * an estimate query (Algorithm 6) takes the waiting estimate queries on the same
//     hypergraph; they share one load and step one, then draw their own samples.
// Several workers, each with its own CUDA stream, run batches at the same time, so
// queries that arrive while others are on the device are admitted as workers and
// memory free up.  Every answer equals the one computed alone: exact counts do not
// depend on the batch, and sample n of a seed is the same Philox draw everywhere.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "hg_internal.cuh"

namespace {

struct ServeGraph {
  int32_t nv = 0, ne = 0;
  int64_t nnz = 0;
  int64_t* d_ptr = nullptr;   // server-owned device copies
  int32_t* d_idx = nullptr;
  uint64_t W = 0;             // hyperwedges (from step one when the hypergraph is added)
  size_t exact_bytes = 0;     // device memory of one exact evaluation (estimate)
  size_t sample_bytes = 0;    // device memory of one estimate evaluation (estimate)
};

struct Pending {
  uint64_t ticket;
  hg_query q;
  double t_submit;
};

constexpr int kMaxEstimateGroup = 256;

}  // namespace

struct hg_server {
  hg_server_options opt{};
  int device = 0;
  size_t budget = 0;
  std::vector<ServeGraph> graphs;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Pending> queue;
  std::unordered_set<uint64_t> outstanding;
  std::unordered_map<uint64_t, hg_result> done;
  uint64_t next_ticket = 1;
  size_t in_flight = 0;
  int running = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  std::chrono::steady_clock::time_point t0;
  hg_server_stats stats{};
};

namespace {

double now(const hg_server* S) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - S->t0).count();
}

bool is_exact(const hg_query& q) { return q.kind == HG_Q_COUNTS || q.kind == HG_Q_CLUSTERING; }

size_t bytes_of(const hg_server* S, const hg_query& q) {
  const ServeGraph& g = S->graphs[(size_t)q.graph];
  return is_exact(q) ? g.exact_bytes : g.sample_bytes;
}

// Device memory of one evaluation: inputs and transposes, step one (rows, degrees,
// oriented entries over all 2W slots), step two (team lists, scratch), with slack.
void size_graph(ServeGraph& g, int packed) {
  const size_t ne = (size_t)g.ne, nv = (size_t)g.nv, nnz = (size_t)g.nnz, W = (size_t)g.W;
  const size_t load = 16 * nnz + 40 * ne + 16 * nv;
  const size_t build = 48 * ne + (packed ? 4 : 8) * 2 * W;
  const size_t count = 32 * ne;
  const size_t slack = size_t(64) << 20;
  g.exact_bytes = load + build + count + slack;
  g.sample_bytes = load + build + 8 * ne + (packed ? 4 : 8) * W + slack;
}

// Take the oldest query and what can join it (the caller holds the lock).
void form_batch(hg_server* S, std::vector<Pending>& out, size_t& bytes) {
  const Pending head = S->queue.front();
  std::deque<Pending> rest;
  bytes = 0;
  if (is_exact(head.q)) {
    std::vector<int32_t> members;
    for (const Pending& p : S->queue) {
      bool take = false;
      if (is_exact(p.q)) {
        if ((int32_t)out.size() >= S->opt.max_batch_queries) {
          take = false;
        } else if (std::find(members.begin(), members.end(), p.q.graph) != members.end()) {
          take = true;
        } else {
          const size_t b = S->graphs[(size_t)p.q.graph].exact_bytes;
          const bool fits = S->in_flight + bytes + b <= S->budget;
          if ((int32_t)members.size() < S->opt.max_batch_graphs &&
              (members.empty() || fits)) {
            members.push_back(p.q.graph);
            bytes += b;
            take = true;
          }
        }
      }
      if (take) out.push_back(p);
      else rest.push_back(p);
    }
  } else {
    bytes = S->graphs[(size_t)head.q.graph].sample_bytes;
    for (const Pending& p : S->queue) {
      if (p.q.kind == HG_Q_ESTIMATE && p.q.graph == head.q.graph &&
          (int)out.size() < std::min(kMaxEstimateGroup, S->opt.max_batch_queries))
        out.push_back(p);
      else
        rest.push_back(p);
    }
  }
  S->queue.swap(rest);
}

using GraphCopies = std::unordered_map<int32_t, ServeGraph>;   // taken under the lock

void run_exact(const GraphCopies& gs, const std::vector<Pending>& batch, cudaStream_t st,
               std::vector<hg_result>& res) {
  std::vector<int32_t> members, nv, ne;
  std::vector<const int64_t*> ptrs;
  std::vector<const int32_t*> idxs;
  std::vector<int32_t> slot(batch.size());
  for (size_t k = 0; k < batch.size(); ++k) {
    const int32_t gid = batch[k].q.graph;
    auto it = std::find(members.begin(), members.end(), gid);
    if (it == members.end()) {
      const ServeGraph& g = gs.at(gid);
      members.push_back(gid);
      nv.push_back(g.nv);
      ne.push_back(g.ne);
      ptrs.push_back(g.d_ptr);
      idxs.push_back(g.d_idx);
      it = members.end() - 1;
    }
    slot[k] = (int32_t)(it - members.begin());
  }
  const int32_t G = (int32_t)members.size();
  std::vector<uint64_t> counts((size_t)G * 21);
  std::vector<double> cc((size_t)G);
  std::vector<uint64_t> open((size_t)G), conn((size_t)G);
  hg_batch* b = nullptr;
  hg_status st_all = hg_load_batch_members(G, nv.data(), ne.data(), ptrs.data(), idxs.data(), 1,
                                           0, st, &b);
  if (st_all == HG_OK) st_all = hg_batch_build_wedges(b, nullptr);
  if (st_all == HG_OK) st_all = hg_batch_count_patterns(b, counts.data(), nullptr);
  for (size_t k = 0; k < batch.size(); ++k) {
    hg_result& r = res[k];
    r.status = st_all;
    if (st_all != HG_OK) continue;
    const size_t m = (size_t)slot[k];
    std::memcpy(r.counts, counts.data() + 21 * m, sizeof(r.counts));
    if (batch[k].q.kind == HG_Q_CLUSTERING) {
      r.status = hg_batch_clustering_coeff(b, batch[k].q.eps, cc.data(), open.data(), conn.data());
      r.cc = cc[m];
      r.open = open[m];
      r.connected = conn[m];
    }
  }
  if (b) hg_batch_free(b);
}

void run_estimate(const GraphCopies& gs, const std::vector<Pending>& batch, cudaStream_t st,
                  std::vector<hg_result>& res) {
  const ServeGraph& g = gs.at(batch[0].q.graph);
  hg_graph* h = nullptr;
  hg_status st_all = hg_load_csr(g.nv, g.ne, g.d_ptr, g.d_idx, 1, st, &h);
  if (st_all == HG_OK) st_all = hg_build_wedges(h, nullptr, nullptr);
  for (size_t k = 0; k < batch.size(); ++k) {
    hg_result& r = res[k];
    r.status = st_all;
    if (st_all != HG_OK) continue;
    const hg_query& q = batch[k].q;
    r.status = hg_sample_estimate(h, q.seed, q.first_sample, q.num_samples, 1.0, r.counts, r.est);
  }
  if (h) hg_free(h);
}

void worker_main(hg_server* S, int wid) {
  cudaSetDevice(S->device);
  hg::alloc_bypass_hooks(true);
  cudaStream_t st = nullptr;
  const bool have_stream = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
  for (;;) {
    std::vector<Pending> batch;
    GraphCopies gs;
    size_t bytes = 0;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] {
        if (S->queue.empty()) return S->stop;
        // head-of-line admission by device memory (always when nothing is running)
        return S->in_flight == 0 || S->in_flight + bytes_of(S, S->queue.front().q) <= S->budget;
      });
      if (S->queue.empty()) break;   // stop requested and nothing left
      form_batch(S, batch, bytes);
      for (const Pending& p : batch) gs.emplace(p.q.graph, S->graphs[(size_t)p.q.graph]);
      S->in_flight += bytes;
      S->running += 1;
      S->stats.batches += 1;
      S->stats.queries_batched += batch.size();
      if (is_exact(batch[0].q)) S->stats.exact_batches += 1;
      S->stats.max_in_flight_bytes = std::max<uint64_t>(S->stats.max_in_flight_bytes, S->in_flight);
      S->stats.max_concurrent_batches =
          std::max<uint64_t>(S->stats.max_concurrent_batches, (uint64_t)S->running);
    }
    const double t_start = now(S);
    std::vector<hg_result> res(batch.size());
    for (auto& r : res) std::memset(&r, 0, sizeof(r));
    if (!have_stream) {
      for (auto& r : res) r.status = HG_ERR_CUDA;
    } else if (is_exact(batch[0].q)) {
      run_exact(gs, batch, st, res);
    } else {
      run_estimate(gs, batch, st, res);
    }
    const double t_done = now(S);
    std::unordered_set<int32_t> distinct;
    for (const Pending& p : batch) distinct.insert(p.q.graph);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->in_flight -= bytes;
      S->running -= 1;
      for (size_t k = 0; k < batch.size(); ++k) {
        hg_result& r = res[k];
        r.kind = batch[k].q.kind;
        r.graph = batch[k].q.graph;
        r.t_submit = batch[k].t_submit;
        r.t_start = t_start;
        r.t_done = t_done;
        r.batch_queries = (int32_t)batch.size();
        r.batch_graphs = (int32_t)distinct.size();
        r.worker = wid;
        S->done[batch[k].ticket] = r;
      }
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
  if (have_stream) cudaStreamDestroy(st);
}

void free_graphs(hg_server* S) {
  for (ServeGraph& g : S->graphs) {
    cudaFree(g.d_ptr);
    cudaFree(g.d_idx);
  }
  S->graphs.clear();
}

}  // namespace

extern "C" {

hg_status hg_server_create(const hg_server_options* opt, hg_server** out) {
  if (!out) return HG_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
    cudaGetLastError();
    return HG_ERR_NO_DEVICE;
  }
  hg_server* S = new hg_server();
  if (opt) S->opt = *opt;
  if (S->opt.workers < 0 || S->opt.max_batch_graphs < 0 || S->opt.memory_budget < 0 ||
      S->opt.max_batch_queries < 0) {
    delete S;
    return HG_ERR_INVALID_ARG;
  }
  if (S->opt.workers == 0) S->opt.workers = 4;
  if (S->opt.max_batch_graphs == 0) S->opt.max_batch_graphs = 64;
  if (S->opt.max_batch_queries == 0) S->opt.max_batch_queries = INT32_MAX;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return HG_ERR_CUDA;
  }
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    delete S;
    return HG_ERR_CUDA;
  }
  S->budget = S->opt.memory_budget > 0 ? (size_t)S->opt.memory_budget : free_b / 2;
  S->t0 = std::chrono::steady_clock::now();
  for (int w = 0; w < S->opt.workers; ++w) S->workers.emplace_back(worker_main, S, w);
  *out = S;
  return HG_OK;
}

hg_status hg_server_add_graph(hg_server* S, int32_t num_vertices, int32_t num_edges,
                              const int64_t* edge_ptr, const int32_t* edge_vtx,
                              int inputs_on_device, int32_t* graph_id) {
  if (!S || !graph_id || num_vertices < 1 || num_edges < 0 || !edge_ptr) return HG_ERR_INVALID_ARG;
  const cudaMemcpyKind kind = inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  ServeGraph g;
  g.nv = num_vertices;
  g.ne = num_edges;
  if (inputs_on_device) {
    if (cudaMemcpy(&g.nnz, edge_ptr + num_edges, sizeof(int64_t), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return HG_ERR_CUDA;
  } else {
    g.nnz = edge_ptr[num_edges];
  }
  if (g.nnz < 0 || (g.nnz > 0 && !edge_vtx)) return HG_ERR_INVALID_ARG;
  if (cudaMalloc(&g.d_ptr, sizeof(int64_t) * ((size_t)num_edges + 1)) != cudaSuccess ||
      cudaMalloc(&g.d_idx, sizeof(int32_t) * (size_t)std::max<int64_t>(g.nnz, 1)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(g.d_ptr);
    return HG_ERR_OOM;
  }
  hg_status st = HG_OK;
  if (cudaMemcpy(g.d_ptr, edge_ptr, sizeof(int64_t) * ((size_t)num_edges + 1), kind) !=
          cudaSuccess ||
      (g.nnz > 0 && cudaMemcpy(g.d_idx, edge_vtx, sizeof(int32_t) * (size_t)g.nnz, kind) !=
                        cudaSuccess))
    st = HG_ERR_CUDA;
  // validate and measure once: step one gives W for the memory estimates
  if (st == HG_OK) {
    hg::alloc_bypass_hooks(true);
    hg_graph* h = nullptr;
    hg_wedge_stats ws{};
    st = hg_load_csr(num_vertices, num_edges, g.d_ptr, g.d_idx, 1, nullptr, &h);
    if (st == HG_OK) st = hg_build_wedges(h, nullptr, &ws);
    if (h) hg_free(h);
    hg::alloc_bypass_hooks(false);
    g.W = ws.W;
  }
  if (st != HG_OK) {
    cudaFree(g.d_ptr);
    cudaFree(g.d_idx);
    return st;
  }
  size_graph(g, 0);   // unpacked entries: an upper bound
  std::lock_guard<std::mutex> lk(S->mu);
  *graph_id = (int32_t)S->graphs.size();
  S->graphs.push_back(g);
  return HG_OK;
}

hg_status hg_server_submit(hg_server* S, const hg_query* q, uint64_t* ticket) {
  if (!S || !q || !ticket) return HG_ERR_INVALID_ARG;
  if (q->kind != HG_Q_COUNTS && q->kind != HG_Q_CLUSTERING && q->kind != HG_Q_ESTIMATE)
    return HG_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop || q->graph < 0 || q->graph >= (int32_t)S->graphs.size()) return HG_ERR_INVALID_ARG;
    if (q->kind == HG_Q_ESTIMATE && q->num_samples > UINT64_MAX - q->first_sample)
      return HG_ERR_INVALID_ARG;
    Pending p{S->next_ticket++, *q, now(S)};
    *ticket = p.ticket;
    S->outstanding.insert(p.ticket);
    S->queue.push_back(p);
    S->stats.submitted += 1;
  }
  S->cv_work.notify_one();
  return HG_OK;
}

hg_status hg_server_wait(hg_server* S, uint64_t ticket, hg_result* out) {
  if (!S || !out) return HG_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  if (!S->outstanding.count(ticket)) return HG_ERR_INVALID_ARG;
  S->cv_done.wait(lk, [&] { return S->done.count(ticket) > 0; });
  *out = S->done[ticket];
  S->done.erase(ticket);
  S->outstanding.erase(ticket);
  return HG_OK;
}

hg_status hg_server_cancel(hg_server* S, uint64_t ticket) {
  if (!S) return HG_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (!S->outstanding.count(ticket)) return HG_ERR_INVALID_ARG;
    auto it = std::find_if(S->queue.begin(), S->queue.end(),
                           [&](const Pending& p) { return p.ticket == ticket; });
    if (it == S->queue.end()) return HG_ERR_STATE;   // taken by a worker, or answered
    hg_result r;
    std::memset(&r, 0, sizeof(r));
    r.status = HG_ERR_CANCELLED;
    r.kind = it->q.kind;
    r.graph = it->q.graph;
    r.t_submit = it->t_submit;
    r.t_start = r.t_done = now(S);
    r.worker = -1;
    S->queue.erase(it);
    S->done[ticket] = r;
  }
  S->cv_done.notify_all();   // its waiter, and a drain the emptier queue may end
  // a cancelled head of the queue may have been what kept the next query out of the
  // memory budget: let idle workers look at the queue again
  S->cv_work.notify_all();
  return HG_OK;
}

hg_status hg_server_drain(hg_server* S) {
  if (!S) return HG_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  S->cv_done.wait(lk, [&] { return S->queue.empty() && S->running == 0; });
  return HG_OK;
}

hg_status hg_server_stats_get(hg_server* S, hg_server_stats* out) {
  if (!S || !out) return HG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  *out = S->stats;
  out->budget_bytes = S->budget;
  out->now = now(S);
  return HG_OK;
}

hg_status hg_server_destroy(hg_server* S) {
  if (!S) return HG_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  free_graphs(S);
  delete S;
  return HG_OK;
}

}  // extern "C"
