// Serving loop (igp_server_*): requests to embed graphs, or to grow a resident graph by an
// edge increment and re-embed it (the merge and FFP of a step of Alg. 2), are queued, admitted into a fixed
// number of slots as device memory and slots free up, and run concurrently: every slot
// is a host worker thread with its own CUDA stream that builds or grows the request's
// CSR and embeds the graph, so the GPU work of admitted requests overlaps. Optionally
// (batch_rows > 0) the FFPs of small graphs are batched continuously instead: a batcher thread
// with its own stream takes every small request whose CSR is ready when it frees up and embeds
// them together in one block-diagonal batch (one launch sequence for all of them, each graph
// with its own Theta seed and column statistics, so every result equals embedding it alone),
// then copies each result to its caller. (On the served stream measured here, slots embedding
// their own graphs on concurrent streams kept the GPU busier than shared batches.)
// Resident graphs keep their CSR and degree state on the device between requests;
// requests on the same resident graph run in submission order.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "igp_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  uint64_t ticket = 0;
  igp_request r;  // pointers of the caller: src/dst replaced by the copies below
  std::vector<int32_t> src, dst;
  int32_t state = IGP_REQ_QUEUED;
  igp_status status = IGP_OK;
  std::string error;
  size_t est = 0;
  igp_graph* g = nullptr;  // the request's graph once its CSR is built or grown
  bool embedded = false;   // set by the batcher once the result is in r.out (or failed)
  int waiters = 0;         // callers inside igp_wait on this request (igp_server_forget refuses then)
  Clock::time_point t_submit, t_start, t_done;
};



}  // namespace

struct igp_server {
  igp_server_opts opts;
  int device = 0;
  size_t budget = 0, admitted = 0;  // device bytes: usable, held by running requests
  size_t resident_bytes = 0;         // device bytes held by resident graphs
  std::map<int64_t, size_t> resident_size;
  std::mutex mu;
  std::condition_variable cv;       // work or completion
  std::deque<Req*> queue;
  std::map<uint64_t, Req*> reqs;
  std::map<int64_t, igp_graph*> resident;
  std::set<int64_t> busy;           // resident graph ids with a running request
  std::vector<std::thread> workers;
  std::vector<std::thread> batchers;
  std::deque<Req*> ready;           // CSR done, waiting for a batcher
  std::vector<double> latencies;   // submit-to-done times of the last kLatencyWindow completions
  size_t latency_next = 0;          // ring position once the window is full
  uint64_t next_ticket = 1;
  int64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, running = 0;
  int64_t batches = 0, batched = 0;  // shared FFP batches and the requests they served
  bool stopping = false;
};

namespace {

constexpr size_t kLatencyWindow = 65536;

// Device memory a new request may take right now: free device memory (re-read, so that memory
// taken or released by other users of the GPU counts) plus what the library's pool holds
// unused, less the reserve.
size_t free_now(const igp_server* sv) {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const size_t avail = fr + igp::pool_idle_bytes();
  const size_t res = (size_t)sv->opts.reserve_bytes;
  return avail > res ? avail - res : 0;
}

// Device bytes a request may hold at its peak (edge copies, CSR build temporaries, the
// CSR, per-node arrays, the two activation buffers and the output staging).
size_t estimate(const igp_server* sv, const igp_request& r) {
  const size_t sb = r.opts.storage == IGP_STORE_BF16 ? 2 : 4;
  size_t n = (size_t)r.N, m = (size_t)r.M;
  size_t bytes = 40 * m + 48 * n + n * (size_t)r.d * (2 * sb + 4) + (1u << 20);
  if (r.kind == IGP_REQ_APPEND) {
    auto it = sv->resident.find(r.graph_id);
    if (it != sv->resident.end()) bytes += 12 * (size_t)it->second->nnz;
  }
  return bytes;
}

// Device bytes a graph handle holds between calls (CSR, Eq. 1 factors, order, workspace).
size_t graph_bytes(const igp_graph* g) {
  return 4 * ((size_t)g->N + 1) + 4 * (size_t)g->nnz + 12 * (size_t)g->N + g->ws_bytes;
}

void set_resident(igp_server* sv, int64_t id, igp_graph* g) {
  auto it = sv->resident_size.find(id);
  if (it != sv->resident_size.end()) sv->resident_bytes -= it->second;
  if (g) {
    const size_t b = graph_bytes(g);
    sv->resident_size[id] = b;
    sv->resident_bytes += b;
  } else if (it != sv->resident_size.end()) {
    sv->resident_size.erase(it);
  }
}

// First queued request that may start now: memory fits, and no earlier request on the
// same resident graph is queued or running.
Req* pick(igp_server* sv) {
  std::set<int64_t> seen;
  size_t avail = 0;
  bool avail_read = false;
  for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it) {
    Req* q = *it;
    const bool on_graph = q->r.kind == IGP_REQ_APPEND || q->r.keep;
    if (on_graph) {
      if (seen.count(q->r.graph_id) || sv->busy.count(q->r.graph_id)) {
        seen.insert(q->r.graph_id);
        continue;
      }
      seen.insert(q->r.graph_id);
    }
    if (q->r.kind == IGP_REQ_APPEND && !sv->resident.count(q->r.graph_id)) {
      // nothing earlier will create this graph: the request fails without running
      q->est = 0;
      q->status = IGP_E_INVAL;
      q->error = "igp_submit: no resident graph with this graph_id";
      sv->queue.erase(it);
      return q;
    }
    q->est = estimate(sv, q->r);
    if (sv->running > 0) {  // wait for memory: the server's budget, and the device's free memory now
      if (sv->admitted + sv->resident_bytes + q->est > sv->budget) continue;
      if (!avail_read) {
        avail = free_now(sv);
        avail_read = true;
      }
      if (q->est > avail) continue;
    }
    sv->queue.erase(it);
    return q;
  }
  return nullptr;
}

// The request's CSR: built from its edges, or its resident graph grown by them (on the slot's
// stream). q->g is the graph to embed.
void run_csr(igp_server* sv, Req* q, cudaStream_t s) {
  igp_request& r = q->r;
  igp_graph* g = nullptr;
  igp_status st = IGP_OK;
  if (r.kind == IGP_REQ_EMBED) {
    st = igp_graph_build(q->src.data(), q->dst.data(), r.M, r.N, s, &g);
  } else {
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      g = sv->resident[r.graph_id];
    }
    st = igp_graph_append(g, q->src.data(), q->dst.data(), r.M, r.N, s);
  }
  if (st != IGP_OK) q->error = igp_last_error();
  q->g = g;
  q->status = st;
}

// After the embedding (lock held): keep or free the graph, account its memory.
void settle(igp_server* sv, Req* q) {
  igp_request& r = q->r;
  igp_graph* g = q->g;
  if (r.kind == IGP_REQ_EMBED) {
    if (q->status == IGP_OK && r.keep) {
      auto it = sv->resident.find(r.graph_id);
      if (it != sv->resident.end()) igp_graph_free(it->second);
      sv->resident[r.graph_id] = g;
      set_resident(sv, r.graph_id, g);
    } else if (g) {
      igp_graph_free(g);
    }
  } else {
    set_resident(sv, r.graph_id, g);  // grown by the increment (unchanged if the merge failed)
  }
  q->g = nullptr;
}

// Requests whose FFPs can share one batch: the same tau, L, d and options, none of them
// outside what batches support.
bool batchable(const igp_request& r) {
  return r.opts.chunk_cols == 0 && (r.opts.gather == IGP_GATHER_AUTO || r.opts.gather == IGP_GATHER_LSU) &&
         r.opts.reserved_test == 0 && r.opts.out_row_begin == 0;
}
bool same_ffp(const igp_request& a, const igp_request& b) {
  return a.tau == b.tau && a.L == b.L && a.d == b.d && a.opts.alpha == b.opts.alpha &&
         a.opts.theta == b.opts.theta && a.opts.eps == b.opts.eps && a.opts.x_scale == b.opts.x_scale &&
         a.opts.znorm_ddof == b.opts.znorm_ddof && a.opts.storage == b.opts.storage &&
         a.opts.out_row_l2 == b.opts.out_row_l2;
}

void fail_all(const std::vector<Req*>& qs, igp_status st) {
  const std::string msg = igp_last_error();
  for (Req* q : qs) {
    q->status = st;
    q->error = msg;
  }
}

// One batch of compatible requests on stream s: pack their graphs, run the FFP of all of
// them in the same launches, copy every result to its caller. Waits for completion.
void embed_batch(const std::vector<Req*>& qs, cudaStream_t s) {
  const igp_request& r0 = qs[0]->r;
  const int32_t G = (int32_t)qs.size();
  std::vector<igp_graph*> graphs(G);
  std::vector<uint64_t> seeds(G);
  for (int32_t k = 0; k < G; ++k) {
    graphs[k] = qs[k]->g;
    seeds[k] = qs[k]->r.seed;
  }
  igp_batch* b = nullptr;
  igp_status st = igp_batch_create(graphs.data(), G, s, &b);
  if (st != IGP_OK) return fail_all(qs, st);
  void* out = nullptr;
  const size_t row_bytes = (size_t)r0.d * sizeof(float);
  st = igp::dev_alloc(&out, (size_t)b->N * row_bytes, s);
  if (st == IGP_OK) st = igp::batch_embed(b, r0.tau, r0.L, r0.d, seeds.data(), (float*)out, r0.opts, s, false);
  for (int32_t k = 0; k < G && st == IGP_OK; ++k) {
    const size_t off = (size_t)b->goff_host[k] * row_bytes;
    const size_t bytes = (size_t)(b->goff_host[k + 1] - b->goff_host[k]) * row_bytes;
    if (cudaMemcpyAsync(qs[k]->r.out, (char*)out + off, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      st = igp::cuda_status(cudaGetLastError(), "result copy", __FILE__, __LINE__);
  }
  if (st == IGP_OK && cudaStreamSynchronize(s) != cudaSuccess)
    st = igp::cuda_status(cudaGetLastError(), "batch", __FILE__, __LINE__);
  if (out) igp::dev_free(out, s);
  igp_batch_free(b);
  if (st != IGP_OK) fail_all(qs, st);
}

void embed_alone(Req* q, cudaStream_t s) {
  igp_request& r = q->r;
  // A page-locked output is formed in device memory (the staging the admission estimate counts)
  // and copied by a copy engine, which overlaps the other slots' kernels; written by the output
  // kernel across the host link instead, it would hold the SMs for the whole transfer. The slot
  // waits for the copy, so the result is final when the request completes.
  igp_embed_opts o = r.opts;
  o.host_async = 1;
  igp_status st = igp_embed(q->g, r.tau, r.L, r.d, r.seed, r.out, &o, s);
  if (st == IGP_OK) st = igp_graph_sync(q->g);
  if (st != IGP_OK) {
    q->status = st;
    q->error = igp_last_error();
  }
}

// The batcher: embeds every request whose CSR is ready, small compatible ones together.
void batcher(igp_server* sv) {
  cudaSetDevice(sv->device);
  cudaStream_t s = nullptr;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  for (;;) {
    std::vector<Req*> group;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv.wait(lk, [&] { return !sv->ready.empty() || (sv->stopping && sv->running == 0); });
      if (sv->ready.empty()) break;
      const Req* first = sv->ready.front();
      for (auto it = sv->ready.begin(); it != sv->ready.end();) {
        Req* q = *it;
        if (q == first || (batchable(first->r) && batchable(q->r) && same_ffp(first->r, q->r))) {
          group.push_back(q);
          it = sv->ready.erase(it);
        } else {
          ++it;
        }
      }
    }
    std::vector<Req*> small;
    for (Req* q : group) small.push_back(q);
    if (small.size() == 1)
      embed_alone(small[0], s);
    else if (!small.empty())
      embed_batch(small, s);
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      for (Req* q : group) q->embedded = true;
      if (small.size() > 1) {
        sv->batches += 1;
        sv->batched += (int64_t)small.size();
      }
    }
    sv->cv.notify_all();
  }
  cudaStreamDestroy(s);
}

void worker(igp_server* sv) {
  cudaSetDevice(sv->device);
  cudaStream_t s = nullptr;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  for (;;) {
    Req* q = nullptr;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      for (;;) {
        if (sv->stopping && sv->queue.empty()) break;
        q = pick(sv);
        if (q || sv->stopping) break;
        sv->cv.wait(lk);
      }
      if (!q) break;
      q->state = IGP_REQ_RUNNING;
      q->t_start = Clock::now();
      sv->admitted += q->est;
      sv->running += 1;
      if (q->r.kind == IGP_REQ_APPEND || q->r.keep) sv->busy.insert(q->r.graph_id);
    }
    if (q->status == IGP_OK) {
      run_csr(sv, q, s);
      if (q->status == IGP_OK && (!batchable(q->r) || q->g->N >= sv->opts.batch_rows)) {
        embed_alone(q, s);  // large: its own launches fill the GPU, next to the other slots'
        std::lock_guard<std::mutex> lk(sv->mu);
        settle(sv, q);
      } else {
        std::unique_lock<std::mutex> lk(sv->mu);
        if (q->status == IGP_OK) {  // small: wait for the batcher
          sv->ready.push_back(q);
          sv->cv.notify_all();
          sv->cv.wait(lk, [&] { return q->embedded; });
        }
        settle(sv, q);
      }
    }
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      q->t_done = Clock::now();
      q->state = q->status == IGP_OK ? IGP_REQ_DONE : IGP_REQ_FAILED;
      sv->admitted -= q->est;
      sv->running -= 1;
      if (q->r.kind == IGP_REQ_APPEND || q->r.keep) sv->busy.erase(q->r.graph_id);
      if (q->status == IGP_OK) {
        sv->completed += 1;
        const double lat = std::chrono::duration<double>(q->t_done - q->t_submit).count();
        if (sv->latencies.size() < kLatencyWindow) {
          sv->latencies.push_back(lat);
        } else {
          sv->latencies[sv->latency_next] = lat;
          sv->latency_next = (sv->latency_next + 1) % kLatencyWindow;
        }
      } else {
        sv->failed += 1;
      }
      q->src.clear();
      q->src.shrink_to_fit();
      q->dst.clear();
      q->dst.shrink_to_fit();
    }
    sv->cv.notify_all();
  }
  cudaStreamDestroy(s);
}

double pct(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const size_t k = (size_t)std::min<double>((double)v.size() - 1, p * (double)(v.size() - 1) + 0.5);
  return v[k];
}

}  // namespace

using namespace igp;

extern "C" {

void igp_server_opts_init(igp_server_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->slots = 4;
  o->max_queue = 0;
  o->reserve_bytes = 1ll << 30;
  o->device = -1;
  o->batch_rows = 0;
}

igp_status igp_server_create(const igp_server_opts* opts, igp_server** out) {
  clear_error();
  if (!out) return IGP_E_INVAL;
  *out = nullptr;
  igp_server_opts o;
  if (opts)
    o = *opts;
  else
    igp_server_opts_init(&o);
  if (o.slots < 1 || o.slots > 64 || o.max_queue < 0 || o.reserve_bytes < 0 || o.batch_rows < 0) {
    set_error("igp_server_create: need 1 <= slots <= 64, max_queue >= 0, reserve_bytes >= 0, batch_rows >= 0");
    return IGP_E_INVAL;
  }
  igp_server* sv = new (std::nothrow) igp_server();
  if (!sv) return IGP_E_NOMEM;
  sv->opts = o;
  if (o.device >= 0) {
    cudaError_t e = cudaSetDevice(o.device);
    if (e != cudaSuccess) {
      delete sv;
      return cuda_status(e, "cudaSetDevice", __FILE__, __LINE__);
    }
  }
  cudaGetDevice(&sv->device);
  size_t fr = 0, tot = 0;
  cudaError_t e = cudaMemGetInfo(&fr, &tot);
  if (e != cudaSuccess) {
    delete sv;
    return cuda_status(e, "cudaMemGetInfo", __FILE__, __LINE__);
  }
  sv->budget = fr > (size_t)o.reserve_bytes ? fr - (size_t)o.reserve_bytes : 0;
  for (int k = 0; k < o.slots; ++k) sv->workers.emplace_back(worker, sv);
  // one batcher (batch_rows > 0): small requests whose CSR is ready while it is busy wait
  // together and are then embedded in one batch
  if (o.batch_rows > 0) sv->batchers.emplace_back(batcher, sv);
  *out = sv;
  return IGP_OK;
}

void igp_server_destroy(igp_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    for (Req* q : sv->queue) {
      q->state = IGP_REQ_CANCELLED;
      sv->cancelled += 1;
    }
    sv->queue.clear();
    sv->stopping = true;
  }
  sv->cv.notify_all();
  for (auto& t : sv->workers) t.join();
  sv->cv.notify_all();
  for (auto& t : sv->batchers) t.join();
  for (auto& kv : sv->resident) igp_graph_free(kv.second);
  for (auto& kv : sv->reqs) delete kv.second;
  delete sv;
}

igp_status igp_submit(igp_server* sv, const igp_request* r, uint64_t* ticket) {
  clear_error();
  if (!sv || !r || !ticket || !r->out || r->N < 1 || r->M < 0 || (r->M > 0 && (!r->src || !r->dst)) ||
      (r->kind != IGP_REQ_EMBED && r->kind != IGP_REQ_APPEND) || r->opts.x_in || r->opts.profile ||
      r->opts.host_async) {
    set_error("igp_submit: invalid request (kind, N, M, edges, out; opts.x_in and opts.profile must be NULL, "
              "opts.host_async 0)");
    return IGP_E_INVAL;
  }
  Req* q = new (std::nothrow) Req();
  if (!q) return IGP_E_NOMEM;
  q->r = *r;
  q->src.assign(r->src, r->src + r->M);
  q->dst.assign(r->dst, r->dst + r->M);
  q->r.src = nullptr;
  q->r.dst = nullptr;
  q->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stopping || (sv->opts.max_queue > 0 && (int)sv->queue.size() >= sv->opts.max_queue)) {
      delete q;
      set_error("igp_submit: the server is stopping or its queue is full");
      return IGP_E_BUSY;
    }
    const size_t est = estimate(sv, q->r);
    if (est > sv->budget) {
      delete q;
      set_error("igp_submit: the request needs about %zu device bytes, more than the server's %zu", est,
                sv->budget);
      return IGP_E_NOMEM;
    }
    q->ticket = sv->next_ticket++;
    sv->reqs[q->ticket] = q;
    sv->queue.push_back(q);
    sv->submitted += 1;
    *ticket = q->ticket;
  }
  sv->cv.notify_all();
  return IGP_OK;
}

static igp_status report(Req* q, int32_t* state, double* latency_s) {
  if (state) *state = q->state;
  if (latency_s)
    *latency_s = q->state == IGP_REQ_DONE || q->state == IGP_REQ_FAILED
                     ? std::chrono::duration<double>(q->t_done - q->t_submit).count()
                     : 0.0;
  if (q->state == IGP_REQ_FAILED) {
    set_error("%s", q->error.c_str());
    return q->status;
  }
  if (q->state == IGP_REQ_CANCELLED) return IGP_E_CANCELLED;
  return (q->state == IGP_REQ_DONE) ? IGP_OK : IGP_E_NOTREADY;
}

igp_status igp_poll(igp_server* sv, uint64_t ticket, int32_t* state, double* latency_s) {
  clear_error();
  if (!sv) return IGP_E_INVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) {
    set_error("igp_poll: unknown ticket %llu", (unsigned long long)ticket);
    return IGP_E_INVAL;
  }
  return report(it->second, state, latency_s);
}

igp_status igp_wait(igp_server* sv, uint64_t ticket, double timeout_s, int32_t* state, double* latency_s) {
  clear_error();
  if (!sv) return IGP_E_INVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) {
    set_error("igp_wait: unknown ticket %llu", (unsigned long long)ticket);
    return IGP_E_INVAL;
  }
  Req* q = it->second;
  auto finished = [&] { return q->state >= IGP_REQ_DONE; };
  q->waiters += 1;  // keeps the record alive while this thread sleeps without the lock
  if (timeout_s < 0)
    sv->cv.wait(lk, finished);
  else
    sv->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), finished);
  q->waiters -= 1;
  return report(q, state, latency_s);
}

igp_status igp_server_forget(igp_server* sv, uint64_t ticket) {
  clear_error();
  if (!sv) return IGP_E_INVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) {
    set_error("igp_server_forget: unknown ticket %llu", (unsigned long long)ticket);
    return IGP_E_INVAL;
  }
  Req* q = it->second;
  // a finished record is no longer referenced by the queue, the batcher or a worker; only
  // callers of igp_wait may still hold it
  if (q->state < IGP_REQ_DONE || q->waiters > 0) {
    set_error("igp_server_forget: request %llu is queued, running or being waited on", (unsigned long long)ticket);
    return IGP_E_BUSY;
  }
  sv->reqs.erase(it);
  delete q;
  return IGP_OK;
}

igp_status igp_cancel(igp_server* sv, uint64_t ticket) {
  clear_error();
  if (!sv) return IGP_E_INVAL;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) {
      set_error("igp_cancel: unknown ticket %llu", (unsigned long long)ticket);
      return IGP_E_INVAL;
    }
    Req* q = it->second;
    if (q->state != IGP_REQ_QUEUED) {
      set_error("igp_cancel: the request is no longer queued");
      return IGP_E_BUSY;
    }
    sv->queue.erase(std::find(sv->queue.begin(), sv->queue.end(), q));
    q->state = IGP_REQ_CANCELLED;
    sv->cancelled += 1;
  }
  sv->cv.notify_all();
  return IGP_OK;
}

igp_status igp_server_release(igp_server* sv, int64_t graph_id) {
  clear_error();
  if (!sv) return IGP_E_INVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  sv->cv.wait(lk, [&] { return !sv->busy.count(graph_id); });
  auto it = sv->resident.find(graph_id);
  if (it == sv->resident.end()) {
    set_error("igp_server_release: no resident graph %lld", (long long)graph_id);
    return IGP_E_INVAL;
  }
  igp_graph_free(it->second);
  sv->resident.erase(it);
  set_resident(sv, graph_id, nullptr);
  return IGP_OK;
}

igp_status igp_server_get_stats(igp_server* sv, igp_server_stats* st) {
  clear_error();
  if (!sv || !st) return IGP_E_INVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  memset(st, 0, sizeof(*st));
  st->submitted = sv->submitted;
  st->completed = sv->completed;
  st->failed = sv->failed;
  st->cancelled = sv->cancelled;
  st->queued = (int64_t)sv->queue.size();
  st->running = sv->running;
  st->resident_graphs = (int64_t)sv->resident.size();
  st->admitted_bytes = (int64_t)sv->admitted;
  st->budget_bytes = (int64_t)sv->budget;
  st->resident_bytes = (int64_t)sv->resident_bytes;
  st->batches = sv->batches;
  st->batched = sv->batched;
  st->latency_p50_s = pct(sv->latencies, 0.50);
  st->latency_p99_s = pct(sv->latencies, 0.99);
  return IGP_OK;
}

}  // extern "C"
