// C-ABI entry points (include/igp.h): argument checks, host/device pointer handling,
// graph handles, the private memory pool, error messages and phase profiling.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "igp_internal.cuh"

namespace igp {

// ------------------------------------------------------------------ errors
static thread_local char t_err[512] = "";
static std::atomic<int64_t> g_launches{0};
static std::atomic<int64_t> g_allocs{0};  // device and pinned-host allocations made by the library

void count_alloc() { g_allocs.fetch_add(1, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(t_err, sizeof(t_err), fmt, ap);
  va_end(ap);
}
void clear_error() { t_err[0] = 0; }

igp_status cuda_status(cudaError_t e, const char* what, const char* file, int line) {
  set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  return e == cudaErrorMemoryAllocation ? IGP_E_NOMEM : IGP_E_CUDA;
}

// Kernel launches made by replaying a captured graph of n kernels (capturing counted them
// once as launches; pass -n to take that back).
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

igp_status after_launch(const char* name) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("launch of %s failed: %s", name, cudaGetErrorString(e));
    return IGP_E_CUDA;
  }
  return IGP_OK;
}

// ------------------------------------------------------------------ memory
static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[64] = {};

static cudaMemPool_t pool_for_current_device() {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
    uint64_t thr = ~0ull;  // keep freed memory in the pool
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr);
    g_pools[dev] = p;
  }
  return g_pools[dev];
}

static std::mutex g_slot_mu;
static std::vector<int*> g_slots;
constexpr int kSlotInts = 16;   // 64 bytes a slot
constexpr int kSlabSlots = 256; // slots page-locked at a time

int* pinned_slot() {
  std::lock_guard<std::mutex> lk(g_slot_mu);
  if (g_slots.empty()) {
    int* slab = nullptr;
    // portable: a slot may serve a handle on any device of the process
    if (cudaHostAlloc((void**)&slab, (size_t)kSlabSlots * kSlotInts * sizeof(int), cudaHostAllocPortable) !=
        cudaSuccess)
      return nullptr;
    for (int k = kSlabSlots - 1; k >= 0; --k) g_slots.push_back(slab + (size_t)k * kSlotInts);
  }
  int* w = g_slots.back();
  g_slots.pop_back();
  memset(w, 0, kSlotInts * sizeof(int));
  return w;
}

void release_slot(int* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_slot_mu);
  g_slots.push_back(p);
}

igp_status dev_alloc(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  cudaMemPool_t pool = pool_for_current_device();
  if (!pool) {
    set_error("cannot create the device memory pool");
    return IGP_E_CUDA;
  }
  count_alloc();
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes > 0 ? bytes : 1, pool, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? IGP_E_NOMEM : IGP_E_CUDA;
  }
  return IGP_OK;
}

void dev_free(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

size_t pool_idle_bytes() {
  cudaMemPool_t pool = pool_for_current_device();
  if (!pool) return 0;
  uint64_t reserved = 0, used = 0;
  if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) != cudaSuccess ||
      cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return reserved > used ? (size_t)(reserved - used) : 0;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device address of page-locked host memory (NULL for any other pointer): kernels write
// such a buffer directly over the host link, with no staging copy.
void* pinned_alias(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int num_sms() {
  static std::atomic<int> sms[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (sms[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    sms[dev] = v > 0 ? v : 1;
  }
  return sms[dev];
}

// ------------------------------------------------------------------ profile
cudaEvent_t Profile::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

PhaseTimer::PhaseTimer(Profile* p_, int ph, cudaStream_t s_) : p(p_), phase(ph), s(s_) {
  if (p) {
    a = p->get();
    cudaEventRecord(a, s);
  }
}
PhaseTimer::~PhaseTimer() {
  if (p) {
    cudaEvent_t b = p->get();
    cudaEventRecord(b, s);
    p->recs.push_back({phase, a, b});
  }
}

// Copy `bytes` from a host or device source into a new device buffer (or alias it).
static igp_status to_device(const void* src, size_t bytes, cudaStream_t s, const void** dev, void** owned) {
  *owned = nullptr;
  if (bytes == 0 || is_device_ptr(src)) {
    *dev = src;
    return IGP_OK;
  }
  void* p = nullptr;
  IGP_TRY(dev_alloc(&p, bytes, s));
  cudaError_t e = cudaMemcpyAsync(p, src, bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    dev_free(p, s);
    return cuda_status(e, "host-to-device copy", __FILE__, __LINE__);
  }
  *dev = p;
  *owned = p;
  return IGP_OK;
}

// Order stream `s` after the handle's previous work / mark the end of this call's work.
static igp_status graph_wait(igp_graph* g, cudaStream_t s) {
  if (g->done) IGP_TRY_CUDA(cudaStreamWaitEvent(s, g->done, 0));
  return IGP_OK;
}
static igp_status graph_mark(igp_graph* g, cudaStream_t s) {
  if (g->done) IGP_TRY_CUDA(cudaEventRecord(g->done, s));
  return IGP_OK;
}

}  // namespace igp

using namespace igp;

extern "C" {

const char* igp_version(void) { return "igp-gb300 0.1.0 (sm_103a)"; }
const char* igp_last_error(void) { return t_err; }
int64_t igp_launch_count(void) { return g_launches.load(); }
int64_t igp_alloc_count(void) { return g_allocs.load(); }

void igp_embed_opts_init(igp_embed_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->alpha = 1.0;
  o->theta = 0.1;
  o->eps = 1e-3;
  o->x_scale = 0.0;
  o->znorm_ddof = 1;
  o->storage = IGP_STORE_F32;
  o->out_row_l2 = 0;
  o->out_row_begin = 0;
  o->host_async = 0;
  o->x_in = nullptr;
  o->profile = nullptr;
}

igp_status igp_graph_build_profiled(const int32_t* src, const int32_t* dst, int64_t M, int32_t N, void* stream,
                                    igp_profile* profile, igp_graph** out) {
  clear_error();
  if (!out) {
    set_error("igp_graph_build: out is NULL");
    return IGP_E_INVAL;
  }
  *out = nullptr;
  if (N < 1 || N >= 2147483647 || M < 0 || M >= (1LL << 30) || (M > 0 && (!src || !dst))) {
    set_error("igp_graph_build: need 1 <= N < 2^31-1, 0 <= M < 2^30 and non-NULL edge arrays (N=%d, M=%lld)", N,
              (long long)M);
    return IGP_E_INVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  igp_graph* g = new (std::nothrow) igp_graph();
  if (!g) {
    set_error("igp_graph_build: host allocation failed");
    return IGP_E_NOMEM;
  }
  cudaGetDevice(&g->device);
  count_alloc();
  if (cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming) != cudaSuccess ||
      (g->err_host = pinned_slot()) == nullptr) {
    igp_status e = cuda_status(cudaGetLastError(), "graph handle set-up", __FILE__, __LINE__);
    if (g->done) cudaEventDestroy(g->done);
    delete g;
    return e;
  }
  *g->err_host = 0;
  const void *ds = nullptr, *dd = nullptr;
  void *os = nullptr, *od = nullptr;
  igp_status st = to_device(src, (size_t)M * sizeof(int32_t), s, &ds, &os);
  if (st == IGP_OK) st = to_device(dst, (size_t)M * sizeof(int32_t), s, &dd, &od);
  if (st == IGP_OK) {
    PhaseTimer pt(profile ? &profile->prof : nullptr, IGP_PHASE_BUILD, s);
    st = build_csr((const int32_t*)ds, (const int32_t*)dd, M, N, s, g);
  }
  dev_free(os, s);
  dev_free(od, s);
  if (st == IGP_OK) st = graph_mark(g, s);
  if (st != IGP_OK) {
    cudaEventDestroy(g->done);
    release_slot(g->err_host);  // the failed build copied nothing into it
    delete g;
    return st;
  }
  *out = g;
  return IGP_OK;
}

igp_status igp_graph_build(const int32_t* src, const int32_t* dst, int64_t M, int32_t N, void* stream,
                           igp_graph** out) {
  return igp_graph_build_profiled(src, dst, M, N, stream, nullptr, out);
}

igp_status igp_graph_append(igp_graph* g, const int32_t* src, const int32_t* dst, int64_t M_new, int32_t N_new,
                            void* stream) {
  clear_error();
  if (!g || N_new < g->N || N_new >= 2147483647 || M_new < 0 || M_new >= (1LL << 30) ||
      (M_new > 0 && (!src || !dst))) {
    set_error("igp_graph_append: need a graph, N_new >= its N (N_new < 2^31-1), 0 <= M_new < 2^30 and edge arrays");
    return IGP_E_INVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  IGP_TRY(graph_wait(g, s));
  const void *ds = nullptr, *dd = nullptr;
  void *os = nullptr, *od = nullptr;
  igp_status st = to_device(src, (size_t)M_new * sizeof(int32_t), s, &ds, &os);
  if (st == IGP_OK) st = to_device(dst, (size_t)M_new * sizeof(int32_t), s, &dd, &od);
  if (st == IGP_OK) st = append_csr(g, (const int32_t*)ds, (const int32_t*)dd, M_new, N_new, s);
  dev_free(os, s);
  dev_free(od, s);
  if (st == IGP_OK) st = graph_mark(g, s);
  return st;
}

igp_status igp_graph_info(const igp_graph* g, int32_t* N, int64_t* nnz, int32_t* max_deg) {
  clear_error();
  if (!g) {
    set_error("igp_graph_info: NULL graph");
    return IGP_E_INVAL;
  }
  if (N) *N = g->N;
  if (nnz) *nnz = g->nnz;
  if (max_deg) *max_deg = g->max_deg;
  return IGP_OK;
}

// Copies `bytes` from the device to `dst` (host or device); a host destination (also with
// bytes == 0) returns after the stream has drained, so host-visible results of it are final.
static igp_status copy_out(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (!dst) return IGP_OK;
  bool dev = is_device_ptr(dst);
  cudaError_t e = cudaSuccess;
  if (bytes > 0) {
    e = cudaMemcpyAsync(dst, src, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_status(e, "copy out", __FILE__, __LINE__);
  }
  if (!dev) {
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e, "stream synchronize", __FILE__, __LINE__);
  }
  return IGP_OK;
}

igp_status igp_graph_export(const igp_graph* g, int32_t* row_ptr, int32_t* col, void* stream) {
  clear_error();
  if (!g) {
    set_error("igp_graph_export: NULL graph");
    return IGP_E_INVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  IGP_TRY(graph_wait(const_cast<igp_graph*>(g), s));
  IGP_TRY(copy_out(row_ptr, g->row_ptr, ((size_t)g->N + 1) * sizeof(int32_t), s));
  IGP_TRY(copy_out(col, g->col, (size_t)g->nnz * sizeof(int32_t), s));
  return graph_mark(const_cast<igp_graph*>(g), s);
}

igp_status igp_degree_factors(igp_graph* g, double tau, double eps, float* dinv, void* stream) {
  clear_error();
  if (!g || !dinv || !std::isfinite(tau) || !(eps > 0) || !std::isfinite(eps)) {
    set_error("igp_degree_factors: need a graph, an output and finite tau, eps > 0");
    return IGP_E_INVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  IGP_TRY(graph_wait(g, s));
  IGP_TRY(compute_dinv(g, tau, eps, s, nullptr));
  IGP_TRY(copy_out(dinv, g->dinv, (size_t)g->N * sizeof(float), s));
  return graph_mark(g, s);
}

void igp_graph_free(igp_graph* g) {
  if (!g) return;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != g->device) cudaSetDevice(g->device);
  // device memory: released in stream order after the handle's last work; the host then waits for
  // that work only because the handle's page-locked error word may be written until it ends
  cudaStream_t s = cudaStreamPerThread;
  if (g->done) cudaStreamWaitEvent(s, g->done, 0);
  if (g->row_ptr) cudaFreeAsync(g->row_ptr, s);
  if (g->col) cudaFreeAsync(g->col, s);
  if (g->dinv) cudaFreeAsync(g->dinv, s);
  if (g->perm) cudaFreeAsync(g->perm, s);
  if (g->ws) cudaFreeAsync(g->ws, s);
  if (g->done) {
    cudaEventSynchronize(g->done);  // the pinned error word may still be written
    cudaEventDestroy(g->done);
  }
  release_slot(g->err_host);  // after the handle's last work
  cudaGetLastError();
  if (cur != g->device) cudaSetDevice(cur);
  delete g;
}

igp_status igp_graph_sync(igp_graph* g) {
  clear_error();
  if (!g) {
    set_error("igp_graph_sync: NULL graph");
    return IGP_E_INVAL;
  }
  if (g->done) IGP_TRY_CUDA(cudaEventSynchronize(g->done));
  if (g->err_host && *g->err_host) {
    set_error("a device-side wait of the last igp_embed ran out; its output is invalid");
    return IGP_E_TIMEOUT;
  }
  return IGP_OK;
}

igp_status igp_generate_x(uint64_t seed, int32_t N, int32_t d, double x_scale, float* out, void* stream) {
  clear_error();
  if (!out || N < 1 || d < 8 || d % 8 != 0 || d > 4096 || (int64_t)N * d >= (1LL << 40)) {
    set_error("igp_generate_x: need an output, N >= 1 and d a multiple of 8 in [8, 4096]");
    return IGP_E_INVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const double xs = x_scale > 0 ? x_scale : 1.0 / std::sqrt((double)d);
  const size_t bytes = (size_t)N * d * sizeof(float);
  if (is_device_ptr(out)) return launch_theta(seed, N, d, d, (float)xs, IGP_STORE_F32, nullptr, out, s);
  void* tmp = nullptr;
  IGP_TRY(dev_alloc(&tmp, bytes, s));
  igp_status st = launch_theta(seed, N, d, d, (float)xs, IGP_STORE_F32, nullptr, tmp, s);
  if (st == IGP_OK) st = copy_out(out, tmp, bytes, s);
  dev_free(tmp, s);
  return st;
}

igp_status igp_embed(igp_graph* g, double tau, int32_t L, int32_t d, uint64_t seed, float* out,
                     const igp_embed_opts* opts, void* stream) {
  clear_error();
  igp_embed_opts o;
  if (opts)
    o = *opts;
  else
    igp_embed_opts_init(&o);
  if (!g || (!out && o.out_row_begin != g->N)) {
    set_error("igp_embed: NULL graph or output");
    return IGP_E_INVAL;
  }
  if (!std::isfinite(tau) || L < 0 || L > 10000 || !std::isfinite(o.alpha) || !std::isfinite(o.theta) ||
      !(o.eps > 0) || !std::isfinite(o.eps) || (o.znorm_ddof != 0 && o.znorm_ddof != 1) ||
      (o.storage != IGP_STORE_F32 && o.storage != IGP_STORE_BF16) || !std::isfinite(o.x_scale) ||
      (o.host_async != 0 && o.host_async != 1)) {
    set_error("igp_embed: invalid tau, L or options");
    return IGP_E_INVAL;
  }
  if (d != 8 && d != 16 && d != 32 && d != 64 && d != 128) {
    set_error("igp_embed: d=%d unsupported (8, 16, 32, 64, 128)", d);
    return IGP_E_INVAL;
  }
  if (o.gather < IGP_GATHER_AUTO || o.gather > IGP_GATHER_TMA4) {
    set_error("igp_embed: unknown gather mode %d", o.gather);
    return IGP_E_INVAL;
  }
  if (o.chunk_cols != 0) {
    const int sb = o.storage == IGP_STORE_BF16 ? 2 : 4;
    const int c = o.chunk_cols;
    if (c < 0 || c > d || d % c != 0 || (c & (c - 1)) != 0 || c * sb < 16) {
      set_error("igp_embed: chunk_cols=%d must be a power of two dividing d=%d with >= 16 bytes per row", c, d);
      return IGP_E_INVAL;
    }
  }
  if (o.x_in && !is_device_ptr(o.x_in)) {
    set_error("igp_embed: opts->x_in must be device memory");
    return IGP_E_INVAL;
  }
  if (o.out_row_begin < 0 || o.out_row_begin > g->N) {
    set_error("igp_embed: opts->out_row_begin=%d outside [0, N=%d]", o.out_row_begin, g->N);
    return IGP_E_INVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)(g->N - o.out_row_begin) * d * sizeof(float);
  IGP_TRY(graph_wait(g, s));
  igp_status st;
  const bool on_device = bytes == 0 || is_device_ptr(out);  // no rows to write: stream-ordered too
  void* host_alias = on_device ? nullptr : pinned_alias(out);
  if (on_device) {
    st = run_ffp(g, tau, L, d, seed, bytes ? out : nullptr, o, s);
  } else if (host_alias && o.host_async) {
    // page-locked host output, asynchronous: the result is formed in device memory and copied by a
    // copy engine in stream order, so the copy overlaps kernels of other streams (the output
    // kernel writing across the host link would hold the SMs for as long); igp_graph_sync waits
    void* tmp = nullptr;
    IGP_TRY(dev_alloc(&tmp, bytes, s));
    st = run_ffp(g, tau, L, d, seed, (float*)tmp, o, s);
    if (st == IGP_OK) {
      const cudaError_t e = cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, s);
      if (e != cudaSuccess) st = cuda_status(e, "copy out", __FILE__, __LINE__);
    }
    dev_free(tmp, s);
    if (st == IGP_OK) st = graph_mark(g, s);
    return st;
  } else if (host_alias) {  // page-locked host output: written by the output kernel itself
    st = run_ffp(g, tau, L, d, seed, (float*)host_alias, o, s);
    if (st == IGP_OK && cudaStreamSynchronize(s) != cudaSuccess)
      st = cuda_status(cudaGetLastError(), "stream synchronize", __FILE__, __LINE__);
    if (st == IGP_OK && *g->err_host) {
      set_error("igp_embed: a device-side wait ran out; the output is invalid");
      st = IGP_E_TIMEOUT;
    }
  } else {
    void* tmp = nullptr;
    IGP_TRY(dev_alloc(&tmp, bytes, s));
    st = run_ffp(g, tau, L, d, seed, (float*)tmp, o, s);
    if (st == IGP_OK) st = copy_out(out, tmp, bytes, s);  // synchronises
    dev_free(tmp, s);
    if (st == IGP_OK && *g->err_host) {
      set_error("igp_embed: a device-side wait ran out; the output is invalid");
      st = IGP_E_TIMEOUT;
    }
  }
  if (st == IGP_OK) st = graph_mark(g, s);
  return st;
}

// ------------------------------------------------------------------ batches
static void batch_release(igp_batch* b) {
  if (!b) return;
  if (b->cs) cudaStreamSynchronize(b->cs);
  cudaDeviceSynchronize();
  void* ptrs[] = {b->row_ptr, b->col, b->row_graph, b->perm, b->pgraph, b->goff, b->seeds_dev, b->dinv, b->ws};
  for (void* q : ptrs)
    if (q) cudaFreeAsync(q, 0);
  for (auto& kv : b->chunks)
    if (kv.second.start) cudaFreeAsync(kv.second.start, 0);
  cudaStreamSynchronize(0);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cs) cudaStreamDestroy(b->cs);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->ev_err) cudaEventDestroy(b->ev_err);
  release_slot(b->err_host);  // after the device synchronisation above
  cudaGetLastError();
  delete b;
}

igp_status igp_batch_create(igp_graph* const* graphs, int32_t G, void* stream, igp_batch** out) {
  clear_error();
  if (!out || !graphs || G < 1) {
    set_error("igp_batch_create: need an output handle and G >= 1 graphs");
    return IGP_E_INVAL;
  }
  *out = nullptr;
  for (int32_t g = 0; g < G; ++g)
    if (!graphs[g]) {
      set_error("igp_batch_create: graph %d is NULL", g);
      return IGP_E_INVAL;
    }
  cudaStream_t s = (cudaStream_t)stream;
  for (int32_t g = 0; g < G; ++g) IGP_TRY(graph_wait(graphs[g], s));
  igp_batch* b = new (std::nothrow) igp_batch();
  if (!b) return IGP_E_NOMEM;
  cudaGetDevice(&b->device);
  igp_status st = batch_create(graphs, G, s, b);
  if (st != IGP_OK) {
    batch_release(b);
    return st;
  }
  *out = b;
  return IGP_OK;
}

igp_status igp_batch_info(const igp_batch* b, int32_t* G, int32_t* N_total, int64_t* nnz_total,
                          int32_t* row_offsets) {
  clear_error();
  if (!b) {
    set_error("igp_batch_info: NULL batch");
    return IGP_E_INVAL;
  }
  if (G) *G = b->G;
  if (N_total) *N_total = b->N;
  if (nnz_total) *nnz_total = b->nnz;
  if (row_offsets) memcpy(row_offsets, b->goff_host.data(), (size_t)(b->G + 1) * sizeof(int32_t));
  return IGP_OK;
}

igp_status igp_batch_embed(igp_batch* b, double tau, int32_t L, int32_t d, const uint64_t* seeds, float* out,
                           const igp_embed_opts* opts, void* stream) {
  clear_error();
  igp_embed_opts o;
  if (opts)
    o = *opts;
  else
    igp_embed_opts_init(&o);
  if (!b || !seeds || !out) {
    set_error("igp_batch_embed: NULL batch, seeds or output");
    return IGP_E_INVAL;
  }
  if (!std::isfinite(tau) || L < 0 || L > 10000 || !std::isfinite(o.alpha) || !std::isfinite(o.theta) ||
      !(o.eps > 0) || !std::isfinite(o.eps) || (o.znorm_ddof != 0 && o.znorm_ddof != 1) ||
      (o.storage != IGP_STORE_F32 && o.storage != IGP_STORE_BF16) || !std::isfinite(o.x_scale)) {
    set_error("igp_batch_embed: invalid tau, L or options");
    return IGP_E_INVAL;
  }
  if (o.x_in || o.chunk_cols != 0 || (o.gather != IGP_GATHER_AUTO && o.gather != IGP_GATHER_LSU) ||
      (o.reserved_test != 0 && (o.reserved_test < 2 || o.reserved_test > 7)) || o.out_row_begin != 0) {
    set_error("igp_batch_embed: x_in, chunk_cols, TMA gathers and out_row_begin are not supported for batches");
    return IGP_E_INVAL;
  }
  if (d != 8 && d != 16 && d != 32 && d != 64 && d != 128) {
    set_error("igp_batch_embed: d=%d unsupported (8, 16, 32, 64, 128)", d);
    return IGP_E_INVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (is_device_ptr(out)) return batch_embed(b, tau, L, d, seeds, out, o, s);
  const size_t bytes = (size_t)b->N * d * sizeof(float);
  void* tmp = nullptr;
  IGP_TRY(dev_alloc(&tmp, bytes, s));
  igp_status st = batch_embed(b, tau, L, d, seeds, (float*)tmp, o, s);
  if (st == IGP_OK) st = copy_out(out, tmp, bytes, s);
  dev_free(tmp, s);
  if (st == IGP_OK && b->err_host && *b->err_host) {
    set_error("igp_batch_embed: a bounded device-side wait of the persistent launch ran out; the output is invalid");
    *b->err_host = 0;
    return IGP_E_TIMEOUT;
  }
  return st;
}

igp_status igp_batch_sync(igp_batch* b) {
  clear_error();
  if (!b) return IGP_E_INVAL;
  if (b->ev_out) IGP_TRY_CUDA(cudaEventSynchronize(b->ev_out));
  if (b->ev_err) IGP_TRY_CUDA(cudaEventSynchronize(b->ev_err));
  if (b->err_host && *b->err_host) {
    set_error("igp_batch_sync: a bounded device-side wait of the last persistent launch ran out; its output is "
              "invalid");
    *b->err_host = 0;
    return IGP_E_TIMEOUT;
  }
  return IGP_OK;
}

void igp_batch_free(igp_batch* b) { batch_release(b); }

igp_status igp_profile_create(igp_profile** p) {
  clear_error();
  if (!p) return IGP_E_INVAL;
  *p = new (std::nothrow) igp_profile();
  return *p ? IGP_OK : IGP_E_NOMEM;
}

void igp_profile_free(igp_profile* p) {
  if (!p) return;
  for (auto& r : p->prof.recs) {
    cudaEventSynchronize(r.b);
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : p->prof.pool) cudaEventDestroy(e);
  delete p;
}

igp_status igp_profile_read(igp_profile* p, double* ms, int64_t* launches) {
  clear_error();
  if (!p) return IGP_E_INVAL;
  double acc[IGP_NUM_PHASES] = {0};
  int64_t cnt[IGP_NUM_PHASES] = {0};
  igp_status st = IGP_OK;
  for (auto& r : p->prof.recs) {
    cudaError_t e = cudaEventSynchronize(r.b);
    float t = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess && st == IGP_OK) st = cuda_status(e, "event timing", __FILE__, __LINE__);
    if (r.phase >= 0 && r.phase < IGP_NUM_PHASES) {
      acc[r.phase] += t;
      cnt[r.phase] += 1;
    }
    p->prof.pool.push_back(r.a);
    p->prof.pool.push_back(r.b);
  }
  p->prof.recs.clear();
  for (int i = 0; i < IGP_NUM_PHASES; ++i) {
    if (ms) ms[i] = acc[i];
    if (launches) launches[i] = cnt[i];
  }
  return st;
}

}  // extern "C"
