// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <string>
#include <vector>

#include "igp.h"

namespace igp {

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
void clear_error();
igp_status cuda_status(cudaError_t e, const char* what, const char* file, int line);

#define IGP_TRY_CUDA(expr)                                                          \
  do {                                                                              \
    cudaError_t _e = (expr);                                                        \
    if (_e != cudaSuccess) return ::igp::cuda_status(_e, #expr, __FILE__, __LINE__); \
  } while (0)

#define IGP_TRY(expr)                  \
  do {                                 \
    igp_status _s = (expr);            \
    if (_s != IGP_OK) return _s;       \
  } while (0)

// Count one kernel launch and surface launch-configuration errors.
igp_status after_launch(const char* name);
// Add n to the launch count (the kernels of a replayed graph; negative to take back captured ones).
void count_launches(int64_t n);

// ---------------------------------------------------------------- memory
// Stream-ordered allocation from a library-private pool that keeps freed memory
// cached (release threshold = max), so per-call workspaces cost no driver calls
// after warm-up.
igp_status dev_alloc(void** p, size_t bytes, cudaStream_t s);
// Count one memory allocation (igp_alloc_count); dev_alloc counts its own.
void count_alloc();
// A zeroed 64-byte page-locked host slot (16 ints) for flags and small readbacks, from a free list
// that keeps slots for the life of the process (cudaFreeHost would synchronise the whole device, so
// releasing a graph handle would wait for the work of every other). NULL if page-locking fails.
int* pinned_slot();
// Back to the free list; the caller makes sure no copy into the slot is still pending.
void release_slot(int* p);
void dev_free(void* p, cudaStream_t s);
// Bytes the current device's library pool holds but does not use (free for dev_alloc).
size_t pool_idle_bytes();
bool is_device_ptr(const void* p);
int num_sms();

// ---------------------------------------------------------------- profile
struct Profile {
  struct Rec {
    int phase;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get();
};
// Records an event pair around a phase when p != nullptr.
struct PhaseTimer {
  Profile* p;
  int phase;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  PhaseTimer(Profile* p_, int ph, cudaStream_t s_);
  ~PhaseTimer();
};

}  // namespace igp

struct igp_profile {
  igp::Profile prof;
};

struct igp_graph {
  int32_t N = 0;
  int64_t nnz = 0;
  int32_t max_deg = 0;
  int device = 0;
  int32_t* row_ptr = nullptr;  // device [N+1]
  int32_t* col = nullptr;      // device [nnz]
  // Eq. 1 factors for the last (tau, eps) asked for, and w_i = sum_{j in N(i)} dinv_j
  float* dinv = nullptr;       // device [N]
  float* wsum = nullptr;       // device [N], same allocation as dinv
  // rows in order of decreasing degree (the layer kernels' processing order), followed in the
  // same allocation by the offsets of each degree in it ([max_deg + 2], see ensure_perm)
  int32_t* perm = nullptr;
  double dinv_tau = 0, dinv_eps = 0;
  bool dinv_valid = false;
  // FFP workspace (grown on demand, kept until free)
  void* ws = nullptr;
  size_t ws_bytes = 0;
  // host copy (pinned) of the device error word of the last igp_embed
  int* err_host = nullptr;
  // recorded on the stream of each call: later calls on another stream, and the
  // stream-ordered release in igp_graph_free, wait for it
  cudaEvent_t done = nullptr;
};

// Many graphs packed block-diagonally for one FFP each (igp_batch_*).
struct igp_batch {
  int32_t G = 0, N = 0;  // graphs, packed rows
  int64_t nnz = 0, P = 0;  // packed CSR entries, processing-order length (padded)
  int device = 0;
  int32_t* row_ptr = nullptr;    // [N+1]
  int32_t* col = nullptr;        // [nnz], packed ids
  int32_t* row_graph = nullptr;  // [N] graph of each packed row
  int32_t* perm = nullptr;       // [P] processing order: each graph's rows by decreasing degree, -1 padded
  int32_t* pgraph = nullptr;     // [P/32] graph of each 32-position block of the order
  int32_t* goff = nullptr;       // [G+1] packed row offset of each graph
  std::vector<int32_t> goff_host;
  uint64_t* seeds_dev = nullptr; // [G]
  float* dinv = nullptr;         // [N], and w [N] after it
  float* wsum = nullptr;
  double dinv_tau = 0, dinv_eps = 0;
  bool dinv_valid = false;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  // captured launch sequence and its parameters, replayed on cs
  cudaStream_t cs = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t exec_kernels = 0;  // kernels in exec
  // launch plan per (d, storage), chosen by the schedule tuner on first use: mode 0 = one launch
  // per layer plus a statistics launch, 1 = one persistent launch for all layers; the claim size
  // (order positions per warp turn); CTAs per SM of the persistent launch
  struct Plan {
    int mode = 0, chunk = 64, ctas = 1;
  };
  std::map<int, Plan> plan;
  // work-balanced chunks of the order, per (rows per warp tile, mean positions per chunk):
  // start[0..K] (start[K] = P) and K on the device, in one allocation
  struct Chunks {
    int32_t* start = nullptr;
    int* count = nullptr;
  };
  std::map<std::pair<int, int>, Chunks> chunks;
  std::string exec_key;
  int* err_host = nullptr;        // pinned copy of the device error word of the last persistent launch
  cudaEvent_t ev_err = nullptr;   // recorded after that copy
};

namespace igp {
// csr_build.cu: exclusive prefix sum of n >= 1 ints; tmp holds ceil(n / 8192) ints.
igp_status exclusive_scan(const int* in, int* out, int64_t n, int* tmp, cudaStream_t s);
// csr_build.cu: CSR of the undirected edge list (device inputs), into g (empty).
igp_status build_csr(const int32_t* src, const int32_t* dst, int64_t M, int32_t N, cudaStream_t s,
                     igp_graph* g);
// csr_build.cu: merge an edge increment (device inputs) into g, growing it to N_new nodes.
igp_status append_csr(igp_graph* g, const int32_t* src, const int32_t* dst, int64_t M, int32_t N_new,
                      cudaStream_t s);
// ffp.cu: batches
igp_status batch_create(igp_graph* const* graphs, int32_t G, cudaStream_t s, igp_batch* b);
igp_status batch_embed(igp_batch* b, double tau, int32_t L, int32_t d, const uint64_t* seeds, float* out_dev,
                       const igp_embed_opts& o, cudaStream_t s,
                       bool capture = true);

// Arguments of one layer launch.
struct LayerArgs {
  const int32_t* row_ptr;
  const int32_t* col;
  const float* dinv;
  const float* wsum;
  const int32_t* perm;  // processing order of the rows (NULL: their own order)
  const void* Tin;
  void* Tout;
  const float* stats_in;
  unsigned long long* gsum;  // per column chunk [2 dc] int64 column sums, zero on entry (left zero)
  float* stats_out;
  unsigned* tickets;  // [2 nchunks]: finish tickets, then tile-claim counters; zero on entry (left zero)
  int* err;       // device word set to 1 by a layer whose bounded wait ran out
  int withhold;   // test hook of the bounded wait (0 in normal use)
  int gather4;    // bulk-copy kernel: 1 = tile::gather4 through a tensor map
  int prefetch;   // register-load kernel: 1 = L2 prefetch of the rows a few trips ahead
  const int* heavy_count;  // register-load kernel: device count of leading heavy rows in perm (NULL: 0)
  int32_t N, d;
  float alpha, theta;
  int ddof, grid;
};

// ffp.cu
igp_status ensure_perm(igp_graph* g, cudaStream_t s);
// dinv and w for (tau, eps), cached on the graph.
igp_status compute_dinv(igp_graph* g, double tau, double eps, cudaStream_t s, Profile* prof);
// Theta (the random input of Alg. 1) into `out` in the storage type, in column blocks of dc columns
// (dc = d: row-major), multiplied row-wise by dinv if non-NULL.
igp_status launch_theta(uint64_t seed, int32_t N, int32_t d, int32_t dc, float x_scale, int storage,
                        const float* dinv, void* out, cudaStream_t s);
igp_status run_ffp(igp_graph* g, double tau, int32_t L, int32_t d, uint64_t seed, float* out_dev,
                   const igp_embed_opts& o, cudaStream_t s);
}  // namespace igp
