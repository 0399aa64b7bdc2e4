/*
 * igp.h -- C-ABI of the GB300 (sm_103a) library for InfraredGP's feed-forward
 * propagation (FFP): Qin, Li, Cui, Pei, "InfraredGP: Efficient Graph
 * Partitioning via Spectral Graph Neural Networks with Negative Corrections",
 * arXiv 2508.19737.
 *
 * What the library computes (Alg. 1 up to its clustering step):
 *   A       symmetric binary adjacency of an undirected simple graph (Sec. II)
 *   D_tau   Eq. 1 for tau < 0: deg_i - min(|tau|, deg_i - eps); deg_i + tau otherwise (Sec. I)
 *   Z^(0)   Theta ~ N(0, 1/d), drawn from a seed on the device (the random input of Alg. 1)
 *   Z^(l)   ZNorm(tanh(theta Z^(l-1) + alpha D_tau^{-1/2} A D_tau^{-1/2} Z^(l-1))), l = 1..L
 *           (Eq. 2-4; the paper's low-pass filter is (alpha, theta) = (1, 0.1))
 *   out     sigmoid(Z^(L)) (Eq. 4), optionally divided by its row L2 norm
 *
 * Conventions for every entry point:
 *   - Node ids are 0-based int32 in [0, N). Edges are undirected; either or both
 *     directions may be given; self-loops are dropped and repeated edges merged.
 *   - A pointer argument may be host memory (pageable or pinned) or device memory
 *     of the current CUDA device; the library asks the CUDA runtime which. Host
 *     inputs are copied before the call returns; host outputs are complete when
 *     the call returns.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream). Work on device
 *     buffers is enqueued on it; a call whose outputs are all device buffers may
 *     return before the work finishes.
 *   - Nothing is thrown across the ABI. A non-zero igp_status is returned on error
 *     and igp_last_error() gives a thread-local message. On error no output is
 *     partially written by the host side and no handle is created.
 *   - A handle may be used from any thread, but calls on the same handle must not
 *     overlap.
 */
#ifndef IGP_H
#define IGP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t igp_status;
#define IGP_OK            0
#define IGP_E_INVAL       1  /* bad argument: id out of range, size limits, unsupported d */
#define IGP_E_NOMEM       2  /* device allocation failed */
#define IGP_E_CUDA        3  /* a CUDA runtime call failed (message has the CUDA error) */
#define IGP_E_TIMEOUT     4  /* a bounded device-side wait gave up */
#define IGP_E_BUSY        5  /* resource held by another request */
#define IGP_E_NOTREADY    6  /* polled work not finished yet */
#define IGP_E_CANCELLED   7  /* request cancelled before it ran */
#define IGP_E_UNSUPPORTED 8

/* Storage type of the N x d layer activations T^(l) and of Theta. Accumulation is
 * always fp32, degree factors are computed in fp64, the output is fp32. */
#define IGP_STORE_F32  0
#define IGP_STORE_BF16 1

/* How a layer brings neighbour rows to the SM (igp_embed_opts.gather). The bulk-copy modes add each
 * row's neighbours in one sequence; the register-load mode gathers rows of a few hundred entries
 * or more with a whole warp (another fp32 summation order), so the modes agree to fp32 rounding. */
#define IGP_GATHER_AUTO 0  /* the measured best (currently register loads for every width) */
#define IGP_GATHER_LSU  1  /* 16-byte register loads by the lanes of each row group */
#define IGP_GATHER_BULK 2  /* one cp.async.bulk copy per row into a per-warp shared-memory ring */
#define IGP_GATHER_TMA4 3  /* cp.async.bulk.tensor tile::gather4 (4 rows per copy); needs chunk_cols 0 */

/* Phases timed by an igp_profile (device time between CUDA events). */
#define IGP_PHASE_DINV   0  /* Eq. 1 degree factors (fp64 on the device) */
#define IGP_PHASE_THETA  1  /* Theta generation (the random input of Alg. 1) */
#define IGP_PHASE_LAYER  2  /* one Eq. 4 layer: gather-SpMM + tanh + column statistics */
#define IGP_PHASE_OUTPUT 3  /* sigmoid(ZNorm(T^(L))) */
#define IGP_PHASE_BUILD  4  /* whole CSR construction from an edge list */
#define IGP_NUM_PHASES   5

typedef struct igp_graph igp_graph;
typedef struct igp_batch igp_batch;
typedef struct igp_profile igp_profile;

/* Options of one FFP. Fill with igp_embed_opts_init() and change fields. */
typedef struct igp_embed_opts {
  double alpha;        /* Eq. 2 slope; 1.0 (low-pass). Negative values give a high-pass filter. */
  double theta;        /* Eq. 2 offset (the self term of Eq. 3); 0.1 */
  double eps;          /* Eq. 1 clamp; 1e-3 */
  double x_scale;      /* Theta = N(0,1) * x_scale; <= 0 means 1/sqrt(d) (the paper's N(0, 1/d)) */
  int32_t znorm_ddof;  /* ZNorm standard deviation divisor N - ddof; 1 (0 allowed) */
  int32_t storage;     /* IGP_STORE_F32 (default) or IGP_STORE_BF16 */
  int32_t out_row_l2;  /* 1: divide each output row by its L2 norm; 0 (default) */
  int32_t chunk_cols;  /* columns per layer pass; 0 (default) picks the widest of d, d/2, d/4, ..
                          whose N x width slice of the activations fits ~72 MB of L2, keeping at
                          least 128 bytes per row. Otherwise a power of two dividing d, >= 8, with
                          at least 16 bytes per row. The statistics are exact integer sums; the
                          fp32 summation order of the highest-degree rows depends on the pass
                          width, so passes change results only by fp32 rounding. */
  int32_t gather;      /* IGP_GATHER_AUTO (default), _LSU, _BULK or _TMA4 */
  int32_t reserved_test;/* 0. (Non-zero only in the library's own test of its bounded device waits.) */
  int32_t out_row_begin;/* first output row, 0 (default) .. N: the call writes rows out_row_begin .. N-1
                           of Z~ (out row 0 = graph row out_row_begin), so `out` holds (N - out_row_begin)
                           x d values. After igp_graph_append grew the graph from N_old nodes, N_old
                           extracts the new nodes' rows (as each step of Alg. 2 does). The FFP and its statistics still
                           run over all N rows. With N (no rows) `out` may be NULL and the call is
                           stream-ordered as for a device output. igp_batch_embed takes only 0. */
  int32_t host_async;  /* 0 (default): with a HOST `out`, the call returns once `out` holds the result.
                          1: a page-locked (pinned) host `out` is filled in stream order and the call
                          returns without waiting: the result is formed in device memory (a temporary
                          of the output's size from the pool) and copied by a copy engine, so the copy
                          overlaps kernels on other streams. Read `out` only after igp_graph_sync(g)
                          (which also reports a device-side timeout) or after the stream has drained.
                          Ignored for device and pageable host outputs. */
  const void* x_in;    /* NULL: Theta from `seed`. Else a DEVICE pointer to N x d row-major values in
                          the storage type, used as Z^(0) instead (not modified). */
  igp_profile* profile;/* NULL, or a profile that records per-phase device times of this call */
} igp_embed_opts;

/* Library version string; never NULL. */
const char* igp_version(void);

/* Message of the last error on this thread ("" if none); owned by the library. */
const char* igp_last_error(void);

/* Number of CUDA kernels this library has launched in this process so far. */
int64_t igp_launch_count(void);

/* Number of memory allocations (device memory from the library's pool, pinned host words of graph
 * handles) this library has made in this process so far. */
int64_t igp_alloc_count(void);

/* Defaults: alpha 1, theta 0.1, eps 1e-3, x_scale 1/sqrt(d), ddof 1, fp32 storage, no row L2. */
void igp_embed_opts_init(igp_embed_opts* opts);

/*
 * Build the CSR adjacency of an undirected graph on the device (Sec. II: A is
 * symmetric, binary, without self-loops). Columns of each row are sorted
 * increasingly. Integer result, identical to sort + unique of the directed pairs.
 *   src, dst : M node ids each (host or device), edge e = {src[e], dst[e]}
 *   M        : 0 <= M < 2^30
 *   N        : 1 <= N < 2^31 - 1
 *   out      : receives a new graph handle (free with igp_graph_free)
 * Errors: IGP_E_INVAL if an id is outside [0, N) (no handle is created),
 * IGP_E_NOMEM, IGP_E_CUDA. Synchronises `stream` once (to size the column array).
 */
igp_status igp_graph_build(const int32_t* src, const int32_t* dst, int64_t M, int32_t N,
                           void* stream, igp_graph** out);

/* Same as igp_graph_build, recording the device time of the build in `profile` (may be NULL). */
igp_status igp_graph_build_profiled(const int32_t* src, const int32_t* dst, int64_t M, int32_t N,
                                    void* stream, igp_profile* profile, igp_graph** out);

/*
 * Streaming update (the merge of each step of Alg. 2): merge an increment of undirected edges into the graph's
 * device-resident CSR, growing it to N_new >= N nodes (new nodes start without edges). The result
 * is the CSR igp_graph_build would give for all edges so far and N_new (sorted, deduplicated,
 * no self-loops). Cached per-graph state (degree factors, processing order) is refreshed on the
 * next use. Errors: IGP_E_INVAL (N_new < N, id outside [0, N_new); the graph is then unchanged),
 * IGP_E_NOMEM, IGP_E_CUDA. Synchronises `stream` once.
 */
igp_status igp_graph_append(igp_graph* g, const int32_t* src, const int32_t* dst, int64_t M_new, int32_t N_new,
                            void* stream);

/* N, number of stored (directed) CSR entries nnz = sum of degrees, and the largest degree. */
igp_status igp_graph_info(const igp_graph* g, int32_t* N, int64_t* nnz, int32_t* max_deg);

/* Copy the CSR out: row_ptr[N+1] and col[nnz] (host or device; either may be NULL). */
igp_status igp_graph_export(const igp_graph* g, int32_t* row_ptr, int32_t* col, void* stream);

/*
 * A graph from its CSR (the form igp_graph_export writes: the symmetric adjacency of Sec. II, no
 * self-loops, every row's columns sorted increasingly without repeats), e.g. to restore a graph
 * saved with igp_graph_export without its edge list.
 *   row_ptr : N+1 int32 (host or device), row_ptr[0] = 0, row_ptr[N] = nnz
 *   col     : nnz int32 (host or device)
 *   validate: 1 = check all of the above on the device (each entry's mirror by binary search;
 *             O(nnz log(max degree))); 0 = trust the input (a CSR that breaks them gives
 *             undefined embeddings, but no out-of-bounds access as long as row_ptr is valid)
 * Both arrays are copied. Errors: IGP_E_INVAL (bad sizes, or a check failed: no handle is
 * created; the message names the broken property), IGP_E_NOMEM, IGP_E_CUDA. Synchronises `stream`.
 */
igp_status igp_graph_import(const int32_t* row_ptr, const int32_t* col, int32_t N, int64_t nnz, int32_t validate,
                            void* stream, igp_graph** out);

/* Eq. 1 degree factors D_tau^{-1/2} as fp32 (computed in fp64, IEEE sqrt and division, then
 * rounded to nearest fp32), dinv[N] host or device. 0 where D_tau == 0 (tau = 0, isolated node). */
igp_status igp_degree_factors(igp_graph* g, double tau, double eps, float* dinv, void* stream);

/* Wait for all work issued on the handle; IGP_E_TIMEOUT if a device-side wait of the last
 * igp_embed on it ran out (about a second without progress: its output is then invalid), else
 * IGP_OK or IGP_E_CUDA. */
igp_status igp_graph_sync(igp_graph* g);

/* Release a graph and its device memory. NULL is a no-op. The call waits until the last work issued
 * on the handle has finished (its page-locked error word may be written until then); the device
 * memory is returned to the library's pool in stream order after that work. */
void igp_graph_free(igp_graph* g);

/*
 * Theta of Alg. 1 (its random input), exactly as igp_embed draws it, as fp32 [N][d] (host or device):
 * Philox4x64-10 (Salmon et al., SC 2011) on counter (i, c/8, 0, 0) with key (seed, 0); its four
 * 64-bit words are split into eight 32-bit halves w_k (low half first); u_k = ((w_k >> 8) + 1) 2^-24;
 * Box-Muller on (u_{2p}, u_{2p+1}) in fp32 gives columns 8(c/8) + 0..7; times x_scale
 * (<= 0: 1/sqrt(d)). d must be a multiple of 8.
 */
igp_status igp_generate_x(uint64_t seed, int32_t N, int32_t d, double x_scale, float* out, void* stream);

/*
 * One FFP (Alg. 1 up to its clustering step) on graph g:
 *   tau  : degree correction (Eq. 1 for tau < 0), any finite value
 *   L    : number of layers, 0 <= L <= 10000 (L = 0 gives sigmoid(Theta))
 *   d    : embedding width, one of 8, 16, 32, 64, 128
 *   seed : Theta seed (ignored when opts->x_in is set)
 *   out  : N x d fp32 row-major (host or device)
 *   opts : NULL for defaults
 * Errors: IGP_E_INVAL (bad d, L, tau, options), IGP_E_NOMEM, IGP_E_CUDA.
 * Uses (and keeps, until igp_graph_free) a per-graph device workspace of about
 * 2 N d storage-size bytes.
 */
igp_status igp_embed(igp_graph* g, double tau, int32_t L, int32_t d, uint64_t seed, float* out,
                     const igp_embed_opts* opts, void* stream);

/*
 * Batches: many independent graphs embedded together (block-diagonal packing). Each graph keeps its
 * own Theta seed and its own ZNorm column statistics (Eq. 4 acts per graph), so every graph's
 * result equals igp_embed on that graph alone, to fp32 rounding (igp_embed gathers a graph's
 * highest-degree rows with a whole warp, in another summation order; every other row and the
 * column statistics are computed identically).
 *
 * igp_batch_create: packs G built graphs (copied; the graphs may be freed afterwards) into one
 *   device CSR, with each graph's rows by decreasing degree as the processing order. Synchronises
 *   `stream`. Errors: IGP_E_INVAL (G < 1, NULL graph, more than 2^31 packed rows/entries), IGP_E_NOMEM.
 */
igp_status igp_batch_create(igp_graph* const* graphs, int32_t G, void* stream, igp_batch** out);

/* G, total rows, total CSR entries, and (if row_offsets is non-NULL) the G+1 row offsets of the
 * graphs in the packed output (host array). */
igp_status igp_batch_info(const igp_batch* b, int32_t* G, int32_t* N_total, int64_t* nnz_total,
                          int32_t* row_offsets);

/*
 * One FFP per graph of the batch (Alg. 1 up to its clustering step), all graphs in the same launches:
 *   seeds : host array of G Theta seeds (graph g's rows draw Theta with seeds[g] and local row ids)
 *   out   : N_total x d fp32 (host or device); graph g's rows at row_offsets[g] ..
 *   opts  : as igp_embed, except x_in, chunk_cols and TMA gathers (not supported here)
 * The layers run in one of two plans, both with the same arithmetic (the results are identical):
 * one launch per layer plus a statistics launch, or one persistent cooperative launch for all L
 * layers, in which each graph moves to its next layer as soon as its own rows are done (Eq. 4's
 * statistics are per graph), with bounded device-side waits. On the first embedding at a (d,
 * storage, mean-degree bucket) in the process, a schedule tuner times every candidate plan (claim
 * sizes, CTAs per SM) on this batch and keeps the fastest for that key. With device output, no
 * profile and the per-layer plan, the launch sequence is captured into a CUDA graph on first use
 * and replayed while (tau, L, d, options, out) stay the same; the replay runs on a library stream
 * ordered after, and before, the caller's `stream` by events. Errors: as igp_embed, and
 * IGP_E_TIMEOUT (host output) when a bounded wait of the persistent launch ran out (device output:
 * reported by igp_batch_sync).
 */
igp_status igp_batch_embed(igp_batch* b, double tau, int32_t L, int32_t d, const uint64_t* seeds, float* out,
                           const igp_embed_opts* opts, void* stream);

/* Wait for the batch's last embedding; IGP_E_TIMEOUT if a bounded device-side wait of its persistent
 * launch ran out (about a second without progress: its output is then invalid), else IGP_OK or
 * IGP_E_CUDA. */
igp_status igp_batch_sync(igp_batch* b);

/* Release a batch (waits for its work). NULL is a no-op. */
void igp_batch_free(igp_batch* b);

/*
 * Serving. A server admits requests into `slots` concurrent slots (host worker threads, each with
 * its own CUDA stream, so the GPU work of admitted requests overlaps) as slots and device memory
 * free up: a request starts only if its estimated peak device memory fits the server's budget
 * (free memory at creation minus reserve_bytes) next to the running ones and the resident graphs,
 * and also fits the device memory free at that moment (re-read with cudaMemGetInfo at each
 * admission, plus what the library's pool holds unused, minus reserve_bytes), so memory that other
 * users of the GPU take or release after igp_server_create counts. A request that finds nothing
 * running starts regardless and fails with IGP_E_NOMEM if the memory is not there. Requests are picked in submission order among those that may start. Resident graphs keep
 * their CSR and degree state on the device between requests (streaming, Alg. 2): an
 * IGP_REQ_APPEND request grows a resident graph by an edge increment and re-embeds it; requests
 * on the same graph_id run in submission order. The slots build or grow the requests' CSRs and
 * embed the graphs, each on its own stream, so admitted requests overlap on the device. With
 * batch_rows > 0 the FFPs of graphs with fewer nodes are batched instead: one batcher thread takes
 * every such request whose CSR is ready when it frees up and embeds those with the same (tau, L, d,
 * options) together in one block-diagonal batch (one launch sequence). Results do not depend on
 * what else runs: each equals igp_embed of that graph alone (bit for bit when embedded by its
 * slot, to fp32 rounding when embedded in a shared batch).
 */
typedef struct igp_server igp_server;

typedef struct igp_server_opts {
  int32_t slots;          /* concurrent requests, 1..64; 4 */
  int32_t max_queue;      /* queued requests allowed (0: no limit); 0 */
  int64_t reserve_bytes;  /* device memory left free; 1 GiB */
  int32_t device;         /* CUDA device (-1: the current one); -1 */
  int32_t batch_rows;     /* graphs of fewer nodes are embedded in shared batches (0: never); 0 */
} igp_server_opts;

#define IGP_REQ_EMBED  0  /* build a graph from the edges (N nodes) and embed it */
#define IGP_REQ_APPEND 1  /* append the edges to resident graph graph_id (grown to N nodes) and embed it */

/* request states reported by igp_poll / igp_wait */
#define IGP_REQ_QUEUED    0
#define IGP_REQ_RUNNING   1
#define IGP_REQ_DONE      2
#define IGP_REQ_FAILED    3
#define IGP_REQ_CANCELLED 4

typedef struct igp_request {
  int32_t kind;         /* IGP_REQ_EMBED or IGP_REQ_APPEND */
  int32_t keep;         /* EMBED: keep the built graph resident under graph_id */
  int64_t graph_id;     /* caller-chosen id of a resident graph */
  const int32_t* src;   /* HOST edge arrays, M entries each; copied by igp_submit */
  const int32_t* dst;
  int64_t M;
  int32_t N;            /* nodes after this request */
  int32_t L;            /* layers */
  double tau;
  int32_t d;
  int32_t reserved0;
  uint64_t seed;
  igp_embed_opts opts;  /* as for igp_embed; x_in and profile must be NULL, host_async 0 */
  float* out;           /* HOST N x d fp32, written when the request is done; keep it valid until then */
} igp_request;

typedef struct igp_server_stats {
  int64_t submitted, completed, failed, cancelled, queued, running, resident_graphs;
  int64_t admitted_bytes;  /* estimated peak device bytes of the running requests */
  int64_t budget_bytes;    /* free device memory at igp_server_create minus reserve_bytes */
  double latency_p50_s, latency_p99_s;  /* submit-to-done latency of the last 65,536 completed requests */
  int64_t resident_bytes;  /* device bytes held by resident graphs */
  int64_t batches;         /* FFP launch sequences that served two or more requests together */
  int64_t batched;         /* requests embedded in such shared batches */
} igp_server_stats;

/* Defaults as listed in igp_server_opts. */
void igp_server_opts_init(igp_server_opts* opts);
/* Start a server (its worker threads). Errors: IGP_E_INVAL, IGP_E_CUDA. */
igp_status igp_server_create(const igp_server_opts* opts, igp_server** out);
/* Cancel queued requests, wait for running ones, free resident graphs and the server. */
void igp_server_destroy(igp_server* sv);
/* Queue a request; *ticket identifies it. Errors: IGP_E_INVAL (bad request), IGP_E_BUSY (queue full
 * or stopping), IGP_E_NOMEM (the request alone exceeds the memory budget). Non-blocking. */
igp_status igp_submit(igp_server* sv, const igp_request* r, uint64_t* ticket);
/* Non-blocking state of a request: IGP_OK when done, IGP_E_NOTREADY while queued or running, the
 * request's own error when it failed, IGP_E_CANCELLED; *latency_s = submit-to-done time. */
igp_status igp_poll(igp_server* sv, uint64_t ticket, int32_t* state, double* latency_s);
/* Like igp_poll after waiting up to timeout_s seconds (< 0: no limit) for the request to finish. */
igp_status igp_wait(igp_server* sv, uint64_t ticket, double timeout_s, int32_t* state, double* latency_s);
/* Cancel a queued request (IGP_E_BUSY once it runs). */
igp_status igp_cancel(igp_server* sv, uint64_t ticket);
/* Drop the server's record of a finished (done, failed or cancelled) request, so that a long-running
 * server does not keep one record per request it ever served. Afterwards the ticket is unknown
 * (IGP_E_INVAL from igp_poll / igp_wait / igp_cancel); the request's output is untouched. Errors:
 * IGP_E_INVAL (unknown ticket), IGP_E_BUSY (the request is queued or running, or another thread is
 * inside igp_wait on it). */
igp_status igp_server_forget(igp_server* sv, uint64_t ticket);
/* Free a resident graph (waits for a request running on it). */
igp_status igp_server_release(igp_server* sv, int64_t graph_id);
igp_status igp_server_get_stats(igp_server* sv, igp_server_stats* stats);

/*
 * igp_embed without any memory allocation. (The paper has no counterpart.) Some callers cannot
 * allocate device memory at the moment they call: an allocator or memory-manager hook, which would
 * re-enter the allocator it is part of; a framework whose caching allocator already holds the free
 * memory, so that a cudaMalloc of the library fails; a long-running loop that must keep a fixed
 * memory footprint. For them this call allocates nothing: no cudaMalloc, cudaFree, pool or other
 * allocating routine (igp_alloc_count does not move).
 *   row_ptr, col : DEVICE CSR of the graph, [N+1] and [row_ptr[N]] int32, in the form igp_graph_export
 *                  writes (symmetric, no self-loops, ids in [0, N)); it is trusted, not checked
 *   out          : DEVICE (N - opts->out_row_begin) x d fp32 output (N x d with default options)
 *   tau, L, d, seed, opts : as for igp_embed; opts->profile and opts->chunk_cols must be 0
 * Same result as igp_embed on the graph built from that CSR, to fp32 rounding (rows are taken in
 * their own order, so the heaviest rows are summed in another order than igp_embed's).
 * All temporaries live in a fixed 16 MiB device array inside the library, reserved on every GPU
 * that loads the library until the process exits. Sizes whose temporaries do not fit (about
 * 2 N d storage-size bytes plus 8 N bytes and 32 d bytes of column statistics) are rejected with
 * IGP_E_INVAL before any GPU work. The first call on each device looks up that device's address
 * of the array (cudaGetSymbolAddress); make that first call before any stream capture. All calls
 * share the array, which keeps the last call's contents: calls whose GPU work overlaps (other
 * streams, other threads) race, so serialise them. Asynchronous on `stream`.
 */
igp_status igp_embed_noalloc(const int32_t* row_ptr, const int32_t* col, int32_t N, double tau, int32_t L, int32_t d,
                             uint64_t seed, float* out, const igp_embed_opts* opts, void* stream);

/*
 * K-agnostic clustering of embeddings on the device: the step that turns the FFP output into
 * blocks (Alg. 1's last step; Alg. 2's fit and assign), done by BIRCH in the paper (Sec. IV-A).
 * The clusterer keeps BIRCH's leaf entries, clustering features CF = (n, LS, SS) (member count,
 * linear sum, sum of squared norms; Zhang, Ramakrishnan, Livny, SIGMOD 1996), and its absorption
 * rule, without the tree: the closest entry is found by an exhaustive search on the GPU. A fit
 * takes the points in index order, in batches of `batch`:
 *   - points are quantised to multiples of 2^-16 (they must lie in [-1, 1]; FFP outputs do);
 *   - each point joins the entry whose centroid is closest (fp32 squared distance, coordinates
 *     summed in order; ties to the smaller id) if the merged entry's radius
 *     sqrt(SS/n - |LS/n|^2) (fp64 from exact integer sums) is at most `threshold`; the entries
 *     are those at the start of the point's batch;
 *   - the batch's other points ("candidates") form new entries: a candidate is a leader if no
 *     earlier candidate of the batch lies within `threshold` of it; the others join the closest
 *     leader within `threshold` (ties to the smaller index) or start an entry of their own; new
 *     entries are numbered on in index order.
 * The number of entries K follows from the threshold (it is not given). Labels and entries are
 * reproducible bit for bit (integer sums, fixed-order fp32/fp64 decisions).
 */
typedef struct igp_clusterer igp_clusterer;

/* d in {8, 16, 32, 64, 128}; threshold > 0; 1 <= batch <= 4096; 1 <= max_entries <= 2^24.
 * The clusterer belongs to the current device. Errors: IGP_E_INVAL, IGP_E_NOMEM, IGP_E_CUDA. */
igp_status igp_clusterer_create(int32_t d, double threshold, int32_t batch, int32_t max_entries,
                                igp_clusterer** out);
/* Fit N more points (a partial fit: the entries so far are kept and grown).
 *   E      : N x d fp32 row-major, host or device, every coordinate in [-1, 1]
 *   labels : N int32 (host or device, or NULL): the entry each point joined
 * Synchronises `stream`. Errors: IGP_E_INVAL (a coordinate outside [-1, 1] or not finite: nothing
 * is fitted), IGP_E_NOMEM (more than max_entries entries: the batches before the one that would
 * exceed it are fitted), IGP_E_CUDA. */
igp_status igp_clusterer_fit(igp_clusterer* c, const float* E, int32_t N, int32_t* labels, void* stream);
/* The closest entry (fp32 squared distance to the centroids, ties to the smaller id) of each of N
 * points, labels[N] host or device; entries unchanged. IGP_E_INVAL before any fit. */
igp_status igp_clusterer_predict(igp_clusterer* c, const float* E, int32_t N, int32_t* labels, void* stream);
/* K (number of entries) and, if non-NULL, the K x d centroids and K member counts (host or device). */
igp_status igp_clusterer_info(igp_clusterer* c, int32_t* K, float* centroids, int64_t* counts, void* stream);
/* Release the clusterer (waits for the legacy default stream). NULL is a no-op. */
void igp_clusterer_free(igp_clusterer* c);

/* Per-phase device timing. Events are recorded on the call's stream around each phase. */
igp_status igp_profile_create(igp_profile** p);
void igp_profile_free(igp_profile* p);
/* Wait for the recorded events, add their durations up per phase (ms) and count the launches per
 * phase; both arrays have IGP_NUM_PHASES entries (either may be NULL). Clears the record. */
igp_status igp_profile_read(igp_profile* p, double* ms, int64_t* launches);

#ifdef __cplusplus
}
#endif
#endif /* IGP_H */
