// igp_graph_import: a graph handle from a CSR in the form igp_graph_export writes (the graph of
// Sec. II: symmetric binary adjacency, no self-loops; every row's columns sorted, no repeats), so
// that a graph can be stored and restored, or built by other means, without its edge list.
//
// Validation (optional) runs on the device, one warp per row: row_ptr starts at 0, does not
// decrease and ends at nnz; every column lies in [0, N), differs from its row and exceeds the
// previous column of the row; and every entry (i, j) has its mirror (j, i), found by binary search
// in row j. The largest degree is computed in any case (the degree order needs it).
#include "igp_internal.cuh"

namespace igp {
namespace {

constexpr int kBadPtr = 1, kBadRange = 2, kBadOrder = 4, kBadLoop = 8, kBadMirror = 16;

__global__ void k_imp_check(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int32_t N,
                            int64_t nnz, int validate, int* __restrict__ flags, int* __restrict__ max_deg) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int bad = 0, md = 0;
  for (int64_t i = w; i < N; i += nw) {
    const int64_t b = row_ptr[i], e = row_ptr[i + 1];
    if (b > e || b < 0 || e > nnz || (i == 0 && b != 0) || (i == N - 1 && e != nnz)) {
      bad |= kBadPtr;
      continue;
    }
    md = max(md, (int)(e - b));
    if (!validate) continue;
    for (int64_t k = b + lane; k < e; k += 32) {
      const int j = col[k];
      if (j < 0 || j >= N) {
        bad |= kBadRange;
        continue;
      }
      if (j == i) bad |= kBadLoop;
      if (k > b && col[k - 1] >= j) bad |= kBadOrder;
      // mirror (j, i): binary search in row j (sorted, if the row is valid)
      int64_t lo = row_ptr[j], hi = row_ptr[j + 1];
      if (lo < 0 || hi > nnz || lo > hi) {
        bad |= kBadPtr;
        continue;
      }
      bool found = false;
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int c = col[mid];
        if (c == (int)i) {
          found = true;
          break;
        }
        if (c < (int)i)
          lo = mid + 1;
        else
          hi = mid;
      }
      if (!found) bad |= kBadMirror;
    }
  }
  bad = __reduce_or_sync(0xffffffffu, bad);
  md = __reduce_max_sync(0xffffffffu, md);
  if (lane == 0) {
    if (bad) atomicOr(flags, bad);
    atomicMax(max_deg, md);
  }
}

}  // namespace
}  // namespace igp

using namespace igp;

extern "C" igp_status igp_graph_import(const int32_t* row_ptr, const int32_t* col, int32_t N, int64_t nnz,
                                       int32_t validate, void* stream, igp_graph** out) {
  clear_error();
  if (!out) {
    set_error("igp_graph_import: out is NULL");
    return IGP_E_INVAL;
  }
  *out = nullptr;
  if (!row_ptr || N < 1 || N >= 2147483647 || nnz < 0 || nnz >= (1LL << 31) || (nnz > 0 && !col)) {
    set_error("igp_graph_import: need row_ptr, 1 <= N < 2^31-1, 0 <= nnz < 2^31 and col (N=%d, nnz=%lld)", N,
              (long long)nnz);
    return IGP_E_INVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  igp_graph* g = new (std::nothrow) igp_graph();
  if (!g) {
    set_error("igp_graph_import: host allocation failed");
    return IGP_E_NOMEM;
  }
  cudaGetDevice(&g->device);
  count_alloc();
  int* host = nullptr;  // [flags, max_deg]
  void *rp = nullptr, *cl = nullptr, *tmp = nullptr;
  igp_status st = IGP_OK;
  auto fail = [&](igp_status e) {
    dev_free(rp, s);
    dev_free(cl, s);
    dev_free(tmp, s);
    cudaStreamSynchronize(s);
    release_slot(host);  // the stream has drained: no copy is pending
    if (g->done) cudaEventDestroy(g->done);
    release_slot(g->err_host);
    delete g;
    return e;
  };
  if (cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming) != cudaSuccess ||
      (g->err_host = pinned_slot()) == nullptr || (host = pinned_slot()) == nullptr)
    return fail(cuda_status(cudaGetLastError(), "graph handle set-up", __FILE__, __LINE__));
  *g->err_host = 0;
  const size_t bp = ((size_t)N + 1) * sizeof(int32_t), bc = (size_t)nnz * sizeof(int32_t);
  st = dev_alloc(&rp, bp, s);
  if (st == IGP_OK) st = dev_alloc(&cl, bc, s);
  if (st == IGP_OK) st = dev_alloc(&tmp, 2 * sizeof(int), s);
  if (st != IGP_OK) return fail(st);
  const cudaMemcpyKind kr = is_device_ptr(row_ptr) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind kc = (nnz > 0 && is_device_ptr(col)) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (cudaMemcpyAsync(rp, row_ptr, bp, kr, s) != cudaSuccess ||
      (nnz > 0 && cudaMemcpyAsync(cl, col, bc, kc, s) != cudaSuccess) ||
      cudaMemsetAsync(tmp, 0, 2 * sizeof(int), s) != cudaSuccess)
    return fail(cuda_status(cudaGetLastError(), "igp_graph_import copies", __FILE__, __LINE__));
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)N * 32 + 255) / 256, (int64_t)num_sms() * 8));
  k_imp_check<<<blocks, 256, 0, s>>>((const int32_t*)rp, (const int32_t*)cl, N, nnz, validate ? 1 : 0, (int*)tmp,
                                     (int*)tmp + 1);
  if ((st = after_launch("k_imp_check")) != IGP_OK) return fail(st);
  if (cudaMemcpyAsync(host, tmp, 2 * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail(cuda_status(cudaGetLastError(), "igp_graph_import check", __FILE__, __LINE__));
  if (host[0]) {
    set_error("igp_graph_import: not a CSR of an undirected simple graph:%s%s%s%s%s", (host[0] & kBadPtr) ? " row_ptr" : "",
              (host[0] & kBadRange) ? " column out of range" : "", (host[0] & kBadOrder) ? " row not sorted or repeated" : "",
              (host[0] & kBadLoop) ? " self-loop" : "", (host[0] & kBadMirror) ? " not symmetric" : "");
    return fail(IGP_E_INVAL);
  }
  g->N = N;
  g->nnz = nnz;
  g->max_deg = host[1];
  g->row_ptr = (int32_t*)rp;
  g->col = (int32_t*)cl;
  dev_free(tmp, s);
  release_slot(host);  // read after the stream synchronisation above
  if (cudaEventRecord(g->done, s) != cudaSuccess) {
    rp = cl = tmp = nullptr;
    host = nullptr;
    igp_graph_free(g);
    return cuda_status(cudaGetLastError(), "cudaEventRecord", __FILE__, __LINE__);
  }
  *out = g;
  return IGP_OK;
}
