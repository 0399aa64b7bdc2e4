// CSR construction of the symmetric binary adjacency A (Sec. II of the paper:
// undirected, unweighted, simple graph) from an undirected edge list.
//
// Pipeline (all on the device, integer-exact, result independent of scheduling):
//   1. k_count     validate ids, count both directions of every non-loop edge per row
//   2. scan        exclusive prefix sum of the counts -> row offsets of the raw buckets
//   3. k_scatter   bucket each directed entry into its row (atomic cursor per row)
//   4. k_sort_rows_warp / k_sort_rows_big
//                  sort every bucket ascending (bitonic network; one warp per short
//                  row, one CTA per long row), drop repeated columns in place and
//                  record the unique count
//   5. scan        exclusive prefix sum of the unique counts -> row_ptr
//   6. k_compact   copy each row's unique columns to the final col[] array
// The order in which the atomics of step 3 fill a bucket does not matter: step 4
// sorts it, so the CSR is the same on every run (sorted, deduplicated rows).
#include <climits>
#include <cstdio>

#include "igp_internal.cuh"

namespace igp {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 8192 elements per tile

constexpr int kWarpCap = 1024;          // rows longer than this go to the CTA sorter
constexpr int kSortWarps = 8;           // warps per CTA in the warp sorter
constexpr int kBigThreads = 1024;
constexpr int kBigSmemCap = 48 * 1024;  // ints staged in shared memory (192 KB)

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ------------------------------------------------------------------ scan
// Block-wide exclusive scan of kScanItems consecutive ints per thread.
__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_tot, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
    int wx = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, wx, o);
      if (lane >= o) wx += y;
    }
    if (lane < (int)(blockDim.x >> 5)) warp_tot[lane] = wx - w;  // exclusive per warp
    if (lane == 31) *total = wx;
  }
  __syncthreads();
  int r = warp_tot[warp] + x - v;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tile_sums(const int* __restrict__ in, int64_t n,
                                                                  int* __restrict__ tile_sums) {
  __shared__ int red[32];
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) s += in[base + k];
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    int w = red[threadIdx.x];
#pragma unroll
    for (int o = 16; o; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = w;
  }
}

// One CTA: exclusive scan of the tile sums in place (any count, chunked with a carry).
__global__ void __launch_bounds__(kScanThreads) k_scan_tile_prefix(int* __restrict__ tile_sums, int64_t ntiles) {
  __shared__ int warp_tot[32];
  __shared__ int total;
  int carry = 0;
  for (int64_t c0 = 0; c0 < ntiles; c0 += kScanTile) {
    int64_t base = c0 + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      v[k] = (base + k < ntiles) ? tile_sums[base + k] : 0;
      s += v[k];
    }
    int ex = block_exclusive_scan(s, warp_tot, &total) + carry;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      if (base + k < ntiles) tile_sums[base + k] = ex;
      ex += v[k];
    }
    carry += total;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const int* __restrict__ in, int64_t n,
                                                              const int* __restrict__ tile_prefix,
                                                              int* __restrict__ out) {
  __shared__ int warp_tot[32];
  __shared__ int total;
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int v[kScanItems];
  int s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    s += v[k];
  }
  int ex = block_exclusive_scan(s, warp_tot, &total) + tile_prefix[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = ex;
    ex += v[k];
  }
}

}  // namespace

// Exclusive scan of n ints (n >= 1). tmp must hold ceil(n / kScanTile) ints.
igp_status exclusive_scan(const int* in, int* out, int64_t n, int* tmp, cudaStream_t s) {
  int64_t ntiles = (n + kScanTile - 1) / kScanTile;
  k_scan_tile_sums<<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, n, tmp);
  IGP_TRY(after_launch("k_scan_tile_sums"));
  k_scan_tile_prefix<<<1, kScanThreads, 0, s>>>(tmp, ntiles);
  IGP_TRY(after_launch("k_scan_tile_prefix"));
  k_scan_tiles<<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, n, tmp, out);
  return after_launch("k_scan_tiles");
}

namespace {

// ------------------------------------------------------------------ count / scatter
__global__ void k_count(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t M,
                        int32_t N, int* __restrict__ cnt, unsigned long long* __restrict__ bad_edge) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < M; e += (int64_t)gridDim.x * blockDim.x) {
    int32_t u = src[e], v = dst[e];
    if ((uint32_t)u >= (uint32_t)N || (uint32_t)v >= (uint32_t)N) {
      atomicMin(bad_edge, (unsigned long long)e);
      continue;
    }
    if (u != v) {
      atomicAdd(&cnt[u], 1);
      atomicAdd(&cnt[v], 1);
    }
  }
}

// cnt[] holds the bucket sizes on entry and is counted down to 0.
__global__ void k_scatter(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t M,
                          int32_t N, const int* __restrict__ off, int* __restrict__ cnt,
                          int32_t* __restrict__ buf) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < M; e += (int64_t)gridDim.x * blockDim.x) {
    int32_t u = src[e], v = dst[e];
    if ((uint32_t)u >= (uint32_t)N || (uint32_t)v >= (uint32_t)N || u == v) continue;
    int pu = atomicSub(&cnt[u], 1) - 1;
    buf[off[u] + pu] = v;
    int pv = atomicSub(&cnt[v], 1) - 1;
    buf[off[v] + pv] = u;
  }
}

// ------------------------------------------------------------------ per-row sort + dedup
// Bitonic sorting network with every comparator ascending (min to the lower index):
// block size k = 2, 4, .., P (P = next power of two >= n); per k one "flip" step
// (i against i ^ (k-1)) then half-cleaners (i against i + j, j = k/4 .. 1). Indices
// >= n act as +infinity, so a comparator whose upper index is >= n is skipped and no
// padding storage is needed.
__device__ __forceinline__ void cswap(int32_t* a, int i, int p) {
  int32_t x = a[i], y = a[p];
  if (x > y) {
    a[i] = y;
    a[p] = x;
  }
}

__device__ void warp_bitonic_smem(int32_t* a, int n) {
  const int lane = threadIdx.x & 31;
  int P = 1;
  while (P < n) P <<= 1;
  for (int k = 2; k <= P; k <<= 1) {
    const int h = k >> 1;
    for (int t = lane; t < (P >> 1); t += 32) {
      int i = ((t & ~(h - 1)) << 1) | (t & (h - 1));
      int p = i ^ (k - 1);
      if (p < n) cswap(a, i, p);
    }
    __syncwarp();
    for (int j = k >> 2; j >= 1; j >>= 1) {
      for (int t = lane; t < (P >> 1); t += 32) {
        int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
        int p = i + j;
        if (p < n) cswap(a, i, p);
      }
      __syncwarp();
    }
  }
}

__device__ void block_bitonic(int32_t* a, int n) {
  int P = 1;
  while (P < n) P <<= 1;
  for (int k = 2; k <= P; k <<= 1) {
    const int h = k >> 1;
    for (int t = threadIdx.x; t < (P >> 1); t += blockDim.x) {
      int i = ((t & ~(h - 1)) << 1) | (t & (h - 1));
      int p = i ^ (k - 1);
      if (p < n) cswap(a, i, p);
    }
    __syncthreads();
    for (int j = k >> 2; j >= 1; j >>= 1) {
      for (int t = threadIdx.x; t < (P >> 1); t += blockDim.x) {
        int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
        int p = i + j;
        if (p < n) cswap(a, i, p);
      }
      __syncthreads();
    }
  }
}

// One warp per row. Rows with more than kWarpCap entries are queued for k_sort_rows_big.
__global__ void __launch_bounds__(kSortWarps * 32) k_sort_rows_warp(const int* __restrict__ off, int32_t N,
                                                                    int32_t* __restrict__ buf, int* __restrict__ ucnt,
                                                                    int* __restrict__ big_rows, int* __restrict__ n_big,
                                                                    int* __restrict__ max_deg) {
  __shared__ int32_t sm[kSortWarps][kWarpCap];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t* a = sm[warp];
  int local_max = 0;
  for (int64_t i = (int64_t)blockIdx.x * kSortWarps + warp; i < N; i += (int64_t)gridDim.x * kSortWarps) {
    const int s = off[i];
    const int n = off[i + 1] - s;
    if (n > kWarpCap) {
      if (lane == 0) big_rows[atomicAdd(n_big, 1)] = (int)i;
      continue;
    }
    int uniq;
    if (n <= 32) {
      int32_t v = (lane < n) ? buf[s + lane] : INT_MAX;
      for (int k = 2; k <= 32; k <<= 1) {
        int32_t w = __shfl_xor_sync(0xffffffffu, v, k - 1);
        bool lower = (lane & (k >> 1)) == 0;  // lane < partner in the flip step
        v = lower ? min(v, w) : max(v, w);
        for (int j = k >> 2; j >= 1; j >>= 1) {
          w = __shfl_xor_sync(0xffffffffu, v, j);
          v = (lane & j) ? max(v, w) : min(v, w);
        }
      }
      int32_t prev = __shfl_up_sync(0xffffffffu, v, 1);
      bool f = lane < n && (lane == 0 || v != prev);
      unsigned m = __ballot_sync(0xffffffffu, f);
      if (f) buf[s + __popc(m & lanemask_lt())] = v;
      uniq = __popc(m);
    } else {
      for (int t = lane; t < n; t += 32) a[t] = buf[s + t];
      __syncwarp();
      warp_bitonic_smem(a, n);
      int base = 0;
      for (int c = 0; c < n; c += 32) {
        int t = c + lane;
        int32_t v = (t < n) ? a[t] : 0;
        bool f = t < n && (t == 0 || v != a[t - 1]);
        unsigned m = __ballot_sync(0xffffffffu, f);
        if (f) buf[s + base + __popc(m & lanemask_lt())] = v;
        base += __popc(m);
      }
      uniq = base;
      __syncwarp();
    }
    if (lane == 0) ucnt[i] = uniq;
    local_max = max(local_max, uniq);
  }
  if (lane == 0 && local_max > 0) atomicMax(max_deg, local_max);
}

// One CTA per long row: sorted in shared memory when it fits, else in place in global memory.
__global__ void __launch_bounds__(kBigThreads) k_sort_rows_big(const int* __restrict__ off, int32_t* buf,
                                                               int* __restrict__ ucnt, const int* __restrict__ big_rows,
                                                               const int* __restrict__ n_big, int* __restrict__ max_deg) {
  extern __shared__ int32_t dyn[];
  __shared__ int warp_tot[32];
  __shared__ int total;
  __shared__ int32_t carry_last;
  const int nb = *n_big;
  for (int r = blockIdx.x; r < nb; r += gridDim.x) {
    const int i = big_rows[r];
    const int s = off[i];
    const int n = off[i + 1] - s;
    int32_t* a;
    if (n <= kBigSmemCap) {
      a = dyn;
      for (int t = threadIdx.x; t < n; t += blockDim.x) a[t] = buf[s + t];
      __syncthreads();
    } else {
      a = buf + s;
    }
    block_bitonic(a, n);
    // dedup in chunks of blockDim: read chunk (and the previous value), then write compacted
    int base = 0;
    if (threadIdx.x == 0) carry_last = INT_MIN;
    __syncthreads();
    for (int c = 0; c < n; c += blockDim.x) {
      int t = c + threadIdx.x;
      int32_t v = (t < n) ? a[t] : 0;
      int32_t prev = (t == c) ? carry_last : ((t < n) ? a[t - 1] : 0);
      int f = (t < n && (t == 0 || v != prev)) ? 1 : 0;
      int ex = block_exclusive_scan(f, warp_tot, &total);  // has __syncthreads inside
      int last_idx = min(n, c + (int)blockDim.x) - 1;
      if (t == last_idx) carry_last = v;
      if (f) buf[s + base + ex] = v;
      base += total;
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      ucnt[i] = base;
      atomicMax(max_deg, base);
    }
    __syncthreads();
  }
}

__global__ void k_compact(const int* __restrict__ off, const int32_t* __restrict__ buf, const int* __restrict__ row_ptr,
                          int32_t N, int32_t* __restrict__ col) {
  const int lane = threadIdx.x & 31;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < N;
       i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int s = off[i];
    const int d = row_ptr[i];
    const int n = row_ptr[i + 1] - d;
    for (int t = lane; t < n; t += 32) col[d + t] = buf[s + t];
  }
}

// ------------------------------------------------------------------ streaming merge
// Union of the sorted, duplicate-free rows of the old CSR (rows < N_old) and of the
// increment's CSR (N_new rows), one warp per row. Pass 1 drops from each increment row
// the columns the old row already has (compacting the increment row in place, in order)
// and counts the union; pass 2 merges the two now disjoint sorted lists: an element's
// place is its index in its own list plus the number of smaller elements of the other.
__device__ __forceinline__ int lower_bound_dev(const int32_t* a, int n, int32_t x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < x)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

__global__ void k_merge_count(const int32_t* __restrict__ rp_a, const int32_t* __restrict__ col_a, int32_t N_old,
                              const int32_t* __restrict__ rp_b, int32_t* col_b, int32_t N_new, int* __restrict__ cnt,
                              int* __restrict__ nbp, int* __restrict__ max_deg) {
  const int lane = threadIdx.x & 31;
  int local_max = 0;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < N_new;
       i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int32_t* A = col_a + (i < N_old ? rp_a[i] : 0);
    const int na = i < N_old ? rp_a[i + 1] - rp_a[i] : 0;
    int32_t* B = col_b + rp_b[i];
    const int nb = rp_b[i + 1] - rp_b[i];
    int base = 0;
    for (int c = 0; c < nb; c += 32) {
      const int k = c + lane;
      const bool valid = k < nb;
      const int32_t x = valid ? B[k] : 0;
      bool keep = false;
      if (valid) {
        const int r = lower_bound_dev(A, na, x);
        keep = !(r < na && A[r] == x);
      }
      const unsigned m = __ballot_sync(0xffffffffu, keep);  // all reads of the chunk precede the writes
      if (keep) B[base + __popc(m & lanemask_lt())] = x;
      base += __popc(m);
    }
    const int n = na + base;
    if (lane == 0) {
      cnt[i] = n;
      nbp[i] = base;
    }
    local_max = max(local_max, n);
  }
  if (lane == 0 && local_max > 0) atomicMax(max_deg, local_max);
}

__global__ void k_merge_write(const int32_t* __restrict__ rp_a, const int32_t* __restrict__ col_a, int32_t N_old,
                              const int32_t* __restrict__ rp_b, const int32_t* __restrict__ col_b,
                              const int* __restrict__ nbp, int32_t N_new, const int32_t* __restrict__ rp_out,
                              int32_t* __restrict__ col_out) {
  const int lane = threadIdx.x & 31;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < N_new;
       i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int32_t* A = col_a + (i < N_old ? rp_a[i] : 0);
    const int na = i < N_old ? rp_a[i + 1] - rp_a[i] : 0;
    const int32_t* B = col_b + rp_b[i];
    const int nb = nbp[i];
    const int o = rp_out[i];
    for (int k = lane; k < na; k += 32) col_out[o + k + lower_bound_dev(B, nb, A[k])] = A[k];
    for (int k = lane; k < nb; k += 32) col_out[o + k + lower_bound_dev(A, na, B[k])] = B[k];
  }
}

}  // namespace

igp_status build_csr(const int32_t* src, const int32_t* dst, int64_t M, int32_t N, cudaStream_t s, igp_graph* g) {
  const int sms = num_sms();
  const int64_t n1 = (int64_t)N + 1;
  const int64_t ntiles = (n1 + kScanTile - 1) / kScanTile;
  const int64_t cap = 2 * M > 0 ? 2 * M : 1;
  const int64_t max_big = cap / kWarpCap + 1;

  // one temporary block: cnt | off | ucnt | tile tmp | big_rows | scalars(4) | buf
  size_t o_cnt = 0;
  size_t o_off = o_cnt + n1;
  size_t o_ucnt = o_off + n1;
  size_t o_tmp = o_ucnt + n1;
  size_t o_big = o_tmp + ntiles;
  size_t o_sc = o_big + max_big;
  size_t o_bad = (o_sc + 4 + 1) & ~(size_t)1;  // 8-byte aligned (in ints)
  size_t o_buf = o_bad + 2;
  size_t total_ints = o_buf + cap;
  void* tmp_raw = nullptr;
  IGP_TRY(dev_alloc(&tmp_raw, total_ints * sizeof(int), s));
  int* T = (int*)tmp_raw;
  int* cnt = T + o_cnt;
  int* off = T + o_off;
  int* ucnt = T + o_ucnt;
  int* tiles = T + o_tmp;
  int* big_rows = T + o_big;
  int* n_big = T + o_sc;
  int* max_deg = T + o_sc + 1;
  unsigned long long* bad = (unsigned long long*)(T + o_bad);
  int32_t* buf = T + o_buf;

  igp_status st = IGP_OK;
  auto fail = [&](igp_status e) {
    dev_free(tmp_raw, s);
    return e;
  };
#define STEP(x)                \
  do {                         \
    st = (x);                  \
    if (st != IGP_OK) return fail(st); \
  } while (0)

  auto cu = [](cudaError_t e, const char* what) {
    return e == cudaSuccess ? IGP_OK : cuda_status(e, what, __FILE__, __LINE__);
  };
  STEP(cu(cudaMemsetAsync(cnt, 0, n1 * sizeof(int), s), "memset cnt"));
  STEP(cu(cudaMemsetAsync(ucnt + N, 0, sizeof(int), s), "memset ucnt"));
  STEP(cu(cudaMemsetAsync(n_big, 0, 2 * sizeof(int), s), "memset scalars"));
  STEP(cu(cudaMemsetAsync(bad, 0xFF, sizeof(unsigned long long), s), "memset bad"));

  const int eblocks = (int)std::min<int64_t>((M + 255) / 256 > 0 ? (M + 255) / 256 : 1, (int64_t)sms * 16);
  k_count<<<eblocks, 256, 0, s>>>(src, dst, M, N, cnt, bad);
  STEP(after_launch("k_count"));
  STEP(exclusive_scan(cnt, off, n1, tiles, s));
  k_scatter<<<eblocks, 256, 0, s>>>(src, dst, M, N, off, cnt, buf);
  STEP(after_launch("k_scatter"));
  const int rblocks = (int)std::min<int64_t>((N + kSortWarps - 1) / kSortWarps, (int64_t)sms * 8);
  k_sort_rows_warp<<<rblocks, kSortWarps * 32, 0, s>>>(off, N, buf, ucnt, big_rows, n_big, max_deg);
  STEP(after_launch("k_sort_rows_warp"));
  STEP(cu(cudaFuncSetAttribute(k_sort_rows_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kBigSmemCap * (int)sizeof(int)),
          "k_sort_rows_big smem"));
  k_sort_rows_big<<<sms, kBigThreads, kBigSmemCap * sizeof(int), s>>>(off, buf, ucnt, big_rows, n_big, max_deg);
  STEP(after_launch("k_sort_rows_big"));
  int32_t* row_ptr = nullptr;
  {
    void* p = nullptr;
    STEP(dev_alloc(&p, n1 * sizeof(int32_t), s));
    row_ptr = (int32_t*)p;
  }
  auto fail2 = [&](igp_status e) {
    dev_free(row_ptr, s);
    return fail(e);
  };
  st = exclusive_scan(ucnt, row_ptr, n1, tiles, s);
  if (st != IGP_OK) return fail2(st);

  // one synchronisation: the column count and the validation result
  int host_sc[2];
  unsigned long long host_bad = 0;
  int host_nnz = 0;
  if (cudaMemcpyAsync(&host_nnz, row_ptr + N, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(host_sc, n_big, 2 * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&host_bad, bad, sizeof(host_bad), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail2(cuda_status(cudaGetLastError(), "igp_graph_build readback", __FILE__, __LINE__));
  if (host_bad != ~0ull) {
    set_error("igp_graph_build: edge %llu has a node id outside [0, %d)", host_bad, N);
    return fail2(IGP_E_INVAL);
  }
  int32_t* col = nullptr;
  {
    void* p = nullptr;
    igp_status e = dev_alloc(&p, (size_t)(host_nnz > 0 ? host_nnz : 1) * sizeof(int32_t), s);
    if (e != IGP_OK) return fail2(e);
    col = (int32_t*)p;
  }
  const int cblocks = (int)std::min<int64_t>((N * 32LL + 255) / 256, (int64_t)sms * 16);
  k_compact<<<cblocks, 256, 0, s>>>(off, buf, row_ptr, N, col);
  st = after_launch("k_compact");
  if (st != IGP_OK) {
    dev_free(col, s);
    return fail2(st);
  }
  dev_free(tmp_raw, s);
  g->N = N;
  g->nnz = host_nnz;
  g->max_deg = host_sc[1];
  g->row_ptr = row_ptr;
  g->col = col;
  return IGP_OK;
#undef STEP
}

// Alg. 2, lines 1-2: merge an increment of edges (and new nodes up to N_new) into g.
igp_status append_csr(igp_graph* g, const int32_t* src, const int32_t* dst, int64_t M, int32_t N_new, cudaStream_t s) {
  igp_graph inc;
  IGP_TRY(build_csr(src, dst, M, N_new, s, &inc));  // validates ids, sorts and dedups the increment
  const int64_t n1 = (int64_t)N_new + 1;
  const int64_t ntiles = (n1 + kScanTile - 1) / kScanTile;
  void* t = nullptr;
  igp_status st = dev_alloc(&t, (size_t)(2 * n1 + ntiles + 1) * sizeof(int), s);
  if (st != IGP_OK) {
    dev_free(inc.row_ptr, s);
    dev_free(inc.col, s);
    return st;
  }
  int* cnt = (int*)t;
  int* nbp = cnt + n1;
  int* tiles = nbp + n1;
  int* max_deg = tiles + ntiles;
  int32_t* rp = nullptr;
  int32_t* col = nullptr;
  int host_nnz = 0, host_max = 0;
  auto cleanup = [&](igp_status e) {
    dev_free(t, s);
    dev_free(inc.row_ptr, s);
    dev_free(inc.col, s);
    if (e != IGP_OK) {
      dev_free(rp, s);
      dev_free(col, s);
    }
    return e;
  };
  if (cudaMemsetAsync(cnt + N_new, 0, sizeof(int), s) != cudaSuccess ||
      cudaMemsetAsync(max_deg, 0, sizeof(int), s) != cudaSuccess)
    return cleanup(cuda_status(cudaGetLastError(), "memset", __FILE__, __LINE__));
  const int blocks = (int)std::min<int64_t>((n1 * 32 + 255) / 256, (int64_t)num_sms() * 16);
  k_merge_count<<<blocks, 256, 0, s>>>(g->row_ptr, g->col, g->N, inc.row_ptr, inc.col, N_new, cnt, nbp, max_deg);
  if ((st = after_launch("k_merge_count")) != IGP_OK) return cleanup(st);
  {
    void* p = nullptr;
    if ((st = dev_alloc(&p, n1 * sizeof(int32_t), s)) != IGP_OK) return cleanup(st);
    rp = (int32_t*)p;
  }
  if ((st = exclusive_scan(cnt, rp, n1, tiles, s)) != IGP_OK) return cleanup(st);
  if (cudaMemcpyAsync(&host_nnz, rp + N_new, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&host_max, max_deg, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return cleanup(cuda_status(cudaGetLastError(), "igp_graph_append readback", __FILE__, __LINE__));
  {
    void* p = nullptr;
    if ((st = dev_alloc(&p, (size_t)std::max(host_nnz, 1) * sizeof(int32_t), s)) != IGP_OK) return cleanup(st);
    col = (int32_t*)p;
  }
  k_merge_write<<<blocks, 256, 0, s>>>(g->row_ptr, g->col, g->N, inc.row_ptr, inc.col, nbp, N_new, rp, col);
  if ((st = after_launch("k_merge_write")) != IGP_OK) return cleanup(st);
  cleanup(IGP_OK);
  dev_free(g->row_ptr, s);
  dev_free(g->col, s);
  g->row_ptr = rp;
  g->col = col;
  g->nnz = host_nnz;
  g->max_deg = host_max;
  if (N_new != g->N) {  // per-node arrays change size
    dev_free(g->dinv, s);
    g->dinv = g->wsum = nullptr;
  }
  g->N = N_new;
  g->dinv_valid = false;
  dev_free(g->perm, s);
  g->perm = nullptr;
  return IGP_OK;
}

}  // namespace igp
