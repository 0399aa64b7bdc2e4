// CSR construction of the symmetric binary adjacency A (Sec. II of the paper:
// undirected, unweighted, simple graph) from an undirected edge list.
//
// Partitioned build (up to 4096 buckets of up to 1024 rows, packed entries in 32 bits; all
// on the device, integer-exact, result independent of scheduling):
//   1. k_part_count   validate ids; per CTA and bucket, count the directed entries of
//                     every non-loop edge (shared-memory histogram, no global atomics)
//   2. scan           exclusive prefix sum over (bucket, CTA): each CTA's run in each bucket
//   3. k_part_scatter write every directed entry, packed (row in bucket, column) in 32
//                     bits, into its CTA's run of its bucket, staged through shared memory
//                     so that the runs fill front to back with contiguous writes
//   4. k_bucket_rows  one CTA per bucket: place the entries by row in shared memory, sort
//                     every row (in registers by one warp up to 512 entries, else by the
//                     whole CTA), drop repeated columns, write the bucket's rows back to
//                     back and record where each row starts and its distinct count
//   5. scan           exclusive prefix sum of the distinct counts -> row_ptr
//   6. k_rows_out     copy each row's distinct columns to its place in col[]
// Row u belongs to bucket u mod NB (NB a power of two) as local row u / NB, so a bucket
// collects rows from the whole id range and bucket sizes stay near their mean whatever
// order the ids come in.
//
// Atomic build (larger graphs):
//   1. k_count     validate ids, count both directions of every non-loop edge per row
//   2. scan        exclusive prefix sum of the counts -> row offsets of the raw buckets
//   3. k_scatter   bucket each directed entry into its row (atomic cursor per row)
//   4. k_sort_rows_warp / k_sort_rows_big
//                  sort every bucket ascending (bitonic network; one warp per short
//                  row, one CTA per long row), drop repeated columns in place and
//                  record the unique count
//   5. scan        exclusive prefix sum of the unique counts -> row_ptr
//   6. k_compact   copy each row's unique columns to the final col[] array
// In both, the order in which atomics fill a row does not matter: every row is sorted
// afterwards, so the CSR is the same on every run (sorted, deduplicated rows).
#include <algorithm>
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

// ------------------------------------------------------------------ partitioned build
// Row u belongs to bucket u & (NB - 1) as its local row u >> kb (NB = 2^kb), so a bucket
// collects rows from the whole id range and bucket sizes stay near their mean whatever
// order the ids come in. A directed entry is packed as local row << colbits | column.
constexpr int kPartThreads = 1024;     // k_part_count / k_part_scatter
constexpr int kPartTile = 8192;        // edges a scatter CTA stages per round
constexpr int kPartMaxBits = 12;       // at most 4096 buckets
constexpr int kPartEntries = 65536;    // target directed entries per bucket
constexpr int kBucketThreads = 1024;   // k_bucket_rows
constexpr int kBucketCap = 52 * 1024;  // entries a bucket places in shared memory (208 KB)
constexpr int kMaxLocalRows = 1024;    // rows per bucket
constexpr int kRegSortMax = 512;       // longest row a warp sorts in registers
constexpr int kGroupWarps = 4;         // warps of a group that sorts one longer row in shared memory
constexpr int kGroupSortMax = 8192;    // longest row a group sorts (longer ones: the whole CTA)
constexpr int kMaxLongRows = 512;      // longer rows of a bucket listed for the groups
constexpr int kLoadBatch = 8;          // independent loads a thread issues before using them

struct PartGeom {
  int kb;       // NB = 2^kb buckets
  int colbits;  // bits of a column id (col < N)
};

// Bucket geometry for `entries` directed entries over N rows; false if the packed entry
// does not fit 32 bits or a bucket would hold more than kMaxLocalRows rows.
bool part_geom(int64_t entries, int32_t N, PartGeom* g) {
  int kb = 0;
  while (kb < kPartMaxBits && ((int64_t)kPartEntries << kb) < entries) ++kb;
  while (kb < kPartMaxBits && ((((int64_t)N + (1ll << kb) - 1) >> kb) > kMaxLocalRows)) ++kb;
  const int64_t R = ((int64_t)N + (1ll << kb) - 1) >> kb;
  if (R > kMaxLocalRows) return false;
  int colbits = 1, rowbits = 0;
  while ((1ll << colbits) < N) ++colbits;
  while ((1ll << rowbits) < R) ++rowbits;
  if (colbits + rowbits > 32) return false;
  g->kb = kb;
  g->colbits = colbits;
  return true;
}

// Edges of CTA c: [c * per, min(M, (c + 1) * per)). cnt[b * gridDim.x + c] = entries of
// CTA c in bucket b (both directions of every valid non-loop edge).
__global__ void __launch_bounds__(kPartThreads) k_part_count(const int32_t* __restrict__ src,
                                                             const int32_t* __restrict__ dst, int64_t M, int32_t N,
                                                             int kb, int64_t per, int* __restrict__ cnt,
                                                             unsigned long long* __restrict__ bad_edge) {
  __shared__ int hist[1 << kPartMaxBits];
  const int NB = 1 << kb;
  for (int b = threadIdx.x; b < NB; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  const int64_t e0 = (int64_t)blockIdx.x * per;
  const int64_t e1 = e0 + per < M ? e0 + per : M;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += (int64_t)kLoadBatch * blockDim.x) {
    int32_t u[kLoadBatch], v[kLoadBatch];
#pragma unroll
    for (int k = 0; k < kLoadBatch; ++k) {
      const int64_t ek = e + (int64_t)k * blockDim.x;
      u[k] = ek < e1 ? src[ek] : 0;
      v[k] = ek < e1 ? dst[ek] : 0;
    }
#pragma unroll
    for (int k = 0; k < kLoadBatch; ++k) {
      const int64_t ek = e + (int64_t)k * blockDim.x;
      if (ek >= e1) continue;
      if ((uint32_t)u[k] >= (uint32_t)N || (uint32_t)v[k] >= (uint32_t)N) {
        atomicMin(bad_edge, (unsigned long long)ek);
        continue;
      }
      if (u[k] == v[k]) continue;
      atomicAdd(&hist[u[k] & (NB - 1)], 1);
      atomicAdd(&hist[v[k] & (NB - 1)], 1);
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < NB; b += blockDim.x) cnt[(int64_t)b * gridDim.x + blockIdx.x] = hist[b];
}

// pos[b * gridDim.x + c]: start of CTA c's run in bucket b (exclusive scan of k_part_count's
// output). Each round stages kPartTile edges' entries in shared memory grouped by bucket,
// then writes every bucket's group to the next free places of the CTA's run, so the run
// fills front to back and the writes of a group are contiguous.
__global__ void __launch_bounds__(kPartThreads) k_part_scatter(const int32_t* __restrict__ src,
                                                               const int32_t* __restrict__ dst, int64_t M,
                                                               int32_t N, int kb, int colbits, int64_t per,
                                                               const int* __restrict__ pos,
                                                               uint32_t* __restrict__ ebuf) {
  constexpr int EPT = kPartTile / kPartThreads;  // edges per thread per round
  extern __shared__ uint32_t sm_p[];
  uint32_t* s_stage = sm_p;                                    // [2 kPartTile] packed entries
  uint16_t* s_sb = (uint16_t*)(sm_p + 2 * kPartTile);          // [2 kPartTile] their buckets
  int* s_cur = (int*)(sm_p + 3 * kPartTile);                   // [NB] next free place of the run
  int* s_cnt = s_cur + (1 << kPartMaxBits);                    // [NB] this round's count
  int* s_base = s_cnt + (1 << kPartMaxBits);                   // [NB] this round's group start
  const int NB = 1 << kb;
  __shared__ int warp_tot[32];
  __shared__ int total;
  for (int b = threadIdx.x; b < NB; b += blockDim.x) s_cur[b] = pos[(int64_t)b * gridDim.x + blockIdx.x];
  const int64_t e0 = (int64_t)blockIdx.x * per;
  const int64_t e1 = e0 + per < M ? e0 + per : M;
  constexpr int BPT = (1 << kPartMaxBits) / kPartThreads;  // buckets per thread in the scan
  for (int64_t t0 = e0; t0 < e1; t0 += kPartTile) {
    {  // the next round's edges into L2, read after this round: kPartTile ids of each array are
       // kPartTile / 32 lines of 128 bytes; one line per thread
      constexpr int kLines = kPartTile / 32;
      const int64_t n0 = t0 + kPartTile;
      if ((int)threadIdx.x < 2 * kLines) {
        const int64_t at = n0 + (int64_t)(threadIdx.x % kLines) * 32;
        const int32_t* arr = (int)threadIdx.x < kLines ? src : dst;
        if (at < e1) asm volatile("prefetch.global.L2 [%0];" ::"l"(arr + at));
      }
    }
    for (int b = threadIdx.x; b < NB; b += blockDim.x) s_cnt[b] = 0;
    __syncthreads();
    int32_t eu[EPT], ev[EPT];  // this thread's edges of the round (eu = -1: none)
    int ru[EPT], rv[EPT];      // their ranks within the round's bucket groups
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int64_t e = t0 + k * kPartThreads + threadIdx.x;
      eu[k] = ev[k] = -1;
      if (e < e1) {
        const int32_t u = src[e], v = dst[e];
        if ((uint32_t)u < (uint32_t)N && (uint32_t)v < (uint32_t)N && u != v) {
          eu[k] = u;
          ev[k] = v;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < EPT; ++k)
      if (eu[k] >= 0) {
        ru[k] = atomicAdd(&s_cnt[eu[k] & (NB - 1)], 1);
        rv[k] = atomicAdd(&s_cnt[ev[k] & (NB - 1)], 1);
      }
    __syncthreads();
    // exclusive scan of s_cnt[0..NB): thread t owns buckets t BPT .. t BPT + BPT - 1
    int c[BPT], sum = 0;
#pragma unroll
    for (int q = 0; q < BPT; ++q) {
      const int b = threadIdx.x * BPT + q;
      c[q] = b < NB ? s_cnt[b] : 0;
      sum += c[q];
    }
    int ex = block_exclusive_scan(sum, warp_tot, &total);
#pragma unroll
    for (int q = 0; q < BPT; ++q) {
      const int b = threadIdx.x * BPT + q;
      if (b < NB) s_base[b] = ex;
      ex += c[q];
    }
    __syncthreads();
    const int staged = total;
#pragma unroll
    for (int k = 0; k < EPT; ++k)
      if (eu[k] >= 0) {
        const int bu = eu[k] & (NB - 1), bv = ev[k] & (NB - 1);
        const int iu = s_base[bu] + ru[k], iv = s_base[bv] + rv[k];
        s_stage[iu] = ((uint32_t)(eu[k] >> kb) << colbits) | (uint32_t)ev[k];
        s_sb[iu] = (uint16_t)bu;
        s_stage[iv] = ((uint32_t)(ev[k] >> kb) << colbits) | (uint32_t)eu[k];
        s_sb[iv] = (uint16_t)bv;
      }
    __syncthreads();
    for (int i = threadIdx.x; i < staged; i += blockDim.x) {
      const int b = s_sb[i];
      ebuf[s_cur[b] + (i - s_base[b])] = s_stage[i];
    }
    __syncthreads();
    for (int b = threadIdx.x; b < NB; b += blockDim.x) s_cur[b] += s_cnt[b];
  }
}

// Bitonic sort of the 32 E values a warp holds (value k of lane l is element 32 k + l),
// ascending.
template <int E>
__device__ __forceinline__ void warp_bitonic_regs(int32_t (&v)[E]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int size = 2; size <= 32 * E; size <<= 1) {
#pragma unroll
    for (int j = size >> 1; j > 0; j >>= 1) {
      if (j >= 32) {
        const int kj = j >> 5;
#pragma unroll
        for (int k = 0; k < E; ++k) {
          if ((k & kj) == 0) {
            const int kp = k | kj;
            const bool up = ((k * 32 + lane) & size) == 0;
            const int32_t a = v[k], b = v[kp];
            v[k] = up ? min(a, b) : max(a, b);
            v[kp] = up ? max(a, b) : min(a, b);
          }
        }
      } else {
#pragma unroll
        for (int k = 0; k < E; ++k) {
          const int32_t w = __shfl_xor_sync(0xffffffffu, v[k], j);
          const bool keep_min = ((lane & j) == 0) == (((k * 32 + lane) & size) == 0);
          v[k] = keep_min ? min(v[k], w) : max(v[k], w);
        }
      }
    }
  }
}

// One warp: sort the n <= 32 E column ids at src (non-negative) and write the distinct
// ones, ascending, to out (which may be src). Returns the distinct count.
template <int E>
__device__ __forceinline__ int warp_sort_unique(const int32_t* src, int n, int32_t* out) {
  const int lane = threadIdx.x & 31;
  int32_t v[E];
#pragma unroll
  for (int k = 0; k < E; ++k) v[k] = (k * 32 + lane < n) ? src[k * 32 + lane] : INT_MAX;
  __syncwarp();  // every lane has read src before any lane writes out
  warp_bitonic_regs<E>(v);
  int base = 0;
  int32_t carry = INT_MIN;  // element 32 k - 1 (none before element 0; ids are >= 0)
#pragma unroll
  for (int k = 0; k < E; ++k) {
    int32_t prev = __shfl_up_sync(0xffffffffu, v[k], 1);
    if (lane == 0) prev = carry;
    const bool f = k * 32 + lane < n && v[k] != prev;
    const unsigned m = __ballot_sync(0xffffffffu, f);
    if (f) out[base + __popc(m & lanemask_lt())] = v[k];
    base += __popc(m);
    carry = __shfl_sync(0xffffffffu, v[k], 31);
  }
  return base;
}

__device__ __forceinline__ int warp_sort_unique_any(const int32_t* src, int n, int32_t* out) {
  if (n <= 32) return warp_sort_unique<1>(src, n, out);
  if (n <= 64) return warp_sort_unique<2>(src, n, out);
  if (n <= 128) return warp_sort_unique<4>(src, n, out);
  if (n <= 256) return warp_sort_unique<8>(src, n, out);
  return warp_sort_unique<16>(src, n, out);
}

// One warp: write the distinct values of the sorted w[0..n) to out (which may be w), ascending;
// returns their count.
__device__ int warp_unique_sorted(const int32_t* w, int n, int32_t* out) {
  const int lane = threadIdx.x & 31;
  int base = 0;
  int32_t carry = INT_MIN;  // last value of the previous chunk, read before any write
  for (int c = 0; c < n; c += 32) {
    const int t = c + lane;
    const int32_t v = t < n ? w[t] : 0;
    int32_t prev = __shfl_up_sync(0xffffffffu, v, 1);
    if (lane == 0) prev = carry;
    const bool f = t < n && v != prev;
    const unsigned m = __ballot_sync(0xffffffffu, f);
    carry = __shfl_sync(0xffffffffu, v, 31);
    __syncwarp();  // the chunk is read before it is overwritten
    if (f) out[base + __popc(m & lanemask_lt())] = v;
    base += __popc(m);
    __syncwarp();
  }
  return base;
}

// Barrier of the kGroupWarps warps of group `id` (named barrier id + 1; 0 is __syncthreads).
__device__ __forceinline__ void group_sync(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id + 1), "r"(kGroupWarps * 32) : "memory");
}

// The warps of one group: bitonic sort of a[0..n) in shared memory (the network of
// block_bitonic, comparators spread over the group's threads).
__device__ void group_bitonic(int32_t* a, int n, int gtid, int gid) {
  int P = 1;
  while (P < n) P <<= 1;
  for (int k = 2; k <= P; k <<= 1) {
    const int h = k >> 1;
    for (int t = gtid; t < (P >> 1); t += kGroupWarps * 32) {
      int i = ((t & ~(h - 1)) << 1) | (t & (h - 1));
      int p = i ^ (k - 1);
      if (p < n) cswap(a, i, p);
    }
    group_sync(gid);
    for (int j = k >> 2; j >= 1; j >>= 1) {
      for (int t = gtid; t < (P >> 1); t += kGroupWarps * 32) {
        int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
        int p = i + j;
        if (p < n) cswap(a, i, p);
      }
      group_sync(gid);
    }
  }
}

// Whole CTA: sort a[0..n) in place (shared or global memory), then write the distinct
// values, ascending, to out (which may be a). Returns the distinct count (all threads).
__device__ int block_sort_unique(int32_t* a, int n, int32_t* out, int* warp_tot, int* total, int32_t* carry_last) {
  block_bitonic(a, n);
  int base = 0;
  if (threadIdx.x == 0) *carry_last = INT_MIN;
  __syncthreads();
  for (int c = 0; c < n; c += blockDim.x) {
    const int t = c + threadIdx.x;
    const int32_t v = (t < n) ? a[t] : 0;
    const int32_t prev = (t == c) ? *carry_last : ((t < n) ? a[t - 1] : 0);
    const int f = (t < n && v != prev) ? 1 : 0;
    const int ex = block_exclusive_scan(f, warp_tot, total);  // synchronises: all reads precede the writes
    if (t == min(n, c + (int)blockDim.x) - 1) *carry_last = v;
    if (f) out[base + ex] = v;
    base += *total;
    __syncthreads();
  }
  return base;
}

// One CTA per bucket b: its entries ebuf[pos[b C] .. pos[(b + 1) C]) (C = CTAs of the
// scatter), E of them, for the rows u = b + r NB. The columns are placed by row in shared
// memory (in obuf's region of the bucket when E > kBucketCap), each row is sorted and made
// distinct in place (by a warp up to kRegSortMax entries, else by the whole CTA in shared
// memory), and the bucket's rows are written back to back to ebuf[pos[b C] ..], which the
// placement has finished reading: toff[u] = where row u starts, ucnt[u] = its length.
__global__ void __launch_bounds__(kBucketThreads) k_bucket_rows(uint32_t* __restrict__ ebuf,
                                                                const int* __restrict__ pos, int nC, int kb,
                                                                int colbits, int32_t N, int32_t* obuf,
                                                                int* __restrict__ toff, int* __restrict__ ucnt,
                                                                int* __restrict__ max_deg) {
  extern __shared__ int32_t s_col[];  // [kBucketCap]
  __shared__ int s_cnt[kMaxLocalRows], s_off[kMaxLocalRows], s_cur[kMaxLocalRows];
  __shared__ int warp_tot[32];
  __shared__ int total;
  __shared__ int32_t carry_last;
  __shared__ int s_max;
  __shared__ int s_long[kMaxLongRows];
  __shared__ int s_nlong;
  const int b = blockIdx.x;
  const int NB = 1 << kb;
  if (b >= N) return;  // no rows
  const int R = (N - 1 - b) / NB + 1;
  const int64_t e0 = pos[(int64_t)b * nC];
  const int E = (int)(pos[(int64_t)(b + 1) * nC] - e0);
  const bool fits = E <= kBucketCap;
  const uint32_t cmask = (uint32_t)((1ull << colbits) - 1);
  uint32_t* ent = ebuf + e0;
  int32_t* place = fits ? s_col : obuf + e0;
  for (int r = threadIdx.x; r < kMaxLocalRows; r += blockDim.x) s_cnt[r] = 0;
  if (threadIdx.x == 0) {
    s_max = 0;
    s_nlong = 0;
  }
  __syncthreads();
  for (int k0 = threadIdx.x; k0 < E; k0 += kLoadBatch * blockDim.x) {
    uint32_t x[kLoadBatch];
#pragma unroll
    for (int q = 0; q < kLoadBatch; ++q) {
      const int k = k0 + q * blockDim.x;
      x[q] = k < E ? ent[k] : 0u;
    }
#pragma unroll
    for (int q = 0; q < kLoadBatch; ++q)
      if (k0 + q * (int)blockDim.x < E) atomicAdd(&s_cnt[x[q] >> colbits], 1);
  }
  __syncthreads();
  {  // exclusive scan of s_cnt (kMaxLocalRows == blockDim)
    const int a0 = s_cnt[threadIdx.x];
    const int ex = block_exclusive_scan(a0, warp_tot, &total);
    s_off[threadIdx.x] = s_cur[threadIdx.x] = ex;
  }
  __syncthreads();
  for (int k0 = threadIdx.x; k0 < E; k0 += kLoadBatch * blockDim.x) {
    uint32_t x[kLoadBatch];
#pragma unroll
    for (int q = 0; q < kLoadBatch; ++q) {
      const int k = k0 + q * blockDim.x;
      x[q] = k < E ? ent[k] : 0u;
    }
#pragma unroll
    for (int q = 0; q < kLoadBatch; ++q)
      if (k0 + q * (int)blockDim.x < E) place[atomicAdd(&s_cur[x[q] >> colbits], 1)] = (int32_t)(x[q] & cmask);
  }
  __syncthreads();
  // sort + distinct in place; s_cur[r] := distinct count of row r. Warps take rows up to
  // kRegSortMax entries (in registers); groups of kGroupWarps warps then take the longer
  // rows up to kGroupSortMax entries of a bucket placed in shared memory, one row per group
  // at a time; the whole CTA takes what is left, one row at a time, in shared memory (a
  // bucket placed in global memory lends its unused shared buffer for that).
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int gmax = fits ? kGroupSortMax : kRegSortMax;  // longest row the groups take
  int local_max = 0;
  for (int r = warp; r < R; r += nwarps) {
    const int n = s_cnt[r];
    if (n > kRegSortMax) {  // below
      if (lane == 0 && n <= gmax) {
        const int k = atomicAdd(&s_nlong, 1);
        if (k < kMaxLongRows) s_long[k] = r;
      }
      continue;
    }
    const int uq = n > 0 ? warp_sort_unique_any(place + s_off[r], n, place + s_off[r]) : 0;
    if (lane == 0) s_cur[r] = uq;
    local_max = max(local_max, uq);
  }
  if (lane == 0 && local_max > 0) atomicMax(&s_max, local_max);
  __syncthreads();
  {
    const int nlong = min(s_nlong, kMaxLongRows);
    const int gid = warp / kGroupWarps, gtid = threadIdx.x - gid * kGroupWarps * 32;
    const int ngroups = nwarps / kGroupWarps;
    for (int k = gid; k < nlong; k += ngroups) {
      const int r = s_long[k];
      int32_t* a = place + s_off[r];
      group_bitonic(a, s_cnt[r], gtid, gid);
      if (gtid < 32) {
        const int uq = warp_unique_sorted(a, s_cnt[r], a);
        if (lane == 0) {
          s_cur[r] = uq;
          atomicMax(&s_max, uq);
        }
      }
      group_sync(gid);
    }
  }
  __syncthreads();
  for (int r = 0; r < R; ++r) {
    const int n = s_cnt[r];
    if (n <= kRegSortMax) continue;
    if (n <= gmax) {  // done by a group, unless the list was full
      bool listed = false;
      for (int k = 0; k < min(s_nlong, kMaxLongRows) && !listed; ++k) listed = s_long[k] == r;
      if (listed) continue;
    }
    int32_t* a = place + s_off[r];
    int uq;
    if (!fits && n <= kBucketCap) {  // global placement: sort a copy in shared memory
      for (int k = threadIdx.x; k < n; k += blockDim.x) s_col[k] = a[k];
      __syncthreads();
      uq = block_sort_unique(s_col, n, a, warp_tot, &total, &carry_last);
    } else {
      uq = block_sort_unique(a, n, a, warp_tot, &total, &carry_last);
    }
    if (threadIdx.x == 0) {
      s_cur[r] = uq;
      s_max = max(s_max, uq);
    }
    __syncthreads();
  }
  {  // exclusive scan of the distinct counts -> s_cnt (row starts in the bucket's output)
    const int a0 = threadIdx.x < R ? s_cur[threadIdx.x] : 0;
    const int ex = block_exclusive_scan(a0, warp_tot, &total);
    s_cnt[threadIdx.x] = ex;
    if (threadIdx.x < R) {
      const int64_t u = b + (int64_t)threadIdx.x * NB;
      ucnt[u] = a0;
      toff[u] = (int)(e0 + ex);
    }
  }
  __syncthreads();
  int32_t* dense = (int32_t*)ent;
  for (int r = warp; r < R; r += nwarps) {
    const int n = s_cur[r];
    for (int k = lane; k < n; k += 32) dense[s_cnt[r] + k] = place[s_off[r] + k];
  }
  if (threadIdx.x == 0 && s_max > 0) atomicMax(max_deg, s_max);
}

// Eight lanes per row: col[row_ptr[i] ..] = src[toff[i] ..], row_ptr[i+1] - row_ptr[i] values;
// each lane issues up to four loads before storing.
__global__ void k_rows_out(const int* __restrict__ toff, const int32_t* __restrict__ srcv,
                           const int* __restrict__ row_ptr, int32_t N, int32_t* __restrict__ col) {
  const int sub = threadIdx.x & 7;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3; i < N;
       i += ((int64_t)gridDim.x * blockDim.x) >> 3) {
    const int d = row_ptr[i];
    const int n = row_ptr[i + 1] - d;
    const int s = toff[i];
    for (int t0 = sub; t0 < n; t0 += 32) {
      int32_t v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = t0 + 8 * q < n ? srcv[s + t0 + 8 * q] : 0;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (t0 + 8 * q < n) col[d + t0 + 8 * q] = v[q];
    }
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

namespace {

// Partitioned build (steps 1-6 of the partitioned pipeline above).
igp_status build_csr_part(const int32_t* src, const int32_t* dst, int64_t M, int32_t N, const PartGeom& pg,
                          cudaStream_t s, igp_graph* g) {
  const int sms = num_sms();
  const int nC = sms;  // count / scatter CTAs: one per SM
  const int NB = 1 << pg.kb;
  const int64_t per = M > 0 ? (M + nC - 1) / nC : 1;
  const int64_t n1 = (int64_t)N + 1;
  const int64_t npos = (int64_t)NB * nC + 1;
  const int64_t cap = 2 * M > 0 ? 2 * M : 1;
  const int64_t ntiles = std::max((npos + kScanTile - 1) / kScanTile, (n1 + kScanTile - 1) / kScanTile);

  // one temporary block: pos | ucnt | toff | tile tmp | scalars | ebuf | obuf (ints)
  size_t o_pos = 0;
  size_t o_ucnt = o_pos + npos;
  size_t o_toff = o_ucnt + n1;
  size_t o_tmp = o_toff + n1;
  size_t o_sc = o_tmp + ntiles;
  size_t o_bad = (o_sc + 2 + 1) & ~(size_t)1;    // 8-byte aligned (in ints)
  size_t o_ebuf = (o_bad + 2 + 3) & ~(size_t)3;  // 16-byte aligned
  size_t o_obuf = (o_ebuf + cap + 3) & ~(size_t)3;
  size_t total_ints = o_obuf + cap;
  void* tmp_raw = nullptr;
  IGP_TRY(dev_alloc(&tmp_raw, total_ints * sizeof(int), s));
  int* T = (int*)tmp_raw;
  int* pos = T + o_pos;
  int* ucnt = T + o_ucnt;
  int* toff = T + o_toff;
  int* tiles = T + o_tmp;
  int* max_deg = T + o_sc;
  unsigned long long* bad = (unsigned long long*)(T + o_bad);
  uint32_t* ebuf = (uint32_t*)(T + o_ebuf);
  int32_t* obuf = T + o_obuf;
  int32_t* row_ptr = nullptr;
  int32_t* col = nullptr;
  auto fail = [&](igp_status e) {
    dev_free(col, s);
    dev_free(row_ptr, s);
    dev_free(tmp_raw, s);
    return e;
  };
  auto cu = [](cudaError_t e, const char* what) {
    return e == cudaSuccess ? IGP_OK : cuda_status(e, what, __FILE__, __LINE__);
  };
  igp_status st = IGP_OK;
#define PSTEP(x)                       \
  do {                                 \
    st = (x);                          \
    if (st != IGP_OK) return fail(st); \
  } while (0)
  PSTEP(cu(cudaMemsetAsync(pos + npos - 1, 0, sizeof(int), s), "memset pos"));
  PSTEP(cu(cudaMemsetAsync(ucnt + N, 0, sizeof(int), s), "memset ucnt"));
  PSTEP(cu(cudaMemsetAsync(max_deg, 0, sizeof(int), s), "memset max_deg"));
  PSTEP(cu(cudaMemsetAsync(bad, 0xFF, sizeof(unsigned long long), s), "memset bad"));
  const size_t ssm = (size_t)3 * kPartTile * sizeof(uint32_t) + (size_t)3 * (1 << kPartMaxBits) * sizeof(int);
  const size_t bsm = (size_t)kBucketCap * sizeof(int32_t);
  PSTEP(cu(cudaFuncSetAttribute(k_part_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm),
           "k_part_scatter smem"));
  PSTEP(cu(cudaFuncSetAttribute(k_bucket_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm),
           "k_bucket_rows smem"));
  k_part_count<<<nC, kPartThreads, 0, s>>>(src, dst, M, N, pg.kb, per, pos, bad);
  PSTEP(after_launch("k_part_count"));
  PSTEP(exclusive_scan(pos, pos, npos, tiles, s));
  k_part_scatter<<<nC, kPartThreads, ssm, s>>>(src, dst, M, N, pg.kb, pg.colbits, per, pos, ebuf);
  PSTEP(after_launch("k_part_scatter"));
  k_bucket_rows<<<NB, kBucketThreads, bsm, s>>>(ebuf, pos, nC, pg.kb, pg.colbits, N, obuf, toff, ucnt, max_deg);
  PSTEP(after_launch("k_bucket_rows"));
  {
    void* p = nullptr;
    PSTEP(dev_alloc(&p, n1 * sizeof(int32_t), s));
    row_ptr = (int32_t*)p;
  }
  PSTEP(exclusive_scan(ucnt, row_ptr, n1, tiles, s));
  // one synchronisation: the column count, the largest degree and the validation result
  int host_nnz = 0, host_max = 0;
  unsigned long long host_bad = 0;
  if (cudaMemcpyAsync(&host_nnz, row_ptr + N, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&host_max, max_deg, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&host_bad, bad, sizeof(host_bad), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail(cuda_status(cudaGetLastError(), "igp_graph_build readback", __FILE__, __LINE__));
  if (host_bad != ~0ull) {
    set_error("igp_graph_build: edge %llu has a node id outside [0, %d)", host_bad, N);
    return fail(IGP_E_INVAL);
  }
  {
    void* p = nullptr;
    PSTEP(dev_alloc(&p, (size_t)(host_nnz > 0 ? host_nnz : 1) * sizeof(int32_t), s));
    col = (int32_t*)p;
  }
  const int cblocks = (int)std::min<int64_t>((N * 8LL + 255) / 256, (int64_t)sms * 16);
  k_rows_out<<<std::max(cblocks, 1), 256, 0, s>>>(toff, (const int32_t*)ebuf, row_ptr, N, col);
  PSTEP(after_launch("k_rows_out"));
#undef PSTEP
  dev_free(tmp_raw, s);
  g->N = N;
  g->nnz = host_nnz;
  g->max_deg = host_max;
  g->row_ptr = row_ptr;
  g->col = col;
  return IGP_OK;
}

// Atomic build (steps 1-6 of the atomic pipeline above).
igp_status build_csr_atomic(const int32_t* src, const int32_t* dst, int64_t M, int32_t N, cudaStream_t s,
                            igp_graph* g) {
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

}  // namespace

igp_status build_csr(const int32_t* src, const int32_t* dst, int64_t M, int32_t N, cudaStream_t s, igp_graph* g) {
  PartGeom pg;
  if (part_geom(2 * M, N, &pg)) return build_csr_part(src, dst, M, N, pg, s, g);
  return build_csr_atomic(src, dst, M, N, s, g);
}

// Alg. 2, the merge of each step: merge an increment of edges (and new nodes up to N_new) into g.
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
