// K-agnostic clustering of FFP embeddings on the device: the leaf level of BIRCH (the clusterer
// of Alg. 1's last step and of Alg. 2's fit and assign, Sec. IV-A), without its tree.
//
// Entries are BIRCH clustering features CF = (n, LS, SS) (member count, linear sum, sum of
// squared norms; Zhang, Ramakrishnan, Livny, SIGMOD 1996), kept as exact integers of the points
// quantised to 2^-16. A fit takes the points in batches of B, in index order:
//   1. quantise: xq = rint(x 2^16), x' = xq 2^-16 (exact in fp32);
//   2. each point (k_clu_best, k_clu_join): the closest entry c* by the fp32 squared distance
//      |x' - C_c|^2 (coordinates summed in order, every difference, product and sum rounded,
//      ties to the smaller c); it joins c* if the radius of CF(c*) + x, evaluated in fp64 from
//      the integer sums (SS'/n' - sum_k (LS'_k/n')^2, coordinates in order), is within T;
//      otherwise it is a candidate;
//   3. candidates (k_clu_leaders, k_clu_targets): a candidate is a leader if no earlier candidate
//      of the batch lies within T of it (fp32 squared distance <= fp32(T^2)); the others join
//      the closest leader within T (ties to the smaller index) or start an entry of their own;
//   4. new entries are numbered on from K in index order (k_clu_number); all joins are added to
//      the sums with 64-bit integer atomics (exact, order-free; k_clu_sums) and the touched
//      entries' centroids refreshed: C_c = fp32((double) LS_c / n_c 2^-16) (k_clu_centroids).
// Every decision is taken in fixed-order IEEE arithmetic (the _rn intrinsics keep the compiler
// from contracting or reordering), so labels and entries are reproducible bit for bit.
// Candidates within a batch are resolved in parallel: leaders by an O(c^2) scan of earlier
// candidates, the rest by a scan of the leaders; the nearest-entry search is exhaustive, split
// over CTAs by entry slices and merged with 64-bit atomicMin on (distance bits, entry id).
#include <cmath>
#include <cstring>
#include <mutex>

#include "igp_internal.cuh"

namespace igp {
namespace {

constexpr float kQ = 65536.0f;                 // 2^16
constexpr double kInvQ = 1.52587890625e-05;    // 2^-16
constexpr int kCluThreads = 128;
constexpr int kCluTile = 32;                   // entries staged in shared memory at a time
constexpr unsigned long long kNoEntry = ~0ull;

// err bits
constexpr int kErrRange = 1;     // a coordinate outside [-1, 1] or not finite
constexpr int kErrCapacity = 2;  // more entries than max_entries

struct ClusterState {
  int32_t d = 0, batch = 0, max_entries = 0;
  double threshold = 0;
  int32_t K = 0;          // host copy of the entry count
  int32_t cap = 0;        // entries the device arrays hold
  int device = 0;
  long long* n = nullptr;             // [cap]
  long long* LS = nullptr;            // [cap][d]
  unsigned long long* SS = nullptr;   // [cap]
  float* C = nullptr;                 // [cap][d]
  // per-batch scratch and the device counters
  unsigned long long* best = nullptr;  // [batch] packed (distance bits, entry)
  int32_t* cand = nullptr;             // [batch] positions (in the batch) of the candidates
  int32_t* flag = nullptr;             // [batch] leader flags of the candidates
  int32_t* target = nullptr;           // [batch] candidate index each candidate joins, or -1 (own entry)
  int32_t* eid = nullptr;              // [batch] entry id of each candidate that starts one
  int32_t* lab = nullptr;              // [batch] labels of the batch
  int32_t* ctr = nullptr;              // [4]: K, number of candidates, err, spare
  int32_t* ctr_host = nullptr;         // pinned copy of ctr
};

// rint(x 2^16) for |x| <= 1, ties to even, in the fp32 adder: x 2^16 + 1.5 2^23 lies in
// [2^23, 2^24), where fp32 values are spaced 1 apart, so one fma rounds x 2^16 to an integer that
// sits in the low bits of the result (no float to int64 conversion: that runs on the FP64 unit).
constexpr float kQMagic = 12582912.0f;  // 1.5 2^23
__device__ __forceinline__ float qmagic(float x) { return __fmaf_rn(x, kQ, kQMagic); }
// x' = rint(x 2^16) 2^-16 (exact in fp32)
__device__ __forceinline__ float qpoint(float x) {
  return __fmul_rn(__fsub_rn(qmagic(x), kQMagic), 1.52587890625e-05f);
}
// xq = rint(x 2^16) as an integer
__device__ __forceinline__ long long qint(float x) {
  return (long long)(int)(__float_as_uint(qmagic(x)) - 0x4B400000u);
}

// fp32 squared distance, coordinates in order, every operation rounded on its own
template <int D>
__device__ __forceinline__ float dist2(const float (&x)[D], const float* __restrict__ c) {
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const float t = __fsub_rn(x[k], c[k]);
    s = __fadd_rn(s, __fmul_rn(t, t));
  }
  return s;
}

template <int D>
__device__ __forceinline__ bool load_point(const float* __restrict__ E, int64_t i, float (&x)[D], long long (&xq)[D]) {
  bool ok = true;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const float v = E[i * D + k];
    ok = ok && (fabsf(v) <= 1.0f);  // false for NaN too
    const float vc = fminf(fmaxf(v, -1.0f), 1.0f);
    xq[k] = qint(vc);
    x[k] = qpoint(vc);
  }
  return ok;
}

// Step 2a: the closest entry of every point of the batch, over entry slice blockIdx.y.
template <int D>
__global__ void __launch_bounds__(kCluThreads) k_clu_best(const float* __restrict__ E, int64_t b0, int m,
                                                         const float* __restrict__ C, const int32_t* __restrict__ ctr,
                                                         unsigned long long* __restrict__ best) {
  __shared__ float sc[kCluTile][D];
  const int K = ctr[0];
  if (K == 0 || ctr[2]) return;
  const int per = (K + gridDim.y - 1) / gridDim.y;
  const int s0 = blockIdx.y * per, s1 = min(K, s0 + per);
  if (s0 >= s1) return;
  const int p = blockIdx.x * kCluThreads + threadIdx.x;
  float x[D];
  long long xq[D];
  if (p < m) load_point<D>(E, b0 + p, x, xq);
  float bd = INFINITY;
  int bc = -1;
  for (int t0 = s0; t0 < s1; t0 += kCluTile) {
    const int nt = min(kCluTile, s1 - t0);
    __syncthreads();
    for (int e = threadIdx.x; e < nt * D; e += kCluThreads) sc[e / D][e % D] = C[(int64_t)(t0 + e / D) * D + e % D];
    __syncthreads();
    if (p < m) {
      int j = 0;
      for (; j + 4 <= nt; j += 4) {  // four entries' distances as independent chains, then in order
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float u0 = __fsub_rn(x[k], sc[j][k]), u1 = __fsub_rn(x[k], sc[j + 1][k]);
          const float u2 = __fsub_rn(x[k], sc[j + 2][k]), u3 = __fsub_rn(x[k], sc[j + 3][k]);
          s0 = __fadd_rn(s0, __fmul_rn(u0, u0));
          s1 = __fadd_rn(s1, __fmul_rn(u1, u1));
          s2 = __fadd_rn(s2, __fmul_rn(u2, u2));
          s3 = __fadd_rn(s3, __fmul_rn(u3, u3));
        }
        const float dd[4] = {s0, s1, s2, s3};
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (dd[q] < bd) {  // strict: the first (smallest id) minimum of the slice
            bd = dd[q];
            bc = t0 + j + q;
          }
      }
      for (; j < nt; ++j) {
        const float dd = dist2<D>(x, sc[j]);
        if (dd < bd) {
          bd = dd;
          bc = t0 + j;
        }
      }
    }
  }
  if (p < m && bc >= 0)
    atomicMin(best + p, ((unsigned long long)__float_as_uint(bd) << 32) | (unsigned)bc);
}

// Step 2b: BIRCH's radius test against the closest entry (entries as at the start of the batch);
// labels of the points that join, candidate flags (-1) of the others. The merged entry's
// radius^2 2^32 is formed in fp64 from the exact integer sums: SS' / (n + 1) minus the sum over
// coordinates, in order, of ((LS_k + xq_k) / (n + 1))^2. One warp per point: lane k takes
// coordinates k, k + 32, ..; the integer sum of squares is exact in any order, and every lane adds
// the squared means in coordinate order.
template <int D>
__global__ void k_clu_join(const float* __restrict__ E, int64_t b0, int m, const long long* __restrict__ n,
                           const long long* __restrict__ LS, const unsigned long long* __restrict__ SS,
                           const unsigned long long* __restrict__ best, double t2r, int32_t* __restrict__ lab,
                           int32_t* __restrict__ ctr) {
  constexpr int KPL = (D + 31) / 32;  // coordinates per lane
  const int p = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (p >= m || ctr[2]) return;  // warp-uniform
  const unsigned long long bst = best[p];
  int l = -1;
  if (bst != kNoEntry) {
    const int c = (int)(bst & 0xffffffffu);
    const double n1 = __ll2double_rn(n[c] + 1);
    unsigned long long ss = 0;
    double m2[KPL];
#pragma unroll
    for (int q = 0; q < KPL; ++q) {
      const int k = lane + 32 * q;
      m2[q] = 0.0;
      if (k < D) {
        const float vc = fminf(fmaxf(E[(b0 + p) * D + k], -1.0f), 1.0f);
        const long long xq = qint(vc);
        ss += (unsigned long long)(xq * xq);
        const double mk = __ddiv_rn(__ll2double_rn(LS[(int64_t)c * D + k] + xq), n1);
        m2[q] = __dmul_rn(mk, mk);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    double b = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) b = __dadd_rn(b, __shfl_sync(0xffffffffu, m2[k / 32], k % 32));
    const double r2 = __ddiv_rn(__ull2double_rn(SS[c] + ss), n1);
    if (__dsub_rn(r2, b) <= t2r) l = c;
  }
  if (lane == 0) lab[p] = l;
}

// Any coordinate outside [-1, 1] (or not finite) sets kErrRange; run over the whole input before
// a fit changes anything.
__global__ void k_clu_check(const float* __restrict__ E, int64_t total, int32_t* __restrict__ ctr) {
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    bad = bad || !(fabsf(E[i]) <= 1.0f);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(ctr + 2, kErrRange);
}

// Step 3a: positions of the candidates (lab = -1) of the batch, in index order (one CTA).
__global__ void __launch_bounds__(1024) k_clu_compact(const int32_t* __restrict__ lab, int m, int32_t* __restrict__ cand,
                                                      int32_t* __restrict__ ctr) {
  __shared__ int wsum[32];
  __shared__ int base;
  if (ctr[2]) return;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int p0 = 0; p0 < m; p0 += blockDim.x) {
    const int p = p0 + threadIdx.x;
    const bool c = p < m && lab[p] < 0;
    const unsigned bal = __ballot_sync(0xffffffffu, c);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    if (c) cand[base + before + __popc(bal & ((1u << lane) - 1u))] = p;
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
      base += t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) ctr[1] = base;
}

// Step 3b: leader flags, one warp per candidate: no earlier candidate of the batch within T.
template <int D>
__global__ void k_clu_leaders(const float* __restrict__ E, int64_t b0, const int32_t* __restrict__ cand,
                              const int32_t* __restrict__ ctr, float t2d, int32_t* __restrict__ flag) {
  const int q = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  const int c = ctr[1];
  if (q >= c || ctr[2]) return;
  float x[D];
#pragma unroll
  for (int k = 0; k < D; ++k) x[k] = qpoint(E[(b0 + cand[q]) * D + k]);
  bool close = false;
  for (int r0 = 0; r0 < q && !close; r0 += 32) {
    const int r = r0 + lane;
    bool cl = false;
    if (r < q) {
      float y[D];
#pragma unroll
      for (int k = 0; k < D; ++k) y[k] = qpoint(E[(b0 + cand[r]) * D + k]);
      cl = dist2<D>(x, y) <= t2d;
    }
    close = __any_sync(0xffffffffu, cl);
  }
  if (lane == 0) flag[q] = close ? 0 : 1;
}

// Step 3c: every other candidate joins the closest leader within T (ties to the smaller index),
// or starts its own entry (target -1). One warp per candidate.
template <int D>
__global__ void k_clu_targets(const float* __restrict__ E, int64_t b0, const int32_t* __restrict__ cand,
                              const int32_t* __restrict__ ctr, const int32_t* __restrict__ flag, float t2d,
                              int32_t* __restrict__ target) {
  const int q = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  const int c = ctr[1];
  if (q >= c || ctr[2]) return;
  if (flag[q]) {
    if (lane == 0) target[q] = q;
    return;
  }
  float x[D];
#pragma unroll
  for (int k = 0; k < D; ++k) x[k] = qpoint(E[(b0 + cand[q]) * D + k]);
  unsigned long long bst = kNoEntry;
  for (int r = lane; r < c; r += 32) {
    if (!flag[r]) continue;
    float y[D];
#pragma unroll
    for (int k = 0; k < D; ++k) y[k] = qpoint(E[(b0 + cand[r]) * D + k]);
    const float dd = dist2<D>(x, y);
    if (dd <= t2d) {
      const unsigned long long key = ((unsigned long long)__float_as_uint(dd) << 32) | (unsigned)r;
      bst = key < bst ? key : bst;
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const unsigned long long other = __shfl_xor_sync(0xffffffffu, bst, o);
    bst = other < bst ? other : bst;
  }
  if (lane == 0) target[q] = bst == kNoEntry ? -1 : (int)(bst & 0xffffffffu);
}

// Step 4a: new entries numbered on from K in index order; labels of the candidates; K updated.
// One CTA. With more entries than the capacity nothing is numbered and kErrCapacity is set.
__global__ void __launch_bounds__(1024) k_clu_number(const int32_t* __restrict__ cand,
                                                     const int32_t* __restrict__ flag,
                                                     const int32_t* __restrict__ target, int cap,
                                                     int32_t* __restrict__ eid, int32_t* __restrict__ lab,
                                                     int32_t* __restrict__ ctr) {
  __shared__ int wsum[32];
  __shared__ int base;
  if (ctr[2]) return;
  const int c = ctr[1];
  const int K0 = ctr[0];
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q0 = 0; q0 < c; q0 += blockDim.x) {
    const int q = q0 + threadIdx.x;
    const bool own = q < c && (flag[q] || target[q] < 0);
    const unsigned bal = __ballot_sync(0xffffffffu, own);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    if (own) eid[q] = K0 + base + before + __popc(bal & ((1u << lane) - 1u));
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
      base += t;
    }
    __syncthreads();
  }
  if (K0 + base > cap) {
    if (threadIdx.x == 0) atomicOr(ctr + 2, kErrCapacity);
    return;
  }
  for (int q = threadIdx.x; q < c; q += blockDim.x) {
    const int t = (flag[q] || target[q] < 0) ? q : target[q];
    lab[cand[q]] = eid[t];
  }
  if (threadIdx.x == 0) ctr[0] = K0 + base;
}

// Step 4b: the batch's points added to their entries' sums (exact integer atomics), and the
// labels written out.
template <int D>
__global__ void k_clu_sums(const float* __restrict__ E, int64_t b0, int m, const int32_t* __restrict__ lab,
                           const int32_t* __restrict__ ctr, long long* __restrict__ n, long long* __restrict__ LS,
                           unsigned long long* __restrict__ SS, int32_t* __restrict__ labels_out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= m || ctr[2]) return;
  float x[D];
  long long xq[D];
  load_point<D>(E, b0 + p, x, xq);
  const int c = lab[p];
  unsigned long long ss = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    atomicAdd((unsigned long long*)(LS + (int64_t)c * D + k), (unsigned long long)xq[k]);
    ss += (unsigned long long)(xq[k] * xq[k]);
  }
  atomicAdd((unsigned long long*)(n + c), 1ull);
  atomicAdd(SS + c, ss);
  if (labels_out) labels_out[b0 + p] = c;
}

// Step 4c: centroids of the entries the batch touched (a thread per point and coordinate; an
// entry with several members is written several times with the same value).
template <int D>
__global__ void k_clu_centroids(int m, const int32_t* __restrict__ lab, const int32_t* __restrict__ ctr,
                                const long long* __restrict__ n, const long long* __restrict__ LS,
                                float* __restrict__ C) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)m * D || ctr[2]) return;
  const int p = (int)(t / D), k = (int)(t % D);
  const int c = lab[p];
  const double v = __dmul_rn(__ddiv_rn(__ll2double_rn(LS[(int64_t)c * D + k]), __ll2double_rn(n[c])), kInvQ);
  C[(int64_t)c * D + k] = __double2float_rn(v);
}

// predict: labels = the closest entry of every point (no radius test, entries unchanged)
__global__ void k_clu_unpack(const unsigned long long* __restrict__ best, int64_t N, int32_t* __restrict__ labels) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    labels[i] = best[i] == kNoEntry ? -1 : (int32_t)(best[i] & 0xffffffffu);
}

}  // namespace
}  // namespace igp

struct igp_clusterer {
  igp::ClusterState st;
};

namespace igp {
namespace {

struct CluOps {
  void (*best)(const float*, int64_t, int, const float*, const int32_t*, unsigned long long*, dim3, cudaStream_t);
  void (*join)(const float*, int64_t, int, const long long*, const long long*, const unsigned long long*,
               const unsigned long long*, double, int32_t*, int32_t*, cudaStream_t);
  void (*leaders)(const float*, int64_t, int, const int32_t*, const int32_t*, float, int32_t*, cudaStream_t);
  void (*targets)(const float*, int64_t, int, const int32_t*, const int32_t*, const int32_t*, float, int32_t*,
                  cudaStream_t);
  void (*sums)(const float*, int64_t, int, const int32_t*, const int32_t*, long long*, long long*,
               unsigned long long*, int32_t*, cudaStream_t);
  void (*centroids)(int, const int32_t*, const int32_t*, const long long*, const long long*, float*, cudaStream_t);
};

template <int D>
CluOps clu_ops() {
  CluOps o;
  o.best = [](const float* E, int64_t b0, int m, const float* C, const int32_t* ctr, unsigned long long* best, dim3 g,
              cudaStream_t s) { k_clu_best<D><<<g, kCluThreads, 0, s>>>(E, b0, m, C, ctr, best); };
  o.join = [](const float* E, int64_t b0, int m, const long long* n, const long long* LS,
              const unsigned long long* SS, const unsigned long long* best, double t2r, int32_t* lab, int32_t* ctr,
              cudaStream_t s) {
    k_clu_join<D><<<(int)(((int64_t)m * 32 + 255) / 256), 256, 0, s>>>(E, b0, m, n, LS, SS, best, t2r, lab, ctr);
  };
  o.leaders = [](const float* E, int64_t b0, int m, const int32_t* cand, const int32_t* ctr, float t2d, int32_t* flag,
                 cudaStream_t s) {
    k_clu_leaders<D><<<(m * 32 + 255) / 256, 256, 0, s>>>(E, b0, cand, ctr, t2d, flag);
  };
  o.targets = [](const float* E, int64_t b0, int m, const int32_t* cand, const int32_t* ctr, const int32_t* flag,
                 float t2d, int32_t* target, cudaStream_t s) {
    k_clu_targets<D><<<(m * 32 + 255) / 256, 256, 0, s>>>(E, b0, cand, ctr, flag, t2d, target);
  };
  o.sums = [](const float* E, int64_t b0, int m, const int32_t* lab, const int32_t* ctr, long long* n, long long* LS,
              unsigned long long* SS, int32_t* out, cudaStream_t s) {
    k_clu_sums<D><<<(m + kCluThreads - 1) / kCluThreads, kCluThreads, 0, s>>>(E, b0, m, lab, ctr, n, LS, SS, out);
  };
  o.centroids = [](int m, const int32_t* lab, const int32_t* ctr, const long long* n, const long long* LS, float* C,
                   cudaStream_t s) {
    k_clu_centroids<D><<<(int)(((int64_t)m * D + 255) / 256), 256, 0, s>>>(m, lab, ctr, n, LS, C);
  };
  return o;
}

bool get_clu_ops(int d, CluOps* o) {
  switch (d) {
    case 8: *o = clu_ops<8>(); return true;
    case 16: *o = clu_ops<16>(); return true;
    case 32: *o = clu_ops<32>(); return true;
    case 64: *o = clu_ops<64>(); return true;
    case 128: *o = clu_ops<128>(); return true;
    default: return false;
  }
}

// Entry slices of the nearest-entry search: enough CTAs for about two per SM.
int slices_for(int m) {
  const int pb = (m + kCluThreads - 1) / kCluThreads;
  return std::max(1, std::min(64, (8 * num_sms() + pb - 1) / pb));  // about 8 CTAs per SM
}

// Device arrays for `need` entries (the first st.K kept, the rest zero).
igp_status ensure_capacity(ClusterState& st, int need, cudaStream_t s) {
  if (need <= st.cap) return IGP_OK;
  const int cap = std::min(st.max_entries, std::max(need, 2 * st.cap));
  const size_t d = (size_t)st.d;
  void *n = nullptr, *LS = nullptr, *SS = nullptr, *C = nullptr;
  igp_status e = dev_alloc(&n, (size_t)cap * 8, s);
  if (e == IGP_OK) e = dev_alloc(&LS, (size_t)cap * d * 8, s);
  if (e == IGP_OK) e = dev_alloc(&SS, (size_t)cap * 8, s);
  if (e == IGP_OK) e = dev_alloc(&C, (size_t)cap * d * 4, s);
  if (e == IGP_OK) {
    cudaError_t r = cudaMemsetAsync(n, 0, (size_t)cap * 8, s);
    if (r == cudaSuccess) r = cudaMemsetAsync(LS, 0, (size_t)cap * d * 8, s);
    if (r == cudaSuccess) r = cudaMemsetAsync(SS, 0, (size_t)cap * 8, s);
    if (r == cudaSuccess) r = cudaMemsetAsync(C, 0, (size_t)cap * d * 4, s);
    if (r == cudaSuccess && st.K > 0) {
      r = cudaMemcpyAsync(n, st.n, (size_t)st.K * 8, cudaMemcpyDeviceToDevice, s);
      if (r == cudaSuccess) r = cudaMemcpyAsync(LS, st.LS, (size_t)st.K * d * 8, cudaMemcpyDeviceToDevice, s);
      if (r == cudaSuccess) r = cudaMemcpyAsync(SS, st.SS, (size_t)st.K * 8, cudaMemcpyDeviceToDevice, s);
      if (r == cudaSuccess) r = cudaMemcpyAsync(C, st.C, (size_t)st.K * d * 4, cudaMemcpyDeviceToDevice, s);
    }
    if (r != cudaSuccess) e = cuda_status(r, "clusterer arrays", __FILE__, __LINE__);
  }
  if (e != IGP_OK) {
    dev_free(n, s);
    dev_free(LS, s);
    dev_free(SS, s);
    dev_free(C, s);
    return e;
  }
  dev_free(st.n, s);
  dev_free(st.LS, s);
  dev_free(st.SS, s);
  dev_free(st.C, s);
  st.n = (long long*)n;
  st.LS = (long long*)LS;
  st.SS = (unsigned long long*)SS;
  st.C = (float*)C;
  st.cap = cap;
  return IGP_OK;
}

// E on the device (the caller's, or a copy in *tmp that the caller frees).
igp_status device_points(const float* E, int64_t count, cudaStream_t s, const float** dev, void** tmp) {
  *tmp = nullptr;
  if (is_device_ptr(E)) {
    *dev = E;
    return IGP_OK;
  }
  IGP_TRY(dev_alloc(tmp, (size_t)count * 4, s));
  IGP_TRY_CUDA(cudaMemcpyAsync(*tmp, E, (size_t)count * 4, cudaMemcpyHostToDevice, s));
  *dev = (const float*)*tmp;
  return IGP_OK;
}

igp_status check_device(const ClusterState& st, const char* who) {
  int dev = -1;
  IGP_TRY_CUDA(cudaGetDevice(&dev));
  if (dev != st.device) {
    set_error("%s: the current device (%d) is not the clusterer's (%d)", who, dev, st.device);
    return IGP_E_INVAL;
  }
  return IGP_OK;
}

}  // namespace
}  // namespace igp

using namespace igp;

extern "C" {

igp_status igp_clusterer_create(int32_t d, double threshold, int32_t batch, int32_t max_entries, igp_clusterer** out) {
  clear_error();
  if (!out) return IGP_E_INVAL;
  *out = nullptr;
  CluOps ops;
  if (!get_clu_ops(d, &ops) || !(threshold > 0) || !std::isfinite(threshold) || batch < 1 || batch > 4096 ||
      max_entries < 1 || max_entries > (1 << 24)) {
    set_error("igp_clusterer_create: need d in {8, 16, 32, 64, 128}, threshold > 0, 1 <= batch <= 4096, "
              "1 <= max_entries <= 2^24");
    return IGP_E_INVAL;
  }
  igp_clusterer* c = new (std::nothrow) igp_clusterer();
  if (!c) return IGP_E_NOMEM;
  ClusterState& st = c->st;
  st.d = d;
  st.threshold = threshold;
  st.batch = batch;
  st.max_entries = max_entries;
  cudaGetDevice(&st.device);
  const size_t B = (size_t)batch;
  void* p = nullptr;
  igp_status e = dev_alloc(&p, B * 8 + 5 * B * 4 + 16, 0);
  if (e == IGP_OK) {
    st.best = (unsigned long long*)p;
    st.cand = (int32_t*)(st.best + B);
    st.flag = st.cand + B;
    st.target = st.flag + B;
    st.eid = st.target + B;
    st.lab = st.eid + B;
    st.ctr = st.lab + B;
    count_alloc();
    if ((st.ctr_host = pinned_slot()) == nullptr) {
      e = cuda_status(cudaGetLastError(), "page-locked counters", __FILE__, __LINE__);
      dev_free(p, 0);
    }
  }
  if (e == IGP_OK) {
    cudaError_t r = cudaMemsetAsync(st.ctr, 0, 16, 0);
    if (r == cudaSuccess) r = cudaStreamSynchronize(0);
    if (r != cudaSuccess) e = cuda_status(r, "clusterer set-up", __FILE__, __LINE__);
  }
  if (e != IGP_OK) {
    delete c;
    return e;
  }
  *out = c;
  return IGP_OK;
}

void igp_clusterer_free(igp_clusterer* c) {
  if (!c) return;
  ClusterState& st = c->st;
  cudaStreamSynchronize(0);
  dev_free(st.n, 0);
  dev_free(st.LS, 0);
  dev_free(st.SS, 0);
  dev_free(st.C, 0);
  dev_free(st.best, 0);
  release_slot(st.ctr_host);  // after the synchronisation above
  delete c;
}

igp_status igp_clusterer_fit(igp_clusterer* c, const float* E, int32_t N, int32_t* labels, void* stream) {
  clear_error();
  if (!c || N < 0 || (N > 0 && !E)) {
    set_error("igp_clusterer_fit: need a clusterer, N >= 0 and the points");
    return IGP_E_INVAL;
  }
  ClusterState& st = c->st;
  IGP_TRY(check_device(st, "igp_clusterer_fit"));
  if (N == 0) return IGP_OK;
  cudaStream_t s = (cudaStream_t)stream;
  CluOps ops;
  get_clu_ops(st.d, &ops);
  const int64_t total = (int64_t)N * st.d;
  const float* Ed = nullptr;
  void* tmpE = nullptr;
  void* tmpL = nullptr;
  igp_status e = device_points(E, total, s, &Ed, &tmpE);
  int32_t* lab_out = labels;
  if (e == IGP_OK && labels && !is_device_ptr(labels)) {
    e = dev_alloc(&tmpL, (size_t)N * 4, s);
    lab_out = (int32_t*)tmpL;
  }
  auto done = [&](igp_status r) {
    dev_free(tmpE, s);
    dev_free(tmpL, s);
    return r;
  };
  if (e != IGP_OK) return done(e);
  // the whole input is checked before anything changes
  st.ctr_host[0] = st.K;
  st.ctr_host[1] = 0;
  st.ctr_host[2] = 0;
  st.ctr_host[3] = 0;
  if (cudaMemcpyAsync(st.ctr, st.ctr_host, 16, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return done(cuda_status(cudaGetLastError(), "cudaMemcpyAsync", __FILE__, __LINE__));
  k_clu_check<<<(int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)num_sms() * 8)), 256, 0,
                s>>>(Ed, total, st.ctr);
  if ((e = after_launch("k_clu_check")) != IGP_OK) return done(e);
  if (cudaMemcpyAsync(st.ctr_host, st.ctr, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return done(cuda_status(cudaGetLastError(), "igp_clusterer_fit", __FILE__, __LINE__));
  if (st.ctr_host[2] & kErrRange) {
    set_error("igp_clusterer_fit: a coordinate is outside [-1, 1] or not finite");
    return done(IGP_E_INVAL);
  }
  if ((e = ensure_capacity(st, (int)std::min<int64_t>(st.max_entries, (int64_t)st.K + N), s)) != IGP_OK)
    return done(e);
  const double tq = st.threshold * 65536.0;
  const double t2r = tq * tq;
  const float t2d = (float)(st.threshold * st.threshold);
  // The batches, in stream order: 8 launches each (and a memset), all of them reading the entry
  // count and the error word from device memory, so the whole sequence is fixed by N and can be
  // recorded once into a CUDA graph and launched as one; launched one by one if recording fails.
  auto enqueue = [&](cudaStream_t q) -> igp_status {
    for (int64_t b0 = 0; b0 < N; b0 += st.batch) {
      const int m = (int)std::min<int64_t>(st.batch, N - b0);
      IGP_TRY_CUDA(cudaMemsetAsync(st.best, 0xff, (size_t)m * 8, q));
      ops.best(Ed, b0, m, st.C, st.ctr, st.best, dim3((m + kCluThreads - 1) / kCluThreads, slices_for(m)), q);
      IGP_TRY(after_launch("k_clu_best"));
      ops.join(Ed, b0, m, st.n, st.LS, st.SS, st.best, t2r, st.lab, st.ctr, q);
      IGP_TRY(after_launch("k_clu_join"));
      k_clu_compact<<<1, 1024, 0, q>>>(st.lab, m, st.cand, st.ctr);
      IGP_TRY(after_launch("k_clu_compact"));
      ops.leaders(Ed, b0, m, st.cand, st.ctr, t2d, st.flag, q);
      IGP_TRY(after_launch("k_clu_leaders"));
      ops.targets(Ed, b0, m, st.cand, st.ctr, st.flag, t2d, st.target, q);
      IGP_TRY(after_launch("k_clu_targets"));
      k_clu_number<<<1, 1024, 0, q>>>(st.cand, st.flag, st.target, st.cap, st.eid, st.lab, st.ctr);
      IGP_TRY(after_launch("k_clu_number"));
      ops.sums(Ed, b0, m, st.lab, st.ctr, st.n, st.LS, st.SS, lab_out, q);
      IGP_TRY(after_launch("k_clu_sums"));
      ops.centroids(m, st.lab, st.ctr, st.n, st.LS, st.C, q);
      IGP_TRY(after_launch("k_clu_centroids"));
    }
    return IGP_OK;
  };
  bool ran = false;
  if (N > st.batch) {  // several batches: record them (on a private stream ordered after s)
    cudaStream_t cs = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventRecord(ev, s) == cudaSuccess && cudaStreamWaitEvent(cs, ev, 0) == cudaSuccess &&
              cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      const int64_t n0 = igp_launch_count();
      const igp_status rec = enqueue(cs);
      const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
      count_launches(-(igp_launch_count() - n0));  // recorded, not run: counted when the graph runs
      ok = rec == IGP_OK && ec == cudaSuccess && graph &&
           cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess && cudaGraphLaunch(exec, cs) == cudaSuccess &&
           cudaEventRecord(ev, cs) == cudaSuccess && cudaStreamWaitEvent(s, ev, 0) == cudaSuccess;
      if (ok) {
        count_launches(8 * ((N + st.batch - 1) / st.batch));
        ran = true;
      }
    }
    cudaGetLastError();
    if (exec) cudaGraphExecDestroy(exec);  // freed when the launch completes
    if (graph) cudaGraphDestroy(graph);
    if (cs) {
      cudaStreamSynchronize(cs);
      cudaStreamDestroy(cs);
    }
    if (ev) cudaEventDestroy(ev);
  }
  if (!ran && (e = enqueue(s)) != IGP_OK) return done(e);
  if (labels && labels != lab_out &&
      cudaMemcpyAsync(labels, lab_out, (size_t)N * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return done(cuda_status(cudaGetLastError(), "cudaMemcpyAsync", __FILE__, __LINE__));
  if (cudaMemcpyAsync(st.ctr_host, st.ctr, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return done(cuda_status(cudaGetLastError(), "igp_clusterer_fit", __FILE__, __LINE__));
  if (st.ctr_host[2] & kErrCapacity) {
    // the batches before the one that overflowed are fitted; K counts them
    st.K = st.ctr_host[0];
    set_error("igp_clusterer_fit: more than max_entries=%d entries; the points before the overflowing batch "
              "are fitted",
              st.max_entries);
    return done(IGP_E_NOMEM);
  }
  st.K = st.ctr_host[0];
  return done(IGP_OK);
}

igp_status igp_clusterer_predict(igp_clusterer* c, const float* E, int32_t N, int32_t* labels, void* stream) {
  clear_error();
  if (!c || N < 0 || (N > 0 && (!E || !labels))) {
    set_error("igp_clusterer_predict: need a clusterer, N >= 0, the points and the labels");
    return IGP_E_INVAL;
  }
  ClusterState& st = c->st;
  IGP_TRY(check_device(st, "igp_clusterer_predict"));
  if (st.K == 0) {
    set_error("igp_clusterer_predict: no entries yet (fit first)");
    return IGP_E_INVAL;
  }
  if (N == 0) return IGP_OK;
  cudaStream_t s = (cudaStream_t)stream;
  CluOps ops;
  get_clu_ops(st.d, &ops);
  const int64_t total = (int64_t)N * st.d;
  const float* Ed = nullptr;
  void *tmpE = nullptr, *best = nullptr, *tmpL = nullptr;
  igp_status e = device_points(E, total, s, &Ed, &tmpE);
  if (e == IGP_OK) e = dev_alloc(&best, (size_t)N * 8, s);
  int32_t* lab = labels;
  const bool host_out = !is_device_ptr(labels);
  if (e == IGP_OK && host_out) {
    e = dev_alloc(&tmpL, (size_t)N * 4, s);
    lab = (int32_t*)tmpL;
  }
  if (e == IGP_OK && cudaMemsetAsync(best, 0xff, (size_t)N * 8, s) != cudaSuccess)
    e = cuda_status(cudaGetLastError(), "cudaMemsetAsync", __FILE__, __LINE__);
  if (e == IGP_OK) {  // the device count of entries, and a clear error word
    st.ctr_host[0] = st.K;
    st.ctr_host[1] = st.ctr_host[2] = st.ctr_host[3] = 0;
    if (cudaMemcpyAsync(st.ctr, st.ctr_host, 16, cudaMemcpyHostToDevice, s) != cudaSuccess)
      e = cuda_status(cudaGetLastError(), "cudaMemcpyAsync", __FILE__, __LINE__);
  }
  if (e == IGP_OK) {
    ops.best(Ed, 0, N, st.C, st.ctr, (unsigned long long*)best, dim3((N + kCluThreads - 1) / kCluThreads,
                                                                     slices_for(N)), s);
    e = after_launch("k_clu_best");
  }
  if (e == IGP_OK) {
    k_clu_unpack<<<(int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)N + 255) / 256, (int64_t)num_sms() * 8)),
                   256, 0, s>>>((const unsigned long long*)best, N, lab);
    e = after_launch("k_clu_unpack");
  }
  if (e == IGP_OK && host_out) {
    if (cudaMemcpyAsync(labels, lab, (size_t)N * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      e = cuda_status(cudaGetLastError(), "igp_clusterer_predict", __FILE__, __LINE__);
  }
  dev_free(tmpE, s);
  dev_free(best, s);
  dev_free(tmpL, s);
  return e;
}

igp_status igp_clusterer_info(igp_clusterer* c, int32_t* K, float* centroids, int64_t* counts, void* stream) {
  clear_error();
  if (!c) return IGP_E_INVAL;
  ClusterState& st = c->st;
  if (K) *K = st.K;
  cudaStream_t s = (cudaStream_t)stream;
  if (st.K > 0 && centroids) {
    const cudaMemcpyKind k = is_device_ptr(centroids) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    IGP_TRY_CUDA(cudaMemcpyAsync(centroids, st.C, (size_t)st.K * st.d * 4, k, s));
    if (k == cudaMemcpyDeviceToHost) IGP_TRY_CUDA(cudaStreamSynchronize(s));
  }
  if (st.K > 0 && counts) {
    const cudaMemcpyKind k = is_device_ptr(counts) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    IGP_TRY_CUDA(cudaMemcpyAsync(counts, st.n, (size_t)st.K * 8, k, s));
    if (k == cudaMemcpyDeviceToHost) IGP_TRY_CUDA(cudaStreamSynchronize(s));
  }
  return IGP_OK;
}

}  // extern "C"
