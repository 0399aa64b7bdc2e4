// The feed-forward propagation (FFP) of InfraredGP, Alg. 1 up to its clustering step:
//   k_dinv        Eq. 1 degree correction D_tau and D_tau^{-1/2} (fp64, rounded to fp32)
//   k_wsum        w_i = sum_{j in N(i)} dinv_j (fp32), once per graph and tau
//   k_deg_*       rows in order of decreasing degree, once per graph
//   k_theta       Z^(0) = Theta ~ N(0, 1/d): Philox4x64-10 + Box-Muller (the random input of Alg. 1)
//   k_layer       one Eq. 4 layer: T^(l) = tanh(theta Z + alpha Ahat Z), Z = ZNorm(T^(l-1)),
//                 fused with the column statistics of T^(l) that the next ZNorm needs
//   k_layer_tma   the same layer with the neighbour rows brought in by the TMA engine
//   k_output      Z~ = sigmoid(ZNorm(T^(L))) (Eq. 4), optional row L2 normalisation
//
// Storage: row i of every N x d activation buffer holds s_i = dinv_i * t_i (t_i itself
// when dinv_i = 0, an isolated node at tau = 0). With Z = ZNorm(T) = (T - mu) inv_s,
//     sum_j dinv_j z_j = inv_s (sum_j s_j - mu w_i),
// so a layer gathers neighbour rows and only adds them: no per-neighbour degree
// factor, no per-neighbour normalisation; the self term uses t_i = s_i / dinv_i.
//
// Layer kernel (bandwidth-bound sparse gather, no tensor cores):
//   * a group of G lanes owns one row; each lane owns 16 bytes of it (8 bf16 or 4 fp32
//     values), so a neighbour row is G coalesced 16-byte loads;
//   * rows are visited in decreasing-degree order (perm) in warp tiles of 32/G rows, so
//     the groups of a warp have (nearly) the same trip count and stay converged;
//   * kChunk (16) neighbour rows per group are in flight per trip; the next trip's column
//     indices and the next tiles' rows (perm entry two tiles ahead, row bounds, self
//     row, dinv, w one tile ahead) are loaded during the current trip;
//   * when the gathered slice of T^(l-1) is larger than L2 can hold, each trip also
//     issues prefetch.global.L2 for the rows of the next trip (past the tile's last trip,
//     the next tile's first), so that the register loads find their lines in L2;
//   * column indices are loaded evict-first (streamed once); outputs stored streaming;
//     bf16 neighbour rows are added with mixed-precision adds (one instruction a value);
//   * wide rows can be split into column chunks (blockIdx.y) over a column-blocked
//     activation layout so that the gathered slice of T^(l-1) fits L2;
//   * epilogue per row: self term, tanh, store s_i, and exact integer column sums of t
//     and t^2 (fixed point 2^-30); a warp/CTA reduction gives one partial per CTA and
//     the last CTA to finish (ticket counter) adds them up and forms mean and 1/std
//     in fp64. Integer sums make the result independent of the row order.
#include <cuda.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "igp_internal.cuh"

namespace igp {
namespace {

constexpr int kLayerThreads = 256;
constexpr int kLayerWarps = kLayerThreads / 32;

// ------------------------------------------------------------------ storage traits
template <typename S>
struct Store;
template <>
struct Store<float> {
  static constexpr int VPL = 4;  // values per 16-byte chunk
};
template <>
struct Store<__nv_bfloat16> {
  static constexpr int VPL = 8;
};

__device__ __forceinline__ float bf_lo(uint32_t x) { return __uint_as_float(x << 16); }
__device__ __forceinline__ float bf_hi(uint32_t x) { return __uint_as_float(x & 0xffff0000u); }
__device__ __forceinline__ uint32_t bf_pack(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

// 16-byte chunk load (read-only path) -> VPL floats
__device__ __forceinline__ void load_chunk(const float* p, float (&v)[4]) {
  float4 x = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
__device__ __forceinline__ void load_chunk(const __nv_bfloat16* p, float (&v)[8]) {
  uint4 x = __ldg(reinterpret_cast<const uint4*>(p));
  v[0] = bf_lo(x.x); v[1] = bf_hi(x.x); v[2] = bf_lo(x.y); v[3] = bf_hi(x.y);
  v[4] = bf_lo(x.z); v[5] = bf_hi(x.z); v[6] = bf_lo(x.w); v[7] = bf_hi(x.w);
}
__device__ __forceinline__ void store_chunk(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store_chunk(__nv_bfloat16* p, const float (&v)[8]) {
  *reinterpret_cast<uint4*>(p) = make_uint4(bf_pack(v[0], v[1]), bf_pack(v[2], v[3]), bf_pack(v[4], v[5]),
                                            bf_pack(v[6], v[7]));
}

constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

// Activation layout: column blocks of dc columns, each block an N x dc row-major array
// (dc = d: plain row-major). Offset of element (i, c).
__device__ __forceinline__ int64_t blk_off(int64_t i, int c, int32_t N, int dc) {
  const int q = c / dc;
  return (int64_t)q * N * dc + i * dc + (c - q * dc);
}

// Streamed-once data (column indices): keep it out of L1 and first in line for L2 eviction,
// so it does not push the gathered rows out of L2.
__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ int ld_stream(const int* p, uint64_t pol) {
  int v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
// Rows written by a layer are read again only by the next layer: streaming stores.
__device__ __forceinline__ void store_chunk_cs(float* p, const float (&v)[4]) {
  __stcs(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
}
__device__ __forceinline__ void store_chunk_cs(__nv_bfloat16* p, const float (&v)[8]) {
  __stcs(reinterpret_cast<uint4*>(p), make_uint4(bf_pack(v[0], v[1]), bf_pack(v[2], v[3]), bf_pack(v[4], v[5]),
                                                 bf_pack(v[6], v[7])));
}

// ------------------------------------------------------------------ Eq. 1
__global__ void k_dinv(const int32_t* __restrict__ row_ptr, int32_t N, double tau, double eps,
                       float* __restrict__ dinv) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double deg = (double)(row_ptr[i + 1] - row_ptr[i]);
    double dt;
    if (tau < 0.0)
      dt = deg - fmin(fabs(tau), deg - eps);  // Eq. 1
    else
      dt = deg + tau;  // D + tau I
    // IEEE-rounded fp64 square root and division, then round to nearest fp32
    dinv[i] = dt > 0.0 ? (float)(1.0 / sqrt(dt)) : 0.0f;
  }
}

// ------------------------------------------------------------------ Theta (random input of Alg. 1)
// Philox4x64-10 (Salmon et al., SC 2011): round multipliers and Weyl key increments.
constexpr uint64_t kPhiloxM0 = 0xD2E7470EE14C6C93ull;
constexpr uint64_t kPhiloxM1 = 0xCA5A826395121157ull;
constexpr uint64_t kPhiloxW0 = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kPhiloxW1 = 0xBB67AE8584CAA73Bull;

__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
    const uint64_t hi0 = __umul64hi(kPhiloxM0, c[0]), lo0 = kPhiloxM0 * c[0];
    const uint64_t hi1 = __umul64hi(kPhiloxM1, c[2]), lo1 = kPhiloxM1 * c[2];
    const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// Eight normals for row i, column block q (columns 8q..8q+7), times x_scale.
__device__ __forceinline__ void theta8(uint64_t seed, uint64_t i, uint64_t q, float xs, float (&z)[8]) {
  uint64_t c[4] = {i, q, 0ull, 0ull};
  philox4x64_10(c, seed, 0ull);
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    // word 2p is the low half of c[p], word 2p+1 the high half
    const uint32_t wa = (uint32_t)(c[p] & 0xffffffffull);
    const uint32_t wb = (uint32_t)(c[p] >> 32);
    const float ua = (float)((wa >> 8) + 1u) * 5.9604644775390625e-08f;  // 2^-24
    const float ub = (float)((wb >> 8) + 1u) * 5.9604644775390625e-08f;
    const float r = sqrtf(-2.0f * logf(ua));
    float sn, cs;
    sincospif(2.0f * ub, &sn, &cs);
    z[2 * p] = r * cs * xs;
    z[2 * p + 1] = r * sn * xs;
  }
}

// Theta, stored as dinv_i * Theta_i when dinv is given (the layer storage convention); thread
// `tid` of `nthreads` takes work items tid, tid + nthreads, ..
template <typename S>
__device__ __forceinline__ void theta_part(uint64_t seed, int32_t N, int32_t d, int32_t dc, float xs,
                                           const float* __restrict__ dinv, S* __restrict__ out, int64_t tid,
                                           int64_t nthreads) {
  const int nq = d >> 3;
  const int64_t total = (int64_t)N * nq;
  for (int64_t t = tid; t < total; t += nthreads) {
    const int64_t i = t / nq;
    const int q = (int)(t - i * nq);
    float z[8];
    theta8(seed, (uint64_t)i, (uint64_t)q, xs, z);
    if (dinv) {
      const float di = __ldg(dinv + i);
      if (di > 0.0f) {
#pragma unroll
        for (int k = 0; k < 8; ++k) z[k] *= di;
      }
    }
    S* p = out + blk_off(i, q * 8, N, dc);
    if constexpr (sizeof(S) == 2) {
      store_chunk(p, z);
    } else {
      float a[4] = {z[0], z[1], z[2], z[3]}, b[4] = {z[4], z[5], z[6], z[7]};
      store_chunk(p, a);
      store_chunk(p + 4, b);
    }
  }
}

template <typename S>
__global__ void k_theta(uint64_t seed, int32_t N, int32_t d, int32_t dc, float xs, const float* __restrict__ dinv,
                        S* __restrict__ out) {
  theta_part<S>(seed, N, d, dc, xs, dinv, out, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                (int64_t)gridDim.x * blockDim.x);
}

// ------------------------------------------------------------------ per-graph helpers
// w_i = sum_{j in N(i)} dinv_j, fixed order: eight lanes per row, lane s adding entries
// s, s + 8, s + 16, .. (four index loads, then four gathers, in flight at a time), then an
// xor tree over the eight lanes. A warp takes four consecutive rows per tile.
// Warp `wid` of `nwarps` takes tiles wid, wid + nwarps, ..
__device__ __forceinline__ void wsum_part(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                          const float* __restrict__ dinv, int32_t N, float* __restrict__ wsum,
                                          int64_t wid, int64_t nwarps) {
  const int sub = threadIdx.x & 7, grp = (threadIdx.x & 31) >> 3;
  const int64_t ntiles = ((int64_t)N + 3) >> 2;
  for (int64_t tile = wid; tile < ntiles; tile += nwarps) {
    const int64_t i = tile * 4 + grp;
    const bool ok = i < N;
    const int b = ok ? row_ptr[i] : 0, e = ok ? row_ptr[i + 1] : 0;
    float a = 0.0f;
    for (int k0 = b + sub; k0 < e; k0 += 32) {
      int j[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) j[q] = k0 + 8 * q < e ? __ldg(col + k0 + 8 * q) : -1;
      float w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) w[q] = j[q] >= 0 ? __ldg(dinv + j[q]) : 0.0f;
#pragma unroll
      for (int q = 0; q < 4; ++q) a += w[q];
    }
#pragma unroll
    for (int o = 4; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (ok && sub == 0) wsum[i] = a;
  }
}

__global__ void k_wsum(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                       const float* __restrict__ dinv, int32_t N, float* __restrict__ wsum) {
  wsum_part(row_ptr, col, dinv, N, wsum, ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5,
            ((int64_t)gridDim.x * blockDim.x) >> 5);
}

// Theta and w in one launch: the first half of every CTA's warps draw Theta (arithmetic-bound),
// the second half sum w (bound by the latency of its gathers), so the two overlap on every SM.
template <typename S>
__global__ void __launch_bounds__(256) k_theta_wsum(uint64_t seed, int32_t N, int32_t d, int32_t dc, float xs,
                                                    const float* __restrict__ dinv, S* __restrict__ out,
                                                    const int32_t* __restrict__ row_ptr,
                                                    const int32_t* __restrict__ col, float* __restrict__ wsum) {
  const int half = blockDim.x >> 1;
  if ((int)threadIdx.x < half)
    theta_part<S>(seed, N, d, dc, xs, dinv, out, (int64_t)blockIdx.x * half + threadIdx.x, (int64_t)gridDim.x * half);
  else
    wsum_part(row_ptr, col, dinv, N, wsum, ((int64_t)blockIdx.x * half + (threadIdx.x - half)) >> 5,
              ((int64_t)gridDim.x * half) >> 5);
}

// Rows in order of decreasing degree (counting sort by key max_deg - deg: block-local
// shared-memory histograms, a scan, one global atomic per block and key, then an atomic
// scatter). The order among rows of equal degree is whatever the atomics give; nothing
// computed from it depends on that order (each row's result, and the exact integer
// column sums of the layer kernel).
constexpr int kPermRowsPerBlock = 4096;
constexpr int kPermSmemBins = 12 * 1024;  // keys handled in shared memory (48 KB)

__device__ __forceinline__ int deg_key(const int32_t* row_ptr, int64_t i, int32_t max_deg) {
  return max_deg - (row_ptr[i + 1] - row_ptr[i]);
}

__global__ void k_deg_hist(const int32_t* __restrict__ row_ptr, int32_t N, int32_t max_deg, int* __restrict__ hist) {
  extern __shared__ int sh[];
  const int nb = max_deg + 1;
  const bool local = nb <= kPermSmemBins;
  const int64_t i0 = (int64_t)blockIdx.x * kPermRowsPerBlock;
  const int64_t i1 = min((int64_t)N, i0 + kPermRowsPerBlock);
  if (local) {
    for (int k = threadIdx.x; k < nb; k += blockDim.x) sh[k] = 0;
    __syncthreads();
  }
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const int k = deg_key(row_ptr, i, max_deg);
    atomicAdd(local ? &sh[k] : &hist[k], 1);
  }
  if (local) {
    __syncthreads();
    for (int k = threadIdx.x; k < nb; k += blockDim.x)
      if (sh[k]) atomicAdd(&hist[k], sh[k]);
  }
}

__global__ void k_deg_scatter(const int32_t* __restrict__ row_ptr, int32_t N, int32_t max_deg,
                              const int* __restrict__ off, int* __restrict__ cur, int32_t* __restrict__ perm) {
  extern __shared__ int sh[];
  const int nb = max_deg + 1;
  const bool local = nb <= kPermSmemBins;
  const int64_t i0 = (int64_t)blockIdx.x * kPermRowsPerBlock;
  const int64_t i1 = min((int64_t)N, i0 + kPermRowsPerBlock);
  if (!local) {
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      const int k = deg_key(row_ptr, i, max_deg);
      perm[off[k] + atomicAdd(&cur[k], 1)] = (int32_t)i;
    }
    return;
  }
  for (int k = threadIdx.x; k < nb; k += blockDim.x) sh[k] = 0;
  __syncthreads();
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) atomicAdd(&sh[deg_key(row_ptr, i, max_deg)], 1);
  __syncthreads();
  for (int k = threadIdx.x; k < nb; k += blockDim.x) {
    const int c = sh[k];
    if (c) sh[k] = off[k] + atomicAdd(&cur[k], c);  // this block's slots for key k
  }
  __syncthreads();
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const int k = deg_key(row_ptr, i, max_deg);
    perm[atomicAdd(&sh[k], 1)] = (int32_t)i;
  }
}

// A caller-supplied Z^(0) in the storage type, copied into the row-scaled storage.
template <typename S>
__global__ void k_prescale(const S* __restrict__ x, const float* __restrict__ dinv, int32_t N, int32_t d,
                           int32_t dc, S* __restrict__ out) {
  constexpr int VPL = Store<S>::VPL;
  const int nc = d / VPL;
  const int64_t total = (int64_t)N * nc;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / nc;
    const int c = (int)(t - i * nc) * VPL;
    float v[VPL];
    load_chunk(x + i * d + c, v);
    const float di = __ldg(dinv + i);
    if (di > 0.0f) {
#pragma unroll
      for (int k = 0; k < VPL; ++k) v[k] *= di;
    }
    store_chunk(out + blk_off(i, c, N, dc), v);
  }
}

// ------------------------------------------------------------------ Eq. 4 layer
#ifndef IGP_LAYER_CHUNK
#define IGP_LAYER_CHUNK 16
#endif
constexpr int kChunk = IGP_LAYER_CHUNK;  // neighbour rows in flight per row group per trip
constexpr int kTmaChunk = 8;             // the same for the bulk-copy kernel (shared-memory stages)
// Neighbour rows per trip for G lanes per row: rows of one or two lanes (16 or 32 bytes) hold
// a trip's indices one per entry per lane, so they take half as many to stay in registers.
constexpr int layer_chunk(int G) { return G >= 4 ? kChunk : (kChunk < 8 ? kChunk : 8); }

// Build-time tuning of the register-load layer kernel (defaults are the measured best).
#ifndef IGP_LAYER_MIN_CTAS
#define IGP_LAYER_MIN_CTAS 2  // resident CTAs per SM the register budget is sized for
#endif
// L2 prefetch distance of the neighbour rows, in trips, used when a layer's gathered slice of
// T^(l-1) is larger than kL2ResidentBytes (the row loads of a trip then find their lines in L2
// instead of waiting on DRAM); smaller slices stay in L2 and are not prefetched.
#ifndef IGP_LAYER_PF
#define IGP_LAYER_PF 1
#endif
constexpr size_t kL2ResidentBytes = 96ull << 20;
constexpr int kClaimTiles = 8;  // tiles a warp claims at a time after its first

// Fetch the 128-byte line holding p into L2 (no data returned to the SM).
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}


// tanh of Eq. 4. With fp32 storage: CUDA's tanhf. With bf16 storage the result is
// rounded to 8 significant bits right after, so the hardware approximation (relative
// error below 2^-10.9, under a quarter of a bf16 rounding step) is used.
template <typename S>
__device__ __forceinline__ float tanh_for(float y);
template <>
__device__ __forceinline__ float tanh_for<float>(float y) {
  return tanhf(y);
}
template <>
__device__ __forceinline__ float tanh_for<__nv_bfloat16>(float y) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(y));
  return t;
}

template <typename S>
struct Raw;
template <>
struct Raw<float> {
  using T = float4;
  static __device__ __forceinline__ float4 load(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
  static __device__ __forceinline__ float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  static __device__ __forceinline__ void add(float (&a)[4], float4 x) {
    a[0] += x.x; a[1] += x.y; a[2] += x.z; a[3] += x.w;
  }
  static __device__ __forceinline__ void unpack(float4 x, float (&v)[4]) {
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  }
};
template <>
struct Raw<__nv_bfloat16> {
  using T = uint4;
  static __device__ __forceinline__ uint4 load(const __nv_bfloat16* p) { return __ldg(reinterpret_cast<const uint4*>(p)); }
  static __device__ __forceinline__ uint4 zero() { return make_uint4(0u, 0u, 0u, 0u); }
  // a[2k] += low bf16 of word k, a[2k+1] += high bf16, each one mixed-precision add
  // (bf16 operand, fp32 accumulator and result; the same value as converting first).
  static __device__ __forceinline__ void add2(float& lo, float& hi, uint32_t w) {
    asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\tadd.rn.f32.bf16 %0, l, %0;\n\t"
        "add.rn.f32.bf16 %1, h, %1;\n\t}"
        : "+f"(lo), "+f"(hi)
        : "r"(w));
  }
  static __device__ __forceinline__ void add(float (&a)[8], uint4 x) {
    add2(a[0], a[1], x.x);
    add2(a[2], a[3], x.y);
    add2(a[4], a[5], x.z);
    add2(a[6], a[7], x.w);
  }
  static __device__ __forceinline__ void unpack(uint4 x, float (&v)[8]) {
    v[0] = bf_lo(x.x); v[1] = bf_hi(x.x); v[2] = bf_lo(x.y); v[3] = bf_hi(x.y);
    v[4] = bf_lo(x.z); v[5] = bf_hi(x.z); v[6] = bf_lo(x.w); v[7] = bf_hi(x.w);
  }
};

// Column sums of t and t^2 are accumulated as integers, t * 2^kQBits rounded to nearest
// (|t| <= 1), so that they are exact and independent of the order rows are summed in. The
// rounding is done in the fp32 adder: t 2^22 + 1.5 2^23 lies in [2^23, 2^24], where fp32 values
// are spaced 1 apart, so one fma rounds t 2^22 to an integer (ties to even) that sits in the low
// bits of the result; subtracting the bits of 1.5 2^23 leaves it as an int32. (A float to int64
// conversion would run on the FP64 unit, which is slow on this GPU.)
constexpr int kQBits = 22;
constexpr float kQScale = 4194304.0f;     // 2^22
constexpr float kQMagic = 12582912.0f;    // 1.5 2^23
constexpr unsigned kQMagicBits = 0x4B400000u;
__device__ __forceinline__ int qfix(float t) {
  return (int)(__float_as_uint(__fmaf_rn(t, kQScale, kQMagic)) - kQMagicBits);
}

// Eq. 4 for the VPL values of one row that a lane owns, after its neighbours were added up:
//   sv  : the row's stored values s_i (= dinv_i t_i; t_i when dinv_i = 0), unpacked
//   acc : sum over neighbours j of their stored values s_j
//   mu, is : the column means and 1/std of T^(l-1) (the previous layer's ZNorm)
// gives T^(l)_i = tanh(theta z_i + alpha dinv_i (sum_j dinv_j z_j)) with z = (t - mu) is, adds t and
// t^2 to the exact column sums, and returns the values to store (dinv_i t, or t). Every layer kernel
// uses this one function, so all of them compute a row in the same way.
template <typename S, int VPL>
__device__ __forceinline__ void layer_epilogue(const float (&sv)[VPL], const float (&acc)[VPL], float di, float wi,
                                               const float* mu, const float* is, float alpha, float theta,
                                               long long (&qs)[VPL], long long (&qq)[VPL], float (&o)[VPL]) {
  const bool scaled = di > 0.0f;
  const float rdi = scaled ? __frcp_rn(di) : 1.0f;
#pragma unroll
  for (int v = 0; v < VPL; ++v) {
    const float ti = scaled ? sv[v] * rdi : sv[v];
    const float zi = (ti - mu[v]) * is[v];
    const float agg = is[v] * fmaf(-mu[v], wi, acc[v]);
    const float y = fmaf(theta, zi, alpha * di * agg);
    const float t = tanh_for<S>(y);
    qs[v] += qfix(t);
    qq[v] += qfix(__fmul_rn(t, t));
    o[v] = scaled ? di * t : t;
  }
}

// Heavy rows: in the single-graph layer, rows of at least layer_heavy_min(G) entries (they
// lead the degree order) are gathered by the whole warp, one row per tile, so that no warp is
// left with a chain of trips longer than the rest of the layer: the row's entries are cut into
// chunks of C, group g (of the warp's GPW groups) adds chunks g, g + GPW, g + 2 GPW, .. in order,
// and the groups' sums are combined by an xor tree over the group bits. (Other paths add every
// row's entries in one sequence, so they agree with it to fp32 rounding.)
constexpr int layer_heavy_min(int G) { return 32 / G > 1 ? (32 / G) * layer_chunk(G) * 4 : 1 << 30; }

// Columns are processed in chunks of D (the template width) out of d per row:
// blockIdx.y selects the chunk, whose N x D slice of T^(l-1) is one contiguous column
// block of the activation layout and can stay in L2 while the chunk is processed.
// Chunks are independent (tanh and the column statistics act per column); each has
// its own column sums, ticket and tile counter.
//
// Rows are taken in `perm` order (NULL: their own order) in warp tiles of GPW rows, one
// row per group of G lanes; with perm sorting rows by degree, the rows of a tile have
// (nearly) equal degree and the groups run their gather loops in lockstep.
template <int D, typename S, int PF>
__global__ void __launch_bounds__(kLayerThreads, IGP_LAYER_MIN_CTAS) k_layer(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col, const float* __restrict__ dinv,
    const float* __restrict__ wsum, const int32_t* __restrict__ perm, const S* __restrict__ Tin_all,
    S* __restrict__ Tout_all, const float* __restrict__ stats_in, unsigned long long* __restrict__ gsum_all,
    float* __restrict__ stats_out, unsigned* __restrict__ tickets, const int* __restrict__ heavy_count, int32_t N,
    int32_t d, float alpha, float theta, int ddof) {
  using RW = Raw<S>;
  using RT = typename RW::T;
  constexpr int VPL = Store<S>::VPL;
  constexpr int G = D / VPL;               // lanes per row
  constexpr int GPW = 32 / G;              // rows per warp tile
  constexpr int C = layer_chunk(G);        // neighbour rows per trip
  constexpr int IPL = C >= G ? C / G : 1;  // trip indices held per lane
  static_assert(G >= 1 && G <= 32 && GPW * G == 32, "unsupported width");
  static_assert(C <= G || C % G == 0, "kChunk must be at most, or a multiple of, the lanes per row");

  __shared__ float s_mu[D], s_is[D];
  __shared__ long long s_red[kLayerWarps][2 * D];
  __shared__ bool s_last;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / G, lig = lane % G;
  const int c0 = blockIdx.y * D;  // first column of this chunk
  const int64_t blk = (int64_t)blockIdx.y * N * D + lig * VPL;  // this lane's part of the column block
  const S* __restrict__ Tin = Tin_all + blk;
  S* __restrict__ Tout = Tout_all + blk;
  unsigned long long* __restrict__ gsum = gsum_all + (int64_t)blockIdx.y * 2 * D;
  unsigned* ticket = tickets + blockIdx.y;
  unsigned* claims = tickets + gridDim.y + blockIdx.y;
  for (int c = threadIdx.x; c < D; c += blockDim.x) {
    s_mu[c] = stats_in ? stats_in[c0 + c] : 0.0f;
    s_is[c] = stats_in ? stats_in[d + c0 + c] : 1.0f;
  }
  __syncthreads();
  const uint64_t pol_first = evict_first_policy();

  long long qs[VPL], qq[VPL];
#pragma unroll
  for (int v = 0; v < VPL; ++v) qs[v] = qq[v] = 0;

  // Tiles: warp w first takes tile w (in decreasing-degree order the heaviest tiles, one per
  // warp), then claims chunks of kClaimTiles tiles from a counter, one chunk ahead of use,
  // so that no warp is left with more than its share of the long rows.
  // The first H rows of the order (the heavy ones, with perm) are one tile each, gathered by
  // the whole warp; the rest go GPW to a tile. (Tile ids fit 32 bits: ntiles <= N.)
  const int H = heavy_count ? __ldg(heavy_count) : 0;
  const int ntiles = H + (int)(((int64_t)N - H + GPW - 1) / GPW);
  const int nw = gridDim.x * kLayerWarps;
  const int w0 = blockIdx.x * kLayerWarps + warp;
  auto claim = [&]() -> int {
    unsigned c = 0;
    if (lane == 0) c = atomicAdd(claims, 1u);
    const int64_t t = nw + (int64_t)__shfl_sync(0xffffffffu, c, 0) * kClaimTiles;
    return t < ntiles ? (int)t : ntiles;
  };
  int next_chunk = claim();
  auto next_tile = [&](int t) -> int {  // the tile after t in this warp's sequence
    if (t >= nw && (t - nw + 1) % kClaimTiles) return t + 1;
    const int c = next_chunk;
    if (c < ntiles) next_chunk = claim();
    return c;
  };

  // lane lig holds trip entries lig + G k (k < IPL) counted from `base`, below `end`
  auto load_idx = [&](int (&jw)[IPL], int base, int end) {
#pragma unroll
    for (int k = 0; k < IPL; ++k) {
      const int t = lig + G * k;
      jw[k] = (t < C && base + t < end) ? ld_stream(col + base + t, pol_first) : 0;
    }
  };
  auto row_at = [&](int tile) -> int {
    if (tile >= ntiles) return -1;
    if (tile < H) return __ldg(perm + tile);
    const int64_t p = H + (int64_t)(tile - H) * GPW + grp;
    if (p >= N) return -1;
    return perm ? __ldg(perm + p) : (int)p;
  };
  struct RowData {
    int b, e;
    RT self;
    float di, wi;
  };
  auto fetch_row = [&](int r, RowData& rd) {
    if (r >= 0) {
      rd.b = __ldg(row_ptr + r);
      rd.e = __ldg(row_ptr + r + 1);
      rd.self = RW::load(Tin + (int64_t)r * D);
      rd.di = __ldg(dinv + r);
      rd.wi = __ldg(wsum + r);
    } else {
      rd.b = rd.e = 0;
      rd.self = RW::zero();
      rd.di = rd.wi = 0.0f;
    }
  };

  // L2 prefetch of neighbour rows: lane lig takes the trip entries it holds indices for
  // (as load_idx) and fetches every 128-byte line of each such row into L2
  const S* __restrict__ Tblk = Tin_all + (int64_t)blockIdx.y * N * D;
  auto load_pf = [&](int (&p)[IPL], int base, int end) {
#pragma unroll
    for (int k = 0; k < IPL; ++k) {
      const int t = lig + G * k;
      p[k] = (t < C && base + t < end) ? __ldg(col + base + t) : -1;
    }
  };
  auto prefetch_rows = [&](const int (&p)[IPL]) {
    constexpr int kLines = (int)(D * sizeof(S)) > 128 ? (int)(D * sizeof(S)) / 128 : 1;
#pragma unroll
    for (int k = 0; k < IPL; ++k)
      if (p[k] >= 0) {
#pragma unroll
        for (int q = 0; q < kLines; ++q) prefetch_l2(Tblk + (int64_t)p[k] * D + q * (128 / (int)sizeof(S)));
      }
  };

  // three-stage pipeline over tiles: row id (t+2), row data (t+1), gathers (t)
  int r = row_at(w0);
  RowData cur;
  fetch_row(r, cur);
  int tn = next_tile(w0);
  int r_n = row_at(tn);
  int jw[IPL];
  load_idx(jw, cur.b + (w0 < H ? grp * C : 0), cur.e);
  for (int tile = w0; tile < ntiles;) {
    const int tnn = next_tile(tn);
    const int r_nn = row_at(tnn);
    RowData nxt;
    fetch_row(r_n, nxt);

    // A heavy tile is one row gathered by all groups (group g takes chunks g, g + GPW, .. of C
    // entries, then an xor tree adds the groups' sums); otherwise every group gathers its own
    // row, C entries a trip, in lockstep.
    const bool heavy = tile < H;  // warp-uniform
    const int cstep = heavy ? GPW * C : C;  // entries between a group's trips
    const int ntrip = heavy ? ((cur.e - cur.b + C - 1) / C + GPW - 1) / GPW : (cur.e - cur.b + C - 1) / C;
    const int mtrip = __reduce_max_sync(0xffffffffu, ntrip);
    float acc[VPL];
#pragma unroll
    for (int v = 0; v < VPL; ++v) acc[v] = 0.0f;
    for (int tr = 0; tr < mtrip; ++tr) {
      const int c = cur.b + (heavy ? grp * C : 0) + tr * cstep;
      int jn[IPL];
      load_idx(jn, c + cstep, cur.e);
      // prefetch target: trip tr + PF of this tile, or past its last trip the next tile's
      // first trip
      int pa[IPL];
      if (PF > 0) {
        if (tr + PF < mtrip)
          load_pf(pa, c + PF * cstep, cur.e);
        else
          load_pf(pa, nxt.b + (tn < H ? grp * C : 0), nxt.e);
      }
      RT x[C];
#pragma unroll
      for (int t = 0; t < C; ++t) {
        const int j = __shfl_sync(0xffffffffu, jw[t / G], t % G, G);
        x[t] = (c + t < cur.e) ? RW::load(Tin + (int64_t)j * D) : RW::zero();
      }
#pragma unroll
      for (int t = 0; t < C; ++t) RW::add(acc, x[t]);
      if (PF > 0) prefetch_rows(pa);
#pragma unroll
      for (int k = 0; k < IPL; ++k) jw[k] = jn[k];
    }
    if (heavy) {
#pragma unroll
      for (int m = G; m < 32; m <<= 1) {
#pragma unroll
        for (int v = 0; v < VPL; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], m);
      }
    }
    // first trip indices of the next tile, then this tile's epilogue (a heavy tile's by its
    // first group)
    load_idx(jw, nxt.b + (tn < H ? grp * C : 0), nxt.e);
    if (r >= 0 && (!heavy || grp == 0)) {
      float sv[VPL];
      RW::unpack(cur.self, sv);
      float o[VPL];
      layer_epilogue<S, VPL>(sv, acc, cur.di, cur.wi, s_mu + lig * VPL, s_is + lig * VPL, alpha, theta, qs, qq, o);
      store_chunk_cs(Tout + (int64_t)r * D, o);
    }
    r = r_n;
    r_n = r_nn;
    cur = nxt;
    tile = tn;
    tn = tnn;
  }

  // ---- column statistics: exact integer sums over groups, warps, CTAs
#pragma unroll
  for (int m = G; m < 32; m <<= 1) {
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
      qs[v] += __shfl_xor_sync(0xffffffffu, qs[v], m);
      qq[v] += __shfl_xor_sync(0xffffffffu, qq[v], m);
    }
  }
  if (grp == 0) {
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
      s_red[warp][lig * VPL + v] = qs[v];
      s_red[warp][D + lig * VPL + v] = qq[v];
    }
  }
  __syncthreads();
  // this CTA's sums are added to the chunk's global int64 sums (exact, in any order)
  for (int c = threadIdx.x; c < 2 * D; c += blockDim.x) {
    long long a = 0;
#pragma unroll
    for (int w = 0; w < kLayerWarps; ++w) a += s_red[w][c];
    atomicAdd(gsum + c, (unsigned long long)a);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int c = threadIdx.x; c < D; c += blockDim.x) {
    const long long sa = (long long)__ldcg(gsum + c), qa = (long long)__ldcg(gsum + D + c);
    const double n = (double)N;
    const double st = (double)sa * (1.0 / (double)(1ll << kQBits));  // sum of t
    const double sq = (double)qa * (1.0 / (double)(1ll << kQBits));  // sum of t^2
    const double mean = st / n;
    const double denom = n - (double)ddof;
    double var = denom > 0.0 ? (sq - st * mean) / denom : 0.0;
    if (!(var > 0.0)) var = 0.0;
    const double sd = sqrt(var);
    stats_out[c0 + c] = (float)mean;
    stats_out[d + c0 + c] = sd > 0.0 ? (float)(1.0 / sd) : 0.0f;
  }
  __syncthreads();  // every read of gsum precedes its reset
  for (int c = threadIdx.x; c < 2 * D; c += blockDim.x) gsum[c] = 0ull;
  if (threadIdx.x == 0) {  // ready for the next launch
    *ticket = 0u;
    *claims = 0u;
  }
}

// ------------------------------------------------------------------ Eq. 4 layer, bulk-copy gathers
// The same layer as k_layer, with the neighbour rows brought in by the TMA engine:
// every warp owns a ring of kTmaStages shared-memory stages (one trip each: 32/G rows x
// kChunk neighbours = 4 KB) completed by mbarriers. Each neighbour row is one
// cp.async.bulk copy issued by the lane that holds its column index, so no registers
// are tied up while rows are in flight and the warp keeps kTmaStages trips in flight;
// lanes then add the rows from shared memory. Waits are bounded (about a second); a
// warp that gives up sets *err, waits (bounded) for its own copies and returns.
constexpr int kTmaStages = 3;
constexpr int kTmaStageBytes = 32 * kTmaChunk * 16;  // rows per trip x row bytes, for any width
constexpr unsigned long long kWaitNs = 1000000000ull;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity` of an mbarrier; false if it did not complete in time.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  if (mbar_try_wait(mbar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    for (int k = 0; k < 64; ++k)
      if (mbar_try_wait(mbar, parity)) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
}

template <typename S>
struct RawSm;
template <>
struct RawSm<float> {
  static __device__ __forceinline__ void add(float (&a)[4], uint32_t addr) {
    float4 x;
    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(x.x), "=f"(x.y), "=f"(x.z), "=f"(x.w) : "r"(addr));
    a[0] += x.x; a[1] += x.y; a[2] += x.z; a[3] += x.w;
  }
};
template <>
struct RawSm<__nv_bfloat16> {
  static __device__ __forceinline__ void add(float (&a)[8], uint32_t addr) {
    uint4 x;
    asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(x.x), "=r"(x.y), "=r"(x.z), "=r"(x.w) : "r"(addr));
    Raw<__nv_bfloat16>::add(a, x);
  }
};

// MODE 1: one cp.async.bulk copy per neighbour row, issued by the lane holding its index.
// MODE 4: cp.async.bulk.tensor tile::gather4 through a tensor map of T^(l-1) (box one row
//         high), four neighbour rows per copy; needs a single column block.
template <int D, typename S, int MODE>
__global__ void __launch_bounds__(kLayerThreads, 2) k_layer_tma(
    const __grid_constant__ CUtensorMap tmap, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
    const float* __restrict__ dinv, const float* __restrict__ wsum, const int32_t* __restrict__ perm,
    const S* __restrict__ Tin_all,
    S* __restrict__ Tout_all, const float* __restrict__ stats_in, unsigned long long* __restrict__ gsum_all,
    float* __restrict__ stats_out, unsigned* __restrict__ tickets, int* __restrict__ err, int32_t N, int32_t d,
    float alpha, float theta, int ddof, int withhold) {
  using RW = Raw<S>;
  using RT = typename RW::T;
  constexpr int VPL = Store<S>::VPL;
  constexpr int G = D / VPL;               // lanes per row
  constexpr int GPW = 32 / G;              // rows per warp tile
  constexpr int C = kTmaChunk;             // neighbour rows per row per trip
  constexpr int IPL = C >= G ? C / G : 1;  // trip entries held per lane
  constexpr int RB = D * (int)sizeof(S);   // bytes per row
  static_assert(GPW * C * RB == kTmaStageBytes, "stage size");
  static_assert(RB % 16 == 0, "bulk copies need 16-byte rows");

  extern __shared__ __align__(128) unsigned char dyn[];
  __shared__ float s_mu[D], s_is[D];
  __shared__ long long s_red[kLayerWarps][2 * D];
  __shared__ bool s_last;
  __shared__ int s_fail;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / G, lig = lane % G;
  const int c0 = blockIdx.y * D;
  const int64_t blk = (int64_t)blockIdx.y * N * D;
  if (threadIdx.x == 0) s_fail = 0;
  const S* __restrict__ Tin = Tin_all + blk;  // row r of this column block at Tin + r * D
  S* __restrict__ Tout = Tout_all + blk + lig * VPL;
  unsigned long long* __restrict__ gsum = gsum_all + (int64_t)blockIdx.y * 2 * D;
  unsigned* ticket = tickets + blockIdx.y;
  const uint32_t ring = smem_addr(dyn) + warp * kTmaStages * kTmaStageBytes;
  const uint32_t mbar0 = smem_addr(dyn) + kLayerWarps * kTmaStages * kTmaStageBytes + warp * kTmaStages * 8;
  for (int c = threadIdx.x; c < D; c += blockDim.x) {
    s_mu[c] = stats_in ? stats_in[c0 + c] : 0.0f;
    s_is[c] = stats_in ? stats_in[d + c0 + c] : 1.0f;
  }
  if (lane == 0) {
    for (int k = 0; k < kTmaStages; ++k) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar0 + 8 * k));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const uint64_t pol_first = evict_first_policy();

  long long qs[VPL], qq[VPL];
#pragma unroll
  for (int v = 0; v < VPL; ++v) qs[v] = qq[v] = 0;

  const int64_t ntiles = ((int64_t)N + GPW - 1) / GPW;
  const int64_t nw = (int64_t)gridDim.x * kLayerWarps;
  const int64_t w0 = (int64_t)blockIdx.x * kLayerWarps + warp;

  auto load_idx = [&](int (&jw)[IPL], int base, int end) {
#pragma unroll
    for (int k = 0; k < IPL; ++k) {
      const int t = lig + G * k;
      jw[k] = (t < C && base + t < end) ? ld_stream(col + base + t, pol_first) : 0;
    }
  };
  auto row_at = [&](int64_t tile) -> int {
    const int64_t p = tile * GPW + grp;
    if (tile >= ntiles || p >= N) return -1;
    return perm ? __ldg(perm + p) : (int)p;
  };
  auto bounds = [&](int64_t tile, int& b, int& e) {
    const int r = row_at(tile);
    if (r >= 0) {
      b = __ldg(row_ptr + r);
      e = __ldg(row_ptr + r + 1);
    } else {
      b = e = 0;
    }
  };
  auto trips = [&](int b, int e) { return __reduce_max_sync(0xffffffffu, (e - b + C - 1) / C); };

  // ---- producer: walks the same tiles and trips as the consumer, up to kTmaStages ahead
  int64_t p_tile = w0;
  int p_trip = 0, p_b, p_e, p_nb, p_ne;
  bounds(p_tile, p_b, p_e);
  bounds(p_tile + nw, p_nb, p_ne);
  int p_mtrip = trips(p_b, p_e);
  int p_jw[IPL];
  load_idx(p_jw, p_b, p_e);
  uint32_t issued = 0;
  // move the producer to the next tile that has trips (or past the end)
  auto p_next_tile = [&]() {
    for (;;) {
      p_tile += nw;
      p_trip = 0;
      p_b = p_nb;
      p_e = p_ne;
      bounds(p_tile + nw, p_nb, p_ne);
      if (p_tile >= ntiles) return;
      p_mtrip = trips(p_b, p_e);
      if (p_mtrip > 0) return;
    }
  };
  if (p_mtrip == 0 && p_tile < ntiles) {
    p_next_tile();
    load_idx(p_jw, p_b, p_e);
  }
  auto issue = [&]() {
    const uint32_t stage = issued % kTmaStages;
    const uint32_t mbar = mbar0 + 8 * stage;
    const int base = p_b + p_trip * C;
    // (withhold != 0 only in the test of the bounded wait: the first trip of the first warp
    // announces its bytes but issues no copy, so that wait runs out)
    const bool skip = withhold && issued == 0 && blockIdx.x == 0 && blockIdx.y == 0 && warp == 0;
    if constexpr (MODE == 1) {
      int cnt = 0;
#pragma unroll
      for (int k = 0; k < IPL; ++k) {
        const int t = lig + G * k;
        cnt += __popc(__ballot_sync(0xffffffffu, t < C && base + t < p_e));
      }
      if (lane == 0)
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(cnt * RB) : "memory");
      __syncwarp();
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
#pragma unroll
      for (int k = 0; k < IPL; ++k) {
        const int t = lig + G * k;
        if (t < C && base + t < p_e && !skip) {
          const uint32_t dst = ring + stage * kTmaStageBytes + (grp * C + t) * RB;
          asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                       "l"(Tin + (int64_t)p_jw[k] * D), "r"(RB), "r"(mbar)
                       : "memory");
        }
      }
    } else {
      // lane q < NOPS issues gather4 #q: stage slots 4q..4q+3 = entries t0..t0+3 of group g
      constexpr int NOPS = GPW * C / 4;
      const int q = lane;
      const int g = (4 * q) / C, t0 = (4 * q) % C;
      const int gl = (g * G) & 31;  // a lane of group g
      const int gbase = __shfl_sync(0xffffffffu, base, gl);
      const int gend = __shfl_sync(0xffffffffu, p_e, gl);
      int rows[4];
      bool any = false;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int t = t0 + u;
        const int src = (g * G + (t % G)) & 31;
        int v = 0;
#pragma unroll
        for (int k = 0; k < IPL; ++k) {
          const int w = __shfl_sync(0xffffffffu, p_jw[k], src);
          if (k == t / G) v = w;
        }
        const bool valid = q < NOPS && gbase + t < gend;
        rows[u] = valid ? v : 0;  // unused slots read row 0 and are not added
        any |= valid;
      }
      const int ops = __popc(__ballot_sync(0xffffffffu, any));
      if (lane == 0)
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(ops * 4 * RB)
                     : "memory");
      __syncwarp();
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (any && !skip) {
        const uint32_t dst = ring + stage * kTmaStageBytes + 4 * q * RB;
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
            "%3, %4, %5, %6}], [%7];" ::"r"(dst),
            "l"(&tmap), "r"(0), "r"(rows[0]), "r"(rows[1]), "r"(rows[2]), "r"(rows[3]), "r"(mbar)
            : "memory");
      }
    }
    ++issued;
    if (++p_trip == p_mtrip) p_next_tile();
    if (p_tile < ntiles) load_idx(p_jw, p_b + p_trip * C, p_e);
  };
  while (p_tile < ntiles && issued < (uint32_t)kTmaStages) issue();

  // ---- consumer
  struct RowData {
    int b, e;
    RT self;
    float di, wi;
  };
  auto fetch_row = [&](int r, RowData& rd) {
    if (r >= 0) {
      rd.b = __ldg(row_ptr + r);
      rd.e = __ldg(row_ptr + r + 1);
      rd.self = RW::load(Tin + (int64_t)r * D + lig * VPL);
      rd.di = __ldg(dinv + r);
      rd.wi = __ldg(wsum + r);
    } else {
      rd.b = rd.e = 0;
      rd.self = RW::zero();
      rd.di = rd.wi = 0.0f;
    }
  };
  uint32_t consumed = 0;
  bool failed = false;
  int r = row_at(w0);
  RowData cur;
  fetch_row(r, cur);
  int r_n = row_at(w0 + nw);
  for (int64_t tile = w0; tile < ntiles; tile += nw) {
    const int r_nn = row_at(tile + 2 * nw);
    RowData nxt;
    fetch_row(r_n, nxt);
    const int mtrip = trips(cur.b, cur.e);
    float acc[VPL];
#pragma unroll
    for (int v = 0; v < VPL; ++v) acc[v] = 0.0f;
    for (int tr = 0; tr < mtrip; ++tr) {
      const uint32_t stage = consumed % kTmaStages;
      const uint32_t parity = (consumed / kTmaStages) & 1u;
      if (!__all_sync(0xffffffffu, mbar_wait(mbar0 + 8 * stage, parity))) {  // warp-uniform
        failed = true;
        break;
      }
      const int c = cur.b + tr * C;
      const uint32_t src = ring + stage * kTmaStageBytes + grp * C * RB + lig * 16;
#pragma unroll
      for (int t = 0; t < C; ++t)
        if (c + t < cur.e) RawSm<S>::add(acc, src + t * RB);
      __syncwarp();
      ++consumed;
      if (p_tile < ntiles) issue();
    }
    if (__any_sync(0xffffffffu, failed)) {
      failed = true;
      break;
    }
    if (r >= 0) {
      float sv[VPL];
      RW::unpack(cur.self, sv);
      float o[VPL];
      layer_epilogue<S, VPL>(sv, acc, cur.di, cur.wi, s_mu + lig * VPL, s_is + lig * VPL, alpha, theta, qs, qq, o);
      store_chunk_cs(Tout + (int64_t)r * D, o);
    }
    r = r_n;
    r_n = r_nn;
    cur = nxt;
  }
  if (failed) {
    // record, and wait (bounded) for this warp's copies still in flight; the CTA then
    // skips its ticket, so this layer's statistics are not formed
    if (lane == 0) {
      atomicOr(err, 1);
      s_fail = 1;
    }
    while (consumed < issued) {
      const uint32_t stage = consumed % kTmaStages;
      (void)mbar_wait(mbar0 + 8 * stage, (consumed / kTmaStages) & 1u);
      ++consumed;
    }
  }

  // ---- column statistics: exact integer sums over groups, warps, CTAs
#pragma unroll
  for (int m = G; m < 32; m <<= 1) {
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
      qs[v] += __shfl_xor_sync(0xffffffffu, qs[v], m);
      qq[v] += __shfl_xor_sync(0xffffffffu, qq[v], m);
    }
  }
  if (grp == 0) {
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
      s_red[warp][lig * VPL + v] = qs[v];
      s_red[warp][D + lig * VPL + v] = qq[v];
    }
  }
  __syncthreads();
  if (s_fail) return;  // uniform over the CTA
  // this CTA's sums are added to the chunk's global int64 sums (exact, in any order)
  for (int c = threadIdx.x; c < 2 * D; c += blockDim.x) {
    long long a = 0;
#pragma unroll
    for (int w = 0; w < kLayerWarps; ++w) a += s_red[w][c];
    atomicAdd(gsum + c, (unsigned long long)a);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int c = threadIdx.x; c < D; c += blockDim.x) {
    const long long sa = (long long)__ldcg(gsum + c), qa = (long long)__ldcg(gsum + D + c);
    const double n = (double)N;
    const double st = (double)sa * (1.0 / (double)(1ll << kQBits));  // sum of t
    const double sq = (double)qa * (1.0 / (double)(1ll << kQBits));  // sum of t^2
    const double mean = st / n;
    const double denom = n - (double)ddof;
    double var = denom > 0.0 ? (sq - st * mean) / denom : 0.0;
    if (!(var > 0.0)) var = 0.0;
    const double sd = sqrt(var);
    stats_out[c0 + c] = (float)mean;
    stats_out[d + c0 + c] = sd > 0.0 ? (float)(1.0 / sd) : 0.0f;
  }
  __syncthreads();  // every read of gsum precedes its reset
  for (int c = threadIdx.x; c < 2 * D; c += blockDim.x) gsum[c] = 0ull;
  if (threadIdx.x == 0) *ticket = 0u;  // ready for the next launch
}


// ------------------------------------------------------------------ output
template <int D, typename S>
__global__ void k_output(const S* __restrict__ T, const float* __restrict__ dinv, const float* __restrict__ stats,
                         int32_t row0, int32_t N, int32_t dc, int row_l2, float* __restrict__ out) {
  constexpr int VPL = Store<S>::VPL;
  constexpr int G = D / VPL;  // lanes per row
  constexpr int RPW = 32 / G;  // rows per warp pass
  const int lane = threadIdx.x & 31;
  const int chunk = lane % G, sub = lane / G;
  const int64_t warp_id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  // rows row0 .. N-1 (Alg. 2 extracts the newest nodes' rows); out row 0 is row row0
  for (int64_t base = row0 + warp_id * RPW; base < N; base += nw * RPW) {  // warp-uniform loop
    const int64_t i = base + sub;
    const bool ok = i < N;
    float v[VPL];
    float di = 0.0f;
    if (ok) {
      load_chunk(T + blk_off(i, chunk * VPL, N, dc), v);
      di = __ldg(dinv + i);
    } else {
#pragma unroll
      for (int e = 0; e < VPL; ++e) v[e] = 0.0f;
    }
    const float rdi = di > 0.0f ? __frcp_rn(di) : 1.0f;
    float o[VPL];
    float ss = 0.0f;
#pragma unroll
    for (int e = 0; e < VPL; ++e) {
      const int c = chunk * VPL + e;
      const float t = v[e] * rdi;
      const float z = stats ? (t - stats[c]) * stats[D + c] : t;
      o[e] = 1.0f / (1.0f + expf(-z));  // sigmoid, Eq. 4
      ss = fmaf(o[e], o[e], ss);
    }
    if (row_l2) {
#pragma unroll
      for (int m = 1; m < G; m <<= 1) ss += __shfl_xor_sync(0xffffffffu, ss, m);
      const float inv = 1.0f / sqrtf(ss);
#pragma unroll
      for (int e = 0; e < VPL; ++e) o[e] *= inv;
    }
    if (ok) {
      float* p = out + (i - row0) * D + chunk * VPL;
#pragma unroll
      for (int e = 0; e < VPL; e += 4)
        *reinterpret_cast<float4*>(p + e) = make_float4(o[e], o[e + 1], o[e + 2], o[e + 3]);
    }
  }
}

// ------------------------------------------------------------------ batches
// Many independent graphs packed block-diagonally (row and column ids shifted by the
// graph's row offset), each keeping its own Theta seed and its own column statistics:
// the FFP of each graph is exactly what it would be alone (Eq. 4 acts per graph).
// The processing order lists each graph's rows by decreasing degree, padded with -1 to
// a multiple of kBatchAlign, so a warp tile never mixes graphs.
constexpr int kBatchAlign = 32;
// Order positions per warp turn (a multiple of kBatchAlign), tried on the first embedding of a
// batch at each (d, storage); the fastest is kept.
constexpr int kBatchChunks[] = {32, 64, 128, 256};

struct PackSrc {
  const int32_t* row_ptr;  // graph's own CSR
  const int32_t* col;
  const int32_t* perm;     // graph's own degree order
  int32_t N, roff, poff;   // rows, packed row offset, packed order offset
  int32_t eoff;            // packed entry offset
};

__global__ void k_batch_pack(const PackSrc* __restrict__ src, int32_t G, int32_t* __restrict__ row_ptr,
                             int32_t* __restrict__ col, int32_t* __restrict__ row_graph, int32_t* __restrict__ perm,
                             int32_t* __restrict__ pgraph) {
  const int g = blockIdx.y;
  const PackSrc ps = src[g];
  const int64_t nnz = ps.row_ptr[ps.N];
  const int64_t P = ((int64_t)ps.N + kBatchAlign - 1) / kBatchAlign * kBatchAlign;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ps.N; i += stride) {
    row_ptr[ps.roff + i] = ps.eoff + ps.row_ptr[i];
    row_graph[ps.roff + i] = g;
  }
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += stride)
    col[ps.eoff + k] = ps.roff + ps.col[k];
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < P; k += stride) {
    perm[ps.poff + k] = k < ps.N ? ps.roff + ps.perm[k] : -1;
    if (k % kBatchAlign == 0) pgraph[(ps.poff + k) / kBatchAlign] = g;
  }
}

// Work-balanced chunks of the processing order. Warps claim chunks of consecutive warp tiles. A
// tile costs about its longest row (its row groups gather in lockstep) plus a fixed part, and each
// graph's rows come by decreasing degree, so chunks of equal length would differ in cost by orders
// of magnitude (a graph's first chunk holds its hubs). Tile t weighs w_t = (largest degree in the
// tile) + kTileWeight; with W_t the sum of the weights before tile t, a chunk is a run of tiles with
// equal floor(W_t / W), W set so that chunks hold `mean` positions on average. A chunk then costs
// at most W plus its last tile. (The sum of the weights is below nnz + 4 P < 2^31.)
constexpr int kTileWeight = 4;

__global__ void k_tile_weight(const int32_t* __restrict__ perm, const int32_t* __restrict__ row_ptr, int64_t T,
                              int gpw, int* __restrict__ w) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (int64_t)gridDim.x * blockDim.x) {
    int m = 0;
    for (int k = 0; k < gpw; ++k) {
      const int r = perm[t * gpw + k];
      if (r >= 0) m = max(m, row_ptr[r + 1] - row_ptr[r]);
    }
    w[t] = m + kTileWeight;
  }
}

// f[t] = 1 where tile t starts a chunk (ex: exclusive prefix sums of w).
__global__ void k_chunk_flags(const int* __restrict__ w, const int* __restrict__ ex, int64_t T, int gpw, int mean,
                              int* __restrict__ f) {
  const int64_t total = (int64_t)ex[T - 1] + w[T - 1];
  const int64_t want = max((int64_t)1, (T * gpw + mean - 1) / mean);  // chunks wanted
  const int64_t W = max((int64_t)1, (total + want - 1) / want);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (int64_t)gridDim.x * blockDim.x)
    f[t] = (t == 0 || ex[t] / W != ex[t - 1] / W) ? 1 : 0;
}

// start[fx[t]] = t gpw for every tile t that starts a chunk; start[K] = T gpw = P and *count = K.
__global__ void k_chunk_starts(const int* __restrict__ f, const int* __restrict__ fx, int64_t T, int gpw,
                               int32_t* __restrict__ start, int* __restrict__ count) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (int64_t)gridDim.x * blockDim.x) {
    if (f[t]) start[fx[t]] = (int32_t)(t * gpw);
    if (t == T - 1) {
      const int K = fx[t] + f[t];
      start[K] = (int32_t)(T * gpw);
      *count = K;
    }
  }
}

// Theta for packed row i: the draw of row i - goff[g] of graph g = row_graph[i] with seeds[g].
template <typename S>
__global__ void k_theta_batch(const uint64_t* __restrict__ seeds, const int32_t* __restrict__ row_graph,
                              const int32_t* __restrict__ goff, int32_t N, int32_t d, float xs,
                              const float* __restrict__ dinv, S* __restrict__ out) {
  const int nq = d >> 3;
  const int64_t total = (int64_t)N * nq;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / nq;
    const int q = (int)(t - i * nq);
    const int g = row_graph[i];
    float z[8];
    theta8(seeds[g], (uint64_t)(i - goff[g]), (uint64_t)q, xs, z);
    const float di = __ldg(dinv + i);
    if (di > 0.0f) {
#pragma unroll
      for (int k = 0; k < 8; ++k) z[k] *= di;
    }
    S* p = out + i * d + q * 8;
    if constexpr (sizeof(S) == 2) {
      store_chunk(p, z);
    } else {
      float a4[4] = {z[0], z[1], z[2], z[3]}, b4[4] = {z[4], z[5], z[6], z[7]};
      store_chunk(p, a4);
      store_chunk(p + 4, b4);
    }
  }
}

// One Eq. 4 layer over a batch: the gather/epilogue of k_layer. The processing order is
// cut into chunks of `chunk` positions that warps claim in order from a global
// counter, so at any time the GPU works on a narrow window of the order, i.e. on a few
// graphs, whose rows (the only ones their neighbours can be) stay in L2; claiming also
// balances the load. (Which warp takes which rows changes nothing in the result.) The column statistics are kept per graph
// (exact int64 sums, added atomically to gsum[g] when a warp leaves a graph) and finished
// by k_batch_stats.
template <int D, typename S>
__global__ void __launch_bounds__(kLayerThreads, IGP_LAYER_MIN_CTAS) k_layer_batch(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col, const float* __restrict__ dinv,
    const float* __restrict__ wsum, const int32_t* __restrict__ perm, const int32_t* __restrict__ pgraph, int64_t P,
    const S* __restrict__ Tin, S* __restrict__ Tout_all, const float* __restrict__ stats_in,
    unsigned long long* __restrict__ gsum, unsigned* __restrict__ chunk_ctr, float alpha, float theta,
    const int32_t* __restrict__ cst, const int* __restrict__ nchunk) {
  using RW = Raw<S>;
  using RT = typename RW::T;
  constexpr int VPL = Store<S>::VPL;
  constexpr int G = D / VPL;
  constexpr int GPW = 32 / G;
  constexpr int C = layer_chunk(G);
  constexpr int IPL = C >= G ? C / G : 1;
  static_assert(kBatchAlign % GPW == 0, "tiles must not straddle graphs");

  __shared__ float s_mu[kLayerWarps][D], s_is[kLayerWarps][D];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / G, lig = lane % G;
  S* __restrict__ Tout = Tout_all + lig * VPL;
  const uint64_t pol_first = evict_first_policy();
  // chunks claimed by this warp, one claim ahead of use; chunk k holds the positions
  // [cst[k], cst[k+1]) (work-balanced, see k_tile_weight), k = K stands for the end (cst[K] = P)
  const int K = __ldg(nchunk);
  auto claim = [&]() -> int {
    unsigned c = 0;
    if (lane == 0) c = atomicAdd(chunk_ctr, 1u);
    return (int)min(__shfl_sync(0xffffffffu, c, 0), (unsigned)K);
  };
  int kn = claim();
  const int64_t p0 = __ldg(cst + kn);
  int64_t fe = __ldg(cst + kn + (kn < K ? 1 : 0));  // end of the chunk of the newest position
  kn = claim();
  // the position after q (the newest one): the next of its chunk, else the start of the chunk
  // claimed ahead (claims only grow, so once the end is returned it is returned again)
  auto next_pos = [&](int64_t q) -> int64_t {
    q += GPW;
    if (q < fe) return q;
    const int k = kn;
    kn = claim();
    fe = __ldg(cst + k + (k < K ? 1 : 0));
    return __ldg(cst + k);
  };

  long long qs[VPL], qq[VPL];
#pragma unroll
  for (int v = 0; v < VPL; ++v) qs[v] = qq[v] = 0;
  int cur_g = -1;
  auto flush = [&]() {  // add this warp's sums for graph cur_g to gsum[cur_g]
#pragma unroll
    for (int m = G; m < 32; m <<= 1) {
#pragma unroll
      for (int v = 0; v < VPL; ++v) {
        qs[v] += __shfl_xor_sync(0xffffffffu, qs[v], m);
        qq[v] += __shfl_xor_sync(0xffffffffu, qq[v], m);
      }
    }
    if (grp == 0 && cur_g >= 0) {
      unsigned long long* gs = gsum + (int64_t)cur_g * 2 * D;
#pragma unroll
      for (int v = 0; v < VPL; ++v) {
        atomicAdd(gs + lig * VPL + v, (unsigned long long)qs[v]);
        atomicAdd(gs + D + lig * VPL + v, (unsigned long long)qq[v]);
      }
    }
#pragma unroll
    for (int v = 0; v < VPL; ++v) qs[v] = qq[v] = 0;
  };
  auto load_idx = [&](int (&jw)[IPL], int base, int end) {
#pragma unroll
    for (int k = 0; k < IPL; ++k) {
      const int t = lig + G * k;
      jw[k] = (t < C && base + t < end) ? ld_stream(col + base + t, pol_first) : 0;
    }
  };
  struct RowData {
    int b, e;
    RT self;
    float di, wi;
  };
  auto row_at = [&](int64_t p) -> int { return p < P ? __ldg(perm + p + grp) : -1; };
  auto fetch_row = [&](int r, RowData& rd) {
    if (r >= 0) {
      rd.b = __ldg(row_ptr + r);
      rd.e = __ldg(row_ptr + r + 1);
      rd.self = RW::load(Tin + (int64_t)r * D + lig * VPL);
      rd.di = __ldg(dinv + r);
      rd.wi = __ldg(wsum + r);
    } else {
      rd.b = rd.e = 0;
      rd.self = RW::zero();
      rd.di = rd.wi = 0.0f;
    }
  };
  int r = row_at(p0);
  RowData cur;
  fetch_row(r, cur);
  int64_t pn = next_pos(p0);
  int r_n = row_at(pn);
  int jw[IPL];
  load_idx(jw, cur.b, cur.e);
  for (int64_t p = p0; p < P;) {
    const int64_t pnn = next_pos(pn);  // (claims a chunk at a boundary: call once per step)
    const int g = __ldg(pgraph + p / kBatchAlign);
    if (g != cur_g) {  // warp-uniform: a tile belongs to one graph
      flush();
      cur_g = g;
      for (int c = lane; c < D; c += 32) {
        s_mu[warp][c] = stats_in ? stats_in[(int64_t)g * 2 * D + c] : 0.0f;
        s_is[warp][c] = stats_in ? stats_in[(int64_t)g * 2 * D + D + c] : 1.0f;
      }
      __syncwarp();
    }
    const int r_nn = row_at(pnn);
    RowData nxt;
    fetch_row(r_n, nxt);
    const int mtrip = __reduce_max_sync(0xffffffffu, (cur.e - cur.b + C - 1) / C);
    float acc[VPL];
#pragma unroll
    for (int v = 0; v < VPL; ++v) acc[v] = 0.0f;
    for (int tr = 0; tr < mtrip; ++tr) {
      const int c = cur.b + tr * C;
      int jn[IPL];
      load_idx(jn, c + C, cur.e);
      RT x[C];
#pragma unroll
      for (int t = 0; t < C; ++t) {
        const int j = __shfl_sync(0xffffffffu, jw[t / G], t % G, G);
        x[t] = (c + t < cur.e) ? RW::load(Tin + (int64_t)j * D + lig * VPL) : RW::zero();
      }
#pragma unroll
      for (int t = 0; t < C; ++t) RW::add(acc, x[t]);
#pragma unroll
      for (int k = 0; k < IPL; ++k) jw[k] = jn[k];
    }
    load_idx(jw, nxt.b, nxt.e);
    if (r >= 0) {
      float sv[VPL];
      RW::unpack(cur.self, sv);
      float o[VPL];
      layer_epilogue<S, VPL>(sv, acc, cur.di, cur.wi, s_mu[warp] + lig * VPL, s_is[warp] + lig * VPL, alpha, theta, qs, qq, o);
      store_chunk_cs(Tout + (int64_t)r * D, o);
    }
    r = r_n;
    r_n = r_nn;
    cur = nxt;
    p = pn;
    pn = pnn;
  }
  flush();
}

// ------------------------------------------------------------------ batches, one persistent launch
// All L layers of a batch in one cooperative launch (every CTA resident). Warps claim chunks of a
// queue of (layer, chunk of the order) pairs, layer-major; a tile of graph g at layer l needs g's
// layer l-1 complete, which the warp that completes it announces: every warp adds its column sums
// and its row count for (g, l) when it leaves (g, l); the one whose count completes g's rows forms
// g's mean and 1/std, clears the sums and the count, and publishes ready[g] = l. So a graph moves
// to its next layer as soon as its own rows are done, without a barrier over the batch. Every wait
// ends: a warp waits only for chunks earlier in the queue than the one it enters, and the earliest
// unfinished chunk is held by a resident warp (as its current chunk, or as the one it claimed
// ahead after a finished one) whose own wait, if any, is for chunks that are all finished. Each
// wait is still bounded (about a second of globaltimer), after which the warp sets *err and returns.
// Rows of T written in this launch are read through L2 only (ld.cg): L1 is not coherent with
// other SMs' stores within one launch.
template <typename S>
struct RawCg;
template <>
struct RawCg<float> {
  static __device__ __forceinline__ float4 load(const float* p) { return __ldcg(reinterpret_cast<const float4*>(p)); }
};
template <>
struct RawCg<__nv_bfloat16> {
  static __device__ __forceinline__ uint4 load(const __nv_bfloat16* p) {
    return __ldcg(reinterpret_cast<const uint4*>(p));
  }
};

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Lane 0 waits until ready[g] >= l (acquire), at most about a second; the result goes to all lanes.
// false: the wait ran out (err set) or another warp already gave up (err seen).
__device__ __forceinline__ bool wait_ready(const int* ready, int g, int l, int* err) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0 && ld_acquire(ready + g) < l) {
    const unsigned long long t0 = globaltimer_ns();
    for (;;) {
      __nanosleep(128);
      if (ld_acquire(ready + g) >= l) break;
      if (ld_acquire(err)) {
        ok = 0;
        break;
      }
      if (globaltimer_ns() - t0 > 1000000000ull) {
        atomicOr(err, 1);
        ok = 0;
        break;
      }
    }
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();  // the other lanes' later reads are ordered after lane 0's acquire
  return ok != 0;
}

template <int D, typename S>
__global__ void __launch_bounds__(kLayerThreads, IGP_LAYER_MIN_CTAS) k_ffp_batch_persistent(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col, const float* __restrict__ dinv,
    const float* __restrict__ wsum, const int32_t* __restrict__ perm, const int32_t* __restrict__ pgraph, int64_t P,
    int L, S* __restrict__ T0, S* __restrict__ T1, float* __restrict__ stats, unsigned long long* __restrict__ gsum,
    unsigned* __restrict__ rows_done, int* __restrict__ ready, const int32_t* __restrict__ goff,
    unsigned long long* __restrict__ qctr, int* __restrict__ err, int32_t G, float alpha, float theta, int ddof,
    const int32_t* __restrict__ cst, const int* __restrict__ nchunk, int withhold) {
  using RT = typename Raw<S>::T;
  constexpr int VPL = Store<S>::VPL;
  constexpr int GW = D / VPL;  // lanes per row
  constexpr int GPW = 32 / GW;
  constexpr int C = layer_chunk(GW);
  constexpr int IPL = C >= GW ? C / GW : 1;
  static_assert(kBatchAlign % GPW == 0, "tiles must not straddle graphs");

  __shared__ float s_mu[kLayerWarps][D], s_is[kLayerWarps][D];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / GW, lig = lane % GW;
  const uint64_t pol_first = evict_first_policy();
  const int K = __ldg(nchunk);  // work-balanced chunks of the order: chunk k = [cst[k], cst[k+1])
  const int64_t Q = (int64_t)L * K;
  auto claim = [&]() -> int64_t {
    unsigned long long c = 0;
    if (lane == 0) c = atomicAdd(qctr, 1ull);
    return (int64_t)__shfl_sync(0xffffffffu, c, 0);
  };

  long long qs[VPL], qq[VPL];
#pragma unroll
  for (int v = 0; v < VPL; ++v) qs[v] = qq[v] = 0;
  int cur_g = -1, cur_l = 0;
  unsigned rows = 0;  // rows of (cur_g, cur_l) this warp has finished since its last flush
  // Add this warp's sums and row count of (cur_g, cur_l); the warp that completes the graph's rows
  // forms its statistics for layer cur_l and publishes ready[cur_g] = cur_l.
  auto flush = [&]() {
#pragma unroll
    for (int m = GW; m < 32; m <<= 1) {
#pragma unroll
      for (int v = 0; v < VPL; ++v) {
        qs[v] += __shfl_xor_sync(0xffffffffu, qs[v], m);
        qq[v] += __shfl_xor_sync(0xffffffffu, qq[v], m);
      }
    }
    if (cur_g >= 0 && rows > 0) {
      unsigned long long* gs = gsum + (int64_t)cur_g * 2 * D;
      if (grp == 0) {
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
          atomicAdd(gs + lig * VPL + v, (unsigned long long)qs[v]);
          atomicAdd(gs + D + lig * VPL + v, (unsigned long long)qq[v]);
        }
      }
      __threadfence();
      __syncwarp();
      unsigned last = 0;
      if (lane == 0) {
        const unsigned n = (unsigned)(goff[cur_g + 1] - goff[cur_g]) + ((withhold && cur_g == 0) ? 1u : 0u);
        last = atomicAdd(rows_done + cur_g, rows) + rows == n;
      }
      last = __shfl_sync(0xffffffffu, last, 0);
      __syncwarp();  // every lane's reads of the sums are ordered after lane 0's count update
      if (last) {
        __threadfence();
        const double n = (double)(goff[cur_g + 1] - goff[cur_g]);
        float* so = stats + ((int64_t)(cur_l & 1) * G + cur_g) * 2 * D;
        for (int c = lane; c < D; c += 32) {
          const long long sa = (long long)__ldcg(gs + c), qa = (long long)__ldcg(gs + D + c);
          const double st = (double)sa * (1.0 / (double)(1ll << kQBits));
          const double sq = (double)qa * (1.0 / (double)(1ll << kQBits));
          const double mean = st / n;
          const double denom = n - (double)ddof;
          double var = denom > 0.0 ? (sq - st * mean) / denom : 0.0;
          if (!(var > 0.0)) var = 0.0;
          const double sd = sqrt(var);
          so[c] = (float)mean;
          so[D + c] = sd > 0.0 ? (float)(1.0 / sd) : 0.0f;
          gs[c] = 0ull;
          gs[D + c] = 0ull;
        }
        __syncwarp();
        if (lane == 0) {
          rows_done[cur_g] = 0u;
          __threadfence();
          st_release(ready + cur_g, cur_l);
        }
      }
    }
#pragma unroll
    for (int v = 0; v < VPL; ++v) qs[v] = qq[v] = 0;
    rows = 0;
  };
  auto load_idx = [&](int (&jw)[IPL], int base, int end) {
#pragma unroll
    for (int k = 0; k < IPL; ++k) {
      const int t = lig + GW * k;
      jw[k] = (t < C && base + t < end) ? ld_stream(col + base + t, pol_first) : 0;
    }
  };

  struct RowData {
    int r, b, e;
    RT self;
    float di, wi;
  };
  const S* __restrict__ Tin = T0;
  S* __restrict__ Tout = T1;
  // A queue position: layer - 1, position in the order and the end of its chunk; the claimed queue
  // index qq = (layer - 1) K + chunk is converted once per chunk (one 64-bit division), then the
  // position is advanced by adding GPW.
  struct Pos {
    int64_t l, p, e;  // l = L marks the end of the queue
  };
  auto at = [&](int64_t qq) -> Pos {
    if (qq >= Q) return Pos{(int64_t)L, 0, 0};
    const int64_t l = qq / K;
    const int k = (int)(qq - l * K);
    return Pos{l, __ldg(cst + k), __ldg(cst + k + 1)};
  };
  // row data of the tile at position x: the parts that do not change during the launch (row,
  // entry range, degree factors), which may be read at any time
  auto fetch = [&](const Pos& x, RowData& rd) {
    rd.r = __ldg(perm + x.p + grp);
    rd.b = rd.e = 0;
    rd.di = rd.wi = 0.0f;
    if (rd.r >= 0) {
      rd.b = __ldg(row_ptr + rd.r);
      rd.e = __ldg(row_ptr + rd.r + 1);
      rd.di = __ldg(dinv + rd.r);
      rd.wi = __ldg(wsum + rd.r);
    }
  };
  // the row's own value of T^(l-1) (through L2), read only once its segment's wait is over
  auto fetch_self = [&](RowData& rd) {
    rd.self = rd.r >= 0 ? RawCg<S>::load(Tin + (int64_t)rd.r * D + lig * VPL) : Raw<S>::zero();
  };
  auto graph_of = [&](const Pos& x) -> int { return __ldg(pgraph + x.p / kBatchAlign); };
  // enter the segment (layer x.l + 1, graph g): flush the last one, wait for the graph's previous
  // layer, load its statistics and pick the layer's buffers; false if a wait gave up
  auto enter = [&](const Pos& x, int g) -> bool {
    const int l = (int)x.l + 1;
    flush();
    cur_g = g;
    cur_l = l;
    if (l > 1 && !wait_ready(ready, g, l - 1, err)) return false;
    const float* si = stats + ((int64_t)((l - 1) & 1) * G + g) * 2 * D;
    for (int c = lane; c < D; c += 32) {
      s_mu[warp][c] = l > 1 ? __ldcg(si + c) : 0.0f;
      s_is[warp][c] = l > 1 ? __ldcg(si + D + c) : 1.0f;
    }
    __syncwarp();
    Tin = (l & 1) ? T0 : T1;  // layer l reads T^(l-1) and writes T^(l); T0 holds Theta
    Tout = (l & 1) ? T1 : T0;
    return true;
  };

  // Chunks are claimed one ahead of use, so that the next tile's row data and column indices are
  // read during the current tile's gathers, across chunk boundaries too. (Its own row of T is read
  // there only when it continues the current segment; otherwise after the segment's wait.) The
  // chunk held ahead delays its graphs' completion by at most one chunk, which work-balanced chunks
  // keep short against the layer of queue between a graph's chunks of two consecutive layers.
  Pos x = at(claim());
  Pos xa = at(claim());  // the chunk claimed ahead
  auto next_of = [&](const Pos& y) -> Pos {  // the position after y (claims only grow: the end stays)
    if (y.p + GPW < y.e) return Pos{y.l, y.p + GPW, y.e};
    const Pos z = xa;
    if (z.l < L) xa = at(claim());
    return z;
  };
  if (x.l >= L) {
    flush();
    return;
  }
  int gx = graph_of(x);
  if (!enter(x, gx)) return;
  RowData cur;
  fetch(x, cur);
  fetch_self(cur);
  int jw[IPL];
  load_idx(jw, cur.b, cur.e);
  while (true) {
    const Pos xn = next_of(x);
    const int gn = xn.l < L ? graph_of(xn) : -1;
    const bool same = xn.l == x.l && gn == gx;  // the next tile continues the segment
    RowData nxt;
    if (xn.l < L) fetch(xn, nxt);
    if (same) fetch_self(nxt);
    const int mtrip = __reduce_max_sync(0xffffffffu, (cur.e - cur.b + C - 1) / C);
    float acc[VPL];
#pragma unroll
    for (int v = 0; v < VPL; ++v) acc[v] = 0.0f;
    for (int tr = 0; tr < mtrip; ++tr) {
      const int c = cur.b + tr * C;
      int jn[IPL];
      load_idx(jn, c + C, cur.e);
      RT x[C];
#pragma unroll
      for (int t = 0; t < C; ++t) {
        const int j = __shfl_sync(0xffffffffu, jw[t / GW], t % GW, GW);
        x[t] = (c + t < cur.e) ? RawCg<S>::load(Tin + (int64_t)j * D + lig * VPL) : Raw<S>::zero();
      }
#pragma unroll
      for (int t = 0; t < C; ++t) Raw<S>::add(acc, x[t]);
#pragma unroll
      for (int k = 0; k < IPL; ++k) jw[k] = jn[k];
    }
    if (xn.l < L) load_idx(jw, nxt.b, nxt.e);
    const int r = cur.r;
    if (r >= 0) {
      float sv[VPL];
      Raw<S>::unpack(cur.self, sv);
      float o[VPL];
      layer_epilogue<S, VPL>(sv, acc, cur.di, cur.wi, s_mu[warp] + lig * VPL, s_is[warp] + lig * VPL, alpha, theta, qs, qq, o);
      store_chunk_cs(Tout + (int64_t)r * D + lig * VPL, o);
    }
    rows += __popc(__ballot_sync(0xffffffffu, lig == 0 && r >= 0));
    x = xn;
    gx = gn;
    if (x.l >= L) break;
    if (!same) {
      if (!enter(x, gx)) return;
      fetch_self(nxt);
    }
    cur = nxt;
  }
  flush();
}

// Per graph and column: mean and 1/std from the exact sums (then cleared for the next layer).
template <int D>
__global__ void k_batch_stats(unsigned long long* __restrict__ gsum, const int32_t* __restrict__ goff, int32_t G,
                              int ddof, float* __restrict__ stats_out, unsigned* __restrict__ chunk_ctr) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *chunk_ctr = 0u;  // for the next layer
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)G * D;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int g = (int)(t / D), c = (int)(t - (int64_t)g * D);
    unsigned long long* gs = gsum + (int64_t)g * 2 * D;
    const double n = (double)(goff[g + 1] - goff[g]);
    const double st = (double)(long long)gs[c] * (1.0 / (double)(1ll << kQBits));
    const double sq = (double)(long long)gs[D + c] * (1.0 / (double)(1ll << kQBits));
    gs[c] = 0ull;
    gs[D + c] = 0ull;
    const double mean = st / n;
    const double denom = n - (double)ddof;
    double var = denom > 0.0 ? (sq - st * mean) / denom : 0.0;
    if (!(var > 0.0)) var = 0.0;
    const double sd = sqrt(var);
    stats_out[(int64_t)g * 2 * D + c] = (float)mean;
    stats_out[(int64_t)g * 2 * D + D + c] = sd > 0.0 ? (float)(1.0 / sd) : 0.0f;
  }
}

template <int D, typename S>
__global__ void k_output_batch(const S* __restrict__ T, const float* __restrict__ dinv,
                               const float* __restrict__ stats, const int32_t* __restrict__ row_graph, int32_t N,
                               int row_l2, float* __restrict__ out) {
  constexpr int VPL = Store<S>::VPL;
  constexpr int G = D / VPL;
  constexpr int RPW = 32 / G;
  const int lane = threadIdx.x & 31;
  const int chunk = lane % G, sub = lane / G;
  const int64_t warp_id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = warp_id * RPW; base < N; base += nw * RPW) {
    const int64_t i = base + sub;
    const bool ok = i < N;
    float v[VPL];
    float di = 0.0f;
    int g = 0;
    if (ok) {
      load_chunk(T + i * D + chunk * VPL, v);
      di = __ldg(dinv + i);
      g = row_graph[i];
    } else {
#pragma unroll
      for (int e = 0; e < VPL; ++e) v[e] = 0.0f;
    }
    const float rdi = di > 0.0f ? __frcp_rn(di) : 1.0f;
    const float* st = stats ? stats + (int64_t)g * 2 * D : nullptr;
    float o[VPL];
    float ss = 0.0f;
#pragma unroll
    for (int e = 0; e < VPL; ++e) {
      const int c = chunk * VPL + e;
      const float t = v[e] * rdi;
      const float z = st ? (t - st[c]) * st[D + c] : t;
      o[e] = 1.0f / (1.0f + expf(-z));
      ss = fmaf(o[e], o[e], ss);
    }
    if (row_l2) {
#pragma unroll
      for (int m = 1; m < G; m <<= 1) ss += __shfl_xor_sync(0xffffffffu, ss, m);
      const float inv = 1.0f / sqrtf(ss);
#pragma unroll
      for (int e = 0; e < VPL; ++e) o[e] *= inv;
    }
    if (ok) {
      float* q = out + i * D + chunk * VPL;
#pragma unroll
      for (int e = 0; e < VPL; e += 4)
        *reinterpret_cast<float4*>(q + e) = make_float4(o[e], o[e + 1], o[e + 2], o[e + 3]);
    }
  }
}

// ------------------------------------------------------------------ host dispatch
template <int D, typename S>
struct LayerCfg {
  static int per_sm() {
    static std::atomic<int> v{0};  // filled once; concurrent server threads may race to fill it
    if (v == 0) {
      int b = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_layer<D, S, IGP_LAYER_PF>, kLayerThreads, 0);
      v = b > 0 ? b : 1;
    }
    return v;
  }
  static constexpr int GPW = 32 / (D / Store<S>::VPL);
  // CTAs per chunk: one full wave, or fewer for small graphs
  static int grid(int32_t N) {
    const int64_t rows_per_cta = (int64_t)kLayerWarps * GPW;
    const int64_t want = ((int64_t)N + rows_per_cta - 1) / rows_per_cta;
    const int64_t cap = (int64_t)per_sm() * num_sms();
    return (int)std::max<int64_t>(1, std::min(want, cap));
  }
};

template <int D, typename S>
igp_status layer_launch(const LayerArgs& a, cudaStream_t s) {
  dim3 gr(a.grid, a.d / D);
  if (a.prefetch)
    k_layer<D, S, IGP_LAYER_PF><<<gr, kLayerThreads, 0, s>>>(a.row_ptr, a.col, a.dinv, a.wsum, a.perm,
                                                             (const S*)a.Tin, (S*)a.Tout, a.stats_in, a.gsum,
                                                             a.stats_out, a.tickets, a.heavy_count, a.N, a.d,
                                                             a.alpha, a.theta, a.ddof);
  else
    k_layer<D, S, 0><<<gr, kLayerThreads, 0, s>>>(a.row_ptr, a.col, a.dinv, a.wsum, a.perm, (const S*)a.Tin,
                                                  (S*)a.Tout, a.stats_in, a.gsum, a.stats_out, a.tickets,
                                                  a.heavy_count, a.N, a.d, a.alpha, a.theta, a.ddof);
  return after_launch("k_layer");
}

constexpr size_t kTmaDynSmem = (size_t)kLayerWarps * kTmaStages * (kTmaStageBytes + 8);

template <int D, typename S>
struct TmaCfg {
  static int per_sm() {
    static std::atomic<int> v{0};  // filled once; concurrent server threads may race to fill it
    if (v == 0) {
      cudaFuncSetAttribute(k_layer_tma<D, S, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTmaDynSmem);
      int b = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_layer_tma<D, S, 1>, kLayerThreads, kTmaDynSmem);
      v = b > 0 ? b : 1;
    }
    return v;
  }
  static constexpr int GPW = 32 / (D / Store<S>::VPL);
  static int grid(int32_t N) {
    const int64_t rows_per_cta = (int64_t)kLayerWarps * GPW;
    const int64_t want = ((int64_t)N + rows_per_cta - 1) / rows_per_cta;
    const int64_t cap = (int64_t)per_sm() * num_sms();
    return (int)std::max<int64_t>(1, std::min(want, cap));
  }
};

// cuTensorMapEncodeTiled, looked up once from the driver (no link-time dependency).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
igp_status encode_tiled_fn(EncodeTiledFn* fn) {
  static EncodeTiledFn f = nullptr;
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  if (!f) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
      set_error("cuTensorMapEncodeTiled is not available from the driver");
      return IGP_E_UNSUPPORTED;
    }
    f = (EncodeTiledFn)p;
  }
  *fn = f;
  return IGP_OK;
}

// Tensor map of an N x D activation block (rows of D values), boxes one row high.
template <int D, typename S>
igp_status make_row_map(const void* base, int32_t N, CUtensorMap* m) {
  EncodeTiledFn fn;
  IGP_TRY(encode_tiled_fn(&fn));
  const cuuint64_t dims[2] = {(cuuint64_t)D, (cuuint64_t)N};
  const cuuint64_t strides[1] = {(cuuint64_t)D * sizeof(S)};
  const cuuint32_t box[2] = {(cuuint32_t)D, 1u};
  const cuuint32_t estr[2] = {1u, 1u};
  const CUtensorMapDataType dt = sizeof(S) == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  CUresult r = fn(m, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d) for a %d x %d map", (int)r, N, D);
    return IGP_E_CUDA;
  }
  return IGP_OK;
}

template <int D, typename S>
igp_status layer_tma_launch(const LayerArgs& a, cudaStream_t s) {
  dim3 gr(a.grid, a.d / D);
  CUtensorMap m;
  memset(&m, 0, sizeof(m));
  if (a.gather4) {
    if (a.d != D) {
      set_error("gather4 needs a single column block");
      return IGP_E_INVAL;
    }
    const igp_status ms = make_row_map<D, S>(a.Tin, a.N, &m);
    if (ms != IGP_OK) return ms;
    IGP_TRY_CUDA(
        cudaFuncSetAttribute(k_layer_tma<D, S, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTmaDynSmem));
    k_layer_tma<D, S, 4><<<gr, kLayerThreads, kTmaDynSmem, s>>>(
        m, a.row_ptr, a.col, a.dinv, a.wsum, a.perm, (const S*)a.Tin, (S*)a.Tout, a.stats_in, a.gsum, a.stats_out,
        a.tickets, a.err, a.N, a.d, a.alpha, a.theta, a.ddof, a.withhold);
  } else {
    IGP_TRY_CUDA(
        cudaFuncSetAttribute(k_layer_tma<D, S, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTmaDynSmem));
    k_layer_tma<D, S, 1><<<gr, kLayerThreads, kTmaDynSmem, s>>>(
        m, a.row_ptr, a.col, a.dinv, a.wsum, a.perm, (const S*)a.Tin, (S*)a.Tout, a.stats_in, a.gsum, a.stats_out,
        a.tickets, a.err, a.N, a.d, a.alpha, a.theta, a.ddof, a.withhold);
  }
  return after_launch("k_layer_tma");
}

template <int D, typename S>
igp_status output_launch(const void* T, const float* dinv, const float* st, int32_t row0, int32_t N, int dc,
                         int row_l2, float* out, cudaStream_t s) {
  if (row0 >= N) return IGP_OK;  // no rows to write
  constexpr int G = D / Store<S>::VPL;
  int64_t threads = (int64_t)(N - row0) * G;
  int blocks = (int)std::min<int64_t>((threads + 255) / 256, (int64_t)num_sms() * 16);
  k_output<D, S><<<std::max(blocks, 1), 256, 0, s>>>((const S*)T, dinv, st, row0, N, dc, row_l2, out);
  return after_launch("k_output");
}

template <typename S>
igp_status prescale_launch(const void* x, const float* dinv, int32_t N, int32_t d, int32_t dc, void* out,
                           cudaStream_t s) {
  int64_t total = (int64_t)N * d / Store<S>::VPL;
  int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms() * 16);
  k_prescale<S><<<std::max(blocks, 1), 256, 0, s>>>((const S*)x, dinv, N, d, dc, (S*)out);
  return after_launch("k_prescale");
}

template <int D, typename S>
struct BatchCfg {
  static int per_sm() {
    static std::atomic<int> v{0};  // filled once; concurrent server threads may race to fill it
    if (v == 0) {
      int b = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_layer_batch<D, S>, kLayerThreads, 0);
      v = b > 0 ? b : 1;
    }
    return v;
  }
};

template <int D, typename S>
igp_status batch_layer_launch(const igp_batch* b, const void* Tin, void* Tout, const float* st_in,
                              unsigned long long* gsum, float alpha, float theta, int grid, const int32_t* cst,
                              const int* nchunk, cudaStream_t s) {
  k_layer_batch<D, S><<<grid, kLayerThreads, 0, s>>>(b->row_ptr, b->col, b->dinv, b->wsum, b->perm, b->pgraph,
                                                     b->P, (const S*)Tin, (S*)Tout, st_in, gsum,
                                                     (unsigned*)(gsum + (int64_t)b->G * 2 * D), alpha, theta,
                                                     cst, nchunk);
  return after_launch("k_layer_batch");
}

// All layers of a batch in one cooperative launch (every CTA resident: the launch fails rather
// than run part of the grid). Arguments as in k_ffp_batch_persistent.
struct PersistArgs {
  void *T0, *T1;
  float* stats;
  unsigned long long* gsum;
  unsigned* rows_done;
  int* ready;
  unsigned long long* qctr;
  int* err;
  const int32_t* cst;  // chunk table of the order: starts [K + 1], and K
  const int* nchunk;
  int L, ddof, grid, withhold;
  float alpha, theta;
};

template <int D, typename S>
int persist_per_sm() {
  static int n = -1;
  if (n < 0) {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_ffp_batch_persistent<D, S>, kLayerThreads, 0);
    n = std::max(b, 1);
  }
  return n;
}

template <int D, typename S>
igp_status batch_persist_launch(const igp_batch* b, const PersistArgs& a, cudaStream_t s) {
  const int32_t* row_ptr = b->row_ptr;
  const int32_t* col = b->col;
  const float* dinv = b->dinv;
  const float* wsum = b->wsum;
  const int32_t* perm = b->perm;
  const int32_t* pgraph = b->pgraph;
  int64_t P = b->P;
  int L = a.L;
  S* T0 = (S*)a.T0;
  S* T1 = (S*)a.T1;
  float* stats = a.stats;
  unsigned long long* gsum = a.gsum;
  unsigned* rows_done = a.rows_done;
  int* ready = a.ready;
  const int32_t* goff = b->goff;
  unsigned long long* qctr = a.qctr;
  int* err = a.err;
  int32_t G = b->G;
  float alpha = a.alpha, theta = a.theta;
  int ddof = a.ddof, withhold = a.withhold;
  const int32_t* cst = a.cst;
  const int* nchunk = a.nchunk;
  void* args[] = {&row_ptr, &col, &dinv, &wsum, &perm, &pgraph, &P, &L, &T0, &T1, &stats, &gsum, &rows_done,
                  &ready, &goff, &qctr, &err, &G, &alpha, &theta, &ddof, &cst, &nchunk, &withhold};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_ffp_batch_persistent<D, S>, dim3(a.grid),
                                              dim3(kLayerThreads), args, 0, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(e, "cudaLaunchCooperativeKernel(k_ffp_batch_persistent)", __FILE__, __LINE__);
  }
  return after_launch("k_ffp_batch_persistent");
}

template <int D, typename S>
igp_status batch_tail_launch(const igp_batch* b, unsigned long long* gsum, int ddof, float* st_out, cudaStream_t s) {
  const int64_t n = (int64_t)b->G * D;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8);
  k_batch_stats<D><<<std::max(blocks, 1), 256, 0, s>>>(gsum, b->goff, b->G, ddof, st_out,
                                                        (unsigned*)(gsum + (int64_t)b->G * 2 * D));
  return after_launch("k_batch_stats");
}

template <int D, typename S>
igp_status batch_output_launch(const igp_batch* b, const void* T, const float* st, int row_l2, float* out,
                               cudaStream_t s) {
  constexpr int G = D / Store<S>::VPL;
  const int64_t threads = (int64_t)b->N * G;
  const int blocks = (int)std::min<int64_t>((threads + 255) / 256, (int64_t)num_sms() * 16);
  k_output_batch<D, S><<<std::max(blocks, 1), 256, 0, s>>>((const S*)T, b->dinv, st, b->row_graph, b->N, row_l2,
                                                            out);
  return after_launch("k_output_batch");
}

template <typename S>
igp_status batch_theta_launch(const igp_batch* b, int d, float xs, void* out, cudaStream_t s) {
  const int64_t total = (int64_t)b->N * (d / 8);
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms() * 16);
  k_theta_batch<S><<<std::max(blocks, 1), 256, 0, s>>>(b->seeds_dev, b->row_graph, b->goff, b->N, d, xs, b->dinv,
                                                        (S*)out);
  return after_launch("k_theta_batch");
}

struct BatchOps {
  int gpw;  // rows per warp tile
  int (*per_sm)();
  int (*persist_per_sm)();
  igp_status (*persist)(const igp_batch*, const PersistArgs&, cudaStream_t);
  igp_status (*layer)(const igp_batch*, const void*, void*, const float*, unsigned long long*, float, float, int,
                      const int32_t*, const int*, cudaStream_t);
  igp_status (*tail)(const igp_batch*, unsigned long long*, int, float*, cudaStream_t);
  igp_status (*output)(const igp_batch*, const void*, const float*, int, float*, cudaStream_t);
  igp_status (*theta)(const igp_batch*, int, float, void*, cudaStream_t);
};

template <int D, typename S>
BatchOps batch_ops_for() {
  return BatchOps{32 / (D / Store<S>::VPL), &BatchCfg<D, S>::per_sm, &persist_per_sm<D, S>, &batch_persist_launch<D, S>,
                  &batch_layer_launch<D, S>, &batch_tail_launch<D, S>, &batch_output_launch<D, S>,
                  &batch_theta_launch<S>};
}

bool get_batch_ops(int d, int storage, BatchOps* o) {
  const bool bf = storage == IGP_STORE_BF16;
  switch (d) {
    case 8: *o = bf ? batch_ops_for<8, __nv_bfloat16>() : batch_ops_for<8, float>(); return true;
    case 16: *o = bf ? batch_ops_for<16, __nv_bfloat16>() : batch_ops_for<16, float>(); return true;
    case 32: *o = bf ? batch_ops_for<32, __nv_bfloat16>() : batch_ops_for<32, float>(); return true;
    case 64: *o = bf ? batch_ops_for<64, __nv_bfloat16>() : batch_ops_for<64, float>(); return true;
    case 128: *o = bf ? batch_ops_for<128, __nv_bfloat16>() : batch_ops_for<128, float>(); return true;
    default: return false;
  }
}

struct Ops {
  int (*grid)(int32_t);
  igp_status (*layer)(const LayerArgs&, cudaStream_t);
  int (*tma_grid)(int32_t);
  igp_status (*layer_tma)(const LayerArgs&, cudaStream_t);
  igp_status (*output)(const void*, const float*, const float*, int32_t, int32_t, int, int, float*, cudaStream_t);
  igp_status (*prescale)(const void*, const float*, int32_t, int32_t, int32_t, void*, cudaStream_t);
};

template <int D, typename S>
Ops ops_for() {
  return Ops{&LayerCfg<D, S>::grid, &layer_launch<D, S>, &TmaCfg<D, S>::grid, &layer_tma_launch<D, S>,
             &output_launch<D, S>, &prescale_launch<S>};
}

// L2 budget for the gathered chunk of T^(l-1): chunks of at most this many bytes.
constexpr size_t kChunkBytes = 72ull << 20;

// Column chunk width for a layer: the widest of d, d/2, d/4, .. whose N x width slice
// fits the L2 budget, but never below 128 bytes per row: a gathered row segment is then
// one full L2 line per request, and splitting it further multiplies the L1->L2 request
// count (measured to cost more than the extra L2 hits gain).
int chunk_width(int32_t N, int d, size_t sb) {
  int w = d;
  while ((size_t)N * w * sb > kChunkBytes && w * sb > 128) w >>= 1;
  return w;
}

// Gather mechanism of a layer: register loads unless a TMA mode is asked for (measured:
// for 128-byte rows at 2M nodes, per-row bulk copies and gather4 copies were 1.8x and
// 1.3x slower than register loads).
bool use_tma(int gather, int dc, size_t sb) {
  if (gather == IGP_GATHER_LSU) return false;
  if (gather == IGP_GATHER_BULK || gather == IGP_GATHER_TMA4) return dc * sb >= 16;
  return false;
}

bool get_ops(int d, int storage, Ops* o) {
  const bool bf = storage == IGP_STORE_BF16;
  switch (d) {
    case 8: *o = bf ? ops_for<8, __nv_bfloat16>() : ops_for<8, float>(); return true;
    case 16: *o = bf ? ops_for<16, __nv_bfloat16>() : ops_for<16, float>(); return true;
    case 32: *o = bf ? ops_for<32, __nv_bfloat16>() : ops_for<32, float>(); return true;
    case 64: *o = bf ? ops_for<64, __nv_bfloat16>() : ops_for<64, float>(); return true;
    case 128: *o = bf ? ops_for<128, __nv_bfloat16>() : ops_for<128, float>(); return true;
    default: return false;
  }
}

igp_status launch_dinv(const int32_t* row_ptr, int32_t N, double tau, double eps, float* dinv, cudaStream_t s) {
  int blocks = (int)std::min<int64_t>(((int64_t)N + 255) / 256, (int64_t)num_sms() * 8);
  k_dinv<<<std::max(blocks, 1), 256, 0, s>>>(row_ptr, N, tau, eps, dinv);
  return after_launch("k_dinv");
}

igp_status launch_dinv_wsum(const int32_t* row_ptr, const int32_t* col, int32_t N, double tau, double eps,
                            float* dinv, float* wsum, cudaStream_t s) {
  IGP_TRY(launch_dinv(row_ptr, N, tau, eps, dinv, s));
  int wblocks = (int)std::min<int64_t>(((int64_t)N * 8 + 255) / 256, (int64_t)num_sms() * 8);
  k_wsum<<<std::max(wblocks, 1), 256, 0, s>>>(row_ptr, col, dinv, N, wsum);
  return after_launch("k_wsum");
}

}  // namespace

// Rows by decreasing degree (g->perm), once per graph. The allocation holds perm[N] and after
// it the offsets off[k] (k = 0..max_deg + 1) of each degree key in perm: off[k] = number of rows
// of degree > max_deg - k, so the rows of degree >= T are perm[0 .. off[max_deg - T + 1]).
igp_status ensure_perm(igp_graph* g, cudaStream_t s) {
  if (g->perm) return IGP_OK;
  const int32_t N = g->N;
  const int64_t nb = (int64_t)g->max_deg + 1;
  void* p = nullptr;
  IGP_TRY(dev_alloc(&p, ((size_t)N + nb + 1) * sizeof(int32_t), s));
  int32_t* perm = (int32_t*)p;
  void* t = nullptr;
  const int64_t ntiles = (nb + 1 + 8191) / 8192;
  igp_status st = dev_alloc(&t, (size_t)(2 * (nb + 1) + ntiles) * sizeof(int), s);
  if (st != IGP_OK) {
    dev_free(p, s);
    return st;
  }
  int* hist = (int*)t;
  int* off = perm + N;
  int* cur = hist + (nb + 1);
  int* tmp = cur + (nb + 1);
  if (cudaMemsetAsync(hist, 0, (nb + 1) * sizeof(int), s) != cudaSuccess ||
      cudaMemsetAsync(cur, 0, (nb + 1) * sizeof(int), s) != cudaSuccess)
    st = cuda_status(cudaGetLastError(), "memset", __FILE__, __LINE__);
  const int blocks = (int)(((int64_t)N + kPermRowsPerBlock - 1) / kPermRowsPerBlock);
  const size_t smem = nb <= kPermSmemBins ? (size_t)nb * sizeof(int) : 0;
  if (st == IGP_OK) {
    k_deg_hist<<<blocks, 512, smem, s>>>(g->row_ptr, N, g->max_deg, hist);
    st = after_launch("k_deg_hist");
  }
  if (st == IGP_OK) st = exclusive_scan(hist, off, nb + 1, tmp, s);
  if (st == IGP_OK) {
    k_deg_scatter<<<blocks, 512, smem, s>>>(g->row_ptr, N, g->max_deg, off, cur, perm);
    st = after_launch("k_deg_scatter");
  }
  dev_free(t, s);
  if (st != IGP_OK) {
    dev_free(p, s);
    return st;
  }
  g->perm = perm;
  return IGP_OK;
}

igp_status compute_dinv(igp_graph* g, double tau, double eps, cudaStream_t s, Profile* prof) {
  if (g->dinv_valid && g->dinv_tau == tau && g->dinv_eps == eps) return IGP_OK;
  if (!g->dinv) {
    void* p = nullptr;
    IGP_TRY(dev_alloc(&p, (size_t)g->N * 2 * sizeof(float), s));
    g->dinv = (float*)p;
    g->wsum = g->dinv + g->N;
  }
  PhaseTimer pt(prof, IGP_PHASE_DINV, s);
  IGP_TRY(launch_dinv_wsum(g->row_ptr, g->col, g->N, tau, eps, g->dinv, g->wsum, s));
  g->dinv_valid = true;
  g->dinv_tau = tau;
  g->dinv_eps = eps;
  return IGP_OK;
}

// Theta into `out` and, in the same launch, w of the graph (row_ptr, col) from dinv.
igp_status launch_theta_wsum(uint64_t seed, int32_t N, int32_t d, int32_t dc, float xs, int storage,
                             const float* dinv, void* out, const int32_t* row_ptr, const int32_t* col, float* wsum,
                             cudaStream_t s) {
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)N * 8 + 127) / 128, (int64_t)num_sms() * 8));
  if (storage == IGP_STORE_BF16)
    k_theta_wsum<__nv_bfloat16><<<blocks, 256, 0, s>>>(seed, N, d, dc, xs, dinv, (__nv_bfloat16*)out, row_ptr, col,
                                                       wsum);
  else
    k_theta_wsum<float><<<blocks, 256, 0, s>>>(seed, N, d, dc, xs, dinv, (float*)out, row_ptr, col, wsum);
  return after_launch("k_theta_wsum");
}

igp_status launch_theta(uint64_t seed, int32_t N, int32_t d, int32_t dc, float xs, int storage, const float* dinv,
                        void* out, cudaStream_t s) {
  int64_t total = (int64_t)N * (d / 8);
  int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms() * 16);
  blocks = std::max(blocks, 1);
  if (storage == IGP_STORE_BF16)
    k_theta<__nv_bfloat16><<<blocks, 256, 0, s>>>(seed, N, d, dc, xs, dinv, (__nv_bfloat16*)out);
  else
    k_theta<float><<<blocks, 256, 0, s>>>(seed, N, d, dc, xs, dinv, (float*)out);
  return after_launch("k_theta");
}

igp_status run_ffp(igp_graph* g, double tau, int32_t L, int32_t d, uint64_t seed, float* out_dev,
                   const igp_embed_opts& o, cudaStream_t s) {
  Profile* prof = o.profile ? &o.profile->prof : nullptr;
  Ops ops, lops;
  const int32_t N = g->N;
  const size_t sb = o.storage == IGP_STORE_BF16 ? 2 : 4;
  const int dc = o.chunk_cols > 0 ? o.chunk_cols : chunk_width(N, d, sb);  // columns per layer chunk
  if (!get_ops(d, o.storage, &ops) || !get_ops(dc, o.storage, &lops)) {
    set_error("igp_embed: d=%d unsupported (8, 16, 32, 64, 128)", d);
    return IGP_E_INVAL;
  }
  const int nchunks = d / dc;
  // Eq. 1 factors (cached per tau); w comes with Theta below when it has to be recomputed
  const bool w_ready = g->dinv_valid && g->dinv_tau == tau && g->dinv_eps == o.eps;
  if (!w_ready) {
    g->dinv_valid = false;
    if (!g->dinv) {
      void* p = nullptr;
      IGP_TRY(dev_alloc(&p, (size_t)g->N * 2 * sizeof(float), s));
      g->dinv = (float*)p;
      g->wsum = g->dinv + g->N;
    }
    PhaseTimer pt(prof, IGP_PHASE_DINV, s);
    IGP_TRY(launch_dinv(g->row_ptr, N, tau, o.eps, g->dinv, s));
  }
  IGP_TRY(ensure_perm(g, s));
  const bool tma = use_tma(o.gather, dc, sb);
  if (o.gather == IGP_GATHER_TMA4 && dc != d) {
    set_error("igp_embed: gather4 needs the whole row in one pass (chunk_cols = 0 or d)");
    return IGP_E_INVAL;
  }
  const int grid = tma ? lops.tma_grid(N) : lops.grid(N);
  // workspace: T0 | T1 | stats[2][2d] | gsum[nchunks][2dc] | err, tickets[nchunks], claims[nchunks]
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t bT = al((size_t)N * d * sb);
  const size_t bS = al(2 * 2 * (size_t)d * sizeof(float));
  const size_t bP = al((size_t)nchunks * 2 * dc * sizeof(unsigned long long));
  const size_t bK = al((size_t)(2 * nchunks + 1) * sizeof(unsigned));
  const size_t need = 2 * bT + bS + bP + bK;
  if (g->ws_bytes < need) {
    if (g->ws) dev_free(g->ws, s);
    g->ws = nullptr;
    g->ws_bytes = 0;
    void* p = nullptr;
    IGP_TRY(dev_alloc(&p, need, s));
    g->ws = p;
    g->ws_bytes = need;
  }
  char* base = (char*)g->ws;
  void* T0 = base;
  void* T1 = base + bT;
  float* stats = (float*)(base + 2 * bT);
  unsigned long long* gsum = (unsigned long long*)(base + 2 * bT + bS);
  int* err = (int*)(base + 2 * bT + bS + bP);
  unsigned* tickets = (unsigned*)(err + 1);
  IGP_TRY_CUDA(cudaMemsetAsync(gsum, 0, bP + (2 * nchunks + 1) * sizeof(unsigned), s));

  {
    PhaseTimer pt(prof, IGP_PHASE_THETA, s);
    if (o.x_in) {
      if (!w_ready) {
        const int wblocks = (int)std::min<int64_t>(((int64_t)N * 8 + 255) / 256, (int64_t)num_sms() * 8);
        k_wsum<<<std::max(wblocks, 1), 256, 0, s>>>(g->row_ptr, g->col, g->dinv, N, g->wsum);
        IGP_TRY(after_launch("k_wsum"));
      }
      IGP_TRY(ops.prescale(o.x_in, g->dinv, N, d, dc, T0, s));
    } else {
      const double xs = o.x_scale > 0 ? o.x_scale : 1.0 / std::sqrt((double)d);
      if (w_ready)
        IGP_TRY(launch_theta(seed, N, d, dc, (float)xs, o.storage, g->dinv, T0, s));
      else
        IGP_TRY(launch_theta_wsum(seed, N, d, dc, (float)xs, o.storage, g->dinv, T0, g->row_ptr, g->col,
                                  g->wsum, s));
    }
  }
  if (!w_ready) {
    g->dinv_valid = true;
    g->dinv_tau = tau;
    g->dinv_eps = o.eps;
  }
  LayerArgs la;
  la.row_ptr = g->row_ptr;
  la.col = g->col;
  la.perm = g->perm;
  la.dinv = g->dinv;
  la.wsum = g->wsum;
  la.gsum = gsum;
  la.tickets = tickets;
  la.err = err;
  la.withhold = o.reserved_test;
  la.gather4 = o.gather == IGP_GATHER_TMA4;
  la.prefetch = (size_t)N * dc * sb > kL2ResidentBytes ? 1 : 0;
  {  // rows of at least layer_heavy_min entries lead the degree order: their count
    const int Gl = std::max(1, (int)(dc * sb / 16));
    const int T = layer_heavy_min(Gl);
    la.heavy_count = (32 / Gl > 1 && T <= g->max_deg) ? g->perm + N + (g->max_deg - T + 1) : nullptr;
  }
  la.N = N;
  la.d = d;

  la.alpha = (float)o.alpha;
  la.theta = (float)o.theta;
  la.ddof = o.znorm_ddof;
  la.grid = grid;
  const void* cur = T0;
  const float* st_prev = nullptr;
  for (int32_t l = 1; l <= L; ++l) {
    void* dst = (cur == T0) ? T1 : T0;
    float* st = stats + (size_t)(l & 1) * 2 * d;
    la.Tin = cur;
    la.Tout = dst;
    la.stats_in = st_prev;
    la.stats_out = st;
    PhaseTimer pt(prof, IGP_PHASE_LAYER, s);
    IGP_TRY(tma ? lops.layer_tma(la, s) : lops.layer(la, s));
    cur = dst;
    st_prev = st;
  }
  {
    PhaseTimer pt(prof, IGP_PHASE_OUTPUT, s);
    IGP_TRY(ops.output(cur, g->dinv, st_prev, o.out_row_begin, N, dc, o.out_row_l2, out_dev, s));
  }
  // the device error word of this call, read by igp_graph_sync / host-output calls
  IGP_TRY_CUDA(cudaMemcpyAsync(g->err_host, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  return IGP_OK;
}

// ------------------------------------------------------------------ batch host side
igp_status batch_create(igp_graph* const* graphs, int32_t G, cudaStream_t s, igp_batch* b) {
  std::vector<PackSrc> src(G);
  int64_t N = 0, nnz = 0, P = 0;
  b->goff_host.assign(G + 1, 0);
  for (int32_t g = 0; g < G; ++g) {
    igp_graph* gr = graphs[g];
    IGP_TRY(ensure_perm(gr, s));
    src[g] = PackSrc{gr->row_ptr, gr->col, gr->perm, gr->N, (int32_t)N, (int32_t)P, (int32_t)nnz};
    b->goff_host[g] = (int32_t)N;
    N += gr->N;
    nnz += gr->nnz;
    P += ((int64_t)gr->N + kBatchAlign - 1) / kBatchAlign * kBatchAlign;
    if (N >= (1ll << 31) - 1 || nnz + 4 * P >= (1ll << 31) - 1) {
      set_error("igp_batch_create: the packed batch exceeds 2^31 rows or entries");
      return IGP_E_INVAL;
    }
  }
  b->goff_host[G] = (int32_t)N;
  b->G = G;
  b->N = (int32_t)N;
  b->nnz = nnz;
  b->P = P;
  auto alloc = [&](void** p, size_t bytes) { return dev_alloc(p, bytes, s); };
  void *rp, *cl, *rg, *pm, *pg, *go, *sd, *ps;
  IGP_TRY(alloc(&rp, (N + 1) * 4));
  b->row_ptr = (int32_t*)rp;
  IGP_TRY(alloc(&cl, std::max<int64_t>(nnz, 1) * 4));
  b->col = (int32_t*)cl;
  IGP_TRY(alloc(&rg, std::max<int64_t>(N, 1) * 4));
  b->row_graph = (int32_t*)rg;
  IGP_TRY(alloc(&pm, std::max<int64_t>(P, 1) * 4));
  b->perm = (int32_t*)pm;
  IGP_TRY(alloc(&pg, std::max<int64_t>(P / kBatchAlign, 1) * 4));
  b->pgraph = (int32_t*)pg;
  IGP_TRY(alloc(&go, (G + 1) * 4));
  b->goff = (int32_t*)go;
  IGP_TRY(alloc(&sd, (size_t)G * 8));
  b->seeds_dev = (uint64_t*)sd;
  IGP_TRY(alloc(&ps, (size_t)G * sizeof(PackSrc)));
  const int32_t nnz32 = (int32_t)nnz;
  IGP_TRY_CUDA(cudaMemcpyAsync(ps, src.data(), (size_t)G * sizeof(PackSrc), cudaMemcpyHostToDevice, s));
  IGP_TRY_CUDA(cudaMemcpyAsync(b->goff, b->goff_host.data(), (G + 1) * 4, cudaMemcpyHostToDevice, s));
  IGP_TRY_CUDA(cudaMemcpyAsync(b->row_ptr + N, &nnz32, 4, cudaMemcpyHostToDevice, s));
  dim3 grid(std::max(1, num_sms() * 4 / std::max(G, 1)), G);
  k_batch_pack<<<grid, 256, 0, s>>>((const PackSrc*)ps, G, b->row_ptr, b->col, b->row_graph, b->perm, b->pgraph);
  IGP_TRY(after_launch("k_batch_pack"));
  IGP_TRY_CUDA(cudaStreamSynchronize(s));  // the host arrays above and the source graphs are read
  dev_free(ps, s);
  return IGP_OK;
}

// The batch's chunk table for warp tiles of gpw rows and chunks of `mean` positions on average,
// built on first use (stream-ordered) and kept with the batch.
igp_status ensure_chunks(igp_batch* b, int gpw, int mean, cudaStream_t s, igp_batch::Chunks* out) {
  const auto key = std::make_pair(gpw, mean);
  auto it = b->chunks.find(key);
  if (it != b->chunks.end()) {
    *out = it->second;
    return IGP_OK;
  }
  const int64_t T = b->P / gpw;  // P is a multiple of kBatchAlign, which gpw divides
  void* p = nullptr;
  IGP_TRY(dev_alloc(&p, (size_t)(T + 2) * 4, s));
  igp_batch::Chunks c{(int32_t*)p, (int*)p + T + 1};
  igp_status st = IGP_OK;
  if (T == 0) {
    if (cudaMemsetAsync(p, 0, 8, s) != cudaSuccess) st = cuda_status(cudaGetLastError(), "chunk table", __FILE__, __LINE__);
  } else {
    void* q = nullptr;
    const int64_t ntile = (T + 8191) / 8192;
    st = dev_alloc(&q, (size_t)(3 * T + ntile) * 4, s);
    if (st == IGP_OK) {
      int* w = (int*)q;
      int* ex = w + T;
      int* f = ex + T;
      int* tmp = f + T;
      const int blocks = (int)std::min<int64_t>((T + 255) / 256, (int64_t)num_sms() * 8);
      k_tile_weight<<<blocks, 256, 0, s>>>(b->perm, b->row_ptr, T, gpw, w);
      st = after_launch("k_tile_weight");
      if (st == IGP_OK) st = exclusive_scan(w, ex, T, tmp, s);
      if (st == IGP_OK) {
        k_chunk_flags<<<blocks, 256, 0, s>>>(w, ex, T, gpw, mean, f);
        st = after_launch("k_chunk_flags");
      }
      if (st == IGP_OK) st = exclusive_scan(f, w, T, tmp, s);  // w := index of each starting tile's chunk
      if (st == IGP_OK) {
        k_chunk_starts<<<blocks, 256, 0, s>>>(f, w, T, gpw, c.start, c.count);
        st = after_launch("k_chunk_starts");
      }
      dev_free(q, s);
    }
  }
  if (st != IGP_OK) {
    dev_free(p, s);
    return st;
  }
  b->chunks[key] = c;
  *out = c;
  return IGP_OK;
}

igp_status batch_embed(igp_batch* b, double tau, int32_t L, int32_t d, const uint64_t* seeds, float* out_dev,
                       const igp_embed_opts& o, cudaStream_t s, bool capture) {
  BatchOps bo;
  Ops ops;
  if (!get_batch_ops(d, o.storage, &bo) || !get_ops(d, o.storage, &ops)) {
    set_error("igp_batch_embed: d=%d unsupported (8, 16, 32, 64, 128)", d);
    return IGP_E_INVAL;
  }
  Profile* prof = o.profile ? &o.profile->prof : nullptr;
  const size_t sb = o.storage == IGP_STORE_BF16 ? 2 : 4;
  const int32_t N = b->N, G = b->G;
  // per-tau factors on the packed (block-diagonal) CSR: every degree is a degree in its own graph
  if (!(b->dinv_valid && b->dinv_tau == tau && b->dinv_eps == o.eps)) {
    if (!b->dinv) {
      void* p = nullptr;
      IGP_TRY(dev_alloc(&p, (size_t)std::max(N, 1) * 8, s));
      b->dinv = (float*)p;
      b->wsum = b->dinv + N;
    }
    PhaseTimer pt(prof, IGP_PHASE_DINV, s);
    IGP_TRY(launch_dinv_wsum(b->row_ptr, b->col, N, tau, o.eps, b->dinv, b->wsum, s));
    b->dinv_valid = true;
    b->dinv_tau = tau;
    b->dinv_eps = o.eps;
    b->exec_key.clear();
  }
  // one full wave of CTAs (fewer for a short order), warps claiming chunks of the order
  auto grid_for = [&](int chunk) {
    const int64_t want = (b->P + (int64_t)kLayerWarps * chunk - 1) / ((int64_t)kLayerWarps * chunk);
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)bo.per_sm() * num_sms()));
  };
  // workspace: T0 | T1 | stats[2][G][2d] | gsum[G][2d] + claim counter | rows_done[G] ready[G] qctr err
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t bT = al((size_t)N * d * sb);
  const size_t bS = al((size_t)2 * G * 2 * d * sizeof(float));
  const size_t bQ = al((size_t)G * 2 * d * sizeof(unsigned long long) + sizeof(unsigned long long));  // + counter
  const size_t offQ = ((size_t)G * 8 + 7) & ~(size_t)7;
  const size_t bX = al(offQ + 16);
  const size_t need = 2 * bT + bS + bQ + bX;
  if (b->ws_bytes < need) {
    if (b->ws) dev_free(b->ws, s);
    b->ws = nullptr;
    b->ws_bytes = 0;
    void* p = nullptr;
    IGP_TRY(dev_alloc(&p, need, s));
    b->ws = p;
    b->ws_bytes = need;
    b->exec_key.clear();
  }
  if (!b->err_host) {
    count_alloc();
    b->err_host = pinned_slot();
    if (!b->err_host) return cuda_status(cudaGetLastError(), "page-locked error word", __FILE__, __LINE__);
  }
  char* base = (char*)b->ws;
  void* T0 = base;
  void* T1 = base + bT;
  float* stats = (float*)(base + 2 * bT);
  unsigned long long* gsum = (unsigned long long*)(base + 2 * bT + bS);
  char* xb = base + 2 * bT + bS + bQ;
  unsigned* rows_done = (unsigned*)xb;
  int* ready = (int*)(xb + (size_t)G * 4);
  unsigned long long* qctr = (unsigned long long*)(xb + offQ);
  int* err = (int*)(xb + offQ + 8);
  const double xs = o.x_scale > 0 ? o.x_scale : 1.0 / std::sqrt((double)d);
  // test hooks (reserved_test, the library's own tests only): 2 = the persistent plan with one row
  // of graph 0 withheld, so that its bounded waits run out; 3, 4 = the persistent plan (claims of
  // 64 at one CTA per SM; of 256 at the resident maximum); 5 = one launch per layer (claims of 64);
  // 6, 7 = the persistent plan with claims of 64, 32 at the resident maximum
  const int withhold = o.reserved_test == 2 ? 1 : 0;

  IGP_TRY_CUDA(cudaMemcpyAsync(b->seeds_dev, seeds, (size_t)G * 8, cudaMemcpyHostToDevice, s));

  // One FFP of every graph with plan pl: Theta, the layers (one launch each plus a statistics
  // launch, or one persistent launch for all of them) and the output.
  auto enqueue_plan = [&](cudaStream_t q, Profile* pf, const igp_batch::Plan& pl) -> igp_status {
    IGP_TRY_CUDA(cudaMemsetAsync(gsum, 0, bQ + bX, q));
    {
      PhaseTimer pt(pf, IGP_PHASE_THETA, q);
      IGP_TRY(bo.theta(b, d, (float)xs, T0, q));
    }
    const void* cur = T0;
    const float* st_prev = nullptr;
    if (pl.mode == 1 && L > 0) {
      igp_batch::Chunks ch;
      IGP_TRY(ensure_chunks(b, bo.gpw, pl.chunk, q, &ch));
      PersistArgs a{T0, T1, stats, gsum, rows_done, ready, qctr, err, ch.start, ch.count, L, o.znorm_ddof,
                    pl.ctas * num_sms(), withhold, (float)o.alpha, (float)o.theta};
      {
        PhaseTimer pt(pf, IGP_PHASE_LAYER, q);
        IGP_TRY(bo.persist(b, a, q));
      }
      IGP_TRY_CUDA(cudaMemcpyAsync(b->err_host, err, sizeof(int), cudaMemcpyDeviceToHost, q));
      if (!b->ev_err) IGP_TRY_CUDA(cudaEventCreateWithFlags(&b->ev_err, cudaEventDisableTiming));
      IGP_TRY_CUDA(cudaEventRecord(b->ev_err, q));
      cur = (L & 1) ? T1 : T0;
      st_prev = stats + (size_t)(L & 1) * G * 2 * d;
    } else {
      for (int32_t l = 1; l <= L; ++l) {
        void* dst = (cur == T0) ? T1 : T0;
        float* st = stats + (size_t)(l & 1) * G * 2 * d;
        PhaseTimer pt(pf, IGP_PHASE_LAYER, q);
        igp_batch::Chunks ch;
        IGP_TRY(ensure_chunks(b, bo.gpw, pl.chunk, q, &ch));
        IGP_TRY(bo.layer(b, cur, dst, st_prev, gsum, (float)o.alpha, (float)o.theta, grid_for(pl.chunk), ch.start,
                         ch.count, q));
        IGP_TRY(bo.tail(b, gsum, o.znorm_ddof, st, q));
        cur = dst;
        st_prev = st;
      }
    }
    PhaseTimer pt(pf, IGP_PHASE_OUTPUT, q);
    return bo.output(b, cur, st_prev, o.out_row_l2, out_dev, q);
  };

  // Schedule tuner: on the first embedding at a (d, storage, mean-degree bucket) in this process,
  // every candidate plan runs one whole FFP of this batch, timed with CUDA events, and the
  // fastest is kept for the key (later batches with the same key reuse it). Candidates: one
  // launch per layer with each claim size (32, 64, 128, 256 positions on average), and the
  // persistent launch at the resident maximum with claims of 32, 64 and 128 (the positions in flight
  // are what its warps gather from at once: larger claims overflow L2).
  const int tkey = d * 2 + o.storage;
  igp_batch::Plan plan;
  if (o.reserved_test >= 2 && o.reserved_test <= 7) {
    const int t = o.reserved_test;
    plan.mode = t == 5 ? 0 : 1;
    plan.chunk = t == 4 ? 256 : t == 7 ? 32 : 64;
    plan.ctas = (t == 4 || t >= 6) ? bo.persist_per_sm() : 1;
  } else {
    if (!b->plan.count(tkey)) {
      const int dbucket = (int)std::lround(std::log2(std::max(1.0, (double)b->nnz / std::max(1, N))));
      const auto gkey = std::make_tuple(d, o.storage, dbucket);
      static std::mutex tmu;
      static std::map<std::tuple<int, int, int>, igp_batch::Plan> tuned;
      bool found = false;
      {
        std::lock_guard<std::mutex> lk(tmu);
        auto it = tuned.find(gkey);
        if (it != tuned.end()) {
          b->plan[tkey] = it->second;
          found = true;
        }
      }
      if (!found) {
        std::vector<igp_batch::Plan> cands;
        for (int c : kBatchChunks) cands.push_back(igp_batch::Plan{0, c, 1});
        const int pm = bo.persist_per_sm();
        for (int c : {32, 64, 128}) cands.push_back(igp_batch::Plan{1, c, pm});
        for (const auto& c : cands) {  // chunk tables first: not part of any plan's time
          igp_batch::Chunks ch;
          IGP_TRY(ensure_chunks(b, bo.gpw, c.chunk, s, &ch));
        }
        std::vector<cudaEvent_t> ev(2 * cands.size() + 2, nullptr);
        for (auto& e : ev) IGP_TRY_CUDA(cudaEventCreate(&e));
        igp_status st = enqueue_plan(s, nullptr, cands[0]);  // warm-up (module loads, first touches)
        for (size_t k = 0; k < cands.size() && st == IGP_OK; ++k) {
          cudaEventRecord(ev[2 * k], s);
          st = enqueue_plan(s, nullptr, cands[k]);
          cudaEventRecord(ev[2 * k + 1], s);
        }
        igp_batch::Plan best = cands[0];
        float best_ms = 1e30f;
        for (size_t k = 0; k < cands.size() && st == IGP_OK; ++k) {
          float ms = 0.0f;
          if (cudaEventSynchronize(ev[2 * k + 1]) != cudaSuccess ||
              cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]) != cudaSuccess) {
            st = cuda_status(cudaGetLastError(), "schedule tuning", __FILE__, __LINE__);
            break;
          }
          if (ms < best_ms) {
            best_ms = ms;
            best = cands[k];
          }
        }
        for (auto& e : ev) cudaEventDestroy(e);
        if (st == IGP_OK && *b->err_host) {
          *b->err_host = 0;
          set_error("igp_batch_embed: a bounded device-side wait ran out while tuning the schedule");
          st = IGP_E_TIMEOUT;
        }
        IGP_TRY(st);
        b->plan[tkey] = best;
        std::lock_guard<std::mutex> lk(tmu);
        tuned[gkey] = best;
      }
      b->exec_key.clear();
    }
    plan = b->plan[tkey];
  }
  const int chunk = plan.chunk;
  {
    igp_batch::Chunks ch;  // built here, before any capture, on first use
    IGP_TRY(ensure_chunks(b, bo.gpw, chunk, s, &ch));
  }

  auto enqueue = [&](cudaStream_t q, Profile* pf) -> igp_status { return enqueue_plan(q, pf, plan); };

  // timed phases, a one-off batch or the persistent launch: plain launches
  if (prof || !capture || plan.mode == 1) return enqueue(s, prof);
  // The launch sequence is captured once into a CUDA graph (on a library stream ordered
  // after `s`) and replayed while its parameters stay the same.
  char key[256];
  snprintf(key, sizeof(key), "%a|%d|%d|%d|%a|%a|%a|%d|%d|%a|%p|%p|%d", tau, L, d, o.storage, o.alpha, o.theta,
           o.eps, o.znorm_ddof, o.out_row_l2, xs, (void*)out_dev, b->ws, chunk);
  if (!b->cs) IGP_TRY_CUDA(cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking));
  if (!b->ev_in) IGP_TRY_CUDA(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
  if (!b->ev_out) IGP_TRY_CUDA(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
  IGP_TRY_CUDA(cudaEventRecord(b->ev_in, s));
  IGP_TRY_CUDA(cudaStreamWaitEvent(b->cs, b->ev_in, 0));
  if (b->exec_key != key) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    const int64_t n0 = igp_launch_count();
    IGP_TRY_CUDA(cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal));
    igp_status st = enqueue(b->cs, nullptr);
    cudaError_t e = cudaStreamEndCapture(b->cs, &graph);
    b->exec_kernels = igp_launch_count() - n0;
    count_launches(-b->exec_kernels);  // captured, not run: counted when the graph runs
    if (st != IGP_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    IGP_TRY_CUDA(e);
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    IGP_TRY_CUDA(e);
    b->exec_key = key;
  }
  IGP_TRY_CUDA(cudaGraphLaunch(b->exec, b->cs));
  count_launches(b->exec_kernels);
  IGP_TRY_CUDA(cudaEventRecord(b->ev_out, b->cs));
  IGP_TRY_CUDA(cudaStreamWaitEvent(s, b->ev_out, 0));
  return IGP_OK;
}

}  // namespace igp

// ============================================================================
// igp_embed_noalloc: one FFP that allocates nothing.
//
// Some callers cannot allocate device memory while they call into this library: an
// allocator hook or custom memory manager that must not re-enter the allocator it is
// part of, a framework whose caching allocator already holds the free memory (so a
// cudaMalloc here would fail), or a long-running loop that has to keep a fixed memory
// footprint. This entry point serves them: the caller passes the CSR, the output and a
// stream; all temporaries live in one fixed device array that is part of the library
// image, and nothing here calls dev_alloc or any other allocating routine.
//
// The array below is reserved on every GPU that loads the library and stays
// reserved until the process exits. Every call shares it, so calls whose GPU work
// overlaps (on different streams, or from different host threads) race with each
// other; serialise them. It keeps the last call's contents; what a call needs zeroed
// (the completion tickets of the column statistics) it clears itself.
// ============================================================================
namespace igp {
namespace {

constexpr size_t kNoAllocScratchBytes = 16ull << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch on the current device (host code may not use the
// symbol itself: on the host it names a stand-in, not device memory).
igp_status noalloc_scratch(void** ptr) {
  static std::mutex mu;
  static void* addr[64] = {};
  int dev = 0;
  IGP_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("igp_embed_noalloc: device ordinal %d out of range", dev);
    return IGP_E_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
    addr[dev] = p;
  }
  *ptr = addr[dev];
  return IGP_OK;
}

}  // namespace
}  // namespace igp

extern "C" igp_status igp_embed_noalloc(const int32_t* row_ptr, const int32_t* col, int32_t N, double tau,
                                        int32_t L, int32_t d, uint64_t seed, float* out,
                                        const igp_embed_opts* opts, void* stream) {
  using namespace igp;
  clear_error();
  igp_embed_opts o;
  if (opts)
    o = *opts;
  else
    igp_embed_opts_init(&o);
  if (!row_ptr || !col || !out || N < 1) {
    set_error("igp_embed_noalloc: need device row_ptr, col and out, and N >= 1");
    return IGP_E_INVAL;
  }
  if (!std::isfinite(tau) || L < 0 || L > 10000 || !std::isfinite(o.alpha) || !std::isfinite(o.theta) ||
      !(o.eps > 0) || !std::isfinite(o.eps) || (o.znorm_ddof != 0 && o.znorm_ddof != 1) ||
      (o.storage != IGP_STORE_F32 && o.storage != IGP_STORE_BF16) || !std::isfinite(o.x_scale)) {
    set_error("igp_embed_noalloc: invalid tau, L or options");
    return IGP_E_INVAL;
  }
  if (o.profile || o.chunk_cols != 0) {
    set_error("igp_embed_noalloc: opts->profile and opts->chunk_cols are not supported here (leave them 0)");
    return IGP_E_INVAL;
  }
  if (o.out_row_begin < 0 || o.out_row_begin > N) {
    set_error("igp_embed_noalloc: opts->out_row_begin=%d outside [0, N=%d]", o.out_row_begin, N);
    return IGP_E_INVAL;
  }
  Ops ops;
  if (!get_ops(d, o.storage, &ops)) {
    set_error("igp_embed_noalloc: d=%d unsupported (8, 16, 32, 64, 128)", d);
    return IGP_E_INVAL;
  }
  if (!is_device_ptr(row_ptr) || !is_device_ptr(col) || !is_device_ptr(out) ||
      (o.x_in && !is_device_ptr(o.x_in))) {
    set_error("igp_embed_noalloc: row_ptr, col, out (and opts->x_in) must be device memory");
    return IGP_E_INVAL;
  }
  // scratch layout: dinv | w | T0 | T1 | stats[2][2d] | gsum[2d] | ticket, claims, err
  const size_t sb = o.storage == IGP_STORE_BF16 ? 2 : 4;
  const int grid = ops.grid(N);
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t bN = al((size_t)N * 4);
  const size_t bT = al((size_t)N * d * sb);
  const size_t bS = al(2 * 2 * (size_t)d * sizeof(float));
  const size_t bP = al((size_t)2 * d * sizeof(unsigned long long));
  const size_t need = 2 * bN + 2 * bT + bS + bP + 256;
  if (need > kNoAllocScratchBytes) {
    set_error("igp_embed_noalloc: N=%d, d=%d needs %zu bytes of scratch, more than the fixed %zu (16 MiB); "
              "use igp_embed for this size",
              N, d, need, kNoAllocScratchBytes);
    return IGP_E_INVAL;
  }
  void* scratch = nullptr;
  IGP_TRY(noalloc_scratch(&scratch));
  cudaStream_t s = (cudaStream_t)stream;
  char* base = (char*)scratch;
  float* dinv = (float*)base;
  float* wsum = (float*)(base + bN);
  void* T0 = base + 2 * bN;
  void* T1 = base + 2 * bN + bT;
  float* stats = (float*)(base + 2 * bN + 2 * bT);
  unsigned long long* gsum = (unsigned long long*)(base + 2 * bN + 2 * bT + bS);
  unsigned* ticket = (unsigned*)(base + 2 * bN + 2 * bT + bS + bP);  // ticket, tile-claim counter
  int* err = (int*)(ticket + 2);
  IGP_TRY_CUDA(cudaMemsetAsync(gsum, 0, bP + 3 * sizeof(unsigned), s));

  // the caller's graph as it is (no relabelling: that would need memory)
  IGP_TRY(launch_dinv_wsum(row_ptr, col, N, tau, o.eps, dinv, wsum, s));
  if (o.x_in) {
    IGP_TRY(ops.prescale(o.x_in, dinv, N, d, d, T0, s));
  } else {
    const double xs = o.x_scale > 0 ? o.x_scale : 1.0 / std::sqrt((double)d);
    IGP_TRY(launch_theta(seed, N, d, d, (float)xs, o.storage, dinv, T0, s));
  }
  LayerArgs la;
  la.row_ptr = row_ptr;
  la.col = col;
  la.perm = nullptr;  // rows in their own order
  la.dinv = dinv;
  la.wsum = wsum;
  la.gsum = gsum;
  la.tickets = ticket;
  la.err = err;
  la.withhold = 0;
  la.gather4 = 0;
  la.prefetch = (size_t)N * d * sb > kL2ResidentBytes ? 1 : 0;
  la.heavy_count = nullptr;  // rows in their own order: no heavy tiles
  la.N = N;
  la.d = d;

  la.alpha = (float)o.alpha;
  la.theta = (float)o.theta;
  la.ddof = o.znorm_ddof;
  la.grid = grid;
  const void* cur = T0;
  const float* st_prev = nullptr;
  for (int32_t l = 1; l <= L; ++l) {
    void* dst = (cur == T0) ? T1 : T0;
    float* st = stats + (size_t)(l & 1) * 2 * d;
    la.Tin = cur;
    la.Tout = dst;
    la.stats_in = st_prev;
    la.stats_out = st;
    IGP_TRY(ops.layer(la, s));
    cur = dst;
    st_prev = st;
  }
  return ops.output(cur, dinv, st_prev, o.out_row_begin, N, d, o.out_row_l2, out, s);
}
