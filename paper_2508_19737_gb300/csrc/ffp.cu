// The feed-forward propagation (FFP) of InfraredGP, Alg. 1 lines 1-6:
//   k_dinv    Eq. 1 degree correction D_tau and D_tau^{-1/2} (fp64, rounded to fp32)
//   k_theta   Z^(0) = Theta ~ N(0, 1/d): Philox4x64-10 + Box-Muller (Alg. 1, line 2)
//   k_layer   one Eq. 4 layer: T^(l) = tanh(theta Z + alpha Ahat Z), Z = ZNorm(T^(l-1)),
//             fused with the column statistics of T^(l) that the next ZNorm needs
//   k_output  Z~ = sigmoid(ZNorm(T^(L))) (Eq. 4), optional row L2 normalisation
//
// Layer kernel design (bandwidth-bound sparse gather, no tensor cores):
//   * one warp per row; its 32 lanes are NS neighbour slots x G column chunks, a chunk
//     being 16 bytes of the stored row (8 bf16 or 4 fp32 values), so a neighbour row
//     is fetched by G lanes with one 16-byte load each;
//   * slot s takes neighbours beg+s, beg+s+NS, ...; U neighbours per slot are in
//     flight per iteration and the next iteration's column indices are prefetched;
//   * ZNorm of the input is applied after the gather, per row:
//       sum_j dinv_j z_j = inv_s (sum_j dinv_j t_j - mu sum_j dinv_j),
//     so a neighbour costs one FMA per element;
//   * the NS slot partial sums are combined by a shuffle reduce-scatter, after which
//     each lane owns EPL columns of the row and applies the epilogue (self term,
//     tanh, store, running column sums) to them only;
//   * column statistics: per-lane fp32 sums of t and t^2, a fixed-order CTA
//     reduction to one partial per CTA, and the last CTA to finish (ticket counter)
//     reduces the partials in fixed order and forms mean and 1/std in fp64.
#include <cmath>
#include <cstdio>

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

// E consecutive values (E = 1, 2, 4; aligned to E elements)
template <int E>
__device__ __forceinline__ void load_small(const float* p, float (&v)[E]) {
  if constexpr (E == 1) {
    v[0] = __ldg(p);
  } else if constexpr (E == 2) {
    float2 x = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = x.x; v[1] = x.y;
  } else {
    float4 x = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  }
}
template <int E>
__device__ __forceinline__ void load_small(const __nv_bfloat16* p, float (&v)[E]) {
  if constexpr (E == 1) {
    uint32_t h = __ldg(reinterpret_cast<const unsigned short*>(p));
    v[0] = __uint_as_float(h << 16);
  } else if constexpr (E == 2) {
    uint32_t x = __ldg(reinterpret_cast<const unsigned int*>(p));
    v[0] = bf_lo(x); v[1] = bf_hi(x);
  } else if constexpr (E == 4) {
    uint2 x = __ldg(reinterpret_cast<const uint2*>(p));
    v[0] = bf_lo(x.x); v[1] = bf_hi(x.x); v[2] = bf_lo(x.y); v[3] = bf_hi(x.y);
  } else {
    uint4 x = __ldg(reinterpret_cast<const uint4*>(p));
    v[0] = bf_lo(x.x); v[1] = bf_hi(x.x); v[2] = bf_lo(x.y); v[3] = bf_hi(x.y);
    v[4] = bf_lo(x.z); v[5] = bf_hi(x.z); v[6] = bf_lo(x.w); v[7] = bf_hi(x.w);
  }
}
template <int E>
__device__ __forceinline__ void store_small(float* p, const float (&v)[E]) {
  if constexpr (E == 1) {
    p[0] = v[0];
  } else if constexpr (E == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
}
template <int E>
__device__ __forceinline__ void store_small(__nv_bfloat16* p, const float (&v)[E]) {
  if constexpr (E == 1) {
    *p = __float2bfloat16_rn(v[0]);
  } else if constexpr (E == 2) {
    *reinterpret_cast<uint32_t*>(p) = bf_pack(v[0], v[1]);
  } else if constexpr (E == 4) {
    *reinterpret_cast<uint2*>(p) = make_uint2(bf_pack(v[0], v[1]), bf_pack(v[2], v[3]));
  } else {
    *reinterpret_cast<uint4*>(p) = make_uint4(bf_pack(v[0], v[1]), bf_pack(v[2], v[3]), bf_pack(v[4], v[5]),
                                              bf_pack(v[6], v[7]));
  }
}

constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

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

// ------------------------------------------------------------------ Theta (Alg. 1, line 2)
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

template <typename S>
__global__ void k_theta(uint64_t seed, int32_t N, int32_t d, float xs, S* __restrict__ out) {
  const int nq = d >> 3;
  const int64_t total = (int64_t)N * nq;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / nq;
    const int q = (int)(t - i * nq);
    float z[8];
    theta8(seed, (uint64_t)i, (uint64_t)q, xs, z);
    S* p = out + i * d + q * 8;
    if constexpr (sizeof(S) == 2) {
      store_chunk(p, z);
    } else {
      float a[4] = {z[0], z[1], z[2], z[3]}, b[4] = {z[4], z[5], z[6], z[7]};
      store_chunk(p, a);
      store_chunk(p + 4, b);
    }
  }
}

// ------------------------------------------------------------------ Eq. 4 layer
template <int D, typename S, int U>
__global__ void __launch_bounds__(kLayerThreads) k_layer(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col, const float* __restrict__ dinv,
    const S* __restrict__ Tin, S* __restrict__ Tout, const float* __restrict__ stats_in,
    float* __restrict__ partials, float* __restrict__ stats_out, unsigned* __restrict__ ticket, int32_t N,
    float alpha, float theta, int ddof) {
  constexpr int VPL = Store<S>::VPL;
  constexpr int G = D / VPL;   // lanes per row copy (16 B each)
  constexpr int NS = 32 / G;   // neighbour slots per warp
  constexpr int EPL = VPL >= NS ? VPL / NS : 1;  // epilogue values per lane
  constexpr int RS = ilog2(VPL / EPL);           // reduce-scatter steps
  constexpr int AR = ilog2(NS) - RS;             // remaining all-reduce steps
  static_assert(G >= 1 && G <= 32 && NS * G == 32, "unsupported width");

  __shared__ float s_mu[D], s_is[D];
  __shared__ float s_red[kLayerWarps][2 * D];
  __shared__ bool s_last;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int chunk = lane % G, slot = lane / G;
  for (int c = threadIdx.x; c < D; c += blockDim.x) {
    s_mu[c] = stats_in ? stats_in[c] : 0.0f;
    s_is[c] = stats_in ? stats_in[D + c] : 1.0f;
  }
  __syncthreads();

  // columns this lane owns after the reduce-scatter
  int off = 0;
#pragma unroll
  for (int b = 0; b < RS; ++b) {
    const int sb = ilog2(NS) - 1 - b;
    if ((slot >> sb) & 1) off += (VPL >> (b + 1));
  }
  const bool owner = AR == 0 || (slot & ((1 << AR) - 1)) == 0;
  const int cc = chunk * VPL + off;

  float mu_e[EPL], is_e[EPL];
#pragma unroll
  for (int e = 0; e < EPL; ++e) {
    mu_e[e] = s_mu[cc + e];
    is_e[e] = s_is[cc + e];
  }
  float csum[EPL], csq[EPL];
#pragma unroll
  for (int e = 0; e < EPL; ++e) csum[e] = csq[e] = 0.0f;

  const int64_t nwarps = (int64_t)gridDim.x * kLayerWarps;
  for (int64_t i = (int64_t)blockIdx.x * kLayerWarps + warp; i < N; i += nwarps) {
    const int beg = row_ptr[i], end = row_ptr[i + 1];
    float acc[VPL];
#pragma unroll
    for (int v = 0; v < VPL; ++v) acc[v] = 0.0f;
    float wsum = 0.0f;
    // neighbours handled by this slot: beg + slot + NS * m
    int k = beg + slot;
    int jn[U];
#pragma unroll
    for (int u = 0; u < U; ++u) jn[u] = (k + u * NS < end) ? __ldg(col + k + u * NS) : -1;
    for (; k < end; k += U * NS) {
      int j[U];
#pragma unroll
      for (int u = 0; u < U; ++u) j[u] = jn[u];
      const int kn = k + U * NS;
#pragma unroll
      for (int u = 0; u < U; ++u) jn[u] = (kn + u * NS < end) ? __ldg(col + kn + u * NS) : -1;
      float w[U];
      float x[U][VPL];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (j[u] >= 0) {
          w[u] = __ldg(dinv + j[u]);
          load_chunk(Tin + (int64_t)j[u] * D + chunk * VPL, x[u]);
        } else {
          w[u] = 0.0f;
#pragma unroll
          for (int v = 0; v < VPL; ++v) x[u][v] = 0.0f;
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        wsum += w[u];
#pragma unroll
        for (int v = 0; v < VPL; ++v) acc[v] = fmaf(w[u], x[u][v], acc[v]);
      }
    }
    // reduce-scatter over the slot bits (highest first), then all-reduce the rest
#pragma unroll
    for (int b = 0; b < RS; ++b) {
      const int sb = ilog2(NS) - 1 - b;
      constexpr int W0 = VPL;
      const int half = W0 >> (b + 1);
      const bool upper = (slot >> sb) & 1;
#pragma unroll
      for (int e = 0; e < (VPL >> (b + 1)); ++e) {
        const float send = upper ? acc[e] : acc[half + e];
        const float keep = upper ? acc[half + e] : acc[e];
        const float recv = __shfl_xor_sync(0xffffffffu, send, G << sb);
        acc[e] = keep + recv;
      }
    }
#pragma unroll
    for (int b = 0; b < AR; ++b) acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], G << b);
#pragma unroll
    for (int b = 0; b < ilog2(NS); ++b) wsum += __shfl_xor_sync(0xffffffffu, wsum, G << b);

    // epilogue on this lane's EPL columns
    const float di = __ldg(dinv + i);
    float ti[EPL];
    load_small<EPL>(Tin + i * D + cc, ti);
    float t[EPL];
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
      const float zi = (ti[e] - mu_e[e]) * is_e[e];
      const float agg = is_e[e] * fmaf(-mu_e[e], wsum, acc[e]);
      const float y = fmaf(theta, zi, alpha * di * agg);
      t[e] = tanhf(y);
    }
    if (owner) {
      store_small<EPL>(Tout + i * D + cc, t);
#pragma unroll
      for (int e = 0; e < EPL; ++e) {
        csum[e] += t[e];
        csq[e] = fmaf(t[e], t[e], csq[e]);
      }
    }
  }

  // ---- column statistics: CTA partial, then the last CTA reduces all partials
  if (owner) {
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
      s_red[warp][cc + e] = csum[e];
      s_red[warp][D + cc + e] = csq[e];
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < 2 * D; c += blockDim.x) {
    float a = 0.0f;
#pragma unroll
    for (int w = 0; w < kLayerWarps; ++w) a += s_red[w][c];
    partials[(int64_t)blockIdx.x * 2 * D + c] = a;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // fixed-order reduction of gridDim.x partials: R threads per value, then R-way combine
  constexpr int R0 = kLayerThreads / (2 * D) > 0 ? kLayerThreads / (2 * D) : 1;
  constexpr int R = R0 < kLayerWarps ? R0 : kLayerWarps;
  float* s_tot = &s_red[0][0];  // reuse: needs R * 2D <= kLayerWarps * 2D floats
  static_assert(R <= kLayerWarps, "reduction scratch too small");
  for (int t = threadIdx.x; t < R * 2 * D; t += blockDim.x) {
    const int c = t % (2 * D), r = t / (2 * D);
    float a = 0.0f;
    for (int b = r; b < (int)gridDim.x; b += R) a += __ldcg(partials + (int64_t)b * 2 * D + c);
    s_tot[r * 2 * D + c] = a;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < D; c += blockDim.x) {
    float sa = 0.0f, qa = 0.0f;
    for (int r = 0; r < R; ++r) {
      sa += s_tot[r * 2 * D + c];
      qa += s_tot[r * 2 * D + D + c];
    }
    const double n = (double)N;
    const double mean = (double)sa / n;
    const double denom = n - (double)ddof;
    double var = denom > 0.0 ? ((double)qa - (double)sa * mean) / denom : 0.0;
    if (!(var > 0.0)) var = 0.0;
    const double sd = sqrt(var);
    stats_out[c] = (float)mean;
    stats_out[D + c] = sd > 0.0 ? (float)(1.0 / sd) : 0.0f;
  }
  if (threadIdx.x == 0) *ticket = 0u;  // ready for the next launch
}

// ------------------------------------------------------------------ output
template <int D, typename S>
__global__ void k_output(const S* __restrict__ T, const float* __restrict__ stats, int32_t N, int row_l2,
                         float* __restrict__ out) {
  constexpr int VPL = Store<S>::VPL;
  constexpr int G = D / VPL;  // lanes per row
  constexpr int RPW = 32 / G;  // rows per warp pass
  const int lane = threadIdx.x & 31;
  const int chunk = lane % G, sub = lane / G;
  const int64_t warp_id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = warp_id * RPW; base < N; base += nw * RPW) {  // warp-uniform loop
    const int64_t i = base + sub;
    const bool ok = i < N;
    float v[VPL];
    if (ok) {
      load_chunk(T + i * D + chunk * VPL, v);
    } else {
#pragma unroll
      for (int e = 0; e < VPL; ++e) v[e] = 0.0f;
    }
    float o[VPL];
    float ss = 0.0f;
#pragma unroll
    for (int e = 0; e < VPL; ++e) {
      const int c = chunk * VPL + e;
      const float z = stats ? (v[e] - stats[c]) * stats[D + c] : v[e];
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
      float* p = out + i * D + chunk * VPL;
#pragma unroll
      for (int e = 0; e < VPL; e += 4)
        *reinterpret_cast<float4*>(p + e) = make_float4(o[e], o[e + 1], o[e + 2], o[e + 3]);
    }
  }
}

// ------------------------------------------------------------------ host dispatch
constexpr int kUnroll = 4;

template <int D, typename S>
struct LayerCfg {
  static int grid(int32_t N) {
    static int per_sm = 0;
    if (per_sm == 0) {
      int b = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_layer<D, S, kUnroll>, kLayerThreads, 0);
      per_sm = b > 0 ? b : 1;
    }
    int64_t want = ((int64_t)N + kLayerWarps - 1) / kLayerWarps;
    int64_t cap = (int64_t)per_sm * num_sms();
    return (int)std::max<int64_t>(1, std::min(want, cap));
  }
};

template <int D, typename S>
igp_status layer_launch(const igp_graph* g, const void* Tin, void* Tout, const float* st_in, float* partials,
                        float* st_out, unsigned* ticket, float alpha, float theta, int ddof, int grid,
                        cudaStream_t s) {
  k_layer<D, S, kUnroll><<<grid, kLayerThreads, 0, s>>>(g->row_ptr, g->col, g->dinv, (const S*)Tin, (S*)Tout, st_in,
                                                        partials, st_out, ticket, g->N, alpha, theta, ddof);
  return after_launch("k_layer");
}

template <int D, typename S>
igp_status output_launch(const void* T, const float* st, int32_t N, int row_l2, float* out, cudaStream_t s) {
  constexpr int G = D / Store<S>::VPL;
  int64_t threads = (int64_t)N * G;
  int blocks = (int)std::min<int64_t>((threads + 255) / 256, (int64_t)num_sms() * 16);
  k_output<D, S><<<std::max(blocks, 1), 256, 0, s>>>((const S*)T, st, N, row_l2, out);
  return after_launch("k_output");
}

struct Ops {
  int (*grid)(int32_t);
  igp_status (*layer)(const igp_graph*, const void*, void*, const float*, float*, float*, unsigned*, float, float,
                      int, int, cudaStream_t);
  igp_status (*output)(const void*, const float*, int32_t, int, float*, cudaStream_t);
};

template <int D, typename S>
Ops ops_for() {
  return Ops{&LayerCfg<D, S>::grid, &layer_launch<D, S>, &output_launch<D, S>};
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

}  // namespace

igp_status compute_dinv(igp_graph* g, double tau, double eps, cudaStream_t s, Profile* prof) {
  if (g->dinv_valid && g->dinv_tau == tau && g->dinv_eps == eps) return IGP_OK;
  if (!g->dinv) {
    void* p = nullptr;
    IGP_TRY(dev_alloc(&p, (size_t)g->N * sizeof(float), s));
    g->dinv = (float*)p;
  }
  PhaseTimer pt(prof, IGP_PHASE_DINV, s);
  int blocks = (int)std::min<int64_t>(((int64_t)g->N + 255) / 256, (int64_t)num_sms() * 8);
  k_dinv<<<std::max(blocks, 1), 256, 0, s>>>(g->row_ptr, g->N, tau, eps, g->dinv);
  IGP_TRY(after_launch("k_dinv"));
  g->dinv_valid = true;
  g->dinv_tau = tau;
  g->dinv_eps = eps;
  return IGP_OK;
}

igp_status launch_theta(uint64_t seed, int32_t N, int32_t d, float xs, int storage, void* out, cudaStream_t s) {
  int64_t total = (int64_t)N * (d / 8);
  int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms() * 16);
  blocks = std::max(blocks, 1);
  if (storage == IGP_STORE_BF16)
    k_theta<__nv_bfloat16><<<blocks, 256, 0, s>>>(seed, N, d, xs, (__nv_bfloat16*)out);
  else
    k_theta<float><<<blocks, 256, 0, s>>>(seed, N, d, xs, (float*)out);
  return after_launch("k_theta");
}

igp_status run_ffp(igp_graph* g, double tau, int32_t L, int32_t d, uint64_t seed, float* out_dev,
                   const igp_embed_opts& o, cudaStream_t s) {
  Profile* prof = o.profile ? &o.profile->prof : nullptr;
  Ops ops;
  if (!get_ops(d, o.storage, &ops)) {
    set_error("igp_embed: d=%d unsupported (8, 16, 32, 64, 128)", d);
    return IGP_E_INVAL;
  }
  IGP_TRY(compute_dinv(g, tau, o.eps, s, prof));
  const int32_t N = g->N;
  const size_t sb = o.storage == IGP_STORE_BF16 ? 2 : 4;
  const int grid = ops.grid(N);
  // workspace: T0 | T1 | stats[2][2d] | partials[grid][2d] | ticket
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t bT = al((size_t)N * d * sb);
  const size_t bS = al(2 * 2 * (size_t)d * sizeof(float));
  const size_t bP = al((size_t)grid * 2 * d * sizeof(float));
  const size_t need = 2 * bT + bS + bP + 256;
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
  float* partials = (float*)(base + 2 * bT + bS);
  unsigned* ticket = (unsigned*)(base + 2 * bT + bS + bP);
  IGP_TRY(cudaMemsetAsync(ticket, 0, sizeof(unsigned), s) == cudaSuccess ? IGP_OK : IGP_E_CUDA);

  const double xs = o.x_scale > 0 ? o.x_scale : 1.0 / std::sqrt((double)d);
  const void* cur = o.x_in;
  if (!cur) {
    PhaseTimer pt(prof, IGP_PHASE_THETA, s);
    IGP_TRY(launch_theta(seed, N, d, (float)xs, o.storage, T0, s));
    cur = T0;
  }
  const float* st_prev = nullptr;
  for (int32_t l = 1; l <= L; ++l) {
    void* dst = (cur == T0) ? T1 : T0;
    float* st = stats + (size_t)(l & 1) * 2 * d;
    PhaseTimer pt(prof, IGP_PHASE_LAYER, s);
    IGP_TRY(ops.layer(g, cur, dst, st_prev, partials, st, ticket, (float)o.alpha, (float)o.theta, o.znorm_ddof,
                      grid, s));
    cur = dst;
    st_prev = st;
  }
  PhaseTimer pt(prof, IGP_PHASE_OUTPUT, s);
  return ops.output(cur, st_prev, N, o.out_row_l2, out_dev, s);
}

}  // namespace igp
