/*
 * Plain FP64 reference of InfraredGP's feed-forward propagation in C, run on all host cores.
 *
 * TEST INFRASTRUCTURE ONLY: the same computation as oracle/fp64.py's ffp(), written as loops so
 * that it can be timed on every host core (OpenMP over rows) as the CPU baseline next to the GPU.
 * It shares no code with the CUDA library. Steps (Alg. 1 up to its clustering step):
 *   1. deg_i = row length of the CSR; D_tau by Eq. 1 for tau < 0 (deg - min(|tau|, deg - eps)),
 *      deg + tau otherwise (Sec. I); dinv_i = 1 / sqrt(D_tau_i), 0 where D_tau_i = 0;
 *   2. Z = X (the random input Theta);
 *   3. L times (Eq. 3 with the Eq. 2 filter, then Eq. 4):
 *        Y_i = theta Z_i + alpha dinv_i sum_{j in N(i)} dinv_j Z_j   (neighbours in CSR order)
 *        T = tanh(Y);  per column: mean, then std with divisor N - ddof (two passes);
 *        Z = (T - mean) / std, 0 in a column whose std is 0;
 *   4. out = sigmoid(Z) = 1 / (1 + exp(-Z)).
 * Column sums are taken per thread over fixed row blocks and then added in block order, so the
 * result does not depend on the number of threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ROW_BLOCK 4096

int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* 0 on success, 1 on an allocation failure, 2 on a bad argument. */
int oracle_ffp(int64_t N, const int64_t* row_ptr, const int64_t* col, const double* X, int32_t d, double tau,
               int32_t L, double alpha, double theta, double eps, int32_t ddof, int32_t threads, double* out) {
  if (N < 1 || d < 1 || L < 0 || !row_ptr || !X || !out) return 2;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#endif
  const int64_t nblk = (N + ROW_BLOCK - 1) / ROW_BLOCK;
  double* dinv = (double*)malloc(sizeof(double) * (size_t)N);
  double* Z = (double*)malloc(sizeof(double) * (size_t)N * d);
  double* T = (double*)malloc(sizeof(double) * (size_t)N * d);
  double* part = (double*)malloc(sizeof(double) * (size_t)nblk * d);
  double* mu = (double*)malloc(sizeof(double) * (size_t)d);
  double* sd = (double*)malloc(sizeof(double) * (size_t)d);
  if (!dinv || !Z || !T || !part || !mu || !sd) {
    free(dinv); free(Z); free(T); free(part); free(mu); free(sd);
    return 1;
  }
  /* 1. degree correction */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; ++i) {
    const double deg = (double)(row_ptr[i + 1] - row_ptr[i]);
    const double dt = tau < 0.0 ? deg - fmin(fabs(tau), deg - eps) : deg + tau;
    dinv[i] = dt > 0.0 ? 1.0 / sqrt(dt) : 0.0;
  }
  /* 2. Z = Theta */
  memcpy(Z, X, sizeof(double) * (size_t)N * d);
  for (int32_t l = 0; l < L; ++l) {
    /* 3a. convolution and tanh */
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < N; ++i) {
      double* t = T + i * d;
      for (int32_t c = 0; c < d; ++c) t[c] = 0.0;
      for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
        const int64_t j = col[k];
        const double w = dinv[j];
        const double* z = Z + j * d;
        for (int32_t c = 0; c < d; ++c) t[c] += w * z[c];
      }
      const double* zi = Z + i * d;
      for (int32_t c = 0; c < d; ++c) t[c] = tanh(theta * zi[c] + alpha * dinv[i] * t[c]);
    }
    /* 3b. column means (per block, then blocks in order) */
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nblk; ++b) {
      double* p = part + b * d;
      for (int32_t c = 0; c < d; ++c) p[c] = 0.0;
      const int64_t e = (b + 1) * ROW_BLOCK < N ? (b + 1) * ROW_BLOCK : N;
      for (int64_t i = b * ROW_BLOCK; i < e; ++i)
        for (int32_t c = 0; c < d; ++c) p[c] += T[i * d + c];
    }
    for (int32_t c = 0; c < d; ++c) {
      double s = 0.0;
      for (int64_t b = 0; b < nblk; ++b) s += part[b * d + c];
      mu[c] = s / (double)N;
    }
    /* 3c. standard deviations, second pass */
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nblk; ++b) {
      double* p = part + b * d;
      for (int32_t c = 0; c < d; ++c) p[c] = 0.0;
      const int64_t e = (b + 1) * ROW_BLOCK < N ? (b + 1) * ROW_BLOCK : N;
      for (int64_t i = b * ROW_BLOCK; i < e; ++i)
        for (int32_t c = 0; c < d; ++c) {
          const double v = T[i * d + c] - mu[c];
          p[c] += v * v;
        }
    }
    const double denom = (double)N - (double)ddof;
    for (int32_t c = 0; c < d; ++c) {
      double s = 0.0;
      for (int64_t b = 0; b < nblk; ++b) s += part[b * d + c];
      sd[c] = denom > 0.0 ? sqrt(s / denom) : 0.0;
    }
    /* 3d. ZNorm */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i)
      for (int32_t c = 0; c < d; ++c) Z[i * d + c] = sd[c] > 0.0 ? (T[i * d + c] - mu[c]) / sd[c] : 0.0;
  }
  /* 4. output */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N * d; ++i) out[i] = 1.0 / (1.0 + exp(-Z[i]));
  free(dinv); free(Z); free(T); free(part); free(mu); free(sd);
  return 0;
}
