// View-independent part of the 6D slice (6DGS section 3.1 and Algorithm 1
// steps 1-3): Cholesky activation, covariance blocks, Sigma_d^-1, the
// regression matrix A = Sigma_pd Sigma_d^-1 and the Schur complement
// Sigma_cond = Sigma_p - A Sigma_pd^T (Eq. sigma).
#pragma once

#include "common.cuh"
#include "mat3.cuh"

namespace sixdgs {

// L, Sigma blocks and the conditional quantities of one Gaussian.
struct CondState {
  M3 A;        // Sigma_pd Sigma_d^-1
  M3 Sdi;      // Sigma_d^-1
  M3 Sc;       // Sigma_cond
  float alpha; // sigmoid(opacity logit)
};

// L from the 21 raw planes; plane(p) returns raw plane p of this Gaussian.
template <typename Plane>
__device__ __forceinline__ void cholesky_from(Plane plane, float L[6][6]) {
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) L[i][j] = 0.f;
#pragma unroll
  for (int i = 0; i < 6; ++i) L[i][i] = __expf(plane(i));
  int k = 6;
#pragma unroll
  for (int i = 1; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < i; ++j) {
      // 2 sigmoid(x) - 1, evaluated as the identical function tanh(x / 2):
      // the subtraction form loses the relative accuracy of small entries
      // (|v| ~ 1e-3 keeps only ~3 significant digits in FP32), tanhf keeps
      // it to a few ulps.
      L[i][j] = tanhf(0.5f * plane(k++));
    }
}

__device__ __forceinline__ void load_cholesky(const float* __restrict__ l_raw, int64_t n, int64_t g,
                                              float L[6][6]) {
  cholesky_from([&](int p) { return __ldg(l_raw + p * n + g); }, L);
}

// Sigma_p = Lpp Lpp^T, Sigma_pd = Lpp Ldp^T, Sigma_d = Ldp Ldp^T + Ldd Ldd^T.
__device__ __forceinline__ void sigma_blocks(const float L[6][6], M3& Sp, M3& Spd, M3& Sd) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float sp = 0.f, spd = 0.f, sd = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        sp += L[i][k] * L[j][k];
        spd += L[i][k] * L[3 + j][k];
        sd += L[3 + i][k] * L[3 + j][k] + L[3 + i][3 + k] * L[3 + j][3 + k];
      }
      Sp(i, j) = sp;
      Spd(i, j) = spd;
      Sd(i, j) = sd;
    }
}

template <typename Plane>
__device__ __forceinline__ bool condition_from(Plane plane, float logit, CondState& s) {
  float L[6][6];
  cholesky_from(plane, L);
  M3 Sp, Spd, Sd;
  sigma_blocks(L, Sp, Spd, Sd);
  if (!spd_inverse(Sd, s.Sdi)) return false;
  s.A = mul(Spd, s.Sdi);
  s.Sc = sub(Sp, mul_bt(s.A, Spd));
  s.alpha = sigmoidf_(logit);
  return true;
}

__device__ __forceinline__ bool condition_gaussian(const float* __restrict__ l_raw, float logit,
                                                   int64_t n, int64_t g, CondState& s) {
  return condition_from([&](int p) { return __ldg(l_raw + p * n + g); }, logit, s);
}

}  // namespace sixdgs
