// Small fixed-size matrix helpers (row-major 3x3 in float[9]).
#pragma once

namespace sixdgs {

struct M3 {
  float m[9];
  __device__ __forceinline__ float& operator()(int i, int j) { return m[i * 3 + j]; }
  __device__ __forceinline__ float operator()(int i, int j) const { return m[i * 3 + j]; }
};

__device__ __forceinline__ M3 mul(const M3& a, const M3& b) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      c(i, j) = a(i, 0) * b(0, j) + a(i, 1) * b(1, j) + a(i, 2) * b(2, j);
  return c;
}

// a * b^T
__device__ __forceinline__ M3 mul_bt(const M3& a, const M3& b) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      c(i, j) = a(i, 0) * b(j, 0) + a(i, 1) * b(j, 1) + a(i, 2) * b(j, 2);
  return c;
}

// a^T * b
__device__ __forceinline__ M3 mul_at(const M3& a, const M3& b) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      c(i, j) = a(0, i) * b(0, j) + a(1, i) * b(1, j) + a(2, i) * b(2, j);
  return c;
}

__device__ __forceinline__ M3 add(const M3& a, const M3& b) {
  M3 c;
#pragma unroll
  for (int k = 0; k < 9; ++k) c.m[k] = a.m[k] + b.m[k];
  return c;
}

__device__ __forceinline__ M3 sub(const M3& a, const M3& b) {
  M3 c;
#pragma unroll
  for (int k = 0; k < 9; ++k) c.m[k] = a.m[k] - b.m[k];
  return c;
}

__device__ __forceinline__ M3 transpose(const M3& a) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) c(i, j) = a(j, i);
  return c;
}

__device__ __forceinline__ M3 zero3() {
  M3 c;
#pragma unroll
  for (int k = 0; k < 9; ++k) c.m[k] = 0.f;
  return c;
}

__device__ __forceinline__ void mat_vec(const M3& a, const float* x, float* y) {
#pragma unroll
  for (int i = 0; i < 3; ++i) y[i] = a(i, 0) * x[0] + a(i, 1) * x[1] + a(i, 2) * x[2];
}

__device__ __forceinline__ void mat_t_vec(const M3& a, const float* x, float* y) {
#pragma unroll
  for (int i = 0; i < 3; ++i) y[i] = a(0, i) * x[0] + a(1, i) * x[1] + a(2, i) * x[2];
}

// Inverse of a symmetric positive definite 3x3 matrix through its Cholesky
// factor C (S = C C^T, S^-1 = C^-T C^-1).  Returns false when S is not
// numerically positive definite.
__device__ __forceinline__ bool spd_inverse(const M3& s, M3& inv) {
  float c00 = s(0, 0);
  if (!(c00 > 0.f)) return false;
  c00 = sqrtf(c00);
  float c10 = s(1, 0) / c00, c20 = s(2, 0) / c00;
  float d11 = s(1, 1) - c10 * c10;
  if (!(d11 > 0.f)) return false;
  float c11 = sqrtf(d11);
  float c21 = (s(2, 1) - c20 * c10) / c11;
  float d22 = s(2, 2) - c20 * c20 - c21 * c21;
  if (!(d22 > 0.f)) return false;
  float c22 = sqrtf(d22);
  // M = C^-1 (lower triangular)
  float m00 = 1.f / c00, m11 = 1.f / c11, m22 = 1.f / c22;
  float m10 = -c10 * m00 * m11;
  float m21 = -c21 * m11 * m22;
  float m20 = -(c20 * m00 + c21 * m10) * m22;
  // S^-1 = M^T M
  inv(0, 0) = m00 * m00 + m10 * m10 + m20 * m20;
  inv(0, 1) = inv(1, 0) = m10 * m11 + m20 * m21;
  inv(0, 2) = inv(2, 0) = m20 * m22;
  inv(1, 1) = m11 * m11 + m21 * m21;
  inv(1, 2) = inv(2, 1) = m21 * m22;
  inv(2, 2) = m22 * m22;
  return true;
}

}  // namespace sixdgs
