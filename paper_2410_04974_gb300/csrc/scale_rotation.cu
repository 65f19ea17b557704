// Scale and rotation of every conditional 3D Gaussian (6DGS section 4.3,
// Algorithm 1 steps 4-5): Sigma_cond = U D U^T, R = U, S = sqrt(diag D),
// with the third column of R multiplied by sign(det R) so that R is a
// proper rotation.  Needed by adaptive density control (clone / split),
// which the paper runs every ~100 iterations.
//
// One thread per Gaussian: Sigma_cond from the raw parameters (the same
// helper as the projection), then a cyclic Jacobi eigen-solve of the
// symmetric 3x3 matrix (each rotation zeroes one off-diagonal entry;
// Golub and Van Loan, "Matrix Computations", section 8.5), eigenvalues
// sorted in decreasing order as a singular value decomposition returns them.
#include "common.cuh"
#include "cond.cuh"
#include "kernels.cuh"
#include "mat3.cuh"

namespace sixdgs {

// One Jacobi rotation in the (p, q) plane of symmetric A, accumulated into V.
__device__ __forceinline__ void jacobi_rotate(float A[3][3], float V[3][3], int p, int q) {
  const float apq = A[p][q];
  if (fabsf(apq) <= 1e-30f) return;
  const float theta = (A[q][q] - A[p][p]) / (2.f * apq);
  const float t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
  const float c = rsqrtf(t * t + 1.f), s = t * c;
  // A <- J^T A J with J the rotation in (p, q)
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float akp = A[k][p], akq = A[k][q];
    A[k][p] = c * akp - s * akq;
    A[k][q] = s * akp + c * akq;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float apk = A[p][k], aqk = A[q][k];
    A[p][k] = c * apk - s * aqk;
    A[q][k] = s * apk + c * aqk;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float vkp = V[k][p], vkq = V[k][q];
    V[k][p] = c * vkp - s * vkq;
    V[k][q] = s * vkp + c * vkq;
  }
}

__global__ void __launch_bounds__(128) scale_rotation_kernel(ScaleRotationArgs a) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.n) return;
  const int64_t n = a.n;
  CondState cs;
  const bool ok = condition_gaussian(a.l_raw, 0.f, n, g, cs);
  float A[3][3], V[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      A[i][j] = 0.5f * (cs.Sc(i, j) + cs.Sc(j, i));
      V[i][j] = i == j ? 1.f : 0.f;
    }
  // Cyclic sweeps until the off-diagonal mass is at FP32 rounding level of
  // the diagonal (about 3-4 sweeps; at most 8).  A residual off-diagonal e
  // moves an eigenvalue by O(e^2 / gap) and an axis by O(e / gap).
  for (int sweep = 0; sweep < 8; ++sweep) {
    const float off = fabsf(A[0][1]) + fabsf(A[0][2]) + fabsf(A[1][2]);
    const float diag = fabsf(A[0][0]) + fabsf(A[1][1]) + fabsf(A[2][2]);
    if (off <= 6e-8f * diag) break;
    jacobi_rotate(A, V, 0, 1);
    jacobi_rotate(A, V, 0, 2);
    jacobi_rotate(A, V, 1, 2);
  }
  // eigenvalues in decreasing order (columns of V permuted alike)
  float d[3] = {A[0][0], A[1][1], A[2][2]};
  int o[3] = {0, 1, 2};
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2 - i; ++j)
      if (d[o[j]] < d[o[j + 1]]) {
        const int t = o[j];
        o[j] = o[j + 1];
        o[j + 1] = t;
      }
  float R[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) R[i][j] = V[i][o[j]];
  const float det = R[0][0] * (R[1][1] * R[2][2] - R[1][2] * R[2][1]) -
                    R[0][1] * (R[1][0] * R[2][2] - R[1][2] * R[2][0]) +
                    R[0][2] * (R[1][0] * R[2][1] - R[1][1] * R[2][0]);
  const float sgn = det < 0.f ? -1.f : 1.f;
#pragma unroll
  for (int i = 0; i < 3; ++i) R[i][2] *= sgn;
  const bool finite = ok && isfinite(det);
  if (!finite) raise_status(a.status, SIXDGS_ERR_NONFINITE);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) a.rotation[(i * 3 + j) * n + g] = finite ? R[i][j] : 0.f;
#pragma unroll
  for (int j = 0; j < 3; ++j) a.scale[j * n + g] = finite ? sqrtf(fmaxf(d[o[j]], 0.f)) : 0.f;
}

void launch_scale_rotation(const ScaleRotationArgs& a, cudaStream_t stream) {
  if (a.n == 0) return;
  scale_rotation_kernel<<<(unsigned)((a.n + 127) / 128), 128, 0, stream>>>(a);
}

}  // namespace sixdgs
