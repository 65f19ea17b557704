// Real orthonormal spherical harmonics up to degree 3 (6DGS section 4.2).
//
// Basis index k = l*l + l + m, no Condon-Shortley phase.  For a unit
// direction (x, y, z) the functions are polynomials; the constants are the
// normalisations sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (times sqrt(2) for
// m != 0) multiplied into each polynomial:
//   C0   = 1/(2 sqrt(pi))         C1  = sqrt(3/(4 pi))
//   C2a  = sqrt(15/(4 pi))        C20 = sqrt(5/(16 pi))   C22 = sqrt(15/(16 pi))
//   C33  = sqrt(35/(32 pi))       C32b = sqrt(105/(4 pi)) C31 = sqrt(21/(32 pi))
//   C30  = sqrt(7/(16 pi))        C32a = sqrt(105/(16 pi))
#pragma once

namespace sixdgs {

constexpr float kC0 = 0.28209479177387814f;
constexpr float kC1 = 0.4886025119029199f;
constexpr float kC2a = 1.0925484305920792f;
constexpr float kC20 = 0.31539156525252005f;
constexpr float kC22 = 0.5462742152960396f;
constexpr float kC33 = 0.5900435899266435f;
constexpr float kC32b = 2.890611442640554f;
constexpr float kC31 = 0.4570457994644658f;
constexpr float kC30 = 0.3731763325901154f;
constexpr float kC32a = 1.445305721320277f;

// Y[k] for k < (deg+1)^2 (entries beyond are left untouched).
__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float* Y) {
  Y[0] = kC0;
  if (deg < 1) return;
  Y[1] = kC1 * y;
  Y[2] = kC1 * z;
  Y[3] = kC1 * x;
  if (deg < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = kC2a * x * y;
  Y[5] = kC2a * y * z;
  Y[6] = kC20 * (3.f * zz - 1.f);
  Y[7] = kC2a * x * z;
  Y[8] = kC22 * (xx - yy);
  if (deg < 3) return;
  Y[9] = kC33 * y * (3.f * xx - yy);
  Y[10] = kC32b * x * y * z;
  Y[11] = kC31 * y * (5.f * zz - 1.f);
  Y[12] = kC30 * z * (5.f * zz - 3.f);
  Y[13] = kC31 * x * (5.f * zz - 1.f);
  Y[14] = kC32a * z * (xx - yy);
  Y[15] = kC33 * x * (xx - 3.f * yy);
}

// g = sum_k w[k] * grad Y_k(x, y, z) (gradient of the polynomial form).
__device__ __forceinline__ void sh_grad(int deg, float x, float y, float z, const float* w,
                                        float* g) {
  float gx = 0.f, gy = 0.f, gz = 0.f;
  if (deg >= 1) {
    gy += kC1 * w[1];
    gz += kC1 * w[2];
    gx += kC1 * w[3];
  }
  if (deg >= 2) {
    gx += kC2a * (y * w[4] + z * w[7]) + 2.f * kC22 * x * w[8];
    gy += kC2a * (x * w[4] + z * w[5]) - 2.f * kC22 * y * w[8];
    gz += kC2a * (y * w[5] + x * w[7]) + 6.f * kC20 * z * w[6];
  }
  if (deg >= 3) {
    const float xx = x * x, yy = y * y, zz = z * z;
    gx += kC33 * 6.f * x * y * w[9] + kC32b * y * z * w[10] + kC31 * (5.f * zz - 1.f) * w[13] +
          kC32a * 2.f * x * z * w[14] + kC33 * 3.f * (xx - yy) * w[15];
    gy += kC33 * 3.f * (xx - yy) * w[9] + kC32b * x * z * w[10] + kC31 * (5.f * zz - 1.f) * w[11] -
          kC32a * 2.f * y * z * w[14] - kC33 * 6.f * x * y * w[15];
    gz += kC32b * x * y * w[10] + kC31 * 10.f * y * z * w[11] + kC30 * (15.f * zz - 3.f) * w[12] +
          kC31 * 10.f * x * z * w[13] + kC32a * (xx - yy) * w[14];
  }
  g[0] = gx;
  g[1] = gy;
  g[2] = gz;
}

}  // namespace sixdgs
