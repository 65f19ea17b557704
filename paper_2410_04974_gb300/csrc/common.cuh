// Shared device-side definitions of the sixdgs library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sixdgs.h"

namespace sixdgs {

// ---- constants of the inherited 3DGS rasteriser (6DGS section 4.4) --------
constexpr float kDilation = 0.3f;       // px^2 added to the 2D covariance diagonal
constexpr float kRadiusSigmas = 3.0f;   // screen extent in standard deviations
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;
constexpr float kFrustumGuard = 1.3f;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
// log2(1/255): an entry is skipped when its log2-alpha q is below this
constexpr float kQMin = -7.994353436858858f;
// log2(0.99): alpha is clamped to 0.99 above this
constexpr float kQMax = -0.014499569695115089f;

constexpr int kMaxShCoeffs = 16;

// Per-camera record stored in the workspace (128 bytes).
struct __align__(16) CamRec {
  float r[9];        // world-to-camera rotation, row-major
  float t[3];        // world-to-camera translation
  float campos[3];
  float fx, fy, cx, cy;
  float znear;
  float limx, limy;  // frustum guard on x/z, y/z for the Jacobian
  int32_t width, height;
  int32_t tiles_x, tiles_y;
  int32_t tile_offset;   // first global tile id of this camera
  int64_t pixel_base;    // pixels of all earlier cameras; image floats start at 3 * pixel_base
  int32_t pad[2];
};
static_assert(sizeof(CamRec) == 128, "CamRec must stay 128 bytes");

// Record of one (view, Gaussian) pair, consumed by the blend (48 bytes).
//  a = (u, v, qa, qb), b = (qc, lo, r, g), c = (b, hx, hy, depth)
// with q(dx, dy) = qa dx^2 + qb dx dy + qc dy^2 + lo = log2(alpha_cond) +
// log2(e) * (-1/2 Delta^T conic Delta), Delta = (u - px, v - py), and
// (hx, hy) the half-extents of the box around (u, v) outside which
// q < log2(1/255) (the entry is skipped at every pixel there).
struct __align__(16) PairRec {
  float4 a, b, c;
};

__device__ __forceinline__ void raise_status(int32_t* status, int code) {
  if (status) atomicOr(status, 1 << code);
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + __expf(-x)); }

// q of one list entry (a, b) at the pixel centre whose negation is npix
// = (-px, -py); d = (u - px, v - py) comes out as one packed subtraction.
// Explicit rounding intrinsics keep the forward and backward walks
// bit-identical.
__device__ __forceinline__ float entry_q(const float4& a, const float4& b, float2 npix, float2& d) {
  d = __fadd2_rn(make_float2(a.x, a.y), npix);
  const float t1 = __fmaf_rn(a.z, d.x, __fmul_rn(a.w, d.y));   // qa dx + qb dy
  const float t2 = __fmaf_rn(__fmul_rn(b.x, d.y), d.y, b.y);   // qc dy^2 + lo
  return __fmaf_rn(t1, d.x, t2);
}

// Decoupled look-back status words: 2-bit flag in the top bits.
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kFlagMask = 3u << 30;
constexpr uint32_t kValMask = ~kFlagMask;

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) {
  return *reinterpret_cast<const volatile uint32_t*>(p);
}
__device__ __forceinline__ void st_volatile(uint32_t* p, uint32_t v) {
  *reinterpret_cast<volatile uint32_t*>(p) = v;
}

__device__ __forceinline__ uint32_t lane_id() {
  uint32_t l;
  asm volatile("mov.u32 %0, %%laneid;" : "=r"(l));
  return l;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace sixdgs
