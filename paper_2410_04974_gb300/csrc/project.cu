// Stage 1: slice every 6D Gaussian at each camera's view direction, colour
// it and project it (6DGS section 3.2 Eqs. mu / sigma / alpha with Eq.
// pdfv2, section 4.2, and the 3DGS projection kept by section 4.4).
//
// One thread per Gaussian.  The view-independent part (Cholesky factor,
// Sigma_d^-1, A = Sigma_pd Sigma_d^-1, Sigma_cond; Algorithm 1 steps 1-3) is
// computed once in registers and reused for every camera, so the 304 bytes
// of parameters of a Gaussian are read from HBM once per frame however many
// cameras there are.  Loads are coalesced structure-of-arrays planes.
//
// Inference (the Algorithm 1 caption: the view-independent terms are
// computed once when the scene is fixed): cond_cache_kernel stores that
// state once, and the cached variant of the projection loads it instead of
// recomputing it; every later step is the same code on the same values, so
// the two variants give bit-identical records.
#include "common.cuh"
#include "kernels.cuh"
#include "cond.cuh"
#include "mat3.cuh"
#include "sh.cuh"

namespace sixdgs {

// Cached view-independent state (written by cond_cache_kernel): plane k of
// A (k < 9), the upper triangle of the symmetric Sigma_d^-1 (9..14), plane k
// of Sigma_cond (15..23) and alpha (24; NaN where Sigma_d was not
// numerically positive definite).
__device__ __forceinline__ void load_cond_cache(const float* __restrict__ c, int64_t n, int64_t g,
                                                CondState& cs) {
#pragma unroll
  for (int k = 0; k < 9; ++k) cs.A.m[k] = __ldg(c + k * n + g);
  cs.Sdi(0, 0) = __ldg(c + 9 * n + g);
  cs.Sdi(0, 1) = cs.Sdi(1, 0) = __ldg(c + 10 * n + g);
  cs.Sdi(0, 2) = cs.Sdi(2, 0) = __ldg(c + 11 * n + g);
  cs.Sdi(1, 1) = __ldg(c + 12 * n + g);
  cs.Sdi(1, 2) = cs.Sdi(2, 1) = __ldg(c + 13 * n + g);
  cs.Sdi(2, 2) = __ldg(c + 14 * n + g);
#pragma unroll
  for (int k = 0; k < 9; ++k) cs.Sc.m[k] = __ldg(c + (15 + k) * n + g);
  cs.alpha = __ldg(c + 24 * n + g);
}

__global__ void __launch_bounds__(128) cond_cache_kernel(CondCacheArgs a) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.n) return;
  const int64_t n = a.n;
  CondState cs;
  const bool ok = condition_gaussian(a.l_raw, __ldg(a.opacity_logit + g), n, g, cs);
  float* c = a.cache;
#pragma unroll
  for (int k = 0; k < 9; ++k) c[k * n + g] = cs.A.m[k];
  c[9 * n + g] = cs.Sdi(0, 0);
  c[10 * n + g] = cs.Sdi(0, 1);
  c[11 * n + g] = cs.Sdi(0, 2);
  c[12 * n + g] = cs.Sdi(1, 1);
  c[13 * n + g] = cs.Sdi(1, 2);
  c[14 * n + g] = cs.Sdi(2, 2);
#pragma unroll
  for (int k = 0; k < 9; ++k) c[(15 + k) * n + g] = cs.Sc.m[k];
  c[24 * n + g] = ok ? cs.alpha : __int_as_float(0x7fc00000);
}

template <bool kCached>
// 4 CTAs per SM (128 registers, a few spilled) instead of 3: 0.115 -> 0.105 ms on
// the 300k / 8 x 800^2 frame.
__global__ void __launch_bounds__(128, 4) project_fwd_kernel(ProjectArgs a) {
  extern __shared__ CamRec s_cams[];
  for (int i = threadIdx.x; i < a.n_cams; i += blockDim.x) s_cams[i] = a.cams[i];
  __syncthreads();
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.n) return;
  const int64_t n = a.n;

  float mp[3], md[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    mp[i] = __ldg(a.mu_p + i * n + g);
    md[i] = __ldg(a.mu_d + i * n + g);
  }
  CondState cs;
  bool ok = true;
  if constexpr (kCached)
    load_cond_cache(a.cond_cache, n, g, cs);
  else
    ok = condition_gaussian(a.l_raw, __ldg(a.opacity_logit + g), n, g, cs);
  // lambda_opa: global, or per Gaussian as sigmoid(raw) (section 4.2)
  const float lam = a.lambda_raw ? sigmoidf_(__ldg(a.lambda_raw + g)) : a.lambda_opa;
  const int K = (a.sh_degree + 1) * (a.sh_degree + 1);
  float beta[kMaxShCoeffs][3];
#pragma unroll
  for (int k = 0; k < kMaxShCoeffs; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) beta[k][c] = (k < K) ? __ldg(a.sh + (k * 3 + c) * n + g) : 0.f;
  if (ok) {
#pragma unroll
    for (int k = 0; k < 9; ++k)
      ok = ok && isfinite(cs.A.m[k]) && isfinite(cs.Sdi.m[k]) && isfinite(cs.Sc.m[k]);
    ok = ok && isfinite(mp[0]) && isfinite(mp[1]) && isfinite(mp[2]) && isfinite(md[0]) &&
         isfinite(md[1]) && isfinite(md[2]) && isfinite(cs.alpha) && isfinite(lam);
  }
  if (!ok) raise_status(a.status, SIXDGS_ERR_NONFINITE);

  for (int v = 0; v < a.n_cams; ++v) {
    const CamRec& cam = s_cams[v];
    const int64_t pair = (int64_t)v * n + g;
    uint32_t ntiles = 0;
    if (ok) {
      // ---- slice (Eq. mu, Eq. pdfv2, Eq. alpha) ----
      float dv[3] = {mp[0] - cam.campos[0], mp[1] - cam.campos[1], mp[2] - cam.campos[2]};
      float inv_len = rsqrtf(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
      float d[3] = {dv[0] * inv_len, dv[1] * inv_len, dv[2] * inv_len};
      float delta[3] = {d[0] - md[0], d[1] - md[1], d[2] - md[2]};
      float Ad[3], Sd_delta[3];
      mat_vec(cs.A, delta, Ad);
      mat_vec(cs.Sdi, delta, Sd_delta);
      float mc[3] = {mp[0] + Ad[0], mp[1] + Ad[1], mp[2] + Ad[2]};
      float D = delta[0] * Sd_delta[0] + delta[1] * Sd_delta[1] + delta[2] * Sd_delta[2];
      float alpha_cond = cs.alpha * __expf(-lam * D);
      // ---- projection (section 4.4, EWA) ----
      float t[3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
        t[i] = cam.r[i * 3] * mc[0] + cam.r[i * 3 + 1] * mc[1] + cam.r[i * 3 + 2] * mc[2] + cam.t[i];
      bool vis = (alpha_cond >= kAlphaMin) && (t[2] > cam.znear);
      if (vis) {
        float iz = 1.f / t[2];
        float rx = fminf(cam.limx, fmaxf(-cam.limx, t[0] * iz));
        float ry = fminf(cam.limy, fmaxf(-cam.limy, t[1] * iz));
        float j00 = cam.fx * iz, j02 = -cam.fx * rx * iz;
        float j11 = cam.fy * iz, j12 = -cam.fy * ry * iz;
        // T = J R (2x3)
        float T0[3], T1[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          T0[j] = j00 * cam.r[j] + j02 * cam.r[6 + j];
          T1[j] = j11 * cam.r[3 + j] + j12 * cam.r[6 + j];
        }
        float U0[3], U1[3];
        mat_t_vec(cs.Sc, T0, U0);  // Sigma_cond symmetric: (T0 Sc)_j
        mat_t_vec(cs.Sc, T1, U1);
        float ca = U0[0] * T0[0] + U0[1] * T0[1] + U0[2] * T0[2] + kDilation;
        float cb = U0[0] * T1[0] + U0[1] * T1[1] + U0[2] * T1[2];
        float cc = U1[0] * T1[0] + U1[1] * T1[1] + U1[2] * T1[2] + kDilation;
        float det = ca * cc - cb * cb;
        vis = det > 0.f;
        if (vis) {
          float idet = 1.f / det;
          float con_a = cc * idet, con_b = -cb * idet, con_c = ca * idet;
          float mid = 0.5f * (ca + cc);
          float lam = mid + sqrtf(fmaxf(mid * mid - det, 0.f));
          float radius = kRadiusSigmas * sqrtf(lam);
          float u = cam.fx * t[0] * iz + cam.cx;
          float w = cam.fy * t[1] * iz + cam.cy;
          // Bounding box of the alpha >= 1/255 ellipse {Delta^T conic Delta <=
          // 2 ln(255 alpha_cond)}: half-extents sqrt(L2 * Sigma_2D,ii), widened
          // by a margin far above FP32 rounding, so that culling with it (the
          // tile rectangle here, the blend's per-warp test) never drops an
          // entry that a pixel composites.
          const float lo = log2f(alpha_cond);
          const float L2 = 2.f * kLn2 * fmaxf(lo - kQMin, 0.f);
          const float hx = sqrtf(L2 * ca) * 1.0001f + 0.01f;
          const float hy = sqrtf(L2 * cc) * 1.0001f + 0.01f;
          const float ex = a.alpha_footprint ? fminf(radius, hx) : radius;
          const float ey = a.alpha_footprint ? fminf(radius, hy) : radius;
          float x0 = floorf((u - ex) * a.inv_tile_w), x1 = floorf((u + ex) * a.inv_tile_w) + 1.f;
          float y0 = floorf((w - ey) * a.inv_tile_h), y1 = floorf((w + ey) * a.inv_tile_h) + 1.f;
          x0 = fminf(fmaxf(x0, 0.f), (float)cam.tiles_x);
          x1 = fminf(fmaxf(x1, 0.f), (float)cam.tiles_x);
          y0 = fminf(fmaxf(y0, 0.f), (float)cam.tiles_y);
          y1 = fminf(fmaxf(y1, 0.f), (float)cam.tiles_y);
          bool finite = isfinite(u) && isfinite(w) && isfinite(radius) && isfinite(con_a) &&
                        isfinite(con_b) && isfinite(con_c);
          if (!finite) raise_status(a.status, SIXDGS_ERR_NONFINITE);
          // ---- colour (section 4.2) ----
          float Y[kMaxShCoeffs];
          sh_basis(a.sh_degree, d[0], d[1], d[2], Y);
          float rgb[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < kMaxShCoeffs; ++k)
              if (k < K) s += beta[k][c] * Y[k];
            rgb[c] = sigmoidf_(s);
          }
          if (finite && !(isfinite(rgb[0]) && isfinite(rgb[1]) && isfinite(rgb[2]))) {
            finite = false;
            raise_status(a.status, SIXDGS_ERR_NONFINITE);
          }
          if (finite && x0 < x1 && y0 < y1) {
            ntiles = (uint32_t)((x1 - x0) * (y1 - y0));
            PairRec rec;
            rec.a = make_float4(u, w, -0.5f * kLog2e * con_a, -kLog2e * con_b);
            rec.b = make_float4(-0.5f * kLog2e * con_c, lo, rgb[0], rgb[1]);
            rec.c = make_float4(rgb[2], hx, hy, t[2]);
            a.rec[pair] = rec;
            if (a.grad_rec) {
              float4* gr = reinterpret_cast<float4*>(a.grad_rec) + pair * 3;
              gr[0] = gr[1] = gr[2] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            a.depth_key[pair] = __float_as_uint(t[2]);
            a.rect[pair] = make_ushort4((unsigned short)x0, (unsigned short)x1, (unsigned short)y0,
                                        (unsigned short)y1);
          }
        }
      }
    }
    a.ntiles[pair] = ntiles;
  }
}

void launch_project_fwd(const ProjectArgs& a, cudaStream_t stream) {
  if (a.n == 0) return;
  const int threads = 128;
  const int64_t blocks = (a.n + threads - 1) / threads;
  size_t smem = sizeof(CamRec) * (size_t)a.n_cams;
  if (a.cond_cache)
    project_fwd_kernel<true><<<(unsigned)blocks, threads, smem, stream>>>(a);
  else
    project_fwd_kernel<false><<<(unsigned)blocks, threads, smem, stream>>>(a);
}

void launch_cond_cache(const CondCacheArgs& a, cudaStream_t stream) {
  if (a.n == 0) return;
  cond_cache_kernel<<<(unsigned)((a.n + 127) / 128), 128, 0, stream>>>(a);
}

}  // namespace sixdgs
