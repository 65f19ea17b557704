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
#include "stage.cuh"

namespace sixdgs {

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

// Planes of the projection's staged tile: mu_p, mu_d, then the raw Cholesky
// factor and opacity logit (or, with a cached slice state, its 25 planes),
// the optional per-Gaussian lambda, and the SH coefficients (last: phase A
// of the projection does not read them).
struct ProjPlanes {
  int mu_p, mu_d, cond, sh, lam, count;
};

__host__ __device__ inline ProjPlanes proj_planes(bool cached, int sh_degree, bool lambda) {
  ProjPlanes p;
  p.mu_p = 0;
  p.mu_d = 3;
  p.cond = 6;
  p.lam = 6 + (cached ? kCondCachePlanes : 23);   // 21 raw Cholesky planes, the logit, one spare
  p.sh = p.lam + (lambda ? 1 : 0);
  p.count = p.sh + (sh_degree + 1) * (sh_degree + 1) * 3;
  return p;
}

__device__ __forceinline__ const float* proj_src(const ProjectArgs& a, const ProjPlanes& pp, int q) {
  if (q < pp.mu_d) return a.mu_p + (int64_t)q * a.n;
  if (q < pp.cond) return a.mu_d + (int64_t)(q - pp.mu_d) * a.n;
  if (q < pp.lam) {
    const int c = q - pp.cond;
    if (a.cond_cache) return a.cond_cache + (int64_t)c * a.n;
    return c < 21 ? a.l_raw + (int64_t)c * a.n : a.opacity_logit;   // the spare plane: the logit again
  }
  if (q < pp.sh) return a.lambda_raw;
  return a.sh + (int64_t)(q - pp.sh) * a.n;
}

// View-dependent slice of one Gaussian for one camera (Eq. mu, Eq. pdfv2,
// Eq. alpha) and its camera-space mean: d = normalize(mu_p - campos),
// mu_cond = mu_p + A (d - mu_d), alpha_cond = alpha exp(-lambda D).
struct SliceView {
  float d[3], t[3], alpha_cond;
};

__device__ __forceinline__ SliceView slice_view(const float* mp, const float* md, const M3& A, const M3& Sdi,
                                                float alpha, float lam, const CamRec& cam) {
  SliceView s;
  float dv[3] = {mp[0] - cam.campos[0], mp[1] - cam.campos[1], mp[2] - cam.campos[2]};
  float inv_len = rsqrtf(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
#pragma unroll
  for (int i = 0; i < 3; ++i) s.d[i] = dv[i] * inv_len;
  float delta[3] = {s.d[0] - md[0], s.d[1] - md[1], s.d[2] - md[2]};
  float Ad[3], Sd_delta[3];
  mat_vec(A, delta, Ad);
  mat_vec(Sdi, delta, Sd_delta);
  float mc[3] = {mp[0] + Ad[0], mp[1] + Ad[1], mp[2] + Ad[2]};
  float D = delta[0] * Sd_delta[0] + delta[1] * Sd_delta[1] + delta[2] * Sd_delta[2];
  s.alpha_cond = alpha * __expf(-lam * D);
#pragma unroll
  for (int i = 0; i < 3; ++i)
    s.t[i] = cam.r[i * 3] * mc[0] + cam.r[i * 3 + 1] * mc[1] + cam.r[i * 3 + 2] * mc[2] + cam.t[i];
  return s;
}

// The matrix with its lower triangle replaced by the upper one (the state
// the projection works with is symmetric by construction).
__device__ __forceinline__ M3 sym_upper(const M3& m) {
  M3 r = m;
  r(1, 0) = m(0, 1);
  r(2, 0) = m(0, 2);
  r(2, 1) = m(1, 2);
  return r;
}

// Per-Gaussian state the second phase reads from shared memory, written over
// the tile's conditioning planes once a thread has read its own: A (9), the
// upper triangles of Sigma_d^-1 and Sigma_cond (6 each: 00 01 02 11 12 22),
// alpha, lambda.
constexpr int kCsPlanes = 23;

__device__ __forceinline__ void store_sym(float* cp, int k0, const M3& m) {
  cp[(k0 + 0) * kStageTile] = m(0, 0);
  cp[(k0 + 1) * kStageTile] = m(0, 1);
  cp[(k0 + 2) * kStageTile] = m(0, 2);
  cp[(k0 + 3) * kStageTile] = m(1, 1);
  cp[(k0 + 4) * kStageTile] = m(1, 2);
  cp[(k0 + 5) * kStageTile] = m(2, 2);
}

__device__ __forceinline__ M3 load_sym(const float* cp, int k0) {
  M3 m;
  m(0, 0) = cp[(k0 + 0) * kStageTile];
  m(0, 1) = m(1, 0) = cp[(k0 + 1) * kStageTile];
  m(0, 2) = m(2, 0) = cp[(k0 + 2) * kStageTile];
  m(1, 1) = cp[(k0 + 3) * kStageTile];
  m(1, 2) = m(2, 1) = cp[(k0 + 4) * kStageTile];
  m(2, 2) = cp[(k0 + 5) * kStageTile];
  return m;
}

// EWA projection, colour and tile rectangle of one pair that passed the
// visibility test (section 4.4, section 4.2): writes the pair's record, depth
// key, rect and tile count (0 when the 2D covariance, the footprint or a
// value is degenerate).  beta(k, c): SH coefficient k of colour channel c.
template <typename Beta>
__device__ __forceinline__ void project_pair(const ProjectArgs& a, Beta beta, const float* mp,
                                             const float* md, const M3& A, const M3& Sdi, const M3& Sc, float alpha,
                                             float lam, const CamRec& cam, int64_t pair, int K) {
  const SliceView sv = slice_view(mp, md, A, Sdi, alpha, lam, cam);
  const float* t = sv.t;
  const float alpha_cond = sv.alpha_cond;
  uint32_t ntiles = 0;
  // ---- projection (section 4.4, EWA) ----
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
  mat_t_vec(Sc, T0, U0);  // Sigma_cond symmetric: (T0 Sc)_j
  mat_t_vec(Sc, T1, U1);
  float ca = U0[0] * T0[0] + U0[1] * T0[1] + U0[2] * T0[2] + kDilation;
  float cb = U0[0] * T1[0] + U0[1] * T1[1] + U0[2] * T1[2];
  float cc = U1[0] * T1[0] + U1[1] * T1[1] + U1[2] * T1[2] + kDilation;
  float det = ca * cc - cb * cb;
  if (det > 0.f) {
    float idet = 1.f / det;
    float con_a = cc * idet, con_b = -cb * idet, con_c = ca * idet;
    float mid = 0.5f * (ca + cc);
    float lmax = mid + sqrtf(fmaxf(mid * mid - det, 0.f));
    float radius = kRadiusSigmas * sqrtf(lmax);
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
    bool finite = isfinite(u) && isfinite(w) && isfinite(radius) && isfinite(con_a) && isfinite(con_b) &&
                  isfinite(con_c);
    if (!finite) raise_status(a.status, SIXDGS_ERR_NONFINITE);
    // ---- colour (section 4.2) ----
    float Y[kMaxShCoeffs];
    sh_basis(a.sh_degree, sv.d[0], sv.d[1], sv.d[2], Y);
    float rgb[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < kMaxShCoeffs; ++k)
        if (k < K) s += beta(k, c) * Y[k];
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
      a.rect[pair] =
          make_ushort4((unsigned short)x0, (unsigned short)x1, (unsigned short)y0, (unsigned short)y1);
    }
  }
  a.ntiles[pair] = ntiles;
}

// kStageTile Gaussians per CTA in two phases:
//  A. one thread per Gaussian: the tile's parameter planes are staged in
//     shared memory (stage.cuh), the view-independent state is computed (or
//     read from the cache) and kept in shared memory, and every camera's
//     slice decides visibility (alpha_cond >= 1/255, in front of the near
//     plane); visible (Gaussian, camera) pairs are queued in shared memory;
//  B. the CTA's threads take the queued pairs densely, one pair each, for
//     the EWA projection, colour and tile rectangle, so that the expensive
//     part runs on full warps however many pairs a Gaussian has visible.
// kStaged (frames of several cameras, where each Gaussian's parameters serve
// several pairs): as above.  Otherwise (one camera: little work to overlap
// with an up-front load, at most one pair per Gaussian) each thread reads its
// Gaussian's planes from global memory where it uses them and projects its
// visible pair itself, with the same arithmetic.
template <bool kCached, bool kStaged>
__global__ void __launch_bounds__(kStageTile, kStaged ? 5 : 4) project_fwd_kernel(ProjectArgs a) {
  extern __shared__ float4 s_dyn[];
  __shared__ uint64_t s_bars[2];
  __shared__ uint32_t s_count;
  CamRec* s_cams = reinterpret_cast<CamRec*>(s_dyn);
  float* tile = reinterpret_cast<float*>(s_cams + a.n_cams);
  const int64_t n = a.n;
  const ProjPlanes pp = proj_planes(kCached, a.sh_degree, a.lambda_raw != nullptr);
  // per-Gaussian state over the staged conditioning planes (read by phase A
  // first); queue after the tile (staged path only)
  float* s_cs = tile + pp.cond * kStageTile;
  uint16_t* s_queue = reinterpret_cast<uint16_t*>(tile + pp.count * kStageTile);
  for (int i = threadIdx.x; i < a.n_cams; i += blockDim.x) s_cams[i] = a.cams[i];
  if (threadIdx.x == 0) s_count = 0;
  const int64_t g0 = (int64_t)blockIdx.x * kStageTile;
  const int m = (int)min((int64_t)kStageTile, n - g0);
  // group 0: mu_p, mu_d, the conditioning planes and lambda (phase A);
  // group 1: the SH coefficients, in flight while phase A runs
  const bool bulk = a.bulk != 0;
  if (kStaged) {
    stage_issue(tile, pp.count, pp.sh, [&](int q) { return proj_src(a, pp, q); }, g0, m, bulk, s_bars);
    if (!stage_wait(s_bars, 0, bulk, a.spin_budget)) raise_status(a.status, SIXDGS_ERR_TIMEOUT);
  } else {
    __syncthreads();
  }
  const int tid = threadIdx.x;

  // ---- phase A: per Gaussian ----
  if (tid < m) {
    const int64_t g = g0 + tid;
    const float* sp = tile + tid;
    auto P = [&](int q) { return kStaged ? sp[q * kStageTile] : __ldg(proj_src(a, pp, q) + g); };
    float mp[3], md[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      mp[i] = P(pp.mu_p + i);
      md[i] = P(pp.mu_d + i);
    }
    // one camera: the SH coefficients are loaded with everything else, into
    // registers (unused in the staged path, which reads shared memory)
    float bt[kMaxShCoeffs][3];
    if (!kStaged) {
      const int Kb = (a.sh_degree + 1) * (a.sh_degree + 1);
#pragma unroll
      for (int k = 0; k < kMaxShCoeffs; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) bt[k][c] = k < Kb ? __ldg(a.sh + (int64_t)(k * 3 + c) * n + g) : 0.f;
    }
    CondState cs;
    bool ok = true;
    if constexpr (kCached) {
      // cached view-independent state (written by cond_cache_kernel): plane k
      // of A (k < 9), the upper triangle of the symmetric Sigma_d^-1 (9..14),
      // plane k of Sigma_cond (15..23) and alpha (24; NaN where Sigma_d was
      // not numerically positive definite)
#pragma unroll
      for (int k = 0; k < 9; ++k) cs.A.m[k] = P(pp.cond + k);
      cs.Sdi(0, 0) = P(pp.cond + 9);
      cs.Sdi(0, 1) = cs.Sdi(1, 0) = P(pp.cond + 10);
      cs.Sdi(0, 2) = cs.Sdi(2, 0) = P(pp.cond + 11);
      cs.Sdi(1, 1) = P(pp.cond + 12);
      cs.Sdi(1, 2) = cs.Sdi(2, 1) = P(pp.cond + 13);
      cs.Sdi(2, 2) = P(pp.cond + 14);
#pragma unroll
      for (int k = 0; k < 9; ++k) cs.Sc.m[k] = P(pp.cond + 15 + k);
      cs.alpha = P(pp.cond + 24);
    } else {
      ok = condition_from([&](int q) { return P(pp.cond + q); }, P(pp.cond + 21), cs);
    }
    // lambda_opa: global, or per Gaussian as sigmoid(raw) (section 4.2)
    const float lam = a.lambda_raw ? sigmoidf_(P(pp.lam)) : a.lambda_opa;
    if (ok) {
#pragma unroll
      for (int k = 0; k < 9; ++k)
        ok = ok && isfinite(cs.A.m[k]) && isfinite(cs.Sdi.m[k]) && isfinite(cs.Sc.m[k]);
      ok = ok && isfinite(mp[0]) && isfinite(mp[1]) && isfinite(mp[2]) && isfinite(md[0]) &&
           isfinite(md[1]) && isfinite(md[2]) && isfinite(cs.alpha) && isfinite(lam);
    }
    if (!ok) raise_status(a.status, SIXDGS_ERR_NONFINITE);
    if (!kStaged) {
      // one camera: project the pair right here (no queue, no second phase),
      // with the same symmetric state the queued path reads
      const M3 Sdi = sym_upper(cs.Sdi), Sc = sym_upper(cs.Sc);
      const int K = (a.sh_degree + 1) * (a.sh_degree + 1);
      for (int v = 0; v < a.n_cams; ++v) {
        const int64_t pair = (int64_t)v * n + g;
        bool vis = false;
        if (ok) {
          const SliceView sv = slice_view(mp, md, cs.A, Sdi, cs.alpha, lam, s_cams[v]);
          vis = (sv.alpha_cond >= kAlphaMin) && (sv.t[2] > s_cams[v].znear);
        }
        if (vis) project_pair(a, [&](int k, int c) { return bt[k][c]; }, mp, md, cs.A, Sdi, Sc, cs.alpha, lam,
                              s_cams[v], pair, K);
        else a.ntiles[pair] = 0u;
      }
      return;
    }
    // this thread's own column of the conditioning planes is read: reuse it
    float* cp = s_cs + tid;
#pragma unroll
    for (int k = 0; k < 9; ++k) cp[k * kStageTile] = cs.A.m[k];
    store_sym(cp, 9, cs.Sdi);
    store_sym(cp, 15, cs.Sc);
    cp[21 * kStageTile] = cs.alpha;
    cp[22 * kStageTile] = lam;
    const int lane = tid & 31;
    const M3 Sdi = sym_upper(cs.Sdi);   // as phase B reads it back
    for (int v = 0; v < a.n_cams; ++v) {
      bool vis = false;
      if (ok) {
        const SliceView sv = slice_view(mp, md, cs.A, Sdi, cs.alpha, lam, s_cams[v]);
        vis = (sv.alpha_cond >= kAlphaMin) && (sv.t[2] > s_cams[v].znear);
      }
      if (!vis) a.ntiles[(int64_t)v * n + g] = 0u;
      // warp-aggregated append to the queue
      const uint32_t active = __activemask();
      const uint32_t bal = __ballot_sync(active, vis);
      uint32_t base = 0;
      const int leader = __ffs(active) - 1;
      if (lane == leader && bal) base = atomicAdd(&s_count, (uint32_t)__popc(bal));
      base = __shfl_sync(active, base, leader);
      if (vis) s_queue[base + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)(tid | (v << 7));
    }
  }
  if (!kStaged) return;
  if (!stage_wait(s_bars, 1, bulk, a.spin_budget)) raise_status(a.status, SIXDGS_ERR_TIMEOUT);
  __syncthreads();

  // ---- phase B: one visible pair per thread ----
  const uint32_t count = s_count;
  const int K = (a.sh_degree + 1) * (a.sh_degree + 1);
  for (uint32_t qi = tid; qi < count; qi += kStageTile) {
    const uint32_t e = s_queue[qi];
    const int gl = (int)(e & 127u);
    const int v = (int)(e >> 7);
    const int64_t pair = (int64_t)v * n + g0 + gl;
    const float* sp = tile + gl;
    auto P = [&](int q) { return kStaged ? sp[q * kStageTile] : __ldg(proj_src(a, pp, q) + g0 + gl); };
    const float* cp = s_cs + gl;
    M3 A;
#pragma unroll
    for (int k = 0; k < 9; ++k) A.m[k] = cp[k * kStageTile];
    const M3 Sdi = load_sym(cp, 9), Sc = load_sym(cp, 15);
    const float mp[3] = {P(pp.mu_p), P(pp.mu_p + 1), P(pp.mu_p + 2)};
    const float md[3] = {P(pp.mu_d), P(pp.mu_d + 1), P(pp.mu_d + 2)};
    const CamRec& cam = s_cams[v];
    project_pair(a, [&](int k, int c) { return P(pp.sh + k * 3 + c); }, mp, md, A, Sdi, Sc, cp[21 * kStageTile],
                 cp[22 * kStageTile], cam, pair, K);
  }
}

template <bool kCached, bool kStaged>
static void launch_project(const ProjectArgs& a, cudaStream_t stream) {
  const int64_t blocks = (a.n + kStageTile - 1) / kStageTile;
  const ProjPlanes pp = proj_planes(kCached, a.sh_degree, a.lambda_raw != nullptr);
  const size_t smem = sizeof(CamRec) * (size_t)a.n_cams +
                      (kStaged ? (size_t)pp.count * kStageTile * sizeof(float) +
                                     (size_t)kStageTile * a.n_cams * sizeof(uint16_t)
                               : 0);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(project_fwd_kernel<kCached, kStaged>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  project_fwd_kernel<kCached, kStaged><<<(unsigned)blocks, kStageTile, smem, stream>>>(a);
}

void launch_project_fwd(const ProjectArgs& a, cudaStream_t stream) {
  if (a.n == 0) return;
  const bool staged = a.n_cams > 1;
  if (a.cond_cache) {
    if (staged) launch_project<true, true>(a, stream);
    else launch_project<true, false>(a, stream);
  } else {
    if (staged) launch_project<false, true>(a, stream);
    else launch_project<false, false>(a, stream);
  }
}

void launch_cond_cache(const CondCacheArgs& a, cudaStream_t stream) {
  if (a.n == 0) return;
  cond_cache_kernel<<<(unsigned)((a.n + 127) / 128), 128, 0, stream>>>(a);
}

}  // namespace sixdgs
