// Stage 4b: per-Gaussian backward of the slice, colour and projection.
//
// The blend backward leaves, for every (view, Gaussian) pair, the gradient
// of the loss with respect to that pair's record (u, v, qa, qb, qc, lo, r, g,
// b).  Two kernels then run one thread per Gaussian, loop over the cameras
// and sum in registers, so no atomics are needed and each parameter
// gradient is written once:
//   sh_bwd_kernel   -- colour = sigmoid(sum_k beta_k Y_k(d)) (section 4.2):
//                      gradients of beta and the d -> mu_p term;
//   geom_bwd_kernel -- conic and 2D mean -> EWA projection -> mu_cond and
//                      Sigma_cond; alpha_cond -> alpha and D (Eq. pdfv2);
//                      mu_cond = mu_p + A (d - mu_d) (Eq. mu); then, once
//                      per Gaussian, the Schur complement (Eq. sigma) and
//                      Sigma_d^-1 back to Sigma = L L^T and the raw Cholesky,
//                      opacity and mean parameters.
// Forward quantities are recomputed from the parameters with the same
// arithmetic as the forward kernel.
#include "common.cuh"
#include "cond.cuh"
#include "kernels.cuh"
#include "mat3.cuh"
#include "sh.cuh"

namespace sixdgs {

// 4 CTAs per SM (128 registers, 32 bytes spilled) instead of 3.
__global__ void __launch_bounds__(128, 4) sh_bwd_kernel(ProjectBwdArgs a) {
  extern __shared__ CamRec s_cams[];
  for (int i = threadIdx.x; i < a.n_cams; i += blockDim.x) s_cams[i] = a.cams[i];
  __syncthreads();
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.n) return;
  const int64_t n = a.n;
  const int K = (a.sh_degree + 1) * (a.sh_degree + 1);
  float mp[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) mp[i] = __ldg(a.mu_p + i * n + g);
  float beta[kMaxShCoeffs][3], dbeta[kMaxShCoeffs][3];
#pragma unroll
  for (int k = 0; k < kMaxShCoeffs; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      beta[k][c] = (k < K) ? __ldg(a.sh + (k * 3 + c) * n + g) : 0.f;
      dbeta[k][c] = 0.f;
    }
  float dmp[3] = {0.f, 0.f, 0.f};
  const float4* grec = reinterpret_cast<const float4*>(a.grad_rec);
  // Loads run ahead of the camera loop: the tile count two cameras ahead,
  // and the next camera's colour gradients only where its pair is visible
  // (its count arrived an iteration earlier), so their latency overlaps this
  // camera's arithmetic and no invisible pair's record is read.
  uint32_t nt_next = a.ntiles[g];
  uint32_t nt_next2 = a.n_cams > 1 ? a.ntiles[n + g] : 0u;
  float4 gb_next = make_float4(0.f, 0.f, 0.f, 0.f);
  float gbz_next = 0.f;
  if (nt_next) {
    gb_next = grec[g * 3 + 1];
    gbz_next = grec[g * 3 + 2].x;
  }
  for (int v = 0; v < a.n_cams; ++v) {
    const uint32_t nt = nt_next;
    const float4 gb = gb_next;
    const float gbz = gbz_next;
    nt_next = nt_next2;
    if (nt_next) {
      const int64_t next = (int64_t)(v + 1) * n + g;
      gb_next = grec[next * 3 + 1];
      gbz_next = grec[next * 3 + 2].x;
    }
    nt_next2 = v + 2 < a.n_cams ? a.ntiles[(int64_t)(v + 2) * n + g] : 0u;
    if (nt == 0u) continue;
    const float drgb[3] = {gb.z, gb.w, gbz};
    if (drgb[0] == 0.f && drgb[1] == 0.f && drgb[2] == 0.f) continue;
    const int64_t pair = (int64_t)v * n + g;
    const PairRec& r = a.rec[pair];
    const float rgb[3] = {r.b.z, r.b.w, r.c.x};
    const CamRec& cam = s_cams[v];
    float dv[3] = {mp[0] - cam.campos[0], mp[1] - cam.campos[1], mp[2] - cam.campos[2]};
    const float inv_len = rsqrtf(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    const float d[3] = {dv[0] * inv_len, dv[1] * inv_len, dv[2] * inv_len};
    float dpre[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) dpre[c] = drgb[c] * rgb[c] * (1.f - rgb[c]);
    float Y[kMaxShCoeffs], w[kMaxShCoeffs];
#pragma unroll
    for (int k = 0; k < kMaxShCoeffs; ++k) Y[k] = 0.f;
    sh_basis(a.sh_degree, d[0], d[1], d[2], Y);
#pragma unroll
    for (int k = 0; k < kMaxShCoeffs; ++k) {
      w[k] = 0.f;
      if (k < K) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          dbeta[k][c] += dpre[c] * Y[k];
          w[k] += dpre[c] * beta[k][c];
        }
      }
    }
    float gd[3];
    sh_grad(a.sh_degree, d[0], d[1], d[2], w, gd);
    // d = v / |v|: dv = (gd - d (d . gd)) / |v|
    const float dot = d[0] * gd[0] + d[1] * gd[1] + d[2] * gd[2];
#pragma unroll
    for (int i = 0; i < 3; ++i) dmp[i] += (gd[i] - d[i] * dot) * inv_len;
  }
  const bool acc = a.accumulate != 0;
#pragma unroll
  for (int k = 0; k < kMaxShCoeffs; ++k)
    if (k < K)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float* o = a.grad_sh + (k * 3 + c) * n + g;
        *o = acc ? *o + dbeta[k][c] : dbeta[k][c];
      }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float* o = a.grad_mu_p + i * n + g;
    *o = acc ? *o + dmp[i] : dmp[i];
  }
}

// 4 CTAs of 128 threads per SM (128 registers, ~130 bytes spilled to L1)
// hide the latency of the per-camera loads better than 3 (168 registers):
// 0.186 -> 0.165 ms for the pair of per-Gaussian backward kernels at 300k /
// 8 x 800^2.
__global__ void __launch_bounds__(128, 4) geom_bwd_kernel(ProjectBwdArgs a) {
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
  float L[6][6];
  load_cholesky(a.l_raw, n, g, L);
  M3 Sp, P, Sd, S;
  sigma_blocks(L, Sp, P, Sd);
  const bool ok = spd_inverse(Sd, S);
  const M3 A = mul(P, S);
  const M3 Sc = sub(Sp, mul_bt(A, P));
  const float alpha = sigmoidf_(__ldg(a.opacity_logit + g));
  const float lam = a.lambda_raw ? sigmoidf_(__ldg(a.lambda_raw + g)) : a.lambda_opa;

  M3 gA = zero3(), gS = zero3(), gSc = zero3();
  float gmp[3] = {0.f, 0.f, 0.f}, gmd[3] = {0.f, 0.f, 0.f}, galpha = 0.f, glam = 0.f;
  const float4* grec = reinterpret_cast<const float4*>(a.grad_rec);

  // the count two cameras ahead and the next camera's record gradients
  // (only where that pair is visible) loaded ahead of the camera loop
  uint32_t nt_next = a.ntiles[g];
  uint32_t nt_next2 = a.n_cams > 1 ? a.ntiles[n + g] : 0u;
  float4 ga_next = make_float4(0.f, 0.f, 0.f, 0.f), gb_next = ga_next;
  if (nt_next) {
    ga_next = grec[g * 3];
    gb_next = grec[g * 3 + 1];
  }
  for (int v = 0; v < a.n_cams && ok; ++v) {
    const uint32_t nt = nt_next;
    const float4 ga = ga_next, gb = gb_next;
    nt_next = nt_next2;
    if (nt_next) {
      const int64_t next = (int64_t)(v + 1) * n + g;
      ga_next = grec[next * 3];
      gb_next = grec[next * 3 + 1];
    }
    nt_next2 = v + 2 < a.n_cams ? a.ntiles[(int64_t)(v + 2) * n + g] : 0u;
    if (nt == 0u) continue;
    const CamRec& cam = s_cams[v];
    // ---- forward recomputation (same arithmetic as project_fwd_kernel) ----
    float dv[3] = {mp[0] - cam.campos[0], mp[1] - cam.campos[1], mp[2] - cam.campos[2]};
    const float inv_len = rsqrtf(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    const float d[3] = {dv[0] * inv_len, dv[1] * inv_len, dv[2] * inv_len};
    const float delta[3] = {d[0] - md[0], d[1] - md[1], d[2] - md[2]};
    float Ad[3], Sdl[3];
    mat_vec(A, delta, Ad);
    mat_vec(S, delta, Sdl);
    const float mc[3] = {mp[0] + Ad[0], mp[1] + Ad[1], mp[2] + Ad[2]};
    const float D = delta[0] * Sdl[0] + delta[1] * Sdl[1] + delta[2] * Sdl[2];
    const float f = __expf(-lam * D);
    const float alpha_cond = alpha * f;
    float t[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
      t[i] = cam.r[i * 3] * mc[0] + cam.r[i * 3 + 1] * mc[1] + cam.r[i * 3 + 2] * mc[2] + cam.t[i];
    const float iz = 1.f / t[2];
    const float rx_raw = t[0] * iz, ry_raw = t[1] * iz;
    const float rx = fminf(cam.limx, fmaxf(-cam.limx, rx_raw));
    const float ry = fminf(cam.limy, fmaxf(-cam.limy, ry_raw));
    const float j00 = cam.fx * iz, j02 = -cam.fx * rx * iz;
    const float j11 = cam.fy * iz, j12 = -cam.fy * ry * iz;
    float T0[3], T1[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      T0[j] = j00 * cam.r[j] + j02 * cam.r[6 + j];
      T1[j] = j11 * cam.r[3 + j] + j12 * cam.r[6 + j];
    }
    float U0[3], U1[3];
    mat_t_vec(Sc, T0, U0);
    mat_t_vec(Sc, T1, U1);
    const float ca = U0[0] * T0[0] + U0[1] * T0[1] + U0[2] * T0[2] + kDilation;
    const float cb = U0[0] * T1[0] + U0[1] * T1[1] + U0[2] * T1[2];
    const float cc = U1[0] * T1[0] + U1[1] * T1[1] + U1[2] * T1[2] + kDilation;
    const float det = ca * cc - cb * cb;
    const float idet = 1.f / det;
    const float idet2 = idet * idet;
    // ---- record gradients -> conic and alpha_cond ----
    // The blend leaves the moments M = sum over pixels of g, g dx, g dy,
    // g dx^2, g dx dy, g dy^2 with g = (dL/dq) / ln 2 and
    // q = qa dx^2 + qb dx dy + qc dy^2 + lo, dx = u - px, dy = v - py.
    const float con_a0 = cc * idet, con_b0 = -cb * idet, con_c0 = ca * idet;
    const float qa = -0.5f * kLog2e * con_a0, qb = -kLog2e * con_b0, qc = -0.5f * kLog2e * con_c0;
    const float du = kLn2 * (2.f * qa * ga.x + qb * ga.y);
    const float dvv = kLn2 * (qb * ga.x + 2.f * qc * ga.y);
    const float dcon_a = -0.5f * kLog2e * kLn2 * ga.z;   // dq/dcon_a = -1/2 log2(e) dx^2
    const float dcon_b = -kLog2e * kLn2 * ga.w;
    const float dcon_c = -0.5f * kLog2e * kLn2 * gb.x;
    const float dalpha_cond = gb.y / alpha_cond;         // lo = log2(alpha_cond): ln 2 cancels
    // conic = (cc, -cb, ca) / det  ->  (ca, cb, cc)
    const float d_ca = (-dcon_a * cc * cc + dcon_b * cb * cc - dcon_c * cb * cb) * idet2;
    const float d_cb = (2.f * dcon_a * cb * cc - dcon_b * (det + 2.f * cb * cb) + 2.f * dcon_c * ca * cb) * idet2;
    const float d_cc = (-dcon_a * cb * cb + dcon_b * ca * cb - dcon_c * ca * ca) * idet2;
    // (ca, cb, cc) = (T0 Sc T0, T0 Sc T1, T1 Sc T1) (+ dilation)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        gSc(i, j) += d_ca * T0[i] * T0[j] + d_cb * T0[i] * T1[j] + d_cc * T1[i] * T1[j];
    float dT0[3], dT1[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      dT0[j] = 2.f * d_ca * U0[j] + d_cb * U1[j];
      dT1[j] = d_cb * U0[j] + 2.f * d_cc * U1[j];
    }
    // T = J R
    const float dj00 = dT0[0] * cam.r[0] + dT0[1] * cam.r[1] + dT0[2] * cam.r[2];
    const float dj02 = dT0[0] * cam.r[6] + dT0[1] * cam.r[7] + dT0[2] * cam.r[8];
    const float dj11 = dT1[0] * cam.r[3] + dT1[1] * cam.r[4] + dT1[2] * cam.r[5];
    const float dj12 = dT1[0] * cam.r[6] + dT1[1] * cam.r[7] + dT1[2] * cam.r[8];
    float dtx = 0.f, dty = 0.f, dtz = 0.f;
    dtz += -j00 * iz * dj00 - j11 * iz * dj11;
    dtz += -j02 * iz * dj02 - j12 * iz * dj12;   // at fixed rx, ry
    const float drx = -cam.fx * iz * dj02, dry = -cam.fy * iz * dj12;
    if (fabsf(rx_raw) <= cam.limx) {
      dtx += drx * iz;
      dtz += -drx * t[0] * iz * iz;
    }
    if (fabsf(ry_raw) <= cam.limy) {
      dty += dry * iz;
      dtz += -dry * t[1] * iz * iz;
    }
    // 2D mean
    dtx += du * cam.fx * iz;
    dty += dvv * cam.fy * iz;
    dtz += -(du * cam.fx * t[0] + dvv * cam.fy * t[1]) * iz * iz;
    // t = R mu_cond + t_w
    float dmc[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) dmc[i] = cam.r[i] * dtx + cam.r[3 + i] * dty + cam.r[6 + i] * dtz;
    // ---- slice backward (Eq. mu, Eq. pdfv2, Eq. alpha) ----
    float ddelta[3];
    mat_t_vec(A, dmc, ddelta);
    const float dD = -lam * alpha_cond * dalpha_cond;
    galpha += f * dalpha_cond;
    glam -= D * alpha_cond * dalpha_cond;   // d alpha_cond / d lambda = -D alpha_cond
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      gmp[i] += dmc[i];
      ddelta[i] += 2.f * dD * Sdl[i];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        gA(i, j) += dmc[i] * delta[j];
        gS(i, j) += dD * delta[i] * delta[j];
      }
    }
    const float dot = d[0] * ddelta[0] + d[1] * ddelta[1] + d[2] * ddelta[2];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      gmd[i] -= ddelta[i];
      gmp[i] += (ddelta[i] - d[i] * dot) * inv_len;
    }
  }

  // ---- Schur complement and inverse (Eq. sigma) back to Sigma blocks ----
  // Sc = Sp - A P^T, A = P S, S = Sd^-1
  const M3 GA = sub(gA, mul(gSc, P));
  const M3 GP = sub(mul(GA, S), mul_at(gSc, A));   // G_A S - gSc^T A
  const M3 GS = add(mul_at(P, GA), gS);
  const M3 GSd = mul(mul(S, GS), S);   // dL/dSd = -S GS S (sign applied below)
  // ---- Sigma = L L^T back to L ----
  float dL[6][6];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) dL[i][j] = 0.f;
  // symmetric parts
  M3 Gp2, Gd2;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Gp2(i, j) = gSc(i, j) + gSc(j, i);
      Gd2(i, j) = -(GSd(i, j) + GSd(j, i));
    }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float lpp = 0.f, ldp = 0.f, ldd = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        lpp += Gp2(i, k) * L[k][j] + GP(i, k) * L[3 + k][j];  // ((G+G^T) Lpp + G_P Ldp)_{ij}
        ldp += GP(k, i) * L[k][j] + Gd2(i, k) * L[3 + k][j];  // (G_P^T Lpp + (Gd+Gd^T) Ldp)_{ij}
        ldd += Gd2(i, k) * L[3 + k][3 + j];                   // ((Gd+Gd^T) Ldd)_{ij}
      }
      dL[i][j] = lpp;
      dL[3 + i][j] = ldp;
      dL[3 + i][3 + j] = ldd;
    }
  if (!ok) {
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j) dL[i][j] = 0.f;
    galpha = 0.f;
    glam = 0.f;
  }
  const bool acc = a.accumulate != 0;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    float* o = a.grad_l_raw + i * n + g;
    const float v = dL[i][i] * L[i][i];
    *o = acc ? *o + v : v;
  }
  int k = 6;
#pragma unroll
  for (int i = 1; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < i; ++j) {
      const float v = L[i][j];
      float* o = a.grad_l_raw + (k++) * n + g;
      const float gv = dL[i][j] * 0.5f * (1.f - v * v);
      *o = acc ? *o + gv : gv;
    }
  const float gl = galpha * alpha * (1.f - alpha);
  a.grad_opacity_logit[g] = acc ? a.grad_opacity_logit[g] + gl : gl;
  if (a.lambda_raw && a.grad_lambda_raw) {
    const float gr = glam * lam * (1.f - lam);
    a.grad_lambda_raw[g] = acc ? a.grad_lambda_raw[g] + gr : gr;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    a.grad_mu_d[i * n + g] = acc ? a.grad_mu_d[i * n + g] + gmd[i] : gmd[i];
    a.grad_mu_p[i * n + g] += gmp[i];   // sh_bwd_kernel wrote (or added) its part first
  }
}

void launch_sh_bwd(const ProjectBwdArgs& a, cudaStream_t stream) {
  if (a.n == 0) return;
  const int threads = 128;
  sh_bwd_kernel<<<(unsigned)((a.n + threads - 1) / threads), threads, sizeof(CamRec) * a.n_cams, stream>>>(a);
}

void launch_geom_bwd(const ProjectBwdArgs& a, cudaStream_t stream) {
  if (a.n == 0) return;
  const int threads = 128;
  geom_bwd_kernel<<<(unsigned)((a.n + threads - 1) / threads), threads, sizeof(CamRec) * a.n_cams, stream>>>(a);
}

}  // namespace sixdgs
