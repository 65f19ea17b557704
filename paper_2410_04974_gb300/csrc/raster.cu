// Stages 3 and 4a: front-to-back blending of every screen tile and its
// reverse (the 3DGS rasteriser that 6DGS section 4.4 keeps after slicing).
//
// One CTA per global tile (all cameras' tiles in one grid, so cameras of
// different resolutions share a launch), one thread per pixel.  The tile's
// sorted list is walked in batches: each batch of pair records is gathered
// into shared memory by the whole CTA, then every thread composites its
// pixel against it.  A CTA leaves as soon as __syncthreads_count reports
// every pixel saturated; in the backward pass a warp leaves a batch as soon
// as all its lanes are done.
//
// Per entry and pixel:  q = qa dx^2 + qb dx dy + qc dy^2 + lo  (log2 alpha),
// skipped when q < log2(1/255); alpha = min(0.99, 2^q); stop (excluding the
// entry) when T (1 - alpha) < 1e-4; C += c alpha T; T *= (1 - alpha).
// Explicit rounding intrinsics make the backward replay bit-identical.
#include "common.cuh"
#include "kernels.cuh"

namespace sixdgs {

__device__ __forceinline__ int find_camera(const CamRec* cams, int n_cams, uint32_t gt) {
  int lo = 0, hi = n_cams - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if ((uint32_t)cams[mid].tile_offset <= gt) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(512) blend_fwd_kernel(BlendArgs a) {
  extern __shared__ float4 s_mem[];
  const int B = a.batch;
  float4* s_a = s_mem;
  float4* s_b = s_mem + B;
  float* s_c = reinterpret_cast<float*>(s_mem + 2 * B);
  __shared__ float s_red[16];

  const uint32_t gt = blockIdx.x;
  const CamRec& cam = a.cams[find_camera(a.cams, a.n_cams, gt)];
  const uint32_t local = gt - (uint32_t)cam.tile_offset;
  const int tx = local % cam.tiles_x, ty = local / cam.tiles_x;
  const int px = tx * a.tile_w + (int)threadIdx.x % a.tile_w;
  const int py = ty * a.tile_h + (int)threadIdx.x / a.tile_w;
  const bool inside = px < cam.width && py < cam.height;
  const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
  const uint2 range = a.ranges[gt];

  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  bool done = !inside;
  uint32_t walked = range.y - range.x;
  uint32_t n_eval = 0, n_comp = 0;
  for (uint32_t start = range.x; start < range.y; start += B) {
    if (__syncthreads_count(done) == (int)blockDim.x) break;
    const int cnt = (int)min((uint32_t)B, range.y - start);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      const uint32_t p = a.sorted[start + i];
      if (p < a.n_pairs) {
        const PairRec& r = a.rec[p];
        s_a[i] = r.a;
        s_b[i] = r.b;
        s_c[i] = r.c.x;
      } else {  // unreachable for a consistent sort; an entry that is always skipped
        s_a[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        s_b[i] = make_float4(0.f, -1e30f, 0.f, 0.f);
        s_c[i] = 0.f;
      }
    }
    __syncthreads();
    if (!done) {
      for (int j = 0; j < cnt; ++j) {
        const float4 ra = s_a[j], rb = s_b[j];
        float dx, dy;
        const float q = entry_q(ra, rb, pxc, pyc, dx, dy);
        ++n_eval;
        if (q < kQMin) continue;
        const float alpha = fminf(kAlphaMax, ex2_approx(q));
        const float test_T = __fmul_rn(T, __fsub_rn(1.f, alpha));
        if (test_T < kTMin) {
          done = true;
          walked = start - range.x + j;
          break;
        }
        ++n_comp;
        const float w = __fmul_rn(alpha, T);
        C0 = __fmaf_rn(rb.z, w, C0);
        C1 = __fmaf_rn(rb.w, w, C1);
        C2 = __fmaf_rn(s_c[j], w, C2);
        T = test_T;
      }
    }
  }

  float l1 = 0.f;
  if (inside) {
    C0 = __fmaf_rn(T, a.bg[0], C0);
    C1 = __fmaf_rn(T, a.bg[1], C1);
    C2 = __fmaf_rn(T, a.bg[2], C2);
    const int64_t hw = (int64_t)cam.width * cam.height;
    const int64_t pix = (int64_t)py * cam.width + px;
    float* img = a.images + 3 * cam.pixel_base;
    img[pix] = C0;
    img[hw + pix] = C1;
    img[2 * hw + pix] = C2;
    if (a.nwalk) a.nwalk[cam.pixel_base + pix] = walked;
    if (a.targets) {
      const float* tg = a.targets + 3 * cam.pixel_base;
      float* gi = a.grad_images + 3 * cam.pixel_base;
      const float c[3] = {C0, C1, C2};
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const float diff = c[ch] - tg[ch * hw + pix];
        gi[ch * hw + pix] = diff > 0.f ? a.inv_count : (diff < 0.f ? -a.inv_count : 0.f);
        l1 += fabsf(diff);
      }
    }
  }
  if (a.pair_counts) {
    unsigned long long e = n_eval, c = n_comp;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_xor_sync(0xffffffffu, e, o);
      c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(a.pair_counts, e);
      atomicAdd(a.pair_counts + 1, c);
    }
  }
  if (a.targets) {
    l1 = warp_sum(l1);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = l1;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) s += s_red[w];
      atomicAdd(a.loss, s * (double)a.inv_count);
    }
  }
}

// Vector reduction of the atomics into the (view, Gaussian) gradient record.
__device__ __forceinline__ void red_add_v4(float* addr, float x, float y, float z, float w) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(x), "f"(y), "f"(z),
               "f"(w)
               : "memory");
}

__global__ void __launch_bounds__(512) blend_bwd_kernel(BlendArgs a) {
  extern __shared__ float4 s_mem[];
  const int B = a.batch;
  float4* s_a = s_mem;
  float4* s_b = s_mem + B;
  float* s_c = reinterpret_cast<float*>(s_mem + 2 * B);
  uint32_t* s_p = reinterpret_cast<uint32_t*>(s_c + B);

  const uint32_t gt = blockIdx.x;
  const CamRec& cam = a.cams[find_camera(a.cams, a.n_cams, gt)];
  const uint32_t local = gt - (uint32_t)cam.tile_offset;
  const int tx = local % cam.tiles_x, ty = local / cam.tiles_x;
  const int px = tx * a.tile_w + (int)threadIdx.x % a.tile_w;
  const int py = ty * a.tile_h + (int)threadIdx.x / a.tile_w;
  const bool inside = px < cam.width && py < cam.height;
  const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
  const uint2 range = a.ranges[gt];
  const int lane = threadIdx.x & 31;

  float Cf[3] = {0.f, 0.f, 0.f}, dC[3] = {0.f, 0.f, 0.f};
  uint32_t bound = range.y - range.x;
  if (inside) {
    const int64_t hw = (int64_t)cam.width * cam.height;
    const int64_t pix = (int64_t)py * cam.width + px;
    const float* img = a.images_in + 3 * cam.pixel_base;
    const float* gi = a.grad_in + 3 * cam.pixel_base;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      Cf[ch] = img[ch * hw + pix];
      dC[ch] = gi[ch * hw + pix];
    }
    if (!a.recompute) bound = a.nwalk[cam.pixel_base + pix];
  }
  float T = 1.f, P0 = 0.f, P1 = 0.f, P2 = 0.f;
  bool done = !inside;

  for (uint32_t start = range.x; start < range.y; start += B) {
    if (__syncthreads_count(done) == (int)blockDim.x) break;
    const int cnt = (int)min((uint32_t)B, range.y - start);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      uint32_t p = a.sorted[start + i];
      if (p < a.n_pairs) {
        const PairRec& r = a.rec[p];
        s_a[i] = r.a;
        s_b[i] = r.b;
        s_c[i] = r.c.x;
      } else {  // unreachable for a consistent sort; an entry that is always skipped
        p = 0;
        s_a[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        s_b[i] = make_float4(0.f, -1e30f, 0.f, 0.f);
        s_c[i] = 0.f;
      }
      s_p[i] = p;
    }
    __syncthreads();
    for (int j = 0; j < cnt; ++j) {
      if (__all_sync(0xffffffffu, done)) break;
      float g[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) g[k] = 0.f;
      bool contrib = false;
      if (!done) {
        const uint32_t idx = start - range.x + j;
        if (!a.recompute && idx >= bound) {
          done = true;
        } else {
          const float4 ra = s_a[j], rb = s_b[j];
          float dx, dy;
          const float q = entry_q(ra, rb, pxc, pyc, dx, dy);
          if (q >= kQMin) {
            const float e = ex2_approx(q);
            const float alpha = fminf(kAlphaMax, e);
            const float test_T = __fmul_rn(T, __fsub_rn(1.f, alpha));
            if (a.recompute && test_T < kTMin) {
              done = true;
            } else {
              const float rgb2 = s_c[j];
              const float w = __fmul_rn(alpha, T);
              P0 = __fmaf_rn(rb.z, w, P0);
              P1 = __fmaf_rn(rb.w, w, P1);
              P2 = __fmaf_rn(rgb2, w, P2);
              // colour behind this entry (background included)
              const float S0 = Cf[0] - P0, S1 = Cf[1] - P1, S2 = Cf[2] - P2;
              const float inv1ma = 1.f / (1.f - alpha);
              g[6] = dC[0] * w;
              g[7] = dC[1] * w;
              g[8] = dC[2] * w;
              const float dLda = dC[0] * (rb.z * T - S0 * inv1ma) + dC[1] * (rb.w * T - S1 * inv1ma) +
                                 dC[2] * (rgb2 * T - S2 * inv1ma);
              const float dq = (e <= kAlphaMax) ? dLda * alpha * kLn2 : 0.f;
              g[0] = dq * (2.f * ra.z * dx + ra.w * dy);
              g[1] = dq * (ra.w * dx + 2.f * rb.x * dy);
              g[2] = dq * dx * dx;
              g[3] = dq * dx * dy;
              g[4] = dq * dy * dy;
              g[5] = dq;
              T = test_T;
              contrib = true;
            }
          }
        }
      }
      if (__any_sync(0xffffffffu, contrib)) {
#pragma unroll
        for (int k = 0; k < 9; ++k) g[k] = warp_sum(g[k]);
        if (lane == 0) {
          float* dst = a.grad_rec + (size_t)s_p[j] * 12;
          red_add_v4(dst, g[0], g[1], g[2], g[3]);
          red_add_v4(dst + 4, g[4], g[5], g[6], g[7]);
          atomicAdd(dst + 8, g[8]);
        }
      }
    }
  }
}

static int blend_smem(int batch, bool bwd) {
  return batch * (2 * (int)sizeof(float4) + (int)sizeof(float) + (bwd ? (int)sizeof(uint32_t) : 0));
}

void launch_blend_fwd(const BlendArgs& a, int64_t total_tiles, cudaStream_t stream) {
  if (total_tiles == 0) return;
  blend_fwd_kernel<<<(unsigned)total_tiles, a.tile_w * a.tile_h, blend_smem(a.batch, false), stream>>>(a);
}

void launch_blend_bwd(const BlendArgs& a, int64_t total_tiles, cudaStream_t stream) {
  if (total_tiles == 0) return;
  blend_bwd_kernel<<<(unsigned)total_tiles, a.tile_w * a.tile_h, blend_smem(a.batch, true), stream>>>(a);
}

}  // namespace sixdgs
