// Stages 3 and 4a: front-to-back blending of every screen tile and its
// reverse (the 3DGS rasteriser that 6DGS section 4.4 keeps after slicing).
//
// One CTA per global tile (all cameras' tiles in one grid, so cameras of
// different resolutions share a launch); each warp owns an 8x4 sub-block of
// the tile, one pixel per lane.  The tile's sorted list is walked in
// batches: each batch of pair records is gathered into shared memory by the
// whole CTA; then every warp tests 32 entries at a time against its
// sub-block (lane-parallel box test with the entry's alpha >= 1/255 box,
// ballot) and composites its pixels only against the entries that can reach
// them, in list order.  An entry a warp passes over would be skipped at
// every pixel of its sub-block (q < log2(1/255)), so the result is the same
// as walking every entry at every pixel.  A CTA leaves as soon as
// __syncthreads_count reports every pixel saturated; a warp leaves a batch
// as soon as all its lanes are done.
//
// Per entry and pixel:  q = qa dx^2 + qb dx dy + qc dy^2 + lo  (log2 alpha),
// skipped when q < log2(1/255); alpha = min(0.99, 2^q); stop (excluding the
// entry) when T (1 - alpha) < 1e-4; C += c alpha T; T *= (1 - alpha).
// Explicit rounding intrinsics make the backward replay bit-identical.
// The stand-alone forward culls with the alpha box only (its per-entry work
// is too cheap for the exact test to pay off); the backward, whose
// per-entry work is several times larger, also applies the exact quadratic
// test, and in the fused kernel the forward applies it and records each
// group's ballot for the backward.  Pairs of values that take the same
// operation (the pixel offset, T (1 - alpha) and alpha T, two colour
// channels) use the packed two-wide FP32 instructions, with the same
// rounding as the scalar ones.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace sixdgs {

constexpr int kSubW = 8;   // warp sub-block: 8 x 4 pixels
constexpr int kSubH = 4;

__device__ __forceinline__ int find_camera(const CamRec* cams, int n_cams, uint32_t gt) {
  int lo = 0, hi = n_cams - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if ((uint32_t)cams[mid].tile_offset <= gt) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Pixel of this thread and the pixel-centre box of its warp's sub-block.
struct PixelMap {
  int px, py;
  float x0, x1, y0, y1;   // pixel centres spanned by the warp
};

__device__ __forceinline__ PixelMap map_pixel(int tile_w, int tx, int ty, int tile_h) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub_per_row = tile_w / kSubW;
  const int sx = (warp % sub_per_row) * kSubW, sy = (warp / sub_per_row) * kSubH;
  PixelMap m;
  m.px = tx * tile_w + sx + (lane % kSubW);
  m.py = ty * tile_h + sy + (lane / kSubW);
  m.x0 = (float)(tx * tile_w + sx) + 0.5f;
  m.x1 = m.x0 + (float)(kSubW - 1);
  m.y0 = (float)(ty * tile_h + sy) + 0.5f;
  m.y1 = m.y0 + (float)(kSubH - 1);
  return m;
}

// Can the entry have q >= log2(1/255) at some pixel centre of the warp's
// sub-block?  First the entry's alpha box (u, v, hx, hy); with kExact also
// the maximum of the concave quadratic q over the sub-block's pixel-centre
// rectangle: the entry's centre if it lies inside, else the best point of
// the four edges (vertex of q along each edge, clamped to the edge).  The
// continuous maximum bounds every pixel centre's q, and the 1e-3 margin (in
// log2 units) is far above FP32 rounding, so no pixel that would composite
// the entry is ever passed over.
template <bool kExact>
__device__ __forceinline__ bool reaches(const PixelMap& m, float4 a, float4 b, float4 c) {
  if (!((a.x + c.y >= m.x0) && (a.x - c.y <= m.x1) && (a.y + c.z >= m.y0) && (a.y - c.z <= m.y1)))
    return false;
  if (!kExact) return true;
  const float dx0 = a.x - m.x1, dx1 = a.x - m.x0;   // dx = u - x over the sub-block
  const float dy0 = a.y - m.y1, dy1 = a.y - m.y0;
  if (dx0 <= 0.f && dx1 >= 0.f && dy0 <= 0.f && dy1 >= 0.f) return true;
  const float qa = a.z, qb = a.w, qc = b.x;
  const float kx = __fdividef(-0.5f * qb, qc), ky = __fdividef(-0.5f * qb, qa);
  float best = -INFINITY;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const float dx = e ? dx1 : dx0;
    const float dy = fminf(fmaxf(kx * dx, dy0), dy1);
    best = fmaxf(best, (qa * dx + qb * dy) * dx + qc * dy * dy);
    const float ey = e ? dy1 : dy0;
    const float ex = fminf(fmaxf(ky * ey, dx0), dx1);
    best = fmaxf(best, (qa * ex + qb * ey) * ex + qc * ey * ey);
  }
  return best + b.y >= kQMin - 1e-3f;
}

// A list entry as staged in shared memory: its blend record (u, v, qa, qb),
// (qc, lo, r, g), (b, hx, hy) and its pair index (bits of c.w).  One struct
// per entry, so a walk addresses all three parts from one index.
struct __align__(16) Entry {
  float4 a, b, c;
};

__device__ __forceinline__ void load_batch(const BlendArgs& a, uint32_t start, int cnt, Entry* s_e) {
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    const uint32_t p = a.sorted[start + i];
    if (p < a.n_pairs) {
      const PairRec& r = a.rec[p];
      s_e[i].a = r.a;
      s_e[i].b = r.b;
      s_e[i].c = make_float4(r.c.x, r.c.y, r.c.z, __uint_as_float(p));
    } else {  // unreachable for a consistent sort: an entry that reaches no pixel
      s_e[i].a = make_float4(-1e30f, -1e30f, 0.f, 0.f);
      s_e[i].b = make_float4(0.f, -1e30f, 0.f, 0.f);
      s_e[i].c = make_float4(0.f, 0.f, 0.f, __uint_as_float(0u));
    }
  }
}

// The backward walk runs in two passes per warp so that no value has to be
// summed across the lanes of a warp for every list entry:
//  1. pixel-parallel (lane = pixel), front to back like the forward: the
//     transmittance T and the running dL/dC . (colour prefix) Q are carried
//     per pixel, and each pixel's dL/dq and blend weight w for the entry are
//     written to the warp's shared-memory slots (kSlots = 8 entries at a
//     time);
//  2. entry-parallel, once the slots are full (or the batch ends): lane
//     8 r + s takes slot s over row r of the 8 x 4 sub-block and sums, over
//     the row's 8 pixels, dq, c dq, c^2 dq and dL/dC . w (c the column
//     relative to the sub-block's centre); the four rows are added with
//     shuffles, and lane s turns the sums into the entry's nine record
//     gradients (moments of dq in dx = u - px, dy = v - py) and adds them to
//     the record gradients in global memory.
// A slot's 32 pixel values are stored with a stride of 33 (one float2 of
// padding per slot), so the row writes of pass 1 and the column reads of
// pass 2 are both free of shared-memory bank conflicts.
constexpr int kSlots = 8;
constexpr int kCullGroups = 64;   // 2,048 list entries
struct __align__(16) WarpScratch {
  float2 dqw[kSlots][33];   // (dL/dq / ln 2, w) of slot s at pixel p, at [s][p]
  float4 pix[35];           // dL/dC of pixel p at p + (p >> 3) (rows in other banks)
  int slot_j[kSlots];       // batch index of the entry in slot s
  // fused kernel: the forward walk's culling ballot of list entries
  // [32 g, 32 g + 32) of the tile's list (first kCullGroups groups)
  uint32_t cull[kCullGroups];
};

__host__ __device__ constexpr int bwd_scratch_bytes(int threads) {
  return (threads / 32) * (int)sizeof(WarpScratch);
}

// Per-pixel front-to-back walk of a tile's list (the forward blend): T and
// C accumulate over the entries that reach the warp's sub-block; walked is
// the number of list entries before the stop (the list length if none).
struct FwdPixel {
  float T, C0, C1, C2;
  uint32_t walked;
  bool staged;   // the whole list was loaded as one batch (CTA-uniform)
};

// cull (fused kernel, else null): the exact sub-block test is used and each
// group's ballot is recorded there for the backward walk.
template <bool kCount>
__device__ __forceinline__ FwdPixel fwd_walk(const BlendArgs& a, const PixelMap& pm, float pxc, float pyc,
                                             uint2 range, bool inside, Entry* s_e,
                                             uint32_t& n_eval, uint32_t& n_comp, uint32_t& n_warp,
                                             uint32_t* cull = nullptr) {
  const int B = a.batch;
  const int lane = threadIdx.x & 31;
  float T = 1.f, C2 = 0.f;
  float2 C01 = make_float2(0.f, 0.f);
  const float2 npix = make_float2(-pxc, -pyc);
  bool done = !inside;
  uint32_t walked = range.y - range.x;
  bool staged = false;
  for (uint32_t start = range.x; start < range.y; start += B) {
    if (__syncthreads_count(done) == (int)blockDim.x) break;
    const int cnt = (int)min((uint32_t)B, range.y - start);
    load_batch(a, start, cnt, s_e);
    staged = start == range.x && start + cnt == range.y;
    __syncthreads();
    if (__all_sync(0xffffffffu, done)) continue;
    for (int base = 0; base < cnt; base += 32) {
      const int jl = base + lane;
      const bool rel = jl < cnt && (cull ? reaches<true>(pm, s_e[jl].a, s_e[jl].b, s_e[jl].c)
                                         : reaches<false>(pm, s_e[jl].a, s_e[jl].b, s_e[jl].c));
      uint32_t mask = __ballot_sync(0xffffffffu, rel);
      if (cull) {
        const uint32_t g = (start - range.x + base) >> 5;
        if (lane == 0 && g < kCullGroups) cull[g] = mask;
      }
      if (kCount) n_warp += __popc(mask);
      while (mask) {
        const int j = base + __ffs(mask) - 1;
        mask &= mask - 1;
        // Branch-free: a skipped (or finished) pixel takes alpha = 0, which
        // leaves T and C bit-for-bit unchanged.
        const float4 ra = s_e[j].a, rb = s_e[j].b;
        const float blue = s_e[j].c.x;
        float2 d;
        const float q = entry_q(ra, rb, npix, d);
        const bool vis = !done && q >= kQMin;
        const float alpha = vis ? fminf(kAlphaMax, ex2_approx(q)) : 0.f;
        // (T (1 - alpha), alpha T) in one packed multiply
        const float2 tw = __fmul2_rn(make_float2(T, T), make_float2(__fsub_rn(1.f, alpha), alpha));
        const bool stop = tw.x < kTMin;
        const float w = stop ? 0.f : tw.y;
        C01 = __ffma2_rn(make_float2(rb.z, rb.w), make_float2(w, w), C01);
        C2 = __fmaf_rn(blue, w, C2);
        T = stop ? T : tw.x;
        if (stop) walked = start - range.x + j;
        if (kCount) {
          n_eval += done ? 0u : 1u;
          n_comp += (vis && !stop) ? 1u : 0u;
        }
        done = done || stop;
      }
      if (__all_sync(0xffffffffu, done)) break;
    }
  }
  return FwdPixel{T, C01.x, C01.y, C2, walked, staged};
}

// Forward blend of global tile gt by the calling CTA.
template <bool kCount, bool kStore>
__device__ __forceinline__ void blend_fwd_tile(const BlendArgs& a, uint32_t gt, float4* s_mem) {
  Entry* s_e = reinterpret_cast<Entry*>(s_mem);
  __shared__ float s_red[16];

  const CamRec& cam = a.cams[find_camera(a.cams, a.n_cams, gt)];
  const uint32_t local = gt - (uint32_t)cam.tile_offset;
  const PixelMap pm = map_pixel(a.tile_w, local % cam.tiles_x, local / cam.tiles_x, a.tile_h);
  const bool inside = pm.px < cam.width && pm.py < cam.height;
  const float pxc = (float)pm.px + 0.5f, pyc = (float)pm.py + 0.5f;
  const uint2 range = a.ranges[gt];
  const int lane = threadIdx.x & 31;

  uint32_t n_eval = 0, n_comp = 0, n_warp = 0;
  const FwdPixel fp = fwd_walk<kCount>(a, pm, pxc, pyc, range, inside, s_e, n_eval, n_comp, n_warp);
  float T = fp.T, C0 = fp.C0, C1 = fp.C1, C2 = fp.C2;
  const uint32_t walked = fp.walked;

  float l1 = 0.f;
  if (inside) {
    C0 = __fmaf_rn(T, a.bg[0], C0);
    C1 = __fmaf_rn(T, a.bg[1], C1);
    C2 = __fmaf_rn(T, a.bg[2], C2);
    const int64_t hw = (int64_t)cam.width * cam.height;
    const int64_t pix = (int64_t)pm.py * cam.width + pm.px;
    float* img = a.images + 3 * cam.pixel_base;
    img[pix] = C0;
    img[hw + pix] = C1;
    img[2 * hw + pix] = C2;
    if (kStore) a.nwalk[cam.pixel_base + pix] = walked;
    if (a.targets) {
      const float* tg = a.targets + 3 * cam.pixel_base + pix;
      float* gi = a.grad_images + 3 * cam.pixel_base + pix;
      const float d0 = C0 - tg[0], d1 = C1 - tg[hw], d2 = C2 - tg[2 * hw];
      gi[0] = d0 > 0.f ? a.inv_count : (d0 < 0.f ? -a.inv_count : 0.f);
      gi[hw] = d1 > 0.f ? a.inv_count : (d1 < 0.f ? -a.inv_count : 0.f);
      gi[2 * hw] = d2 > 0.f ? a.inv_count : (d2 < 0.f ? -a.inv_count : 0.f);
      l1 = fabsf(d0) + fabsf(d1) + fabsf(d2);
    }
  }
  if (kCount) {
    unsigned long long e = n_eval, c = n_comp;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_xor_sync(0xffffffffu, e, o);
      c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if (lane == 0) {
      atomicAdd(a.pair_counts, e);
      atomicAdd(a.pair_counts + 1, c);
      atomicAdd(a.pair_counts + 2, (unsigned long long)n_warp);
    }
  }
  if (a.targets) {
    l1 = warp_sum(l1);
    if (lane == 0) s_red[threadIdx.x >> 5] = l1;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) s += s_red[w];
      atomicAdd(a.loss, s * (double)a.inv_count);
    }
  }
}

__device__ __forceinline__ void red_add(float* addr, float x) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(addr), "f"(x) : "memory");
}

// Four consecutive floats (16-byte aligned) added in one vector reduction.
__device__ __forceinline__ void red_add4(float* addr, float x, float y, float z, float w) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(x), "f"(y), "f"(z), "f"(w)
               : "memory");
}

// Pass 2 over slots [0, k).  xc, yc: centre of the 8 x 4 sub-block.
__device__ __forceinline__ void flush_slots(const BlendArgs& a, WarpScratch& ws, int k, const Entry* s_e,
                                            float xc, float yc) {
  static_assert(kSlots == kSubW && kSubH == 4, "one row of the sub-block per slot group");
  __syncwarp();
  const int lane = threadIdx.x & 31;
  const int s = lane & (kSlots - 1);
  const int r = lane >> 3;                 // row of the sub-block
  const float2* row = ws.dqw[s];
  float R1 = 0.f, R2 = 0.f;
  float2 RG = make_float2(0.f, 0.f);    // (sum dq, sum dC2 w)
  float2 G01 = make_float2(0.f, 0.f);   // (sum dC0 w, sum dC1 w)
#pragma unroll
  for (int c = 0; c < kSubW; ++c) {
    const int p = r * kSubW + c;
    const float2 v = row[p];
    const float4 dc = ws.pix[p + (p >> 3)];   // (dC0, dC1, 1, dC2)
    const float cc = (float)c - 0.5f * (float)(kSubW - 1);   // column about the centre
    R1 = fmaf(cc, v.x, R1);
    R2 = fmaf(cc * cc, v.x, R2);
    RG = __ffma2_rn(make_float2(dc.z, dc.w), v, RG);
    G01 = __ffma2_rn(make_float2(dc.x, dc.y), make_float2(v.y, v.y), G01);
  }
  const float R0 = RG.x, G0 = G01.x, G1 = G01.y, G2 = RG.y;
  const float rr = (float)r - 0.5f * (float)(kSubH - 1);      // row about the centre
  // moments of dq in (c, r) about the centre: 1, c, r, c^2, c r, r^2; then dL/dC . w
  float m[9] = {R0, R1, rr * R0, R2, rr * R1, rr * rr * R0, G0, G1, G2};
#pragma unroll
  for (int o = kSlots; o < 32; o <<= 1)
#pragma unroll
    for (int q = 0; q < 9; ++q) m[q] += __shfl_xor_sync(0xffffffffu, m[q], o);
  if (lane < k) {
    const int j = ws.slot_j[lane];
    const float U = s_e[j].a.x - xc, V = s_e[j].a.y - yc;   // dx = U - c, dy = V - r
    float g[9];
    g[0] = fmaf(U, m[0], -m[1]);                          // sum dq dx
    g[1] = fmaf(V, m[0], -m[2]);                          // sum dq dy
    g[2] = fmaf(U, fmaf(U, m[0], -2.f * m[1]), m[3]);     // sum dq dx^2
    g[3] = fmaf(U, fmaf(V, m[0], -m[2]), fmaf(-V, m[1], m[4]));   // sum dq dx dy
    g[4] = fmaf(V, fmaf(V, m[0], -2.f * m[2]), m[5]);     // sum dq dy^2
    g[5] = m[0];
    g[6] = m[6];
    g[7] = m[7];
    g[8] = m[8];
    float* dst = a.grad_rec + (size_t)__float_as_uint(s_e[j].c.w) * 12;
    // a record is 48 bytes, 16-byte aligned: floats 0-3 and 4-7 as vectors
    red_add4(dst, g[0], g[1], g[2], g[3]);
    red_add4(dst + 4, g[4], g[5], g[6], g[7]);
    if (g[8] != 0.f) red_add(dst + 8, g[8]);
  }
  __syncwarp();
}

// Backward replay of a tile's list for the calling thread's pixel, front to
// back (as the forward), accumulating the record gradients of every entry.
// kRecompute: re-derive the stop from the transmittance; otherwise the pixel
// walks `bound` entries.  staged (CTA-uniform): the whole list is already in
// shared memory (a single batch that the forward of the same CTA staged).
template <bool kRecompute>
__device__ __forceinline__ void bwd_walk(const BlendArgs& a, const PixelMap& pm, float pxc, float pyc,
                                         uint2 range, bool inside, const float* Cf, const float* dC,
                                         uint32_t bound, bool staged, Entry* s_e, WarpScratch& ws,
                                         bool recorded = false) {
  const int B = a.batch;
  const int lane = threadIdx.x & 31;
  // dL/dalpha_i = sum_c dC_c (c_i T_i - S_c / (1 - alpha_i)) with S the colour
  // behind entry i, S_c = C_c - P_c (P the running front-to-back sum), so
  // sum_c dC_c S_c = D0 - Q with D0 = dC . C and Q = dC . P kept as a scalar.
  const float D0 = dC[0] * Cf[0] + dC[1] * Cf[1] + dC[2] * Cf[2];
  float T = 1.f, Q = 0.f;
  const float2 npix = make_float2(-pxc, -pyc);
  bool done = !inside;
  if (kRecompute || !inside) bound = inside ? 0xffffffffu : 0u;   // outside the image: an empty walk
  // (dC0, dC1, 1, dC2): pass 2 pairs the 1 with dq and dC2 with w
  ws.pix[lane + (lane >> 3)] = make_float4(dC[0], dC[1], 1.f, dC[2]);
  int k = 0;          // slots filled (warp-uniform)

  for (uint32_t start = range.x; start < range.y; start += B) {
    // a staged list is already in shared memory (read-only): no CTA barrier
    if (!staged && __syncthreads_count(done) == (int)blockDim.x) break;
    const int cnt = (int)min((uint32_t)B, range.y - start);
    if (!staged) {
      load_batch(a, start, cnt, s_e);
      __syncthreads();
    }
    if (__all_sync(0xffffffffu, done)) continue;
    // entries j < lim of this batch lie within the pixel's walk
    const int lim = (int)min((uint32_t)cnt, bound - min(bound, start - range.x));
    for (int base = 0; base < cnt; base += 32) {
      // the sub-block test of these 32 entries: recorded by the fused
      // kernel's forward walk (the list is the same), else evaluated here
      const uint32_t g = (start - range.x + base) >> 5;
      uint32_t mask;
      if (recorded && g < kCullGroups) {
        mask = ws.cull[g];
      } else {
        const int jl = base + lane;
        const bool rel = jl < cnt && reaches<true>(pm, s_e[jl].a, s_e[jl].b, s_e[jl].c);
        mask = __ballot_sync(0xffffffffu, rel);
      }
      while (mask) {
        const int j = base + __ffs(mask) - 1;
        mask &= mask - 1;
        // Branch-free, as in the forward: alpha = 0 for a pixel that skips
        // the entry or is finished, which leaves T and Q unchanged and gives
        // zero dq and w.
        const float4 ra = s_e[j].a, rb = s_e[j].b;
        const float blue = s_e[j].c.x;
        float2 d;
        const float q = entry_q(ra, rb, npix, d);
        const bool vis = (kRecompute ? !done : j < lim) && q >= kQMin;
        const float e = ex2_approx(q);
        const float alpha = vis ? fminf(kAlphaMax, e) : 0.f;
        const float om = __fsub_rn(1.f, alpha);
        const float2 tw = __fmul2_rn(make_float2(T, T), make_float2(om, alpha));   // (T (1 - alpha), alpha T)
        const float test_T = tw.x;
        // stored walk: never a stop inside it, and alpha = 0 past it
        const bool stop = kRecompute && test_T < kTMin;
        const float w = stop ? 0.f : tw.y;
        const float G = dC[0] * rb.z + dC[1] * rb.w + dC[2] * blue;
        Q = fmaf(w, G, Q);   // now includes this entry: D0 - Q is behind it
        const float dLda = T * G - (D0 - Q) * __fdividef(1.f, om);
        // dL/dq / ln 2 (the factor ln 2 of d 2^q / dq is applied by the
        // per-Gaussian backward); no gradient through the 0.99 clamp; alpha = 0
        // (skipped, off the walk) gives dq = 0
        const float dq = (!stop && e <= kAlphaMax) ? dLda * alpha : 0.f;
        T = stop ? T : test_T;
        if (kRecompute) done = done || stop;
        ws.dqw[k][lane] = make_float2(dq, w);
        if (lane == 0) ws.slot_j[k] = j;
        if (++k == kSlots) {
          flush_slots(a, ws, k, s_e, 0.5f * (pm.x0 + pm.x1), 0.5f * (pm.y0 + pm.y1));
          k = 0;
        }
      }
      if (__all_sync(0xffffffffu, kRecompute ? done : base + 32 >= lim)) break;
    }
    if (!kRecompute) done = done || start - range.x + cnt >= bound;
    if (k) {   // the slots refer to this batch's shared-memory records
      flush_slots(a, ws, k, s_e, 0.5f * (pm.x0 + pm.x1), 0.5f * (pm.y0 + pm.y1));
      k = 0;
    }
  }
}

// Backward blend of global tile gt by the calling CTA.  kRecompute: re-derive
// the stop from the transmittance (no per-pixel state); otherwise walk each
// pixel's stored number of entries.
template <bool kRecompute>
__device__ __forceinline__ void blend_bwd_tile(const BlendArgs& a, uint32_t gt, float4* s_mem) {
  const int B = a.batch;

  const CamRec& cam = a.cams[find_camera(a.cams, a.n_cams, gt)];
  const uint32_t local = gt - (uint32_t)cam.tile_offset;
  const PixelMap pm = map_pixel(a.tile_w, local % cam.tiles_x, local / cam.tiles_x, a.tile_h);
  const bool inside = pm.px < cam.width && pm.py < cam.height;
  const float pxc = (float)pm.px + 0.5f, pyc = (float)pm.py + 0.5f;
  const uint2 range = a.ranges[gt];

  float Cf[3] = {0.f, 0.f, 0.f}, dC[3] = {0.f, 0.f, 0.f};
  uint32_t bound = range.y - range.x;
  if (inside) {
    const int64_t hw = (int64_t)cam.width * cam.height;
    const int64_t pix = (int64_t)pm.py * cam.width + pm.px;
    const float* img = a.images_in + 3 * cam.pixel_base;
    const float* gi = a.grad_in + 3 * cam.pixel_base;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      Cf[ch] = img[ch * hw + pix];
      dC[ch] = gi[ch * hw + pix];
    }
    if (!kRecompute) bound = a.nwalk[cam.pixel_base + pix];
  }
  WarpScratch* ws = reinterpret_cast<WarpScratch*>(s_mem + 3 * B);
  bwd_walk<kRecompute>(a, pm, pxc, pyc, range, inside, Cf, dC, bound, false, reinterpret_cast<Entry*>(s_mem),
                       ws[threadIdx.x >> 5]);
}

// Forward blend, fused L1 loss and backward blend of global tile gt by the
// calling CTA, for the training step whose loss is the L1 term (section
// 4.4): each pixel's dL/dC = sign(C - target) / M is known as soon as its
// forward walk ends, so the backward replay follows in the same CTA with C,
// dL/dC and the walk length in registers, and a list that fitted in one
// batch is replayed from the shared memory the forward filled, each warp
// starting its backward as soon as its own forward ends (the loss partials
// are summed after the backward, at the CTA's only barrier past the load).
// Images,
// dL/dC, loss and record gradients equal those of raster_fwd followed by
// blend_bwd in stored-walk mode, bit for bit up to the order of the atomic
// additions.
__device__ __forceinline__ void blend_fused_tile(const BlendArgs& a, uint32_t gt, float4* s_mem) {
  const int B = a.batch;
  Entry* s_e = reinterpret_cast<Entry*>(s_mem);
  __shared__ float s_red[16];

  const CamRec& cam = a.cams[find_camera(a.cams, a.n_cams, gt)];
  const uint32_t local = gt - (uint32_t)cam.tile_offset;
  const PixelMap pm = map_pixel(a.tile_w, local % cam.tiles_x, local / cam.tiles_x, a.tile_h);
  const bool inside = pm.px < cam.width && pm.py < cam.height;
  const float pxc = (float)pm.px + 0.5f, pyc = (float)pm.py + 0.5f;
  const uint2 range = a.ranges[gt];
  const int lane = threadIdx.x & 31;

  WarpScratch& ws = reinterpret_cast<WarpScratch*>(s_mem + 3 * B)[threadIdx.x >> 5];
  uint32_t n_eval = 0, n_comp = 0, n_warp = 0;
  const FwdPixel fp =
      fwd_walk<false>(a, pm, pxc, pyc, range, inside, s_e, n_eval, n_comp, n_warp, ws.cull);
  float Cf[3] = {0.f, 0.f, 0.f}, dC[3] = {0.f, 0.f, 0.f};
  float l1 = 0.f;
  if (inside) {
    Cf[0] = __fmaf_rn(fp.T, a.bg[0], fp.C0);
    Cf[1] = __fmaf_rn(fp.T, a.bg[1], fp.C1);
    Cf[2] = __fmaf_rn(fp.T, a.bg[2], fp.C2);
    const int64_t hw = (int64_t)cam.width * cam.height;
    const int64_t pix = (int64_t)pm.py * cam.width + pm.px;
    float* img = a.images + 3 * cam.pixel_base;
    const float* tg = a.targets + 3 * cam.pixel_base + pix;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      img[ch * hw + pix] = Cf[ch];
      const float d = Cf[ch] - tg[ch * hw];
      dC[ch] = d > 0.f ? a.inv_count : (d < 0.f ? -a.inv_count : 0.f);
      l1 += fabsf(d);
    }
    if (a.grad_images) {
      float* gi = a.grad_images + 3 * cam.pixel_base + pix;
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) gi[ch * hw] = dC[ch];
    }
    if (a.nwalk) a.nwalk[cam.pixel_base + pix] = fp.walked;
  }
  l1 = warp_sum(l1);
  if (lane == 0) s_red[threadIdx.x >> 5] = l1;
  __syncwarp();
  bwd_walk<false>(a, pm, pxc, pyc, range, inside, Cf, dC, fp.walked, fp.staged, s_e, ws, true);
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) sum += s_red[w];
    atomicAdd(a.loss, sum * (double)a.inv_count);
  }
}

// Register budgets of the kernels that run the backward walk (swept on the
// 300k / 8 x 800^2 frame).
#ifndef SIXDGS_FUSED_MAXNREG
#define SIXDGS_FUSED_MAXNREG 64
#endif
#ifndef SIXDGS_BWD_MAXNREG
#define SIXDGS_BWD_MAXNREG 64
#endif
__global__ void __maxnreg__(SIXDGS_FUSED_MAXNREG) blend_fused_kernel(BlendArgs a) {
  extern __shared__ float4 s_mem[];
  if (!a.tile_queue) {
    blend_fused_tile(a, blockIdx.x, s_mem);
    return;
  }
  __shared__ uint32_t s_next;
  while (true) {
    if (threadIdx.x == 0) s_next = atomicAdd(a.tile_queue, 1u);
    __syncthreads();
    const uint32_t gt = s_next;
    if (gt >= a.total_tiles) break;
    blend_fused_tile(a, gt, s_mem);
    __syncthreads();
  }
}

// One CTA per tile (grid = tiles), or persistent: a grid of as many CTAs as
// fit on the GPU at once, each taking tiles from a device counter until all
// cameras' tiles are done.
template <bool kCount, bool kStore>
__global__ void __launch_bounds__(512) blend_fwd_kernel(BlendArgs a) {
  extern __shared__ float4 s_mem[];
  if (!a.tile_queue) {
    blend_fwd_tile<kCount, kStore>(a, blockIdx.x, s_mem);
    return;
  }
  __shared__ uint32_t s_next;
  while (true) {
    if (threadIdx.x == 0) s_next = atomicAdd(a.tile_queue, 1u);
    __syncthreads();
    const uint32_t gt = s_next;
    if (gt >= a.total_tiles) break;
    blend_fwd_tile<kCount, kStore>(a, gt, s_mem);
    __syncthreads();
  }
}

template <bool kRecompute>
__global__ void __maxnreg__(SIXDGS_BWD_MAXNREG) blend_bwd_kernel(BlendArgs a) {
  extern __shared__ float4 s_mem[];
  if (!a.tile_queue) {
    blend_bwd_tile<kRecompute>(a, blockIdx.x, s_mem);
    return;
  }
  __shared__ uint32_t s_next;
  while (true) {
    if (threadIdx.x == 0) s_next = atomicAdd(a.tile_queue, 1u);
    __syncthreads();
    const uint32_t gt = s_next;
    if (gt >= a.total_tiles) break;
    blend_bwd_tile<kRecompute>(a, gt, s_mem);
    __syncthreads();
  }
}

static int blend_smem(int batch) { return batch * 3 * (int)sizeof(float4); }

// Batches near or above 48 KB of shared memory (with the kernels' static
// shared memory) need the opt-in limit.
static void allow_smem(const void* fn, int bytes) {
  if (bytes > 40 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// CTAs of `fn` resident on the whole GPU at once (the persistent grid).
static int resident_grid(const void* fn, int threads, int smem, int64_t tiles) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
  const int64_t g = (int64_t)std::max(per_sm, 1) * std::max(sms, 1);
  return (int)std::min<int64_t>(g, tiles);
}

// scratch: the backward walk's per-warp shared memory (0 for the forward)
template <typename K>
static void launch_blend(K kernel, const BlendArgs& a, int64_t total_tiles, bool scratch, cudaStream_t stream) {
  const int threads = a.tile_w * a.tile_h;
  const int smem = blend_smem(a.batch) + (scratch ? bwd_scratch_bytes(threads) : 0);
  allow_smem((const void*)kernel, smem);
  if (a.tile_queue) {
    cudaMemsetAsync(a.tile_queue, 0, sizeof(uint32_t), stream);
    const int grid = resident_grid((const void*)kernel, threads, smem, total_tiles);
    kernel<<<grid, threads, smem, stream>>>(a);
  } else {
    kernel<<<(unsigned)total_tiles, threads, smem, stream>>>(a);
  }
}

void launch_blend_fwd(const BlendArgs& a, int64_t total_tiles, cudaStream_t stream) {
  if (total_tiles == 0) return;
  if (a.pair_counts) {
    if (a.nwalk) launch_blend(blend_fwd_kernel<true, true>, a, total_tiles, false, stream);
    else launch_blend(blend_fwd_kernel<true, false>, a, total_tiles, false, stream);
  } else {
    if (a.nwalk) launch_blend(blend_fwd_kernel<false, true>, a, total_tiles, false, stream);
    else launch_blend(blend_fwd_kernel<false, false>, a, total_tiles, false, stream);
  }
}

void launch_blend_fused(const BlendArgs& a, int64_t total_tiles, cudaStream_t stream) {
  if (total_tiles == 0) return;
  launch_blend(blend_fused_kernel, a, total_tiles, true, stream);
}

void launch_blend_bwd(const BlendArgs& a, int64_t total_tiles, cudaStream_t stream) {
  if (total_tiles == 0) return;
  if (a.recompute) launch_blend(blend_bwd_kernel<true>, a, total_tiles, true, stream);
  else launch_blend(blend_bwd_kernel<false>, a, total_tiles, true, stream);
}

}  // namespace sixdgs
