// Staging of per-Gaussian structure-of-arrays planes into shared memory.
//
// A CTA that works on a contiguous range of Gaussians copies the range of
// every parameter plane it needs into shared memory with bulk asynchronous
// copies (cp.async.bulk, one 16-byte-aligned segment per plane), whose
// completion is counted in bytes on one mbarrier.  All of a tile's loads are
// in flight at once and hold no registers; the compute then reads its
// Gaussian's values from shared memory (plane q of the tile at
// tile[q * kStageTile + i]).  When a plane segment cannot be copied in bulk
// (a base address or the plane length not a multiple of 16 bytes) the CTA
// loads the same layout with ordinary coalesced loads instead.
#pragma once

#include "common.cuh"

namespace sixdgs {

constexpr int kStageTile = 128;   // Gaussians per staged tile (one per thread)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t arrivals) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(arrivals) : "memory");
  // make the initialised barrier visible to the bulk-copy (async) proxy
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Waits until the barrier's phase `parity` completed, for at most `budget`
// clock cycles; false when the budget ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int64_t budget) {
  const long long t0 = clock64();
  while (!mbar_test(bar, parity)) {
    if (clock64() - t0 > budget) return false;
  }
  return true;
}

// Copies planes [0, np) of the tile of m Gaussians starting at g0 into
// `tile` (np * kStageTile floats, 16-byte aligned); plane q is read from
// src(q) + g0.  bulk: every src(q) + g0 is 16-byte aligned and m * 4 is a
// multiple of 16.  The planes arrive in two groups, [0, split) on bars[0]
// and [split, np) on bars[1], so that work on the first group can start
// while the second is in flight: call stage_wait(bars, 0 or 1, ...) before
// reading a group.  Must be called by the whole CTA.
template <typename Src>
__device__ __forceinline__ void stage_issue(float* tile, int np, int split, Src src, int64_t g0, int m, bool bulk,
                                            uint64_t* bars) {
  if (!bulk) {
    // plain coalesced loads, kBurst planes in flight per thread
    constexpr int kBurst = 16;
    if ((int)threadIdx.x < m) {
      for (int q0 = 0; q0 < np; q0 += kBurst) {
        float v[kBurst];
#pragma unroll
        for (int i = 0; i < kBurst; ++i) v[i] = q0 + i < np ? __ldg(src(q0 + i) + g0 + threadIdx.x) : 0.f;
#pragma unroll
        for (int i = 0; i < kBurst; ++i)
          if (q0 + i < np) tile[(q0 + i) * kStageTile + threadIdx.x] = v[i];
      }
    }
    __syncthreads();
    return;
  }
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    if (threadIdx.x == 0) {
      mbar_arrive_expect_tx(&bars[0], (uint32_t)(split * m * 4));
      mbar_arrive_expect_tx(&bars[1], (uint32_t)((np - split) * m * 4));
    }
    __syncwarp();
    for (int q = threadIdx.x; q < np; q += 32)
      bulk_copy_g2s(tile + q * kStageTile, src(q) + g0, (uint32_t)(m * 4), &bars[q < split ? 0 : 1]);
  }
}

// Waits for group `grp` of stage_issue (bulk mode; a no-op otherwise).  False
// when the bounded wait ran out, after which that group's contents are
// unspecified.
__device__ __forceinline__ bool stage_wait(uint64_t* bars, int grp, bool bulk, int64_t budget) {
  if (!bulk) return true;
  bool ok = mbar_wait(&bars[grp], 0, budget);
  if (!ok) ok = mbar_wait(&bars[grp], 0, budget);   // the copies land in this CTA's memory: let them finish
  return ok;
}

}  // namespace sixdgs
