// Stage 2: binning and sorting of (view, Gaussian) pairs into per-tile lists
// ordered by depth (the 3DGS duplicate/sort step kept by 6DGS section 4.4).
//
// The composite key (global tile, depth, Gaussian id) is sorted LSD-first:
//   1. compact_kernel   -- visible pairs in (view, id) order, with the depth
//                          digits' histograms (single-pass scan, decoupled
//                          look-back);
//   2. onesweep passes  -- stable 8-bit digit passes over the depth key;
//   3. emit_kernel      -- duplicate each pair once per touched tile, in depth
//                          order, with the tile digits' histograms;
//   4. onesweep passes  -- stable passes over the global tile id;
//   5. ranges_kernel    -- [start, end) of every tile's list.
// Because every pass is stable and the depth passes run before duplication,
// the result equals one LSD sort of the full key while the depth passes
// touch each visible pair once instead of once per tile.
//
// The per-digit passes follow the single-pass "onesweep" design (Adinets and
// Merrill, 2022): a tile's digit counts are published with decoupled
// look-back (Merrill and Garland, 2016) so each pass reads and writes the
// data once.  Every spin is bounded by a clock budget; on expiry the kernel
// reports SIXDGS_ERR_TIMEOUT and carries on with in-bounds writes only.
#include "common.cuh"
#include "kernels.cuh"

namespace sixdgs {

constexpr unsigned long long kScanAgg = 1ull << 62;
constexpr unsigned long long kScanInc = 2ull << 62;
constexpr unsigned long long kScanValMask = (1ull << 62) - 1;

__device__ __forceinline__ unsigned long long ld_volatile64(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}
__device__ __forceinline__ void st_volatile64(unsigned long long* p, unsigned long long v) {
  *reinterpret_cast<volatile unsigned long long*>(p) = v;
}

// Exclusive block scan of one value per thread; returns the thread's prefix
// and the block total through `total`.  s_warp needs THREADS/32 + 1 words.
template <int THREADS>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t& total, uint32_t* s_warp) {
  constexpr int WARPS = THREADS / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < WARPS ? s_warp[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < WARPS) s_warp[lane] = wi - w;
    if (lane == WARPS - 1) s_warp[WARPS] = wi;
  }
  __syncthreads();
  total = s_warp[WARPS];
  uint32_t r = s_warp[warp] + incl - v;
  __syncthreads();
  return r;
}

// Decoupled look-back over 64-bit scan state, run by one full warp.
// Publishes this tile's aggregate, waits for the predecessors and
// publishes the inclusive prefix.  Returns the exclusive prefix.
__device__ unsigned long long scan_lookback(unsigned long long* state, uint32_t tile,
                                            unsigned long long block_total, int64_t budget,
                                            int32_t* status) {
  const int lane = threadIdx.x & 31;
  if (tile == 0) {
    if (lane == 0) st_volatile64(&state[0], kScanInc | block_total);
    return 0;
  }
  if (lane == 0) st_volatile64(&state[tile], kScanAgg | block_total);
  unsigned long long excl = 0;
  long long p = (long long)tile - 1;
  const long long t0 = clock64();
  bool timed_out = false;
  while (true) {
    long long idx = p - lane;
    unsigned long long w = idx >= 0 ? ld_volatile64(&state[idx]) : kScanInc;
    uint32_t flag = (uint32_t)(w >> 62);
    uint32_t inc = __ballot_sync(0xffffffffu, flag == 2u);
    uint32_t not_ready = __ballot_sync(0xffffffffu, flag == 0u);
    int i_inc = inc ? __ffs(inc) - 1 : 32;
    uint32_t need = i_inc >= 31 ? 0xffffffffu : ((2u << i_inc) - 1u);
    if (not_ready & need) {
      bool expired = __shfl_sync(0xffffffffu, (clock64() - t0) > budget, 0);
      if (expired) {
        timed_out = true;
        break;
      }
      continue;
    }
    unsigned long long val = (lane <= i_inc) ? (w & kScanValMask) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
    excl += val;
    if (i_inc < 32) break;
    p -= 32;
  }
  if (lane == 0) {
    if (timed_out) raise_status(status, SIXDGS_ERR_TIMEOUT);
    st_volatile64(&state[tile], kScanInc | ((excl + block_total) & kScanValMask));
  }
  return excl;
}

// --------------------------------------------------------------------------
// 1. Visible-pair compaction + depth-digit histograms
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(kScanThreads) compact_kernel(CompactArgs a) {
  __shared__ uint32_t s_warp[kScanThreads / 32 + 1];
  __shared__ uint32_t s_hist[4 * 256];
  __shared__ uint32_t s_tile;
  __shared__ unsigned long long s_excl;
  for (int i = threadIdx.x; i < 4 * 256; i += kScanThreads) s_hist[i] = 0;
  const uint64_t n = (uint64_t)a.n_pairs;
  const uint32_t num_tiles = (uint32_t)((n + kCompactTile - 1) / kCompactTile);
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) s_tile = atomicAdd(a.tile_counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= num_tiles) break;
    const uint64_t base = (uint64_t)tile * kCompactTile + (uint64_t)threadIdx.x * kCompactItems;
    uint32_t cnt[kCompactItems];
    if (base + kCompactItems <= n) {
#pragma unroll
      for (int k = 0; k < kCompactItems; k += 4) {
        const uint4 q = *reinterpret_cast<const uint4*>(a.ntiles + base + k);
        cnt[k] = q.x; cnt[k + 1] = q.y; cnt[k + 2] = q.z; cnt[k + 3] = q.w;
      }
    } else {
#pragma unroll
      for (int k = 0; k < kCompactItems; ++k) cnt[k] = (base + k < n) ? a.ntiles[base + k] : 0u;
    }
    // the depth keys of all items, loaded together (an invisible pair's key is
    // not used)
    uint32_t key[kCompactItems];
#pragma unroll
    for (int k = 0; k < kCompactItems; ++k) key[k] = (base + k < n) ? a.depth_key[base + k] : 0u;
    uint32_t vis = 0;
#pragma unroll
    for (int k = 0; k < kCompactItems; ++k) vis += cnt[k] > 0u;
    uint32_t total;
    uint32_t excl = block_excl_scan<kScanThreads>(vis, total, s_warp);
    if (threadIdx.x < 32) {
      unsigned long long e = scan_lookback(a.scan_state, tile, total, a.spin_budget, a.status);
      if (threadIdx.x == 0) s_excl = e;
    }
    __syncthreads();
    uint64_t off = s_excl + excl;
#pragma unroll
    for (int k = 0; k < kCompactItems; ++k) {
      if (cnt[k] > 0u) {
        if (off < n) {
          a.keys_out[off] = key[k];
          a.vals_out[off] = (uint32_t)(base + k);
        }
        ++off;
        for (int p = 0; p < a.passes; ++p) atomicAdd(&s_hist[p * 256 + ((key[k] >> (8 * p)) & 255u)], 1u);
      }
    }
    if (tile == num_tiles - 1 && threadIdx.x == 0) *a.n_vis_out = (uint32_t)(s_excl + total);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < a.passes * 256; i += kScanThreads)
    if (s_hist[i]) atomicAdd(&a.hist[i], s_hist[i]);
}

// --------------------------------------------------------------------------
// 2/4. One stable 8-bit digit pass (onesweep)
// --------------------------------------------------------------------------
// 80 registers, 3 CTAs per SM (2 at the unbounded 128): bin_sort 0.327 -> 0.320 ms
// on the 300k / 8 x 800^2 frame.
__global__ void __launch_bounds__(kSortThreads, 3) onesweep_kernel(OnesweepArgs a) {
  constexpr int WARPS = kSortThreads / 32;
  static_assert(kSortThreads == 256, "one thread per digit");
  __shared__ uint32_t s_whist[WARPS][256];
  __shared__ uint32_t s_keys[kSortTile];
  __shared__ uint32_t s_vals[kSortTile];
  __shared__ uint32_t s_dstart[256];
  __shared__ uint32_t s_glob[256];
  __shared__ uint32_t s_warp[WARPS + 1];
  __shared__ uint32_t s_tile;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // input buffer: fixed (parity == null) or as the previous pass left it
  const uint32_t par = a.parity ? *a.parity : 0u;
  // (selects, not an index: a runtime index into the parameter arrays would
  // copy them to local memory)
  const uint32_t* keys_in = par ? a.keys[1] : a.keys[0];
  const uint32_t* vals_in = par ? a.vals[1] : a.vals[0];
  uint32_t* keys_out = par ? a.keys[0] : a.keys[1];
  uint32_t* vals_out = par ? a.vals[0] : a.vals[1];
  const uint32_t n = min(*a.n_ptr, a.capacity);
  const uint32_t num_tiles = (n + kSortTile - 1) / kSortTile;
  // exclusive digit offsets of the whole pass (thread tid owns digit tid)
  uint32_t htot;
  const uint32_t my_count = a.hist[tid];
  const uint32_t hist_excl = block_excl_scan<kSortThreads>(my_count, htot, s_warp);
  const uint32_t lt_mask = (1u << lane) - 1u;
  // Every key has the same digit: the stable pass is the identity.  With a
  // parity word the data stays where it is (the next reader is told so);
  // otherwise the tiles are copied through without ranking or look-back.
  if (__syncthreads_or(n > 0u && my_count == n)) {
    if (a.parity) {
      if (blockIdx.x == 0 && tid == 0) a.parity[1] = par;
      return;
    }
    for (uint32_t i = blockIdx.x * kSortThreads + tid; i < n; i += gridDim.x * kSortThreads) {
      keys_out[i] = keys_in[i];
      vals_out[i] = vals_in[i];
    }
    return;
  }
  if (a.parity && blockIdx.x == 0 && tid == 0) a.parity[1] = par ^ 1u;
  while (true) {
    __syncthreads();
    if (tid == 0) s_tile = atomicAdd(a.tile_counter, 1u);
#pragma unroll
    for (int w = 0; w < WARPS; ++w) s_whist[w][tid] = 0u;
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= num_tiles) break;
    const uint32_t base = tile * kSortTile;
    const uint32_t wbase = base + warp * (32 * kSortItems);
    uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
      uint32_t idx = wbase + j * 32 + lane;
      bool valid = idx < n;
      key[j] = valid ? keys_in[idx] : 0xffffffffu;
      val[j] = valid ? vals_in[idx] : 0u;
    }
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
      uint32_t idx = wbase + j * 32 + lane;
      uint32_t d = idx < n ? (key[j] >> a.shift) & 255u : 256u;
      // lanes with the same digit, from one ballot per digit bit
      uint32_t peers = __ballot_sync(0xffffffffu, d < 256u);
      if (d >= 256u) peers = ~peers;
#pragma unroll
      for (int bit = 0; bit < 8; ++bit) {
        const uint32_t set = (d >> bit) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, set);
        peers &= set ? bal : ~bal;
      }
      uint32_t before = d < 256u ? s_whist[warp][d] : 0u;
      __syncwarp();
      if (d < 256u && lane == (uint32_t)(__ffs(peers) - 1)) s_whist[warp][d] = before + __popc(peers);
      __syncwarp();
      rank[j] = before + __popc(peers & lt_mask);
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, block count
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) {
      uint32_t c = s_whist[w][tid];
      s_whist[w][tid] = run;
      run += c;
    }
    const uint32_t cnt = run;
    uint32_t btot;
    const uint32_t dstart = block_excl_scan<kSortThreads>(cnt, btot, s_warp);
    s_dstart[tid] = dstart;
    // decoupled look-back for digit tid
    uint32_t* lb = a.lookback;
    uint32_t excl = 0;
    if (tile == 0) {
      st_volatile(&lb[tid], kFlagInc | cnt);
    } else {
      st_volatile(&lb[tile * 256 + tid], kFlagAgg | cnt);
      // Walk back over the predecessors' words for this digit, kWindow at a
      // time (all loads in flight together), summing aggregates up to the
      // first inclusive prefix; a word not yet published is waited for.
      constexpr int kWindow = 8;
      long long p = (long long)tile - 1;
      const long long t0 = clock64();
      while (p >= 0) {
        uint32_t w[kWindow];
#pragma unroll
        for (int i = 0; i < kWindow; ++i) w[i] = (p - i >= 0) ? ld_volatile(&lb[(p - i) * 256 + tid]) : kFlagInc;
        int used = 0;
        bool found = false, waiting = false;
#pragma unroll
        for (int i = 0; i < kWindow; ++i) {
          if (found || waiting) continue;
          const uint32_t f = w[i] & kFlagMask;
          if (f == 0u) {
            waiting = true;
            continue;
          }
          excl += w[i] & kValMask;
          ++used;
          found = f == kFlagInc;
        }
        if (found) break;
        p -= used;
        if (waiting && clock64() - t0 > a.spin_budget) {
          raise_status(a.status, SIXDGS_ERR_TIMEOUT);
          break;
        }
      }
      st_volatile(&lb[tile * 256 + tid], kFlagInc | ((excl + cnt) & kValMask));
    }
    s_glob[tid] = hist_excl + excl - dstart;
    __syncthreads();
    // local scatter into digit order
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
      uint32_t idx = wbase + j * 32 + lane;
      if (idx < n) {
        uint32_t d = (key[j] >> a.shift) & 255u;
        uint32_t pos = s_dstart[d] + s_whist[warp][d] + rank[j];
        s_keys[pos] = key[j];
        s_vals[pos] = val[j];
      }
    }
    __syncthreads();
    const uint32_t tile_n = min((uint32_t)kSortTile, n - base);
    for (uint32_t i = tid; i < tile_n; i += kSortThreads) {
      uint32_t k = s_keys[i];
      uint32_t out = s_glob[(k >> a.shift) & 255u] + i;
      if (out < n) {
        keys_out[out] = k;
        vals_out[out] = s_vals[i];
      }
    }
  }
}

// --------------------------------------------------------------------------
// 3. Duplicate emission in depth order + tile-digit histograms
//
// Two kernels, so that the work is spread over the duplicates, not over the
// visible pairs (a few large Gaussians can own most of the duplicates):
//   emit_scan_kernel   -- exclusive scan of the depth-sorted pairs' tile
//                         counts (decoupled look-back): every pair's first
//                         output, the pair owning the first output of every
//                         chunk of kEmitChunk outputs, and the total K;
//   emit_expand_kernel -- one chunk per CTA at a time: the chunk's pairs
//                         (at most kEmitChunk + 1, since every visible pair
//                         has at least one tile) are staged in shared
//                         memory, each marks the chunk position where its
//                         outputs start, a prefix maximum over the positions
//                         gives every output its pair, and consecutive
//                         threads write consecutive duplicates, so stores are
//                         coalesced.
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(kScanThreads) emit_scan_kernel(EmitArgs a) {
  __shared__ uint32_t s_warp[kScanThreads / 32 + 1];
  __shared__ uint32_t s_tile;
  __shared__ unsigned long long s_excl;
  const uint32_t n_vis = *a.n_vis;
  const uint32_t num_tiles = (n_vis + kScanTile - 1) / kScanTile;
  const unsigned long long cap = a.capacity;
  const uint32_t par = *a.depth_parity;
  const uint32_t* pairs = par ? a.pairs[1] : a.pairs[0];
  uint32_t* dup_off = par ? a.dup_off[1] : a.dup_off[0];
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) s_tile = atomicAdd(a.tile_counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= num_tiles) break;
    const uint32_t base = tile * kScanTile + threadIdx.x * kScanItems;
    // all pair indices first, then all their tile counts (two rounds of
    // loads in flight instead of a dependent pair per item)
    uint32_t cnt[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) cnt[k] = base + k < n_vis ? pairs[base + k] : 0xffffffffu;
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      cnt[k] = cnt[k] < a.n_pairs ? a.ntiles[cnt[k]] : 0u;
      sum += cnt[k];
    }
    uint32_t total;
    const uint32_t run = block_excl_scan<kScanThreads>(sum, total, s_warp);
    if (threadIdx.x < 32) {
      unsigned long long e = scan_lookback(a.scan_state, tile, total, a.spin_budget, a.status);
      if (threadIdx.x == 0) s_excl = e;
    }
    __syncthreads();
    unsigned long long off = s_excl + run;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      if (base + k < n_vis) {
        dup_off[base + k] = (uint32_t)min(off, 0xffffffffull);
        // chunk boundaries b in [off, off + cnt) below the capacity
        const unsigned long long end = min(off + cnt[k], cap);
        for (unsigned long long b = (off + kEmitChunk - 1) / kEmitChunk * kEmitChunk; b < end; b += kEmitChunk)
          a.chunk_first[b / kEmitChunk] = base + k;
      }
      off += cnt[k];
    }
    if (tile == num_tiles - 1 && threadIdx.x == 0) {
      const unsigned long long k_total = s_excl + total;
      *a.k_out = (uint32_t)min(k_total, 0xffffffffull);
      if (k_total > cap) raise_status(a.status, SIXDGS_ERR_CAPACITY);
    }
  }
}

// row = local / w for the small integers of a tile rectangle: a float
// estimate corrected to the exact quotient.
// (64-bit, so that the correction terminates for any 32-bit input; w >= 1).
__device__ __forceinline__ uint32_t rect_row(uint32_t local, uint32_t w) {
  uint64_t row = (uint64_t)__fdividef((float)local, (float)w);
  while (row > 0u && row * w > local) --row;
  while ((row + 1u) * w <= local) ++row;
  return (uint32_t)row;
}

__global__ void __launch_bounds__(kScanThreads) emit_expand_kernel(EmitArgs a) {
  constexpr int kMaxPairs = kEmitChunk + 1;
  __shared__ uint32_t s_start[kMaxPairs];      // first output of each staged pair
  __shared__ uint32_t s_pair[kMaxPairs];
  __shared__ uint32_t s_base[kMaxPairs];       // key of the pair's top-left tile
  __shared__ uint32_t s_shape[kMaxPairs];      // rect width | tiles_x << 16
  __shared__ uint32_t s_owner[kEmitChunk];     // staged pair of every output of the chunk
  __shared__ uint32_t s_wmax[kScanThreads / 32];
  __shared__ uint32_t s_hist[4 * 256];
  static_assert(kEmitChunk == 2 * kScanThreads, "two outputs per thread in the owner scan");
  for (int i = threadIdx.x; i < 4 * 256; i += kScanThreads) s_hist[i] = 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t n_vis = *a.n_vis;
  const uint32_t k_all = (uint32_t)min((unsigned long long)*a.k_out, (unsigned long long)a.capacity);
  const uint32_t n_chunks = n_vis ? (k_all + kEmitChunk - 1) / kEmitChunk : 0u;
  const uint32_t par = *a.depth_parity;
  const uint32_t* pairs = par ? a.pairs[1] : a.pairs[0];
  const uint32_t* dup_off = par ? a.dup_off[1] : a.dup_off[0];
  for (uint32_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
    const uint32_t o0 = c * kEmitChunk;
    const uint32_t o1 = min(k_all, o0 + kEmitChunk);
    // Every visible pair owns at least one output, so a chunk spans at most
    // kMaxPairs pairs.  The clamps keep every index in bounds even if the
    // scan gave up on a look-back wait (then the status word already
    // reports the timeout).
    const uint32_t e0 = min(a.chunk_first[c], n_vis - 1);
    uint32_t e1 = (c + 1 < n_chunks) ? a.chunk_first[c + 1] : n_vis - 1;
    e1 = max(min(e1, n_vis - 1), e0);
    const int m = (int)min(e1 - e0 + 1u, (uint32_t)kMaxPairs);
    __syncthreads();
    for (int i = threadIdx.x; i < kEmitChunk; i += kScanThreads) s_owner[i] = 0u;
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += kScanThreads) {
      const uint32_t e = e0 + i;
      const uint32_t p = pairs[e];
      const uint32_t st = dup_off[e];
      s_start[i] = st;
      s_pair[i] = p;
      // a pair's outputs start at most once in the chunk (every visible pair
      // has at least one), so each position is marked by at most one pair
      const int64_t lp = (int64_t)st - (int64_t)o0;
      if (lp >= 0 && lp < kEmitChunk) s_owner[lp] = (uint32_t)i;
      uint32_t base = 0, shape = 1;
      if (p < a.n_pairs) {
        const CamRec& cam = a.cams[p / (uint32_t)a.n];
        const ushort4 r = a.rect[p];
        base = (uint32_t)cam.tile_offset + (uint32_t)r.z * (uint32_t)cam.tiles_x + r.x;
        shape = max((uint32_t)(r.y - r.x), 1u) | ((uint32_t)cam.tiles_x << 16);
      }
      s_base[i] = base;
      s_shape[i] = shape;
    }
    __syncthreads();
    // The owner of output o is the last staged pair whose outputs start at
    // or before o: an inclusive prefix maximum of the marks (unmarked
    // positions hold 0, the chunk's first pair).  Thread t scans positions
    // 2t and 2t + 1.
    {
      const uint32_t m0 = s_owner[2 * threadIdx.x];
      const uint32_t m1 = max(m0, s_owner[2 * threadIdx.x + 1]);
      uint32_t x = m1;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x = max(x, y);
      }
      if (lane == 31) s_wmax[warp] = x;
      uint32_t before = __shfl_up_sync(0xffffffffu, x, 1);
      if (lane == 0) before = 0u;
      __syncthreads();
      for (int w = 0; w < warp; ++w) before = max(before, s_wmax[w]);
      s_owner[2 * threadIdx.x] = max(before, m0);
      s_owner[2 * threadIdx.x + 1] = max(before, m1);
    }
    __syncthreads();
    for (uint32_t o1r = o0; o1r < o1; o1r += kScanThreads) {
      const uint32_t o = o1r + threadIdx.x;
      uint32_t key = 0xffffffffu;
      if (o < o1) {
        const int lo = (int)min(s_owner[o - o0], (uint32_t)(m - 1));
        const uint32_t local = o - s_start[lo];
        const uint32_t shape = s_shape[lo];
        const uint32_t w = shape & 0xffffu, tiles_x = shape >> 16;
        const uint32_t row = rect_row(local, w);
        key = s_base[lo] + row * tiles_x + (local - row * w);
        a.keys_out[o] = key;
        a.vals_out[o] = s_pair[lo];
      }
      if (key != 0xffffffffu)
        for (int q = 0; q < a.passes; ++q) atomicAdd(&s_hist[q * 256 + ((key >> (8 * q)) & 255u)], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < a.passes * 256; i += kScanThreads)
    if (s_hist[i]) atomicAdd(&a.hist[i], s_hist[i]);
}

// --------------------------------------------------------------------------
// 5. Per-tile ranges in the sorted duplicate list
// --------------------------------------------------------------------------
__global__ void ranges_kernel(RangesArgs a) {
  const uint32_t k = min(*a.k_ptr, a.capacity);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
    const uint32_t t = a.keys[i];
    if (t >= a.total_tiles) continue;
    if (i == 0 || a.keys[i - 1] != t) a.ranges[t].x = i;
    if (i == k - 1 || a.keys[i + 1] != t) a.ranges[t].y = i + 1;
  }
}

void launch_compact(const CompactArgs& a, int grid, cudaStream_t stream) {
  compact_kernel<<<grid, kScanThreads, 0, stream>>>(a);
}
void launch_onesweep(const OnesweepArgs& a, int grid, cudaStream_t stream) {
  onesweep_kernel<<<grid, kSortThreads, 0, stream>>>(a);
}
void launch_emit(const EmitArgs& a, int scan_grid, int expand_grid, cudaStream_t stream) {
  emit_scan_kernel<<<scan_grid, kScanThreads, 0, stream>>>(a);
  emit_expand_kernel<<<expand_grid, kScanThreads, 0, stream>>>(a);
}
void launch_ranges(const RangesArgs& a, int grid, cudaStream_t stream) {
  ranges_kernel<<<grid, 256, 0, stream>>>(a);
}

}  // namespace sixdgs
