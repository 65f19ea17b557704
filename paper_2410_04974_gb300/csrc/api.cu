// C ABI of the sixdgs library: plan and workspace layout, argument checks
// and the launch sequence of each stage (declared in include/sixdgs.h).
#include <cstring>
#include <initializer_list>

#include "common.cuh"
#include "kernels.cuh"

using namespace sixdgs;

namespace {

// Internal workspace sections (after the public ones of sixdgs.h).
enum {
  WS_ZERO = 11,        // start of the region cleared by bin_sort
  WS_ZERO_END = 12,
  WS_COUNTERS = 13,    // uint32 tile counters of the persistent kernels
  WS_SCAN_C = 14,      // compaction scan state
  WS_SCAN_E = 15,      // emission scan state
  WS_HIST = 16,        // (depth + tile passes) x 256 digit counts
  WS_LB_DEPTH = 17,    // look-back words of the depth passes
  WS_LB_TILE = 18,     // look-back words of the tile passes
  WS_DEPTH_A_K = 19,
  WS_DEPTH_A_V = 20,
  WS_DEPTH_B_K = 21,
  WS_DEPTH_B_V = 22,
  WS_DUP_A_K = 23,
  WS_DUP_A_V = 24,
  WS_DUP_B_K = 25,
  WS_DUP_B_V = 26,
  WS_CHUNK_FIRST = 27, // first pair of every emission chunk
  WS_COUNT = 28
};

constexpr int kMaxCams = 256;
// WS_COUNTERS words: 0 compaction, 1-4 depth passes, 8 emission, 9-12 tile
// passes, 32 persistent blend queue, 40-44 depth-pass buffer parities
constexpr int kDepthParityWord = 40;
constexpr int kCamsPerUpload = 48;   // 6 KB of kernel parameters per upload

int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (!cached[dev]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
    cached[dev] = v;
  }
  return cached[dev];
}

struct CamUpload {
  CamRec cams[kCamsPerUpload];
  int32_t count;
};

__global__ void upload_cams_kernel(CamUpload up, CamRec* dst) {
  for (int i = threadIdx.x; i < up.count; i += blockDim.x) dst[i] = up.cams[i];
}

CamRec make_cam_rec(const sixdgs_camera& c, const sixdgs_settings& st, int32_t tile_offset,
                    int64_t pixel_base) {
  CamRec r;
  std::memset(&r, 0, sizeof(r));
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) r.r[i * 3 + j] = c.world_to_cam[i * 4 + j];
    r.t[i] = c.world_to_cam[i * 4 + 3];
    r.campos[i] = c.campos[i];
  }
  r.fx = c.fx;
  r.fy = c.fy;
  r.cx = c.cx;
  r.cy = c.cy;
  r.znear = c.znear;
  r.limx = kFrustumGuard * (0.5f * (float)c.width) / c.fx;
  r.limy = kFrustumGuard * (0.5f * (float)c.height) / c.fy;
  r.width = c.width;
  r.height = c.height;
  r.tiles_x = (c.width + st.tile_w - 1) / st.tile_w;
  r.tiles_y = (c.height + st.tile_h - 1) / st.tile_h;
  r.tile_offset = tile_offset;
  r.pixel_base = pixel_base;
  return r;
}

template <typename T>
T* ws_ptr(void* ws, const sixdgs_plan* p, int section) {
  return reinterpret_cast<T*>(static_cast<char*>(ws) + p->off[section]);
}

int64_t spin_budget(const sixdgs_plan* p) {
  return p->settings.spin_budget > 0 ? p->settings.spin_budget : (int64_t)1 << 31;
}

sixdgs_status check_ws(const sixdgs_plan* p, void* ws, size_t ws_bytes) {
  if (!p || !ws) return SIXDGS_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return SIXDGS_ERR_INVALID_ARG;
  if ((int64_t)ws_bytes < p->ws_bytes) return SIXDGS_ERR_WORKSPACE;
  return SIXDGS_OK;
}

// Can every plane segment of a staged tile of Gaussians be copied in bulk
// (16-byte-aligned source, length a multiple of 16 bytes)?  Null pointers
// (absent planes) do not count.
bool bulk_planes(int64_t n, std::initializer_list<const float*> arrays) {
  if (n % 4 != 0) return false;
  for (const float* p : arrays)
    if (p && (reinterpret_cast<uintptr_t>(p) & 15u) != 0) return false;
  return true;
}

sixdgs_status launch_status() {
  return cudaPeekAtLastError() == cudaSuccess ? SIXDGS_OK : SIXDGS_ERR_CUDA;
}

bool valid_scene(const sixdgs_plan* p, const sixdgs_scene* s) {
  return s && s->n == p->n && s->sh_degree == p->sh_degree &&
         (p->n == 0 || (s->mu_p && s->mu_d && s->l_raw && s->opacity_logit && s->sh));
}

// The projection needs l_raw and opacity_logit only without a cached state.
bool valid_fwd_scene(const sixdgs_plan* p, const sixdgs_scene* s) {
  return s && s->n == p->n && s->sh_degree == p->sh_degree &&
         (p->n == 0 || (s->mu_p && s->mu_d && s->sh && (s->cond_cache || (s->l_raw && s->opacity_logit))));
}

}  // namespace

extern "C" {

const char* sixdgs_version(void) { return "0.1.0"; }

const char* sixdgs_status_string(int32_t status) {
  switch (status) {
    case SIXDGS_OK: return "ok";
    case SIXDGS_ERR_INVALID_ARG: return "invalid argument";
    case SIXDGS_ERR_CUDA: return "CUDA error";
    case SIXDGS_ERR_CAPACITY: return "duplicate capacity exceeded";
    case SIXDGS_ERR_TIMEOUT: return "device wait timed out";
    case SIXDGS_ERR_NONFINITE: return "non-finite Gaussian";
    case SIXDGS_ERR_WORKSPACE: return "workspace too small";
    default: return "unknown status";
  }
}

sixdgs_status sixdgs_plan_init(int64_t n, int32_t sh_degree, const sixdgs_camera* cams,
                               int32_t n_cams, const sixdgs_settings* st, int64_t dup_capacity,
                               sixdgs_plan* plan) {
  if (!plan || !st || !cams || n < 0 || n_cams < 1 || n_cams > kMaxCams) return SIXDGS_ERR_INVALID_ARG;
  if (sh_degree < 0 || sh_degree > 3) return SIXDGS_ERR_INVALID_ARG;
  if (!(st->tile_w == 8 || st->tile_w == 16 || st->tile_w == 32)) return SIXDGS_ERR_INVALID_ARG;
  if (!(st->tile_h == 8 || st->tile_h == 16)) return SIXDGS_ERR_INVALID_ARG;
  if (st->batch < 32 || st->batch > 1024 || st->batch % 32) return SIXDGS_ERR_INVALID_ARG;
  if (!(st->lambda_opa >= 0.f) || !(st->lambda_opa <= 1.f)) return SIXDGS_ERR_INVALID_ARG;
  if (st->inference != 0 && st->inference != 1) return SIXDGS_ERR_INVALID_ARG;
  if (st->inference && st->store_aux) return SIXDGS_ERR_INVALID_ARG;
  if (st->alpha_footprint != 0 && st->alpha_footprint != 1) return SIXDGS_ERR_INVALID_ARG;
  const int64_t n_pairs = (int64_t)n_cams * n;
  if (n_pairs >= ((int64_t)1 << 31)) return SIXDGS_ERR_INVALID_ARG;
  std::memset(plan, 0, sizeof(*plan));
  int64_t tiles = 0, pixels = 0;
  for (int i = 0; i < n_cams; ++i) {
    const sixdgs_camera& c = cams[i];
    if (c.width <= 0 || c.height <= 0 || !(c.fx > 0.f) || !(c.fy > 0.f)) return SIXDGS_ERR_INVALID_ARG;
    const int64_t tx = (c.width + st->tile_w - 1) / st->tile_w;
    const int64_t ty = (c.height + st->tile_h - 1) / st->tile_h;
    if (tx > 65535 || ty > 65535) return SIXDGS_ERR_INVALID_ARG;
    tiles += tx * ty;
    pixels += (int64_t)c.width * c.height;
  }
  if (tiles >= ((int64_t)1 << 31)) return SIXDGS_ERR_INVALID_ARG;
  if (dup_capacity <= 0) dup_capacity = 4 * n_pairs + 4096;
  if (dup_capacity >= ((int64_t)1 << 30)) return SIXDGS_ERR_INVALID_ARG;

  plan->n = n;
  plan->sh_degree = sh_degree;
  plan->n_cams = n_cams;
  plan->settings = *st;
  plan->n_pairs = n_pairs;
  plan->total_tiles = tiles;
  plan->total_pixels = pixels;
  plan->dup_capacity = dup_capacity;
  plan->depth_passes = 4;
  int bits = 1;
  while (((int64_t)1 << bits) < tiles) ++bits;
  plan->tile_passes = (bits + 7) / 8;

  const int64_t np4 = align_up(n_pairs, 4);
  const int64_t scan_tiles = (n_pairs + kScanTile - 1) / kScanTile + 1;
  const int64_t sort_tiles_d = (n_pairs + kSortTile - 1) / kSortTile + 1;
  const int64_t sort_tiles_t = (dup_capacity + kSortTile - 1) / kSortTile + 1;
  int64_t o = 0;
  auto take = [&](int section, int64_t bytes) {
    plan->off[section] = o;
    o = align_up(o + bytes, 256);
  };
  take(SIXDGS_WS_CAMS, (int64_t)n_cams * (int64_t)sizeof(CamRec));
  take(SIXDGS_WS_REC, n_pairs * (int64_t)sizeof(PairRec));
  take(SIXDGS_WS_NTILES, np4 * 4);
  take(SIXDGS_WS_RECT, n_pairs * 8);
  take(SIXDGS_WS_DEPTHKEY, n_pairs * 4);
  take(SIXDGS_WS_GRADREC, st->inference ? 0 : n_pairs * 48);
  take(SIXDGS_WS_RANGES, tiles * 8);
  take(SIXDGS_WS_NWALK, st->store_aux ? pixels * 4 : 0);
  // cleared at the start of every bin_sort
  plan->off[WS_ZERO] = o;
  take(SIXDGS_WS_COUNTS, 48);
  take(WS_COUNTERS, 64 * 4);
  take(WS_SCAN_C, scan_tiles * 8);
  take(WS_SCAN_E, scan_tiles * 8);
  take(WS_HIST, (int64_t)(plan->depth_passes + plan->tile_passes) * 256 * 4);
  take(WS_LB_DEPTH, (int64_t)plan->depth_passes * sort_tiles_d * 256 * 4);
  take(WS_LB_TILE, (int64_t)plan->tile_passes * sort_tiles_t * 256 * 4);
  plan->off[WS_ZERO_END] = o;
  take(WS_DEPTH_A_K, n_pairs * 4);
  take(WS_DEPTH_A_V, n_pairs * 4);
  take(WS_DEPTH_B_K, n_pairs * 4);
  take(WS_DEPTH_B_V, n_pairs * 4);
  take(WS_DUP_A_K, dup_capacity * 4);
  take(WS_DUP_A_V, dup_capacity * 4);
  take(WS_DUP_B_K, dup_capacity * 4);
  take(WS_DUP_B_V, dup_capacity * 4);
  take(WS_CHUNK_FIRST, (dup_capacity / kEmitChunk + 2) * 4);
  const bool odd = plan->tile_passes & 1;
  plan->off[SIXDGS_WS_SORTED] = plan->off[odd ? WS_DUP_B_V : WS_DUP_A_V];
  plan->off[SIXDGS_WS_SORTEDKEY] = plan->off[odd ? WS_DUP_B_K : WS_DUP_A_K];
  plan->ws_bytes = o;
  return SIXDGS_OK;
}

size_t sixdgs_workspace_size(const sixdgs_plan* plan) { return plan ? (size_t)plan->ws_bytes : 0; }

sixdgs_status sixdgs_condition_project(const sixdgs_plan* p, const sixdgs_scene* scene,
                                       const sixdgs_camera* cams, void* ws, size_t ws_bytes,
                                       int32_t* status_dev, sixdgs_stream_t stream_) {
  sixdgs_status e = check_ws(p, ws, ws_bytes);
  if (e != SIXDGS_OK) return e;
  if (!valid_fwd_scene(p, scene) || !cams) return SIXDGS_ERR_INVALID_ARG;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  CamRec* dcams = ws_ptr<CamRec>(ws, p, SIXDGS_WS_CAMS);
  int32_t tile_offset = 0;
  int64_t pixel_base = 0;
  for (int first = 0; first < p->n_cams; first += kCamsPerUpload) {
    CamUpload up;
    std::memset(&up, 0, sizeof(up));
    up.count = std::min(kCamsPerUpload, p->n_cams - first);
    for (int i = 0; i < up.count; ++i) {
      const sixdgs_camera& c = cams[first + i];
      up.cams[i] = make_cam_rec(c, p->settings, tile_offset, pixel_base);
      tile_offset += up.cams[i].tiles_x * up.cams[i].tiles_y;
      pixel_base += (int64_t)c.width * c.height;
    }
    upload_cams_kernel<<<1, 64, 0, stream>>>(up, dcams + first);
  }
  if (tile_offset != p->total_tiles || pixel_base != p->total_pixels) return SIXDGS_ERR_INVALID_ARG;
  ProjectArgs a;
  a.cams = dcams;
  a.n_cams = p->n_cams;
  a.n = p->n;
  a.sh_degree = p->sh_degree;
  a.lambda_opa = p->settings.lambda_opa;
  a.inv_tile_w = 1.f / (float)p->settings.tile_w;
  a.inv_tile_h = 1.f / (float)p->settings.tile_h;
  a.alpha_footprint = p->settings.alpha_footprint;
  a.mu_p = scene->mu_p;
  a.mu_d = scene->mu_d;
  a.l_raw = scene->l_raw;
  a.opacity_logit = scene->opacity_logit;
  a.sh = scene->sh;
  a.lambda_raw = scene->lambda_raw;
  a.cond_cache = scene->cond_cache;
  a.rec = ws_ptr<PairRec>(ws, p, SIXDGS_WS_REC);
  a.ntiles = ws_ptr<uint32_t>(ws, p, SIXDGS_WS_NTILES);
  a.rect = ws_ptr<ushort4>(ws, p, SIXDGS_WS_RECT);
  a.depth_key = ws_ptr<uint32_t>(ws, p, SIXDGS_WS_DEPTHKEY);
  a.grad_rec = p->settings.inference ? nullptr : ws_ptr<float>(ws, p, SIXDGS_WS_GRADREC);
  a.bulk = bulk_planes(p->n, {a.mu_p, a.mu_d, a.sh, a.lambda_raw, a.cond_cache,
                              a.cond_cache ? nullptr : a.l_raw, a.cond_cache ? nullptr : a.opacity_logit});
  a.spin_budget = spin_budget(p);
  a.status = status_dev;
  launch_project_fwd(a, stream);
  return launch_status();
}

sixdgs_status sixdgs_bin_sort(const sixdgs_plan* p, void* ws, size_t ws_bytes, int32_t* status_dev,
                              sixdgs_stream_t stream_) {
  sixdgs_status e = check_ws(p, ws, ws_bytes);
  if (e != SIXDGS_OK) return e;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  const int sms = sm_count();
  char* base = static_cast<char*>(ws);
  if (cudaMemsetAsync(base + p->off[WS_ZERO], 0, p->off[WS_ZERO_END] - p->off[WS_ZERO], stream) != cudaSuccess)
    return SIXDGS_ERR_CUDA;
  uint32_t* counts = ws_ptr<uint32_t>(ws, p, SIXDGS_WS_COUNTS);
  uint32_t* counters = ws_ptr<uint32_t>(ws, p, WS_COUNTERS);
  uint32_t* hist = ws_ptr<uint32_t>(ws, p, WS_HIST);
  const int64_t budget = spin_budget(p);
  const int64_t sort_tiles_d = (p->n_pairs + kSortTile - 1) / kSortTile + 1;
  const int64_t sort_tiles_t = (p->dup_capacity + kSortTile - 1) / kSortTile + 1;

  // 1. compaction of visible pairs + depth histograms
  {
    CompactArgs a;
    a.ntiles = ws_ptr<uint32_t>(ws, p, SIXDGS_WS_NTILES);
    a.depth_key = ws_ptr<uint32_t>(ws, p, SIXDGS_WS_DEPTHKEY);
    a.n_pairs = p->n_pairs;
    a.keys_out = ws_ptr<uint32_t>(ws, p, WS_DEPTH_A_K);
    a.vals_out = ws_ptr<uint32_t>(ws, p, WS_DEPTH_A_V);
    a.n_vis_out = counts + 0;
    a.scan_state = ws_ptr<unsigned long long>(ws, p, WS_SCAN_C);
    a.tile_counter = counters + 0;
    a.hist = hist;
    a.passes = p->depth_passes;
    a.spin_budget = budget;
    a.status = status_dev;
    const int64_t tiles = (p->n_pairs + kCompactTile - 1) / kCompactTile;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sms * 8));
    launch_compact(a, grid, stream);
  }
  // 2. depth passes between buffers A and B; each pass records in a parity
  // word where its output is, so that a pass whose digit is the same for
  // every key (the high byte of depths within a factor of two) moves nothing
  uint32_t* depth_parity = counters + kDepthParityWord;   // zeroed above: input in A
  const int depth_grid = (int)std::max<int64_t>(1, std::min<int64_t>((p->n_pairs + kSortTile - 1) / kSortTile, (int64_t)sms * 4));
  for (int pass = 0; pass < p->depth_passes; ++pass) {
    OnesweepArgs a;
    a.keys[0] = ws_ptr<uint32_t>(ws, p, WS_DEPTH_A_K);
    a.vals[0] = ws_ptr<uint32_t>(ws, p, WS_DEPTH_A_V);
    a.keys[1] = ws_ptr<uint32_t>(ws, p, WS_DEPTH_B_K);
    a.vals[1] = ws_ptr<uint32_t>(ws, p, WS_DEPTH_B_V);
    a.parity = depth_parity + pass;
    a.n_ptr = counts + 0;
    a.capacity = (uint32_t)p->n_pairs;
    a.hist = hist + pass * 256;
    a.lookback = ws_ptr<uint32_t>(ws, p, WS_LB_DEPTH) + (int64_t)pass * sort_tiles_d * 256;
    a.tile_counter = counters + 1 + pass;
    a.shift = 8 * pass;
    a.spin_budget = budget;
    a.status = status_dev;
    launch_onesweep(a, depth_grid, stream);
  }
  // 3. duplicate emission in depth order + tile histograms
  {
    EmitArgs a;
    a.pairs[0] = ws_ptr<uint32_t>(ws, p, WS_DEPTH_A_V);
    a.pairs[1] = ws_ptr<uint32_t>(ws, p, WS_DEPTH_B_V);
    a.depth_parity = depth_parity + p->depth_passes;
    a.n_vis = counts + 0;
    a.ntiles = ws_ptr<uint32_t>(ws, p, SIXDGS_WS_NTILES);
    a.rect = ws_ptr<ushort4>(ws, p, SIXDGS_WS_RECT);
    a.cams = ws_ptr<CamRec>(ws, p, SIXDGS_WS_CAMS);
    a.n = p->n;
    a.n_pairs = (uint32_t)p->n_pairs;
    a.keys_out = ws_ptr<uint32_t>(ws, p, WS_DUP_A_K);
    a.vals_out = ws_ptr<uint32_t>(ws, p, WS_DUP_A_V);
    // the depth keys are not needed once the depth passes are done
    a.dup_off[0] = ws_ptr<uint32_t>(ws, p, WS_DEPTH_A_K);
    a.dup_off[1] = ws_ptr<uint32_t>(ws, p, WS_DEPTH_B_K);
    a.chunk_first = ws_ptr<uint32_t>(ws, p, WS_CHUNK_FIRST);
    a.capacity = (uint64_t)p->dup_capacity;
    a.k_out = counts + 1;
    a.scan_state = ws_ptr<unsigned long long>(ws, p, WS_SCAN_E);
    a.tile_counter = counters + 8;
    a.hist = hist + p->depth_passes * 256;
    a.passes = p->tile_passes;
    a.spin_budget = budget;
    a.status = status_dev;
    const int64_t tiles = (p->n_pairs + kScanTile - 1) / kScanTile;
    const int scan_grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sms * 8));
    const int64_t chunks = (p->dup_capacity + kEmitChunk - 1) / kEmitChunk;
    const int expand_grid = (int)std::max<int64_t>(1, std::min<int64_t>(chunks, (int64_t)sms * 6));
    launch_emit(a, scan_grid, expand_grid, stream);
  }
  // 4. tile passes
  const int tile_grid = (int)std::max<int64_t>(1, std::min<int64_t>((p->dup_capacity + kSortTile - 1) / kSortTile, (int64_t)sms * 4));
  for (int pass = 0; pass < p->tile_passes; ++pass) {
    // fixed ping-pong: the sorted duplicates end in the buffer the plan names
    OnesweepArgs a;
    const bool even = (pass % 2) == 0;
    a.keys[0] = ws_ptr<uint32_t>(ws, p, even ? WS_DUP_A_K : WS_DUP_B_K);
    a.vals[0] = ws_ptr<uint32_t>(ws, p, even ? WS_DUP_A_V : WS_DUP_B_V);
    a.keys[1] = ws_ptr<uint32_t>(ws, p, even ? WS_DUP_B_K : WS_DUP_A_K);
    a.vals[1] = ws_ptr<uint32_t>(ws, p, even ? WS_DUP_B_V : WS_DUP_A_V);
    a.parity = nullptr;
    a.n_ptr = counts + 1;
    a.capacity = (uint32_t)p->dup_capacity;
    a.hist = hist + (p->depth_passes + pass) * 256;
    a.lookback = ws_ptr<uint32_t>(ws, p, WS_LB_TILE) + (int64_t)pass * sort_tiles_t * 256;
    a.tile_counter = counters + 9 + pass;
    a.shift = 8 * pass;
    a.spin_budget = budget;
    a.status = status_dev;
    launch_onesweep(a, tile_grid, stream);
  }
  // 5. tile ranges
  if (cudaMemsetAsync(base + p->off[SIXDGS_WS_RANGES], 0, p->total_tiles * 8, stream) != cudaSuccess)
    return SIXDGS_ERR_CUDA;
  {
    RangesArgs a;
    a.keys = ws_ptr<uint32_t>(ws, p, SIXDGS_WS_SORTEDKEY);
    a.k_ptr = counts + 1;
    a.capacity = (uint32_t)p->dup_capacity;
    a.total_tiles = (uint32_t)p->total_tiles;
    a.ranges = ws_ptr<uint2>(ws, p, SIXDGS_WS_RANGES);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((p->dup_capacity + 255) / 256, (int64_t)sms * 8));
    launch_ranges(a, grid, stream);
  }
  return launch_status();
}

static BlendArgs blend_args(const sixdgs_plan* p, void* ws) {
  BlendArgs a;
  std::memset(&a, 0, sizeof(a));
  a.cams = ws_ptr<CamRec>(ws, p, SIXDGS_WS_CAMS);
  a.n_cams = p->n_cams;
  a.tile_w = p->settings.tile_w;
  a.tile_h = p->settings.tile_h;
  a.batch = p->settings.batch;
  a.rec = ws_ptr<PairRec>(ws, p, SIXDGS_WS_REC);
  a.n_pairs = (uint32_t)p->n_pairs;
  a.sorted = ws_ptr<uint32_t>(ws, p, SIXDGS_WS_SORTED);
  a.ranges = ws_ptr<uint2>(ws, p, SIXDGS_WS_RANGES);
  for (int i = 0; i < 3; ++i) a.bg[i] = p->settings.bg[i];
  const double norm = p->settings.loss_norm > 0.f ? (double)p->settings.loss_norm
                                                   : 3.0 * (double)p->total_pixels;
  a.inv_count = (float)(1.0 / norm);
  a.nwalk = p->settings.store_aux ? ws_ptr<uint32_t>(ws, p, SIXDGS_WS_NWALK) : nullptr;
  a.pair_counts = p->settings.count_pairs
                      ? reinterpret_cast<unsigned long long*>(ws_ptr<char>(ws, p, SIXDGS_WS_COUNTS) + 16)
                      : nullptr;
  a.tile_queue = p->settings.persistent ? ws_ptr<uint32_t>(ws, p, WS_COUNTERS) + 32 : nullptr;
  a.total_tiles = (uint32_t)p->total_tiles;
  a.spin_budget = spin_budget(p);
  return a;
}

sixdgs_status sixdgs_raster_fwd(const sixdgs_plan* p, void* ws, size_t ws_bytes, float* images_dev,
                                const float* targets_dev, float* grad_images_dev, double* loss_dev,
                                int32_t* status_dev, sixdgs_stream_t stream_) {
  sixdgs_status e = check_ws(p, ws, ws_bytes);
  if (e != SIXDGS_OK) return e;
  if (!images_dev) return SIXDGS_ERR_INVALID_ARG;
  const bool any = targets_dev || grad_images_dev || loss_dev;
  const bool all = targets_dev && grad_images_dev && loss_dev;
  if (any && !all) return SIXDGS_ERR_INVALID_ARG;
  BlendArgs a = blend_args(p, ws);
  a.images = images_dev;
  a.targets = targets_dev;
  a.grad_images = grad_images_dev;
  a.loss = loss_dev;
  a.status = status_dev;
  launch_blend_fwd(a, p->total_tiles, reinterpret_cast<cudaStream_t>(stream_));
  return launch_status();
}

sixdgs_status sixdgs_raster_fwd_bwd(const sixdgs_plan* p, void* ws, size_t ws_bytes, float* images_dev,
                                    const float* targets_dev, float* grad_images_dev, double* loss_dev,
                                    int32_t* status_dev, sixdgs_stream_t stream_) {
  sixdgs_status e = check_ws(p, ws, ws_bytes);
  if (e != SIXDGS_OK) return e;
  if (p->settings.inference || !images_dev || !targets_dev || !loss_dev) return SIXDGS_ERR_INVALID_ARG;
  BlendArgs a = blend_args(p, ws);
  a.images = images_dev;
  a.targets = targets_dev;
  a.grad_images = grad_images_dev;
  a.loss = loss_dev;
  a.grad_rec = ws_ptr<float>(ws, p, SIXDGS_WS_GRADREC);
  a.status = status_dev;
  launch_blend_fused(a, p->total_tiles, reinterpret_cast<cudaStream_t>(stream_));
  return launch_status();
}

sixdgs_status sixdgs_blend_bwd(const sixdgs_plan* p, void* ws, size_t ws_bytes, const float* images_dev,
                               const float* grad_images_dev, int32_t* status_dev, sixdgs_stream_t stream_) {
  sixdgs_status e = check_ws(p, ws, ws_bytes);
  if (e != SIXDGS_OK) return e;
  if (p->settings.inference) return SIXDGS_ERR_INVALID_ARG;
  if (!images_dev || !grad_images_dev) return SIXDGS_ERR_INVALID_ARG;
  BlendArgs a = blend_args(p, ws);
  a.images_in = images_dev;
  a.grad_in = grad_images_dev;
  a.grad_rec = ws_ptr<float>(ws, p, SIXDGS_WS_GRADREC);
  a.recompute = p->settings.store_aux ? 0 : 1;
  a.status = status_dev;
  launch_blend_bwd(a, p->total_tiles, reinterpret_cast<cudaStream_t>(stream_));
  return launch_status();
}

sixdgs_status sixdgs_project_bwd(const sixdgs_plan* p, const sixdgs_scene* scene, void* ws,
                                 size_t ws_bytes, float* grad_mu_p, float* grad_mu_d, float* grad_l_raw,
                                 float* grad_opacity_logit, float* grad_sh, float* grad_lambda_raw,
                                 int32_t accumulate, int32_t* status_dev, sixdgs_stream_t stream_) {
  sixdgs_status e = check_ws(p, ws, ws_bytes);
  if (e != SIXDGS_OK) return e;
  if (p->settings.inference) return SIXDGS_ERR_INVALID_ARG;
  if (!valid_scene(p, scene)) return SIXDGS_ERR_INVALID_ARG;
  if (p->n > 0 && (!grad_mu_p || !grad_mu_d || !grad_l_raw || !grad_opacity_logit || !grad_sh))
    return SIXDGS_ERR_INVALID_ARG;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  ProjectBwdArgs b;
  b.cams = ws_ptr<CamRec>(ws, p, SIXDGS_WS_CAMS);
  b.n_cams = p->n_cams;
  b.n = p->n;
  b.sh_degree = p->sh_degree;
  b.lambda_opa = p->settings.lambda_opa;
  b.mu_p = scene->mu_p;
  b.mu_d = scene->mu_d;
  b.l_raw = scene->l_raw;
  b.opacity_logit = scene->opacity_logit;
  b.sh = scene->sh;
  b.lambda_raw = scene->lambda_raw;
  b.rec = ws_ptr<PairRec>(ws, p, SIXDGS_WS_REC);
  b.ntiles = ws_ptr<uint32_t>(ws, p, SIXDGS_WS_NTILES);
  b.grad_rec = ws_ptr<float>(ws, p, SIXDGS_WS_GRADREC);
  b.grad_mu_p = grad_mu_p;
  b.grad_mu_d = grad_mu_d;
  b.grad_l_raw = grad_l_raw;
  b.grad_opacity_logit = grad_opacity_logit;
  b.grad_sh = grad_sh;
  b.grad_lambda_raw = grad_lambda_raw;
  b.accumulate = accumulate;
  b.bulk = bulk_planes(p->n, {b.mu_p, b.mu_d, b.l_raw, b.opacity_logit, b.sh, b.lambda_raw});
  b.spin_budget = spin_budget(p);
  b.status = status_dev;
  launch_sh_bwd(b, stream);
  launch_geom_bwd(b, stream);
  return launch_status();
}

sixdgs_status sixdgs_raster_bwd(const sixdgs_plan* p, const sixdgs_scene* scene, void* ws,
                                size_t ws_bytes, const float* images_dev,
                                const float* grad_images_dev, float* grad_mu_p, float* grad_mu_d,
                                float* grad_l_raw, float* grad_opacity_logit, float* grad_sh,
                                float* grad_lambda_raw, int32_t accumulate, int32_t* status_dev,
                                sixdgs_stream_t stream) {
  sixdgs_status e = check_ws(p, ws, ws_bytes);
  if (e != SIXDGS_OK) return e;
  if (p->settings.inference) return SIXDGS_ERR_INVALID_ARG;
  if (!valid_scene(p, scene)) return SIXDGS_ERR_INVALID_ARG;
  if (p->n > 0 && (!grad_mu_p || !grad_mu_d || !grad_l_raw || !grad_opacity_logit || !grad_sh))
    return SIXDGS_ERR_INVALID_ARG;
  e = sixdgs_blend_bwd(p, ws, ws_bytes, images_dev, grad_images_dev, status_dev, stream);
  if (e != SIXDGS_OK) return e;
  return sixdgs_project_bwd(p, scene, ws, ws_bytes, grad_mu_p, grad_mu_d, grad_l_raw, grad_opacity_logit,
                            grad_sh, grad_lambda_raw, accumulate, status_dev, stream);
}

sixdgs_status sixdgs_render_batched(const sixdgs_plan* p, const sixdgs_scene* scene,
                                    const sixdgs_camera* cams_host, void* ws, size_t ws_bytes,
                                    float* images_dev, const float* targets_dev, float* grad_images_dev,
                                    double* loss_dev, float* grad_mu_p, float* grad_mu_d, float* grad_l_raw,
                                    float* grad_opacity_logit, float* grad_sh, float* grad_lambda_raw,
                                    int32_t* status_dev, sixdgs_stream_t stream) {
  sixdgs_status e = check_ws(p, ws, ws_bytes);
  if (e != SIXDGS_OK) return e;
  const bool train = targets_dev != nullptr;
  if (train) {
    if (p->settings.inference || !loss_dev || !valid_scene(p, scene)) return SIXDGS_ERR_INVALID_ARG;
    if (p->n > 0 && (!grad_mu_p || !grad_mu_d || !grad_l_raw || !grad_opacity_logit || !grad_sh))
      return SIXDGS_ERR_INVALID_ARG;
    if (cudaMemsetAsync(loss_dev, 0, sizeof(double), reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
      return SIXDGS_ERR_CUDA;
  }
  e = sixdgs_condition_project(p, scene, cams_host, ws, ws_bytes, status_dev, stream);
  if (e != SIXDGS_OK) return e;
  e = sixdgs_bin_sort(p, ws, ws_bytes, status_dev, stream);
  if (e != SIXDGS_OK) return e;
  if (!train) return sixdgs_raster_fwd(p, ws, ws_bytes, images_dev, nullptr, nullptr, nullptr, status_dev, stream);
  e = sixdgs_raster_fwd_bwd(p, ws, ws_bytes, images_dev, targets_dev, grad_images_dev, loss_dev, status_dev,
                            stream);
  if (e != SIXDGS_OK) return e;
  return sixdgs_project_bwd(p, scene, ws, ws_bytes, grad_mu_p, grad_mu_d, grad_l_raw, grad_opacity_logit,
                            grad_sh, grad_lambda_raw, 0, status_dev, stream);
}

sixdgs_status sixdgs_peak_probe(int32_t kind, int64_t iters, float* out_dev, int32_t blocks,
                                sixdgs_stream_t stream) {
  if ((kind != 0 && kind != 1) || iters < 0 || blocks < 1 || !out_dev) return SIXDGS_ERR_INVALID_ARG;
  launch_peak_probe(kind, iters, out_dev, blocks, reinterpret_cast<cudaStream_t>(stream));
  return launch_status();
}

sixdgs_status sixdgs_condition_cache(int64_t n, const float* l_raw_dev, const float* opacity_logit_dev,
                                     float* cache_dev, sixdgs_stream_t stream) {
  if (n < 0 || (n > 0 && (!l_raw_dev || !opacity_logit_dev || !cache_dev))) return SIXDGS_ERR_INVALID_ARG;
  CondCacheArgs a;
  a.n = n;
  a.l_raw = l_raw_dev;
  a.opacity_logit = opacity_logit_dev;
  a.cache = cache_dev;
  launch_cond_cache(a, reinterpret_cast<cudaStream_t>(stream));
  return launch_status();
}

sixdgs_status sixdgs_scale_rotation(int64_t n, const float* l_raw_dev, float* rotation_dev, float* scale_dev,
                                    int32_t* status_dev, sixdgs_stream_t stream) {
  if (n < 0 || (n > 0 && (!l_raw_dev || !rotation_dev || !scale_dev))) return SIXDGS_ERR_INVALID_ARG;
  ScaleRotationArgs a;
  a.n = n;
  a.l_raw = l_raw_dev;
  a.rotation = rotation_dev;
  a.scale = scale_dev;
  a.status = status_dev;
  launch_scale_rotation(a, reinterpret_cast<cudaStream_t>(stream));
  return launch_status();
}

}  // extern "C"
