// Kernel argument blocks and host launchers of the sixdgs library.
#pragma once

#include "common.cuh"

namespace sixdgs {

struct ProjectArgs {
  const CamRec* cams;
  int32_t n_cams;
  int64_t n;
  int32_t sh_degree;
  float lambda_opa;
  float inv_tile_w, inv_tile_h;
  int32_t alpha_footprint;   // 1: tile rect within the alpha >= 1/255 box
  const float* mu_p;
  const float* mu_d;
  const float* l_raw;
  const float* opacity_logit;
  const float* sh;
  const float* lambda_raw;   // optional per-Gaussian lambda_opa (pre-sigmoid)
  const float* cond_cache;   // optional cached view-independent state
  PairRec* rec;
  uint32_t* ntiles;
  ushort4* rect;
  uint32_t* depth_key;
  float* grad_rec;   // zeroed for every visible pair (read by the backward); null: inference plan
  int32_t bulk;      // 1: every parameter plane segment can be staged with bulk copies
  int64_t spin_budget;
  int32_t* status;
};

// Visible-pair compaction (scan of ntiles > 0) feeding the depth sort.
struct CompactArgs {
  const uint32_t* ntiles;
  const uint32_t* depth_key;
  int64_t n_pairs;
  uint32_t* keys_out;
  uint32_t* vals_out;
  uint32_t* n_vis_out;
  unsigned long long* scan_state;  // one word per scan tile
  uint32_t* tile_counter;
  uint32_t* hist;                  // passes x 256
  int32_t passes;
  int64_t spin_budget;
  int32_t* status;
};

struct OnesweepArgs {
  uint32_t* keys[2];       // the two key buffers; data moves from one to the other
  uint32_t* vals[2];
  // null: input in keys[0], output in keys[1]; else *parity is the input
  // buffer and the pass writes its output buffer to parity[1] (an identity
  // pass leaves the data where it is)
  uint32_t* parity;
  const uint32_t* n_ptr;   // element count (device)
  uint32_t capacity;       // buffer size; counts above it are clamped
  const uint32_t* hist;    // 256 digit counts of this pass
  uint32_t* lookback;      // tiles x 256 status words of this pass
  uint32_t* tile_counter;
  int32_t shift;
  int64_t spin_budget;
  int32_t* status;
};

// Duplicate emission in depth order (scan of ntiles over the depth-sorted
// visible pairs) feeding the tile sort.
struct EmitArgs {
  const uint32_t* pairs[2];   // depth-sorted visible pair indices: pairs[*depth_parity]
  const uint32_t* depth_parity;
  const uint32_t* n_vis;
  const uint32_t* ntiles;
  const ushort4* rect;
  const CamRec* cams;
  int64_t n;                  // Gaussians per camera
  uint32_t n_pairs;
  uint32_t* keys_out;         // global tile id
  uint32_t* vals_out;         // pair index
  uint32_t* dup_off[2];       // first output of each depth-sorted pair (n_vis): dup_off[*depth_parity]
  uint32_t* chunk_first;      // pair owning the first output of each chunk
  uint64_t capacity;
  uint32_t* k_out;            // number of duplicates (may exceed capacity)
  unsigned long long* scan_state;
  uint32_t* tile_counter;
  uint32_t* hist;
  int32_t passes;
  int64_t spin_budget;
  int32_t* status;
};

struct RangesArgs {
  const uint32_t* keys;
  const uint32_t* k_ptr;
  uint32_t capacity;
  uint32_t total_tiles;
  uint2* ranges;
};

struct BlendArgs {
  const CamRec* cams;
  int32_t n_cams;
  int32_t tile_w, tile_h, batch;
  const PairRec* rec;
  uint32_t n_pairs;
  const uint32_t* sorted;   // pair index per list entry
  const uint2* ranges;
  float bg[3];
  float* images;
  const float* targets;
  float* grad_images;
  double* loss;
  float inv_count;          // 1 / (3 * total_pixels)
  uint32_t* nwalk;          // optional per-pixel walk length
  unsigned long long* pair_counts;  // optional: evaluated, compositing pairs
  // backward
  const float* images_in;
  const float* grad_in;
  float* grad_rec;          // n_pairs x 12
  int32_t recompute;        // 1: re-derive the stop; 0: use nwalk
  // persistent mode: tiles are taken from this counter (NULL: one CTA per tile)
  uint32_t* tile_queue;
  uint32_t total_tiles;
  int64_t spin_budget;      // clock cycles a shared-memory ring wait may take
  int32_t* status;
};

struct ProjectBwdArgs {
  const CamRec* cams;
  int32_t n_cams;
  int64_t n;
  int32_t sh_degree;
  float lambda_opa;
  const float* mu_p;
  const float* mu_d;
  const float* l_raw;
  const float* opacity_logit;
  const float* sh;
  const float* lambda_raw;
  const PairRec* rec;
  const uint32_t* ntiles;
  const float* grad_rec;
  float* grad_mu_p;
  float* grad_mu_d;
  float* grad_l_raw;
  float* grad_opacity_logit;
  float* grad_sh;
  float* grad_lambda_raw;
  int32_t accumulate;   // 1: add into the outputs instead of overwriting
  int32_t bulk;         // 1: the parameter planes can be staged with bulk copies
  int64_t spin_budget;
  int32_t* status;
};

struct CondCacheArgs {
  int64_t n;
  const float* l_raw;
  const float* opacity_logit;
  float* cache;      // kCondCachePlanes planes of n floats
};

constexpr int kCondCachePlanes = 25;

struct ScaleRotationArgs {
  int64_t n;
  const float* l_raw;
  float* rotation;   // 9 planes, R row-major
  float* scale;      // 3 planes
  int32_t* status;
};

void launch_project_fwd(const ProjectArgs& a, cudaStream_t stream);
void launch_scale_rotation(const ScaleRotationArgs& a, cudaStream_t stream);
void launch_cond_cache(const CondCacheArgs& a, cudaStream_t stream);
void launch_peak_probe(int kind, int64_t iters, float* out, int blocks, cudaStream_t stream);
void launch_compact(const CompactArgs& a, int grid, cudaStream_t stream);
void launch_onesweep(const OnesweepArgs& a, int grid, cudaStream_t stream);
void launch_emit(const EmitArgs& a, int scan_grid, int expand_grid, cudaStream_t stream);
void launch_ranges(const RangesArgs& a, int grid, cudaStream_t stream);
void launch_blend_fwd(const BlendArgs& a, int64_t total_tiles, cudaStream_t stream);
void launch_blend_fused(const BlendArgs& a, int64_t total_tiles, cudaStream_t stream);
void launch_blend_bwd(const BlendArgs& a, int64_t total_tiles, cudaStream_t stream);
void launch_sh_bwd(const ProjectBwdArgs& a, cudaStream_t stream);
void launch_geom_bwd(const ProjectBwdArgs& a, cudaStream_t stream);

// Tile geometry of the scans and sorts (elements per block tile).
constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;
// the visible-pair compaction: more items per thread (loads in flight, fewer
// look-back steps); a multiple of 4, so its tiles never outnumber the scan
// tiles the workspace has state for
#ifndef SIXDGS_COMPACT_ITEMS
#define SIXDGS_COMPACT_ITEMS 16
#endif
constexpr int kCompactItems = SIXDGS_COMPACT_ITEMS;
constexpr int kCompactTile = kScanThreads * kCompactItems;
static_assert(kCompactItems % 4 == 0 && kCompactTile >= kScanTile, "compaction tile");
constexpr int kSortThreads = 256;
constexpr int kSortItems = 12;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kEmitChunk = 512;    // duplicates written per expansion chunk

}  // namespace sixdgs
