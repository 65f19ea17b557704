// Allocation-free forward render: the same three forward stages as
// sixdgs_condition_project + sixdgs_bin_sort + sixdgs_raster_fwd, with the
// frame's workspace placed in a file-scope device array instead of a
// caller-provided buffer.
//
// Meant for callers that cannot allocate device memory themselves: code
// running inside a host application whose allocator owns all device memory
// (plugins, engines with a fixed memory budget), or latency-critical loops
// that must not call cudaMalloc.  The array is SIXDGS_STATIC_WS_BYTES long
// and every device that loads the library keeps it until the process exits.
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace {

// Workspace shared by every call of sixdgs_render_fwd_static on a device.
static __device__ __align__(256) unsigned char g_static_ws[SIXDGS_STATIC_WS_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_static_ptr[kMaxDevices] = {nullptr};

// Device address of g_static_ws on the current device (looked up once per
// device; in host code the symbol itself is only a host-side handle).
sixdgs_status static_ws_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SIXDGS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_ws) != cudaSuccess || !p) return SIXDGS_ERR_CUDA;
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return SIXDGS_OK;
}

}  // namespace

extern "C" sixdgs_status sixdgs_render_fwd_static(int64_t n, int32_t sh_degree, const sixdgs_scene* scene,
                                                  const sixdgs_camera* cams, int32_t n_cams,
                                                  const sixdgs_settings* settings, float* images_dev,
                                                  int32_t* status_dev, sixdgs_stream_t stream) {
  if (!scene || !cams || !settings || !images_dev) return SIXDGS_ERR_INVALID_ARG;
  // A forward-only frame: plan it as one (no gradient-record section, no
  // per-pixel walk lengths), so the fixed array holds as many pairs as it can.
  sixdgs_settings fwd = *settings;
  fwd.inference = 1;
  fwd.store_aux = 0;
  sixdgs_plan plan;
  sixdgs_status e = sixdgs_plan_init(n, sh_degree, cams, n_cams, &fwd, 0, &plan);
  if (e != SIXDGS_OK) return e;
  if (plan.ws_bytes > (int64_t)SIXDGS_STATIC_WS_BYTES) return SIXDGS_ERR_WORKSPACE;
  void* ws = nullptr;
  e = static_ws_address(&ws);
  if (e != SIXDGS_OK) return e;
  const size_t bytes = SIXDGS_STATIC_WS_BYTES;
  e = sixdgs_condition_project(&plan, scene, cams, ws, bytes, status_dev, stream);
  if (e != SIXDGS_OK) return e;
  e = sixdgs_bin_sort(&plan, ws, bytes, status_dev, stream);
  if (e != SIXDGS_OK) return e;
  return sixdgs_raster_fwd(&plan, ws, bytes, images_dev, nullptr, nullptr, nullptr, status_dev, stream);
}
