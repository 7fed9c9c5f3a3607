// Host-side helpers of libgs: status strings, version, frame layout.
#include <string.h>

#include <atomic>

#include "gs_common.cuh"

extern "C" const char *gs_status_str(gs_status_t s) {
  switch (s) {
    case GS_OK: return "ok";
    case GS_ERR_INVALID_ARG: return "invalid argument";
    case GS_ERR_CAPACITY: return "device-side capacity exceeded";
    case GS_ERR_CUDA: return "CUDA error";
    case GS_ERR_TIMEOUT: return "bounded device wait timed out";
    case GS_ERR_UNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}

namespace gs {
static std::atomic<uint64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace gs

extern "C" uint64_t gs_launch_count(void) { return gs::g_launches.load(std::memory_order_relaxed); }

extern "C" const char *gs_version(void) { return "libgs 0.1 (sm_103a)"; }

extern "C" gs_status_t gs_frame_init(gs_camera_t *cams, int32_t n_views, int32_t tile_w, int32_t tile_h,
                                     gs_frame_t *frame) {
  if (!cams || !frame || n_views <= 0 || !gs_tile_supported(tile_w, tile_h)) return GS_ERR_INVALID_ARG;
  int64_t tiles = 0, pixels = 0;
  int32_t mw = 0, mh = 0;
  for (int v = 0; v < n_views; ++v) {
    gs_camera_t &c = cams[v];
    if (c.width <= 0 || c.height <= 0 || !(c.fx > 0.f) || !(c.fy > 0.f) || !(c.near_plane > 0.f))
      return GS_ERR_INVALID_ARG;
    c.grid_x = (c.width + tile_w - 1) / tile_w;
    c.grid_y = (c.height + tile_h - 1) / tile_h;
    if (c.grid_x > 65535 || c.grid_y > 65535) return GS_ERR_INVALID_ARG;
    c.tile_offset = (int32_t)tiles;
    c.pixel_offset = pixels;
    tiles += (int64_t)c.grid_x * c.grid_y;
    pixels += (int64_t)c.width * c.height;
    if (tiles >= (1ll << 31)) return GS_ERR_INVALID_ARG;
    mw = c.width > mw ? c.width : mw;
    mh = c.height > mh ? c.height : mh;
  }
  memset(frame, 0, sizeof(*frame));
  frame->n_views = n_views;
  frame->tile_w = tile_w;
  frame->tile_h = tile_h;
  frame->n_tiles = (int32_t)tiles;
  frame->n_pixels = pixels;
  frame->max_width = mw;
  frame->max_height = mh;
  return GS_OK;
}

// The first failed bounds check of a debug build since the last call, as
// (code << 48 | index), 0 if none; clears it. Release builds: GS_ERR_UNSUPPORTED.
extern "C" gs_status_t gs_debug_status(uint64_t *word) {
  if (!word) return GS_ERR_INVALID_ARG;
  *word = 0;
#ifdef GS_DEBUG
  const uint64_t a = gs::debug_take_raster(), b = gs::debug_take_bin_sort();
  if (a == ~0ull || b == ~0ull) return GS_ERR_CUDA;
  *word = a ? a : b;
  return GS_OK;
#else
  return GS_ERR_UNSUPPORTED;
#endif
}
