// vg_downsample_noalloc: the same decimation as vg_downsample for callers that cannot
// call cudaMalloc, because they run where an allocation is not allowed or not possible:
// a real-time sensor callback that must never block (cudaMalloc can synchronise the
// whole device), or a host program whose device memory belongs to another allocator and
// that has no way to hand the library a workspace.
//
// The scratch lives in a file-scope __device__ array sized for VG_NOALLOC_MAX_POINTS
// points (the sort-path workspace for that many points, about 25 MB).  Every GPU that
// loads this module keeps the array until the process exits.  Nothing here allocates:
// the call looks up the array's device address once per device and then runs the
// ordinary vg_downsample (sort path only) on it.  A cudaDeviceReset unloads the module;
// the cached address is then stale, so the entry point is not for use after a reset.
#include <mutex>

#include "../../include/vg.h"
#include "vg_internal.h"

namespace {

constexpr int64_t kMaxPoints = VG_NOALLOC_MAX_POINTS;
constexpr size_t kScratchBytes = vg::sort_layout(kMaxPoints).total;

// Device scratch shared by every call on a device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (host code may not use the symbol
// itself: on the host it names a stand-in object, not device memory).
vg_status scratch_for_current_device(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return VG_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) return VG_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return VG_OK;
}

}  // namespace

extern "C" {

vg_status vg_downsample_noalloc(const float* xyz, int64_t n, float* origin, float leaf,
                                uint64_t* out_keys, float* out_centroids, uint32_t* out_counts,
                                int64_t cap, int64_t* out_num_voxels, int32_t* out_point_to_voxel,
                                int32_t* out_error, int flags, vg_stream_t stream) {
  if (n < 0 || n > kMaxPoints) return VG_ERR_INVALID_ARG;
  // The array is sized for the sort path's workspace; the hash path and the single-frame
  // bin grouping need more.
  if ((flags & VG_METHOD_MASK) == VG_METHOD_HASH || (flags & VG_SORT_FRAME) != 0)
    return VG_ERR_INVALID_ARG;
  void* scratch = nullptr;
  const vg_status s = scratch_for_current_device(&scratch);
  if (s != VG_OK) return s;
  return vg_downsample(xyz, n, origin, leaf, out_keys, out_centroids, out_counts, cap,
                       out_num_voxels, out_point_to_voxel, out_error, scratch, kScratchBytes,
                       flags, stream);
}

size_t vg_downsample_noalloc_scratch_bytes(void) { return kScratchBytes; }

}  // extern "C"
