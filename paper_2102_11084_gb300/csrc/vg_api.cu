// C ABI entry points of libvg.so (declared in include/vg.h): argument checks, workspace
// layout and the launch sequence of each call.  No allocation happens here.
#include <atomic>
#include <cmath>
#include <cstring>

#include "../../include/vg.h"
#include "vg_internal.h"

namespace vg {

namespace {
std::atomic<uint32_t> g_spin_limit{0};
void** g_events = nullptr;
int g_max_events = 0;
constexpr int kSortStages = 3 + kMaxPasses;

// Records profiling event k on `stream` when the stage-event hook is on.
void mark(int k, cudaStream_t stream) {
  if (g_events && k < g_max_events && g_events[k])
    cudaEventRecord(static_cast<cudaEvent_t>(g_events[k]), stream);
}
int g_sms[64] = {0};
}  // namespace

uint32_t spin_limit() {
  const uint32_t v = g_spin_limit.load(std::memory_order_relaxed);
  return v ? v : kDefaultSpinLimit;
}

int num_sms() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 132;
  if (g_sms[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
      v = 132;
    g_sms[dev] = v;
  }
  return g_sms[dev];
}

}  // namespace vg

using namespace vg;

namespace {

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

vg_status cuda_status(cudaError_t e) { return e == cudaSuccess ? VG_OK : VG_ERR_CUDA; }

}  // namespace

extern "C" {

const char* vg_status_string(int status) {
  switch (status) {
    case VG_OK: return "ok";
    case VG_ERR_INVALID_ARG: return "invalid argument";
    case VG_ERR_ALIGN: return "misaligned pointer";
    case VG_ERR_RANGE: return "voxel index out of range [0, 2^21)";
    case VG_ERR_CAPACITY: return "more voxels than the output capacity";
    case VG_ERR_WORKSPACE: return "workspace missing or too small";
    case VG_ERR_TIMEOUT: return "chained-scan wait timed out";
    case VG_ERR_CUDA: return "CUDA error";
    default: return "unknown status";
  }
}

int vg_version(void) { return 100; }

int vg_set_stage_events(void** events, int max_events) {
  g_events = events;
  g_max_events = events ? max_events : 0;
  return kSortStages;
}

void vg_debug_set_spin_limit(uint32_t limit) {
  g_spin_limit.store(limit, std::memory_order_relaxed);
}

size_t vg_downsample_workspace_bytes(int64_t n_points, int flags) {
  (void)flags;
  if (n_points < 0) return 0;
  return sort_layout(n_points).total;
}

vg_status vg_downsample(const float* xyz, int64_t n, float* origin, float leaf,
                        uint64_t* out_keys, float* out_centroids, uint32_t* out_counts,
                        int64_t cap, int64_t* out_num_voxels, int32_t* out_point_to_voxel,
                        int32_t* out_error, void* workspace, size_t workspace_bytes, int flags,
                        vg_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (n < 0 || n > kMaxPoints || cap < 0) return VG_ERR_INVALID_ARG;
  if (!(leaf > 0.0f) || !std::isfinite(leaf)) return VG_ERR_INVALID_ARG;
  if ((flags & ~(VG_ORIGIN_FROM_MIN | VG_METHOD_SORT)) != 0) return VG_ERR_INVALID_ARG;
  if (!origin || !out_num_voxels || (n > 0 && !xyz)) return VG_ERR_INVALID_ARG;
  if (cap > 0 && (!out_keys || !out_centroids || !out_counts)) return VG_ERR_INVALID_ARG;
  if (!aligned(xyz, 4) || !aligned(origin, 4) || !aligned(out_keys, 8) ||
      !aligned(out_centroids, 4) || !aligned(out_counts, 4) || !aligned(out_num_voxels, 8) ||
      !aligned(out_point_to_voxel, 4) || !aligned(out_error, 4) || !aligned(workspace, 256))
    return VG_ERR_ALIGN;
  const SortLayout L = sort_layout(n);
  if (!workspace || workspace_bytes < L.total) return VG_ERR_WORKSPACE;

  char* ws = static_cast<char*>(workspace);
  State* st = reinterpret_cast<State*>(ws + L.state);
  uint64_t* keys0 = reinterpret_cast<uint64_t*>(ws + L.keys0);
  uint64_t* keys1 = reinterpret_cast<uint64_t*>(ws + L.keys1);
  uint32_t* idx0 = reinterpret_cast<uint32_t*>(ws + L.idx0);
  uint32_t* idx1 = reinterpret_cast<uint32_t*>(ws + L.idx1);
  uint32_t* lb_a = reinterpret_cast<uint32_t*>(ws + L.lb_a);
  uint32_t* lb_b = reinterpret_cast<uint32_t*>(ws + L.lb_b);
  SegStatus* seg_lb = reinterpret_cast<SegStatus*>(ws + L.seg_lb);
  int* err = out_error ? reinterpret_cast<int*>(out_error) : &st->error;
  const uint32_t spins = spin_limit();
  const bool from_min = (flags & VG_ORIGIN_FROM_MIN) != 0;

  cudaError_t e = cudaMemsetAsync(ws, 0, L.zero_bytes, stream);
  if (e == cudaSuccess && out_error) e = cudaMemsetAsync(out_error, 0, sizeof(int32_t), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(out_num_voxels, 0, sizeof(int64_t), stream);
  if (e == cudaSuccess && out_point_to_voxel && n > 0)
    e = cudaMemsetAsync(out_point_to_voxel, 0xff, size_t(n) * sizeof(int32_t), stream);
  mark(0, stream);
  if (e == cudaSuccess && from_min) e = launch_origin(xyz, n, st, stream);
  mark(1, stream);
  if (e == cudaSuccess) e = launch_keys(xyz, n, origin, from_min, leaf, st, keys0, err, stream);
  mark(2, stream);
  for (int p = 0; p < kMaxPasses && e == cudaSuccess; ++p) {
    e = launch_sort_pass(st, keys0, idx0, keys1, idx1, lb_a, lb_b, n, p, spins, err, stream);
    mark(3 + p, stream);
  }
  if (e == cudaSuccess)
    e = launch_segreduce(st, keys0, idx0, keys1, idx1, xyz, leaf, seg_lb, n, out_keys,
                         out_centroids, out_counts, cap, out_num_voxels, out_point_to_voxel,
                         spins, err, stream);
  mark(3 + kMaxPasses, stream);
  return cuda_status(e);
}

}  // extern "C"
