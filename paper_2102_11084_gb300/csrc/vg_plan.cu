// The batch plan: a reusable object for step a8 (many frames of uneven size per call).
//
// A plan owns the workspace for up to max_points points in max_frames frames (allocated
// once, at creation -- never on the hot path), the grouping method and streaming-grid
// size chosen by its autotuner, and a CUDA graph of the whole launch sequence (memsets,
// origin, keys or hash insert, radix passes, reduction) so that a batch costs one graph
// launch on the host.  The graph is captured on first use and replayed while the call's
// pointers, sizes and flags stay the same; kernels read the frame table, leaves and
// counts from device memory, so new data in the same buffers needs no re-capture.
//
// The paper spreads the subdivisions of space over all CUDA processors (Sec. II-C,
// "processed independently"); here every frame's chunks go to the same persistent
// streaming grid and one radix sort orders all frames at once (frame id above the
// voxel key).
#include <cstring>
#include <new>

#include "../../include/vg.h"
#include "vg_api_internal.h"
#include "vg_internal.h"

struct vg_plan {
  int device = 0;
  int max_frames = 0;
  int64_t max_points = 0;
  int method = VG_METHOD_SORT;
  int grid_per_sm = 0;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  cudaGraphExec_t exec = nullptr;
  // arguments the captured graph was built with
  struct Key {
    const void* p[10];
    int64_t n_total, cap;
    int n_frames, flags;
    bool operator==(const Key& o) const { return std::memcmp(this, &o, sizeof(Key)) == 0; }
  } key{};
};

namespace {

int plan_flags(const vg_plan* p, int flags) {
  return (flags & VG_ORIGIN_FROM_MIN) | p->method | (p->grid_per_sm << VG_GRID_SHIFT);
}

// The grouping choices a plan holds: the sort (bucket grouping for 32-bit keys), the sort
// with every digit in global radix passes, the single-frame bin grouping, and the hash
// path.
bool plan_method_ok(int m) {
  return m == VG_METHOD_AUTO || m == VG_METHOD_SORT || m == (VG_METHOD_SORT | VG_SORT_LSD) ||
         m == (VG_METHOD_SORT | VG_SORT_FRAME) || m == VG_METHOD_HASH;
}

void drop_graph(vg_plan* p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  p->exec = nullptr;
}

}  // namespace

extern "C" {

vg_status vg_plan_create(vg_plan** out, int max_frames, int64_t max_points, int flags) {
  if (!out || max_frames < 1 || max_frames > vg::kMaxFrames || max_points < 0 ||
      max_points > vg::kMaxPoints)
    return VG_ERR_INVALID_ARG;
  const int m = flags & VG_METHOD_MASK;
  if (m == VG_METHOD_MASK) return VG_ERR_INVALID_ARG;
  *out = nullptr;
  vg_plan* p = new (std::nothrow) vg_plan();
  if (!p) return VG_ERR_CUDA;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    return VG_ERR_CUDA;
  }
  p->max_frames = max_frames;
  p->max_points = max_points;
  p->method = m == VG_METHOD_HASH
                  ? VG_METHOD_HASH
                  : (m == VG_METHOD_AUTO ? VG_METHOD_AUTO
                                         : (VG_METHOD_SORT | (flags & (VG_SORT_LSD | VG_SORT_FRAME))));
  if (p->method == (VG_METHOD_SORT | VG_SORT_LSD | VG_SORT_FRAME)) {
    delete p;
    return VG_ERR_INVALID_ARG;
  }
  // room for every grouping a later configure may pick
  const size_t a = vg::frames_workspace_bytes(max_points, max_frames, VG_METHOD_SORT | VG_SORT_FRAME);
  const size_t b = vg::frames_workspace_bytes(max_points, max_frames, VG_METHOD_HASH);
  p->ws_bytes = a > b ? a : b;
  if (cudaMalloc(&p->ws, p->ws_bytes) != cudaSuccess) {
    delete p;
    return VG_ERR_CUDA;
  }
  vg::warm_launch_config();  // occupancy queries happen here, never inside a capture
  *out = p;
  return VG_OK;
}

vg_status vg_plan_destroy(vg_plan* p) {
  if (!p) return VG_ERR_INVALID_ARG;
  drop_graph(p);
  cudaError_t e = cudaFree(p->ws);
  delete p;
  return e == cudaSuccess ? VG_OK : VG_ERR_CUDA;
}

vg_status vg_plan_configure(vg_plan* p, int method, int grid_per_sm) {
  if (!p || !plan_method_ok(method) || grid_per_sm < 0 || grid_per_sm > 255)
    return VG_ERR_INVALID_ARG;
  if (method != p->method || grid_per_sm != p->grid_per_sm) drop_graph(p);
  p->method = method;
  p->grid_per_sm = grid_per_sm;
  return VG_OK;
}

vg_status vg_plan_get(const vg_plan* p, int* method, int* grid_per_sm, size_t* workspace_bytes) {
  if (!p) return VG_ERR_INVALID_ARG;
  if (method) *method = p->method;
  if (grid_per_sm) *grid_per_sm = p->grid_per_sm;
  if (workspace_bytes) *workspace_bytes = p->ws_bytes;
  return VG_OK;
}

vg_status vg_downsample_batch(vg_plan* p, const float* xyz, int64_t n_total,
                              const int64_t* frame_offsets, int n_frames, float* origins,
                              const float* leaves, uint64_t* out_keys, float* out_centroids,
                              uint32_t* out_counts, int64_t cap, int64_t* out_frame_offsets,
                              int32_t* out_point_to_voxel, int32_t* out_error, int flags,
                              vg_stream_t stream_) {
  if (!p) return VG_ERR_INVALID_ARG;
  if ((flags & ~(VG_ORIGIN_FROM_MIN | VG_USE_GRAPH)) != 0) return VG_ERR_INVALID_ARG;
  if (n_total > p->max_points || n_frames > p->max_frames) return VG_ERR_INVALID_ARG;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  const int f = plan_flags(p, flags);
  if (!(flags & VG_USE_GRAPH))
    return vg_downsample_frames(xyz, n_total, frame_offsets, n_frames, origins, leaves, out_keys,
                                out_centroids, out_counts, cap, out_frame_offsets,
                                out_point_to_voxel, out_error, p->ws, p->ws_bytes, f, stream_);
  if (!stream) return VG_ERR_INVALID_ARG;  // the legacy stream cannot be captured
  vg_plan::Key k{};
  const void* ptrs[10] = {xyz, frame_offsets, origins, leaves, out_keys, out_centroids,
                          out_counts, out_frame_offsets, out_point_to_voxel, out_error};
  std::memcpy(k.p, ptrs, sizeof(ptrs));
  k.n_total = n_total;
  k.cap = cap;
  k.n_frames = n_frames;
  k.flags = f;
  if (!p->exec || !(k == p->key)) {
    drop_graph(p);
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return VG_ERR_CUDA;
    vg::pause_stage_events(true);
    const vg_status s = vg_downsample_frames(xyz, n_total, frame_offsets, n_frames, origins,
                                             leaves, out_keys, out_centroids, out_counts, cap,
                                             out_frame_offsets, out_point_to_voxel, out_error,
                                             p->ws, p->ws_bytes, f, stream_);
    vg::pause_stage_events(false);
    const cudaError_t ec = cudaStreamEndCapture(stream, &g);
    if (s != VG_OK || ec != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return s != VG_OK ? s : VG_ERR_CUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&p->exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      p->exec = nullptr;
      return VG_ERR_CUDA;
    }
    p->key = k;
  }
  return cudaGraphLaunch(p->exec, stream) == cudaSuccess ? VG_OK : VG_ERR_CUDA;
}

vg_status vg_plan_tune(vg_plan* p, const float* xyz, int64_t n_total,
                       const int64_t* frame_offsets, int n_frames, float* origins,
                       const float* leaves, uint64_t* out_keys, float* out_centroids,
                       uint32_t* out_counts, int64_t cap, int64_t* out_frame_offsets,
                       int32_t* out_error, int flags, int reps, vg_stream_t stream_,
                       float* out_ms) {
  if (!p || reps < 1) return VG_ERR_INVALID_ARG;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  const int methods[4] = {VG_METHOD_SORT, VG_METHOD_SORT | VG_SORT_LSD,
                          VG_METHOD_SORT | VG_SORT_FRAME, VG_METHOD_HASH};
  const int grids[3] = {4, 8, 16};
  // the device error word of the tuning runs: a grouping that records an error (the bin
  // grouping of keys wider than 32 bits) is not a candidate
  const int32_t* errw = out_error ? out_error : &reinterpret_cast<const vg::State*>(p->ws)->error;
  float best = 3.0e38f;
  int best_m = p->method, best_g = p->grid_per_sm;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return VG_ERR_CUDA;
  vg_status result = VG_OK;
  int slot = 0;
  for (int mi = 0; mi < 4 && result == VG_OK; ++mi) {
    for (int gi = 0; gi < 3 && result == VG_OK; ++gi, ++slot) {
      if ((methods[mi] & VG_SORT_FRAME) != 0 && n_frames != 1) {  // several frames: SORT
        if (out_ms) out_ms[slot] = -1.0f;
        continue;
      }
      vg_plan_configure(p, methods[mi], grids[gi]);
      // one untimed run (captures the graph), then `reps` timed replays
      result = vg_downsample_batch(p, xyz, n_total, frame_offsets, n_frames, origins, leaves,
                                   out_keys, out_centroids, out_counts, cap, out_frame_offsets,
                                   nullptr, out_error, flags | VG_USE_GRAPH, stream_);
      if (result != VG_OK) break;
      cudaEventRecord(e0, stream);
      for (int r = 0; r < reps && result == VG_OK; ++r)
        result = vg_downsample_batch(p, xyz, n_total, frame_offsets, n_frames, origins, leaves,
                                     out_keys, out_centroids, out_counts, cap, out_frame_offsets,
                                     nullptr, out_error, flags | VG_USE_GRAPH, stream_);
      cudaEventRecord(e1, stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        result = VG_ERR_CUDA;
        break;
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= float(reps);
      int32_t werr = 0;
      if (cudaMemcpy(&werr, errw, sizeof(werr), cudaMemcpyDeviceToHost) != cudaSuccess) {
        result = VG_ERR_CUDA;
        break;
      }
      if (werr != 0) {  // not a candidate; the next runs start from a clear word
        ms = -1.0f;
        if (cudaMemset(const_cast<int32_t*>(errw), 0, sizeof(int32_t)) != cudaSuccess) {
          result = VG_ERR_CUDA;
          break;
        }
      }
      if (out_ms) out_ms[slot] = ms;
      if (ms < 0.0f) continue;
      if (ms < best) {
        best = ms;
        best_m = methods[mi];
        best_g = grids[gi];
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  vg_plan_configure(p, best_m, best_g);
  return result;
}

}  // extern "C"
