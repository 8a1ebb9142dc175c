// C ABI entry points of libvg.so (declared in include/vg.h): argument checks, workspace
// layouts and the launch sequence of each call.  No allocation happens here (the plan
// object in vg_plan.cu is the only owner of device memory in the library).
#include <atomic>
#include <mutex>
#include <cmath>
#include <cstring>

#include <nvtx3/nvToolsExt.h>

#include "../../include/vg.h"
#include "vg_api_internal.h"
#include "vg_internal.h"
#include "vg_frame.h"

namespace vg {

namespace {
std::atomic<uint32_t> g_spin_limit{0};
void** g_events = nullptr;
int g_max_events = 0;
bool g_events_paused = false;
int g_sms[64] = {0};
constexpr int kMaxStages = 20;
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

void pause_stage_events(bool paused) { g_events_paused = paused; }

namespace {
struct OccEntry {
  const void* fn;
  int dev;
  int blocks;
};
std::mutex g_occ_mu;
OccEntry g_occ[64];
int g_occ_n = 0;
}  // namespace

void warm_launch_config() {
  num_sms();
  warm_sort_config();
  warm_reduce_config();
  warm_filter_config();
  warm_msd_config();
  warm_frame_config();
}

int persistent_grid(const void* kernel, int threads, size_t dyn_smem, int64_t work_tiles) {
  int dev = 0;
  cudaGetDevice(&dev);
  int blocks = 0;
  {
    std::lock_guard<std::mutex> lock(g_occ_mu);
    for (int i = 0; i < g_occ_n; ++i)
      if (g_occ[i].fn == kernel && g_occ[i].dev == dev) blocks = g_occ[i].blocks;
    if (blocks == 0) {
      if (dyn_smem > 48 * 1024 - 4096)
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(dyn_smem));
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, threads, dyn_smem) !=
              cudaSuccess ||
          blocks < 1)
        blocks = 1;
      if (g_occ_n < 64) g_occ[g_occ_n++] = OccEntry{kernel, dev, blocks};
    }
  }
  const int64_t cap = int64_t(blocks) * num_sms();
  const int64_t g = work_tiles < cap ? work_tiles : cap;
  return static_cast<int>(g < 1 ? 1 : g);
}

namespace {

// Records profiling event k on `stream` when the stage-event hook is on.
void mark(int k, cudaStream_t stream) {
  if (!g_events_paused && g_events && k < g_max_events && g_events[k])
    cudaEventRecord(static_cast<cudaEvent_t>(g_events[k]), stream);
}

// NVTX range around a call's host-side launch sequence (seen by NVTX-aware profilers;
// free when none is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

vg_status cuda_status(cudaError_t e) { return e == cudaSuccess ? VG_OK : VG_ERR_CUDA; }

int grid_per_sm_of(int flags) { return (flags >> VG_GRID_SHIFT) & 0xff; }

int method_of(int flags) {
  const int m = flags & VG_METHOD_MASK;
  return m == VG_METHOD_HASH ? VG_METHOD_HASH : VG_METHOD_SORT;
}

}  // namespace

size_t frames_workspace_bytes(int64_t n, int frames, int flags) {
  if (n < 0 || frames < 1) return 0;
  if (method_of(flags) == VG_METHOD_HASH) return hash_layout(n, frames).total;
  const SortLayout L = sort_layout(n, frames);
  if ((flags & VG_SORT_FRAME) == 0) return L.total;
  // the bin grouping after the sort layout, or the one-launch grouping after the frame state
  const size_t a = frame_layout(n, L.total).total, b = fused_layout(n, L.lb_a).total;
  return a > b ? a : b;
}

vg_status check_outputs(int64_t n, const float* xyz, uint64_t* out_keys, float* out_centroids,
                        uint32_t* out_counts, int64_t cap, const int64_t* num_voxels,
                        const int32_t* p2v, const int32_t* out_error, const void* workspace) {
  if (n < 0 || n > kMaxPoints || cap < 0) return VG_ERR_INVALID_ARG;
  if (n > 0 && !xyz) return VG_ERR_INVALID_ARG;
  if (cap > 0 && (!out_keys || !out_centroids || !out_counts)) return VG_ERR_INVALID_ARG;
  if (!aligned(xyz, 4) || !aligned(out_keys, 8) || !aligned(out_centroids, 4) ||
      !aligned(out_counts, 4) || !aligned(num_voxels, 8) || !aligned(p2v, 4) ||
      !aligned(out_error, 4) || !aligned(workspace, 256))
    return VG_ERR_ALIGN;
  return VG_OK;
}

// The launch sequence shared by every decimation entry point.
vg_status run_frames(const float* xyz, const FramesArg& fr, bool from_min, const SegOut& out,
                     int32_t* out_error, void* workspace, size_t workspace_bytes, int flags,
                     cudaStream_t stream) {
  const int64_t n = fr.n;
  const int F = fr.nframes;
  const int method = method_of(flags);
  const NvtxRange range(method == VG_METHOD_HASH ? "vg: decimate (hash)" : "vg: decimate (sort)");
  const size_t need = frames_workspace_bytes(n, F, flags);
  if (!workspace || workspace_bytes < need) return VG_ERR_WORKSPACE;
  char* ws = static_cast<char*>(workspace);
  const uint32_t spins = spin_limit();
  int stage = 0;

  if (method == VG_METHOD_SORT) {
    // The narrow layout (no gather) needs the extents up front and no point_to_voxel; it
    // is grouped by buckets unless the caller asks for every digit in global passes.
    FramesArg frn = fr;
    frn.allow_narrow = out.p2v == nullptr && out.attrs_in == nullptr;
    // AUTO takes the bucket grouping only for large clouds (see kAutoBucketMinPoints); the
    // frame method, when the call is not one frame for its own grouping, the radix sort
    frn.lsd_narrow = (flags & (VG_SORT_LSD | VG_SORT_FRAME)) != 0 ||
                     ((flags & VG_METHOD_MASK) == VG_METHOD_AUTO && n < kAutoBucketMinPoints);
    const bool maybe_msd = frn.allow_narrow && !frn.lsd_narrow;
    // VG_SORT_FRAME: one frame, no point_to_voxel or attributes (else the plain sort path)
    const bool frame_path = (flags & VG_SORT_FRAME) != 0 && F == 1 && frn.allow_narrow && n > 0;
    // a frame that one cooperative launch holds: that launch alone (it finds the extents)
    const bool fused = frame_path && frame_fused_fits(n, posed(frn));
    const bool have_extent = from_min || F > 1 || frn.allow_narrow;
    const SortLayout L = sort_layout(n, F);
    State* st = reinterpret_cast<State*>(ws + L.state);
    FrameState* fs = reinterpret_cast<FrameState*>(ws + L.frames);
    uint64_t* keys0 = reinterpret_cast<uint64_t*>(ws + L.keys0);
    uint64_t* keys1 = reinterpret_cast<uint64_t*>(ws + L.keys1);
    uint32_t* idx0 = reinterpret_cast<uint32_t*>(ws + L.idx0);
    uint32_t* idx1 = reinterpret_cast<uint32_t*>(ws + L.idx1);
    uint32_t* lb_a = reinterpret_cast<uint32_t*>(ws + L.lb_a);
    uint32_t* lb_b = reinterpret_cast<uint32_t*>(ws + L.lb_b);
    TileRec* recs = reinterpret_cast<TileRec*>(ws + L.seg_lb);
    const int64_t nn = n < 1 ? 1 : n;
    uint32_t* k32_0 = reinterpret_cast<uint32_t*>(ws + L.keys0);
    uint32_t* k32_1 = k32_0 + align_up(size_t(nn), 4);  // 16-byte aligned, like k32_0
    uint64_t* pay_0 = reinterpret_cast<uint64_t*>(ws + L.keys1);
    uint64_t* pay_1 = reinterpret_cast<uint64_t*>(ws + L.idx0);
    int* err = out_error ? reinterpret_cast<int*>(out_error) : &st->error;

    // (the frame path needs only the state and frame state cleared: its last kernel
    // writes the voxel count and the frame offsets)
    // (the one-launch grouping clears the few state words it reads itself)
    cudaError_t e = fused ? cudaSuccess
                          : cudaMemsetAsync(ws, 0, frame_path ? L.lb_a : L.zero_bytes, stream);
    if (e == cudaSuccess && maybe_msd && !frame_path)  // points per bucket
      e = cudaMemsetAsync(ws + L.mhist, 0, L.mvcnt - L.mhist, stream);
    if (e == cudaSuccess && out_error && !fused)  // (the one-launch kernel clears it)
      e = cudaMemsetAsync(out_error, 0, sizeof(int32_t), stream);
    if (e == cudaSuccess && !frame_path)
      e = cudaMemsetAsync(out.num_voxels, 0, sizeof(int64_t), stream);
    if (e == cudaSuccess && out.frame_offsets && !frame_path)
      e = cudaMemsetAsync(out.frame_offsets, 0, size_t(F + 1) * sizeof(int64_t), stream);
    if (e == cudaSuccess && out.p2v && n > 0)
      e = cudaMemsetAsync(out.p2v, 0xff, size_t(n) * sizeof(int32_t), stream);
    mark(stage++, stream);
    if (fused) {
      if (e == cudaSuccess)
        e = launch_frame_fused(xyz, frn, st, fs, ws, fused_layout(n, L.lb_a), out, spins, err,
                               stream);
      for (int k = 0; k < 1 + 1 + 3 + kMaxPasses + 1; ++k) mark(stage++, stream);
      return cuda_status(e);
    }
    if (e == cudaSuccess && have_extent) {
      if (frame_path) {
        const FrameLayout FL = frame_layout(n, L.total);
        e = launch_origin(xyz, frn, st, fs, err, stream, ws + FL.zero, FL.zero_bytes);
      } else {
        e = launch_origin(xyz, frn, st, fs, err, stream);
      }
    }
    mark(stage++, stream);
    if (e == cudaSuccess && !frame_path)
      e = launch_keys_any(xyz, frn, have_extent, st, fs, keys0, k32_0, pay_0, err, stream);
    if (!frame_path) mark(stage++, stream);
    // The layout and the grouping are chosen on the device (they depend on the largest
    // key); the kernels of the ones not chosen return at once.
    const NarrowBuffers nb{k32_0, pay_0, k32_1, pay_1};
    if (frame_path) {
      // one camera frame: bins of 2^12 keys (vg_frame.cu); the extent kernel clears the
      // bin counts
      const FrameLayout FL = frame_layout(n, L.total);
      if (e == cudaSuccess) e = launch_frame(xyz, frn, st, fs, nb, ws, FL, out, spins, err, stream);
      for (int k = 0; k < 1 + 3 + kMaxPasses + 1; ++k) mark(stage++, stream);
      return cuda_status(e);
    }
    if (maybe_msd) {
      if (e == cudaSuccess)
        e = launch_msd(st, fs, F, nb, ws, L, n, out, spins, err, stream, stage, mark);
    } else {
      for (int k = 0; k < 3; ++k) mark(stage + k, stream);
    }
    stage += 3;
    for (int p = 0; p < kMaxPasses && e == cudaSuccess; ++p) {
      e = launch_sort_pass(st, keys0, idx0, keys1, idx1, lb_a, lb_b, n, p, false, spins, err,
                           stream, &nb);
      mark(stage++, stream);
    }
    if (e == cudaSuccess)
      e = launch_segreduce(st, fs, F, keys0, idx0, keys1, idx1, xyz, recs, n, out, err, stream,
                           &nb, frn.poses);
    mark(stage++, stream);
    return cuda_status(e);
  }

  // hash path
  const bool have_extent = from_min || F > 1;
  const HashLayout L = hash_layout(n, F);
  State* st = reinterpret_cast<State*>(ws + L.state);
  FrameState* fs = reinterpret_cast<FrameState*>(ws + L.frames);
  uint64_t* keys0 = reinterpret_cast<uint64_t*>(ws + L.keys0);
  uint64_t* keys1 = reinterpret_cast<uint64_t*>(ws + L.keys1);
  uint32_t* idx0 = reinterpret_cast<uint32_t*>(ws + L.idx0);
  uint32_t* idx1 = reinterpret_cast<uint32_t*>(ws + L.idx1);
  uint32_t* lb_a = reinterpret_cast<uint32_t*>(ws + L.lb_a);
  uint32_t* lb_b = reinterpret_cast<uint32_t*>(ws + L.lb_b);
  HashTable tab{reinterpret_cast<unsigned long long*>(ws + L.tkeys),
                reinterpret_cast<HashAcc*>(ws + L.tacc), static_cast<uint32_t>(L.slots - 1)};
  uint32_t* slot_rank = out.p2v ? reinterpret_cast<uint32_t*>(ws + L.slot_rank) : nullptr;
  uint32_t* point_slot = out.p2v ? reinterpret_cast<uint32_t*>(ws + L.point_slot) : nullptr;
  int* err = out_error ? reinterpret_cast<int*>(out_error) : &st->error;

  cudaError_t e = cudaMemsetAsync(ws, 0, L.zero_bytes, stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(tab.keys, 0xff, size_t(L.slots) * sizeof(unsigned long long), stream);
  if (e == cudaSuccess && out_error) e = cudaMemsetAsync(out_error, 0, sizeof(int32_t), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(out.num_voxels, 0, sizeof(int64_t), stream);
  if (e == cudaSuccess && out.frame_offsets)
    e = cudaMemsetAsync(out.frame_offsets, 0, size_t(F + 1) * sizeof(int64_t), stream);
  mark(stage++, stream);
  if (e == cudaSuccess && have_extent) e = launch_origin(xyz, fr, st, fs, err, stream);
  mark(stage++, stream);
  if (e == cudaSuccess)
    e = launch_hash_insert(xyz, fr, have_extent, st, fs, tab, point_slot, spins, err, stream);
  mark(stage++, stream);
  if (e == cudaSuccess) e = launch_hash_compact(tab, st, keys0, idx0, err, stream);
  mark(stage++, stream);
  for (int p = 0; p < kMaxPasses && e == cudaSuccess; ++p) {
    e = launch_sort_pass(st, keys0, idx0, keys1, idx1, lb_a, lb_b, n, p, true, spins, err, stream);
    mark(stage++, stream);
  }
  if (e == cudaSuccess)
    e = launch_hash_finalize(st, fs, F, keys0, idx0, keys1, idx1, tab, slot_rank, n, out, err,
                             stream);
  mark(stage++, stream);
  if (e == cudaSuccess && out.p2v) e = launch_hash_p2v(point_slot, slot_rank, n, out.p2v, err, stream);
  mark(stage++, stream);
  return cuda_status(e);
}

// Pyramid workspace: the sort path's, then two fixed-point sum buffers and the merge
// chained-scan status of every level.
struct PyramidLayout {
  size_t base, sums_a, sums_b, merge_lb, total;
  int64_t merge_tiles;
};

PyramidLayout pyramid_layout(int64_t n, int levels) {
  PyramidLayout L{};
  const int64_t nn = n < 1 ? 1 : n;
  L.base = sort_layout(n, 1).total;
  size_t off = L.base;
  L.sums_a = off;
  off = align_up(off + size_t(nn) * 3 * sizeof(long long), 256);
  L.sums_b = off;
  off = align_up(off + size_t(nn) * 3 * sizeof(long long), 256);
  L.merge_tiles = ceil_div(nn, kMergeTile);
  L.merge_lb = off;
  off = align_up(off + size_t(levels) * size_t(L.merge_tiles) * sizeof(uint32_t), 256);
  L.total = off;
  return L;
}

}  // namespace vg

using namespace vg;

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
  return kMaxStages;
}

void vg_debug_set_spin_limit(uint32_t limit) {
  g_spin_limit.store(limit, std::memory_order_relaxed);
}

vg_status vg_debug_wait_timeout(uint32_t* scratch_words, uint32_t limit, int32_t* out_error,
                                vg_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (!scratch_words || !out_error || limit == 0 || limit > kDefaultSpinLimit)
    return VG_ERR_INVALID_ARG;
  if (!aligned(scratch_words, 4) || !aligned(out_error, 4)) return VG_ERR_ALIGN;
  cudaError_t e = cudaMemsetAsync(scratch_words, 0, 4 * sizeof(uint32_t), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(out_error, 0, sizeof(int32_t), stream);
  if (e == cudaSuccess)
    e = launch_debug_wait(scratch_words, 3, limit, reinterpret_cast<int*>(out_error), stream);
  return cuda_status(e);
}

vg_status vg_debug_grid_barrier_timeout(uint32_t* scratch_words, uint32_t limit,
                                        int32_t* out_error, vg_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (!scratch_words || !out_error || limit == 0 || limit > kDefaultSpinLimit)
    return VG_ERR_INVALID_ARG;
  if (!aligned(scratch_words, 4) || !aligned(out_error, 4)) return VG_ERR_ALIGN;
  cudaError_t e = cudaMemsetAsync(scratch_words, 0, sizeof(uint32_t), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(out_error, 0, sizeof(int32_t), stream);
  if (e == cudaSuccess)
    e = launch_debug_grid_barrier(scratch_words, limit, reinterpret_cast<int*>(out_error), stream);
  return cuda_status(e);
}

size_t vg_downsample_workspace_bytes(int64_t n_points, int flags) {
  return frames_workspace_bytes(n_points, 1, flags);
}

int64_t vg_frame_one_launch_points(int posed) { return frame_fused_max_points(posed != 0); }

size_t vg_batch_workspace_bytes(int64_t n_total, int n_frames, int flags) {
  if (n_frames < 1 || n_frames > kMaxFrames) return 0;
  return frames_workspace_bytes(n_total, n_frames, flags);
}

vg_status vg_downsample(const float* xyz, int64_t n, float* origin, float leaf,
                        uint64_t* out_keys, float* out_centroids, uint32_t* out_counts,
                        int64_t cap, int64_t* out_num_voxels, int32_t* out_point_to_voxel,
                        int32_t* out_error, void* workspace, size_t workspace_bytes, int flags,
                        vg_stream_t stream) {
  if (!(leaf > 0.0f) || !std::isfinite(leaf)) return VG_ERR_INVALID_ARG;
  if ((flags & ~(VG_ORIGIN_FROM_MIN | VG_METHOD_MASK | VG_SORT_BUCKETS | VG_SORT_LSD |
                 VG_SORT_FRAME)) != 0)
    return VG_ERR_INVALID_ARG;
  if ((flags & VG_METHOD_MASK) == VG_METHOD_MASK) return VG_ERR_INVALID_ARG;
  if ((flags & VG_SORT_FRAME) != 0 && (flags & VG_METHOD_MASK) != VG_METHOD_SORT)
    return VG_ERR_INVALID_ARG;
  if (!origin || !out_num_voxels) return VG_ERR_INVALID_ARG;
  vg_status s = check_outputs(n, xyz, out_keys, out_centroids, out_counts, cap, out_num_voxels,
                              out_point_to_voxel, out_error, workspace);
  if (s != VG_OK) return s;
  if (!aligned(origin, 4)) return VG_ERR_ALIGN;
  const bool from_min = (flags & VG_ORIGIN_FROM_MIN) != 0;
  FramesArg fr{nullptr, 1, n, from_min ? nullptr : origin, from_min ? origin : nullptr, nullptr, leaf, 0};
  SegOut out{out_keys, out_centroids, out_counts, nullptr, cap, out_num_voxels, nullptr,
             out_point_to_voxel};
  return run_frames(xyz, fr, from_min, out, out_error, workspace, workspace_bytes, flags,
                    reinterpret_cast<cudaStream_t>(stream));
}

vg_status vg_downsample_frames(const float* xyz, int64_t n_total, const int64_t* frame_offsets,
                               int n_frames, float* origins, const float* leaves,
                               uint64_t* out_keys, float* out_centroids, uint32_t* out_counts,
                               int64_t cap, int64_t* out_frame_offsets,
                               int32_t* out_point_to_voxel, int32_t* out_error, void* workspace,
                               size_t workspace_bytes, int flags, vg_stream_t stream) {
  return vg_downsample_frames_posed(xyz, n_total, frame_offsets, n_frames, nullptr, nullptr,
                                    origins, leaves, out_keys, out_centroids, out_counts, cap,
                                    out_frame_offsets, out_point_to_voxel, out_error, workspace,
                                    workspace_bytes, flags, stream);
}

vg_status vg_downsample_frames_posed(const float* xyz, int64_t n_total,
                                     const int64_t* frame_offsets, int n_frames,
                                     const float* poses, const float* z_limits, float* origins,
                                     const float* leaves, uint64_t* out_keys,
                                     float* out_centroids, uint32_t* out_counts, int64_t cap,
                                     int64_t* out_frame_offsets, int32_t* out_point_to_voxel,
                                     int32_t* out_error, void* workspace, size_t workspace_bytes,
                                     int flags, vg_stream_t stream) {
  return vg_downsample_frames_ex(xyz, n_total, frame_offsets, n_frames, poses, z_limits, origins,
                                 leaves, out_keys, out_centroids, out_counts, cap,
                                 out_frame_offsets, out_point_to_voxel, nullptr, out_error,
                                 workspace, workspace_bytes, flags, stream);
}

size_t vg_downsample_ex_workspace_bytes(int64_t n_total, int n_frames, int flags,
                                        const vg_voxel_extras* extras) {
  if (n_total < 0 || n_frames < 1 || n_frames > kMaxFrames) return 0;
  const size_t base = frames_workspace_bytes(n_total, n_frames, flags);
  if (!extras || extras->min_count <= 1) return base;
  return filter_layout(n_total, base).total;
}

vg_status vg_downsample_frames_ex(const float* xyz, int64_t n_total,
                                  const int64_t* frame_offsets, int n_frames, const float* poses,
                                  const float* z_limits, float* origins, const float* leaves,
                                  uint64_t* out_keys, float* out_centroids, uint32_t* out_counts,
                                  int64_t cap, int64_t* out_frame_offsets,
                                  int32_t* out_point_to_voxel, const vg_voxel_extras* extras,
                                  int32_t* out_error, void* workspace, size_t workspace_bytes,
                                  int flags, vg_stream_t stream) {
  if (n_frames < 1 || n_frames > kMaxFrames) return VG_ERR_INVALID_ARG;
  if (!aligned(poses, 4) || !aligned(z_limits, 4)) return VG_ERR_ALIGN;
  const uint8_t* attrs = extras ? extras->attrs : nullptr;
  const int channels = attrs ? extras->attr_channels : 0;
  if (attrs) {
    if (channels < 1 || channels > 4 || !extras->out_attrs) return VG_ERR_INVALID_ARG;
    if (method_of(flags) == VG_METHOD_HASH) return VG_ERR_INVALID_ARG;
    if (!aligned(extras->out_attrs, 4)) return VG_ERR_ALIGN;
  }
  const bool filtered = extras && extras->min_count > 1;
  if ((flags & ~(VG_ORIGIN_FROM_MIN | VG_METHOD_MASK | VG_GRID_MASK | VG_SORT_BUCKETS |
                 VG_SORT_LSD | VG_SORT_FRAME)) != 0)
    return VG_ERR_INVALID_ARG;
  if ((flags & VG_METHOD_MASK) == VG_METHOD_MASK) return VG_ERR_INVALID_ARG;
  if ((flags & VG_SORT_FRAME) != 0 && (flags & VG_METHOD_MASK) != VG_METHOD_SORT)
    return VG_ERR_INVALID_ARG;
  if (!frame_offsets || !origins || !leaves || !out_frame_offsets) return VG_ERR_INVALID_ARG;
  vg_status s = check_outputs(n_total, xyz, out_keys, out_centroids, out_counts, cap,
                              out_frame_offsets, out_point_to_voxel, out_error, workspace);
  if (s != VG_OK) return s;
  if (!aligned(frame_offsets, 8) || !aligned(origins, 4) || !aligned(leaves, 4))
    return VG_ERR_ALIGN;
  const bool from_min = (flags & VG_ORIGIN_FROM_MIN) != 0;
  FramesArg fr{frame_offsets, n_frames, n_total, from_min ? nullptr : origins,
               from_min ? origins : nullptr, leaves, 0.0f, grid_per_sm_of(flags), 0, poses,
               z_limits};
  // V lands in out_frame_offsets[n_frames]; the segmented reduction also writes it there.
  SegOut out{out_keys, out_centroids, out_counts, nullptr, cap, out_frame_offsets + n_frames,
             out_frame_offsets, out_point_to_voxel, attrs, channels,
             attrs ? extras->out_attrs : nullptr};
  const size_t base = frames_workspace_bytes(n_total, n_frames, flags);
  FilterLayout FL{};
  if (filtered) {
    FL = filter_layout(n_total, base);
    if (!workspace || workspace_bytes < FL.total) return VG_ERR_WORKSPACE;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  s = run_frames(xyz, fr, from_min, out, out_error, workspace, workspace_bytes, flags, st);
  if (s != VG_OK || !filtered) return s;
  char* ws = static_cast<char*>(workspace);
  int* err = out_error ? reinterpret_cast<int*>(out_error) : &reinterpret_cast<State*>(ws)->error;
  return cuda_status(launch_filter(ws, FL, cap < n_total ? cap : n_total, extras->min_count, out,
                                   n_frames, n_total, spin_limit(), err, st));
}

size_t vg_pyramid_workspace_bytes(int64_t n_points, int levels, int flags) {
  (void)flags;
  if (n_points < 0 || levels < 1 || levels > kMaxLevels) return 0;
  return pyramid_layout(n_points, levels).total;
}

vg_status vg_pyramid(const float* xyz, int64_t n, float* origin, float leaf, int levels,
                     uint64_t* out_keys, float* out_centroids, uint32_t* out_counts,
                     int64_t cap_total, int64_t* out_level_offsets, int32_t* out_point_to_voxel,
                     int32_t* out_error, void* workspace, size_t workspace_bytes, int flags,
                     vg_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (!(leaf > 0.0f) || !std::isfinite(leaf)) return VG_ERR_INVALID_ARG;
  if (levels < 1 || levels > kMaxLevels) return VG_ERR_INVALID_ARG;
  if ((flags & ~(VG_ORIGIN_FROM_MIN | VG_SORT_BUCKETS | VG_SORT_LSD)) != 0)
    return VG_ERR_INVALID_ARG;
  if (!origin || !out_level_offsets) return VG_ERR_INVALID_ARG;
  if (!std::isfinite(leaf * float(1u << (levels - 1)))) return VG_ERR_INVALID_ARG;
  vg_status s = check_outputs(n, xyz, out_keys, out_centroids, out_counts, cap_total,
                              out_level_offsets, out_point_to_voxel, out_error, workspace);
  if (s != VG_OK) return s;
  if (!aligned(origin, 4)) return VG_ERR_ALIGN;
  const PyramidLayout P = pyramid_layout(n, levels);
  if (!workspace || workspace_bytes < P.total) return VG_ERR_WORKSPACE;
  char* ws = static_cast<char*>(workspace);
  const SortLayout L = sort_layout(n, 1);
  State* st = reinterpret_cast<State*>(ws + L.state);
  const FrameState* fs = reinterpret_cast<const FrameState*>(ws + L.frames);
  long long* sums[2] = {reinterpret_cast<long long*>(ws + P.sums_a),
                        reinterpret_cast<long long*>(ws + P.sums_b)};
  uint32_t* merge_lb = reinterpret_cast<uint32_t*>(ws + P.merge_lb);
  int* err = out_error ? reinterpret_cast<int*>(out_error) : &st->error;
  const bool from_min = (flags & VG_ORIGIN_FROM_MIN) != 0;

  cudaError_t e = cudaMemsetAsync(out_level_offsets, 0, size_t(levels + 1) * sizeof(int64_t), stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(merge_lb, 0, size_t(levels) * size_t(P.merge_tiles) * sizeof(uint32_t),
                        stream);
  if (e != cudaSuccess) return VG_ERR_CUDA;
  FramesArg fr{nullptr, 1, n, from_min ? nullptr : origin, from_min ? origin : nullptr, nullptr, leaf, 0};
  SegOut out{out_keys, out_centroids, out_counts, sums[0], cap_total, out_level_offsets + 1,
             nullptr, out_point_to_voxel};
  // level 0 by the sort method's grouping (the AUTO choice unless the flags name one)
  s = run_frames(xyz, fr, from_min, out, out_error, workspace, L.total,
                 flags & (VG_SORT_BUCKETS | VG_SORT_LSD), stream);
  if (s != VG_OK) return s;
  const uint32_t spins = spin_limit();
  for (int k = 1; k < levels && e == cudaSuccess; ++k)
    e = launch_pyramid_merge(st, fs, k, out_keys, out_centroids, out_counts, sums[(k - 1) & 1],
                             sums[k & 1], out_level_offsets, cap_total,
                             merge_lb + size_t(k - 1) * size_t(P.merge_tiles), n, spins, err,
                             stream);
  return cuda_status(e);
}

vg_status vg_downsample_backward(const float* grad_centroids, const uint32_t* counts,
                                 const int32_t* point_to_voxel, int64_t n, int64_t num_voxels,
                                 float* grad_xyz, int32_t* out_error, vg_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (n < 0 || num_voxels < 0 || n > kMaxPoints) return VG_ERR_INVALID_ARG;
  if (n > 0 && (!point_to_voxel || !grad_xyz || !out_error)) return VG_ERR_INVALID_ARG;
  if (num_voxels > 0 && (!grad_centroids || !counts)) return VG_ERR_INVALID_ARG;
  if (!aligned(grad_centroids, 4) || !aligned(counts, 4) || !aligned(point_to_voxel, 4) ||
      !aligned(grad_xyz, 4) || !aligned(out_error, 4))
    return VG_ERR_ALIGN;
  if (n == 0) return VG_OK;
  cudaError_t e = cudaMemsetAsync(out_error, 0, sizeof(int32_t), stream);
  if (e == cudaSuccess)
    e = launch_backward(grad_centroids, counts, point_to_voxel, n, num_voxels, grad_xyz,
                        reinterpret_cast<int*>(out_error), stream);
  return cuda_status(e);
}

}  // extern "C"
