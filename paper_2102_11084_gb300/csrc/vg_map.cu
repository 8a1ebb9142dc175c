// Persistent voxel map (vg_map_*): many frames merged into one device-resident table.
//
// arXiv 2102.11084 Sec. II-C: STVL marks the cells of a global map with every filtered
// camera cloud.  The map here keeps, per occupied voxel of one fixed lattice, the point
// count and the fixed-point offset sums that the decimation accumulates (the same
// quantisation as every other path), in an open-addressing table in HBM.  Inserting is
// the hash path's insert kernel with all frames keyed into one voxel space; extracting
// is its compaction, the radix sort of the occupied keys and the finalisation.  Integer
// sums make the map independent of how the points were split into inserts.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/vg.h"
#include "vg_api_internal.h"
#include "vg_internal.h"

struct vg_map {
  int device = 0;
  float origin[3] = {0, 0, 0};
  float leaf = 1.0f;
  int64_t slots = 0;
  int64_t sort_tiles = 0;
  void* mem = nullptr;
  vg::State* st = nullptr;   // insert state (maximum key, counters), kept across calls
  vg::State* xst = nullptr;  // extraction state, reset by every extraction
  vg::FrameState* fs = nullptr;
  float* origins = nullptr;  // [kMaxFrames,3] the map origin, once per frame slot
  float* leaves = nullptr;   // [kMaxFrames]
  vg::HashTable tab{};
  uint32_t* lb_a = nullptr;
  uint32_t* lb_b = nullptr;
  uint64_t* keys0 = nullptr;
  uint64_t* keys1 = nullptr;
  uint32_t* idx0 = nullptr;
  uint32_t* idx1 = nullptr;
};

namespace {

using vg::align_up;

// Byte offsets of the map's single allocation.
struct MapLayout {
  size_t st, xst, fs, origins, leaves, tkeys, tacc, lb_a, lb_b, keys0, keys1, idx0, idx1, total;
};

MapLayout map_layout(int64_t slots, int64_t sort_tiles) {
  MapLayout L{};
  size_t off = 0;
  auto take = [&](size_t* at, size_t bytes) {
    *at = off;
    off = align_up(off + bytes, 256);
  };
  take(&L.st, sizeof(vg::State));
  take(&L.xst, sizeof(vg::State));
  take(&L.fs, size_t(vg::kMaxFrames) * sizeof(vg::FrameState));
  take(&L.origins, size_t(vg::kMaxFrames) * 3 * sizeof(float));
  take(&L.leaves, size_t(vg::kMaxFrames) * sizeof(float));
  take(&L.tkeys, size_t(slots) * sizeof(unsigned long long));
  take(&L.tacc, size_t(slots) * sizeof(vg::HashAcc));
  take(&L.lb_a, size_t(sort_tiles) * vg::kRadix * sizeof(uint32_t));
  take(&L.lb_b, size_t(sort_tiles) * vg::kRadix * sizeof(uint32_t));
  take(&L.keys0, size_t(slots) * sizeof(uint64_t));
  take(&L.keys1, size_t(slots) * sizeof(uint64_t));
  take(&L.idx0, size_t(slots) * sizeof(uint32_t));
  take(&L.idx1, size_t(slots) * sizeof(uint32_t));
  L.total = off;
  return L;
}

// The extraction sorts the occupied keys of the whole lattice: no frame id, wide layout,
// and the largest key any insert has seen.
__global__ void map_extract_init(const vg::State* st, vg::State* xst) {
  xst->maxkey = st->maxkey;
  xst->key_shift = 64;
  xst->nframes = 1;
  xst->narrow = 0;
}

vg_status cuda_status(cudaError_t e) { return e == cudaSuccess ? VG_OK : VG_ERR_CUDA; }

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

extern "C" {

vg_status vg_map_create(vg_map** out, int64_t capacity, const float* origin, float leaf) {
  if (!out || !origin || capacity < 1 || capacity > vg::kMaxPoints) return VG_ERR_INVALID_ARG;
  if (!(leaf > 0.0f) || !std::isfinite(leaf)) return VG_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(origin[a])) return VG_ERR_INVALID_ARG;
  *out = nullptr;
  vg_map* m = new (std::nothrow) vg_map();
  if (!m) return VG_ERR_CUDA;
  if (cudaGetDevice(&m->device) != cudaSuccess) {
    delete m;
    return VG_ERR_CUDA;
  }
  std::memcpy(m->origin, origin, sizeof(m->origin));
  m->leaf = leaf;
  m->slots = vg::hash_slots(capacity);
  m->sort_tiles = vg::ceil_div(m->slots, vg::kSortTile);
  const MapLayout L = map_layout(m->slots, m->sort_tiles);
  if (cudaMalloc(&m->mem, L.total) != cudaSuccess) {
    delete m;
    return VG_ERR_CUDA;
  }
  char* base = static_cast<char*>(m->mem);
  m->st = reinterpret_cast<vg::State*>(base + L.st);
  m->xst = reinterpret_cast<vg::State*>(base + L.xst);
  m->fs = reinterpret_cast<vg::FrameState*>(base + L.fs);
  m->origins = reinterpret_cast<float*>(base + L.origins);
  m->leaves = reinterpret_cast<float*>(base + L.leaves);
  m->tab = vg::HashTable{reinterpret_cast<unsigned long long*>(base + L.tkeys),
                         reinterpret_cast<vg::HashAcc*>(base + L.tacc),
                         static_cast<uint32_t>(m->slots - 1)};
  m->lb_a = reinterpret_cast<uint32_t*>(base + L.lb_a);
  m->lb_b = reinterpret_cast<uint32_t*>(base + L.lb_b);
  m->keys0 = reinterpret_cast<uint64_t*>(base + L.keys0);
  m->keys1 = reinterpret_cast<uint64_t*>(base + L.keys1);
  m->idx0 = reinterpret_cast<uint32_t*>(base + L.idx0);
  m->idx1 = reinterpret_cast<uint32_t*>(base + L.idx1);
  // every frame slot carries the map's origin and leaf
  std::vector<float> frame_tab(size_t(vg::kMaxFrames) * 4);
  for (int f = 0; f < vg::kMaxFrames; ++f) {
    for (int a = 0; a < 3; ++a) frame_tab[3 * f + a] = origin[a];
    frame_tab[size_t(vg::kMaxFrames) * 3 + f] = leaf;
  }
  cudaError_t e = cudaMemset(m->mem, 0, L.tkeys);
  if (e == cudaSuccess)
    e = cudaMemcpy(m->origins, frame_tab.data(), size_t(vg::kMaxFrames) * 3 * sizeof(float),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(m->leaves, frame_tab.data() + size_t(vg::kMaxFrames) * 3,
                   size_t(vg::kMaxFrames) * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemset(m->tab.keys, 0xff, size_t(m->slots) * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaFree(m->mem);
    delete m;
    return VG_ERR_CUDA;
  }
  vg::warm_launch_config();  // occupancy queries now, not inside a later capture
  *out = m;
  return VG_OK;
}

vg_status vg_map_destroy(vg_map* m) {
  if (!m) return VG_ERR_INVALID_ARG;
  const cudaError_t e = cudaFree(m->mem);
  delete m;
  return cuda_status(e);
}

vg_status vg_map_clear(vg_map* m, vg_stream_t stream_) {
  if (!m) return VG_ERR_INVALID_ARG;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  cudaError_t e = cudaMemsetAsync(m->st, 0, sizeof(vg::State), stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(m->tab.keys, 0xff, size_t(m->slots) * sizeof(unsigned long long),
                        stream);
  return cuda_status(e);
}

vg_status vg_map_insert(vg_map* m, const float* xyz, int64_t n_total,
                        const int64_t* frame_offsets, int n_frames, const float* poses,
                        const float* z_limits, int32_t* out_error, vg_stream_t stream_) {
  if (!m || n_total < 0 || n_total > vg::kMaxPoints) return VG_ERR_INVALID_ARG;
  if (n_frames < 1 || n_frames > vg::kMaxFrames) return VG_ERR_INVALID_ARG;
  if (!frame_offsets && n_frames != 1) return VG_ERR_INVALID_ARG;
  if (n_total > 0 && !xyz) return VG_ERR_INVALID_ARG;
  if (!aligned(xyz, 4) || !aligned(frame_offsets, 8) || !aligned(poses, 4) ||
      !aligned(z_limits, 4) || !aligned(out_error, 4))
    return VG_ERR_ALIGN;
  if (n_total == 0) return VG_OK;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  vg::FramesArg fr{frame_offsets, n_frames, n_total, m->origins, nullptr, m->leaves, m->leaf,
                   0, 0, poses, z_limits, 1};
  int* err = out_error ? reinterpret_cast<int*>(out_error) : &m->st->error;
  return cuda_status(vg::launch_hash_insert(xyz, fr, false, m->st, m->fs, m->tab, nullptr,
                                            vg::spin_limit(), err, stream));
}

vg_status vg_map_extract(vg_map* m, uint64_t* out_keys, float* out_centroids,
                         uint32_t* out_counts, int64_t cap, int64_t* out_num_voxels,
                         int32_t* out_error, vg_stream_t stream_) {
  if (!m || !out_num_voxels || cap < 0) return VG_ERR_INVALID_ARG;
  if (cap > 0 && (!out_keys || !out_centroids || !out_counts)) return VG_ERR_INVALID_ARG;
  if (!aligned(out_keys, 8) || !aligned(out_centroids, 4) || !aligned(out_counts, 4) ||
      !aligned(out_num_voxels, 8) || !aligned(out_error, 4))
    return VG_ERR_ALIGN;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  int* err = out_error ? reinterpret_cast<int*>(out_error) : &m->xst->error;
  cudaError_t e = cudaMemsetAsync(m->xst, 0, sizeof(vg::State), stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(m->lb_a, 0, size_t(m->sort_tiles) * vg::kRadix * sizeof(uint32_t), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(out_num_voxels, 0, sizeof(int64_t), stream);
  if (e != cudaSuccess) return VG_ERR_CUDA;
  map_extract_init<<<1, 1, 0, stream>>>(m->st, m->xst);
  e = vg::launch_hash_compact(m->tab, m->xst, m->keys0, m->idx0, err, stream);
  const uint32_t spins = vg::spin_limit();
  for (int p = 0; p < vg::kMaxPasses && e == cudaSuccess; ++p)
    e = vg::launch_sort_pass(m->xst, m->keys0, m->idx0, m->keys1, m->idx1, m->lb_a, m->lb_b,
                             m->slots, p, true, spins, err, stream);
  vg::SegOut out{out_keys, out_centroids, out_counts, nullptr, cap, out_num_voxels, nullptr,
                 nullptr};
  if (e == cudaSuccess)
    e = vg::launch_hash_finalize(m->xst, m->fs, 1, m->keys0, m->idx0, m->keys1, m->idx1, m->tab,
                                 nullptr, m->slots, out, err, stream);
  return cuda_status(e);
}

}  // extern "C"
