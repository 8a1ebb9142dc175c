// Minimum points per voxel: removes the output rows of voxels holding fewer than m
// points, in place and in order, after the decimation has written them.
//
// The voxel-grid filter the paper replaces (Sec. I and II-C, PCL's filter in STVL) can
// drop sparsely occupied voxels; here that is a stable compaction of the V rows (keys,
// counts, centroids, attribute means) with a chained scan over tiles of 1024 rows:
//   filter_kernel   a tile reads its rows, ranks the kept ones, waits (bounded) for the
//                   kept-row count of all earlier tiles, then writes its kept rows at
//                   their new place.  Tiles start in ticket order and a tile's prefix is
//                   complete only once every earlier tile has read its rows, so the
//                   in-place writes (always to rows at or before the tile's own) never
//                   overwrite a row not yet read.  Every row also gets its remap word:
//                   bit 31 = kept, bits 0-30 = kept rows before it.
//   filter_fix      one block: the new voxel count and per-frame row offsets.
//   filter_p2v      point_to_voxel through the remap (-1 for removed voxels).
#include "vg_device.cuh"
#include "vg_internal.h"

namespace vg {
namespace {

constexpr int kFiltThreads = 256;
constexpr int kFiltRows = 4;
constexpr int kFiltTile = kFiltThreads * kFiltRows;
constexpr uint32_t kKeptBit = 0x80000000u;

__global__ __launch_bounds__(kFiltThreads) void filter_kernel(
    const int64_t* __restrict__ num_voxels, int64_t cap, uint32_t min_count, uint64_t* keys,
    uint32_t* counts, float* centroids, float* attrs, int channels, uint32_t* remap,
    uint32_t* status, uint32_t* ticket, uint32_t spin_limit, int* err) {
  __shared__ uint32_t s_tmp[kFiltThreads / 32];
  __shared__ int s_tile;
  __shared__ uint32_t s_prefix;
  const int t = threadIdx.x;
  const int64_t V = *num_voxels < cap ? *num_voxels : cap;  // rows beyond cap were not written
  const int64_t ntiles = ceil_div(V, kFiltTile);
  for (;;) {
    // After an error (an earlier step, or a chained-scan timeout here) a block takes no
    // more tickets; every ticket taken is processed, so no tile waits on a skipped one.
    if (t == 0) s_tile = error_raised(err) ? 0x7fffffff : static_cast<int>(atomicAdd(ticket, 1u));
    __syncthreads();
    const int tile = s_tile;
    if (tile >= ntiles) break;
    const int64_t base = int64_t(tile) * kFiltTile;
    // this thread's rows: base + 4t .. base + 4t + 3, read before anything is written
    uint64_t k[kFiltRows];
    uint32_t n[kFiltRows];
    float c[kFiltRows][3];
    float a[kFiltRows][4];
    uint32_t kept = 0, mine = 0;
#pragma unroll
    for (int j = 0; j < kFiltRows; ++j) {
      const int64_t r = base + kFiltRows * t + j;
      const bool in = r < V;
      k[j] = in ? keys[r] : 0;
      n[j] = in ? counts[r] : 0;
#pragma unroll
      for (int x = 0; x < 3; ++x) c[j][x] = in ? centroids[3 * r + x] : 0.0f;
#pragma unroll
      for (int x = 0; x < 4; ++x) a[j][x] = (in && x < channels) ? attrs[r * channels + x] : 0.0f;
      const bool keep = in && n[j] >= min_count;
      kept |= uint32_t(keep) << j;
      mine += keep;
    }
    uint32_t tile_kept;
    const uint32_t rank = block_excl_scan(mine, &tile_kept, s_tmp);
    if (t == 0) {
      uint32_t excl = 0;
      if (tile == 0) {
        st_relaxed(status, kFlagPrefix | tile_kept);
      } else {
        st_relaxed(status + tile, kFlagAggregate | tile_kept);
        excl = lookback_u32(status, 1, tile, spin_limit, err);
        st_relaxed(status + tile, kFlagPrefix | ((excl + tile_kept) & kValueMask));
      }
      s_prefix = excl;
    }
    __syncthreads();
    uint32_t dst = s_prefix + rank;
#pragma unroll
    for (int j = 0; j < kFiltRows; ++j) {
      const int64_t r = base + kFiltRows * t + j;
      if (r >= V) break;
      const bool keep = (kept >> j) & 1u;
      remap[r] = (keep ? kKeptBit : 0u) | dst;
      if (keep) {
        keys[dst] = k[j];
        counts[dst] = n[j];
#pragma unroll
        for (int x = 0; x < 3; ++x) centroids[3 * size_t(dst) + x] = c[j][x];
#pragma unroll
        for (int x = 0; x < 4; ++x)
          if (x < channels) attrs[size_t(dst) * channels + x] = a[j][x];
        ++dst;
      }
    }
    __syncthreads();
  }
}

// New voxel count, and per-frame offsets (kept rows before each frame's first row).
__global__ __launch_bounds__(1024) void filter_fix_kernel(int64_t* num_voxels, int64_t cap,
                                                          int64_t* frame_offsets, int nframes,
                                                          const uint32_t* __restrict__ remap,
                                                          const int* err) {
  if (block_error_raised(err)) return;  // the remap may be incomplete
  const int64_t V = *num_voxels < cap ? *num_voxels : cap;
  const uint32_t last = V > 0 ? remap[V - 1] : 0u;
  const int64_t total = V > 0 ? int64_t(last & ~kKeptBit) + (last >> 31) : 0;
  if (frame_offsets)
    for (int f = threadIdx.x; f <= nframes; f += blockDim.x) {
      const int64_t old = frame_offsets[f];
      frame_offsets[f] = old < V ? int64_t(remap[old] & ~kKeptBit) : total;
    }
  __syncthreads();
  if (threadIdx.x == 0) *num_voxels = total;
}

__global__ void filter_p2v_kernel(int32_t* p2v, int64_t n, int64_t cap,
                                  const uint32_t* __restrict__ remap, const int* err) {
  if (error_raised(err)) return;  // the remap may be incomplete
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int32_t v = p2v[i];
    if (v >= cap) {  // a row the capacity error left unwritten
      p2v[i] = -1;
    } else if (v >= 0) {
      const uint32_t m = remap[v];
      p2v[i] = (m & kKeptBit) ? static_cast<int32_t>(m & ~kKeptBit) : -1;
    }
  }
}

}  // namespace

FilterLayout filter_layout(int64_t cap, size_t base) {
  FilterLayout L{};
  const int64_t cc = cap < 1 ? 1 : cap;
  size_t off = align_up(base, 256);
  L.ticket = off;
  L.status = off + 256;
  off = align_up(L.status + size_t(ceil_div(cc, kFiltTile)) * sizeof(uint32_t), 256);
  L.zero_bytes = off - L.ticket;
  L.remap = off;
  off = align_up(off + size_t(cc) * sizeof(uint32_t), 256);
  L.total = off;
  return L;
}

cudaError_t launch_filter(char* ws, const FilterLayout& L, int64_t cap, uint32_t min_count,
                          const SegOut& out, int nframes, int64_t n_points, uint32_t spin_limit,
                          int* err, cudaStream_t stream) {
  if (cap == 0) return cudaSuccess;
  uint32_t* ticket = reinterpret_cast<uint32_t*>(ws + L.ticket);
  uint32_t* status = reinterpret_cast<uint32_t*>(ws + L.status);
  uint32_t* remap = reinterpret_cast<uint32_t*>(ws + L.remap);
  cudaError_t e = cudaMemsetAsync(ticket, 0, L.zero_bytes, stream);
  if (e != cudaSuccess) return e;
  const int grid = persistent_grid(reinterpret_cast<const void*>(filter_kernel), kFiltThreads, 0,
                                   ceil_div(cap, kFiltTile));
  filter_kernel<<<grid, kFiltThreads, 0, stream>>>(out.num_voxels, cap, min_count, out.keys,
                                                   out.counts, out.centroids, out.attrs_out,
                                                   out.attrs_out ? out.channels : 0, remap,
                                                   status, ticket, spin_limit, err);
  filter_fix_kernel<<<1, 1024, 0, stream>>>(out.num_voxels, cap, out.frame_offsets, nframes,
                                            remap, err);
  if (out.p2v && n_points > 0) {
    const int blocks = static_cast<int>(ceil_div(n_points, 256) < 4096 ? ceil_div(n_points, 256)
                                                                         : 4096);
    filter_p2v_kernel<<<blocks, 256, 0, stream>>>(out.p2v, n_points, cap, remap, err);
  }
  return cudaGetLastError();
}

void warm_filter_config() {
  persistent_grid(reinterpret_cast<const void*>(filter_kernel), kFiltThreads, 0, 1);
}

}  // namespace vg
