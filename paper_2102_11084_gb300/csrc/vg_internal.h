// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace vg {

// Radix sort geometry (8-bit digits, 256 threads x 16 keys per tile).
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kMaxPasses = 8;  // 64-bit keys
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;

// Segmented reduction geometry (256 threads x 8 keys per tile).
constexpr int kSegThreads = 256;
constexpr int kSegItems = 8;
constexpr int kSegTile = kSegThreads * kSegItems;

// Streaming kernels (origin, keys): 256 threads, 4 points per thread per iteration.
constexpr int kStreamThreads = 256;
constexpr int kStreamPoints = 4;

// Chained-scan status flags (top two bits of a 32-bit status word).
constexpr uint32_t kFlagAggregate = 1u << 30;
constexpr uint32_t kFlagPrefix = 2u << 30;
constexpr uint32_t kValueMask = (1u << 30) - 1;

// Largest cloud a call accepts: counts live in 30-bit chained-scan values.
constexpr int64_t kMaxPoints = (int64_t(1) << 30) - 1;

// Default spin limit of a chained-scan wait before it gives up with a timeout status.
constexpr uint32_t kDefaultSpinLimit = 1u << 22;

// Per-call device state, at the start of the workspace.  Zeroed by the call.
struct alignas(256) State {
  uint32_t ord_min_inv[3];   // max over valid points of ~ordered(x): min via atomicMax
  uint32_t pad0;
  float origin[3];           // origin used by the call
  uint32_t pad1;
  unsigned long long maxkey; // largest valid key
  uint32_t nvalid;           // number of valid points (compacted key count)
  uint32_t pad3;
  uint32_t tile_ctr[kMaxPasses + 4];
  int32_t error;             // internal error word when the caller passes none
  uint32_t pad2[3];
  uint32_t hist[kMaxPasses][kRadix];
};

// Segmented-reduction chained-scan record of one tile.
struct alignas(16) SegStatus {
  uint32_t flag;
  uint32_t heads_agg;
  uint32_t heads_incl;
  uint32_t n_agg;
  uint32_t n_incl;
  uint32_t pad[3];
  long long s_agg[3];
  long long pad2;
  long long s_incl[3];
  long long pad3;
};

constexpr int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
constexpr size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Workspace layout of the sort path for n points.
struct SortLayout {
  size_t state, keys0, keys1, idx0, idx1, lb_a, lb_b, seg_lb, total;
  size_t zero_bytes;  // bytes from `state` that must be zero at call start
  int64_t sort_tiles, seg_tiles;
};
constexpr SortLayout sort_layout(int64_t n) {
  SortLayout L{};
  const int64_t nn = n < 1 ? 1 : n;
  L.sort_tiles = ceil_div(nn, kSortTile);
  L.seg_tiles = ceil_div(nn, kSegTile);
  size_t off = 0;
  L.state = off;
  off = align_up(off + sizeof(State), 256);
  L.lb_a = off;
  off = align_up(off + size_t(L.sort_tiles) * kRadix * sizeof(uint32_t), 256);
  L.seg_lb = off;
  off = align_up(off + size_t(L.seg_tiles) * sizeof(SegStatus), 256);
  L.zero_bytes = off;  // state, pass-0 status rows and segment status: zeroed per call
  L.lb_b = off;
  off = align_up(off + size_t(L.sort_tiles) * kRadix * sizeof(uint32_t), 256);
  L.keys0 = off;
  off = align_up(off + size_t(nn) * sizeof(uint64_t), 256);
  L.keys1 = off;
  off = align_up(off + size_t(nn) * sizeof(uint64_t), 256);
  L.idx0 = off;
  off = align_up(off + size_t(nn) * sizeof(uint32_t), 256);
  L.idx1 = off;
  off = align_up(off + size_t(nn) * sizeof(uint32_t), 256);
  L.total = off;
  return L;
}

int num_sms();

uint32_t spin_limit();

// Launchers (all asynchronous on `stream`).
cudaError_t launch_origin(const float* xyz, int64_t n, State* st, cudaStream_t stream);
cudaError_t launch_keys(const float* xyz, int64_t n, float* origin_user, bool from_min,
                        float leaf, State* st, uint64_t* keys, int* err, cudaStream_t stream);
cudaError_t launch_sort_pass(State* st, uint64_t* keys0, uint32_t* idx0, uint64_t* keys1,
                             uint32_t* idx1, uint32_t* lb_a, uint32_t* lb_b, int64_t n_max,
                             int pass, uint32_t spin_limit, int* err, cudaStream_t stream);
cudaError_t launch_segreduce(State* st, const uint64_t* keys0, const uint32_t* idx0,
                             const uint64_t* keys1, const uint32_t* idx1, const float* xyz,
                             float leaf, SegStatus* lb, int64_t n_max, uint64_t* out_keys,
                             float* out_centroids, uint32_t* out_counts, int64_t cap,
                             int64_t* out_num_voxels, int32_t* out_p2v, uint32_t spin_limit,
                             int* err, cudaStream_t stream);

}  // namespace vg
