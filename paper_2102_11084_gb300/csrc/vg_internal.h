// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace vg {

// Tile geometry (build-time choices; the defaults are the measured best on GB300).
#ifndef VG_SORT_ITEMS
#define VG_SORT_ITEMS 12
#endif
#ifndef VG_SORT_MINB
#define VG_SORT_MINB 4
#endif
#ifndef VG_RED_MINB
#define VG_RED_MINB 4
#endif
#ifndef VG_KEY_MINB  // blocks/SM of the (unposed) key kernel: 4 fits 64 registers
#define VG_KEY_MINB 4
#endif
#ifndef VG_SORT_PREFETCH
#define VG_SORT_PREFETCH 1
#endif
#ifndef VG_SORT_EARLY_TICKET
#define VG_SORT_EARLY_TICKET 1
#endif

// Radix sort geometry (8-bit digits, 256 threads x VG_SORT_ITEMS keys per tile).
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kMaxPasses = 8;  // 64-bit keys
constexpr int kSortThreads = 256;
constexpr int kSortItems = VG_SORT_ITEMS;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kSortMinBlocks = VG_SORT_MINB;

// Bucket grouping of the narrow layout (the default for 32-bit keys, vg_msd.cu): the top
// key bits (the bucket, key >> lowbits) are split in one or two most-significant-digit
// partition passes of at most 8 bits each; every bucket's low lowbits <= 16 bits are then
// reduced on chip.
constexpr int kMsdMaxLow = 16;                 // largest bucket-local key width
constexpr int kMsdMaxTop = 16;                 // largest bucket id width (two 8-bit levels)
constexpr int kMsdBuckets = 1 << kMsdMaxTop;   // bucket ids
#ifndef VG_MSD_TARGET
#define VG_MSD_TARGET 2048
#endif
constexpr int kMsdTarget = VG_MSD_TARGET;               // average points per bucket the split aims at
// Clouds from this many points on take the bucket grouping under VG_METHOD_AUTO; smaller
// ones (camera frames, whose dense surfaces make large buckets of few cells) take the
// global radix sort, which is faster there (measured: a 640x480 frame 0.10 vs 0.20 ms,
// the 50M-point map 2.78 vs 2.24 ms).
constexpr int64_t kAutoBucketMinPoints = int64_t(1) << 22;
constexpr int kPartThreads = 256;              // partition pass: 256 threads x 16 records
constexpr int kPartItems = 16;
constexpr int kPartTile = kPartThreads * kPartItems;
// Entries the bucket kernel stages per job (build-time); larger buckets are cut into
// windows of at most this many entries by key range.
#ifndef VG_BK_STAGE
#define VG_BK_STAGE 3072
#endif
constexpr int kBkStage = VG_BK_STAGE;
constexpr int kJobWords = 8;                   // 32-bit words of one bucket-kernel job

// Segmented reduction geometry (256 threads x 4 sorted entries per tile).
constexpr int kRedThreads = 256;
constexpr int kRedItems = 4;
constexpr int kRedTile = kRedThreads * kRedItems;

// Streaming kernels (origin, keys, hash insert): 256 threads, 4 points per thread; the
// cloud is cut into chunks of 1024 points that never cross a frame boundary.
constexpr int kStreamThreads = 256;
constexpr int kStreamPoints = 4;
constexpr int kChunk = kStreamThreads * kStreamPoints;

// Frames per batched call.
constexpr int kMaxFrames = 1024;

// Chained-scan status flags (top two bits of a 32-bit status word).
constexpr uint32_t kFlagAggregate = 1u << 30;
constexpr uint32_t kFlagPrefix = 2u << 30;
constexpr uint32_t kValueMask = (1u << 30) - 1;

// Predecessor status words a chained-scan wait loads per round trip.
#ifndef VG_LOOKBACK_WINDOW
#define VG_LOOKBACK_WINDOW 1
#endif
constexpr int kLookbackWindow = VG_LOOKBACK_WINDOW;

// Largest cloud a call accepts: counts live in 30-bit chained-scan values.
constexpr int64_t kMaxPoints = (int64_t(1) << 30) - 1;

// Default spin limit of a chained-scan wait before it gives up with a timeout status.
constexpr uint32_t kDefaultSpinLimit = 1u << 22;

// Status codes shared with include/vg.h (device side).
constexpr int kErrInvalidArg = 1;
constexpr int kErrRange = 3;
constexpr int kErrCapacity = 4;
constexpr int kErrTimeout = 6;

// Per-frame device state (workspace, zeroed by every call).
struct FrameState {
  uint32_t ord_min_inv[3];  // max of ~ordered(x) over valid points: the min, via atomicMax
  uint32_t ord_max[3];      // max of ordered(x) over valid points
  float origin[3];          // origin used for the frame
  float leaf;               // leaf used for the frame
  uint32_t pad[2];
};

// Per-call device state, at the start of the workspace.  Zeroed by the call.
struct alignas(256) State {
  unsigned long long maxkey;  // largest sort key
  uint32_t nvalid;            // number of valid points
  uint32_t nitems;            // number of entries the radix sort orders
  uint32_t key_shift;         // bits of the per-frame key field (frame id above it)
  uint32_t nframes;
  uint32_t nchunks;           // chunks of the frame decomposition
  uint32_t narrow;            // 1: 32-bit sort keys + packed-offset payload (no gather)
  int32_t error;              // internal error word when the caller passes none
  uint32_t msd;               // 1: narrow layout grouped by buckets (vg_msd.cu)
  uint32_t lowbits;           // bucket = key >> lowbits; the low bits are reduced on chip
  uint32_t levels;            // partition passes over the bucket bits (1 or 2)
  uint32_t b1, b2;            // digit widths of the two passes (b2 = 0 with one pass)
  uint32_t njobs2;            // second-pass jobs (chunks of the first pass's digit runs)
  uint32_t nbjobs;            // non-empty buckets (in key order)
  uint32_t nmjobs;            // bucket-kernel jobs of whole buckets (runs of small ones)
  uint32_t nwjobs;            // bucket-kernel jobs of windows of large buckets
  uint32_t nbig;              // buckets of more than kBkStage entries
  uint32_t njobs3;            // chunks of large buckets the third partition pass splits
  uint32_t fspan;             // single-frame bins: bin = key >> fspan (vg_frame.cu)
  uint32_t ftop;              // single-frame bins: 2^ftop bins
  uint32_t fz_bar;            // one-launch frame grouping: grid-barrier arrivals
  uint32_t fz_rows;           // one-launch frame grouping: rows (occupied cells)
  uint32_t ctot[64];          // entries of every 1024 consecutive buckets
  uint32_t nztot[64];         // non-empty buckets of every 1024 consecutive buckets
  uint32_t vtot[64];          // cells of every 1024 consecutive non-empty buckets
  uint32_t tile_ctr[kMaxPasses + 8];
  uint32_t hist[kMaxPasses][kRadix];
};

// Per-tile record of the segmented reduction: run heads in the tile, the tile's first
// output row, and the sums of its leading entries (those continuing an earlier run).
struct alignas(8) TileRec {
  uint32_t heads;
  uint32_t vbase;
  uint32_t lead_n;
  uint32_t pad;
  long long lead_s[3];
  unsigned long long lead_a[4];  // attribute channel sums of the leading entries
};

// Frames of one call.  A single cloud is one frame [0, n) with offsets == nullptr.
struct FramesArg {
  const int64_t* offsets;  // device [F+1], or nullptr for one frame
  int nframes;
  int64_t n;               // total points
  const float* origin_in;  // device [F,3] origins to use, or nullptr: per-frame minimum
  float* origin_out;       // device [F,3] receives the minimum (when origin_in == nullptr)
  const float* leaves;     // device [F] per-frame leaves, or nullptr: `leaf` for all
  float leaf;
  int grid_per_sm;         // blocks per SM of the streaming kernels (0 = default 8)
  int allow_narrow;        // the key kernel may pick the narrow layout (no point_to_voxel)
  const float* poses;      // device [F,12] row-major [R|t] sensor poses, or nullptr
  const float* zlims;      // device [F,2] [z_min, z_max] after the pose, or nullptr
  int merge_frames;        // 1: every frame keys into one voxel space (no frame id)
  int lsd_narrow;          // 1: a narrow layout sorts every key digit in global radix passes
                           //    (the segmented reduction follows) instead of by buckets
};

// A posed call maps every point into the common frame, p' = R p + t, before anything
// else reads it, and drops points whose z' leaves [z_min, z_max].
inline bool posed(const FramesArg& fr) { return fr.poses != nullptr || fr.zlims != nullptr; }

// Grid of the streaming kernels: one block per chunk, at most grid_per_sm blocks per SM.
int stream_grid(const FramesArg& fr);

constexpr int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
constexpr size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Upper bound of the chunk count of n points in F frames.
constexpr int64_t max_chunks(int64_t n, int frames) { return ceil_div(n, kChunk) + frames; }

// Workspace layout of the sort path for n points in `frames` frames.  The narrow layout
// (32-bit keys, 64-bit packed offsets) aliases the same bytes: keys32 ping-pong in keys0,
// payload ping-pong in keys1 and in idx0..idx1.
struct SortLayout {
  size_t state, frames, keys0, keys1, idx0, idx1, lb_a, lb_b, seg_lb, mhist, mvcnt, mcur,
      mjob, mjob2, mjobm, mjobw, mcur3, mjob3, total;
  size_t zero_bytes;  // bytes from `state` that must be zero at call start
  int64_t sort_tiles, seg_tiles, jobs2, jobsw, big, jobs3;
};

// Second-pass jobs of the bucket grouping: the first pass's digit runs cut into pieces of
// at most kPartTile entries.
constexpr int64_t max_jobs2(int64_t n) { return ceil_div(n, kPartTile) + 256; }
// Window jobs of large buckets: two consecutive windows of a bucket hold more than
// kBkStage entries (or the first is one oversized key range), so a bucket of m entries
// has at most 2m/kBkStage + 1 windows, and only buckets above kBkStage entries have any.
constexpr int64_t max_jobsw(int64_t n) { return 3 * ceil_div(n, kBkStage) + 16; }
// Buckets of more than kBkStage entries, and their chunks of at most kPartTile entries.
constexpr int64_t max_big(int64_t n) { return n / (kBkStage + 1) + 1; }
constexpr int64_t max_jobs3(int64_t n) { return ceil_div(n, kPartTile) + max_big(n); }

constexpr SortLayout sort_layout(int64_t n, int frames = 1) {
  SortLayout L{};
  const int64_t nn = n < 1 ? 1 : n;
  const int64_t ff = frames < 1 ? 1 : frames;
  L.sort_tiles = ceil_div(nn, kSortTile);
  L.seg_tiles = ceil_div(nn, kRedTile);
  L.jobs2 = max_jobs2(nn);
  L.jobsw = max_jobsw(nn);
  L.big = max_big(nn);
  L.jobs3 = max_jobs3(nn);
  size_t off = 0;
  L.state = off;
  off = align_up(off + sizeof(State), 256);
  L.frames = off;
  off = align_up(off + size_t(ff) * sizeof(FrameState), 256);
  L.lb_a = off;
  off = align_up(off + size_t(L.sort_tiles) * kRadix * sizeof(uint32_t), 256);
  L.seg_lb = off;  // per-tile records, then the tiles' head counts as a compact array
  off = align_up(off + size_t(L.seg_tiles) * (sizeof(TileRec) + sizeof(uint32_t)), 256);
  L.zero_bytes = off;  // state, frames, pass-0 status rows and segment status
  // bucket grouping: points per bucket (zeroed by calls that may take the grouping)
  L.mhist = off;
  off = align_up(off + size_t(kMsdBuckets) * sizeof(uint32_t), 256);
  L.mvcnt = off;  // cells of every non-empty bucket
  off = align_up(off + size_t(kMsdBuckets) * sizeof(uint32_t), 256);
  L.mcur = off;  // write cursors: 256 of the first pass, then one per bucket (which later
                 // hold every non-empty bucket's first row)
  off = align_up(off + size_t(256 + kMsdBuckets) * sizeof(uint32_t), 256);
  L.mjob = off;  // non-empty buckets: first entry, entries, bucket id (kMsdBuckets each)
  off = align_up(off + size_t(kMsdBuckets) * 3 * sizeof(uint32_t), 256);
  L.mjob2 = off;  // tables of the first pass's digit runs (first entries, first jobs)
  off = align_up(off + 2 * 257 * sizeof(uint32_t), 256);
  L.mjobm = off;  // bucket-kernel jobs of whole buckets
  off = align_up(off + size_t(kMsdBuckets) * kJobWords * sizeof(uint32_t), 256);
  L.mjobw = off;  // bucket-kernel jobs of windows of large buckets
  off = align_up(off + size_t(L.jobsw) * kJobWords * sizeof(uint32_t), 256);
  L.mcur3 = off;  // third-pass write cursors: 256 per large bucket
  off = align_up(off + size_t(L.big) * 256 * sizeof(uint32_t), 256);
  L.mjob3 = off;  // third-pass jobs: first entry, entries, large-bucket index
  off = align_up(off + size_t(L.jobs3) * 4 * sizeof(uint32_t), 256);
  L.lb_b = off;
  off = align_up(off + size_t(L.sort_tiles) * kRadix * sizeof(uint32_t), 256);
  L.keys0 = off;  // also the two 32-bit key arrays of the narrow layout, 16-byte aligned
  off = align_up(off + size_t(nn) * sizeof(uint64_t) + 16, 256);
  L.keys1 = off;
  off = align_up(off + size_t(nn) * sizeof(uint64_t), 256);
  L.idx0 = off;
  off = align_up(off + size_t(nn) * sizeof(uint32_t), 256);
  L.idx1 = off;
  off = align_up(off + size_t(nn) * sizeof(uint32_t), 256);
  // bulk copies of the bucket kernel read whole 16-byte granules: up to 16 bytes past the
  // last entry of an array
  L.total = off + 256;
  return L;
}

int num_sms();
uint32_t spin_limit();
// Grid of a persistent kernel: all its blocks resident at once (occupancy x SMs), at most
// one block per unit of work.  Sets the dynamic shared-memory limit when needed.
int persistent_grid(const void* kernel, int threads, size_t dyn_smem, int64_t work_tiles);
// Runs the occupancy queries of every persistent kernel on the current device (so that a
// later CUDA-graph capture makes none).
void warm_launch_config();
void warm_sort_config();
void warm_reduce_config();

// Launchers (all asynchronous on `stream`).
// a1: per-frame min (and max) of the valid points into FrameState.
// `zero`/`zero_bytes` (16-byte multiple, or 0): a region the kernel also clears.
cudaError_t launch_origin(const float* xyz, const FramesArg& fr, State* st, FrameState* fs,
                          int* err, cudaStream_t stream, void* zero = nullptr,
                          size_t zero_bytes = 0);
// a2: per-point sort keys (frame id above a key_shift-bit Morton field; ~0 = invalid).
cudaError_t launch_keys(const float* xyz, const FramesArg& fr, bool have_extent, State* st,
                        FrameState* fs, uint64_t* keys, int* err, cudaStream_t stream);
// Buffers of the narrow layout (32-bit keys, packed-offset payloads), ping-pong.
struct NarrowBuffers {
  uint32_t* k0;
  uint64_t* p0;
  uint32_t* k1;
  uint64_t* p1;
};
constexpr int kNarrowPasses = 4;
// a3: one radix pass of the layout the key kernel chose.  compact_input: pass 0 reads
// st->nitems compacted keys with their payload from idx0 (hash path, wide layout only)
// instead of n raw keys with an implicit index.  nb = nullptr: wide layout only.
cudaError_t launch_sort_pass(State* st, uint64_t* keys0, uint32_t* idx0, uint64_t* keys1,
                             uint32_t* idx1, uint32_t* lb_a, uint32_t* lb_b, int64_t n_max,
                             int pass, bool compact_input, uint32_t spin_limit, int* err,
                             cudaStream_t stream, const NarrowBuffers* nb = nullptr);
// a4 + a5: reduce-by-key of the sorted table into key-ordered voxels.
struct SegOut {
  uint64_t* keys;
  float* centroids;
  uint32_t* counts;
  long long* sums;         // optional [cap,3] fixed-point sums (pyramid input)
  int64_t cap;
  int64_t* num_voxels;
  int64_t* frame_offsets;  // optional [F+1] per-frame output offsets
  int32_t* p2v;
  const uint8_t* attrs_in;  // optional [n, channels] per-point attributes (wide layout)
  int channels;
  float* attrs_out;         // [cap, channels] per-voxel means
};
cudaError_t launch_segreduce(State* st, const FrameState* fs, int nframes,
                             const uint64_t* keys0, const uint32_t* idx0, const uint64_t* keys1,
                             const uint32_t* idx1, const float* xyz, TileRec* recs,
                             int64_t n_max, const SegOut& out, int* err, cudaStream_t stream,
                             const NarrowBuffers* nb = nullptr, const float* poses = nullptr);
// Bucket grouping of the narrow layout (vg_msd.cu): the partition passes over the bucket
// bits, then every bucket reduced on chip into its rows.  Kernels return at once unless
// the key kernel chose the narrow layout with bucket grouping.
cudaError_t launch_msd(State* st, const FrameState* fs, int nframes, const NarrowBuffers& nb,
                       char* ws, const SortLayout& L, int64_t n_max, const SegOut& out,
                       uint32_t spin_limit, int* err, cudaStream_t stream, int stage0,
                       void (*mark)(int, cudaStream_t));
void warm_msd_config();
// Minimum-count filter (vg_filter.cu): its scratch follows the grouping method's layout.
struct FilterLayout {
  size_t ticket, status, remap, zero_bytes, total;
};
FilterLayout filter_layout(int64_t cap, size_t base);
cudaError_t launch_filter(char* ws, const FilterLayout& L, int64_t cap, uint32_t min_count,
                          const SegOut& out, int nframes, int64_t n_points, uint32_t spin_limit,
                          int* err, cudaStream_t stream);
void warm_filter_config();
// a2, narrow-capable key kernel: writes either 64-bit keys to keys64 (wide) or 32-bit keys
// and packed offsets (narrow, when allowed and the sort key fits in 32 bits).
cudaError_t launch_keys_any(const float* xyz, const FramesArg& fr, bool have_extent, State* st,
                            FrameState* fs, uint64_t* keys64, uint32_t* keys32,
                            uint64_t* payload, int* err, cudaStream_t stream);

// ---- hash path ----
struct alignas(32) HashAcc {
  uint32_t n;
  uint32_t pad;
  long long s[3];
};
struct HashTable {
  unsigned long long* keys;  // [H], ~0 = empty
  HashAcc* acc;              // [H]
  uint32_t mask;             // H - 1, H a power of two
};

// Slot count of the hash table for n points: a power of two >= 2n (never fills).
constexpr int64_t hash_slots(int64_t n) {
  int64_t h = 1024;
  while (h < 2 * n) h <<= 1;
  return h;
}

struct HashLayout {
  size_t state, frames, lb_a, zero_bytes, lb_b, keys0, keys1, idx0, idx1, tkeys, tacc, slot_rank,
      point_slot, total;
  int64_t slots, sort_tiles;
};

constexpr HashLayout hash_layout(int64_t n, int frames = 1) {
  HashLayout L{};
  const int64_t nn = n < 1 ? 1 : n;
  const int64_t ff = frames < 1 ? 1 : frames;
  L.slots = hash_slots(nn);
  L.sort_tiles = ceil_div(nn, kSortTile);
  size_t off = 0;
  L.state = off;
  off = align_up(off + sizeof(State), 256);
  L.frames = off;
  off = align_up(off + size_t(ff) * sizeof(FrameState), 256);
  L.lb_a = off;
  off = align_up(off + size_t(L.sort_tiles) * kRadix * sizeof(uint32_t), 256);
  L.zero_bytes = off;
  L.lb_b = off;
  off = align_up(off + size_t(L.sort_tiles) * kRadix * sizeof(uint32_t), 256);
  L.keys0 = off;  // also the two 32-bit key arrays of the narrow layout, 16-byte aligned
  off = align_up(off + size_t(nn) * sizeof(uint64_t) + 16, 256);
  L.keys1 = off;
  off = align_up(off + size_t(nn) * sizeof(uint64_t), 256);
  L.idx0 = off;
  off = align_up(off + size_t(nn) * sizeof(uint32_t), 256);
  L.idx1 = off;
  off = align_up(off + size_t(nn) * sizeof(uint32_t), 256);
  L.tkeys = off;
  off = align_up(off + size_t(L.slots) * sizeof(unsigned long long), 256);
  L.tacc = off;
  off = align_up(off + size_t(L.slots) * sizeof(HashAcc), 256);
  L.slot_rank = off;
  off = align_up(off + size_t(L.slots) * sizeof(uint32_t), 256);
  L.point_slot = off;
  off = align_up(off + size_t(nn) * sizeof(uint32_t), 256);
  L.total = off;
  return L;
}

cudaError_t launch_hash_insert(const float* xyz, const FramesArg& fr, bool have_extent, State* st,
                               FrameState* fs, const HashTable& tab, uint32_t* point_slot,
                               uint32_t spin_limit, int* err, cudaStream_t stream);
cudaError_t launch_hash_compact(const HashTable& tab, State* st, uint64_t* keys, uint32_t* slots,
                                const int* err, cudaStream_t stream);
cudaError_t launch_hash_finalize(const State* st, const FrameState* fs, int nframes,
                                 const uint64_t* keys0, const uint32_t* idx0,
                                 const uint64_t* keys1, const uint32_t* idx1,
                                 const HashTable& tab, uint32_t* slot_rank, int64_t n_max,
                                 const SegOut& out, int* err, cudaStream_t stream);
cudaError_t launch_hash_p2v(const uint32_t* point_slot, const uint32_t* slot_rank, int64_t n,
                            int32_t* p2v, const int* err, cudaStream_t stream);

// ---- pyramid ----
constexpr int kMaxLevels = 8;
constexpr int kMergeThreads = 256;
constexpr int kMergeItems = 8;
constexpr int kMergeTile = kMergeThreads * kMergeItems;
// Merges pyramid level k-1 (rows [off[k-1], off[k])) into level k (written from off[k]).
cudaError_t launch_pyramid_merge(State* st, const FrameState* fs, int level, uint64_t* keys,
                                 float* centroids, uint32_t* counts, const long long* sums_in,
                                 long long* sums_out, int64_t* level_offsets, int64_t cap,
                                 uint32_t* lb, int64_t n_max, uint32_t spin_limit, int* err,
                                 cudaStream_t stream);

// Test: a bounded chained-scan wait on words nobody sets (records kErrTimeout).
cudaError_t launch_debug_wait(const uint32_t* status, int tile, uint32_t limit, int* err,
                              cudaStream_t stream);

// ---- backward ----
cudaError_t launch_backward(const float* grad_centroids, const uint32_t* counts,
                            const int32_t* p2v, int64_t n, int64_t num_voxels, float* grad_xyz,
                            int* err, cudaStream_t stream);

}  // namespace vg
