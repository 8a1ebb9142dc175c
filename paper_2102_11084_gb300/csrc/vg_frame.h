// Scratch layouts and launches of the single-frame groupings (VG_SORT_FRAME, vg_frame.cu):
// the one-launch grouping and the bin grouping of frames above its capacity.
#pragma once
#include "vg_internal.h"

namespace vg {

// The single-frame bin grouping (VG_SORT_FRAME, vg_frame.cu): the sort layout's key
// arrays, then the runs of equal keys and their places in their bins, the zeroed bin
// counts and scan status words, the bins' first entries and cells.
constexpr int kFrSpanBits = 12;  // a bin holds 2^12 consecutive keys
constexpr int kFrMaxTop = 20;    // at most 2^20 bins (32-bit keys)
constexpr int kFrMaxUnitBits = 12;  // at most 2^12 look-back units of bins
constexpr int kFrScanBins = 4096;   // bins per tile of the bin-count scan
struct FrameLayout {
  size_t pos, rin, rout, zero, hist, ustat, pstat, tick, start, vcnt, zero_bytes, total;
};
constexpr FrameLayout frame_layout(int64_t n, size_t base) {
  FrameLayout L{};
  const int64_t nn = n < 1 ? 1 : n;
  size_t off = align_up(base, 256);
  L.pos = off;  // each run's place in its bin (at its last point)
  off = align_up(off + size_t(nn) * sizeof(uint32_t), 256);
  L.rin = off;  // runs (three offset sums and the points) at their last point
  off = align_up(off + size_t(nn) * 4 * sizeof(uint32_t), 256);
  L.rout = off;  // the runs grouped by bin
  off = align_up(off + size_t(nn) * 4 * sizeof(uint32_t), 256);
  L.zero = off;
  L.hist = off;
  off = align_up(off + (size_t(1) << kFrMaxTop) * sizeof(uint32_t), 256);
  L.ustat = off;
  off = align_up(off + (size_t(1) << kFrMaxUnitBits) * sizeof(uint32_t), 256);
  L.pstat = off;
  off = align_up(off + ((size_t(1) << kFrMaxTop) / kFrScanBins) * sizeof(uint32_t), 256);
  L.tick = off;
  off = align_up(off + 4 * sizeof(uint32_t), 256);
  L.zero_bytes = off - L.zero;
  L.start = off;
  off = align_up(off + ((size_t(1) << kFrMaxTop) + 1) * sizeof(uint32_t), 256);
  L.vcnt = off;  // cells of every bin
  off = align_up(off + (size_t(1) << kFrMaxTop) * sizeof(uint32_t), 256);
  L.total = off;
  return L;
}

// The single-frame grouping in one cooperative launch (vg_frame.cu): an occupancy bitmap
// over the frame's keys (every key of up to kFzDenseBits bits, else bitmaps of the occupied
// blocks of 2^kFzBlockBits keys) ranks the cells in key order, and the cells' counts and
// sums are added at their rows.  Scratch after the sort layout's frame state.
constexpr int kFzThreads = 1024;   // threads of a block (one block per SM)
constexpr int kFzPer = 14;         // points a thread holds at most
constexpr int kFzMaxPointsBits = 21;  // a frame of at most 2^21 points
constexpr int kFzDenseBits = 26;   // keys of up to 26 bits: one bitmap over every key
constexpr int kFzZeroBits = 24;    // bitmap bits the kernel clears before the extents
constexpr int kFzBlockBits = 9;    // wider keys: bitmaps of the occupied blocks of 2^9 keys
constexpr int kFzMaxGrid = 1024;   // blocks of the launch at most (chained-scan words)
constexpr size_t kFzDenseWords = size_t(1) << (kFzDenseBits - 5);
constexpr size_t kFzZeroWords = size_t(1) << (kFzZeroBits - 5);
static_assert(kFzZeroWords >= (size_t(1) << (32 - kFzBlockBits - 5)), "block bitmap cleared");
struct FusedLayout {
  size_t bits, rank, slotmap, slotbin, sbits, srank, acc, rowkey, stat, total;
};
constexpr FusedLayout fused_layout(int64_t n, size_t base) {
  FusedLayout L{};
  const size_t nn = size_t(n < 1 ? 1 : n);
  size_t off = align_up(base, 256);
  L.bits = off;  // key bitmap, or the occupied-block bitmap of wide keys (zeroed by the kernel)
  off = align_up(off + kFzDenseWords * sizeof(uint32_t), 256);
  L.rank = off;  // set bits before every word of `bits`
  off = align_up(off + kFzDenseWords * sizeof(uint32_t), 256);
  L.slotmap = off;  // block -> slot, written for occupied blocks only
  off = align_up(off + (size_t(1) << (32 - kFzBlockBits)) * sizeof(uint32_t), 256);
  L.slotbin = off;  // slot -> block (at most one slot a point)
  off = align_up(off + nn * sizeof(uint32_t), 256);
  L.sbits = off;  // 16 words of key bitmap a slot
  off = align_up(off + nn * 16 * sizeof(uint32_t), 256);
  L.srank = off;
  off = align_up(off + nn * 16 * sizeof(uint32_t), 256);
  L.acc = off;  // three arrays of 64-bit sums, one entry a row (at most one row a point)
  off = align_up(off + nn * 3 * sizeof(unsigned long long), 256);
  L.rowkey = off;  // the key of every row
  off = align_up(off + nn * sizeof(uint32_t), 256);
  L.stat = off;  // the two rankings' per-block totals
  off = align_up(off + 2 * size_t(kFzMaxGrid) * sizeof(uint32_t), 256);
  L.total = off;
  return L;
}

// The single-frame bin grouping after the extent kernel (which cleared the layout's zero
// region): keys and bin places, bin starts, the scatter into bins, and the rows.
cudaError_t launch_frame(const float* xyz, const FramesArg& fr, State* st, FrameState* fs,
                         const NarrowBuffers& nb, char* ws, const FrameLayout& FL,
                         const SegOut& out, uint32_t spin_limit, int* err, cudaStream_t stream);
void warm_frame_config();
// Whether one cooperative launch holds a frame of n points (the grid resident at once, at
// most kFzPer points a thread); the caller then runs launch_frame_fused in place of the
// extent kernel and launch_frame.
bool frame_fused_fits(int64_t n, bool posed);
int64_t frame_fused_max_points(bool posed);
cudaError_t launch_frame_fused(const float* xyz, const FramesArg& fr, State* st, FrameState* fs,
                               char* ws, const FusedLayout& ZL, const SegOut& out,
                               uint32_t spin_limit, int* err, cudaStream_t stream);
// Test of the grid barrier's bounded wait (a two-block cooperative launch whose barrier
// waits for one block more than it has).
cudaError_t launch_debug_grid_barrier(uint32_t* ctr, uint32_t limit, int* err,
                                      cudaStream_t stream);
}  // namespace vg
