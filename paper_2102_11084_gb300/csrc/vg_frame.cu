// Steps a1-a5 for one camera frame (VG_SORT_FRAME).
//
// arXiv 2102.11084 Sec. II-C filters one camera cloud per call (Table I times that call),
// and a frame's points all fall in a few thousand cells per axis at most, so its keys fit
// 32 bits and its cells are few: launches, not bytes, cost the time.  A frame the grid
// holds (vg_frame_one_launch_points) is grouped by frame_fused_kernel, ONE cooperative
// launch (below): the rank of each occupied key's bit in an occupancy bitmap over the
// keys is its row, and every run of points adds its sums at its row.  A larger frame's
// Morton keys split into bins of 2^12 consecutive keys (a 16-cell cube) with at most 2^20
// bins; order inside a bin is the only sorting left, and a bin's cells fit one block's
// shared memory densely (one counter and three sums per key of the bin), so that grouping
// is a counting pass, one scatter and one reduction:
//   frame_key_kernel     the key and corner offsets of every point (the key kernel's
//                        arithmetic); runs of equal keys among 32 consecutive pixels
//                        summed into one entry, and its place in its bin (one global
//                        atomic per warp and bin, which also counts the bins);
//   frame_prefix_kernel  the bins' first entries (a chained scan over tiles of 4096 bins);
//   frame_scatter_kernel every entry to its bin's first entry plus its place;
//   frame_count_kernel   every bin's cells (the population of an occupancy bitmap);
//   frame_bin_kernel     units of consecutive bins (at most 4096 units) in ticket order:
//                        a chained scan over the units' cells gives each unit's first row
//                        as soon as it is taken; each bin's entries add into its 4096
//                        counters and sums (runs of equal keys summed across a warp first,
//                        then shared-memory atomics), an occupancy bitmap ranks its cells,
//                        and one thread per occupied key writes its row (the centroid
//                        formula of acc_centroid).
// Same cells, counts and integer sums as every other grouping in both: the rows are
// bit-identical.  Before the bin grouping, the extent kernel clears the bin counts and
// status words.
#include <cstddef>

#include "vg_device.cuh"
#include "vg_internal.h"
#include "vg_frame.h"
#include "vg_rows.cuh"
#include "vg_stream.cuh"

namespace vg {
namespace {

constexpr uint32_t kFrSpan = 1u << kFrSpanBits;
constexpr int kFrThreads = 512;
constexpr int kFrWords = kFrSpan / 32;  // occupancy words of a bin
constexpr int kFrPer = kFrSpan / kFrThreads;  // keys of a bin per thread
static_assert(kFrWords <= 4 * 32, "one warp scans a bin's occupancy words, four a lane");
static_assert(kFrScanBins == 16 * 256, "prefix tile: 16 bins per thread");

// Runs of equal keys among a warp's 32 consecutive points: a segmented scan sums each run's
// offsets and points (32 offsets of 21 bits fit 32 bits) into v = {x, y, z, points} of
// its last lane, which returns true (invalid points, key all ones, form no run).
__device__ __forceinline__ bool warp_run(uint32_t k, uint64_t pw, bool ok, uint32_t v[4]) {
  const uint32_t lane = threadIdx.x & 31u;
  v[0] = uint32_t(pw) & 0x1fffffu;
  v[1] = uint32_t(pw >> 21) & 0x1fffffu;
  v[2] = uint32_t(pw >> 42) & 0x1fffffu;
  v[3] = ok ? 1u : 0u;
  const uint32_t prev = __shfl_up_sync(kFullMask, k, 1);
  const uint32_t heads = __ballot_sync(kFullMask, lane == 0 || k != prev);
  const uint32_t head = 31u - __clz(heads & (0xffffffffu >> (31u - lane)));
#pragma unroll
  for (uint32_t d = 1; d < 32; d <<= 1) {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const uint32_t yv = __shfl_up_sync(kFullMask, v[a], d);
      if (lane >= head + d) v[a] += yv;
    }
  }
  return ok && (lane == 31u || ((heads >> (lane + 1u)) & 1u) != 0u);
}

// ---- keys, runs and places in bins ---------------------------------------------------------
// Lane l of warp w takes point start + 256 s + 32 w + l of every chunk (s = 0..3), so a
// warp holds 32 consecutive points at a time: neighbouring pixels of a camera frame, which
// often share a cell.  Equal keys of consecutive lanes form a run; a segmented scan sums
// its points and offsets (32 offsets of 21 bits fit 32 bits), and the run's last lane
// writes it -- key, then {sum x, sum y, sum z, points} -- at its own point index, with its
// place in its bin (one global atomic per warp and bin).  Every other index gets the
// all-ones key.  st->nvalid counts the valid points, st->nitems the runs.
template <bool kPosed>
__global__ __launch_bounds__(kStreamThreads) void frame_key_kernel(
    const float* __restrict__ xyz, FramesArg fr, State* st, FrameState* fs,
    uint32_t* __restrict__ keys, uint4* __restrict__ runs, uint32_t* __restrict__ pos,
    uint32_t* __restrict__ hist, int* err) {
  __shared__ ChunkSmem sm;
  __shared__ unsigned long long wmax[kStreamThreads / 32];
  __shared__ uint32_t wcount[kStreamThreads / 32], wruns[kStreamThreads / 32];
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t T = build_chunk_map(fr, sm.off, sm.cstart, sm.tmp, err);
  bool narrow = false;
  uint32_t kb = 0;
  const uint32_t key_shift =
      frame_prologue(fr, true, st, fs, T, sm, err, &narrow, nullptr, &kb);
  const uint32_t span = kb < kFrSpanBits ? kb : uint32_t(kFrSpanBits);  // bin = key >> span
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->fspan = span;
    st->ftop = kb - span;
    if (!narrow) set_error(err, kErrRange);  // keys of more than 32 bits
  }
  if (!narrow) return;  // (uniform: the prologue's decision)
  uint32_t c0, c1;
  block_range(T, &c0, &c1);
  uint32_t nvalid = 0, nruns = 0, kmax = 0;
  bool range_bad = false;
  Pose P;
  int pose_f = -1;
  for (uint32_t c = c0; c < c1; ++c) {
    const int f = chunk_frame(sm.cstart, fr.nframes, c);
    const int64_t start = sm.off[f] + int64_t(c - sm.cstart[f]) * kChunk;
    const int64_t end = min(start + kChunk, sm.off[f + 1]);
    if (kPosed && f != pose_f) {
      load_pose(fr, f, P);
      pose_f = f;
    }
    const float o[3] = {sm.org[f][0], sm.org[f][1], sm.org[f][2]};
#pragma unroll 1
    for (int s4 = 0; s4 < kStreamPoints; ++s4) {
      const int64_t p = start + int64_t(s4) * kStreamThreads + threadIdx.x;
      const bool in = p < end;
      float x = in ? __ldcs(xyz + 3 * p) : __int_as_float(0x7fc00000);
      float y = in ? __ldcs(xyz + 3 * p + 1) : x;
      float z = in ? __ldcs(xyz + 3 * p + 2) : x;
      if (kPosed) pose_point(P, x, y, z);
      uint32_t k = kFullMask;
      uint64_t pw = 0;
      const bool ok = narrow_entry(x, y, z, o, sm.leaf[f], sm.rleaf[f], sm.inv_unit[f],
                                   static_cast<uint32_t>(f), key_shift, &k, &pw, &range_bad);
      if (!ok) k = kFullMask;
      nvalid += ok;
      kmax = ok && k > kmax ? k : kmax;
      uint32_t v[4];
      const bool emit = warp_run(k, pw, ok, v);
      const uint32_t em = __ballot_sync(kFullMask, emit);
      uint32_t q = 0;
      if (emit) {
        ++nruns;
        const uint32_t bin = k >> span;
        const uint32_t peers = __match_any_sync(em, bin);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (int(lane) == leader) base = atomicAdd(&hist[bin], uint32_t(__popc(peers)));
        base = __shfl_sync(peers, base, leader);
        q = base + __popc(peers & ((1u << lane) - 1u));
      }
      if (in) {
        __stcg(keys + p, emit ? k : kFullMask);
        if (emit) {
          __stcg(pos + p, q);
          __stcg(runs + p, make_uint4(v[0], v[1], v[2], v[3]));
        }
      }
    }
  }
  if (__any_sync(kFullMask, range_bad) && lane == 0) set_error(err, kErrRange);
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    nvalid += __shfl_xor_sync(kFullMask, nvalid, off);
    nruns += __shfl_xor_sync(kFullMask, nruns, off);
    kmax = max(kmax, __shfl_xor_sync(kFullMask, kmax, off));
  }
  if (lane == 0) {
    wcount[warp] = nvalid;
    wruns[warp] = nruns;
    wmax[warp] = kmax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t cnt = 0, rc = 0;
    unsigned long long m = 0;
    for (int w = 0; w < kStreamThreads / 32; ++w) {
      cnt += wcount[w];
      rc += wruns[w];
      m = wmax[w] > m ? wmax[w] : m;
    }
    if (cnt) {
      atomicAdd(&st->nvalid, cnt);
      atomicAdd(&st->nitems, rc);
      atomicMax(&st->maxkey, m);
    }
  }
}

// ---- first entry of every bin -----------------------------------------------------------
// Tiles of kFrScanBins bins in ticket order; start[2^ftop] = the entries, which must be the
// runs the key kernel counted.
__global__ __launch_bounds__(256) void frame_prefix_kernel(State* st, const uint32_t* hist,
                                                           uint32_t* __restrict__ start,
                                                           uint32_t* status, uint32_t* ticket,
                                                           uint32_t spin_limit, int* err) {
  __shared__ uint32_t tmp[8];
  __shared__ int s_tile;
  __shared__ uint32_t s_excl;
  if (block_error_raised(err)) return;
  const int t = threadIdx.x;
  const uint32_t nb = 1u << st->ftop;
  const int tiles = int((nb + kFrScanBins - 1) / kFrScanBins);
  for (;;) {
    if (t == 0) s_tile = static_cast<int>(atomicAdd(ticket, 1u));
    __syncthreads();
    const int tile = s_tile;
    if (tile >= tiles) break;
    const uint32_t b0 = uint32_t(tile) * kFrScanBins + 16u * uint32_t(t);
    uint32_t c[16], mine = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint4 w = make_uint4(0u, 0u, 0u, 0u);
      if (b0 + 4u * q < nb) w = *reinterpret_cast<const uint4*>(hist + b0 + 4u * q);
      c[4 * q] = w.x;
      c[4 * q + 1] = w.y;
      c[4 * q + 2] = w.z;
      c[4 * q + 3] = w.w;
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) mine += c[q];
    uint32_t total;
    uint32_t run = block_excl_scan(mine, &total, tmp);
    if (t == 0) {
      uint32_t excl = 0;
      if (tile == 0) {
        st_relaxed(status, kFlagPrefix | total);
      } else {
        st_relaxed(status + tile, kFlagAggregate | total);
        excl = lookback_u32(status, 1, tile, spin_limit, err);
        st_relaxed(status + tile, kFlagPrefix | ((excl + total) & kValueMask));
      }
      s_excl = excl;
      if (tile == tiles - 1) {
        start[nb] = excl + total;
        if (excl + total != st->nitems) set_error(err, kErrInvalidArg);
      }
    }
    __syncthreads();
    run += s_excl;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      if (b0 + q < nb) start[b0 + q] = run;
      run += c[q];
    }
  }
}

// ---- runs into their bins ------------------------------------------------------------------
__global__ __launch_bounds__(256) void frame_scatter_kernel(
    const State* st, const uint32_t* __restrict__ kin, const uint4* __restrict__ rin,
    const uint32_t* __restrict__ pos, const uint32_t* __restrict__ start,
    uint32_t* __restrict__ kout, uint4* __restrict__ rout, int64_t n, const int* err) {
  if (error_raised(err)) return;
  const uint32_t span = st->fspan;
  const uint32_t cap = st->nitems;
  for (int64_t i = int64_t(blockIdx.x) * 256 + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * 256) {
    const uint32_t k = __ldcs(kin + i);
    if (k == kFullMask) continue;
    const uint32_t d = __ldg(start + (k >> span)) + __ldcs(pos + i);
    if (d < cap) {
      kout[d] = k;
      rout[d] = __ldcs(rin + i);
    }
  }
}

// ---- cells of every bin -------------------------------------------------------------------
// Block b takes bins b, b + G, ...: the occupancy bitmap of the bin's keys (a lane skips a
// key equal to the one before it), its population into cells[bin].
__global__ __launch_bounds__(256) void frame_count_kernel(const State* st,
                                                          const uint32_t* __restrict__ keys,
                                                          const uint32_t* __restrict__ hist,
                                                          const uint32_t* __restrict__ start,
                                                          uint32_t* __restrict__ cells,
                                                          const int* err) {
  __shared__ uint32_t bits[kFrWords];
  __shared__ uint32_t red[8];
  if (block_error_raised(err)) return;
  const int t = threadIdx.x, lane = t & 31;
  const uint32_t span = 1u << st->fspan, mask = span - 1u;
  const int nw = int((span + 31u) >> 5);
  const uint32_t nb = 1u << st->ftop;
  if (t < kFrWords) bits[t] = 0;
  __syncthreads();
  for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x) {
    const uint32_t m = __ldg(hist + b);
    if (m == 0) {
      if (t == 0) cells[b] = 0;
      continue;
    }
    const uint32_t s0 = __ldg(start + b);
    for (uint32_t i0 = 0; i0 < m; i0 += 4 * 256) {  // four loads in flight a thread
      uint32_t off[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t i = i0 + uint32_t(q) * 256 + uint32_t(t);
        off[q] = i < m ? (__ldcg(keys + s0 + i) & mask) : 0xffffffffu;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t prev = __shfl_up_sync(kFullMask, off[q], 1);
        if (off[q] != 0xffffffffu && (lane == 0 || off[q] != prev))
          atomicOr(&bits[off[q] >> 5], 1u << (off[q] & 31u));
      }
    }
    __syncthreads();
    uint32_t c = 0;
    if (t < nw) {
      c = __popc(bits[t]);
      bits[t] = 0;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(kFullMask, c, o);
    if (lane == 0) red[t >> 5] = c;
    __syncthreads();
    if (t == 0) {
      uint32_t v = 0;
      for (int w = 0; w < 8; ++w) v += red[w];
      cells[b] = v;
    }
  }
}

// ---- rows ---------------------------------------------------------------------------------
struct alignas(16) FrSmem {
  // biased offset sums of every key of the bin, 64 bits a sum: a 32-bit low word per axis,
  // and the three axes' carries (an addition below 2^31 that wraps a low word adds one)
  // packed 21 bits apart in one 64-bit word (fewer than 2^32 points keep every carry
  // count below 2^21, so no field overflows into the next)
  uint32_t lo[3][kFrSpan];
  unsigned long long hi[kFrSpan];
  uint32_t cnt[kFrSpan];               // entries of every key of the bin
  uint32_t bits[2][kFrWords];          // occupancy of alternate bins (kept clean)
  uint16_t wrank[kFrWords];            // occupied keys before every word
  uint32_t tmp[kFrThreads / 32];
  uint32_t s_v, s_excl;
  int s_unit;
};

// The bin's runs into the counters and sums, and its occupancy bitmap.  Every warp takes 32
// consecutive runs at a time; equal keys among them (runs cut at warp boundaries of the
// key kernel) are summed again by a segmented scan across the lanes (32 runs of at most
// 32 offsets of 21 bits fit 32 bits), and only each group's last lane adds into shared
// memory.
__device__ __forceinline__ void frame_accumulate(FrSmem& sm, uint32_t* bits,
                                                 const uint32_t* __restrict__ keys,
                                                 const uint4* __restrict__ runs, uint32_t s0,
                                                 uint32_t m, uint32_t mask) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  constexpr int kU = 2;  // groups of 32 runs a warp loads before reducing
  for (uint32_t b = warp * 32u; b < m; b += kU * kFrThreads) {
    uint32_t off[kU];
    uint4 r[kU];
#pragma unroll
    for (int g = 0; g < kU; ++g) {
      const uint32_t i = b + uint32_t(g) * kFrThreads + lane;
      const bool in = i < m;
      off[g] = in ? (__ldcg(keys + s0 + i) & mask) : 0xffffffffu;
      r[g] = in ? __ldcg(runs + s0 + i) : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int g = 0; g < kU; ++g) {
      uint32_t v[4] = {r[g].w, r[g].x, r[g].y, r[g].z};
      const uint32_t prev = __shfl_up_sync(kFullMask, off[g], 1);
      const uint32_t heads = __ballot_sync(kFullMask, lane == 0 || off[g] != prev);
      const uint32_t head = 31u - __clz(heads & (0xffffffffu >> (31u - lane)));  // my group's
#pragma unroll
      for (uint32_t d = 1; d < 32; d <<= 1) {
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const uint32_t y = __shfl_up_sync(kFullMask, v[a], d);
          if (lane >= head + d) v[a] += y;
        }
      }
      const bool tail = lane == 31u || ((heads >> (lane + 1u)) & 1u) != 0u;
      if (off[g] != 0xffffffffu && tail) {
        const uint32_t o = off[g];
        atomicOr(&bits[o >> 5], 1u << (o & 31u));
        atomicAdd(&sm.cnt[o], v[0]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const uint32_t old = atomicAdd(&sm.lo[a][o], v[a + 1]);
          if (old + v[a + 1] < old) atomicAdd(&sm.hi[o], 1ull << (21 * a));
        }
      }
    }
  }
}

// Warp 0: occupied keys before every word of the bitmap (wrank) and their total.
__device__ __forceinline__ uint32_t frame_rank_words(FrSmem& sm, const uint32_t* bits, int nw) {
  const int lane = threadIdx.x & 31;
  uint32_t pc[4], mine = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int w = 4 * lane + q;
    pc[q] = w < nw ? __popc(bits[w]) : 0u;
    mine += pc[q];
  }
  uint32_t inc = mine;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(kFullMask, inc, off);
    if (lane >= off) inc += y;
  }
  uint32_t run = inc - mine;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int w = 4 * lane + q;
    if (w < nw) sm.wrank[w] = static_cast<uint16_t>(run);
    run += pc[q];
  }
  return __shfl_sync(kFullMask, inc, 31);
}

// One thread per key of the bin: the occupied keys' rows from row0 on (the bin's key
// order), counters and sums cleared behind.
__device__ __forceinline__ void frame_rows(FrSmem& sm, const uint32_t* bits, uint32_t span,
                                           uint32_t key0, uint32_t row0, const RowCtx& rc,
                                           const SegOut& out, int* err) {
#pragma unroll 1
  for (int q = 0; q < kFrPer; ++q) {
    const uint32_t off = uint32_t(q) * kFrThreads + threadIdx.x;
    if (off >= span) break;
    const uint32_t n = sm.cnt[off];
    if (n == 0) continue;
    const uint32_t w = off >> 5;
    const uint32_t r = uint32_t(sm.wrank[w]) + __popc(bits[w] & ((1u << (off & 31u)) - 1u));
    float sf[3];
    long long s64[3];
    const unsigned long long carries = sm.hi[off];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const unsigned long long b = (((carries >> (21 * a)) & 0x1fffffull) << 32) | sm.lo[a][off];
      s64[a] = static_cast<long long>(b) + static_cast<long long>(n) * kQMin;
      sf[a] = __ll2float_rn(s64[a]);
      sm.lo[a][off] = 0;
    }
    sm.hi[off] = 0;
    sm.cnt[off] = 0;
    put_row32(rc, out, row0 + r, key0 + off, n, sf, s64, err);
  }
}

// Publishes unit u's cells (v) in the chained scan and returns the unit's first row; the
// last unit also writes the voxel count (and the one frame's end).
__device__ __forceinline__ uint32_t frame_unit_prefix(uint32_t* status, uint32_t u,
                                                      uint32_t units, uint32_t v,
                                                      const SegOut& out, uint32_t spin_limit,
                                                      int* err) {
  uint32_t excl = 0;
  if (u == 0) {
    st_relaxed(status, kFlagPrefix | v);
  } else {
    st_relaxed(status + u, kFlagAggregate | v);
    excl = lookback_u32(status, 1, int(u), spin_limit, err);
    st_relaxed(status + u, kFlagPrefix | ((excl + v) & kValueMask));
  }
  if (u == 0 && out.frame_offsets) out.frame_offsets[0] = 0;
  if (u == units - 1) {
    *out.num_voxels = excl + v;
    if (out.frame_offsets) out.frame_offsets[1] = excl + v;
  }
  return excl;
}

// Units of 2^(ftop - u) consecutive bins (2^u units, u = min(ftop, 12)) in ticket order.
// A unit's cells are known (the counting kernel) when it is taken, so it joins the chained
// scan at once and no unit waits on another's reduction.  Invariant at the start of every
// bin: bits[jb] is clear, counters and sums are zero.
__global__ __launch_bounds__(kFrThreads) void frame_bin_kernel(
    State* st, const FrameState* __restrict__ fs, const uint32_t* __restrict__ keys,
    const uint4* __restrict__ runs, const uint32_t* __restrict__ hist,
    const uint32_t* __restrict__ start, const uint32_t* __restrict__ cells, uint32_t* status,
    uint32_t* ticket, SegOut out, uint32_t spin_limit, int* err) {
  extern __shared__ __align__(16) unsigned char fr_smem[];
  FrSmem& sm = *reinterpret_cast<FrSmem*>(fr_smem);
  if (block_error_raised(err)) return;
  const int t = threadIdx.x;
  const uint32_t span_bits = st->fspan, top = st->ftop;
  const uint32_t span = 1u << span_bits, mask = span - 1u;
  const int nw = int((span + 31u) >> 5);
  const uint32_t ubits = top < uint32_t(kFrMaxUnitBits) ? top : uint32_t(kFrMaxUnitBits);
  const uint32_t units = 1u << ubits, per = 1u << (top - ubits);
  RowCtx rc;
  rc.fs = fs;
  rc.key_shift = st->key_shift;
  rc.o1[0] = fs[0].origin[0];
  rc.o1[1] = fs[0].origin[1];
  rc.o1[2] = fs[0].origin[2];
  rc.leaf1 = fs[0].leaf;
  for (uint32_t i = t; i < kFrSpan; i += kFrThreads) {
    sm.cnt[i] = 0;
    sm.hi[i] = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) sm.lo[a][i] = 0;
  }
  for (int w = t; w < 2 * kFrWords; w += kFrThreads) sm.bits[w / kFrWords][w % kFrWords] = 0;
  int jb = 0;
  for (;;) {
    if (t < 32) {
      uint32_t u = 0;
      if (t == 0) u = atomicAdd(ticket, 1u);
      u = __shfl_sync(kFullMask, u, 0);
      if (u < units) {  // the unit's cells, then its place in the chained scan
        uint32_t v = 0;
        for (uint32_t b = u * per + uint32_t(t); b < (u + 1) * per; b += 32) v += __ldg(cells + b);
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
        if (t == 0) sm.s_excl = frame_unit_prefix(status, u, units, v, out, spin_limit, err);
      }
      if (t == 0) sm.s_unit = static_cast<int>(u);
    }
    __syncthreads();
    const uint32_t u = static_cast<uint32_t>(sm.s_unit);
    if (u >= units) break;
    uint32_t row = sm.s_excl;
    for (uint32_t b = u * per; b < (u + 1) * per; ++b) {
      const uint32_t m = __ldg(hist + b);
      if (m == 0) continue;
      uint32_t* bits = sm.bits[jb];
      frame_accumulate(sm, bits, keys, runs, __ldg(start + b), m, mask);
      for (int w = t; w < kFrWords; w += kFrThreads) sm.bits[jb ^ 1][w] = 0;  // last bin's
      __syncthreads();
      if (t < 32) (void)frame_rank_words(sm, bits, nw);
      __syncthreads();
      frame_rows(sm, bits, span, b << span_bits, row, rc, out, err);
      row += __ldg(cells + b);
      jb ^= 1;
      __syncthreads();  // counters and sums cleared, the ranks read
    }
    __syncthreads();  // every thread has read the unit before warp 0 takes the next
  }
}

// ---- the whole frame in one launch --------------------------------------------------------
// A cooperative grid (every block resident, one a SM) takes the frame in phases separated
// by grid barriers, each point held by one thread (point (s G' + w) 32 + lane for step s,
// w = the warp's index in the grid, G' = the grid's warps, so a warp holds 32 consecutive
// points a step):
//   0  extents (the origin kernel's minima and maxima); the key bitmap's first
//      kFzZeroWords words cleared (the rest, for wider keys, once the extents give the
//      width);
//   1  key and corner offsets of every point; runs of equal keys among a warp's 32 points
//      kept in shared memory; one bit a run in the key bitmap (one atomic a bitmap word of
//      the warp's step) -- or, for keys of more than kFzDenseBits bits, in a bitmap of
//      blocks of 2^kFzBlockBits keys, whose set bits are ranked into slots before each run
//      sets its key's bit in its slot's 16-word bitmap;
//   2  the bitmap's set bits ranked in word order (counts per block, a barrier, every
//      block's predecessors summed at once): an occupied key's row is its rank, so rows
//      come out in key order; the rows' sums cleared;
//   3  every run adds its points and offset sums at its row (two global atomics and a
//      rare carry) and stores the row's key;
//   4  one thread a row: the centroid (put_row32: the other groupings' formula and integer
//      sums, so the rows are bit-identical to theirs).
// Every wait is bounded (kErrTimeout after the limit), every index read back from scratch
// is checked against its buffer, and every block passes every barrier, so an error never
// leaves a block waiting on another.
struct FzArgs {
  const float* xyz;
  FramesArg fr;
  State* st;
  FrameState* fs;
  uint32_t* bits;      // kFzDenseWords words
  uint32_t* rank;      // kFzDenseWords words
  uint32_t* slotmap;   // 2^(32 - kFzBlockBits) words
  uint32_t* slotbin;   // rows_cap words
  uint32_t* sbits;     // 16 rows_cap words
  uint32_t* srank;     // 16 rows_cap words
  unsigned long long* acc;  // 3 arrays of rows_cap: A, B and C of every row (see below)
  uint32_t* rowkey;    // rows_cap words
  uint32_t* stat;      // 2 kFzMaxGrid words
  SegOut out;
  int64_t rows_cap;    // the frame's points (bounds slots and rows)
  int per;             // points a thread
  uint32_t spin_limit;
  int* err;
};

// A cell's three sums and points in two words and a carry word: A = x + y 2^32 and
// B = z + points 2^32 (mod 2^64), C = the carries out of A's and B's low halves and out of
// A, 21 bits each.  A frame of at most 2^21 points keeps every sum below 2^42, so each
// carry count below 2^10.
static_assert(kFzMaxPointsBits + 21 <= 42 && 42 - 32 < 21, "carry counts fit their fields");

// Grid barrier on an arrival counter the call zeroes; `target` (thread 0's) grows by the
// grid each barrier.  The wait is bounded.
__device__ __forceinline__ void fz_grid_sync(uint32_t* ctr, uint32_t& target, uint32_t spin,
                                             int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    target += gridDim.x;
    __threadfence();
    atomicAdd(ctr, 1u);
    uint32_t spins = 0;
    while (ld_acquire(ctr) < target) {
      if (++spins > spin) {
        set_error(err, kErrTimeout);
        break;
      }
      if (spins > 16) __nanosleep(32);
    }
    __threadfence();
  }
  __syncthreads();
}

// Ranking the set bits of words [0, nw) in word order takes two steps around a grid
// barrier: block b takes a contiguous slice of the words and publishes the slice's set
// bits in agg[b]; after the barrier every block sums its predecessors' totals (all at
// once, one per thread) for its slice's first rank, and ranks the slice tile by tile
// (thread t: word t of a tile of kFzThreads consecutive words), so that the 32 words of a
// warp are consecutive and so are their ranks.
__device__ __forceinline__ void fz_slice(uint32_t nw, uint32_t* s0, uint32_t* s1) {
  const uint32_t q = (nw + gridDim.x - 1u) / gridDim.x;
  *s0 = min(nw, blockIdx.x * q);
  *s1 = min(nw, *s0 + q);
}

// Step one: agg[blockIdx.x] = set bits of the block's slice.  Contains __syncthreads.
__device__ __forceinline__ void fz_count(const uint32_t* w, uint32_t nw, uint32_t* agg,
                                         uint32_t* tmp) {
  uint32_t s0, s1;
  fz_slice(nw, &s0, &s1);
  uint32_t mine = 0;
  for (uint32_t i = s0 + threadIdx.x; i < s1; i += kFzThreads) mine += __popc(__ldcg(w + i));
  uint32_t total;
  (void)block_excl_scan(mine, &total, tmp);
  if (threadIdx.x == 0) agg[blockIdx.x] = total;
}

// Lane-parallel walk over the set bits of a warp's 32 consecutive words: lane i holds word
// index wi, bits vi and ri = the rank of its first set bit, the ranks consecutive across
// the lanes (r[i+1] = r[i] + popc(v[i])).  The bits are taken 32 at a time, lane l the
// (j + l)-th: its word is the last lane whose first rank is at most that (a binary search
// over the lanes), its position the matching set bit of that word; f(word, position, rank)
// then runs with consecutive ranks across the lanes, so row writes coalesce.
template <typename F>
__device__ __forceinline__ void warp_expand(uint32_t wi, uint32_t vi, uint32_t ri, F f) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t r0 = __shfl_sync(kFullMask, ri, 0);
  const uint32_t e = ri - r0;
  const uint32_t total = __shfl_sync(kFullMask, e + __popc(vi), 31);
  for (uint32_t j = 0; j < total; j += 32) {
    const uint32_t b = j + lane;
    uint32_t lo = 0;
#pragma unroll
    for (uint32_t step = 16; step; step >>= 1) {
      const uint32_t ec = __shfl_sync(kFullMask, e, lo + step);
      if (ec <= b) lo += step;
    }
    const uint32_t eo = __shfl_sync(kFullMask, e, lo);
    const uint32_t vo = __shfl_sync(kFullMask, vi, lo);
    const uint32_t wo = __shfl_sync(kFullMask, wi, lo);
    if (b < total) f(wo, __fns(vo, 0u, int(b - eo + 1u)), r0 + b);
  }
}

struct FzNoBits {
  __device__ void operator()(uint32_t, uint32_t, uint32_t) const {}
};

// Step two (after a grid barrier): rk[i] = set bits before word i for the block's slice;
// with kExpand, f(word, position, rank) for every set bit (warp_expand).  Returns the grand
// total (in every block).  The grid has at most kFzThreads blocks.  Contains
// __syncthreads.
template <bool kExpand, typename F>
__device__ __forceinline__ uint32_t fz_rank(const uint32_t* w, uint32_t* rk, uint32_t nw,
                                            const uint32_t* agg, uint32_t* tmp,
                                            uint32_t* s_first, F f) {
  uint32_t s0, s1;
  fz_slice(nw, &s0, &s1);
  const uint32_t g = threadIdx.x < gridDim.x ? __ldcg(agg + threadIdx.x) : 0u;
  uint32_t all;
  const uint32_t pre = block_excl_scan(g, &all, tmp);
  if (threadIdx.x == blockIdx.x) *s_first = pre;  // the blocks before this one
  __syncthreads();
  uint32_t base = *s_first;
  for (uint32_t t0 = s0; t0 < s1; t0 += kFzThreads) {  // (the same trips in every thread)
    const uint32_t i = t0 + threadIdx.x;
    const uint32_t v = i < s1 ? __ldcg(w + i) : 0u;
    uint32_t tot;
    const uint32_t r = base + block_excl_scan(__popc(v), &tot, tmp);
    if (i < s1) rk[i] = r;
    if (kExpand) warp_expand(i, v, r, f);
    base += tot;
  }
  return all;
}

template <bool kPosed>
__global__ __launch_bounds__(kFzThreads, 1) void frame_fused_kernel(const FzArgs a) {
  extern __shared__ uint4 fz_runs[];  // [per][kFzThreads]: key, x, y, z | points << 26
  __shared__ float red[kFzThreads / 32][6];
  __shared__ uint32_t tmp[kFzThreads / 32];
  __shared__ uint32_t s_excl;
  __shared__ float s_o[3], s_leaf, s_rleaf, s_inv;
  __shared__ uint32_t s_kb;
  __shared__ int s_go;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t gthreads = gridDim.x * kFzThreads;
  const int64_t n = a.fr.n;
  const int64_t gwarps = int64_t(gridDim.x) * (kFzThreads / 32);
  const int64_t gw = int64_t(blockIdx.x) * (kFzThreads / 32) + warp;
  int* err = a.err;
  uint32_t target = 0;

  // The call clears the error word here, before the first barrier (no step records an
  // error before it).  One frame: offsets, when given, must be {0, n}.
  if (blockIdx.x == 0 && threadIdx.x == 0) *err = 0;
  const bool bad_offsets =
      a.fr.offsets && (__ldg(a.fr.offsets) != 0 || __ldg(a.fr.offsets + 1) != n);
  Pose P;
  if (kPosed) load_pose(a.fr, 0, P);

  // ---- phase 0: extents; the bitmap's first kFzZeroWords words cleared ----
  for (uint32_t i = blockIdx.x * kFzThreads + threadIdx.x; i < kFzZeroWords / 4; i += gthreads)
    reinterpret_cast<uint4*>(a.bits)[i] = make_uint4(0u, 0u, 0u, 0u);
  {
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll 2
    for (int s = 0; s < (bad_offsets ? 0 : a.per); ++s) {
      const int64_t p = (int64_t(s) * gwarps + gw) * 32 + lane;
      if (p >= n) continue;
      float x = __ldg(a.xyz + 3 * p), y = __ldg(a.xyz + 3 * p + 1), z = __ldg(a.xyz + 3 * p + 2);
      if (kPosed) pose_point(P, x, y, z);
      if (point_valid(x, y, z)) {
        mn[0] = fminf(mn[0], x), mx[0] = fmaxf(mx[0], x);
        mn[1] = fminf(mn[1], y), mx[1] = fmaxf(mx[1], y);
        mn[2] = fminf(mn[2], z), mx[2] = fmaxf(mx[2], z);
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
      for (int off = 16; off; off >>= 1) {
        mn[c] = fminf(mn[c], __shfl_xor_sync(kFullMask, mn[c], off));
        mx[c] = fmaxf(mx[c], __shfl_xor_sync(kFullMask, mx[c], off));
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        red[warp][c] = mn[c];
        red[warp][3 + c] = mx[c];
      }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      const int c = threadIdx.x;
      float m = INFINITY, M = -INFINITY;
      for (int w = 0; w < kFzThreads / 32; ++w) {
        m = fminf(m, red[w][c]);
        M = fmaxf(M, red[w][3 + c]);
      }
      if (m != INFINITY) {
        atomicMax(&a.fs[0].ord_min_inv[c], ~float_to_ordered(m));
        atomicMax(&a.fs[0].ord_max[c], float_to_ordered(M));
      }
    }
  }
  fz_grid_sync(&a.st->fz_bar, target, a.spin_limit, err);
  if (bad_offsets) {  // (uniform: every block read the same offsets)
    if (blockIdx.x == 0 && threadIdx.x == 0) set_error(err, kErrInvalidArg);
    return;
  }

  // ---- the frame's origin, leaf and key width (the same in every block) ----
  if (threadIdx.x == 0) {
    const float leaf = a.fr.leaves ? __ldg(a.fr.leaves) : a.fr.leaf;
    const bool bad_leaf = !(leaf > 0.0f) || !isfinite(leaf);
    const bool any = __ldcg(&a.fs[0].ord_min_inv[0]) != 0u;
    float o[3];
    for (int c = 0; c < 3; ++c) {
      if (a.fr.origin_in) {
        o[c] = __ldg(a.fr.origin_in + c);
      } else {
        const uint32_t u = __ldcg(&a.fs[0].ord_min_inv[c]);
        o[c] = u == 0u ? 0.0f : ordered_to_float(~u);
      }
      s_o[c] = o[c];
    }
    uint64_t kbound = 0;
    if (any && !bad_leaf) {
      uint32_t ii[3];
      bool ok = true;
      for (int c = 0; c < 3; ++c)
        ok = ok && axis_index(ordered_to_float(__ldcg(&a.fs[0].ord_max[c])), o[c], leaf, &ii[c]);
      kbound = ok ? morton3(ii[0], ii[1], ii[2]) : ~0ull >> 1;
    }
    const uint32_t kb = kbound ? 64u - __clzll(static_cast<long long>(kbound)) : 0u;
    const bool narrow = kb <= 32u && kbound < 0xffffffffull;
    s_leaf = leaf;
    s_rleaf = fast_leaf(leaf) ? __fdiv_rn(1.0f, leaf) : 0.0f;
    s_inv = quant_inv_unit(leaf);
    s_kb = kb;
    s_go = !bad_leaf && narrow;
    if (blockIdx.x == 0) {
      for (int c = 0; c < 3; ++c) {
        a.fs[0].origin[c] = o[c];
        if (!a.fr.origin_in && a.fr.origin_out) a.fr.origin_out[c] = o[c];
      }
      a.fs[0].leaf = leaf;
      a.st->key_shift = 64;
      a.st->nframes = 1;
      a.st->narrow = narrow ? 1u : 0u;
      a.st->maxkey = kbound;
      if (bad_leaf) set_error(err, kErrInvalidArg);
      else if (!narrow) set_error(err, kErrRange);  // keys of more than 32 bits
      if (bad_leaf || !narrow) {
        *a.out.num_voxels = 0;
        if (a.out.frame_offsets) a.out.frame_offsets[0] = a.out.frame_offsets[1] = 0;
      }
    }
  }
  __syncthreads();
  if (!s_go) return;  // (uniform across the grid)
  const uint32_t kb = s_kb;
  const bool dense = kb <= uint32_t(kFzDenseBits);
  const float o[3] = {s_o[0], s_o[1], s_o[2]};
  const float leaf = s_leaf, rleaf = s_rleaf, inv_unit = s_inv;
  if (dense && kb > uint32_t(kFzZeroBits)) {  // the rest of a wider key bitmap (uniform)
    const uint32_t end = (1u << (kb - 5u)) / 4u;
    for (uint32_t i = uint32_t(kFzZeroWords / 4) + blockIdx.x * kFzThreads + threadIdx.x; i < end;
         i += gthreads)
      reinterpret_cast<uint4*>(a.bits)[i] = make_uint4(0u, 0u, 0u, 0u);
    fz_grid_sync(&a.st->fz_bar, target, a.spin_limit, err);
  }

  // ---- phase 1: keys, runs, bitmap ----
  {
    bool range_bad = false;
    float nx[3];  // the next point's coordinates, loaded one step ahead
    {
      const int64_t p = gw * 32 + lane;
      const bool in = p < n;
      nx[0] = in ? __ldg(a.xyz + 3 * p) : __int_as_float(0x7fc00000);
      nx[1] = in ? __ldg(a.xyz + 3 * p + 1) : nx[0];
      nx[2] = in ? __ldg(a.xyz + 3 * p + 2) : nx[0];
    }
    for (int s = 0; s < a.per; ++s) {
      float x = nx[0], y = nx[1], z = nx[2];
      if (s + 1 < a.per) {
        const int64_t p = (int64_t(s + 1) * gwarps + gw) * 32 + lane;
        const bool in = p < n;
        nx[0] = in ? __ldg(a.xyz + 3 * p) : __int_as_float(0x7fc00000);
        nx[1] = in ? __ldg(a.xyz + 3 * p + 1) : nx[0];
        nx[2] = in ? __ldg(a.xyz + 3 * p + 2) : nx[0];
      }
      if (kPosed) pose_point(P, x, y, z);
      uint32_t k = kFullMask;
      uint64_t pw = 0;
      const bool ok = narrow_entry(x, y, z, o, leaf, rleaf, inv_unit, 0u, 64u, &k, &pw,
                                   &range_bad);
      if (!ok) k = kFullMask;
      uint32_t v[4];
      const bool emit = warp_run(k, pw, ok, v);
      fz_runs[s * kFzThreads + threadIdx.x] =
          emit ? make_uint4(k, v[0], v[1], v[2] | (v[3] << 26)) : make_uint4(kFullMask, 0u, 0u, 0u);
      // one atomic a bitmap word among the warp's runs
      const uint32_t em = __ballot_sync(kFullMask, emit);
      if (emit) {
        const uint32_t word = dense ? (k >> 5) : (k >> (kFzBlockBits + 5));
        const uint32_t bit = 1u << (dense ? (k & 31u) : ((k >> kFzBlockBits) & 31u));
        const uint32_t peers = __match_any_sync(em, word);
        const uint32_t orv = __reduce_or_sync(peers, bit);
        if (int(lane) == __ffs(peers) - 1) atomicOr(a.bits + word, orv);
      }
    }
    if (__any_sync(kFullMask, range_bad) && lane == 0) set_error(err, kErrRange);
  }
  fz_grid_sync(&a.st->fz_bar, target, a.spin_limit, err);

  uint32_t* wbits = a.bits;
  uint32_t* wrank = a.rank;
  uint32_t nw = kb > 5u ? 1u << (kb - 5u) : 1u;
  uint32_t nslots = 0;
  if (!dense) {
    // ---- phase 1b: occupied blocks numbered (slots); their bitmaps cleared ----
    const uint32_t nw1 = kb > uint32_t(kFzBlockBits + 5) ? 1u << (kb - kFzBlockBits - 5u) : 1u;
    fz_count(a.bits, nw1, a.stat, tmp);
    fz_grid_sync(&a.st->fz_bar, target, a.spin_limit, err);
    uint32_t* slotmap = a.slotmap;
    uint32_t* slotbin = a.slotbin;
    const int64_t cap = a.rows_cap;
    const uint32_t slots = fz_rank<true>(
        a.bits, a.rank, nw1, a.stat, tmp, &s_excl,
        [&](uint32_t i, uint32_t bit, uint32_t slot) {
          if (slot >= cap) return;  // (more slots than points: reported below)
          const uint32_t blk = (i << 5) | bit;
          slotmap[blk] = slot;
          slotbin[slot] = blk;
        });
    nslots = static_cast<uint32_t>(min(int64_t(slots), a.rows_cap));
    if (slots > nslots && blockIdx.x == 0 && threadIdx.x == 0) set_error(err, kErrInvalidArg);
    for (uint32_t i = blockIdx.x * kFzThreads + threadIdx.x; i < nslots * 4u; i += gthreads)
      reinterpret_cast<uint4*>(a.sbits)[i] = make_uint4(0u, 0u, 0u, 0u);
    fz_grid_sync(&a.st->fz_bar, target, a.spin_limit, err);
    // ---- phase 1c: every run's bit in its slot's bitmap ----
    for (int s = 0; s < a.per; ++s) {
      const uint4 r = fz_runs[s * kFzThreads + threadIdx.x];
      const bool emit = r.x != kFullMask;
      const uint32_t em = __ballot_sync(kFullMask, emit);
      if (emit) {
        const uint32_t slot = __ldcg(a.slotmap + (r.x >> kFzBlockBits));
        const bool good = slot < nslots;
        const uint32_t word = good ? slot * 16u + ((r.x >> 5) & 15u) : ~0u;
        const uint32_t peers = __match_any_sync(em, word);
        const uint32_t orv = __reduce_or_sync(peers, 1u << (r.x & 31u));
        if (!good) set_error(err, kErrInvalidArg);
        else if (int(lane) == __ffs(peers) - 1) atomicOr(a.sbits + word, orv);
      }
    }
    fz_grid_sync(&a.st->fz_bar, target, a.spin_limit, err);
    wbits = a.sbits;
    wrank = a.srank;
    nw = nslots * 16u;
  }

  // ---- phase 2: rows in key order (the rank of each occupied key's bit); sums cleared ----
  fz_count(wbits, nw, a.stat + kFzMaxGrid, tmp);
  fz_grid_sync(&a.st->fz_bar, target, a.spin_limit, err);
  const uint32_t rows_all =
      fz_rank<false>(wbits, wrank, nw, a.stat + kFzMaxGrid, tmp, &s_excl, FzNoBits());
  const uint32_t rows = static_cast<uint32_t>(min(int64_t(rows_all), a.rows_cap));
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (rows_all > rows) set_error(err, kErrInvalidArg);
    // more cells than output rows: the first out.cap rows are written (phase 4 writes only
    // those), so the shortfall is recorded once, here, for every block to see alike
    if (int64_t(rows_all) > a.out.cap) set_error(err, kErrCapacity);
    a.st->fz_rows = rows_all;
    *a.out.num_voxels = rows_all;
    if (a.out.frame_offsets) {
      a.out.frame_offsets[0] = 0;
      a.out.frame_offsets[1] = rows_all;
    }
  }
  for (uint32_t i = blockIdx.x * kFzThreads + threadIdx.x; i < rows; i += gthreads) {
    a.acc[i] = 0ull;
    a.acc[i + a.rows_cap] = 0ull;
    a.acc[i + 2 * a.rows_cap] = 0ull;
  }
  fz_grid_sync(&a.st->fz_bar, target, a.spin_limit, err);

  // ---- phase 3: every run's points and sums at its row ----
  {
    // the rows of all the thread's runs first (their loads in flight together), then the
    // atomics
    uint32_t rw[kFzPer];
#pragma unroll
    for (int s = 0; s < kFzPer; ++s) {
      rw[s] = ~0u;
      if (s < a.per) {
        const uint32_t k = fz_runs[s * kFzThreads + threadIdx.x].x;
        if (k != kFullMask) {
          uint32_t word;
          if (dense) {
            word = k >> 5;
          } else {
            const uint32_t slot = __ldcg(a.slotmap + (k >> kFzBlockBits));
            word = slot < nslots ? slot * 16u + ((k >> 5) & 15u) : ~0u;
          }
          if (word < nw) {
            rw[s] = __ldcg(wrank + word) + __popc(__ldcg(wbits + word) & ((1u << (k & 31u)) - 1u));
            if (rw[s] >= rows) rw[s] = ~1u;
          } else {
            rw[s] = ~1u;
          }
        }
      }
    }
    // two atomics a run: A += x | y << 32, B += z | points << 32; the old values they return
    // tell every carry out of a 32-bit half (x into y, A out of 64 bits, z into points),
    // counted in a third word (rare: a cell of more than 2^11 points)
    unsigned long long* accA = a.acc;
    unsigned long long* accB = a.acc + a.rows_cap;
    unsigned long long* accC = a.acc + 2 * a.rows_cap;
#pragma unroll
    for (int s0 = 0; s0 < kFzPer; s0 += 2) {
      unsigned long long oa[2], ob[2], va[2], vb[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int s = s0 + q;
        oa[q] = ob[q] = va[q] = vb[q] = 0ull;
        if (s >= kFzPer || rw[s] >= ~1u) continue;
        const uint4 r = fz_runs[s * kFzThreads + threadIdx.x];
        a.rowkey[rw[s]] = r.x;  // (every run of the row stores the same key)
        va[q] = (unsigned long long)r.y | ((unsigned long long)r.z << 32);
        vb[q] = (unsigned long long)(r.w & 0x3ffffffu) | ((unsigned long long)(r.w >> 26) << 32);
        oa[q] = atomicAdd(accA + rw[s], va[q]);
        ob[q] = atomicAdd(accB + rw[s], vb[q]);
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int s = s0 + q;
        if (s >= kFzPer || rw[s] == ~0u) continue;
        if (rw[s] == ~1u) {
          set_error(err, kErrInvalidArg);
          continue;
        }
        const unsigned long long cx = ((oa[q] & 0xffffffffull) + (va[q] & 0xffffffffull)) >> 32;
        const unsigned long long cy = oa[q] + va[q] < oa[q] ? 1ull : 0ull;
        const unsigned long long cz = ((ob[q] & 0xffffffffull) + (vb[q] & 0xffffffffull)) >> 32;
        if (cx | cy | cz) atomicAdd(accC + rw[s], cx | (cy << 21) | (cz << 42));
      }
    }
  }
  fz_grid_sync(&a.st->fz_bar, target, a.spin_limit, err);

  // ---- phase 4: rows (a thread a row), the first out.cap of them ----
  // (every error but the capacity one stops it; none is set from here on)
  if (__syncthreads_or(threadIdx.x == 0 && error_raised(err) &&
                       *reinterpret_cast<const volatile int*>(err) != kErrCapacity))
    return;
  const uint32_t wrows = static_cast<uint32_t>(min(int64_t(rows), a.out.cap));
  RowCtx rc;
  rc.fs = a.fs;
  rc.key_shift = 64;
  rc.o1[0] = o[0];
  rc.o1[1] = o[1];
  rc.o1[2] = o[2];
  rc.leaf1 = leaf;
  for (uint32_t row = blockIdx.x * kFzThreads + threadIdx.x; row < wrows; row += gthreads) {
    const unsigned long long* ap = a.acc + row;
    const unsigned long long A = __ldcg(ap), B = __ldcg(ap + a.rows_cap),
                             C = __ldcg(ap + 2 * a.rows_cap);
    const unsigned long long cx = C & 0x1fffffull, cy = (C >> 21) & 0x1fffffull, cz = C >> 42;
    // x = low(A) + cx 2^32; y = high(A) + cy 2^32 - cx; z = low(B) + cz 2^32;
    // points = high(B) - cz
    const unsigned long long sb[3] = {(A & 0xffffffffull) + (cx << 32),
                                      (A >> 32) + (cy << 32) - cx,
                                      (B & 0xffffffffull) + (cz << 32)};
    const uint32_t cnt = static_cast<uint32_t>((B >> 32) - cz);
    float sf[3];
    long long s64[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      s64[c] = static_cast<long long>(sb[c]) + static_cast<long long>(cnt) * kQMin;
      sf[c] = __ll2float_rn(s64[c]);
    }
    put_row32(rc, a.out, row, __ldcg(a.rowkey + row), cnt, sf, s64, err);
  }
}

// The only state the one-launch kernel reads before writing it: the barrier's arrival
// counter and the frame's extent words (atomic maxima).  A one-thread-block kernel costs the
// stream less than a memset of the state.
__global__ void fz_clear_kernel(State* st, FrameState* fs) {
  if (threadIdx.x == 0) st->fz_bar = 0u;
  if (threadIdx.x < 3) {
    fs[0].ord_min_inv[threadIdx.x] = 0u;
    fs[0].ord_max[threadIdx.x] = 0u;
  }
}

// Test of the grid barrier's bounded wait: the target counts one arrival more than the grid
// makes, so every block's wait runs out after `limit` polls and records kErrTimeout.
__global__ void debug_grid_barrier_kernel(uint32_t* ctr, uint32_t limit, int* err) {
  uint32_t target = 1;
  fz_grid_sync(ctr, target, limit, err);
}

constexpr size_t kFzSmem = size_t(kFzPer) * kFzThreads * sizeof(uint4);
static_assert(kFzSmem + 2048 <= 227 * 1024, "one-launch block shared memory");

constexpr size_t kFrSmem = sizeof(FrSmem);
static_assert(kFrSmem + 1024 <= 227 * 1024, "bin block shared memory");

}  // namespace

namespace {
// Blocks of the one-launch kernel resident on an SM (0: it cannot run), per device.
int fused_blocks_per_sm(bool posed) {
  static int cache[64][2];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  int& b = cache[dev][posed ? 1 : 0];
  if (b == 0) {
    const void* fn = posed ? reinterpret_cast<const void*>(frame_fused_kernel<true>)
                           : reinterpret_cast<const void*>(frame_fused_kernel<false>);
    int v = 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kFzSmem)) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, fn, kFzThreads, kFzSmem) != cudaSuccess)
      v = 0;
    (void)cudaGetLastError();
    b = v > 0 ? v : -1;
  }
  return b > 0 ? b : 0;
}

int fused_grid(bool posed) {
  const int64_t g = int64_t(fused_blocks_per_sm(posed)) * num_sms();
  return static_cast<int>(g < kFzMaxGrid ? g : kFzMaxGrid);
}
}  // namespace

void warm_frame_config() {
  persistent_grid(reinterpret_cast<const void*>(frame_bin_kernel), kFrThreads, kFrSmem, 1);
  (void)fused_blocks_per_sm(false);
  (void)fused_blocks_per_sm(true);
}

int64_t frame_fused_max_points(bool posed) {
  // (and at most 2^21 points, so a cell's carry counts fit their fields)
  const int64_t g = int64_t(fused_grid(posed)) * kFzThreads * kFzPer;
  return g < (int64_t(1) << kFzMaxPointsBits) ? g : (int64_t(1) << kFzMaxPointsBits);
}

bool frame_fused_fits(int64_t n, bool posed) {
  return n > 0 && n <= frame_fused_max_points(posed);
}

cudaError_t launch_debug_grid_barrier(uint32_t* ctr, uint32_t limit, int* err,
                                      cudaStream_t stream) {
  void* args[] = {&ctr, &limit, &err};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(debug_grid_barrier_kernel),
                                     dim3(2), dim3(32), args, 0, stream);
}

cudaError_t launch_frame_fused(const float* xyz, const FramesArg& fr, State* st, FrameState* fs,
                               char* ws, const FusedLayout& ZL, const SegOut& out,
                               uint32_t spin_limit, int* err, cudaStream_t stream) {
  const bool ps = posed(fr);
  const int g = fused_grid(ps);
  if (g <= 0) return cudaErrorInvalidConfiguration;
  const int64_t per = ceil_div(fr.n, int64_t(g) * kFzThreads);
  if (per > kFzPer) return cudaErrorInvalidValue;
  FzArgs a;
  a.xyz = xyz;
  a.fr = fr;
  a.st = st;
  a.fs = fs;
  a.bits = reinterpret_cast<uint32_t*>(ws + ZL.bits);
  a.rank = reinterpret_cast<uint32_t*>(ws + ZL.rank);
  a.slotmap = reinterpret_cast<uint32_t*>(ws + ZL.slotmap);
  a.slotbin = reinterpret_cast<uint32_t*>(ws + ZL.slotbin);
  a.sbits = reinterpret_cast<uint32_t*>(ws + ZL.sbits);
  a.srank = reinterpret_cast<uint32_t*>(ws + ZL.srank);
  a.acc = reinterpret_cast<unsigned long long*>(ws + ZL.acc);
  a.rowkey = reinterpret_cast<uint32_t*>(ws + ZL.rowkey);
  a.stat = reinterpret_cast<uint32_t*>(ws + ZL.stat);
  a.out = out;
  a.rows_cap = fr.n;
  a.per = static_cast<int>(per);
  a.spin_limit = spin_limit;
  a.err = err;
  fz_clear_kernel<<<1, 32, 0, stream>>>(st, fs);
  void* args[] = {&a};
  const void* fn = ps ? reinterpret_cast<const void*>(frame_fused_kernel<true>)
                      : reinterpret_cast<const void*>(frame_fused_kernel<false>);
  // shared memory for the runs of the points a thread holds (the rest stays L1 cache)
  const size_t smem = size_t(per) * kFzThreads * sizeof(uint4);
  return cudaLaunchCooperativeKernel(fn, dim3(g), dim3(kFzThreads), args, smem, stream);
}

cudaError_t launch_frame(const float* xyz, const FramesArg& fr, State* st, FrameState* fs,
                         const NarrowBuffers& nb, char* ws, const FrameLayout& FL,
                         const SegOut& out, uint32_t spin_limit, int* err, cudaStream_t stream) {
  if (fr.n == 0) return cudaSuccess;
  uint32_t* pos = reinterpret_cast<uint32_t*>(ws + FL.pos);
  uint32_t* hist = reinterpret_cast<uint32_t*>(ws + FL.hist);
  uint32_t* ustat = reinterpret_cast<uint32_t*>(ws + FL.ustat);
  uint32_t* pstat = reinterpret_cast<uint32_t*>(ws + FL.pstat);
  uint32_t* tick = reinterpret_cast<uint32_t*>(ws + FL.tick);
  uint32_t* start = reinterpret_cast<uint32_t*>(ws + FL.start);
  uint32_t* cells = reinterpret_cast<uint32_t*>(ws + FL.vcnt);
  uint4* rin = reinterpret_cast<uint4*>(ws + FL.rin);
  uint4* rout = reinterpret_cast<uint4*>(ws + FL.rout);
  if (posed(fr))
    frame_key_kernel<true><<<stream_grid(fr), kStreamThreads, 0, stream>>>(
        xyz, fr, st, fs, nb.k0, rin, pos, hist, err);
  else
    frame_key_kernel<false><<<stream_grid(fr), kStreamThreads, 0, stream>>>(
        xyz, fr, st, fs, nb.k0, rin, pos, hist, err);
  frame_prefix_kernel<<<32, 256, 0, stream>>>(st, hist, start, pstat, tick, spin_limit, err);
  const int64_t want = ceil_div(fr.n, 256);
  const int64_t cap = int64_t(num_sms()) * 8;
  frame_scatter_kernel<<<static_cast<int>(want < cap ? want : cap), 256, 0, stream>>>(
      st, nb.k0, rin, pos, start, nb.k1, rout, fr.n, err);
  frame_count_kernel<<<num_sms() * 8, 256, 0, stream>>>(st, nb.k1, hist, start, cells, err);
  const int gb = persistent_grid(reinterpret_cast<const void*>(frame_bin_kernel), kFrThreads,
                                 kFrSmem, int64_t(1) << kFrMaxUnitBits);
  frame_bin_kernel<<<gb, kFrThreads, kFrSmem, stream>>>(st, fs, nb.k1, rout, hist, start, cells,
                                                        ustat, tick + 1, out, spin_limit, err);
  return cudaGetLastError();
}

}  // namespace vg
