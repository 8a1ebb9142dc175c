// Steps a2-a5 for one camera frame (VG_SORT_FRAME): grouping by bins of 2^12 keys.
//
// arXiv 2102.11084 Sec. II-C filters one camera cloud per call (Table I times that call),
// and a frame's points all fall in a few thousand cells per axis at most, so its 32-bit
// Morton keys split into bins of 2^12 consecutive keys (a 16-cell cube) with at most
// 2^20 bins.  Order inside a bin is the only sorting left, and a bin's cells fit one
// block's shared memory densely (one counter and three sums per key of the bin), so the
// whole grouping is a counting pass, one scatter and one reduction:
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
// Same cells, counts and integer sums as every other grouping: the rows are bit-identical.
// The extent kernel, which runs first, clears the bin counts and status words.
#include <cstddef>

#include "vg_device.cuh"
#include "vg_internal.h"
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
      // runs of equal keys among the warp's 32 consecutive points
      uint32_t v[4] = {uint32_t(pw) & 0x1fffffu, uint32_t(pw >> 21) & 0x1fffffu,
                       uint32_t(pw >> 42) & 0x1fffffu, ok ? 1u : 0u};
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
      const bool emit = ok && (lane == 31u || ((heads >> (lane + 1u)) & 1u) != 0u);
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

constexpr size_t kFrSmem = sizeof(FrSmem);
static_assert(kFrSmem + 1024 <= 227 * 1024, "bin block shared memory");

}  // namespace

void warm_frame_config() {
  persistent_grid(reinterpret_cast<const void*>(frame_bin_kernel), kFrThreads, kFrSmem, 1);
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
