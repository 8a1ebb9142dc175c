// Steps a3-a5 for 32-bit keys (the narrow layout): grouping by buckets.
//
// arXiv 2102.11084 Sec. II-C / Algorithm 1 sorts the (cell, point) table with a radix sort
// so that the points of every cell become contiguous, then keeps one point per cell.  The
// order of the cells is all that the output needs; the order of the points inside a cell
// is irrelevant, because every cell's sum is an exact integer.  So the sort here is a
// most-significant-digit partition, and no pass has to be stable:
//   * the key kernel histograms the first digit of every key (the top bits);
//   * one or two partition passes split the entries by the top <= 16 key bits (the
//     bucket).  Each tile of 4096 entries is ranked by shared-memory atomics (in any
//     order), reserves a run per digit with one global atomic, and writes its runs
//     contiguously (whole sectors).  The second pass splits every run of the first one,
//     with its digit counts from a small histogram pass over the keys alone;
//   * a counting kernel finds every bucket's cells (the population of an occupancy bitmap
//     of its low key bits) and cuts every bucket of more than kBkStage entries into
//     windows of consecutive key ranges of at most kBkStage entries each (a single range
//     of at most 256 keys may hold more: an oversized window);
//   * a one-block plan kernel scans the cell counts into every bucket's first row, writes
//     the frame offsets, and merges runs of small consecutive buckets into jobs of at
//     most kBkStage entries whose keys span at most 2^16;
//   * the bucket kernel runs the jobs, largest kind first, none waiting on another.  A
//     job's entries arrive in shared memory by bulk asynchronous copies, double-buffered
//     (the next job's copy runs while this one is reduced), or, for a window, are gathered
//     by key from its bucket; an occupancy bitmap over the job's key range ranks its cells
//     (prefix popcounts: the cells in key order); a counting sort by rank puts each cell's
//     entries together; one thread per cell sums them into its row.  An oversized window
//     accumulates into one shared-memory slot per key instead.
// Same cells, counts and sums as the global radix sort and its segmented reduction, so
// the rows are bit-identical to theirs.
#include <cstddef>

#include "vg_device.cuh"
#include "vg_internal.h"
#include "vg_rows.cuh"

namespace vg {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ bool msd_on(const State* st) { return st->narrow && st->msd; }

// ---- scan of the first digit ----------------------------------------------------------

// Tables of the first pass's digit runs: start1[d] = first entry of digit d (start1[256] =
// entries), jp[d] = the second pass's first job of digit d (jp[256] = jobs): the run of
// digit d is cut into pieces of at most kPartTile entries.
constexpr int kT1 = 257;

// Second-pass job q: its digit (the largest d with jp[d] <= q: digits without jobs have
// jp[d] == jp[d + 1]), first entry and entries.
__device__ __forceinline__ uint32_t job2_digit(const uint32_t* jp, uint32_t q) {
  int lo = 0, hi = 255;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jp[mid] <= q) lo = mid;
    else hi = mid - 1;
  }
  return uint32_t(lo);
}
__device__ __forceinline__ void job2_range(const uint32_t* start1, const uint32_t* jp, uint32_t q,
                                           uint32_t* d1, uint32_t* base, uint32_t* m) {
  const uint32_t d = job2_digit(jp, q);
  const uint32_t k = q - jp[d];
  *d1 = d;
  *base = start1[d] + k * kPartTile;
  const uint32_t end = start1[d + 1];
  *m = min(uint32_t(kPartTile), end - *base);
}

// One block of 256 threads (thread t = digit t): the first pass's write cursors (each
// digit's first entry) and the two tables above.
__global__ __launch_bounds__(256) void msd_scan1_kernel(State* st, uint32_t* __restrict__ cur1,
                                                        uint32_t* __restrict__ t1, int* err) {
  __shared__ uint32_t tmp[8];
  if (!msd_on(st) || block_error_raised(err)) return;
  const uint32_t t = threadIdx.x;
  const uint32_t c = st->hist[0][t];  // digits at or above 2^b1 count nothing
  const uint32_t nj = (c + kPartTile - 1) / kPartTile;
  uint32_t total_c, total_j;
  const uint32_t start = block_excl_scan(c, &total_c, tmp);
  __syncthreads();
  const uint32_t j0 = block_excl_scan(nj, &total_j, tmp);
  cur1[t] = start;
  t1[t] = start;
  t1[kT1 + t] = j0;
  if (t == 0) {
    t1[256] = total_c;
    t1[kT1 + 256] = total_j;
    // the counts cover exactly the valid points the key kernel counted
    const bool ok = total_c == st->nvalid;
    st->njobs2 = ok ? total_j : 0u;
    if (!ok) set_error(err, kErrInvalidArg);
  }
}

// ---- partition pass ---------------------------------------------------------------------

struct PartSmem {
  uint32_t t1[2 * kT1];  // first-pass run tables (second pass)
  uint32_t cnt[256];
  uint32_t loff[256];
  int32_t gofs[256];  // output position of local slot i of digit d: gofs[d] + i
  uint32_t tmp[kPartThreads / 32];
  uint32_t keys[kPartTile];
  unsigned long long pay[kPartTile];
};

// kLevel 1: tiles of the point-order table (invalid rows, all-ones keys, are dropped), by
// the first digit.  kLevel 2: second-pass jobs, each inside one run of the first pass, by
// the second digit; the run's digit selects 256 of the bucket cursors.  kLevel 3: chunks
// of the buckets of more than kBkStage entries (the counting kernel's list), by coarse key
// range (the top 8 of the bucket's low key bits), into the other buffer; each large
// bucket has its own 256 cursors.  Arguments: (ka, pa) in and (kb, pb) out for levels 1
// and 2; for level 3 (ka, pa) = (k0, p0) and (kb, pb) = (k1, p1), the last pass's output
// being read and the other buffer written.
template <int kLevel>
__global__ __launch_bounds__(kPartThreads, 3) void msd_part_kernel(
    State* st, uint32_t* ka, uint64_t* pa, uint32_t* kb, uint64_t* pb, uint32_t* cursor,
    const uint32_t* __restrict__ t1, int64_t n_max, int* err) {
  __shared__ PartSmem sm;
  if (!msd_on(st) || block_error_raised(err)) return;
  if (kLevel == 2 && st->levels != 2) return;
  if (kLevel == 3 && st->njobs3 == 0) return;
  const int t = threadIdx.x;
  const uint32_t* __restrict__ kin = ka;
  const uint64_t* __restrict__ pin = pa;
  uint32_t* __restrict__ kout = kb;
  uint64_t* __restrict__ pout = pb;
  if (kLevel == 3 && st->levels != 2) {  // one pass: its output is (k1, p1)
    kin = kb;
    pin = pb;
    kout = ka;
    pout = pa;
  }
  if (kLevel == 2) {
    for (int i = t; i < 2 * kT1; i += kPartThreads) sm.t1[i] = t1[i];
    __syncthreads();
  }
  const uint32_t L = st->lowbits;
  const uint32_t kmask = kLevel == 3 ? (1u << L) - 1u : kFull;
  const uint32_t shift =
      kLevel == 1 ? L + st->b2 : (kLevel == 2 ? L : (L > 8 ? L - 8 : 0u));
  const uint32_t mask = kLevel == 1 ? (1u << st->b1) - 1u : 0xffu;
  const uint32_t cap = st->nvalid;  // every position lies below the number of valid points
  const int64_t ntiles = kLevel == 1 ? ceil_div(n_max, kPartTile)
                                     : int64_t(kLevel == 2 ? st->njobs2 : st->njobs3);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int64_t base;
    uint32_t m, cbase = 0;
    if (kLevel == 1) {
      base = tile * kPartTile;
      m = static_cast<uint32_t>(n_max - base < kPartTile ? n_max - base : kPartTile);
    } else if (kLevel == 2) {
      uint32_t d1, b0;
      job2_range(sm.t1, sm.t1 + kT1, uint32_t(tile), &d1, &b0, &m);
      base = b0;
      cbase = 256u + (d1 << 8);
    } else {
      const uint4 j3 = reinterpret_cast<const uint4*>(t1)[tile];
      base = j3.x;
      m = j3.y;
      cbase = j3.z << 8;
    }
    sm.cnt[t] = 0;
    __syncthreads();
    uint32_t k[kPartItems], slot[kPartItems];
    unsigned long long p[kPartItems];  // loaded with the keys: both latencies overlap
#pragma unroll
    for (int j = 0; j < kPartItems; ++j) {
      const uint32_t i = uint32_t(j) * kPartThreads + uint32_t(t);
      k[j] = i < m ? __ldcs(kin + base + i) : kFull;
      p[j] = i < m ? __ldcs(pin + base + i) : 0ull;
    }
#pragma unroll
    for (int j = 0; j < kPartItems; ++j) {
      const uint32_t i = uint32_t(j) * kPartThreads + uint32_t(t);
      const bool ok = i < m && (kLevel != 1 || k[j] != kFull);
      slot[j] = ok ? atomicAdd(&sm.cnt[((k[j] & kmask) >> shift) & mask], 1u) : kFull;
    }
    __syncthreads();
    const uint32_t c = sm.cnt[t];
    uint32_t total;
    const uint32_t lo = block_excl_scan(c, &total, sm.tmp);
    sm.loff[t] = lo;
    if (c) sm.gofs[t] = static_cast<int32_t>(atomicAdd(&cursor[cbase + t], c)) - int32_t(lo);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kPartItems; ++j)
      if (slot[j] != kFull) {
        slot[j] += sm.loff[((k[j] & kmask) >> shift) & mask];
        sm.keys[slot[j]] = k[j];
      }
#pragma unroll
    for (int j = 0; j < kPartItems; ++j)
      if (slot[j] != kFull) sm.pay[slot[j]] = p[j];
    __syncthreads();
    for (uint32_t i = t; i < total; i += kPartThreads) {
      const uint32_t key = sm.keys[i];
      const uint32_t pos =
          static_cast<uint32_t>(sm.gofs[((key & kmask) >> shift) & mask] + int32_t(i));
      if (pos < cap) {
        __stcg(kout + pos, key);
        __stcg(pout + pos, static_cast<uint64_t>(sm.pay[i]));
      }
    }
    __syncthreads();
  }
}

// Second-digit counts of every bucket (two passes only): per second-pass job, a histogram
// of its keys' second digit, added into the bucket counts; also the entries and the
// non-empty buckets of every 1024 consecutive buckets (a job's buckets share its first
// digit, so all of them lie in block d1 / 4).  Jobs run from the last one down, so that
// the keys the second pass reads first are the ones left in L2.
__global__ __launch_bounds__(256) void msd_upsweep_kernel(State* st, const uint32_t* __restrict__ k1,
                                                          const uint32_t* __restrict__ t1,
                                                          uint32_t* hist2, int* err) {
  __shared__ uint32_t h[256];
  __shared__ uint32_t tab[2 * kT1];
  __shared__ uint32_t nzw[8];
  if (!msd_on(st) || st->levels != 2 || block_error_raised(err)) return;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int i = t; i < 2 * kT1; i += 256) tab[i] = t1[i];
  const uint32_t shift = st->lowbits;
  const int64_t nj = st->njobs2;
  for (int64_t jr = blockIdx.x; jr < nj; jr += gridDim.x) {
    const uint32_t j = uint32_t(nj - 1 - jr);
    h[t] = 0;
    __syncthreads();
    uint32_t d1, base, m;
    job2_range(tab, tab + kT1, j, &d1, &base, &m);
    uint32_t k[kPartItems];
#pragma unroll
    for (int q = 0; q < kPartItems; ++q) {
      const uint32_t i = uint32_t(q) * 256u + uint32_t(t);
      k[q] = i < m ? __ldcg(k1 + base + i) : kFull;
    }
#pragma unroll
    for (int q = 0; q < kPartItems; ++q)
      if (uint32_t(q) * 256u + uint32_t(t) < m) atomicAdd(&h[(k[q] >> shift) & 255u], 1u);
    __syncthreads();
    bool became = false;  // this job made bucket (d1, t) non-empty
    if (h[t]) became = atomicAdd(&hist2[(d1 << 8) | uint32_t(t)], h[t]) == 0u;
    const uint32_t nb_w = __popc(__ballot_sync(kFull, became));
    if (lane == 0) nzw[warp] = nb_w;
    __syncthreads();
    if (t == 0) {
      uint32_t nz = 0;
      for (int w = 0; w < 8; ++w) nz += nzw[w];
      atomicAdd(&st->ctot[d1 >> 2], m);
      if (nz) atomicAdd(&st->nztot[d1 >> 2], nz);
    }
  }
}

// Sum over the first `nblk` of 64 per-block totals (warp 0), broadcast through `out`.
// Contains __syncthreads.
__device__ __forceinline__ void sum_before(const uint32_t* tot, uint32_t nblk, uint32_t* out,
                                           uint32_t* out2 = nullptr,
                                           const uint32_t* tot2 = nullptr) {
  if (threadIdx.x < 32) {
    const uint32_t l = threadIdx.x;
    uint32_t a = (l < nblk ? tot[l] : 0u) + (l + 32 < nblk ? tot[l + 32] : 0u);
    uint32_t b = 0;
    if (tot2) b = (l < nblk ? tot2[l] : 0u) + (l + 32 < nblk ? tot2[l + 32] : 0u);
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      a += __shfl_xor_sync(kFull, a, off);
      b += __shfl_xor_sync(kFull, b, off);
    }
    if (l == 0) {
      *out = a;
      if (out2) *out2 = b;
    }
  }
  __syncthreads();
}

// Blocks of 1024 buckets, one per thread: every bucket's first entry (the second pass's
// write cursors) and the non-empty buckets in key order (first entry, entries, bucket); a
// block's offsets come from the per-block totals of the earlier blocks.  With one pass the
// buckets are the first digits (at most 256, one block) and their counts the key kernel's.
__global__ __launch_bounds__(1024) void msd_scan2_kernel(State* st, const uint32_t* __restrict__ hist2,
                                                         uint32_t* __restrict__ cur2,
                                                         uint32_t* __restrict__ bjob, int* err) {
  __shared__ uint32_t tmp[32];
  __shared__ uint32_t s_be, s_bj;
  if (!msd_on(st) || block_error_raised(err)) return;
  const int t = threadIdx.x;
  const bool two = st->levels == 2;
  const uint32_t nb = 1u << (st->b1 + st->b2);
  const uint32_t blk = blockIdx.x;
  if (blk * 1024u >= nb) return;
  if (two) {
    sum_before(st->ctot, blk, &s_be, &s_bj, st->nztot);
  } else if (t == 0) {
    s_be = 0;
    s_bj = 0;
  }
  __syncthreads();
  const uint32_t b = blk * 1024u + uint32_t(t);
  const uint32_t c = b < nb ? (two ? hist2[b] : st->hist[0][b]) : 0u;
  uint32_t tot_e, tot_j;
  const uint32_t e = s_be + block_excl_scan(c, &tot_e, tmp);
  __syncthreads();
  const uint32_t q = s_bj + block_excl_scan(c ? 1u : 0u, &tot_j, tmp);
  if (two && b < nb) cur2[b] = e;
  if (c) {
    bjob[q] = e;
    bjob[kMsdBuckets + q] = c;
    bjob[2 * kMsdBuckets + q] = b;
  }
  if (t == 0 && (blk + 1) * 1024u >= nb) {  // the last block
    const bool ok = s_be + tot_e == st->nvalid;
    st->nbjobs = ok ? s_bj + tot_j : 0u;
    if (!ok) set_error(err, kErrInvalidArg);
  }
}

// ---- the bucket kernel's jobs --------------------------------------------------------------

constexpr int kBkWords = 1 << (kMsdMaxLow - 5);  // bitmap words of a 2^16-key range
constexpr uint32_t kJobRun = 0xffffffffu;        // bj of a job of whole buckets

// A job of the bucket kernel (kJobWords words): its mw entries [start, start + mw), keys in
// [key_lo, key_lo + span), in the last partition pass's output (a run of whole buckets) or
// in the other buffer (a window of a large bucket, `scratch` = 1); its cells' rows start at
// `row` (a run) or at the first row of non-empty bucket `bj` plus `row` (a window).
struct Job {
  uint32_t start, mw, key_lo, span, row, scratch, bj, pad;
};

__device__ __forceinline__ void put_job(uint32_t* dst, const Job& j) {
  uint4* d = reinterpret_cast<uint4*>(dst);
  d[0] = make_uint4(j.start, j.mw, j.key_lo, j.span);
  d[1] = make_uint4(j.row, j.scratch, j.bj, 0u);
}

// Rank of key offset k among the occupied ones (ranks of the words set).
__device__ __forceinline__ uint32_t rank_of(const uint32_t* bits, const uint16_t* rank, uint32_t k) {
  const uint32_t w = k >> 5;
  return uint32_t(rank[w]) + __popc(bits[w] & ((1u << (k & 31u)) - 1u));
}

// Exclusive popcount prefix of words [0, nw) into rank (when with_ranks) and their total.
// kThreads threads, (2^16 / 32) / kThreads words per thread.  Contains __syncthreads.
template <int kThreads>
__device__ __forceinline__ uint32_t bitmap_popc(const uint32_t* bits, uint16_t* rank, int nw,
                                                bool with_ranks, uint32_t* tmp) {
  constexpr int kPer = kBkWords / kThreads;
  const int t = threadIdx.x;
  uint32_t pc[kPer], mine = 0;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int w = kPer * t + q;
    pc[q] = w < nw ? __popc(bits[w]) : 0u;
    mine += pc[q];
  }
  uint32_t V;
  uint32_t run = block_excl_scan(mine, &V, tmp);
  if (with_ranks) {
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int w = kPer * t + q;
      if (w < nw) {
        rank[w] = static_cast<uint16_t>(run);
        run += pc[q];
      }
    }
  }
  return V;
}

// ---- cells of every bucket; windows of the large ones -----------------------------------

constexpr int kCntThreads = 256;
constexpr int kCntItems = kBkStage / kCntThreads;
static_assert(kBkStage % kCntThreads == 0, "count stage");
struct CntSmem {
  uint32_t keys[2][kBkStage + 4];  // staged keys of the current and the next bucket
  uint32_t bits[kBkWords];         // occupancy of the bucket's low key bits (kept clean)
  uint32_t coarse[256];            // entries per coarse key range, then fill counters
  uint32_t ccell[256];             // cells per coarse key range
  uint32_t pfx[257];               // first entry of every coarse range inside the bucket
  uint32_t cpfx[257];              // first cell of every coarse range inside the bucket
  uint32_t nxt[256];               // end of the window that starts at a coarse range
  uint16_t winlo[256], winhi[256];  // windows as coarse-range intervals
  uint32_t tmp[kCntThreads / 32];
  unsigned long long bar[2];
  uint32_t jb[2][4];  // bucket index, first entry, entries, bucket id
  uint32_t s_v, s_nwin, s_q, s_bi, s_q3;
};
static_assert(offsetof(CntSmem, keys) % 16 == 0, "count stage buffers on 16-byte boundaries");
static_assert(offsetof(CntSmem, bar) % 8 == 0, "mbarrier alignment");

// Descriptor of non-empty bucket j (first entry, entries, bucket id), or j itself past nb.
struct BDesc {
  uint32_t j, start, m, bucket;
};
__device__ __forceinline__ BDesc bdesc_load(const uint32_t* bjob, uint32_t j, uint32_t nb) {
  BDesc d{j, 0u, 0u, 0u};
  if (j < nb) {
    d.start = bjob[j];
    d.m = bjob[kMsdBuckets + j];
    d.bucket = bjob[2 * kMsdBuckets + j];
  }
  return d;
}
// Slot b takes descriptor d, and buffer b its keys when they fit (bulk copy from the
// 16-byte boundary at or below its first entry).
__device__ __forceinline__ void cnt_stage(CntSmem& sm, int b, const BDesc& d, uint32_t nb,
                                          const uint32_t* K) {
  sm.jb[b][0] = d.j;
  sm.jb[b][1] = d.start;
  sm.jb[b][2] = d.m;
  sm.jb[b][3] = d.bucket;
  if (d.j < nb && d.m <= uint32_t(kBkStage)) {
    const uint32_t kg = ((d.start & 3u) + d.m + 3u) >> 2;
    mbar_arrive_expect_tx(&sm.bar[b], 16u * kg);
    bulk_copy_g2s(sm.keys[b], K + (d.start & ~3u), 16u * kg, &sm.bar[b]);
  }
}

// Marks key offset k in the bitmap; true when the key was not there yet (a new cell).
__device__ __forceinline__ bool mark_new(uint32_t* bits, uint32_t k) {
  const uint32_t bit = 1u << (k & 31u);
  return (atomicOr(&bits[k >> 5], bit) & bit) == 0u;
}

// Every non-empty bucket (block b takes buckets b, b + G, ...; a bucket's keys are copied
// while the one before is counted, its descriptor read two buckets ahead): its cells, the
// keys that find their bit of the occupancy bitmap still clear, added into the cells of
// its block of 1024 buckets.  A bucket of more than kBkStage entries is also cut into
// windows of consecutive coarse key ranges (the bucket's key range in 256 equal parts) of
// at most kBkStage entries each (a range of more entries is a window of its own); its
// entries are written, grouped by coarse range, to the same place of the other buffer,
// and every window becomes a job with the number of cells before it.
__global__ __launch_bounds__(kCntThreads) void msd_count_kernel(
    State* st, const uint32_t* k0, const uint32_t* k1, const uint32_t* __restrict__ bjob,
    uint32_t* __restrict__ vcnt, uint32_t* __restrict__ jobsw, uint32_t jobsw_cap,
    uint32_t* __restrict__ cur3, uint32_t big_cap, uint32_t* __restrict__ jobs3,
    uint32_t jobs3_cap, int* err) {
  extern __shared__ __align__(128) unsigned char cnt_smem[];
  CntSmem& sm = *reinterpret_cast<CntSmem*>(cnt_smem);
  if (!msd_on(st) || block_error_raised(err)) return;
  const uint32_t nb = st->nbjobs;
  if (blockIdx.x >= nb) return;
  const uint32_t* K = st->levels == 2 ? k0 : k1;  // the last partition pass's output
  const uint32_t L = st->lowbits;
  const uint32_t lowmask = (1u << L) - 1u;
  const int nw = L >= 5 ? 1 << (L - 5) : 1;
  const uint32_t cs = L > 8 ? L - 8 : 0;  // coarse range width (log2)
  const uint32_t nco = 1u << (L - cs);
  const uint32_t G = gridDim.x;
  const int t = threadIdx.x, lane = t & 31;
  for (int w = t; w < nw; w += kCntThreads) sm.bits[w] = 0;
  BDesc ahead{};  // thread 0: the bucket after the next one
  if (t == 0) {
    mbar_init(&sm.bar[0], 1);
    mbar_init(&sm.bar[1], 1);
    fence_mbar_init();
    cnt_stage(sm, 0, bdesc_load(bjob, blockIdx.x, nb), nb, K);
    ahead = bdesc_load(bjob, blockIdx.x + G, nb);
  }
  __syncthreads();
  uint32_t phase = 0;
  for (int b = 0;; b ^= 1) {
    const uint32_t j = sm.jb[b][0];
    if (j >= nb) break;
    const uint32_t start = sm.jb[b][1], m = sm.jb[b][2], bucket = sm.jb[b][3];
    const bool big = m > uint32_t(kBkStage);
    if (t == 0) {
      fence_proxy_async();
      cnt_stage(sm, b ^ 1, ahead, nb, K);
      ahead = bdesc_load(bjob, ahead.j + G, nb);
      sm.s_v = 0;
    }
    uint32_t nc = 0;  // new cells this thread found
    const uint32_t* sk = sm.keys[b] + (start & 3u);
    if (!big) {
      bool ok = true;
      const uint32_t par = (phase >> b) & 1u;
      if (t < 32) ok = mbar_wait(&sm.bar[b], par, kDefaultSpinLimit);
      phase ^= 1u << b;
      if (__syncthreads_or(!ok)) {  // a copy that never completed: report, drain, stop
        if (t == 0) {
          set_error(err, kErrTimeout);
          mbar_wait(&sm.bar[b], par, kDefaultSpinLimit);
          if (sm.jb[b ^ 1][0] < nb && sm.jb[b ^ 1][2] <= uint32_t(kBkStage))
            mbar_wait(&sm.bar[b ^ 1], (phase >> (b ^ 1)) & 1u, kDefaultSpinLimit);
        }
        return;
      }
#pragma unroll
      for (int q = 0; q < kCntItems; ++q) {
        if (uint32_t(q) * kCntThreads >= m) break;
        const uint32_t i = uint32_t(q) * kCntThreads + uint32_t(t);
        if (i < m) nc += mark_new(sm.bits, sk[i] & lowmask);
      }
    } else {
      sm.coarse[t] = 0;
      sm.ccell[t] = 0;
      __syncthreads();
      for (uint32_t i0 = 0; i0 < m; i0 += 8u * kCntThreads) {
        uint32_t k[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const uint32_t i = i0 + uint32_t(q) * kCntThreads + uint32_t(t);
          k[q] = i < m ? (__ldcg(K + start + i) & lowmask) : kFull;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (k[q] != kFull) {
            const bool fresh = mark_new(sm.bits, k[q]);
            nc += fresh;
            atomicAdd(&sm.coarse[k[q] >> cs], 1u);
            if (fresh) atomicAdd(&sm.ccell[k[q] >> cs], 1u);
          }
      }
    }
    // the bucket's cells
#pragma unroll
    for (int off = 16; off; off >>= 1) nc += __shfl_xor_sync(kFull, nc, off);
    if (lane == 0 && nc) atomicAdd(&sm.s_v, nc);
    __syncthreads();
    if (t == 0) {
      vcnt[j] = sm.s_v;
      atomicAdd(&st->vtot[j >> 10], sm.s_v);
    }
    if (!big) {
      // the bitmap clean again: only the words this bucket touched
#pragma unroll
      for (int q = 0; q < kCntItems; ++q) {
        if (uint32_t(q) * kCntThreads >= m) break;
        const uint32_t i = uint32_t(q) * kCntThreads + uint32_t(t);
        if (i < m) sm.bits[(sk[i] & lowmask) >> 5] = 0;
      }
    } else {
      // windows: every coarse range's first entry and first cell; from each range, the end
      // of the widest window of at most kBkStage entries starting there (a range of more
      // entries is a window of its own); walked from range 0, skipping windows without
      // entries
      const uint32_t h = uint32_t(t) < nco ? sm.coarse[t] : 0u;
      const uint32_t hc = uint32_t(t) < nco ? sm.ccell[t] : 0u;
      // (coarse counts stay where they are: the third pass needs none of them)
      uint32_t tot, totc;
      const uint32_t ex = block_excl_scan(h, &tot, sm.tmp);
      const uint32_t exc = block_excl_scan(hc, &totc, sm.tmp);
      if (uint32_t(t) < nco) {
        sm.pfx[t] = ex;
        sm.cpfx[t] = exc;
      }
      if (t == 0) {
        sm.pfx[nco] = tot;
        sm.cpfx[nco] = totc;
      }
      __syncthreads();
      if (uint32_t(t) < nco) {
        const uint32_t c = t, lim = sm.pfx[c] + uint32_t(kBkStage);
        uint32_t e = c + 1;
        if (sm.pfx[e] <= lim) {  // the largest e <= nco with pfx[e] <= lim
          uint32_t lo = e, hi = nco;
          while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (sm.pfx[mid] <= lim) lo = mid;
            else hi = mid - 1;
          }
          e = lo;
        }
        sm.nxt[c] = e;
      }
      __syncthreads();
      if (t == 0) {
        uint32_t k = 0;
        for (uint32_t c = 0; c < nco;) {
          const uint32_t e = sm.nxt[c];
          if (sm.pfx[e] > sm.pfx[c]) {
            sm.winlo[k] = static_cast<uint16_t>(c);
            sm.winhi[k] = static_cast<uint16_t>(e);
            ++k;
          }
          c = e;
        }
        sm.s_nwin = k;
        sm.s_q = atomicAdd(&st->nwjobs, k);
        sm.s_bi = atomicAdd(&st->nbig, 1u);
        sm.s_q3 = atomicAdd(&st->njobs3, (m + kPartTile - 1) / kPartTile);
      }
      __syncthreads();
      // the window jobs, in the other buffer at the bucket's own entries, which the third
      // partition pass groups there by coarse range: its cursors and its chunks
      const uint32_t nwin = sm.s_nwin, q0 = sm.s_q, bi = sm.s_bi, q3 = sm.s_q3;
      const uint32_t nch = (m + kPartTile - 1) / kPartTile;
      const bool room = q0 + nwin <= jobsw_cap && bi < big_cap && q3 + nch <= jobs3_cap;
      if (room) {
        if (uint32_t(t) < nwin) {
          const uint32_t lo = sm.winlo[t], hi = sm.winhi[t];
          put_job(jobsw + size_t(q0 + t) * kJobWords,
                  Job{start + sm.pfx[lo], sm.pfx[hi] - sm.pfx[lo], (bucket << L) + (lo << cs),
                      (hi - lo) << cs, sm.cpfx[lo], 1u, j, 0u});
        }
        if (uint32_t(t) < nco) cur3[size_t(bi) * 256 + t] = start + sm.pfx[t];
        for (uint32_t c = t; c < nch; c += kCntThreads)
          reinterpret_cast<uint4*>(jobs3)[q3 + c] =
              make_uint4(start + c * kPartTile, min(uint32_t(kPartTile), m - c * kPartTile), bi, 0u);
      } else if (t == 0) {
        set_error(err, kErrInvalidArg);
      }
      // the bitmap clean again (a large bucket touches many words)
      for (int w = t; w < nw; w += kCntThreads) sm.bits[w] = 0;
    }
    fence_proxy_async();  // this thread's reads of buffer b precede later bulk copies
    __syncthreads();
  }
}

// Blocks of 1024 non-empty buckets, one per thread: every bucket's first row (its block's
// offset from the cells of the earlier blocks, then a block scan) and V; the frame offsets
// (a bucket lies inside one frame); and the jobs of whole buckets: within each warp's 32
// buckets, runs of consecutive buckets of at most kBkStage entries each, of at most
// kBkStage entries and a key span of at most 2^16 together (a large bucket ends a run),
// appended in any order (every job carries its own first row).
__global__ __launch_bounds__(1024) void msd_plan_kernel(State* st, const uint32_t* __restrict__ bjob,
                                                        const uint32_t* __restrict__ vcnt,
                                                        uint32_t* __restrict__ vbase,
                                                        uint32_t* __restrict__ jobsm, SegOut out,
                                                        int nframes, int* err) {
  __shared__ uint32_t tmp[32];
  __shared__ uint32_t s_base;
  __shared__ uint32_t wm[32][32], wb[32][32], wrow[32][32], wst[32][32];
  if (!msd_on(st) || block_error_raised(err)) return;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const uint32_t nb = st->nbjobs;
  const uint32_t blk = blockIdx.x;
  if (blk * 1024u >= nb) return;
  const uint32_t L = st->lowbits;
  const uint32_t key_shift = st->key_shift;
  sum_before(st->vtot, blk, &s_base);
  const uint32_t j = blk * 1024u + uint32_t(t);
  const bool in = j < nb;
  const uint32_t v = in ? vcnt[j] : 0u;
  const uint32_t m = in ? bjob[kMsdBuckets + j] : 0u;
  const uint32_t bk = in ? bjob[2 * kMsdBuckets + j] : 0u;
  const uint32_t st0 = in ? bjob[j] : 0u;
  uint32_t tot;
  const uint32_t row = s_base + block_excl_scan(v, &tot, tmp);
  if (in) vbase[j] = row;
  // frame offsets (frames before the first bucket's keep the zero they start with)
  if (in && out.frame_offsets && key_shift < 64) {
    const uint32_t fk = key_frame(uint64_t(bk) << L, key_shift);
    if (j > 0) {
      const uint32_t fp = key_frame(uint64_t(bjob[2 * kMsdBuckets + j - 1]) << L, key_shift);
      for (uint32_t f = fp + 1; f <= fk; ++f) out.frame_offsets[f] = row;
    }
    if (j + 1 == nb)
      for (uint32_t f = fk + 1; f <= uint32_t(nframes); ++f) out.frame_offsets[f] = row + v;
  }
  if (in && j + 1 == nb) *out.num_voxels = int64_t(row) + v;
  // runs of whole buckets within the warp's 32 buckets (lane 0 walks them twice: counting,
  // then writing after one append)
  wm[warp][lane] = in ? m : 0xffffffffu;  // past the end: ends any run
  wb[warp][lane] = bk;
  wrow[warp][lane] = row;
  wst[warp][lane] = st0;
  __syncwarp();
  if (lane == 0) {
    const uint32_t max_run = L >= 16 ? 1u : (1u << (16 - L));  // buckets a 2^16 span holds
    uint32_t njobs = 0, q = 0;
    for (int pass = 0; pass < 2; ++pass) {
      bool open = false;
      uint32_t sum = 0, b0 = 0, b1 = 0, f = 0;
      for (int i = 0; i <= 32; ++i) {
        const bool end = i == 32;
        const uint32_t mi = end ? 0xffffffffu : wm[warp][i], bi = end ? 0u : wb[warp][i];
        const bool small = mi <= uint32_t(kBkStage);
        const bool joins = small && open && sum + mi <= uint32_t(kBkStage) && bi - b0 < max_run;
        if (open && !joins) {  // the run [f, i) ends
          if (pass == 0) {
            ++njobs;
          } else {
            put_job(jobsm + size_t(q) * kJobWords,
                    Job{wst[warp][f], sum, b0 << L, (b1 - b0 + 1u) << L, wrow[warp][f], 0u,
                        kJobRun, 0u});
            ++q;
          }
          open = false;
        }
        if (end) break;
        if (!small) continue;
        if (joins) {
          sum += mi;
          b1 = bi;
        } else {
          open = true;
          f = uint32_t(i);
          sum = mi;
          b0 = b1 = bi;
        }
      }
      if (pass == 0) {
        if (njobs == 0) break;
        q = atomicAdd(&st->nmjobs, njobs);
      }
    }
  }
}

// ---- the bucket kernel ------------------------------------------------------------------

// Geometry (build-time): 512 threads, two blocks per SM.
#ifndef VG_BK_THREADS
#define VG_BK_THREADS 512
#endif
#ifndef VG_BK_MINB
#define VG_BK_MINB 2
#endif
constexpr int kBkThreads = VG_BK_THREADS;
constexpr int kBkWarps = kBkThreads / 32;
constexpr int kBkItems = kBkStage / kBkThreads;
constexpr int kBkPer = kBkWords / kBkThreads;  // bitmap words per thread
constexpr int kSlotMax = 256;  // keys of an oversized window (one coarse range)
// A cell's first kSumSplit entries are summed in 32 bits (kSumSplit biased 21-bit offsets
// stay below 2^32).  A job holds at most kBkStage < 2 kSumSplit entries, so at most one of
// its cells has more; their further entries go into one 64-bit sum per axis.
constexpr uint32_t kSumSplit = 2048;
static_assert(kBkStage % kBkThreads == 0, "bucket stage");
static_assert(kBkWords % kBkThreads == 0, "bucket bitmap");
static_assert(kBkStage < 2 * int(kSumSplit), "at most one cell per job above the 32-bit sums");
static_assert(uint64_t(kSumSplit) * 0x1fffffu <= 0xffffffffull, "32-bit sums");
static_assert(kBkStage < 65536, "16-bit ranks and key offsets");
static_assert(kSlotMax <= kBkThreads && 6 * kSlotMax <= 3 * kBkStage, "slots fit the sums");
static_assert(kBkWarps <= 32, "one warp scans the warp totals");

struct BkSmem {
  uint32_t keys[kBkStage + 4];           // staged keys, from a 16-byte boundary
  unsigned long long pay[kBkStage + 2];  // staged payloads, from a 16-byte boundary
  unsigned long long big[4];             // 64-bit sums past kSumSplit entries (kept zero)
  uint32_t bits[2][kBkWords];            // occupancy bitmaps of alternate jobs (kept clean)
  uint32_t cnt[kBkStage];                // entries per cell (kept zero)
  uint32_t sum[3][kBkStage];             // biased offset sums per cell and axis (kept zero)
  uint16_t rank[kBkWords];               // occupied cells before each word
  uint16_t vkey[kBkStage];               // key offset of each cell in the job's range
  uint32_t tmp[kBkWarps];
  unsigned long long bar[2];             // [0] key copies, [1] payload copies
  Job job[2];                            // this job and the next (alternating slots)
  Job ahd;                               // the one after (copied in asynchronously)
  uint32_t jid[2];
  RowCtx rc;
};
static_assert(offsetof(BkSmem, keys) % 16 == 0 && (sizeof(uint32_t) * (kBkStage + 4)) % 16 == 0,
              "key stage buffer on a 16-byte boundary");
static_assert(offsetof(BkSmem, pay) % 16 == 0 && (8 * (kBkStage + 2)) % 16 == 0,
              "payload stage buffer on a 16-byte boundary");
static_assert(offsetof(BkSmem, sum) % 8 == 0, "oversized windows sum in 64 bits there");
static_assert(offsetof(BkSmem, bar) % 8 == 0, "mbarrier alignment");
static_assert(offsetof(BkSmem, job) % 16 == 0 && offsetof(BkSmem, ahd) % 16 == 0 &&
                  sizeof(Job) == 32,
              "descriptors copied in 16-byte pieces");
static_assert((sizeof(BkSmem) + 1024) * VG_BK_MINB <= 228 * 1024, "bucket block shared memory");

// Job q of the bucket kernel's order (the windows, then the runs of whole buckets), or an
// empty job past the last one.
__device__ __forceinline__ Job job_load(uint32_t q, uint32_t nwin, uint32_t njobs,
                                        const uint32_t* jobsw, const uint32_t* jobsm) {
  if (q >= njobs) return Job{0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
  const uint4* p = reinterpret_cast<const uint4*>(
      q < nwin ? jobsw + size_t(q) * kJobWords : jobsm + size_t(q - nwin) * kJobWords);
  const uint4 a = p[0], b = p[1];
  return Job{a.x, a.y, a.z, a.w, b.x, b.y, b.z, 0u};
}

// The same, copied into *dst asynchronously (complete after cp_async_wait_all).
__device__ __forceinline__ void job_fetch(Job* dst, uint32_t q, uint32_t nwin, uint32_t njobs,
                                          const uint32_t* jobsw, const uint32_t* jobsm) {
  if (q >= njobs) {
    *dst = Job{0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    return;
  }
  const uint32_t* p = q < nwin ? jobsw + size_t(q) * kJobWords : jobsm + size_t(q - nwin) * kJobWords;
  cp_async16(dst, p);
  cp_async16(reinterpret_cast<uint32_t*>(dst) + 4, p + 4);
}

__device__ __forceinline__ bool staged_by_copy(const Job& j) {
  return j.mw <= uint32_t(kBkStage);
}

// The buffers holding a job's entries.
struct Bufs {
  const uint32_t* K;
  const uint64_t* P;
  const uint32_t* KS;
  const uint64_t* PS;
};


// Bulk copies of a job's keys (barrier 0) or payloads (barrier 1) into the stage buffer,
// from the 16-byte boundary at or below its first entry, in whole granules.
__device__ __forceinline__ void issue_keys(BkSmem& sm, const Bufs& bf, const Job& d) {
  const uint32_t* K = d.scratch ? bf.KS : bf.K;
  const uint32_t kg = ((d.start & 3u) + d.mw + 3u) >> 2;  // 16-byte granules of keys
  mbar_arrive_expect_tx(&sm.bar[0], 16u * kg);
  bulk_copy_g2s(sm.keys, K + (d.start & ~3u), 16u * kg, &sm.bar[0]);
}
__device__ __forceinline__ void issue_pays(BkSmem& sm, const Bufs& bf, const Job& d) {
  const uint64_t* P = d.scratch ? bf.PS : bf.P;
  const uint32_t pg = ((d.start & 1u) + d.mw + 1u) >> 1;  // 16-byte granules of payloads
  mbar_arrive_expect_tx(&sm.bar[1], 16u * pg);
  bulk_copy_g2s(sm.pay, P + (d.start & ~1u), 16u * pg, &sm.bar[1]);
}

// An oversized window: at most kSlotMax keys, any number of entries (contiguous in the
// job's buffer), read from global memory; one slot per key (the cell counters and, as
// 64-bit words, the first sums), warp sums first when a whole warp meets one key.  Leaves
// the slots zero again.
__device__ __forceinline__ void slot_window(BkSmem& sm, const Bufs& bf, const Job& d,
                                            uint32_t row0, const RowCtx& rc, const SegOut& out,
                                            int* err) {
  const uint32_t* __restrict__ K = d.scratch ? bf.KS : bf.K;
  const uint64_t* __restrict__ P = d.scratch ? bf.PS : bf.P;
  const int t = threadIdx.x, lane = t & 31;
  uint32_t* wcnt = sm.cnt;
  unsigned long long* wsum = reinterpret_cast<unsigned long long*>(&sm.sum[0][0]);  // [3][256]
  const uint32_t span = d.span;  // <= kSlotMax
  __syncthreads();  // the job before has read and cleared the slots
  for (uint32_t i0 = 0; i0 < d.mw; i0 += 4u * kBkThreads) {
    uint32_t k[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t i = i0 + uint32_t(q) * kBkThreads + uint32_t(t);
      k[q] = i < d.mw ? __ldcg(K + d.start + i) : kFull;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t i = i0 + uint32_t(q) * kBkThreads + uint32_t(t);
      const uint32_t s = k[q] != kFull ? k[q] - d.key_lo : kFull;
      const bool in = s < span;
      long long v[3] = {0, 0, 0};
      if (in) {
        const uint64_t p = __ldcg(P + d.start + i);
        v[0] = unpack_offset(p, 0);
        v[1] = unpack_offset(p, 1);
        v[2] = unpack_offset(p, 2);
      }
      const uint32_t s0 = __shfl_sync(kFull, s, 0);
      if (__all_sync(kFull, s == s0) && s0 < span) {  // one key for the whole warp
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int off = 16; off; off >>= 1) v[a] += __shfl_xor_sync(kFull, v[a], off);
        if (lane == 0) {
          atomicAdd(&wcnt[s0], 32u);
#pragma unroll
          for (int a = 0; a < 3; ++a)
            atomicAdd(&wsum[a * kSlotMax + s0], static_cast<unsigned long long>(v[a]));
        }
      } else if (in) {
        atomicAdd(&wcnt[s], 1u);
#pragma unroll
        for (int a = 0; a < 3; ++a)
          atomicAdd(&wsum[a * kSlotMax + s], static_cast<unsigned long long>(v[a]));
      }
    }
  }
  __syncthreads();
  // rows of the occupied keys, in key order
  const uint32_t n = uint32_t(t) < span ? wcnt[t] : 0u;
  Acc a;
  a.n = n;
  a.s[0] = a.s[1] = a.s[2] = 0;
  if (uint32_t(t) < span) {
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      a.s[x] = static_cast<long long>(wsum[x * kSlotMax + t]);
      wsum[x * kSlotMax + t] = 0;
    }
    wcnt[t] = 0;
  }
  uint32_t unused;
  const uint32_t r = block_excl_scan(n ? 1u : 0u, &unused, sm.tmp);
  if (n) put_row(rc, out, row0 + r, d.key_lo + uint32_t(t), a, err);
}

// Block b runs jobs b, b + G, ... (the windows first: the larger jobs).  A job's keys are
// copied in while the job before ranks its entries, and its payloads while the job before
// writes its rows; descriptors are read two jobs ahead.  Per job:
//   1. every thread waits for the keys and marks its entries' key offsets in the job's
//      occupancy bitmap (two bitmaps, alternate jobs: one is cleared while the other fills);
//   2. the prefix popcounts of the bitmap's words: every cell's rank, in key order;
//   3. every thread waits for the payloads and adds each entry into its cell's counter and
//      per-axis sums (shared-memory atomics; integers, so the order does not matter);
//   4. one thread per cell writes its row and clears its counter and sums.
// Four barriers a job; counters, sums and bitmaps are left clean for the next one.
__global__ __launch_bounds__(kBkThreads, VG_BK_MINB) void msd_bucket_kernel(
    State* st, const FrameState* __restrict__ fs, const uint32_t* k0, const uint64_t* p0,
    const uint32_t* k1, const uint64_t* p1, const uint32_t* __restrict__ jobsw,
    const uint32_t* __restrict__ jobsm, const uint32_t* __restrict__ vbase, SegOut out,
    int* err) {
  extern __shared__ __align__(128) unsigned char bk_smem[];
  BkSmem& sm = *reinterpret_cast<BkSmem*>(bk_smem);
  if (!msd_on(st) || block_error_raised(err)) return;
  const uint32_t nwin = st->nwjobs, njobs = nwin + st->nmjobs;
  if (blockIdx.x >= njobs) return;
  const bool two = st->levels == 2;
  // the last partition pass's output, and the other buffer (windows of large buckets)
  const Bufs bf{two ? k0 : k1, two ? p0 : p1, two ? k1 : k0, two ? p1 : p0};
  const uint32_t G = gridDim.x;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const RowCtx& rc = sm.rc;

  for (int i = t; i < kBkStage; i += kBkThreads) {
    sm.cnt[i] = 0;
    sm.sum[0][i] = sm.sum[1][i] = sm.sum[2][i] = 0;
  }
  for (int w = t; w < 2 * kBkWords; w += kBkThreads) sm.bits[w / kBkWords][w % kBkWords] = 0;
  if (t < 4) sm.big[t] = 0;
  // thread 0 keeps the job numbers: slot s holds job jid[s] (this one), slot s ^ 1 the
  // next (whose copies are issued during this one), ahd the one after (jid qa)
  uint32_t qa = 0;
  if (t == 0) {
    sm.rc.fs = fs;
    sm.rc.key_shift = st->key_shift;
    sm.rc.o1[0] = fs[0].origin[0];
    sm.rc.o1[1] = fs[0].origin[1];
    sm.rc.o1[2] = fs[0].origin[2];
    sm.rc.leaf1 = fs[0].leaf;
    mbar_init(&sm.bar[0], 1);
    mbar_init(&sm.bar[1], 1);
    fence_mbar_init();
    const uint32_t q = blockIdx.x, qn = q + G;
    sm.jid[0] = q;
    sm.job[0] = job_load(q, nwin, njobs, jobsw, jobsm);
    if (staged_by_copy(sm.job[0])) {
      issue_keys(sm, bf, sm.job[0]);
      issue_pays(sm, bf, sm.job[0]);
    }
    sm.jid[1] = qn;
    sm.job[1] = job_load(qn, nwin, njobs, jobsw, jobsm);
    qa = qn < njobs ? qn + G : qn;
    job_fetch(&sm.ahd, qa, nwin, njobs, jobsw, jobsm);
  }
  __syncthreads();
  uint32_t par = 0;  // parity of both copy barriers' next completion
  int jb = 0;        // the bitmap of the next staged job
  for (int s = 0;; s ^= 1) {
    const uint32_t q = sm.jid[s];
    if (q >= njobs) break;
    const Job d = sm.job[s];
    // this job's first row (a window's: its bucket's first row plus its first cell's rank)
    const uint32_t row0 = d.row + (d.bj != kJobRun ? vbase[d.bj] : 0u);
    const Job& nxt = sm.job[s ^ 1];  // (thread 0 issues its copies)
    const bool nxt_copy = t == 0 && sm.jid[s ^ 1] < njobs && staged_by_copy(nxt);
    if (!staged_by_copy(d)) {  // an oversized window: nothing of it is staged
      if (nxt_copy) {
        issue_keys(sm, bf, nxt);
        issue_pays(sm, bf, nxt);
      }
      slot_window(sm, bf, d, row0, rc, out, err);
    } else {
      const uint32_t m = d.mw;
      const uint32_t* sk = sm.keys + (d.start & 3u);
      const unsigned long long* sp = sm.pay + (d.start & 1u);
      uint32_t* bits = sm.bits[jb];
      const int nw = int((d.span + 31u) >> 5);
      // (item loops stop at the job's entries: the break is the same in every thread)

      // 1. the keys, and the occupancy bitmap of the job's key range
      bool ok = mbar_wait(&sm.bar[0], par, kDefaultSpinLimit);
      uint32_t kl[kBkItems];
#pragma unroll
      for (int q2 = 0; q2 < kBkItems; ++q2) {
        kl[q2] = kFull;
        if (uint32_t(q2) * kBkThreads >= m) break;
        const uint32_t i = uint32_t(q2) * kBkThreads + uint32_t(t);
        kl[q2] = i < m ? sk[i] - d.key_lo : kFull;
        if (kl[q2] != kFull) atomicOr(&bits[kl[q2] >> 5], 1u << (kl[q2] & 31u));
      }
      fence_proxy_async();  // this thread's reads of the key buffer precede the next copy
      if (__syncthreads_or(!ok)) {  // a copy that never completed: report, drain, stop
        if (t == 0) {
          set_error(err, kErrTimeout);
          mbar_wait(&sm.bar[0], par, kDefaultSpinLimit);
          mbar_wait(&sm.bar[1], par, kDefaultSpinLimit);
          cp_async_wait_all();
        }
        return;
      }
      if (nxt_copy) issue_keys(sm, bf, nxt);

      // 2. cells before every word (exclusive prefix of the popcounts) and the cell count
      uint32_t pc[kBkPer], mine = 0;
#pragma unroll
      for (int q2 = 0; q2 < kBkPer; ++q2) {
        const int w = kBkPer * t + q2;
        pc[q2] = w < nw ? __popc(bits[w]) : 0u;
        mine += pc[q2];
      }
      uint32_t inc = mine;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, inc, off);
        if (lane >= off) inc += y;
      }
      if (lane == 31) sm.tmp[warp] = inc;
      __syncthreads();
      uint32_t wt = lane < kBkWarps ? sm.tmp[lane] : 0u;
#pragma unroll
      for (int off = 1; off < kBkWarps; off <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, wt, off);
        if (lane >= off) wt += y;
      }
      const uint32_t V = __shfl_sync(kFull, wt, kBkWarps - 1);
      const uint32_t wex = __shfl_sync(kFull, wt, (warp + 31) & 31);
      uint32_t run = (warp ? wex : 0u) + inc - mine;
#pragma unroll
      for (int q2 = 0; q2 < kBkPer; ++q2) {
        const int w = kBkPer * t + q2;
        if (w < nw) sm.rank[w] = static_cast<uint16_t>(run);
        run += pc[q2];
      }
      __syncthreads();

      // 3. the payloads, into their cells' counters and sums
      ok = mbar_wait(&sm.bar[1], par, kDefaultSpinLimit);
#pragma unroll
      for (int q2 = 0; q2 < kBkItems; ++q2) {
        if (uint32_t(q2) * kBkThreads >= m) break;
        if (kl[q2] != kFull) {
          const uint32_t i = uint32_t(q2) * kBkThreads + uint32_t(t);
          const uint32_t r = rank_of(bits, sm.rank, kl[q2]);
          const uint64_t p = sp[i];
          const uint32_t f[3] = {uint32_t(p) & 0x1fffffu, uint32_t(p >> 21) & 0x1fffffu,
                                 uint32_t(p >> 42) & 0x1fffffu};
          const uint32_t old = atomicAdd(&sm.cnt[r], 1u);
          if (old < kSumSplit) {
#pragma unroll
            for (int a = 0; a < 3; ++a) atomicAdd(&sm.sum[a][r], f[a]);
          } else {
#pragma unroll
            for (int a = 0; a < 3; ++a) atomicAdd(&sm.big[a], static_cast<unsigned long long>(f[a]));
          }
          if (old == 0) sm.vkey[r] = static_cast<uint16_t>(kl[q2]);
        }
      }
      fence_proxy_async();  // this thread's reads of the payload buffer precede the next copy
      if (__syncthreads_or(!ok)) {
        if (t == 0) {
          set_error(err, kErrTimeout);
          mbar_wait(&sm.bar[1], par, kDefaultSpinLimit);
          if (nxt_copy) mbar_wait(&sm.bar[0], par ^ 1u, kDefaultSpinLimit);
          cp_async_wait_all();
        }
        return;
      }
      if (nxt_copy) issue_pays(sm, bf, nxt);
      par ^= 1u;

      // 4. one row per cell (biased sums, the bias n * kQMin removed once); clean up for
      //    the next job.  Up to 1024 entries the unbiased sum fits 32 bits (|s| < 1.5 2^30),
      //    and the 32-bit difference of the biased sum and n 2^19 is that exact integer.
      for (uint32_t r = t; r < V; r += kBkThreads) {
        const uint32_t n = sm.cnt[r];
        uint32_t b[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          b[a] = sm.sum[a][r];
          sm.sum[a][r] = 0;
        }
        sm.cnt[r] = 0;
        float sf[3];
        long long s64[3];
        if (n <= 1024u) {
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const int s32 = static_cast<int>(b[a] - (n << 19));
            sf[a] = __int2float_rn(s32);
            s64[a] = s32;
          }
        } else {
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            unsigned long long bb = b[a];
            if (n > kSumSplit) {
              bb += sm.big[a];
              sm.big[a] = 0;
            }
            s64[a] = static_cast<long long>(bb) + static_cast<long long>(n) * kQMin;
            sf[a] = __ll2float_rn(s64[a]);
          }
        }
        put_row32(rc, out, row0 + r, d.key_lo + sm.vkey[r], n, sf, s64, err);
      }
#pragma unroll
      for (int q2 = 0; q2 < kBkPer; ++q2) {
        const int w = kBkPer * t + q2;
        if (w < nw) bits[w] = 0;
      }
      jb ^= 1;
    }
    if (t == 0) {  // slot s takes the job after the next; every thread has read this one
      cp_async_wait_all();
      sm.jid[s] = qa;
      sm.job[s] = sm.ahd;
      qa = qa < njobs ? qa + G : qa;
      job_fetch(&sm.ahd, qa, nwin, njobs, jobsw, jobsm);
    }
  }
  if (t == 0) cp_async_wait_all();  // (nothing is in flight: the jobs past the last are empty)
}


constexpr size_t kBkSmem = sizeof(BkSmem);

}  // namespace

void warm_msd_config() {
  persistent_grid(reinterpret_cast<const void*>(msd_part_kernel<1>), kPartThreads, 0, 1);
  persistent_grid(reinterpret_cast<const void*>(msd_part_kernel<2>), kPartThreads, 0, 1);
  persistent_grid(reinterpret_cast<const void*>(msd_part_kernel<3>), kPartThreads, 0, 1);
  persistent_grid(reinterpret_cast<const void*>(msd_count_kernel), kCntThreads, sizeof(CntSmem),
                  1);
  persistent_grid(reinterpret_cast<const void*>(msd_bucket_kernel), kBkThreads, kBkSmem, 1);
}

cudaError_t launch_msd(State* st, const FrameState* fs, int nframes, const NarrowBuffers& nb,
                       char* ws, const SortLayout& L, int64_t n_max, const SegOut& out,
                       uint32_t spin_limit, int* err, cudaStream_t stream, int stage0,
                       void (*mark)(int, cudaStream_t)) {
  (void)spin_limit;
  if (n_max == 0) return cudaSuccess;
  uint32_t* mhist = reinterpret_cast<uint32_t*>(ws + L.mhist);
  uint32_t* mvcnt = reinterpret_cast<uint32_t*>(ws + L.mvcnt);
  uint32_t* mcur = reinterpret_cast<uint32_t*>(ws + L.mcur);
  uint32_t* mjob = reinterpret_cast<uint32_t*>(ws + L.mjob);
  uint32_t* mt1 = reinterpret_cast<uint32_t*>(ws + L.mjob2);
  uint32_t* mjobm = reinterpret_cast<uint32_t*>(ws + L.mjobm);
  uint32_t* mjobw = reinterpret_cast<uint32_t*>(ws + L.mjobw);
  const int blocks1024 = kMsdBuckets / 1024;
  msd_scan1_kernel<<<1, 256, 0, stream>>>(st, mcur, mt1, err);
  const int64_t tiles = ceil_div(n_max, kPartTile);
  const int g1 = persistent_grid(reinterpret_cast<const void*>(msd_part_kernel<1>), kPartThreads,
                                 0, tiles);
  msd_part_kernel<1><<<g1, kPartThreads, 0, stream>>>(st, nb.k0, nb.p0, nb.k1, nb.p1, mcur,
                                                      mt1, n_max, err);
  mark(stage0, stream);
  const int64_t jobs2 = max_jobs2(n_max);
  const int gu = static_cast<int>(jobs2 < int64_t(num_sms()) * 8 ? jobs2 : int64_t(num_sms()) * 8);
  msd_upsweep_kernel<<<gu, 256, 0, stream>>>(st, nb.k1, mt1, mhist, err);
  msd_scan2_kernel<<<blocks1024, 1024, 0, stream>>>(st, mhist, mcur + 256, mjob, err);
  const int g2 = persistent_grid(reinterpret_cast<const void*>(msd_part_kernel<2>), kPartThreads,
                                 0, jobs2);
  msd_part_kernel<2><<<g2, kPartThreads, 0, stream>>>(st, nb.k1, nb.p1, nb.k0, nb.p0, mcur,
                                                      mt1, n_max, err);
  mark(stage0 + 1, stream);
  const int gc = persistent_grid(reinterpret_cast<const void*>(msd_count_kernel), kCntThreads,
                                 sizeof(CntSmem), int64_t(kMsdBuckets));
  uint32_t* mcur3 = reinterpret_cast<uint32_t*>(ws + L.mcur3);
  uint32_t* mjob3 = reinterpret_cast<uint32_t*>(ws + L.mjob3);
  msd_count_kernel<<<gc, kCntThreads, sizeof(CntSmem), stream>>>(
      st, nb.k0, nb.k1, mjob, mvcnt, mjobw, static_cast<uint32_t>(L.jobsw), mcur3,
      static_cast<uint32_t>(L.big), mjob3, static_cast<uint32_t>(L.jobs3), err);
  const int g3 = persistent_grid(reinterpret_cast<const void*>(msd_part_kernel<3>), kPartThreads,
                                 0, L.jobs3);
  msd_part_kernel<3><<<g3, kPartThreads, 0, stream>>>(st, nb.k0, nb.p0, nb.k1, nb.p1, mcur3,
                                                      mjob3, n_max, err);
  msd_plan_kernel<<<blocks1024, 1024, 0, stream>>>(st, mjob, mvcnt, mcur + 256, mjobm, out,
                                                   nframes, err);
  const int gb = persistent_grid(reinterpret_cast<const void*>(msd_bucket_kernel), kBkThreads,
                                 kBkSmem, int64_t(kMsdBuckets) + L.jobsw);
  msd_bucket_kernel<<<gb, kBkThreads, kBkSmem, stream>>>(st, fs, nb.k0, nb.p0, nb.k1, nb.p1, mjobw,
                                                          mjobm, mcur + 256, out, err);
  mark(stage0 + 2, stream);
  return cudaGetLastError();
}

}  // namespace vg
