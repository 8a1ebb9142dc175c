// Bucket tail of the narrow sort path (opt-in): the radix passes (vg_sort.cu) order the
// points by their bucket, the top L <= 16 bits of the sort key (key >> bshift), and count
// the points of every bucket.  Here a one-block scan turns the counts into jobs (the
// non-empty buckets, in key order); a counting kernel finds every job's voxel count (the
// population of an occupancy bitmap over the bucket's low key bits) and largest key; a
// one-block scan turns the counts into each job's first row; and a persistent kernel
// reduces the buckets in shared memory without sorting them:
//   * the occupancy bitmap again (2^bshift <= 65536 bits, 8 KB);
//   * a prefix popcount over the bitmap gives every occupied key its rank, i.e. its row
//     within the bucket (the bucket's voxels in key order);
//   * every point adds its count and fixed-point offsets into its voxel's slot with
//     shared-memory atomics (32-bit sums plus a carry count per axis, so the totals are
//     exact integers: the rows are bit-identical to the sorted path's);
//   * the slots are finalised into rows from the job's first row on.
// No job waits for another.  Buckets of any size: points are streamed in chunks of
// kBmChunk, voxels in windows of kBmWindow slots.
//
// arXiv 2102.11084 Sec. II-C / Algorithm 1 sorts the (cell, point) table with a radix
// sort so that the points of each cell are contiguous, then reduces every cell.  Here the
// radix sort orders the cells by their top key bits only; inside a bucket the order of
// the cells is the order of the bits of the bitmap, and the points of a cell meet in its
// slot instead of in a contiguous run: the same cells, in the same order, with the same
// sums.
#include "vg_device.cuh"
#include "vg_internal.h"

namespace vg {
namespace {

constexpr unsigned kFull = 0xffffffffu;
// Geometry (build-time; the defaults are the measured best on the 50M map: 256 threads x 4
// blocks with 1792 slots, 128 x 6 with 1024 and 256 x 2 with 3584 were slower, and with
// the chained-scan wait taken out 256 x 4 was still slower than 512 x 2).
#ifndef VG_BM_THREADS
#define VG_BM_THREADS 512
#endif
#ifndef VG_BM_WINDOW
#define VG_BM_WINDOW 4096
#endif
#ifndef VG_BM_MINB
#define VG_BM_MINB 2
#endif
constexpr int kBmThreads = VG_BM_THREADS;
constexpr int kBmWarps = kBmThreads / 32;
constexpr int kBmItems = 16;                              // keys a thread holds per chunk
constexpr int kBmChunk = kBmThreads * kBmItems;           // points per chunk
#ifndef VG_BM_GROUP  // (2, 4 and 8 measured 1.41, 1.40 and 1.39 ms for the bucket stage)
#define VG_BM_GROUP 8
#endif
constexpr int kBmGroup = VG_BM_GROUP;                     // payload loads in flight
constexpr int kBmWords = 1 << (kBucketMaxBits - 5);       // bitmap words (bshift <= 16)
constexpr int kBmWindow = VG_BM_WINDOW;                   // voxel slots per window
constexpr int kBmWordsPerThread = kBmWords / kBmThreads;
constexpr uint32_t kCarryField = 10;                      // carry bits per axis
constexpr uint32_t kExactLimit = 1u << 21;                // points of a slot the carries hold

// Job table (bjob, kBucketSlots entries per array): first point at [0, S), points at
// [S, 2S), largest key at [2S, 3S), S = kBucketSlots.

// A job's descriptor: first point, points, bucket, first row, and the largest key of the
// job before it (frame marks).  Independent loads (the bucket comes from the job's own
// largest key).
struct JobDesc {
  uint32_t a, m, bucket, vbase, prev;
};
struct BmSmem {
  uint32_t bits[kBmWords];            // occupancy of the low key bits
  uint16_t rank[kBmWords];            // occupied keys before each word (exclusive)
  uint32_t cnt[kBmWindow];            // points per slot
  uint32_t lo[3][kBmWindow];          // per-axis sums of the biased offsets, mod 2^32
  uint32_t hi[kBmWindow];             // per-axis wrap counts, kCarryField bits each
  uint16_t vkey[kBmWindow];           // low key bits of every slot
  uint32_t tmp[kBmWarps];
  long long red[kBmWarps][4];
  JobDesc s_desc;                       // the job about to run
  uint32_t s_prev16, s_big;             // last slot key of the window; big-slot flag
};
// VG_BM_MINB blocks per SM: each takes this + 1 KB reserved of the SM's 228 KB.
static_assert((sizeof(BmSmem) + 1024) * VG_BM_MINB <= 228 * 1024, "bucket block shared memory");

// L2 prefetch of the 16-byte-aligned interior of [p, p + bytes).
__device__ __forceinline__ void prefetch_range(const void* p, size_t bytes) {
  const uintptr_t a = (reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15);
  const uintptr_t b = (reinterpret_cast<uintptr_t>(p) + bytes) & ~uintptr_t(15);
  if (b > a) prefetch_l2(reinterpret_cast<const void*>(a), static_cast<uint32_t>(b - a));
}

// One output row: voxel `key` (the full sort key) at row `cur`, plus the frame marks.
struct RowCtx {
  const FrameState* fs;
  uint32_t key_shift;
  int nframes;
  float o1[3];
  float leaf1;
};

__device__ __forceinline__ void write_row(const RowCtx& rc, const SegOut& out, uint32_t cur,
                                          uint32_t key, uint32_t prev_key, bool has_prev,
                                          bool last, const Acc& run, int* err) {
  const uint64_t local = key_local(key, rc.key_shift);
  if (int64_t(cur) >= out.cap) {
    set_error(err, kErrCapacity);
  } else {
    float o[3] = {rc.o1[0], rc.o1[1], rc.o1[2]};
    float leaf = rc.leaf1;
    if (rc.key_shift < 64) {
      const uint32_t f = key_frame(key, rc.key_shift);
      o[0] = rc.fs[f].origin[0];
      o[1] = rc.fs[f].origin[1];
      o[2] = rc.fs[f].origin[2];
      leaf = rc.fs[f].leaf;
    }
    float c[3];
    acc_centroid(local, run, o, leaf, leaf, c);
    out.keys[cur] = local;
    out.counts[cur] = run.n;
    out.centroids[3 * size_t(cur)] = c[0];
    out.centroids[3 * size_t(cur) + 1] = c[1];
    out.centroids[3 * size_t(cur) + 2] = c[2];
    if (out.sums) {
      out.sums[3 * size_t(cur)] = run.s[0];
      out.sums[3 * size_t(cur) + 1] = run.s[1];
      out.sums[3 * size_t(cur) + 2] = run.s[2];
    }
  }
  if (out.frame_offsets) {
    const uint32_t fk = key_frame(key, rc.key_shift);
    if (has_prev) {
      const uint32_t fp = key_frame(prev_key, rc.key_shift);
      for (uint32_t f = fp + 1; f <= fk; ++f) out.frame_offsets[f] = cur;
    }
    if (last)
      for (uint32_t f = fk + 1; f <= uint32_t(rc.nframes); ++f) out.frame_offsets[f] = cur + 1;
  }
  if (last) *out.num_voxels = int64_t(cur) + 1;
}

// ---- the jobs -------------------------------------------------------------------------

// One block: the non-empty buckets in key order become jobs (first point, points), in
// rounds of 16 consecutive buckets per thread (four 16-byte loads in flight), so that a
// thread writes consecutive jobs.
__global__ __launch_bounds__(1024) void bucket_scan_kernel(State* st, const uint32_t* __restrict__ bcount,
                                                           uint32_t* __restrict__ bjob) {
  __shared__ uint32_t tmp[32];
  if (!(st->narrow && st->bucket)) return;
  constexpr int kPer = 16;
  const int t = threadIdx.x;
  uint32_t* job_start = bjob;
  uint32_t* job_count = bjob + kBucketSlots;
  uint32_t base_e = 0, base_j = 0;
  for (int r0 = 0; r0 < kBucketSlots; r0 += kPer * 1024) {
    const uint4* c4 = reinterpret_cast<const uint4*>(bcount + r0 + kPer * t);
    uint32_t c[kPer];
#pragma unroll
    for (int q = 0; q < kPer / 4; ++q) {
      const uint4 v = c4[q];
      c[4 * q] = v.x;
      c[4 * q + 1] = v.y;
      c[4 * q + 2] = v.z;
      c[4 * q + 3] = v.w;
    }
    uint32_t sum = 0, nz = 0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      sum += c[q];
      nz += c[q] != 0;
    }
    uint32_t tot_e, tot_j;
    uint32_t run_e = base_e + block_excl_scan(sum, &tot_e, tmp);
    __syncthreads();
    uint32_t run_j = base_j + block_excl_scan(nz, &tot_j, tmp);
#pragma unroll
    for (int q = 0; q < kPer; ++q)
      if (c[q]) {
        job_start[run_j] = run_e;
        job_count[run_j] = c[q];
        ++run_j;
        run_e += c[q];
      }
    base_e += tot_e;
    base_j += tot_j;
    __syncthreads();
  }
  // the counts cover exactly the valid points, unless the call already failed before the
  // keys were written (bad frame offsets): then there is nothing to reduce
  if (t == 0) st->njobs = base_e == st->nitems ? base_j : 0u;
}

__device__ __forceinline__ JobDesc load_desc(const uint32_t* bjob, const uint32_t* vbase, int j,
                                             uint32_t bshift) {
  JobDesc d;
  d.a = bjob[j];
  d.m = bjob[kBucketSlots + j];
  d.bucket = bjob[2 * size_t(kBucketSlots) + j] >> bshift;
  d.vbase = vbase[j];
  d.prev = j > 0 ? bjob[2 * size_t(kBucketSlots) + j - 1] : 0u;
  return d;
}

// Rank of low key bits k16 among the bucket's occupied keys.
__device__ __forceinline__ uint32_t key_rank(const BmSmem& sm, uint32_t k16) {
  const uint32_t w = k16 >> 5;
  return uint32_t(sm.rank[w]) + __popc(sm.bits[w] & ((1u << (k16 & 31u)) - 1u));
}

// Exact biased sum of one axis of slot i: 32-bit sum plus the wrap count.
__device__ __forceinline__ long long slot_sum(const BmSmem& sm, int axis, int i) {
  const uint64_t carry = (sm.hi[i] >> (kCarryField * axis)) & ((1u << kCarryField) - 1u);
  return static_cast<long long>((carry << 32) | sm.lo[axis][i]);
}

// One job: the bucket's m points at [a, a + m), its rows from row vbase on; prev_last is
// the largest key of the job before it (frame marks).
__device__ __forceinline__ void bucket_job(BmSmem& sm, const uint32_t* __restrict__ K,
                                           const uint64_t* __restrict__ P, uint32_t a, uint32_t m,
                                           uint32_t bucket, uint32_t bshift, uint32_t vbase,
                                           uint32_t prev_last, bool last_job, const RowCtx& rc,
                                           const SegOut& out, int* err) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const uint32_t smask = (1u << bshift) - 1u;  // bshift <= 16
  const int nw = bshift >= 5 ? 1 << (bshift - 5) : 1;
  const bool resident = m <= uint32_t(kBmChunk);  // keys stay in registers
  for (int w = t; w < nw; w += kBmThreads) sm.bits[w] = 0;
  __syncthreads();

  // 1. occupancy bitmap
  uint32_t k16[kBmItems];
  for (uint32_t c0 = 0; c0 < m; c0 += kBmChunk) {
    // all loads first, then the atomics (so the loads overlap)
#pragma unroll
    for (int i = 0; i < kBmItems; ++i) {
      const uint32_t e = c0 + uint32_t(i) * kBmThreads + uint32_t(t);
      k16[i] = e < m ? (__ldcs(K + a + e) & smask) : kFull;
    }
#pragma unroll
    for (int i = 0; i < kBmItems; ++i)
      if (k16[i] != kFull) atomicOr(&sm.bits[k16[i] >> 5], 1u << (k16[i] & 31u));
  }
  __syncthreads();

  // 2. ranks: exclusive popcounts of the words, the voxel count, the largest key
  uint32_t pc[kBmWordsPerThread], mine = 0;
#pragma unroll
  for (int q = 0; q < kBmWordsPerThread; ++q) {
    const int w = kBmWordsPerThread * t + q;
    pc[q] = w < nw ? __popc(sm.bits[w]) : 0u;
    mine += pc[q];
  }
  uint32_t V;
  uint32_t run = block_excl_scan(mine, &V, sm.tmp);
#pragma unroll
  for (int q = 0; q < kBmWordsPerThread; ++q) {
    const int w = kBmWordsPerThread * t + q;
    if (w < nw) {
      sm.rank[w] = static_cast<uint16_t>(run);
      run += pc[q];
    }
  }
  __syncthreads();

  // 3. windows of kBmWindow voxel slots: accumulate, then finalise into rows
  for (uint32_t w0 = 0; w0 < V; w0 += kBmWindow) {
    const uint32_t wn = V - w0 < uint32_t(kBmWindow) ? V - w0 : uint32_t(kBmWindow);
    if (t == 0) sm.s_big = 0;
    for (uint32_t i = t; i < wn; i += kBmThreads) {
      sm.cnt[i] = 0;
      sm.lo[0][i] = 0;
      sm.lo[1][i] = 0;
      sm.lo[2][i] = 0;
      sm.hi[i] = 0;
    }
    // the keys of the window's slots, from the bitmap
    for (int w = t; w < nw; w += kBmThreads) {
      uint32_t b = sm.bits[w];
      uint32_t r = sm.rank[w];
      while (b) {
        const uint32_t bit = __ffs(static_cast<int>(b)) - 1;
        if (r >= w0 && r < w0 + wn) sm.vkey[r - w0] = static_cast<uint16_t>(uint32_t(w) * 32u + bit);
        b &= b - 1;
        ++r;
      }
    }
    __syncthreads();
    for (uint32_t c0 = 0; c0 < m; c0 += kBmChunk) {
      // in groups of kBmGroup items: the group's payload loads first, then its atomics
#pragma unroll
      for (int h = 0; h < kBmItems; h += kBmGroup) {
        uint64_t pl[kBmGroup];
        uint32_t sl[kBmGroup];
#pragma unroll
        for (int i = 0; i < kBmGroup; ++i) {
          const uint32_t e = c0 + uint32_t(h + i) * kBmThreads + uint32_t(t);
          sl[i] = kFull;
          pl[i] = 0;
          if (e < m) {
            const uint32_t k = resident ? k16[h + i] : (__ldcs(K + a + e) & smask);
            const uint32_t s = key_rank(sm, k) - w0;
            if (s < wn) {
              sl[i] = s;
              pl[i] = __ldcs(P + a + e);
            }
          }
        }
#pragma unroll
        for (int i = 0; i < kBmGroup; ++i) {
          if (sl[i] == kFull) continue;
          const uint32_t s = sl[i];
          // the point that fills a slot to kExactLimit flags the window for the exact pass
          if (atomicAdd(&sm.cnt[s], 1u) + 1u == kExactLimit) sm.s_big = 1u;
#pragma unroll
          for (int ax = 0; ax < 3; ++ax) {
            const uint32_t v = static_cast<uint32_t>(pl[i] >> (21 * ax)) & 0x1fffffu;
            const uint32_t old = atomicAdd(&sm.lo[ax][s], v);
            if (old + v < old) atomicAdd(&sm.hi[s], 1u << (kCarryField * ax));
          }
        }
      }
    }
    __syncthreads();
    // slots with kExactLimit points or more may have overflowed their carry fields: those
    // (only in clouds with millions of points in one voxel) are summed again exactly
    const bool exact_pass = sm.s_big != 0;
    for (uint32_t i = t; i < wn; i += kBmThreads) {
      const uint32_t n = sm.cnt[i];
      if (exact_pass && n >= kExactLimit) continue;  // written below
      Acc acc;
      acc.n = n;
      const long long bias = static_cast<long long>(n) * kQMin;
      acc.s[0] = slot_sum(sm, 0, int(i)) + bias;
      acc.s[1] = slot_sum(sm, 1, int(i)) + bias;
      acc.s[2] = slot_sum(sm, 2, int(i)) + bias;
      const uint32_t r = w0 + i;
      const uint32_t key = (bucket << bshift) | sm.vkey[i];
      const uint32_t prev_key =
          i > 0 ? ((bucket << bshift) | sm.vkey[i - 1])
                : (r > 0 ? ((bucket << bshift) | sm.s_prev16) : prev_last);
      write_row(rc, out, vbase + r, key, prev_key, vbase + r > 0, last_job && r + 1 == V, acc,
                err);
    }
    if (exact_pass) {
      for (uint32_t i = 0; i < wn; ++i) {
        if (sm.cnt[i] < kExactLimit) continue;  // (uniform: every thread reads the same slot)
        const uint32_t kk = sm.vkey[i];
        Acc part = acc_zero();
        for (uint32_t e = t; e < m; e += kBmThreads)
          if ((__ldcs(K + a + e) & smask) == kk) {
            const uint64_t p = __ldcs(P + a + e);
            part.s[0] += unpack_offset(p, 0);
            part.s[1] += unpack_offset(p, 1);
            part.s[2] += unpack_offset(p, 2);
          }
        // block sum of the three axes
        long long v3[3] = {part.s[0], part.s[1], part.s[2]};
#pragma unroll
        for (int ax = 0; ax < 3; ++ax)
#pragma unroll
          for (int off = 16; off; off >>= 1) v3[ax] += __shfl_xor_sync(kFull, v3[ax], off);
        __syncthreads();
        if (lane == 0)
#pragma unroll
          for (int ax = 0; ax < 3; ++ax) sm.red[warp][ax] = v3[ax];
        __syncthreads();
        if (t == 0) {
          Acc acc = acc_zero();
          acc.n = sm.cnt[i];
          for (int w = 0; w < kBmWarps; ++w) {
            acc.s[0] += sm.red[w][0];
            acc.s[1] += sm.red[w][1];
            acc.s[2] += sm.red[w][2];
          }
          const uint32_t r = w0 + i;
          const uint32_t key = (bucket << bshift) | kk;
          const uint32_t prev_key =
              i > 0 ? ((bucket << bshift) | sm.vkey[i - 1])
                    : (r > 0 ? ((bucket << bshift) | sm.s_prev16) : prev_last);
          write_row(rc, out, vbase + r, key, prev_key, vbase + r > 0, last_job && r + 1 == V,
                    acc, err);
        }
      }
    }
    __syncthreads();
    if (t == 0) sm.s_prev16 = sm.vkey[wn - 1];
    __syncthreads();
  }
}

// Voxels of every job: its bitmap's population (no accumulation), then the job's largest
// key.  Small blocks, many per SM: a job here is one pass over its keys.
constexpr int kCountThreads = 256;
__global__ __launch_bounds__(kCountThreads) void bucket_count_kernel(State* st, const uint32_t* k0,
                                                                     const uint32_t* k1,
                                                                     uint32_t* __restrict__ vox,
                                                                     uint32_t* __restrict__ bjob) {
  __shared__ uint32_t bits[kBmWords];
  __shared__ uint32_t s_sum[kCountThreads / 32];
  __shared__ int s_max[kCountThreads / 32];
  if (!(st->narrow && st->bucket)) return;
  const int njobs = static_cast<int>(st->njobs);
  const uint32_t* K = (pass_count(st) & 1) ? k1 : k0;
  const uint32_t bshift = st->bshift;
  const uint32_t smask = (1u << bshift) - 1u;
  const int nw = bshift >= 5 ? 1 << (bshift - 5) : 1;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int j = blockIdx.x; j < njobs; j += gridDim.x) {
    const uint32_t a = bjob[j], m = bjob[kBucketSlots + j];
    for (int w = t; w < nw; w += kCountThreads) bits[w] = 0;
    __syncthreads();
    for (uint32_t e0 = t; e0 < m; e0 += 4 * kCountThreads) {
      uint32_t k16[4];  // four loads in flight, then their atomics
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t e = e0 + uint32_t(q) * kCountThreads;
        k16[q] = e < m ? (__ldcs(K + a + e) & smask) : kFull;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (k16[q] != kFull) atomicOr(&bits[k16[q] >> 5], 1u << (k16[q] & 31u));
    }
    __syncthreads();
    uint32_t c = 0;
    int last = -1;  // largest occupied low key
    for (int w = t; w < nw; w += kCountThreads) {
      const uint32_t b = bits[w];
      c += __popc(b);
      if (b) last = w * 32 + 31 - __clz(static_cast<int>(b));
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      c += __shfl_xor_sync(kFull, c, off);
      last = max(last, __shfl_xor_sync(kFull, last, off));
    }
    if (lane == 0) {
      s_sum[warp] = c;
      s_max[warp] = last;
    }
    __syncthreads();
    if (t == 0) {
      uint32_t v = 0;
      int l = -1;
      for (int w = 0; w < kCountThreads / 32; ++w) {
        v += s_sum[w];
        l = max(l, s_max[w]);
      }
      vox[j] = v;
      bjob[2 * size_t(kBucketSlots) + j] = ((K[a] >> bshift) << bshift) | uint32_t(l);
    }
    __syncthreads();
  }
}

// One block: the jobs' voxel counts become their first rows (exclusive scan in place),
// 16 consecutive counts per thread per round.
__global__ __launch_bounds__(1024) void bucket_vscan_kernel(const State* st, uint32_t* vox) {
  __shared__ uint32_t tmp[32];
  if (!(st->narrow && st->bucket)) return;
  constexpr int kPer = 16;
  const int njobs = static_cast<int>(st->njobs);
  uint32_t carry = 0;
  for (int base = 0; base < njobs; base += kPer * 1024) {
    const int i0 = base + kPer * int(threadIdx.x);
    uint32_t c[kPer], sum = 0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      c[q] = i0 + q < njobs ? vox[i0 + q] : 0u;
      sum += c[q];
    }
    uint32_t total;
    uint32_t run = carry + block_excl_scan(sum, &total, tmp);
#pragma unroll
    for (int q = 0; q < kPer; ++q)
      if (i0 + q < njobs) {
        vox[i0 + q] = run;
        run += c[q];
      }
    carry += total;
    __syncthreads();
  }
}

// Jobs j = blockIdx.x + k * gridDim.x (no job waits for another: every job's first row is
// known).  Thread 0 keeps the next two descriptors in flight: the one after next is loaded
// while a job runs, the next one's rows start their way into L2 as that job starts.
__global__ __launch_bounds__(kBmThreads, VG_BM_MINB) void bucket_local_kernel(
    State* st, const FrameState* __restrict__ fs, int nframes, uint32_t* k0, uint64_t* p0,
    uint32_t* k1, uint64_t* p1, const uint32_t* __restrict__ vbase, uint32_t* bjob, SegOut out,
    int* err) {
  extern __shared__ __align__(128) unsigned char bm_smem[];
  BmSmem& sm = *reinterpret_cast<BmSmem*>(bm_smem);
  if (!(st->narrow && st->bucket)) return;
  const int njobs = static_cast<int>(st->njobs);
  const int G = static_cast<int>(gridDim.x);
  const int j0 = static_cast<int>(blockIdx.x);
  if (j0 >= njobs) return;
  const bool odd = pass_count(st) & 1;
  const uint32_t* K = odd ? k1 : k0;
  const uint64_t* P = odd ? p1 : p0;
  const uint32_t bshift = st->bshift;
  RowCtx rc{fs, st->key_shift, nframes, {fs[0].origin[0], fs[0].origin[1], fs[0].origin[2]},
            fs[0].leaf};
  const int t = threadIdx.x;
  JobDesc d1{}, d2{};  // thread 0: the next job's descriptor, and the one after
  if (t == 0) {
    sm.s_desc = load_desc(bjob, vbase, j0, bshift);
    if (j0 + G < njobs) d1 = load_desc(bjob, vbase, j0 + G, bshift);
  }
  __syncthreads();
  for (int j = j0; j < njobs; j += G) {
    const JobDesc d = sm.s_desc;
    __syncthreads();  // (the slot is refilled at the end of this job)
    if (t == 0) {
      if (j + G < njobs) {
        prefetch_range(K + d1.a, size_t(d1.m) * sizeof(uint32_t));
        prefetch_range(P + d1.a, size_t(d1.m) * sizeof(uint64_t));
      }
      if (j + 2 * G < njobs) d2 = load_desc(bjob, vbase, j + 2 * G, bshift);
    }
    bucket_job(sm, K, P, d.a, d.m, d.bucket, bshift, d.vbase, d.prev, j + 1 == njobs, rc, out,
               err);
    if (t == 0) {
      sm.s_desc = d1;
      d1 = d2;
    }
    __syncthreads();
  }
}

}  // namespace

void warm_bucket_config() {
  persistent_grid(reinterpret_cast<const void*>(bucket_local_kernel), kBmThreads, sizeof(BmSmem),
                  1);
  persistent_grid(reinterpret_cast<const void*>(bucket_count_kernel), kCountThreads, 0, 1);
}

cudaError_t launch_bucket_tail(State* st, const FrameState* fs, int nframes,
                               const NarrowBuffers& nb, const uint32_t* bcount, uint32_t* bstat,
                               uint32_t* bjob, int64_t n_max, const SegOut& out,
                               uint32_t spin_limit, int* err, cudaStream_t stream) {
  (void)spin_limit;  // no job of the bucket tail waits for another
  if (n_max == 0) return cudaSuccess;
  bucket_scan_kernel<<<1, 1024, 0, stream>>>(st, bcount, bjob);
  // bstat holds the jobs' voxel counts, then (scanned in place) their first rows
  const int cgrid = persistent_grid(reinterpret_cast<const void*>(bucket_count_kernel),
                                    kCountThreads, 0, kBucketSlots);
  bucket_count_kernel<<<cgrid, kCountThreads, 0, stream>>>(st, nb.k0, nb.k1, bstat, bjob);
  bucket_vscan_kernel<<<1, 1024, 0, stream>>>(st, bstat);
  const int grid = persistent_grid(reinterpret_cast<const void*>(bucket_local_kernel),
                                   kBmThreads, sizeof(BmSmem), kBucketSlots);
  bucket_local_kernel<<<grid, kBmThreads, sizeof(BmSmem), stream>>>(
      st, fs, nframes, nb.k0, nb.p0, nb.k1, nb.p1, bstat, bjob, out, err);
  return cudaGetLastError();
}

}  // namespace vg
