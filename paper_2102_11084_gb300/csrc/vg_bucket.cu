// Bucket tail of the narrow sort path: the radix passes (vg_sort.cu) order the points by
// their bucket, the top L <= 16 bits of the sort key (key >> bshift), and count the
// points of every bucket.  Here a one-block scan turns the counts into jobs (the
// non-empty buckets, in key order), and a persistent kernel takes the jobs in ticket
// order: it sorts each bucket by the low bshift <= 16 key bits in shared memory and
// reduces the sorted runs into voxels, as the segmented reduction does.
//
// arXiv 2102.11084 Sec. II-C / Algorithm 1 sorts the (cell, point) table with a radix
// sort so that the points of each cell are contiguous and then reduces every cell.  A
// radix sort may split its digits between passes over the whole table and passes inside
// independent key ranges (an MSD step followed by per-range LSD passes gives the same
// order), so this is still that sort: the ranges here are buckets small enough for one
// block's shared memory, which saves the low digits' trips through HBM and the separate
// reduction kernels.  Centroid sums are exact integers, so the order of equal keys does
// not change any output bit.
//
// Jobs publish their voxel counts through a chained scan over the ticket order (bounded
// waits, as everywhere else).  A bucket larger than one block's capacity (kLocalCap
// points) is sorted through global scratch in chunks, with the same ranking code.
#include "vg_device.cuh"
#include "vg_internal.h"

namespace vg {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kLW = kLocalThreads / 32;

// Per-job words of the bjob array.
constexpr int kJobStart = 0, kJobCount = 1, kJobLast = 2;

struct LocalSmem {
  uint32_t words[kLocalCap];             // sort words (key16 << 16 | local index); scratch
  unsigned long long pay[kLocalCap];     // payloads by local index
  union {
    uint16_t whist[kLW][kRadix];         // per-warp digit counts (sort passes)
    uint16_t hpos[kLocalCap + 2];        // run heads (reduction)
  } u;
  uint16_t cnt[kRadix];                  // digit counts, then (in place) digit starts
  uint32_t tmp[kLW];
  int s_job, s_next;
  uint32_t s_vbase, s_prev_last, s_v;
  uint32_t s_a, s_m, s_bucket, s_na, s_nm, s_nbucket;  // current and next job descriptor
};
// Two blocks per SM: 2 x (this + 1 KB reserved) within the SM's 228 KB.
static_assert(sizeof(LocalSmem) + 1024 <= 228 * 1024 / 2, "bucket block shared memory");

__device__ __forceinline__ void cp_async8(void* smem, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(smem)), "l"(g)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// L2 prefetch of the 16-byte-aligned interior of [p, p + bytes).
__device__ __forceinline__ void prefetch_range(const void* p, size_t bytes) {
  const uintptr_t a = (reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15);
  const uintptr_t b = (reinterpret_cast<uintptr_t>(p) + bytes) & ~uintptr_t(15);
  if (b > a) prefetch_l2(reinterpret_cast<const void*>(a), static_cast<uint32_t>(b - a));
}

// Stable rank of the block's items by the 8-bit digit (x >> sh) & 255.  Items are
// warp-striped (item j of lane l in warp w is element w*32*ipt + j*32 + l of the block's
// sequence); bit j of `valid` says item j exists.  On return rank[j] = number of earlier
// elements with the same digit, and cnt[d] (shared) = the block's count of digit d
// (threads < 256 write it; at most kLocalCap).  Contains __syncthreads.
__device__ __forceinline__ void rank_items(const uint32_t (&x)[kLocalItems], uint32_t sh,
                                           uint32_t valid, int ipt, uint16_t (*whist)[kRadix],
                                           uint32_t (&rank)[kLocalItems], uint16_t* cnt) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int d = lane; d < kRadix; d += 32) whist[warp][d] = 0;
  __syncwarp();
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int j = 0; j < kLocalItems; ++j) {
    if (j < ipt) {
      const bool ok = (valid >> j) & 1u;
      const uint32_t d = (x[j] >> sh) & (kRadix - 1);
      uint32_t peers = __ballot_sync(kFull, ok);
#pragma unroll
      for (int b = 0; b < kRadixBits; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t bal = __ballot_sync(kFull, bit);
        peers &= bit ? bal : ~bal;
      }
      const uint32_t lower = peers & lt;
      uint32_t old = 0;
      if (ok) old = whist[warp][d];
      __syncwarp();
      if (ok && lower == 0) whist[warp][d] = static_cast<uint16_t>(old + __popc(peers));
      __syncwarp();
      rank[j] = old + __popc(lower);
    }
  }
  __syncthreads();
  if (t < kRadix) {
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kLW; ++w) {
      const uint32_t c = whist[w][t];
      whist[w][t] = static_cast<uint16_t>(run);
      run += c;
    }
    cnt[t] = static_cast<uint16_t>(run);
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kLocalItems; ++j)
    if (j < ipt && ((valid >> j) & 1u)) rank[j] += whist[warp][(x[j] >> sh) & (kRadix - 1)];
}

// Exclusive scan of cnt[0..256) into dst (may be cnt itself), over the whole block.
template <typename T>
__device__ __forceinline__ void digit_starts(const T* cnt, T* dst, uint32_t* tmp) {
  const int t = threadIdx.x;
  uint32_t total;
  const uint32_t e = block_excl_scan(t < kRadix ? uint32_t(cnt[t]) : 0u, &total, tmp);
  if (t < kRadix) dst[t] = static_cast<T>(e);
  __syncthreads();
}

// Sum of a block's Acc values (all threads receive it).  Contains __syncthreads.
__device__ __forceinline__ Acc block_sum_acc(Acc a, long long (*red)[4]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long v[4] = {a.s[0], a.s[1], a.s[2], static_cast<long long>(a.n)};
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int off = 16; off; off >>= 1) v[k] += __shfl_xor_sync(kFull, v[k], off);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 4; ++k) red[warp][k] = v[k];
  __syncthreads();
  Acc r = acc_zero();
  for (int w = 0; w < kLW; ++w) {
    r.s[0] += red[w][0];
    r.s[1] += red[w][1];
    r.s[2] += red[w][2];
    r.n += static_cast<uint32_t>(red[w][3]);
  }
  return r;
}

__device__ __forceinline__ void acc_add_payload(Acc& a, uint64_t w) {
  a.s[0] += unpack_offset(w, 0);
  a.s[1] += unpack_offset(w, 1);
  a.s[2] += unpack_offset(w, 2);
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

// Warp-wide chained-scan wait over the jobs before j: every round trip loads 32
// predecessors' status words (a wave of jobs publishes its aggregates at about the same
// time, so a one-word walk would pay one L2 round trip per job).  Returns the exclusive
// prefix of job j (the same in every lane).  Bounded like every other wait.
__device__ __forceinline__ uint32_t warp_lookback(const uint32_t* status, int j,
                                                  uint32_t spin_limit, int* err) {
  const int lane = threadIdx.x & 31;
  uint32_t excl = 0, spins = 0;
  int base = j - 1;
  while (base >= 0) {
    const int idx = base - lane;
    const uint32_t w = idx >= 0 ? ld_relaxed(status + idx) : kFlagPrefix;  // before job 0: 0
    const uint32_t f = w & ~kValueMask;
    const uint32_t notready = __ballot_sync(kFull, f == 0);
    const uint32_t prefix = __ballot_sync(kFull, f == kFlagPrefix);
    const int first_nr = notready ? __ffs(static_cast<int>(notready)) - 1 : 32;
    const int first_p = prefix ? __ffs(static_cast<int>(prefix)) - 1 : 32;
    const bool done = first_p < first_nr;
    const int take = done ? first_p + 1 : first_nr;
    uint32_t v = lane < take ? (w & kValueMask) : 0u;
#pragma unroll
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    excl += v;
    if (done) break;
    base -= take;
    if (take == 0) {
      if (++spins > spin_limit) {
        if (lane == 0) set_error(err, kErrTimeout);
        break;
      }
      if (spins > 64) __nanosleep(64);
    }
  }
  return excl;
}

// Warp 0: publishes `v` voxels for job j (its aggregate, unless a pre-pass already did,
// after its largest key), waits for the rows before it, publishes its prefix.  Returns
// the rows before it; *prev_last = the largest key of job j - 1.
__device__ __forceinline__ uint32_t publish_job(uint32_t* bstat, uint32_t* bjob, int j, uint32_t v,
                                                bool publish_aggregate, uint32_t last_key,
                                                uint32_t spins, int* err, uint32_t* prev_last) {
  const int lane = threadIdx.x & 31;
  if (publish_aggregate && lane == 0) {
    bjob[3 * size_t(j) + kJobLast] = last_key;
    __threadfence();
    st_relaxed(bstat + j, (j == 0 ? kFlagPrefix : kFlagAggregate) | v);
  }
  if (j == 0) {
    if (lane == 0 && !publish_aggregate) st_relaxed(bstat, kFlagPrefix | v);
    return 0;
  }
  const uint32_t excl = warp_lookback(bstat, j, spins, err);
  if (lane == 0) {
    st_relaxed(bstat + j, kFlagPrefix | ((excl + v) & kValueMask));
    __threadfence();
    *prev_last = ld_relaxed(bjob + 3 * size_t(j - 1) + kJobLast);
  }
  return excl;
}

// Thread 0, once the current job's prefix is out: the next ticket and its descriptor,
// whose rows start their way into L2 while this job reduces (taken any earlier, the
// ticket would hold up every later job's look-back for a whole job).
__device__ __forceinline__ void take_next(LocalSmem& sm, uint32_t* job_ctr, const uint32_t* K,
                                          const uint64_t* P, const uint32_t* bjob, int njobs,
                                          uint32_t bshift) {
  const int nx = static_cast<int>(atomicAdd(job_ctr, 1u));
  sm.s_next = nx;
  if (nx < njobs) {
    const uint32_t na = bjob[3 * size_t(nx) + kJobStart];
    const uint32_t nm = bjob[3 * size_t(nx) + kJobCount];
    prefetch_range(K + na, size_t(nm) * sizeof(uint32_t));
    prefetch_range(P + na, size_t(nm) * sizeof(uint64_t));
    sm.s_na = na;
    sm.s_nm = nm;
    sm.s_nbucket = K[na] >> bshift;
  }
}

// ---- the jobs -------------------------------------------------------------------------

__global__ __launch_bounds__(1024) void bucket_scan_kernel(State* st, const uint32_t* __restrict__ bcount,
                                                           uint32_t* __restrict__ bjob) {
  __shared__ uint32_t tmp[32];
  __shared__ uint32_t smax[32];
  if (!(st->narrow && st->bucket)) return;
  constexpr int kPer = kBucketSlots / 1024;
  const int t = threadIdx.x;
  const uint4* c4 = reinterpret_cast<const uint4*>(bcount + size_t(t) * kPer);
  uint32_t sum = 0, nz = 0, mx = 0;
#pragma unroll 4
  for (int k = 0; k < kPer / 4; ++k) {
    const uint4 v = c4[k];
    sum += v.x + v.y + v.z + v.w;
    nz += (v.x != 0) + (v.y != 0) + (v.z != 0) + (v.w != 0);
    mx = max(max(mx, max(v.x, v.y)), max(v.z, v.w));
  }
  uint32_t nbig = 0;
  for (int k = 0; k < kPer / 4; ++k) {
    const uint4 v = c4[k];
    nbig += (v.x > uint32_t(kLocalCap)) + (v.y > uint32_t(kLocalCap)) +
            (v.z > uint32_t(kLocalCap)) + (v.w > uint32_t(kLocalCap));
  }
  uint32_t tot_e, tot_j, tot_b;
  uint32_t run_e = block_excl_scan(sum, &tot_e, tmp);
  __syncthreads();
  uint32_t run_j = block_excl_scan(nz, &tot_j, tmp);
  __syncthreads();
  uint32_t run_b = block_excl_scan(nbig, &tot_b, tmp);
  uint32_t* big = bjob + 3 * size_t(kBucketSlots);
#pragma unroll
  for (int off = 16; off; off >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, off));
  if ((t & 31) == 0) smax[t >> 5] = mx;
  // The counts cover exactly the valid points, unless the call already failed before the
  // keys were written (bad frame offsets): then there is nothing to reduce.
  const bool consistent = tot_e == st->nitems;
  for (int k = 0; consistent && k < kPer / 4; ++k) {
    const uint4 v = c4[k];
    const uint32_t c[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (c[q]) {
        bjob[3 * size_t(run_j) + kJobStart] = run_e;
        bjob[3 * size_t(run_j) + kJobCount] = c[q];
        if (c[q] > uint32_t(kLocalCap)) big[run_b++] = run_j;
        ++run_j;
        run_e += c[q];
      }
  }
  __syncthreads();
  if (t == 0) {
    uint32_t m = 0;
    for (int w = 0; w < 32; ++w) m = max(m, smax[w]);
    st->njobs = consistent ? tot_j : 0u;
    st->nbig = consistent ? tot_b : 0u;
    st->bmax = m;
  }
}

// Small job: the bucket's m <= kLocalCap points sorted and reduced in shared memory.
__device__ __forceinline__ void small_job(LocalSmem& sm, const uint32_t* __restrict__ K,
                                          const uint64_t* __restrict__ P, uint32_t a, uint32_t m,
                                          uint32_t bucket, uint32_t bshift, int j, int njobs,
                                          uint32_t* bstat, uint32_t* bjob, uint32_t* job_ctr,
                                          const RowCtx& rc, const SegOut& out, uint32_t spins,
                                          int* err) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int ipt = static_cast<int>((m + kLocalThreads - 1) / kLocalThreads);
  const uint32_t smask = bshift >= 32 ? kFull : ((1u << bshift) - 1u);
  uint32_t w[kLocalItems];
  uint32_t valid = 0;
  const uint32_t ebase = uint32_t(warp) * 32u * uint32_t(ipt) + uint32_t(lane);
#pragma unroll
  for (int j2 = 0; j2 < kLocalItems; ++j2) {
    w[j2] = 0;
    if (j2 < ipt) {
      const uint32_t e = ebase + uint32_t(j2) * 32u;
      if (e < m) {
        cp_async8(&sm.pay[e], P + a + e);
        w[j2] = ((__ldcs(K + a + e) & smask) << 16) | e;
        valid |= 1u << j2;
      }
    }
  }
  const int npl = bshift == 0 ? 0 : (bshift <= 8 ? 1 : 2);
  for (int q = 0; q < npl; ++q) {
    const uint32_t sh = 16u + 8u * uint32_t(q);
    uint32_t rank[kLocalItems];
    rank_items(w, sh, valid, ipt, sm.u.whist, rank, sm.cnt);
    digit_starts(sm.cnt, sm.cnt, sm.tmp);
#pragma unroll
    for (int j2 = 0; j2 < kLocalItems; ++j2)
      if (j2 < ipt && ((valid >> j2) & 1u))
        sm.words[sm.cnt[(w[j2] >> sh) & (kRadix - 1)] + rank[j2]] = w[j2];
    __syncthreads();
    if (q + 1 < npl) {
#pragma unroll
      for (int j2 = 0; j2 < kLocalItems; ++j2)
        if (j2 < ipt && ((valid >> j2) & 1u)) w[j2] = sm.words[ebase + uint32_t(j2) * 32u];
    }
  }
  if (npl == 0) {
#pragma unroll
    for (int j2 = 0; j2 < kLocalItems; ++j2)
      if (j2 < ipt && ((valid >> j2) & 1u)) sm.words[ebase + uint32_t(j2) * 32u] = w[j2];
  }
  cp_async_wait_all();
  __syncthreads();

  // run heads over blocked positions [t*ipt, t*ipt + ipt)
  const uint32_t p0 = uint32_t(t) * uint32_t(ipt);
  uint32_t hmask = 0, hc = 0;
#pragma unroll
  for (int j2 = 0; j2 < kLocalItems; ++j2) {
    const uint32_t p = p0 + uint32_t(j2);
    if (j2 < ipt && p < m) {
      const bool head = p == 0 || (sm.words[p] >> 16) != (sm.words[p - 1] >> 16);
      hmask |= uint32_t(head) << j2;
      hc += head;
    }
  }
  uint32_t V;
  uint32_t r = block_excl_scan(hc, &V, sm.tmp);
#pragma unroll
  for (int j2 = 0; j2 < kLocalItems; ++j2)
    if ((hmask >> j2) & 1u) sm.u.hpos[r++] = static_cast<uint16_t>(p0 + uint32_t(j2));
  if (warp == 0) {
    const uint32_t last_key = (bucket << bshift) | (sm.words[m - 1] >> 16);
    uint32_t prev_last = 0;
    const uint32_t vb = publish_job(bstat, bjob, j, V, true, last_key, spins, err, &prev_last);
    if (lane == 0) {
      sm.u.hpos[V] = static_cast<uint16_t>(m);
      sm.s_vbase = vb;
      sm.s_prev_last = prev_last;
      take_next(sm, job_ctr, K, P, bjob, njobs, bshift);
    }
  }
  __syncthreads();
  const uint32_t vbase = sm.s_vbase;
  const bool last_job = j + 1 == njobs;
  for (uint32_t v = t; v < V; v += kLocalThreads) {
    const uint32_t e0 = sm.u.hpos[v], e1 = sm.u.hpos[v + 1];
    const uint32_t key = (bucket << bshift) | (sm.words[e0] >> 16);
    Acc run = acc_zero();
    run.n = e1 - e0;
    for (uint32_t e = e0; e < e1; ++e) acc_add_payload(run, sm.pay[sm.words[e] & 0xffffu]);
    const uint32_t cur = vbase + v;
    const uint32_t prev_key = v > 0 ? ((bucket << bshift) | (sm.words[e0 - 1] >> 16)) : sm.s_prev_last;
    write_row(rc, out, cur, key, prev_key, cur > 0, last_job && v + 1 == V, run, err);
  }
  __syncthreads();
}

// Rows of a large job after large_sort: sorted keys and payloads, and the run heads.
struct LargeRows {
  uint32_t* keys;
  uint64_t* pay;
  uint32_t* heads;
};
__device__ __forceinline__ LargeRows large_rows(uint32_t* K, uint64_t* P, uint32_t* K2,
                                                uint64_t* P2, uint32_t bshift) {
  // one on-chip digit pass leaves the rows in the other buffer; zero or two in this one
  const bool moved = bshift != 0 && bshift <= 8;
  return moved ? LargeRows{K2, P2, K} : LargeRows{K, P, K2};
}

// Large job, pre-pass: m > kLocalCap points, sorted through the other ping-pong buffer in
// chunks of kLocalCap (stable LSD passes on the low digits, the same ranking as on chip);
// the run heads go to the free key buffer and the voxel count is published as the job's
// chained-scan aggregate before the main kernel starts, so no later job ever waits for a
// large one's sort.
__device__ void large_sort(LocalSmem& sm, uint32_t* K, uint64_t* P, uint32_t* K2, uint64_t* P2,
                           uint32_t a, uint32_t m, uint32_t bucket, uint32_t bshift, int j,
                           uint32_t* bstat, uint32_t* bjob) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const uint32_t smask = bshift >= 32 ? kFull : ((1u << bshift) - 1u);
  const int npl = bshift == 0 ? 0 : (bshift <= 8 ? 1 : 2);
  uint32_t* hist = sm.words;              // [2][256]
  uint32_t* base = sm.words + 2 * kRadix;  // [2][256]
  uint32_t* runc = sm.words + 4 * kRadix;  // [256]
  uint16_t* cnt = sm.cnt;
  for (int d = t; d < 2 * kRadix; d += kLocalThreads) hist[d] = 0;
  __syncthreads();
  for (uint32_t e = t; e < m; e += kLocalThreads) {
    const uint32_t k16 = K[a + e] & smask;
    atomicAdd(&hist[k16 & (kRadix - 1)], 1u);
    if (npl == 2) atomicAdd(&hist[kRadix + (k16 >> 8)], 1u);
  }
  __syncthreads();
  digit_starts(hist, base, sm.tmp);
  digit_starts(hist + kRadix, base + kRadix, sm.tmp);
  uint32_t* sk = K;
  uint64_t* sp = P;
  uint32_t* dk = K2;
  uint64_t* dp = P2;
  for (int q = 0; q < npl; ++q) {
    if (t < kRadix) runc[t] = 0;
    __syncthreads();
    for (uint32_t c0 = 0; c0 < m; c0 += kLocalCap) {
      const uint32_t mc = m - c0 < uint32_t(kLocalCap) ? m - c0 : uint32_t(kLocalCap);
      const int ipt = static_cast<int>((mc + kLocalThreads - 1) / kLocalThreads);
      const uint32_t ebase = uint32_t(warp) * 32u * uint32_t(ipt) + uint32_t(lane);
      uint32_t key[kLocalItems], rank[kLocalItems];
      uint32_t valid = 0;
#pragma unroll
      for (int j2 = 0; j2 < kLocalItems; ++j2) {
        key[j2] = 0;
        if (j2 < ipt) {
          const uint32_t e = ebase + uint32_t(j2) * 32u;
          if (e < mc) {
            cp_async8(&sm.pay[e], sp + a + c0 + e);
            key[j2] = sk[a + c0 + e] & smask;  // the bits above are the job's bucket
            valid |= 1u << j2;
          }
        }
      }
      const uint32_t sh = 8u * uint32_t(q);
      rank_items(key, sh, valid, ipt, sm.u.whist, rank, cnt);
      cp_async_wait_all();
      __syncthreads();
#pragma unroll
      for (int j2 = 0; j2 < kLocalItems; ++j2)
        if (j2 < ipt && ((valid >> j2) & 1u)) {
          const uint32_t d = (key[j2] >> sh) & (kRadix - 1);
          const uint32_t g = base[q * kRadix + d] + runc[d] + rank[j2];
          dk[a + g] = (bucket << bshift) | key[j2];
          dp[a + g] = sm.pay[ebase + uint32_t(j2) * 32u];
        }
      __syncthreads();
      if (t < kRadix) runc[t] += cnt[t];
      __syncthreads();
    }
    uint32_t* xk = sk;
    uint64_t* xp = sp;
    sk = dk;
    sp = dp;
    dk = xk;
    dp = xp;
  }
  // sorted rows in (sk, sp); dk is free scratch for the run heads
  uint32_t V = 0;
  for (uint32_t c0 = 0; c0 < m; c0 += kLocalCap) {
    const uint32_t mc = m - c0 < uint32_t(kLocalCap) ? m - c0 : uint32_t(kLocalCap);
    const int ipt = static_cast<int>((mc + kLocalThreads - 1) / kLocalThreads);
    const uint32_t p0 = c0 + uint32_t(t) * uint32_t(ipt);
    uint32_t hmask = 0, hc = 0;
#pragma unroll
    for (int j2 = 0; j2 < kLocalItems; ++j2) {
      const uint32_t p = p0 + uint32_t(j2);
      if (j2 < ipt && p < c0 + mc) {
        const bool head = p == 0 || sk[a + p] != sk[a + p - 1];
        hmask |= uint32_t(head) << j2;
        hc += head;
      }
    }
    uint32_t tot;
    uint32_t r = V + block_excl_scan(hc, &tot, sm.tmp);
#pragma unroll
    for (int j2 = 0; j2 < kLocalItems; ++j2)
      if ((hmask >> j2) & 1u) dk[a + r++] = p0 + uint32_t(j2);
    V += tot;
    __syncthreads();
  }
  if (t == 0) {
    bjob[3 * size_t(j) + kJobLast] = sk[a + m - 1];
    st_relaxed(bstat + j, kFlagAggregate | (V & kValueMask));
  }
  __syncthreads();
}

// Large job, main kernel: the rows before it from the chained scan, then its voxels from
// the sorted rows in global memory (one voxel per thread; a single voxel block-wide).
__device__ __noinline__ void large_reduce(LocalSmem& sm, uint32_t* K, uint64_t* P, uint32_t* K2,
                                          uint64_t* P2, uint32_t a, uint32_t m, uint32_t bshift,
                                          int j, int njobs, uint32_t* bstat, uint32_t* bjob,
                                          uint32_t* job_ctr, const RowCtx& rc, const SegOut& out,
                                          uint32_t spins, int* err) {
  const int t = threadIdx.x;
  const LargeRows R = large_rows(K, P, K2, P2, bshift);
  const uint32_t* sk = R.keys;
  const uint64_t* sp = R.pay;
  const uint32_t* dk = R.heads;
  if (t < 32) {
    const uint32_t V = ld_relaxed(bstat + j) & kValueMask;  // the pre-pass's aggregate
    uint32_t prev_last = 0;
    const uint32_t vb = publish_job(bstat, bjob, j, V, false, 0u, spins, err, &prev_last);
    if (t == 0) {
      sm.s_vbase = vb;
      sm.s_prev_last = prev_last;
      sm.s_v = V;
      take_next(sm, job_ctr, K, P, bjob, njobs, bshift);
    }
  }
  __syncthreads();
  const uint32_t vbase = sm.s_vbase, V = sm.s_v;
  const bool last_job = j + 1 == njobs;
  if (V == 1) {  // one voxel: a block-wide sum
    Acc part = acc_zero();
    for (uint32_t e = t; e < m; e += kLocalThreads) acc_add_payload(part, sp[a + e]);
    part.n = 0;
    Acc run = block_sum_acc(part, reinterpret_cast<long long (*)[4]>(&sm.u));
    run.n = m;
    if (t == 0) write_row(rc, out, vbase, sk[a], sm.s_prev_last, vbase > 0, last_job, run, err);
  } else {
    for (uint32_t v = t; v < V; v += kLocalThreads) {
      const uint32_t e0 = dk[a + v], e1 = v + 1 < V ? dk[a + v + 1] : m;
      Acc run = acc_zero();
      run.n = e1 - e0;
      for (uint32_t e = e0; e < e1; ++e) acc_add_payload(run, sp[a + e]);
      const uint32_t cur = vbase + v;
      const uint32_t prev_key = v > 0 ? sk[a + e0 - 1] : sm.s_prev_last;
      write_row(rc, out, cur, sk[a + e0], prev_key, cur > 0, last_job && v + 1 == V, run, err);
    }
  }
  __syncthreads();
}


__global__ __launch_bounds__(kLocalThreads, 2) void bucket_local_kernel(
    State* st, const FrameState* __restrict__ fs, int nframes, uint32_t* k0, uint64_t* p0,
    uint32_t* k1, uint64_t* p1, uint32_t* bstat, uint32_t* bjob, SegOut out, uint32_t spins,
    int* err) {
  extern __shared__ __align__(128) unsigned char local_smem[];
  LocalSmem& sm = *reinterpret_cast<LocalSmem*>(local_smem);
  if (!(st->narrow && st->bucket)) return;
  const int njobs = static_cast<int>(st->njobs);
  if (njobs == 0) return;
  const bool odd = pass_count(st) & 1;
  uint32_t* K = odd ? k1 : k0;
  uint64_t* P = odd ? p1 : p0;
  uint32_t* K2 = odd ? k0 : k1;
  uint64_t* P2 = odd ? p0 : p1;
  const uint32_t bshift = st->bshift;
  RowCtx rc{fs, st->key_shift, nframes, {fs[0].origin[0], fs[0].origin[1], fs[0].origin[2]},
            fs[0].leaf};
  const int t = threadIdx.x;
  if (t == 0) {
    take_next(sm, &st->job_ctr, K, P, bjob, njobs, bshift);
    sm.s_job = sm.s_next;
  }
  __syncthreads();
  for (;;) {
    const int j = sm.s_job;
    if (j >= njobs) break;
    const uint32_t a = sm.s_na, m = sm.s_nm, bucket = sm.s_nbucket;
    __syncthreads();  // (the descriptor slots are refilled by this job's take_next)
    if (m <= uint32_t(kLocalCap))
      small_job(sm, K, P, a, m, bucket, bshift, j, njobs, bstat, bjob, &st->job_ctr, rc, out,
                spins, err);
    else
      large_reduce(sm, K, P, K2, P2, a, m, bshift, j, njobs, bstat, bjob, &st->job_ctr, rc, out,
                   spins, err);
    if (t == 0) sm.s_job = sm.s_next;
    __syncthreads();
  }
}

// Pre-pass over the large jobs (in any order: each publishes only its own aggregate).
__global__ __launch_bounds__(kLocalThreads, 2) void bucket_large_kernel(State* st, uint32_t* k0,
                                                                        uint64_t* p0, uint32_t* k1,
                                                                        uint64_t* p1,
                                                                        uint32_t* bstat,
                                                                        uint32_t* bjob) {
  extern __shared__ __align__(128) unsigned char local_smem[];
  LocalSmem& sm = *reinterpret_cast<LocalSmem*>(local_smem);
  if (!(st->narrow && st->bucket)) return;
  const int nbig = static_cast<int>(st->nbig);
  if (nbig == 0) return;
  const bool odd = pass_count(st) & 1;
  uint32_t* K = odd ? k1 : k0;
  uint64_t* P = odd ? p1 : p0;
  uint32_t* K2 = odd ? k0 : k1;
  uint64_t* P2 = odd ? p0 : p1;
  const uint32_t bshift = st->bshift;
  const uint32_t* big = bjob + 3 * size_t(kBucketSlots);
  for (;;) {
    if (threadIdx.x == 0) sm.s_job = static_cast<int>(atomicAdd(&st->big_ctr, 1u));
    __syncthreads();
    const int b = sm.s_job;
    __syncthreads();
    if (b >= nbig) break;
    const int j = static_cast<int>(big[b]);
    const uint32_t a = bjob[3 * size_t(j) + kJobStart];
    const uint32_t m = bjob[3 * size_t(j) + kJobCount];
    large_sort(sm, K, P, K2, P2, a, m, K[a] >> bshift, bshift, j, bstat, bjob);
  }
}

}  // namespace

void warm_bucket_config() {
  persistent_grid(reinterpret_cast<const void*>(bucket_local_kernel), kLocalThreads,
                  sizeof(LocalSmem), 1);
  persistent_grid(reinterpret_cast<const void*>(bucket_large_kernel), kLocalThreads,
                  sizeof(LocalSmem), 1);
}

cudaError_t launch_bucket_tail(State* st, const FrameState* fs, int nframes,
                               const NarrowBuffers& nb, const uint32_t* bcount, uint32_t* bstat,
                               uint32_t* bjob, int64_t n_max, const SegOut& out,
                               uint32_t spin_limit, int* err, cudaStream_t stream) {
  if (n_max == 0) return cudaSuccess;
  bucket_scan_kernel<<<1, 1024, 0, stream>>>(st, bcount, bjob);
  const int lgrid = persistent_grid(reinterpret_cast<const void*>(bucket_large_kernel),
                                    kLocalThreads, sizeof(LocalSmem), kBucketSlots);
  bucket_large_kernel<<<lgrid, kLocalThreads, sizeof(LocalSmem), stream>>>(
      st, nb.k0, nb.p0, nb.k1, nb.p1, bstat, bjob);
  const int grid = persistent_grid(reinterpret_cast<const void*>(bucket_local_kernel),
                                   kLocalThreads, sizeof(LocalSmem), kBucketSlots);
  bucket_local_kernel<<<grid, kLocalThreads, sizeof(LocalSmem), stream>>>(
      st, fs, nframes, nb.k0, nb.p0, nb.k1, nb.p1, bstat, bjob, out, spin_limit, err);
  return cudaGetLastError();
}

}  // namespace vg
