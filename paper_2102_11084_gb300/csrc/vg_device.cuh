// Device helpers shared by the voxel-grid kernels (sm_103a).
//
// Voxel key (arXiv 2102.11084 Sec. II-C, ordered subdivision of space): per axis, in
// IEEE binary32 with round-to-nearest and no contraction, i = floor(fl(fl(p-o)/leaf)),
// 0 <= i < 2^21; the key interleaves bit b of ix, iy, iz into bits 3b, 3b+1, 3b+2.
// Batched calls put the frame id above a key_shift-bit key field, so one sort orders
// every frame's voxels at once.
//
// Centroid accumulator (not fixed by the paper): each point contributes the offset from
// its voxel corner c = fl(o + fl(i*leaf)), quantised to a signed integer in units of
// leaf/2^20; sums are int64, so any summation order gives the same bits.  The centroid is
// c + (sum/n)/2^20*leaf evaluated in binary32.  Every path (sort, hash, batch, pyramid
// level 0) uses exactly these functions, so their outputs agree bit for bit.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "vg_internal.h"

namespace vg {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr float kAxisLimitF = 2097152.0f;   // 2^21
constexpr float kQuantScale = 1048576.0f;   // 2^20 units per leaf
constexpr uint64_t kKeySentinel = ~0ull;    // invalid point

// ---- error word -------------------------------------------------------------------
// The first error code wins; later ones are dropped.
__device__ __forceinline__ void set_error(int* err, int code) {
  atomicCAS(err, 0, code);
}
// True once some step has set the error word: every kernel after the key kernel then
// returns at once, so no step reads a row, an index or a count an earlier step left
// unwritten.
__device__ __forceinline__ bool error_raised(const int* err) {
  return *reinterpret_cast<const volatile int*>(err) != 0;
}
// The same test taken once for the whole block (thread 0 reads, a barrier shares the
// answer), for kernels with barriers: a block of a kernel that sets errors itself could
// otherwise see the word change between its warps' reads.  Every thread must call it.
__device__ __forceinline__ bool block_error_raised(const int* err) {
  return __syncthreads_or(threadIdx.x == 0 && error_raised(err)) != 0;
}

// ---- voxel index and Morton key -----------------------------------------------------
// Returns false when the index leaves [0, 2^21) (also for an infinite quotient).
__device__ __forceinline__ bool axis_index(float p, float o, float leaf, uint32_t* i) {
  const float t = __fsub_rn(p, o);
  const float q = __fdiv_rn(t, leaf);
  if (!(q >= 0.0f) || !(q < kAxisLimitF)) return false;
  *i = static_cast<uint32_t>(__float2int_rd(q));
  return true;
}

// The same index as axis_index, cheaper: q1 = fl(fl(p-o) * r) with r = fl(1/leaf) is
// within 1.5*2^-23*|q| of fl((p-o)/leaf), so whenever q1 lies farther than |q1|*2^-20 from
// every integer both have the same floor (and the same side of 0 and 2^21, which are
// integers); otherwise the exact division decides.  Valid for 2^-100 < leaf < 2^100
// (r is then a normal number); callers check that range.
__device__ __forceinline__ bool axis_index_fast(float p, float o, float leaf, float r,
                                                uint32_t* i) {
  const float t = __fsub_rn(p, o);
  const float q1 = __fmul_rn(t, r);
  const float fl = floorf(q1);
  const float d = q1 - fl;
  const float margin = fabsf(q1) * 9.5367431640625e-07f;  // 2^-20
  if (d > margin && 1.0f - d > margin) {
    if (!(fl >= 0.0f) || !(fl < kAxisLimitF)) return false;
    *i = static_cast<uint32_t>(fl);
    return true;
  }
  return axis_index(p, o, leaf, i);
}

// leaf range in which axis_index_fast may be used
__device__ __forceinline__ bool fast_leaf(float leaf) {
  return leaf > 7.8886090522101181e-31f && leaf < 1.2676506002282294e30f;  // 2^-100, 2^100
}

__device__ __forceinline__ bool point_valid(float x, float y, float z) {
  return isfinite(x) && isfinite(y) && isfinite(z);
}

// Spread the low 21 bits of v so that bit b lands on bit 3b.
__device__ __forceinline__ uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1fffffu;
  x = (x | (x << 32)) & 0x001f00000000ffffull;
  x = (x | (x << 16)) & 0x001f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

// Inverse of spread3: gather bits 0, 3, 6, ... into the low 21 bits.
__device__ __forceinline__ uint32_t compact3(uint64_t x) {
  x &= 0x1249249249249249ull;
  x = (x | (x >> 2)) & 0x10c30c30c30c30c3ull;
  x = (x | (x >> 4)) & 0x100f00f00f00f00full;
  x = (x | (x >> 8)) & 0x001f0000ff0000ffull;
  x = (x | (x >> 16)) & 0x001f00000000ffffull;
  x = (x | (x >> 32)) & 0x00000000001fffffull;
  return static_cast<uint32_t>(x);
}

// spread3 for indices below 2^11, with 32-bit operations (bit b -> bit 3b, up to bit 30).
__device__ __forceinline__ uint32_t spread3_32(uint32_t x) {
  x &= 0x7ffu;
  x = (x | (x << 16)) & 0x070000ffu;
  x = (x | (x << 8)) & 0x0700f00fu;
  x = (x | (x << 4)) & 0x430c30c3u;
  x = (x | (x << 2)) & 0x49249249u;
  return x;
}

// compact3 for keys below 2^32 (11 bits of x and y, 10 of z), with 32-bit operations.
__device__ __forceinline__ uint32_t compact3_32(uint32_t x) {
  x &= 0x49249249u;
  x = (x | (x >> 2)) & 0xc30c30c3u;
  x = (x | (x >> 4)) & 0x0f00f00fu;
  x = (x | (x >> 8)) & 0xff0000ffu;
  x = (x | (x >> 16)) & 0x000007ffu;
  return x;
}

// Voxel index on `axis` (0, 1, 2) of a per-frame Morton key.
__device__ __forceinline__ uint32_t key_axis(uint64_t key, int axis) {
  return (key >> 32) == 0 ? compact3_32(static_cast<uint32_t>(key) >> axis) : compact3(key >> axis);
}

__device__ __forceinline__ uint64_t morton3(uint32_t ix, uint32_t iy, uint32_t iz) {
  return spread3(ix) | (spread3(iy) << 1) | (spread3(iz) << 2);
}

// Validity and voxel indices of a point (no key); *range_bad set when out of range.
__device__ __forceinline__ bool point_index(float x, float y, float z, const float o[3],
                                            float leaf, float rleaf, uint32_t ijk[3],
                                            bool* range_bad) {
  if (!point_valid(x, y, z)) return false;
  bool ok;
  if (rleaf != 0.0f)
    ok = axis_index_fast(x, o[0], leaf, rleaf, &ijk[0]) &
         axis_index_fast(y, o[1], leaf, rleaf, &ijk[1]) &
         axis_index_fast(z, o[2], leaf, rleaf, &ijk[2]);
  else
    ok = axis_index(x, o[0], leaf, &ijk[0]) & axis_index(y, o[1], leaf, &ijk[1]) &
         axis_index(z, o[2], leaf, &ijk[2]);
  if (!ok) *range_bad = true;
  return ok;
}

// point_key that also returns the voxel indices.
// rleaf = fl(1/leaf) when fast_leaf(leaf), else 0 (exact division for every point).
__device__ __forceinline__ bool point_key_ijk(float x, float y, float z, const float o[3],
                                              float leaf, float rleaf, uint64_t* key,
                                              uint32_t ijk[3], bool* range_bad) {
  if (!point_valid(x, y, z)) return false;
  bool ok;
  if (rleaf != 0.0f)
    ok = axis_index_fast(x, o[0], leaf, rleaf, &ijk[0]) &
         axis_index_fast(y, o[1], leaf, rleaf, &ijk[1]) &
         axis_index_fast(z, o[2], leaf, rleaf, &ijk[2]);
  else
    ok = axis_index(x, o[0], leaf, &ijk[0]) & axis_index(y, o[1], leaf, &ijk[1]) &
         axis_index(z, o[2], leaf, &ijk[2]);
  if (!ok) {
    *range_bad = true;
    return false;
  }
  *key = morton3(ijk[0], ijk[1], ijk[2]);
  return true;
}

// Morton key of a point, or false if the point is invalid / out of range (*range_bad
// set for the latter).
__device__ __forceinline__ bool point_key(float x, float y, float z, const float o[3],
                                          float leaf, float rleaf, uint64_t* key,
                                          bool* range_bad) {
  uint32_t ijk[3];
  return point_key_ijk(x, y, z, o, leaf, rleaf, key, ijk, range_bad);
}

// Split a sort key into (frame, per-frame voxel key).  key_shift == 64: one frame.
__device__ __forceinline__ uint32_t key_frame(uint64_t key, uint32_t key_shift) {
  return key_shift >= 64 ? 0u : static_cast<uint32_t>(key >> key_shift);
}
__device__ __forceinline__ uint64_t key_local(uint64_t key, uint32_t key_shift) {
  return key_shift >= 64 ? key : (key & ((1ull << key_shift) - 1ull));
}
__device__ __forceinline__ uint64_t key_compose(uint32_t frame, uint64_t local,
                                                uint32_t key_shift) {
  return key_shift >= 64 ? local : ((uint64_t(frame) << key_shift) | local);
}

// ---- fixed-point centroid accumulator ------------------------------------------------
struct Acc {
  uint32_t n;
  long long s[3];
};

__device__ __forceinline__ Acc acc_zero() {
  Acc a;
  a.n = 0;
  a.s[0] = a.s[1] = a.s[2] = 0;
  return a;
}

__device__ __forceinline__ void acc_add(Acc& a, const Acc& b) {
  a.n += b.n;
  a.s[0] += b.s[0];
  a.s[1] += b.s[1];
  a.s[2] += b.s[2];
}

__device__ __forceinline__ float quant_inv_unit(float leaf) {
  return __fdiv_rn(kQuantScale, leaf);
}

__device__ __forceinline__ float voxel_corner(uint32_t i, float o, float leaf) {
  return __fadd_rn(o, __fmul_rn(__uint2float_rn(i), leaf));
}

// Quantised offset of coordinate p from its voxel corner c, clamped to
// [-2^19, 3*2^19): half a voxel of slack on either side of [0, leaf), so that it packs in
// 21 bits.  An offset leaves that range only when the leaf is within a few binary32 ulps
// of the coordinates, where the clamp moves a centroid by less than those ulps.
constexpr int kQMin = -(1 << 19);
constexpr int kQMax = (3 << 19) - 1;
__device__ __forceinline__ int quant_offset(float p, float c, float inv_unit) {
  const int q = __float2int_rn(__fmul_rn(__fsub_rn(p, c), inv_unit));
  return q < kQMin ? kQMin : (q > kQMax ? kQMax : q);
}

// Three quantised offsets packed in one 64-bit word (21 bits each, biased by 2^19);
// bit 63 set marks an invalid point.
constexpr uint64_t kPayloadInvalid = 1ull << 63;
__device__ __forceinline__ uint64_t pack_offsets(int qx, int qy, int qz) {
  return uint64_t(uint32_t(qx - kQMin)) | (uint64_t(uint32_t(qy - kQMin)) << 21) |
         (uint64_t(uint32_t(qz - kQMin)) << 42);
}
__device__ __forceinline__ int unpack_offset(uint64_t w, int axis) {
  return int(uint32_t(w >> (21 * axis)) & 0x1fffffu) + kQMin;
}

// Offsets of point (x,y,z) from the corner of voxel `local` (a per-frame Morton key).
__device__ __forceinline__ Acc point_acc(uint64_t local, float x, float y, float z,
                                         const float o[3], float leaf, float inv_unit) {
  Acc a;
  a.n = 1;
  a.s[0] = quant_offset(x, voxel_corner(key_axis(local, 0), o[0], leaf), inv_unit);
  a.s[1] = quant_offset(y, voxel_corner(key_axis(local, 1), o[1], leaf), inv_unit);
  a.s[2] = quant_offset(z, voxel_corner(key_axis(local, 2), o[2], leaf), inv_unit);
  return a;
}

// Centroid of voxel `local` (edge `leaf`) from n points whose offsets from its corner sum
// to S, in units of unit_leaf/2^20: c + S * (unit_leaf / (n * 2^20)), one division per
// voxel.  (unit_leaf = leaf except in the pyramid, whose sums keep the level-0 unit.)
__device__ __forceinline__ void acc_centroid(uint64_t local, const Acc& a, const float o[3],
                                             float leaf, float unit_leaf, float out[3]) {
  // For n = 2^k the divisor n * 2^20 = 2^(20+k) is exact and so is the quotient (a normal
  // number when unit_leaf >= 2^-76 and k <= 30): the same bits as the division, cheaper.
  float scale;
  if ((a.n & (a.n - 1u)) == 0u && a.n != 0u && unit_leaf >= 1.3234889800848443e-23f)
    scale = __fmul_rn(unit_leaf, __int_as_float((127 - 20 - (__ffs(int(a.n)) - 1)) << 23));
  else
    scale = __fdiv_rn(unit_leaf, __fmul_rn(__uint2float_rn(a.n), kQuantScale));
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const float c = voxel_corner(key_axis(local, ax), o[ax], leaf);
    out[ax] = __fadd_rn(c, __fmul_rn(__ll2float_rn(a.s[ax]), scale));
  }
}

// ---- ordered float <-> uint (for atomic min/max) -------------------------------------
__device__ __forceinline__ uint32_t float_to_ordered(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ordered_to_float(uint32_t u) {
  const uint32_t b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
  return __uint_as_float(b);
}

// ---- memory-model helpers for chained scans -------------------------------------------
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Number of 8-bit digit passes needed for keys <= maxkey.
__device__ __forceinline__ int sort_passes(unsigned long long maxkey) {
  if (maxkey == 0) return 0;
  const int bits = 64 - __clzll(static_cast<long long>(maxkey));
  return (bits + kRadixBits - 1) / kRadixBits;
}

// Radix passes a call runs: every significant digit of the largest key (at least one,
// which also drops the invalid rows); none when the narrow layout is grouped by buckets.
__device__ __forceinline__ int pass_count(const State* st) {
  if (st->narrow && st->msd) return 0;
  return max(1, sort_passes(st->maxkey));
}

// Bounded chained-scan wait on a tile status word (flag | 30-bit value).  Returns the
// exclusive prefix of tile `tile`'s value over tiles 0..tile-1.
__device__ __forceinline__ uint32_t lookback_u32(const uint32_t* status, size_t stride,
                                                 int tile, uint32_t spin_limit, int* err) {
  // The status words of up to VG_LOOKBACK_WINDOW predecessors are loaded at once (one
  // round trip to L2 per window instead of per tile) and consumed in tile order until a
  // prefix or a word not yet published; a window that makes no progress counts as one
  // poll against spin_limit.
  uint32_t excl = 0;
  int j = tile - 1;
  uint32_t spins = 0;
  while (j >= 0) {
    uint32_t s[kLookbackWindow];
#pragma unroll
    for (int k = 0; k < kLookbackWindow; ++k)
      s[k] = j - k >= 0 ? ld_relaxed(status + size_t(j - k) * stride) : 0u;
    int adv = 0;
    bool found = false, blocked = false;
#pragma unroll
    for (int k = 0; k < kLookbackWindow; ++k) {
      if (!found && !blocked && j - k >= 0) {
        const uint32_t f = s[k] & ~kValueMask;
        if (f == 0) {
          blocked = true;
        } else {
          excl += s[k] & kValueMask;
          ++adv;
          found = f == kFlagPrefix;
        }
      }
    }
    if (found) break;
    j -= adv;
    if (adv == 0) {
      if (++spins > spin_limit) {
        set_error(err, kErrTimeout);
        break;
      }
      if (spins > 64) __nanosleep(64);
    }
  }
  return excl;
}

// ---- bulk asynchronous copies (TMA unit) completed on a shared-memory mbarrier ------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t arrivals) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(arrivals)
               : "memory");
}
// Makes mbarrier initialisation visible to the asynchronous proxy (the bulk-copy unit).
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n\tfence.proxy.async.shared::cta;" ::
                   : "memory");
}
// Orders this thread's earlier shared-memory accesses before later bulk copies.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// One arrival that also announces `bytes` of bulk-copy data for the current phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// Global -> shared bulk copy; dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Asynchronous 16-byte global -> shared copy (both addresses 16-byte aligned); complete
// once this thread has executed cp_async_wait_all.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}
// Hint: bring [p, p + bytes) into L2 (bulk prefetch; p and bytes multiples of 16).
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Waits (bounded: `limit` polls) for the phase of parity `parity` to complete.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity,
                                          uint32_t limit) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (i > 32) __nanosleep(32);
  }
  return false;
}

// ---- block-wide helpers (256 threads) -------------------------------------------------
// Exclusive scan of one u32 per thread; *total receives the block sum.  `tmp` holds
// blockDim/32 words of shared memory (blockDim <= 1024).  The warp totals are scanned by
// every warp with shuffles.  Contains __syncthreads.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* total,
                                                    uint32_t* tmp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(kFullMask, inc, off);
    if (lane >= off) inc += y;
  }
  __syncthreads();  // earlier readers of tmp are done
  if (lane == 31) tmp[warp] = inc;
  __syncthreads();
  const uint32_t wt = lane < nw ? tmp[lane] : 0u;
  uint32_t ws = wt;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(kFullMask, ws, off);
    if (lane >= off) ws += y;
  }
  *total = __shfl_sync(kFullMask, ws, 31);
  return __shfl_sync(kFullMask, ws - wt, warp) + inc - v;
}

// ---- frame decomposition (chunks of kChunk points inside one frame) -----------------------
// Loads the frame offsets into s_off[0..F] and the chunk prefix into s_cstart[0..F];
// returns the number of chunks.  Bad offsets (not starting at 0, not ending at n, or
// decreasing) record kErrInvalidArg and yield zero chunks.  Contains __syncthreads.
__device__ __forceinline__ uint32_t build_chunk_map(const FramesArg& fr, int64_t* s_off,
                                                    uint32_t* s_cstart, uint32_t* tmp,
                                                    int* err) {
  const int F = fr.nframes;
  for (int f = threadIdx.x; f <= F; f += blockDim.x)
    s_off[f] = fr.offsets ? fr.offsets[f] : (f == 0 ? 0 : fr.n);
  __syncthreads();
  // chunk counts of the frames owned by this thread: frames [4t, 4t+4)
  constexpr int kPer = kMaxFrames / kStreamThreads;
  uint32_t c[kPer];
  uint32_t mine = 0;
  bool bad = false;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int f = threadIdx.x * kPer + k;
    c[k] = 0;
    if (f < F) {
      const int64_t a = s_off[f], b = s_off[f + 1];
      if (b < a || a < 0 || b > fr.n) bad = true;
      else c[k] = static_cast<uint32_t>(ceil_div(b - a, kChunk));
    }
    mine += c[k];
  }
  if (threadIdx.x == 0 && (s_off[0] != 0 || s_off[F] != fr.n)) bad = true;
  const int any_bad = __syncthreads_or(bad);
  uint32_t total;
  uint32_t run = block_excl_scan(any_bad ? 0u : mine, &total, tmp);
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int f = threadIdx.x * kPer + k;
    if (f <= F) s_cstart[f] = run;
    if (!any_bad) run += c[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) s_cstart[F] = any_bad ? 0u : total;
  if (any_bad && threadIdx.x == 0 && blockIdx.x == 0) set_error(err, kErrInvalidArg);
  __syncthreads();
  return any_bad ? 0u : total;
}

// Frame holding chunk c (largest f with s_cstart[f] <= c, skipping empty frames).
__device__ __forceinline__ int chunk_frame(const uint32_t* s_cstart, int F, uint32_t c) {
  int lo = 0, hi = F - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (s_cstart[mid] <= c) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Loads points p0..p0+3 (x,y,z interleaved) into v[12]; rows at or beyond `end` are NaN.
__device__ __forceinline__ void load4(const float* __restrict__ xyz, int64_t p0, int64_t end,
                                      bool vec, float v[12]) {
  if (vec && p0 + 4 <= end) {
    const float4* q = reinterpret_cast<const float4*>(xyz + 3 * p0);
    const float4 a = __ldcs(q), b = __ldcs(q + 1), c = __ldcs(q + 2);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    v[8] = c.x; v[9] = c.y; v[10] = c.z; v[11] = c.w;
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const bool in = p0 + j < end;
#pragma unroll
      for (int a = 0; a < 3; ++a)
        v[3 * j + a] = in ? __ldcs(xyz + 3 * (p0 + j) + a) : __int_as_float(0x7fc00000);
    }
  }
}

// 64-bit mixer (the MurmurHash3 finaliser) for the voxel hash table.
__device__ __forceinline__ uint64_t hash64(uint64_t x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}

}  // namespace vg
