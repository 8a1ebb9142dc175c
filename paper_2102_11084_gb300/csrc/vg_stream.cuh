// Block-level pieces shared by the streaming kernels (origin, keys, hash insert): the
// frame/chunk decomposition held in shared memory and the per-frame prologue.
#pragma once
#include "vg_device.cuh"
#include "vg_internal.h"

namespace vg {

struct ChunkSmem {
  int64_t off[kMaxFrames + 1];
  uint32_t cstart[kMaxFrames + 1];
  uint32_t tmp[kStreamThreads / 32];
  float org[kMaxFrames][3];
  float leaf[kMaxFrames];
  float rleaf[kMaxFrames];  // fl(1/leaf) when the fast index applies, else 0
  float inv_unit[kMaxFrames];  // the fixed-point scale of the frame's offsets
  uint32_t bits[kStreamThreads / 32];
  unsigned long long kmax[kStreamThreads / 32];
};

// Pose and height limits of one frame (registers of a posed streaming kernel).
struct Pose {
  float r[12];  // row-major [R|t]
  float zlo, zhi;
  bool rigid;   // false: identity pose (only the height limits apply)
};

__device__ __forceinline__ void load_pose(const FramesArg& fr, int f, Pose& P) {
  P.rigid = fr.poses != nullptr;
#pragma unroll
  for (int i = 0; i < 12; ++i) P.r[i] = P.rigid ? __ldg(fr.poses + 12 * f + i) : 0.0f;
  P.zlo = fr.zlims ? __ldg(fr.zlims + 2 * f) : -INFINITY;
  P.zhi = fr.zlims ? __ldg(fr.zlims + 2 * f + 1) : INFINITY;
}

// p' = R p + t in FP32, each product and sum rounded on its own in the order
// ((r0 x + r1 y) + r2 z) + t (no fused multiply-add); a point whose z' is outside
// [zlo, zhi] (or not a number) becomes NaN, i.e. invalid.
__device__ __forceinline__ void pose_point(const Pose& P, float& x, float& y, float& z) {
  float g[3] = {x, y, z};
  if (P.rigid) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float* r = P.r + 4 * a;
      g[a] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(r[0], x), __fmul_rn(r[1], y)),
                                 __fmul_rn(r[2], z)),
                       r[3]);
    }
  }
  const bool keep = g[2] >= P.zlo && g[2] <= P.zhi;
  x = keep ? g[0] : NAN;
  y = keep ? g[1] : NAN;
  z = keep ? g[2] : NAN;
}

// Key (the narrow layout's 32 bits) and packed corner offsets of one point of frame f;
// false for an invalid or out-of-range point (*range_bad set for the latter).  The key
// kernel and the single-frame bin grouping both call this, so they agree bit for bit.
__device__ __forceinline__ bool narrow_entry(float x, float y, float z, const float o[3],
                                             float leaf, float rleaf, float inv_unit,
                                             uint32_t f, uint32_t key_shift, uint32_t* key,
                                             uint64_t* pay, bool* range_bad) {
  uint32_t ijk[3];
  if (!point_index(x, y, z, o, leaf, rleaf, ijk, range_bad)) return false;
  // the indices have at most 11 bits: the interleave runs on 32-bit words
  const uint32_t local =
      spread3_32(ijk[0]) | (spread3_32(ijk[1]) << 1) | (spread3_32(ijk[2]) << 2);
  *key = static_cast<uint32_t>(key_compose(f, local, key_shift));
  const float v[3] = {x, y, z};
  int qq[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) qq[a] = quant_offset(v[a], voxel_corner(ijk[a], o[a], leaf), inv_unit);
  *pay = pack_offsets(qq[0], qq[1], qq[2]);
  return true;
}

// Contiguous chunk range of this block.
__device__ __forceinline__ void block_range(uint32_t T, uint32_t* c0, uint32_t* c1) {
  *c0 = static_cast<uint32_t>((uint64_t(T) * blockIdx.x) / gridDim.x);
  *c1 = static_cast<uint32_t>((uint64_t(T) * (blockIdx.x + 1)) / gridDim.x);
}

// Resolves every frame's origin (given, or the minimum found by the origin kernel) and
// leaf into shared memory, checks the leaves, and returns the key shift: 64 for one
// frame, else the bit length of the largest per-frame key (from the frame maxima).  Block
// 0 publishes origins, leaves and the shift.  Contains __syncthreads.
__device__ __forceinline__ uint32_t frame_prologue(const FramesArg& fr, bool have_extent,
                                                   State* st, FrameState* fs, uint32_t T,
                                                   ChunkSmem& sm, int* err,
                                                   bool* narrow = nullptr,
                                                   uint32_t* bshift = nullptr,
                                                   uint32_t* kbits = nullptr) {
  const int F = fr.nframes;
  // per-frame origin and leaf; bits of the largest key of each frame
  uint32_t bits = 0;
  unsigned long long kmax = 0;  // largest per-frame key bound (Morton code of the maxima)
  bool bad_leaf = false;
  for (int f = threadIdx.x; f < F; f += kStreamThreads) {
    const float leaf = fr.leaves ? fr.leaves[f] : fr.leaf;
    if (!(leaf > 0.0f) || !isfinite(leaf)) bad_leaf = true;
    float o[3];
    const bool any = fs[f].ord_min_inv[0] != 0;
    for (int a = 0; a < 3; ++a) {
      if (fr.origin_in) {
        o[a] = fr.origin_in[3 * f + a];
      } else {
        const uint32_t u = fs[f].ord_min_inv[a];
        o[a] = (u == 0) ? 0.0f : ordered_to_float(~u);
      }
      sm.org[f][a] = o[a];
    }
    sm.leaf[f] = leaf;
    sm.rleaf[f] = fast_leaf(leaf) ? __fdiv_rn(1.0f, leaf) : 0.0f;
    sm.inv_unit[f] = quant_inv_unit(leaf);
    if (blockIdx.x == 0) {
      for (int a = 0; a < 3; ++a) {
        fs[f].origin[a] = o[a];
        if (!fr.origin_in && fr.origin_out) fr.origin_out[3 * f + a] = o[a];
      }
      fs[f].leaf = leaf;
    }
    if (have_extent && any) {
      uint32_t ii[3];
      bool ok = true;
      for (int a = 0; a < 3; ++a)
        ok = ok && axis_index(ordered_to_float(fs[f].ord_max[a]), o[a], leaf, &ii[a]);
      const uint64_t m = ok ? morton3(ii[0], ii[1], ii[2]) : ~0ull >> 1;
      const uint32_t b = m ? 64u - __clzll(static_cast<long long>(m)) : 0u;
      bits = b > bits ? b : bits;
      kmax = m > kmax ? m : kmax;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    bits = max(bits, __shfl_xor_sync(kFullMask, bits, off));
    const unsigned long long o = __shfl_xor_sync(kFullMask, kmax, off);
    kmax = o > kmax ? o : kmax;
  }
  if (lane == 0) {
    sm.bits[warp] = bits;
    sm.kmax[warp] = kmax;
  }
  if (__syncthreads_or(bad_leaf) && threadIdx.x == 0 && blockIdx.x == 0)
    set_error(err, kErrInvalidArg);
  uint32_t maxbits = 0;
  unsigned long long maxkey = 0;
  for (int w = 0; w < kStreamThreads / 32; ++w) {
    maxbits = max(maxbits, sm.bits[w]);
    maxkey = sm.kmax[w] > maxkey ? sm.kmax[w] : maxkey;
  }
  uint32_t key_shift = 64, total_bits = maxbits;
  if (F > 1 && !fr.merge_frames) {
    key_shift = maxbits;
    const uint32_t fbits = 32u - __clz(static_cast<int>(F - 1));
    total_bits = key_shift + fbits;
    if (total_bits > 63 && threadIdx.x == 0 && blockIdx.x == 0) set_error(err, kErrRange);
  }
  // The narrow layout needs the largest key known in advance (the extents), below
  // 0xffffffff: a 32-bit key of all ones then marks an invalid row by itself.  Morton codes
  // grow with each index, so the code of the per-axis maxima bounds every key of a frame.
  const uint64_t key_bound =
      key_shift < 64 ? ((uint64_t(F - 1) << key_shift) | ((uint64_t(1) << key_shift) - 1))
                     : maxkey;
  const bool nar = fr.allow_narrow && have_extent && total_bits <= 32 && key_bound < 0xffffffffull;
  if (narrow) *narrow = nar;
  // Bucket grouping (narrow layout unless the caller forces the global radix sort): the
  // top `top` key bits name the bucket, aimed at kMsdTarget points per bucket, at most
  // kMsdMaxTop bits, and enough that the low kb - top bits reduced on chip are at most
  // kMsdMaxLow -- and, with several frames, at most the frame key field, so that a bucket
  // never holds two frames.  One partition pass splits up to 8 bucket bits, two up to 16.
  bool mmode = nar && !fr.lsd_narrow;
  uint32_t low = 0, levels = 0, b1 = 0, b2 = 0;
  const uint32_t kb = key_bound ? 64u - __clzll(static_cast<long long>(key_bound)) : 0u;
  const uint32_t lmax = key_shift < 64 ? min(uint32_t(kMsdMaxLow), key_shift)
                                       : uint32_t(kMsdMaxLow);
  const uint32_t lo = max(1u, kb > lmax ? kb - lmax : 0u);
  // (kb <= 32 and the frame id takes at most 10 bits keep lo <= 16; checked all the same)
  mmode = mmode && lo <= uint32_t(kMsdMaxTop);
  if (mmode) {
    const int64_t q = (fr.n + kMsdTarget - 1) / kMsdTarget;
    const uint32_t want = q > 1 ? 64u - __clzll(static_cast<long long>(q - 1)) : 0u;
    const uint32_t hi = max(lo, min(uint32_t(kMsdMaxTop), kb));
    const uint32_t top = min(hi, max(lo, want));
    low = kb > top ? kb - top : 0u;
    levels = top > uint32_t(kRadixBits) ? 2u : 1u;
    b2 = levels == 2 ? uint32_t(kRadixBits) : 0u;
    b1 = top - b2;
  }
  // the key kernel histograms the first partition pass's digit
  if (bshift) *bshift = mmode ? low + b2 : 0u;
  if (kbits) *kbits = kb;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->key_shift = key_shift;
    st->nframes = F;
    st->nchunks = T;
    st->narrow = nar ? 1u : 0u;
    st->msd = mmode ? 1u : 0u;
    st->lowbits = low;
    st->levels = levels;
    st->b1 = b1;
    st->b2 = b2;
  }

  __syncthreads();
  return key_shift;
}

}  // namespace vg
