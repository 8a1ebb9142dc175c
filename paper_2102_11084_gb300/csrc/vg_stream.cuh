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
  uint32_t bits[kStreamThreads / 32];
};

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
                                                   bool* narrow = nullptr) {
  const int F = fr.nframes;
  // per-frame origin and leaf; bits of the largest key of each frame
  uint32_t bits = 0;
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
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off; off >>= 1) bits = max(bits, __shfl_xor_sync(kFullMask, bits, off));
  if (lane == 0) sm.bits[warp] = bits;
  if (__syncthreads_or(bad_leaf) && threadIdx.x == 0 && blockIdx.x == 0)
    set_error(err, kErrInvalidArg);
  uint32_t maxbits = 0;
  for (int w = 0; w < kStreamThreads / 32; ++w) maxbits = max(maxbits, sm.bits[w]);
  uint32_t key_shift = 64, total_bits = maxbits;
  if (F > 1) {
    key_shift = maxbits;
    const uint32_t fbits = 32u - __clz(static_cast<int>(F - 1));
    total_bits = key_shift + fbits;
    if (total_bits > 63 && threadIdx.x == 0 && blockIdx.x == 0) set_error(err, kErrRange);
  }
  // The narrow layout needs the largest key known in advance (the extents) and <= 32 bits.
  const bool nar = fr.allow_narrow && have_extent && total_bits <= 32;
  if (narrow) *narrow = nar;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->key_shift = key_shift;
    st->nframes = F;
    st->nchunks = T;
    st->narrow = nar ? 1u : 0u;
  }

  __syncthreads();
  return key_shift;
}

}  // namespace vg
