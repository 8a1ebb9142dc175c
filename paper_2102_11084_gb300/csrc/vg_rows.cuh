// Output rows of the groupings that reduce one cell at a time in shared memory (the
// bucket grouping and the single-frame bin grouping): the centroid formula of
// acc_centroid, written to the caller's keys, counts and centroids (and the fixed-point
// sums when the pyramid asks for them).
#pragma once
#include "vg_device.cuh"
#include "vg_internal.h"

namespace vg {

// Origin and leaf of a single frame (o1, leaf1), else each row's frame from fs.
struct RowCtx {
  const FrameState* fs;
  uint32_t key_shift;
  float o1[3];
  float leaf1;
};

// Row `cur`: cell `key` (the full sort key) with n entries whose offsets sum to s.
__device__ __forceinline__ void put_row(const RowCtx& rc, const SegOut& out, uint32_t cur,
                                        uint32_t key, const Acc& a, int* err) {
  if (int64_t(cur) >= out.cap) {
    set_error(err, kErrCapacity);
    return;
  }
  const uint64_t local = key_local(key, rc.key_shift);
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
  acc_centroid(local, a, o, leaf, leaf, c);
  out.keys[cur] = local;
  out.counts[cur] = a.n;
  out.centroids[3 * size_t(cur)] = c[0];
  out.centroids[3 * size_t(cur) + 1] = c[1];
  out.centroids[3 * size_t(cur) + 2] = c[2];
  if (out.sums) {
    out.sums[3 * size_t(cur)] = a.s[0];
    out.sums[3 * size_t(cur) + 1] = a.s[1];
    out.sums[3 * size_t(cur) + 2] = a.s[2];
  }
}

// Row `cur` of a 32-bit key: the same operations as put_row (acc_centroid), with the
// key's indices de-interleaved in 32-bit words; sf = the offset sums, already converted
// to binary32 (round to nearest, as acc_centroid converts them).
__device__ __forceinline__ void put_row32(const RowCtx& rc, const SegOut& out, uint32_t cur,
                                          uint32_t key, uint32_t n, const float sf[3],
                                          const long long* s64, int* err) {
  if (int64_t(cur) >= out.cap) {
    set_error(err, kErrCapacity);
    return;
  }
  const uint32_t local = rc.key_shift < 32 ? key & ((1u << rc.key_shift) - 1u) : key;
  float o[3] = {rc.o1[0], rc.o1[1], rc.o1[2]};
  float leaf = rc.leaf1;
  if (rc.key_shift < 64) {
    const uint32_t f = rc.key_shift < 32 ? key >> rc.key_shift : 0u;
    o[0] = rc.fs[f].origin[0];
    o[1] = rc.fs[f].origin[1];
    o[2] = rc.fs[f].origin[2];
    leaf = rc.fs[f].leaf;
  }
  float scale;
  if ((n & (n - 1u)) == 0u && n != 0u && leaf >= 1.3234889800848443e-23f)
    scale = __fmul_rn(leaf, __int_as_float((127 - 20 - (__ffs(int(n)) - 1)) << 23));
  else
    scale = __fdiv_rn(leaf, __fmul_rn(__uint2float_rn(n), kQuantScale));
  float c[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float corner = __fadd_rn(o[a], __fmul_rn(__uint2float_rn(compact3_32(local >> a)), leaf));
    c[a] = __fadd_rn(corner, __fmul_rn(sf[a], scale));
  }
  out.keys[cur] = local;
  out.counts[cur] = n;
  out.centroids[3 * size_t(cur)] = c[0];
  out.centroids[3 * size_t(cur) + 1] = c[1];
  out.centroids[3 * size_t(cur) + 2] = c[2];
  if (out.sums) {
    out.sums[3 * size_t(cur)] = s64[0];
    out.sums[3 * size_t(cur) + 1] = s64[1];
    out.sums[3 * size_t(cur) + 2] = s64[2];
  }
}

}  // namespace vg
