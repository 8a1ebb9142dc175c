// Device helpers shared by the voxel-grid kernels (sm_103a).
//
// Voxel key (arXiv 2102.11084 Sec. II-C, ordered subdivision of space): per axis, in
// IEEE binary32 with round-to-nearest and no contraction, i = floor(fl(fl(p-o)/leaf)),
// 0 <= i < 2^21; the key interleaves bit b of ix, iy, iz into bits 3b, 3b+1, 3b+2.
//
// Centroid accumulator (not fixed by the paper): each point contributes the offset from
// its voxel corner c = fl(o + fl(i*leaf)), quantised to a signed integer in units of
// leaf/2^20; sums are int64, so any summation order gives the same bits.  The centroid is
// c + (sum/n)/2^20*leaf evaluated in binary32.  Every path (sort, hash, batch, pyramid)
// uses exactly these functions, so their outputs agree bit for bit.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "vg_internal.h"

namespace vg {

constexpr float kAxisLimitF = 2097152.0f;   // 2^21
constexpr float kQuantScale = 1048576.0f;   // 2^20 units per leaf

// ---- error word -------------------------------------------------------------------
// The first error code wins; later ones are dropped.
__device__ __forceinline__ void set_error(int* err, int code) {
  atomicCAS(err, 0, code);
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

__device__ __forceinline__ uint64_t morton3(uint32_t ix, uint32_t iy, uint32_t iz) {
  return spread3(ix) | (spread3(iy) << 1) | (spread3(iz) << 2);
}

// Key of a point, or false if the point is invalid / out of range (*range_bad set for
// the latter).
__device__ __forceinline__ bool point_key(float x, float y, float z, const float o[3],
                                          float leaf, uint64_t* key, bool* range_bad) {
  if (!point_valid(x, y, z)) return false;
  uint32_t ix, iy, iz;
  const bool ok = axis_index(x, o[0], leaf, &ix) & axis_index(y, o[1], leaf, &iy) &
                  axis_index(z, o[2], leaf, &iz);
  if (!ok) {
    *range_bad = true;
    return false;
  }
  *key = morton3(ix, iy, iz);
  return true;
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

// Quantised offset of coordinate p from its voxel corner c.
__device__ __forceinline__ int quant_offset(float p, float c, float inv_unit) {
  return __float2int_rn(__fmul_rn(__fsub_rn(p, c), inv_unit));
}

// Offsets of point (x,y,z) from the corner of voxel `key`, as one accumulator entry.
__device__ __forceinline__ Acc point_acc(uint64_t key, float x, float y, float z,
                                         const float o[3], float leaf, float inv_unit) {
  Acc a;
  a.n = 1;
  a.s[0] = quant_offset(x, voxel_corner(compact3(key), o[0], leaf), inv_unit);
  a.s[1] = quant_offset(y, voxel_corner(compact3(key >> 1), o[1], leaf), inv_unit);
  a.s[2] = quant_offset(z, voxel_corner(compact3(key >> 2), o[2], leaf), inv_unit);
  return a;
}

// Centroid of voxel `key` from its accumulator (n >= 1).
__device__ __forceinline__ void acc_centroid(uint64_t key, const Acc& a, const float o[3],
                                             float leaf, float inv_unit, float out[3]) {
  const float fn = __uint2float_rn(a.n);
  const uint32_t ii[3] = {compact3(key), compact3(key >> 1), compact3(key >> 2)};
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const float c = voxel_corner(ii[ax], o[ax], leaf);
    const float m = __fdiv_rn(__fdiv_rn(__ll2float_rn(a.s[ax]), fn), inv_unit);
    out[ax] = __fadd_rn(c, m);
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
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
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

}  // namespace vg
