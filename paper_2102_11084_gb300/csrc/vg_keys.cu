// Steps a1 (origin = cloud minimum) and a2 (voxel key per point).
//
// arXiv 2102.11084 Sec. II-C normalises each point and classifies it into one cell of an
// ordered subdivision of space ("buscar subdiv" / "actualizar tabla_subdiv" of
// Algorithm 1); here the cell is the voxel of an unbounded lattice with a caller-chosen
// origin and leaf, keyed by a 63-bit Morton code.  Both kernels stream the xyz array
// once with 16-byte loads (4 points = 3 float4 per lane) and are HBM-bound.
#include "vg_device.cuh"
#include "vg_internal.h"

namespace vg {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint64_t kSentinel = ~0ull;

// Loads points p0..p0+3 (x,y,z interleaved) into v[12]; rows at or beyond n are NaN.
template <bool kVec>
__device__ __forceinline__ void load4(const float* __restrict__ xyz, int64_t p0, int64_t n,
                                      float v[12]) {
  if (kVec && p0 + 4 <= n) {
    const float4* q = reinterpret_cast<const float4*>(xyz + 3 * p0);
    const float4 a = __ldcs(q), b = __ldcs(q + 1), c = __ldcs(q + 2);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    v[8] = c.x; v[9] = c.y; v[10] = c.z; v[11] = c.w;
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const bool in = p0 + j < n;
#pragma unroll
      for (int a = 0; a < 3; ++a) v[3 * j + a] = in ? __ldcs(xyz + 3 * (p0 + j) + a) : __int_as_float(0x7fc00000);
    }
  }
}

// a1: per-axis minimum over the valid points, folded into st->ord_min_inv with atomicMax
// on ~ordered(x) (so that a zeroed word means "no valid point").
template <bool kVec>
__global__ __launch_bounds__(kStreamThreads) void origin_kernel(const float* __restrict__ xyz,
                                                                int64_t n, State* st) {
  float mn[3] = {INFINITY, INFINITY, INFINITY};
  const int64_t stride = int64_t(gridDim.x) * kStreamThreads * kStreamPoints;
  for (int64_t p0 = (int64_t(blockIdx.x) * kStreamThreads + threadIdx.x) * kStreamPoints; p0 < n;
       p0 += stride) {
    float v[12];
    load4<kVec>(xyz, p0, n, v);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (point_valid(v[3 * j], v[3 * j + 1], v[3 * j + 2])) {
#pragma unroll
        for (int a = 0; a < 3; ++a) mn[a] = fminf(mn[a], v[3 * j + a]);
      }
    }
  }
  __shared__ float red[kStreamThreads / 32][3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int off = 16; off; off >>= 1) mn[a] = fminf(mn[a], __shfl_xor_sync(kFull, mn[a], off));
    if (lane == 0) red[warp][a] = mn[a];
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    float m = INFINITY;
    for (int w = 0; w < kStreamThreads / 32; ++w) m = fminf(m, red[w][threadIdx.x]);
    if (m != INFINITY) atomicMax(&st->ord_min_inv[threadIdx.x], ~float_to_ordered(m));
  }
}

// a2: key per point (kSentinel for invalid or out-of-range rows), plus the digit-0
// histogram of the valid keys, the number of valid points and the largest valid key.
// Each warp handles 128 consecutive points per iteration (4 per lane).
template <bool kVec>
__global__ __launch_bounds__(kStreamThreads) void key_kernel(
    const float* __restrict__ xyz, int64_t n, float* origin_user, int from_min, float leaf,
    State* st, uint64_t* __restrict__ keys, int* err) {
  __shared__ float so[3];
  __shared__ uint32_t hist[kRadix];
  __shared__ uint32_t wcount[kStreamThreads / 32];
  __shared__ unsigned long long wmax[kStreamThreads / 32];
  if (threadIdx.x < 3) {
    float o;
    if (from_min) {
      const uint32_t u = st->ord_min_inv[threadIdx.x];
      o = (u == 0) ? 0.0f : ordered_to_float(~u);
    } else {
      o = origin_user[threadIdx.x];
    }
    so[threadIdx.x] = o;
    if (blockIdx.x == 0) {
      st->origin[threadIdx.x] = o;
      if (from_min) origin_user[threadIdx.x] = o;
    }
  }
  for (int d = threadIdx.x; d < kRadix; d += kStreamThreads) hist[d] = 0;
  __syncthreads();
  const float o[3] = {so[0], so[1], so[2]};

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t warp_global = int64_t(blockIdx.x) * (kStreamThreads / 32) + warp;
  const int64_t warp_stride = int64_t(gridDim.x) * (kStreamThreads / 32) * 32 * kStreamPoints;
  uint32_t nvalid = 0;
  unsigned long long kmax = 0;
  bool range_bad = false;
  for (int64_t w0 = warp_global * 32 * kStreamPoints; w0 < n; w0 += warp_stride) {
    const int64_t p0 = w0 + int64_t(lane) * kStreamPoints;
    float v[12];
    load4<kVec>(xyz, p0, n, v);
    uint64_t k[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      uint64_t key;
      const bool ok = point_key(v[3 * j], v[3 * j + 1], v[3 * j + 2], o, leaf, &key, &range_bad);
      k[j] = ok ? key : kSentinel;
      if (ok) {
        ++nvalid;
        kmax = key > kmax ? key : kmax;
        atomicAdd(&hist[key & (kRadix - 1)], 1u);
      }
    }
    if (kVec && p0 + 4 <= n) {
      ulonglong2* dst = reinterpret_cast<ulonglong2*>(keys + p0);
      __stcg(dst, make_ulonglong2(k[0], k[1]));
      __stcg(dst + 1, make_ulonglong2(k[2], k[3]));
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (p0 + j < n) keys[p0 + j] = k[j];
    }
  }
  if (__any_sync(kFull, range_bad) && lane == 0) set_error(err, 3 /* VG_ERR_RANGE */);
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    nvalid += __shfl_xor_sync(kFull, nvalid, off);
    const unsigned long long other = __shfl_xor_sync(kFull, kmax, off);
    kmax = other > kmax ? other : kmax;
  }
  if (lane == 0) {
    wcount[warp] = nvalid;
    wmax[warp] = kmax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t c = 0;
    unsigned long long m = 0;
    for (int w = 0; w < kStreamThreads / 32; ++w) {
      c += wcount[w];
      m = wmax[w] > m ? wmax[w] : m;
    }
    if (c) {
      atomicAdd(&st->nvalid, c);
      atomicMax(&st->maxkey, m);
    }
  }
  for (int d = threadIdx.x; d < kRadix; d += kStreamThreads)
    if (hist[d]) atomicAdd(&st->hist[0][d], hist[d]);
}

int stream_grid(int64_t n) {
  const int64_t per_block = int64_t(kStreamThreads) * kStreamPoints;
  const int64_t want = ceil_div(n, per_block);
  const int64_t cap = int64_t(num_sms()) * 8;
  return static_cast<int>(want < 1 ? 1 : (want < cap ? want : cap));
}

}  // namespace

cudaError_t launch_origin(const float* xyz, int64_t n, State* st, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const bool vec = (reinterpret_cast<uintptr_t>(xyz) & 15) == 0;
  if (vec)
    origin_kernel<true><<<stream_grid(n), kStreamThreads, 0, stream>>>(xyz, n, st);
  else
    origin_kernel<false><<<stream_grid(n), kStreamThreads, 0, stream>>>(xyz, n, st);
  return cudaGetLastError();
}

cudaError_t launch_keys(const float* xyz, int64_t n, float* origin_user, bool from_min, float leaf,
                        State* st, uint64_t* keys, int* err, cudaStream_t stream) {
  const bool vec = (reinterpret_cast<uintptr_t>(xyz) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(keys) & 15) == 0;
  // One block even for n == 0: it publishes the origin the call used.
  if (vec)
    key_kernel<true><<<stream_grid(n), kStreamThreads, 0, stream>>>(xyz, n, origin_user,
                                                                    from_min, leaf, st, keys, err);
  else
    key_kernel<false><<<stream_grid(n), kStreamThreads, 0, stream>>>(xyz, n, origin_user,
                                                                     from_min, leaf, st, keys, err);
  return cudaGetLastError();
}

}  // namespace vg
