// Steps a1 (origin = per-frame cloud minimum) and a2 (sort key per point).
//
// arXiv 2102.11084 Sec. II-C normalises each point and classifies it into one cell of an
// ordered subdivision of space (the classification and table update of Algorithm 1);
// here the cell is the voxel of an unbounded lattice with a caller-chosen origin and
// leaf, keyed by a 63-bit Morton code.  Both kernels stream xyz once with 16-byte loads
// (4 points = 3 float4 per lane) over chunks of 1024 points that never cross a frame,
// each block walking a contiguous run of chunks; they are HBM-bound.
#include <type_traits>

#include "vg_device.cuh"
#include "vg_internal.h"
#include "vg_stream.cuh"

namespace vg {
namespace {

// Reduces per-thread min/max over the block and folds them into frame f's state.
__device__ __forceinline__ void flush_extent(float mn[3], float mx[3], FrameState* fs, int f,
                                             float (*red)[6]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      mn[a] = fminf(mn[a], __shfl_xor_sync(kFullMask, mn[a], off));
      mx[a] = fmaxf(mx[a], __shfl_xor_sync(kFullMask, mx[a], off));
    }
  }
  __syncthreads();
  if (lane == 0) {
    for (int a = 0; a < 3; ++a) {
      red[warp][a] = mn[a];
      red[warp][3 + a] = mx[a];
    }
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    const int a = threadIdx.x;
    float m = INFINITY, M = -INFINITY;
    for (int w = 0; w < kStreamThreads / 32; ++w) {
      m = fminf(m, red[w][a]);
      M = fmaxf(M, red[w][3 + a]);
    }
    if (m != INFINITY) {
      atomicMax(&fs[f].ord_min_inv[a], ~float_to_ordered(m));
      atomicMax(&fs[f].ord_max[a], float_to_ordered(M));
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    mn[a] = INFINITY;
    mx[a] = -INFINITY;
  }
}

// a1: per-frame minimum and maximum over the valid points.
template <bool kPosed>
__global__ __launch_bounds__(kStreamThreads) void origin_kernel(const float* __restrict__ xyz,
                                                                FramesArg fr, FrameState* fs,
                                                                int* err, uint4* zero,
                                                                size_t zero16) {
  // only the frame/chunk map (no per-frame origin or leaf is needed here)
  __shared__ struct {
    int64_t off[kMaxFrames + 1];
    uint32_t cstart[kMaxFrames + 1];
    uint32_t tmp[kStreamThreads / 32];
  } sm;
  __shared__ float red[kStreamThreads / 32][6];
  for (size_t i = size_t(blockIdx.x) * kStreamThreads + threadIdx.x; i < zero16;
       i += size_t(gridDim.x) * kStreamThreads)
    zero[i] = make_uint4(0u, 0u, 0u, 0u);
  const uint32_t T = build_chunk_map(fr, sm.off, sm.cstart, sm.tmp, err);
  uint32_t c0, c1;
  block_range(T, &c0, &c1);
  const bool xyz_vec = (reinterpret_cast<uintptr_t>(xyz) & 15) == 0;
  float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  int cur = -1;
  Pose P;
  for (uint32_t c = c0; c < c1; ++c) {
    const int f = chunk_frame(sm.cstart, fr.nframes, c);
    if (f != cur) {
      if (cur >= 0) flush_extent(mn, mx, fs, cur, red);
      cur = f;
      if (kPosed) load_pose(fr, f, P);
    }
    const int64_t start = sm.off[f] + int64_t(c - sm.cstart[f]) * kChunk;
    const int64_t end = min(start + kChunk, sm.off[f + 1]);
    const int64_t p0 = start + int64_t(threadIdx.x) * kStreamPoints;
    float v[12];
    load4(xyz, p0, end, xyz_vec && (start & 3) == 0, v);
    if (kPosed) {
#pragma unroll
      for (int j = 0; j < 4; ++j) pose_point(P, v[3 * j], v[3 * j + 1], v[3 * j + 2]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (point_valid(v[3 * j], v[3 * j + 1], v[3 * j + 2])) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          mn[a] = fminf(mn[a], v[3 * j + a]);
          mx[a] = fmaxf(mx[a], v[3 * j + a]);
        }
      }
    }
  }
  if (cur >= 0) flush_extent(mn, mx, fs, cur, red);
}

// The streaming loop of the key kernel over this block's chunks.  kNarrow: 32-bit keys
// (every key fits, checked from the extents) and packed corner offsets as payload;
// otherwise 64-bit keys only.  Accumulates the first sorted digit's histogram (digit 0,
// or the digit at the bucket shift in the bucket tail), #valid and the largest
// key.
template <bool kPosed, bool kNarrow>
__device__ __forceinline__ void key_loop(const float* __restrict__ xyz, const FramesArg& fr,
                                         const ChunkSmem& sm, uint32_t c0, uint32_t c1,
                                         uint32_t key_shift, uint64_t* __restrict__ keys,
                                         uint32_t* __restrict__ keys32,
                                         uint64_t* __restrict__ payload, uint32_t* hist,
                                         uint32_t hshift, uint32_t& nvalid,
                                         unsigned long long& kmax_out, bool& range_bad) {
  using KeyT = typename std::conditional<kNarrow, uint32_t, uint64_t>::type;
  const int F = fr.nframes;
  const bool xyz_vec = (reinterpret_cast<uintptr_t>(xyz) & 15) == 0;
  const bool key_vec = kNarrow ? (reinterpret_cast<uintptr_t>(keys32) & 15) == 0
                               : (reinterpret_cast<uintptr_t>(keys) & 15) == 0;
  const bool pay_vec = !kNarrow || (reinterpret_cast<uintptr_t>(payload) & 15) == 0;
  KeyT kmax = 0;
  // software pipeline: the next chunk's points are loaded while this one is computed
  float vn[12];
  if (c0 < c1) {
    const int f = chunk_frame(sm.cstart, F, c0);
    const int64_t start = sm.off[f] + int64_t(c0 - sm.cstart[f]) * kChunk;
    load4(xyz, start + int64_t(threadIdx.x) * kStreamPoints, min(start + kChunk, sm.off[f + 1]),
          xyz_vec && (start & 3) == 0, vn);
  }
  Pose P;
  int pose_f = -1;
  for (uint32_t c = c0; c < c1; ++c) {
    const int f = chunk_frame(sm.cstart, F, c);
    const int64_t start = sm.off[f] + int64_t(c - sm.cstart[f]) * kChunk;
    const int64_t end = min(start + kChunk, sm.off[f + 1]);
    const int64_t p0 = start + int64_t(threadIdx.x) * kStreamPoints;
    const bool vec = (start & 3) == 0;
    float v[12];
#pragma unroll
    for (int x = 0; x < 12; ++x) v[x] = vn[x];
    if (kPosed) {
      if (f != pose_f) {
        load_pose(fr, f, P);
        pose_f = f;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) pose_point(P, v[3 * j], v[3 * j + 1], v[3 * j + 2]);
    }
    if (c + 1 < c1) {
      const int fn = chunk_frame(sm.cstart, F, c + 1);
      const int64_t sn = sm.off[fn] + int64_t(c + 1 - sm.cstart[fn]) * kChunk;
      load4(xyz, sn + int64_t(threadIdx.x) * kStreamPoints, min(sn + kChunk, sm.off[fn + 1]),
            xyz_vec && (sn & 3) == 0, vn);
    }
    const float o[3] = {sm.org[f][0], sm.org[f][1], sm.org[f][2]};
    const float leaf = sm.leaf[f];
    const float rleaf = sm.rleaf[f];
    const float inv_unit = sm.inv_unit[f];
    KeyT k[4];
    uint64_t pay[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      bool ok;
      pay[j] = kPayloadInvalid;
      if (kNarrow) {
        uint32_t k32 = 0;
        ok = narrow_entry(v[3 * j], v[3 * j + 1], v[3 * j + 2], o, leaf, rleaf, inv_unit,
                          static_cast<uint32_t>(f), key_shift, &k32, &pay[j], &range_bad);
        k[j] = ok ? static_cast<KeyT>(k32) : static_cast<KeyT>(kKeySentinel);
      } else {
        uint32_t ijk[3];
        ok = point_index(v[3 * j], v[3 * j + 1], v[3 * j + 2], o, leaf, rleaf, ijk, &range_bad);
        k[j] = ok ? key_compose(static_cast<uint32_t>(f), morton3(ijk[0], ijk[1], ijk[2]),
                                key_shift)
                  : kKeySentinel;
      }
      if (ok) {
        ++nvalid;
        kmax = k[j] > kmax ? k[j] : kmax;
        atomicAdd(&hist[uint32_t(k[j] >> hshift) & (kRadix - 1)], 1u);
      }
    }
    if (kNarrow) {
      if (key_vec && pay_vec && vec && p0 + 4 <= end) {
        __stcg(reinterpret_cast<uint4*>(keys32 + p0),
               make_uint4(uint32_t(k[0]), uint32_t(k[1]), uint32_t(k[2]), uint32_t(k[3])));
        ulonglong2* dst = reinterpret_cast<ulonglong2*>(payload + p0);
        __stcg(dst, make_ulonglong2(pay[0], pay[1]));
        __stcg(dst + 1, make_ulonglong2(pay[2], pay[3]));
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (p0 + j < end) {
            keys32[p0 + j] = uint32_t(k[j]);
            payload[p0 + j] = pay[j];
          }
      }
    } else if (key_vec && vec && p0 + 4 <= end) {
      ulonglong2* dst = reinterpret_cast<ulonglong2*>(keys + p0);
      __stcg(dst, make_ulonglong2(uint64_t(k[0]), uint64_t(k[1])));
      __stcg(dst + 1, make_ulonglong2(uint64_t(k[2]), uint64_t(k[3])));
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (p0 + j < end) keys[p0 + j] = uint64_t(k[j]);
    }
  }
  kmax_out = kmax;
}

// a2: sort key per point (kKeySentinel for invalid or out-of-range rows), plus the
// histogram of the first sorted digit of the valid keys, the number of valid points and
// the largest key.
// Block 0 also publishes every frame's origin and leaf (and the minimum to the caller
// when the origin is computed) and the key shift.
template <bool kPosed>
__global__ __launch_bounds__(kStreamThreads, kPosed ? 1 : VG_KEY_MINB) void key_kernel(
    const float* __restrict__ xyz, FramesArg fr, int have_extent, State* st, FrameState* fs,
    uint64_t* __restrict__ keys, uint32_t* __restrict__ keys32, uint64_t* __restrict__ payload,
    int* err) {
  __shared__ ChunkSmem sm;
  __shared__ uint32_t hist[kRadix];
  __shared__ unsigned long long wmax[kStreamThreads / 32];
  __shared__ uint32_t wcount[kStreamThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kRadix; d += kStreamThreads) hist[d] = 0;
  const uint32_t T = build_chunk_map(fr, sm.off, sm.cstart, sm.tmp, err);
  bool narrow = false;
  uint32_t bshift = 0;
  const uint32_t key_shift =
      frame_prologue(fr, have_extent != 0, st, fs, T, sm, err, &narrow, &bshift);
  narrow = narrow && keys32 && payload;
  uint32_t c0, c1;
  block_range(T, &c0, &c1);
  uint32_t nvalid = 0;
  unsigned long long kmax = 0;
  bool range_bad = false;
  if (narrow)
    key_loop<kPosed, true>(xyz, fr, sm, c0, c1, key_shift, keys, keys32, payload, hist, bshift,
                           nvalid, kmax, range_bad);
  else
    key_loop<kPosed, false>(xyz, fr, sm, c0, c1, key_shift, keys, keys32, payload, hist, 0u,
                            nvalid, kmax, range_bad);
  if (__any_sync(kFullMask, range_bad) && lane == 0) set_error(err, kErrRange);
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    nvalid += __shfl_xor_sync(kFullMask, nvalid, off);
    const unsigned long long other = __shfl_xor_sync(kFullMask, kmax, off);
    kmax = other > kmax ? other : kmax;
  }
  if (lane == 0) {
    wcount[warp] = nvalid;
    wmax[warp] = kmax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t cnt = 0;
    unsigned long long m = 0;
    for (int w = 0; w < kStreamThreads / 32; ++w) {
      cnt += wcount[w];
      m = wmax[w] > m ? wmax[w] : m;
    }
    if (cnt) {
      atomicAdd(&st->nvalid, cnt);
      atomicAdd(&st->nitems, cnt);
      atomicMax(&st->maxkey, m);
    }
  }
  for (int d = threadIdx.x; d < kRadix; d += kStreamThreads)
    if (hist[d]) atomicAdd(&st->hist[0][d], hist[d]);
}

}  // namespace

int stream_grid(const FramesArg& fr) {
  const int64_t want = max_chunks(fr.n, fr.nframes);
  const int64_t cap = int64_t(num_sms()) * (fr.grid_per_sm > 0 ? fr.grid_per_sm : 8);
  return static_cast<int>(want < 1 ? 1 : (want < cap ? want : cap));
}

cudaError_t launch_origin(const float* xyz, const FramesArg& fr, State* st, FrameState* fs,
                          int* err, cudaStream_t stream, void* zero, size_t zero_bytes) {
  (void)st;
  if (fr.n == 0) {
    return zero_bytes ? cudaMemsetAsync(zero, 0, zero_bytes, stream) : cudaSuccess;
  }
  uint4* z = static_cast<uint4*>(zero);
  const size_t z16 = zero ? zero_bytes / 16 : 0;
  if (posed(fr))
    origin_kernel<true><<<stream_grid(fr), kStreamThreads, 0, stream>>>(xyz, fr, fs, err, z, z16);
  else
    origin_kernel<false><<<stream_grid(fr), kStreamThreads, 0, stream>>>(xyz, fr, fs, err, z, z16);
  return cudaGetLastError();
}

cudaError_t launch_keys(const float* xyz, const FramesArg& fr, bool have_extent, State* st,
                        FrameState* fs, uint64_t* keys, int* err, cudaStream_t stream) {
  return launch_keys_any(xyz, fr, have_extent, st, fs, keys, nullptr, nullptr, err, stream);
}

cudaError_t launch_keys_any(const float* xyz, const FramesArg& fr, bool have_extent, State* st,
                            FrameState* fs, uint64_t* keys64, uint32_t* keys32,
                            uint64_t* payload, int* err, cudaStream_t stream) {
  // Always at least one block: it publishes the origins and leaves the call used.
  if (posed(fr))
    key_kernel<true><<<stream_grid(fr), kStreamThreads, 0, stream>>>(
        xyz, fr, have_extent ? 1 : 0, st, fs, keys64, keys32, payload, err);
  else
    key_kernel<false><<<stream_grid(fr), kStreamThreads, 0, stream>>>(
        xyz, fr, have_extent ? 1 : 0, st, fs, keys64, keys32, payload, err);
  return cudaGetLastError();
}

}  // namespace vg
