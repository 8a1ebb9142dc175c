// Grouping by hashing (the alternative to sorting every point): steps a2-a5 for clouds
// with many points per voxel.
//
// arXiv 2102.11084 Sec. II-C keeps a (cell, point) table in GPU global memory from which
// the number of points of every cell is known.  Here that table is an open-addressing
// hash table in HBM keyed by the voxel's sort key: every point adds its fixed-point
// offset and a count into its voxel's slot, so only the V occupied slots -- not the N
// points -- are then radix-sorted into key order.  Same key, same accumulator and same
// centroid formula as the sort path, so both paths give identical bits.
//
//   hash_insert_kernel   key per point; points of a warp with equal keys are merged
//                        (match.any) and their leader claims/updates one slot
//   hash_compact_kernel  occupied slots -> dense (key, slot) list, digit-0 histogram
//   (radix passes over the V entries, compacted-input mode)
//   hash_finalize_kernel sorted (key, slot) -> key, count, centroid rows; slot -> row
//   hash_p2v_kernel      point -> row through its slot (only when asked for)
//
// Slot claiming: EMPTY -> LOCKED by compare-and-swap, the winner writes the slot's
// accumulator and then publishes the key with a release store; others that see LOCKED
// wait (bounded) and then add with atomics after an acquire load of the key.
#include "vg_device.cuh"
#include "vg_internal.h"
#include "vg_stream.cuh"

namespace vg {
namespace {

constexpr unsigned long long kEmpty = ~0ull;
constexpr unsigned long long kLocked = ~0ull - 1ull;
constexpr uint32_t kNoSlot = 0xffffffffu;

// Inserts accumulator `a` for `key`; returns the slot or kNoSlot (error recorded).
__device__ __forceinline__ uint32_t table_add(unsigned long long* tkeys, HashAcc* tacc,
                                              uint32_t mask, uint64_t key, const Acc& a,
                                              uint32_t spin_limit, int* err) {
  uint32_t h = static_cast<uint32_t>(hash64(key)) & mask;
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    unsigned long long k = ld_acquire64(&tkeys[h]);
    if (k == kEmpty) {
      const unsigned long long prev = atomicCAS(&tkeys[h], kEmpty, kLocked);
      if (prev == kEmpty) {
        tacc[h].n = a.n;
        tacc[h].s[0] = a.s[0];
        tacc[h].s[1] = a.s[1];
        tacc[h].s[2] = a.s[2];
        st_release64(&tkeys[h], key);
        return h;
      }
      k = ld_acquire64(&tkeys[h]);
    }
    uint32_t spins = 0;
    while (k == kLocked) {
      if (++spins > spin_limit) {
        set_error(err, kErrTimeout);
        return kNoSlot;
      }
      if (spins > 16) __nanosleep(32);
      k = ld_acquire64(&tkeys[h]);
    }
    if (k == key) {
      atomicAdd(&tacc[h].n, a.n);
      atomicAdd(reinterpret_cast<unsigned long long*>(&tacc[h].s[0]),
                static_cast<unsigned long long>(a.s[0]));
      atomicAdd(reinterpret_cast<unsigned long long*>(&tacc[h].s[1]),
                static_cast<unsigned long long>(a.s[1]));
      atomicAdd(reinterpret_cast<unsigned long long*>(&tacc[h].s[2]),
                static_cast<unsigned long long>(a.s[2]));
      return h;
    }
    h = (h + 1) & mask;
  }
  set_error(err, kErrCapacity);
  return kNoSlot;
}

template <bool kPosed>
__global__ __launch_bounds__(kStreamThreads) void hash_insert_kernel(
    const float* __restrict__ xyz, FramesArg fr, int have_extent, State* st, FrameState* fs,
    HashTable tab, uint32_t* __restrict__ point_slot, uint32_t spin_limit, int* err) {
  __shared__ ChunkSmem sm;
  __shared__ int s_q[kStreamThreads / 32][32][3];
  __shared__ unsigned long long wmax[kStreamThreads / 32];
  __shared__ uint32_t wcount[kStreamThreads / 32];
  const int F = fr.nframes;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t T = build_chunk_map(fr, sm.off, sm.cstart, sm.tmp, err);
  const uint32_t key_shift = frame_prologue(fr, have_extent != 0, st, fs, T, sm, err);
  uint32_t c0, c1;
  block_range(T, &c0, &c1);
  const bool xyz_vec = (reinterpret_cast<uintptr_t>(xyz) & 15) == 0;
  uint32_t nvalid = 0;
  unsigned long long kmax = 0;
  bool range_bad = false;
  Pose P;
  int pose_f = -1;
  for (uint32_t c = c0; c < c1; ++c) {
    const int f = chunk_frame(sm.cstart, F, c);
    const int64_t start = sm.off[f] + int64_t(c - sm.cstart[f]) * kChunk;
    const int64_t end = min(start + kChunk, sm.off[f + 1]);
    const int64_t p0 = start + int64_t(threadIdx.x) * kStreamPoints;
    float v[12];
    load4(xyz, p0, end, xyz_vec && (start & 3) == 0, v);
    if (kPosed) {
      if (f != pose_f) {
        load_pose(fr, f, P);
        pose_f = f;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) pose_point(P, v[3 * j], v[3 * j + 1], v[3 * j + 2]);
    }
    const float o[3] = {sm.org[f][0], sm.org[f][1], sm.org[f][2]};
    const float leaf = sm.leaf[f];
    const float rleaf = sm.rleaf[f];
    const float inv_unit = sm.inv_unit[f];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      uint64_t local = 0;
      const bool ok = point_key(v[3 * j], v[3 * j + 1], v[3 * j + 2], o, leaf, rleaf, &local, &range_bad);
      const uint64_t key = ok ? key_compose(static_cast<uint32_t>(f), local, key_shift) : 0;
      uint32_t slot = kNoSlot;
      const uint32_t vm = __ballot_sync(kFullMask, ok);
      if (ok) {
        ++nvalid;
        kmax = key > kmax ? key : kmax;
        const Acc a = point_acc(local, v[3 * j], v[3 * j + 1], v[3 * j + 2], o, leaf, inv_unit);
        s_q[warp][lane][0] = static_cast<int>(a.s[0]);
        s_q[warp][lane][1] = static_cast<int>(a.s[1]);
        s_q[warp][lane][2] = static_cast<int>(a.s[2]);
        const uint32_t peers = __match_any_sync(vm, key);
        const int leader = __ffs(peers) - 1;
        __syncwarp(vm);
        if (lane == leader) {
          Acc g = acc_zero();
          for (uint32_t m = peers; m; m &= m - 1) {
            const int l = __ffs(m) - 1;
            g.n += 1;
            g.s[0] += s_q[warp][l][0];
            g.s[1] += s_q[warp][l][1];
            g.s[2] += s_q[warp][l][2];
          }
          slot = table_add(tab.keys, tab.acc, tab.mask, key, g, spin_limit, err);
        }
        slot = __shfl_sync(vm, slot, leader);
        __syncwarp(vm);
      }
      if (point_slot && p0 + j < end) point_slot[p0 + j] = slot;
    }
  }
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
      atomicMax(&st->maxkey, m);
    }
  }
}

// Occupied slots -> dense (key, slot) entries for the radix sort; counts them into
// st->nitems and histograms their digit 0.
__global__ __launch_bounds__(256) void hash_compact_kernel(HashTable tab, State* st,
                                                           uint64_t* __restrict__ keys,
                                                           uint32_t* __restrict__ slots,
                                                           const int* err) {
  __shared__ uint32_t hist[kRadix];
  if (block_error_raised(err)) return;  // an earlier step failed
  hist[threadIdx.x] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint32_t H = tab.mask + 1;
  for (uint32_t base = blockIdx.x * 256u; base < H; base += gridDim.x * 256u) {
    const uint32_t h = base + threadIdx.x;
    const unsigned long long k = h < H ? __ldcg(&tab.keys[h]) : kEmpty;
    const bool occ = k != kEmpty && k != kLocked;
    const uint32_t bal = __ballot_sync(kFullMask, occ);
    uint32_t pos = 0;
    if (lane == 0 && bal) pos = atomicAdd(&st->nitems, __popc(bal));
    pos = __shfl_sync(kFullMask, pos, 0) + __popc(bal & ((1u << lane) - 1u));
    if (occ) {
      keys[pos] = k;
      slots[pos] = h;
      atomicAdd(&hist[k & (kRadix - 1)], 1u);
    }
  }
  __syncthreads();
  if (hist[threadIdx.x]) atomicAdd(&st->hist[0][threadIdx.x], hist[threadIdx.x]);
}

// Sorted (key, slot) entries -> output rows.
__global__ __launch_bounds__(256) void hash_finalize_kernel(
    const State* st, const FrameState* __restrict__ fs, int nframes,
    const uint64_t* __restrict__ keys0, const uint32_t* __restrict__ idx0,
    const uint64_t* __restrict__ keys1, const uint32_t* __restrict__ idx1, HashTable tab,
    uint32_t* __restrict__ slot_rank, SegOut out, int* err) {
  if (error_raised(err)) return;  // an earlier step failed
  const int64_t V = st->nitems;
  const int64_t i = int64_t(blockIdx.x) * 256 + threadIdx.x;
  if (i >= V) return;
  const int passes = max(1, sort_passes(st->maxkey));
  const uint64_t* K = (passes & 1) ? keys1 : keys0;
  const uint32_t* I = (passes & 1) ? idx1 : idx0;
  const uint32_t key_shift = st->key_shift;
  const uint64_t key = K[i];
  const uint32_t slot = I[i];
  const uint32_t f = key_frame(key, key_shift);
  if (i >= out.cap) {
    set_error(err, kErrCapacity);
  } else {
    Acc a;
    a.n = __ldcg(&tab.acc[slot].n);
    a.s[0] = __ldcg(&tab.acc[slot].s[0]);
    a.s[1] = __ldcg(&tab.acc[slot].s[1]);
    a.s[2] = __ldcg(&tab.acc[slot].s[2]);
    const uint64_t local = key_local(key, key_shift);
    const float o[3] = {fs[f].origin[0], fs[f].origin[1], fs[f].origin[2]};
    const float leaf = fs[f].leaf;
    float c[3];
    acc_centroid(local, a, o, leaf, leaf, c);
    out.keys[i] = local;
    out.counts[i] = a.n;
    out.centroids[3 * i] = c[0];
    out.centroids[3 * i + 1] = c[1];
    out.centroids[3 * i + 2] = c[2];
    if (out.sums) {
      out.sums[3 * i] = a.s[0];
      out.sums[3 * i + 1] = a.s[1];
      out.sums[3 * i + 2] = a.s[2];
    }
  }
  if (slot_rank) slot_rank[slot] = static_cast<uint32_t>(i);
  if (out.frame_offsets) {
    if (i > 0) {
      const uint32_t fp = key_frame(K[i - 1], key_shift);
      for (uint32_t g = fp + 1; g <= f; ++g) out.frame_offsets[g] = i;
    }
    if (i == V - 1)
      for (uint32_t g = f + 1; g <= uint32_t(nframes); ++g) out.frame_offsets[g] = V;
  }
  if (i == V - 1) *out.num_voxels = V;
}

__global__ __launch_bounds__(256) void hash_p2v_kernel(const uint32_t* __restrict__ point_slot,
                                                       const uint32_t* __restrict__ slot_rank,
                                                       int64_t n, int32_t* __restrict__ p2v,
                                                       const int* err) {
  if (error_raised(err)) return;  // an earlier step failed
  for (int64_t i = int64_t(blockIdx.x) * 256 + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * 256) {
    const uint32_t s = point_slot[i];
    p2v[i] = s == kNoSlot ? -1 : static_cast<int32_t>(slot_rank[s]);
  }
}

}  // namespace

cudaError_t launch_hash_insert(const float* xyz, const FramesArg& fr, bool have_extent, State* st,
                               FrameState* fs, const HashTable& tab, uint32_t* point_slot,
                               uint32_t spin_limit, int* err, cudaStream_t stream) {
  if (posed(fr))
    hash_insert_kernel<true><<<stream_grid(fr), kStreamThreads, 0, stream>>>(
        xyz, fr, have_extent ? 1 : 0, st, fs, tab, point_slot, spin_limit, err);
  else
    hash_insert_kernel<false><<<stream_grid(fr), kStreamThreads, 0, stream>>>(
        xyz, fr, have_extent ? 1 : 0, st, fs, tab, point_slot, spin_limit, err);
  return cudaGetLastError();
}

cudaError_t launch_hash_compact(const HashTable& tab, State* st, uint64_t* keys, uint32_t* slots,
                                const int* err, cudaStream_t stream) {
  const int64_t H = int64_t(tab.mask) + 1;
  const int64_t want = ceil_div(H, 256);
  const int64_t cap = int64_t(num_sms()) * 16;
  hash_compact_kernel<<<static_cast<int>(want < cap ? want : cap), 256, 0, stream>>>(tab, st, keys,
                                                                                    slots, err);
  return cudaGetLastError();
}

cudaError_t launch_hash_finalize(const State* st, const FrameState* fs, int nframes,
                                 const uint64_t* keys0, const uint32_t* idx0,
                                 const uint64_t* keys1, const uint32_t* idx1,
                                 const HashTable& tab, uint32_t* slot_rank, int64_t n_max,
                                 const SegOut& out, int* err, cudaStream_t stream) {
  if (n_max == 0) return cudaSuccess;
  hash_finalize_kernel<<<static_cast<int>(ceil_div(n_max, 256)), 256, 0, stream>>>(
      st, fs, nframes, keys0, idx0, keys1, idx1, tab, slot_rank, out, err);
  return cudaGetLastError();
}

cudaError_t launch_hash_p2v(const uint32_t* point_slot, const uint32_t* slot_rank, int64_t n,
                            int32_t* p2v, const int* err, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const int64_t want = ceil_div(n, 256);
  const int64_t cap = int64_t(num_sms()) * 16;
  hash_p2v_kernel<<<static_cast<int>(want < cap ? want : cap), 256, 0, stream>>>(
      point_slot, slot_rank, n, p2v, err);
  return cudaGetLastError();
}

}  // namespace vg
