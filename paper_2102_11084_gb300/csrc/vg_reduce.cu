// Steps a4 + a5 (sort path): one output voxel per run of equal keys in the sorted table,
// with its point count and centroid, written densely in ascending key order.
//
// arXiv 2102.11084 Sec. II-C: once "tabla_subdiv" is sorted, the points of each cell are
// contiguous and the number of points per cell is known; the filtered cloud keeps one
// point per occupied cell (the centroid, as the voxel-grid filter the paper replaces).
//
// One kernel: every tile (256 threads x 8 sorted entries, tile id from an atomic ticket)
//   1. flags run heads, gathers its points and quantises each offset from the voxel
//      corner (see vg_device.cuh);
//   2. does a block-wide segmented scan of (heads, open-run partial) over its threads;
//   3. joins a chained scan over tiles (decoupled look-back with separate aggregate and
//      inclusive records, release/acquire ordering, bounded waits) that gives it the
//      number of voxels before it and the partial of the run still open at its start;
//   4. emits each run at its last entry: key, count and centroid at the run's rank.
// Integer sums make the result independent of tile size and of the order of the points.
#include <type_traits>

#include "vg_device.cuh"
#include "vg_internal.h"

namespace vg {
namespace {

constexpr unsigned kFull = kFullMask;

// A segmented-scan value: number of run heads, and the partial sums of the run that is
// open at the end of the segment.
struct Seg {
  uint32_t h;
  Acc a;
};

__device__ __forceinline__ Seg seg_identity() {
  Seg s;
  s.h = 0;
  s.a = acc_zero();
  return s;
}

// x (earlier) then y (later).
__device__ __forceinline__ Seg seg_combine(const Seg& x, const Seg& y) {
  Seg r;
  r.h = x.h + y.h;
  if (y.h > 0) {
    r.a = y.a;
  } else {
    r.a = x.a;
    acc_add(r.a, y.a);
  }
  return r;
}

__device__ __forceinline__ Seg seg_shfl_up(const Seg& s, int off) {
  Seg r;
  r.h = __shfl_up_sync(kFull, s.h, off);
  r.a.n = __shfl_up_sync(kFull, s.a.n, off);
#pragma unroll
  for (int a = 0; a < 3; ++a) r.a.s[a] = __shfl_up_sync(kFull, s.a.s[a], off);
  return r;
}

__device__ __forceinline__ Seg seg_shfl_down(const Seg& s, int off) {
  Seg r;
  r.h = __shfl_down_sync(kFull, s.h, off);
  r.a.n = __shfl_down_sync(kFull, s.a.n, off);
#pragma unroll
  for (int a = 0; a < 3; ++a) r.a.s[a] = __shfl_down_sync(kFull, s.a.s[a], off);
  return r;
}

// Exclusive prefix of tile `tile` over tiles 0..tile-1, by one warp: each round reads the
// status of 32 predecessors at once (lane l: tile j - l), waits (bounded) until every
// tile up to the nearest one with an inclusive prefix is ready, and folds them in tile
// order with a shuffle tree.  Returns the same value to every lane.
__device__ __forceinline__ Seg warp_lookback(const SegStatus* lb, int tile, int lane,
                                             uint32_t spin_limit, int* err) {
  Seg suffix = seg_identity();
  int j = tile - 1;
  uint32_t spins = 0;
  while (true) {
    const int jt = j - lane;
    const uint32_t f = jt >= 0 ? ld_acquire(&lb[jt].flag) : 2u;
    const uint32_t prefix_lanes = __ballot_sync(kFull, f == 2u);
    const int plane = prefix_lanes ? __ffs(prefix_lanes) - 1 : 31;
    const uint32_t need = plane == 31 ? kFull : ((2u << plane) - 1u);
    const uint32_t not_ready = __ballot_sync(kFull, f == 0u) & need;
    if (not_ready) {
      if (++spins > spin_limit) {
        set_error(err, kErrTimeout);
        return suffix;
      }
      if (spins > 64) __nanosleep(64);
      continue;
    }
    Seg v = seg_identity();
    if (((need >> lane) & 1u) && jt >= 0) {
      const SegStatus* o = lb + jt;
      if (f == 1u) {
        v.h = __ldcg(&o->heads_agg);
        v.a.n = __ldcg(&o->n_agg);
        for (int a = 0; a < 3; ++a) v.a.s[a] = __ldcg(&o->s_agg[a]);
      } else {
        v.h = __ldcg(&o->heads_incl);
        v.a.n = __ldcg(&o->n_incl);
        for (int a = 0; a < 3; ++a) v.a.s[a] = __ldcg(&o->s_incl[a]);
      }
    }
    // lane l holds tile j - l: higher lanes are earlier tiles
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const Seg o = seg_shfl_down(v, off);
      if (lane + off < 32) v = seg_combine(o, v);
    }
    Seg w;
    w.h = __shfl_sync(kFull, v.h, 0);
    w.a.n = __shfl_sync(kFull, v.a.n, 0);
    for (int a = 0; a < 3; ++a) w.a.s[a] = __shfl_sync(kFull, v.a.s[a], 0);
    suffix = seg_combine(w, suffix);
    if (prefix_lanes) return suffix;
    j -= 32;
  }
}

// Output rows of one tile, staged in shared memory and written out coalesced.
struct Stage {
  uint64_t* key;    // [kSegTile + 1]
  uint32_t* count;  // [kSegTile + 1]; 0 = not emitted by this tile
  float* cent;      // [3 * (kSegTile + 1)]
};

// Stages voxel v (sort key `key`, sums `a`) at e = v - e0 of this tile.  o1/leaf1: the
// frame's origin and leaf when the call has one frame (key_shift == 64).
__device__ __forceinline__ void emit_voxel(uint32_t v, int64_t e0, uint64_t key, const Acc& a,
                                           const FrameState* fs, uint32_t key_shift,
                                           const float o1[3], float leaf1, const SegOut& out,
                                           const Stage& sg, int* err) {
  if (int64_t(v) >= out.cap) {
    set_error(err, kErrCapacity);
    return;
  }
  const uint64_t local = key_local(key, key_shift);
  float o[3] = {o1[0], o1[1], o1[2]};
  float leaf = leaf1;
  if (key_shift < 64) {
    const uint32_t f = key_frame(key, key_shift);
    o[0] = fs[f].origin[0];
    o[1] = fs[f].origin[1];
    o[2] = fs[f].origin[2];
    leaf = fs[f].leaf;
  }
  float c[3];
  acc_centroid(local, a, o, leaf, leaf, c);
  const int e = static_cast<int>(int64_t(v) - e0);
  sg.key[e] = local;
  sg.count[e] = a.n;
  sg.cent[3 * e] = c[0];
  sg.cent[3 * e + 1] = c[1];
  sg.cent[3 * e + 2] = c[2];
  if (out.sums) {
    out.sums[3 * size_t(v)] = a.s[0];
    out.sums[3 * size_t(v) + 1] = a.s[1];
    out.sums[3 * size_t(v) + 2] = a.s[2];
  }
}

// Output offsets of frames (f_prev, f_new] start at voxel v.
__device__ __forceinline__ void mark_frames(int64_t* fo, uint32_t f_prev, uint32_t f_new,
                                            uint32_t v) {
  if (!fo) return;
  for (uint32_t f = f_prev + 1; f <= f_new; ++f) fo[f] = v;
}

}  // namespace

// Shared-memory bytes of the reduction: the staged rows; the sorted input entries of a tile
// (keys and payloads) overlay the same bytes before they are consumed.
constexpr size_t kSegStageBytes =
    size_t(kSegTile + 1) * (sizeof(uint64_t) + sizeof(uint32_t) + 3 * sizeof(float));
static_assert(kSegStageBytes >= size_t(kSegTile) * 2 * sizeof(uint64_t), "stage overlay");

namespace {

// kNarrow: 32-bit keys with the packed offsets as payload (no gather); otherwise 64-bit
// keys with the point index as payload, whose coordinates are gathered.  Persistent: each
// block takes tiles from a ticket until none is left.  A launch whose layout was not
// chosen returns before taking a ticket.
template <bool kNarrow>
__global__ __launch_bounds__(kSegThreads, kSegMinBlocks) void segreduce_kernel(
    State* st, const FrameState* __restrict__ fs, int nframes, const void* keys0_,
    const void* pay0_, const void* keys1_, const void* pay1_, const float* __restrict__ xyz,
    SegStatus* lb, SegOut out, uint32_t spin_limit, int* err) {
  using KeyT = typename std::conditional<kNarrow, uint32_t, uint64_t>::type;
  using PayT = typename std::conditional<kNarrow, uint64_t, uint32_t>::type;
  extern __shared__ __align__(16) unsigned char seg_smem[];
  __shared__ Seg wtot[kSegThreads / 32];
  __shared__ Seg s_tile_excl;
  __shared__ uint32_t s_tile_heads;
  __shared__ uint64_t s_prev_key;
  __shared__ int s_tile;
  if ((st->narrow != 0) != kNarrow) return;

  uint64_t* skeys = reinterpret_cast<uint64_t*>(seg_smem);
  PayT* sidx = reinterpret_cast<PayT*>(seg_smem + size_t(kSegTile) * sizeof(uint64_t));
  Stage sg;
  sg.key = reinterpret_cast<uint64_t*>(seg_smem);
  sg.count = reinterpret_cast<uint32_t*>(seg_smem + size_t(kSegTile + 1) * sizeof(uint64_t));
  sg.cent = reinterpret_cast<float*>(seg_smem + size_t(kSegTile + 1) * (sizeof(uint64_t) +
                                                                         sizeof(uint32_t)));

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t nitems = st->nitems;
  const int64_t ntiles = ceil_div(nitems, kSegTile);
  const uint32_t key_shift = st->key_shift;
  const int passes = max(1, sort_passes(st->maxkey));
  const KeyT* K = static_cast<const KeyT*>((passes & 1) ? keys1_ : keys0_);
  const PayT* I = static_cast<const PayT*>((passes & 1) ? pay1_ : pay0_);
  (void)xyz;
  const float o1[3] = {fs[0].origin[0], fs[0].origin[1], fs[0].origin[2]};
  const float leaf1 = fs[0].leaf;

  for (;;) {
    if (t == 0) s_tile = static_cast<int>(atomicAdd(&st->tile_ctr[kMaxPasses], 1u));
    __syncthreads();
    const int tile = s_tile;
    if (tile >= ntiles) break;
    const int64_t base = int64_t(tile) * kSegTile;
    const int cnt = static_cast<int>(nitems - base < kSegTile ? nitems - base : kSegTile);

    for (int i = t; i < cnt; i += kSegThreads) {
      skeys[i] = uint64_t(__ldcs(K + base + i));
      sidx[i] = __ldcs(I + base + i);
    }
    if (t == 0) s_prev_key = base > 0 ? uint64_t(K[base - 1]) : 0ull;
    __syncthreads();

    // ---- this thread's entries (blocked: t*8 .. t*8+7) ----
    uint64_t k[kSegItems];
    uint32_t pi[kSegItems];
    int q[kSegItems][3];
    uint32_t headmask = 0;
    const int first = t * kSegItems;
    const uint64_t prev0 = first == 0 ? s_prev_key : skeys[first > 0 ? first - 1 : 0];
    Seg mine = seg_identity();
#pragma unroll
    for (int j = 0; j < kSegItems; ++j) {
      const int li = first + j;
      if (li < cnt) {
        k[j] = skeys[li];
        const uint64_t pk = j == 0 ? prev0 : k[j - 1];
        const bool head = (base + li == 0) || (k[j] != pk);
        headmask |= uint32_t(head) << j;
        Acc a;
        if (kNarrow) {
          const uint64_t w = uint64_t(sidx[li]);
          pi[j] = 0;
          a.n = 1;
          a.s[0] = unpack_offset(w, 0);
          a.s[1] = unpack_offset(w, 1);
          a.s[2] = unpack_offset(w, 2);
        } else {
          pi[j] = uint32_t(sidx[li]);
          const uint32_t f = key_frame(k[j], key_shift);
          const float o[3] = {fs[f].origin[0], fs[f].origin[1], fs[f].origin[2]};
          const float leaf = fs[f].leaf;
          const float* p = xyz + 3 * size_t(pi[j]);
          a = point_acc(key_local(k[j], key_shift), __ldg(p), __ldg(p + 1), __ldg(p + 2), o,
                        leaf, quant_inv_unit(leaf));
        }
        q[j][0] = static_cast<int>(a.s[0]);
        q[j][1] = static_cast<int>(a.s[1]);
        q[j][2] = static_cast<int>(a.s[2]);
        if (head) {
          mine.h += 1;
          mine.a = acc_zero();
        }
        acc_add(mine.a, a);
      } else {
        k[j] = 0;
        pi[j] = 0;
        q[j][0] = q[j][1] = q[j][2] = 0;
      }
    }

    // ---- block segmented scan over threads ----
    Seg incl = mine;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const Seg y = seg_shfl_up(incl, off);
      if (lane >= off) incl = seg_combine(y, incl);
    }
    Seg lane_excl = seg_shfl_up(incl, 1);
    if (lane == 0) lane_excl = seg_identity();
    if (lane == 31) wtot[warp] = incl;
    __syncthreads();

    if (warp == 0) {
      Seg agg = seg_identity();
      for (int w = 0; w < kSegThreads / 32; ++w) agg = seg_combine(agg, wtot[w]);
      SegStatus* me = lb + tile;
      Seg excl = seg_identity();
      if (tile == 0) {
        if (lane == 0) {
          me->heads_incl = agg.h;
          me->n_incl = agg.a.n;
          for (int a = 0; a < 3; ++a) me->s_incl[a] = agg.a.s[a];
          st_release(&me->flag, 2u);
        }
      } else {
        if (lane == 0) {
          me->heads_agg = agg.h;
          me->n_agg = agg.a.n;
          for (int a = 0; a < 3; ++a) me->s_agg[a] = agg.a.s[a];
          st_release(&me->flag, 1u);
        }
        excl = warp_lookback(lb, tile, lane, spin_limit, err);
        if (lane == 0) {
          const Seg inc = seg_combine(excl, agg);
          me->heads_incl = inc.h;
          me->n_incl = inc.a.n;
          for (int a = 0; a < 3; ++a) me->s_incl[a] = inc.a.s[a];
          st_release(&me->flag, 2u);
        }
      }
      if (lane == 0) {
        s_tile_excl = excl;
        s_tile_heads = agg.h;
      }
    }
    __syncthreads();

    // rows this tile can emit: [e0, e0 + span), staged from here on (inputs are consumed)
    const uint32_t H0 = s_tile_excl.h;
    const int64_t e0 = H0 > 0 ? int64_t(H0) - 1 : 0;
    const int span = static_cast<int>(int64_t(H0) + s_tile_heads - e0);
    for (int e = t; e < span; e += kSegThreads) sg.count[e] = 0;
    Seg wexcl = seg_identity();
    for (int w = 0; w < warp; ++w) wexcl = seg_combine(wexcl, wtot[w]);
    const Seg pre = seg_combine(seg_combine(s_tile_excl, wexcl), lane_excl);
    __syncthreads();

    // ---- emit every run at its last entry ----
    uint32_t H = pre.h;
    Acc run = pre.a;
#pragma unroll
    for (int j = 0; j < kSegItems; ++j) {
      const int li = first + j;
      if (li >= cnt) break;
      const int64_t gi = base + li;
      if ((headmask >> j) & 1u) {
        if (gi > 0) {
          const uint64_t pk = j == 0 ? prev0 : k[j - 1];
          emit_voxel(H - 1, e0, pk, run, fs, key_shift, o1, leaf1, out, sg, err);
          mark_frames(out.frame_offsets, key_frame(pk, key_shift), key_frame(k[j], key_shift), H);
        }
        H += 1;
        run = acc_zero();
      }
      run.n += 1;
      run.s[0] += q[j][0];
      run.s[1] += q[j][1];
      run.s[2] += q[j][2];
      if (!kNarrow && out.p2v) out.p2v[pi[j]] = static_cast<int32_t>(H - 1);
      if (gi == nitems - 1) {
        emit_voxel(H - 1, e0, k[j], run, fs, key_shift, o1, leaf1, out, sg, err);
        *out.num_voxels = H;
        mark_frames(out.frame_offsets, key_frame(k[j], key_shift), uint32_t(nframes), H);
      }
    }
    __syncthreads();

    // ---- coalesced write-out of the staged rows ----
    for (int e = t; e < span; e += kSegThreads) {
      if (sg.count[e]) {
        out.keys[e0 + e] = sg.key[e];
        out.counts[e0 + e] = sg.count[e];
      }
    }
    for (int x = t; x < 3 * span; x += kSegThreads)
      if (sg.count[x / 3]) out.centroids[3 * e0 + x] = sg.cent[x];
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_segreduce(State* st, const FrameState* fs, int nframes,
                             const uint64_t* keys0, const uint32_t* idx0, const uint64_t* keys1,
                             const uint32_t* idx1, const float* xyz, SegStatus* lb,
                             int64_t n_max, const SegOut& out, uint32_t spin_limit, int* err,
                             cudaStream_t stream) {
  if (n_max == 0) return cudaSuccess;
  const int grid = persistent_grid(reinterpret_cast<const void*>(segreduce_kernel<false>),
                                   kSegThreads, kSegStageBytes, ceil_div(n_max, kSegTile));
  segreduce_kernel<false><<<grid, kSegThreads, kSegStageBytes, stream>>>(
      st, fs, nframes, keys0, idx0, keys1, idx1, xyz, lb, out, spin_limit, err);
  return cudaGetLastError();
}

void warm_reduce_config() {
  persistent_grid(reinterpret_cast<const void*>(segreduce_kernel<false>), kSegThreads,
                  kSegStageBytes, 1);
  persistent_grid(reinterpret_cast<const void*>(segreduce_kernel<true>), kSegThreads,
                  kSegStageBytes, 1);
}

cudaError_t launch_segreduce_narrow(State* st, const FrameState* fs, int nframes,
                                    const uint32_t* k0, const uint64_t* p0, const uint32_t* k1,
                                    const uint64_t* p1, SegStatus* lb, int64_t n_max,
                                    const SegOut& out, uint32_t spin_limit, int* err,
                                    cudaStream_t stream) {
  if (n_max == 0) return cudaSuccess;
  const int grid = persistent_grid(reinterpret_cast<const void*>(segreduce_kernel<true>),
                                   kSegThreads, kSegStageBytes, ceil_div(n_max, kSegTile));
  segreduce_kernel<true><<<grid, kSegThreads, kSegStageBytes, stream>>>(
      st, fs, nframes, k0, p0, k1, p1, nullptr, lb, out, spin_limit, err);
  return cudaGetLastError();
}

}  // namespace vg
