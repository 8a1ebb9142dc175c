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
#include "vg_device.cuh"
#include "vg_internal.h"

namespace vg {
namespace {

constexpr unsigned kFull = 0xffffffffu;

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

__device__ __forceinline__ void emit_voxel(uint32_t v, uint64_t key, const Acc& a,
                                           const float o[3], float leaf, float inv_unit,
                                           uint64_t* out_keys, float* out_centroids,
                                           uint32_t* out_counts, int64_t cap, int* err) {
  if (int64_t(v) >= cap) {
    set_error(err, 4 /* VG_ERR_CAPACITY */);
    return;
  }
  float c[3];
  acc_centroid(key, a, o, leaf, inv_unit, c);
  out_keys[v] = key;
  out_counts[v] = a.n;
  out_centroids[3 * size_t(v)] = c[0];
  out_centroids[3 * size_t(v) + 1] = c[1];
  out_centroids[3 * size_t(v) + 2] = c[2];
}

__global__ __launch_bounds__(kSegThreads) void segreduce_kernel(
    State* st, const uint64_t* __restrict__ keys0, const uint32_t* __restrict__ idx0,
    const uint64_t* __restrict__ keys1, const uint32_t* __restrict__ idx1,
    const float* __restrict__ xyz, float leaf, SegStatus* lb, uint64_t* __restrict__ out_keys,
    float* __restrict__ out_centroids, uint32_t* __restrict__ out_counts, int64_t cap,
    int64_t* out_num_voxels, int32_t* __restrict__ out_p2v, uint32_t spin_limit, int* err) {
  __shared__ uint64_t skeys[kSegTile];
  __shared__ uint32_t sidx[kSegTile];
  __shared__ Seg wtot[kSegThreads / 32];
  __shared__ Seg s_tile_excl;
  __shared__ uint64_t s_prev_key;
  __shared__ int s_tile;

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t == 0) s_tile = static_cast<int>(atomicAdd(&st->tile_ctr[kMaxPasses], 1u));
  __syncthreads();
  const int tile = s_tile;
  const int64_t nvalid = st->nvalid;
  const int64_t base = int64_t(tile) * kSegTile;
  if (base >= nvalid) return;
  const int passes = max(1, sort_passes(st->maxkey));
  const uint64_t* K = (passes & 1) ? keys1 : keys0;
  const uint32_t* I = (passes & 1) ? idx1 : idx0;
  const int cnt = static_cast<int>(nvalid - base < kSegTile ? nvalid - base : kSegTile);
  const float o[3] = {st->origin[0], st->origin[1], st->origin[2]};
  const float inv_unit = quant_inv_unit(leaf);

  for (int i = t; i < cnt; i += kSegThreads) {
    skeys[i] = __ldcs(K + base + i);
    sidx[i] = __ldcs(I + base + i);
  }
  if (t == 0) s_prev_key = base > 0 ? K[base - 1] : 0ull;
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
      pi[j] = sidx[li];
      const uint64_t pk = j == 0 ? prev0 : k[j - 1];
      const bool head = (base + li == 0) || (k[j] != pk);
      headmask |= uint32_t(head) << j;
      const float* p = xyz + 3 * size_t(pi[j]);
      const Acc a = point_acc(k[j], __ldg(p), __ldg(p + 1), __ldg(p + 2), o, leaf, inv_unit);
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

  if (t == 0) {
    Seg agg = seg_identity();
    for (int w = 0; w < kSegThreads / 32; ++w) agg = seg_combine(agg, wtot[w]);
    SegStatus* me = lb + tile;
    Seg excl = seg_identity();
    if (tile == 0) {
      me->heads_incl = agg.h;
      me->n_incl = agg.a.n;
      for (int a = 0; a < 3; ++a) me->s_incl[a] = agg.a.s[a];
      st_release(&me->flag, 2u);
    } else {
      me->heads_agg = agg.h;
      me->n_agg = agg.a.n;
      for (int a = 0; a < 3; ++a) me->s_agg[a] = agg.a.s[a];
      st_release(&me->flag, 1u);
      Seg suffix = seg_identity();
      int j = tile - 1;
      uint32_t spins = 0;
      while (j >= 0) {
        const SegStatus* other = lb + j;
        const uint32_t f = ld_acquire(&other->flag);
        if (f == 0) {
          if (++spins > spin_limit) {
            set_error(err, 6 /* VG_ERR_TIMEOUT */);
            break;
          }
          if (spins > 64) __nanosleep(64);
          continue;
        }
        Seg v;
        if (f == 1u) {
          v.h = __ldcg(&other->heads_agg);
          v.a.n = __ldcg(&other->n_agg);
          for (int a = 0; a < 3; ++a) v.a.s[a] = __ldcg(&other->s_agg[a]);
        } else {
          v.h = __ldcg(&other->heads_incl);
          v.a.n = __ldcg(&other->n_incl);
          for (int a = 0; a < 3; ++a) v.a.s[a] = __ldcg(&other->s_incl[a]);
        }
        suffix = seg_combine(v, suffix);
        if (f != 1u) break;
        --j;
      }
      excl = suffix;
      const Seg inc = seg_combine(excl, agg);
      me->heads_incl = inc.h;
      me->n_incl = inc.a.n;
      for (int a = 0; a < 3; ++a) me->s_incl[a] = inc.a.s[a];
      st_release(&me->flag, 2u);
    }
    s_tile_excl = excl;
  }
  __syncthreads();

  Seg wexcl = seg_identity();
  for (int w = 0; w < warp; ++w) wexcl = seg_combine(wexcl, wtot[w]);
  const Seg pre = seg_combine(seg_combine(s_tile_excl, wexcl), lane_excl);

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
        emit_voxel(H - 1, pk, run, o, leaf, inv_unit, out_keys, out_centroids, out_counts, cap, err);
      }
      H += 1;
      run = acc_zero();
    }
    run.n += 1;
    run.s[0] += q[j][0];
    run.s[1] += q[j][1];
    run.s[2] += q[j][2];
    if (out_p2v) out_p2v[pi[j]] = static_cast<int32_t>(H - 1);
    if (gi == nvalid - 1) {
      emit_voxel(H - 1, k[j], run, o, leaf, inv_unit, out_keys, out_centroids, out_counts, cap, err);
      *out_num_voxels = H;
    }
  }
}

}  // namespace

cudaError_t launch_segreduce(State* st, const uint64_t* keys0, const uint32_t* idx0,
                             const uint64_t* keys1, const uint32_t* idx1, const float* xyz,
                             float leaf, SegStatus* lb, int64_t n_max, uint64_t* out_keys,
                             float* out_centroids, uint32_t* out_counts, int64_t cap,
                             int64_t* out_num_voxels, int32_t* out_p2v, uint32_t spin_limit,
                             int* err, cudaStream_t stream) {
  if (n_max == 0) return cudaSuccess;
  const int tiles = static_cast<int>(ceil_div(n_max, kSegTile));
  segreduce_kernel<<<tiles, kSegThreads, 0, stream>>>(st, keys0, idx0, keys1, idx1, xyz, leaf, lb,
                                                      out_keys, out_centroids, out_counts, cap,
                                                      out_num_voxels, out_p2v, spin_limit, err);
  return cudaGetLastError();
}

}  // namespace vg
