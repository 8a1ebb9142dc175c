// Steps a4 + a5: one output voxel per run of equal keys in the sorted table, with its
// point count and centroid, written densely in ascending key order.
//
// arXiv 2102.11084 Sec. II-C: once "tabla_subdiv" is sorted, the points of each cell are
// contiguous and the number of points per cell is known; the filtered cloud keeps one
// point per occupied cell (the centroid, as the voxel-grid filter the paper replaces).
//
// Three kernels over tiles of 1024 sorted entries, with no waits between tiles:
//   seg_count  run heads per tile (keys only), and the fixed-point sum of the tile's
//              leading entries that continue a run begun in an earlier tile (usually
//              none or a few; the whole tile when it holds no head);
//   seg_scan   one block: exclusive scan of the head counts = each tile's first row, V;
//   seg_reduce every run is reduced by the thread holding its head: it reads the run's
//              entries from shared memory and, if the run crosses the tile end, adds the
//              leading sums of the following tiles; rows are staged in shared memory and
//              written out coalesced.
// Integer sums make the result independent of tiling and of the order of the points.
// Two layouts: narrow (32-bit keys, packed offsets as payload) and wide (64-bit keys,
// point index as payload, coordinates gathered; also gives point_to_voxel).  The
// kernels of the layout the key kernel did not choose return at once.
#include <type_traits>

#include "vg_device.cuh"
#include "vg_internal.h"

namespace vg {
namespace {

template <bool kNarrow>
struct Layout {
  using KeyT = typename std::conditional<kNarrow, uint32_t, uint64_t>::type;
  using PayT = typename std::conditional<kNarrow, uint64_t, uint32_t>::type;
};

// Quantised offsets of a sorted entry (narrow: unpacked; wide: gathered and quantised).
template <bool kNarrow>
__device__ __forceinline__ void entry_offsets(uint64_t key, uint64_t pay,
                                              const float* __restrict__ xyz,
                                              const FrameState* __restrict__ fs,
                                              uint32_t key_shift, const float o1[3],
                                              float leaf1, int q[3]) {
  if (kNarrow) {
    q[0] = unpack_offset(pay, 0);
    q[1] = unpack_offset(pay, 1);
    q[2] = unpack_offset(pay, 2);
  } else {
    float o[3] = {o1[0], o1[1], o1[2]};
    float leaf = leaf1;
    if (key_shift < 64) {
      const uint32_t f = key_frame(key, key_shift);
      o[0] = fs[f].origin[0];
      o[1] = fs[f].origin[1];
      o[2] = fs[f].origin[2];
      leaf = fs[f].leaf;
    }
    const float* p = xyz + 3 * size_t(uint32_t(pay));
    const Acc a = point_acc(key_local(key, key_shift), __ldg(p), __ldg(p + 1), __ldg(p + 2), o,
                            leaf, quant_inv_unit(leaf));
    q[0] = int(a.s[0]);
    q[1] = int(a.s[1]);
    q[2] = int(a.s[2]);
  }
}

// Block-wide sum of an accumulator (kRedThreads threads); result valid in thread 0.
__device__ __forceinline__ Acc block_sum_acc(Acc a, Acc* tmp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    a.n += __shfl_xor_sync(kFullMask, a.n, off);
#pragma unroll
    for (int x = 0; x < 3; ++x) a.s[x] += __shfl_xor_sync(kFullMask, a.s[x], off);
  }
  if (lane == 0) tmp[warp] = a;
  __syncthreads();
  Acc r = acc_zero();
  if (threadIdx.x == 0)
    for (int w = 0; w < kRedThreads / 32; ++w) acc_add(r, tmp[w]);
  return r;
}

template <bool kNarrow>
__device__ __forceinline__ void seg_count_body(
    const State* st, const FrameState* __restrict__ fs, const void* k0_, const void* p0_,
    const void* k1_, const void* p1_, const float* __restrict__ xyz, TileRec* recs) {
  using KeyT = typename Layout<kNarrow>::KeyT;
  using PayT = typename Layout<kNarrow>::PayT;
  __shared__ uint32_t s_heads[kRedThreads / 32];
  __shared__ int s_first[kRedThreads / 32];
  __shared__ Acc s_acc[kRedThreads / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t nitems = st->nitems;
  const int64_t ntiles = ceil_div(nitems, kRedTile);
  const int passes = max(1, sort_passes(st->maxkey));
  const KeyT* K = static_cast<const KeyT*>((passes & 1) ? k1_ : k0_);
  const PayT* P = static_cast<const PayT*>((passes & 1) ? p1_ : p0_);
  const uint32_t key_shift = st->key_shift;
  const float o1[3] = {fs[0].origin[0], fs[0].origin[1], fs[0].origin[2]};
  const float leaf1 = fs[0].leaf;

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t base = tile * kRedTile;
    const int cnt = static_cast<int>(nitems - base < kRedTile ? nitems - base : kRedTile);
    uint32_t heads = 0;
    int first = kRedTile;
    uint64_t rk[kRedItems], rq[kRedItems];
#pragma unroll
    for (int j = 0; j < kRedItems; ++j) {
      const int li = j * kRedThreads + t;
      const int64_t gi = base + li;
      rk[j] = li < cnt ? uint64_t(K[gi]) : 0ull;
      rq[j] = (li < cnt && gi > 0) ? uint64_t(K[gi - 1]) : ~rk[j];
    }
#pragma unroll
    for (int j = 0; j < kRedItems; ++j) {
      const int li = j * kRedThreads + t;
      const bool head = li < cnt && rk[j] != rq[j];
      heads += head;
      if (head && li < first) first = li;
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      heads += __shfl_xor_sync(kFullMask, heads, off);
      first = min(first, __shfl_xor_sync(kFullMask, first, off));
    }
    if (lane == 0) {
      s_heads[warp] = heads;
      s_first[warp] = first;
    }
    __syncthreads();
    uint32_t th = 0;
    int fh = kRedTile;
    for (int w = 0; w < kRedThreads / 32; ++w) {
      th += s_heads[w];
      fh = min(fh, s_first[w]);
    }
    if (fh > cnt) fh = cnt;
    // leading entries [0, fh): the continuation of a run begun before this tile
    Acc lead = acc_zero();
    for (int li = t; li < fh; li += kRedThreads) {
      const int64_t gi = base + li;
      int q[3];
      entry_offsets<kNarrow>(uint64_t(K[gi]), uint64_t(P[gi]), xyz, fs, key_shift, o1, leaf1, q);
      lead.n += 1;
      lead.s[0] += q[0];
      lead.s[1] += q[1];
      lead.s[2] += q[2];
    }
    lead = block_sum_acc(lead, s_acc);
    if (t == 0) {
      TileRec r;
      r.heads = th;
      r.vbase = 0;
      r.lead_n = lead.n;
      r.pad = 0;
      r.lead_s[0] = lead.s[0];
      r.lead_s[1] = lead.s[1];
      r.lead_s[2] = lead.s[2];
      recs[tile] = r;
    }
    __syncthreads();
  }
}

// One block of 1024 threads: exclusive scan of the tiles' head counts into vbase, and V.
// Thread t owns a contiguous run of ceil(ntiles/1024) tiles, so its loads are all in
// flight at once; one block-wide scan of the 1024 run totals joins them.
__global__ __launch_bounds__(1024) void seg_scan_kernel(const State* st, TileRec* recs,
                                                        int64_t* num_voxels) {
  __shared__ uint32_t s_tmp[32];
  const int64_t ntiles = ceil_div(int64_t(st->nitems), kRedTile);
  const int64_t per = ceil_div(ntiles, 1024);
  const int64_t t0 = int64_t(threadIdx.x) * per;
  const int64_t t1 = t0 + per < ntiles ? t0 + per : ntiles;
  uint32_t sum = 0;
  for (int64_t i = t0; i < t1; ++i) sum += recs[i].heads;
  uint32_t total;
  uint32_t run = block_excl_scan(sum, &total, s_tmp);
  for (int64_t i = t0; i < t1; ++i) {
    const uint32_t h = recs[i].heads;
    recs[i].vbase = run;
    run += h;
  }
  if (threadIdx.x == 0) *num_voxels = total;
}

// Output offsets of frames (f_prev, f_new] start at voxel v.
__device__ __forceinline__ void mark_frames(int64_t* fo, uint32_t f_prev, uint32_t f_new,
                                            uint32_t v) {
  if (!fo) return;
  for (uint32_t f = f_prev + 1; f <= f_new; ++f) fo[f] = v;
}

template <bool kNarrow>
__device__ __forceinline__ void seg_reduce_body(
    const State* st, const FrameState* __restrict__ fs, int nframes, const void* k0_,
    const void* p0_, const void* k1_, const void* p1_, const float* __restrict__ xyz,
    const TileRec* __restrict__ recs, const SegOut& out, int* err) {
  using KeyT = typename Layout<kNarrow>::KeyT;
  using PayT = typename Layout<kNarrow>::PayT;
  extern __shared__ __align__(16) unsigned char red_smem[];
  __shared__ uint32_t s_tmp[kRedThreads / 32];
  __shared__ uint64_t s_prev;
  uint64_t* skey = reinterpret_cast<uint64_t*>(red_smem);           // [kRedTile]
  uint64_t* gkey = skey + kRedTile;                                 // [kRedTile]
  int* sq = reinterpret_cast<int*>(gkey + kRedTile);                // [3][kRedTile]
  uint32_t* sidx = reinterpret_cast<uint32_t*>(sq + 3 * kRedTile);  // [kRedTile]
  uint32_t* gcnt = sidx + kRedTile;                                 // [kRedTile]
  float* gcen = reinterpret_cast<float*>(gcnt + kRedTile);          // [3 * kRedTile]

  const int t = threadIdx.x;
  const int64_t nitems = st->nitems;
  const int64_t ntiles = ceil_div(nitems, kRedTile);
  const int passes = max(1, sort_passes(st->maxkey));
  const KeyT* K = static_cast<const KeyT*>((passes & 1) ? k1_ : k0_);
  const PayT* P = static_cast<const PayT*>((passes & 1) ? p1_ : p0_);
  const uint32_t key_shift = st->key_shift;
  const float o1[3] = {fs[0].origin[0], fs[0].origin[1], fs[0].origin[2]};
  const float leaf1 = fs[0].leaf;

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t base = tile * kRedTile;
    const int cnt = static_cast<int>(nitems - base < kRedTile ? nitems - base : kRedTile);
    const uint32_t vbase = recs[tile].vbase;
    const uint32_t theads = recs[tile].heads;
    // all of this thread's loads first (kRedItems in flight), then unpack into shared memory
    uint64_t rk[kRedItems], rp[kRedItems];
#pragma unroll
    for (int j = 0; j < kRedItems; ++j) {
      const int li = j * kRedThreads + t;
      rk[j] = li < cnt ? uint64_t(__ldcs(K + base + li)) : 0ull;
      rp[j] = li < cnt ? uint64_t(__ldcs(P + base + li)) : 0ull;
    }
#pragma unroll
    for (int j = 0; j < kRedItems; ++j) {
      const int li = j * kRedThreads + t;
      if (li < cnt) {
        skey[li] = rk[j];
        int q[3];
        entry_offsets<kNarrow>(rk[j], rp[j], xyz, fs, key_shift, o1, leaf1, q);
        sq[li] = q[0];
        sq[kRedTile + li] = q[1];
        sq[2 * kRedTile + li] = q[2];
        if (!kNarrow) sidx[li] = uint32_t(rp[j]);
      }
    }
    if (t == 0) s_prev = base > 0 ? uint64_t(K[base - 1]) : ~uint64_t(0);
    __syncthreads();

    // this thread's entries: [t*kRedItems, t*kRedItems + kRedItems)
    const int first = t * kRedItems;
    uint32_t headmask = 0, mine = 0;
#pragma unroll
    for (int j = 0; j < kRedItems; ++j) {
      const int li = first + j;
      if (li < cnt) {
        const uint64_t pk = li == 0 ? s_prev : skey[li - 1];
        const bool head = (base + li == 0) || skey[li] != pk;
        headmask |= uint32_t(head) << j;
        mine += head;
      }
    }
    uint32_t unused;
    const uint32_t rank = block_excl_scan(mine, &unused, s_tmp);  // heads before my entries

    // reduce the runs whose head is here; record point_to_voxel (wide layout)
    uint32_t cur = vbase + rank - 1;  // voxel of entries before my first head
#pragma unroll
    for (int j = 0; j < kRedItems; ++j) {
      const int li = first + j;
      if (li >= cnt) break;
      if ((headmask >> j) & 1u) {
        ++cur;
        const uint64_t key0 = skey[li];
        Acc run = acc_zero();
        int e = li;
        while (e < cnt && skey[e] == key0) {
          run.n += 1;
          run.s[0] += sq[e];
          run.s[1] += sq[kRedTile + e];
          run.s[2] += sq[2 * kRedTile + e];
          ++e;
        }
        bool last_run = false;
        if (e == cnt) {  // the run may continue in the following tiles
          int64_t tt = tile + 1;
          for (; tt < ntiles; ++tt) {
            const TileRec& r = recs[tt];
            run.n += r.lead_n;
            run.s[0] += r.lead_s[0];
            run.s[1] += r.lead_s[1];
            run.s[2] += r.lead_s[2];
            if (r.heads > 0) break;
          }
          last_run = tt >= ntiles;
        }
        const uint32_t row = cur - vbase;
        if (int64_t(cur) >= out.cap) {
          set_error(err, kErrCapacity);
        } else {
          const uint64_t local = key_local(key0, key_shift);
          float o[3] = {o1[0], o1[1], o1[2]};
          float leaf = leaf1;
          if (key_shift < 64) {
            const uint32_t f = key_frame(key0, key_shift);
            o[0] = fs[f].origin[0];
            o[1] = fs[f].origin[1];
            o[2] = fs[f].origin[2];
            leaf = fs[f].leaf;
          }
          float c[3];
          acc_centroid(local, run, o, leaf, leaf, c);
          gkey[row] = local;
          gcnt[row] = run.n;
          gcen[3 * row] = c[0];
          gcen[3 * row + 1] = c[1];
          gcen[3 * row + 2] = c[2];
          if (out.sums) {
            out.sums[3 * size_t(cur)] = run.s[0];
            out.sums[3 * size_t(cur) + 1] = run.s[1];
            out.sums[3 * size_t(cur) + 2] = run.s[2];
          }
        }
        if (out.frame_offsets) {
          const uint32_t fk = key_frame(key0, key_shift);
          if (base + li > 0) {
            const uint64_t pk = li == 0 ? s_prev : skey[li - 1];
            mark_frames(out.frame_offsets, key_frame(pk, key_shift), fk, cur);
          }
          if (last_run) mark_frames(out.frame_offsets, fk, uint32_t(nframes), cur + 1);
        }
      }
      if (!kNarrow && out.p2v) out.p2v[sidx[li]] = static_cast<int32_t>(cur);
    }
    __syncthreads();

    // coalesced write-out of this tile's rows [vbase, vbase + theads)
    const int span = static_cast<int>(theads);
    for (int r = t; r < span; r += kRedThreads) {
      if (int64_t(vbase) + r < out.cap) {
        out.keys[vbase + r] = gkey[r];
        out.counts[vbase + r] = gcnt[r];
      }
    }
    for (int x = t; x < 3 * span; x += kRedThreads)
      if (int64_t(vbase) + x / 3 < out.cap) out.centroids[3 * size_t(vbase) + x] = gcen[x];
    __syncthreads();
  }
}

// Pointers of both layouts; the kernels dispatch on the layout the key kernel chose.
struct RedPtrs {
  const void* wk0;
  const void* wp0;
  const void* wk1;
  const void* wp1;
  const void* nk0;
  const void* np0;
  const void* nk1;
  const void* np1;
};

__global__ __launch_bounds__(kRedThreads) void seg_count_kernel(
    const State* st, const FrameState* __restrict__ fs, RedPtrs rp, const float* __restrict__ xyz,
    TileRec* recs) {
  if (st->narrow)
    seg_count_body<true>(st, fs, rp.nk0, rp.np0, rp.nk1, rp.np1, xyz, recs);
  else
    seg_count_body<false>(st, fs, rp.wk0, rp.wp0, rp.wk1, rp.wp1, xyz, recs);
}

__global__ __launch_bounds__(kRedThreads, 4) void seg_reduce_kernel(
    const State* st, const FrameState* __restrict__ fs, int nframes, RedPtrs rp,
    const float* __restrict__ xyz, const TileRec* __restrict__ recs, SegOut out, int* err) {
  if (st->narrow)
    seg_reduce_body<true>(st, fs, nframes, rp.nk0, rp.np0, rp.nk1, rp.np1, xyz, recs, out, err);
  else
    seg_reduce_body<false>(st, fs, nframes, rp.wk0, rp.wp0, rp.wk1, rp.wp1, xyz, recs, out, err);
}

// Bytes of dynamic shared memory of seg_reduce_kernel.
constexpr size_t kRedSmem = size_t(kRedTile) * (2 * sizeof(uint64_t) + 3 * sizeof(int) +
                                                2 * sizeof(uint32_t) + 3 * sizeof(float));

}  // namespace

void warm_reduce_config() {
  persistent_grid(reinterpret_cast<const void*>(seg_count_kernel), kRedThreads, 0, 1);
  persistent_grid(reinterpret_cast<const void*>(seg_reduce_kernel), kRedThreads, kRedSmem, 1);
}

cudaError_t launch_segreduce(State* st, const FrameState* fs, int nframes,
                             const uint64_t* keys0, const uint32_t* idx0, const uint64_t* keys1,
                             const uint32_t* idx1, const float* xyz, TileRec* recs,
                             int64_t n_max, const SegOut& out, int* err, cudaStream_t stream,
                             const NarrowBuffers* nb) {
  if (n_max == 0) return cudaSuccess;
  RedPtrs rp{keys0, idx0, keys1, idx1, nb ? nb->k0 : nullptr, nb ? nb->p0 : nullptr,
             nb ? nb->k1 : nullptr, nb ? nb->p1 : nullptr};
  const int64_t tiles = ceil_div(n_max, kRedTile);
  const int gc = persistent_grid(reinterpret_cast<const void*>(seg_count_kernel), kRedThreads, 0,
                                 tiles);
  seg_count_kernel<<<gc, kRedThreads, 0, stream>>>(st, fs, rp, xyz, recs);
  seg_scan_kernel<<<1, 1024, 0, stream>>>(st, recs, out.num_voxels);
  const int gr = persistent_grid(reinterpret_cast<const void*>(seg_reduce_kernel), kRedThreads,
                                 kRedSmem, tiles);
  seg_reduce_kernel<<<gr, kRedThreads, kRedSmem, stream>>>(st, fs, nframes, rp, xyz, recs, out,
                                                          err);
  return cudaGetLastError();
}

}  // namespace vg
