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
//   seg_scan   one block: exclusive scan of the head counts (from a compact array) =
//              each tile's first row, and V;
//   seg_reduce the tile's entries are staged in shared memory and its run heads
//              compacted in order, so consecutive threads take consecutive voxels: each
//              sums its run and, if the run crosses the tile end, adds the leading sums
//              of the following tiles, and writes its row (consecutive threads write
//              consecutive rows).
// Integer sums make the result independent of tiling and of the order of the points.
// Two layouts: narrow (32-bit keys, packed offsets as payload) and wide (64-bit keys,
// point index as payload, coordinates gathered; also gives point_to_voxel).  The
// kernels of the layout the key kernel did not choose return at once.
#include <type_traits>

#include "vg_device.cuh"
#include "vg_internal.h"
#include "vg_stream.cuh"

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
                                              const float* __restrict__ poses,
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
    const uint32_t f = key_shift < 64 ? key_frame(key, key_shift) : 0u;
    if (key_shift < 64) {
      o[0] = fs[f].origin[0];
      o[1] = fs[f].origin[1];
      o[2] = fs[f].origin[2];
      leaf = fs[f].leaf;
    }
    const float* p = xyz + 3 * size_t(uint32_t(pay));
    float x = __ldg(p), y = __ldg(p + 1), z = __ldg(p + 2);
    if (poses) {  // the gathered point in the common frame, as the key kernel saw it
      Pose P;
      P.rigid = true;
#pragma unroll
      for (int i = 0; i < 12; ++i) P.r[i] = __ldg(poses + 12 * f + i);
      P.zlo = -INFINITY;
      P.zhi = INFINITY;
      pose_point(P, x, y, z);
    }
    const Acc a = point_acc(key_local(key, key_shift), x, y, z, o, leaf, quant_inv_unit(leaf));
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

// Block-wide sums of four 64-bit counters (kRedThreads threads); result valid in thread 0.
__device__ __forceinline__ void block_sum_u64x4(unsigned long long a[4],
                                                unsigned long long (*tmp)[4]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int off = 16; off; off >>= 1) a[c] += __shfl_xor_sync(kFullMask, a[c], off);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < 4; ++c) tmp[warp][c] = a[c];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      a[c] = 0;
      for (int w = 0; w < kRedThreads / 32; ++w) a[c] += tmp[w][c];
    }
}

template <bool kNarrow>
__device__ __forceinline__ void seg_count_body(
    const State* st, const FrameState* __restrict__ fs, const void* k0_, const void* p0_,
    const void* k1_, const void* p1_, const float* __restrict__ xyz,
    const float* __restrict__ poses, const uint8_t* __restrict__ attrs, int channels,
    TileRec* recs, uint32_t* tile_heads) {
  __shared__ unsigned long long s_attr[kRedThreads / 32][4];
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
    // (fh is the same in every thread: the block skips the sums when the tile opens with
    // a head, as most tiles do)
    for (int li = t; li < fh; li += kRedThreads) {
      const int64_t gi = base + li;
      int q[3];
      entry_offsets<kNarrow>(uint64_t(K[gi]), uint64_t(P[gi]), xyz, poses, fs, key_shift, o1, leaf1,
                            q);
      lead.n += 1;
      lead.s[0] += q[0];
      lead.s[1] += q[1];
      lead.s[2] += q[2];
    }
    if (fh > 0) lead = block_sum_acc(lead, s_acc);
    unsigned long long la[4] = {0, 0, 0, 0};
    if (!kNarrow && attrs && fh > 0) {  // attribute sums of the same leading entries
      for (int li = t; li < fh; li += kRedThreads) {
        const uint8_t* a = attrs + size_t(uint32_t(P[base + li])) * channels;
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (c < channels) la[c] += a[c];
      }
      block_sum_u64x4(la, s_attr);
    }
    if (t == 0) {
      TileRec r;
      r.heads = th;
      r.vbase = 0;
      r.lead_n = lead.n;
      r.pad = 0;
      r.lead_s[0] = lead.s[0];
      r.lead_s[1] = lead.s[1];
      r.lead_s[2] = lead.s[2];
      for (int c = 0; c < 4; ++c) r.lead_a[c] = la[c];
      recs[tile] = r;
      tile_heads[tile] = th;
    }
    __syncthreads();
  }
}

// One block of 1024 threads: exclusive scan of the tiles' head counts into vbase, and V.
// The counts come from a compact array, 4096 per round: coalesced loads, one block-wide
// scan per round, a running carry between rounds.
__global__ __launch_bounds__(1024) void seg_scan_kernel(const State* st,
                                                        const uint32_t* __restrict__ tile_heads,
                                                        TileRec* recs, int64_t* num_voxels,
                                                        const int* err) {
  __shared__ uint32_t s_tmp[32];
  if (st->narrow && st->msd) return;
  if (block_error_raised(err)) return;  // an earlier step failed
  const int64_t ntiles = ceil_div(int64_t(st->nitems), kRedTile);
  uint32_t carry = 0;
  for (int64_t base = 0; base < ntiles; base += 4 * 1024) {
    const int64_t i0 = base + 4 * int64_t(threadIdx.x);
    uint32_t h[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) h[j] = i0 + j < ntiles ? tile_heads[i0 + j] : 0u;
    uint32_t total;
    uint32_t run = carry + block_excl_scan(h[0] + h[1] + h[2] + h[3], &total, s_tmp);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (i0 + j < ntiles) {
        recs[i0 + j].vbase = run;
        run += h[j];
      }
    carry += total;
  }
  if (threadIdx.x == 0) *num_voxels = carry;
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
    const float* __restrict__ poses, const TileRec* __restrict__ recs, const SegOut& out,
    int* err) {
  using KeyT = typename Layout<kNarrow>::KeyT;
  using PayT = typename Layout<kNarrow>::PayT;
  extern __shared__ __align__(128) unsigned char red_smem[];
  __shared__ uint32_t s_tmp[kRedThreads / 32];
  __shared__ uint64_t s_prev;
  uint64_t* skey = reinterpret_cast<uint64_t*>(red_smem);           // [kRedTile]
  int* sq = reinterpret_cast<int*>(skey + kRedTile);                // [3][kRedTile]
  uint32_t* sidx = reinterpret_cast<uint32_t*>(sq + 3 * kRedTile);  // [kRedTile]
  uint32_t* hpos = sidx + kRedTile;                                 // [kRedTile + 1]

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
    const int theads = static_cast<int>(recs[tile].heads);
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
        entry_offsets<kNarrow>(rk[j], rp[j], xyz, poses, fs, key_shift, o1, leaf1, q);
        sq[li] = q[0];
        sq[kRedTile + li] = q[1];
        sq[2 * kRedTile + li] = q[2];
        if (!kNarrow) sidx[li] = uint32_t(rp[j]);
      }
    }
    if (t == 0) s_prev = base > 0 ? uint64_t(K[base - 1]) : ~uint64_t(0);
    __syncthreads();

    // run heads among this thread's entries [t*kRedItems, t*kRedItems + kRedItems), then
    // their positions, compacted in order: hpos[r] = first entry of the tile's r-th voxel
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
    uint32_t r = block_excl_scan(mine, &unused, s_tmp);
#pragma unroll
    for (int j = 0; j < kRedItems; ++j)
      if ((headmask >> j) & 1u) hpos[r++] = first + j;
    if (t == 0) hpos[theads] = cnt;
    __syncthreads();

    // entries before the first head continue the previous tile's last voxel
    if (!kNarrow && out.p2v) {
      const int lead_end = static_cast<int>(hpos[0]);
      for (int li = t; li < lead_end; li += kRedThreads)
        out.p2v[sidx[li]] = static_cast<int32_t>(vbase) - 1;
    }

    // one voxel per thread: its run is [hpos[v], hpos[v + 1])
    for (int v = t; v < theads; v += kRedThreads) {
      const int e0 = static_cast<int>(hpos[v]), e1 = static_cast<int>(hpos[v + 1]);
      const uint64_t key0 = skey[e0];
      const uint32_t cur = vbase + v;
      Acc run = acc_zero();
      run.n = uint32_t(e1 - e0);
      for (int e = e0; e < e1; ++e) {
        run.s[0] += sq[e];
        run.s[1] += sq[kRedTile + e];
        run.s[2] += sq[2 * kRedTile + e];
      }
      if (!kNarrow && out.p2v)
        for (int e = e0; e < e1; ++e) out.p2v[sidx[e]] = static_cast<int32_t>(cur);
      unsigned long long asum[4] = {0, 0, 0, 0};
      const bool with_attrs = !kNarrow && out.attrs_in != nullptr;
      if (with_attrs)
        for (int e = e0; e < e1; ++e) {
          const uint8_t* a = out.attrs_in + size_t(sidx[e]) * out.channels;
#pragma unroll
          for (int c = 0; c < 4; ++c)
            if (c < out.channels) asum[c] += a[c];
        }
      bool last_run = false;
      if (e1 == cnt) {  // the run may continue in the following tiles
        int64_t tt = tile + 1;
        for (; tt < ntiles; ++tt) {
          const TileRec& rr = recs[tt];
          run.n += rr.lead_n;
          run.s[0] += rr.lead_s[0];
          run.s[1] += rr.lead_s[1];
          run.s[2] += rr.lead_s[2];
          if (with_attrs)
#pragma unroll
            for (int c = 0; c < 4; ++c) asum[c] += rr.lead_a[c];
          if (rr.heads > 0) break;
        }
        last_run = tt >= ntiles;
      }
      if (with_attrs && int64_t(cur) < out.cap)  // exact sums, one FP64 division each
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (c < out.channels)
            out.attrs_out[size_t(cur) * out.channels + c] = __double2float_rn(
                __ddiv_rn(static_cast<double>(asum[c]), static_cast<double>(run.n)));
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
        out.keys[cur] = local;
        out.counts[cur] = run.n;
        out.centroids[3 * size_t(cur)] = c[0];
        out.centroids[3 * size_t(cur) + 1] = c[1];
        out.centroids[3 * size_t(cur) + 2] = c[2];
        if (out.sums) {
          out.sums[3 * size_t(cur)] = run.s[0];
          out.sums[3 * size_t(cur) + 1] = run.s[1];
          out.sums[3 * size_t(cur) + 2] = run.s[2];
        }
      }
      if (out.frame_offsets) {
        const uint32_t fk = key_frame(key0, key_shift);
        if (base + e0 > 0) {
          const uint64_t pk = e0 == 0 ? s_prev : skey[e0 - 1];
          mark_frames(out.frame_offsets, key_frame(pk, key_shift), fk, cur);
        }
        if (last_run) mark_frames(out.frame_offsets, fk, uint32_t(nframes), cur + 1);
      }
    }
    __syncthreads();
  }
}

// Narrow layout: the tile's 32-bit keys and packed offsets arrive in shared memory by
// bulk asynchronous copies (the TMA unit), double-buffered, so the next tile's loads run
// while this one is reduced; offsets are unpacked where they are summed.
struct NarrowRedSmem {
  uint32_t keys[2][kRedTile];
  unsigned long long pay[2][kRedTile];
  uint32_t hpos[kRedTile + 4];
  unsigned long long bar[2];
  TileRec after;  // record of the tile that follows the current one
};

__device__ __forceinline__ void narrow_issue(NarrowRedSmem& sm, int b, const uint32_t* K,
                                             const uint64_t* P, int64_t tile) {
  const int64_t base = tile * kRedTile;
  mbar_arrive_expect_tx(&sm.bar[b], kRedTile * (sizeof(uint32_t) + sizeof(uint64_t)));
  bulk_copy_g2s(sm.keys[b], K + base, kRedTile * sizeof(uint32_t), &sm.bar[b]);
  bulk_copy_g2s(sm.pay[b], P + base, kRedTile * sizeof(uint64_t), &sm.bar[b]);
}

__device__ __forceinline__ void seg_reduce_narrow(const State* st, const FrameState* __restrict__ fs,
                                                  int nframes, const uint32_t* __restrict__ K,
                                                  const uint64_t* __restrict__ P,
                                                  const TileRec* __restrict__ recs,
                                                  const SegOut& out, int* err) {
  extern __shared__ __align__(128) unsigned char red_smem[];
  NarrowRedSmem& sm = *reinterpret_cast<NarrowRedSmem*>(red_smem);
  __shared__ uint32_t s_tmp[kRedThreads / 32];
  const int t = threadIdx.x;
  const int64_t nitems = st->nitems;
  const int64_t ntiles = ceil_div(nitems, kRedTile);
  // Full tiles take the bulk copy (16-byte aligned buffers); a ragged last tile, or
  // buffers that are not aligned, take plain loads.
  const bool aligned = ((reinterpret_cast<uintptr_t>(K) | reinterpret_cast<uintptr_t>(P)) & 15) == 0;
  const int64_t bulk_tiles = aligned ? nitems / kRedTile : 0;
  const uint32_t key_shift = st->key_shift;
  const float o1[3] = {fs[0].origin[0], fs[0].origin[1], fs[0].origin[2]};
  const float leaf1 = fs[0].leaf;

  int64_t tile = blockIdx.x;
  if (tile >= ntiles) return;
  if (t == 0) {
    mbar_init(&sm.bar[0], 1);
    mbar_init(&sm.bar[1], 1);
    fence_mbar_init();
    if (tile < bulk_tiles) narrow_issue(sm, 0, K, P, tile);
  }
  __syncthreads();
  uint32_t phase = 0;  // bit b: parity of buffer b's next completion
  uint32_t vbase = recs[tile].vbase, theads = recs[tile].heads, lead = recs[tile].lead_n;
  for (int b = 0; tile < ntiles; tile += gridDim.x, b ^= 1) {
    const int64_t next = tile + gridDim.x;
    const int64_t base = tile * kRedTile;
    const int cnt = static_cast<int>(nitems - base < kRedTile ? nitems - base : kRedTile);
    if (t == 0 && next < bulk_tiles) {
      fence_proxy_async();  // this block's reads of the buffer precede the copy into it
      narrow_issue(sm, b ^ 1, K, P, next);
    }
    // records for later: the next tile of this block, and the tile after this one
    uint32_t nvbase = 0, ntheads = 0, nlead = 0;
    if (next < ntiles) {
      nvbase = recs[next].vbase;
      ntheads = recs[next].heads;
      nlead = recs[next].lead_n;
    }
    TileRec after{};
    if (t == 0 && tile + 1 < ntiles) after = recs[tile + 1];

    bool ok = true;
    const uint32_t par = (phase >> b) & 1u;
    if (tile < bulk_tiles) {
      // one warp polls; the barrier below passes the completed copy on to the others
      if (t < 32) ok = mbar_wait(&sm.bar[b], par, kDefaultSpinLimit);
      phase ^= 1u << b;
    } else {
      for (int li = t; li < cnt; li += kRedThreads) {
        sm.keys[b][li] = K[base + li];
        sm.pay[b][li] = P[base + li];
      }
    }
    if (__syncthreads_or(!ok)) {  // a copy that never completed: report, drain, stop
      if (t == 0) {
        set_error(err, kErrTimeout);
        mbar_wait(&sm.bar[b], par, kDefaultSpinLimit);
        if (next < bulk_tiles) mbar_wait(&sm.bar[b ^ 1], (phase >> (b ^ 1)) & 1u, kDefaultSpinLimit);
      }
      return;
    }
    const uint32_t* kk = sm.keys[b];
    const unsigned long long* pp = sm.pay[b];

    // run heads among entries [4t, 4t + 4); entry 0 is a head unless the tile opens with
    // the continuation of an earlier run
    const int first = t * kRedItems;
    uint32_t headmask = 0, mine = 0;
    if (first < cnt) {
      uint32_t prev = first > 0 ? kk[first - 1] : 0u;
#pragma unroll
      for (int j = 0; j < kRedItems; ++j) {
        const int li = first + j;
        if (li < cnt) {
          const uint32_t k = kk[li];
          const bool head = li == 0 ? (tile == 0 || lead == 0) : k != prev;
          headmask |= uint32_t(head) << j;
          mine += head;
          prev = k;
        }
      }
    }
    uint32_t unused;
    uint32_t r = block_excl_scan(mine, &unused, s_tmp);
#pragma unroll
    for (int j = 0; j < kRedItems; ++j)
      if ((headmask >> j) & 1u) sm.hpos[r++] = first + j;
    if (t == 0) {
      sm.hpos[theads] = cnt;
      sm.after = after;
    }
    __syncthreads();

    for (int v = t; v < static_cast<int>(theads); v += kRedThreads) {
      const int e0 = static_cast<int>(sm.hpos[v]), e1 = static_cast<int>(sm.hpos[v + 1]);
      const uint64_t key0 = kk[e0];
      const uint32_t cur = vbase + v;
      Acc run = acc_zero();
      run.n = uint32_t(e1 - e0);
      for (int e = e0; e < e1; ++e) {
        const uint64_t w = pp[e];
        run.s[0] += unpack_offset(w, 0);
        run.s[1] += unpack_offset(w, 1);
        run.s[2] += unpack_offset(w, 2);
      }
      bool last_run = false;
      if (e1 == cnt) {  // the run may continue in the following tiles
        int64_t tt = tile + 1;
        for (; tt < ntiles; ++tt) {
          const TileRec rr = tt == tile + 1 ? sm.after : recs[tt];
          run.n += rr.lead_n;
          run.s[0] += rr.lead_s[0];
          run.s[1] += rr.lead_s[1];
          run.s[2] += rr.lead_s[2];
          if (rr.heads > 0) break;
        }
        last_run = tt >= ntiles;
      }
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
        out.keys[cur] = local;
        out.counts[cur] = run.n;
        out.centroids[3 * size_t(cur)] = c[0];
        out.centroids[3 * size_t(cur) + 1] = c[1];
        out.centroids[3 * size_t(cur) + 2] = c[2];
        if (out.sums) {
          out.sums[3 * size_t(cur)] = run.s[0];
          out.sums[3 * size_t(cur) + 1] = run.s[1];
          out.sums[3 * size_t(cur) + 2] = run.s[2];
        }
      }
      if (out.frame_offsets) {
        const uint32_t fk = key_frame(key0, key_shift);
        if (base + e0 > 0) {
          const uint64_t pk = e0 == 0 ? uint64_t(K[base - 1]) : uint64_t(kk[e0 - 1]);
          mark_frames(out.frame_offsets, key_frame(pk, key_shift), fk, cur);
        }
        if (last_run) mark_frames(out.frame_offsets, fk, uint32_t(nframes), cur + 1);
      }
    }
    __syncthreads();
    vbase = nvbase;
    theads = ntheads;
    lead = nlead;
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
    const float* __restrict__ poses, const uint8_t* __restrict__ attrs, int channels,
    TileRec* recs, uint32_t* tile_heads, const int* err) {
  if (st->narrow && st->msd) return;  // the bucket grouping reduces instead
  if (block_error_raised(err)) return;  // an earlier step failed
  if (st->narrow)
    seg_count_body<true>(st, fs, rp.nk0, rp.np0, rp.nk1, rp.np1, xyz, poses, nullptr, 0, recs,
                         tile_heads);
  else
    seg_count_body<false>(st, fs, rp.wk0, rp.wp0, rp.wk1, rp.wp1, xyz, poses, attrs, channels,
                          recs, tile_heads);
}

__global__ __launch_bounds__(kRedThreads, VG_RED_MINB) void seg_reduce_kernel(
    const State* st, const FrameState* __restrict__ fs, int nframes, RedPtrs rp,
    const float* __restrict__ xyz, const float* __restrict__ poses,
    const TileRec* __restrict__ recs, SegOut out, int* err) {
  if (st->narrow && st->msd) return;
  if (block_error_raised(err)) return;  // an earlier step failed
  if (st->narrow) {
    const bool odd = max(1, sort_passes(st->maxkey)) & 1;
    seg_reduce_narrow(st, fs, nframes, static_cast<const uint32_t*>(odd ? rp.nk1 : rp.nk0),
                      static_cast<const uint64_t*>(odd ? rp.np1 : rp.np0), recs, out, err);
  } else
    seg_reduce_body<false>(st, fs, nframes, rp.wk0, rp.wp0, rp.wk1, rp.wp1, xyz, poses, recs, out,
                           err);
}

// Bytes of dynamic shared memory of seg_reduce_kernel.
constexpr size_t kRedSmemWide = size_t(kRedTile) * (sizeof(uint64_t) + 3 * sizeof(int) +
                                                    2 * sizeof(uint32_t)) +
                                4 * sizeof(uint32_t);
constexpr size_t kRedSmem =
    kRedSmemWide > sizeof(NarrowRedSmem) ? kRedSmemWide : sizeof(NarrowRedSmem);

}  // namespace

void warm_reduce_config() {
  persistent_grid(reinterpret_cast<const void*>(seg_count_kernel), kRedThreads, 0, 1);
  persistent_grid(reinterpret_cast<const void*>(seg_reduce_kernel), kRedThreads, kRedSmem, 1);
}

cudaError_t launch_segreduce(State* st, const FrameState* fs, int nframes,
                             const uint64_t* keys0, const uint32_t* idx0, const uint64_t* keys1,
                             const uint32_t* idx1, const float* xyz, TileRec* recs,
                             int64_t n_max, const SegOut& out, int* err, cudaStream_t stream,
                             const NarrowBuffers* nb, const float* poses) {
  if (n_max == 0) return cudaSuccess;
  RedPtrs rp{keys0, idx0, keys1, idx1, nb ? nb->k0 : nullptr, nb ? nb->p0 : nullptr,
             nb ? nb->k1 : nullptr, nb ? nb->p1 : nullptr};
  const int64_t tiles = ceil_div(n_max, kRedTile);
  const int gc = persistent_grid(reinterpret_cast<const void*>(seg_count_kernel), kRedThreads, 0,
                                 tiles);
  uint32_t* tile_heads = reinterpret_cast<uint32_t*>(recs + tiles);  // after the records
  seg_count_kernel<<<gc, kRedThreads, 0, stream>>>(st, fs, rp, xyz, poses, out.attrs_in,
                                                   out.channels, recs, tile_heads, err);
  seg_scan_kernel<<<1, 1024, 0, stream>>>(st, tile_heads, recs, out.num_voxels, err);
  const int gr = persistent_grid(reinterpret_cast<const void*>(seg_reduce_kernel), kRedThreads,
                                 kRedSmem, tiles);
  seg_reduce_kernel<<<gr, kRedThreads, kRedSmem, stream>>>(st, fs, nframes, rp, xyz, poses, recs,
                                                          out, err);
  return cudaGetLastError();
}

}  // namespace vg
