// Step a3 (sort path): stable LSD radix sort of the voxel keys with the point index as
// payload, one kernel per 8-bit digit ("onesweep": per-tile digit ranks, a chained scan
// with decoupled look-back for the tile's offset inside each digit bucket, and a
// locally-sorted, coalesced scatter).
//
// arXiv 2102.11084 Sec. II-C / Algorithm 1 sorts the (cell, point) table "tabla_subdiv"
// with a radix sort so that the points of every cell become contiguous.  This kernel is
// that sort, restated for sm_103a:
//   * only the significant digits are sorted: the number of passes comes from the
//     largest valid key (found by the key kernel), read on the device, so launched
//     passes beyond it return at once and the data stays in the right buffer;
//   * pass 0 reads the raw per-point keys, drops invalid rows (sentinel keys) and
//     generates the payload index itself, so compaction costs nothing extra;
//   * every pass also histograms the next digit, so no separate upsweep pass exists;
//   * tile ids come from an atomic ticket (a waiting tile only waits on tiles that have
//     already started), and every wait is bounded: after the limit the kernel records
//     a timeout status and carries on, so a fault can never hang the GPU.
#include "vg_device.cuh"
#include "vg_internal.h"

namespace vg {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint64_t kSentinel = kKeySentinel;

// Exclusive scans of two values over a 256-thread block; also returns the totals.
__device__ __forceinline__ void block_excl_scan2(uint32_t a, uint32_t b, uint32_t* ea,
                                                 uint32_t* eb, uint32_t* ta, uint32_t* tb,
                                                 uint32_t (*tmp)[2]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t ia = a, ib = b;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t ya = __shfl_up_sync(kFull, ia, off);
    const uint32_t yb = __shfl_up_sync(kFull, ib, off);
    if (lane >= off) {
      ia += ya;
      ib += yb;
    }
  }
  if (lane == 31) {
    tmp[warp][0] = ia;
    tmp[warp][1] = ib;
  }
  __syncthreads();
  uint32_t wa = 0, wb = 0, sa = 0, sb = 0;
#pragma unroll
  for (int w = 0; w < kSortThreads / 32; ++w) {
    if (w < warp) {
      wa += tmp[w][0];
      wb += tmp[w][1];
    }
    sa += tmp[w][0];
    sb += tmp[w][1];
  }
  *ea = wa + ia - a;
  *eb = wb + ib - b;
  *ta = sa;
  *tb = sb;
}

// Shared memory of one radix-pass block.
struct SortSmem {
  uint32_t warp_hist[kSortThreads / 32][kRadix];
  uint32_t digit_start[kRadix];
  int32_t gofs[kRadix];  // output position of local slot i of digit d: gofs[d] + i
  uint32_t next_hist[kRadix];
  uint32_t scan_tmp[kSortThreads / 32][2];
  uint64_t sbuf[kSortTile];  // keys, then payloads, in local (digit) order
  uint32_t sdst[kSortTile];  // output position of each local slot
  int s_tile;
  uint32_t s_tile_n;
};

// One radix pass.  KeyT/PayT: (uint64, uint32 point index) for the wide layout, or
// (uint32, uint64 packed offsets) for the narrow one.  A pass beyond the needed ones
// returns before taking a tile ticket.  Keys are loaded, ranked and written first; the
// payloads are loaded only once the keys sit in shared memory (their loads overlap the
// key write-out), so the ranking holds no payload registers.
template <typename KeyT, typename PayT, bool kNarrow>
__device__ __forceinline__ void onesweep_body(
    const KeyT* __restrict__ keys_in, const PayT* __restrict__ pay_in,
    KeyT* __restrict__ keys_out, PayT* __restrict__ pay_out, State* st, uint32_t* lb_cur,
    uint32_t* lb_next, int pass, int64_t n_host, int compact_input, uint32_t spin_limit,
    int* err, SortSmem& sm) {
  uint32_t (&warp_hist)[kSortThreads / 32][kRadix] = sm.warp_hist;
  uint32_t* digit_start = sm.digit_start;
  int32_t* gofs = sm.gofs;
  uint32_t* next_hist = sm.next_hist;
  uint32_t (&scan_tmp)[kSortThreads / 32][2] = sm.scan_tmp;
  uint64_t* sbuf = sm.sbuf;
  uint32_t* sdst = sm.sdst;
  int& s_tile = sm.s_tile;
  uint32_t& s_tile_n = sm.s_tile_n;

  const int passes = pass_count(st);
  if (pass >= passes) return;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  // Pass 0 of the sort path reads all n raw entries and drops the invalid rows (sentinel
  // keys); every other pass, and pass 0 of compacted input, reads st->nitems entries.
  const bool raw = pass == 0 && !compact_input;
  const int64_t n_items = raw ? n_host : int64_t(st->nitems);
  const int64_t ntiles = ceil_div(n_items, kSortTile);
  const int shift = pass * kRadixBits;
  const bool has_next = shift + kRadixBits < int(8 * sizeof(KeyT));

  // The next digit's histogram is accumulated over all tiles of this block and folded
  // into the global one once, at exit.
  next_hist[t] = 0;
#if VG_SORT_EARLY_TICKET
  // The next ticket is taken once this tile's prefixes are out, its latency hidden
  // behind the scatter.  The next tile is then held, unstarted, for the scatter only
  // (holding it for a whole tile stalled every later look-back and was slower; this
  // is faster by about 2 % a pass on the 50M-point map).
  if (t == 0) s_tile = static_cast<int>(atomicAdd(&st->tile_ctr[pass], 1u));
  __syncthreads();
  int next_tile = 0;
#endif
  for (;;) {  // persistent: tiles from a ticket until none is left
#if !VG_SORT_EARLY_TICKET
  // (a ticket is taken only when the block can start the tile at once)
  if (t == 0) s_tile = static_cast<int>(atomicAdd(&st->tile_ctr[pass], 1u));
  __syncthreads();
#endif
  const int tile = s_tile;
  if (tile >= ntiles) break;
  // The next pass uses the other status region; every tile clears its own row of it.
  lb_next[size_t(tile) * kRadix + t] = 0;
  const int64_t tile_base = int64_t(tile) * kSortTile;
  // item j of lane l (warp-striped): tile_base + warp * 32 * kSortItems + j * 32 + l
  const int64_t my_base = tile_base + warp * (32 * kSortItems) + lane;

  // ---- keys ----
  KeyT key[kSortItems];
  uint32_t vmask = 0;
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    const int64_t i = my_base + j * 32;
    const bool in = i < n_items;
    key[j] = in ? __ldcs(keys_in + i) : KeyT(0);
    bool ok = in;
    // raw rows: the sentinel key (all ones, in either width) marks an invalid point; the
    // narrow layout is chosen only when no valid key can be all ones
    if (raw) ok = ok && key[j] != KeyT(kSentinel);
    vmask |= uint32_t(ok) << j;
  }
  for (int d = lane; d < kRadix; d += 32) warp_hist[warp][d] = 0;
  __syncwarp();

  // ---- stable rank of every item among the same digit within its warp ----
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t rank[kSortItems];
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    const bool ok = (vmask >> j) & 1u;
    const uint32_t d = static_cast<uint32_t>(uint64_t(key[j]) >> shift) & (kRadix - 1);
    uint32_t peers = __ballot_sync(kFull, ok);
#pragma unroll
    for (int b = 0; b < kRadixBits; ++b) {
      const bool bit = (d >> b) & 1u;
      const uint32_t bal = __ballot_sync(kFull, bit);
      peers &= bit ? bal : ~bal;
    }
    const uint32_t lower = peers & lt;
    uint32_t old = 0;
    if (ok) old = warp_hist[warp][d];
    __syncwarp();
    if (ok && lower == 0) warp_hist[warp][d] = old + __popc(peers);
    __syncwarp();
    rank[j] = old + __popc(lower);
  }
  __syncthreads();

  // ---- per digit (thread t = digit t): offsets of the warps, tile count, scans ----
  uint32_t run = 0;
#pragma unroll
  for (int w = 0; w < kSortThreads / 32; ++w) {
    const uint32_t c = warp_hist[w][t];
    warp_hist[w][t] = run;
    run += c;
  }
  const uint32_t tile_count = run;
  uint32_t local_excl, global_excl, tile_total, global_total;
  block_excl_scan2(tile_count, st->hist[pass][t], &local_excl, &global_excl, &tile_total,
                   &global_total, scan_tmp);

  // ---- chained scan over tiles, one digit per thread ----
  uint32_t excl = 0;
  uint32_t* my = lb_cur + size_t(tile) * kRadix + t;
  if (tile == 0) {
    st_relaxed(my, kFlagPrefix | tile_count);
  } else {
    st_relaxed(my, kFlagAggregate | tile_count);
    excl = lookback_u32(lb_cur + t, kRadix, tile, spin_limit, err);
    st_relaxed(my, kFlagPrefix | ((excl + tile_count) & kValueMask));
  }
  digit_start[t] = local_excl;
  gofs[t] = static_cast<int32_t>(global_excl + excl) - static_cast<int32_t>(local_excl);
  if (t == 0) s_tile_n = tile_total;
  __syncthreads();
#if VG_SORT_EARLY_TICKET
  if (t == 0) next_tile = static_cast<int>(atomicAdd(&st->tile_ctr[pass], 1u));
#endif

  // ---- keys: locally sorted in shared memory, then written digit run by digit run ----
  KeyT* skey = reinterpret_cast<KeyT*>(sbuf);
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    if ((vmask >> j) & 1u) {
      const uint32_t d = static_cast<uint32_t>(uint64_t(key[j]) >> shift) & (kRadix - 1);
      rank[j] += digit_start[d] + warp_hist[warp][d];
      skey[rank[j]] = key[j];
    }
  }
  __syncthreads();
  // payload loads, in flight while the keys are written out
  PayT pay[kSortItems];
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    const int64_t i = my_base + j * 32;
    if (!kNarrow && raw)
      pay[j] = static_cast<PayT>(i);
    else
      pay[j] = ((vmask >> j) & 1u) ? __ldcs(pay_in + i) : PayT(0);
  }
  const uint32_t tile_n = s_tile_n;
  for (uint32_t i = t; i < tile_n; i += kSortThreads) {
    const KeyT k = skey[i];
    const uint32_t d = static_cast<uint32_t>(uint64_t(k) >> shift) & (kRadix - 1);
    const uint32_t dst = static_cast<uint32_t>(gofs[d] + static_cast<int32_t>(i));
    sdst[i] = dst;
    __stcg(keys_out + dst, k);
    if (has_next)
      atomicAdd(&next_hist[static_cast<uint32_t>(uint64_t(k) >> (shift + kRadixBits)) & (kRadix - 1)],
                1u);
  }
  __syncthreads();
#if VG_SORT_EARLY_TICKET && VG_SORT_PREFETCH
  // the next tile's keys and payloads start their way into L2 while this one scatters
  if (t == 0 && next_tile < ntiles) {
    const int64_t b = int64_t(next_tile) * kSortTile;
    const int64_t m = n_items - b < kSortTile ? n_items - b : kSortTile;
    const uint32_t kb = static_cast<uint32_t>(m * sizeof(KeyT)) & ~15u;
    const uint32_t pb = static_cast<uint32_t>(m * sizeof(PayT)) & ~15u;
    if (kb && ((reinterpret_cast<uintptr_t>(keys_in + b) & 15) == 0)) prefetch_l2(keys_in + b, kb);
    if (pb && !(raw && !kNarrow) && ((reinterpret_cast<uintptr_t>(pay_in + b) & 15) == 0))
      prefetch_l2(pay_in + b, pb);
  }
#endif
  PayT* spay = reinterpret_cast<PayT*>(sbuf);
#pragma unroll
  for (int j = 0; j < kSortItems; ++j)
    if ((vmask >> j) & 1u) spay[rank[j]] = pay[j];
  __syncthreads();
  for (uint32_t i = t; i < tile_n; i += kSortThreads) __stcg(pay_out + sdst[i], spay[i]);
  __syncthreads();
#if VG_SORT_EARLY_TICKET
  if (t == 0) s_tile = next_tile;
  __syncthreads();
#endif
  }
  __syncthreads();
  if (has_next && pass + 1 < kMaxPasses && next_hist[t])
    atomicAdd(&st->hist[pass + 1][t], next_hist[t]);
}

// One radix pass of whichever layout the key kernel chose (read on the device).
__global__ __launch_bounds__(kSortThreads, kSortMinBlocks) void onesweep_kernel(
    const uint64_t* kw_in, const uint32_t* iw_in, uint64_t* kw_out, uint32_t* iw_out,
    const uint32_t* kn_in, const uint64_t* pn_in, uint32_t* kn_out, uint64_t* pn_out, State* st,
    uint32_t* lb_cur, uint32_t* lb_next, int pass, int64_t n_host, int compact_input,
    uint32_t spin_limit, int* err) {
  __shared__ SortSmem sm;
  if (block_error_raised(err)) return;  // an earlier step failed
  if (st->narrow)
    onesweep_body<uint32_t, uint64_t, true>(kn_in, pn_in, kn_out, pn_out, st, lb_cur, lb_next, pass,
                                            n_host, compact_input, spin_limit, err, sm);
  else
    onesweep_body<uint64_t, uint32_t, false>(kw_in, iw_in, kw_out, iw_out, st, lb_cur, lb_next,
                                             pass, n_host, compact_input, spin_limit, err, sm);
}

// Test kernel: one chained-scan wait of tile `tile` on status words nobody publishes; it
// must give up after `limit` polls and record kErrTimeout.
__global__ void debug_wait_kernel(const uint32_t* status, int tile, uint32_t limit, int* err) {
  if (threadIdx.x == 0 && blockIdx.x == 0) (void)lookback_u32(status, 1, tile, limit, err);
}

}  // namespace

cudaError_t launch_debug_wait(const uint32_t* status, int tile, uint32_t limit, int* err,
                              cudaStream_t stream) {
  debug_wait_kernel<<<1, 32, 0, stream>>>(status, tile, limit, err);
  return cudaGetLastError();
}

cudaError_t launch_sort_pass(State* st, uint64_t* keys0, uint32_t* idx0, uint64_t* keys1,
                             uint32_t* idx1, uint32_t* lb_a, uint32_t* lb_b, int64_t n_max,
                             int pass, bool compact_input, uint32_t spin_limit, int* err,
                             cudaStream_t stream, const NarrowBuffers* nb) {
  if (n_max == 0) return cudaSuccess;
  const int tiles = persistent_grid(reinterpret_cast<const void*>(onesweep_kernel), kSortThreads,
                                    0, ceil_div(n_max, kSortTile));
  const bool even = (pass & 1) == 0;
  // pass p reads buffer (p odd ? 1 : 0) and writes the other; pass 0 reads raw keys.
  const bool raw = pass == 0 && !compact_input;
  const uint32_t* kn_in = nb ? (even ? nb->k0 : nb->k1) : nullptr;
  const uint64_t* pn_in = nb ? (even ? nb->p0 : nb->p1) : nullptr;
  uint32_t* kn_out = nb ? (even ? nb->k1 : nb->k0) : nullptr;
  uint64_t* pn_out = nb ? (even ? nb->p1 : nb->p0) : nullptr;
  onesweep_kernel<<<tiles, kSortThreads, 0, stream>>>(
      even ? keys0 : keys1, raw ? nullptr : (even ? idx0 : idx1), even ? keys1 : keys0,
      even ? idx1 : idx0, kn_in, pn_in, kn_out, pn_out, st, even ? lb_a : lb_b,
      even ? lb_b : lb_a, pass, n_max, compact_input ? 1 : 0, spin_limit, err);
  return cudaGetLastError();
}

void warm_sort_config() {
  persistent_grid(reinterpret_cast<const void*>(onesweep_kernel), kSortThreads, 0, 1);
}

}  // namespace vg
