// Step a6: the count-weighted octree pyramid.
//
// arXiv 2102.11084 reduces the cloud "iteratively with an ordered subdivision of space"
// (abstract, Sec. II-C) and recalls the octree, whose cells split into eight children
// (Sec. I).  Level 0 is the decimation at leaf L; level k+1 merges level k into parents
// key >> 3 (edge 2L): because Morton order is preserved by the shift, the children of a
// parent are adjacent rows of level k (at most 8), so no re-sort is needed.  n' = sum n;
// the parent's fixed-point sum is the children's sums moved to the parent corner:
//   S' = sum (S_child + n_child * round((c_child - C_parent) / u0)),
// all in units u0 = L/2^20 (the level-0 unit), and the centroid is C' + (S'/n')*u0 in
// binary32 -- the same formula as level 0 with leaf 2^k L for the corner.
//
// One kernel per level: tiles of 2048 rows (ticketed), run heads counted and ranked by a
// bounded chained scan, each head row gathers its (<= 8) children.
#include "vg_device.cuh"
#include "vg_internal.h"

namespace vg {
namespace {

__global__ __launch_bounds__(kMergeThreads) void pyramid_merge_kernel(
    State* st, const FrameState* __restrict__ fs, int level, uint64_t* keys, float* centroids,
    uint32_t* counts, const long long* __restrict__ sums_in, long long* __restrict__ sums_out,
    int64_t* level_offsets, int64_t cap, uint32_t* lb, uint32_t spin_limit, int* err) {
  __shared__ int s_tile;
  __shared__ uint32_t s_tmp[kMergeThreads / 32];
  __shared__ uint32_t s_excl;
  const int t = threadIdx.x;
  // An earlier step failed: take no ticket.  Every ticket taken is processed, so no tile
  // ever waits for one that a returning block skipped.
  if (block_error_raised(err)) return;
  if (t == 0) s_tile = static_cast<int>(atomicAdd(&st->tile_ctr[kMaxPasses + level], 1u));
  __syncthreads();
  const int tile = s_tile;
  const int64_t off_prev = level_offsets[level - 1];
  const int64_t off_cur = level_offsets[level];
  const int64_t vprev = off_cur - off_prev;
  const int64_t base = int64_t(tile) * kMergeTile;
  if (base >= vprev) return;

  const float o[3] = {fs[0].origin[0], fs[0].origin[1], fs[0].origin[2]};
  const float leaf0 = fs[0].leaf;
  const float inv_unit0 = quant_inv_unit(leaf0);
  const float leaf_child = __fmul_rn(leaf0, float(1u << (level - 1)));
  const float leaf_par = __fmul_rn(leaf0, float(1u << level));
  const uint64_t* ck = keys + off_prev;
  const uint32_t* cn = counts + off_prev;
  const long long* cs = sums_in;

  // heads among this thread's rows
  const int64_t r0 = base + int64_t(t) * kMergeItems;
  uint32_t heads = 0, headmask = 0;
#pragma unroll
  for (int j = 0; j < kMergeItems; ++j) {
    const int64_t r = r0 + j;
    if (r < vprev) {
      const bool h = (r == 0) || ((ck[r] >> 3) != (ck[r - 1] >> 3));
      headmask |= uint32_t(h) << j;
      heads += h;
    }
  }
  uint32_t total;
  const uint32_t texcl = block_excl_scan(heads, &total, s_tmp);
  if (t == 0) {
    uint32_t* status = lb;
    uint32_t excl = 0;
    if (tile == 0) {
      st_relaxed(status, kFlagPrefix | total);
    } else {
      st_relaxed(status + tile, kFlagAggregate | total);
      excl = lookback_u32(status, 1, tile, spin_limit, err);
      st_relaxed(status + tile, kFlagPrefix | ((excl + total) & kValueMask));
    }
    s_excl = excl;
    if (base + kMergeTile >= vprev) level_offsets[level + 1] = off_cur + excl + total;
  }
  __syncthreads();
  uint32_t rank = s_excl + texcl;
#pragma unroll
  for (int j = 0; j < kMergeItems; ++j) {
    if (!((headmask >> j) & 1u)) continue;
    const int64_t r = r0 + j;
    const uint64_t pkey = ck[r] >> 3;
    const uint32_t pi[3] = {key_axis(pkey, 0), key_axis(pkey, 1), key_axis(pkey, 2)};
    float C[3];
    for (int a = 0; a < 3; ++a) C[a] = voxel_corner(pi[a], o[a], leaf_par);
    Acc acc = acc_zero();
    for (int64_t c = r; c < vprev && c < r + 8; ++c) {
      const uint64_t k = ck[c];
      if ((k >> 3) != pkey) break;
      const uint32_t n = cn[c];
      acc.n += n;
      const uint32_t ci[3] = {key_axis(k, 0), key_axis(k, 1), key_axis(k, 2)};
      for (int a = 0; a < 3; ++a) {
        const float cc = voxel_corner(ci[a], o[a], leaf_child);
        const double shift = (double(cc) - double(C[a])) * double(inv_unit0);
        acc.s[a] += cs[3 * c + a] + static_cast<long long>(n) * __double2ll_rn(shift);
      }
    }
    const int64_t out = off_cur + rank;
    ++rank;
    if (out >= cap) {
      set_error(err, kErrCapacity);
      continue;
    }
    float cent[3];
    acc_centroid(pkey, acc, o, leaf_par, leaf0, cent);
    keys[out] = pkey;
    counts[out] = acc.n;
    centroids[3 * out] = cent[0];
    centroids[3 * out + 1] = cent[1];
    centroids[3 * out + 2] = cent[2];
    const int64_t lr = out - off_cur;
    sums_out[3 * lr] = acc.s[0];
    sums_out[3 * lr + 1] = acc.s[1];
    sums_out[3 * lr + 2] = acc.s[2];
  }
}

}  // namespace

cudaError_t launch_pyramid_merge(State* st, const FrameState* fs, int level, uint64_t* keys,
                                 float* centroids, uint32_t* counts, const long long* sums_in,
                                 long long* sums_out, int64_t* level_offsets, int64_t cap,
                                 uint32_t* lb, int64_t n_max, uint32_t spin_limit, int* err,
                                 cudaStream_t stream) {
  if (n_max == 0) return cudaSuccess;
  const int tiles = static_cast<int>(ceil_div(n_max, kMergeTile));
  pyramid_merge_kernel<<<tiles, kMergeThreads, 0, stream>>>(st, fs, level, keys, centroids, counts,
                                                            sums_in, sums_out, level_offsets, cap,
                                                            lb, spin_limit, err);
  return cudaGetLastError();
}

}  // namespace vg
