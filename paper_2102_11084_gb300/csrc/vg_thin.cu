// Neighbour-count thinning (vg_thin): the paper's own filter loop.
//
// arXiv 2102.11084 Sec. II-C, Algorithm 1: every point is placed in a cell of a regular
// grid, the (cell, point) table is radix-sorted, and then, pass after pass, every point
// counts its neighbours in its own and the 26 surrounding cells (Euclidean distance,
// Eq. 1), is marked when the count exceeds a threshold, and a batch of the marked points
// is deleted; when no more than a batch is marked, all of them are deleted and the loop
// ends.  The paper deletes a random batch; here the batch is the marked points of lowest
// caller-given priority (ties by point index), so the result is reproducible.
//
// GPU layout of the loop:
//   grouping   the sort path (wide layout, point_to_voxel on) gives the occupied cells
//              in key order and the points in cell order;
//   setup      per point of the sorted table: its coordinates, priority and index; per
//              cell: its first entry and the rows of its 26 neighbour cells (binary
//              search in the sorted cell keys, once);
//   per pass   thin_count_kernel counts and marks; the host reads the number marked;
//              if it exceeds the batch, a radix select over the 64-bit keys
//              (priority << 32 | index) of the marked points finds the batch, 8 bits a
//              round, on 256-bin histograms (thin_hist_kernel); thin_delete_kernel
//              removes it (or every marked point, in the last pass).
//   output     keep flag per input point and the number kept.
// The host synchronises the stream once per pass and once per select round.
#include <cmath>

#include "../../include/vg.h"
#include "vg_api_internal.h"
#include "vg_device.cuh"
#include "vg_internal.h"

namespace vg {
namespace {

constexpr int kNb = 27;
constexpr uint32_t kNoCell = 0xffffffffu;
constexpr uint8_t kAlive = 1, kMarked = 2;

struct ThinLayout {
  size_t base, vkeys, vcent, vcnt, vnum, p2v, cstart, nb, sx, sprio, sidx, state, ctr, hist,
      total;
};

ThinLayout thin_layout(int64_t n) {
  ThinLayout L{};
  const int64_t nn = n < 1 ? 1 : n;
  size_t off = frames_workspace_bytes(n, 1, VG_METHOD_SORT);
  L.base = 0;
  auto take = [&](size_t* at, size_t bytes) {
    *at = off;
    off = align_up(off + bytes, 256);
  };
  take(&L.vkeys, size_t(nn) * sizeof(uint64_t));
  take(&L.vcent, size_t(nn) * 3 * sizeof(float));
  take(&L.vcnt, size_t(nn) * sizeof(uint32_t));
  take(&L.vnum, sizeof(int64_t));
  take(&L.p2v, size_t(nn) * sizeof(int32_t));
  take(&L.cstart, size_t(nn) * sizeof(uint32_t));
  take(&L.nb, size_t(nn) * kNb * sizeof(uint32_t));
  take(&L.sx, size_t(nn) * 3 * sizeof(float));
  take(&L.sprio, size_t(nn) * sizeof(uint32_t));
  take(&L.sidx, size_t(nn) * sizeof(uint32_t));
  take(&L.state, size_t(nn));
  take(&L.ctr, 4 * sizeof(uint32_t));  // [0] marked, [1] kept
  take(&L.hist, 256 * sizeof(uint32_t));
  L.total = off;
  return L;
}

__device__ __forceinline__ const uint32_t* sorted_idx(const State* st, const uint32_t* idx0,
                                                      const uint32_t* idx1) {
  return (max(1, sort_passes(st->maxkey)) & 1) ? idx1 : idx0;
}

// Per sorted entry: gather coordinates, priority and index; mark cell starts.
__global__ void thin_setup_kernel(const State* st, const uint32_t* idx0, const uint32_t* idx1,
                                  const float* __restrict__ xyz, const uint32_t* __restrict__ prio,
                                  const int32_t* __restrict__ p2v, uint32_t* cstart, float* sx,
                                  uint32_t* sprio, uint32_t* sidx, uint8_t* state,
                                  const int* err) {
  if (error_raised(err)) return;  // the grouping failed: point_to_voxel is unwritten
  const int64_t m = st->nitems;
  const uint32_t* I = sorted_idx(st, idx0, idx1);
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m;
       i += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t p = I[i];
    const int32_t row = p2v[p];
    const int32_t prev = i > 0 ? p2v[I[i - 1]] : -1;
    if (row != prev) cstart[row] = static_cast<uint32_t>(i);
    sx[3 * i] = xyz[3 * size_t(p)];
    sx[3 * i + 1] = xyz[3 * size_t(p) + 1];
    sx[3 * i + 2] = xyz[3 * size_t(p) + 2];
    sprio[i] = prio[p];
    sidx[i] = p;
    state[i] = kAlive;
  }
}

// Per cell: rows of the 27 cells around it (itself included), kNoCell where empty.
__global__ void thin_neighbors_kernel(const int64_t* __restrict__ num_cells,
                                      const uint64_t* __restrict__ vkeys, uint32_t* nb,
                                      const int* err) {
  if (error_raised(err)) return;
  const int64_t V = *num_cells;
  for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < V;
       v += int64_t(gridDim.x) * blockDim.x) {
    const uint64_t key = vkeys[v];
    const int64_t c[3] = {int64_t(compact3(key)), int64_t(compact3(key >> 1)),
                          int64_t(compact3(key >> 2))};
    int o = 0;
    for (int dx = -1; dx <= 1; ++dx)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dz = -1; dz <= 1; ++dz, ++o) {
          const int64_t a = c[0] + dx, b = c[1] + dy, d = c[2] + dz;
          uint32_t row = kNoCell;
          const int64_t lim = int64_t(1) << 21;
          if (a >= 0 && b >= 0 && d >= 0 && a < lim && b < lim && d < lim) {
            const uint64_t want = morton3(uint32_t(a), uint32_t(b), uint32_t(d));
            int64_t lo = 0, hi = V;  // first key >= want
            while (lo < hi) {
              const int64_t mid = (lo + hi) >> 1;
              if (vkeys[mid] < want) lo = mid + 1; else hi = mid;
            }
            if (lo < V && vkeys[lo] == want) row = static_cast<uint32_t>(lo);
          }
          nb[v * kNb + o] = row;
        }
  }
}

// One pass: every remaining point counts the other remaining points within r in the 27
// cells around it (squared distance, binary32, ((dx*dx + dy*dy) + dz*dz)) and is marked
// when the count exceeds the threshold.  Counting stops once it exceeds the threshold.
__global__ __launch_bounds__(256) void thin_count_kernel(
    const State* st, const int32_t* __restrict__ p2v, const uint32_t* __restrict__ sidx,
    const uint32_t* __restrict__ cstart, const uint32_t* __restrict__ vcnt,
    const uint32_t* __restrict__ nb, const float* __restrict__ sx, uint8_t* state, float r2,
    int64_t threshold, uint32_t* marked_count, const int* err) {
  if (error_raised(err)) return;  // nothing marked: the loop ends after one pass
  const int64_t m = st->nitems;
  uint32_t marked = 0;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m;
       i += int64_t(gridDim.x) * blockDim.x) {
    if (!(state[i] & kAlive)) continue;
    const float x = sx[3 * i], y = sx[3 * i + 1], z = sx[3 * i + 2];
    const uint32_t row = static_cast<uint32_t>(p2v[sidx[i]]);
    int64_t cnt = 0;
    for (int o = 0; o < kNb && cnt <= threshold; ++o) {
      const uint32_t c = nb[size_t(row) * kNb + o];
      if (c == kNoCell) continue;
      const int64_t j0 = cstart[c], j1 = j0 + vcnt[c];
      for (int64_t j = j0; j < j1 && cnt <= threshold; ++j) {
        if (j == i || !(state[j] & kAlive)) continue;
        const float ex = __fsub_rn(sx[3 * j], x);
        const float ey = __fsub_rn(sx[3 * j + 1], y);
        const float ez = __fsub_rn(sx[3 * j + 2], z);
        const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)),
                                   __fmul_rn(ez, ez));
        if (d2 <= r2) ++cnt;
      }
    }
    if (cnt > threshold) {
      state[i] = kAlive | kMarked;
      ++marked;
    }
  }
  for (int off = 16; off; off >>= 1) marked += __shfl_xor_sync(kFullMask, marked, off);
  if ((threadIdx.x & 31) == 0 && marked) atomicAdd(marked_count, marked);
}

__device__ __forceinline__ uint64_t select_key(const uint32_t* sprio, const uint32_t* sidx,
                                               int64_t i) {
  return (uint64_t(sprio[i]) << 32) | sidx[i];
}

// Histogram of one 8-bit digit of the marked points' keys that match the prefix so far.
__global__ __launch_bounds__(256) void thin_hist_kernel(const State* st, const uint8_t* state,
                                                        const uint32_t* __restrict__ sprio,
                                                        const uint32_t* __restrict__ sidx,
                                                        uint64_t prefix, uint64_t mask, int shift,
                                                        uint32_t* hist, const int* err) {
  __shared__ uint32_t h[256];
  if (block_error_raised(err)) return;
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t m = st->nitems;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m;
       i += int64_t(gridDim.x) * blockDim.x) {
    if (state[i] != (kAlive | kMarked)) continue;
    const uint64_t k = select_key(sprio, sidx, i);
    if ((k & mask) == prefix) atomicAdd(&h[(k >> shift) & 255u], 1u);
  }
  __syncthreads();
  if (h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

// Deletes the marked points whose key, cut to the decided digits, is <= prefix (all
// marked points when mask == 0); unmarks the rest for the next pass.
__global__ __launch_bounds__(256) void thin_delete_kernel(const State* st, uint8_t* state,
                                                          const uint32_t* __restrict__ sprio,
                                                          const uint32_t* __restrict__ sidx,
                                                          uint64_t prefix, uint64_t mask,
                                                          const int* err) {
  if (error_raised(err)) return;
  const int64_t m = st->nitems;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m;
       i += int64_t(gridDim.x) * blockDim.x) {
    if (state[i] != (kAlive | kMarked)) continue;
    const bool del = (select_key(sprio, sidx, i) & mask) <= prefix;
    state[i] = del ? 0 : kAlive;
  }
}

// keep flag per input point (the buffer was zeroed: invalid points stay 0), number kept.
__global__ __launch_bounds__(256) void thin_output_kernel(const State* st, const uint8_t* state,
                                                          const uint32_t* __restrict__ sidx,
                                                          uint8_t* keep, uint32_t* kept,
                                                          const int* err) {
  if (error_raised(err)) return;  // every keep flag stays 0, the count 0
  const int64_t m = st->nitems;
  uint32_t c = 0;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m;
       i += int64_t(gridDim.x) * blockDim.x) {
    const bool a = state[i] & kAlive;
    keep[sidx[i]] = a ? 1 : 0;
    c += a;
  }
  for (int off = 16; off; off >>= 1) c += __shfl_xor_sync(kFullMask, c, off);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(kept, c);
}

__global__ void thin_finish_kernel(const uint32_t* kept, int64_t* out_num_kept) {
  *out_num_kept = *kept;
}

vg_status thin_status(cudaError_t e) { return e == cudaSuccess ? VG_OK : VG_ERR_CUDA; }

int grid_for(int64_t n) {
  const int64_t b = ceil_div(n < 1 ? 1 : n, 256);
  const int64_t cap = int64_t(num_sms()) * 8;
  return static_cast<int>(b < cap ? b : cap);
}

}  // namespace
}  // namespace vg

using namespace vg;

extern "C" {

size_t vg_thin_workspace_bytes(int64_t n_points) {
  if (n_points < 0 || n_points > kMaxPoints) return 0;
  return thin_layout(n_points).total;
}

vg_status vg_thin(const float* xyz, int64_t n, float* origin, float cell, float radius,
                  int64_t threshold, int64_t batch, const uint32_t* priority, uint8_t* out_keep,
                  int64_t* out_num_kept, int32_t* out_passes, int32_t* out_error,
                  void* workspace, size_t workspace_bytes, int flags, vg_stream_t stream_) {
  if (!(cell > 0.0f) || !std::isfinite(cell)) return VG_ERR_INVALID_ARG;
  if (!(radius > 0.0f) || !(radius <= cell)) return VG_ERR_INVALID_ARG;  // 27 cells suffice
  if (threshold < 0 || batch < 1) return VG_ERR_INVALID_ARG;
  if ((flags & ~VG_ORIGIN_FROM_MIN) != 0) return VG_ERR_INVALID_ARG;
  if (!origin || !out_keep || !out_num_kept || (n > 0 && (!xyz || !priority)))
    return VG_ERR_INVALID_ARG;
  if (n < 0 || n > kMaxPoints) return VG_ERR_INVALID_ARG;
  const ThinLayout L = thin_layout(n);
  if (!workspace || workspace_bytes < L.total) return VG_ERR_WORKSPACE;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0 ||
      (reinterpret_cast<uintptr_t>(xyz) & 3) != 0 || (reinterpret_cast<uintptr_t>(priority) & 3) != 0 ||
      (reinterpret_cast<uintptr_t>(out_num_kept) & 7) != 0 || (reinterpret_cast<uintptr_t>(origin) & 3) != 0)
    return VG_ERR_ALIGN;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  char* ws = static_cast<char*>(workspace);
  const SortLayout S = sort_layout(n, 1);
  State* st = reinterpret_cast<State*>(ws + S.state);
  int* err = out_error ? reinterpret_cast<int*>(out_error) : &st->error;
  uint64_t* vkeys = reinterpret_cast<uint64_t*>(ws + L.vkeys);
  float* vcent = reinterpret_cast<float*>(ws + L.vcent);
  uint32_t* vcnt = reinterpret_cast<uint32_t*>(ws + L.vcnt);
  int64_t* vnum = reinterpret_cast<int64_t*>(ws + L.vnum);
  int32_t* p2v = reinterpret_cast<int32_t*>(ws + L.p2v);
  uint32_t* cstart = reinterpret_cast<uint32_t*>(ws + L.cstart);
  uint32_t* nb = reinterpret_cast<uint32_t*>(ws + L.nb);
  float* sx = reinterpret_cast<float*>(ws + L.sx);
  uint32_t* sprio = reinterpret_cast<uint32_t*>(ws + L.sprio);
  uint32_t* sidx = reinterpret_cast<uint32_t*>(ws + L.sidx);
  uint8_t* state = reinterpret_cast<uint8_t*>(ws + L.state);
  uint32_t* ctr = reinterpret_cast<uint32_t*>(ws + L.ctr);
  uint32_t* hist = reinterpret_cast<uint32_t*>(ws + L.hist);
  if (out_passes) *out_passes = 0;

  // grouping: the decimation's sort path, wide layout (point_to_voxel = each point's cell)
  const bool from_min = (flags & VG_ORIGIN_FROM_MIN) != 0;
  FramesArg fr{nullptr, 1, n, from_min ? nullptr : origin, from_min ? origin : nullptr, nullptr,
               cell, 0};
  SegOut out{vkeys, vcent, vcnt, nullptr, n, vnum, nullptr, p2v};
  vg_status s = run_frames(xyz, fr, from_min, out, out_error, workspace,
                           frames_workspace_bytes(n, 1, VG_METHOD_SORT), VG_METHOD_SORT, stream);
  if (s != VG_OK) return s;
  cudaError_t e = n > 0 ? cudaMemsetAsync(out_keep, 0, size_t(n), stream) : cudaSuccess;
  if (e == cudaSuccess) e = cudaMemsetAsync(ctr, 0, 4 * sizeof(uint32_t), stream);
  if (e != cudaSuccess) return VG_ERR_CUDA;
  const uint32_t* idx0 = reinterpret_cast<const uint32_t*>(ws + S.idx0);
  const uint32_t* idx1 = reinterpret_cast<const uint32_t*>(ws + S.idx1);
  const int g = grid_for(n);
  if (n > 0) {
    thin_setup_kernel<<<g, 256, 0, stream>>>(st, idx0, idx1, xyz, priority, p2v, cstart, sx,
                                             sprio, sidx, state, err);
    thin_neighbors_kernel<<<g, 256, 0, stream>>>(vnum, vkeys, nb, err);
  }
  const float r2 = radius * radius;
  const int64_t max_passes = n / batch + 2;  // every pass but the last deletes `batch` points
  int32_t passes = 0;
  for (; n > 0 && passes < max_passes; ++passes) {
    uint32_t marked = 0;
    e = cudaMemsetAsync(ctr, 0, sizeof(uint32_t), stream);
    if (e != cudaSuccess) return VG_ERR_CUDA;
    thin_count_kernel<<<g, 256, 0, stream>>>(st, p2v, sidx, cstart, vcnt, nb, sx, state, r2,
                                             threshold, ctr, err);
    e = cudaMemcpyAsync(&marked, ctr, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return VG_ERR_CUDA;
    if (int64_t(marked) <= batch) {  // the last pass: every marked point goes
      thin_delete_kernel<<<g, 256, 0, stream>>>(st, state, sprio, sidx, ~0ull, 0ull, err);
      ++passes;
      break;
    }
    // radix select of the `batch` smallest keys among the marked, 8 bits a round
    uint64_t prefix = 0, mask = 0;
    int64_t want = batch;
    for (int shift = 56; shift >= 0; shift -= 8) {
      uint32_t h[256];
      e = cudaMemsetAsync(hist, 0, sizeof(h), stream);
      if (e != cudaSuccess) return VG_ERR_CUDA;
      thin_hist_kernel<<<g, 256, 0, stream>>>(st, state, sprio, sidx, prefix, mask, shift, hist,
                                                  err);
      e = cudaMemcpyAsync(h, hist, sizeof(h), cudaMemcpyDeviceToHost, stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
      if (e != cudaSuccess) return VG_ERR_CUDA;
      int d = 0;
      while (d < 255 && want > int64_t(h[d])) want -= h[d++];
      prefix |= uint64_t(d) << shift;
      mask |= 0xffull << shift;
      if (want == int64_t(h[d])) break;  // the whole bucket goes: no finer digit needed
    }
    thin_delete_kernel<<<g, 256, 0, stream>>>(st, state, sprio, sidx, prefix, mask, err);
  }
  if (n > 0) {
    thin_output_kernel<<<g, 256, 0, stream>>>(st, state, sidx, out_keep, ctr + 1, err);
    thin_finish_kernel<<<1, 1, 0, stream>>>(ctr + 1, out_num_kept);
  } else {
    e = cudaMemsetAsync(out_num_kept, 0, sizeof(int64_t), stream);
  }
  if (out_passes) *out_passes = passes;
  return thin_status(e == cudaSuccess ? cudaGetLastError() : e);
}

}  // extern "C"
