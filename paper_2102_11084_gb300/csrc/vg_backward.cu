// Step a7: backward of the centroid map.
//
// A voxel's centroid is the mean of its n member points, so d c_v / d p_i = 1/n_v (per
// axis) for every member i and 0 otherwise; the gradient of any loss L(c) with respect
// to the points is grad_xyz[i] = dL/dc_v(i) / n_v(i), and 0 for an invalid point
// (point_to_voxel = -1).  Keys depend on the points only piecewise-constantly, so they
// carry no gradient.  (The paper has no training pass; this is the differentiable form
// of the decimation of Sec. II-C.)
//
// One pass over the points: 4 points per thread, int4 load of point_to_voxel, gathers of
// the voxel gradient rows and counts (voxel-ordered, mostly cached), 3 float4 stores.
#include "vg_device.cuh"
#include "vg_internal.h"

namespace vg {
namespace {

__global__ __launch_bounds__(256) void backward_kernel(const float* __restrict__ gc,
                                                       const uint32_t* __restrict__ counts,
                                                       const int32_t* __restrict__ p2v, int64_t n,
                                                       int64_t nv, float* __restrict__ gx,
                                                       int vec, int* err) {
  const int64_t stride = int64_t(gridDim.x) * 256 * 4;
  for (int64_t p0 = (int64_t(blockIdx.x) * 256 + threadIdx.x) * 4; p0 < n; p0 += stride) {
    int32_t v[4];
    if (vec && p0 + 4 <= n) {
      const int4 q = __ldcs(reinterpret_cast<const int4*>(p2v + p0));
      v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
      for (int j = 0; j < 4; ++j) v[j] = p0 + j < n ? p2v[p0 + j] : -1;
    }
    float g[12];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int32_t r = v[j];
      if (r >= 0 && r < nv) {
        const float inv = __uint2float_rn(__ldg(counts + r));
#pragma unroll
        for (int a = 0; a < 3; ++a) g[3 * j + a] = __fdiv_rn(__ldg(gc + 3 * size_t(r) + a), inv);
      } else {
        if (r >= nv || r < -1) set_error(err, kErrInvalidArg);
#pragma unroll
        for (int a = 0; a < 3; ++a) g[3 * j + a] = 0.0f;
      }
    }
    if (vec && p0 + 4 <= n) {
      float4* dst = reinterpret_cast<float4*>(gx + 3 * p0);
      __stcs(dst, make_float4(g[0], g[1], g[2], g[3]));
      __stcs(dst + 1, make_float4(g[4], g[5], g[6], g[7]));
      __stcs(dst + 2, make_float4(g[8], g[9], g[10], g[11]));
    } else {
      for (int j = 0; j < 4; ++j)
        if (p0 + j < n)
          for (int a = 0; a < 3; ++a) gx[3 * (p0 + j) + a] = g[3 * j + a];
    }
  }
}

}  // namespace

cudaError_t launch_backward(const float* grad_centroids, const uint32_t* counts,
                            const int32_t* p2v, int64_t n, int64_t num_voxels, float* grad_xyz,
                            int* err, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const bool vec = (reinterpret_cast<uintptr_t>(p2v) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(grad_xyz) & 15) == 0;
  const int64_t want = ceil_div(n, 1024);
  const int64_t cap = int64_t(num_sms()) * 8;
  backward_kernel<<<static_cast<int>(want < cap ? want : cap), 256, 0, stream>>>(
      grad_centroids, counts, p2v, n, num_voxels, grad_xyz, vec ? 1 : 0, err);
  return cudaGetLastError();
}

}  // namespace vg
