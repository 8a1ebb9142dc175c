// TEST INFRASTRUCTURE ONLY.  This file is the CPU oracle of voxel-grid decimation.
// It is a plain, slow, obviously-correct restatement of what the GPU library computes,
// used by the tests, by __graft_entry__.smoke() and by bench.py's CPU baseline.  Nothing
// in the product path may call it, and it shares no code with the CUDA sources.
//
// What it follows (arXiv 2102.11084, "Paralelizacion del submuestreo de nube de puntos
// para plataformas con memoria unificada"):
//   * Sec. II-C: every point of the cloud is placed in one cell of an ordered
//     subdivision of space; a key-value table (cell -> points) is sorted by cell so
//     that the number of points of every cell is known; the filtered cloud replaces
//     the cell's points by one point.  The voxel-grid filter that the paper replaces
//     (Sec. I and II-C, the PCL filter used by STVL) outputs the centroid of each
//     occupied voxel; that is the definition written out here.
//   * Sec. I (Octomap background): an octree cell is split into eight children, so the
//     parent of a Morton-coded voxel is key >> 3 (the "iterative reduction with an
//     ordered subdivision of space" of the abstract is read as this pyramid).
//
// Readings where the paper is silent:
//   R1  a point is valid iff x, y and z are all finite (NaN marks a missing depth);
//   R2  per axis, in IEEE binary32 with round-to-nearest and no contraction:
//         t = fl(p - o), q = fl(t / leaf), i = floor(q);  a point on a face goes up;
//   R3  0 <= i < 2^21 on every axis, otherwise the whole call fails (status 3);
//   R4  Morton key: bit b of ix -> key bit 3b, iy -> 3b+1, iz -> 3b+2;
//   R5  every occupied voxel is output (no minimum count), in ascending key order;
//   R6  centroid = mean of the raw member points, accumulated in FP64;
//   R7  pyramid level k+1 = level k merged by key >> 3, count-weighted, in FP64;
//   R8  backward of L = (1/(3V)) sum_v |c_v - t_v|^2 : dL/dp_i = dL/dc_v(i) / n_v(i);
//   R12 posed clouds (Sec. II-C: camera clouds are taken into the global frame by tf2
//       and the filter limits the height there): p' = R p + t with R, t row-major
//       [R|t], each coordinate in binary32 as ((r0 x + r1 y) + r2 z) + t, one rounding
//       per operation; a point is kept iff p' is finite and z_min <= z' <= z_max; the
//       kept points are then decimated as any cloud;
//   R13 per-voxel attributes (the RGB-D camera's colour, Sec. II-B): the mean of each
//       8-bit channel over the voxel's points, summed exactly and divided in FP64, then
//       rounded to binary32;
//   R14 minimum points per voxel (the PCL voxel filter's option): voxels with fewer
//       than m points are removed after grouping; the others keep their order, and
//       their points' point_to_voxel rows follow them (removed voxels' points get -1).
//   R16 neighbour-count thinning (Sec. II-C, Algorithm 1, its loop; Eq. 1 distance):
//       the valid points live in the cells of the lattice (origin, cell edge) (R2/R3);
//       repeat: every remaining point counts the other remaining points j in its own
//       and the 26 surrounding cells with d2 = ((dx*dx + dy*dy) + dz*dz) <= r*r in
//       binary32 (dx = x_j - x_i), and is marked when the count exceeds the threshold;
//       if more than K points are marked, the K marked points of lowest priority are
//       deleted (priority: a caller-given distinct rank per point, standing in for the
//       paper's random choice) and the loop repeats; otherwise every marked point is
//       deleted and the loop ends.  r <= cell edge makes the 27 cells hold every
//       neighbour.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fno-fast-math -shared -fPIC.
// Parity status: every function below is pinned by the tests in tests/test_oracle_*.py
// (brute force, closed forms, special cases and invariants); none is unpinned.

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <map>
#include <utility>
#include <vector>

namespace {

const int kStatusOk = 0;
const int kStatusRange = 3;
const int kStatusCapacity = 4;
const int64_t kAxisLimit = int64_t(1) << 21;

// R1: finite on all three axes.
bool point_is_valid(const float* p) {
  return std::isfinite(p[0]) && std::isfinite(p[1]) && std::isfinite(p[2]);
}

// R2 + R3 for one axis.  Every operation is a binary32 operation: operands are
// float, the build forbids contraction, and float arithmetic on x86-64 / aarch64
// has no excess precision.  Returns false when the index leaves [0, 2^21).
bool axis_index(float p, float o, float leaf, int64_t* out) {
  float t = p - o;     // fl(p - o)
  float q = t / leaf;  // fl(t / leaf)
  if (!(q >= 0.0f) || !(q < 2097152.0f)) return false;
  *out = static_cast<int64_t>(std::floor(q));
  return *out >= 0 && *out < kAxisLimit;
}

// R4: bit-by-bit interleave, the plainest possible form.
uint64_t morton_key(int64_t ix, int64_t iy, int64_t iz) {
  uint64_t key = 0;
  for (int b = 0; b < 21; ++b) {
    key |= static_cast<uint64_t>((ix >> b) & 1) << (3 * b);
    key |= static_cast<uint64_t>((iy >> b) & 1) << (3 * b + 1);
    key |= static_cast<uint64_t>((iz >> b) & 1) << (3 * b + 2);
  }
  return key;
}

struct VoxelSum {
  double sx = 0.0, sy = 0.0, sz = 0.0;
  uint64_t n = 0;
};

}  // namespace

extern "C" {

// Step a1: origin = per-axis minimum over the valid points (FP32 min is exact).
// Writes (0,0,0) when there is no valid point.  Returns the number of valid points.
int64_t oracle_origin(const float* xyz, int64_t n, float* origin_out) {
  int64_t valid = 0;
  float mn[3] = {0.0f, 0.0f, 0.0f};
  for (int64_t i = 0; i < n; ++i) {
    const float* p = xyz + 3 * i;
    if (!point_is_valid(p)) continue;
    for (int a = 0; a < 3; ++a) mn[a] = (valid == 0) ? p[a] : std::min(mn[a], p[a]);
    ++valid;
  }
  for (int a = 0; a < 3; ++a) origin_out[a] = mn[a];
  return valid;
}

// Step a2: per-point voxel index triple and Morton key.  valid[i] = 0 for an invalid
// point (its key and ijk are left as 0).  Returns 0, or 3 if any valid point falls
// outside [0, 2^21) on some axis.
int oracle_keys(const float* xyz, int64_t n, const float* origin, float leaf,
                uint64_t* keys, int64_t* ijk, uint8_t* valid) {
  int status = kStatusOk;
  for (int64_t i = 0; i < n; ++i) {
    const float* p = xyz + 3 * i;
    keys[i] = 0;
    if (ijk) ijk[3 * i] = ijk[3 * i + 1] = ijk[3 * i + 2] = 0;
    valid[i] = 0;
    if (!point_is_valid(p)) continue;
    int64_t idx[3];
    bool ok = true;
    for (int a = 0; a < 3; ++a) ok = ok && axis_index(p[a], origin[a], leaf, &idx[a]);
    if (!ok) {
      status = kStatusRange;
      continue;
    }
    valid[i] = 1;
    keys[i] = morton_key(idx[0], idx[1], idx[2]);
    if (ijk) {
      ijk[3 * i] = idx[0];
      ijk[3 * i + 1] = idx[1];
      ijk[3 * i + 2] = idx[2];
    }
  }
  return status;
}

// Steps a2-a5: group the valid points by voxel triple (std::map), accumulate the raw
// coordinates in FP64, and emit one centroid per occupied voxel in ascending Morton
// key order.  point_to_voxel (may be null) receives each point's output row, or -1.
// Returns V; *status is 0, 3 (range: nothing is written) or 4 (V > cap: the first cap
// voxels are written).
int64_t oracle_downsample(const float* xyz, int64_t n, const float* origin, float leaf,
                          uint64_t* out_keys, double* out_centroids, uint64_t* out_counts,
                          int64_t cap, int32_t* point_to_voxel, int* status) {
  *status = kStatusOk;
  std::map<std::array<int64_t, 3>, VoxelSum> voxels;
  for (int64_t i = 0; i < n; ++i) {
    const float* p = xyz + 3 * i;
    if (!point_is_valid(p)) continue;
    std::array<int64_t, 3> v;
    bool ok = true;
    for (int a = 0; a < 3; ++a) ok = ok && axis_index(p[a], origin[a], leaf, &v[a]);
    if (!ok) {
      *status = kStatusRange;
      return 0;
    }
    VoxelSum& s = voxels[v];
    s.sx += static_cast<double>(p[0]);
    s.sy += static_cast<double>(p[1]);
    s.sz += static_cast<double>(p[2]);
    s.n += 1;
  }
  // R5: ascending Morton key.  Keys are unique per voxel, so the order is unique.
  std::vector<std::pair<uint64_t, std::array<int64_t, 3>>> order;
  order.reserve(voxels.size());
  for (const auto& kv : voxels)
    order.emplace_back(morton_key(kv.first[0], kv.first[1], kv.first[2]), kv.first);
  std::sort(order.begin(), order.end());
  const int64_t V = static_cast<int64_t>(order.size());
  if (V > cap) *status = kStatusCapacity;
  std::map<std::array<int64_t, 3>, int64_t> rank;
  for (int64_t r = 0; r < V; ++r) {
    rank[order[r].second] = r;
    if (r >= cap) continue;
    const VoxelSum& s = voxels[order[r].second];
    out_keys[r] = order[r].first;
    out_counts[r] = s.n;
    out_centroids[3 * r] = s.sx / static_cast<double>(s.n);
    out_centroids[3 * r + 1] = s.sy / static_cast<double>(s.n);
    out_centroids[3 * r + 2] = s.sz / static_cast<double>(s.n);
  }
  if (point_to_voxel) {
    for (int64_t i = 0; i < n; ++i) {
      const float* p = xyz + 3 * i;
      point_to_voxel[i] = -1;
      if (!point_is_valid(p)) continue;
      std::array<int64_t, 3> v;
      for (int a = 0; a < 3; ++a) axis_index(p[a], origin[a], leaf, &v[a]);
      point_to_voxel[i] = static_cast<int32_t>(rank[v]);
    }
  }
  return V;
}

// Step a6: one pyramid level.  Level k (ascending keys) is merged into level k+1 by
// parent = key >> 3 with count-weighted FP64 centroids:  n' = sum n,
// c' = sum(n * c) / n'.  Output is in ascending parent key.  Returns V_{k+1}.
int64_t oracle_pyramid_merge(const uint64_t* keys, const double* centroids,
                             const uint64_t* counts, int64_t v, uint64_t* out_keys,
                             double* out_centroids, uint64_t* out_counts) {
  std::map<uint64_t, VoxelSum> parents;
  for (int64_t r = 0; r < v; ++r) {
    VoxelSum& s = parents[keys[r] >> 3];
    const double w = static_cast<double>(counts[r]);
    s.sx += w * centroids[3 * r];
    s.sy += w * centroids[3 * r + 1];
    s.sz += w * centroids[3 * r + 2];
    s.n += counts[r];
  }
  int64_t r = 0;
  for (const auto& kv : parents) {
    out_keys[r] = kv.first;
    out_counts[r] = kv.second.n;
    out_centroids[3 * r] = kv.second.sx / static_cast<double>(kv.second.n);
    out_centroids[3 * r + 1] = kv.second.sy / static_cast<double>(kv.second.n);
    out_centroids[3 * r + 2] = kv.second.sz / static_cast<double>(kv.second.n);
    ++r;
  }
  return r;
}

// Step a7: backward of the centroid map.  A centroid is the mean of its n members, so
// d c_v / d p_i = 1/n_v for each member i (per axis) and 0 otherwise:
// grad_xyz[i] = grad_centroids[v(i)] / n_v(i); invalid points (v = -1) get 0.
void oracle_backward(const double* grad_centroids, const uint64_t* counts,
                     const int32_t* point_to_voxel, int64_t n, double* grad_xyz) {
  for (int64_t i = 0; i < n; ++i) {
    const int32_t v = point_to_voxel[i];
    for (int a = 0; a < 3; ++a)
      grad_xyz[3 * i + a] =
          (v < 0) ? 0.0 : grad_centroids[3 * v + a] / static_cast<double>(counts[v]);
  }
}

// R13: mean attributes of voxels 0..V-1 from each point's voxel row (p2v, -1 = none).
void oracle_voxel_attrs(const int32_t* p2v, int64_t n, const uint8_t* attrs, int channels,
                        int64_t num_voxels, float* out) {
  std::vector<double> sum(size_t(num_voxels) * channels, 0.0);
  std::vector<uint64_t> cnt(size_t(num_voxels), 0);
  for (int64_t i = 0; i < n; ++i) {
    const int32_t v = p2v[i];
    if (v < 0) continue;
    cnt[size_t(v)] += 1;
    for (int c = 0; c < channels; ++c) sum[size_t(v) * channels + c] += double(attrs[i * channels + c]);
  }
  for (int64_t v = 0; v < num_voxels; ++v)
    for (int c = 0; c < channels; ++c)
      out[v * channels + c] =
          cnt[size_t(v)] ? float(sum[size_t(v) * channels + c] / double(cnt[size_t(v)])) : 0.0f;
}

// R14: removes voxels with fewer than m points, in place and in order; remaps p2v.
// Returns the new voxel count.
int64_t oracle_min_count(uint64_t* keys, double* centroids, uint64_t* counts, float* attrs,
                         int channels, int64_t num_voxels, uint64_t m, int32_t* p2v, int64_t n) {
  std::vector<int64_t> row(size_t(num_voxels), -1);
  int64_t w = 0;
  for (int64_t v = 0; v < num_voxels; ++v) {
    if (counts[v] < m) continue;
    row[size_t(v)] = w;
    keys[w] = keys[v];
    counts[w] = counts[v];
    for (int a = 0; a < 3; ++a) centroids[3 * w + a] = centroids[3 * v + a];
    for (int c = 0; c < channels; ++c) attrs[w * channels + c] = attrs[v * channels + c];
    ++w;
  }
  for (int64_t i = 0; p2v && i < n; ++i)
    if (p2v[i] >= 0) p2v[i] = int32_t(row[size_t(p2v[i])]);
  return w;
}

// R16: neighbour counts of the remaining points (alive[i] != 0), the plain 27-cell search.
void oracle_neighbor_counts(const float* xyz, int64_t n, const int64_t* ijk,
                            const uint8_t* alive, float r, int64_t* counts) {
  std::map<std::array<int64_t, 3>, std::vector<int64_t>> cells;
  for (int64_t i = 0; i < n; ++i)
    if (alive[i]) cells[{ijk[3 * i], ijk[3 * i + 1], ijk[3 * i + 2]}].push_back(i);
  const float r2 = r * r;
  for (int64_t i = 0; i < n; ++i) {
    counts[i] = 0;
    if (!alive[i]) continue;
    for (int64_t dx = -1; dx <= 1; ++dx)
      for (int64_t dy = -1; dy <= 1; ++dy)
        for (int64_t dz = -1; dz <= 1; ++dz) {
          auto it = cells.find({ijk[3 * i] + dx, ijk[3 * i + 1] + dy, ijk[3 * i + 2] + dz});
          if (it == cells.end()) continue;
          for (int64_t j : it->second) {
            if (j == i) continue;
            const float ex = xyz[3 * j] - xyz[3 * i];
            const float ey = xyz[3 * j + 1] - xyz[3 * i + 1];
            const float ez = xyz[3 * j + 2] - xyz[3 * i + 2];
            float d2 = ex * ex;
            d2 = d2 + ey * ey;
            d2 = d2 + ez * ez;
            if (d2 <= r2) ++counts[i];
          }
        }
  }
}

// R16: the thinning loop.  keep[i] = 1 for the points that remain; returns the number of
// passes of the loop, or -status when a voxel index leaves [0, 2^21).
int64_t oracle_thin(const float* xyz, int64_t n, const float* origin, float cell, float r,
                    int64_t threshold, int64_t batch, const uint32_t* priority, uint8_t* keep) {
  std::vector<int64_t> ijk(size_t(3 * (n > 0 ? n : 1)), 0);
  for (int64_t i = 0; i < n; ++i) {
    keep[i] = 0;
    if (!point_is_valid(xyz + 3 * i)) continue;
    for (int a = 0; a < 3; ++a)
      if (!axis_index(xyz[3 * i + a], origin[a], cell, &ijk[size_t(3 * i + a)]))
        return -kStatusRange;
    keep[i] = 1;
  }
  std::vector<int64_t> counts(size_t(n > 0 ? n : 1));
  int64_t passes = 0;
  for (;;) {
    ++passes;
    oracle_neighbor_counts(xyz, n, ijk.data(), keep, r, counts.data());
    std::vector<std::pair<uint32_t, int64_t>> marked;  // (priority, point)
    for (int64_t i = 0; i < n; ++i)
      if (keep[i] && counts[size_t(i)] > threshold) marked.push_back({priority[i], i});
    if (int64_t(marked.size()) > batch) {
      std::sort(marked.begin(), marked.end());
      for (int64_t k = 0; k < batch; ++k) keep[marked[size_t(k)].second] = 0;
      continue;
    }
    for (const auto& m : marked) keep[m.second] = 0;
    return passes;
  }
}

// R12: the posed cloud.  Dropped points come out as NaN (R1 then rejects them).
void oracle_pose(const float* xyz, int64_t n, const float* pose, const float* zlim,
                 float* out) {
  const float nan = std::nanf("");
  for (int64_t i = 0; i < n; ++i) {
    const float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    float g[3] = {x, y, z};
    if (pose) {
      for (int a = 0; a < 3; ++a) {
        const float* r = pose + 4 * a;
        float acc = r[0] * x;   // fl(r0 x)
        acc = acc + r[1] * y;   // fl(acc + fl(r1 y))
        acc = acc + r[2] * z;   // fl(acc + fl(r2 z))
        g[a] = acc + r[3];      // fl(acc + t)
      }
    }
    const bool finite = std::isfinite(g[0]) && std::isfinite(g[1]) && std::isfinite(g[2]);
    const bool in_band = !zlim || (g[2] >= zlim[0] && g[2] <= zlim[1]);
    for (int a = 0; a < 3; ++a) out[3 * i + a] = finite && in_band ? g[a] : nan;
  }
}

// The loss whose gradient oracle_backward propagates, as a function of FP64 point
// coordinates with the voxel membership held fixed (point_to_voxel from an
// oracle_downsample of the FP32 cloud):  L = (1/(3V)) sum_v |c_v - t_v|^2 where
// c_v is the mean of the member points.  Used for central finite differences.
double oracle_centroid_loss(const double* xyz, int64_t n, const int32_t* point_to_voxel,
                            int64_t v, const double* targets) {
  std::vector<double> sums(3 * v, 0.0);
  std::vector<uint64_t> counts(v, 0);
  for (int64_t i = 0; i < n; ++i) {
    const int32_t k = point_to_voxel[i];
    if (k < 0) continue;
    for (int a = 0; a < 3; ++a) sums[3 * k + a] += xyz[3 * i + a];
    counts[k] += 1;
  }
  double loss = 0.0;
  for (int64_t k = 0; k < v; ++k)
    for (int a = 0; a < 3; ++a) {
      const double c = sums[3 * k + a] / static_cast<double>(counts[k]);
      const double e = c - targets[3 * k + a];
      loss += e * e;
    }
  return v > 0 ? loss / (3.0 * static_cast<double>(v)) : 0.0;
}

}  // extern "C"
