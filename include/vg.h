/*
 * vg.h -- C ABI of the GB300 (sm_103a) voxel-grid decimation library (libvg.so).
 *
 * The operation (arXiv 2102.11084, "Paralelizacion del submuestreo de nube de puntos
 * para plataformas con memoria unificada"):
 *   Sec. II-C and Algorithm 1: the filter takes a pointer to the camera cloud and
 *   returns a pointer to the filtered cloud; every point is classified into one cell
 *   of an ordered subdivision of space, a (cell, point) table is radix-sorted by cell
 *   so that each cell's points are contiguous and counted, and each occupied cell is
 *   replaced by one point -- the centroid, as in the voxel-grid filter of PCL that the
 *   paper replaces (Sec. I, II-C).  The block ("leaf") size is chosen at start
 *   (Sec. II-C).  The abstract's "iterative reduction with an ordered subdivision of
 *   space" is provided as a count-weighted octree pyramid (vg_pyramid).
 *
 * Definitions used by every entry point:
 *   valid point : x, y and z all finite (NaN marks a missing depth).
 *   voxel index : per axis, in IEEE binary32 round-to-nearest without contraction,
 *                 i = floor(fl(fl(p - origin) / leaf)); a point on a face goes to the
 *                 upper voxel.  0 <= i < 2^21 is required on every axis.
 *   voxel key   : 63-bit Morton code, bit b of ix/iy/iz -> key bit 3b/3b+1/3b+2.
 *   output      : one row per occupied voxel, in ascending key order: key (uint64),
 *                 count (uint32, number of valid points) and centroid (float32[3],
 *                 within 1e-5 m of the exact mean for coordinates below 64 m).
 *
 * Conventions:
 *   * Every pointer argument is DEVICE memory (cudaMalloc'd or equivalent) on the
 *     current device unless stated otherwise; the caller owns all of it.  The library
 *     allocates nothing in vg_downsample / vg_pyramid / vg_downsample_backward; scratch
 *     memory is the caller's `workspace`, sized by the matching *_workspace_bytes query.
 *   * xyz is float32 [n, 3], row-major (x, y, z interleaved), 4-byte aligned (16-byte
 *     alignment enables vector loads).  workspace must be 256-byte aligned.
 *   * Calls are asynchronous on `stream` (cudaStream_t; NULL = legacy default stream).
 *     Argument errors are returned synchronously and nothing is launched.  Errors found
 *     on the device (index out of range, output capacity, chained-scan timeout) are
 *     written to *out_error (device int32, first error wins, 0 = none) and are visible
 *     once the stream has completed; the outputs are then unspecified.
 *   * No C++ exception crosses this interface.
 */
#ifndef VG_H_
#define VG_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define VG_API __attribute__((visibility("default")))
#else
#define VG_API
#endif

typedef struct CUstream_st* vg_stream_t; /* same type as cudaStream_t */

typedef enum {
  VG_OK = 0,
  VG_ERR_INVALID_ARG = 1, /* a null pointer, a negative size, a bad leaf or flag      */
  VG_ERR_ALIGN = 2,       /* a pointer below its required alignment                  */
  VG_ERR_RANGE = 3,       /* device: a valid point's voxel index left [0, 2^21)        */
  VG_ERR_CAPACITY = 4,    /* device: more voxels than `cap` (first `cap` rows written)  */
  VG_ERR_WORKSPACE = 5,   /* workspace null or smaller than the query's answer          */
  VG_ERR_TIMEOUT = 6,     /* device: a chained-scan wait gave up (never expected)       */
  VG_ERR_CUDA = 7         /* a CUDA launch or runtime call failed                       */
} vg_status;

/* flags */
#define VG_ORIGIN_FROM_MIN 1 /* compute origin = per-axis min of the valid points and
                                write it to `origin` (else `origin` is read)            */
#define VG_METHOD_AUTO 0     /* let the library choose the grouping method             */
#define VG_METHOD_SORT 16    /* radix sort + segmented reduction                       */

/* Largest number of points one call accepts (2^30 - 1). */
#define VG_MAX_POINTS 1073741823LL

/* Human-readable name of a vg_status value (static string, never NULL). */
VG_API const char* vg_status_string(int status);

/* Library ABI version (major * 100 + minor). */
VG_API int vg_version(void);

/* Bytes of device workspace vg_downsample needs for a cloud of n_points with `flags`.
 * Pure host function; returns 0 for a negative n_points. */
VG_API size_t vg_downsample_workspace_bytes(int64_t n_points, int flags);

/*
 * vg_downsample -- steps a1..a5: origin (optional), voxel key per point, grouping by
 * key, per-voxel count and centroid, dense key-ordered output.
 * Sec. II-C and Algorithm 1 of arXiv 2102.11084 (classification into cells, radix sort
 * of the cell table, one output point per cell); centroid as in the PCL voxel filter.
 *
 *   xyz            [n,3] float32 input cloud (device).  Rows with a non-finite
 *                  coordinate are ignored.
 *   n              number of rows, 0 <= n <= VG_MAX_POINTS.
 *   origin         float32[3] (device).  Read, or written with the cloud minimum when
 *                  flags has VG_ORIGIN_FROM_MIN (then (0,0,0) if no point is valid).
 *   leaf           voxel edge length, finite and > 0.
 *   out_keys       uint64 [cap]   ascending voxel keys.
 *   out_centroids  float32 [cap,3] centroids.
 *   out_counts     uint32 [cap]   points per voxel.
 *   cap            capacity of the three outputs in rows (n is always enough).
 *   out_num_voxels int64 scalar: V, the number of occupied voxels.
 *   out_point_to_voxel  int32 [n] or NULL: output row of each point, -1 if invalid.
 *   out_error      int32 scalar or NULL: device error word (see conventions).
 *   workspace      scratch of at least vg_downsample_workspace_bytes(n, flags) bytes,
 *                  256-byte aligned; its contents on entry do not matter.
 *   flags          VG_ORIGIN_FROM_MIN | one VG_METHOD_*.
 *   stream         CUDA stream for every launch.
 */
VG_API vg_status vg_downsample(const float* xyz, int64_t n, float* origin, float leaf,
                        uint64_t* out_keys, float* out_centroids, uint32_t* out_counts,
                        int64_t cap, int64_t* out_num_voxels, int32_t* out_point_to_voxel,
                        int32_t* out_error, void* workspace, size_t workspace_bytes,
                        int flags, vg_stream_t stream);

/* Largest cloud vg_downsample_noalloc accepts (2^20 points: a 1280 x 720 frame fits). */
#define VG_NOALLOC_MAX_POINTS 1048576LL

/*
 * vg_downsample_noalloc -- vg_downsample without a caller workspace, for callers that
 * cannot call cudaMalloc: code that runs where allocating is not allowed or not possible,
 * such as a real-time sensor callback that must never block (cudaMalloc can synchronise
 * the device), or a host program whose device memory is owned by another allocator and
 * that cannot hand out scratch.  The paper has no counterpart of this entry point; it
 * exists only for such callers.
 *
 * Arguments are those of vg_downsample minus workspace/workspace_bytes; the caller still
 * passes (and owns) the input cloud and all outputs.  The scratch is a static device
 * array of vg_downsample_noalloc_scratch_bytes() bytes (about 25 MB, the workspace of
 * VG_NOALLOC_MAX_POINTS points) that every GPU loading the library keeps until the
 * process exits.  The call allocates nothing.
 *   * n > VG_NOALLOC_MAX_POINTS is rejected with VG_ERR_INVALID_ARG before any launch.
 *   * The first call on a device looks up the array's device address (once per device,
 *     with that device current); make that first call before any stream capture.
 *   * All calls on a device share the one array; it keeps the last call's contents and
 *     every call clears what must start at zero.  Calls whose work overlaps on the GPU
 *     (different streams, or different host threads) race on it: serialise them.
 */
VG_API vg_status vg_downsample_noalloc(const float* xyz, int64_t n, float* origin, float leaf,
                                       uint64_t* out_keys, float* out_centroids,
                                       uint32_t* out_counts, int64_t cap,
                                       int64_t* out_num_voxels, int32_t* out_point_to_voxel,
                                       int32_t* out_error, int flags, vg_stream_t stream);

/* Bytes of the static scratch array behind vg_downsample_noalloc. */
VG_API size_t vg_downsample_noalloc_scratch_bytes(void);

/* Profiling hook.  When `events` is non-NULL, every later vg_downsample call records
 * events[0] on its stream before its first kernel and events[k] after stage k, for
 * k = 1 .. min(max_events - 1, number of stages); NULL turns it off.  The events are
 * cudaEvent_t handles owned by the caller.  Stages of the sort path, in order: origin
 * (recorded even when the origin is given), keys, 8 radix passes, segmented reduction.
 * Returns the number of stages of the sort path (11). */
VG_API int vg_set_stage_events(void** events, int max_events);

/* Test hook: limit of every chained-scan wait in later calls (0 restores the default
 * of about a second).  A wait that reaches it records VG_ERR_TIMEOUT and returns. */
VG_API void vg_debug_set_spin_limit(uint32_t limit);

#ifdef __cplusplus
}
#endif

#endif /* VG_H_ */
