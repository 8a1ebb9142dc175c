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
 *   * The radix passes and reductions are persistent kernels sized to fill the GPU, and a
 *     tile may wait (bounded) on tiles other blocks of its grid hold.  Two large calls
 *     running at the same time on different streams share the SMs and slow each other
 *     down several times over: order such calls (an event between them); their copies
 *     may still overlap.
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
#define VG_METHOD_AUTO 0     /* the library's choice: SORT, with the bucket grouping
                                from 4,194,304 points on and every digit in global radix
                                passes (VG_SORT_LSD) below.  A single camera frame is
                                fastest with VG_SORT_FRAME, which AUTO does not take: it
                                needs 32-bit keys, known only on the device, and AUTO
                                serves every cloud without a host synchronisation        */
#define VG_METHOD_SORT 16    /* sort the points by key and reduce each run of equal keys.
                                32-bit keys (no point_to_voxel, no attributes, extents
                                bound the keys): the top <= 16 key bits are split by one
                                or two most-significant-digit partition passes and every
                                bucket of the low bits is reduced in one block's shared
                                memory; otherwise a global LSD radix sort of every digit
                                and a segmented reduction                                 */
#define VG_METHOD_HASH 32    /* hash-table accumulation + radix sort of the voxels     */
#define VG_METHOD_MASK 48
#define VG_SORT_BUCKETS 2    /* accepted for compatibility; changes nothing (32-bit keys
                                are grouped by buckets by default)                       */
#define VG_SORT_LSD 4        /* SORT with 32-bit keys: every key digit in a global LSD
                                radix pass, then the segmented reduction, instead of the
                                bucket grouping (same rows; for comparison)              */
#define VG_USE_GRAPH 64      /* vg_downsample_batch: capture / replay a CUDA graph      */
#define VG_SORT_FRAME 128    /* SORT for one camera frame (vg_downsample, or a batch of
                                one frame), for clouds whose launches cost more than their
                                bytes.  A frame of up to vg_frame_one_launch_points()
                                points is grouped by ONE cooperative launch: an occupancy
                                bitmap over the keys ranks the cells in key order and the
                                cells' sums are added at their rows.  A larger frame is
                                counted into bins of 2^12 consecutive keys, scattered
                                once, and every bin reduced in one block's shared memory
                                (five kernels after the extent kernel).  Needs 32-bit
                                keys (the Morton code of the frame's per-axis maximum
                                index below 2^32 - 1), else the call records
                                VG_ERR_RANGE.  Several frames, point_to_voxel or
                                attributes take the global radix sort (as with
                                VG_SORT_LSD).  Same rows as SORT                          */
#define VG_GRID_SHIFT 8      /* vg_downsample_frames: blocks per SM of the streaming    */
#define VG_GRID_MASK (0xff << VG_GRID_SHIFT) /* kernels (0 = default 8)                */

/* Largest number of frames of one batched call, and of pyramid levels. */
#define VG_MAX_FRAMES 1024
#define VG_MAX_LEVELS 8

/* Largest number of points one call accepts (2^30 - 1). */
#define VG_MAX_POINTS 1073741823LL

/* Human-readable name of a vg_status value (static string, never NULL). */
VG_API const char* vg_status_string(int status);

/* Library ABI version (major * 100 + minor). */
VG_API int vg_version(void);

/* Bytes of device workspace vg_downsample needs for a cloud of n_points with `flags`.
 * Pure host function; returns 0 for a negative n_points. */
VG_API size_t vg_downsample_workspace_bytes(int64_t n_points, int flags);

/* Largest frame, in points, that VG_SORT_FRAME groups in one cooperative launch on the
 * current device: its grid (one block of 1024 threads per SM) holding 14 points a thread,
 * and at most 2^21 points (2,097,152: a 1920x1080 frame fits); 0 when the device cannot
 * run that launch.  posed != 0 asks for calls with a pose or height limits.  Larger frames
 * take the bin grouping.  Reads device attributes only. */
VG_API int64_t vg_frame_one_launch_points(int posed);

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
 *   flags          VG_ORIGIN_FROM_MIN | one VG_METHOD_* (| VG_SORT_BUCKETS with SORT).
 *                  SORT and HASH give identical results; HASH needs more workspace and
 *                  wins when voxels hold many points.  VG_SORT_BUCKETS changes how the
 *                  narrow layout sorts, not the rows.
 *   stream         CUDA stream for every launch.
 */
VG_API vg_status vg_downsample(const float* xyz, int64_t n, float* origin, float leaf,
                        uint64_t* out_keys, float* out_centroids, uint32_t* out_counts,
                        int64_t cap, int64_t* out_num_voxels, int32_t* out_point_to_voxel,
                        int32_t* out_error, void* workspace, size_t workspace_bytes,
                        int flags, vg_stream_t stream);

/*
 * Batched frames -- step a8: many clouds of uneven size in one call.  Every frame is
 * decimated exactly as vg_downsample would decimate it alone (same keys, counts and
 * centroid bits); all frames share the launches and one radix sort (frame id above the
 * voxel key).  The paper distributes the subdivisions of space over every CUDA processor
 * (Sec. II-C, grid sized to the processor count).
 *
 *   xyz               [n_total,3] float32, the frames concatenated.
 *   frame_offsets     int64 [n_frames+1] (device): frame f is rows [off[f], off[f+1]);
 *                     off[0] = 0, non-decreasing, off[n_frames] = n_total (checked on the
 *                     device: VG_ERR_INVALID_ARG).  1 <= n_frames <= VG_MAX_FRAMES.
 *   origins           float32 [n_frames,3] (device): read, or written with each frame's
 *                     minimum when flags has VG_ORIGIN_FROM_MIN.
 *   leaves            float32 [n_frames] (device): each frame's leaf (finite, > 0).
 *   out_keys/out_centroids/out_counts  rows of all frames, frame by frame, each frame in
 *                     ascending key order; keys are the frames' own voxel keys.
 *   out_frame_offsets int64 [n_frames+1] (device): frame f's rows are
 *                     [out[f], out[f+1]); out[n_frames] = total voxels.
 *   out_point_to_voxel int32 [n_total] or NULL: global output row of each point, or -1.
 * The per-frame key field plus the frame id must fit in 63 bits (VG_ERR_RANGE otherwise).
 */
VG_API size_t vg_batch_workspace_bytes(int64_t n_total, int n_frames, int flags);
VG_API vg_status vg_downsample_frames(const float* xyz, int64_t n_total,
                                      const int64_t* frame_offsets, int n_frames,
                                      float* origins, const float* leaves, uint64_t* out_keys,
                                      float* out_centroids, uint32_t* out_counts, int64_t cap,
                                      int64_t* out_frame_offsets, int32_t* out_point_to_voxel,
                                      int32_t* out_error, void* workspace,
                                      size_t workspace_bytes, int flags, vg_stream_t stream);

/*
 * Posed frames: vg_downsample_frames for clouds given in their sensors' frames.  The
 * paper's pipeline takes each camera cloud into the global frame (the tf2 step) and the
 * voxel filter limits the height of the cloud there (Sec. II-C); here both are fused
 * into the first read of every point, so they cost no extra pass over the cloud:
 *
 *   p' = R p + t, each of x', y', z' computed in float32 as ((r0*x + r1*y) + r2*z) + t
 *   with every product and sum rounded on its own (no fused multiply-add);
 *   the point is kept iff x', y', z' are finite and z_min <= z' <= z_max.
 *
 * Everything else (origin = minimum of the kept points, keys, centroids in the common
 * frame, outputs, workspace: vg_batch_workspace_bytes) is as in vg_downsample_frames.
 *
 *   poses     float32 [n_frames,12] (device) row-major [R|t] of each frame, or NULL for
 *             the identity.
 *   z_limits  float32 [n_frames,2] (device) [z_min, z_max] of each frame, or NULL for no
 *             limit.
 * Both NULL is exactly vg_downsample_frames.  Misaligned poses/z_limits: VG_ERR_ALIGN.
 */
VG_API vg_status vg_downsample_frames_posed(
    const float* xyz, int64_t n_total, const int64_t* frame_offsets, int n_frames,
    const float* poses, const float* z_limits, float* origins, const float* leaves,
    uint64_t* out_keys, float* out_centroids, uint32_t* out_counts, int64_t cap,
    int64_t* out_frame_offsets, int32_t* out_point_to_voxel, int32_t* out_error, void* workspace,
    size_t workspace_bytes, int flags, vg_stream_t stream);

/*
 * Voxel extras: per-voxel attributes and a minimum point count, on top of posed frames.
 * The paper's camera is an RGB-D sensor (Sec. II-B), so a voxel can carry the mean
 * colour of its points next to their centroid; the PCL voxel filter that the paper
 * replaces can also drop voxels holding fewer than a given number of points.
 *
 *   attrs          uint8 [n_total, attr_channels] (device), row i belongs to point i, or
 *                  NULL for none.  1 <= attr_channels <= 4 when attrs is given.
 *   out_attrs      float32 [cap, attr_channels] (device): each voxel's channel means,
 *                  sum over its points (exact) / count, divided in FP64 and rounded to
 *                  float32.  Needs the sort path (VG_METHOD_HASH: VG_ERR_INVALID_ARG).
 *   min_count      voxels with fewer points are removed after grouping (0 or 1 keeps
 *                  them all); the kept voxels keep their order, out_frame_offsets and
 *                  the voxel count refer to them, and points of removed voxels get -1 in
 *                  out_point_to_voxel.
 * The workspace must hold vg_downsample_ex_workspace_bytes(n_total, n_frames, flags,
 * extras) bytes.  extras == NULL is exactly vg_downsample_frames_posed.
 */
typedef struct vg_voxel_extras {
  const uint8_t* attrs;
  int attr_channels;
  float* out_attrs;
  uint32_t min_count;
} vg_voxel_extras;

VG_API size_t vg_downsample_ex_workspace_bytes(int64_t n_total, int n_frames, int flags,
                                               const vg_voxel_extras* extras);
VG_API vg_status vg_downsample_frames_ex(
    const float* xyz, int64_t n_total, const int64_t* frame_offsets, int n_frames,
    const float* poses, const float* z_limits, float* origins, const float* leaves,
    uint64_t* out_keys, float* out_centroids, uint32_t* out_counts, int64_t cap,
    int64_t* out_frame_offsets, int32_t* out_point_to_voxel, const vg_voxel_extras* extras,
    int32_t* out_error, void* workspace, size_t workspace_bytes, int flags, vg_stream_t stream);

/*
 * Persistent voxel map.  In the paper's pipeline every filtered camera cloud is merged
 * into a global map (STVL marks the cells of its OpenVDB grid, Sec. II-C).  A vg_map is
 * that map kept on the GPU: an open-addressing table in device memory, keyed by the
 * 63-bit Morton key of the voxel (R4) on one fixed lattice (origin, leaf), holding each
 * voxel's point count and fixed-point offset sums.  Inserting frames one call at a time
 * and extracting gives exactly what one vg_downsample of all the inserted points with
 * that origin would give (same keys, counts and centroid bits), whatever the order and
 * grouping of the inserts.
 *
 *   vg_map_create    allocates the table for about `capacity` voxels (2x slots, power
 *                    of two) and the scratch of the extraction, once; origin is host
 *                    float32[3], leaf finite > 0.  No other call allocates.
 *   vg_map_insert    adds the valid points of a batch of frames (layout as in
 *                    vg_downsample_frames; frame_offsets NULL means one frame of
 *                    n_total points), each taken through its pose and height band
 *                    first when poses / z_limits are given (see
 *                    vg_downsample_frames_posed).  A point whose voxel index leaves
 *                    [0, 2^21) on an axis records VG_ERR_RANGE and is skipped; a full
 *                    table records VG_ERR_CAPACITY; both in *out_error (device int32,
 *                    set, never cleared, by the call's kernels; may be NULL).
 *   vg_map_extract   writes every voxel of the map in ascending key order: keys,
 *                    centroids, counts (device, capacity cap), *out_num_voxels (device).
 *                    The map is unchanged.
 *   vg_map_clear     empties the map (asynchronous on the stream).
 * All calls are asynchronous on `stream`; calls on one map must not overlap on the GPU.
 */
typedef struct vg_map vg_map;
VG_API vg_status vg_map_create(vg_map** map, int64_t capacity, const float* origin, float leaf);
VG_API vg_status vg_map_destroy(vg_map* map);
VG_API vg_status vg_map_clear(vg_map* map, vg_stream_t stream);
VG_API vg_status vg_map_insert(vg_map* map, const float* xyz, int64_t n_total,
                               const int64_t* frame_offsets, int n_frames, const float* poses,
                               const float* z_limits, int32_t* out_error, vg_stream_t stream);
VG_API vg_status vg_map_extract(vg_map* map, uint64_t* out_keys, float* out_centroids,
                                uint32_t* out_counts, int64_t cap, int64_t* out_num_voxels,
                                int32_t* out_error, vg_stream_t stream);

/*
 * Neighbour-count thinning: the paper's own filter loop (Sec. II-C, Algorithm 1).  The
 * valid points are placed in the cells (edge `cell`, origin as in vg_downsample) of a
 * regular grid; then, pass after pass, every remaining point counts the other
 * remaining points in its own and the 26 surrounding cells within distance `radius`
 * (Eq. 1; squared distance in float32 as ((dx*dx + dy*dy) + dz*dz) with dx = x_j - x_i,
 * compared with radius*radius) and is marked when the count exceeds `threshold`.  When
 * more than `batch` points are marked, the `batch` marked points of lowest `priority`
 * (ties by point index) are deleted and the loop goes on; otherwise every marked point
 * is deleted and the loop ends.  The paper deletes a random batch of 1000; priority
 * stands in for that random choice (pass a random permutation for the paper's
 * behaviour).
 *
 *   xyz, n         as vg_downsample; origin float32[3] (device), read or written as
 *                  there (VG_ORIGIN_FROM_MIN).
 *   cell, radius   finite, 0 < radius <= cell (so the 27 cells hold every neighbour).
 *   threshold      >= 0; batch >= 1.
 *   priority       uint32 [n] (device).
 *   out_keep       uint8 [n] (device): 1 for the points that remain, 0 otherwise
 *                  (invalid points included); *out_num_kept (device int64) their number.
 *   out_passes     host int32 or NULL: passes of the loop.
 * Workspace: vg_thin_workspace_bytes(n) bytes.  The call synchronises the stream once per
 * pass and once per round of the batch selection (8 bits a round).
 */
VG_API size_t vg_thin_workspace_bytes(int64_t n_points);
VG_API vg_status vg_thin(const float* xyz, int64_t n, float* origin, float cell, float radius,
                         int64_t threshold, int64_t batch, const uint32_t* priority,
                         uint8_t* out_keep, int64_t* out_num_kept, int32_t* out_passes,
                         int32_t* out_error, void* workspace, size_t workspace_bytes, int flags,
                         vg_stream_t stream);

/*
 * Batch plan: owns a workspace for up to max_points points in max_frames frames
 * (allocated here, once), the grouping method and grid size, and a CUDA graph of the
 * batched launch sequence.  vg_downsample_batch takes the arguments of
 * vg_downsample_frames without the workspace; with VG_USE_GRAPH (non-NULL stream
 * required) the first call captures the sequence and later calls with the same pointers,
 * sizes and flags replay it with one cudaGraphLaunch.  A plan is not thread-safe and its
 * workspace is shared by its calls: calls that overlap on the GPU race.
 * vg_plan_tune times four groupings -- VG_METHOD_SORT, VG_METHOD_SORT | VG_SORT_LSD,
 * VG_METHOD_SORT | VG_SORT_FRAME (one-frame batches only) and VG_METHOD_HASH -- x
 * streaming grids {4,8,16} blocks/SM on the given batch (`reps` replays each,
 * host-synchronising) and keeps the fastest; out_ms (12 floats or NULL) receives
 * sort@4,8,16, sort_lsd@4,8,16, frame@4,8,16 then hash@4,8,16 in ms per batch, -1 for a
 * grouping not timed (frame with several frames) or one whose runs recorded a device
 * error (frame with keys wider than 32 bits; the error word is cleared again).  A plan's
 * method (vg_plan_create flags, vg_plan_configure, vg_plan_get) is one of those four or
 * VG_METHOD_AUTO (the library's choice by cloud size, the default of a new plan).
 */
typedef struct vg_plan vg_plan;
VG_API vg_status vg_plan_create(vg_plan** plan, int max_frames, int64_t max_points, int flags);
VG_API vg_status vg_plan_destroy(vg_plan* plan);
VG_API vg_status vg_plan_configure(vg_plan* plan, int method, int grid_per_sm);
VG_API vg_status vg_plan_get(const vg_plan* plan, int* method, int* grid_per_sm,
                             size_t* workspace_bytes);
VG_API vg_status vg_downsample_batch(vg_plan* plan, const float* xyz, int64_t n_total,
                                     const int64_t* frame_offsets, int n_frames, float* origins,
                                     const float* leaves, uint64_t* out_keys,
                                     float* out_centroids, uint32_t* out_counts, int64_t cap,
                                     int64_t* out_frame_offsets, int32_t* out_point_to_voxel,
                                     int32_t* out_error, int flags, vg_stream_t stream);
VG_API vg_status vg_plan_tune(vg_plan* plan, const float* xyz, int64_t n_total,
                              const int64_t* frame_offsets, int n_frames, float* origins,
                              const float* leaves, uint64_t* out_keys, float* out_centroids,
                              uint32_t* out_counts, int64_t cap, int64_t* out_frame_offsets,
                              int32_t* out_error, int flags, int reps, vg_stream_t stream,
                              float* out_ms);

/*
 * vg_pyramid -- step a6: the count-weighted octree pyramid ("iterative reduction with an
 * ordered subdivision of space", abstract and Sec. II-C; octree cells split in eight,
 * Sec. I).  Level 0 is vg_downsample at `leaf`; level k+1 merges level k by key >> 3
 * (edge doubles), n' = sum n, centroid' = count-weighted mean.  Levels are written one
 * after another into the outputs: level k is rows [off[k], off[k+1]) of out_keys /
 * out_centroids / out_counts, with out_level_offsets int64 [levels+1] (device).  Keys and
 * counts of level k equal vg_downsample at leaf 2^k * leaf exactly; centroids agree within
 * the library's tolerance.  cap_total >= levels * n always suffices.  Single cloud,
 * sort method, 1 <= levels <= VG_MAX_LEVELS.  point_to_voxel refers to level 0.  flags:
 * VG_ORIGIN_FROM_MIN | VG_SORT_BUCKETS (level 0's grouping; anything else is
 * VG_ERR_INVALID_ARG).
 */
VG_API size_t vg_pyramid_workspace_bytes(int64_t n_points, int levels, int flags);
VG_API vg_status vg_pyramid(const float* xyz, int64_t n, float* origin, float leaf, int levels,
                            uint64_t* out_keys, float* out_centroids, uint32_t* out_counts,
                            int64_t cap_total, int64_t* out_level_offsets,
                            int32_t* out_point_to_voxel, int32_t* out_error, void* workspace,
                            size_t workspace_bytes, int flags, vg_stream_t stream);

/*
 * vg_downsample_backward -- step a7: gradient of a loss of the centroids with respect to
 * the input points.  A centroid is the mean of its n members, so
 * grad_xyz[i] = grad_centroids[v(i)] / counts[v(i)] for a valid point i (v = point_to_voxel
 * from the forward call) and 0 for an invalid one (v = -1); keys are piecewise constant and
 * carry no gradient.  (The paper has no training pass; this differentiates its decimation.)
 *   grad_centroids float32 [num_voxels,3], counts uint32 [num_voxels],
 *   point_to_voxel int32 [n], grad_xyz float32 [n,3] (written, every row), out_error int32
 *   scalar: VG_ERR_INVALID_ARG if an entry of point_to_voxel is outside [-1, num_voxels).
 */
VG_API vg_status vg_downsample_backward(const float* grad_centroids, const uint32_t* counts,
                                        const int32_t* point_to_voxel, int64_t n,
                                        int64_t num_voxels, float* grad_xyz, int32_t* out_error,
                                        vg_stream_t stream);

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
 *   * Only the sort method runs here (VG_METHOD_AUTO, VG_METHOD_SORT, with or without
 *     VG_SORT_BUCKETS or VG_SORT_LSD): the array holds the sort path's workspace, so
 *     VG_METHOD_HASH and VG_SORT_FRAME are rejected with VG_ERR_INVALID_ARG before any
 *     launch.
 *   * The device address of the array is cached per device; cudaDeviceReset invalidates
 *     it, so do not call this entry point after resetting the device.
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
 * cudaEvent_t handles owned by the caller.  Stages of the sort path, in order: extent /
 * origin (recorded even when skipped), keys, then the bucket grouping's first partition
 * pass (with the scan of its digit counts), second partition pass (with its digit
 * histogram and bucket scan) and bucket kernel (all three return at once, or are not
 * launched, when the call takes the global radix sort), then 8 radix passes (those
 * beyond the key's significant digits, and all of them with the bucket grouping, return
 * at once) and the segmented reduction (count, scan, reduce); of the hash path: origin,
 * insert, compaction, 8 radix passes, finalize, point-to-voxel.
 * Returns the largest number of events a call records (20). */
VG_API int vg_set_stage_events(void** events, int max_events);

/* Test of the bounded waits: runs one chained-scan wait on four device words
 * (scratch_words, caller-owned) that nothing publishes, with a limit of `limit` polls
 * (1 .. 2^22); the wait gives up and *out_error becomes VG_ERR_TIMEOUT.  No hang, no
 * fault: this is how a lost predecessor is reported. */
VG_API vg_status vg_debug_wait_timeout(uint32_t* scratch_words, uint32_t limit,
                                       int32_t* out_error, vg_stream_t stream);

/* Test of the grid barrier of the one-launch frame grouping: a two-block cooperative
 * launch whose barrier waits for one block more than it has, on one device word
 * (scratch_words, caller-owned, zeroed by the call) with a limit of `limit` polls
 * (1 .. 2^22); every block's wait gives up and *out_error becomes VG_ERR_TIMEOUT. */
VG_API vg_status vg_debug_grid_barrier_timeout(uint32_t* scratch_words, uint32_t limit,
                                               int32_t* out_error, vg_stream_t stream);

/* Test hook: limit of every chained-scan wait in later calls (0 restores the default
 * of about a second).  A wait that reaches it records VG_ERR_TIMEOUT and returns. */
VG_API void vg_debug_set_spin_limit(uint32_t limit);

#ifdef __cplusplus
}
#endif

#endif /* VG_H_ */
