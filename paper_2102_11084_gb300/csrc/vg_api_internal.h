// Host-side pieces of the C ABI shared between vg_api.cu and vg_plan.cu.
#pragma once
#include "../../include/vg.h"
#include "vg_internal.h"

namespace vg {

size_t frames_workspace_bytes(int64_t n, int frames, int flags);
vg_status check_outputs(int64_t n, const float* xyz, uint64_t* out_keys, float* out_centroids,
                        uint32_t* out_counts, int64_t cap, const int64_t* num_voxels,
                        const int32_t* p2v, const int32_t* out_error, const void* workspace);
vg_status run_frames(const float* xyz, const FramesArg& fr, bool from_min, const SegOut& out,
                     int32_t* out_error, void* workspace, size_t workspace_bytes, int flags,
                     cudaStream_t stream);
// Suspends the stage-event hook (used while a CUDA graph is being captured).
void pause_stage_events(bool paused);

}  // namespace vg
