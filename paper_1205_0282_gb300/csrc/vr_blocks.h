// Brick blocks for the out-of-core paths, from a host cube or a provider callback
// (host code only: vr_ooc.cu and the host planner).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/vr.h"

namespace vr {

// Where a brick's block comes from: the caller's host cube, or a provider callback
// (vr_block_provider) that fills a box of voxels on request.
struct BlockSource {
    const float* cube = nullptr;
    vr_block_provider fn = nullptr;
    void* user = nullptr;
    int threads = 0;  // host threads (<= 0: the hardware's)
    bool valid() const { return cube || fn; }
};
// Blocks of bricks ids[i] (or i when ids is null), i < count, into store + i *
// slot_floats (zero beyond the cube), with each block's [min, max] over its voxels
// inside the cube when minmax is not null.  Returns VR_OK, or VR_ESOURCE when the
// provider reported a failure (the first failing brick in *bad_brick).
int read_blocks(const BlockSource& src, const int64_t n[3], const int32_t B[3], const int32_t nb[3],
                const int32_t* ids, int64_t count, float* store, int64_t slot_floats, float2* minmax,
                int64_t* bad_brick);

}  // namespace vr
