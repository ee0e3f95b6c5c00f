// Out-of-core brick residency (host side).  The cube stays in host memory; the
// brick store holds every brick as one dense block so that a brick reaches the
// device with one contiguous copy, and the device keeps a cache of brick slots.
//
//   build_brick_store  copy the cube into the pinned store, brick b as a
//                      (Bz+1) x (By+1) x (Bx+1) block of its voxels [b*B,
//                      min((b+1)*B, n-1)] per axis (its own plus the one-voxel
//                      apron its samples read), zero beyond the cube, and the
//                      brick's [min, max] over the same voxels (Section 2.3.1's
//                      per-sub-cube range, used for empty-space skipping).
//   plan_residency     assign a device slot to every brick a frame renders:
//                      when they fit, resident bricks are reused and missing ones
//                      take free or least recently used slots; otherwise the
//                      bricks stream through two alternating halves of the cache.
#include <algorithm>
#include <cfloat>
#include <cstring>
#include <thread>
#include <vector>

#include "vr_internal.cuh"

namespace vr {

void build_brick_store(const float* src, const int64_t n[3], const int32_t B[3], const int32_t nb[3],
                       float* store, int64_t slot_floats, float2* minmax) {
    const int64_t total = (int64_t)nb[0] * nb[1] * nb[2];
    const int64_t sx = B[0] + 1, sy = B[1] + 1;
    auto work = [&](int64_t b0, int64_t b1) {
        for (int64_t id = b0; id < b1; ++id) {
            const int64_t ix = id % nb[0], iy = (id / nb[0]) % nb[1], iz = id / ((int64_t)nb[0] * nb[1]);
            const int64_t x0 = ix * B[0], y0 = iy * B[1], z0 = iz * B[2];
            const int64_t x1 = std::min<int64_t>(x0 + B[0], n[0] - 1);
            const int64_t y1 = std::min<int64_t>(y0 + B[1], n[1] - 1);
            const int64_t z1 = std::min<int64_t>(z0 + B[2], n[2] - 1);
            float* blk = store + id * slot_floats;
            std::memset(blk, 0, (size_t)slot_floats * sizeof(float));
            float mn = FLT_MAX, mx = -FLT_MAX;
            for (int64_t z = z0; z <= z1; ++z)
                for (int64_t y = y0; y <= y1; ++y) {
                    const float* row = src + (z * n[1] + y) * n[0] + x0;
                    float* dst = blk + ((z - z0) * sy + (y - y0)) * sx;
                    const int64_t len = x1 - x0 + 1;
                    std::memcpy(dst, row, (size_t)len * sizeof(float));
                    for (int64_t x = 0; x < len; ++x) {
                        mn = std::min(mn, row[x]);
                        mx = std::max(mx, row[x]);
                    }
                }
            minmax[id] = make_float2(mn, mx);
        }
    };
    const int64_t threads = std::max<int64_t>(1, std::min<int64_t>(std::thread::hardware_concurrency(), total));
    std::vector<std::thread> pool;
    for (int64_t t = 0; t < threads; ++t)
        pool.emplace_back(work, total * t / threads, total * (t + 1) / threads);
    for (auto& th : pool) th.join();
}

int plan_residency(Residency& r, const std::vector<int32_t>& bricks, int64_t frame, std::vector<int32_t>& slot,
                   std::vector<int32_t>& upload_chunks) {
    const int32_t S = (int32_t)r.brick_in_slot.size();
    const int32_t P = (int32_t)bricks.size();
    slot.assign(P, -1);
    upload_chunks.clear();
    if (P <= S) {
        // cache: mark this frame's resident bricks, then give every missing brick
        // a free slot or the least recently used slot not needed by this frame
        std::vector<char> needed(S, 0);
        for (int32_t k = 0; k < P; ++k) {
            const int32_t s = r.slot_of_brick[bricks[k]];
            if (s >= 0) {
                slot[k] = s;
                needed[s] = 1;
                r.last_used[s] = frame;
            }
        }
        std::vector<int32_t> victims;
        for (int32_t s = 0; s < S; ++s)
            if (!needed[s]) victims.push_back(s);
        // free slots first (brick -1), then oldest use
        std::sort(victims.begin(), victims.end(), [&](int32_t a, int32_t b) {
            const bool fa = r.brick_in_slot[a] < 0, fb = r.brick_in_slot[b] < 0;
            if (fa != fb) return fa;
            return r.last_used[a] < r.last_used[b];
        });
        size_t v = 0;
        for (int32_t k = 0; k < P; ++k) {
            if (slot[k] >= 0) continue;
            const int32_t s = victims[v++];
            if (r.brick_in_slot[s] >= 0) r.slot_of_brick[r.brick_in_slot[s]] = -1;
            r.brick_in_slot[s] = bricks[k];
            r.slot_of_brick[bricks[k]] = s;
            r.last_used[s] = frame;
            slot[k] = s;
            upload_chunks.push_back(k);
        }
        return 0;  // cache mode: upload_chunks lists the bricks to copy
    }
    // streaming: drop the cache; chunk c (bricks [c*H, (c+1)*H)) uses half c % 2
    std::fill(r.slot_of_brick.begin(), r.slot_of_brick.end(), -1);
    std::fill(r.brick_in_slot.begin(), r.brick_in_slot.end(), -1);
    const int32_t H = S / 2;
    for (int32_t k = 0; k < P; ++k) {
        const int32_t c = k / H;
        slot[k] = (c % 2) * H + k % H;
        upload_chunks.push_back(k);
    }
    return H;  // streaming mode: chunks of H bricks
}

}  // namespace vr
