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
//   build_brick_blocks the same blocks for a list of bricks only (the plain
//                      copies a learned context keeps for its fallback bricks).
//   read_blocks        blocks of a list of bricks from the host cube or from a
//                      provider callback (cubes that exist only as a function:
//                      generated, or read from storage on request).
//   launch_brick_error per brick, the largest difference between its decoded
//                      and its plain block, both clipped from below at a floor.
//   plan_residency     assign a device slot to every brick a frame renders:
//                      resident bricks are reused and missing ones take free or
//                      least recently used slots; when the frame needs more bricks
//                      than the cache holds, the last 2H slots become a streaming
//                      ring (two halves of H, alternating), the rest stays resident
//                      across frames, and the bricks left over stream through the
//                      ring.
#include <algorithm>
#include <atomic>
#include <cfloat>
#include <climits>
#include <cstring>
#include <thread>
#include <vector>

#include "vr_blocks.h"
#include "vr_internal.cuh"

namespace vr {

namespace {

// Blocks of bricks ids[i] (or i when ids is null), i < count, into store + i *
// slot_floats, from the host cube or the provider; bricks are dealt to the threads
// one at a time (a provider's cost per brick can vary).
int build_blocks(const BlockSource& src, const int64_t n[3], const int32_t B[3], const int32_t nb[3],
                 const int32_t* ids, int64_t count, float* store, int64_t slot_floats, float2* minmax,
                 int64_t* bad_brick) {
    const int64_t sx = B[0] + 1, sy = B[1] + 1;
    std::atomic<int64_t> next{0};
    std::atomic<int64_t> bad{INT64_MAX};
    auto work = [&]() {
        for (int64_t i = next++; i < count && bad.load() == INT64_MAX; i = next++) {
            const int64_t id = ids ? ids[i] : i;
            const int64_t ix = id % nb[0], iy = (id / nb[0]) % nb[1], iz = id / ((int64_t)nb[0] * nb[1]);
            const int64_t x0 = ix * B[0], y0 = iy * B[1], z0 = iz * B[2];
            const int64_t x1 = std::min<int64_t>(x0 + B[0], n[0] - 1);
            const int64_t y1 = std::min<int64_t>(y0 + B[1], n[1] - 1);
            const int64_t z1 = std::min<int64_t>(z0 + B[2], n[2] - 1);
            float* blk = store + i * slot_floats;
            // zero the part of the block beyond the cube (all of it when clipped)
            if (x1 - x0 < B[0] || y1 - y0 < B[1] || z1 - z0 < B[2])
                std::memset(blk, 0, (size_t)slot_floats * sizeof(float));
            const int64_t len = x1 - x0 + 1;
            if (src.fn) {
                const int64_t origin[3] = {x0, y0, z0};
                const int32_t extent[3] = {(int32_t)len, (int32_t)(y1 - y0 + 1), (int32_t)(z1 - z0 + 1)};
                if (src.fn(src.user, origin, extent, blk, sx, sx * sy) != 0) {
                    int64_t cur = bad.load();
                    while (id < cur && !bad.compare_exchange_weak(cur, id)) {
                    }
                    break;
                }
            } else {
                for (int64_t z = z0; z <= z1; ++z)
                    for (int64_t y = y0; y <= y1; ++y)
                        std::memcpy(blk + ((z - z0) * sy + (y - y0)) * sx, src.cube + (z * n[1] + y) * n[0] + x0,
                                    (size_t)len * sizeof(float));
            }
            if (minmax) {
                float mn = FLT_MAX, mx = -FLT_MAX;
                for (int64_t z = 0; z <= z1 - z0; ++z)
                    for (int64_t y = 0; y <= y1 - y0; ++y) {
                        const float* row = blk + (z * sy + y) * sx;
                        for (int64_t x = 0; x < len; ++x) {
                            mn = std::min(mn, row[x]);
                            mx = std::max(mx, row[x]);
                        }
                    }
                minmax[i] = make_float2(mn, mx);
            }
        }
    };
    const int64_t hw = src.threads > 0 ? src.threads : (int64_t)std::max(1u, std::thread::hardware_concurrency());
    const int64_t threads = std::max<int64_t>(1, std::min<int64_t>(hw, count));
    if (threads == 1) {
        work();
    } else {
        std::vector<std::thread> pool;
        for (int64_t t = 0; t < threads; ++t) pool.emplace_back(work);
        for (auto& th : pool) th.join();
    }
    if (bad.load() != INT64_MAX) {
        if (bad_brick) *bad_brick = bad.load();
        return VR_ESOURCE;
    }
    return VR_OK;
}

// One block of threads per (part of a) brick: the largest clipped difference over
// the brick's voxels inside the cube, folded into err_bits (non-negative floats
// order like their bit patterns).
__global__ void brick_error_kernel(const float* __restrict__ decoded, const float* __restrict__ plain, int64_t first,
                                   int3 n, int3 B, int3 nb, float floor_v, uint32_t* err_bits) {
    const int k = blockIdx.y;
    const int64_t id = first + k;
    const int ix = (int)(id % nb.x), iy = (int)((id / nb.x) % nb.y), iz = (int)(id / ((int64_t)nb.x * nb.y));
    // extent of the brick's block inside the cube, per axis: voxels 0 .. e
    const int ex = min(B.x, n.x - 1 - ix * B.x), ey = min(B.y, n.y - 1 - iy * B.y), ez = min(B.z, n.z - 1 - iz * B.z);
    const int sx = B.x + 1, sy = B.y + 1;
    const int64_t V = (int64_t)sx * sy * (B.z + 1);
    const float* d = decoded + (int64_t)k * V;
    const float* p = plain + (int64_t)k * V;
    float m = 0.0f;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < V; q += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(q % sx), y = (int)((q / sx) % sy), z = (int)(q / ((int64_t)sx * sy));
        if (x <= ex && y <= ey && z <= ez) m = fmaxf(m, fabsf(fmaxf(d[q], floor_v) - fmaxf(p[q], floor_v)));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(err_bits + k, __float_as_uint(m));
}

}  // namespace

int read_blocks(const BlockSource& src, const int64_t n[3], const int32_t B[3], const int32_t nb[3],
                const int32_t* ids, int64_t count, float* store, int64_t slot_floats, float2* minmax,
                int64_t* bad_brick) {
    if (count <= 0) return VR_OK;
    return build_blocks(src, n, B, nb, ids, count, store, slot_floats, minmax, bad_brick);
}

void build_brick_store(const float* src, const int64_t n[3], const int32_t B[3], const int32_t nb[3],
                       float* store, int64_t slot_floats, float2* minmax) {
    BlockSource bs;
    bs.cube = src;
    build_blocks(bs, n, B, nb, nullptr, (int64_t)nb[0] * nb[1] * nb[2], store, slot_floats, minmax, nullptr);
}

void build_brick_blocks(const float* src, const int64_t n[3], const int32_t B[3], const int32_t nb[3],
                        const int32_t* ids, int64_t count, float* store, int64_t slot_floats) {
    BlockSource bs;
    bs.cube = src;
    build_blocks(bs, n, B, nb, ids, count, store, slot_floats, nullptr, nullptr);
}

cudaError_t launch_brick_error(const float* decoded, const float* plain, int64_t first, int32_t count,
                               const int64_t n[3], const int32_t B[3], const int32_t nb[3], float floor_v,
                               uint32_t* err_bits, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int64_t V = (int64_t)(B[0] + 1) * (B[1] + 1) * (B[2] + 1);
    const int per_brick = (int)std::min<int64_t>(64, (V + 255) / 256);
    brick_error_kernel<<<dim3(per_brick, count), 256, 0, s>>>(
        decoded, plain, first, make_int3((int)n[0], (int)n[1], (int)n[2]), make_int3(B[0], B[1], B[2]),
        make_int3(nb[0], nb[1], nb[2]), floor_v, err_bits);
    return cudaGetLastError();
}

int plan_residency(Residency& r, const std::vector<int32_t>& bricks, int64_t frame, int32_t first_half,
                   std::vector<int32_t>& slot, std::vector<int32_t>& upload, std::vector<int32_t>& ring) {
    const int32_t S = (int32_t)r.brick_in_slot.size();
    const int32_t P = (int32_t)bricks.size();
    slot.assign(P, -1);
    upload.clear();
    ring.clear();
    // Streaming ring for frames larger than the cache: two halves of H slots at the
    // end of the cache; the first R = S - 2H slots stay resident across frames.
    int32_t H = 0;
    if (P > S) H = std::max<int32_t>(1, std::min<int32_t>(S / 8, 32));
    const int32_t R = S - 2 * H;
    // slots no longer resident (a smaller resident part than the last frame's)
    for (int32_t s = R; s < S; ++s)
        if (r.brick_in_slot[s] >= 0) {
            r.slot_of_brick[r.brick_in_slot[s]] = -1;
            r.brick_in_slot[s] = -1;
        }
    // resident hits, then free or least recently used resident slots for the rest
    // (each brick is listed once, so the hits of different threads touch different
    // slots)
    std::vector<char> needed(R, 0);
    const int32_t hw = (int32_t)std::max(1u, std::thread::hardware_concurrency());
    const int32_t n_th = std::max(1, std::min({hw, 16, P / 16384}));
    std::vector<int32_t> miss(n_th, 0);
    auto hits = [&](int32_t t) {
        for (int32_t k = (int32_t)((int64_t)P * t / n_th); k < (int32_t)((int64_t)P * (t + 1) / n_th); ++k) {
            const int32_t s = r.slot_of_brick[bricks[k]];
            if (s >= 0) {
                slot[k] = s;
                needed[s] = 1;
                r.last_used[s] = frame;
            } else {
                ++miss[t];
            }
        }
    };
    std::vector<std::thread> pool;
    for (int32_t t = 1; t < n_th; ++t) pool.emplace_back(hits, t);
    hits(0);
    for (auto& th : pool) th.join();
    int32_t misses = 0;
    for (int32_t m : miss) misses += m;
    // the misses' slots: free ones first, then the least recently used (ties by
    // slot), found without ordering the whole cache
    std::vector<int32_t> victims;
    if (misses > 0) {
        for (int32_t s = 0; s < R; ++s)
            if (!needed[s]) victims.push_back(s);
        const size_t m = std::min<size_t>((size_t)misses, victims.size());
        std::partial_sort(victims.begin(), victims.begin() + m, victims.end(), [&](int32_t a, int32_t b) {
            const bool fa = r.brick_in_slot[a] < 0, fb = r.brick_in_slot[b] < 0;
            if (fa != fb) return fa;
            if (r.last_used[a] != r.last_used[b]) return r.last_used[a] < r.last_used[b];
            return a < b;
        });
        victims.resize(m);
    }
    size_t v = 0;
    int32_t streamed = 0;
    for (int32_t k = 0; k < P; ++k) {
        if (slot[k] >= 0) continue;
        if (v < victims.size()) {
            const int32_t s = victims[v++];
            if (r.brick_in_slot[s] >= 0) r.slot_of_brick[r.brick_in_slot[s]] = -1;
            r.brick_in_slot[s] = bricks[k];
            r.slot_of_brick[bricks[k]] = s;
            r.last_used[s] = frame;
            slot[k] = s;
            upload.push_back(k);
        } else {
            // through the ring: the j-th streamed brick goes to half (first_half + j / H) % 2
            const int32_t half = (first_half + streamed / H) % 2;
            slot[k] = R + half * H + streamed % H;
            ring.push_back(k);
            ++streamed;
        }
    }
    return H;
}

}  // namespace vr
