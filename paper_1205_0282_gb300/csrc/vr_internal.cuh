// Structures shared by the host planner (vr_host.cu) and the kernels (vr_kernels.cu).
#pragma once
#include <cstdint>
#include <vector>
#include <cuda.h>
#include <cuda_runtime.h>

#include "df.cuh"

namespace vr {

constexpr int kTile = 8;                    // tile edge of the direct-gather march (8x8 items)
constexpr int kTilePixels = kTile * kTile;  // 64 rays per item, one per thread
constexpr int kTileTma = 16;                // tile edge of the TMA-staged march (16x16 items)
constexpr int kTmaClasses = 8;              // staged-box classes of the TMA march
constexpr int kPrecF32 = 0, kPrecF16 = 1, kPrecF8 = 2;  // texture storage precisions
constexpr int kMaxTexSlabs = 16;  // texture march: slabs per layered copy at most
constexpr int kMaxTfPoints = 256;
constexpr int kAlphaPolyTerms = 11;         // coefficients of the opacity-correction polynomial
constexpr int kAlphaSmallTerms = 6;         // ... and of its short form for small opacities

// Device error flags (OR-ed into Stats::errors).
constexpr int kErrBounds = 1;               // a sample fell outside its staged box (clamped)
constexpr int kErrTimeout = 2;              // a bounded mbarrier wait gave up

// One work item: the rays of one pixel tile restricted to the samples one brick owns.
struct Item {
    int32_t brick;  // brick id = ix + nbx*(iy + nby*iz)
    int32_t tile;   // tile id = tx + tiles_x*ty
    int32_t frag;   // fragment slot: its 64 float4 sub-image pixels live at frag*64
    int32_t sweep;  // TMA march: sweep axis (0 = x, 1 = y, 2 = z) | 4 if it runs towards -axis
};

// Per-frame device counters.
struct Stats {
    unsigned long long samples;
    unsigned long long chunks_staged;  // TMA march: chunks read from shared memory
    unsigned long long chunks_direct;  // TMA march: chunks that fell back to global loads
    int errors;
    int work_next;  // texture march: next half item (32 rays) for a warp to take
};

// One frame of a batch (the serving loop): its camera, tiles and image.  The
// frames of a batch share everything else in FrameParams (cube, transfer
// function, step, termination, fragment buffer).
struct FrameCam {
    df eye[3];
    df f[3], r[3], u[3];
    const df* qx;
    const df* qy;
    int32_t width, height, tiles_x, tiles_y;
    const int32_t* tile_start;  // fragments of tile t: [tile_start[t], tile_start[t+1])
    float4* out;                // float4[height][width]
    int32_t tile_base;          // first composite block of this frame in the batch
    int32_t tf_off;             // the frame's transfer function: entries [tf_off, tf_off + tf_n]
    int32_t tf_n;               // of the batch's tables (control points, the last repeated)
    float tf_v0, tf_inv_dv;     // uniform control points: v_i = v0 + i / inv_dv
    float tau;                  // termination threshold
    int32_t tf_uniform;         // 1: look the transfer function up by its uniform spacing
};

// Everything a frame's kernels need, passed by value.
struct FrameParams {
    // camera (double-float)
    df eye[3];
    df f[3], r[3], u[3];
    const df* qx;  // per column: (2(i+.5)/W - 1) tan(fovy/2) W/H
    const df* qy;  // per row:    (1 - 2(j+.5)/H) tan(fovy/2)
    int32_t width, height, tiles_x, tiles_y;
    int32_t tile;   // tile edge in pixels (fragments hold tile*tile pixels)
    df dt;          // step (voxels)
    df inv_dt;      // 1 / dt
    int32_t step_mode;  // 0: fixed step dt; 1: dynamic (dt along the ray's dominant axis)
    float dt_f;
    float tau;      // termination opacity

    // volume
    const float* cube;
    int32_t n[3];          // nx, ny, nz
    int32_t B[3];          // brick size
    int32_t nb[3];         // bricks per axis
    int64_t stride_y, stride_z;
    int32_t offsets32;     // 1: (B+1) * stride_z < 2^32, brick-local offsets fit in uint32_t

    // transfer function: control points (r,g,b,a) and their values; tf_rgba has
    // tf_n + 1 entries, the last one repeating point tf_n - 1
    const float4* tf_rgba;
    const float* tf_v;
    int32_t tf_n;
    int32_t tf_uniform;    // 1: v_i = v0 + i*dv
    float tf_v0, tf_inv_dv;
    // opacity correction alpha(a) = 1 - (1-a)^dt as a * Q(a): Q in powers of
    // t = a * scale - 1, a short fit for a <= small_split, a long one up to alpha_split
    float alpha_small[kAlphaSmallTerms];
    float small_scale, small_split;
    float alpha_poly[kAlphaPolyTerms];
    float poly_scale;
    float alpha_split;
    int32_t mode;               // 0 = emission-absorption, 1 = MIP
    float gmax;                 // MIP: the cube's global maximum (rays stop on reaching it)

    // plan
    const Item* items;
    int32_t n_items;
    const CUtensorMap* tmaps;   // TMA march: tensor maps in device memory
    int32_t tmaps_per_brick;    // 1: one set per brick (brick-local coordinates)
    // texture march: layered copies with layers along x, y, z, each split into slabs
    // of tex_slab_bricks[S] bricks along its layer axis (slab j holds layers
    // [j K B_S, min((j + 1) K B_S, n_S - 1)], its last one the apron of the next)
    cudaTextureObject_t tex[3][kMaxTexSlabs];
    int32_t tex_slab_bricks[3];
    int32_t precision;          // texture storage: kPrecF32, kPrecF16, kPrecF8
    const float* brick_scale;   // FP8: per-brick scale (value = code * scale)
    const int32_t* tile_start;  // fragments of tile t: [tile_start[t], tile_start[t+1])
    const float* pool;          // out-of-core: device brick cache, or nullptr (read `cube`)
    // out-of-core texture march: the cache's slots as layered copies, one per sweep
    // axis S (slot k's block at texel (k % pool_cols[S], k / pool_cols[S]) x (B+1)
    // across, layers = its coordinate along S), or 0
    cudaTextureObject_t pool_tex[3];
    int32_t pool_cols[3];
    int32_t* work_next;         // texture march: the launch's half-item counter (nullptr: stats->work_next)
    const int32_t* slot_of;     // out-of-core: cache slot of each brick rendered this frame
    int64_t slot_stride;        // floats per slot, (Bx+1)(By+1)(Bz+1)
    int32_t pool_sy, pool_sz;   // row and plane strides inside a slot
    float4* frags;
    const FrameCam* cams;       // batch: per-frame cameras (items carry the frame in sweep >> 3)
    int32_t n_cams;
    float4* out;                // image window: pixel (i, j) of the frame goes to
    int32_t out_x0, out_y0;     // out[(j - out_y0) * out_w + (i - out_x0)] if it lies in
    int32_t out_w, out_h;       // [out_x0, out_x0 + out_w) x [out_y0, out_y0 + out_h)
    Stats* stats;
};

// Sub-images for the root's sort-last fold (vr_shard.cu): a rectangle
// [x0, x1] x [y0, y1] of the frame, row-major RGBA.
constexpr int kMaxSubimages = 256;
struct SubimageRef {
    const float4* data;
    int32_t x0, y0, x1, y1;
};
struct SubimageList {
    int32_t n;
    SubimageRef s[kMaxSubimages];
};

// Launchers (vr_kernels.cu).
cudaError_t launch_brick_minmax(const float* cube, int64_t pitch, const int32_t n[3], const int32_t B[3],
                                const int32_t nb[3], float2* out, cudaStream_t s);
cudaError_t launch_march(const FrameParams& p, cudaStream_t s);
cudaError_t launch_march_tma(const FrameParams& p, cudaStream_t s);
cudaError_t launch_march_tex(const FrameParams& p, cudaStream_t s);
// Out-of-core texture march: copy the blocks of the cache slots slots[0..count)
// (device list) into the layered copies of the slot pool (surfaces by sweep axis,
// null for a copy the pool does not keep; slot k at texel (k % cols[S], k / cols[S])
// x (B+1)).  staged: slot slots[i]'s block is block i of `pool` (the staging area);
// otherwise block slots[i].
cudaError_t fill_pool_tex(const float* pool, int64_t slot_floats, const int32_t* slots, int32_t count, bool staged,
                          const int32_t B[3], const cudaSurfaceObject_t surf[3], const int32_t cols[3],
                          cudaStream_t s);
// Batch (vr_serve.cu): the texture march over items of several frames, and the
// composite of every tile of every frame (p.n_cams frames, total_tiles blocks).
cudaError_t launch_march_tex_batch(const FrameParams& p, cudaStream_t s);
cudaError_t launch_composite_batch(const FrameParams& p, int32_t total_tiles, cudaStream_t s);
// Layers [l0, l0 + nl) along axis S of the cube into the layered array behind surf
// (its layer 0 = coordinate l0).
cudaError_t fill_tex_layers(const float* a, int64_t nx, int64_t ny, int64_t nz, int64_t a_pitch, int S,
                            int64_t l0, int64_t nl, int precision, cudaSurfaceObject_t surf, const float* scale,
                            const int32_t B[3], const int32_t nb[3], cudaStream_t s);
cudaError_t launch_brick_scale(const float* a, int64_t nx, int64_t ny, int64_t nz, int64_t a_pitch,
                               const int32_t B[3], const int32_t nb[3], float* scale, cudaStream_t s);
cudaError_t launch_stored_minmax(const float* a, int64_t pitch, const int32_t n[3], const int32_t B[3],
                                 const int32_t nb[3], int precision, const float* scale, float2* out,
                                 cudaStream_t s);
cudaError_t make_tma_maps(const float* a, int64_t nx, int64_t ny, int64_t nz, int64_t a_pitch,
                          const float* b, int64_t b_pitch, const int32_t B[3], const int32_t nb[3],
                          std::vector<CUtensorMap>& out, int& per_brick);
cudaError_t launch_transpose_xzy(const float* a, int64_t nx, int64_t ny, int64_t nz, int64_t a_pitch,
                                 float* b, int64_t b_pitch, cudaStream_t s);
cudaError_t launch_composite(const FrameParams& p, cudaStream_t s);

// Out-of-core residency (vr_ooc.cu).
struct Residency {
    std::vector<int32_t> slot_of_brick;  // per brick: its cache slot, -1 if not resident
    std::vector<int32_t> brick_in_slot;  // per slot: its brick, -1 if free
    std::vector<int64_t> last_used;      // per slot: last frame that rendered it
};
void build_brick_store(const float* src, const int64_t n[3], const int32_t B[3], const int32_t nb[3],
                       float* store, int64_t slot_floats, float2* minmax);
// The blocks of the listed bricks ids[0..count) only, block i at store + i * slot_floats.
void build_brick_blocks(const float* src, const int64_t n[3], const int32_t B[3], const int32_t nb[3],
                        const int32_t* ids, int64_t count, float* store, int64_t slot_floats);
// Decode error of `count` consecutive bricks first, first + 1, ...: decoded and
// plain hold their (B+1)^3 blocks back to back; err_bits[k] (zeroed by the caller)
// receives the bits of max |max(d, floor) - max(v, floor)| over brick first + k's
// voxels inside the cube.
cudaError_t launch_brick_error(const float* decoded, const float* plain, int64_t first, int32_t count,
                               const int64_t n[3], const int32_t B[3], const int32_t nb[3], float floor_v,
                               uint32_t* err_bits, cudaStream_t s);
// Slots for the frame's bricks (in render order).  upload: positions (in
// `bricks`) of bricks copied into resident slots; ring: positions of bricks that
// stream through the ring, in order, the j-th into half (first_half + j / H) % 2.
// Returns H (0 when every brick of the frame is resident).
int plan_residency(Residency& r, const std::vector<int32_t>& bricks, int64_t frame, int32_t first_half,
                   std::vector<int32_t>& slot, std::vector<int32_t>& upload, std::vector<int32_t>& ring);

// k-d distribution and the root's fold (vr_shard.cu).  ranges: parts x 6 int32
// (brick lo x, y, z then hi x, y, z, half-open), leaves in tree order.
bool kd_partition(const int64_t n[3], const int32_t B[3], int32_t parts, int32_t* ranges);
bool kd_order(const int64_t n[3], const int32_t B[3], int32_t parts, const double eye[3], int32_t* order);
cudaError_t launch_subimage_composite(const SubimageList& L, int32_t width, int32_t height, float tau,
                                      float4* out, cudaStream_t s);

}  // namespace vr
