/*
 * vr.h -- C ABI of the GB300 bricked volume ray caster.
 *
 * Renders a float32 data cube by per-pixel ray casting (tri-linear sampling,
 * a 1D transfer function with step-size opacity correction, front-to-back
 * compositing with early ray termination) and sort-last 'over' compositing of
 * per-brick sub-images in view order, after Hassan, Fluke & Barnes, "A
 * Distributed GPU-based Framework for real-time 3D Volume Rendering of Large
 * Astronomical Data Cubes" (arXiv:1205.0282):
 *   Section 2.3.1  data partitioning into sub-cubes, per-sub-cube min/max;
 *   Section 2.3.2  ray casting: rendering rectangle from the projected sub-cube
 *                  vertices, entry/exit with the bounding cube, tri-linear
 *                  sampling, termination at exit or on opacity;
 *   Section 2.3.3  composition of sub-images, associativity of alpha blending,
 *                  maximum intensity projection with a colour map.
 *
 * Conventions for every call:
 *   - Return value: VR_OK (0) or a negative VR_E* code; no exception crosses the
 *     ABI.  vr_last_error() gives a message for the last failing call on a context.
 *   - The library owns all device memory it allocates (released by vr_destroy).
 *     Callers own every buffer they pass; the library keeps no pointer to a
 *     caller buffer after a call returns, except where the call says so: an
 *     output buffer written asynchronously on the given stream (device memory,
 *     or page-locked host memory with VR_OPT_HOST_OUTPUT_ASYNC), the host cube
 *     of vr_load_cube_host, a brick provider and its user data, and a learned
 *     context's fallback cube or provider (read at the next vr_brick).
 *   - Pointers may be host or device (CUDA unified addressing decides).
 *   - Coordinates: voxel (i,j,k) of a cube float32[nz][ny][nx] (x fastest) sits
 *     at the point (i,j,k); the domain is [0,nx-1] x [0,ny-1] x [0,nz-1]; all
 *     distances are in voxel units.
 *   - A context is not thread-safe: one host thread at a time.
 */
#ifndef VR_H
#define VR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VR_OK 0
#define VR_EINVAL (-1)   /* bad argument */
#define VR_ENOMEM (-2)   /* device or pinned-host allocation failed */
#define VR_ECUDA (-3)    /* a CUDA runtime/driver call failed */
#define VR_ESTATE (-4)   /* call out of order (e.g. render before cube/brick/TF/camera) */
#define VR_ETIMEOUT (-5) /* a bounded device wait gave up; the frame is invalid */
#define VR_ESOURCE (-6)  /* a brick provider (vr_block_provider) reported a failure */

typedef struct vr_ctx vr_ctx;

/*
 * Pinhole camera (Section 2.3.2 passes the viewer's projection and view
 * transforms; this is the equivalent look-at form).  Basis f = |target-eye|,
 * r = |f x up|, u = r x f.  Pixel (i,j), row j = 0 at the top, is cast along
 * |f + qx r + qy u| with qx = (2(i+0.5)/width - 1) tan(fovy/2) width/height and
 * qy = (1 - 2(j+0.5)/height) tan(fovy/2).  Samples are taken every `step`
 * voxels from the ray's entry into the domain (or from the eye if it is
 * inside); compositing stops once the accumulated opacity reaches
 * `term_alpha` (1.0 disables early termination).
 */
typedef struct {
    double eye[3], target[3], up[3];
    double fovy_deg;      /* vertical field of view, (0, 180) */
    int32_t width, height;
    double step;          /* sample spacing in voxels, [0.01, 1000] */
    double term_alpha;    /* early-termination opacity, (0, 1] */
} vr_camera;

/* Render statistics (cumulative since vr_create or the last vr_reset_stats). */
typedef struct {
    int64_t frames;          /* completed vr_render calls */
    int64_t samples;         /* samples composited (after termination, excluding skipped bricks) */
    int64_t items;           /* (brick, pixel tile) work items launched */
    int64_t fragments;       /* per-brick sub-image pixels written (items x tile pixels) */
    int64_t bricks_rendered; /* bricks with at least one work item, summed over frames */
    int64_t bricks_skipped;  /* bricks dropped because the TF opacity is zero on [min,max] */
    int64_t touched_bytes;   /* sum over rendered bricks of their voxel bytes (no apron) */
    double march_ms;         /* device time of the ray-march kernel (CUDA events) */
    double composite_ms;     /* device time of the sort-last compositing kernel */
    double frame_ms;         /* device time from plan upload to image written */
    double plan_ms;          /* host time of the per-frame planner */
    int64_t h2d_bytes;       /* host->device bytes copied by vr_render (plans, camera, TF) */
    int64_t d2h_bytes;       /* device->host bytes copied by vr_render (counters, host images) */
    int64_t launches;        /* kernels launched by vr_render */
    int64_t chunks_staged;   /* TMA march: sample chunks read from TMA-staged shared memory */
    int64_t chunks_direct;   /* TMA march: chunks whose footprint did not fit the staged box
                                (read through L1 instead) */
    int64_t bricks_uploaded; /* out-of-core: bricks copied host->device (their bytes are in
                                h2d_bytes) */
    int64_t bricks_cached;   /* out-of-core: rendered bricks found resident in the device cache */
    int32_t device_errors;   /* OR of device-side error flags seen (0 = none; 1 = a sample
                                outside its staged box was clamped; 2 = a bounded wait on a
                                TMA copy gave up and the frame is invalid) */
    int32_t reserved;
} vr_stats;

/* Options for vr_set_option. */
#define VR_OPT_SKIP_EMPTY 1  /* 1 (default): drop bricks whose TF opacity is 0 on [min,max] */
#define VR_OPT_RECT_CULL 2   /* 1 (default): items only for tiles inside a brick's rendering
                                rectangle (Section 2.3.2) that its silhouette reaches (see
                                vr_plan_brick_tiles); 0: every tile for every brick */
#define VR_OPT_MODE 3        /* 0 (default): emission-absorption compositing;
                                1: maximum intensity projection + colour map (Section 2.3.3) */
#define VR_OPT_KERNEL 4      /* ray-march kernel for emission-absorption frames:
                                VR_KERNEL_AUTO (default): VR_KERNEL_TEX when the cube fits the
                                device's layered-texture limits, else VR_KERNEL_TMA;
                                VR_KERNEL_TEX: 8x8-pixel items, corners gathered unfiltered
                                (tld4) from three layered-texture copies of the cube (three
                                times the cube's size in extra device memory);
                                VR_KERNEL_TMA: 16x16-pixel items, voxel boxes staged in shared
                                memory by TMA (one transposed copy extra); VR_KERNEL_DIRECT:
                                8x8-pixel items, corners read through the L1 cache.  MIP frames
                                use the texture march under VR_KERNEL_AUTO (cube within the
                                limits) or VR_KERNEL_TEX with FP32 storage, else the direct
                                kernel.  All give the same image up to FP32 rounding. */
#define VR_KERNEL_TMA 0
#define VR_KERNEL_DIRECT 1
#define VR_KERNEL_TEX 2
#define VR_KERNEL_AUTO 3
#define VR_OPT_PRECISION 5   /* storage of the texture march's copies of the cube (no
                                counterpart in the paper, which samples FP32 sub-cubes):
                                VR_PRECISION_F32 (default): the values as loaded;
                                VR_PRECISION_F16: each value rounded to the nearest FP16
                                (VR_EINVAL at render time if |value| > 65504);
                                VR_PRECISION_F8: each value v of a voxel owned by brick b
                                (voxel g lies in brick min(g / B, nb - 1) along each axis)
                                stored as the E4M3 code nearest to v / s_b, saturated at
                                448, with s_b = max|v| over the voxels b owns / 448 (1 for
                                an all-zero brick); it reads back as code * s_b.
                                Interpolation, transfer function and compositing stay in
                                FP32; the image is the FP32 render of the cube of
                                read-back values (up to FP32 rounding order: F8
                                interpolates code values and applies the brick's scale
                                once per sample), and empty-space skipping uses the
                                read-back values' per-brick range.  F16 and F8 need the
                                texture march (VR_OPT_MODE 0 and VR_KERNEL_TEX, or
                                VR_KERNEL_AUTO on a cube within the texture limits):
                                vr_render returns VR_EINVAL otherwise.  Changing it waits
                                for frames in flight and rebuilds the copies on the next
                                render (F8 also after vr_brick). */
#define VR_OPT_DEVICE_BUDGET 6 /* out-of-core contexts (vr_load_cube_host): bytes of device
                                memory for the brick cache, a brick's block being
                                (bx+1)(by+1)(bz+1) floats: with the direct march one block
                                per slot; with the texture march (VR_OPT_OOC_MARCH) one
                                block's bytes per layered copy of a slot, plus a staging
                                area of max(min(64 MiB of blocks, S0/8), H0) blocks (S0:
                                the slots the budget holds without it, H0 its ring half)
                                through which the blocks are copied or decoded.  Default
                                (and any value <= 0): room for every brick.  A frame whose rendered bricks fit
                                keeps bricks resident across frames (least recently used
                                evicted); in a larger frame the last 2H slots (H = S/8
                                clamped to [1, 32], S slots) form a ring of two halves that
                                the bricks not resident stream through, each half refilled
                                once its previous bricks are marched, while the other
                                S - 2H slots stay resident.  Needs room for 2 bricks.
                                Takes effect at the next vr_brick. */
#define VR_OPT_STEP_MODE 7   /* 0 (default): samples every cam.step voxels along each ray;
                                1: dynamic step (Section 2.3.2: discrete ray casting, at
                                least one sample per voxel crossed along the ray's
                                dominant axis): a ray with unit direction d samples every
                                cam.step / max_a |d_a| voxels, i.e. every cam.step voxels
                                along its dominant axis, the opacity correction using that
                                spacing; the first sample sits half a step after the
                                ray's entry (a ray crossing whole voxel slabs samples their
                                middles, never their faces).
                                Rendered by the texture or the direct march (VR_KERNEL_TMA
                                with it: VR_EINVAL at render time). */
#define VR_OPT_TEX_SLAB_LAYERS 8 /* texture march: the layered copies are split along their
                                layer axis into slabs of whole bricks plus one apron layer,
                                each a layered texture of at most this many layers (0,
                                default: the device's layer limit, 2048 on this GPU), so
                                that cubes longer than that limit along any axis keep the
                                texture march (memory permitting; up to 16 slabs per axis).
                                Values below B + 1 make the texture march unavailable
                                (VR_KERNEL_AUTO then picks VR_KERNEL_TMA).  Changing it drops
                                the current copies (rebuilt at the next render). */
#define VR_OPT_OOC_MARCH 9     /* out-of-core and learned contexts: 1: the texture march
                                (VR_KERNEL_TEX's gathers) on three layered copies of the
                                device cache's slots, one per sweep axis, filled from each
                                brick's block after it is copied or decoded into the
                                staging area; each slot takes three times its block's
                                bytes of VR_OPT_DEVICE_BUDGET.  If the device's
                                layered-texture limits cannot tile the slots, the direct
                                march is used.  3: the same march on one layered copy,
                                layers along z (every ray sweeps along z, about 17% slower
                                than with the ray's dominant axis), each slot taking its
                                block's bytes.  4: two layered copies, layers along x and
                                along z (each ray sweeps along the larger of |d_x|, |d_z|:
                                for camera paths about the y axis, the paper's orbit, as
                                fast as three copies), each slot taking twice its block's
                                bytes.  0: the direct march on blocks kept in the
                                slots (a block per slot).  2 (default): 1 when every brick
                                fits the budget with three copies, else 4 when every brick
                                fits it with two, else 3 when every brick fits it with one,
                                else 0 (a cache that streams is bound by its uploads, which
                                the direct march does not follow with fills).  Takes effect
                                at the next vr_brick. */
#define VR_OPT_PROVIDER_THREADS 10 /* host threads that call a brick provider (and copy a
                                host cube into the brick store) at once; <= 0 (default):
                                the machine's hardware threads. */
#define VR_OPT_HOST_OUTPUT_ASYNC 11 /* 0 (default): vr_render into host memory returns with
                                the image there.  1: a page-locked host buffer (cudaHostAlloc
                                or cudaHostRegister) is filled by a copy enqueued on the
                                call's stream after the frame's kernels, and the call returns
                                without waiting, so that the host plans the next frame while
                                this one renders; the image is there once the stream has
                                reached that point (synchronise it or wait on an event
                                recorded after the call).  Pageable host memory is then
                                refused (VR_EINVAL). */
#define VR_PRECISION_F32 0
#define VR_PRECISION_F16 1
#define VR_PRECISION_F8 2

/*
 * Create a context on CUDA device `device`.  *out receives the context.
 * Errors: VR_EINVAL (null out, bad device), VR_ECUDA.
 */
int vr_create(vr_ctx** out, int32_t device);

/* Destroy a context and free everything it owns; NULL is ignored.  Waits for
 * the context's outstanding work first. */
void vr_destroy(vr_ctx* ctx);

/*
 * Load the data cube (Section 2.3.1: the cube is moved into GPU memory).
 * data: float32[nz][ny][nx], x fastest, host or device; the library copies it
 * into memory it owns (the caller keeps ownership of `data`).  2 <= nx, ny, nz <= 65536.
 * Invalidates any previous bricking.  Synchronous.
 * Errors: VR_EINVAL, VR_ENOMEM, VR_ECUDA.
 */
int vr_load_cube(vr_ctx* ctx, const float* data, int64_t nx, int64_t ny, int64_t nz);

/*
 * Out-of-core load (no counterpart in the paper, which keeps the cube in GPU
 * memory): the cube stays in host memory.  data: host memory, float32[nz][ny][nx];
 * the context reads it at every vr_brick, so it must stay valid and unchanged
 * until the context is destroyed or another cube is loaded.  vr_brick then copies
 * it brick by brick into a pinned host brick store (brick b as a dense
 * (bx+1)(by+1)(bz+1) block holding its voxels and apron, zero beyond the cube)
 * and computes the brick ranges on the host; vr_render copies the bricks a frame
 * needs into a device cache (VR_OPT_DEVICE_BUDGET) with cudaMemcpyAsync on a side
 * stream, overlapped with the ray march of bricks already resident, and marches
 * them with the texture march on layered copies of the cache's slots
 * (VR_OPT_OOC_MARCH).  Images are those of vr_load_cube with the same data (up
 * to FP32 rounding between march kernels).
 * Errors: VR_EINVAL (bad sizes, device memory), VR_ECUDA.
 */
int vr_load_cube_host(vr_ctx* ctx, const float* data, int64_t nx, int64_t ny, int64_t nz);

/*
 * A brick provider: fills one box of the cube on request, for cubes that exist only
 * as a function (read from storage, received, or generated).  The paper's render
 * nodes likewise load their sub-cubes from a file server on request (Sections 2.2
 * and 2.3.1).  Voxel (origin[0] + i, origin[1] + j, origin[2] + k), i < extent[0],
 * j < extent[1], k < extent[2], goes to dst[k * slice_stride + j * row_stride + i]
 * (strides in floats, row_stride >= extent[0], slice_stride >= row_stride *
 * extent[1]); the box always lies inside the cube and dst is host memory the
 * library owns.  Returns 0 on success, anything else on failure.  The library
 * calls it from up to VR_OPT_PROVIDER_THREADS host threads at once, so it must be
 * thread-safe, and it must return the same values for a voxel every time.
 */
typedef int (*vr_block_provider)(void* user, const int64_t origin[3], const int32_t extent[3], float* dst,
                                 int64_t row_stride, int64_t slice_stride);

/*
 * Out-of-core load from a provider (no counterpart in the paper): like
 * vr_load_cube_host, but no host copy of the cube or of its bricks is kept.
 * vr_brick calls the provider once for every brick's block (its voxels plus the
 * one-voxel apron, clipped to the cube) to compute the bricks' ranges; vr_render
 * calls it for every brick the frame needs that is not in the device cache
 * (VR_OPT_DEVICE_BUDGET), into pinned staging buffers the library owns, copies the
 * blocks into their cache slots with cudaMemcpyAsync on a side stream, and marches
 * them as vr_load_cube_host does, while the bricks already resident march.  fn and
 * user must stay valid until the context is destroyed or another cube is loaded.
 * Images are those of vr_load_cube_host with the same values, bit for bit.
 * Errors: VR_EINVAL (null fn, bad sizes), VR_ECUDA; a failing provider makes
 * vr_brick or vr_render return VR_ESOURCE (vr_last_error names the brick; a frame
 * that fails leaves the cache's failed slots empty and can be rendered again).
 */
int vr_load_cube_provider(vr_ctx* ctx, vr_block_provider fn, void* user, int64_t nx, int64_t ny, int64_t nz);

/*
 * Partition the loaded cube into bricks of bx x by x bz voxels (Section 2.3.1;
 * the unit of sort-last compositing) and compute each brick's [min, max] over
 * the voxels its samples can touch: along each axis brick b covers voxels
 * [b*B, min((b+1)*B, n-1)] (its own plus a one-voxel apron on the high side).
 * Bricks per axis: ceil((n-1)/B).  Sample p belongs to brick floor(p/B) per
 * axis, the last brick being closed.  1 <= B <= 4096.  Synchronous.
 * Errors: VR_EINVAL, VR_ESTATE (no cube), VR_ENOMEM, VR_ECUDA.
 */
int vr_brick(vr_ctx* ctx, int32_t bx, int32_t by, int32_t bz);

/*
 * Set the transfer function (Section 1.2): n >= 2 control points given as
 * rows of 5 doubles (v, r, g, b, a), host memory, v strictly increasing,
 * r, g, b, a in [0, 1]; a is the opacity per unit voxel of path.  Values
 * between points are interpolated linearly, values outside take the end
 * points.  Per sample alpha = 1 - (1 - a)^(step / 1 voxel).  n <= 256.
 * The rows are doubles (the camera is given in doubles too): the kernels use
 * each value rounded to FP32, the difference lying far below the image
 * tolerance.  Host-side only: takes effect for the next vr_render.
 * Errors: VR_EINVAL.
 */
int vr_set_transfer_function(vr_ctx* ctx, const double* points, int32_t n);

/* Set the camera (Section 2.3.2: the viewer's projection and view transforms
 * fix every pixel's ray; see vr_camera for the equivalent look-at form).
 * width, height in [1, 16384].  Host-side only: takes effect for the next
 * vr_render, frames already enqueued are not affected.
 * Errors: VR_EINVAL (degenerate basis, bad sizes). */
int vr_set_camera(vr_ctx* ctx, const vr_camera* cam);

/*
 * The camera from the viewer's OpenGL matrices (Section 2.3.2: the viewer sends
 * its projection and transformation matrices and the rendering threads project
 * with them).  view: the modelview matrix (world -> eye, a rotation and a
 * translation), proj: a symmetric perspective projection, both 16 doubles in
 * OpenGL's column-major order (element (row r, column c) at [4 c + r]).  The eye
 * is -R^T t, the viewing direction minus the third row of R, up its second row;
 * fovy = 2 atan(1 / proj[5]).  The aspect proj[5] / proj[0] must equal width /
 * height (square pixels) within 1e-6, R must be orthonormal within 1e-6, and
 * the projection must have no skew or off-centre terms (proj[4], proj[8],
 * proj[9] zero, proj[11] = -1, proj[15] = 0).  width, height, step and
 * term_alpha as in vr_camera.  vr_camera_from_matrices only fills *out (host
 * code, no context); vr_set_camera_matrices then sets it as vr_set_camera does.
 * Errors: VR_EINVAL.
 */
int vr_camera_from_matrices(const double view[16], const double proj[16], int32_t width, int32_t height,
                            double step, double term_alpha, vr_camera* out);
int vr_set_camera_matrices(vr_ctx* ctx, const double view[16], const double proj[16], int32_t width,
                           int32_t height, double step, double term_alpha);

/* Set an option (VR_OPT_*).  Errors: VR_EINVAL. */
int vr_set_option(vr_ctx* ctx, int32_t option, int64_t value);

/*
 * Render one frame (Section 2.3.2, ray casting: for every brick that is not
 * empty for the transfer function, the pixels of its rendering rectangle cast
 * rays through it, sampling tri-linearly from the ray's entry into the cube and
 * stopping at the brick's exit or once the opacity reaches term_alpha;
 * Section 2.3.3, composition: the per-brick sub-images are folded front to back
 * with the associative 'over' operator, stopping once a pixel's opacity reaches
 * term_alpha) into out_rgba: float32[height][width][4], premultiplied
 * (r, g, b, alpha), row 0 at the top, no background.  out_rgba may be device
 * memory (written asynchronously on `cuda_stream`, a cudaStream_t or NULL for
 * the legacy default stream) or host memory (the call then copies the image
 * back and synchronises the stream, or only enqueues the copy with
 * VR_OPT_HOST_OUTPUT_ASYNC).  Stream-ordered: the call returns after enqueueing
 * work unless out_rgba is host memory and VR_OPT_HOST_OUTPUT_ASYNC is 0.  Calls on different streams
 * with one context must not overlap in time on the device.
 * Errors: VR_ESTATE (missing cube/brick/TF/camera), VR_EINVAL, VR_ENOMEM,
 * VR_ECUDA.
 */
int vr_render(vr_ctx* ctx, float* out_rgba, void* cuda_stream);

/* Copy the statistics out (waits for the context's outstanding frames).
 * Errors: VR_EINVAL, VR_ECUDA. */
int vr_get_stats(vr_ctx* ctx, vr_stats* out);

/* Zero the statistics (waits for outstanding frames).  Errors: VR_EINVAL, VR_ECUDA. */
int vr_reset_stats(vr_ctx* ctx);

/* Copy the per-brick [min, max] pairs (float32, n_bricks x 2, host memory,
 * brick id = ix + nbx*(iy + nby*iz)) computed by vr_brick.
 * Errors: VR_EINVAL (n_bricks mismatch), VR_ESTATE (no bricking), VR_ECUDA. */
int vr_get_brick_minmax(vr_ctx* ctx, float* out, int64_t n_bricks);

/*
 * Host-only planner query, no device needed: the rendering rectangle of every
 * brick (Section 2.3.2: the bounding rectangle of the brick's projected
 * vertices, clipped to the image).  rects: int32[n_bricks][4] receiving
 * (x0, y0, x1, y1) inclusive pixel bounds, or (0, 0, -1, -1) when the brick is
 * off screen.  n_bricks must equal the brick count for the given sizes.
 * Errors: VR_EINVAL.
 */
int vr_plan_brick_rects(const vr_camera* cam, int64_t nx, int64_t ny, int64_t nz,
                        int32_t bx, int32_t by, int32_t bz, int32_t* rects, int64_t n_bricks);

/* Host-only, like vr_plan_brick_rects: the (brick, 8x8 tile) work items the
 * planner emits for every brick (no empty-space skipping), as mask[brick *
 * n_tiles + tile] = 1 (tiles row-major, ceil(width / 8) per row).  A brick's
 * items are the tiles of its rendering rectangle that its silhouette reaches:
 * with all eight box corners in front of the eye, the convex hull of their
 * projections widened by one pixel; otherwise the whole rectangle.
 * Errors: VR_EINVAL. */
int vr_plan_brick_tiles(const vr_camera* cam, int64_t nx, int64_t ny, int64_t nz, int32_t bx, int32_t by,
                        int32_t bz, uint8_t* mask, int64_t n_bricks, int64_t n_tiles);

/* ---------------------------------------------------------------------------
 * Sort-last distribution over ranks (Sections 2.3.1, 2.3.3, 2.3.4).  Each rank
 * renders the bricks of its k-d leaf into a sub-image clipped to the leaf's
 * rendering rectangle; the root folds the sub-images front to back with 'over'.
 * A ray meets each leaf in one contiguous run (leaves are boxes), so with
 * term_alpha = 1 the fold equals the single-context render; with term_alpha < 1
 * each leaf stops at term_alpha on its own and the root stops once a pixel
 * reaches it, as bricks do within one context.
 * ------------------------------------------------------------------------- */

/*
 * Host-only, no device needed.  k-d partition of the brick grid of an nx x ny x nz
 * cube with brick size B into n_parts boxes of bricks of near-equal volume
 * (Section 2.3.1): each tree node cuts its longest axis (voxel extent; ties go to
 * the lower axis; an axis of one brick is not cut), the low side taking
 * floor(parts/2) of the node's parts and round(bricks * floor(parts/2) / parts)
 * of its bricks along that axis (at least one brick a side).
 *   ranges: int32[n_parts][6] receiving brick (lo x, y, z, hi x, y, z), hi
 *           exclusive, leaves numbered depth first, low side first.
 * Errors: VR_EINVAL (bad sizes, n_parts < 1 or more parts than bricks, or a node
 * that cannot be cut).
 */
int vr_kd_partition(int64_t nx, int64_t ny, int64_t nz, const int32_t B[3], int32_t n_parts,
                    int32_t* ranges);

/*
 * Host-only.  Front-to-back visibility order of the leaves of vr_kd_partition
 * (same arguments) from eye (voxel coordinates): the tree is walked with the
 * eye's side of each cut first (a cut at brick index k along axis a is the plane
 * a = k * B[a]; an eye on the plane counts as the high side).
 *   order: int32[n_parts] receiving leaf numbers, nearest first.
 * Errors: VR_EINVAL.
 */
int vr_kd_order(int64_t nx, int64_t ny, int64_t nz, const int32_t B[3], int32_t n_parts,
                const double eye[3], int32_t* order);

/*
 * Restrict this context's renders to the bricks [lo, hi) (brick indices per axis,
 * 0 <= lo < hi <= bricks along the axis).  vr_brick resets it to all bricks.
 * Errors: VR_EINVAL, VR_ESTATE (no bricking).
 */
int vr_set_region(vr_ctx* ctx, const int32_t lo[3], const int32_t hi[3]);

/*
 * Rendering rectangle of the current region for the current camera (Section
 * 2.3.2), int32[4] = (x0, y0, x1, y1) inclusive, or (0, 0, -1, -1) when no pixel
 * sees it.  Host-only computation.  Errors: VR_EINVAL, VR_ESTATE.
 */
int vr_region_rect(vr_ctx* ctx, int32_t rect[4]);

/* Host-only: the same rectangle for the brick range [lo, hi) of a cube of the
 * given sizes and brick size B, without a context.  Errors: VR_EINVAL. */
int vr_plan_region_rect(const vr_camera* cam, int64_t nx, int64_t ny, int64_t nz, const int32_t B[3],
                        const int32_t lo[3], const int32_t hi[3], int32_t rect[4]);

/*
 * vr_render restricted to the pixel rectangle rect = (x0, y0, x1, y1) inclusive
 * (within the image): only those pixels are computed, and out_rgba receives them
 * as float32[y1-y0+1][x1-x0+1][4] (device memory written on the stream, or host
 * memory filled before return, as for vr_render).  An empty rect (x1 < x0 or
 * y1 < y0) renders nothing and returns VR_OK.  The pixels equal those of
 * vr_render.  Errors: as vr_render, VR_EINVAL (rect outside the image).
 */
int vr_render_rect(vr_ctx* ctx, const int32_t rect[4], float* out_rgba, void* cuda_stream);

/*
 * Root fold (Sections 2.3.3-2.3.4): out_rgba (float32[H][W][4] of the context's
 * camera; device memory written on the stream, or host memory filled before
 * return) receives, per pixel, the front-to-back 'over' fold of the sub-images
 * whose rectangle holds it, in the order given, stopping once the pixel's alpha
 * reaches term_alpha; pixels no sub-image covers are 0.
 *   images: n device pointers, sub-image k = float32[rows][cols][4] of rects[k];
 *   rects:  int32[n][4] (x0, y0, x1, y1) inclusive, within the image; an empty
 *           rect (x1 < x0 or y1 < y0) is skipped and its pointer may be NULL.
 *   n:      0 <= n <= 256.
 * The sub-images must be complete on the device before the fold's stream reaches
 * it (the caller orders streams).  Errors: VR_EINVAL, VR_ESTATE (no camera),
 * VR_ENOMEM, VR_ECUDA.
 */
int vr_composite_subimages(vr_ctx* ctx, int32_t n, const float* const* images, const int32_t* rects,
                           float* out_rgba, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Serving loop (no counterpart in the paper): requests for frames arrive at any
 * time and are rendered in batches, each batch one texture-march launch over the
 * tiles of all its frames and one composite launch.
 * ------------------------------------------------------------------------- */
typedef struct vr_server vr_server;

typedef struct {
    int64_t submitted;       /* requests accepted by vr_server_submit */
    int64_t completed;       /* requests rendered */
    int64_t failed;          /* requests that could not be rendered (their wait returns the error) */
    int64_t batches;         /* batches launched */
    int64_t batched_frames;  /* frames in those batches (mean batch size = batched_frames / batches) */
    int64_t samples;         /* samples composited by completed batches */
    int64_t items;           /* (brick, tile) items marched by completed batches */
} vr_server_stats;

/*
 * Start a serving loop on ctx, which must hold a loaded, bricked cube, a transfer
 * function and a camera, in emission-absorption mode with the texture march
 * (VR_KERNEL_TEX or VR_KERNEL_AUTO on a cube within the texture limits; any
 * VR_OPT_PRECISION).  The loop owns ctx until vr_server_destroy: no other call
 * may use ctx meanwhile.  It allocates arena_bytes of device memory (>= 64 MiB)
 * in two halves, one per batch in flight, and pinned staging of the same size.
 * A worker thread admits queued requests in arrival order into a batch while
 * they share the step, number at most max_batch, their transfer functions fit
 * the batch's tables (512 control points in all) and their work lists and
 * fragments fit one half; frames of one batch may differ in transfer function
 * and term_alpha, each rendered as vr_render renders it.  It plans the next
 * batch while the GPU renders the current one.  A completion thread marks
 * requests done when their batch's event fires.
 * Errors: VR_EINVAL, VR_ESTATE, VR_ENOMEM, VR_ECUDA.
 */
int vr_server_create(vr_ctx* ctx, int64_t arena_bytes, int32_t max_batch, vr_server** out);

/*
 * Queue a frame.  cam: its camera (any resolution, step, term_alpha);
 * tf_points: NULL for the transfer function in force, else n_tf rows (v, r, g, b,
 * a) that take effect from this request on; out_rgba: device memory,
 * float32[height][width][4], written when the request completes (keep it
 * allocated until vr_server_wait returns).  *ticket identifies the request.
 * Errors: VR_EINVAL, VR_ESTATE (the loop has stopped after a CUDA error).
 */
int vr_server_submit(vr_server* srv, const vr_camera* cam, const double* tf_points, int32_t n_tf,
                     float* out_rgba, int64_t* ticket);

/*
 * Wait for a request: at most timeout_s seconds (< 0: no limit; VR_ETIMEOUT when
 * it runs out, the ticket staying valid).  On return the ticket is released and
 * *latency_ms (nullable) holds the time from submission to completion.  Returns
 * the request's status: VR_OK, VR_ENOMEM (its frame does not fit half the arena),
 * VR_EINVAL, VR_ECUDA.
 */
int vr_server_wait(vr_server* srv, int64_t ticket, double timeout_s, double* latency_ms);

/* Counters since vr_server_create.  Errors: VR_EINVAL. */
int vr_server_get_stats(vr_server* srv, vr_server_stats* out);

/* Finish every queued request, stop the threads and free the loop; NULL is ignored. */
void vr_server_destroy(vr_server* srv);

/*
 * Diagnostic of the tensor-core path used by the learned brick codec (no
 * counterpart in the paper): D = A * B^T on one CTA with tcgen05.mma (BF16
 * operands staged in shared memory K-major, or MN-major when *_mn_major is 1;
 * FP32 accumulation in tensor memory; read back with tcgen05.ld).
 *   a_bf16: host, 128 x K BF16 bit patterns, row-major; b_bf16: host, N x K;
 *   16 <= K <= 64 and 16 <= N <= 64, multiples of 16; d_out: host, 128 x N FP32.
 * Runs on the current CUDA device.  Errors: VR_EINVAL, VR_ENOMEM, VR_ECUDA,
 * VR_ETIMEOUT (the kernel's bounded wait for the MMA gave up).
 */
int vr_codec_gemm_check(const uint16_t* a_bf16, const uint16_t* b_bf16, int32_t K, int32_t N,
                        int32_t a_mn_major, int32_t b_mn_major, float* d_out);

/* ---------------------------------------------------------------------------
 * Learned brick codec (no counterpart in the paper): brick b is stored as a
 * latent grid of 8 x 8 x 8 nodes x 16 channels and decoded by an MLP shared by
 * all bricks.  The value at local voxel position u in [0, B]^3 is
 *   x = u / B;  z = trilinear interpolation of the latents at 7 x;
 *   in = [z (16), sin(pi x_a), cos(pi x_a), sin(2 pi x_a), cos(2 pi x_a) for
 *         a = x, y, z (12), 0 (4)];
 *   h1 = silu(W1 in + b1) (64);  h2 = silu(W2 h1 + b2) (64);
 *   v = (w3 . h2 + b3) s_b + m_b,   silu(t) = t / (1 + exp(-t)).
 * The MLP runs on the tensor cores (tcgen05.mma, BF16 operands: in, W1, W2,
 * h1, w3 rounded to BF16; FP32 accumulation in tensor memory; biases FP32), 128
 * points per CTA tile; training runs forward and backward in one kernel (the
 * weight gradients accumulate in tensor memory across a CTA's tiles) and Adam.
 *
 * Parameter vector (FP32, vr_codec_param_count entries): W1 [64][32] (columns
 * 28..31 unused), b1 [64], W2 [64][64], b2 [64], w3 [64], b3 [1], then the
 * latents [brick][z][y][x][16].  m and s: per-brick offset and scale.
 * Every call runs on the CUDA device current at vr_codec_create and blocks until
 * done, except vr_codec_decode_bricks (asynchronous on its stream).
 * ------------------------------------------------------------------------- */
typedef struct vr_codec vr_codec;

/* A codec for n_bricks bricks of size B (parameters zero).  Errors: VR_EINVAL, VR_ENOMEM. */
int vr_codec_create(int32_t n_bricks, const int32_t B[3], vr_codec** out);
void vr_codec_destroy(vr_codec* codec);
int64_t vr_codec_param_count(const vr_codec* codec);

/* Host copies of the parameters (set also resets the optimiser).  Errors: VR_EINVAL, VR_ECUDA. */
int vr_codec_set_params(vr_codec* codec, const float* theta, const float* m, const float* s);
int vr_codec_get_params(vr_codec* codec, float* theta, float* m, float* s);

/* Decoded values of n points (host float32[n][4]: u_x, u_y, u_z, brick index as
 * the bit pattern of an int32) into host values[n].  Errors: VR_EINVAL, VR_ENOMEM,
 * VR_ECUDA, VR_ETIMEOUT (a bounded wait for the tensor cores gave up). */
int vr_codec_forward(vr_codec* codec, const float* points, int64_t n, float* values);

/* Loss mean((v - target)^2) over n points and its gradient (host float32 in the
 * parameter layout; zero for latents no point touches).  Errors: as forward. */
int vr_codec_gradient(vr_codec* codec, const float* points, const float* targets, int64_t n, float* grad,
                      double* loss);

/* Fit the codec's per-brick data to a device cube float32[nz][ny][nx] bricked by
 * B: m_b, s_b = mean and standard deviation (>= 1e-3) of max(value, floor_v) over
 * each brick's voxels and apron, and the brick's [min, max] of the values (for
 * empty-space skipping when rendering the codec).  floor_v: training targets are
 * max(value, floor_v) (-FLT_MAX: the values themselves); choose a value below
 * which the transfer function is transparent, so that the codec spends nothing
 * on invisible noise.  Errors: VR_EINVAL, VR_ECUDA. */
int vr_codec_fit_stats(vr_codec* codec, const float* cube, int64_t nx, int64_t ny, int64_t nz, float floor_v);

/* The per-brick [min, max] recorded by vr_codec_fit_stats (host float32[n][2]). */
int vr_codec_get_minmax(vr_codec* codec, float* out);
int32_t vr_codec_brick_count(const vr_codec* codec);
void vr_codec_brick_size(const vr_codec* codec, int32_t B[3]);

/* `steps` Adam steps (lr; betas 0.9, 0.999; eps 1e-8) on `batch` voxels drawn per
 * step from the device cube (counter-based generator seeded by seed): with
 * probability active_frac a voxel above floor_v (listed by vr_codec_fit_stats,
 * cubes of up to 2^32 voxels) in the brick that owns it, otherwise a uniform
 * brick among those holding values above floor_v (all bricks when the floor is
 * -FLT_MAX; the others render empty) and a uniform voxel of its block clipped to
 * the cube; targets
 * max(value, floor_v); *last_loss = the last step's loss.  Errors: as forward. */
int vr_codec_train(vr_codec* codec, const float* cube, int64_t nx, int64_t ny, int64_t nz, int32_t steps,
                   int32_t batch, float lr, float active_frac, uint64_t seed, double* last_loss);

/* The same two steps for a cube that does not fit the device, one slab of brick
 * layers at a time.  slab: device float32[z1 - z0 + 1][ny][nx], the planes z0 =
 * bz0 * bz .. z1 = min(bz1 * bz, nz - 1) of the (nx, ny, nz) cube (bz the codec's
 * brick depth), holding the bricks whose z index lies in [bz0, bz1) with their
 * aprons (brick ids bz0 * nbx * nby .. bz1 * nbx * nby - 1, x fastest).
 * vr_codec_fit_stats_slab fits those bricks' offset, scale and range as
 * vr_codec_fit_stats does.  vr_codec_train_slab takes `steps` Adam steps on
 * `batch` voxels drawn from the slab's bricks above the floor (uniform brick, then
 * uniform voxel of its block; all bricks when the floor is -FLT_MAX; no step when
 * none is above it): the shared network at rate mlp_lr (0: kept as it is, e.g.
 * to fit latents to a trained decoder), the slab's latents at rate lr; other
 * bricks' latents, gradients and moments are not touched.  A slab's latents count
 * their own Adam steps (bias correction), the network its own.  Training over all
 * layers at once with mlp_lr = lr is vr_codec_train with active_frac 0.
 * Errors: VR_EINVAL (sizes, layers), VR_ENOMEM, VR_ECUDA, VR_ETIMEOUT. */
int vr_codec_fit_stats_slab(vr_codec* codec, const float* slab, int64_t nx, int64_t ny, int64_t nz, int32_t bz0,
                            int32_t bz1, float floor_v);
int vr_codec_train_slab(vr_codec* codec, const float* slab, int64_t nx, int64_t ny, int64_t nz, int32_t bz0,
                        int32_t bz1, int32_t steps, int32_t batch, float lr, float mlp_lr, uint64_t seed,
                        double* last_loss);

/* Decode the blocks of n bricks (device list of valid brick indices) into device
 * memory: brick k's V = (bx+1)(by+1)(bz+1) values (x fastest) go to out + k V, or
 * to out + slots[k] V when slots (device) is not NULL; on `stream`.
 * Errors: VR_EINVAL, VR_ECUDA. */
int vr_codec_decode_bricks(vr_codec* codec, const int32_t* bricks, const int32_t* slots, int32_t n, float* out,
                           void* stream);

/*
 * Render from a codec instead of a cube (no counterpart in the paper): like
 * vr_load_cube_host, the context keeps a device brick cache (VR_OPT_DEVICE_BUDGET)
 * and marches bricks from it (VR_OPT_OOC_MARCH), but fills a slot by decoding
 * the brick on the tensor cores instead of copying it from host memory.  Empty-
 * space skipping uses the ranges recorded by vr_codec_fit_stats.  The codec must
 * outlive the context's use of it; vr_brick must give the codec's brick size.
 * Errors: VR_EINVAL (sizes or bricking do not match the codec), VR_ECUDA.
 */
int vr_load_cube_codec(vr_ctx* ctx, vr_codec* codec, int64_t nx, int64_t ny, int64_t nz);

/*
 * Per-brick fallback of a learned context to the plain voxels (no counterpart in
 * the paper): at the next vr_brick every brick is decoded and compared with its
 * block of the plain cube `data` (host memory, float32[nz][ny][nx] of the sizes
 * given to vr_load_cube_codec; read during that vr_brick only, the caller keeps
 * ownership).  The error of a brick is the largest |max(d, floor_v) -
 * max(v, floor_v)| over the voxels of its (bx+1)(by+1)(bz+1) block that lie
 * inside the cube (d decoded, v plain): values at or below floor_v, where the
 * transfer function is transparent, count as floor_v.  A brick whose error
 * exceeds `bound` keeps a pinned host copy of its plain block and is copied into
 * its cache slot (as vr_load_cube_host does) instead of decoded.  bound < 0: every
 * brick falls back; bound = +inf: none.  data = NULL turns the fallback off.
 * Errors: VR_ESTATE (not a learned context), VR_EINVAL (NaN bound or floor); the
 * scan's own errors (VR_ENOMEM, VR_ECUDA) are reported by vr_brick.
 */
int vr_set_codec_fallback(vr_ctx* ctx, const float* data, float bound, float floor_v);

/*
 * The same fallback with the plain blocks taken from a brick provider (see
 * vr_load_cube_provider) instead of a host cube: the scan at vr_brick calls fn for
 * every brick's block, and the bricks over the bound keep pinned host copies of
 * their blocks.  fn = NULL turns the fallback off.  fn and user are used during
 * vr_brick only.  Errors: as vr_set_codec_fallback; a failing provider makes
 * vr_brick return VR_ESOURCE.
 */
int vr_set_codec_fallback_provider(vr_ctx* ctx, vr_block_provider fn, void* user, float bound, float floor_v);

/* The per-brick errors measured by the last vr_brick's fallback scan (host
 * float32[n_bricks], may be NULL) and the number of bricks that fall back (may be
 * NULL).  Errors: VR_ESTATE (no scan since the last load). */
int vr_codec_brick_errors(vr_ctx* ctx, float* err, int64_t* n_plain);

/*
 * Allocation-free render (the paper has no counterpart; this serves callers that
 * may not allocate device memory while rendering: an application or plugin that
 * owns the device-memory budget, a real-time loop that cannot take the implicit
 * synchronisation of cudaMalloc/cudaFree, or an embedding with its own allocator).
 * It renders the same image as vr_render (emission-absorption mode, every brick
 * marched, rendering-rectangle culling on) but calls no cudaMalloc, cudaFree or
 * other allocating routine and needs no context: its scratch (work list,
 * per-brick sub-image fragments, counters) lives in one static device array of
 * VR_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library holds until
 * the process exits.
 *   cube:      device memory, float32[nz][ny][nx], x fastest, 2 <= n <= 65536.
 *   bx,by,bz:  brick size (>= 1), at most 4096 bricks.
 *   tf_points: host memory, n_tf rows (v, r, g, b, a) as for vr_set_transfer_function.
 *   cam:       as for vr_set_camera, with width and height <= 1024.
 *   out_rgba:  device memory, float32[height][width][4], written on cuda_stream.
 * Runs on the current CUDA device; cube and out_rgba must be device memory of
 * that device.  The frame is marched by the direct-gather kernel (corners read
 * through the L1 cache), which gives the same image as vr_render's other
 * kernels up to FP32 rounding.  Set-up: the first call on each device looks up
 * the scratch array's device address (cudaGetSymbolAddress) and creates two
 * events, and the first call in the process page-locks the library's two static
 * host staging sets of the plan (cudaHostRegister, which allocates nothing);
 * make that first call before any stream capture.  Each call's plan uploads are
 * then asynchronous copies from one staging set; a call waits (on the host)
 * until the uploads of the call two before it, which used the same set, are
 * done.  All calls share the device scratch, which keeps the last call's
 * contents (the counters are cleared by each call, everything else is
 * rewritten): calls that overlap on the GPU race, and the function must not be
 * called from two host threads at once.
 * Errors: VR_EINVAL (bad argument, a cube or image that is host memory or
 * memory of another device, or a frame whose work list needs more than
 * VR_NOALLOC_SCRATCH_BYTES), VR_ECUDA.
 */
#define VR_NOALLOC_SCRATCH_BYTES (16 * 1024 * 1024)
int vr_render_noalloc(const float* cube, int64_t nx, int64_t ny, int64_t nz, int32_t bx, int32_t by,
                      int32_t bz, const double* tf_points, int32_t n_tf, const vr_camera* cam,
                      float* out_rgba, void* cuda_stream);

/* Message describing the last failing call on ctx (never NULL). */
const char* vr_last_error(const vr_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* VR_H */
