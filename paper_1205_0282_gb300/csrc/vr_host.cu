// Host side of the C ABI declared in include/vr.h: context, brick store, transfer
// function and camera state, the per-frame planner (rendering rectangles, exact
// empty-space skipping, view-order sort, work-list build; Sections 2.3.1-2.3.3 of
// arXiv:1205.0282) and the stream-ordered frame pipeline.
#include <thread>

#include "vr_ctx.cuh"

using namespace vrh;

namespace vrh {
int retire(vr_ctx* c, Slot& s) {
    if (!s.pending) return VR_OK;
    VR_CUDA(c, cudaEventSynchronize(s.ev_end));
    float ms_march = 0, ms_frame = 0, ms_comp = 0;
    VR_CUDA(c, cudaEventElapsedTime(&ms_march, s.ev_march0, s.ev_march1));
    VR_CUDA(c, cudaEventElapsedTime(&ms_comp, s.ev_march1, s.ev_end));
    VR_CUDA(c, cudaEventElapsedTime(&ms_frame, s.ev_begin, s.ev_end));
    c->acc.frames += 1;
    c->acc.samples += (int64_t)s.h_stats->samples;
    c->acc.chunks_staged += (int64_t)s.h_stats->chunks_staged;
    c->acc.chunks_direct += (int64_t)s.h_stats->chunks_direct;
    c->acc.items += s.items;
    c->acc.fragments += s.fragments;
    c->acc.bricks_rendered += s.bricks_rendered;
    c->acc.bricks_skipped += s.bricks_skipped;
    c->acc.touched_bytes += s.touched_bytes;
    c->acc.march_ms += ms_march;
    c->acc.composite_ms += ms_comp;
    c->acc.frame_ms += ms_frame;
    c->acc.plan_ms += s.plan_ms;
    c->acc.h2d_bytes += s.h2d_bytes;
    c->acc.d2h_bytes += s.d2h_bytes;
    c->acc.launches += s.launches;
    c->acc.bricks_uploaded += s.bricks_uploaded;
    c->acc.bricks_cached += s.bricks_cached;
    c->acc.device_errors |= s.h_stats->errors;
    s.pending = false;
    return VR_OK;
}

int retire_all(vr_ctx* c) {
    for (auto& s : c->slots) {
        int rc = retire(c, s);
        if (rc) return rc;
    }
    return VR_OK;
}

// Build the frame's work list into slot s (host).  Returns VR_OK.
// Kernel selection for emission-absorption frames: VR_KERNEL_AUTO takes the
// texture-gather march when the cube fits the device's layered-texture limits and
// the TMA-staged march otherwise.
// Bricks per slab of the layered copy whose layers run along axis S: as many as
// fit the device's layer limit (or VR_OPT_TEX_SLAB_LAYERS) with their apron layer.
int32_t tex_slab_bricks(vr_ctx* c, int S, int max_layers) {
    int64_t lim = max_layers;
    if (c->tex_slab_layers > 0) lim = std::min<int64_t>(lim, c->tex_slab_layers);
    return (int32_t)std::max<int64_t>((lim - 1) / c->B[S], 0);
}
bool tex_fits(vr_ctx* c) {
    if (c->tex_fits < 0) {
        int maxw = 0, maxh = 0, maxl = 0;
        cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxTexture2DLayeredWidth, c->device);
        cudaDeviceGetAttribute(&maxh, cudaDevAttrMaxTexture2DLayeredHeight, c->device);
        cudaDeviceGetAttribute(&maxl, cudaDevAttrMaxTexture2DLayeredLayers, c->device);
        bool ok = c->n[1] <= 65535 && c->n[2] <= 65535;
        for (int S = 0; S < 3; ++S) {
            const int U = S == 0 ? 1 : 0, V = S == 2 ? 1 : 2;
            const int32_t K = tex_slab_bricks(c, S, maxl);
            ok = ok && c->n[U] <= maxw && c->n[V] <= maxh && K > 0 &&
                 (c->nb[S] + K - 1) / K <= vr::kMaxTexSlabs;
        }
        c->tex_fits = ok ? 1 : 0;
    }
    return c->tex_fits == 1;
}
bool use_tex(vr_ctx* c) {
    // MIP frames run on the texture march with FP32 storage only
    return !c->ooc && (c->mode == 0 || c->precision == VR_PRECISION_F32) &&
           (c->kernel == VR_KERNEL_TEX || (c->kernel == VR_KERNEL_AUTO && tex_fits(c)));
}
bool use_tma(vr_ctx* c) {
    return !c->ooc && c->mode == 0 && c->step_mode == 0 && (c->kernel == VR_KERNEL_TMA || (c->kernel == VR_KERNEL_AUTO && !tex_fits(c)));
}

// The layered copies of the out-of-core cache (texture march).
void free_pool_tex(vr_ctx* c) {
    for (int a = 0; a < 3; ++a) {
        if (c->pool_tex[a]) cudaDestroyTextureObject(c->pool_tex[a]);
        if (c->pool_surf[a]) cudaDestroySurfaceObject(c->pool_surf[a]);
        if (c->pool_arr[a]) cudaFreeArray(c->pool_arr[a]);
        c->pool_tex[a] = 0;
        c->pool_surf[a] = 0;
        c->pool_arr[a] = nullptr;
        c->pool_cols[a] = 0;
    }
    c->pool_tex_on = false;
    c->pool_axes = 0;
    c->pool_stage = 0;
}

bool use_pool_tex(vr_ctx* c) { return c->ooc && c->pool_tex_on; }

void free_ooc(vr_ctx* c) {
    free_pool_tex(c);
    if (c->h_store) cudaFreeHost(c->h_store);
    cudaFree(c->d_pool);
    c->h_store = nullptr;
    c->d_pool = nullptr;
    c->store_bytes = 0;
    c->res = vr::Residency();
    for (int j = 0; j < vr_ctx::kStage; ++j) {
        if (c->ev_stage[j]) cudaEventSynchronize(c->ev_stage[j]);
        if (c->h_stage[j]) cudaFreeHost(c->h_stage[j]);
        c->h_stage[j] = nullptr;
    }
    c->stage_cap = 0;
    c->h_src = nullptr;
    c->prov_fn = nullptr;
    c->prov_user = nullptr;
    c->codec = nullptr;
    c->fb_src = nullptr;
    c->fb_fn = nullptr;
    c->fb_user = nullptr;
    c->fb_measured = false;
    c->brick_err.clear();
    c->plain_index.clear();
    c->n_plain = 0;
    c->ooc = false;
}

// Side streams and events of the out-of-core pipeline (created once per context).
int ensure_ooc_streams(vr_ctx* c) {
    if (c->copy_stream) return VR_OK;
    int lo_prio = 0, hi_prio = 0;
    VR_CUDA(c, cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio));
    // high priority: a learned context's decodes (kernels on this stream) feed the
    // ring and should not queue behind the resident bricks' long march
    VR_CUDA(c, cudaStreamCreateWithPriority(&c->copy_stream, cudaStreamNonBlocking, hi_prio));
    VR_CUDA(c, cudaEventCreateWithFlags(&c->ev_march_done, cudaEventDisableTiming));
    VR_CUDA(c, cudaEventCreateWithFlags(&c->ev_copy_done, cudaEventDisableTiming));
    for (cudaEvent_t& ev : c->ev_half_read) VR_CUDA(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    // the ring's marches free its halves for the next copies: schedule their
    // blocks ahead of the resident bricks' long launch
    VR_CUDA(c, cudaStreamCreateWithPriority(&c->ring_stream, cudaStreamNonBlocking, hi_prio));
    VR_CUDA(c, cudaEventCreateWithFlags(&c->ev_ring_start, cudaEventDisableTiming));
    VR_CUDA(c, cudaEventCreateWithFlags(&c->ev_ring_end, cudaEventDisableTiming));
    for (cudaEvent_t& ev : c->ev_stage) VR_CUDA(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    return VR_OK;
}

vr::BlockSource brick_source(vr_ctx* c) {
    vr::BlockSource bs;
    bs.cube = c->h_src;
    bs.fn = c->prov_fn;
    bs.user = c->prov_user;
    bs.threads = c->prov_threads;
    return bs;
}

int source_fail(vr_ctx* c, int64_t brick) {
    return fail(c, VR_ESOURCE, "the brick provider failed for brick " + std::to_string(brick));
}

// Learned residency's fallback (at vr_brick): decode every brick, compare it with
// its plain block, and keep pinned plain blocks of the bricks over the bound.
int codec_fallback_scan(vr_ctx* c) {
    const int64_t nb = c->n_bricks;
    c->brick_err.assign(nb, 0.0f);
    c->plain_index.assign(nb, -1);
    c->n_plain = 0;
    c->fb_measured = false;
    vr::BlockSource fb;
    fb.cube = c->fb_src;
    fb.fn = c->fb_fn;
    fb.user = c->fb_user;
    fb.threads = c->prov_threads;
    if (!fb.valid()) return VR_OK;
    const size_t slot_bytes = (size_t)c->slot_floats * sizeof(float);
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(nb, ((int64_t)256 << 20) / (int64_t)slot_bytes));
    float *d_dec = nullptr, *d_plain = nullptr, *h_stage = nullptr;
    int32_t *d_ids = nullptr, *h_ids = nullptr;
    uint32_t* d_err = nullptr;
    int rc = VR_OK;
    if (cudaMalloc((void**)&d_dec, chunk * slot_bytes) != cudaSuccess ||
        cudaMalloc((void**)&d_plain, chunk * slot_bytes) != cudaSuccess ||
        cudaMalloc((void**)&d_ids, chunk * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc((void**)&d_err, nb * sizeof(uint32_t)) != cudaSuccess ||
        cudaHostAlloc((void**)&h_stage, chunk * slot_bytes, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void**)&h_ids, chunk * sizeof(int32_t), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        rc = fail(c, VR_ENOMEM, "cannot allocate the fallback scan's buffers");
    }
    if (!rc && cudaMemsetAsync(d_err, 0, nb * sizeof(uint32_t), c->copy_stream) != cudaSuccess)
        rc = fail(c, VR_ECUDA, "fallback scan: memset failed");
    for (int64_t b0 = 0; !rc && b0 < nb; b0 += chunk) {
        const int32_t k = (int32_t)std::min<int64_t>(chunk, nb - b0);
        for (int32_t i = 0; i < k; ++i) h_ids[i] = (int32_t)(b0 + i);
        int64_t bad = -1;
        if (vr::read_blocks(fb, c->n, c->B, c->nb, h_ids, k, h_stage, c->slot_floats, nullptr, &bad)) {
            rc = source_fail(c, bad);
            break;
        }
        if (cudaMemcpyAsync(d_ids, h_ids, k * sizeof(int32_t), cudaMemcpyHostToDevice, c->copy_stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(d_plain, h_stage, k * slot_bytes, cudaMemcpyHostToDevice, c->copy_stream) != cudaSuccess) {
            rc = fail(c, VR_ECUDA, "fallback scan: copy failed");
            break;
        }
        if ((rc = vr_codec_decode_bricks(c->codec, d_ids, nullptr, k, d_dec, c->copy_stream))) {
            rc = fail(c, rc, "fallback scan: brick decode failed");
            break;
        }
        if (vr::launch_brick_error(d_dec, d_plain, b0, k, c->n, c->B, c->nb, c->fb_floor, d_err + b0,
                                   c->copy_stream) != cudaSuccess ||
            cudaStreamSynchronize(c->copy_stream) != cudaSuccess) {  // the staging buffers are reused
            rc = fail(c, VR_ECUDA, "fallback scan: comparison failed");
            break;
        }
    }
    if (!rc && cudaMemcpy(c->brick_err.data(), d_err, nb * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = fail(c, VR_ECUDA, "fallback scan: cannot read the errors");
    cudaFree(d_dec);
    cudaFree(d_plain);
    cudaFree(d_ids);
    cudaFree(d_err);
    if (h_stage) cudaFreeHost(h_stage);
    if (h_ids) cudaFreeHost(h_ids);
    if (rc) return rc;
    std::vector<int32_t> plain;
    for (int64_t b = 0; b < nb; ++b)
        if (c->brick_err[b] > c->fb_bound) {
            c->plain_index[b] = (int64_t)plain.size();
            plain.push_back((int32_t)b);
        }
    c->n_plain = (int64_t)plain.size();
    c->fb_measured = true;
    if (plain.empty()) return VR_OK;
    c->store_bytes = slot_bytes * plain.size();
    if (cudaHostAlloc((void**)&c->h_store, c->store_bytes, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        c->h_store = nullptr;
        c->store_bytes = 0;
        return fail(c, VR_ENOMEM, "cannot allocate the pinned store of the fallback bricks");
    }
    int64_t bad = -1;
    if (vr::read_blocks(fb, c->n, c->B, c->nb, plain.data(), (int64_t)plain.size(), c->h_store, c->slot_floats,
                        nullptr, &bad))
        return source_fail(c, bad);
    return VR_OK;
}

// Layered copies of the cache's slots for the texture march: for each sweep axis S
// in `axes` (bit S) a layered array with layers along S (B_S + 1 of them) and the
// slots' (U, V) faces tiled pool_cols[S] per row (an item then sweeps along the
// ray's dominant axis among those kept).  If the device's layered-texture limits
// do not admit the tiling, the context keeps the direct march.
int make_pool_tex(vr_ctx* c, int64_t slots, int axes) {
    int maxw = 0, maxh = 0, maxl = 0;
    VR_CUDA(c, cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxTexture2DLayeredWidth, c->device));
    VR_CUDA(c, cudaDeviceGetAttribute(&maxh, cudaDevAttrMaxTexture2DLayeredHeight, c->device));
    VR_CUDA(c, cudaDeviceGetAttribute(&maxl, cudaDevAttrMaxTexture2DLayeredLayers, c->device));
    int64_t cols[3], rows[3];
    for (int S = 0; S < 3; ++S) {
        if (!(axes >> S & 1)) continue;
        const int U = S == 0 ? 1 : 0, V = S == 2 ? 1 : 2;
        cols[S] = std::min<int64_t>(slots, maxw / (c->B[U] + 1));
        if (cols[S] < 1) return VR_OK;
        rows[S] = (slots + cols[S] - 1) / cols[S];
        if (rows[S] * (c->B[V] + 1) > maxh || c->B[S] + 1 > maxl) return VR_OK;
    }
    cudaChannelFormatDesc ch = cudaCreateChannelDesc<float>();
    for (int S = 0; S < 3; ++S) {
        if (!(axes >> S & 1)) continue;
        const int U = S == 0 ? 1 : 0, V = S == 2 ? 1 : 2;
        if (cudaMalloc3DArray(&c->pool_arr[S], &ch,
                              make_cudaExtent((size_t)(cols[S] * (c->B[U] + 1)), (size_t)(rows[S] * (c->B[V] + 1)),
                                              (size_t)(c->B[S] + 1)),
                              cudaArrayLayered | cudaArraySurfaceLoadStore) != cudaSuccess) {
            cudaGetLastError();
            free_pool_tex(c);
            return fail(c, VR_ENOMEM, "cannot allocate the layered copies of the brick cache");
        }
        cudaResourceDesc rd;
        std::memset(&rd, 0, sizeof(rd));
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = c->pool_arr[S];
        cudaTextureDesc td;
        std::memset(&td, 0, sizeof(td));
        td.addressMode[0] = td.addressMode[1] = td.addressMode[2] = cudaAddressModeClamp;
        td.filterMode = cudaFilterModePoint;
        td.readMode = cudaReadModeElementType;
        td.normalizedCoords = 0;
        if (cudaCreateTextureObject(&c->pool_tex[S], &rd, &td, nullptr) != cudaSuccess ||
            cudaCreateSurfaceObject(&c->pool_surf[S], &rd) != cudaSuccess) {
            cudaGetLastError();
            free_pool_tex(c);
            return fail(c, VR_ECUDA, "cannot create the brick cache's texture objects");
        }
        c->pool_cols[S] = (int32_t)cols[S];
    }
    c->pool_tex_on = true;
    c->pool_axes = axes;
    return VR_OK;
}

// Blocks of the texture march's staging area for a cache of `slots` slots: one
// launch's uploads, i.e. a group of resident uploads (about 64 MiB, and no more
// than an eighth of the cache) or a ring half (max(1, min(slots / 8, 32))
// bricks), whichever is larger.
int64_t ooc_stage_blocks(int64_t slots, size_t slot_bytes) {
    const int64_t group = std::max<int64_t>(1, ((int64_t)64 << 20) / (int64_t)slot_bytes);
    const int64_t eighth = std::max<int64_t>(1, slots / 8);
    const int64_t half = std::max<int64_t>(1, std::min<int64_t>(slots / 8, 32));
    return std::max(std::min(group, eighth), half);
}

// Brick store and device cache of an out-of-core context (at vr_brick).
int build_ooc_store(vr_ctx* c) {
    free_pool_tex(c);
    for (int j = 0; j < vr_ctx::kStage; ++j) {
        if (c->ev_stage[j]) cudaEventSynchronize(c->ev_stage[j]);
        if (c->h_stage[j]) cudaFreeHost(c->h_stage[j]);
        c->h_stage[j] = nullptr;
    }
    c->stage_cap = 0;
    if (c->h_store) cudaFreeHost(c->h_store);
    cudaFree(c->d_pool);
    c->h_store = nullptr;
    c->d_pool = nullptr;
    c->slot_floats = (int64_t)(c->B[0] + 1) * (c->B[1] + 1) * (c->B[2] + 1);
    const size_t slot_bytes = (size_t)c->slot_floats * sizeof(float);
    if (c->codec) {
        int32_t cb[3];
        vr_codec_brick_size(c->codec, cb);
        if (cb[0] != c->B[0] || cb[1] != c->B[1] || cb[2] != c->B[2] || vr_codec_brick_count(c->codec) != c->n_bricks)
            return fail(c, VR_EINVAL, "the bricking does not match the codec's");
        if (vr_codec_get_minmax(c->codec, reinterpret_cast<float*>(c->h_minmax.data())))
            return fail(c, VR_ECUDA, "cannot read the codec's brick ranges");
    } else if (c->prov_fn) {
        // no store: every brick once through the provider for its range, then the
        // pinned staging the uploads go through (one launch's bricks per buffer:
        // at most a 64 MiB group of resident uploads or a 32-brick ring half)
        const int64_t per_chunk = std::max<int64_t>(1, ((int64_t)256 << 20) / (int64_t)slot_bytes);
        std::vector<float> buf((size_t)(std::min<int64_t>(per_chunk, c->n_bricks) * c->slot_floats));
        for (int64_t b0 = 0; b0 < c->n_bricks; b0 += per_chunk) {
            const int64_t k = std::min<int64_t>(per_chunk, c->n_bricks - b0);
            std::vector<int32_t> ids(k);
            for (int64_t i = 0; i < k; ++i) ids[i] = (int32_t)(b0 + i);
            int64_t bad = -1;
            if (vr::read_blocks(brick_source(c), c->n, c->B, c->nb, ids.data(), k, buf.data(), c->slot_floats,
                                c->h_minmax.data() + b0, &bad))
                return source_fail(c, bad);
        }
        const size_t group = std::max<size_t>(1, ((size_t)64 << 20) / slot_bytes);
        c->stage_cap = std::max<size_t>(group, 32) * slot_bytes;
        for (int j = 0; j < vr_ctx::kStage; ++j)
            if (cudaHostAlloc((void**)&c->h_stage[j], c->stage_cap, cudaHostAllocDefault) != cudaSuccess) {
                cudaGetLastError();
                c->h_stage[j] = nullptr;
                return fail(c, VR_ENOMEM, "cannot allocate the provider's pinned staging");
            }
    } else {
        c->store_bytes = slot_bytes * (size_t)c->n_bricks;
        if (cudaHostAlloc((void**)&c->h_store, c->store_bytes, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            c->h_store = nullptr;
            return fail(c, VR_ENOMEM, "cannot allocate the pinned brick store");
        }
        vr::read_blocks(brick_source(c), c->n, c->B, c->nb, nullptr, c->n_bricks, c->h_store, c->slot_floats,
                        c->h_minmax.data(), nullptr);
    }
    // The texture march keeps each slot as layered copies only, three (one per
    // sweep axis), the ones along x and z, or the one along z, and the blocks pass
    // through a staging area
    // holding one launch's uploads.  The direct march keeps a block per slot.
    // Automatically: as many copies (three, the two along x and z, the one along
    // z) as let every brick fit the budget, else the direct march (a streaming
    // cache is bound by its uploads, which the direct march does not follow with
    // fills).
    const int64_t budget_blocks = c->budget > 0 ? c->budget / (int64_t)slot_bytes : -1;
    auto fits = [&](int64_t copies) {
        return budget_blocks < 0 ||
               (budget_blocks - ooc_stage_blocks(budget_blocks / copies, slot_bytes)) / copies >= c->n_bricks;
    };
    int axes = 0;  // bit S: the copy along axis S (0: the direct march)
    if (c->ooc_march == 1) axes = 7;
    else if (c->ooc_march == 4) axes = 5;
    else if (c->ooc_march == 3) axes = 4;
    else if (c->ooc_march == 2) axes = fits(3) ? 7 : (fits(2) ? 5 : (fits(1) ? 4 : 0));
    const bool tex_march = axes != 0;
    int64_t slots = 0;
    c->pool_stage = 0;
    if (tex_march) {
        const int64_t copies = (axes & 1) + (axes >> 1 & 1) + (axes >> 2 & 1);
        int64_t stage = ooc_stage_blocks(c->n_bricks, slot_bytes);
        slots = c->n_bricks;
        if (budget_blocks >= 0) {
            stage = ooc_stage_blocks(budget_blocks / copies, slot_bytes);
            slots = std::min<int64_t>(slots, (budget_blocks - stage) / copies);
        }
        if (slots < 2) return fail(c, VR_EINVAL, "VR_OPT_DEVICE_BUDGET holds fewer than 2 bricks");
        int rc = make_pool_tex(c, slots, axes);
        if (rc) return rc;
        if (c->pool_tex_on) c->pool_stage = stage;
    }
    if (!c->pool_tex_on) {
        slots = budget_blocks >= 0 ? std::min<int64_t>(c->n_bricks, budget_blocks) : c->n_bricks;
        if (slots < 2) return fail(c, VR_EINVAL, "VR_OPT_DEVICE_BUDGET holds fewer than 2 bricks");
    }
    const int64_t blocks = c->pool_stage > 0 ? c->pool_stage : slots;
    if (cudaMalloc((void**)&c->d_pool, slot_bytes * (size_t)blocks) != cudaSuccess) {
        cudaGetLastError();
        c->d_pool = nullptr;
        free_pool_tex(c);
        return fail(c, VR_ENOMEM, "cannot allocate the device brick cache");
    }
    c->res.slot_of_brick.assign(c->n_bricks, -1);
    c->res.brick_in_slot.assign(slots, -1);
    c->res.last_used.assign(slots, -1);
    return c->codec ? codec_fallback_scan(c) : VR_OK;
}

int64_t precision_bytes(int precision) {
    return precision == VR_PRECISION_F16 ? 2 : (precision == VR_PRECISION_F8 ? 1 : 4);
}

void free_tex(vr_ctx* c) {
    for (int a = 0; a < 3; ++a) {
        for (int j = 0; j < vr::kMaxTexSlabs; ++j) {
            if (c->tex_obj[a][j]) cudaDestroyTextureObject(c->tex_obj[a][j]);
            if (c->tex_arr[a][j]) cudaFreeArray(c->tex_arr[a][j]);
            c->tex_obj[a][j] = 0;
            c->tex_arr[a][j] = nullptr;
        }
        c->tex_slab_bricks[a] = 0;
    }
    cudaFree(c->d_brick_scale);
    c->d_brick_scale = nullptr;
    c->tex_ready = false;
}

int plan_frame(vr_ctx* c, Slot& s, const int32_t win[4], int32_t& tiles_x, int32_t& tiles_y, int32_t& T,
               int64_t& n_items, bool emit) {
    const vr_camera& cam = c->cam;
    T = use_tma(c) ? vr::kTileTma : vr::kTile;  // the direct and texture marches use 8x8 tiles
    tiles_x = (cam.width + T - 1) / T;
    tiles_y = (cam.height + T - 1) / T;
    const int64_t n_tiles = (int64_t)tiles_x * tiles_y;
    // sweep axis of each tile for the TMA march: the dominant axis of the ray
    // through the tile's centre pixel, and its sign
    c->plan_sweep.assign(n_tiles, 0);
    if (use_tma(c) || use_tex(c) || use_pool_tex(c)) {
        // view-plane offsets of the tile centres' columns and rows, then per tile
        // d = f + qx r + qy u (no division in the tile loop)
        c->plan_qx.resize(tiles_x);
        c->plan_qy.resize(tiles_y);
        for (int tx = 0; tx < tiles_x; ++tx) {
            const int i = std::min(tx * T + T / 2, cam.width - 1);
            c->plan_qx[tx] = (2.0 * (i + 0.5) / cam.width - 1.0) * c->basis.tan_half * c->basis.aspect;
        }
        for (int ty = 0; ty < tiles_y; ++ty) {
            const int j = std::min(ty * T + T / 2, cam.height - 1);
            c->plan_qy[ty] = (1.0 - 2.0 * (j + 0.5) / cam.height) * c->basis.tan_half;
        }
        const double* f = c->basis.f;
        const double* r = c->basis.r;
        const double* u = c->basis.u;
        const int axes = use_pool_tex(c) ? c->pool_axes : 7;  // the cache's copies
        for (int ty = 0; ty < tiles_y; ++ty) {
            const double qy = c->plan_qy[ty];
            const double g0 = f[0] + qy * u[0], g1 = f[1] + qy * u[1], g2 = f[2] + qy * u[2];
            int32_t* sweep = c->plan_sweep.data() + (int64_t)ty * tiles_x;
            for (int tx = 0; tx < tiles_x; ++tx) {
                const double qx = c->plan_qx[tx];
                const double d[3] = {g0 + qx * r[0], g1 + qx * r[1], g2 + qx * r[2]};
                // the dominant axis among those with a copy (ties to the lower axis)
                int ax = -1;
                for (int a = 0; a < 3; ++a)
                    if ((axes >> a & 1) && (ax < 0 || std::fabs(d[a]) > std::fabs(d[ax]))) ax = a;
                sweep[tx] = ax | (d[ax] < 0.0 ? 4 : 0);
            }
        }
    }

    // eye's brick index per axis, -1 / nb when outside (view-order key, see below)
    int64_t e[3];
    for (int a = 0; a < 3; ++a) {
        double E = cam.eye[a];
        if (E < 0.0) e[a] = -1;
        else if (E > (double)(c->n[a] - 1)) e[a] = c->nb[a];
        else e[a] = std::min<int64_t>((int64_t)std::floor(E / c->B[a]), c->nb[a] - 1);
    }

    // projections of the brick grid's corner points: each brick box spans eight
    // of them, so each is projected once, not per brick
    const int64_t nb64[3] = {c->nb[0], c->nb[1], c->nb[2]};
    if (c->rect_cull) project_brick_grid(cam, c->basis, c->n, c->B, nb64, c->plan_proj);

    // Opacity runs of the TF that reach its first or its last control point: a brick
    // whose value range lies within one has zero opacity, the empty-space test's
    // answer without evaluating the TF (its other bricks go through tf_alpha_max).
    const std::vector<double>& tf = c->tf;
    const int n_tf = (int)(tf.size() / 5);
    double zero_to = -INFINITY, zero_from = INFINITY;
    {
        int z = -1, w = n_tf;
        while (z + 1 < n_tf && tf[5 * (z + 1) + 4] == 0.0) ++z;
        while (w > 0 && tf[5 * (w - 1) + 4] == 0.0) --w;
        if (z >= 0) zero_to = tf[5 * z];
        if (w < n_tf) zero_from = tf[5 * w];
    }

    // Per brick: region, empty-space test, rectangle, silhouette spans and the
    // per-tile item counts.  Host threads take consecutive chunks of bricks.
    const bool lowp = use_tex(c) && c->precision != VR_PRECISION_F32;
    const int64_t vox_bytes = use_tex(c) ? precision_bytes(c->precision) : (int64_t)sizeof(float);
    const int64_t dw = tiles_x + 1;
    const int32_t n_keys = c->nb[0] + c->nb[1] + c->nb[2] + 1;  // keys are at most the sum of the brick counts
    using Part = vr_ctx::PlanPart;
    auto plan_range = [&](int64_t id0, int64_t id1, int32_t part) {
        Part& out = c->plan_parts[part];
        out.bricks.clear();
        out.keys.clear();
        out.spans.clear();
        out.diff.assign((size_t)(dw * tiles_y), 0);
        out.key_count.assign((size_t)n_keys, 0);
        out.skipped = out.touched = out.items = 0;
        int64_t idx[3] = {id0 % c->nb[0], (id0 / c->nb[0]) % c->nb[1], id0 / ((int64_t)c->nb[0] * c->nb[1])};
        auto next = [&]() {
            if (++idx[0] < c->nb[0]) return;
            idx[0] = 0;
            if (++idx[1] < c->nb[1]) return;
            idx[1] = 0;
            ++idx[2];
        };
        for (int64_t id = id0; id < id1; ++id, next()) {
            bool inside = true;
            for (int a = 0; a < 3; ++a) inside = inside && idx[a] >= c->region_lo[a] && idx[a] < c->region_hi[a];
            if (!inside) continue;
            if (c->skip_empty && c->mode == 0) {
                const float2 mm = lowp ? c->h_minmax_q[id] : c->h_minmax[id];
                if ((double)mm.y <= zero_to || (double)mm.x >= zero_from || tf_alpha_max(tf, mm.x, mm.y) == 0.0) {
                    ++out.skipped;
                    continue;
                }
            }
            int32_t rect[4];
            if (c->rect_cull) {
                if (!brick_rect_from_grid(cam, c->plan_proj, nb64, idx, rect)) continue;
            } else {
                rect[0] = rect[1] = 0;
                rect[2] = cam.width - 1;
                rect[3] = cam.height - 1;
            }
            // only the output window's pixels are computed
            rect[0] = std::max(rect[0], win[0]);
            rect[1] = std::max(rect[1], win[1]);
            rect[2] = std::min(rect[2], win[2]);
            rect[3] = std::min(rect[3], win[3]);
            if (rect[2] < rect[0] || rect[3] < rect[1]) continue;
            // the tiles its silhouette reaches, row by row (the rectangle's in full
            // without culling), rows ascending
            vr_ctx::PB pb;
            pb.id = (int32_t)id;
            pb.part = part;
            pb.span0 = (int32_t)out.spans.size();
            if (c->rect_cull) {
                const CornerProj* q[8];
                grid_corners(c->plan_proj, nb64, idx, q);
                brick_spans(q, rect, T, out.spans);
            } else {
                for (int ty = rect[1] / T; ty <= rect[3] / T; ++ty)
                    out.spans.push_back(Span{ty, rect[0] / T, rect[2] / T});
            }
            pb.nspan = (int32_t)out.spans.size() - pb.span0;
            pb.n_items = 0;
            for (int32_t k = pb.span0; k < pb.span0 + pb.nspan; ++k) {
                const Span& sp = out.spans[k];
                pb.n_items += sp.tx1 - sp.tx0 + 1;
                out.diff[(size_t)(sp.ty * dw + sp.tx0)] += 1;
                out.diff[(size_t)(sp.ty * dw + sp.tx1 + 1)] -= 1;
            }
            if (pb.n_items == 0) {
                out.spans.resize(pb.span0);
                continue;
            }
            out.items += pb.n_items;
            // Along any ray from the eye each axis index moves monotonically away from
            // the eye's index, so sum |b - e| strictly increases from one brick to the
            // next: ordering by it is a valid front-to-back order for every ray.
            int32_t key = 0;
            for (int a = 0; a < 3; ++a) key += (int32_t)std::llabs(idx[a] - e[a]);
            out.bricks.push_back(pb);
            out.keys.push_back(key);
            ++out.key_count[key];
            int64_t vox = 1;
            for (int a = 0; a < 3; ++a) vox *= std::min<int64_t>(c->B[a], c->n[a] - idx[a] * c->B[a]);
            out.touched += vox * vox_bytes;
        }
    };
    const int32_t n_parts = (int32_t)std::max<int64_t>(1, std::min<int64_t>(plan_threads(), c->n_bricks / 256));
    if ((int32_t)c->plan_parts.size() < n_parts) c->plan_parts.resize(n_parts);
    auto run_parts = [&](auto&& fn) {
        if (n_parts == 1) {
            fn(0);
            return;
        }
        std::vector<std::thread> pool;
        for (int32_t t = 1; t < n_parts; ++t) pool.emplace_back(fn, t);
        fn(0);
        for (auto& th : pool) th.join();
    };
    run_parts([&](int32_t t) { plan_range(c->n_bricks * t / n_parts, c->n_bricks * (t + 1) / n_parts, t); });

    // the bricks in view order: a stable counting sort by key.  Bricks of one key
    // go part after part, each part's in brick order (the chunks are consecutive),
    // so the order is the same whatever the thread count; each part scatters its
    // own bricks.
    size_t n_bricks = 0;
    s.bricks_skipped = 0;
    s.touched_bytes = 0;
    n_items = 0;
    for (int32_t t = 0; t < n_parts; ++t) {
        const Part& pt = c->plan_parts[t];
        n_bricks += pt.bricks.size();
        s.bricks_skipped += pt.skipped;
        s.touched_bytes += pt.touched;
        n_items += pt.items;
    }
    {
        int64_t run = 0;
        for (int32_t k = 0; k < n_keys; ++k)
            for (int32_t t = 0; t < n_parts; ++t) {
                int32_t& cnt = c->plan_parts[t].key_count[k];
                const int32_t here = cnt;
                cnt = (int32_t)run;  // where the part's first brick of key k goes
                run += here;
            }
    }
    c->plan_bricks.resize(n_bricks);
    run_parts([&](int32_t t) {
        Part& pt = c->plan_parts[t];
        for (size_t i = 0; i < pt.bricks.size(); ++i) c->plan_bricks[(size_t)pt.key_count[pt.keys[i]]++] = pt.bricks[i];
    });
    s.bricks_rendered = (int64_t)n_bricks;

    // items per tile: the parts' difference arrays summed, then prefix sums per row
    std::vector<int32_t>& diff = c->plan_parts[0].diff;
    for (int64_t t = 1; t < n_parts; ++t) {
        const int32_t* d = c->plan_parts[t].diff.data();
        for (size_t i = 0; i < diff.size(); ++i) diff[i] += d[i];
    }
    c->plan_count.assign(n_tiles + 1, 0);
    for (int ty = 0; ty < tiles_y; ++ty) {
        int32_t run = 0;
        for (int tx = 0; tx < tiles_x; ++tx) {
            run += diff[(size_t)(ty * dw + tx)];
            c->plan_count[(int64_t)ty * tiles_x + tx] = run;
        }
    }
    if (n_items > (int64_t)INT32_MAX / (T * T)) return fail(c, VR_ENOMEM, "frame too large");
    int rc = grow_pinned(c, s.h_items, s.cap_items, (size_t)n_items);
    if (rc) return rc;
    rc = grow_pinned(c, s.h_tile_start, s.cap_tiles, (size_t)n_tiles + 1);
    if (rc) return rc;
    int32_t run = 0;
    for (int64_t t = 0; t < n_tiles; ++t) {
        s.h_tile_start[t] = run;
        run += c->plan_count[t];
    }
    s.h_tile_start[n_tiles] = run;
    s.items = n_items;
    if (emit) {
        // the items brick after brick in view order
        c->plan_dst.resize(n_bricks);
        int64_t w = 0;
        for (size_t k = 0; k < n_bricks; ++k) {
            c->plan_dst[k] = w;
            w += c->plan_bricks[k].n_items;
        }
        emit_items(c, s, tiles_x, tiles_y, n_items);
    }
    return VR_OK;
}

// The frame's items: brick k's items, one per tile of its spans, start at
// plan_dst[k] of the list; each gets its tile's next fragment slot in view order
// of the bricks, so every tile's fragments run front to back.  Rows of tiles are
// split among host threads by their item counts, each thread filling its rows'
// items wherever they sit in the list (the same list whatever the thread count).
void emit_items(vr_ctx* c, Slot& s, int32_t tiles_x, int32_t tiles_y, int64_t n_items) {
    const int64_t P = (int64_t)c->plan_bricks.size();
    c->plan_fill.assign((size_t)tiles_x * tiles_y, 0);
    auto rows = [&](int32_t ty0, int32_t ty1) {
        for (int64_t k = 0; k < P; ++k) {
            const vr_ctx::PB& pb = c->plan_bricks[k];
            const Span* sp = c->plan_parts[pb.part].spans.data() + pb.span0;
            if (sp[pb.nspan - 1].ty < ty0 || sp[0].ty >= ty1) continue;
            int64_t w = c->plan_dst[k];
            for (int32_t j = 0; j < pb.nspan; ++j) {
                const Span& q = sp[j];
                if (q.ty >= ty0 && q.ty < ty1) {
                    const int64_t t0 = (int64_t)q.ty * tiles_x;
                    for (int32_t tx = q.tx0; tx <= q.tx1; ++tx) {
                        const int64_t t = t0 + tx;
                        s.h_items[w + (tx - q.tx0)] =
                            vr::Item{pb.id, (int32_t)t, s.h_tile_start[t] + c->plan_fill[t]++, c->plan_sweep[t]};
                    }
                }
                w += q.tx1 - q.tx0 + 1;
            }
        }
    };
    const int64_t n_parts = std::max<int64_t>(1, std::min<int64_t>({plan_threads(), n_items / 65536, (int64_t)tiles_y}));
    if (n_parts == 1) {
        rows(0, tiles_y);
        return;
    }
    // row boundaries at about equal item counts
    std::vector<int32_t> cut(1, 0);
    for (int32_t ty = 0; ty < tiles_y && (int64_t)cut.size() < n_parts; ++ty) {
        const int64_t upto = s.h_tile_start[(int64_t)(ty + 1) * tiles_x];
        if (upto * n_parts >= n_items * (int64_t)cut.size()) cut.push_back(ty + 1);
    }
    cut.push_back(tiles_y);
    std::vector<std::thread> pool;
    for (size_t p = 1; p + 1 < cut.size(); ++p) pool.emplace_back(rows, cut[p], cut[p + 1]);
    rows(cut[0], cut[1]);
    for (auto& th : pool) th.join();
}

}  // namespace vrh

// =============================================================================== ABI

extern "C" {

int vr_create(vr_ctx** out, int32_t device) {
    if (!out) return VR_EINVAL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) {
        cudaGetLastError();
        return VR_ECUDA;
    }
    if (device < 0 || device >= count) return VR_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return VR_ECUDA;
    vr_ctx* c = new vr_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    for (auto& s : c->slots) {
        if (cudaEventCreate(&s.ev_begin) != cudaSuccess || cudaEventCreate(&s.ev_march0) != cudaSuccess ||
            cudaEventCreate(&s.ev_march1) != cudaSuccess || cudaEventCreate(&s.ev_end) != cudaSuccess ||
            cudaMalloc(&s.d_stats, sizeof(vr::Stats)) != cudaSuccess ||
            cudaMallocHost(&s.h_stats, sizeof(vr::Stats)) != cudaSuccess) {
            vr_destroy(c);
            return VR_ECUDA;
        }
        std::memset(s.h_stats, 0, sizeof(vr::Stats));
    }
    *out = c;
    return VR_OK;
}

void vr_destroy(vr_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    for (auto& s : c->slots) {
        if (s.pending) cudaEventSynchronize(s.ev_end);
        if (s.h_items) cudaFreeHost(s.h_items);
        if (s.h_tile_start) cudaFreeHost(s.h_tile_start);
        if (s.h_stats) cudaFreeHost(s.h_stats);
        if (s.h_frame) cudaFreeHost(s.h_frame);
        if (s.h_slot_of) cudaFreeHost(s.h_slot_of);
        cudaFree(s.d_slot_of);
        if (s.h_decode) cudaFreeHost(s.h_decode);
        cudaFree(s.d_decode);
        if (s.h_fill) cudaFreeHost(s.h_fill);
        cudaFree(s.d_fill);
        cudaFree(s.d_work);
        cudaFree(s.d_frame);
        cudaFree(s.d_items);
        cudaFree(s.d_tile_start);
        cudaFree(s.d_frags);
        cudaFree(s.d_img);
        cudaFree(s.d_stats);
        for (cudaEvent_t ev : {s.ev_begin, s.ev_march0, s.ev_march1, s.ev_end})
            if (ev) cudaEventDestroy(ev);
    }
    cudaFree(c->d_cube);
    cudaFree(c->d_cube_xzy);
    cudaFree(c->d_tmaps);
    free_tex(c);
    cudaFree(c->d_minmax);
    cudaFree(c->d_comp);
    free_ooc(c);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->ring_stream) cudaStreamDestroy(c->ring_stream);
    for (cudaEvent_t ev : {c->ev_march_done, c->ev_copy_done, c->ev_ring_start, c->ev_ring_end})
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : c->ev_chunk) cudaEventDestroy(ev);
    for (cudaEvent_t ev : c->ev_half_read)
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : c->ev_stage)
        if (ev) cudaEventDestroy(ev);
    delete c;
}

const char* vr_last_error(const vr_ctx* c) {
    if (!c) return "null context";
    return c->err.c_str();
}

int vr_load_cube(vr_ctx* c, const float* data, int64_t nx, int64_t ny, int64_t nz) {
    if (!c) return VR_EINVAL;
    if (!data) return fail(c, VR_EINVAL, "null cube");
    if (nx < 2 || ny < 2 || nz < 2 || nx > 65536 || ny > 65536 || nz > 65536)
        return fail(c, VR_EINVAL, "cube sizes must be in [2, 65536]");
    VR_CUDA(c, cudaSetDevice(c->device));
    int rc = retire_all(c);
    if (rc) return rc;
    const int64_t nx_pad = (nx + 3) / 4 * 4;
    const size_t bytes = (size_t)nx_pad * ny * nz * sizeof(float);
    cudaFree(c->d_cube);
    cudaFree(c->d_cube_xzy);
    c->d_cube = nullptr;
    c->d_cube_xzy = nullptr;
    c->bricked = false;
    c->tma_ready = false;
    c->tex_fits = -1;
    free_tex(c);
    free_ooc(c);
    if (cudaMalloc((void**)&c->d_cube, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, VR_ENOMEM, "cannot allocate the cube on the device");
    }
    if (nx_pad != nx) VR_CUDA(c, cudaMemset(c->d_cube, 0, bytes));
    VR_CUDA(c, cudaMemcpy2D(c->d_cube, nx_pad * sizeof(float), data, nx * sizeof(float), nx * sizeof(float),
                            (size_t)ny * nz, cudaMemcpyDefault));
    c->nx_pad = nx_pad;
    c->n[0] = nx;
    c->n[1] = ny;
    c->n[2] = nz;
    return VR_OK;
}

int vr_load_cube_host(vr_ctx* c, const float* data, int64_t nx, int64_t ny, int64_t nz) {
    if (!c) return VR_EINVAL;
    if (!data) return fail(c, VR_EINVAL, "null cube");
    if (nx < 2 || ny < 2 || nz < 2 || nx > 65536 || ny > 65536 || nz > 65536)
        return fail(c, VR_EINVAL, "cube sizes must be in [2, 65536]");
    VR_CUDA(c, cudaSetDevice(c->device));
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, data) == cudaSuccess) {
        if (attr.type == cudaMemoryTypeDevice) return fail(c, VR_EINVAL, "vr_load_cube_host needs host memory");
    } else {
        cudaGetLastError();
    }
    int rc = retire_all(c);
    if (rc) return rc;
    cudaFree(c->d_cube);
    cudaFree(c->d_cube_xzy);
    c->d_cube = nullptr;
    c->d_cube_xzy = nullptr;
    c->bricked = false;
    c->tma_ready = false;
    c->tex_fits = -1;
    free_tex(c);
    free_ooc(c);
    if ((rc = ensure_ooc_streams(c))) return rc;
    c->ooc = true;
    c->h_src = data;
    c->nx_pad = nx;
    c->n[0] = nx;
    c->n[1] = ny;
    c->n[2] = nz;
    return VR_OK;
}

int vr_load_cube_provider(vr_ctx* c, vr_block_provider fn, void* user, int64_t nx, int64_t ny, int64_t nz) {
    if (!c) return VR_EINVAL;
    if (!fn) return fail(c, VR_EINVAL, "null brick provider");
    if (nx < 2 || ny < 2 || nz < 2 || nx > 65536 || ny > 65536 || nz > 65536)
        return fail(c, VR_EINVAL, "cube sizes must be in [2, 65536]");
    VR_CUDA(c, cudaSetDevice(c->device));
    int rc = retire_all(c);
    if (rc) return rc;
    cudaFree(c->d_cube);
    cudaFree(c->d_cube_xzy);
    c->d_cube = nullptr;
    c->d_cube_xzy = nullptr;
    c->bricked = false;
    c->tma_ready = false;
    c->tex_fits = -1;
    free_tex(c);
    free_ooc(c);
    if ((rc = ensure_ooc_streams(c))) return rc;
    c->ooc = true;
    c->prov_fn = fn;
    c->prov_user = user;
    c->nx_pad = nx;
    c->n[0] = nx;
    c->n[1] = ny;
    c->n[2] = nz;
    return VR_OK;
}

int vr_load_cube_codec(vr_ctx* c, vr_codec* codec, int64_t nx, int64_t ny, int64_t nz) {
    if (!c) return VR_EINVAL;
    if (!codec) return fail(c, VR_EINVAL, "null codec");
    if (nx < 2 || ny < 2 || nz < 2 || nx > 65536 || ny > 65536 || nz > 65536)
        return fail(c, VR_EINVAL, "cube sizes must be in [2, 65536]");
    VR_CUDA(c, cudaSetDevice(c->device));
    int rc = retire_all(c);
    if (rc) return rc;
    cudaFree(c->d_cube);
    cudaFree(c->d_cube_xzy);
    c->d_cube = nullptr;
    c->d_cube_xzy = nullptr;
    c->bricked = false;
    c->tma_ready = false;
    c->tex_fits = -1;
    free_tex(c);
    free_ooc(c);
    if ((rc = ensure_ooc_streams(c))) return rc;
    c->ooc = true;
    c->codec = codec;
    c->nx_pad = nx;
    c->n[0] = nx;
    c->n[1] = ny;
    c->n[2] = nz;
    return VR_OK;
}

int vr_set_codec_fallback(vr_ctx* c, const float* data, float bound, float floor_v) {
    if (!c) return VR_EINVAL;
    if (!c->codec) return fail(c, VR_ESTATE, "the fallback needs a learned context (vr_load_cube_codec)");
    if (std::isnan(bound) || std::isnan(floor_v)) return fail(c, VR_EINVAL, "NaN bound or floor");
    c->fb_src = data;
    c->fb_fn = nullptr;
    c->fb_user = nullptr;
    c->fb_bound = bound;
    c->fb_floor = floor_v;
    return VR_OK;
}

int vr_set_codec_fallback_provider(vr_ctx* c, vr_block_provider fn, void* user, float bound, float floor_v) {
    if (!c) return VR_EINVAL;
    if (!c->codec) return fail(c, VR_ESTATE, "the fallback needs a learned context (vr_load_cube_codec)");
    if (std::isnan(bound) || std::isnan(floor_v)) return fail(c, VR_EINVAL, "NaN bound or floor");
    c->fb_src = nullptr;
    c->fb_fn = fn;
    c->fb_user = fn ? user : nullptr;
    c->fb_bound = bound;
    c->fb_floor = floor_v;
    return VR_OK;
}

int vr_codec_brick_errors(vr_ctx* c, float* err, int64_t* n_plain) {
    if (!c) return VR_EINVAL;
    if (!c->codec || !c->bricked || !c->fb_measured)
        return fail(c, VR_ESTATE, "no fallback scan: vr_set_codec_fallback, then vr_brick, on a learned context");
    if (err) std::copy(c->brick_err.begin(), c->brick_err.end(), err);
    if (n_plain) *n_plain = c->n_plain;
    return VR_OK;
}

int vr_brick(vr_ctx* c, int32_t bx, int32_t by, int32_t bz) {
    if (!c) return VR_EINVAL;
    if (!c->d_cube && !c->ooc) return fail(c, VR_ESTATE, "vr_brick before vr_load_cube");
    int32_t B[3] = {bx, by, bz};
    for (int a = 0; a < 3; ++a)
        if (B[a] < 1 || B[a] > 4096) return fail(c, VR_EINVAL, "brick sizes must be in [1, 4096]");
    VR_CUDA(c, cudaSetDevice(c->device));
    int rc = retire_all(c);
    if (rc) return rc;
    int64_t total = 1;
    for (int a = 0; a < 3; ++a) {
        c->B[a] = B[a];
        c->nb[a] = (int32_t)bricks_along(c->n[a], B[a]);
        total *= c->nb[a];
    }
    if (total > (1 << 26)) return fail(c, VR_EINVAL, "too many bricks");
    c->n_bricks = total;
    c->tma_ready = false;  // tensor maps are per brick
    if (c->precision == VR_PRECISION_F8) free_tex(c);  // so are the FP8 scales
    cudaFree(c->d_minmax);
    c->d_minmax = nullptr;
    c->h_minmax.resize(total);
    if (c->ooc) {
        if ((rc = build_ooc_store(c))) return rc;
    } else {
        if (cudaMalloc((void**)&c->d_minmax, total * sizeof(float2)) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, VR_ENOMEM, "cannot allocate brick min/max");
        }
        int32_t n32[3] = {(int32_t)c->n[0], (int32_t)c->n[1], (int32_t)c->n[2]};
        VR_CUDA(c, vr::launch_brick_minmax(c->d_cube, c->nx_pad, n32, c->B, c->nb, c->d_minmax, 0));
        VR_CUDA(c, cudaMemcpy(c->h_minmax.data(), c->d_minmax, total * sizeof(float2), cudaMemcpyDeviceToHost));
    }
    for (int a = 0; a < 3; ++a) {
        c->region_lo[a] = 0;
        c->region_hi[a] = c->nb[a];
    }
    c->bricked = true;
    return VR_OK;
}

}  // extern "C"

namespace vrh {

// Transposed copy and tensor maps for the TMA-staged march (built on first use).
int prepare_tma(vr_ctx* c) {
    if (c->tma_ready) return VR_OK;
    const int64_t nx = c->n[0], ny = c->n[1], nz = c->n[2];
    const int64_t ny_pad = (ny + 3) / 4 * 4;
    if (!c->d_cube_xzy) {
        const size_t bytes = (size_t)ny_pad * nz * nx * sizeof(float);
        if (cudaMalloc((void**)&c->d_cube_xzy, bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, VR_ENOMEM, "cannot allocate the transposed cube for the TMA march");
        }
        if (ny_pad != ny) VR_CUDA(c, cudaMemset(c->d_cube_xzy, 0, bytes));
        VR_CUDA(c, vr::launch_transpose_xzy(c->d_cube, nx, ny, nz, c->nx_pad, c->d_cube_xzy, ny_pad, 0));
        VR_CUDA(c, cudaDeviceSynchronize());
    }
    c->ny_pad = ny_pad;
    std::vector<CUtensorMap> maps;
    VR_CUDA(c, vr::make_tma_maps(c->d_cube, nx, ny, nz, c->nx_pad, c->d_cube_xzy, ny_pad, c->B, c->nb, maps,
                                 c->tmaps_per_brick));
    cudaFree(c->d_tmaps);
    c->d_tmaps = nullptr;
    if (cudaMalloc((void**)&c->d_tmaps, maps.size() * sizeof(CUtensorMap)) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, VR_ENOMEM, "cannot allocate tensor maps");
    }
    VR_CUDA(c, cudaMemcpy(c->d_tmaps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
    c->tma_ready = true;
    return VR_OK;
}

// Layered texture copies for the texture-gather march (built on first use): the copy
// for sweeps along axis S has layers along S and texels over the two other axes.
int prepare_tex(vr_ctx* c) {
    if (c->tex_ready) return VR_OK;
    int maxw = 0, maxh = 0, maxl = 0;
    VR_CUDA(c, cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxTexture2DLayeredWidth, c->device));
    VR_CUDA(c, cudaDeviceGetAttribute(&maxh, cudaDevAttrMaxTexture2DLayeredHeight, c->device));
    VR_CUDA(c, cudaDeviceGetAttribute(&maxl, cudaDevAttrMaxTexture2DLayeredLayers, c->device));
    const int64_t* n = c->n;
    if (n[1] > 65535 || n[2] > 65535) return fail(c, VR_EINVAL, "cube too large for the texture march");
    for (int S = 0; S < 3; ++S) {
        const int U = S == 0 ? 1 : 0, V = S == 2 ? 1 : 2;
        const int32_t K = tex_slab_bricks(c, S, maxl);
        if (n[U] > maxw || n[V] > maxh || K == 0 || (c->nb[S] + K - 1) / K > vr::kMaxTexSlabs)
            return fail(c, VR_EINVAL, "cube exceeds the layered-texture limits of this device");
    }
    if (c->precision == VR_PRECISION_F16)
        for (const float2& mm : c->h_minmax)
            if (mm.x < -65504.0f || mm.y > 65504.0f)
                return fail(c, VR_EINVAL, "FP16 storage: the cube has values beyond the FP16 range");
    const int prec = c->precision == VR_PRECISION_F8 ? vr::kPrecF8
                     : c->precision == VR_PRECISION_F16 ? vr::kPrecF16 : vr::kPrecF32;
    free_tex(c);
    if (c->precision == VR_PRECISION_F8) {
        if (cudaMalloc((void**)&c->d_brick_scale, c->n_bricks * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, VR_ENOMEM, "cannot allocate the brick scales");
        }
        VR_CUDA(c, vr::launch_brick_scale(c->d_cube, n[0], n[1], n[2], c->nx_pad, c->B, c->nb, c->d_brick_scale, 0));
    }
    for (int S = 0; S < 3; ++S) {
        const int U = S == 0 ? 1 : 0, V = S == 2 ? 1 : 2;
        cudaChannelFormatDesc ch = c->precision == VR_PRECISION_F16 ? cudaCreateChannelDescHalf()
                                   : c->precision == VR_PRECISION_F8 ? cudaCreateChannelDesc<signed char>()
                                                                     : cudaCreateChannelDesc<float>();
        const int32_t K = tex_slab_bricks(c, S, maxl);
        c->tex_slab_bricks[S] = K;
        const int64_t n_slabs = (c->nb[S] + K - 1) / K;
        for (int64_t j = 0; j < n_slabs; ++j) {
            const int64_t l0 = j * K * c->B[S];
            const int64_t l1 = std::min<int64_t>((j + 1) * K * c->B[S], n[S] - 1);  // apron included
            if (cudaMalloc3DArray(&c->tex_arr[S][j], &ch,
                                  make_cudaExtent((size_t)n[U], (size_t)n[V], (size_t)(l1 - l0 + 1)),
                                  cudaArrayLayered | cudaArraySurfaceLoadStore) != cudaSuccess) {
                cudaGetLastError();
                free_tex(c);
                return fail(c, VR_ENOMEM, "cannot allocate the layered textures");
            }
            cudaResourceDesc rd;
            std::memset(&rd, 0, sizeof(rd));
            rd.resType = cudaResourceTypeArray;
            rd.res.array.array = c->tex_arr[S][j];
            cudaSurfaceObject_t surf = 0;
            VR_CUDA(c, cudaCreateSurfaceObject(&surf, &rd));
            cudaError_t e = vr::fill_tex_layers(c->d_cube, n[0], n[1], n[2], c->nx_pad, S, l0, l1 - l0 + 1, prec,
                                                surf, c->d_brick_scale, c->B, c->nb, 0);
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
            cudaDestroySurfaceObject(surf);
            if (e != cudaSuccess) return cuda_fail(c, e, "fill_tex_layers");
            cudaTextureDesc td;
            std::memset(&td, 0, sizeof(td));
            td.addressMode[0] = td.addressMode[1] = td.addressMode[2] = cudaAddressModeClamp;
            td.filterMode = cudaFilterModePoint;
            td.readMode = cudaReadModeElementType;
            td.normalizedCoords = 0;
            VR_CUDA(c, cudaCreateTextureObject(&c->tex_obj[S][j], &rd, &td, nullptr));
        }
    }
    if (c->precision != VR_PRECISION_F32) {
        float2* d_mm = nullptr;
        if (cudaMalloc((void**)&d_mm, c->n_bricks * sizeof(float2)) != cudaSuccess) {
            cudaGetLastError();
            free_tex(c);
            return fail(c, VR_ENOMEM, "cannot allocate the stored-value min/max");
        }
        const int32_t n32[3] = {(int32_t)n[0], (int32_t)n[1], (int32_t)n[2]};
        cudaError_t e = vr::launch_stored_minmax(c->d_cube, c->nx_pad, n32, c->B, c->nb, prec, c->d_brick_scale,
                                                 d_mm, 0);
        c->h_minmax_q.resize(c->n_bricks);
        if (e == cudaSuccess)
            e = cudaMemcpy(c->h_minmax_q.data(), d_mm, c->n_bricks * sizeof(float2), cudaMemcpyDeviceToHost);
        cudaFree(d_mm);
        if (e != cudaSuccess) return cuda_fail(c, e, "stored min/max");
    }
    c->tex_ready = true;
    return VR_OK;
}

}  // namespace vrh

extern "C" {

int vr_get_brick_minmax(vr_ctx* c, float* out, int64_t n_bricks) {
    if (!c) return VR_EINVAL;
    if (!c->bricked) return fail(c, VR_ESTATE, "no bricking");
    if (!out || n_bricks != c->n_bricks) return fail(c, VR_EINVAL, "n_bricks mismatch");
    std::memcpy(out, c->h_minmax.data(), n_bricks * sizeof(float2));
    return VR_OK;
}

int vr_set_transfer_function(vr_ctx* c, const double* pts, int32_t n) {
    if (!c) return VR_EINVAL;
    if (!pts || n < 2 || n > vr::kMaxTfPoints) return fail(c, VR_EINVAL, "need 2..256 control points");
    for (int i = 0; i < n; ++i) {
        for (int k = 0; k < 5; ++k)
            if (!std::isfinite(pts[5 * i + k])) return fail(c, VR_EINVAL, "non-finite control point");
        for (int k = 1; k < 5; ++k)
            if (pts[5 * i + k] < 0.0 || pts[5 * i + k] > 1.0)
                return fail(c, VR_EINVAL, "colour and opacity must be in [0, 1]");
        if (i > 0 && !(pts[5 * i] > pts[5 * (i - 1)]))
            return fail(c, VR_EINVAL, "control values must increase strictly");
    }
    c->tf.assign(pts, pts + 5 * n);
    c->tf_rgba.resize(n + 1);
    c->tf_v.resize(n);
    for (int i = 0; i < n; ++i) {
        c->tf_rgba[i] = make_float4((float)pts[5 * i + 1], (float)pts[5 * i + 2], (float)pts[5 * i + 3],
                                    (float)pts[5 * i + 4]);
        c->tf_v[i] = (float)pts[5 * i];
    }
    c->tf_rgba[n] = c->tf_rgba[n - 1];
    const double v0 = pts[0], dv = (pts[5 * (n - 1)] - pts[0]) / (n - 1);
    bool uniform = true;
    for (int i = 0; i < n; ++i)
        if (std::fabs(pts[5 * i] - (v0 + i * dv)) > 1e-9 * std::max(1.0, std::fabs(pts[5 * i])))
            uniform = false;
    c->tf_uniform = uniform ? 1 : 0;
    c->tf_v0 = (float)v0;
    c->tf_inv_dv = (float)(1.0 / dv);
    c->tf_set = true;
    return VR_OK;
}

int vr_set_camera(vr_ctx* c, const vr_camera* cam) {
    if (!c) return VR_EINVAL;
    if (!cam || !camera_valid(*cam)) return fail(c, VR_EINVAL, "invalid camera");
    Basis b;
    if (!make_basis(*cam, b)) return fail(c, VR_EINVAL, "degenerate camera basis (eye == target or up parallel to view)");
    c->q.resize((size_t)cam->width + cam->height);
    for (int i = 0; i < cam->width; ++i)
        c->q[i] = vr::df_from_double((2.0 * (i + 0.5) / cam->width - 1.0) * b.tan_half * b.aspect);
    for (int j = 0; j < cam->height; ++j)
        c->q[cam->width + j] = vr::df_from_double((1.0 - 2.0 * (j + 0.5) / cam->height) * b.tan_half);
    if (!c->cam_set || cam->step != c->cam.step)
    {
        static const double long_splits[] = {0.5, 0.4, 0.3, 0.25, 0.2};
        static const double short_splits[] = {0.1, 0.08, 0.06, 0.04, 0.02};
        c->alpha_split = vr::fit_alpha(cam->step / 1.0, long_splits, vr::kAlphaPolyTerms, c->alpha_poly, 5e-10);
        c->small_split = vr::fit_alpha(cam->step / 1.0, short_splits, vr::kAlphaSmallTerms, c->alpha_small, 5e-10);
    }
    c->cam = *cam;
    c->basis = b;
    c->cam_set = true;
    return VR_OK;
}

int vr_camera_from_matrices(const double view[16], const double proj[16], int32_t width, int32_t height,
                            double step, double term_alpha, vr_camera* out) {
    if (!view || !proj || !out || width < 1 || height < 1) return VR_EINVAL;
    for (int k = 0; k < 16; ++k)
        if (!std::isfinite(view[k]) || !std::isfinite(proj[k])) return VR_EINVAL;
    // rows of the rotation R (column-major: element (r, c) at [4c + r]) and t
    double R[3][3], t[3];
    for (int r = 0; r < 3; ++r) {
        for (int cc = 0; cc < 3; ++cc) R[r][cc] = view[4 * cc + r];
        t[r] = view[12 + r];
    }
    if (view[3] != 0.0 || view[7] != 0.0 || view[11] != 0.0 || view[15] != 1.0) return VR_EINVAL;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const double dot = R[a][0] * R[b][0] + R[a][1] * R[b][1] + R[a][2] * R[b][2];
            if (std::fabs(dot - (a == b ? 1.0 : 0.0)) > 1e-6) return VR_EINVAL;
        }
    // a symmetric perspective projection with square pixels
    const double p0 = proj[0], p5 = proj[5];
    if (!(p0 > 0.0) || !(p5 > 0.0) || proj[1] != 0.0 || proj[4] != 0.0 || proj[8] != 0.0 || proj[9] != 0.0 ||
        proj[11] != -1.0 || proj[15] != 0.0 || proj[3] != 0.0 || proj[7] != 0.0 || proj[2] != 0.0 ||
        proj[6] != 0.0)
        return VR_EINVAL;
    const double aspect = p5 / p0;
    if (std::fabs(aspect - (double)width / height) > 1e-6 * ((double)width / height)) return VR_EINVAL;
    vr_camera cam{};
    for (int a = 0; a < 3; ++a) {
        // eye = -R^T t; forward = -(third row), up = second row
        cam.eye[a] = -(R[0][a] * t[0] + R[1][a] * t[1] + R[2][a] * t[2]);
        cam.target[a] = cam.eye[a] - R[2][a];
        cam.up[a] = R[1][a];
    }
    cam.fovy_deg = 2.0 * std::atan(1.0 / p5) * (180.0 / M_PI);
    cam.width = width;
    cam.height = height;
    cam.step = step;
    cam.term_alpha = term_alpha;
    *out = cam;
    return VR_OK;
}

int vr_set_camera_matrices(vr_ctx* c, const double view[16], const double proj[16], int32_t width, int32_t height,
                           double step, double term_alpha) {
    if (!c) return VR_EINVAL;
    vr_camera cam;
    if (vr_camera_from_matrices(view, proj, width, height, step, term_alpha, &cam))
        return fail(c, VR_EINVAL, "the matrices are not a rigid view and a symmetric perspective with square pixels");
    return vr_set_camera(c, &cam);
}

int vr_set_option(vr_ctx* c, int32_t option, int64_t value) {
    if (!c) return VR_EINVAL;
    switch (option) {
        case VR_OPT_SKIP_EMPTY: c->skip_empty = value != 0; return VR_OK;
        case VR_OPT_RECT_CULL: c->rect_cull = value != 0; return VR_OK;
        case VR_OPT_MODE:
            if (value != 0 && value != 1) return fail(c, VR_EINVAL, "mode must be 0 or 1");
            c->mode = (int)value;
            return VR_OK;
        case VR_OPT_KERNEL:
            if (value != VR_KERNEL_AUTO && value != VR_KERNEL_TMA && value != VR_KERNEL_DIRECT &&
                value != VR_KERNEL_TEX)
                return fail(c, VR_EINVAL, "unknown kernel");
            c->kernel = (int)value;
            return VR_OK;
        case VR_OPT_DEVICE_BUDGET: c->budget = value; return VR_OK;
        case VR_OPT_HOST_OUTPUT_ASYNC:
            if (value != 0 && value != 1) return fail(c, VR_EINVAL, "asynchronous host output must be 0 or 1");
            c->host_async = value != 0;
            return VR_OK;
        case VR_OPT_PROVIDER_THREADS: c->prov_threads = (int)std::max<int64_t>(0, std::min<int64_t>(value, 4096)); return VR_OK;
        case VR_OPT_OOC_MARCH:
            if (value < 0 || value > 4) return fail(c, VR_EINVAL, "out-of-core march must be 0, 1, 2, 3 or 4");
            c->ooc_march = (int)value;
            return VR_OK;
        case VR_OPT_TEX_SLAB_LAYERS:
            if (value < 0) return fail(c, VR_EINVAL, "layers per texture slab must be >= 0");
            if (value != c->tex_slab_layers) {
                int rc = retire_all(c);  // frames in flight may read the old textures
                if (rc) return rc;
                free_tex(c);
                c->tex_slab_layers = value;
                c->tex_fits = -1;
            }
            return VR_OK;
        case VR_OPT_STEP_MODE:
            if (value != 0 && value != 1) return fail(c, VR_EINVAL, "step mode must be 0 or 1");
            c->step_mode = (int)value;
            return VR_OK;
        case VR_OPT_PRECISION:
            if (value != VR_PRECISION_F32 && value != VR_PRECISION_F16 && value != VR_PRECISION_F8)
                return fail(c, VR_EINVAL, "unknown precision");
            if ((int)value != c->precision) {
                int rc = retire_all(c);  // frames in flight may read the old textures
                if (rc) return rc;
                free_tex(c);
                c->precision = (int)value;
            }
            return VR_OK;
        default: return fail(c, VR_EINVAL, "unknown option");
    }
}

}  // extern "C"

namespace vrh {

// The frame parameters that do not depend on the camera or the frame's buffers:
// cube, bricking, step, termination, transfer-function scalars, opacity-correction
// fits, mode, storage.  Everything else is zero.
void fill_common_params(vr_ctx* c, vr::FrameParams& p) {
    std::memset(&p, 0, sizeof(p));
    for (int a = 0; a < 3; ++a) {
        p.n[a] = (int32_t)c->n[a];
        p.B[a] = c->B[a];
        p.nb[a] = c->nb[a];
    }
    p.dt = vr::df_from_double(c->cam.step);
    p.inv_dt = vr::df_from_double(1.0 / c->cam.step);
    p.dt_f = (float)c->cam.step;
    p.step_mode = c->step_mode;
    p.tau = (float)c->cam.term_alpha;
    p.cube = c->d_cube;
    p.stride_y = c->nx_pad;
    p.stride_z = c->nx_pad * c->n[1];
    p.offsets32 = ((int64_t)c->B[2] + 1) * p.stride_z + ((int64_t)c->B[1] + 1) * p.stride_y +
                      c->B[0] + 1 < ((int64_t)1 << 32) ? 1 : 0;
    p.tf_n = (int32_t)(c->tf.size() / 5);
    p.tf_uniform = c->tf_uniform;
    p.tf_v0 = c->tf_v0;
    p.tf_inv_dv = c->tf_inv_dv;
    std::memcpy(p.alpha_poly, c->alpha_poly, sizeof(p.alpha_poly));
    p.alpha_split = (float)c->alpha_split;
    p.poly_scale = (float)(2.0 / c->alpha_split);
    std::memcpy(p.alpha_small, c->alpha_small, sizeof(p.alpha_small));
    p.small_split = (float)c->small_split;
    p.small_scale = (float)(2.0 / c->small_split);
    p.mode = c->mode;
    p.gmax = FLT_MAX;
    for (const float2& mm : c->h_minmax) p.gmax = p.gmax == FLT_MAX ? mm.y : std::max(p.gmax, mm.y);
    p.tmaps = c->d_tmaps;
    p.tmaps_per_brick = c->tmaps_per_brick;
    for (int a = 0; a < 3; ++a) {
        for (int j = 0; j < vr::kMaxTexSlabs; ++j) p.tex[a][j] = c->tex_obj[a][j];
        p.tex_slab_bricks[a] = c->tex_slab_bricks[a];
    }
    p.precision = c->precision == VR_PRECISION_F8 ? vr::kPrecF8
                  : c->precision == VR_PRECISION_F16 ? vr::kPrecF16 : vr::kPrecF32;
    p.brick_scale = c->d_brick_scale;
}

// Out-of-core frame: cache slots for the frame's bricks, the slot table, the
// march launches, each a contiguous range of items with the bricks it must wait
// for: first the items of resident bricks (no wait), then bricks copied into
// resident slots in groups of about 64 MiB, then bricks streamed through the ring,
// one launch per half-ring; and the items, written straight into that order.
struct OocLaunch {
    int64_t lo, hi;             // items [lo, hi)
    std::vector<int32_t> up;    // bricks (ids) to copy before the launch
    std::vector<int32_t> slot;  // and their slots
    int32_t half = -1;          // ring half the bricks go to (-1: resident slots)
};

int ooc_prepare(vr_ctx* c, Slot& s, int32_t tiles_x, int32_t tiles_y, int64_t n_items,
                std::vector<OocLaunch>& launches) {
    const int32_t P = (int32_t)c->plan_bricks.size();
    c->ooc_bricks.resize(P);
    int64_t total = 0;
    for (int32_t k = 0; k < P; ++k) {
        c->ooc_bricks[k] = c->plan_bricks[k].id;
        total += c->plan_bricks[k].n_items;
    }
    if (total != n_items) return fail(c, VR_EINVAL, "internal: out-of-core item count mismatch");
    const int32_t H = vr::plan_residency(c->res, c->ooc_bricks, c->ooc_frame++, c->ring_first_half, c->ooc_slot,
                                         c->ooc_up, c->ooc_ring);
    int rc = grow_pinned(c, s.h_slot_of, s.cap_slot_of, (size_t)c->n_bricks);
    if (rc) return rc;
    if ((rc = grow_device(c, s.d_slot_of, s.dcap_slot_of, (size_t)c->n_bricks))) return rc;
    std::fill(s.h_slot_of, s.h_slot_of + c->n_bricks, -1);
    for (int32_t k = 0; k < P; ++k) s.h_slot_of[c->ooc_bricks[k]] = c->ooc_slot[k];
    // where each brick's items go: resident hits, then the uploads, then the ring
    c->plan_dst.assign(P, -1);
    for (int32_t k : c->ooc_up) c->plan_dst[k] = -2;
    for (int32_t k : c->ooc_ring) c->plan_dst[k] = -2;
    int64_t w = 0;
    auto take = [&](int32_t k, OocLaunch* L) {
        c->plan_dst[k] = w;
        w += c->plan_bricks[k].n_items;
        if (L) {
            L->up.push_back(c->ooc_bricks[k]);
            L->slot.push_back(c->ooc_slot[k]);
        }
    };
    launches.clear();
    OocLaunch hits;
    hits.lo = 0;
    for (int32_t k = 0; k < P; ++k)
        if (c->plan_dst[k] == -1) take(k, nullptr);
    hits.hi = w;
    launches.push_back(std::move(hits));
    const size_t slot_bytes = (size_t)c->slot_floats * sizeof(float);
    size_t group = std::max<size_t>(1, ((size_t)64 << 20) / slot_bytes);
    if (c->pool_stage > 0) group = std::min(group, (size_t)c->pool_stage);  // one staging area's blocks
    if (c->pool_stage > 0 && H > c->pool_stage) return fail(c, VR_EINVAL, "internal: ring half larger than the staging");
    for (size_t g0 = 0; g0 < c->ooc_up.size(); g0 += group) {
        OocLaunch L;
        L.lo = w;
        for (size_t g = g0; g < std::min(c->ooc_up.size(), g0 + group); ++g) take(c->ooc_up[g], &L);
        L.hi = w;
        launches.push_back(std::move(L));
    }
    int32_t halves = 0;
    for (size_t g0 = 0; g0 < c->ooc_ring.size(); g0 += (size_t)H, ++halves) {
        OocLaunch L;
        L.lo = w;
        L.half = (c->ring_first_half + halves) % 2;
        for (size_t g = g0; g < std::min(c->ooc_ring.size(), g0 + (size_t)H); ++g) take(c->ooc_ring[g], &L);
        L.hi = w;
        launches.push_back(std::move(L));
    }
    c->ring_first_half = (c->ring_first_half + halves) % 2;
    emit_items(c, s, tiles_x, tiles_y, n_items);
    s.bricks_uploaded = (int64_t)(c->ooc_up.size() + c->ooc_ring.size());
    s.bricks_cached = P - s.bricks_uploaded;
    return VR_OK;
}

// Fill the bricks' cache slots on the copy stream: copy them from the pinned
// store, or decode them (learned residency; list_off: where this launch's
// (brick, slot) lists sit in the frame's list buffers).
// Returns the bytes copied from host memory in *copied.
int ooc_upload(vr_ctx* c, Slot& s, const OocLaunch& L, size_t list_off, size_t* copied) {
    const size_t slot_bytes = (size_t)c->slot_floats * sizeof(float);
    *copied = 0;
    // where brick k of the launch lands: its slot's block, or (texture march) block
    // k of the staging area, from which its layered copies are filled
    if (c->pool_stage > 0 && (int64_t)L.up.size() > c->pool_stage)
        return fail(c, VR_EINVAL, "internal: upload group larger than the staging");
    auto dst = [&](size_t k) -> int32_t { return c->pool_stage > 0 ? (int32_t)k : L.slot[k]; };
    if (c->codec) {
        // fallback bricks are copied from their plain blocks, the others decoded
        int32_t* lb = s.h_decode + list_off;
        size_t n = 0;
        for (size_t k = 0; k < L.up.size(); ++k) {
            const int64_t pi = c->plain_index.empty() ? -1 : c->plain_index[L.up[k]];
            if (pi >= 0) {
                VR_CUDA(c, cudaMemcpyAsync(c->d_pool + (size_t)dst(k) * c->slot_floats,
                                           c->h_store + (size_t)pi * c->slot_floats, slot_bytes,
                                           cudaMemcpyHostToDevice, c->copy_stream));
                *copied += slot_bytes;
            } else {
                lb[n++] = L.up[k];
            }
        }
        if (n == 0) return VR_OK;
        size_t m = 0;
        for (size_t k = 0; k < L.up.size(); ++k)
            if (c->plain_index.empty() || c->plain_index[L.up[k]] < 0) lb[n + m++] = dst(k);
        VR_CUDA(c, cudaMemcpyAsync(s.d_decode + list_off, lb, 2 * n * sizeof(int32_t), cudaMemcpyHostToDevice,
                                   c->copy_stream));
        const int rc = vr_codec_decode_bricks(c->codec, s.d_decode + list_off, s.d_decode + list_off + n, (int32_t)n,
                                              c->d_pool, c->copy_stream);
        if (rc) return fail(c, rc, "brick decode failed");
        return VR_OK;
    }
    if (c->prov_fn) {
        // the provider fills a staging buffer whose earlier copies have finished
        const int j = c->stage_next;
        c->stage_next = (j + 1) % vr_ctx::kStage;
        if (L.up.size() * slot_bytes > c->stage_cap) return fail(c, VR_EINVAL, "internal: upload group too large");
        VR_CUDA(c, cudaEventSynchronize(c->ev_stage[j]));
        int64_t bad = -1;
        if (vr::read_blocks(brick_source(c), c->n, c->B, c->nb, L.up.data(), (int64_t)L.up.size(), c->h_stage[j],
                            c->slot_floats, nullptr, &bad))
            return source_fail(c, bad);
        for (size_t k = 0; k < L.up.size(); ++k)
            VR_CUDA(c, cudaMemcpyAsync(c->d_pool + (size_t)dst(k) * c->slot_floats,
                                       c->h_stage[j] + k * c->slot_floats, slot_bytes, cudaMemcpyHostToDevice,
                                       c->copy_stream));
        VR_CUDA(c, cudaEventRecord(c->ev_stage[j], c->copy_stream));
        *copied = L.up.size() * slot_bytes;
        return VR_OK;
    }
    for (size_t k = 0; k < L.up.size(); ++k)
        VR_CUDA(c, cudaMemcpyAsync(c->d_pool + (size_t)dst(k) * c->slot_floats,
                                   c->h_store + (size_t)L.up[k] * c->slot_floats, slot_bytes,
                                   cudaMemcpyHostToDevice, c->copy_stream));
    *copied = L.up.size() * slot_bytes;
    return VR_OK;
}

// A frame whose provider failed: let the work already issued finish (it reads the
// frame's buffers), and forget the resident slots this frame was to fill, so
// that the next frame asks for those bricks again.
int abort_frame(vr_ctx* c, cudaStream_t st, const std::vector<OocLaunch>& launches, int rc) {
    cudaStreamSynchronize(st);
    cudaStreamSynchronize(c->copy_stream);
    cudaStreamSynchronize(c->ring_stream);
    for (const OocLaunch& L : launches)
        if (L.half < 0)
            for (size_t k = 0; k < L.up.size(); ++k) {
                const int32_t b = L.up[k], sl = L.slot[k];
                if (c->res.slot_of_brick[b] == sl) c->res.slot_of_brick[b] = -1;
                if (c->res.brick_in_slot[sl] == b) c->res.brick_in_slot[sl] = -1;
            }
    return rc;
}

int ensure_events(vr_ctx* c, std::vector<cudaEvent_t>& ev, size_t n) {
    while (ev.size() < n) {
        cudaEvent_t e;
        VR_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ev.push_back(e);
    }
    return VR_OK;
}

// One frame into the output window win = {x0, y0, x1, y1} (inclusive) of the image;
// out_rgba holds the window's pixels row-major.
int render_impl(vr_ctx* c, float* out_rgba, void* stream_ptr, const int32_t win[4]) {
    VR_CUDA(c, cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream_ptr;
    cudaPointerAttributes attr;
    bool out_on_device = false, out_pinned = false;
    if (cudaPointerGetAttributes(&attr, out_rgba) == cudaSuccess) {
        out_on_device = attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
        out_pinned = attr.type == cudaMemoryTypeHost;
    } else {
        cudaGetLastError();
    }
    if (c->host_async && !out_on_device && !out_pinned)
        return fail(c, VR_EINVAL, "asynchronous host output needs page-locked host memory");

    Slot& s = c->slots[c->next_slot];
    c->next_slot = (c->next_slot + 1) % kSlots;
    int rc = retire(c, s);
    if (rc) return rc;

    auto t0 = std::chrono::steady_clock::now();
    int32_t tiles_x, tiles_y, T;
    int64_t n_items;
    if (c->step_mode && c->kernel == VR_KERNEL_TMA)
        return fail(c, VR_EINVAL, "the dynamic step needs the texture or the direct march");
    if (c->precision != VR_PRECISION_F32 && !use_tex(c))
        return fail(c, VR_EINVAL, "FP16/FP8 storage needs the texture march (emission-absorption mode, "
                                  "VR_KERNEL_TEX or VR_KERNEL_AUTO on a cube within the texture limits)");
    if (use_tma(c) && (rc = prepare_tma(c))) return rc;
    if (use_tex(c) && (rc = prepare_tex(c))) return rc;
    rc = plan_frame(c, s, win, tiles_x, tiles_y, T, n_items, !c->ooc);
    if (rc) return rc;
    std::vector<OocLaunch> ooc_launches;
    s.bricks_uploaded = s.bricks_cached = 0;
    if (c->ooc && (rc = ooc_prepare(c, s, tiles_x, tiles_y, n_items, ooc_launches))) return rc;
    s.plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    const int64_t n_tiles = (int64_t)tiles_x * tiles_y;
    const size_t img_px = (size_t)(win[2] - win[0] + 1) * (size_t)(win[3] - win[1] + 1);

    if ((rc = grow_device(c, s.d_items, s.dcap_items, (size_t)std::max<int64_t>(n_items, 1)))) return rc;
    if ((rc = grow_device(c, s.d_tile_start, s.dcap_tiles, (size_t)n_tiles + 1))) return rc;
    if ((rc = grow_device(c, s.d_frags, s.cap_frags, (size_t)std::max<int64_t>(n_items, 1) * T * T)))
        return rc;
    if (!out_on_device && (rc = grow_device(c, s.d_img, s.cap_img, img_px))) return rc;
    // per-frame constants: camera tables (df) and the transfer function
    const size_t q_bytes = c->q.size() * sizeof(df);
    const size_t tf_rgba_off = (q_bytes + 15) / 16 * 16;
    const size_t tf_v_off = tf_rgba_off + c->tf_rgba.size() * sizeof(float4);
    const size_t frame_bytes = tf_v_off + c->tf_v.size() * sizeof(float);
    if ((rc = grow_pinned(c, s.h_frame, s.cap_frame, frame_bytes))) return rc;
    if ((rc = grow_device(c, s.d_frame, s.dcap_frame, frame_bytes))) return rc;
    std::memcpy(s.h_frame, c->q.data(), q_bytes);
    std::memcpy(s.h_frame + tf_rgba_off, c->tf_rgba.data(), c->tf_rgba.size() * sizeof(float4));
    std::memcpy(s.h_frame + tf_v_off, c->tf_v.data(), c->tf_v.size() * sizeof(float));

    vr::FrameParams p;
    fill_common_params(c, p);
    for (int a = 0; a < 3; ++a) {
        p.eye[a] = vr::df_from_double(c->cam.eye[a]);
        p.f[a] = vr::df_from_double(c->basis.f[a]);
        p.r[a] = vr::df_from_double(c->basis.r[a]);
        p.u[a] = vr::df_from_double(c->basis.u[a]);
    }
    p.qx = reinterpret_cast<const df*>(s.d_frame);
    p.qy = reinterpret_cast<const df*>(s.d_frame) + c->cam.width;
    p.width = c->cam.width;
    p.height = c->cam.height;
    p.tiles_x = tiles_x;
    p.tiles_y = tiles_y;
    p.tile = T;
    if (c->ooc) {
        p.pool = c->d_pool;
        p.slot_of = s.d_slot_of;
        p.slot_stride = c->slot_floats;
        p.pool_sy = c->B[0] + 1;
        p.pool_sz = (c->B[0] + 1) * (c->B[1] + 1);
        for (int a = 0; a < 3; ++a) {
            p.pool_tex[a] = c->pool_tex[a];
            p.pool_cols[a] = c->pool_cols[a];
        }
    }
    p.tf_rgba = reinterpret_cast<const float4*>(s.d_frame + tf_rgba_off);
    p.tf_v = reinterpret_cast<const float*>(s.d_frame + tf_v_off);
    p.items = s.d_items;
    p.n_items = (int32_t)n_items;
    p.tile_start = s.d_tile_start;
    p.frags = s.d_frags;
    p.out = out_on_device ? reinterpret_cast<float4*>(out_rgba) : s.d_img;
    p.out_x0 = win[0];
    p.out_y0 = win[1];
    p.out_w = win[2] - win[0] + 1;
    p.out_h = win[3] - win[1] + 1;
    p.stats = s.d_stats;

    VR_CUDA(c, cudaEventRecord(s.ev_begin, st));
    VR_CUDA(c, cudaMemcpyAsync(s.d_frame, s.h_frame, frame_bytes, cudaMemcpyHostToDevice, st));
    VR_CUDA(c, cudaMemcpyAsync(s.d_items, s.h_items, (size_t)n_items * sizeof(vr::Item),
                               cudaMemcpyHostToDevice, st));
    VR_CUDA(c, cudaMemcpyAsync(s.d_tile_start, s.h_tile_start, ((size_t)n_tiles + 1) * sizeof(int32_t),
                               cudaMemcpyHostToDevice, st));
    VR_CUDA(c, cudaMemsetAsync(s.d_stats, 0, sizeof(vr::Stats), st));
    int64_t march_launches = n_items > 0 ? 1 : 0;
    size_t upload_bytes = 0;
    if (c->ooc) {
        p.offsets32 = c->slot_floats < ((int64_t)1 << 32) ? 1 : 0;  // offsets inside one slot
        VR_CUDA(c, cudaMemcpyAsync(s.d_slot_of, s.h_slot_of, (size_t)c->n_bricks * sizeof(int32_t),
                                   cudaMemcpyHostToDevice, st));
        // this frame reads bricks that earlier frames copied into resident slots
        VR_CUDA(c, cudaStreamWaitEvent(st, c->ev_copy_done, 0));
        const size_t nl = ooc_launches.size();
        int rc2 = ensure_events(c, c->ev_chunk, nl);
        if (rc2) return rc2;
        // learned residency: room for every launch's (brick, slot) lists
        std::vector<size_t> list_off(nl + 1, 0);
        for (size_t k = 0; k < nl; ++k) list_off[k + 1] = list_off[k] + 2 * ooc_launches[k].up.size();
        if (c->codec) {
            if ((rc2 = grow_pinned(c, s.h_decode, s.cap_decode, std::max<size_t>(list_off[nl], 1)))) return rc2;
            if ((rc2 = grow_device(c, s.d_decode, s.dcap_decode, std::max<size_t>(list_off[nl], 1)))) return rc2;
        }
        // texture march: each launch's refilled slots, and one half-item counter per launch
        const bool pool_tex = use_pool_tex(c);
        if (pool_tex) {
            if ((rc2 = grow_pinned(c, s.h_fill, s.cap_fill, std::max<size_t>(list_off[nl] / 2, 1)))) return rc2;
            if ((rc2 = grow_device(c, s.d_fill, s.dcap_fill, std::max<size_t>(list_off[nl] / 2, 1)))) return rc2;
            if ((rc2 = grow_device(c, s.d_work, s.dcap_work, std::max<size_t>(nl, 1)))) return rc2;
            VR_CUDA(c, cudaMemsetAsync(s.d_work, 0, nl * sizeof(int32_t), st));
        }
        auto issue_upload = [&](size_t k) -> int {
            const OocLaunch& L = ooc_launches[k];
            if (L.up.empty()) return VR_OK;
            // a ring half is refilled once its last reader has marched (host issue
            // order puts that reader's event record before this wait)
            if (L.half >= 0) VR_CUDA(c, cudaStreamWaitEvent(c->copy_stream, c->ev_half_read[L.half], 0));
            size_t copied = 0;
            int r = ooc_upload(c, s, L, list_off[k], &copied);
            if (r) return r;
            upload_bytes += copied;
            if (pool_tex) {
                // the slots' layered copies, from their blocks
                int32_t* hf = s.h_fill + list_off[k] / 2;
                std::copy(L.slot.begin(), L.slot.end(), hf);
                VR_CUDA(c, cudaMemcpyAsync(s.d_fill + list_off[k] / 2, hf, L.slot.size() * sizeof(int32_t),
                                           cudaMemcpyHostToDevice, c->copy_stream));
                // (from the staging area, in launch order, on the copy stream: the next
                // launch's blocks overwrite it only after this fill)
                VR_CUDA(c, vr::fill_pool_tex(c->d_pool, c->slot_floats, s.d_fill + list_off[k] / 2,
                                             (int32_t)L.slot.size(), c->pool_stage > 0, c->B, c->pool_surf,
                                             c->pool_cols, c->copy_stream));
            }
            VR_CUDA(c, cudaEventRecord(c->ev_chunk[k], c->copy_stream));
            VR_CUDA(c, cudaEventRecord(c->ev_copy_done, c->copy_stream));
            return VR_OK;
        };
        // uploads into resident slots may overwrite bricks the previous frame still reads
        bool resident_uploads = false;
        for (const OocLaunch& L : ooc_launches) resident_uploads = resident_uploads || (L.half < 0 && !L.up.empty());
        if (resident_uploads) VR_CUDA(c, cudaStreamWaitEvent(c->copy_stream, c->ev_march_done, 0));
        // every resident upload at once (with a provider, each just before its own
        // launch, so that the host fills a group while the earlier ones march); the
        // ring two launches ahead of the march
        const bool lazy = c->prov_fn != nullptr;
        std::vector<size_t> ring_launches;
        for (size_t k = 0; k < nl; ++k) {
            if (ooc_launches[k].half < 0) {
                if (!lazy && (rc2 = issue_upload(k))) return abort_frame(c, st, ooc_launches, rc2);
            } else {
                ring_launches.push_back(k);
            }
        }
        size_t ring_issued = 0;
        while (ring_issued < std::min<size_t>(2, ring_launches.size()))
            if ((rc2 = issue_upload(ring_launches[ring_issued++]))) return abort_frame(c, st, ooc_launches, rc2);
        VR_CUDA(c, cudaEventRecord(s.ev_march0, st));
        // the streamed bricks march on their own stream, beside the resident ones,
        // so that waiting for a ring half never holds back the resident work
        const bool ring = !ring_launches.empty();
        if (ring) {
            VR_CUDA(c, cudaEventRecord(c->ev_ring_start, st));
            VR_CUDA(c, cudaStreamWaitEvent(c->ring_stream, c->ev_ring_start, 0));
        }
        march_launches = 0;
        for (size_t k = 0; k < nl; ++k) {
            const OocLaunch& L = ooc_launches[k];
            cudaStream_t ms = L.half >= 0 ? c->ring_stream : st;
            if (lazy && L.half < 0 && (rc2 = issue_upload(k))) return abort_frame(c, st, ooc_launches, rc2);
            if (!L.up.empty()) VR_CUDA(c, cudaStreamWaitEvent(ms, c->ev_chunk[k], 0));
            if (L.hi > L.lo) {
                vr::FrameParams q = p;
                q.items = s.d_items + L.lo;
                q.n_items = (int32_t)(L.hi - L.lo);
                if (pool_tex) {
                    q.work_next = s.d_work + k;
                    VR_CUDA(c, vr::launch_march_tex(q, ms));
                } else {
                    VR_CUDA(c, vr::launch_march(q, ms));
                }
                ++march_launches;
            }
            if (L.half >= 0) {
                VR_CUDA(c, cudaEventRecord(c->ev_half_read[L.half], ms));
                if (ring_issued < ring_launches.size())
                    if ((rc2 = issue_upload(ring_launches[ring_issued++])))
                        return abort_frame(c, st, ooc_launches, rc2);
            }
        }
        if (ring) {
            VR_CUDA(c, cudaEventRecord(c->ev_ring_end, c->ring_stream));
            VR_CUDA(c, cudaStreamWaitEvent(st, c->ev_ring_end, 0));
        }
        VR_CUDA(c, cudaEventRecord(c->ev_march_done, st));
    } else {
        VR_CUDA(c, cudaEventRecord(s.ev_march0, st));
        if (use_tma(c)) {
            VR_CUDA(c, vr::launch_march_tma(p, st));
        } else if (use_tex(c)) {
            VR_CUDA(c, vr::launch_march_tex(p, st));
        } else {
            VR_CUDA(c, vr::launch_march(p, st));
        }
    }
    VR_CUDA(c, cudaEventRecord(s.ev_march1, st));
    VR_CUDA(c, vr::launch_composite(p, st));
    VR_CUDA(c, cudaMemcpyAsync(s.h_stats, s.d_stats, sizeof(vr::Stats), cudaMemcpyDeviceToHost, st));
    VR_CUDA(c, cudaEventRecord(s.ev_end, st));
    s.pending = true;
    s.launches = march_launches + 1;
    s.fragments = n_items * T * T;
    s.h2d_bytes = (int64_t)(frame_bytes + (size_t)n_items * sizeof(vr::Item) +
                            ((size_t)n_tiles + 1) * sizeof(int32_t) + upload_bytes +
                            (c->ooc ? (size_t)c->n_bricks * sizeof(int32_t) : 0));
    s.d2h_bytes = (int64_t)sizeof(vr::Stats) + (out_on_device ? 0 : (int64_t)(img_px * sizeof(float4)));
    if (!out_on_device) {
        VR_CUDA(c, cudaMemcpyAsync(out_rgba, s.d_img, img_px * sizeof(float4), cudaMemcpyDeviceToHost, st));
        if (!c->host_async) VR_CUDA(c, cudaStreamSynchronize(st));
    }
    return VR_OK;
}

int render_checks(vr_ctx* c, const float* out_rgba) {
    if (!c) return VR_EINVAL;
    if ((!c->d_cube && !c->ooc) || !c->bricked || !c->tf_set || !c->cam_set)
        return fail(c, VR_ESTATE, "vr_render needs vr_load_cube, vr_brick, vr_set_transfer_function and vr_set_camera first");
    if (!out_rgba) return fail(c, VR_EINVAL, "null output");
    return VR_OK;
}

// Rendering rectangle of the brick range [lo, hi) (inclusive pixel bounds; x1 < x0
// when no pixel can see it).
void region_rect(const vr_camera& cam, const Basis& b, const int64_t n[3], const int32_t B[3],
                 const int32_t lo[3], const int32_t hi[3], int32_t rect[4]) {
    double blo[3], bhi[3];
    for (int a = 0; a < 3; ++a) {
        blo[a] = (double)lo[a] * B[a];
        bhi[a] = std::min((double)hi[a] * B[a], (double)(n[a] - 1));
    }
    box_rect(cam, b, blo, bhi, rect);
}

}  // namespace vrh

extern "C" {

int vr_render(vr_ctx* c, float* out_rgba, void* stream_ptr) {
    int rc = render_checks(c, out_rgba);
    if (rc) return rc;
    const int32_t win[4] = {0, 0, c->cam.width - 1, c->cam.height - 1};
    return render_impl(c, out_rgba, stream_ptr, win);
}

int vr_render_rect(vr_ctx* c, const int32_t rect[4], float* out_rgba, void* stream_ptr) {
    int rc = render_checks(c, out_rgba);
    if (rc) return rc;
    if (!rect) return fail(c, VR_EINVAL, "null rect");
    if (rect[2] < rect[0] || rect[3] < rect[1]) return VR_OK;  // empty: nothing to render
    if (rect[0] < 0 || rect[1] < 0 || rect[2] >= c->cam.width || rect[3] >= c->cam.height)
        return fail(c, VR_EINVAL, "rect outside the image");
    return render_impl(c, out_rgba, stream_ptr, rect);
}

int vr_set_region(vr_ctx* c, const int32_t lo[3], const int32_t hi[3]) {
    if (!c) return VR_EINVAL;
    if (!c->bricked) return fail(c, VR_ESTATE, "vr_set_region needs vr_brick first");
    if (!lo || !hi) return fail(c, VR_EINVAL, "null region");
    for (int a = 0; a < 3; ++a)
        if (lo[a] < 0 || hi[a] > c->nb[a] || lo[a] >= hi[a]) return fail(c, VR_EINVAL, "bad brick range");
    for (int a = 0; a < 3; ++a) {
        c->region_lo[a] = lo[a];
        c->region_hi[a] = hi[a];
    }
    return VR_OK;
}

int vr_region_rect(vr_ctx* c, int32_t rect[4]) {
    if (!c) return VR_EINVAL;
    if (!c->bricked || !c->cam_set) return fail(c, VR_ESTATE, "vr_region_rect needs vr_brick and vr_set_camera first");
    if (!rect) return fail(c, VR_EINVAL, "null rect");
    region_rect(c->cam, c->basis, c->n, c->B, c->region_lo, c->region_hi, rect);
    return VR_OK;
}

int vr_plan_region_rect(const vr_camera* cam, int64_t nx, int64_t ny, int64_t nz, const int32_t B[3],
                        const int32_t lo[3], const int32_t hi[3], int32_t rect[4]) {
    if (!cam || !B || !lo || !hi || !rect || !camera_valid(*cam)) return VR_EINVAL;
    if (nx < 2 || ny < 2 || nz < 2 || B[0] < 1 || B[1] < 1 || B[2] < 1) return VR_EINVAL;
    const int64_t n[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a)
        if (lo[a] < 0 || lo[a] >= hi[a] || hi[a] > bricks_along(n[a], B[a])) return VR_EINVAL;
    Basis b;
    if (!make_basis(*cam, b)) return VR_EINVAL;
    region_rect(*cam, b, n, B, lo, hi, rect);
    return VR_OK;
}

int vr_kd_partition(int64_t nx, int64_t ny, int64_t nz, const int32_t B[3], int32_t n_parts,
                    int32_t* ranges) {
    if (!B || !ranges || n_parts < 1 || nx < 2 || ny < 2 || nz < 2 || B[0] < 1 || B[1] < 1 || B[2] < 1)
        return VR_EINVAL;
    const int64_t n[3] = {nx, ny, nz};
    int64_t total = 1;
    for (int a = 0; a < 3; ++a) total *= bricks_along(n[a], B[a]);
    if (n_parts > total) return VR_EINVAL;
    return vr::kd_partition(n, B, n_parts, ranges) ? VR_OK : VR_EINVAL;
}

int vr_kd_order(int64_t nx, int64_t ny, int64_t nz, const int32_t B[3], int32_t n_parts, const double eye[3],
                int32_t* order) {
    if (!B || !eye || !order || n_parts < 1 || nx < 2 || ny < 2 || nz < 2 || B[0] < 1 || B[1] < 1 || B[2] < 1)
        return VR_EINVAL;
    const int64_t n[3] = {nx, ny, nz};
    int64_t total = 1;
    for (int a = 0; a < 3; ++a) total *= bricks_along(n[a], B[a]);
    if (n_parts > total) return VR_EINVAL;
    return vr::kd_order(n, B, n_parts, eye, order) ? VR_OK : VR_EINVAL;
}

int vr_composite_subimages(vr_ctx* c, int32_t n, const float* const* images, const int32_t* rects,
                           float* out_rgba, void* stream_ptr) {
    if (!c) return VR_EINVAL;
    if (!c->cam_set) return fail(c, VR_ESTATE, "vr_composite_subimages needs vr_set_camera first");
    if (n < 0 || n > vr::kMaxSubimages) return fail(c, VR_EINVAL, "1..256 sub-images");
    if (!out_rgba || (n > 0 && (!images || !rects))) return fail(c, VR_EINVAL, "null argument");
    VR_CUDA(c, cudaSetDevice(c->device));
    const int32_t W = c->cam.width, H = c->cam.height;
    vr::SubimageList L;
    std::memset(&L, 0, sizeof(L));
    for (int32_t k = 0; k < n; ++k) {
        const int32_t* r = rects + 4 * k;
        if (r[2] < r[0] || r[3] < r[1]) continue;  // an empty sub-image
        if (r[0] < 0 || r[1] < 0 || r[2] >= W || r[3] >= H) return fail(c, VR_EINVAL, "rect outside the image");
        if (!images[k]) return fail(c, VR_EINVAL, "null sub-image");
        vr::SubimageRef& e = L.s[L.n++];
        e.data = reinterpret_cast<const float4*>(images[k]);
        e.x0 = r[0];
        e.y0 = r[1];
        e.x1 = r[2];
        e.y1 = r[3];
    }
    cudaStream_t st = (cudaStream_t)stream_ptr;
    cudaPointerAttributes attr;
    bool out_on_device = false;
    if (cudaPointerGetAttributes(&attr, out_rgba) == cudaSuccess)
        out_on_device = attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
    else
        cudaGetLastError();
    const size_t px = (size_t)W * H;
    float4* dst = reinterpret_cast<float4*>(out_rgba);
    if (!out_on_device) {
        int rc = retire_all(c);  // d_comp may still be read by an earlier call's copy
        if (rc) return rc;
        if ((rc = grow_device(c, c->d_comp, c->cap_comp, px))) return rc;
        dst = c->d_comp;
    }
    VR_CUDA(c, vr::launch_subimage_composite(L, W, H, (float)c->cam.term_alpha, dst, st));
    if (!out_on_device) {
        VR_CUDA(c, cudaMemcpyAsync(out_rgba, dst, px * sizeof(float4), cudaMemcpyDeviceToHost, st));
        VR_CUDA(c, cudaStreamSynchronize(st));
    }
    return VR_OK;
}

int vr_get_stats(vr_ctx* c, vr_stats* out) {
    if (!c) return VR_EINVAL;
    if (!out) return fail(c, VR_EINVAL, "null stats");
    VR_CUDA(c, cudaSetDevice(c->device));
    int rc = retire_all(c);
    if (rc) return rc;
    *out = c->acc;
    return VR_OK;
}

int vr_reset_stats(vr_ctx* c) {
    if (!c) return VR_EINVAL;
    VR_CUDA(c, cudaSetDevice(c->device));
    int rc = retire_all(c);
    if (rc) return rc;
    std::memset(&c->acc, 0, sizeof(c->acc));
    return VR_OK;
}

int vr_plan_brick_rects(const vr_camera* cam, int64_t nx, int64_t ny, int64_t nz, int32_t bx,
                        int32_t by, int32_t bz, int32_t* rects, int64_t n_bricks) {
    if (!cam || !rects || !camera_valid(*cam)) return VR_EINVAL;
    if (nx < 2 || ny < 2 || nz < 2 || bx < 1 || by < 1 || bz < 1) return VR_EINVAL;
    Basis b;
    if (!make_basis(*cam, b)) return VR_EINVAL;
    const int64_t n[3] = {nx, ny, nz};
    const int32_t B[3] = {bx, by, bz};
    const int64_t nb[3] = {bricks_along(nx, bx), bricks_along(ny, by), bricks_along(nz, bz)};
    if (nb[0] * nb[1] * nb[2] != n_bricks) return VR_EINVAL;
    // the planner's computation (grid-corner projections, then each brick's box)
    std::vector<CornerProj> proj;
    project_brick_grid(*cam, b, n, B, nb, proj);
    for (int64_t id = 0; id < n_bricks; ++id) {
        int64_t idx[3] = {id % nb[0], (id / nb[0]) % nb[1], id / (nb[0] * nb[1])};
        brick_rect_from_grid(*cam, proj, nb, idx, rects + 4 * id);
    }
    return VR_OK;
}

int vr_plan_brick_tiles(const vr_camera* cam, int64_t nx, int64_t ny, int64_t nz, int32_t bx, int32_t by,
                        int32_t bz, uint8_t* mask, int64_t n_bricks, int64_t n_tiles) {
    if (!cam || !mask || !camera_valid(*cam)) return VR_EINVAL;
    if (nx < 2 || ny < 2 || nz < 2 || bx < 1 || by < 1 || bz < 1) return VR_EINVAL;
    Basis b;
    if (!make_basis(*cam, b)) return VR_EINVAL;
    const int64_t n[3] = {nx, ny, nz};
    const int32_t B[3] = {bx, by, bz};
    const int64_t nb[3] = {bricks_along(nx, bx), bricks_along(ny, by), bricks_along(nz, bz)};
    const int T = vr::kTile;
    const int64_t tiles_x = (cam->width + T - 1) / T, tiles_y = (cam->height + T - 1) / T;
    if (nb[0] * nb[1] * nb[2] != n_bricks || tiles_x * tiles_y != n_tiles) return VR_EINVAL;
    std::memset(mask, 0, (size_t)(n_bricks * n_tiles));
    // the planner's computation: grid-corner projections, rectangle, silhouette spans
    std::vector<CornerProj> proj;
    project_brick_grid(*cam, b, n, B, nb, proj);
    std::vector<Span> spans;
    for (int64_t id = 0; id < n_bricks; ++id) {
        const int64_t idx[3] = {id % nb[0], (id / nb[0]) % nb[1], id / (nb[0] * nb[1])};
        int32_t rect[4];
        if (!brick_rect_from_grid(*cam, proj, nb, idx, rect)) continue;
        const CornerProj* q[8];
        grid_corners(proj, nb, idx, q);
        spans.clear();
        brick_spans(q, rect, T, spans);
        for (const Span& sp : spans)
            for (int tx = sp.tx0; tx <= sp.tx1; ++tx) mask[id * n_tiles + (int64_t)sp.ty * tiles_x + tx] = 1;
    }
    return VR_OK;
}

}  // extern "C"
