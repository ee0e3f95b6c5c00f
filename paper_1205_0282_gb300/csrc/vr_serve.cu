// Serving loop (no counterpart in the paper, whose server renders one view at a
// time for one viewer): requests for frames (camera and resolution, optionally a
// new transfer function) arrive at any time; a worker thread admits them in
// arrival order into batches that fit half of a device arena, plans each frame
// (the planner of vr_render), and renders a whole batch with one texture-march
// launch over the items of all its frames and one composite launch over all its
// tiles.  Two batches can be in flight (one per arena half): the worker plans and
// uploads the next batch while the GPU renders the current one.  A completion
// thread waits for each batch's event and stamps its requests done.
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "vr_ctx.cuh"

using namespace vrh;

namespace {

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

enum ReqState { kQueued = 0, kRunning = 1, kDone = 2, kFailed = 3 };

// A transfer function as the march reads it: control points with the last one
// repeated, their values (the last repeated too), and the uniform spacing if any.
struct TfTable {
    std::vector<float4> rgba;
    std::vector<float> v;
    int32_t n = 0;
    bool uniform = false;
    float v0 = 0.0f, inv_dv = 0.0f;
    bool same(const TfTable& o) const {
        return n == o.n && std::memcmp(rgba.data(), o.rgba.data(), rgba.size() * sizeof(float4)) == 0 &&
               std::memcmp(v.data(), o.v.data(), v.size() * sizeof(float)) == 0;
    }
};

// Entries of all the transfer functions of one batch (shared memory of the march)
constexpr int32_t kBatchTfEntries = 512;

struct Req {
    int64_t id = 0;
    vr_camera cam{};
    std::vector<double> tf;  // empty: the transfer function in force
    float* out = nullptr;
    int state = kQueued;
    int err = VR_OK;
    double t_submit = 0, t_done = 0;
    // the frame's plan (made when the request is admitted)
    std::vector<vr::Item> items;
    std::vector<int32_t> tile_start;
    std::vector<df> q;
    double f[3], r[3], u[3];
    int32_t tiles_x = 0, tiles_y = 0;
    std::shared_ptr<const TfTable> tft;  // the transfer function it was planned with
    int32_t tf_slot = -1;                // its table in the batch
};

struct Batch {
    int half = -1;
    std::vector<Req*> reqs;
    int64_t items = 0;
    std::vector<const TfTable*> tfs;  // distinct transfer functions, in order of first use
    std::vector<int32_t> tf_off;      // their first entries in the concatenated tables
    int32_t tf_entries = 0;
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

struct vr_server {
    vr_ctx* c = nullptr;
    std::thread worker, completer;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_flight;
    bool stop = false, worker_done = false;
    std::deque<Req*> queue;
    std::unordered_map<int64_t, Req*> reqs;
    int64_t next_id = 1;
    int32_t max_batch = 64;
    std::string worker_err;  // a CUDA failure of the worker (the server stops serving)

    // arena: two halves, one per batch in flight
    size_t half_bytes = 0;
    char* d_arena[2] = {nullptr, nullptr};
    char* h_stage[2] = {nullptr, nullptr};
    vr::Stats* d_stats[2] = {nullptr, nullptr};
    vr::Stats* h_stats[2] = {nullptr, nullptr};
    cudaEvent_t ev_half[2] = {nullptr, nullptr};
    bool half_busy[2] = {false, false};
    cudaStream_t stream = nullptr;
    std::deque<Batch> inflight;

    Slot plan;  // planner scratch (host arrays)
    std::vector<double> tf_now;
    std::shared_ptr<const TfTable> tf_table;  // tf_now as the march reads it
    vr_server_stats st{};
};

namespace {

std::shared_ptr<const TfTable> table_of(const vr_ctx* c) {
    auto t = std::make_shared<TfTable>();
    t->n = (int32_t)c->tf_v.size();
    t->rgba = c->tf_rgba;
    t->v = c->tf_v;
    t->v.push_back(c->tf_v.back());
    t->uniform = c->tf_uniform != 0;
    t->v0 = c->tf_v0;
    t->inv_dv = c->tf_inv_dv;
    return t;
}

// Device bytes a planned frame takes in the arena.
size_t frame_bytes(const vr_camera& cam, int64_t n_items, int64_t n_tiles) {
    return align256(sizeof(vr::FrameCam)) + align256((size_t)(cam.width + cam.height) * sizeof(df)) +
           align256((size_t)n_items * sizeof(vr::Item)) + align256(((size_t)n_tiles + 1) * sizeof(int32_t)) +
           (size_t)n_items * vr::kTilePixels * sizeof(float4);
}

void finish(vr_server* S, Req* r, int state, int err) {
    r->state = state;
    r->err = err;
    r->t_done = now_ms();
    if (state == kDone) ++S->st.completed;
    else ++S->st.failed;
}

// Render one admitted batch (every frame planned, one step; each frame with its
// own transfer function and termination) into arena half b.half.  Returns VR_OK
// or a CUDA error.
int run_batch(vr_server* S, Batch& b) {
    vr_ctx* c = S->c;
    const int h = b.half;
    char* stage = S->h_stage[h];
    char* arena = S->d_arena[h];
    // layout: [TF rgba][TF v][cams][all items][per frame: q tables, tile_start][frags];
    // the batch's transfer functions concatenated (n + 1 entries each)
    int64_t n_items = 0;
    for (Req* r : b.reqs) n_items += (int64_t)r->items.size();
    size_t off = 0;
    const size_t o_rgba = off;
    off += align256((size_t)b.tf_entries * sizeof(float4));
    const size_t o_v = off;
    off += align256((size_t)b.tf_entries * sizeof(float));
    const size_t o_cams = off;
    off += align256(b.reqs.size() * sizeof(vr::FrameCam));
    const size_t o_items = off;
    off += align256((size_t)n_items * sizeof(vr::Item));
    for (size_t k = 0; k < b.tfs.size(); ++k) {
        const TfTable* t = b.tfs[k];
        std::memcpy(stage + o_rgba + (size_t)b.tf_off[k] * sizeof(float4), t->rgba.data(),
                    t->rgba.size() * sizeof(float4));
        std::memcpy(stage + o_v + (size_t)b.tf_off[k] * sizeof(float), t->v.data(), t->v.size() * sizeof(float));
    }
    vr::FrameCam* cams = reinterpret_cast<vr::FrameCam*>(stage + o_cams);
    vr::Item* items = reinterpret_cast<vr::Item*>(stage + o_items);
    int64_t frag_base = 0, tile_base = 0;
    for (size_t k = 0; k < b.reqs.size(); ++k) {
        const Req* r = b.reqs[k];
        const int64_t n_tiles = (int64_t)r->tiles_x * r->tiles_y;
        const size_t o_q = off;
        off += align256(r->q.size() * sizeof(df));
        const size_t o_tiles = off;
        off += align256(((size_t)n_tiles + 1) * sizeof(int32_t));
        std::memcpy(stage + o_q, r->q.data(), r->q.size() * sizeof(df));
        for (size_t i = 0; i < r->items.size(); ++i) {
            vr::Item it = r->items[i];
            it.frag += (int32_t)frag_base;
            it.sweep = (it.sweep & 7) | ((int32_t)k << 3);
            items[frag_base + (int64_t)i] = it;
        }
        int32_t* ts = reinterpret_cast<int32_t*>(stage + o_tiles);
        for (int64_t t = 0; t <= n_tiles; ++t) ts[t] = r->tile_start[t] + (int32_t)frag_base;
        vr::FrameCam& fc = cams[k];
        std::memset(&fc, 0, sizeof(fc));
        for (int a = 0; a < 3; ++a) {
            fc.eye[a] = vr::df_from_double(r->cam.eye[a]);
            fc.f[a] = vr::df_from_double(r->f[a]);
            fc.r[a] = vr::df_from_double(r->r[a]);
            fc.u[a] = vr::df_from_double(r->u[a]);
        }
        fc.qx = reinterpret_cast<const df*>(arena + o_q);
        fc.qy = fc.qx + r->cam.width;
        fc.width = r->cam.width;
        fc.height = r->cam.height;
        fc.tiles_x = r->tiles_x;
        fc.tiles_y = r->tiles_y;
        fc.tile_start = reinterpret_cast<const int32_t*>(arena + o_tiles);
        fc.out = reinterpret_cast<float4*>(r->out);
        fc.tile_base = (int32_t)tile_base;
        fc.tf_off = b.tf_off[r->tf_slot];
        fc.tf_n = r->tft->n;
        fc.tf_v0 = r->tft->v0;
        fc.tf_inv_dv = r->tft->inv_dv;
        fc.tau = (float)r->cam.term_alpha;
        fc.tf_uniform = r->tft->uniform ? 1 : 0;
        frag_base += (int64_t)r->items.size();
        tile_base += n_tiles;
    }
    const size_t upload = off;
    const size_t o_frags = align256(off);
    if (o_frags + (size_t)n_items * vr::kTilePixels * sizeof(float4) > S->half_bytes)
        return fail(c, VR_ENOMEM, "internal: batch exceeds its arena half");

    vr::FrameParams p;
    fill_common_params(c, p);
    p.tau = (float)b.reqs[0]->cam.term_alpha;
    p.tile = vr::kTile;
    p.tf_rgba = reinterpret_cast<const float4*>(arena + o_rgba);
    p.tf_v = reinterpret_cast<const float*>(arena + o_v);
    p.tf_n = b.tf_entries - 1;  // the shared-memory copy takes every entry
    p.cams = reinterpret_cast<const vr::FrameCam*>(arena + o_cams);
    p.n_cams = (int32_t)b.reqs.size();
    p.items = reinterpret_cast<const vr::Item*>(arena + o_items);
    p.n_items = (int32_t)n_items;
    p.frags = reinterpret_cast<float4*>(arena + o_frags);
    p.stats = S->d_stats[h];
    VR_CUDA(c, cudaMemcpyAsync(arena, stage, upload, cudaMemcpyHostToDevice, S->stream));
    VR_CUDA(c, cudaMemsetAsync(S->d_stats[h], 0, sizeof(vr::Stats), S->stream));
    VR_CUDA(c, vr::launch_march_tex_batch(p, S->stream));
    VR_CUDA(c, vr::launch_composite_batch(p, (int32_t)tile_base, S->stream));
    VR_CUDA(c, cudaMemcpyAsync(S->h_stats[h], S->d_stats[h], sizeof(vr::Stats), cudaMemcpyDeviceToHost,
                               S->stream));
    VR_CUDA(c, cudaEventRecord(S->ev_half[h], S->stream));
    b.items = n_items;
    return VR_OK;
}

// Plan request r (its transfer function must be in force): camera, work list and
// the bytes it takes in an arena half.
int plan_request(vr_server* S, Req* r, size_t& bytes) {
    vr_ctx* c = S->c;
    int rc = vr_set_camera(c, &r->cam);
    if (rc) return rc;
    int32_t tx = 0, ty = 0, T = 0;
    int64_t n_items = 0;
    const int32_t win[4] = {0, 0, r->cam.width - 1, r->cam.height - 1};
    if ((rc = plan_frame(c, S->plan, win, tx, ty, T, n_items))) return rc;
    r->items.assign(S->plan.h_items, S->plan.h_items + n_items);
    r->tile_start.assign(S->plan.h_tile_start, S->plan.h_tile_start + (int64_t)tx * ty + 1);
    r->q = c->q;
    for (int a = 0; a < 3; ++a) {
        r->f[a] = c->basis.f[a];
        r->r[a] = c->basis.r[a];
        r->u[a] = c->basis.u[a];
    }
    r->tiles_x = tx;
    r->tiles_y = ty;
    bytes = frame_bytes(r->cam, n_items, (int64_t)tx * ty);
    return VR_OK;
}

// Frames of one batch share the step (its opacity-correction fit is per launch);
// transfer functions and termination thresholds may differ.
bool same_group(const Req* a, const Req* b) { return a->cam.step == b->cam.step; }

// The request's table in the batch (added if no equal one is there).
void use_table(Batch& b, Req* r) {
    for (size_t k = 0; k < b.tfs.size(); ++k)
        if (b.tfs[k]->same(*r->tft)) {
            r->tf_slot = (int32_t)k;
            return;
        }
    r->tf_slot = (int32_t)b.tfs.size();
    b.tfs.push_back(r->tft.get());
    b.tf_off.push_back(b.tf_entries);
    b.tf_entries += (int32_t)r->tft->rgba.size();
}

void worker_main(vr_server* S) {
    vr_ctx* c = S->c;
    cudaSetDevice(c->device);
    for (;;) {
        Batch b;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] {
                return (S->stop && S->queue.empty()) ||
                       (!S->queue.empty() && (!S->half_busy[0] || !S->half_busy[1]));
            });
            if (S->queue.empty()) break;  // stop requested and drained
            b.half = S->half_busy[0] ? 1 : 0;
            S->half_busy[b.half] = true;
        }
        // admit in arrival order while the frames share the step, number at most
        // max_batch, their transfer functions fit the batch's tables and their
        // plans fit half the arena
        size_t bytes = 4096 + align256((size_t)kBatchTfEntries * sizeof(float4)) + align256((size_t)kBatchTfEntries * sizeof(float));
        for (;;) {
            Req* r = nullptr;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                if (S->queue.empty() || (int32_t)b.reqs.size() >= S->max_batch) break;
                r = S->queue.front();
                const bool tf_change = !r->tf.empty() && r->tf != S->tf_now;
                const int32_t tf_new = tf_change ? (int32_t)(r->tf.size() / 5) + 1 : 0;
                if (!b.reqs.empty() && (!same_group(r, b.reqs[0]) || b.tf_entries + tf_new > kBatchTfEntries))
                    break;
                S->queue.pop_front();
                r->state = kRunning;
            }
            int rc = VR_OK;
            if (!r->tf.empty() && r->tf != S->tf_now) {
                rc = vr_set_transfer_function(c, r->tf.data(), (int32_t)(r->tf.size() / 5));
                if (!rc) {
                    S->tf_now = r->tf;
                    S->tf_table = table_of(c);
                }
            }
            r->tft = S->tf_table;
            size_t need = 0;
            if (!rc) rc = plan_request(S, r, need);
            std::lock_guard<std::mutex> lk(S->mu);
            if (rc) {
                finish(S, r, kFailed, rc);
                continue;
            }
            if (bytes + need > S->half_bytes) {
                if (b.reqs.empty()) {
                    finish(S, r, kFailed, VR_ENOMEM);  // larger than half the arena
                    continue;
                }
                r->state = kQueued;
                S->queue.push_front(r);  // first of the next batch (planned again then)
                break;
            }
            bytes += need;
            use_table(b, r);
            b.reqs.push_back(r);
        }
        const int rc = b.reqs.empty() ? VR_OK : run_batch(S, b);
        std::lock_guard<std::mutex> lk(S->mu);
        if (rc) {
            S->worker_err = c->err;
            for (Req* r : b.reqs) finish(S, r, kFailed, rc);
            for (Req* r : S->queue) finish(S, r, kFailed, rc);
            S->queue.clear();
            S->half_busy[b.half] = false;
            S->stop = true;
            S->cv_done.notify_all();
            break;
        }
        if (b.reqs.empty()) {
            S->half_busy[b.half] = false;
            continue;
        }
        for (Req* r : b.reqs) {
            // the plan is in the arena now
            std::vector<vr::Item>().swap(r->items);
            std::vector<int32_t>().swap(r->tile_start);
            std::vector<df>().swap(r->q);
        }
        ++S->st.batches;
        S->st.batched_frames += (int64_t)b.reqs.size();
        S->inflight.push_back(std::move(b));
        S->cv_flight.notify_all();
    }
    std::lock_guard<std::mutex> lk(S->mu);
    S->worker_done = true;
    S->cv_flight.notify_all();
}

void completer_main(vr_server* S) {
    cudaSetDevice(S->c->device);
    for (;;) {
        Batch b;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_flight.wait(lk, [&] { return !S->inflight.empty() || S->worker_done; });
            if (S->inflight.empty()) return;  // the worker has finished and nothing is in flight
            b = std::move(S->inflight.front());
            S->inflight.pop_front();
        }
        const cudaError_t e = cudaEventSynchronize(S->ev_half[b.half]);
        std::lock_guard<std::mutex> lk(S->mu);
        for (Req* r : b.reqs) finish(S, r, e == cudaSuccess ? kDone : kFailed, e == cudaSuccess ? VR_OK : VR_ECUDA);
        if (e == cudaSuccess) {
            S->st.samples += (int64_t)S->h_stats[b.half]->samples;
            S->st.items += b.items;
        }
        S->half_busy[b.half] = false;
        S->cv_work.notify_all();
        S->cv_done.notify_all();
    }
}

}  // namespace

extern "C" {

int vr_server_create(vr_ctx* c, int64_t arena_bytes, int32_t max_batch, vr_server** out) {
    if (!c || !out) return VR_EINVAL;
    *out = nullptr;
    if (arena_bytes < (64 << 20) || max_batch < 1 || max_batch > (1 << 20))
        return fail(c, VR_EINVAL, "arena of at least 64 MiB and 1 <= max_batch");
    if (!c->d_cube || !c->bricked || !c->tf_set || !c->cam_set)
        return fail(c, VR_ESTATE, "vr_server_create needs a loaded, bricked cube, a transfer function and a camera");
    if (c->mode != 0 || c->step_mode != 0 || !use_tex(c))
        return fail(c, VR_EINVAL,
                    "the serving loop renders emission-absorption frames with a fixed step and the texture march");
    VR_CUDA(c, cudaSetDevice(c->device));
    int rc = retire_all(c);
    if (rc) return rc;
    if ((rc = prepare_tex(c))) return rc;
    vr_server* S = new vr_server();
    S->c = c;
    S->max_batch = max_batch;
    S->half_bytes = (size_t)arena_bytes / 2 / 256 * 256;
    S->tf_now = c->tf;
    S->tf_table = table_of(c);
    bool ok = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) == cudaSuccess;
    for (int h = 0; h < 2 && ok; ++h) {
        ok = cudaMalloc((void**)&S->d_arena[h], S->half_bytes) == cudaSuccess &&
             cudaHostAlloc((void**)&S->h_stage[h], S->half_bytes, cudaHostAllocDefault) == cudaSuccess &&
             cudaMalloc((void**)&S->d_stats[h], sizeof(vr::Stats)) == cudaSuccess &&
             cudaHostAlloc((void**)&S->h_stats[h], sizeof(vr::Stats), cudaHostAllocDefault) == cudaSuccess &&
             cudaEventCreateWithFlags(&S->ev_half[h], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        vr_server_destroy(S);
        return fail(c, VR_ENOMEM, "cannot allocate the serving arena");
    }
    S->worker = std::thread(worker_main, S);
    S->completer = std::thread(completer_main, S);
    *out = S;
    return VR_OK;
}

int vr_server_submit(vr_server* S, const vr_camera* cam, const double* tf_points, int32_t n_tf, float* out_rgba,
                     int64_t* ticket) {
    if (!S || !cam || !out_rgba || !ticket) return VR_EINVAL;
    if (!camera_valid(*cam)) return fail(S->c, VR_EINVAL, "bad camera");
    if (tf_points && (n_tf < 2 || n_tf > vr::kMaxTfPoints)) return fail(S->c, VR_EINVAL, "bad transfer function");
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, out_rgba) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return fail(S->c, VR_EINVAL, "the serving loop writes device memory");
    }
    Req* r = new Req();
    r->cam = *cam;
    if (tf_points) r->tf.assign(tf_points, tf_points + 5 * (size_t)n_tf);
    r->out = out_rgba;
    r->t_submit = now_ms();
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) {
        delete r;
        return fail(S->c, VR_ESTATE, "the serving loop has stopped: " + S->worker_err);
    }
    r->id = S->next_id++;
    S->reqs[r->id] = r;
    S->queue.push_back(r);
    ++S->st.submitted;
    *ticket = r->id;
    S->cv_work.notify_all();
    return VR_OK;
}

int vr_server_wait(vr_server* S, int64_t ticket, double timeout_s, double* latency_ms) {
    if (!S) return VR_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(S->c, VR_EINVAL, "unknown ticket");
    Req* r = it->second;
    auto ready = [&] { return r->state == kDone || r->state == kFailed; };
    if (timeout_s < 0) {
        S->cv_done.wait(lk, ready);
    } else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
        return VR_ETIMEOUT;
    }
    const int err = r->err;
    if (latency_ms) *latency_ms = r->t_done - r->t_submit;
    S->reqs.erase(it);
    delete r;
    return err;
}

int vr_server_get_stats(vr_server* S, vr_server_stats* out) {
    if (!S || !out) return VR_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->st;
    return VR_OK;
}

void vr_server_destroy(vr_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
        S->cv_flight.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    if (S->completer.joinable()) S->completer.join();
    cudaSetDevice(S->c->device);
    if (S->stream) cudaStreamSynchronize(S->stream);
    for (int h = 0; h < 2; ++h) {
        cudaFree(S->d_arena[h]);
        cudaFree(S->d_stats[h]);
        if (S->h_stage[h]) cudaFreeHost(S->h_stage[h]);
        if (S->h_stats[h]) cudaFreeHost(S->h_stats[h]);
        if (S->ev_half[h]) cudaEventDestroy(S->ev_half[h]);
    }
    if (S->stream) cudaStreamDestroy(S->stream);
    if (S->plan.h_items) cudaFreeHost(S->plan.h_items);
    if (S->plan.h_tile_start) cudaFreeHost(S->plan.h_tile_start);
    for (auto& kv : S->reqs) delete kv.second;
    delete S;
}

}  // extern "C"
