// vr_render_noalloc: a render entry point that allocates no memory.
//
// Some callers cannot allocate device memory while they render: a host
// application or plugin that owns the whole device-memory budget and forbids
// libraries from calling cudaMalloc, a real-time loop that cannot accept the
// implicit device synchronisation of cudaMalloc/cudaFree, or an embedding whose
// allocator is not CUDA's.  For them this file keeps all of the frame's scratch
// (frame constants, work list, per-brick sub-image fragments, counters) in one
// file-scope static device array, and the planner's lists in static host
// arrays.  The caller passes the cube (device memory), the transfer function,
// the camera and the output image (device memory).
//
// The kernels are the library's direct-gather ray march and sort-last composite
// kernels; only where their scratch lives differs.  Every call shares the same
// device scratch: calls that overlap on the GPU (for example on two streams)
// race, and the host-side lists make the function unsafe to call from two host
// threads at once.
//
// Set-up, done by the first call on each device (and once per process): the
// device address of the scratch array (cudaGetSymbolAddress), two events that
// mark when each of the two host staging sets has been uploaded, and the
// page-locking of those sets (cudaHostRegister, which pins the existing static
// arrays and allocates nothing), so that the uploads are asynchronous copies.
// Call n fills staging set n % 2 after waiting for the uploads of call n - 2.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "../../include/vr.h"
#include "vr_alpha_fit.h"
#include "vr_internal.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)VR_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxSide = 1024;        // image width and height
constexpr int kMaxBricks = 4096;
constexpr size_t kStatsBytes = 256;
constexpr size_t kConstBytes = 64 * 1024;  // camera tables + transfer function

// The scratch array.  In host code its name is only a stand-in: the device
// address comes from cudaGetSymbolAddress (see scratch_on_current_device).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
static void* g_scratch_ptr[kMaxDevices];  // device address per device, set on first use

// Static host-side planner lists (no heap use per call).
constexpr int kTileSide = vr::kTile;
constexpr int kMaxTiles = (kMaxSide / kTileSide) * (kMaxSide / kTileSide);
constexpr size_t kFragBytesPerItem = (size_t)vr::kTilePixels * sizeof(float4);
constexpr size_t kMaxItems =
    (kScratchBytes - kStatsBytes - kConstBytes - ((size_t)kMaxTiles + 1) * sizeof(int32_t)) /
    (kFragBytesPerItem + sizeof(vr::Item));

// Host staging of what each call uploads (two sets, page-locked at set-up).
struct alignas(4096) HostStage {
    vr::Item items[kMaxItems];
    int32_t tile_start[kMaxTiles + 1];
    unsigned char cst[kConstBytes];
};
static HostStage g_stage[2];
static int g_stage_pinned = -1;          // -1: not tried; 0: pageable; 1: page-locked
static unsigned long long g_calls = 0;   // calls that uploaded (picks the staging set)
static int g_stage_dev[2] = {-1, -1};    // device whose event marks each set's last upload
static cudaEvent_t g_stage_done[kMaxDevices][2];
static bool g_events_made[kMaxDevices];

// Planner lists that stay on the host.
static int32_t h_fill[kMaxTiles];
struct PlanBrick {
    int32_t key, id, rect[4];
};
static PlanBrick h_bricks[kMaxBricks];
static PlanBrick h_sorted[kMaxBricks];
// View-order keys sum |b_a - e_a| over the axes, with 0 <= b_a < nb_a and
// -1 <= e_a <= nb_a, so a key is at most nb_x + nb_y + nb_z <= 3 * kMaxBricks.
constexpr int kMaxKey = 3 * kMaxBricks;
static int32_t h_key_start[kMaxKey + 2];

// Set-up, once per device, with that device current: the device address of the
// scratch array and the staging events; once per process: the page-locking of
// the staging sets (if that fails they stay pageable: still correct, but the
// copies may then wait for the stream).  Returns nullptr on failure.
void* scratch_on_current_device(int dev) {
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    if (!g_events_made[dev]) {
        if (cudaEventCreateWithFlags(&g_stage_done[dev][0], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        if (cudaEventCreateWithFlags(&g_stage_done[dev][1], cudaEventDisableTiming) != cudaSuccess) {
            cudaEventDestroy(g_stage_done[dev][0]);
            cudaGetLastError();
            return nullptr;
        }
        g_events_made[dev] = true;
    }
    if (g_stage_pinned < 0) {
        g_stage_pinned =
            cudaHostRegister(g_stage, sizeof(g_stage), cudaHostRegisterPortable) == cudaSuccess ? 1 : 0;
        cudaGetLastError();
    }
    if (g_scratch_ptr[dev]) return g_scratch_ptr[dev];
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    g_scratch_ptr[dev] = ptr;
    return ptr;
}

struct Basis {
    double f[3], r[3], u[3], tan_half, aspect;
};

bool basis_of(const vr_camera& c, Basis& b) {
    double n = 0;
    for (int a = 0; a < 3; ++a) {
        b.f[a] = c.target[a] - c.eye[a];
        n += b.f[a] * b.f[a];
    }
    n = std::sqrt(n);
    if (!(n > 0)) return false;
    for (int a = 0; a < 3; ++a) b.f[a] /= n;
    b.r[0] = b.f[1] * c.up[2] - b.f[2] * c.up[1];
    b.r[1] = b.f[2] * c.up[0] - b.f[0] * c.up[2];
    b.r[2] = b.f[0] * c.up[1] - b.f[1] * c.up[0];
    n = std::sqrt(b.r[0] * b.r[0] + b.r[1] * b.r[1] + b.r[2] * b.r[2]);
    if (!(n > 1e-300)) return false;
    for (int a = 0; a < 3; ++a) b.r[a] /= n;
    b.u[0] = b.r[1] * b.f[2] - b.r[2] * b.f[1];
    b.u[1] = b.r[2] * b.f[0] - b.r[0] * b.f[2];
    b.u[2] = b.r[0] * b.f[1] - b.r[1] * b.f[0];
    b.tan_half = std::tan(c.fovy_deg * 3.14159265358979323846 / 360.0);
    b.aspect = (double)c.width / (double)c.height;
    return true;
}

// Bounding rectangle of the projected box corners, one pixel wider on each side;
// the whole image if a corner is not in front of the eye.  False if off screen.
bool rect_of(const vr_camera& c, const Basis& b, const double lo[3], const double hi[3],
             int32_t rect[4]) {
    double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
    for (int k = 0; k < 8; ++k) {
        double v[3] = {((k & 1) ? hi[0] : lo[0]) - c.eye[0], ((k & 2) ? hi[1] : lo[1]) - c.eye[1],
                       ((k & 4) ? hi[2] : lo[2]) - c.eye[2]};
        double zc = v[0] * b.f[0] + v[1] * b.f[1] + v[2] * b.f[2];
        if (!(zc > 1e-9)) {
            rect[0] = rect[1] = 0;
            rect[2] = c.width - 1;
            rect[3] = c.height - 1;
            return true;
        }
        double xc = v[0] * b.r[0] + v[1] * b.r[1] + v[2] * b.r[2];
        double yc = v[0] * b.u[0] + v[1] * b.u[1] + v[2] * b.u[2];
        double pi = (xc / (zc * b.tan_half * b.aspect) + 1.0) * 0.5 * c.width - 0.5;
        double pj = (1.0 - yc / (zc * b.tan_half)) * 0.5 * c.height - 0.5;
        x0 = std::min(x0, pi);
        x1 = std::max(x1, pi);
        y0 = std::min(y0, pj);
        y1 = std::max(y1, pj);
    }
    x0 = std::max(std::floor(x0) - 1, 0.0);
    y0 = std::max(std::floor(y0) - 1, 0.0);
    x1 = std::min(std::ceil(x1) + 1, (double)c.width - 1);
    y1 = std::min(std::ceil(y1) + 1, (double)c.height - 1);
    if (x1 < x0 || y1 < y0) return false;
    rect[0] = (int32_t)x0;
    rect[1] = (int32_t)y0;
    rect[2] = (int32_t)x1;
    rect[3] = (int32_t)y1;
    return true;
}

}  // namespace

extern "C" int vr_render_noalloc(const float* cube, int64_t nx, int64_t ny, int64_t nz,
                                 int32_t bx, int32_t by, int32_t bz, const double* tf, int32_t n_tf,
                                 const vr_camera* cam, float* out_rgba, void* cuda_stream) {
    if (!cube || !tf || !cam || !out_rgba) return VR_EINVAL;
    if (nx < 2 || ny < 2 || nz < 2 || nx > 65536 || ny > 65536 || nz > 65536) return VR_EINVAL;
    if (bx < 1 || by < 1 || bz < 1 || n_tf < 2 || n_tf > vr::kMaxTfPoints) return VR_EINVAL;
    if (cam->width < 1 || cam->height < 1 || cam->width > kMaxSide || cam->height > kMaxSide)
        return VR_EINVAL;
    if (!(cam->step >= 0.01 && cam->step <= 1000.0) || !(cam->term_alpha > 0.0 && cam->term_alpha <= 1.0) ||
        !(cam->fovy_deg > 0.0 && cam->fovy_deg < 180.0))
        return VR_EINVAL;
    for (int i = 0; i < n_tf; ++i) {
        for (int k = 1; k < 5; ++k)
            if (!(tf[5 * i + k] >= 0.0 && tf[5 * i + k] <= 1.0)) return VR_EINVAL;
        if (i > 0 && !(tf[5 * i] > tf[5 * (i - 1)])) return VR_EINVAL;
    }
    const int64_t nb[3] = {(nx - 1 + bx - 1) / bx, (ny - 1 + by - 1) / by, (nz - 1 + bz - 1) / bz};
    const int64_t n_bricks = nb[0] * nb[1] * nb[2];
    if (n_bricks > kMaxBricks) return VR_EINVAL;
    Basis b;
    if (!basis_of(*cam, b)) return VR_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return VR_ECUDA;
    // both the cube and the image must be device memory of the current device
    // (the kernels run there and read and write them without peer access)
    cudaPointerAttributes a_out, a_cube;
    if (cudaPointerGetAttributes(&a_out, out_rgba) != cudaSuccess ||
        cudaPointerGetAttributes(&a_cube, cube) != cudaSuccess) {
        cudaGetLastError();
        return VR_EINVAL;
    }
    if (a_out.type != cudaMemoryTypeDevice || a_cube.type != cudaMemoryTypeDevice || a_out.device != dev ||
        a_cube.device != dev)
        return VR_EINVAL;
    unsigned char* scratch = static_cast<unsigned char*>(scratch_on_current_device(dev));
    if (!scratch) return VR_ECUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;

    // ---- plan (host, static lists): rendering rectangles, view order, work list
    const int32_t B[3] = {bx, by, bz};
    const int64_t n[3] = {nx, ny, nz};
    int64_t e[3];
    for (int a = 0; a < 3; ++a) {
        double E = cam->eye[a];
        e[a] = E < 0.0 ? -1 : (E > (double)(n[a] - 1) ? nb[a] : std::min<int64_t>((int64_t)std::floor(E / B[a]), nb[a] - 1));
    }
    int n_pb = 0;
    for (int64_t id = 0; id < n_bricks; ++id) {
        int64_t idx[3] = {id % nb[0], (id / nb[0]) % nb[1], id / (nb[0] * nb[1])};
        double lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            lo[a] = (double)(idx[a] * B[a]);
            hi[a] = (double)std::min<int64_t>((idx[a] + 1) * B[a], n[a] - 1);
        }
        PlanBrick pb;
        pb.id = (int32_t)id;
        if (!rect_of(*cam, b, lo, hi, pb.rect)) continue;
        pb.key = 0;
        for (int a = 0; a < 3; ++a) pb.key += (int32_t)std::llabs(idx[a] - e[a]);
        h_bricks[n_pb++] = pb;
    }
    // front-to-back order: a stable counting sort on the view-order key
    std::memset(h_key_start, 0, sizeof(h_key_start));
    for (int q = 0; q < n_pb; ++q) h_key_start[h_bricks[q].key + 1]++;
    for (int k = 0; k <= kMaxKey; ++k) h_key_start[k + 1] += h_key_start[k];
    for (int q = 0; q < n_pb; ++q) h_sorted[h_key_start[h_bricks[q].key]++] = h_bricks[q];
    const int tiles_x = (cam->width + kTileSide - 1) / kTileSide, tiles_y = (cam->height + kTileSide - 1) / kTileSide;
    const int n_tiles = tiles_x * tiles_y;
    std::memset(h_fill, 0, sizeof(int32_t) * n_tiles);
    int64_t n_items = 0;
    for (int q = 0; q < n_pb; ++q) {
        const PlanBrick& pb = h_sorted[q];
        for (int ty = pb.rect[1] / kTileSide; ty <= pb.rect[3] / kTileSide; ++ty)
            for (int tx = pb.rect[0] / kTileSide; tx <= pb.rect[2] / kTileSide; ++tx) h_fill[ty * tiles_x + tx]++;
        n_items += (int64_t)(pb.rect[2] / kTileSide - pb.rect[0] / kTileSide + 1) *
                   (pb.rect[3] / kTileSide - pb.rect[1] / kTileSide + 1);
    }
    if (n_items > (int64_t)kMaxItems) return VR_EINVAL;  // frame needs more scratch than the array holds
    // the staging set of this call: wait until the call that used it last has
    // uploaded it (two calls back; normally long done)
    const int set = (int)(g_calls & 1);
    if (g_stage_dev[set] >= 0 && cudaEventSynchronize(g_stage_done[g_stage_dev[set]][set]) != cudaSuccess) {
        cudaGetLastError();
        return VR_ECUDA;
    }
    HostStage& hs = g_stage[set];
    int32_t run = 0;
    for (int t = 0; t < n_tiles; ++t) {
        hs.tile_start[t] = run;
        run += h_fill[t];
        h_fill[t] = 0;
    }
    hs.tile_start[n_tiles] = run;
    int64_t k = 0;
    for (int q = 0; q < n_pb; ++q) {
        const PlanBrick& pb = h_sorted[q];
        for (int ty = pb.rect[1] / kTileSide; ty <= pb.rect[3] / kTileSide; ++ty)
            for (int tx = pb.rect[0] / kTileSide; tx <= pb.rect[2] / kTileSide; ++tx) {
                const int t = ty * tiles_x + tx;
                hs.items[k++] = vr::Item{pb.id, t, hs.tile_start[t] + h_fill[t]++, 0};
            }
    }

    // ---- frame constants (camera tables, transfer function) into the const block
    const size_t q_bytes = (size_t)(cam->width + cam->height) * sizeof(vr::df);
    const size_t tf_rgba_off = (q_bytes + 15) / 16 * 16;
    const size_t tf_v_off = tf_rgba_off + (size_t)(n_tf + 1) * sizeof(float4);
    const size_t const_bytes = tf_v_off + (size_t)n_tf * sizeof(float);
    if (const_bytes > kConstBytes) return VR_EINVAL;
    vr::df* hq = reinterpret_cast<vr::df*>(hs.cst);
    for (int i = 0; i < cam->width; ++i)
        hq[i] = vr::df_from_double((2.0 * (i + 0.5) / cam->width - 1.0) * b.tan_half * b.aspect);
    for (int j = 0; j < cam->height; ++j)
        hq[cam->width + j] = vr::df_from_double((1.0 - 2.0 * (j + 0.5) / cam->height) * b.tan_half);
    float4* hrgba = reinterpret_cast<float4*>(hs.cst + tf_rgba_off);
    float* hv = reinterpret_cast<float*>(hs.cst + tf_v_off);
    for (int i = 0; i < n_tf; ++i) {
        hrgba[i] = make_float4((float)tf[5 * i + 1], (float)tf[5 * i + 2], (float)tf[5 * i + 3], (float)tf[5 * i + 4]);
        hv[i] = (float)tf[5 * i];
    }
    hrgba[n_tf] = hrgba[n_tf - 1];  // the kernels read one entry past the last point
    const double v0 = tf[0], dv = (tf[5 * (n_tf - 1)] - tf[0]) / (n_tf - 1);
    bool uniform = true;
    for (int i = 0; i < n_tf; ++i)
        if (std::fabs(tf[5 * i] - (v0 + i * dv)) > 1e-9 * std::max(1.0, std::fabs(tf[5 * i]))) uniform = false;

    // ---- scratch layout: [stats][constants][tile_start][items][fragments]
    unsigned char* d_stats = scratch;
    unsigned char* d_const = scratch + kStatsBytes;
    unsigned char* d_tiles = d_const + kConstBytes;
    unsigned char* d_items = d_tiles + ((size_t)kMaxTiles + 1) * sizeof(int32_t);
    unsigned char* d_frags = d_items + kMaxItems * sizeof(vr::Item);
    d_frags = scratch + ((size_t)(d_frags - scratch) + 255) / 256 * 256;
    if ((size_t)(d_frags - scratch) + (size_t)n_items * kFragBytesPerItem > kScratchBytes) return VR_EINVAL;

    vr::FrameParams p;
    std::memset(&p, 0, sizeof(p));
    for (int a = 0; a < 3; ++a) {
        p.eye[a] = vr::df_from_double(cam->eye[a]);
        p.f[a] = vr::df_from_double(b.f[a]);
        p.r[a] = vr::df_from_double(b.r[a]);
        p.u[a] = vr::df_from_double(b.u[a]);
        p.n[a] = (int32_t)n[a];
        p.B[a] = B[a];
        p.nb[a] = (int32_t)nb[a];
    }
    p.qx = reinterpret_cast<const vr::df*>(d_const);
    p.qy = reinterpret_cast<const vr::df*>(d_const) + cam->width;
    p.width = cam->width;
    p.height = cam->height;
    p.tiles_x = tiles_x;
    p.tiles_y = tiles_y;
    p.tile = kTileSide;
    p.dt = vr::df_from_double(cam->step);
    p.inv_dt = vr::df_from_double(1.0 / cam->step);
    p.dt_f = (float)cam->step;
    p.tau = (float)cam->term_alpha;
    p.cube = cube;
    p.stride_y = nx;
    p.stride_z = nx * ny;
    p.offsets32 = ((int64_t)bz + 1) * p.stride_z + ((int64_t)by + 1) * p.stride_y + bx + 1 < ((int64_t)1 << 32) ? 1 : 0;
    p.tf_rgba = reinterpret_cast<const float4*>(d_const + tf_rgba_off);
    p.tf_v = reinterpret_cast<const float*>(d_const + tf_v_off);
    p.tf_n = n_tf;
    p.tf_uniform = uniform ? 1 : 0;
    p.tf_v0 = (float)v0;
    p.tf_inv_dv = (float)(1.0 / dv);
    static const double long_splits[] = {0.5, 0.4, 0.3, 0.25, 0.2};
    static const double short_splits[] = {0.1, 0.08, 0.06, 0.04, 0.02};
    const double split = vr::fit_alpha(cam->step, long_splits, vr::kAlphaPolyTerms, p.alpha_poly, 5e-10);
    p.alpha_split = (float)split;
    p.poly_scale = (float)(2.0 / split);
    const double small = vr::fit_alpha(cam->step, short_splits, vr::kAlphaSmallTerms, p.alpha_small, 5e-10);
    p.small_split = (float)small;
    p.small_scale = (float)(2.0 / small);
    p.mode = 0;
    p.items = reinterpret_cast<const vr::Item*>(d_items);
    p.n_items = (int32_t)n_items;
    p.tile_start = reinterpret_cast<const int32_t*>(d_tiles);
    p.frags = reinterpret_cast<float4*>(d_frags);
    p.out = reinterpret_cast<float4*>(out_rgba);
    p.out_x0 = p.out_y0 = 0;
    p.out_w = p.width;
    p.out_h = p.height;
    p.stats = reinterpret_cast<vr::Stats*>(d_stats);

    // The counters must start at zero; the rest of the scratch is fully rewritten.
    // The staging set is marked in use by this call from its first copy on.
    g_stage_dev[set] = -1;
    if (cudaMemsetAsync(d_stats, 0, sizeof(vr::Stats), st) != cudaSuccess ||
        cudaMemcpyAsync(d_const, hs.cst, const_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_tiles, hs.tile_start, ((size_t)n_tiles + 1) * sizeof(int32_t), cudaMemcpyHostToDevice,
                        st) != cudaSuccess ||
        cudaMemcpyAsync(d_items, hs.items, (size_t)n_items * sizeof(vr::Item), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaEventRecord(g_stage_done[dev][set], st) != cudaSuccess) {
        // copies may be in flight: wait for the stream before the set is reused
        cudaGetLastError();
        cudaStreamSynchronize(st);
        cudaGetLastError();
        return VR_ECUDA;
    }
    g_stage_dev[set] = dev;
    ++g_calls;
    if (vr::launch_march(p, st) != cudaSuccess || vr::launch_composite(p, st) != cudaSuccess) {
        cudaGetLastError();
        return VR_ECUDA;
    }
    return VR_OK;
}
