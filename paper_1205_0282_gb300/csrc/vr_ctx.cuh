// Context of the C ABI (shared by vr_host.cu and vr_serve.cu): the per-frame
// slot ring, the camera basis, the context state and the host helpers that both
// translation units use.
#pragma once
#include <algorithm>
#include <cfloat>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/vr.h"
#include "vr_alpha_fit.h"
#include "vr_blocks.h"
#include "vr_internal.cuh"

using vr::df;

namespace vrh {

constexpr int kSlots = 3;  // frames that may be in flight per context

struct Slot {
    vr::Item* h_items = nullptr;
    int32_t* h_tile_start = nullptr;
    size_t cap_items = 0, cap_tiles = 0;
    vr::Item* d_items = nullptr;
    int32_t* d_tile_start = nullptr;
    size_t dcap_items = 0, dcap_tiles = 0;
    float4* d_frags = nullptr;
    size_t cap_frags = 0;  // float4 pixels
    float4* d_img = nullptr;
    size_t cap_img = 0;    // float4 pixels
    unsigned char* h_frame = nullptr;  // camera tables + transfer function, pinned
    unsigned char* d_frame = nullptr;
    size_t cap_frame = 0, dcap_frame = 0;
    vr::Stats* d_stats = nullptr;
    vr::Stats* h_stats = nullptr;
    int32_t* h_slot_of = nullptr;  // out-of-core: cache slot of each brick (pinned)
    int32_t* d_slot_of = nullptr;
    size_t cap_slot_of = 0, dcap_slot_of = 0;
    int32_t* h_fill = nullptr;    // out-of-core texture march: slots whose layered copies are refilled
    int32_t* d_fill = nullptr;
    size_t cap_fill = 0, dcap_fill = 0;
    int32_t* d_work = nullptr;    // out-of-core texture march: one half-item counter per launch
    size_t dcap_work = 0;
    int32_t* h_decode = nullptr;  // learned residency: (brick, slot) lists of the frame's decodes
    int32_t* d_decode = nullptr;
    size_t cap_decode = 0, dcap_decode = 0;
    cudaEvent_t ev_begin = nullptr, ev_march0 = nullptr, ev_march1 = nullptr, ev_end = nullptr;
    bool pending = false;
    // host-side facts of the frame in flight
    int64_t items = 0, bricks_rendered = 0, bricks_skipped = 0, touched_bytes = 0;
    int64_t h2d_bytes = 0, d2h_bytes = 0, launches = 0, fragments = 0;
    int64_t bricks_uploaded = 0, bricks_cached = 0;
    double plan_ms = 0.0;
};

struct Basis {
    double f[3], r[3], u[3];
    double tan_half, aspect;
};

inline bool make_basis(const vr_camera& c, Basis& b) {
    double f[3], n = 0;
    for (int a = 0; a < 3; ++a) {
        f[a] = c.target[a] - c.eye[a];
        n += f[a] * f[a];
    }
    n = std::sqrt(n);
    if (!(n > 0)) return false;
    for (int a = 0; a < 3; ++a) b.f[a] = f[a] / n;
    double r[3] = {b.f[1] * c.up[2] - b.f[2] * c.up[1], b.f[2] * c.up[0] - b.f[0] * c.up[2],
                   b.f[0] * c.up[1] - b.f[1] * c.up[0]};
    n = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (!(n > 1e-300)) return false;
    for (int a = 0; a < 3; ++a) b.r[a] = r[a] / n;
    b.u[0] = b.r[1] * b.f[2] - b.r[2] * b.f[1];
    b.u[1] = b.r[2] * b.f[0] - b.r[0] * b.f[2];
    b.u[2] = b.r[0] * b.f[1] - b.r[1] * b.f[0];
    b.tan_half = std::tan(c.fovy_deg * 3.14159265358979323846 / 360.0);
    b.aspect = (double)c.width / (double)c.height;
    return true;
}

inline bool camera_valid(const vr_camera& c) {
    if (c.width < 1 || c.height < 1 || c.width > 16384 || c.height > 16384) return false;
    if (!(c.fovy_deg > 0.0 && c.fovy_deg < 180.0)) return false;
    // step >= 0.01 keeps every sample index below 2^24 (exact in FP32) for cubes up
    // to 65536 voxels per axis
    if (!(c.step >= 0.01 && c.step <= 1000.0)) return false;
    if (!(c.term_alpha > 0.0 && c.term_alpha <= 1.0)) return false;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(c.eye[a]) || !std::isfinite(c.target[a]) || !std::isfinite(c.up[a]))
            return false;
    return true;
}

inline int64_t bricks_along(int64_t n, int64_t B) { return (n - 1 + B - 1) / B; }

// Rendering rectangle of the box [lo, hi] (Section 2.3.2: project the sub-cube's
// vertices, take their bounding rectangle).  Pixel (i, j) has its centre at
// ((i+.5)/W, (j+.5)/H) of the image; the rectangle is widened by one pixel so that
// rounding can never drop a pixel whose ray touches the box.  Returns false if the
// rectangle is empty after clipping, or if the whole box lies behind the eye plane
// (every ray leaves the eye forward along f).  A box reaching across the eye plane
// maps to the whole image.
inline bool box_rect(const vr_camera& c, const Basis& b, const double lo[3], const double hi[3],
              int32_t rect[4]) {
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
    bool behind = false;
    int back = 0;
    for (int k = 0; k < 8; ++k) {
        double P[3] = {(k & 1) ? hi[0] : lo[0], (k & 2) ? hi[1] : lo[1], (k & 4) ? hi[2] : lo[2]};
        double v[3] = {P[0] - c.eye[0], P[1] - c.eye[1], P[2] - c.eye[2]};
        double zc = v[0] * b.f[0] + v[1] * b.f[1] + v[2] * b.f[2];
        if (zc < -1e-6) ++back;
        if (!(zc > 1e-9)) behind = true;
        if (behind) continue;
        double xc = v[0] * b.r[0] + v[1] * b.r[1] + v[2] * b.r[2];
        double yc = v[0] * b.u[0] + v[1] * b.u[1] + v[2] * b.u[2];
        double sx = xc / (zc * b.tan_half * b.aspect), sy = yc / (zc * b.tan_half);
        double pi = (sx + 1.0) * 0.5 * c.width - 0.5;
        double pj = (1.0 - sy) * 0.5 * c.height - 0.5;
        xmin = std::min(xmin, pi);
        xmax = std::max(xmax, pi);
        ymin = std::min(ymin, pj);
        ymax = std::max(ymax, pj);
    }
    if (back == 8) {
        rect[0] = rect[1] = 0;
        rect[2] = rect[3] = -1;
        return false;
    }
    if (behind) {
        rect[0] = 0;
        rect[1] = 0;
        rect[2] = c.width - 1;
        rect[3] = c.height - 1;
        return true;
    }
    double x0 = std::floor(xmin) - 1, x1 = std::ceil(xmax) + 1;
    double y0 = std::floor(ymin) - 1, y1 = std::ceil(ymax) + 1;
    x0 = std::max(x0, 0.0);
    y0 = std::max(y0, 0.0);
    x1 = std::min(x1, (double)c.width - 1);
    y1 = std::min(y1, (double)c.height - 1);
    if (x1 < x0 || y1 < y0) {
        rect[0] = rect[1] = 0;
        rect[2] = rect[3] = -1;
        return false;
    }
    rect[0] = (int32_t)x0;
    rect[1] = (int32_t)y0;
    rect[2] = (int32_t)x1;
    rect[3] = (int32_t)y1;
    return true;
}

// A box corner seen from the camera: depth along the view axis and, for
// corners in front of the eye, its pixel coordinates (box_rect's arithmetic).
struct CornerProj {
    double zc, pi, pj;
};
inline CornerProj project_corner(const vr_camera& c, const Basis& b, const double P[3]) {
    CornerProj q;
    const double v[3] = {P[0] - c.eye[0], P[1] - c.eye[1], P[2] - c.eye[2]};
    q.zc = v[0] * b.f[0] + v[1] * b.f[1] + v[2] * b.f[2];
    q.pi = q.pj = 0.0;
    if (q.zc > 1e-9) {
        const double xc = v[0] * b.r[0] + v[1] * b.r[1] + v[2] * b.r[2];
        const double yc = v[0] * b.u[0] + v[1] * b.u[1] + v[2] * b.u[2];
        const double sx = xc / (q.zc * b.tan_half * b.aspect), sy = yc / (q.zc * b.tan_half);
        q.pi = (sx + 1.0) * 0.5 * c.width - 0.5;
        q.pj = (1.0 - sy) * 0.5 * c.height - 0.5;
    }
    return q;
}
// box_rect from the eight corners' projections (the same result as box_rect on
// the box they span).
inline bool rect_from_corners(const vr_camera& c, const CornerProj* const q[8], int32_t rect[4]) {
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
    bool behind = false;
    int back = 0;
    for (int k = 0; k < 8; ++k) {
        if (q[k]->zc < -1e-6) ++back;
        if (!(q[k]->zc > 1e-9)) behind = true;
        if (behind) continue;
        xmin = std::min(xmin, q[k]->pi);
        xmax = std::max(xmax, q[k]->pi);
        ymin = std::min(ymin, q[k]->pj);
        ymax = std::max(ymax, q[k]->pj);
    }
    if (back == 8) {
        rect[0] = rect[1] = 0;
        rect[2] = rect[3] = -1;
        return false;
    }
    if (behind) {
        rect[0] = 0;
        rect[1] = 0;
        rect[2] = c.width - 1;
        rect[3] = c.height - 1;
        return true;
    }
    double x0 = std::floor(xmin) - 1, x1 = std::ceil(xmax) + 1;
    double y0 = std::floor(ymin) - 1, y1 = std::ceil(ymax) + 1;
    x0 = std::max(x0, 0.0);
    y0 = std::max(y0, 0.0);
    x1 = std::min(x1, (double)c.width - 1);
    y1 = std::min(y1, (double)c.height - 1);
    if (x1 < x0 || y1 < y0) {
        rect[0] = rect[1] = 0;
        rect[2] = rect[3] = -1;
        return false;
    }
    rect[0] = (int32_t)x0;
    rect[1] = (int32_t)y0;
    rect[2] = (int32_t)x1;
    rect[3] = (int32_t)y1;
    return true;
}

// Host threads the planner splits its loops over (no more than the machine has);
// the plan is the same whatever the count.
constexpr int64_t kPlanThreads = 16;
inline int64_t plan_threads() {
    return std::max<int64_t>(1, std::min<int64_t>((int64_t)std::thread::hardware_concurrency(), kPlanThreads));
}

// Projections of the brick grid's corner points x_i = min(i B, n - 1), i = 0..nb
// per axis (x fastest): every brick box spans eight of them.
inline void project_brick_grid(const vr_camera& cam, const Basis& b, const int64_t n[3], const int32_t B[3],
                               const int64_t nb[3], std::vector<CornerProj>& proj) {
    const int64_t g[3] = {nb[0] + 1, nb[1] + 1, nb[2] + 1};
    proj.resize((size_t)(g[0] * g[1] * g[2]));
    auto planes = [&](int64_t k0, int64_t k1) {
        for (int64_t k = k0; k < k1; ++k)
            for (int64_t j = 0; j < g[1]; ++j)
                for (int64_t i = 0; i < g[0]; ++i) {
                    const double P[3] = {(double)std::min<int64_t>(i * B[0], n[0] - 1),
                                         (double)std::min<int64_t>(j * B[1], n[1] - 1),
                                         (double)std::min<int64_t>(k * B[2], n[2] - 1)};
                    proj[(size_t)((k * g[1] + j) * g[0] + i)] = project_corner(cam, b, P);
                }
    };
    // large grids (tens of thousands of points) on a few host threads, by planes
    const int64_t parts = std::min<int64_t>({g[2], plan_threads(), g[0] * g[1] * g[2] / 16384 + 1});
    if (parts <= 1) {
        planes(0, g[2]);
        return;
    }
    std::vector<std::thread> pool;
    for (int64_t t = 1; t < parts; ++t) pool.emplace_back(planes, g[2] * t / parts, g[2] * (t + 1) / parts);
    planes(0, g[2] / parts);
    for (auto& th : pool) th.join();
}

// Rendering rectangle of brick idx from the grid projections (box_rect of its box).
inline void grid_corners(const std::vector<CornerProj>& proj, const int64_t nb[3], const int64_t idx[3],
                         const CornerProj* q[8]) {
    const int64_t g0 = nb[0] + 1, g1 = nb[1] + 1;
    for (int k = 0; k < 8; ++k) {
        const int64_t gi = idx[0] + (k & 1), gj = idx[1] + ((k >> 1) & 1), gk = idx[2] + ((k >> 2) & 1);
        q[k] = &proj[(size_t)((gk * g1 + gj) * g0 + gi)];
    }
}
inline bool brick_rect_from_grid(const vr_camera& cam, const std::vector<CornerProj>& proj, const int64_t nb[3],
                                 const int64_t idx[3], int32_t rect[4]) {
    const CornerProj* q[8];
    grid_corners(proj, nb, idx, q);
    return rect_from_corners(cam, q, rect);
}

// Tiles of T x T pixels that brick idx's silhouette reaches, as one span [tx0, tx1]
// per tile row ty.  With all eight corners in front of the eye, the silhouette is
// the convex hull of their projections; a tile is kept if a pixel centre of it lies
// within one pixel of the hull (the rectangle's margin), so every pixel whose ray
// crosses the brick keeps its tile.  Otherwise (a corner at or behind the eye
// plane) every tile of the rendering rectangle is kept.  Spans are clipped to the
// rectangle rect (the brick's rendering rectangle within the output window).
struct Span {
    int32_t ty, tx0, tx1;
};
inline void brick_spans(const CornerProj* const q[8], const int32_t rect[4], int T, std::vector<Span>& out) {
    const int tx_lo = rect[0] / T, tx_hi = rect[2] / T, ty_lo = rect[1] / T, ty_hi = rect[3] / T;
    bool front = true;
    for (int k = 0; k < 8; ++k) front = front && q[k]->zc > 1e-9;
    if (!front) {
        for (int ty = ty_lo; ty <= ty_hi; ++ty) out.push_back(Span{ty, tx_lo, tx_hi});
        return;
    }
    // convex hull (monotone chain) of the projected corners, counter-clockwise
    double px[8], py[8];
    int ord[8];
    for (int k = 0; k < 8; ++k) {
        px[k] = q[k]->pi;
        py[k] = q[k]->pj;
        ord[k] = k;
    }
    for (int i = 1; i < 8; ++i)  // insertion sort by (x, y)
        for (int j = i; j > 0 && (px[ord[j]] < px[ord[j - 1]] ||
                                  (px[ord[j]] == px[ord[j - 1]] && py[ord[j]] < py[ord[j - 1]]));
             --j)
            std::swap(ord[j], ord[j - 1]);
    int hull[16], h = 0;
    auto cross = [&](int o, int a, int b) {
        return (px[a] - px[o]) * (py[b] - py[o]) - (py[a] - py[o]) * (px[b] - px[o]);
    };
    for (int i = 0; i < 8; ++i) {
        while (h >= 2 && cross(hull[h - 2], hull[h - 1], ord[i]) <= 0.0) --h;
        hull[h++] = ord[i];
    }
    for (int i = 6, lo = h + 1; i >= 0; --i) {
        while (h >= lo && cross(hull[h - 2], hull[h - 1], ord[i]) <= 0.0) --h;
        hull[h++] = ord[i];
    }
    const int nh = h - 1;  // the last point repeats the first
    const double m = 1.0;  // margin in pixels
    const double inv_t = 1.0 / T;  // x / T exactly for the power-of-two tiles (columns are integers < 2^24)
    // x-extent of the silhouette within each tile row's band of pixel-centre rows
    // (widened by the margin): the extremes lie on its edges, so each edge updates
    // the rows its y-range overlaps, clipped to each band
    const int nrows = ty_hi - ty_lo + 1;
    constexpr int kRows = 2048;  // image heights up to 16384 pixels in tiles of 8 or more
    double xmn[kRows], xmx[kRows];
    for (int k = 0; k < nrows; ++k) {
        xmn[k] = 1e300;
        xmx[k] = -1e300;
    }
    auto band_lo = [&](int ty) { return std::max((double)(ty * T), (double)rect[1]) - m; };
    auto band_hi = [&](int ty) { return std::min((double)(ty * T + T - 1), (double)rect[3]) + m; };
    auto add_segment = [&](double xa, double ya, double xb, double yb) {
        if (ya > yb) {
            std::swap(xa, xb);
            std::swap(ya, yb);
        }
        const int r0 = std::max(ty_lo, (int)std::floor((ya - m - (T - 1)) * inv_t));
        const int r1 = std::min(ty_hi, (int)std::floor((yb + m) * inv_t));
        const double slope = yb > ya ? (xb - xa) / (yb - ya) : 0.0;
        for (int ty = r0; ty <= r1; ++ty) {
            const double lo = std::max(ya, band_lo(ty)), hi = std::min(yb, band_hi(ty));
            if (lo > hi) continue;
            double x0 = xa, x1 = xb;
            if (yb > ya) {
                x0 = xa + (lo - ya) * slope;
                x1 = xa + (hi - ya) * slope;
            }
            const int k = ty - ty_lo;
            xmn[k] = std::min(xmn[k], std::min(x0, x1));
            xmx[k] = std::max(xmx[k], std::max(x0, x1));
        }
    };
    if (nh >= 1) {
        for (int e = 0; e < nh; ++e) add_segment(px[hull[e]], py[hull[e]], px[hull[e + 1]], py[hull[e + 1]]);
    } else {
        for (int k = 0; k < 8; ++k) add_segment(px[k], py[k], px[k], py[k]);
    }
    for (int ty = ty_lo; ty <= ty_hi; ++ty) {
        const int k = ty - ty_lo;
        if (xmx[k] < xmn[k]) continue;  // the band misses the silhouette
        const double c0 = std::ceil(xmn[k] - m), c1 = std::floor(xmx[k] + m);
        if (c1 < c0) continue;
        const int tx0 = std::max(tx_lo, (int)(std::max(c0, 0.0) * inv_t));
        const int tx1 = std::min(tx_hi, (int)(std::max(c1, 0.0) * inv_t));
        if (tx0 <= tx1) out.push_back(Span{ty, tx0, tx1});
    }
}

// Sampling region of brick (ix, iy, iz): [b*B, min((b+1)*B, n-1)] per axis.
inline void brick_box(const int64_t n[3], const int32_t B[3], const int64_t idx[3], double lo[3],
               double hi[3]) {
    for (int a = 0; a < 3; ++a) {
        lo[a] = (double)(idx[a] * B[a]);
        hi[a] = (double)std::min<int64_t>((idx[a] + 1) * B[a], n[a] - 1);
    }
}

// Maximum of the piecewise-linear opacity over [lo, hi] (exact: endpoints and the
// control points strictly inside).
inline double tf_alpha_max(const std::vector<double>& tf, double lo, double hi) {
    const int n = (int)(tf.size() / 5);
    auto eval = [&](double v) {
        if (v <= tf[0]) return tf[4];
        if (v >= tf[5 * (n - 1)]) return tf[5 * (n - 1) + 4];
        int s = 0;
        while (!(v < tf[5 * (s + 1)])) ++s;
        double w = (v - tf[5 * s]) / (tf[5 * (s + 1)] - tf[5 * s]);
        return tf[5 * s + 4] + w * (tf[5 * (s + 1) + 4] - tf[5 * s + 4]);
    };
    double m = std::max(eval(lo), eval(hi));
    for (int s = 0; s < n; ++s)
        if (tf[5 * s] > lo && tf[5 * s] < hi) m = std::max(m, tf[5 * s + 4]);
    return m;
}

}  // namespace vrh

struct vr_ctx {
    using Slot = vrh::Slot;
    using Basis = vrh::Basis;
    static constexpr int kSlots = vrh::kSlots;
    int device = 0;
    std::string err;
    int sm_count = 0;

    float* d_cube = nullptr;     // [z][y][x], row pitch nx_pad floats (16-byte rows for TMA)
    int64_t n[3] = {0, 0, 0};
    int64_t nx_pad = 0;
    float* d_cube_xzy = nullptr; // transposed copy [x][z][y], row pitch ny_pad (sweeps along x)
    int64_t ny_pad = 0;
    CUtensorMap* d_tmaps = nullptr;  // tensor maps of the TMA march (device memory)
    cudaArray_t tex_arr[3][vr::kMaxTexSlabs] = {};  // texture march: layered copies, by slab
    cudaTextureObject_t tex_obj[3][vr::kMaxTexSlabs] = {};
    int32_t tex_slab_bricks[3] = {0, 0, 0};         // bricks per slab along each layer axis
    int64_t tex_slab_layers = 0;                     // VR_OPT_TEX_SLAB_LAYERS (0: device limit)
    bool tex_ready = false;
    int precision = VR_PRECISION_F32;  // storage of the layered copies
    float* d_brick_scale = nullptr;    // FP8 storage: per-brick scale
    std::vector<float2> h_minmax_q;    // FP16/FP8 storage: per-brick [min, max] of the stored values
    int tmaps_per_brick = 0;
    bool tma_ready = false;

    bool bricked = false;
    int32_t B[3] = {0, 0, 0};
    int32_t nb[3] = {0, 0, 0};
    int64_t n_bricks = 0;
    float2* d_minmax = nullptr;
    std::vector<float2> h_minmax;

    bool tf_set = false;
    std::vector<double> tf;
    std::vector<float4> tf_rgba;
    std::vector<float> tf_v;
    int tf_uniform = 0;
    float tf_v0 = 0, tf_inv_dv = 0;

    bool cam_set = false;
    vr_camera cam{};
    Basis basis{};
    std::vector<df> q;  // qx (width entries) then qy (height entries)
    float alpha_poly[vr::kAlphaPolyTerms] = {};
    double alpha_split = 0.5;
    float alpha_small[vr::kAlphaSmallTerms] = {};
    double small_split = 0.1;

    bool skip_empty = true, rect_cull = true;
    int mode = 0;
    int step_mode = 0;  // VR_OPT_STEP_MODE
    int kernel = VR_KERNEL_AUTO;
    int tex_fits = -1;  // -1 unknown, 0/1: the cube fits the layered-texture limits

    // out-of-core mode (vr_load_cube_host): cube in host memory, bricks cached on the device
    bool ooc = false;
    const float* h_src = nullptr;      // the caller's cube
    vr_block_provider prov_fn = nullptr;  // vr_load_cube_provider: bricks come from the provider
    void* prov_user = nullptr;
    int prov_threads = 0;              // VR_OPT_PROVIDER_THREADS
    bool host_async = false;           // VR_OPT_HOST_OUTPUT_ASYNC
    // provider contexts: pinned staging for the blocks of one upload launch, the
    // buffers taken in turn (a buffer is refilled once its copies have finished)
    static constexpr int kStage = 3;
    float* h_stage[kStage] = {nullptr, nullptr, nullptr};
    size_t stage_cap = 0;              // bytes of each staging buffer
    cudaEvent_t ev_stage[kStage] = {nullptr, nullptr, nullptr};
    int stage_next = 0;
    vr_codec* codec = nullptr;         // learned residency: slots are filled by decoding
    // learned residency's fallback: bricks whose decode error exceeds fb_bound are
    // copied from plain blocks in h_store (block plain_index[b]) instead
    const float* fb_src = nullptr;     // the caller's plain cube, read at vr_brick
    vr_block_provider fb_fn = nullptr; // or a provider of the plain blocks
    void* fb_user = nullptr;
    float fb_bound = 0.0f, fb_floor = 0.0f;
    bool fb_measured = false;          // brick_err holds the last vr_brick's errors
    std::vector<float> brick_err;
    std::vector<int64_t> plain_index;  // per brick: its block in h_store, or -1 (decoded)
    int64_t n_plain = 0;
    float* h_store = nullptr;          // pinned brick store, brick b at b * slot_floats
    size_t store_bytes = 0;
    int64_t slot_floats = 0;           // (Bx+1)(By+1)(Bz+1)
    int64_t budget = 0;                // VR_OPT_DEVICE_BUDGET (<= 0: every brick)
    float* d_pool = nullptr;           // device brick cache
    int ooc_march = 2;                 // VR_OPT_OOC_MARCH: 2 auto, 1 texture march on three layered slot
                                       // copies, 3 on one (along z), 0 direct
    bool pool_tex_on = false;          // the current cache has its layered copies
    int pool_axes = 0;                 // bit S: the cache keeps the copy along axis S
    int64_t pool_stage = 0;            // texture march: d_pool holds this many blocks, one
                                       // launch's uploads on their way into the layered
                                       // copies (0: d_pool is the cache, a block per slot)
    cudaArray_t pool_arr[3] = {nullptr, nullptr, nullptr};  // by sweep axis
    cudaTextureObject_t pool_tex[3] = {0, 0, 0};
    cudaSurfaceObject_t pool_surf[3] = {0, 0, 0};
    int32_t pool_cols[3] = {0, 0, 0};  // slots per row of each copy's texel tiling
    vr::Residency res;
    int64_t ooc_frame = 0;
    cudaStream_t copy_stream = nullptr;
    cudaStream_t ring_stream = nullptr;   // marches of streamed bricks, beside the resident ones
    cudaEvent_t ev_ring_start = nullptr, ev_ring_end = nullptr;
    cudaEvent_t ev_march_done = nullptr;  // end of the last out-of-core frame's marching
    cudaEvent_t ev_copy_done = nullptr;   // end of the last upload issued
    std::vector<cudaEvent_t> ev_chunk;
    cudaEvent_t ev_half_read[2] = {nullptr, nullptr};  // last march that read each ring half
    int32_t ring_first_half = 0;                       // ring half the next frame starts in
    std::vector<int32_t> ooc_ring;
    std::vector<int32_t> ooc_bricks, ooc_slot, ooc_up;

    // sort-last distribution: the bricks this context renders, [region_lo, region_hi)
    int32_t region_lo[3] = {0, 0, 0}, region_hi[3] = {0, 0, 0};
    float4* d_comp = nullptr;  // root fold output when the caller passes a host buffer
    size_t cap_comp = 0;

    Slot slots[kSlots];
    int next_slot = 0;
    vr_stats acc{};

    // planner scratch (host)
    std::vector<int32_t> plan_count, plan_fill, plan_sweep;
    std::vector<double> plan_qx, plan_qy;  // view-plane offsets of tile-centre columns and rows
    std::vector<vrh::CornerProj> plan_proj;  // projections of the brick grid's corner points
    std::vector<int64_t> plan_dst;          // per planned brick: where its items start in the frame's list
    struct PB {
        int32_t id;
        int32_t part;          // the host thread's share that planned it (plan_parts)
        int32_t span0, nspan;  // its tile spans there
        int32_t n_items;       // tiles it covers
    };
    std::vector<PB> plan_bricks;  // in view order
    struct PlanPart {  // one host thread's share of the bricks, kept from frame to frame
        std::vector<PB> bricks;
        std::vector<int32_t> keys;       // their view-order keys
        std::vector<int32_t> key_count;  // bricks per key, then where the first of each goes
        std::vector<vrh::Span> spans;
        std::vector<int32_t> diff;  // items per tile as a difference array per tile row
        int64_t skipped = 0, touched = 0, items = 0;
    };
    std::vector<PlanPart> plan_parts;
};

namespace vrh {

inline int fail(vr_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

inline int cuda_fail(vr_ctx* c, cudaError_t e, const char* what) {
    return fail(c, VR_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define VR_CUDA(ctx, call)                                      \
    do {                                                        \
        cudaError_t _e = (call);                                \
        if (_e != cudaSuccess) return cuda_fail(ctx, _e, #call); \
    } while (0)

template <typename T>
inline int grow_device(vr_ctx* c, T*& p, size_t& cap, size_t need) {
    if (need <= cap && p) return VR_OK;
    size_t n = std::max(need, cap + cap / 2);
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    if (cudaMalloc((void**)&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, VR_ENOMEM, "device allocation failed");
    }
    cap = n;
    return VR_OK;
}

template <typename T>
inline int grow_pinned(vr_ctx* c, T*& p, size_t& cap, size_t need) {
    if (need <= cap && p) return VR_OK;
    size_t n = std::max(need, cap + cap / 2);
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    if (cudaMallocHost((void**)&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, VR_ENOMEM, "pinned host allocation failed");
    }
    cap = n;
    return VR_OK;
}

// Wait for a slot's frame, fold its numbers into the statistics.
}  // namespace vrh

namespace vrh {

// defined in vr_host.cu
int retire(vr_ctx* c, Slot& s);
int retire_all(vr_ctx* c);
bool use_tex(vr_ctx* c);
bool use_tma(vr_ctx* c);
int prepare_tex(vr_ctx* c);
int64_t precision_bytes(int precision);
int plan_frame(vr_ctx* c, Slot& s, const int32_t win[4], int32_t& tiles_x, int32_t& tiles_y, int32_t& T,
               int64_t& n_items, bool emit = true);
void emit_items(vr_ctx* c, Slot& s, int32_t tiles_x, int32_t tiles_y, int64_t n_items);
void fill_common_params(vr_ctx* c, vr::FrameParams& p);

}  // namespace vrh
