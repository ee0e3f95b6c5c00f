/*
 * FP64 CPU oracle for the bricked volume ray caster -- TEST INFRASTRUCTURE.
 *
 * Only the test suite, the package's smoke check and the benchmark's CPU
 * baseline leg may load this file's library.  The product (the CUDA library
 * under paper_1205_0282_gb300/) never calls it and shares no code with it.
 *
 * What it computes (Hassan, Fluke & Barnes, arXiv:1205.0282):
 *   Section 2.3.2: per pixel, a ray from the viewpoint, its entry and exit with
 *   the bounding cube (rays that miss it return at once), sampling of the cube
 *   with tri-linear interpolation, accumulation of colour and opacity, and
 *   termination at the exit point or once the opacity limit is reached.
 *   Section 2.3.3: sub-images of the sub-cubes are merged by compositing; the
 *   alpha-blending operator is associative, so per-brick segments may be
 *   composited separately and folded in view order.
 *   Section 1.2: the transfer function maps each data value to colour and
 *   opacity, accumulated along the ray.
 *
 * The paper fixes none of the constants below; the readings used are:
 *   - voxel (i,j,k) sits at the point (i,j,k); the domain is [0,nx-1]x[0,ny-1]x[0,nz-1];
 *   - pinhole camera: f = |target-eye|, r = |f x up|, u = r x f; pixel (i,j), row 0 at
 *     the top, looks along |f + qx r + qy u| with qx = (2(i+.5)/W-1) tan(fovy/2) W/H,
 *     qy = (1-2(j+.5)/H) tan(fovy/2);
 *   - entry/exit by the slab test, t0 = max(t_near, 0), t1 = t_far, empty if t1 <= t0;
 *   - samples p_k = p_entry + (k dt) d for k = 0,1,... while k dt < t1 - t0;
 *   - tri-linear interpolation with p clamped to the domain, i0 = min(floor p, n-2);
 *   - piecewise-linear transfer function over control points (v,r,g,b,a), clamped
 *     to its end points; a is opacity per unit voxel of path;
 *   - opacity correction alpha = 1 - (1-a)^(dt/1 voxel);
 *   - front-to-back premultiplied compositing C += (1-A) alpha c, A += (1-A) alpha,
 *     termination once A >= term_alpha;
 *   - bricked mode: sample p_k belongs to brick floor(p/B) per axis (last brick
 *     closed); each brick's run of samples is composited from zero with its own
 *     termination, and runs are folded front to back with the 'over' operator,
 *     stopping once the accumulated A >= term_alpha.  Brick size 0 = monolithic.
 *   - maximum intensity projection (the paper's own transfer function,
 *     Section 2.3.3): the maximum interpolated value along the ray, then the
 *     colour map (the transfer function's colour and opacity at that value).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double eye[3], target[3], up[3];
    double fovy_deg;
    int32_t width, height;
    double step;
    double term_alpha;
} orc_camera;

enum { ORC_MODE_EA = 0, ORC_MODE_MIP = 1 };
enum { ORC_AMB_STEPS = 1, ORC_AMB_TERM = 2 };

/* ------------------------------------------------------------------ geometry */

static void normalize3(double v[3]) {
    double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= n;
    v[1] /= n;
    v[2] /= n;
}

static void cross3(const double a[3], const double b[3], double o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

typedef struct {
    double f[3], r[3], u[3];
    double tan_half, aspect;
} basis_t;

static void camera_basis(const orc_camera* c, basis_t* b) {
    for (int a = 0; a < 3; ++a) b->f[a] = c->target[a] - c->eye[a];
    normalize3(b->f);
    cross3(b->f, c->up, b->r);
    normalize3(b->r);
    cross3(b->r, b->f, b->u);
    b->tan_half = tan(c->fovy_deg * 3.14159265358979323846 / 360.0);
    b->aspect = (double)c->width / (double)c->height;
}

static void pixel_direction(const orc_camera* c, const basis_t* b, int i, int j, double d[3]) {
    double qx = (2.0 * (i + 0.5) / c->width - 1.0) * b->tan_half * b->aspect;
    double qy = (1.0 - 2.0 * (j + 0.5) / c->height) * b->tan_half;
    for (int a = 0; a < 3; ++a) d[a] = b->f[a] + qx * b->r[a] + qy * b->u[a];
    normalize3(d);
}

/* Slab test against [lo,hi]; returns 0 if the line misses the box. */
static int slab(const double e[3], const double d[3], const double lo[3], const double hi[3],
                double* tn, double* tf) {
    double t_near = -INFINITY, t_far = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (e[a] < lo[a] || e[a] > hi[a]) return 0;
            continue;
        }
        double ta = (lo[a] - e[a]) / d[a];
        double tb = (hi[a] - e[a]) / d[a];
        double t_min = ta < tb ? ta : tb;
        double t_max = ta < tb ? tb : ta;
        if (t_min > t_near) t_near = t_min;
        if (t_max < t_far) t_far = t_max;
    }
    *tn = t_near;
    *tf = t_far;
    return 1;
}

/* ------------------------------------------------------------- per-sample ops */

typedef struct {
    const float* v;
    int64_t n[3];
} cube_t;

static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

static double trilinear(const cube_t* c, const double p[3]) {
    int64_t i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double q = clampd(p[a], 0.0, (double)(c->n[a] - 1));
        int64_t i = (int64_t)floor(q);
        if (i > c->n[a] - 2) i = c->n[a] - 2;
        i0[a] = i;
        f[a] = q - (double)i;
    }
    const int64_t sx = 1, sy = c->n[0], sz = c->n[0] * c->n[1];
    const float* b = c->v + i0[2] * sz + i0[1] * sy + i0[0] * sx;
    /* interpolate along x, then y, then z */
    double c00 = b[0] + f[0] * ((double)b[sx] - b[0]);
    double c10 = b[sy] + f[0] * ((double)b[sy + sx] - b[sy]);
    double c01 = b[sz] + f[0] * ((double)b[sz + sx] - b[sz]);
    double c11 = b[sz + sy] + f[0] * ((double)b[sz + sy + sx] - b[sz + sy]);
    double c0 = c00 + f[1] * (c10 - c00);
    double c1 = c01 + f[1] * (c11 - c01);
    return c0 + f[2] * (c1 - c0);
}

/* Piecewise-linear transfer function; rows of 5 doubles (v, r, g, b, a). */
static void tf_eval(const double* tf, int n, double v, double out[4]) {
    if (v <= tf[0]) {
        memcpy(out, tf + 1, 4 * sizeof(double));
        return;
    }
    if (v >= tf[5 * (n - 1)]) {
        memcpy(out, tf + 5 * (n - 1) + 1, 4 * sizeof(double));
        return;
    }
    int s = 0;
    while (!(v < tf[5 * (s + 1)])) ++s; /* v_s <= v < v_{s+1} */
    const double* p0 = tf + 5 * s;
    const double* p1 = p0 + 5;
    double w = (v - p0[0]) / (p1[0] - p0[0]);
    for (int ch = 0; ch < 4; ++ch) out[ch] = p0[1 + ch] + w * (p1[1 + ch] - p0[1 + ch]);
}

static double opacity_correct(double a, double dt) { return 1.0 - pow(1.0 - a, dt / 1.0); }

/* ----------------------------------------------------------------- one pixel */

typedef struct {
    const cube_t* cube;
    const double* tf;
    int ntf;
    const orc_camera* cam;
    basis_t basis;
    int64_t brick[3]; /* 0 = monolithic */
    int64_t nb[3];
    int mode;
    double amb_alpha, amb_steps;
    const int32_t* region; /* NULL, or the region of each brick (-1: not rendered) */
    int step_mode;         /* 0: fixed step; 1: dynamic step (see render_pixel) */
} job_t;

static int64_t owner_of(const job_t* J, const double p[3]) {
    if (J->brick[0] == 0) return 0;
    int64_t id = 0, mul = 1;
    for (int a = 0; a < 3; ++a) {
        double q = clampd(p[a], 0.0, (double)(J->cube->n[a] - 1));
        int64_t b = (int64_t)floor(q / (double)J->brick[a]);
        if (b > J->nb[a] - 1) b = J->nb[a] - 1;
        if (b < 0) b = 0;
        id += b * mul;
        mul *= J->nb[a];
    }
    return id;
}

static void near_tau(const job_t* J, double A, int* amb) {
    if (fabs(A - J->cam->term_alpha) < J->amb_alpha) *amb |= ORC_AMB_TERM;
}

/* Front-to-back compositing of one sample (premultiplied): the sample's colour
 * and opacity alpha enter through the transmittance 1 - seg[3] left so far. */
static void accumulate(double seg[4], const double rgba[4], double alpha) {
    double w = (1.0 - seg[3]) * alpha;
    seg[0] += w * rgba[0];
    seg[1] += w * rgba[1];
    seg[2] += w * rgba[2];
    seg[3] += w;
}

/* over: acc <- acc over seg */
static void fold(double acc[4], const double seg[4]) {
    double t = 1.0 - acc[3];
    for (int ch = 0; ch < 4; ++ch) acc[ch] += t * seg[ch];
}

static void render_pixel(const job_t* J, int i, int j, double out[4], int* amb_out,
                         int64_t* samples_out) {
    const orc_camera* cam = J->cam;
    const cube_t* cube = J->cube;
    double d[3];
    pixel_direction(cam, &J->basis, i, j, d);
    double lo[3] = {0, 0, 0}, hi[3];
    for (int a = 0; a < 3; ++a) hi[a] = (double)(cube->n[a] - 1);
    double tn, tf;
    int amb = 0;
    int64_t ns = 0;
    out[0] = out[1] = out[2] = out[3] = 0.0;
    if (!slab(cam->eye, d, lo, hi, &tn, &tf)) goto done;
    double t0 = tn > 0.0 ? tn : 0.0, t1 = tf;
    if (!(t1 > t0)) goto done;
    /* Dynamic step (Section 2.3.2, discrete ray casting with at least one sample
     * per voxel crossed): successive samples are cam->step voxels apart along the
     * ray's dominant axis, i.e. cam->step / max_a |d_a| apart along the ray, and
     * the first sits half a step after the entry (so a ray crossing whole voxel
     * slabs samples their middles, never a face). */
    double dmax = 0.0;
    for (int a = 0; a < 3; ++a) dmax = fabs(d[a]) > dmax ? fabs(d[a]) : dmax;
    const double dt = J->step_mode ? cam->step / dmax : cam->step, tau = cam->term_alpha;
    if (J->step_mode) {
        t0 += 0.5 * dt;
        if (!(t1 > t0)) goto done;
    }
    const double L = t1 - t0;
    {
        double x = L / dt;
        if (fabs(x - nearbyint(x)) < J->amb_steps) amb |= ORC_AMB_STEPS;
    }
    double pe[3];
    for (int a = 0; a < 3; ++a) pe[a] = cam->eye[a] + t0 * d[a];

    if (J->mode == ORC_MODE_MIP) {
        double vmax = -INFINITY;
        for (int64_t k = 0;; ++k) {
            double s = (double)k * dt;
            if (!(s < L)) break;
            double p[3];
            for (int a = 0; a < 3; ++a) p[a] = pe[a] + s * d[a];
            double v = trilinear(cube, p);
            if (v > vmax) vmax = v;
            ++ns;
        }
        if (ns > 0) {
            double rgba[4];
            tf_eval(J->tf, J->ntf, vmax, rgba);
            /* colour map of the maximum, premultiplied by its opacity */
            out[0] = rgba[0] * rgba[3];
            out[1] = rgba[1] * rgba[3];
            out[2] = rgba[2] * rgba[3];
            out[3] = rgba[3];
        }
        goto done;
    }

    if (J->region) {
        /* Two-level sort-last fold (Sections 2.3.3-2.3.4): each brick's run is
         * folded into the run of its region (a box of bricks, crossed by the ray
         * in one piece), which stops taking runs once its opacity reaches tau;
         * region runs are folded into the pixel, which stops at tau.  Bricks of
         * region -1 are not rendered. */
        double acc[4] = {0, 0, 0, 0}, racc[4] = {0, 0, 0, 0}, seg[4] = {0, 0, 0, 0};
        int64_t cur = -1;
        int32_t rcur = -1;
        int seg_done = 0, stopped = 0;
        for (int64_t k = 0;; ++k) {
            double s = (double)k * dt;
            int more = s < L;
            int64_t b = -1;
            double p[3];
            if (more) {
                for (int a = 0; a < 3; ++a) p[a] = pe[a] + s * d[a];
                b = owner_of(J, p);
            }
            if (!more || b != cur) {
                /* close the run of brick cur */
                if (cur >= 0 && J->region[cur] >= 0) {
                    const int32_t r = J->region[cur];
                    if (r != rcur) {
                        if (rcur >= 0) {
                            near_tau(J, acc[3], &amb);
                            if (acc[3] < tau) fold(acc, racc);
                            near_tau(J, acc[3], &amb);
                            if (acc[3] >= tau) {
                                stopped = 1;
                                break;
                            }
                        }
                        racc[0] = racc[1] = racc[2] = racc[3] = 0.0;
                        rcur = r;
                    }
                    near_tau(J, racc[3], &amb);
                    if (racc[3] < tau) fold(racc, seg);
                    near_tau(J, racc[3], &amb);
                }
                if (!more) break;
                cur = b;
                seg[0] = seg[1] = seg[2] = seg[3] = 0.0;
                seg_done = 0;
            }
            if (seg_done || J->region[cur] < 0) continue;
            double v = trilinear(cube, p);
            double rgba[4];
            tf_eval(J->tf, J->ntf, v, rgba);
            accumulate(seg, rgba, opacity_correct(rgba[3], dt));
            ++ns;
            near_tau(J, seg[3], &amb);
            if (seg[3] >= tau) seg_done = 1;
        }
        if (!stopped && rcur >= 0) {
            near_tau(J, acc[3], &amb);
            if (acc[3] < tau) fold(acc, racc);
        }
        memcpy(out, acc, sizeof(acc));
        goto done;
    }

    double acc[4] = {0, 0, 0, 0}, seg[4] = {0, 0, 0, 0};
    int64_t cur = -1;
    int seg_done = 0, stopped = 0;
    for (int64_t k = 0;; ++k) {
        double s = (double)k * dt;
        if (!(s < L)) break;
        double p[3];
        for (int a = 0; a < 3; ++a) p[a] = pe[a] + s * d[a];
        int64_t b = owner_of(J, p);
        if (b != cur) {
            if (cur >= 0) {
                near_tau(J, acc[3], &amb);
                if (acc[3] < tau) fold(acc, seg);
                near_tau(J, acc[3], &amb);
                if (acc[3] >= tau) {
                    stopped = 1;
                    break;
                }
            }
            cur = b;
            seg[0] = seg[1] = seg[2] = seg[3] = 0.0;
            seg_done = 0;
        }
        if (seg_done) continue;
        double v = trilinear(cube, p);
        double rgba[4];
        tf_eval(J->tf, J->ntf, v, rgba);
        accumulate(seg, rgba, opacity_correct(rgba[3], dt));
        ++ns;
        near_tau(J, seg[3], &amb);
        if (seg[3] >= tau) seg_done = 1;
    }
    if (!stopped && cur >= 0) {
        near_tau(J, acc[3], &amb);
        if (acc[3] < tau) fold(acc, seg);
    }
    memcpy(out, acc, sizeof(acc));
done:
    if (amb_out) *amb_out = amb;
    if (samples_out) *samples_out = ns;
}

/* ------------------------------------------------------------------ exports */

static void setup_job(job_t* J, const cube_t* cube, const double* tf, int ntf,
                      const orc_camera* cam, const int64_t brick[3], int mode,
                      double amb_alpha, double amb_steps) {
    J->cube = cube;
    J->tf = tf;
    J->ntf = ntf;
    J->cam = cam;
    camera_basis(cam, &J->basis);
    for (int a = 0; a < 3; ++a) {
        J->brick[a] = brick[a];
        J->nb[a] = brick[a] > 0 ? (cube->n[a] - 1 + brick[a] - 1) / brick[a] : 1;
    }
    if (brick[0] <= 0 || brick[1] <= 0 || brick[2] <= 0) J->brick[0] = J->brick[1] = J->brick[2] = 0;
    J->mode = mode;
    J->amb_alpha = amb_alpha;
    J->amb_steps = amb_steps;
    J->region = NULL;
    J->step_mode = 0;
}

/*
 * Render pixels.  pixels: list of j*W+i (NULL = all W*H in row-major order).
 * out_rgba: npix x 4 doubles (premultiplied).  ambiguous: npix bytes of flag
 * bits (nullable).  samples: npix int64 counts of composited samples (nullable).
 * Returns 0 on success, -1 on bad arguments.
 */
int orc_render(const float* cube_data, int64_t nx, int64_t ny, int64_t nz,
               const double* tf, int32_t ntf, const orc_camera* cam,
               int64_t bx, int64_t by, int64_t bz, int32_t mode, int32_t step_mode,
               const int64_t* pixels, int64_t npix,
               double* out_rgba, uint8_t* ambiguous, int64_t* samples,
               double amb_alpha, double amb_steps, int32_t nthreads) {
    if (!cube_data || nx < 2 || ny < 2 || nz < 2 || !tf || ntf < 1 || !cam || !out_rgba) return -1;
    if (cam->width < 1 || cam->height < 1 || !(cam->step > 0.0)) return -1;
    cube_t cube = {cube_data, {nx, ny, nz}};
    int64_t brick[3] = {bx, by, bz};
    job_t J;
    setup_job(&J, &cube, tf, ntf, cam, brick, mode, amb_alpha, amb_steps);
    J.step_mode = step_mode;
    const int64_t W = cam->width;
    const int64_t total = pixels ? npix : W * cam->height;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < total; ++q) {
        int64_t pix = pixels ? pixels[q] : q;
        int i = (int)(pix % W), j = (int)(pix / W);
        int amb = 0;
        int64_t ns = 0;
        render_pixel(&J, i, j, out_rgba + 4 * q, &amb, &ns);
        if (ambiguous) ambiguous[q] = (uint8_t)amb;
        if (samples) samples[q] = ns;
    }
    return 0;
}

/*
 * orc_render with the two-level fold: region[b] is the region of brick b
 * (-1: brick not rendered); n_bricks must match the bricking.  Emission-
 * absorption only.  Returns 0, or -1 on bad arguments.
 */
int orc_render_regions(const float* cube_data, int64_t nx, int64_t ny, int64_t nz,
                       const double* tf, int32_t ntf, const orc_camera* cam,
                       int64_t bx, int64_t by, int64_t bz, const int32_t* region, int64_t n_bricks,
                       const int64_t* pixels, int64_t npix,
                       double* out_rgba, uint8_t* ambiguous, int64_t* samples,
                       double amb_alpha, double amb_steps, int32_t nthreads) {
    if (!cube_data || nx < 2 || ny < 2 || nz < 2 || !tf || ntf < 1 || !cam || !out_rgba || !region) return -1;
    if (cam->width < 1 || cam->height < 1 || !(cam->step > 0.0)) return -1;
    if (bx < 1 || by < 1 || bz < 1) return -1;
    cube_t cube = {cube_data, {nx, ny, nz}};
    int64_t brick[3] = {bx, by, bz};
    job_t J;
    setup_job(&J, &cube, tf, ntf, cam, brick, ORC_MODE_EA, amb_alpha, amb_steps);
    if (J.nb[0] * J.nb[1] * J.nb[2] != n_bricks) return -1;
    J.region = region;
    const int64_t W = cam->width;
    const int64_t total = pixels ? npix : W * cam->height;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < total; ++q) {
        int64_t pix = pixels ? pixels[q] : q;
        int i = (int)(pix % W), j = (int)(pix / W);
        int amb = 0;
        int64_t ns = 0;
        render_pixel(&J, i, j, out_rgba + 4 * q, &amb, &ns);
        if (ambiguous) ambiguous[q] = (uint8_t)amb;
        if (samples) samples[q] = ns;
    }
    return 0;
}

/* Ray of pixel (i,j): out = d[3], t0, t1, p_entry[3], n_samples (as double). */
int orc_pixel_ray(const orc_camera* cam, int64_t nx, int64_t ny, int64_t nz, int32_t i, int32_t j,
                  double* out) {
    basis_t b;
    camera_basis(cam, &b);
    double d[3];
    pixel_direction(cam, &b, i, j, d);
    double lo[3] = {0, 0, 0}, hi[3] = {(double)(nx - 1), (double)(ny - 1), (double)(nz - 1)};
    double tn = 0, tf = 0;
    int hit = slab(cam->eye, d, lo, hi, &tn, &tf);
    double t0 = tn > 0 ? tn : 0, t1 = tf;
    out[0] = d[0];
    out[1] = d[1];
    out[2] = d[2];
    out[3] = t0;
    out[4] = t1;
    for (int a = 0; a < 3; ++a) out[5 + a] = cam->eye[a] + t0 * d[a];
    double n = 0;
    if (hit && t1 > t0) {
        int64_t k = 0;
        while ((double)k * cam->step < t1 - t0) ++k;
        n = (double)k;
    }
    out[8] = n;
    return hit && t1 > t0;
}

/*
 * For each listed pixel, mark every brick that owns at least one of its
 * samples (no early termination): mask is npix x n_bricks bytes.
 */
int orc_pixel_bricks(const orc_camera* cam, int64_t nx, int64_t ny, int64_t nz,
                     int64_t bx, int64_t by, int64_t bz, const int64_t* pixels, int64_t npix,
                     uint8_t* mask, int64_t n_bricks) {
    cube_t cube = {NULL, {nx, ny, nz}};
    int64_t brick[3] = {bx, by, bz};
    job_t J;
    double dummy_tf[5] = {0, 0, 0, 0, 0};
    setup_job(&J, &cube, dummy_tf, 1, cam, brick, 0, 0, 0);
    if (J.nb[0] * J.nb[1] * J.nb[2] != n_bricks) return -1;
    memset(mask, 0, (size_t)(npix * n_bricks));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < npix; ++q) {
        int i = (int)(pixels[q] % cam->width), j = (int)(pixels[q] / cam->width);
        double d[3];
        pixel_direction(cam, &J.basis, i, j, d);
        double lo[3] = {0, 0, 0}, hi[3] = {(double)(nx - 1), (double)(ny - 1), (double)(nz - 1)};
        double tn, tf;
        if (!slab(cam->eye, d, lo, hi, &tn, &tf)) continue;
        double t0 = tn > 0 ? tn : 0, L = tf - t0;
        if (!(L > 0)) continue;
        double pe[3];
        for (int a = 0; a < 3; ++a) pe[a] = cam->eye[a] + t0 * d[a];
        for (int64_t k = 0;; ++k) {
            double s = (double)k * cam->step;
            if (!(s < L)) break;
            double p[3];
            for (int a = 0; a < 3; ++a) p[a] = pe[a] + s * d[a];
            mask[q * n_bricks + owner_of(&J, p)] = 1;
        }
    }
    return 0;
}

/*
 * Per-brick [min, max] over the voxels a brick's samples can touch: brick b
 * along an axis covers voxels [b*B, min((b+1)*B, n-1)] (its own plus the
 * one-voxel apron on the high side).  out: n_bricks x 2 floats, brick id
 * = bx_i + nbx*(by_i + nby*bz_i).
 */
int orc_brick_minmax(const float* cube_data, int64_t nx, int64_t ny, int64_t nz,
                     int64_t bx, int64_t by, int64_t bz, float* out) {
    int64_t n[3] = {nx, ny, nz}, B[3] = {bx, by, bz}, nb[3];
    for (int a = 0; a < 3; ++a) {
        if (B[a] < 1) return -1;
        nb[a] = (n[a] - 1 + B[a] - 1) / B[a];
    }
    const int64_t total = nb[0] * nb[1] * nb[2];
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t id = 0; id < total; ++id) {
        int64_t ix = id % nb[0], iy = (id / nb[0]) % nb[1], iz = id / (nb[0] * nb[1]);
        int64_t lo[3] = {ix * B[0], iy * B[1], iz * B[2]}, hi[3];
        int64_t idx[3] = {ix, iy, iz};
        for (int a = 0; a < 3; ++a) {
            hi[a] = (idx[a] + 1) * B[a];
            if (hi[a] > n[a] - 1) hi[a] = n[a] - 1;
        }
        float mn = INFINITY, mx = -INFINITY;
        for (int64_t z = lo[2]; z <= hi[2]; ++z)
            for (int64_t y = lo[1]; y <= hi[1]; ++y)
                for (int64_t x = lo[0]; x <= hi[0]; ++x) {
                    float v = cube_data[(z * ny + y) * nx + x];
                    if (v < mn) mn = v;
                    if (v > mx) mx = v;
                }
        out[2 * id] = mn;
        out[2 * id + 1] = mx;
    }
    return 0;
}

/* Maximum of the transfer function's opacity a over the closed interval [lo, hi]. */
double orc_tf_alpha_max(const double* tf, int32_t ntf, double lo, double hi) {
    double rgba[4];
    tf_eval(tf, ntf, lo, rgba);
    double m = rgba[3];
    tf_eval(tf, ntf, hi, rgba);
    if (rgba[3] > m) m = rgba[3];
    for (int s = 0; s < ntf; ++s) {
        double v = tf[5 * s];
        if (v > lo && v < hi && tf[5 * s + 4] > m) m = tf[5 * s + 4];
    }
    return m;
}
