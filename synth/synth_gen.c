/*
 * Seeded synthetic spectral-cube generator (inputs only).
 *
 * This file produces the float32 data cubes that both the GPU renderer and the
 * FP64 oracle consume.  It holds none of the rendering method's arithmetic:
 * no rays, no interpolation, no transfer function, no compositing.
 *
 * Cube layout: float32[nz][ny][nx], x fastest.  Axes follow an HI survey cube
 * (x = RA, y = Dec, z = frequency), the data type the paper renders
 * (Section 1.1, Table 1).
 *
 * Noise: for voxel linear index i, two 64-bit words come from SplitMix64
 * (Steele, Lea & Flood 2014, the published finaliser constants) applied to a
 * counter built from (seed, 2i) and (seed, 2i+1); each gives a uniform in
 * (0, 1], and the Box-Muller transform turns the pair into one N(0, sigma^2)
 * value.  Voxels are independent, so any thread split gives the same bytes.
 *
 * Sources: a list of axis-aligned 3D Gaussians, each
 *   A * exp(-((x-x0)^2 + (y-y0)^2) / (2 s_sp^2) - (z-z0)^2 / (2 s_sp_f^2)),
 * summed over a +-4 sigma box; "continuum" sources have no spectral term and
 * extend over the whole z axis.  Sources are added in list order per z plane,
 * so the result does not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

static inline uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* uniform in (0, 1] with 53 random bits */
static inline double u01(uint64_t h) {
    return (double)((h >> 11) + 1) * (1.0 / 9007199254740992.0);
}

static inline uint64_t counter_key(uint64_t seed, uint64_t c) {
    return splitmix64(seed * 0xD1B54A32D192ED03ULL) ^ (c * 0x9E3779B97F4A7C15ULL);
}

/* Fill cube[0 .. nx*ny*nz) with N(0, sigma^2) noise. */
void synth_noise(float* cube, int64_t nx, int64_t ny, int64_t nz, uint64_t seed, double sigma) {
    const int64_t n = nx * ny * nz;
    const double two_pi = 6.283185307179586476925286766559;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double u1 = u01(splitmix64(counter_key(seed, 2 * (uint64_t)i)));
        double u2 = u01(splitmix64(counter_key(seed, 2 * (uint64_t)i + 1)));
        double r = sqrt(-2.0 * log(u1));
        cube[i] = (float)(sigma * r * cos(two_pi * u2));
    }
}

/*
 * Add Gaussian sources.  src is n_src rows of 7 doubles:
 *   amplitude, x0, y0, z0, sigma_spatial, sigma_spectral, continuum_flag
 * continuum_flag != 0 means no spectral profile (constant along z).
 */
void synth_add_sources(float* cube, int64_t nx, int64_t ny, int64_t nz,
                       const double* src, int64_t n_src) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t z = 0; z < nz; ++z) {
        for (int64_t s = 0; s < n_src; ++s) {
            const double* p = src + 7 * s;
            const double amp = p[0], x0 = p[1], y0 = p[2], z0 = p[3];
            const double ss = p[4], sf = p[5];
            const int continuum = p[6] != 0.0;
            double wz = 1.0;
            if (!continuum) {
                double dz = (double)z - z0;
                if (fabs(dz) > 4.0 * sf) continue;
                wz = exp(-dz * dz / (2.0 * sf * sf));
            }
            int64_t xlo = (int64_t)floor(x0 - 4.0 * ss), xhi = (int64_t)ceil(x0 + 4.0 * ss);
            int64_t ylo = (int64_t)floor(y0 - 4.0 * ss), yhi = (int64_t)ceil(y0 + 4.0 * ss);
            if (xlo < 0) xlo = 0;
            if (ylo < 0) ylo = 0;
            if (xhi > nx - 1) xhi = nx - 1;
            if (yhi > ny - 1) yhi = ny - 1;
            for (int64_t y = ylo; y <= yhi; ++y) {
                double dy = (double)y - y0;
                for (int64_t x = xlo; x <= xhi; ++x) {
                    double dx = (double)x - x0;
                    double w = exp(-(dx * dx + dy * dy) / (2.0 * ss * ss)) * wz;
                    float* c = cube + (z * ny + y) * nx + x;
                    *c = (float)((double)*c + amp * w);
                }
            }
        }
    }
}

/*
 * One block of a cube of nx x ny x nz voxels, without the rest of the cube:
 * voxel (origin[0] + i, origin[1] + j, origin[2] + k), i < extent[0], j < extent[1],
 * k < extent[2], goes to dst[k * slice + j * row + i].  The values are those that
 * synth_noise followed by synth_add_sources give for the whole cube with the same
 * seed, sigma and source list, bit for bit: a voxel's noise depends only on its
 * linear index, and the sources whose boxes reach the block are added to each
 * voxel in list order with the same expressions.  Single-threaded: callers run
 * blocks in parallel.
 */
void synth_block(float* dst, int64_t row, int64_t slice, const int64_t origin[3], const int32_t extent[3],
                 int64_t nx, int64_t ny, int64_t nz, uint64_t seed, double sigma, const double* src, int64_t n_src) {
    const double two_pi = 6.283185307179586476925286766559;
    const int64_t bx0 = origin[0], by0 = origin[1], bz0 = origin[2];
    const int64_t bx1 = bx0 + extent[0] - 1, by1 = by0 + extent[1] - 1, bz1 = bz0 + extent[2] - 1;
    (void)nz;
    for (int64_t z = bz0; z <= bz1; ++z)
        for (int64_t y = by0; y <= by1; ++y) {
            float* out = dst + (z - bz0) * slice + (y - by0) * row - bx0;
            const uint64_t base = (uint64_t)((z * ny + y) * nx);
            for (int64_t x = bx0; x <= bx1; ++x) {
                const uint64_t i = base + (uint64_t)x;
                double u1 = u01(splitmix64(counter_key(seed, 2 * i)));
                double u2 = u01(splitmix64(counter_key(seed, 2 * i + 1)));
                double r = sqrt(-2.0 * log(u1));
                out[x] = (float)(sigma * r * cos(two_pi * u2));
            }
        }
    for (int64_t s = 0; s < n_src; ++s) {
        const double* p = src + 7 * s;
        const double amp = p[0], x0 = p[1], y0 = p[2], z0 = p[3];
        const double ss = p[4], sf = p[5];
        const int continuum = p[6] != 0.0;
        int64_t xlo = (int64_t)floor(x0 - 4.0 * ss), xhi = (int64_t)ceil(x0 + 4.0 * ss);
        int64_t ylo = (int64_t)floor(y0 - 4.0 * ss), yhi = (int64_t)ceil(y0 + 4.0 * ss);
        if (xlo < 0) xlo = 0;
        if (ylo < 0) ylo = 0;
        if (xhi > nx - 1) xhi = nx - 1;
        if (yhi > ny - 1) yhi = ny - 1;
        if (xlo < bx0) xlo = bx0;
        if (ylo < by0) ylo = by0;
        if (xhi > bx1) xhi = bx1;
        if (yhi > by1) yhi = by1;
        if (xlo > xhi || ylo > yhi) continue;
        if (!continuum && (z0 + 4.0 * sf < (double)bz0 || z0 - 4.0 * sf > (double)bz1)) continue;
        for (int64_t z = bz0; z <= bz1; ++z) {
            double wz = 1.0;
            if (!continuum) {
                double dz = (double)z - z0;
                if (fabs(dz) > 4.0 * sf) continue;
                wz = exp(-dz * dz / (2.0 * sf * sf));
            }
            for (int64_t y = ylo; y <= yhi; ++y) {
                double dy = (double)y - y0;
                float* out = dst + (z - bz0) * slice + (y - by0) * row - bx0;
                for (int64_t x = xlo; x <= xhi; ++x) {
                    double dx = (double)x - x0;
                    double w = exp(-(dx * dx + dy * dy) / (2.0 * ss * ss)) * wz;
                    float* c = out + x;
                    *c = (float)((double)*c + amp * w);
                }
            }
        }
    }
}

/* A procedural cube as a block source: the layout of the renderer library's
 * brick-provider callback (origin, extent, destination, row and slice strides in
 * floats), returning 0. */
typedef struct {
    int64_t n[3];
    uint64_t seed;
    double sigma;
    const double* src;
    int64_t n_src;
} synth_cube;

int synth_cube_block(void* user, const int64_t origin[3], const int32_t extent[3], float* dst, int64_t row,
                     int64_t slice) {
    const synth_cube* c = (const synth_cube*)user;
    if (!c || !dst) return 1;
    for (int a = 0; a < 3; ++a)
        if (origin[a] < 0 || extent[a] < 1 || origin[a] + extent[a] > c->n[a]) return 2;
    if (row < extent[0] || slice < row * extent[1]) return 3;
    synth_block(dst, row, slice, origin, extent, c->n[0], c->n[1], c->n[2], c->seed, c->sigma, c->src, c->n_src);
    return 0;
}
