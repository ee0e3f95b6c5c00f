// Texture-gather ray march: the same per-pixel ray casting of one brick as the
// direct kernel (Section 2.3.2 of arXiv:1205.0282), with the eight trilinear
// corners fetched by two 4-texel gathers (tld4) from layered 2D textures.
//
// The paper stores its sub-cubes in texture memory and lets the texture unit
// interpolate; here the texture unit only gathers: tld4 returns the four texels of
// a 2x2 footprint unchanged, and the interpolation weights are applied in FP32 as
// in the other kernels, so no reduced-precision filtering enters the result.  The
// cube is held three times, as layered textures whose layers run along x, y and z;
// an item reads the copy whose layers run along its dominant ray axis, so the 32
// rays of a warp sample one or two layers at a time and the gathers stay local in
// the texture cache.
#include <cuda.h>

#include <cfloat>
#include <cstdint>

#include "vr_device.cuh"

namespace vr {

namespace texm {

// Layered texture of the sweep axis S: layer index = coordinate along S, texel
// (x, y) = coordinates along (U, V) with U < V the two other axes.
template <int S>
struct Axes {
    static constexpr int U = S == 0 ? 1 : 0;
    static constexpr int V = S == 2 ? 1 : 2;
};

// 2x2 texels (u, v), (u+1, v), (u, v+1), (u+1, v+1) of one layer.  With
// unnormalised coordinates the gather footprint of point (x, y) starts at texel
// floor(x - 0.5), so (u + 1, v + 1) selects texels u, u+1 and v, v+1; the four
// components come back as (u, v+1), (u+1, v+1), (u+1, v), (u, v).
__device__ __forceinline__ void gather4(cudaTextureObject_t t, int layer, float x, float y, float& c00,
                                        float& c10, float& c01, float& c11) {
    float r0, r1, r2, r3;
    asm("tld4.r.a2d.v4.f32.f32 {%0, %1, %2, %3}, [%4, {%5, %6, %7, %8}];"
                 : "=f"(r0), "=f"(r1), "=f"(r2), "=f"(r3)
                 : "l"(t), "r"(layer), "f"(x), "f"(y), "f"(0.0f));
    c01 = r0;
    c11 = r1;
    c10 = r2;
    c00 = r3;
}

template <int S, bool UNIFORM>
__device__ __forceinline__ void march_item(const FrameParams& p, const Item& item, const float4* s_rgba,
                                           const float* s_v) {
    constexpr int U = Axes<S>::U, V = Axes<S>::V;
    const cudaTextureObject_t tex = p.tex[S];
    const int lx = threadIdx.x % kTile, ly = threadIdx.x / kTile;
    const int tx = item.tile % p.tiles_x, ty = item.tile / p.tiles_x;
    const int i = tx * kTile + lx, j = ty * kTile + ly;
    int bidx[3], O[3], imax[3];
    bidx[0] = item.brick % p.nb[0];
    bidx[1] = (item.brick / p.nb[0]) % p.nb[1];
    bidx[2] = item.brick / (p.nb[0] * p.nb[1]);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        O[a] = bidx[a] * p.B[a];
        imax[a] = min(p.B[a] - 1, p.n[a] - 2 - O[a]);
    }
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float fk = 0.0f, fn = 0.0f;
    float qs[3] = {0, 0, 0}, dq[3] = {0, 0, 0};
    {
        df d[3], pe[3];
        int n_samples = 0;
        if (i < p.width && j < p.height && setup_ray(p, i, j, d, pe, n_samples)) {
            int klo, khi;
            brick_range(p, bidx, d, pe, n_samples, klo, khi);
            if (khi > klo) {
                fn = (float)(khi - klo);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const df D = df_mul(p.dt, d[a]);
                    qs[a] = df_to_float(df_add_f(df_add(pe[a], df_mul_f(D, (float)klo)), -(float)O[a]));
                    dq[a] = df_to_float(D);
                }
            }
        }
    }
    const float tau = p.tau;
    // brick origin along U, V plus one: gather coordinate of texel (u, v) is (u + 1, v + 1)
    const float ou = (float)(O[U] + 1), ov = (float)(O[V] + 1);
    // Sample k's eight corners and weights.  The loop is software-pipelined: the
    // gathers of sample k + 1 are issued before sample k is interpolated and
    // composited, so texture latency overlaps the arithmetic.
    struct Corners {
        float c[8];  // (u, v, s) corners: c[0..3] in plane ps, c[4..7] in plane ps + 1
        float fu, fv, fs;
    };
    auto fetch = [&](float f, Corners& s) {
        const float qS = fmaf(f, dq[S], qs[S]);
        const float qU = fmaf(f, dq[U], qs[U]);
        const float qV = fmaf(f, dq[V], qs[V]);
        // samples sit inside the brick up to rounding: truncation is the floor for
        // q > -1; the lattice clamp matters only at the far face
        const int ps = min(__float2int_rz(qS), imax[S]);
        const int iu = min(__float2int_rz(qU), imax[U]);
        const int iv = min(__float2int_rz(qV), imax[V]);
        s.fs = qS - (float)ps;
        s.fu = qU - (float)iu;
        s.fv = qV - (float)iv;
        const float x = ou + (float)iu, y = ov + (float)iv;
        gather4(tex, O[S] + ps, x, y, s.c[0], s.c[1], s.c[2], s.c[3]);
        gather4(tex, O[S] + ps + 1, x, y, s.c[4], s.c[5], s.c[6], s.c[7]);
    };
    Corners nxt;
    if (fk < fn) fetch(fk, nxt);
    while (fk < fn) {
        const Corners cur = nxt;
        if (fk + 1.0f < fn) fetch(fk + 1.0f, nxt);
        const float e00 = fmaf(cur.fu, cur.c[1] - cur.c[0], cur.c[0]);
        const float e10 = fmaf(cur.fu, cur.c[3] - cur.c[2], cur.c[2]);
        const float e01 = fmaf(cur.fu, cur.c[5] - cur.c[4], cur.c[4]);
        const float e11 = fmaf(cur.fu, cur.c[7] - cur.c[6], cur.c[6]);
        const float e0 = fmaf(cur.fv, e10 - e00, e00);
        const float e1 = fmaf(cur.fv, e11 - e01, e01);
        const float val = fmaf(cur.fs, e1 - e0, e0);
        const float4 col = tf_lookup<UNIFORM>(p, s_rgba, s_v, val);
        const float alpha = opacity_correct(p, col.w);
        const float w = (1.0f - acc.w) * alpha;
        acc.x = fmaf(w, col.x, acc.x);
        acc.y = fmaf(w, col.y, acc.y);
        acc.z = fmaf(w, col.z, acc.z);
        acc.w += w;
        fk += 1.0f;
        if (acc.w >= tau) fn = fk;
    }
    p.frags[(int64_t)item.frag * kTilePixels + threadIdx.x] = acc;
    unsigned long long t = (unsigned long long)fk;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0 && t) atomicAdd(&p.stats->samples, t);
}

// The transfer function lives in dynamic shared memory sized to the control points,
// so that almost all of the SM's L1/shared array stays texture cache.
template <bool UNIFORM>
__global__ void __launch_bounds__(kTilePixels, 20) march_tex_kernel(const FrameParams p) {
    extern __shared__ float4 s_dyn[];
    float4* s_rgba = s_dyn;
    float* s_v = reinterpret_cast<float*>(s_dyn + p.tf_n + 1);
    for (int k = threadIdx.x; k <= p.tf_n; k += blockDim.x) {
        s_rgba[k] = p.tf_rgba[k];
        if (k < p.tf_n) s_v[k] = p.tf_v[k];
    }
    __syncthreads();
    const Item item = p.items[blockIdx.x];
    switch (item.sweep & 3) {
        case 0: march_item<0, UNIFORM>(p, item, s_rgba, s_v); break;
        case 1: march_item<1, UNIFORM>(p, item, s_rgba, s_v); break;
        default: march_item<2, UNIFORM>(p, item, s_rgba, s_v); break;
    }
}

// Copy the stored cube a[z][y][x] (row pitch a_pitch floats) into the layered
// array of sweep axis S through its surface: layer = coordinate along S.
template <int S>
__global__ void fill_layers_kernel(const float* __restrict__ a, int64_t nx, int64_t ny, int64_t nz,
                                   int64_t a_pitch, cudaSurfaceObject_t surf) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t y = blockIdx.y;
    const int64_t z = blockIdx.z;
    if (x >= nx) return;
    const float v = a[(z * ny + y) * a_pitch + x];
    const int64_t c[3] = {x, y, z};
    constexpr int U = Axes<S>::U, V = Axes<S>::V;
    surf2DLayeredwrite(v, surf, (int)(c[U] * sizeof(float)), (int)c[V], (int)c[S]);
}

}  // namespace texm

cudaError_t launch_march_tex(const FrameParams& p, cudaStream_t s) {
    if (p.n_items == 0) return cudaSuccess;
    const size_t smem = (size_t)(p.tf_n + 1) * sizeof(float4) + (size_t)p.tf_n * sizeof(float);
    // shared-memory carveout just large enough for 20 resident CTAs (each also
    // reserves 1 KB); the rest of the SM's 256 KB array is L1/texture cache
    const int pct = (int)((20 * (smem + 1024) * 100 + 233471) / 233472) + 2;
    auto go = [&](auto kern) {
        static int carveout = -1;
        if (carveout != pct) {
            cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
            carveout = pct;
        }
        kern<<<p.n_items, kTilePixels, smem, s>>>(p);
    };
    if (p.tf_uniform) go(texm::march_tex_kernel<true>);
    else go(texm::march_tex_kernel<false>);
    return cudaGetLastError();
}

cudaError_t fill_tex_layers(const float* a, int64_t nx, int64_t ny, int64_t nz, int64_t a_pitch, int S,
                            cudaSurfaceObject_t surf, cudaStream_t s) {
    dim3 grid((unsigned)((nx + 255) / 256), (unsigned)ny, (unsigned)nz);
    if (S == 0) texm::fill_layers_kernel<0><<<grid, 256, 0, s>>>(a, nx, ny, nz, a_pitch, surf);
    else if (S == 1) texm::fill_layers_kernel<1><<<grid, 256, 0, s>>>(a, nx, ny, nz, a_pitch, surf);
    else texm::fill_layers_kernel<2><<<grid, 256, 0, s>>>(a, nx, ny, nz, a_pitch, surf);
    return cudaGetLastError();
}

}  // namespace vr
