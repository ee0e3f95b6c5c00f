// Texture-gather ray march: the same per-pixel ray casting of one brick as the
// direct kernel (Section 2.3.2 of arXiv:1205.0282), with the eight trilinear
// corners fetched by two 4-texel gathers (tld4) from layered 2D textures.
//
// The paper stores its sub-cubes in texture memory and lets the texture unit
// interpolate; here the texture unit only gathers: tld4 returns the four texels of
// a 2x2 footprint unchanged, and the interpolation weights are applied in FP32 as
// in the other kernels, so no reduced-precision filtering enters the result.  The
// cube is held three times, as layered textures whose layers run along x, y and z
// (each split along its layers into slabs of whole bricks plus one apron layer);
// an item reads the copy whose layers run along its dominant ray axis, so the 32
// rays of a warp sample one or two layers at a time and the gathers stay local in
// the texture cache.
#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cfloat>
#include <cstdint>

#include "vr_device.cuh"

namespace vr {

namespace texm {

#ifndef VR_TEX_DEPTH_F32
#define VR_TEX_DEPTH_F32 3
#endif
#ifndef VR_TEX_BLOCKS_F32
#define VR_TEX_BLOCKS_F32 12
#endif
#ifndef VR_TEX_DEPTH_F16
#define VR_TEX_DEPTH_F16 2
#endif
#ifndef VR_TEX_BLOCKS_F16
#define VR_TEX_BLOCKS_F16 14
#endif
#ifndef VR_TEX_DEPTH_F8
#define VR_TEX_DEPTH_F8 1
#endif
#ifndef VR_TEX_BLOCKS_F8
#define VR_TEX_BLOCKS_F8 16
#endif
// Samples whose gathers are in flight ahead of the one being composited, and
// resident CTAs per SM the kernels are compiled for (12: 80 registers a thread;
// 14: 72; 16: 64).  Measured on the 1080p orbit of the 8 GiB cube: for FP32, three
// samples ahead at 12 CTAs (1.5% faster than two ahead at 14, which beat one
// ahead at 16-20 and four ahead at 10); FP16 two ahead at 14; FP8, whose decode
// makes it ALU-bound, is fastest one ahead at 16 (two ahead: 10% slower).
__host__ __device__ constexpr int tex_depth(int prec) {
    return prec == kPrecF8 ? VR_TEX_DEPTH_F8 : (prec == kPrecF16 ? VR_TEX_DEPTH_F16 : VR_TEX_DEPTH_F32);
}
__host__ __device__ constexpr int tex_blocks_per_sm(int prec) {
    return prec == kPrecF8 ? VR_TEX_BLOCKS_F8 : (prec == kPrecF16 ? VR_TEX_BLOCKS_F16 : VR_TEX_BLOCKS_F32);
}

// Transfer-function colour at v from the control points rgba[] and their forward
// differences drgba[k] = rgba[k + 1] - rgba[k] (formed in FP32 once per CTA, so
// rgba[k] + w drgba[k] rounds exactly like the per-sample lerp of two points).
// The transfer function and termination an item composites with: the launch's
// (single frames), or its frame's own (a serving batch that mixes transfer
// functions and termination thresholds; its control points sit at offset tf_off
// of the batch's shared-memory arrays).
struct TfView {
    float v0, inv_dv, tau;
    int n;
};
__device__ __forceinline__ TfView tf_view(const FrameParams& p, const FrameParams&) {
    return TfView{p.tf_v0, p.tf_inv_dv, p.tau, p.tf_n};
}
__device__ __forceinline__ TfView tf_view(const FrameParams&, const FrameCam& c) {
    return TfView{c.tf_v0, c.tf_inv_dv, c.tau, c.tf_n};
}

template <bool UNIFORM>
__device__ __forceinline__ float4 tf_lerp(const TfView& p, const float4* __restrict__ rgba,
                                          const float4* __restrict__ drgba, const float* __restrict__ vals,
                                          float v) {
    int seg;
    float w;
    if (UNIFORM) {
        // drgba[n - 1] = 0 (rgba[n] repeats the last point): x = n - 1 needs no
        // segment clamp
        float x = (v - p.v0) * p.inv_dv;
        x = fminf(fmaxf(x, 0.0f), (float)(p.n - 1));
        seg = __float2int_rz(x);
        w = x - (float)seg;
    } else {
        int lo = 0, hi = p.n - 1;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (v >= vals[mid]) lo = mid;
            else hi = mid;
        }
        seg = lo;
        w = (v - vals[seg]) / (vals[seg + 1] - vals[seg]);
        w = fminf(fmaxf(w, 0.0f), 1.0f);
    }
    const float4 c0 = rgba[seg], d = drgba[seg];
    return make_float4(fmaf(w, d.x, c0.x), fmaf(w, d.y, c0.y), fmaf(w, d.z, c0.z), fmaf(w, d.w, c0.w));
}

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

// FP8 E4M3 storage: the codes sit in a signed 8-bit texture, so the gather
// returns each code sign-extended to 32 bits.
__device__ __forceinline__ void gather4_codes(cudaTextureObject_t t, int layer, float x, float y,
                                              int& c00, int& c10, int& c01, int& c11) {
    int r0, r1, r2, r3;
    asm("tld4.r.a2d.v4.s32.f32 {%0, %1, %2, %3}, [%4, {%5, %6, %7, %8}];"
        : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
        : "l"(t), "r"(layer), "f"(x), "f"(y), "f"(0.0f));
    c01 = r0;
    c11 = r1;
    c10 = r2;
    c00 = r3;
}

// Value of a sign-extended E4M3 code r times 2^-120, by moving its fields into an
// FP32 word: shifted left by 20, the code's sign lands in bit 31 (the sign
// extension fills bits 27..30, which the mask clears) and its exponent e (bias 7)
// and 3 mantissa bits in bits 26..20, i.e. in the low exponent bits and the top
// of the FP32 mantissa.  A normal code then reads as 2^(e-127) (1 + m/8) and a
// subnormal one (e = 0) as the FP32 denormal m 2^20 2^-149 = (m/8) 2^-6 2^-120:
// both are the code's value times 2^-120, exactly.
__device__ __forceinline__ float e4m3_times_2m120(int r) {
    return __uint_as_float(((unsigned)r << 20) & 0x87f00000u);
}

// (lo, hi) E4M3 codes -> their values through the hardware conversion e4m3x2 ->
// f16x2 (used by the per-brick range of the stored values)
__device__ __forceinline__ float2 e4m3_pair(unsigned lo, unsigned hi) {
    const unsigned short packed = (unsigned short)((lo & 0xffu) | ((hi & 0xffu) << 8));
    unsigned h2;
    asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h2) : "h"(packed));
    const __half2 hh = *reinterpret_cast<const __half2*>(&h2);
    return __half22float2(hh);
}

// E4M3 code of x (saturating to the largest finite value 448)
__device__ __forceinline__ unsigned e4m3_code(float x) {
    unsigned short d;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(d) : "f"(0.0f), "f"(x));
    return d & 0xffu;
}

// Brick-index step along axis a.
__device__ __forceinline__ int step_of(const FrameParams& p, int a) {
    return a == 0 ? 1 : (a == 1 ? p.nb[0] : p.nb[0] * p.nb[1]);
}

// MODE 0: emission-absorption compositing; MODE 1: maximum intensity projection
// (Section 2.3.2; the colour map is applied by the composite), FP32 storage only.
// POOL: the brick is read from its out-of-core cache slot's layered copy (FP32).
template <int S, bool UNIFORM, int PREC, bool DYN, class Cam, int MODE = 0, bool POOL = false>
__device__ __forceinline__ void march_item(const FrameParams& p, const Cam& cam, const Item& item,
                                           const float4* s_rgba, const float4* s_drgba, const float* s_v,
                                           int t) {
    constexpr int U = Axes<S>::U, V = Axes<S>::V;
    const int lx = t % kTile, ly = t / kTile;  // pixel t of the item's tile
    const int tx = item.tile % cam.tiles_x, ty = item.tile / cam.tiles_x;
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
    // the slab of the layered copy that holds this brick, and the brick's first
    // layer in it (out-of-core: the brick's slot in the pool's layered copy, its
    // layers 0..B)
    cudaTextureObject_t tex;
    int lay0;
    int slot_u = 0, slot_v = 0;
    if constexpr (POOL) {
        const int slot = p.slot_of[item.brick];
        tex = p.pool_tex[S];
        lay0 = 0;
        slot_u = (slot % p.pool_cols[S]) * (p.B[U] + 1) - O[U];
        slot_v = (slot / p.pool_cols[S]) * (p.B[V] + 1) - O[V];
    } else {
        const int slab = bidx[S] / p.tex_slab_bricks[S];
        tex = p.tex[S][slab];
        lay0 = O[S] - slab * p.tex_slab_bricks[S] * p.B[S];
    }
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float vmax = -FLT_MAX;  // MIP: running maximum
    float fn = 0.0f;  // samples this ray owes the brick (after termination: those composited)
    float qs[3] = {0, 0, 0}, dq[3] = {0, 0, 0};
    float dt_ray = 0.0f;  // dynamic step: this ray's spacing (voxels)
    {
        df d[3], pe[3], dt, inv_D[3];
        int n_samples = 0;
        if (i < cam.width && j < cam.height && setup_ray<DYN>(p, cam, i, j, d, pe, n_samples, dt, inv_D)) {
            int klo, khi;
            brick_range(p, bidx, d, pe, n_samples, inv_D, klo, khi);
            if (DYN) dt_ray = df_to_float(dt);
            if (khi > klo) {
                fn = (float)(khi - klo);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const df D = df_mul(dt, d[a]);
                    qs[a] = df_to_float(df_add_f(df_add(pe[a], df_mul_f(D, (float)klo)), -(float)O[a]));
                    dq[a] = df_to_float(D);
                }
            }
        }
    }
    const TfView tfv = tf_view(p, cam);
    const float tau = tfv.tau;
    // brick origin along U, V plus one: gather coordinate of texel (u, v) is (u + 1, v + 1)
    const float ou = (float)(O[U] + slot_u + 1), ov = (float)(O[V] + slot_v + 1);
    // Sample k's eight corners and weights, gathered D samples ahead of their use
    // (the software pipeline below).
    struct Corners {
        float c[8];  // (u, v, s) corners: c[0..3] in plane ps, c[4..7] in plane ps + 1
                     // (FP8: the raw codes, decoded when the sample is used, so that the
                     // gathers stay in flight across one sample's compositing)
        float fu, fv, fs;
        int halo;    // FP8: bit a set if the cell's +1 corners along U, V, S (a = 0, 1, 2)
                     // lie in the next brick
    };
    // FP8: corners read back as code * scale of the brick that owns them.  The
    // interpolation runs on code values * 2^-120 and the result is multiplied once
    // by k0 = 2^120 s_b (trilinear weights sum to one; the power of two is exact).
    // The +1 corners on the brick's far faces belong to the next brick along that
    // axis, if there is one (a rare case: those corners are rescaled by the ratio
    // of the two bricks' scales).  lim_a is the cell index along axis a whose +1
    // corner lies in the next brick (-1: none).
    float k0 = 1.0f, s0 = 1.0f;
    int lim_u = -1, lim_v = -1, lim_s = -1;
    if (PREC == kPrecF8) {
        s0 = p.brick_scale[item.brick];
        k0 = s0 * 0x1p120f;
        if (bidx[U] + 1 < p.nb[U]) lim_u = p.B[U] - 1;
        if (bidx[V] + 1 < p.nb[V]) lim_v = p.B[V] - 1;
        if (bidx[S] + 1 < p.nb[S]) lim_s = p.B[S] - 1;
    }
    const float2 dqUV = make_float2(dq[U], dq[V]), qsUV = make_float2(qs[U], qs[V]);
    const float2 oUV = make_float2(ou, ov);
    auto fetch = [&](float f, Corners& s) {
        // positions, fractions and texel coordinates along (U, V) as packed FP32x2
        // operations (each lane rounds like the scalar one)
        const float qS = fmaf(f, dq[S], qs[S]);
        const float2 qUV = __ffma2_rn(make_float2(f, f), dqUV, qsUV);
        // Samples sit inside the brick up to rounding: truncation is the floor for
        // q > -1.  A sample on the brick's far face (q = B: the cube's far face, or
        // rounding) has cell index B and weight 0 on its +1 corners, which FP32 and
        // FP16 read from the global texture (at a clamped coordinate beyond the
        // cube).  FP8 clamps the index to the lattice instead, since its +1 corners
        // are rescaled by the scale of the brick that owns them.
        int ps = __float2int_rz(qS), iu = __float2int_rz(qUV.x), iv = __float2int_rz(qUV.y);
        if (PREC == kPrecF8) {
            ps = min(ps, imax[S]);
            iu = min(iu, imax[U]);
            iv = min(iv, imax[V]);
        }
        const float2 fUV = make_float2((float)iu, (float)iv);
        s.fs = qS - (float)ps;
        const float2 fr = __fadd2_rn(qUV, make_float2(-fUV.x, -fUV.y));
        s.fu = fr.x;
        s.fv = fr.y;
        const float2 xy = __fadd2_rn(oUV, fUV);
        if (PREC != kPrecF8) {
            // FP32 and FP16 textures both return FP32 values
            gather4(tex, lay0 + ps, xy.x, xy.y, s.c[0], s.c[1], s.c[2], s.c[3]);
            gather4(tex, lay0 + ps + 1, xy.x, xy.y, s.c[4], s.c[5], s.c[6], s.c[7]);
        } else {
            int k[8];
            gather4_codes(tex, lay0 + ps, xy.x, xy.y, k[0], k[1], k[2], k[3]);
            gather4_codes(tex, lay0 + ps + 1, xy.x, xy.y, k[4], k[5], k[6], k[7]);
#pragma unroll
            for (int c = 0; c < 8; ++c) s.c[c] = __int_as_float(k[c]);
            s.halo = (iu == lim_u ? 1 : 0) | (iv == lim_v ? 2 : 0) | (ps == lim_s ? 4 : 0);
        }
    };
    // FP8 corners of a fetched sample: code value * 2^-120 (* s_owner / s_b on the
    // far faces)
    auto decode = [&](Corners& s) {
        if (PREC != kPrecF8) return;
#pragma unroll
        for (int c = 0; c < 8; ++c) s.c[c] = e4m3_times_2m120(__float_as_int(s.c[c]));
        if (s.halo) {
#pragma unroll
            for (int c = 1; c < 8; ++c) {
                const int off = ((c & 1) && (s.halo & 1) ? step_of(p, U) : 0) +
                                ((c & 2) && (s.halo & 2) ? step_of(p, V) : 0) +
                                ((c & 4) && (s.halo & 4) ? step_of(p, S) : 0);
                if (off) s.c[c] *= __ldg(p.brick_scale + item.brick + off) / s0;
            }
        }
    };
    // Step fi of the march: interpolate the fetched corners, look up and correct
    // the transfer function and composite sample fi if it is still owed (fi < fn;
    // fn drops to the terminating sample's index + 1 when alpha reaches tau).  A
    // step past the end composites with weight 0, which leaves acc unchanged: the
    // gathered values are finite (clamped texture reads) and the transfer-function
    // index is clamped, so col and alpha are finite too.
    float fi = 0.0f;
    auto step = [&](Corners& cur) {
        decode(cur);
        // along S first, two corners per packed FP32x2 operation: the gather leaves
        // (c[2], c[3]) and (c[1], c[0]) in register pairs (FP8: the decoded values)
        const float2 fs2 = make_float2(cur.fs, cur.fs);
        const float2 a10 = make_float2(cur.c[1], cur.c[0]), a23 = make_float2(cur.c[2], cur.c[3]);
        const float2 b10 = make_float2(cur.c[5], cur.c[4]), b23 = make_float2(cur.c[6], cur.c[7]);
        const float2 s10 = __ffma2_rn(fs2, __fadd2_rn(b10, make_float2(-a10.x, -a10.y)), a10);
        const float2 s23 = __ffma2_rn(fs2, __fadd2_rn(b23, make_float2(-a23.x, -a23.y)), a23);
        const float e0 = fmaf(cur.fu, s10.x - s10.y, s10.y);   // row v
        const float e1 = fmaf(cur.fu, s23.y - s23.x, s23.x);   // row v + 1
        float val = fmaf(cur.fv, e1 - e0, e0);
        if (PREC == kPrecF8) val *= k0;
        if constexpr (MODE == 1) {
            // a MIP ray stops once it reaches the data's global maximum (Section
            // 2.3.2): no later sample can exceed it
            const bool owed = fi < fn;
            if (owed) vmax = fmaxf(vmax, val);
            if (owed && vmax >= p.gmax) fn = fi + 1.0f;
            fi += 1.0f;
            return;
        }
        const float4 col = tf_lerp<UNIFORM>(tfv, s_rgba, s_drgba, s_v, val);
        const float alpha = DYN ? opacity_correct_dt(col.w, dt_ray) : opacity_correct(p, col.w);
        const bool owed = fi < fn;
        const float w = owed ? (1.0f - acc.w) * alpha : 0.0f;
        acc.x = fmaf(w, col.x, acc.x);
        acc.y = fmaf(w, col.y, acc.y);
        acc.z = fmaf(w, col.z, acc.z);
        acc.w += w;
        if (owed && acc.w >= tau) fn = fi + 1.0f;
        fi += 1.0f;
    };
    // Software pipeline of depth D: the gathers of sample k + D are issued before
    // sample k is composited, so D samples' texture reads are in flight per ray.
    // The D + 1 corner buffers form a ring indexed by compile-time constants: the
    // loop body is D + 1 straight-line steps, so that no buffer is copied (a copy of
    // a buffer whose gathers are in flight would wait for them) and the steps'
    // independent arithmetic can overlap.  The gathers are unconditional: those
    // past a segment's end read points up to 2D steps beyond it, which texture
    // addressing clamps (a texture read never faults).
    constexpr int D = tex_depth(PREC);
    Corners ring[D + 1];
#pragma unroll
    for (int d = 0; d < D; ++d) fetch((float)d, ring[d]);
    while (fi < fn) {
#pragma unroll
        for (int r = 0; r <= D; ++r) {
            fetch(fi + (float)D, ring[(r + D) % (D + 1)]);
            step(ring[r]);
        }
    }
    if (MODE == 1) acc = make_float4(vmax, fn > 0.0f ? 1.0f : 0.0f, 0.0f, 0.0f);
    p.frags[(int64_t)item.frag * kTilePixels + t] = acc;
    unsigned long long ns = (unsigned long long)fn;
    for (int o = 16; o > 0; o >>= 1) ns += __shfl_xor_sync(0xffffffffu, ns, o);
    if ((threadIdx.x & 31) == 0 && ns) atomicAdd(&p.stats->samples, ns);
}

// Copy the transfer function into dynamic shared memory sized to its control
// points (so that almost all of the SM's L1/shared array stays texture cache):
// the points, their forward differences and their values.
__device__ __forceinline__ void load_tf(const FrameParams& p, float4*& s_rgba, float4*& s_drgba, float*& s_v) {
    extern __shared__ float4 s_dyn[];
    s_rgba = s_dyn;
    s_drgba = s_dyn + p.tf_n + 1;
    s_v = reinterpret_cast<float*>(s_drgba + p.tf_n);
    for (int k = threadIdx.x; k <= p.tf_n; k += blockDim.x) {
        const float4 c = p.tf_rgba[k];
        s_rgba[k] = c;
        if (k < p.tf_n) {
            const float4 c1 = p.tf_rgba[k + 1];
            s_drgba[k] = make_float4(c1.x - c.x, c1.y - c.y, c1.z - c.z, c1.w - c.w);
            s_v[k] = p.tf_v[k];
        }
    }
    __syncthreads();
}

// Persistent CTAs (as many as are resident), each warp taking half items (the 32
// rays of an 8x4 half tile) in list order from a counter: a warp that finishes
// its rays starts the next half item at once instead of waiting for the other
// warp of its CTA, and the list order (brick-major, front to back) is kept.
template <bool UNIFORM, int PREC, bool DYN, int MODE = 0, bool POOL = false>
__global__ void __launch_bounds__(kTilePixels, tex_blocks_per_sm(PREC)) march_tex_kernel(const FrameParams p) {
    float4 *s_rgba, *s_drgba;
    float* s_v;
    load_tf(p, s_rgba, s_drgba, s_v);
    const int lane = threadIdx.x & 31;
    const int total = 2 * p.n_items;
    int* counter = p.work_next ? p.work_next : &p.stats->work_next;
    for (;;) {
        int w = 0;
        if (lane == 0) w = atomicAdd(counter, 1);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= total) break;
        const Item item = p.items[w >> 1];
        const int t = (w & 1) * 32 + lane;
        switch (item.sweep & 3) {
            case 0: march_item<0, UNIFORM, PREC, DYN, FrameParams, MODE, POOL>(p, p, item, s_rgba, s_drgba, s_v, t); break;
            case 1: march_item<1, UNIFORM, PREC, DYN, FrameParams, MODE, POOL>(p, p, item, s_rgba, s_drgba, s_v, t); break;
            default: march_item<2, UNIFORM, PREC, DYN, FrameParams, MODE, POOL>(p, p, item, s_rgba, s_drgba, s_v, t); break;
        }
    }
}

// Batch of frames (the serving loop): the same persistent march, each item's
// camera, transfer function and termination threshold read from the frame it
// belongs to (item.sweep >> 3).  The batch's transfer functions are concatenated
// (tf_n + 1 entries each, the last point repeated), p.tf_n = their total - 1.
template <int PREC>
__global__ void __launch_bounds__(kTilePixels, tex_blocks_per_sm(PREC)) march_tex_batch_kernel(const FrameParams p) {
    float4 *s_rgba, *s_drgba;
    float* s_v;
    load_tf(p, s_rgba, s_drgba, s_v);
    const int lane = threadIdx.x & 31;
    const int total = 2 * p.n_items;
    for (;;) {
        int w = 0;
        if (lane == 0) w = atomicAdd(&p.stats->work_next, 1);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= total) break;
        const Item item = p.items[w >> 1];
        const FrameCam& cam = p.cams[item.sweep >> 3];
        const int t = (w & 1) * 32 + lane;
        // the frame's transfer function within the batch's concatenated tables
        const float4* rgba = s_rgba + cam.tf_off;
        const float4* drgba = s_drgba + cam.tf_off;
        const float* vals = s_v + cam.tf_off;
        // the lookup each frame's own vr_render would use (uniform spacing or
        // search), so that its image is the same alone and in the batch
        if (cam.tf_uniform) {
            switch (item.sweep & 3) {
                case 0: march_item<0, true, PREC, false>(p, cam, item, rgba, drgba, vals, t); break;
                case 1: march_item<1, true, PREC, false>(p, cam, item, rgba, drgba, vals, t); break;
                default: march_item<2, true, PREC, false>(p, cam, item, rgba, drgba, vals, t); break;
            }
        } else {
            switch (item.sweep & 3) {
                case 0: march_item<0, false, PREC, false>(p, cam, item, rgba, drgba, vals, t); break;
                case 1: march_item<1, false, PREC, false>(p, cam, item, rgba, drgba, vals, t); break;
                default: march_item<2, false, PREC, false>(p, cam, item, rgba, drgba, vals, t); break;
            }
        }
    }
}

// Copy layers [l0, l0 + nl) along axis S of the stored cube a[z][y][x] (row pitch
// a_pitch floats) into the layered array of sweep axis S through its surface:
// layer = coordinate along S - l0.  FP16 stores the nearest half; FP8 stores the
// E4M3 code of v / scale, the scale of the brick that owns the voxel (voxel g
// belongs to brick min(g / B, nb - 1)).  The grid covers (x, y, z) of the slab:
// x in [x0, x0 + gridDim.x * blockDim.x), y = y0 + blockIdx.y, z = z0 + blockIdx.z.
template <int S, int PREC>
__global__ void fill_layers_kernel(const float* __restrict__ a, int64_t nx, int64_t ny, int64_t nz,
                                   int64_t a_pitch, int64_t l0, int64_t x_end, cudaSurfaceObject_t surf,
                                   const float* __restrict__ scale, int3 B, int3 nb) {
    const int64_t x = (S == 0 ? l0 : 0) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t y = (S == 1 ? l0 : 0) + blockIdx.y;
    const int64_t z = (S == 2 ? l0 : 0) + blockIdx.z;
    if (x >= x_end) return;
    const float v = a[(z * ny + y) * a_pitch + x];
    const int64_t c[3] = {x, y, z};
    constexpr int U = Axes<S>::U, V = Axes<S>::V;
    const int cx = (int)(c[U] * (PREC == kPrecF32 ? 4 : (PREC == kPrecF16 ? 2 : 1)));
    const int layer = (int)(c[S] - l0);
    if (PREC == kPrecF32) {
        surf2DLayeredwrite(v, surf, cx, (int)c[V], layer);
    } else if (PREC == kPrecF16) {
        surf2DLayeredwrite(__half_as_ushort(__float2half_rn(v)), surf, cx, (int)c[V], layer);
    } else {
        const int bx = min((int)(x / B.x), nb.x - 1), by = min((int)(y / B.y), nb.y - 1);
        const int bz = min((int)(z / B.z), nb.z - 1);
        const float sc = scale[bx + nb.x * (by + nb.y * bz)];
        surf2DLayeredwrite((signed char)e4m3_code(v / sc), surf, cx, (int)c[V], layer);
    }
}

// Per-brick FP8 scale: the largest |value| over the voxels the brick owns, / 448
// (the largest finite E4M3 value); 1 for an all-zero brick.
__global__ void brick_scale_kernel(const float* __restrict__ a, int64_t nx, int64_t ny, int64_t nz,
                                   int64_t a_pitch, int3 B, int3 nb, float* __restrict__ scale) {
    const int id = blockIdx.x;
    const int bx = id % nb.x, by = (id / nb.x) % nb.y, bz = id / (nb.x * nb.y);
    const int x0 = bx * B.x, y0 = by * B.y, z0 = bz * B.z;
    const int x1 = bx == nb.x - 1 ? (int)nx : x0 + B.x;
    const int y1 = by == nb.y - 1 ? (int)ny : y0 + B.y;
    const int z1 = bz == nb.z - 1 ? (int)nz : z0 + B.z;
    const int rows_y = y1 - y0, rows = rows_y * (z1 - z0);
    float m = 0.0f;
    for (int r = threadIdx.x >> 5; r < rows; r += blockDim.x >> 5) {
        const int64_t y = y0 + r % rows_y, z = z0 + r / rows_y;
        const float* row = a + (z * ny + y) * a_pitch;
        for (int x = x0 + (threadIdx.x & 31); x < x1; x += 32) m = fmaxf(m, fabsf(row[x]));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float sm[32];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, sm[w]);
        scale[id] = m > 0.0f ? m / 448.0f : 1.0f;
    }
}

// Per-brick [min, max] of the values the march reads back from reduced-precision
// storage (the brick's voxels plus its +1 apron, each decoded with the scale of the
// brick that owns it), so that empty-space skipping stays exact for that storage.
template <int PREC>
__global__ void stored_minmax_kernel(const float* __restrict__ a, int64_t pitch, int3 n, int3 B, int3 nb,
                                     const float* __restrict__ scale, float2* __restrict__ out) {
    const int id = blockIdx.x;
    const int bx = id % nb.x, by = (id / nb.x) % nb.y, bz = id / (nb.x * nb.y);
    const int x0 = bx * B.x, y0 = by * B.y, z0 = bz * B.z;
    const int x1 = min(x0 + B.x, n.x - 1), y1 = min(y0 + B.y, n.y - 1), z1 = min(z0 + B.z, n.z - 1);
    const int ny_rows = y1 - y0 + 1, rows = ny_rows * (z1 - z0 + 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    float mn = FLT_MAX, mx = -FLT_MAX;
    for (int r = warp; r < rows; r += nwarps) {
        const int z = z0 + r / ny_rows, y = y0 + r % ny_rows;
        const float* row = a + ((int64_t)z * n.y + y) * pitch;
        const int oyz = min(y / B.y, nb.y - 1) * nb.x + min(z / B.z, nb.z - 1) * nb.x * nb.y;
        for (int x = x0 + lane; x <= x1; x += 32) {
            const float v = row[x];
            float q;
            if (PREC == kPrecF16) {
                q = __half2float(__float2half_rn(v));
            } else {
                const float sc = scale[oyz + min(x / B.x, nb.x - 1)];
                q = e4m3_pair(e4m3_code(v / sc), 0).x * sc;
            }
            mn = fminf(mn, q);
            mx = fmaxf(mx, q);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    __shared__ float smn[32], smx[32];
    if (lane == 0) {
        smn[warp] = mn;
        smx[warp] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nwarps; ++w) {
            mn = fminf(mn, smn[w]);
            mx = fmaxf(mx, smx[w]);
        }
        out[id] = make_float2(mn, mx);
    }
}

// Out-of-core texture pool: slot slots[blockIdx.z]'s block (B+1)^3, x fastest,
// into the layered copy of sweep axis S: layer = coordinate along S, texel =
// (coordinates along U, V) + the slot's tile origin.  The grid covers (x, y) of
// the block with (z) in a loop.
template <int S>
__global__ void fill_pool_kernel(const float* __restrict__ pool, int64_t slot_floats, const int32_t* slots,
                                 bool staged, int3 B1, cudaSurfaceObject_t surf, int32_t cols) {
    constexpr int U = Axes<S>::U, V = Axes<S>::V;
    const int k = slots[blockIdx.z];
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= B1.x) return;
    const int n1[3] = {B1.x, B1.y, B1.z};
    const int tu = (k % cols) * n1[U], tv = (k / cols) * n1[V];
    const float* blk = pool + (int64_t)(staged ? (int)blockIdx.z : k) * slot_floats;
    for (int z = 0; z < B1.z; ++z) {
        const float v = blk[((int64_t)z * B1.y + y) * B1.x + x];
        const int c[3] = {x, y, z};
        surf2DLayeredwrite(v, surf, (tu + c[U]) * 4, tv + c[V], c[S]);
    }
}

// One wave of persistent CTAs (no more than there are items).
inline unsigned persistent_grid(const FrameParams& p, int blocks_per_sm) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (unsigned)std::min<int64_t>((int64_t)sms * blocks_per_sm, (int64_t)p.n_items);
}

}  // namespace texm

cudaError_t launch_march_tex(const FrameParams& p, cudaStream_t s) {
    if (p.n_items == 0) return cudaSuccess;
    const size_t smem = (size_t)(2 * p.tf_n + 1) * sizeof(float4) + (size_t)p.tf_n * sizeof(float);
    // shared-memory carveout just large enough for the resident CTAs the kernel is
    // compiled for (each also reserves 1 KB); the rest of the SM's 256 KB array is
    // L1/texture cache
    auto go = [&](auto kern) {
        const int blocks = texm::tex_blocks_per_sm(p.precision);
        const int pct = std::min(100, (int)((blocks * (smem + 1024) * 100 + 233471) / 233472) + 2);
        static int carveout = -1;
        if (carveout != pct) {
            cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
            carveout = pct;
        }
        kern<<<texm::persistent_grid(p, blocks), kTilePixels, smem, s>>>(p);
    };
    auto by_tf = [&](auto uniform_kern, auto general_kern) {
        if (p.tf_uniform) go(uniform_kern);
        else go(general_kern);
    };
    using namespace texm;
    if (p.pool) {  // out-of-core texture march (FP32 slots)
        if (p.mode == 1) {
            if (p.step_mode) go(march_tex_kernel<true, kPrecF32, true, 1, true>);
            else go(march_tex_kernel<true, kPrecF32, false, 1, true>);
        } else if (p.step_mode) {
            by_tf(march_tex_kernel<true, kPrecF32, true, 0, true>, march_tex_kernel<false, kPrecF32, true, 0, true>);
        } else {
            by_tf(march_tex_kernel<true, kPrecF32, false, 0, true>, march_tex_kernel<false, kPrecF32, false, 0, true>);
        }
        return cudaGetLastError();
    }
    if (p.mode == 1) {  // MIP (FP32 storage; the march does not read the transfer function)
        if (p.step_mode) go(march_tex_kernel<true, kPrecF32, true, 1>);
        else go(march_tex_kernel<true, kPrecF32, false, 1>);
    } else if (p.step_mode) {  // the dynamic step (any storage; uniform or not)
        if (p.precision == kPrecF8) by_tf(march_tex_kernel<true, kPrecF8, true>, march_tex_kernel<false, kPrecF8, true>);
        else if (p.precision == kPrecF16) by_tf(march_tex_kernel<true, kPrecF16, true>, march_tex_kernel<false, kPrecF16, true>);
        else by_tf(march_tex_kernel<true, kPrecF32, true>, march_tex_kernel<false, kPrecF32, true>);
    } else if (p.precision == kPrecF8) {
        by_tf(march_tex_kernel<true, kPrecF8, false>, march_tex_kernel<false, kPrecF8, false>);
    } else if (p.precision == kPrecF16) {
        by_tf(march_tex_kernel<true, kPrecF16, false>, march_tex_kernel<false, kPrecF16, false>);
    } else {
        by_tf(march_tex_kernel<true, kPrecF32, false>, march_tex_kernel<false, kPrecF32, false>);
    }
    return cudaGetLastError();
}

cudaError_t launch_march_tex_batch(const FrameParams& p, cudaStream_t s) {
    if (p.n_items == 0) return cudaSuccess;
    const size_t smem = (size_t)(2 * p.tf_n + 1) * sizeof(float4) + (size_t)p.tf_n * sizeof(float);
    auto go = [&](auto kern) {
        const int blocks = texm::tex_blocks_per_sm(p.precision);
        const int pct = std::min(100, (int)((blocks * (smem + 1024) * 100 + 233471) / 233472) + 2);
        static int carveout = -1;
        if (carveout != pct) {
            cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
            carveout = pct;
        }
        kern<<<texm::persistent_grid(p, blocks), kTilePixels, smem, s>>>(p);
    };
    using namespace texm;
    if (p.precision == kPrecF8) {
        go(march_tex_batch_kernel<kPrecF8>);
    } else if (p.precision == kPrecF16) {
        go(march_tex_batch_kernel<kPrecF16>);
    } else {
        go(march_tex_batch_kernel<kPrecF32>);
    }
    return cudaGetLastError();
}

cudaError_t fill_pool_tex(const float* pool, int64_t slot_floats, const int32_t* slots, int32_t count, bool staged,
                          const int32_t B[3], const cudaSurfaceObject_t surf[3], const int32_t cols[3],
                          cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int3 b1 = make_int3(B[0] + 1, B[1] + 1, B[2] + 1);
    const dim3 grid((unsigned)((b1.x + 127) / 128), (unsigned)b1.y, (unsigned)count);
    // the copies the pool keeps (all three, or the one along z)
    if (surf[0])
        texm::fill_pool_kernel<0><<<grid, 128, 0, s>>>(pool, slot_floats, slots, staged, b1, surf[0], cols[0]);
    if (surf[1])
        texm::fill_pool_kernel<1><<<grid, 128, 0, s>>>(pool, slot_floats, slots, staged, b1, surf[1], cols[1]);
    if (surf[2])
        texm::fill_pool_kernel<2><<<grid, 128, 0, s>>>(pool, slot_floats, slots, staged, b1, surf[2], cols[2]);
    return cudaGetLastError();
}

cudaError_t fill_tex_layers(const float* a, int64_t nx, int64_t ny, int64_t nz, int64_t a_pitch, int S,
                            int64_t l0, int64_t nl, int precision, cudaSurfaceObject_t surf, const float* scale,
                            const int32_t B[3], const int32_t nb[3], cudaStream_t s) {
    // the slab's extent along each axis (S restricted to [l0, l0 + nl))
    const int64_t ex = S == 0 ? nl : nx, ey = S == 1 ? nl : ny, ez = S == 2 ? nl : nz;
    const int64_t x_end = S == 0 ? l0 + nl : nx;
    dim3 grid((unsigned)((ex + 255) / 256), (unsigned)ey, (unsigned)ez);
    const int3 b3 = make_int3(B[0], B[1], B[2]), n3 = make_int3(nb[0], nb[1], nb[2]);
    auto go = [&](auto kern) { kern<<<grid, 256, 0, s>>>(a, nx, ny, nz, a_pitch, l0, x_end, surf, scale, b3, n3); };
    if (precision == kPrecF16) {
        if (S == 0) go(texm::fill_layers_kernel<0, kPrecF16>);
        else if (S == 1) go(texm::fill_layers_kernel<1, kPrecF16>);
        else go(texm::fill_layers_kernel<2, kPrecF16>);
    } else if (precision == kPrecF8) {
        if (S == 0) go(texm::fill_layers_kernel<0, kPrecF8>);
        else if (S == 1) go(texm::fill_layers_kernel<1, kPrecF8>);
        else go(texm::fill_layers_kernel<2, kPrecF8>);
    } else {
        if (S == 0) go(texm::fill_layers_kernel<0, kPrecF32>);
        else if (S == 1) go(texm::fill_layers_kernel<1, kPrecF32>);
        else go(texm::fill_layers_kernel<2, kPrecF32>);
    }
    return cudaGetLastError();
}

cudaError_t launch_brick_scale(const float* a, int64_t nx, int64_t ny, int64_t nz, int64_t a_pitch,
                               const int32_t B[3], const int32_t nb[3], float* scale, cudaStream_t s) {
    texm::brick_scale_kernel<<<nb[0] * nb[1] * nb[2], 256, 0, s>>>(a, nx, ny, nz, a_pitch,
                                                                   make_int3(B[0], B[1], B[2]),
                                                                   make_int3(nb[0], nb[1], nb[2]), scale);
    return cudaGetLastError();
}

cudaError_t launch_stored_minmax(const float* a, int64_t pitch, const int32_t n[3], const int32_t B[3],
                                 const int32_t nb[3], int precision, const float* scale, float2* out,
                                 cudaStream_t s) {
    const int total = nb[0] * nb[1] * nb[2];
    const int3 n3 = make_int3(n[0], n[1], n[2]), b3 = make_int3(B[0], B[1], B[2]);
    const int3 nb3 = make_int3(nb[0], nb[1], nb[2]);
    if (precision == kPrecF8)
        texm::stored_minmax_kernel<kPrecF8><<<total, 256, 0, s>>>(a, pitch, n3, b3, nb3, scale, out);
    else
        texm::stored_minmax_kernel<kPrecF16><<<total, 256, 0, s>>>(a, pitch, n3, b3, nb3, scale, out);
    return cudaGetLastError();
}

}  // namespace vr
