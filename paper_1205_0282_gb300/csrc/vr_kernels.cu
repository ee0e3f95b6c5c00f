// Device code of the bricked ray caster (Hassan, Fluke & Barnes, arXiv:1205.0282).
//
//   brick_minmax_kernel   Section 2.3.1: per-sub-cube minimum and maximum, computed on
//                         the GPU once the data is resident (used for exact empty-space
//                         skipping of bricks whose transfer-function opacity is zero).
//   march_kernel          Section 2.3.2: per-pixel ray casting restricted to one brick's
//                         samples (entry/exit, tri-linear sampling, transfer function,
//                         opacity correction, front-to-back compositing, termination).
//                         One CTA renders one (brick, 8x8 pixel tile) work item into a
//                         sub-image fragment.
//   composite_kernel      Section 2.3.3: sort-last composition of the per-brick
//                         sub-images with the associative 'over' operator, in view
//                         order, stopping once the pixel is opaque; or, for maximum
//                         intensity projection, the maximum then the colour map.
#include <cfloat>
#include <cstdint>

#include "vr_device.cuh"

namespace vr {

// ------------------------------------------------------------------ brick min/max

__global__ void brick_minmax_kernel(const float* __restrict__ cube, int64_t pitch, int3 n, int3 B,
                                    int3 nb, float2* __restrict__ out) {
    const int id = blockIdx.x;
    const int bx = id % nb.x, by = (id / nb.x) % nb.y, bz = id / (nb.x * nb.y);
    const int x0 = bx * B.x, y0 = by * B.y, z0 = bz * B.z;
    const int x1 = min(x0 + B.x, n.x - 1), y1 = min(y0 + B.y, n.y - 1), z1 = min(z0 + B.z, n.z - 1);
    const int ny_rows = y1 - y0 + 1, rows = ny_rows * (z1 - z0 + 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    float mn = FLT_MAX, mx = -FLT_MAX;
    for (int r = warp; r < rows; r += nwarps) {
        const int z = z0 + r / ny_rows, y = y0 + r % ny_rows;
        const float* row = cube + ((int64_t)z * n.y + y) * pitch;
        for (int x = x0 + lane; x <= x1; x += 32) {
            float v = __ldg(row + x);
            mn = fminf(mn, v);
            mx = fmaxf(mx, v);
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

cudaError_t launch_brick_minmax(const float* cube, int64_t pitch, const int32_t n[3], const int32_t B[3],
                                const int32_t nb[3], float2* out, cudaStream_t s) {
    const int total = nb[0] * nb[1] * nb[2];
    brick_minmax_kernel<<<total, 256, 0, s>>>(cube, pitch, make_int3(n[0], n[1], n[2]),
                                              make_int3(B[0], B[1], B[2]),
                                              make_int3(nb[0], nb[1], nb[2]), out);
    return cudaGetLastError();
}

// Off: type of brick-local voxel offsets (uint32_t when (B+1) * nx * ny < 2^32).
template <bool UNIFORM, int MODE, typename Off, bool DYN>
__global__ void __launch_bounds__(kTilePixels) march_kernel(const FrameParams p) {
    __shared__ TfShared s_tf;
    for (int k = threadIdx.x; k <= p.tf_n; k += blockDim.x) {
        s_tf.rgba[k] = p.tf_rgba[k];
        if (k < p.tf_n) s_tf.v[k] = p.tf_v[k];
    }
    __syncthreads();

    const Item item = p.items[blockIdx.x];
    const int lx = threadIdx.x % kTile, ly = threadIdx.x / kTile;
    const int tx = item.tile % p.tiles_x, ty = item.tile / p.tiles_x;
    const int i = tx * kTile + lx, j = ty * kTile + ly;
    int bidx[3];
    bidx[0] = item.brick % p.nb[0];
    bidx[1] = (item.brick / p.nb[0]) % p.nb[1];
    bidx[2] = item.brick / (p.nb[0] * p.nb[1]);

    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float vmax = -FLT_MAX;
    int taken = 0;
    df d[3], pe[3], dt, inv_D[3];
    int n_samples = 0;
    if (i < p.width && j < p.height && setup_ray<DYN>(p, i, j, d, pe, n_samples, dt, inv_D)) {
        int klo, khi;
        brick_range(p, bidx, d, pe, n_samples, inv_D, klo, khi);
        const float dt_ray = df_to_float(dt);
        if (khi > klo) {
            int O[3], imax[3];
            float qs[3], dq[3];
            for (int a = 0; a < 3; ++a) {
                O[a] = bidx[a] * p.B[a];
                imax[a] = min(p.B[a] - 1, p.n[a] - 2 - O[a]);
                const df D = df_mul(dt, d[a]);
                qs[a] = df_to_float(df_add_f(df_add(pe[a], df_mul_f(D, (float)klo)), -(float)O[a]));
                dq[a] = df_to_float(D);
            }
            // Sample positions stay inside the brick's owned box up to rounding
            // (ownership), so a truncating conversion plus an upper clamp keeps the
            // eight corners inside the brick and its one-voxel apron.
            // the brick's voxels: in the resident cube, or in its out-of-core cache slot
            const float* __restrict__ base =
                p.pool ? p.pool + (int64_t)p.slot_of[item.brick] * p.slot_stride
                       : p.cube + (int64_t)O[2] * p.stride_z + (int64_t)O[1] * p.stride_y + O[0];
            const Off sy = (Off)(p.pool ? p.pool_sy : p.stride_y), sz = (Off)(p.pool ? p.pool_sz : p.stride_z);
            const int nk = khi - klo;
            for (int kk = 0; kk < nk; ++kk) {
                const float fk = (float)kk;
                const float qx = fmaf(fk, dq[0], qs[0]);
                const float qy = fmaf(fk, dq[1], qs[1]);
                const float qz = fmaf(fk, dq[2], qs[2]);
                const int ix = min(max(__float2int_rz(qx), 0), imax[0]);
                const int iy = min(max(__float2int_rz(qy), 0), imax[1]);
                const int iz = min(max(__float2int_rz(qz), 0), imax[2]);
                const float fx = qx - (float)ix, fy = qy - (float)iy, fz = qz - (float)iz;
                const float* __restrict__ r0 = base + ((Off)iz * sz + (Off)iy * sy + (Off)ix);
                const float* __restrict__ r1 = r0 + sy;
                const float* __restrict__ r2 = r0 + sz;
                const float* __restrict__ r3 = r2 + sy;
                const float v000 = __ldg(r0), v100 = __ldg(r0 + 1);
                const float v010 = __ldg(r1), v110 = __ldg(r1 + 1);
                const float v001 = __ldg(r2), v101 = __ldg(r2 + 1);
                const float v011 = __ldg(r3), v111 = __ldg(r3 + 1);
                const float c00 = fmaf(fx, v100 - v000, v000);
                const float c10 = fmaf(fx, v110 - v010, v010);
                const float c01 = fmaf(fx, v101 - v001, v001);
                const float c11 = fmaf(fx, v111 - v011, v011);
                const float c0 = fmaf(fy, c10 - c00, c00);
                const float c1 = fmaf(fy, c11 - c01, c01);
                const float v = fmaf(fz, c1 - c0, c0);
                ++taken;
                if (MODE == 1) {
                    vmax = fmaxf(vmax, v);
                    // Section 2.3.2: a ray stops once it reaches the data's global
                    // maximum (nothing later can exceed it)
                    if (vmax >= p.gmax) break;
                    continue;
                }
                const float4 col = tf_lookup<UNIFORM>(p, s_tf.rgba, s_tf.v, v);
                const float alpha = DYN ? opacity_correct_dt(col.w, dt_ray) : opacity_correct(p, col.w);
                const float w = (1.0f - acc.w) * alpha;
                acc.x = fmaf(w, col.x, acc.x);
                acc.y = fmaf(w, col.y, acc.y);
                acc.z = fmaf(w, col.z, acc.z);
                acc.w += w;
                if (acc.w >= p.tau) break;
            }
        }
    }
    if (MODE == 1) acc = make_float4(vmax, taken > 0 ? 1.0f : 0.0f, 0.0f, 0.0f);
    p.frags[(int64_t)item.frag * kTilePixels + threadIdx.x] = acc;

    // sample count: warp reduction then one atomic per warp
    unsigned long long t = (unsigned long long)taken;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0 && t) atomicAdd(&p.stats->samples, t);
}

template <bool UNIFORM, int MODE, bool DYN>
static void launch_march_t(const FrameParams& p, cudaStream_t s) {
    if (p.offsets32)
        march_kernel<UNIFORM, MODE, uint32_t, DYN><<<p.n_items, kTilePixels, 0, s>>>(p);
    else
        march_kernel<UNIFORM, MODE, int64_t, DYN><<<p.n_items, kTilePixels, 0, s>>>(p);
}

cudaError_t launch_march(const FrameParams& p, cudaStream_t s) {
    if (p.n_items == 0) return cudaSuccess;
    // (MIP needs no opacity correction: there the dynamic step only moves the samples)
    if (p.mode == 1) {
        if (p.step_mode) {
            if (p.tf_uniform) launch_march_t<true, 1, true>(p, s);
            else launch_march_t<false, 1, true>(p, s);
        } else {
            if (p.tf_uniform) launch_march_t<true, 1, false>(p, s);
            else launch_march_t<false, 1, false>(p, s);
        }
    } else if (p.step_mode) {
        if (p.tf_uniform) launch_march_t<true, 0, true>(p, s);
        else launch_march_t<false, 0, true>(p, s);
    } else {
        if (p.tf_uniform) launch_march_t<true, 0, false>(p, s);
        else launch_march_t<false, 0, false>(p, s);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ composite
//
// Sort-last composition (Section 2.3.3): a pixel's fragments, one per brick in
// view order, are folded front to back with the associative 'over' operator
// until the accumulated opacity reaches tau.  A warp folds eight pixels at a
// time: lane l holds fragment j = l / 8 of a chunk of four fragments of pixel
// l % 8 (the eight pixels' fragments of one brick are contiguous, so each load
// is coalesced).  An inclusive scan over the four lanes of a pixel (shuffles up
// by 8 and 16 lanes) gives every prefix of the chunk, the prefix of the earlier
// chunks is put in front, and the first prefix whose opacity reaches tau is the
// pixel's value, as in the serial fold that stops after that fragment.

// 'over' of a front and a back fragment (premultiplied RGBA)
__device__ __forceinline__ float4 over(const float4 f, const float4 b) {
    const float tr = 1.0f - f.w;
    return make_float4(fmaf(tr, b.x, f.x), fmaf(tr, b.y, f.y), fmaf(tr, b.z, f.z), fmaf(tr, b.w, f.w));
}

__device__ __forceinline__ float4 shfl_up4(const float4 v, int d) {
    return make_float4(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d),
                       __shfl_up_sync(0xffffffffu, v.z, d), __shfl_up_sync(0xffffffffu, v.w, d));
}

__device__ __forceinline__ float4 shfl4(const float4 v, int src) {
    return make_float4(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src),
                       __shfl_sync(0xffffffffu, v.z, src), __shfl_sync(0xffffffffu, v.w, src));
}

// Front-to-back fold of the fragments [f0, f1) of pixel group g (pixels 8g..8g+7
// of a tile of TT pixels; fragment f of pixel q at frags[f TT + q]).  Called by
// a whole warp; lanes l and l + 8, l + 16, l + 24 return pixel 8g + l % 8's value.
__device__ __forceinline__ float4 fold_over_warp(const float4* __restrict__ frags, int TT, int g, int f0, int f1,
                                                 float tau) {
    const int lane = threadIdx.x & 31, q = lane & 7, j = lane >> 3;
    const int pix = g * 8 + q;
    float4 carry = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    bool done = false;
    for (int c = f0; c < f1; c += 4) {
        const int f = c + j;
        float4 v = f < f1 ? frags[(int64_t)f * TT + pix] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        // inclusive 'over' scan of the chunk across the four lanes of each pixel
        float4 u = shfl_up4(v, 8);
        if (j >= 1) v = over(u, v);
        u = shfl_up4(v, 16);
        if (j >= 2) v = over(u, v);
        const float4 total = over(carry, v);
        // first fragment of the chunk at which the pixel's opacity reaches tau
        const unsigned hit = __ballot_sync(0xffffffffu, !done && f < f1 && total.w >= tau);
        const unsigned mine = (hit >> q) & 0x01010101u;
        const int src = mine ? (__ffs(mine) - 1) + q : 24 + q;
        const float4 pick = shfl4(total, src);
        if (!done) carry = pick;
        done = done || mine != 0;
        if (__all_sync(0xffffffffu, done)) break;
    }
    return carry;
}

// Maximum intensity projection: the colour map of the largest value over the
// fragments that saw samples (fragment = (max, 1 if any sample, 0, 0)).
__device__ __forceinline__ float fold_max_warp(const float4* __restrict__ frags, int TT, int g, int f0, int f1,
                                               bool& any) {
    const int lane = threadIdx.x & 31, q = lane & 7, j = lane >> 3;
    const int pix = g * 8 + q;
    float vmax = -FLT_MAX;
    int seen = 0;
    for (int f = f0 + j; f < f1; f += 4) {
        const float4 fr = frags[(int64_t)f * TT + pix];
        if (fr.y > 0.0f) {
            vmax = fmaxf(vmax, fr.x);
            seen = 1;
        }
    }
    vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, 8));
    vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, 16));
    seen |= __shfl_xor_sync(0xffffffffu, seen, 8);
    seen |= __shfl_xor_sync(0xffffffffu, seen, 16);
    any = seen != 0;
    return vmax;
}

// One CTA of 256 threads (8 warps) per tile; warp w folds pixel groups w, w + 8, ...
__global__ void __launch_bounds__(256) composite_kernel(const FrameParams p) {
    __shared__ TfShared s_tf;
    if (p.mode == 1) {
        for (int k = threadIdx.x; k <= p.tf_n; k += blockDim.x) {
            s_tf.rgba[k] = p.tf_rgba[k];
            if (k < p.tf_n) s_tf.v[k] = p.tf_v[k];
        }
        __syncthreads();
    }
    const int t = blockIdx.x;
    const int T = p.tile, TT = p.tile * p.tile;
    const int tx = t % p.tiles_x, ty = t / p.tiles_x;
    const int f0 = p.tile_start[t], f1 = p.tile_start[t + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int g = warp; g < TT / 8; g += 8) {
        float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (p.mode == 0) {
            acc = fold_over_warp(p.frags, TT, g, f0, f1, p.tau);
        } else {
            bool any;
            const float vmax = fold_max_warp(p.frags, TT, g, f0, f1, any);
            if (any) {
                const float4 c = p.tf_uniform ? tf_lookup<true>(p, s_tf.rgba, s_tf.v, vmax)
                                             : tf_lookup<false>(p, s_tf.rgba, s_tf.v, vmax);
                acc = make_float4(c.x * c.w, c.y * c.w, c.z * c.w, c.w);
            }
        }
        const int pix = g * 8 + (lane & 7);
        const int i = tx * T + pix % T, j = ty * T + pix / T;
        const int wi = i - p.out_x0, wj = j - p.out_y0;
        if (lane < 8 && i < p.width && j < p.height && wi >= 0 && wi < p.out_w && wj >= 0 && wj < p.out_h)
            p.out[(int64_t)wj * p.out_w + wi] = acc;
    }
}

// Batch composite (emission-absorption, 8x8 tiles): block b is tile
// b - cams[k].tile_base of the frame k whose blocks contain b.
__global__ void __launch_bounds__(256) composite_batch_kernel(const FrameParams p) {
    int k = 0;
    while (k + 1 < p.n_cams && (int)blockIdx.x >= p.cams[k + 1].tile_base) ++k;
    const FrameCam& cam = p.cams[k];
    const int t = blockIdx.x - cam.tile_base;
    const int tx = t % cam.tiles_x, ty = t / cam.tiles_x;
    const int f0 = cam.tile_start[t], f1 = cam.tile_start[t + 1];
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;  // 8 warps, one pixel group each
    const float4 acc = fold_over_warp(p.frags, kTilePixels, g, f0, f1, cam.tau);
    const int pix = g * 8 + (lane & 7);
    const int i = tx * kTile + pix % kTile, j = ty * kTile + pix / kTile;
    if (lane < 8 && i < cam.width && j < cam.height) cam.out[(int64_t)j * cam.width + i] = acc;
}

cudaError_t launch_composite_batch(const FrameParams& p, int32_t total_tiles, cudaStream_t s) {
    if (total_tiles > 0) composite_batch_kernel<<<total_tiles, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_composite(const FrameParams& p, cudaStream_t s) {
    composite_kernel<<<p.tiles_x * p.tiles_y, 256, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace vr
