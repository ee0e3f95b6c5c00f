// TMA-staged ray march (Section 2.3.2 of arXiv:1205.0282: per-pixel ray casting of
// one sub-cube with tri-linear sampling, transfer function, front-to-back
// compositing and termination), restructured for sm_103a shared memory.
//
// One CTA of 256 threads renders one (brick, 16x16 pixel tile) item, one ray per
// thread.  The CTA sweeps the brick along the item's dominant ray axis ("sweep
// axis") in chunks of C sample planes.  For each chunk the voxels that the tile's
// rays can touch -- a square box across the sweep axis and C + 1 planes along it,
// placed from the tile's four corner rays -- are copied from HBM into shared memory
// by one TMA bulk-tensor load (mbarrier transaction count, bounded wait), and the
// eight trilinear corners of every sample are read from shared memory.  The box
// is chosen per item from eight classes that trade side (24..80 voxels) against
// depth (8..2 planes) at about the same size, matching the tile's footprint; the
// tensor maps cover one brick plus its apron each, so box parts outside the brick
// are zero-filled without being read.  Four CTAs share an SM, so one CTA's copy
// overlaps the others' compute.
//
// The box's innermost axis must be contiguous in memory and must not be the sweep
// axis, so sweeps along y and z read the cube as stored ([z][y][x]) and sweeps
// along x read a transposed copy ([x][z][y]).  A chunk whose footprint does not
// fit the largest box falls back to direct global loads for that chunk only.
#include <cuda.h>

#include <cfloat>
#include <cstdint>

#include "vr_device.cuh"

namespace vr {

namespace tma {

constexpr int kT = kTileTma;           // tile edge (pixels)
constexpr int kThreads = kT * kT;      // one ray per thread
constexpr uint32_t kWaitLimit = 1u << 22;  // try_wait rounds before a wait gives up

// Box classes: side (across the sweep axis, a multiple of 4) and depth (planes along
// it; a chunk covers depth - 1 sample planes).
__host__ __device__ constexpr int class_side(int c) { return 24 + 8 * c; }
__host__ __device__ constexpr int class_depth(int c) {
    return c < 3 ? 8 : (c == 3 ? 5 : (c == 4 ? 4 : (c == 5 ? 3 : 2)));
}
constexpr int kMaxSide = class_side(kTmaClasses - 1);
constexpr int kMaxBoxFloats = 12800;  // max over classes of side^2 * depth
static_assert(class_side(0) * class_side(0) * class_depth(0) <= kMaxBoxFloats &&
              class_side(2) * class_side(2) * class_depth(2) <= kMaxBoxFloats &&
              class_side(3) * class_side(3) * class_depth(3) <= kMaxBoxFloats &&
              class_side(4) * class_side(4) * class_depth(4) <= kMaxBoxFloats &&
              class_side(5) * class_side(5) * class_depth(5) <= kMaxBoxFloats &&
              class_side(6) * class_side(6) * class_depth(6) <= kMaxBoxFloats &&
              class_side(7) * class_side(7) * class_depth(7) <= kMaxBoxFloats,
              "box buffer too small");

struct alignas(16) Shared {
    unsigned long long bar;
    float coef[4][4];     // per corner ray: u = A_u + B_u * sigma, v = A_v + B_v * sigma
    int red[2][kThreads / 32];
    int cls;              // box class of this item, -1: every chunk reads global memory
    int timeout;
    int toward[4];        // corner ray c runs along the sweep direction
    int box[2][4];        // chunk boxes (u0, v0, ok), double-indexed by chunk parity
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait for the phase with the given parity; false if it gave up.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity) {
    for (uint32_t k = 0; k < kWaitLimit; ++k)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Footprint of chunk g (sample planes [g*C, g*C + C] along the sweep axis) from
// the corner-ray coefficients: lower corner (u0, v0) of a box of side `side`, with
// two voxels of margin on each side (the corner rays are evaluated in FP32 from the
// eye, the samples in brick-local coordinates) and the global u start rounded down
// to a multiple of 4 (16-byte TMA alignment of the innermost coordinate).  Returns
// false if the footprint does not fit.
__device__ __forceinline__ bool place_box(const float (*coef)[4], int g, int C, int side, int Ou, int& u0,
                                          int& v0) {
    float umin = FLT_MAX, umax = -FLT_MAX, vmin = FLT_MAX, vmax = -FLT_MAX;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float sig = (float)(g * C + e * C);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float pu = fmaf(coef[c][1], sig, coef[c][0]);
            const float pv = fmaf(coef[c][3], sig, coef[c][2]);
            umin = fminf(umin, pu);
            umax = fmaxf(umax, pu);
            vmin = fminf(vmin, pv);
            vmax = fmaxf(vmax, pv);
        }
    }
    if (!(umin > -1e6f && umax < 1e6f && vmin > -1e6f && vmax < 1e6f)) return false;
    const int gu = Ou + (int)floorf(umin) - 2;
    u0 = ((gu >> 2) << 2) - Ou;
    v0 = (int)floorf(vmin) - 2;
    return umax + 3.0f <= (float)(u0 + side) && vmax + 3.0f <= (float)(v0 + side);
}

template <int S>
struct Axes {
    static constexpr int U = S == 0 ? 1 : 0;  // contiguous axis of the staged box
    static constexpr int V = S == 2 ? 1 : 2;
};

template <int S, bool DESC, bool UNIFORM, typename Off>
__device__ __forceinline__ void march_item(const FrameParams& p, const Item& item, float* box, Shared& sh,
                                           const float4* s_rgba, const float* s_v) {
    constexpr int U = Axes<S>::U, V = Axes<S>::V;
    const int tid = threadIdx.x;
    const int tx = item.tile % p.tiles_x, ty = item.tile / p.tiles_x;
    const int i = tx * kT + tid % kT, j = ty * kT + tid / kT;
    int bidx[3], O[3], imax[3];
    bidx[0] = item.brick % p.nb[0];
    bidx[1] = (item.brick / p.nb[0]) % p.nb[1];
    bidx[2] = item.brick / (p.nb[0] * p.nb[1]);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        O[a] = bidx[a] * p.B[a];
        imax[a] = min(p.B[a] - 1, p.n[a] - 2 - O[a]);
    }

    // ---- per-ray set-up (double-float), then FP32 brick-local march state
    float qs[3] = {0, 0, 0}, dq[3] = {0, 0, 0};
    int nk = 0;
    {
        df d[3], pe[3], inv_D[3];
        int n_samples = 0;
        df dt;
        if (i < p.width && j < p.height && setup_ray(p, i, j, d, pe, n_samples, dt, inv_D)) {
            int klo, khi;
            brick_range(p, bidx, d, pe, n_samples, inv_D, klo, khi);
            nk = khi - klo;
            if (nk > 0) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const df D = df_mul(dt, d[a]);
                    qs[a] = df_to_float(df_add_f(df_add(pe[a], df_mul_f(D, (float)klo)), -(float)O[a]));
                    dq[a] = df_to_float(D);
                }
            }
        }
    }
    // sample-plane range of this ray along the sweep axis, reduced over the tile
    int g_lo = INT_MAX, g_hi = INT_MIN;
    if (nk > 0) {
        const int p0 = min(max(__float2int_rd(qs[S]), 0), imax[S]);
        const int p1 = min(max(__float2int_rd(fmaf((float)(nk - 1), dq[S], qs[S])), 0), imax[S]);
        g_lo = min(p0, p1);
        g_hi = max(p0, p1);
    }
    for (int o = 16; o > 0; o >>= 1) {
        g_lo = min(g_lo, __shfl_xor_sync(0xffffffffu, g_lo, o));
        g_hi = max(g_hi, __shfl_xor_sync(0xffffffffu, g_hi, o));
    }
    if ((tid & 31) == 0) {
        sh.red[0][tid >> 5] = g_lo;
        sh.red[1][tid >> 5] = g_hi;
    }
    // corner rays of the tile (float; they only place boxes, with margins): threads
    // 0..3 each turn one corner into u, v as linear functions of the sweep coordinate
    if (tid < 4) {
        const int xi = min(tx * kT + (tid & 1) * (kT - 1), p.width - 1);
        const int yj = min(ty * kT + (tid >> 1) * (kT - 1), p.height - 1);
        const float qx = df_to_float(p.qx[xi]), qy = df_to_float(p.qy[yj]);
        float cd[3], e[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cd[a] = p.f[a].hi + qx * p.r[a].hi + qy * p.u[a].hi;
            e[a] = (p.eye[a].hi - (float)O[a]) + p.eye[a].lo;
        }
        sh.toward[tid] = DESC ? (cd[S] < 0.0f) : (cd[S] > 0.0f);
        const float bu = cd[U] / cd[S], bv = cd[V] / cd[S];
        sh.coef[tid][0] = e[U] - e[S] * bu;
        sh.coef[tid][1] = bu;
        sh.coef[tid][2] = e[V] - e[S] * bv;
        sh.coef[tid][3] = bv;
    }
    __syncthreads();  // also publishes the TF table and the barrier initialisation
    g_lo = INT_MAX;
    g_hi = INT_MIN;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) {
        g_lo = min(g_lo, sh.red[0][w]);
        g_hi = max(g_hi, sh.red[1][w]);
    }
    const int p_lo = g_lo, p_hi = g_hi;  // sample planes of the whole tile
    if (tid == 0) {
        // box class: the first (smallest) class whose box holds the first and the
        // last chunk (the footprint's extent is convex in the sweep coordinate, so
        // every chunk in between fits as well).  Corner rays must run along the
        // sweep direction and reach every plane in front of the eye; otherwise the
        // item reads global memory.
        int cls = -1;
        if (p_hi >= p_lo) {
            const float e_s = (p.eye[S].hi - (float)O[S]) + p.eye[S].lo;
            bool front = sh.toward[0] && sh.toward[1] && sh.toward[2] && sh.toward[3];
            front = front && (DESC ? ((float)(p_hi + 1) < e_s) : ((float)p_lo > e_s));
            for (int c = 0; front && c < kTmaClasses; ++c) {
                const int C = class_depth(c) - 1;
                int u0, v0;
                if (place_box(sh.coef, p_lo / C, C, class_side(c), O[U], u0, v0) &&
                    place_box(sh.coef, p_hi / C, C, class_side(c), O[U], u0, v0)) {
                    cls = c;
                    break;
                }
            }
            const int C = cls >= 0 ? class_depth(cls) - 1 : 7;
            int u0 = 0, v0 = 0;
            const bool ok = cls >= 0 && place_box(sh.coef, (DESC ? p_hi : p_lo) / C, C, class_side(cls), O[U], u0, v0);
            sh.box[0][0] = u0;
            sh.box[0][1] = v0;
            sh.box[0][2] = ok ? 1 : 0;
        }
        sh.cls = cls;
        sh.timeout = 0;
    }
    __syncthreads();
    const int cls = sh.cls;
    const int side = cls >= 0 ? class_side(cls) : kMaxSide;
    const int depth = cls >= 0 ? class_depth(cls) : 8;
    const int C = depth - 1;  // sample planes per chunk
    g_lo = p_hi >= p_lo ? p_lo / C : 0;
    g_hi = p_hi >= p_lo ? p_hi / C : -1;
    const int nchunks = g_hi - g_lo + 1;
    // shared-memory strides of the staged box: u contiguous, then v, then the sweep
    // axis; a y-sweep box is stored [v][s][u]
    const int SV = S == 1 ? side * depth : side;
    const int SP = S == 1 ? side : side * side;
    const int max_off = side * side * depth - 1 - (SP + SV + 1);
    const uint32_t box_bytes = (uint32_t)(side * side * depth * 4);
    // tensor maps: one set per brick (brick-local coordinates) or one for the cube
    const CUtensorMap* map = p.tmaps + ((p.tmaps_per_brick ? item.brick * 3 : 0) + S) * kTmaClasses +
                             (cls >= 0 ? cls : 0);
    int corg[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) corg[a] = p.tmaps_per_brick ? 0 : O[a];

    const float* __restrict__ gbase =
        p.cube + (int64_t)O[2] * p.stride_z + (int64_t)O[1] * p.stride_y + O[0];
    const Off gsy = (Off)p.stride_y, gsz = (Off)p.stride_z;
    const Off gsu = U == 0 ? (Off)1 : gsy;               // u is x or y
    const Off gsv = V == 1 ? gsy : gsz;                  // v is y or z
    const Off gsp = S == 0 ? (Off)1 : (S == 1 ? gsy : gsz);

    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    // float sample counter: fk runs over 0 .. fn - 1; termination sets fn = fk
    float fk = 0.0f, fn = (float)nk;
    int err = 0, staged = 0, direct = 0;
    uint32_t phase = 0u;
    const float tau = p.tau;

    for (int ci = 0; ci < nchunks; ++ci) {
        const int g = DESC ? g_hi - ci : g_lo + ci;
        const int plo = g * C, phi = plo + C - 1;
        const int u0 = sh.box[ci & 1][0], v0 = sh.box[ci & 1][1];
        const bool ok = sh.box[ci & 1][2] != 0;
        if (ok) {
            if (tid == 0) {
                int c[3];
                c[U] = corg[U] + u0;
                c[V] = corg[V] + v0;
                c[S] = corg[S] + plo;
                // tensor-map coordinate order: (x, y, z) for the stored cube, (y, z, x)
                // for the transposed copy
                fence_proxy_async();
                mbar_expect_tx(&sh.bar, box_bytes);
                if (S == 0) tma_load_3d(box, map, c[1], c[2], c[0], &sh.bar);
                else tma_load_3d(box, map, c[0], c[1], c[2], &sh.bar);
            }
            if (!mbar_wait(&sh.bar, phase)) sh.timeout = 1;
            phase ^= 1u;
            // offset of voxel (iu, iv, ps) in the box: iu + iv*SV + ps*SP - base
            const int base = u0 + v0 * SV + plo * SP;
            while (fk < fn) {
                const float qS = fmaf(fk, dq[S], qs[S]);
                // samples sit inside the brick up to rounding: truncation is the floor
                // for q > -1, and only the far face needs the clamp of the lattice
                const int ps = min(__float2int_rz(qS), imax[S]);
                if (DESC ? ps < plo : ps > phi) break;  // belongs to a later chunk
                const float qU = fmaf(fk, dq[U], qs[U]);
                const float qV = fmaf(fk, dq[V], qs[V]);
                const int iu = __float2int_rz(qU), iv = __float2int_rz(qV);
                const float fu = qU - (float)iu, fv = qV - (float)iv, fs = qS - (float)ps;
                int off = iu + iv * SV + ps * SP - base;
                if ((unsigned)off > (unsigned)max_off) {
                    err |= kErrBounds;
                    off = min(max(off, 0), max_off);
                }
                const float* a0 = box + off;
                const float c000 = a0[0], c100 = a0[1], c010 = a0[SV], c110 = a0[SV + 1];
                const float c001 = a0[SP], c101 = a0[SP + 1], c011 = a0[SP + SV], c111 = a0[SP + SV + 1];
                const float e00 = fmaf(fu, c100 - c000, c000);
                const float e10 = fmaf(fu, c110 - c010, c010);
                const float e01 = fmaf(fu, c101 - c001, c001);
                const float e11 = fmaf(fu, c111 - c011, c011);
                const float e0 = fmaf(fv, e10 - e00, e00);
                const float e1 = fmaf(fv, e11 - e01, e01);
                const float val = fmaf(fs, e1 - e0, e0);
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
        } else {
            while (fk < fn) {
                const float qS = fmaf(fk, dq[S], qs[S]);
                const int ps = min(max(__float2int_rz(qS), 0), imax[S]);
                if (DESC ? ps < plo : ps > phi) break;
                const float qU = fmaf(fk, dq[U], qs[U]);
                const float qV = fmaf(fk, dq[V], qs[V]);
                const int iu = min(max(__float2int_rz(qU), 0), imax[U]);
                const int iv = min(max(__float2int_rz(qV), 0), imax[V]);
                const float fu = qU - (float)iu, fv = qV - (float)iv, fs = qS - (float)ps;
                int ix[3];
                ix[U] = iu;
                ix[V] = iv;
                ix[S] = ps;
                const float* __restrict__ r0 = gbase + ((Off)ix[2] * gsz + (Off)ix[1] * gsy + (Off)ix[0]);
                const float c000 = __ldg(r0), c100 = __ldg(r0 + gsu);
                const float c010 = __ldg(r0 + gsv), c110 = __ldg(r0 + gsv + gsu);
                const float c001 = __ldg(r0 + gsp), c101 = __ldg(r0 + gsp + gsu);
                const float c011 = __ldg(r0 + gsp + gsv), c111 = __ldg(r0 + gsp + gsv + gsu);
                const float e00 = fmaf(fu, c100 - c000, c000);
                const float e10 = fmaf(fu, c110 - c010, c010);
                const float e01 = fmaf(fu, c101 - c001, c001);
                const float e11 = fmaf(fu, c111 - c011, c011);
                const float e0 = fmaf(fv, e10 - e00, e00);
                const float e1 = fmaf(fv, e11 - e01, e01);
                const float val = fmaf(fs, e1 - e0, e0);
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
        }
        if (tid == 0) {
            if (ok) ++staged;
            else ++direct;
            // place the next chunk's box while the other threads finish this one
            if (ci + 1 < nchunks) {
                int nu0 = 0, nv0 = 0;
                const bool nok = cls >= 0 && place_box(sh.coef, DESC ? g - 1 : g + 1, C, side, O[U], nu0, nv0);
                sh.box[(ci + 1) & 1][0] = nu0;
                sh.box[(ci + 1) & 1][1] = nv0;
                sh.box[(ci + 1) & 1][2] = nok ? 1 : 0;
            }
        }
        // every thread is done with the box before the next copy overwrites it; stop
        // early once every ray of the tile has terminated or left the brick, or once
        // a wait gave up (a block-wide decision: all threads leave together)
        const int more = __syncthreads_or(fk < fn);
        if (!more || sh.timeout) break;
    }
    if (sh.timeout) {
        // a copy whose wait gave up may still be in flight: wait for it once more
        // (bounded) before the CTA's shared memory is released
        mbar_wait(&sh.bar, phase ^ 1u);
        err |= kErrTimeout;
    }

    p.frags[(int64_t)item.frag * kThreads + tid] = acc;
    unsigned long long t = (unsigned long long)fk;  // samples composited by this ray
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((tid & 31) == 0 && t) atomicAdd(&p.stats->samples, t);
    if (err) atomicOr(&p.stats->errors, err);
    if (tid == 0) {
        if (staged) atomicAdd(&p.stats->chunks_staged, (unsigned long long)staged);
        if (direct) atomicAdd(&p.stats->chunks_direct, (unsigned long long)direct);
    }
}

template <bool UNIFORM, typename Off>
__global__ void __launch_bounds__(kThreads, 4) march_tma_kernel(const FrameParams p) {
    extern __shared__ __align__(128) unsigned char smem[];
    float* box = reinterpret_cast<float*>(smem);
    Shared& sh = *reinterpret_cast<Shared*>(smem + kMaxBoxFloats * 4);
    float4* s_rgba = reinterpret_cast<float4*>(smem + kMaxBoxFloats * 4 + sizeof(Shared));
    float* s_v = reinterpret_cast<float*>(s_rgba + p.tf_n + 1);
    const int tid = threadIdx.x;
    for (int k = tid; k <= p.tf_n; k += kThreads) {
        s_rgba[k] = p.tf_rgba[k];
        if (k < p.tf_n) s_v[k] = p.tf_v[k];
    }
    if (tid == 0) {
        mbar_init(&sh.bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const Item item = p.items[blockIdx.x];
    switch (item.sweep & 7) {
        case 0: march_item<0, false, UNIFORM, Off>(p, item, box, sh, s_rgba, s_v); break;
        case 1: march_item<1, false, UNIFORM, Off>(p, item, box, sh, s_rgba, s_v); break;
        case 2: march_item<2, false, UNIFORM, Off>(p, item, box, sh, s_rgba, s_v); break;
        case 4: march_item<0, true, UNIFORM, Off>(p, item, box, sh, s_rgba, s_v); break;
        case 5: march_item<1, true, UNIFORM, Off>(p, item, box, sh, s_rgba, s_v); break;
        default: march_item<2, true, UNIFORM, Off>(p, item, box, sh, s_rgba, s_v); break;
    }
}

}  // namespace tma

cudaError_t launch_march_tma(const FrameParams& p, cudaStream_t s) {
    if (p.n_items == 0) return cudaSuccess;
    static_assert(sizeof(tma::Shared) % 16 == 0, "TF table alignment");
    const size_t smem = (size_t)tma::kMaxBoxFloats * 4 + sizeof(tma::Shared) +
                        (size_t)(p.tf_n + 1) * sizeof(float4) + (size_t)p.tf_n * sizeof(float);
    auto launch = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<p.n_items, tma::kThreads, smem, s>>>(p);
    };
    if (p.tf_uniform) {
        if (p.offsets32) launch(tma::march_tma_kernel<true, uint32_t>);
        else launch(tma::march_tma_kernel<true, int64_t>);
    } else {
        if (p.offsets32) launch(tma::march_tma_kernel<false, uint32_t>);
        else launch(tma::march_tma_kernel<false, int64_t>);
    }
    return cudaGetLastError();
}

// Transposed copy for sweeps along x: b[x][z][y] (row pitch b_pitch floats along y)
// from a[z][y][x] (row pitch a_pitch floats along x), through 32x32 shared tiles.
__global__ void transpose_xzy_kernel(const float* __restrict__ a, int64_t nx, int64_t ny, int64_t nz,
                                     int64_t a_pitch, float* __restrict__ b, int64_t b_pitch) {
    __shared__ float tile[32][33];
    const int64_t z = blockIdx.z;
    const int64_t x0 = (int64_t)blockIdx.x * 32, y0 = (int64_t)blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t y = y0 + r, x = x0 + threadIdx.x;
        if (y < ny && x < nx) tile[r][threadIdx.x] = a[(z * ny + y) * a_pitch + x];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t x = x0 + r, y = y0 + threadIdx.x;
        if (x < nx && y < ny) b[(x * nz + z) * b_pitch + y] = tile[threadIdx.x][r];
    }
}

cudaError_t launch_transpose_xzy(const float* a, int64_t nx, int64_t ny, int64_t nz, int64_t a_pitch,
                                 float* b, int64_t b_pitch, cudaStream_t s) {
    dim3 grid((unsigned)((nx + 31) / 32), (unsigned)((ny + 31) / 32), (unsigned)nz);
    transpose_xzy_kernel<<<grid, dim3(32, 8), 0, s>>>(a, nx, ny, nz, a_pitch, b, b_pitch);
    return cudaGetLastError();
}

}  // namespace vr

// ------------------------------------------------------------------ tensor maps (host)

#include <cudaTypedefs.h>

#include <algorithm>
#include <vector>

namespace vr {

// Encode the tensor maps of the TMA march into `out`.  Per-brick maps (when the
// brick origins keep the 16-byte alignment TMA needs: B_x and B_y multiples of 4)
// cover one brick plus its one-voxel apron, so box parts outside the brick are
// zero-filled without memory traffic; index ((brick * 3 + S) * kTmaClasses + c).
// Otherwise one set covers the cube; index (S * kTmaClasses + c).  a: cube
// [z][y][x] with row pitch a_pitch floats; b: transposed copy [x][z][y] with row
// pitch b_pitch.  Sweeps along z and y read a (dims x, y, z; a y-sweep box is
// u = x, sweep = y, v = z), sweeps along x read b (dims y, z, x).
cudaError_t make_tma_maps(const float* a, int64_t nx, int64_t ny, int64_t nz, int64_t a_pitch,
                          const float* b, int64_t b_pitch, const int32_t B[3], const int32_t nb[3],
                          std::vector<CUtensorMap>& out, int& per_brick) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    per_brick = (B[0] % 4 == 0 && B[1] % 4 == 0) ? 1 : 0;
    const int64_t n_bricks = per_brick ? (int64_t)nb[0] * nb[1] * nb[2] : 1;
    out.resize((size_t)n_bricks * 3 * kTmaClasses);
    const cuuint32_t estr[3] = {1, 1, 1};
    const cuuint64_t str_a[2] = {(cuuint64_t)a_pitch * 4, (cuuint64_t)(a_pitch * ny) * 4};
    const cuuint64_t str_b[2] = {(cuuint64_t)b_pitch * 4, (cuuint64_t)(b_pitch * nz) * 4};
    for (int64_t id = 0; id < n_bricks; ++id) {
        int64_t O[3] = {0, 0, 0}, E[3] = {nx, ny, nz};
        if (per_brick) {
            const int64_t idx[3] = {id % nb[0], (id / nb[0]) % nb[1], id / ((int64_t)nb[0] * nb[1])};
            const int64_t n[3] = {nx, ny, nz};
            for (int k = 0; k < 3; ++k) {
                O[k] = idx[k] * B[k];
                E[k] = std::min<int64_t>(B[k] + 1, n[k] - O[k]);
            }
        }
        const float* base_a = a + (O[2] * ny + O[1]) * a_pitch + O[0];
        const float* base_b = b + (O[0] * nz + O[2]) * b_pitch + O[1];
        const cuuint64_t dims_a[3] = {(cuuint64_t)E[0], (cuuint64_t)E[1], (cuuint64_t)E[2]};
        const cuuint64_t dims_b[3] = {(cuuint64_t)E[1], (cuuint64_t)E[2], (cuuint64_t)E[0]};
        for (int S = 0; S < 3; ++S)
            for (int c = 0; c < kTmaClasses; ++c) {
                const cuuint32_t side = (cuuint32_t)tma::class_side(c), depth = (cuuint32_t)tma::class_depth(c);
                cuuint32_t box[3] = {side, side, depth};
                if (S == 1) box[1] = depth, box[2] = side;
                const bool tr = S == 0;
                CUresult r = encode(&out[(size_t)(id * 3 + S) * kTmaClasses + c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                                    const_cast<float*>(tr ? base_b : base_a), tr ? dims_b : dims_a,
                                    tr ? str_b : str_a, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
            }
    }
    return cudaSuccess;
}

}  // namespace vr
