// Device helpers shared by the ray-march kernels: double-float ray set-up,
// per-brick sample ranges, transfer-function lookup and opacity correction.
#pragma once
#include <cfloat>
#include <cstdint>

#include "vr_internal.cuh"

namespace vr {

// ------------------------------------------------------------------ ray set-up

// Ray of pixel (i, j) in double-float: unit direction d, entry point pe, the
// sample count n = #{k >= 0 : k dt < t1 - t0} and inv_D[a] = 1 / (dt d[a]) (0 where
// d[a] = 0), which brick_range multiplies by instead of dividing.  Returns false if
// the ray misses the domain [0, n-1]^3.  Four df divisions per ray (1 / |d| and one
// reciprocal per axis); every other quotient is a product with a reciprocal.
// Cam: FrameParams (one frame) or FrameCam (a frame of a batch): eye, f, r, u, qx, qy.
// dt: the ray's sample spacing, p.dt, or with the dynamic step (DYN, Section
// 2.3.2's discrete ray casting) p.dt / max_a |d_a|, so that successive samples
// are p.dt voxels apart along the ray's dominant axis, the first half a step
// after the entry.
template <bool DYN = false, class Cam = FrameParams>
__device__ __forceinline__ bool setup_ray(const FrameParams& p, const Cam& cam, int i, int j, df d[3], df pe[3],
                                          int& n_samples, df& dt, df inv_D[3]) {
    const df qx = cam.qx[i], qy = cam.qy[j];
    df dun[3];
    for (int a = 0; a < 3; ++a) dun[a] = df_add(df_add(cam.f[a], df_mul(qx, cam.r[a])), df_mul(qy, cam.u[a]));
    df n2 = df_add(df_add(df_mul(dun[0], dun[0]), df_mul(dun[1], dun[1])), df_mul(dun[2], dun[2]));
    const df inv_len = df_div(df_make(1.0f), df_sqrt(n2));
    df inv_d[3];
    for (int a = 0; a < 3; ++a) {
        d[a] = df_mul(dun[a], inv_len);
        inv_d[a] = df_is_zero(d[a]) ? df_make(0.0f) : df_div(df_make(1.0f), d[a]);
    }

    df tn = df_make(-FLT_MAX), tf = df_make(FLT_MAX);
    for (int a = 0; a < 3; ++a) {
        const df hi = df_make((float)(p.n[a] - 1));
        if (df_is_zero(d[a])) {
            if (df_lt(cam.eye[a], df_make(0.0f)) || df_gt(cam.eye[a], hi)) return false;
            continue;
        }
        df ta = df_mul(df_neg(cam.eye[a]), inv_d[a]);
        df tb = df_mul(df_sub(hi, cam.eye[a]), inv_d[a]);
        tn = df_max(tn, df_min(ta, tb));
        tf = df_min(tf, df_max(ta, tb));
    }
    df t0 = df_max(tn, df_make(0.0f));
    if (!df_gt(tf, t0)) return false;
    dt = p.dt;
    df inv_dt = p.inv_dt;
    if (DYN) {
        // |d| along the dominant axis (selects, no indexed access); the first
        // sample sits half a step after the entry
        df dm = d[0], inv_dm = inv_d[0];
        if (fabsf(d[1].hi) > fabsf(dm.hi)) { dm = d[1]; inv_dm = inv_d[1]; }
        if (fabsf(d[2].hi) > fabsf(dm.hi)) { dm = d[2]; inv_dm = inv_d[2]; }
        if (dm.hi < 0.0f) { dm = df_neg(dm); inv_dm = df_neg(inv_dm); }
        dt = df_mul(p.dt, inv_dm);
        inv_dt = df_mul(dm, p.inv_dt);
        t0 = df_add(t0, df_mul_f(dt, 0.5f));
        if (!df_gt(tf, t0)) return false;
    }
    const df L = df_sub(tf, t0);
    n_samples = (int)df_ceil(df_mul(L, inv_dt));
    for (int a = 0; a < 3; ++a) {
        pe[a] = df_add(cam.eye[a], df_mul(t0, d[a]));
        inv_D[a] = df_mul(inv_d[a], inv_dt);
    }
    return n_samples > 0;
}

template <bool DYN = false>
__device__ __forceinline__ bool setup_ray(const FrameParams& p, int i, int j, df d[3], df pe[3], int& n_samples,
                                          df& dt, df inv_D[3]) {
    return setup_ray<DYN>(p, p, i, j, d, pe, n_samples, dt, inv_D);
}

// Sample range [klo, khi) owned by brick bidx (sample p_k = pe + k dt d belongs to
// brick floor(p/B) per axis, first and last bricks open towards the outside).
// The crossing index of the plane x_a = O is (O - pe_a) / (dt d_a), formed as a
// product with inv_D[a]; a face shared by two bricks gives both the same value.
__device__ __forceinline__ void brick_range(const FrameParams& p, const int bidx[3], const df d[3], const df pe[3],
                                            int n_samples, const df inv_D[3], int& klo, int& khi) {
    float lo = 0.0f, hi = (float)n_samples;
    for (int a = 0; a < 3; ++a) {
        const float dir = d[a].hi;
        const float O = (float)(bidx[a] * p.B[a]);
        const float OB = (float)(bidx[a] * p.B[a] + p.B[a]);
        if (bidx[a] > 0) {
            if (dir > 0.0f) {
                lo = fmaxf(lo, df_ceil(df_mul(df_sub(df_make(O), pe[a]), inv_D[a])));
            } else if (dir < 0.0f) {
                hi = fminf(hi, df_floor(df_mul(df_sub(df_make(O), pe[a]), inv_D[a])) + 1.0f);
            } else if (df_lt(pe[a], df_make(O))) {
                hi = -1.0f;
            }
        }
        if (bidx[a] < p.nb[a] - 1) {
            if (dir > 0.0f) {
                hi = fminf(hi, df_ceil(df_mul(df_sub(df_make(OB), pe[a]), inv_D[a])));
            } else if (dir < 0.0f) {
                lo = fmaxf(lo, df_floor(df_mul(df_sub(df_make(OB), pe[a]), inv_D[a])) + 1.0f);
            } else if (!df_lt(pe[a], df_make(OB))) {
                hi = -1.0f;
            }
        }
    }
    lo = fmaxf(lo, 0.0f);
    hi = fminf(hi, (float)n_samples);
    klo = (int)lo;
    khi = hi > lo ? (int)hi : klo;
}

// ------------------------------------------------------------------ per-sample ops

struct TfShared {
    float4 rgba[kMaxTfPoints + 1];
    float v[kMaxTfPoints];
};

template <bool UNIFORM>
__device__ __forceinline__ float4 tf_lookup(const FrameParams& p, const float4* __restrict__ rgba,
                                            const float* __restrict__ vals, float v) {
    int seg;
    float w;
    if (UNIFORM) {
        // rgba[tf_n] repeats the last point, so x = tf_n - 1 needs no segment clamp
        float x = (v - p.tf_v0) * p.tf_inv_dv;
        x = fminf(fmaxf(x, 0.0f), (float)(p.tf_n - 1));
        seg = __float2int_rz(x);
        w = x - (float)seg;
    } else {
        int lo = 0, hi = p.tf_n - 1;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (v >= vals[mid]) lo = mid;
            else hi = mid;
        }
        seg = lo;
        w = (v - vals[seg]) / (vals[seg + 1] - vals[seg]);
        w = fminf(fmaxf(w, 0.0f), 1.0f);
    }
    const float4 c0 = rgba[seg], c1 = rgba[seg + 1];
    return make_float4(fmaf(w, c1.x - c0.x, c0.x), fmaf(w, c1.y - c0.y, c0.y),
                       fmaf(w, c1.z - c0.z, c0.z), fmaf(w, c1.w - c0.w, c0.w));
}

// alpha = 1 - (1 - a)^dt as a * Q(t): a short polynomial for small a (noise, the
// common case), a long one up to alpha_split (both accurate to ~1e-10 in Q and
// exactly 0 at a = 0), the exponential form above.
// Opacity correction for a per-ray step of dt voxels (the dynamic step).
__device__ __forceinline__ float opacity_correct_dt(float a, float dt) {
    return a >= 1.0f ? 1.0f : 1.0f - exp2f(dt * __log2f(1.0f - a));
}

__device__ __forceinline__ float opacity_correct(const FrameParams& p, float a) {
    if (a <= p.small_split) {
        const float t = fmaf(a, p.small_scale, -1.0f);
        float q = p.alpha_small[kAlphaSmallTerms - 1];
#pragma unroll
        for (int k = kAlphaSmallTerms - 2; k >= 0; --k) q = fmaf(q, t, p.alpha_small[k]);
        return a * q;
    }
    if (a <= p.alpha_split) {
        const float t = fmaf(a, p.poly_scale, -1.0f);
        float q = p.alpha_poly[kAlphaPolyTerms - 1];
#pragma unroll
        for (int k = kAlphaPolyTerms - 2; k >= 0; --k) q = fmaf(q, t, p.alpha_poly[k]);
        return a * q;
    }
    return 1.0f - exp2f(p.dt_f * __log2f(1.0f - a));
}

}  // namespace vr
