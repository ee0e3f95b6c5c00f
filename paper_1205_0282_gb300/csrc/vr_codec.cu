// Learned brick codec: a shared MLP decoder evaluated on the fifth-generation
// tensor cores (tcgen05, BF16 operands, FP32 accumulation in tensor memory).
//
// This file holds the tensor-core building blocks and their self-check: a
// 128 x N x K product through the same shared-memory layouts, descriptors and
// tensor-memory reads that the codec's kernels use.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cfloat>
#include <cstring>
#include <vector>

#include "../../include/vr.h"
#include "tc.cuh"

namespace vr {
namespace codec {

constexpr uint32_t kWaitLimit = 1u << 26;  // mbarrier polls before a kernel gives up

// D (128 x N, FP32 row-major) = A (128 x K) * B (N x K)^T, A and B BF16 row-major
// in global memory.  a_mn / b_mn: stage the operand MN-major instead of K-major.
// Each operand region of shared memory is 64 KiB, large enough for any reading of
// the descriptor offsets, and zero-filled.
__global__ void __launch_bounds__(128) gemm_check_kernel(const __nv_bfloat16* __restrict__ A,
                                                         const __nv_bfloat16* __restrict__ B, float* __restrict__ D,
                                                         int K, int N, int a_mn, int b_mn, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* a_s = smem;
    unsigned char* b_s = smem + 65536;
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < 2 * 65536 / 16; i += 128) reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    // stage A (M = 128 rows) and B (N rows)
    for (int idx = tid; idx < 128 * K; idx += 128) {
        const int m = idx / K, k = idx % K;
        uint32_t off;
        if (a_mn) off = (uint32_t)((((k >> 3) * 16 + (m >> 3)) * 128) + (k & 7) * 16 + (m & 7) * 2);
        else off = tc::kmajor_offset(m, k, K);
        *reinterpret_cast<__nv_bfloat16*>(a_s + off) = A[idx];
    }
    for (int idx = tid; idx < N * K; idx += 128) {
        const int n = idx / K, k = idx % K;
        uint32_t off;
        if (b_mn) off = (uint32_t)((((k >> 3) * (N >> 3) + (n >> 3)) * 128) + (k & 7) * 16 + (n & 7) * 2);
        else off = tc::kmajor_offset(n, k, K);
        *reinterpret_cast<__nv_bfloat16*>(b_s + off) = B[idx];
    }
    tc::fence_smem_to_async();
    if (warp == 0) tc::tmem_alloc(&tmem_slot, 256);
    if (tid == 0) tc::bar_init(&bar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    if (tid == 0) {
        const uint32_t idesc = tc::make_idesc_bf16(128, N, a_mn, b_mn);
        for (int j = 0; j < K / 16; ++j) {
            uint64_t ad, bd;
            if (a_mn) ad = tc::make_desc(tc::smem_addr(a_s) + j * 2 * 2048, 2048, 128);
            else ad = tc::make_desc(tc::smem_addr(a_s) + j * 256, 128, (uint32_t)K * 16);
            if (b_mn) bd = tc::make_desc(tc::smem_addr(b_s) + j * 2 * N * 16, (uint32_t)N * 16, 128);
            else bd = tc::make_desc(tc::smem_addr(b_s) + j * 256, 128, (uint32_t)K * 16);
            tc::mma_bf16(tmem, ad, bd, idesc, j > 0 ? 1u : 0u);
        }
        tc::mma_commit(&bar);
    }
    const bool ok = tc::bar_wait(&bar, 0, kWaitLimit);
    if (!ok && tid == 0) atomicOr(err, 1);
    tc::fence_after_sync();
    if (ok) {
        for (int c = 0; c < N; c += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) D[(int64_t)tid * N + c + i] = v[i];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

}  // namespace codec
}  // namespace vr

extern "C" int vr_codec_gemm_check(const uint16_t* a_bf16, const uint16_t* b_bf16, int32_t K, int32_t N,
                                   int32_t a_mn_major, int32_t b_mn_major, float* d_out) {
    if (!a_bf16 || !b_bf16 || !d_out) return VR_EINVAL;
    if (K < 16 || K > 64 || K % 16 || N < 16 || N > 64 || N % 16) return VR_EINVAL;
    __nv_bfloat16 *A = nullptr, *B = nullptr;
    float* D = nullptr;
    int* err = nullptr;
    int rc = VR_OK;
    const size_t smem = 2 * 65536;
    if (cudaMalloc(&A, 128 * K * 2) != cudaSuccess || cudaMalloc(&B, (size_t)N * K * 2) != cudaSuccess ||
        cudaMalloc(&D, 128 * (size_t)N * 4) != cudaSuccess || cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
        rc = VR_ENOMEM;
    } else if (cudaMemcpy(A, a_bf16, 128 * K * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
               cudaMemcpy(B, b_bf16, (size_t)N * K * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
               cudaMemset(err, 0, sizeof(int)) != cudaSuccess ||
               cudaFuncSetAttribute(vr::codec::gemm_check_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem) != cudaSuccess) {
        rc = VR_ECUDA;
    } else {
        vr::codec::gemm_check_kernel<<<1, 128, smem>>>(A, B, D, K, N, a_mn_major, b_mn_major, err);
        int h_err = 0;
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(d_out, D, 128 * (size_t)N * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = VR_ECUDA;
        else if (h_err)
            rc = VR_ETIMEOUT;
    }
    cudaFree(A);
    cudaFree(B);
    cudaFree(D);
    cudaFree(err);
    return rc;
}

// ============================================================================ codec

namespace vr {
namespace codec {

constexpr int kLatent = 16, kNodes = 8, kHidden = 64, kIn = 32, kTileP = 128;

// Device state of the codec's MLP and latents.
struct Net {
    const __nv_bfloat16* lat;  // [brick][z][y][x][16] BF16
    const float* latf;         // the same BF16 values in FP32 (brick decode for rendering)
    const float4* four;        // brick decode: Fourier features of grid coordinate u along
                               // axis a at four[four_off[a] + u], u = 0..B_a
    int32_t four_off[3];
    const __nv_bfloat16* W1;   // [64][32] BF16 (inputs 28..31 zero)
    const __nv_bfloat16* W2;   // [64][64] BF16
    const float* b1;           // [64]
    const float* b2;           // [64]
    const float* w3;           // [64] (BF16 values)
    const float* b3;           // [1]
    const float* m;            // per-brick offset
    const float* s;            // per-brick scale
    float inv_b[3];            // 1 / brick size
};

// Gradient accumulators of a training step (FP32, zeroed by the caller).
struct Grads {
    float* W1;   // [64][32]
    float* W2;   // [64][64]
    float* b1;   // [64]
    float* b2;   // [64]
    float* w3;   // [64]
    float* b3;   // [1]
    float* lat;  // like Net::lat
    double* loss;
    float dy_scale;  // 2 / (number of points of the step)
};

// Shared-memory layout of the step kernel (bytes).  G2 is followed by G1 and G1
// by Z1: the padded weight-gradient products read up to 1 KiB past either.
// Inference keeps H1 where IN was (IN is consumed by the first product before
// H1 is written) and uses 28 KiB: 7 CTAs of 64 tensor-memory columns per SM.
constexpr uint32_t kOffW1 = 0, kOffW2 = 4096, kOffIN = 12288, kOffH1 = 20480, kOffG2 = 36864, kOffG1 = 53248,
                   kOffZ1 = 69632, kSmemInfer = 28672, kSmemTrain = 102400;
constexpr int kCtasInfer = 7, kCtasTrain = 2;

// SiLU with the hardware base-2 exponential and reciprocal (relative errors ~2^-22,
// far below the BF16 rounding the MLP's operands take): t / (1 + 2^(-t log2 e)).
// Very negative t gives 2^(+big) = inf and a reciprocal of 0, i.e. silu = -0.
__device__ __forceinline__ float silu(float t) {
    float e, r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(t * -1.4426950408889634f));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(1.0f + e));
    return t * r;
}
// The same on two values, the multiplications and additions as packed FP32x2
// operations (each lane rounded like the scalar operation).
__device__ __forceinline__ float2 silu2(float2 t) {
    const float2 a = __fmul2_rn(t, make_float2(-1.4426950408889634f, -1.4426950408889634f));
    float2 e, r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e.x) : "f"(a.x));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e.y) : "f"(a.y));
    const float2 d = __fadd2_rn(e, make_float2(1.0f, 1.0f));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.x) : "f"(d.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.y) : "f"(d.y));
    return __fmul2_rn(t, r);
}
// Rendering decode: silu(t) = h + h tanh(h) with h = t / 2 (the same function,
// t sigmoid(t) = t (1 + tanh(t / 2)) / 2), one hardware tanh (relative error
// about 2^-11) instead of an exponential and a reciprocal, on two values with
// packed FP32x2 multiplication and FMA.
__device__ __forceinline__ float2 silu2_fast(float2 t) {
    const float2 h = __fmul2_rn(t, make_float2(0.5f, 0.5f));
    float2 r;
    asm("tanh.approx.f32 %0, %1;" : "=f"(r.x) : "f"(h.x));
    asm("tanh.approx.f32 %0, %1;" : "=f"(r.y) : "f"(h.y));
    return __ffma2_rn(h, r, h);
}
__device__ __forceinline__ float silu_grad(float t) {
    const float s = __fdividef(1.0f, 1.0f + __expf(-t));
    return s * (1.0f + t * (1.0f - s));
}

// Column sums of a 32 x 16 block held one row per lane (v = this lane's row):
// after halving exchanges lane l holds the sum of column colsum16_index(l), each
// column held by the lane pair (l, l ^ 1).  16 shuffles instead of 16 atomic
// additions per lane to the same 16 addresses.
__device__ __forceinline__ int colsum16_index(int lane) {
    return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}
__device__ __forceinline__ float warp_colsum16(float v[16], int lane) {
#pragma unroll
    for (int h = 8; h >= 1; h >>= 1) {
        const int m = 2 * h;
        const bool hi = (lane & m) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float keep = hi ? v[i + h] : v[i];
            const float send = hi ? v[i] : v[i + h];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

__device__ __forceinline__ void store_bf16(unsigned char* base, uint32_t off, float v) {
    *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
}

// Eight consecutive K elements of one operand row: one core-matrix row, 16 bytes.
__device__ __forceinline__ void store_bf16x8(unsigned char* dst, const float* v) {
    __nv_bfloat162 h[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
    *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(h);
}

// Point p: brick (bits of .w) and local voxel position (.x, .y, .z) in [0, B].
// Builds its input row in IN_s and returns the interpolation corners.
struct Corner {
    int node[8];
    float w[8];
};

// GRID: pt is a voxel of the brick's grid (integer u): latents read in FP32 and the
// Fourier features from the per-axis table (the rendering decode).
template <bool GRID = false>
__device__ __forceinline__ void build_input(const Net& net, float4 pt, bool valid, int row, unsigned char* in_s,
                                            int& brick, Corner& cr) {
    float in[kIn];
    float2* in2 = reinterpret_cast<float2*>(in);
#pragma unroll
    for (int i = 0; i < kIn; ++i) in[i] = 0.0f;
    brick = __float_as_int(pt.w);
    if (valid) {
        const float x[3] = {pt.x * net.inv_b[0], pt.y * net.inv_b[1], pt.z * net.inv_b[2]};
        int i0[3];
        float f[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float g = x[a] * (float)(kNodes - 1);
            i0[a] = min(max((int)floorf(g), 0), kNodes - 2);
            f[a] = g - (float)i0[a];
        }
        const __nv_bfloat16* L = net.lat + (int64_t)brick * kNodes * kNodes * kNodes * kLatent;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
            const float w = (cx ? f[0] : 1.0f - f[0]) * (cy ? f[1] : 1.0f - f[1]) * (cz ? f[2] : 1.0f - f[2]);
            const int node = ((i0[2] + cz) * kNodes + (i0[1] + cy)) * kNodes + (i0[0] + cx);
            cr.node[c] = node;
            cr.w[c] = w;
            const float2 w2 = make_float2(w, w);
            if (GRID) {
                const float4* src = reinterpret_cast<const float4*>(
                    net.latf + ((int64_t)brick * kNodes * kNodes * kNodes + node) * kLatent);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float4 q = __ldg(src + k);
                    in2[2 * k] = __ffma2_rn(w2, make_float2(q.x, q.y), in2[2 * k]);
                    in2[2 * k + 1] = __ffma2_rn(w2, make_float2(q.z, q.w), in2[2 * k + 1]);
                }
            } else {
                const uint4* src = reinterpret_cast<const uint4*>(L + node * kLatent);
                const uint4 q0 = __ldg(src), q1 = __ldg(src + 1);
                const __nv_bfloat162* h0 = reinterpret_cast<const __nv_bfloat162*>(&q0);
                const __nv_bfloat162* h1 = reinterpret_cast<const __nv_bfloat162*>(&q1);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    in2[k] = __ffma2_rn(w2, __bfloat1622float2(h0[k]), in2[k]);
                    in2[4 + k] = __ffma2_rn(w2, __bfloat1622float2(h1[k]), in2[4 + k]);
                }
            }
        }
        if (GRID) {
            const float u[3] = {pt.x, pt.y, pt.z};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float4 f4 = __ldg(net.four + net.four_off[a] + (int)u[a]);
                in[16 + 4 * a] = f4.x;
                in[17 + 4 * a] = f4.y;
                in[18 + 4 * a] = f4.z;
                in[19 + 4 * a] = f4.w;
            }
        } else {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                // sin(2 pi x) = 2 sin cos, cos(2 pi x) = (cos - sin)(cos + sin)
                float sn, cs;
                sincospif(x[a], &sn, &cs);
                in[16 + 4 * a] = sn;
                in[17 + 4 * a] = cs;
                in[18 + 4 * a] = 2.0f * sn * cs;
                in[19 + 4 * a] = (cs - sn) * (cs + sn);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < kIn; i += 8) store_bf16x8(in_s + tc::kmajor_offset(row, i, kIn), in + i);
}

// Issue a chain of K = 16 MMAs (nk of them) and leave the commit to the caller.
__device__ __forceinline__ void mma_chain(uint32_t d_tmem, uint32_t a_start, uint32_t a_step, uint32_t a_lbo,
                                          uint32_t a_sbo, uint32_t b_start, uint32_t b_step, uint32_t b_lbo,
                                          uint32_t b_sbo, uint32_t idesc, int nk, bool accumulate) {
    for (int j = 0; j < nk; ++j)
        tc::mma_bf16(d_tmem, tc::make_desc(a_start + j * a_step, a_lbo, a_sbo),
                     tc::make_desc(b_start + j * b_step, b_lbo, b_sbo), idesc, (accumulate || j > 0) ? 1u : 0u);
}

// One CTA of 128 threads processes tiles of 128 points (tile t, t + gridDim.x, ...).
// TRAIN = false: out[p] = decoded value.  TRAIN = true: the step's loss and
// gradients (targets in tgt) are accumulated into g.
// Points come from pts, or (pts == nullptr) from the voxel grids of the bricks
// listed in grid.bricks: point q is voxel (q % V) of brick grid.bricks[q / V], V =
// (Bx+1)(By+1)(Bz+1) voxels x fastest, written to out[q] (or, with grid.slots, to
// out[grid.slots[q / V] * V + q % V]).
struct Grid {
    const int32_t* bricks;
    const int32_t* slots;  // nullptr: brick k's block at k * V; else at slots[k] * V
    int32_t dims[3];       // B + 1 per axis
};

// FAST (inference only): SiLU through the hardware tanh (silu2_fast), used when
// bricks are decoded for rendering; the point queries and training use the
// exponential form.
template <bool TRAIN, bool FAST = false>
__global__ void __launch_bounds__(kTileP) codec_kernel(const Net net, const float4* __restrict__ pts,
                                                       const Grid grid, const float* __restrict__ tgt,
                                                       int64_t n_points, float* __restrict__ out, const Grads g,
                                                       int* err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_slot;
    __shared__ float s_db1[kHidden], s_db2[kHidden], s_dw3[kHidden], s_db3;
    __shared__ __align__(16) float s_b1[kHidden], s_b2[kHidden], s_w3[kHidden];
    __shared__ double s_loss;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t tcols = TRAIN ? 256 : 64;
    constexpr uint32_t kH1 = TRAIN ? kOffH1 : kOffIN;  // inference: H1 over IN
    // weights into shared memory (K-major, rows = outputs)
    for (int i = tid; i < kHidden * kIn; i += kTileP)
        *reinterpret_cast<__nv_bfloat16*>(sm + kOffW1 + tc::kmajor_offset(i / kIn, i % kIn, kIn)) = net.W1[i];
    for (int i = tid; i < kHidden * kHidden; i += kTileP)
        *reinterpret_cast<__nv_bfloat16*>(sm + kOffW2 + tc::kmajor_offset(i / kHidden, i % kHidden, kHidden)) =
            net.W2[i];
    for (int i = tid; i < kHidden; i += kTileP) {
        s_b1[i] = net.b1[i];
        s_b2[i] = net.b2[i];
        s_w3[i] = net.w3[i];
    }
    if (TRAIN) {
        for (int i = tid; i < kHidden; i += kTileP) s_db1[i] = s_db2[i] = s_dw3[i] = 0.0f;
        // the bytes the padded gradient products read beyond G1 must be initialised
        for (int i = tid; i < (int)(kSmemTrain - kOffG2) / 16; i += kTileP)
            reinterpret_cast<uint4*>(sm + kOffG2)[i] = make_uint4(0, 0, 0, 0);
        if (tid == 0) {
            s_db3 = 0.0f;
            s_loss = 0.0;
        }
    }
    if (warp == 0) tc::tmem_alloc(&tmem_slot, tcols);
    if (tid == 0) tc::bar_init(&bar, 1);
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    const uint32_t sbase = tc::smem_addr(sm);
    // inference: D2 reuses D1's columns (D1 is read out before the second product)
    const uint32_t T_D1 = tmem, T_D2 = TRAIN ? tmem + 64 : tmem, T_DW2 = tmem + 128, T_DW1 = tmem + 192,
                   T_DIN = tmem + 224;
    const uint32_t id_64 = tc::make_idesc_bf16(128, 64, 0, 0);
    uint32_t phase = 0;
    bool ok = true;
    int tiles_done = 0;
    // the issuing thread waits for the MMAs (the others sleep at the block barrier
    // instead of polling); the block then agrees on the outcome, so that a wait that
    // gave up stops the whole block at the same point.  The mbarrier's completion
    // (acquire), the barrier and the fence order every thread's tensor-memory reads
    // after the products.
    auto wait_mma = [&]() {
        const bool mine = tid != 0 || tc::bar_wait(&bar, phase, kWaitLimit);
        phase ^= 1u;
        ok = __syncthreads_and(mine ? 1 : 0) != 0;
        if (!ok && tid == 0) atomicOr(err, 1);
        tc::fence_after_sync();
    };
    const int64_t n_tiles = (n_points + kTileP - 1) / kTileP;
    for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        const int64_t idx = t * kTileP + tid;
        const bool valid = idx < n_points;
        float4 pt = make_float4(0.f, 0.f, 0.f, 0.f);
        int64_t gk = 0, gq = 0;  // grid points: list entry and voxel within the brick
        if (valid) {
            if (pts) {
                pt = pts[idx];
            } else {
                const int64_t V = (int64_t)grid.dims[0] * grid.dims[1] * grid.dims[2];
                if (n_points <= 0x7FFFFFFF) {  // block-uniform: 32-bit division
                    gk = (uint32_t)idx / (uint32_t)V;
                } else {
                    gk = idx / V;
                }
                const int q = (int)(idx - gk * V);
                gq = q;
                const int qy = q / grid.dims[0];
                pt = make_float4((float)(q - qy * grid.dims[0]), (float)(qy % grid.dims[1]),
                                 (float)(qy / grid.dims[1]), __int_as_float(grid.bricks[gk]));
            }
        }
        int brick = 0;
        Corner cr;
        build_input<FAST>(net, pt, valid, tid, sm + kOffIN, brick, cr);
        tc::fence_smem_to_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        // layer 1: D1 = IN W1^T (M 128, N 64, K 32)
        if (tid == 0) {
            mma_chain(T_D1, sbase + kOffIN, 256, 128, 512, sbase + kOffW1, 256, 128, 512, id_64, 2, false);
            tc::mma_commit(&bar);
        }
        wait_mma();
#pragma unroll 1
        for (int c = 0; c < kHidden; c += 32) {
            float d[32];
            tc::tmem_ld32(T_D1 + lane_base + c, d);
#pragma unroll
            for (int i = 0; i < 32; i += 8) {
                float h[8];
#pragma unroll
                for (int e = 0; e < 8; e += 4) {
                    const float4 b = *reinterpret_cast<const float4*>(s_b1 + c + i + e);
                    const float2 za = __fadd2_rn(make_float2(d[i + e], d[i + e + 1]), make_float2(b.x, b.y));
                    const float2 zb = __fadd2_rn(make_float2(d[i + e + 2], d[i + e + 3]), make_float2(b.z, b.w));
                    if (TRAIN)
                        *reinterpret_cast<float4*>(reinterpret_cast<float*>(sm + kOffZ1) + tid * kHidden + c + i +
                                                   e) = make_float4(za.x, za.y, zb.x, zb.y);
                    const float2 ha = FAST ? silu2_fast(za) : silu2(za), hb = FAST ? silu2_fast(zb) : silu2(zb);
                    h[e] = ha.x;
                    h[e + 1] = ha.y;
                    h[e + 2] = hb.x;
                    h[e + 3] = hb.y;
                }
                store_bf16x8(sm + kH1 + tc::kmajor_offset(tid, c + i, kHidden), h);
            }
        }
        tc::fence_smem_to_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        // layer 2: D2 = H1 W2^T (K 64)
        if (tid == 0) {
            mma_chain(T_D2, sbase + kH1, 256, 128, 1024, sbase + kOffW2, 256, 128, 1024, id_64, 4, false);
            tc::mma_commit(&bar);
        }
        wait_mma();
        // two partial sums (even and odd units) in one packed register pair
        float2 y2 = make_float2(net.b3[0], 0.0f);
#pragma unroll 1
        for (int c = 0; c < kHidden; c += 32) {
            float d[32];
            tc::tmem_ld32(T_D2 + lane_base + c, d);
#pragma unroll
            for (int i = 0; i < 32; i += 4) {
                const float4 b = *reinterpret_cast<const float4*>(s_b2 + c + i);
                const float4 w = *reinterpret_cast<const float4*>(s_w3 + c + i);
                const float2 za = __fadd2_rn(make_float2(d[i], d[i + 1]), make_float2(b.x, b.y));
                const float2 zb = __fadd2_rn(make_float2(d[i + 2], d[i + 3]), make_float2(b.z, b.w));
                y2 = __ffma2_rn(FAST ? silu2_fast(za) : silu2(za), make_float2(w.x, w.y), y2);
                y2 = __ffma2_rn(FAST ? silu2_fast(zb) : silu2(zb), make_float2(w.z, w.w), y2);
            }
        }
        const float y = y2.x + y2.y;
        const float sb = valid ? net.s[brick] : 0.0f;
        const float v = valid ? fmaf(y, sb, net.m[brick]) : 0.0f;
        if (!TRAIN) {
            if (valid) {
                int64_t o = idx;
                if (!pts && grid.slots)
                    o = (int64_t)grid.slots[gk] * ((int64_t)grid.dims[0] * grid.dims[1] * grid.dims[2]) + gq;
                out[o] = v;
            }
            tc::fence_before_sync();
            __syncthreads();  // D1 / D2 and the operand tiles are reused by the next tile
            tc::fence_after_sync();
            ++tiles_done;
            continue;
        }
        // ---- backward
        const float r = valid ? v - tgt[idx] : 0.0f;
        const float dy = r * sb * g.dy_scale;
        {
            double l = (double)r * (double)r;
            for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
            if ((tid & 31) == 0 && l != 0.0) atomicAdd(&s_loss, l);
            float d3 = dy;
            for (int o = 16; o > 0; o >>= 1) d3 += __shfl_xor_sync(0xffffffffu, d3, o);
            if ((tid & 31) == 0 && d3 != 0.0f) atomicAdd(&s_db3, d3);
        }
        const int lane = tid & 31, col = colsum16_index(lane);
#pragma unroll 1
        for (int c = 0; c < kHidden; c += 16) {
            float d[16], gg[16];
            tc::tmem_ld16(T_D2 + lane_base + c, d);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float z2 = d[i] + s_b2[c + i];
                gg[i] = dy * s_w3[c + i] * silu_grad(z2);
                d[i] = dy * silu(z2);  // this point's term of dL/dw3
            }
#pragma unroll
            for (int i = 0; i < 16; i += 8)
                store_bf16x8(sm + kOffG2 + tc::kmajor_offset(tid, c + i, kHidden), gg + i);
            const float sb2 = warp_colsum16(gg, lane), sw3 = warp_colsum16(d, lane);
            if ((lane & 1) == 0) {
                atomicAdd(&s_db2[c + col], sb2);
                atomicAdd(&s_dw3[c + col], sw3);
            }
        }
        tc::fence_smem_to_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            // dH1 = G2 W2: A = G2 (K-major, K = o), B = W2 read MN-major (K = o, N = i)
            mma_chain(T_D1, sbase + kOffG2, 256, 128, 1024, sbase + kOffW2, 2048, 1024, 128,
                      tc::make_idesc_bf16(128, 64, 0, 1), 4, false);
            // dW2 += G2^T H1: A = G2 read MN-major (K = p, M = o, padded to 128),
            // B = H1 read MN-major (K = p, N = i)
            mma_chain(T_DW2, sbase + kOffG2, 2048, 1024, 128, sbase + kOffH1, 2048, 1024, 128,
                      tc::make_idesc_bf16(128, 64, 1, 1), 8, tiles_done > 0);
            tc::mma_commit(&bar);
        }
        wait_mma();
#pragma unroll 1
        for (int c = 0; c < kHidden; c += 16) {
            float d[16];
            tc::tmem_ld16(T_D1 + lane_base + c, d);
            const float* zr = reinterpret_cast<const float*>(sm + kOffZ1) + tid * kHidden + c;
#pragma unroll
            for (int i = 0; i < 16; i += 4) {
                const float4 z = *reinterpret_cast<const float4*>(zr + i);
                d[i] *= silu_grad(z.x);
                d[i + 1] *= silu_grad(z.y);
                d[i + 2] *= silu_grad(z.z);
                d[i + 3] *= silu_grad(z.w);
            }
#pragma unroll
            for (int i = 0; i < 16; i += 8)
                store_bf16x8(sm + kOffG1 + tc::kmajor_offset(tid, c + i, kHidden), d + i);
            const float sb1 = warp_colsum16(d, lane);
            if ((lane & 1) == 0) atomicAdd(&s_db1[c + col], sb1);
        }
        tc::fence_smem_to_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            // dIN = G1 W1: A = G1 (K-major, K = o), B = W1 read MN-major (K = o, N = i 32)
            mma_chain(T_DIN, sbase + kOffG1, 256, 128, 1024, sbase + kOffW1, 1024, 512, 128,
                      tc::make_idesc_bf16(128, 32, 0, 1), 4, false);
            // dW1 += G1^T IN: A = G1 read MN-major (K = p, M = o padded), B = IN read MN-major (K = p, N = i)
            mma_chain(T_DW1, sbase + kOffG1, 2048, 1024, 128, sbase + kOffIN, 1024, 512, 128,
                      tc::make_idesc_bf16(128, 32, 1, 1), 8, tiles_done > 0);
            tc::mma_commit(&bar);
        }
        wait_mma();
        {
            float d[16];
            tc::tmem_ld16(T_DIN + lane_base, d);
            if (dy != 0.0f) {
                float* gl = g.lat + (int64_t)brick * kNodes * kNodes * kNodes * kLatent;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    // 16-byte aligned: the latent gradients start on 16 bytes, 16 channels per node
                    float4* dst = reinterpret_cast<float4*>(gl + cr.node[k] * kLatent);
                    const float w = cr.w[k];
#pragma unroll
                    for (int q = 0; q < kLatent / 4; ++q)
                        atomicAdd(dst + q, make_float4(w * d[4 * q], w * d[4 * q + 1], w * d[4 * q + 2],
                                                       w * d[4 * q + 3]));
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        ++tiles_done;
    }
    if (TRAIN && ok && tiles_done > 0) {
        // rows 0..63 of the weight-gradient accumulators hold dW2 and dW1
        if (tid < kHidden) {
            for (int c = 0; c < kHidden; c += 16) {
                float d[16];
                tc::tmem_ld16(T_DW2 + lane_base + c, d);
#pragma unroll
                for (int i = 0; i < 16; ++i) atomicAdd(g.W2 + tid * kHidden + c + i, d[i]);
            }
            for (int c = 0; c < kIn; c += 16) {
                float d[16];
                tc::tmem_ld16(T_DW1 + lane_base + c, d);
#pragma unroll
                for (int i = 0; i < 16; ++i) atomicAdd(g.W1 + tid * kIn + c + i, d[i]);
            }
        } else {
            // the other warps of the pair must take part in the aligned loads
            float d[16];
            for (int c = 0; c < kHidden; c += 16) tc::tmem_ld16(T_DW2 + lane_base + c, d);
            for (int c = 0; c < kIn; c += 16) tc::tmem_ld16(T_DW1 + lane_base + c, d);
        }
        __syncthreads();
        for (int i = tid; i < kHidden; i += kTileP) {
            atomicAdd(g.b1 + i, s_db1[i]);
            atomicAdd(g.b2 + i, s_db2[i]);
            atomicAdd(g.w3 + i, s_dw3[i]);
        }
        if (tid == 0) {
            atomicAdd(g.b3, s_db3);
            atomicAdd(g.loss, s_loss);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, tcols);
}

}  // namespace codec
}  // namespace vr

// ============================================================================ host side

namespace vr {
namespace codec {

// Parameter vector layout (FP32): W1 [64][32], b1 [64], W2 [64][64], b2 [64],
// w3 [64], b3 [1], then the latents [brick][8][8][8][16].
constexpr int64_t kOfsW1 = 0, kOfsB1 = kOfsW1 + kHidden * kIn, kOfsW2 = kOfsB1 + kHidden,
                  kOfsB2 = kOfsW2 + kHidden * kHidden, kOfsW3 = kOfsB2 + kHidden, kOfsB3 = kOfsW3 + kHidden,
                  kOfsLat = kOfsB3 + 1;
// floats in front of the gradient vector so that its latent part starts on 16 bytes
// (the latent gradients are accumulated four channels at a time)
constexpr int64_t kGradPad = (4 - kOfsLat % 4) % 4;
constexpr int64_t kLatPerBrick = (int64_t)kNodes * kNodes * kNodes * kLatent;

__global__ void to_bf16_kernel(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16_rn(src[i]);
}
__global__ void round_bf16_kernel(const float* __restrict__ src, float* __restrict__ dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __bfloat162float(__float2bfloat16_rn(src[i]));
}

// Adam (bias-corrected), one step over the whole parameter vector.
__global__ void adam_kernel(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m1,
                            float* __restrict__ m2, int64_t n, float lr, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = m1[i] = 0.9f * m1[i] + 0.1f * gi;
        const float b = m2[i] = 0.999f * m2[i] + 0.001f * gi * gi;
        th[i] -= lr * (a * c1) / (sqrtf(b * c2) + 1e-8f);
    }
}

// splitmix64 (a counter-based generator): 64 random bits of counter x.
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Training points: uniform brick, uniform voxel of its (B+1)^3 block clipped to
// the cube; target = the cube's value there.  cube holds the planes from z = zoff
// on (the whole cube when zoff = 0); without a list of shown bricks the brick is
// uniform among [b_lo, b_hi).
__global__ void sample_kernel(const float* __restrict__ cube, int64_t zoff, int3 n, int3 B, int3 nb,
                              int32_t b_lo, int32_t b_hi, int64_t n_points, uint64_t seed, float floor_v,
                              const uint32_t* __restrict__ active, uint64_t n_active, float active_frac,
                              const int32_t* __restrict__ shown, int32_t n_shown, float4* __restrict__ pts,
                              float* __restrict__ tgt) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_points) return;
    const uint64_t r0 = mix64(seed ^ (uint64_t)(3 * i)), r1 = mix64(seed ^ (uint64_t)(3 * i + 1));
    const uint64_t r2 = mix64(seed ^ (uint64_t)(3 * i + 2));
    int b, gx, gy, gz, bx, by, bz;
    if (n_active > 0 && (float)(r2 >> 40) * (1.0f / 16777216.0f) < active_frac) {
        // a voxel the transfer function can show, in the brick that owns it
        const uint64_t v = active[r0 % n_active];
        gx = (int)(v % (uint64_t)n.x);
        gy = (int)((v / (uint64_t)n.x) % (uint64_t)n.y);
        gz = (int)(v / ((uint64_t)n.x * (uint64_t)n.y));
        bx = min(gx / B.x, nb.x - 1);
        by = min(gy / B.y, nb.y - 1);
        bz = min(gz / B.z, nb.z - 1);
        b = (bz * nb.y + by) * nb.x + bx;
    } else {
        // a uniform brick among those the transfer function can show (all bricks
        // when none is listed), then a uniform voxel of its block
        b = n_shown > 0 ? shown[r0 % (uint64_t)n_shown] : b_lo + (int)(r0 % (uint64_t)(b_hi - b_lo));
        bx = b % nb.x;
        by = (b / nb.x) % nb.y;
        bz = b / (nb.x * nb.y);
        const int ux = (int)((r1 & 0xFFFFF) % (uint64_t)(B.x + 1));
        const int uy = (int)(((r1 >> 20) & 0xFFFFF) % (uint64_t)(B.y + 1));
        const int uz = (int)(((r1 >> 40) & 0xFFFFF) % (uint64_t)(B.z + 1));
        gx = min(bx * B.x + ux, n.x - 1);
        gy = min(by * B.y + uy, n.y - 1);
        gz = min(bz * B.z + uz, n.z - 1);
    }
    pts[i] = make_float4((float)(gx - bx * B.x), (float)(gy - by * B.y), (float)(gz - bz * B.z), __int_as_float(b));
    tgt[i] = fmaxf(cube[(((int64_t)gz - zoff) * n.y + gy) * n.x + gx], floor_v);
}

// Voxels above the floor (the ones the transfer function can show): count, then
// list (global linear indices; order unspecified).
__global__ void active_kernel(const float* __restrict__ cube, int64_t n, float floor_v, unsigned long long* count,
                              uint32_t* __restrict__ list, unsigned long long cap) {
    // every warp runs the same number of iterations (the ballot needs all its lanes)
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n_round = (n + stride - 1) / stride * stride;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_round; i += stride) {
        const bool a = i < n && cube[i] > floor_v;
        const unsigned mask = __ballot_sync(0xffffffffu, a);
        unsigned long long base = 0;
        if ((threadIdx.x & 31) == 0 && mask) base = atomicAdd(count, (unsigned long long)__popc(mask));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (list && a) {
            const unsigned long long k = base + __popc(mask & ((1u << (threadIdx.x & 31)) - 1u));
            if (k < cap) list[k] = (uint32_t)i;
        }
    }
}

// Per-brick offset and scale: mean and standard deviation (at least 1e-3) over
// the brick's voxels and apron.
__global__ void brick_stats_kernel(const float* __restrict__ cube, int64_t zoff, int3 n, int3 B, int3 nb, int32_t b0,
                                   float floor_v, float* m, float* s, float2* mm) {
    const int b = b0 + (int)blockIdx.x;
    const int bx = b % nb.x, by = (b / nb.x) % nb.y, bz = b / (nb.x * nb.y);
    const int x0 = bx * B.x, y0 = by * B.y, z0 = bz * B.z;
    const int x1 = min(x0 + B.x, n.x - 1), y1 = min(y0 + B.y, n.y - 1), z1 = min(z0 + B.z, n.z - 1);
    double s1 = 0, s2 = 0;
    float lo = FLT_MAX, hi = -FLT_MAX;
    const int64_t cnt = (int64_t)(x1 - x0 + 1) * (y1 - y0 + 1) * (z1 - z0 + 1);
    for (int64_t q = threadIdx.x; q < cnt; q += blockDim.x) {
        const int x = x0 + (int)(q % (x1 - x0 + 1));
        const int y = y0 + (int)((q / (x1 - x0 + 1)) % (y1 - y0 + 1));
        const int z = z0 + (int)(q / ((int64_t)(x1 - x0 + 1) * (y1 - y0 + 1)));
        const float raw = cube[(((int64_t)z - zoff) * n.y + y) * n.x + x];
        lo = fminf(lo, raw);
        hi = fmaxf(hi, raw);
        const double v = fmaxf(raw, floor_v);
        s1 += v;
        s2 += v * v;
    }
    __shared__ double a1[256], a2[256];
    __shared__ float l1[256], h1[256];
    a1[threadIdx.x] = s1;
    a2[threadIdx.x] = s2;
    l1[threadIdx.x] = lo;
    h1[threadIdx.x] = hi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            a1[threadIdx.x] += a1[threadIdx.x + o];
            a2[threadIdx.x] += a2[threadIdx.x + o];
            l1[threadIdx.x] = fminf(l1[threadIdx.x], l1[threadIdx.x + o]);
            h1[threadIdx.x] = fmaxf(h1[threadIdx.x], h1[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mean = a1[0] / (double)cnt;
        const double var = fmax(a2[0] / (double)cnt - mean * mean, 0.0);
        m[b] = (float)mean;
        s[b] = (float)fmax(sqrt(var), 1e-3);
        mm[b] = make_float2(l1[0], h1[0]);
    }
}

}  // namespace codec
}  // namespace vr

struct vr_codec {
    int device = 0;
    int32_t n_bricks = 0;
    int32_t B[3] = {0, 0, 0};
    int64_t n_params = 0;
    float* theta = nullptr;  // FP32 parameters
    float* grad = nullptr;       // grad_mem + kGradPad: the latents' gradients 16-byte aligned
    float* grad_mem = nullptr;
    float* adam1 = nullptr;
    float* adam2 = nullptr;
    __nv_bfloat16* W1h = nullptr;
    __nv_bfloat16* W2h = nullptr;
    __nv_bfloat16* lath = nullptr;
    float* latf = nullptr;   // the BF16 latents as FP32 values (brick decode)
    float4* four = nullptr;  // Fourier features of the grid coordinates (brick decode)
    float* w3r = nullptr;  // w3 rounded to BF16 values
    float* m = nullptr;
    float* s = nullptr;
    float2* minmax = nullptr;  // per-brick range of the data the codec was fitted to
    float floor_v = -FLT_MAX;  // training targets are max(value, floor_v)
    uint32_t* active = nullptr;  // voxels above the floor (global linear indices)
    uint64_t n_active = 0;
    int32_t* shown = nullptr;    // bricks with values above the floor (the others render empty)
    int32_t n_shown = 0;
    unsigned long long* d_count = nullptr;
    double* loss = nullptr;
    int* err = nullptr;
    float4* pts = nullptr;
    float* tgt = nullptr;
    int64_t cap_pts = 0;
    int64_t adam_t = 0;               // Adam steps of the shared network
    std::vector<int64_t> lat_t;       // per brick: Adam steps of its latents
    std::vector<float2> h_minmax;     // host copy of minmax
    int32_t* shown_range = nullptr;   // shown bricks of the last slab trained
    int32_t cap_shown_range = 0;
    int sm_count = 0;
};

namespace {

using vr::codec::Net;

uint64_t mix64_host(uint64_t seed, uint64_t step) {
    uint64_t x = seed + 0x9E3779B97F4A7C15ull * (step + 1);
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

int codec_cuda(cudaError_t e) { return e == cudaSuccess ? VR_OK : (cudaGetLastError(), VR_ECUDA); }
#define CODEC_CUDA(call)                        \
    do {                                        \
        int _rc = codec_cuda(call);             \
        if (_rc) return _rc;                    \
    } while (0)

// Refresh the BF16 operand copies from the FP32 parameters (the latents of
// bricks [b0, b1) only; b1 < 0: every brick).
int sync_bf16(vr_codec* c, int32_t b0 = 0, int32_t b1 = -1) {
    using namespace vr::codec;
    if (b1 < 0) b1 = c->n_bricks;
    to_bf16_kernel<<<64, 256>>>(c->theta + kOfsW1, c->W1h, kHidden * kIn);
    to_bf16_kernel<<<64, 256>>>(c->theta + kOfsW2, c->W2h, kHidden * kHidden);
    round_bf16_kernel<<<1, 64>>>(c->theta + kOfsW3, c->w3r, kHidden);
    const int64_t o = (int64_t)b0 * kLatPerBrick, k = (int64_t)(b1 - b0) * kLatPerBrick;
    if (k > 0) {
        to_bf16_kernel<<<1024, 256>>>(c->theta + kOfsLat + o, c->lath + o, k);
        round_bf16_kernel<<<1024, 256>>>(c->theta + kOfsLat + o, c->latf + o, k);
    }
    return codec_cuda(cudaGetLastError());
}

Net make_net(const vr_codec* c) {
    using namespace vr::codec;
    Net n;
    n.lat = c->lath;
    n.latf = c->latf;
    n.four = c->four;
    n.four_off[0] = 0;
    n.four_off[1] = c->B[0] + 1;
    n.four_off[2] = c->B[0] + c->B[1] + 2;
    n.W1 = c->W1h;
    n.W2 = c->W2h;
    n.b1 = c->theta + kOfsB1;
    n.b2 = c->theta + kOfsB2;
    n.w3 = c->w3r;
    n.b3 = c->theta + kOfsB3;
    n.m = c->m;
    n.s = c->s;
    for (int a = 0; a < 3; ++a) n.inv_b[a] = 1.0f / (float)c->B[a];
    return n;
}

int grow_points(vr_codec* c, int64_t n) {
    if (n <= c->cap_pts) return VR_OK;
    cudaFree(c->pts);
    cudaFree(c->tgt);
    c->pts = nullptr;
    c->tgt = nullptr;
    c->cap_pts = 0;
    if (cudaMalloc(&c->pts, n * sizeof(float4)) != cudaSuccess || cudaMalloc(&c->tgt, n * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return VR_ENOMEM;
    }
    c->cap_pts = n;
    return VR_OK;
}

template <bool TRAIN, bool FAST = false>
int launch_codec(vr_codec* c, const float4* pts, vr::codec::Grid grid, const float* tgt, int64_t n, float* out,
                 cudaStream_t st) {
    using namespace vr::codec;
    if (n == 0) return VR_OK;
    const int smem = TRAIN ? (int)kSmemTrain : (int)kSmemInfer;
    static bool attr = false;
    if (!attr) {
        CODEC_CUDA(cudaFuncSetAttribute(codec_kernel<TRAIN, FAST>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr = true;
    }
    Grads g{};
    if (TRAIN) {
        g.W1 = c->grad + kOfsW1;
        g.W2 = c->grad + kOfsW2;
        g.b1 = c->grad + kOfsB1;
        g.b2 = c->grad + kOfsB2;
        g.w3 = c->grad + kOfsW3;
        g.b3 = c->grad + kOfsB3;
        g.lat = c->grad + kOfsLat;
        g.loss = c->loss;
        g.dy_scale = 2.0f / (float)n;
    }
    const int64_t tiles = (n + kTileP - 1) / kTileP;
    const int64_t grid_ctas = std::min<int64_t>(tiles, (int64_t)c->sm_count * (TRAIN ? kCtasTrain : kCtasInfer));
    codec_kernel<TRAIN, FAST><<<(unsigned)grid_ctas, kTileP, smem, st>>>(make_net(c), pts, grid, tgt, n, out, g, c->err);
    return codec_cuda(cudaGetLastError());
}

int check_err(vr_codec* c) {
    int h = 0;
    CODEC_CUDA(cudaMemcpy(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost));
    return h ? VR_ETIMEOUT : VR_OK;
}

// Bricks per axis of an (nx, ny, nz) cube bricked by the codec's B; false when
// the count differs from the codec's.
bool codec_grid(const vr_codec* c, int64_t nx, int64_t ny, int64_t nz, int3& n, int3& B, int3& nb) {
    if (nx < 2 || ny < 2 || nz < 2 || nx > 65536 || ny > 65536 || nz > 65536) return false;
    n = make_int3((int)nx, (int)ny, (int)nz);
    B = make_int3(c->B[0], c->B[1], c->B[2]);
    nb = make_int3((int)((nx - 2 + B.x) / B.x), (int)((ny - 2 + B.y) / B.y), (int)((nz - 2 + B.z) / B.z));
    return (int64_t)nb.x * nb.y * nb.z == c->n_bricks;
}

// Offset, scale and range of bricks [b0, b1) from cube planes zoff on.
int fit_range(vr_codec* c, const float* cube, int64_t zoff, int3 n, int3 B, int3 nb, int32_t b0, int32_t b1,
              float floor_v) {
    using namespace vr::codec;
    c->floor_v = floor_v;
    if (b1 <= b0) return VR_OK;
    brick_stats_kernel<<<b1 - b0, 256>>>(cube, zoff, n, B, nb, b0, floor_v, c->m, c->s, c->minmax);
    CODEC_CUDA(cudaGetLastError());
    CODEC_CUDA(cudaMemcpy(c->h_minmax.data() + b0, c->minmax + b0, (size_t)(b1 - b0) * sizeof(float2),
                          cudaMemcpyDeviceToHost));
    return VR_OK;
}

// `steps` Adam steps on points of bricks [b0, b1) (from `shown` when listed) read
// from cube planes zoff on: the shared network at rate mlp_lr (0: unchanged), the
// latents of bricks [b0, b1) at rate lr; gradients, moments and BF16 copies of
// other bricks' latents are not touched.
int train_range(vr_codec* c, const float* cube, int64_t zoff, int3 n, int3 B, int3 nb, int32_t b0, int32_t b1,
                const int32_t* shown, int32_t n_shown, float active_frac, int32_t steps, int32_t batch, float lr,
                float mlp_lr, uint64_t seed, double* last_loss) {
    using namespace vr::codec;
    int rc = grow_points(c, batch);
    if (rc) return rc;
    const int64_t lo = kOfsLat + (int64_t)b0 * kLatPerBrick, cnt = (int64_t)(b1 - b0) * kLatPerBrick;
    const bool whole = zoff == 0 && b0 == 0 && b1 == c->n_bricks;
    int64_t t_lat = 0;
    for (int32_t b = b0; b < b1; ++b) t_lat = std::max(t_lat, c->lat_t[b]);
    for (int32_t it = 0; it < steps; ++it) {
        sample_kernel<<<(batch + 255) / 256, 256>>>(cube, zoff, n, B, nb, b0, b1, batch, mix64_host(seed, it),
                                                    c->floor_v, whole ? c->active : nullptr, whole ? c->n_active : 0,
                                                    active_frac, shown, n_shown, c->pts, c->tgt);
        CODEC_CUDA(cudaMemsetAsync(c->grad, 0, (size_t)kOfsLat * 4));
        CODEC_CUDA(cudaMemsetAsync(c->grad + lo, 0, (size_t)cnt * 4));
        CODEC_CUDA(cudaMemsetAsync(c->loss, 0, sizeof(double)));
        if ((rc = launch_codec<true>(c, c->pts, Grid{}, c->tgt, batch, nullptr, 0))) return rc;
        if (mlp_lr > 0.0f) {
            ++c->adam_t;
            const float c1 = 1.0f / (1.0f - powf(0.9f, (float)c->adam_t));
            const float c2 = 1.0f / (1.0f - powf(0.999f, (float)c->adam_t));
            adam_kernel<<<64, 256>>>(c->theta, c->grad, c->adam1, c->adam2, kOfsLat, mlp_lr, c1, c2);
        }
        ++t_lat;
        const float c1 = 1.0f / (1.0f - powf(0.9f, (float)t_lat));
        const float c2 = 1.0f / (1.0f - powf(0.999f, (float)t_lat));
        adam_kernel<<<1024, 256>>>(c->theta + lo, c->grad + lo, c->adam1 + lo, c->adam2 + lo, cnt, lr, c1, c2);
        if ((rc = sync_bf16(c, b0, b1))) return rc;
    }
    for (int32_t b = b0; b < b1; ++b) c->lat_t[b] = t_lat;
    CODEC_CUDA(cudaDeviceSynchronize());
    if ((rc = check_err(c))) return rc;
    if (last_loss) {
        double l = 0;
        CODEC_CUDA(cudaMemcpy(&l, c->loss, sizeof(double), cudaMemcpyDeviceToHost));
        *last_loss = l / (double)batch;
    }
    return VR_OK;
}

}  // namespace

extern "C" {

int vr_codec_create(int32_t n_bricks, const int32_t B[3], vr_codec** out) {
    using namespace vr::codec;
    if (!out || !B || n_bricks < 1 || B[0] < 1 || B[1] < 1 || B[2] < 1) return VR_EINVAL;
    *out = nullptr;
    vr_codec* c = new vr_codec();
    cudaGetDevice(&c->device);
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
    c->n_bricks = n_bricks;
    for (int a = 0; a < 3; ++a) c->B[a] = B[a];
    c->n_params = kOfsLat + (int64_t)n_bricks * kLatPerBrick;
    c->lat_t.assign(n_bricks, 0);
    c->h_minmax.assign(n_bricks, make_float2(0.0f, 0.0f));
    const size_t pb = (size_t)c->n_params * sizeof(float);
    bool ok = cudaMalloc(&c->theta, pb) == cudaSuccess &&
              cudaMalloc(&c->grad_mem, pb + kGradPad * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&c->adam1, pb) == cudaSuccess && cudaMalloc(&c->adam2, pb) == cudaSuccess &&
              cudaMalloc(&c->W1h, kHidden * kIn * 2) == cudaSuccess &&
              cudaMalloc(&c->W2h, kHidden * kHidden * 2) == cudaSuccess &&
              cudaMalloc(&c->lath, (size_t)n_bricks * kLatPerBrick * 2) == cudaSuccess &&
              cudaMalloc(&c->latf, (size_t)n_bricks * kLatPerBrick * 4) == cudaSuccess &&
              cudaMalloc(&c->four, (size_t)(B[0] + B[1] + B[2] + 3) * sizeof(float4)) == cudaSuccess &&
              cudaMalloc(&c->w3r, kHidden * 4) == cudaSuccess && cudaMalloc(&c->m, n_bricks * 4) == cudaSuccess &&
              cudaMalloc(&c->s, n_bricks * 4) == cudaSuccess && cudaMalloc(&c->minmax, n_bricks * 8) == cudaSuccess &&
              cudaMalloc(&c->loss, sizeof(double)) == cudaSuccess &&
              cudaMalloc(&c->err, sizeof(int)) == cudaSuccess;
    if (ok) c->grad = c->grad_mem + kGradPad;
    if (ok) {
        // Fourier features of the grid coordinates x = u / B_a (u = 0..B_a) along each
        // axis: sin(pi x), cos(pi x), sin(2 pi x), cos(2 pi x), rounded from FP64
        std::vector<float4> tab;
        for (int a = 0; a < 3; ++a)
            for (int u = 0; u <= B[a]; ++u) {
                const double x = (double)u / (double)B[a];
                tab.push_back(make_float4((float)std::sin(M_PI * x), (float)std::cos(M_PI * x),
                                          (float)std::sin(2.0 * M_PI * x), (float)std::cos(2.0 * M_PI * x)));
            }
        ok = cudaMemcpy(c->four, tab.data(), tab.size() * sizeof(float4), cudaMemcpyHostToDevice) == cudaSuccess;
    }
    if (ok) ok = cudaMemset(c->theta, 0, pb) == cudaSuccess && cudaMemset(c->adam1, 0, pb) == cudaSuccess &&
                 cudaMemset(c->adam2, 0, pb) == cudaSuccess && cudaMemset(c->err, 0, sizeof(int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        vr_codec_destroy(c);
        return VR_ENOMEM;
    }
    *out = c;
    return VR_OK;
}

void vr_codec_destroy(vr_codec* c) {
    if (!c) return;
    for (void* p : {(void*)c->theta, (void*)c->grad_mem, (void*)c->adam1, (void*)c->adam2, (void*)c->W1h, (void*)c->W2h,
                    (void*)c->lath, (void*)c->latf, (void*)c->four, (void*)c->w3r, (void*)c->m, (void*)c->s,
                    (void*)c->minmax, (void*)c->loss,
                    (void*)c->err, (void*)c->active, (void*)c->d_count, (void*)c->shown, (void*)c->shown_range,
                    (void*)c->pts, (void*)c->tgt})
        cudaFree(p);
    delete c;
}

int64_t vr_codec_param_count(const vr_codec* c) { return c ? c->n_params : -1; }

int vr_codec_set_params(vr_codec* c, const float* theta, const float* m, const float* s) {
    if (!c || !theta || !m || !s) return VR_EINVAL;
    CODEC_CUDA(cudaMemcpy(c->theta, theta, (size_t)c->n_params * 4, cudaMemcpyHostToDevice));
    CODEC_CUDA(cudaMemcpy(c->m, m, (size_t)c->n_bricks * 4, cudaMemcpyHostToDevice));
    CODEC_CUDA(cudaMemcpy(c->s, s, (size_t)c->n_bricks * 4, cudaMemcpyHostToDevice));
    c->adam_t = 0;
    std::fill(c->lat_t.begin(), c->lat_t.end(), 0);
    CODEC_CUDA(cudaMemset(c->adam1, 0, (size_t)c->n_params * 4));
    CODEC_CUDA(cudaMemset(c->adam2, 0, (size_t)c->n_params * 4));
    return sync_bf16(c);
}

int vr_codec_get_params(vr_codec* c, float* theta, float* m, float* s) {
    if (!c || !theta) return VR_EINVAL;
    CODEC_CUDA(cudaMemcpy(theta, c->theta, (size_t)c->n_params * 4, cudaMemcpyDeviceToHost));
    if (m) CODEC_CUDA(cudaMemcpy(m, c->m, (size_t)c->n_bricks * 4, cudaMemcpyDeviceToHost));
    if (s) CODEC_CUDA(cudaMemcpy(s, c->s, (size_t)c->n_bricks * 4, cudaMemcpyDeviceToHost));
    return VR_OK;
}

// Every point names an existing brick.
bool points_valid(const vr_codec* c, const float* points, int64_t n) {
    for (int64_t i = 0; i < n; ++i) {
        int32_t b;
        std::memcpy(&b, points + 4 * i + 3, 4);
        if (b < 0 || b >= c->n_bricks) return false;
    }
    return true;
}

int vr_codec_forward(vr_codec* c, const float* points, int64_t n, float* values) {
    if (!c || !points || !values || n < 0 || !points_valid(c, points, n)) return VR_EINVAL;
    int rc = grow_points(c, std::max<int64_t>(n, 1));
    if (rc) return rc;
    float* d_out = nullptr;
    CODEC_CUDA(cudaMalloc(&d_out, std::max<int64_t>(n, 1) * 4));
    CODEC_CUDA(cudaMemcpy(c->pts, points, n * 16, cudaMemcpyHostToDevice));
    rc = launch_codec<false>(c, c->pts, vr::codec::Grid{}, nullptr, n, d_out, 0);
    if (!rc) rc = codec_cuda(cudaDeviceSynchronize());
    if (!rc) rc = check_err(c);
    if (!rc) rc = codec_cuda(cudaMemcpy(values, d_out, n * 4, cudaMemcpyDeviceToHost));
    cudaFree(d_out);
    return rc;
}

int vr_codec_gradient(vr_codec* c, const float* points, const float* targets, int64_t n, float* grad, double* loss) {
    if (!c || !points || !targets || !grad || n < 1 || !points_valid(c, points, n)) return VR_EINVAL;
    int rc = grow_points(c, n);
    if (rc) return rc;
    CODEC_CUDA(cudaMemcpy(c->pts, points, n * 16, cudaMemcpyHostToDevice));
    CODEC_CUDA(cudaMemcpy(c->tgt, targets, n * 4, cudaMemcpyHostToDevice));
    CODEC_CUDA(cudaMemset(c->grad, 0, (size_t)c->n_params * 4));
    CODEC_CUDA(cudaMemset(c->loss, 0, sizeof(double)));
    if ((rc = launch_codec<true>(c, c->pts, vr::codec::Grid{}, c->tgt, n, nullptr, 0))) return rc;
    CODEC_CUDA(cudaDeviceSynchronize());
    if ((rc = check_err(c))) return rc;
    CODEC_CUDA(cudaMemcpy(grad, c->grad, (size_t)c->n_params * 4, cudaMemcpyDeviceToHost));
    double l = 0;
    CODEC_CUDA(cudaMemcpy(&l, c->loss, sizeof(double), cudaMemcpyDeviceToHost));
    if (loss) *loss = l / (double)n;
    return VR_OK;
}

int vr_codec_fit_stats(vr_codec* c, const float* cube, int64_t nx, int64_t ny, int64_t nz, float floor_v) {
    using namespace vr::codec;
    if (!c || !cube) return VR_EINVAL;
    int3 n, B, nb;
    if (!codec_grid(c, nx, ny, nz, n, B, nb)) return VR_EINVAL;
    int rc = fit_range(c, cube, 0, n, B, nb, 0, c->n_bricks, floor_v);
    if (rc) return rc;
    // the bricks with values above the floor: training samples only those (the
    // others are skipped by the renderer's empty-space test whenever the transfer
    // function is transparent up to the floor)
    {
        const std::vector<float2>& mm = c->h_minmax;
        std::vector<int32_t> shown;
        for (int32_t b = 0; b < c->n_bricks; ++b)
            if (mm[b].y > floor_v) shown.push_back(b);
        cudaFree(c->shown);
        c->shown = nullptr;
        c->n_shown = 0;
        if (!shown.empty() && floor_v > -FLT_MAX) {
            CODEC_CUDA(cudaMalloc(&c->shown, shown.size() * sizeof(int32_t)));
            CODEC_CUDA(cudaMemcpy(c->shown, shown.data(), shown.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
            c->n_shown = (int32_t)shown.size();
        }
    }
    // the voxels above the floor, for importance sampling in training
    cudaFree(c->active);
    c->active = nullptr;
    c->n_active = 0;
    if (!c->d_count) CODEC_CUDA(cudaMalloc(&c->d_count, sizeof(unsigned long long)));
    const int64_t nv = nx * ny * nz;
    unsigned long long cnt = 0;
    CODEC_CUDA(cudaMemset(c->d_count, 0, sizeof(cnt)));
    active_kernel<<<4096, 256>>>(cube, nv, floor_v, c->d_count, nullptr, 0);
    CODEC_CUDA(cudaMemcpy(&cnt, c->d_count, sizeof(cnt), cudaMemcpyDeviceToHost));
    if (cnt > 0 && nv <= 0xFFFFFFFFll) {
        if (cudaMalloc(&c->active, cnt * sizeof(uint32_t)) != cudaSuccess) {
            cudaGetLastError();
            return VR_ENOMEM;
        }
        CODEC_CUDA(cudaMemset(c->d_count, 0, sizeof(cnt)));
        active_kernel<<<4096, 256>>>(cube, nv, floor_v, c->d_count, c->active, cnt);
        c->n_active = cnt;
    }
    return codec_cuda(cudaDeviceSynchronize());
}

int vr_codec_get_minmax(vr_codec* c, float* out) {
    if (!c || !out) return VR_EINVAL;
    return codec_cuda(cudaMemcpy(out, c->minmax, (size_t)c->n_bricks * 8, cudaMemcpyDeviceToHost));
}

int vr_codec_train(vr_codec* c, const float* cube, int64_t nx, int64_t ny, int64_t nz, int32_t steps, int32_t batch,
                   float lr, float active_frac, uint64_t seed, double* last_loss) {
    if (!c || !cube || steps < 0 || batch < 1) return VR_EINVAL;
    int3 n, B, nb;
    if (!codec_grid(c, nx, ny, nz, n, B, nb)) return VR_EINVAL;
    return train_range(c, cube, 0, n, B, nb, 0, c->n_bricks, c->shown, c->n_shown, active_frac, steps, batch, lr, lr,
                       seed, last_loss);
}

int vr_codec_fit_stats_slab(vr_codec* c, const float* slab, int64_t nx, int64_t ny, int64_t nz, int32_t bz0,
                            int32_t bz1, float floor_v) {
    if (!c || !slab) return VR_EINVAL;
    int3 n, B, nb;
    if (!codec_grid(c, nx, ny, nz, n, B, nb) || bz0 < 0 || bz1 > nb.z || bz0 >= bz1) return VR_EINVAL;
    const int32_t layer = nb.x * nb.y;
    int rc = fit_range(c, slab, (int64_t)bz0 * B.z, n, B, nb, bz0 * layer, bz1 * layer, floor_v);
    if (rc) return rc;
    return codec_cuda(cudaDeviceSynchronize());
}

int vr_codec_train_slab(vr_codec* c, const float* slab, int64_t nx, int64_t ny, int64_t nz, int32_t bz0, int32_t bz1,
                        int32_t steps, int32_t batch, float lr, float mlp_lr, uint64_t seed, double* last_loss) {
    if (!c || !slab || steps < 0 || batch < 1 || !(lr >= 0.0f) || !(mlp_lr >= 0.0f)) return VR_EINVAL;
    int3 n, B, nb;
    if (!codec_grid(c, nx, ny, nz, n, B, nb) || bz0 < 0 || bz1 > nb.z || bz0 >= bz1) return VR_EINVAL;
    const int32_t layer = nb.x * nb.y, b0 = bz0 * layer, b1 = bz1 * layer;
    // the slab's bricks with values above the floor (all of them when none has)
    std::vector<int32_t> shown;
    if (c->floor_v > -FLT_MAX)
        for (int32_t b = b0; b < b1; ++b)
            if (c->h_minmax[b].y > c->floor_v) shown.push_back(b);
    if (shown.empty() && c->floor_v > -FLT_MAX) {   // nothing to learn: the renderer skips these bricks
        if (last_loss) *last_loss = 0.0;
        return VR_OK;
    }
    if ((int32_t)shown.size() > c->cap_shown_range) {
        cudaFree(c->shown_range);
        c->shown_range = nullptr;
        c->cap_shown_range = 0;
        if (cudaMalloc(&c->shown_range, shown.size() * sizeof(int32_t)) != cudaSuccess) {
            cudaGetLastError();
            return VR_ENOMEM;
        }
        c->cap_shown_range = (int32_t)shown.size();
    }
    if (!shown.empty())
        CODEC_CUDA(cudaMemcpy(c->shown_range, shown.data(), shown.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    return train_range(c, slab, (int64_t)bz0 * B.z, n, B, nb, b0, b1, shown.empty() ? nullptr : c->shown_range,
                       (int32_t)shown.size(), 0.0f, steps, batch, lr, mlp_lr, seed, last_loss);
}

int vr_codec_decode_bricks(vr_codec* c, const int32_t* bricks, const int32_t* slots, int32_t n, float* out,
                           void* stream) {
    using namespace vr::codec;
    if (!c || (!bricks && n > 0) || !out || n < 0) return VR_EINVAL;
    if (n == 0) return VR_OK;
    Grid grid;
    grid.bricks = bricks;
    grid.slots = slots;
    for (int a = 0; a < 3; ++a) grid.dims[a] = c->B[a] + 1;
    const int64_t pts = (int64_t)n * grid.dims[0] * grid.dims[1] * grid.dims[2];
    return launch_codec<false, true>(c, nullptr, grid, nullptr, pts, out, (cudaStream_t)stream);
}

int32_t vr_codec_brick_count(const vr_codec* c) { return c ? c->n_bricks : -1; }
void vr_codec_brick_size(const vr_codec* c, int32_t B[3]) {
    for (int a = 0; a < 3; ++a) B[a] = c ? c->B[a] : 0;
}

}  // extern "C"
