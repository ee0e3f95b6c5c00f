// Learned brick codec: a shared MLP decoder evaluated on the fifth-generation
// tensor cores (tcgen05, BF16 operands, FP32 accumulation in tensor memory).
//
// This file holds the tensor-core building blocks and their self-check: a
// 128 x N x K product through the same shared-memory layouts, descriptors and
// tensor-memory reads that the codec's kernels use.
#include <cuda_bf16.h>

#include <cstdint>

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
