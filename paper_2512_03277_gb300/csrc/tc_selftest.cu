// Diagnostic: one 128 x N tile of C = A B^T on the fifth-generation tensor cores (BF16 in, FP32
// accumulate in TMEM), through the same building blocks the coupling contraction uses.
#include <cuda_bf16.h>

#include <string>

#include "tc_common.cuh"

namespace {

constexpr int KB = 64;                     // K elements staged per step
constexpr uint32_t SMEM_BYTES = 200 * 1024;   // room beyond the operand tiles (see the host side)

template <int N>
__global__ void __launch_bounds__(128) k_tc_selftest(const __nv_bfloat16 *__restrict__ A,
                                                     const __nv_bfloat16 *__restrict__ B, int K,
                                                     float *__restrict__ C, unsigned *__restrict__ status) {
    extern __shared__ __align__(1024) uint8_t smem[];
    constexpr uint32_t LBO_A = (128 / 8) * 128, LBO_B = (N / 8) * 128;
    uint8_t *sa = smem;
    uint8_t *sb = smem + 128 * KB * 2;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + SMEM_BYTES - 64);
    uint32_t *slot = reinterpret_cast<uint32_t *>(smem + SMEM_BYTES - 32);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(slot, N);
    if (tid == 0) tc::mbar_init(bar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    const uint32_t idesc = tc::idesc_bf16(128, N);
    uint32_t phase = 0;
    bool ok = true;
    for (int kb = 0; kb < K && ok; kb += KB) {
        for (int e = tid; e < 128 * KB; e += 128) {
            const int r = e / KB, k = e - r * KB;
            *reinterpret_cast<__nv_bfloat16 *>(sa + tc::core_offset(r, k, LBO_A)) = A[(size_t)r * K + kb + k];
        }
        for (int e = tid; e < N * KB; e += 128) {
            const int r = e / KB, k = e - r * KB;
            *reinterpret_cast<__nv_bfloat16 *>(sb + tc::core_offset(r, k, LBO_B)) = B[(size_t)r * K + kb + k];
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            for (int kk = 0; kk < KB / 16; ++kk) {
                const uint64_t ad = tc::make_desc(tc::smem_u32(sa) + kk * 2 * LBO_A, LBO_A, 128);
                const uint64_t bd = tc::make_desc(tc::smem_u32(sb) + kk * 2 * LBO_B, LBO_B, 128);
                tc::mma_bf16(tmem, ad, bd, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
            }
            tc::mma_commit(bar);
        }
        const bool got = tc::mbar_wait(bar, phase);
        ok = __syncthreads_and(got) != 0;
        phase ^= 1u;
    }
    if (!ok) {
        tc::mbar_wait(bar, phase ^ 1u);   // one more bounded wait for the MMAs still in flight
        if (tid == 0) atomicOr(status, (unsigned)ERRBIT_TIMEOUT);
    }
    tc::fence_after_sync();
    if (ok) {
        for (int c0 = 0; c0 < N; c0 += 32) {
            float v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
            const int row = 32 * warp + lane;
#pragma unroll
            for (int i = 0; i < 32; ++i) C[(size_t)row * N + c0 + i] = v[i];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, N);
}

}  // namespace

extern "C" int cavmd_tc_selftest(const uint16_t *A, const uint16_t *B, int32_t K, int32_t N, float *C) {
    if (!A || !B || !C || K < 64 || K % 64 != 0 || (N != 128 && N != 256)) {
        cavmd_set_global_error("cavmd_tc_selftest: need K a positive multiple of 64 and N of 128 or 256");
        return CAVMD_ERR_INVALID_ARG;
    }
    void *dA = nullptr, *dB = nullptr, *dC = nullptr, *dS = nullptr;
    auto cleanup = [&]() { cudaFree(dA); cudaFree(dB); cudaFree(dC); cudaFree(dS); };
    cudaError_t e = cudaMalloc(&dA, (size_t)128 * K * 2);
    if (e == cudaSuccess) e = cudaMalloc(&dB, (size_t)N * K * 2);
    if (e == cudaSuccess) e = cudaMalloc(&dC, (size_t)128 * N * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dS, 4);
    if (e == cudaSuccess) e = cudaMemcpy(dA, A, (size_t)128 * K * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dB, B, (size_t)N * K * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(dS, 0, 4);
    if (e == cudaSuccess) {
        if (N == 128) {
            e = cudaFuncSetAttribute(k_tc_selftest<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
            if (e == cudaSuccess)
                k_tc_selftest<128><<<1, 128, SMEM_BYTES>>>((const __nv_bfloat16 *)dA, (const __nv_bfloat16 *)dB, K,
                                                          (float *)dC, (unsigned *)dS);
        } else {
            e = cudaFuncSetAttribute(k_tc_selftest<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
            if (e == cudaSuccess)
                k_tc_selftest<256><<<1, 128, SMEM_BYTES>>>((const __nv_bfloat16 *)dA, (const __nv_bfloat16 *)dB, K,
                                                          (float *)dC, (unsigned *)dS);
        }
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    unsigned st = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&st, dS, 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(C, dC, (size_t)128 * N * 4, cudaMemcpyDeviceToHost);
    cleanup();
    if (e != cudaSuccess) {
        cavmd_set_global_error(std::string("cavmd_tc_selftest: ") + cudaGetErrorString(e));
        return CAVMD_ERR_CUDA;
    }
    if (st) {
        cavmd_set_global_error("cavmd_tc_selftest: tensor-core wait timed out");
        return CAVMD_ERR_DEVICE_TIMEOUT;
    }
    return CAVMD_OK;
}
