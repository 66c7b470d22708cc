// Self-test of the tensor-core building blocks used by the BF16-sound bound
// kernel: a 256 x 144 x 256 BF16 GEMM D = W X^T with W loaded by TMA into
// 128-byte-swizzled K-major tiles, X written by threads into the same layout
// (as the bound kernel's epilogue writes its operands), tcgen05.mma into TMEM
// for an N=128 and an N=16 tile, and tcgen05.ld back to registers.
#include <cuda_bf16.h>

#include <cstring>

#include "tc_ptx.cuh"
#include "tc_host.h"

namespace sra {

namespace {

constexpr int kM = 256, kK = 256, kNA = 128, kNC = 16;
constexpr uint32_t kSpin = 1u << 24;

__global__ void __launch_bounds__(256) tc_gemm_selftest_kernel(const __grid_constant__ CUtensorMap wmap,
                                                              const __nv_bfloat16 *X, float *D,
                                                              int *status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *Ws = smem;                  // 2 M-tiles x 4 K-slices x 16 KB
    unsigned char *XA = smem + 131072;         // 4 K-slices x (128 rows x 128 B)
    unsigned char *XC = XA + 65536;            // 4 K-slices x (16 rows x 128 B)
    uint64_t *bars = (uint64_t *)(XC + 8192);  // [0] full, [1] acc
    uint32_t *tmem_slot = (uint32_t *)(bars + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        ptx::mbar_init(&bars[0], 1);
        ptx::mbar_init(&bars[1], 1);
        ptx::fence_mbar_init();
    }
    if (warp == 0) ptx::tmem_alloc(tmem_slot, 512);
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (tid == 0) {
        ptx::mbar_arrive_expect_tx(&bars[0], 2 * 4 * 16384);
        for (int m = 0; m < 2; ++m)
            for (int s = 0; s < 4; ++s)
                ptx::tma_load_2d(Ws + (m * 4 + s) * 16384, &wmap, s * 64, m * 128, &bars[0]);
    }
    // thread-written B operands (K-major, swizzled)
    for (int e = tid; e < (kNA + kNC) * kK; e += 256) {
        const int n = e / kK, k = e % kK;
        const __nv_bfloat16 v = X[n * kK + k];
        const int s = k >> 6;
        if (n < kNA) *(__nv_bfloat16 *)(XA + s * 16384 + ptx::sw128_offset(n, k & 63)) = v;
        else *(__nv_bfloat16 *)(XC + s * 2048 + ptx::sw128_offset(n - kNA, k & 63)) = v;
    }
    ptx::fence_proxy_async();
    __syncthreads();

    bool ok = ptx::mbar_wait(&bars[0], 0, kSpin);
    if (!ok && lane == 0) atomicExch(status, 1);
    if (tid == 0 && ok) {
        ptx::tc_fence_after();
        const uint32_t ia = ptx::idesc_bf16(128, kNA), ic = ptx::idesc_bf16(128, kNC);
        for (int s = 0; s < 4; ++s)
            for (int ks = 0; ks < 4; ++ks) {
                const uint32_t acc = (s | ks) ? 1u : 0u;
                const uint64_t bA = ptx::desc_kmajor_sw128(ptx::smem_u32(XA + s * 16384)) + (uint64_t)(2 * ks);
                const uint64_t bC = ptx::desc_kmajor_sw128(ptx::smem_u32(XC + s * 2048)) + (uint64_t)(2 * ks);
                for (int m = 0; m < 2; ++m) {
                    const uint64_t a =
                        ptx::desc_kmajor_sw128(ptx::smem_u32(Ws + (m * 4 + s) * 16384)) + (uint64_t)(2 * ks);
                    ptx::mma_bf16(tmem + m * 128, a, bA, ia, acc);
                    ptx::mma_bf16(tmem + 256 + m * 16, a, bC, ic, acc);
                }
            }
        ptx::mma_commit(&bars[1]);
    }
    __syncthreads();
    ok = ok && ptx::mbar_wait(&bars[1], 0, kSpin);
    if (!ok && lane == 0) atomicExch(status, 2);
    ptx::tc_fence_after();
    if (ok) {
        const int m = warp >> 2, q = warp & 3;
        const int row = m * 128 + q * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
        for (int c0 = 0; c0 < kNA; c0 += 16) {
            float v[16];
            ptx::tmem_ld16(tl + m * 128 + c0, v);
            ptx::tmem_wait_ld();
            for (int k = 0; k < 16; ++k) D[row * (kNA + kNC) + c0 + k] = v[k];
        }
        float v[16];
        ptx::tmem_ld16(tl + 256 + m * 16, v);
        ptx::tmem_wait_ld();
        for (int k = 0; k < 16; ++k) D[row * (kNA + kNC) + kNA + k] = v[k];
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 0) ptx::tmem_dealloc(tmem, 512);
}

}  // namespace

// W: device bf16 [256][256] row-major; X: device bf16 [144][256]; D: device
// float [256][144]. Returns 0, or a CUDA / encode / timeout code.
int tc_gemm_selftest(const void *W, const void *X, float *D, int *status, cudaStream_t st) {
    CUtensorMap map;
    if (make_bf16_tile_map(&map, W, kM, kK, 128, 64) != 0) return 10;
    const int smem = 131072 + 65536 + 8192 + 64 + 1024;
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return 11;
    tc_gemm_selftest_kernel<<<1, 256, smem, st>>>(map, (const __nv_bfloat16 *)X, D, status);
    return cudaGetLastError() == cudaSuccess ? 0 : 12;
}

}  // namespace sra
