// tc_probe.cu -- test-only check of the tensor-core operand layouts used by the BF16
// network kernel: one 128 x 208 x 32 tcgen05 MMA from shared memory (A written by
// threads, B by a bulk copy), tensor-memory loads, and a 2-D TMA box load with
// out-of-bounds zero fill.  Every shared-memory access stays inside a 192 KiB
// allocation even if a descriptor field were read with another meaning, and every wait
// is bounded.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../paper_1709_05418_gb300/csrc/tc_ptx.cuh"

using namespace rpnn::tc;

namespace {

constexpr int M = 128, N = 208, KK = 32;
constexpr uint32_t A_OFF = 0, B_OFF = 8192, T_OFF = 24576, BAR_OFF = 65536, SLOT_OFF = 65600;
constexpr int SMEM = 192 * 1024;

__global__ void __launch_bounds__(128) k_probe(const __nv_bfloat16* __restrict__ A,
                                               const __nv_bfloat16* __restrict__ Bimg,
                                               const __grid_constant__ CUtensorMap tmap,
                                               float* __restrict__ D, uint4* __restrict__ tma_out,
                                               int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const uint32_t base = smem_u32(sm);
    const uint32_t bar = base + BAR_OFF, bar_mma = base + BAR_OFF + 8;
    if (tid == 0) {
        abort_flag = 0;
        mbar_init(bar, 1);
        mbar_init(bar_mma, 1);
        fence_mbar_init();
    }
    // A: row r, col c at (c/8)*2048 + r*16 + (c%8)*2
    for (int i = tid; i < M * KK; i += 128) {
        const int r = i / KK, c = i % KK;
        *reinterpret_cast<__nv_bfloat16*>(sm + A_OFF + (c / 8) * 2048 + r * 16 + (c % 8) * 2) = A[i];
    }
    fence_proxy_async_smem();
    if (warp == 0) tmem_alloc(base + SLOT_OFF, 256);
    if (warp == 0) tmem_relinquish();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(sm + SLOT_OFF);
    if (tid == 0) {
        mbar_expect_tx(bar, 4 * 3328 + 2 * 2048);
        bulk_g2s(base + B_OFF, Bimg, 4 * 3328, bar);
        tma_load_2d(base + T_OFF, &tmap, 16, 0, bar);
        tma_load_2d(base + T_OFF + 2048, &tmap, 8, 64, bar);
        if (!mbar_wait(bar, 0, &abort_flag)) { atomicOr(err, 1); }
        else {
            tc_fence_after();
            const uint32_t id = idesc_bf16(M, N);
            for (int j = 0; j < 2; ++j) {
                const uint64_t a = smem_desc(base + A_OFF + 2 * j * 2048, 2048, 128);
                const uint64_t b = smem_desc(base + B_OFF + 2 * j * 3328, 3328, 128);
                mma_bf16(tmem, a, b, id, j > 0);
            }
            mma_commit(bar_mma);
        }
    }
    __syncwarp();
    if (!mbar_wait(bar_mma, 0, &abort_flag)) atomicOr(err, 2);
    tc_fence_after();
    if (!abort_flag) {
        const uint32_t lane_base = (uint32_t)(32 * (warp % 4)) << 16;
        for (int c = 0; c < N; c += 16) {
            float v[16];
            tmem_ld16(tmem + lane_base + c, v);
            const int row = 32 * (warp % 4) + lane;
            for (int i = 0; i < 16; ++i) D[row * N + c + i] = v[i];
        }
        for (int i = tid; i < 256; i += 128) tma_out[i] = reinterpret_cast<const uint4*>(sm + T_OFF)[i];
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 256);
}

}  // namespace

extern "C" int tc_probe(const void* A, const void* Bimg, const void* T2d, int t_rows, int t_cols,
                        float* D, void* tma_out, int* err) {
    typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess || !fn)
        return -10;
    CUtensorMap tmap;
    const cuuint64_t dims[2] = {(cuuint64_t)t_cols, (cuuint64_t)t_rows};
    const cuuint64_t strides[1] = {(cuuint64_t)t_cols * 2};
    const cuuint32_t box[2] = {8, 128};
    const cuuint32_t es[2] = {1, 1};
    CUresult r = ((EncodeFn)fn)(&tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(T2d), dims, strides,
                                box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return -11;
    if (cudaFuncSetAttribute(k_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM) != cudaSuccess) return -12;
    k_probe<<<1, 128, SMEM>>>((const __nv_bfloat16*)A, (const __nv_bfloat16*)Bimg, tmap, D, (uint4*)tma_out, err);
    if (cudaGetLastError() != cudaSuccess) return -13;
    if (cudaDeviceSynchronize() != cudaSuccess) return -14;
    return 0;
}
