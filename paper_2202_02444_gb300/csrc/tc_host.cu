// TMA descriptor creation through the driver entry point (no link-time
// dependency on libcuda), and the tensor-core self-test entry of the C ABI.
#include <cstring>
#include <mutex>

#include "../../include/sra.h"
#include "tc_host.h"

namespace sra {

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                 CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                 CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiled)p;
    });
    return fn;
}

}  // namespace

int make_bf16_tile_map(CUtensorMap *map, const void *base, int rows, int cols, int box_rows, int box_cols) {
    EncodeTiled fn = encode_fn();
    if (!fn) return 1;
    if (((uintptr_t)base & 15u) || ((cols * 2) & 15) || box_cols * 2 != 128) return 2;
    memset(map, 0, sizeof *map);
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : 3;
}

}  // namespace sra

extern "C" sra_status sra_selftest_tc_gemm(const void *W, const void *X, float *D, int *status, void *stream) {
    if (!W || !X || !D || !status) return SRA_EINVAL;
    const int r = sra::tc_gemm_selftest(W, X, D, status, (cudaStream_t)stream);
    return r == 0 ? SRA_OK : (r == 10 ? SRA_EUNSUPPORTED : SRA_ECUDA);
}
