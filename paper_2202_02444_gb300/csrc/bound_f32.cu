// FP32 instantiations of the SIMT engine (plain single-precision form).
#include "engine_simt.cuh"
#include "launch.h"

namespace sra {

template <typename T, int KMAX>
static cudaError_t launch_bound_t(const NetDev &net, const BoxSrc &src, const BoundOut &out,
                                  const RangeCfg &cfg, long long grid, cudaStream_t st) {
    auto k = bound_kernel<T, KMAX>;
    const int smem = cfg.NB * cfg.slot_bytes;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)grid, cfg.NB * cfg.H, smem, st>>>(net, src, out, cfg);
    return cudaGetLastError();
}

template <typename T, int KMAX>
static cudaError_t launch_rays_t(const NetDev &net, const void *rp, const RangeCfg &cfg, int grid,
                                 cudaStream_t st) {
    auto k = ray_kernel<T, KMAX>;
    const int smem = cfg.NB * cfg.slot_bytes;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, cfg.NB * cfg.H, smem, st>>>(net, *(const RayParams *)rp, cfg);
    return cudaGetLastError();
}

template <typename T, int KMAX> static int rays_occ(const RangeCfg &cfg) {
    auto k = ray_kernel<T, KMAX>;
    const int smem = cfg.NB * cfg.slot_bytes;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, cfg.NB * cfg.H, smem) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

#define SRA_KMAX_SWITCH(F, ...)                              \
    switch (kmax) {                                          \
    case 1: return F<float, 1>(__VA_ARGS__);                 \
    case 4: return F<float, 4>(__VA_ARGS__);                 \
    case 8: return F<float, 8>(__VA_ARGS__);                 \
    case 16: return F<float, 16>(__VA_ARGS__);               \
    case 32: return F<float, 32>(__VA_ARGS__);               \
    case 64: return F<float, 64>(__VA_ARGS__);               \
    case 128: return F<float, 128>(__VA_ARGS__);             \
    default: break;                                          \
    }

cudaError_t launch_bound_f32(int kmax, const NetDev &net, const BoxSrc &src, const BoundOut &out,
                             const RangeCfg &cfg, long long grid, cudaStream_t st) {
    SRA_KMAX_SWITCH(launch_bound_t, net, src, out, cfg, grid, st)
    return cudaErrorInvalidValue;
}

cudaError_t launch_rays_f32(int kmax, const NetDev &net, const void *rp, const RangeCfg &cfg, int grid,
                            cudaStream_t st) {
    SRA_KMAX_SWITCH(launch_rays_t, net, rp, cfg, grid, st)
    return cudaErrorInvalidValue;
}

template <typename T, int KMAX>
static cudaError_t launch_multi_t(const BatchSegDev *segs, const int *order, int nseg, long long nchunks,
                                  unsigned long long *next, int threads, int smem, cudaStream_t st) {
    auto k = multi_bound_kernel<T, KMAX>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem)) != cudaSuccess) return e;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long grid = (long long)(per_sm > 0 ? per_sm : 1) * sms;
    if (grid > nchunks) grid = nchunks;
    if (grid < 1) return cudaSuccess;
    k<<<(unsigned)grid, threads, smem, st>>>(segs, order, nseg, nchunks, next);
    return cudaGetLastError();
}

cudaError_t launch_multi_bound_f32(int kmax, const BatchSegDev *segs, const int *order, int nseg,
                                   long long nchunks, unsigned long long *next, int threads, int smem,
                                   cudaStream_t st) {
    SRA_KMAX_SWITCH(launch_multi_t, segs, order, nseg, nchunks, next, threads, smem, st)
    return cudaErrorInvalidValue;
}

int rays_blocks_per_sm_f32(int kmax, const RangeCfg &cfg) {
    SRA_KMAX_SWITCH(rays_occ, cfg)
    return 1;
}

}  // namespace sra
