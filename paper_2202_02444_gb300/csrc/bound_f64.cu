// FP64 instantiations of the SIMT engine (re-check pass and FP64 option).
#include "engine_simt.cuh"
#include "launch.h"

namespace sra {

template <int KMAX>
static cudaError_t launch_bound_d(const NetDev &net, const BoxSrc &src, const BoundOut &out,
                                  const RangeCfg &cfg, long long grid, cudaStream_t st) {
    auto k = bound_kernel<double, KMAX>;
    const int smem = cfg.NB * cfg.slot_bytes;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)grid, cfg.NB * cfg.H, smem, st>>>(net, src, out, cfg);
    return cudaGetLastError();
}

cudaError_t launch_bound_f64(int kmax, const NetDev &net, const BoxSrc &src, const BoundOut &out,
                             const RangeCfg &cfg, long long grid, cudaStream_t st) {
    switch (kmax) {
    case 1: return launch_bound_d<1>(net, src, out, cfg, grid, st);
    case 4: return launch_bound_d<4>(net, src, out, cfg, grid, st);
    case 8: return launch_bound_d<8>(net, src, out, cfg, grid, st);
    case 16: return launch_bound_d<16>(net, src, out, cfg, grid, st);
    case 32: return launch_bound_d<32>(net, src, out, cfg, grid, st);
    case 64: return launch_bound_d<64>(net, src, out, cfg, grid, st);
    case 128: return launch_bound_d<128>(net, src, out, cfg, grid, st);
    default: break;
    }
    return cudaErrorInvalidValue;
}

template <int KMAX>
static cudaError_t launch_rays_d(const NetDev &net, const void *rp, const RangeCfg &cfg, int grid, cudaStream_t st) {
    auto k = ray_kernel<double, KMAX>;
    const int smem = cfg.NB * cfg.slot_bytes;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, cfg.NB * cfg.H, smem, st>>>(net, *(const RayParams *)rp, cfg);
    return cudaGetLastError();
}

template <int KMAX> static int rays_occ_d(const RangeCfg &cfg) {
    auto k = ray_kernel<double, KMAX>;
    const int smem = cfg.NB * cfg.slot_bytes;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, cfg.NB * cfg.H, smem) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

// CastRay in FP64: the FP64 option of sra_cast_rays and its re-check pass.
cudaError_t launch_rays_f64(int kmax, const NetDev &net, const void *rp, const RangeCfg &cfg, int grid,
                            cudaStream_t st) {
    switch (kmax) {
    case 1: return launch_rays_d<1>(net, rp, cfg, grid, st);
    case 4: return launch_rays_d<4>(net, rp, cfg, grid, st);
    case 8: return launch_rays_d<8>(net, rp, cfg, grid, st);
    case 16: return launch_rays_d<16>(net, rp, cfg, grid, st);
    case 32: return launch_rays_d<32>(net, rp, cfg, grid, st);
    case 64: return launch_rays_d<64>(net, rp, cfg, grid, st);
    case 128: return launch_rays_d<128>(net, rp, cfg, grid, st);
    default: break;
    }
    return cudaErrorInvalidValue;
}

int rays_blocks_per_sm_f64(int kmax, const RangeCfg &cfg) {
    switch (kmax) {
    case 1: return rays_occ_d<1>(cfg);
    case 4: return rays_occ_d<4>(cfg);
    case 8: return rays_occ_d<8>(cfg);
    case 16: return rays_occ_d<16>(cfg);
    case 32: return rays_occ_d<32>(cfg);
    case 64: return rays_occ_d<64>(cfg);
    case 128: return rays_occ_d<128>(cfg);
    default: break;
    }
    return 1;
}

}  // namespace sra
