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

}  // namespace sra
