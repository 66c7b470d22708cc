// Parameters of the tensor-core CastRay kernel (BF16 layers on tcgen05).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "sra_common.cuh"

namespace sra {

constexpr int kMaxRayTc = 8;  // hidden H -> H layers served by the tensor cores

// One linear layer as three BF16 matrices, row-major [H][K] (K-major tiles):
// W_b = bf16(W), W_r = bf16(W - W_b) (W_b + W_r ~ W), and |W| rounded up to
// BF16 (an upper bound of |W| for the x_inf product).
struct TcLayerMaps {
    CUtensorMap wb, wr, wa;
};

struct TcRayParams {
    TcLayerMaps first;              // layer 0, K padded to 64 with zero columns
    TcLayerMaps hidden[kMaxRayTc];  // H -> H layers
    const float *b[kMaxRayTc + 2];
    int act[kMaxRayTc + 1];  // activation after linear layer l
    const float *wout;       // output layer [H]
    float bout;
    int L, din, pe, slope;
    int *status;
    // CastRay (Proc. 2)
    const float *origins, *dirs, *f0;
    const float *t_start, *sigma_start;  // optional per-ray march state to resume from
    float *t_hit;
    int *iters;
    long long n;
    unsigned long long *next;
    float delta, t_max, sigma0, eta_plus, eta_minus, safety;
    long long max_iters;
    // optional: each ray that met a near-zero decision (near_zero_step) is
    // appended once, when it ends, to flag_list[atomicAdd(flag_count, 1)]
    int *flag_list, *flag_count;
    float band;
    // sound form (BF16 with a rounding radius): FP32 accumulation factors of
    // the |W| x_inf sums (layer 0, hidden layers), the products' rounding
    // errors per unit of |W| (|c| + |A|) times that factor, and the output
    // layer's FP32 dot-product error factor
    float kx0, kx, rhok0, rhok, gam_out;
};

int tc_ray_smem_bytes(int H, bool sound);
int tc_ray_max_din();
int tc_ray_slots();  // rays per CTA
cudaError_t launch_tc_rays(int H, bool sound, const TcRayParams &p, int grid, cudaStream_t st);

}  // namespace sra
