// Parameters of the tensor-core CastRay kernel (BF16 hidden layers).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "sra_common.cuh"

namespace sra {

constexpr int kMaxRayTc = 8;  // hidden H -> H layers served by the tensor cores

struct TcRayParams {
    CUtensorMap wb[kMaxRayTc];  // W_b = bf16(W)                 [H][H] row-major
    CUtensorMap wr[kMaxRayTc];  // W_r = bf16(W - W_b)
    CUtensorMap wa[kMaxRayTc];  // |W_b|
    CUtensorMap ws[kMaxRayTc];  // sign(W_b) W_r, so |W_b| + sign(W_b) W_r = |W_b + W_r|
    const float *W0t;           // first layer, transposed [din][H] (FP32)
    const float *b[kMaxRayTc + 2];
    int act[kMaxRayTc + 1];     // activation after linear layer l
    const float *wout;          // output layer [H]
    float bout;
    int L, din, pe, slope;
    int *status;
    // CastRay (Proc. 2)
    const float *origins, *dirs, *f0;
    float *t_hit;
    int *iters;
    long long n;
    unsigned long long *next;
    float delta, t_max, sigma0, eta_plus, eta_minus, safety;
    long long max_iters;
};

int tc_ray_smem_bytes(int H);
int tc_ray_max_din();
cudaError_t launch_tc_rays(int H, const TcRayParams &p, int grid, cudaStream_t st);

}  // namespace sra
