// Parameters of the BF16-sound tensor-core bound kernel.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "sra_common.cuh"

namespace sra {

constexpr int kMaxTcLayers = 12;  // hidden H -> H layers served by the tensor cores

struct TcParams {
    CUtensorMap wb[kMaxTcLayers];  // W_b = bf16(W), row-major [H][H]
    CUtensorMap wr[kMaxTcLayers];  // W_r = bf16(W - W_b)
    const float *W0;               // first layer, row-major [H][3]
    const float *b[kMaxTcLayers + 2];
    const float *wout;             // output layer [H]
    float bout;
    int L;                         // linear layers
    int *status;                   // device status word (non-zero: a bounded wait ran out)
    float rho1;    // relative error of the BF16 products per unit of |W| (|x| + |c|)
    float kappa;   // |W| <= kappa |W_b|
    float ub2u;    // bf16 + fp32 rounding of the scaled noise entries
    float gam_out, gam_c_out;  // FP32 dot-product error factors of the output layer
    int test_stall;  // 0; > 0 (tests only): no weight copies and this many spins per bounded wait
    int act;         // SRA_ACT_RELU, SRA_ACT_ELU or SRA_ACT_SIN: the rule of every hidden layer (selects the instantiation)
};

int tc_smem_bytes(int H);
int tc_boxes_per_tile(int H, int K);  // boxes one CTA bounds at a time
bool tc_kt_served(int K, int H);      // kept-symbol counts with a kernel: 16, 32, 64; 128 for H <= 256
// K kept noise symbols (16, 32, 64, or 128 for H <= 256), width H (128, 256 or 512)
cudaError_t launch_tc_bound(int H, int K, bool sound, const TcParams &p, const BoxSrc &src, const BoundOut &out,
                            int grid, cudaStream_t st);
template <int KT>
cudaError_t launch_tc_bound_kt(int H, bool sound, const TcParams &p, const BoxSrc &src, const BoundOut &out,
                               int grid, cudaStream_t st);

}  // namespace sra
