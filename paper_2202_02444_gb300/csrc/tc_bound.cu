// BF16-sound RangeBound on the tensor cores (tcgen05 + TMEM + TMA).
//
// Network shape served: 3 -> H -> ... -> H -> 1 ReLU, ELU or sin MLP (H = 128,
// 256 or 512), affine-truncate with K = 16, 32, 64 or (H <= 256) 128 kept
// noise symbols (Sec. 3.3; one instantiation file per K), the
// dense layers of App. A Table "affine_update_rules" on tensor cores. One
// persistent CTA per SM runs the whole network for a tile of NB boxes with
// NB x H threads (NB = 2 for H <= 256, 1 for H = 512): thread group g (H
// threads, one per neuron) owns box g, so two boxes' SIMT work runs
// concurrently. The per-box affine state never leaves the SM:
//   * operand B of every hidden layer: the NB x K noise columns (BF16) and a
//     16-column chunk holding each box's center as a BF16 hi/lo pair, written
//     by the epilogue threads in the K-major 128-byte-swizzled layout; the
//     chunk follows the noise rows of each K slice, so one MMA of N = NB x K
//     + 16 covers both;
//   * operand A: W as BF16 hi + lo (W = W_b + W_r + rho, |rho| <= u_b^2 |W|),
//     streamed per 64-wide K slice (at H = 512 per half of its M tiles) by
//     TMA into a two-stage ring (lane 0 of the last warp issues the copies;
//     one thread per M tile issues that tile's MMAs, so no MMA issue waits on
//     a refill);
//   * D = (W_b + W_r) [X | c_hi c_lo] accumulates in TMEM (FP32);
//   * x_inf' >= |W| v is accumulated by the SIMT threads from the resident
//     W_b slice with round-up FMAs (|W| <= |W_b| / (1 - u_b));
//   * epilogue, one thread per neuron (tcgen05.ld of its TMEM row): outward
//     rounded range, the activation rule, truncation to the K largest
//     columns, and the a-priori rounding radius of every FP operation folded
//     into x_inf.
// The first layer (3 inputs) and the output layer (1 output) run on the SIMT
// cores with directed rounding. Every bounded wait that runs out writes a
// status word and the CTA leaves through its normal exit (TMEM freed).
#include "tc_bound_impl.cuh"

namespace sra {

template cudaError_t launch_tc_bound_kt<64>(int, bool, const TcParams &, const BoxSrc &, const BoundOut &, int,
                                            cudaStream_t);
extern template cudaError_t launch_tc_bound_kt<32>(int, bool, const TcParams &, const BoxSrc &, const BoundOut &,
                                                   int, cudaStream_t);
extern template cudaError_t launch_tc_bound_kt<16>(int, bool, const TcParams &, const BoxSrc &, const BoundOut &,
                                                   int, cudaStream_t);
extern template cudaError_t launch_tc_bound_kt<128>(int, bool, const TcParams &, const BoxSrc &, const BoundOut &,
                                                    int, cudaStream_t);

int tc_smem_bytes(int H) {
    return H == 512   ? tc::Layout<512, 64, tc::boxes_per_tile(512, 64)>::ALLOC
           : H == 256 ? tc::Layout<256, 64, tc::boxes_per_tile(256, 64)>::ALLOC
           : H == 128 ? tc::Layout<128, 64, tc::boxes_per_tile(128, 64)>::ALLOC
                      : 0;
}

int tc_boxes_per_tile(int H, int K) { return tc::boxes_per_tile(H, K); }

bool tc_kt_served(int K, int H) { return K == 16 || K == 32 || K == 64 || (K == 128 && H <= 256); }

cudaError_t launch_tc_bound(int H, int K, bool sound, const TcParams &p, const BoxSrc &src, const BoundOut &out,
                            int grid, cudaStream_t st) {
    if (K == 64) return launch_tc_bound_kt<64>(H, sound, p, src, out, grid, st);
    if (K == 32) return launch_tc_bound_kt<32>(H, sound, p, src, out, grid, st);
    if (K == 16) return launch_tc_bound_kt<16>(H, sound, p, src, out, grid, st);
    if (K == 128) return launch_tc_bound_kt<128>(H, sound, p, src, out, grid, st);
    return cudaErrorInvalidValue;
}

}  // namespace sra
