// Host-side launch interface between the C-ABI layer and the kernels.
#pragma once

#include <cuda_runtime.h>

#include "sra_common.cuh"

namespace sra {

// Record an error message for sra_last_error() and return s.
sra_status set_error(sra_status s, const char *fmt, ...);

__host__ __device__ constexpr int engine_row_stride(int kmax) { return ((kmax + 3 + 3) / 4) * 4; }

// KMAX values the engine is instantiated for.
constexpr int kKmaxList[] = {1, 4, 8, 16, 32, 64, 128};

// y = f(x) for the FP32 math functions of sra_test_math_f32 (math_probe.cu).
cudaError_t launch_math_f32(int fn, const float *x, long long n, float *y, cudaStream_t st);

cudaError_t launch_bound_f32(int kmax, const NetDev &net, const BoxSrc &src, const BoundOut &out,
                             const RangeCfg &cfg, long long grid, cudaStream_t st);
cudaError_t launch_bound_f64(int kmax, const NetDev &net, const BoxSrc &src, const BoundOut &out,
                             const RangeCfg &cfg, long long grid, cudaStream_t st);

// Affine-full RangeBound past the SIMT engine's register row: one CTA per
// box, the noise matrix (rows x KS) in shared memory (full.cu).
constexpr int kFullMaxWidth = 64;
struct FullCfg {
    int rows;   // state rows: the largest layer width
    int KS;     // row stride: total symbols rounded up to 4
    int slope;  // SRA_SLOPE_*
    int x_off, w_off, smem;  // byte offsets and total dynamic shared memory
};
sra_status full_cfg(int rows, int total_syms, int slope, int tsize, FullCfg *fc);
cudaError_t launch_full_bound(bool fp64, const NetDev &net, const BoxSrc &src, const BoundOut &out,
                              const FullCfg &fc, long long n_hint, cudaStream_t st);

// Affine-full RangeBound with each box's noise matrix in device memory
// (full_hbm.cu): any width, with or without positional encoding. A pass
// takes `chunk` boxes; `bytes` of scratch hold two [rows][LD] noise matrices
// and two FP64 center vectors [rows] per box.
struct FullHbmCfg {
    int rows;        // state rows: the largest layer width
    int LD;          // row stride: 1 + symbols, rounded up to 4
    int slope;       // SRA_SLOPE_*
    int syms;        // symbols after the last nonlinearity
    long long chunk; // boxes per pass
    size_t bytes;    // scratch of one pass
};
constexpr size_t kFullHbmBudget = (size_t)1 << 30;  // scratch bytes of one pass
sra_status full_hbm_cfg(const NetDev &net, int rows, int slope, int tsize, size_t budget, FullHbmCfg *fc);
cudaError_t launch_full_hbm(bool fp64, const NetDev &net, const FullHbmCfg &fc, const BoxSrc &src,
                            const BoundOut &out, long long n_hint, void *scratch, cudaStream_t st);

struct RayParams;
cudaError_t launch_rays_f32(int kmax, const NetDev &net, const void *rp, const RangeCfg &cfg,
                            int grid, cudaStream_t st);
int rays_blocks_per_sm_f32(int kmax, const RangeCfg &cfg);
cudaError_t launch_rays_f64(int kmax, const NetDev &net, const void *rp, const RangeCfg &cfg,
                            int grid, cudaStream_t st);
int rays_blocks_per_sm_f64(int kmax, const RangeCfg &cfg);

// Frontier round (Proc. 3 split) after classification.
struct SplitArgs {
    const uint8_t *cls;
    const sra_node *in;
    long long n;
    int max_level;
    int split;                           // SRA_SPLIT_*
    unsigned char kd_axis[kMaxKdLevels]; // k-d split axis leaving each level
    sra_node *out;
    long long cap_out;
    sra_node *leaves;
    long long cap_leaves;
    unsigned long long *counts;          // device int64[SRA_CNT_N]
    long long *blk;                      // scratch: 2 * nblocks
};
cudaError_t launch_split(const SplitArgs &a, cudaStream_t st);
long long split_blocks(long long n);

// Batched round over many networks: the persistent multi-network bound
// kernel (one launch per KMAX) and the segmented split.
cudaError_t launch_multi_bound_f32(int kmax, const BatchSegDev *segs, const int *order, int nseg,
                                   long long nchunks, unsigned long long *next, int threads, int smem,
                                   cudaStream_t st);
struct BatchSplitSeg {
    long long first, n;          // nodes in[first, first + n) and their classes
    long long out_first, cap_out;
    long long leaf_first, cap_leaves;
    long long blk0;              // first split block of the segment
    int max_level, split;
    unsigned char kd_axis[kMaxKdLevels];
};
// Mesh of the zero set inside leaves (marching tetrahedra on a 2^sub grid per leaf).
struct MeshArgs {
    const sra_node *leaves;
    long long n;
    int sub;
    float lo[3], ext[3];
};
long long mesh_points(const MeshArgs &a);  // corner points of the leaves
long long mesh_blocks(const MeshArgs &a);  // scan blocks of the cells
cudaError_t launch_mesh_points(const MeshArgs &a, float *pts, cudaStream_t st);
cudaError_t launch_mesh_tris(const MeshArgs &a, const float *vals, long long *blk, unsigned long long *counter,
                             float *tris, long long cap, cudaStream_t st);

// Empty-sphere rounds over a device-side list of open points.
cudaError_t launch_sphere_init(long long n, int *list, int *count, float *radius, cudaStream_t st);
cudaError_t launch_sphere_halfw(long long n, const int *list, const int *count, float r, float *halfw,
                                cudaStream_t st);
cudaError_t launch_sphere_update(long long n, const int *list, const int *count, const uint8_t *cls, float r,
                                 float *radius, int *next_list, int *next_count, cudaStream_t st);

// Frustum ray casting: frusta over pixel rectangles of one eye.
struct Frustum {
    int x0, y0, x1, y1;  // pixels [x0, x1) x [y0, y1)
    float t, sigma;
};
struct FrustumArgs {
    const float *dirs;  // unit pixel directions [H * W][3], row-major
    int W, H;
    float eye[3];
    float sigma0, t_max, eta_plus, eta_minus, safety, delta;
};
cudaError_t launch_frustum_init(const FrustumArgs &a, int grid, Frustum *out, int *count, cudaStream_t st);
cudaError_t launch_frustum_boxes(const FrustumArgs &a, const Frustum *fr, const int *count, long long n_hint,
                                 float *centers, float *halfw, cudaStream_t st);
cudaError_t launch_frustum_update(const FrustumArgs &a, const Frustum *fr, const int *count, long long n_hint,
                                  const uint8_t *cls, Frustum *out, int *out_count, int *ray_pix, float *ray_t,
                                  float *ray_sigma, int *ray_count, int *boxes, float *t_hit, int *iters,
                                  cudaStream_t st);
cudaError_t launch_ray_gather(const FrustumArgs &a, const int *ray_pix, int n, float *origins, float *dirs,
                              cudaStream_t st);
cudaError_t launch_ray_scatter(const int *ray_pix, int n, const float *t_ray, const int *it_ray, float *t_hit,
                               int *iters, cudaStream_t st);

// Convergence test of Proc. 3 (opts->converge): class code of the nodes it
// returns as leaves, and the launches that find them.
constexpr uint8_t kClsConverged = 3;
cudaError_t launch_conv_points(const BoxSrc &geo, const uint8_t *cls, long long n, float wlim, int *list,
                               int *count, int *count6, float *pts, cudaStream_t st);
cudaError_t launch_iota(int *a, long long n, cudaStream_t st);
cudaError_t launch_conv_mark(const int *list, const int *count, long long n_hint, const float *vals, uint8_t *cls,
                             cudaStream_t st);

// counts: device int64[nseg][SRA_CNT_N]; blk: scratch 2 * nblk
cudaError_t launch_split_batch(const uint8_t *cls, const sra_node *in, const BatchSplitSeg *segs, int nseg,
                               long long nblk, sra_node *out, sra_node *leaves, unsigned long long *counts,
                               long long *blk, cudaStream_t st);

}  // namespace sra
