// The convergence test of Proc. 3 inside a classify-and-split round: an
// UNKNOWN node narrower than delta / sqrt(3) whose sample points, one per
// face (the face centres), take both signs lies within delta of the level set
// and is returned as a leaf instead of being split. The round lists those
// nodes with their six face centres, evaluates f there with the plain forward
// pass, and marks the nodes whose samples change sign; the split then emits
// marked nodes as leaves.
#include "launch.h"

namespace sra {

__global__ void conv_points_kernel(BoxSrc geo, const uint8_t *cls, long long n, float wlim, int *list, int *count,
                                   int *count6, float *pts) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (cls[i] != SRA_UNKNOWN) continue;
        float c[3], h[3];
        node_geometry<float>(geo, geo.nodes[i], c, h);
        if (!(2.f * fmaxf(h[0], fmaxf(h[1], h[2])) < wlim)) continue;
        const int k = atomicAdd(count, 1);
        atomicAdd(count6, 6);
        list[k] = (int)i;
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            const int d = f >> 1;
            float p[3] = {c[0], c[1], c[2]};
            p[d] = (f & 1) ? c[d] + h[d] : c[d] - h[d];
#pragma unroll
            for (int q = 0; q < 3; ++q) pts[((long long)k * 6 + f) * 3 + q] = p[q];
        }
    }
}

__global__ void iota_kernel(int *a, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] = (int)i;
}

__global__ void conv_mark_kernel(const int *list, const int *count, const float *vals, uint8_t *cls) {
    const int n = *count;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        bool neg = false, pos = false;
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            const float v = vals[(long long)k * 6 + f];
            neg |= v < 0.f;
            pos |= v > 0.f;
        }
        if (neg && pos) cls[list[k]] = kClsConverged;
    }
}

static unsigned grid_for(long long n) {
    long long b = (n + 255) / 256;
    if (b > 8192) b = 8192;
    return (unsigned)(b > 0 ? b : 1);
}

cudaError_t launch_conv_points(const BoxSrc &geo, const uint8_t *cls, long long n, float wlim, int *list,
                               int *count, int *count6, float *pts, cudaStream_t st) {
    conv_points_kernel<<<grid_for(n), 256, 0, st>>>(geo, cls, n, wlim, list, count, count6, pts);
    return cudaGetLastError();
}

cudaError_t launch_iota(int *a, long long n, cudaStream_t st) {
    iota_kernel<<<grid_for(n), 256, 0, st>>>(a, n);
    return cudaGetLastError();
}

cudaError_t launch_conv_mark(const int *list, const int *count, long long n_hint, const float *vals, uint8_t *cls,
                             cudaStream_t st) {
    conv_mark_kernel<<<grid_for(n_hint), 256, 0, st>>>(list, count, vals, cls);
    return cudaGetLastError();
}

}  // namespace sra
