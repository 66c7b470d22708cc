// Empty-sphere queries (Sec. 4.4): shrink a box around each query point until
// range analysis (Proc. 1) proves it POSITIVE or NEGATIVE. Rounds run over a
// device-side list of the points still open, so the whole query is a fixed
// sequence of launches with no host synchronisation: per round, write the
// round's half-width for the open points, bound their boxes (the list-driven
// bound kernel), then record the radius of the decided points and append the
// others to the next round's list.
#include "launch.h"

namespace sra {

__global__ void sphere_init_kernel(long long n, int *list, int *count, float *radius) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *count = (int)n;
    if (i < n) {
        list[i] = (int)i;
        radius[i] = 0.f;
    }
}

__global__ void sphere_halfw_kernel(const int *list, const int *count, float r, float *halfw) {
    const int n = *count;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n; b += gridDim.x * blockDim.x) {
        const int g = list[b];
        halfw[3 * (long long)g] = r;
        halfw[3 * (long long)g + 1] = r;
        halfw[3 * (long long)g + 2] = r;
    }
}

__global__ void sphere_update_kernel(const int *list, const int *count, const uint8_t *cls, float r, float *radius,
                                     int *next_list, int *next_count) {
    const int n = *count;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n; b += gridDim.x * blockDim.x) {
        const int g = list[b];
        if (cls[g] != SRA_UNKNOWN) radius[g] = r;
        else next_list[atomicAdd(next_count, 1)] = g;
    }
}

cudaError_t launch_sphere_init(long long n, int *list, int *count, float *radius, cudaStream_t st) {
    sphere_init_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, list, count, radius);
    return cudaGetLastError();
}

cudaError_t launch_sphere_halfw(long long n, const int *list, const int *count, float r, float *halfw,
                                cudaStream_t st) {
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    sphere_halfw_kernel<<<(unsigned)blocks, 256, 0, st>>>(list, count, r, halfw);
    return cudaGetLastError();
}

cudaError_t launch_sphere_update(long long n, const int *list, const int *count, const uint8_t *cls, float r,
                                 float *radius, int *next_list, int *next_count, cudaStream_t st) {
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    sphere_update_kernel<<<(unsigned)blocks, 256, 0, st>>>(list, count, cls, r, radius, next_list, next_count);
    return cudaGetLastError();
}

}  // namespace sra
