// Device evaluation of the FP32 math functions whose errors the sound
// activation rules pad (sinf, cosf, sinpif, acosf, expm1f, expf, logf), for
// tests that measure those errors against FP64 on many arguments.
#include "launch.h"

namespace sra {

__global__ void math_f32_kernel(int fn, const float *__restrict__ x, long long n, float *__restrict__ y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float v = x[i];
        float r;
        switch (fn) {
            case 0: r = sinf(v); break;
            case 1: r = cosf(v); break;
            case 2: r = sinpif(v); break;
            case 3: r = acosf(v); break;
            case 4: r = expm1f(v); break;
            case 5: r = expf(v); break;
            default: r = logf(v); break;
        }
        y[i] = r;
    }
}

cudaError_t launch_math_f32(int fn, const float *x, long long n, float *y, cudaStream_t st) {
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    math_f32_kernel<<<(int)blocks, 256, 0, st>>>(fn, x, n, y);
    return cudaGetLastError();
}

}  // namespace sra
