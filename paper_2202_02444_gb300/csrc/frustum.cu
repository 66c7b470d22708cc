// Frustum ray casting (Sec. 4.3): blocks of pixel rays from one eye march
// together. A frustum (pixel rectangle [x0,x1) x [y0,y1), march state t,
// sigma) bounds its segment [t, t + sigma] by one 3-D box and steps like
// CastRay (Proc. 2): a POSITIVE / NEGATIVE box advances t by safety * sigma
// and grows sigma by eta+, an UNKNOWN box shrinks sigma by eta-. A frustum
// splits in half across its longer pixel side when that side's width at the
// far face exceeds 2 sigma (or sigma falls below delta), and a single-pixel
// frustum is handed to the ray kernels, which resume Proc. 2 from its
// (t, sigma).
//
// The box must contain every pixel ray's points e + s d, s in [t, t + sigma].
// The unit directions d of the pixels are positive combinations of the four
// corner directions c_i (a pinhole camera maps pixels affinely before
// normalising), so d = lambda * sum w_i c_i with convex weights w_i and
// 1 <= lambda <= 1 / cos(theta), cos(theta) = min_i c_i . m for the unit mean
// direction m. Hence e + s d lies in the truncated pyramid with vertices
// e + t c_i and e + ((t + sigma) / cos(theta)) c_i, and the box of those eight
// vertices (padded outward for FP32 rounding) bounds it.
#include "launch.h"

namespace sra {

__device__ __forceinline__ void corner_dirs(const FrustumArgs &a, const Frustum &f, float c[4][3]) {
    const int xs[2] = {f.x0, f.x1 - 1}, ys[2] = {f.y0, f.y1 - 1};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const long long pix = (long long)ys[k >> 1] * a.W + xs[k & 1];
#pragma unroll
        for (int d = 0; d < 3; ++d) c[k][d] = a.dirs[pix * 3 + d];
    }
}

__global__ void frustum_init_kernel(FrustumArgs a, int grid, Frustum *out, int *count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int tw = (a.W + grid - 1) / grid, th = (a.H + grid - 1) / grid;
    const int nx = (a.W + tw - 1) / tw, ny = (a.H + th - 1) / th;
    if (i == 0) *count = nx * ny;
    if (i >= nx * ny) return;
    Frustum f;
    f.x0 = (i % nx) * tw;
    f.y0 = (i / nx) * th;
    f.x1 = min(f.x0 + tw, a.W);
    f.y1 = min(f.y0 + th, a.H);
    f.t = 0.f;
    f.sigma = a.sigma0;
    out[i] = f;
}

__global__ void frustum_box_kernel(FrustumArgs a, const Frustum *fr, const int *count, float *centers,
                                   float *halfw) {
    const int n = *count;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Frustum f = fr[i];
        float c[4][3];
        corner_dirs(a, f, c);
        float m[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int d = 0; d < 3; ++d) m[d] += c[k][d];
        const float mn = sqrtf(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
        float cosq = 1.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) cosq = fminf(cosq, (c[k][0] * m[0] + c[k][1] * m[1] + c[k][2] * m[2]) / mn);
        cosq = fmaxf(cosq * (1.f - 1e-6f), 1e-3f);  // rounded down: the far face only grows
        const float nearv = f.t, farv = (f.t + f.sigma) / cosq * (1.f + 1e-6f);
        float lo[3], hi[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) { lo[d] = INFINITY; hi[d] = -INFINITY; }
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float p0 = a.eye[d] + nearv * c[k][d], p1 = a.eye[d] + farv * c[k][d];
                lo[d] = fminf(lo[d], fminf(p0, p1));
                hi[d] = fmaxf(hi[d], fmaxf(p0, p1));
            }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float pad = 1e-6f * (fabsf(lo[d]) + fabsf(hi[d])) + 1e-7f;
            const float l = lo[d] - pad, u = hi[d] + pad;
            centers[i * 3 + d] = 0.5f * (l + u);
            halfw[i * 3 + d] = 0.5f * (u - l) * (1.f + 1e-6f) + 1e-7f;
        }
    }
}

__global__ void frustum_update_kernel(FrustumArgs a, const Frustum *fr, const int *count, const uint8_t *cls,
                                      Frustum *out, int *out_count, int *ray_pix, float *ray_t, float *ray_sigma,
                                      int *ray_count, int *boxes, float *t_hit, int *iters) {
    const int n = *count;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(boxes, n);  // frustum boxes bounded this round
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        Frustum f = fr[i];
        if (cls[i] != SRA_UNKNOWN) {
            f.t += a.safety * f.sigma;
            f.sigma *= a.eta_plus;
        } else {
            f.sigma *= a.eta_minus;
        }
        if (!(f.t < a.t_max)) {  // every ray of the frustum leaves the domain: NO_HIT
            for (int y = f.y0; y < f.y1; ++y)
                for (int x = f.x0; x < f.x1; ++x) {
                    t_hit[(long long)y * a.W + x] = INFINITY;
                    if (iters) iters[(long long)y * a.W + x] = 0;
                }
            continue;
        }
        const int w = f.x1 - f.x0, h = f.y1 - f.y0;
        if (w == 1 && h == 1) {
            const int k = atomicAdd(ray_count, 1);
            ray_pix[k] = f.y0 * a.W + f.x0;
            ray_t[k] = f.t;
            ray_sigma[k] = f.sigma;
            continue;
        }
        // width of the longer pixel side at the far face
        float c[4][3];
        corner_dirs(a, f, c);
        const int j = (w >= h) ? 1 : 2;  // corner across the longer side from corner 0
        const float dx = c[j][0] - c[0][0], dy = c[j][1] - c[0][1], dz = c[j][2] - c[0][2];
        const float width = (f.t + f.sigma) * sqrtf(dx * dx + dy * dy + dz * dz);
        // below the tolerance delta the frustum splits regardless (Proc. 2's
        // single rays take over there; also ends the shrinking at t = 0)
        if (width > 2.f * f.sigma || f.sigma < a.delta) {
            Frustum g = f, q = f;
            if (w >= h) { g.x1 = f.x0 + w / 2; q.x0 = g.x1; }
            else { g.y1 = f.y0 + h / 2; q.y0 = g.y1; }
            const int k = atomicAdd(out_count, 2);
            out[k] = g;
            out[k + 1] = q;
        } else {
            out[atomicAdd(out_count, 1)] = f;
        }
    }
}

__global__ void ray_gather_kernel(FrustumArgs a, const int *ray_pix, int n, float *origins, float *dirs) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const long long p = ray_pix[k];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        origins[k * 3 + d] = a.eye[d];
        dirs[k * 3 + d] = a.dirs[p * 3 + d];
    }
}

__global__ void ray_scatter_kernel(const int *ray_pix, int n, const float *t_ray, const int *it_ray, float *t_hit,
                                   int *iters) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    t_hit[ray_pix[k]] = t_ray[k];
    if (iters) iters[ray_pix[k]] = it_ray[k];
}

static unsigned blocks_for(long long n) {
    long long b = (n + 255) / 256;
    if (b > 8192) b = 8192;
    return (unsigned)(b > 0 ? b : 1);
}

cudaError_t launch_frustum_init(const FrustumArgs &a, int grid, Frustum *out, int *count, cudaStream_t st) {
    frustum_init_kernel<<<(unsigned)((grid * grid + 255) / 256), 256, 0, st>>>(a, grid, out, count);
    return cudaGetLastError();
}

cudaError_t launch_frustum_boxes(const FrustumArgs &a, const Frustum *fr, const int *count, long long n_hint,
                                 float *centers, float *halfw, cudaStream_t st) {
    frustum_box_kernel<<<blocks_for(n_hint), 256, 0, st>>>(a, fr, count, centers, halfw);
    return cudaGetLastError();
}

cudaError_t launch_frustum_update(const FrustumArgs &a, const Frustum *fr, const int *count, long long n_hint,
                                  const uint8_t *cls, Frustum *out, int *out_count, int *ray_pix, float *ray_t,
                                  float *ray_sigma, int *ray_count, int *boxes, float *t_hit, int *iters,
                                  cudaStream_t st) {
    frustum_update_kernel<<<blocks_for(n_hint), 256, 0, st>>>(a, fr, count, cls, out, out_count, ray_pix, ray_t,
                                                                ray_sigma, ray_count, boxes, t_hit, iters);
    return cudaGetLastError();
}

cudaError_t launch_ray_gather(const FrustumArgs &a, const int *ray_pix, int n, float *origins, float *dirs,
                              cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    ray_gather_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, ray_pix, n, origins, dirs);
    return cudaGetLastError();
}

cudaError_t launch_ray_scatter(const int *ray_pix, int n, const float *t_ray, const int *it_ray, float *t_hit,
                               int *iters, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    ray_scatter_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ray_pix, n, t_ray, it_ray, t_hit, iters);
    return cudaGetLastError();
}

}  // namespace sra
