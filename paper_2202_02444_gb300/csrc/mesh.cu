// Mesh of the zero level set inside octree leaves: the dense bottom levels of
// hierarchical mesh extraction (Sec. 4.7). Each leaf is split into 2^s cells
// per axis; f is evaluated at the cell corners; every cell is cut into the six
// Kuhn tetrahedra along its main diagonal (vertex bits x = 1, y = 2, z = 4,
// paths 0 -> e_a -> e_a + e_b -> 7 over the six axis orders), and each
// tetrahedron is meshed on its own: one triangle when one corner differs in
// sign from the other three, two when two and two differ.
//
// The Kuhn split is the same in every cell, so neighbouring cells cut their
// shared faces along the same diagonals, and a crossing on a grid edge is
// interpolated from the endpoint with the lower grid index to the higher
// one. Leaves of one level therefore give a closed, crack-free surface: a
// shared edge gets bit-identical vertices from both sides. Corner positions
// come from the global grid index (exact for dyadic roots), so points that
// two leaves share are evaluated identically. Triangles face the side where
// f >= 0 (the side DifferentSigns calls positive).
//
// Output order is deterministic: leaf, cell (x fastest), tetrahedron, then
// triangle, through a count / scan / emit pass like the frontier split.
#include "launch.h"

namespace sra {

constexpr int kMeshBlock = 256;

__device__ __forceinline__ void mesh_corner(const MeshArgs &a, const sra_node &nd, int ca, int cb, int cc,
                                            float *p) {
    const int n = (int)nd.level + a.sub;  // global grid resolution 2^n per axis
    const long long g[3] = {((long long)nd.ix << a.sub) + ca, ((long long)nd.iy << a.sub) + cb,
                            ((long long)nd.iz << a.sub) + cc};
#pragma unroll
    for (int d = 0; d < 3; ++d) p[d] = a.lo[d] + ldexpf(a.ext[d], -n) * (float)g[d];
}

// Corner grid of every leaf of the chunk: (2^s + 1)^3 points per leaf.
__global__ void mesh_points_kernel(MeshArgs a, float *pts) {
    const int G = (1 << a.sub) + 1;
    const long long per = (long long)G * G * G;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n * per) return;
    const long long leaf = i / per;
    const int r = (int)(i - leaf * per);
    const int ca = r % G, cb = (r / G) % G, cc = r / (G * G);
    mesh_corner(a, a.leaves[leaf], ca, cb, cc, pts + i * 3);
}

// The six Kuhn tetrahedra: cube-corner bits of each path 0 -> v1 -> v2 -> 7
// and the axis of each step.
__constant__ unsigned char kKuhnV[6][4] = {{0, 1, 3, 7}, {0, 1, 5, 7}, {0, 2, 3, 7},
                                           {0, 2, 6, 7}, {0, 4, 5, 7}, {0, 4, 6, 7}};
__constant__ unsigned char kKuhnAxis[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2},
                                              {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

__device__ __forceinline__ int tet_triangles(const float *f, int t) {
    int neg = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) neg += f[kKuhnV[t][k]] < 0.f;
    return (neg == 1 || neg == 3) ? 1 : (neg == 2 ? 2 : 0);
}

struct CellView {
    float f[8];
    long long gid[8];  // global grid index (for the canonical edge direction)
    float p[8][3];
};

__device__ __forceinline__ void load_cell(const MeshArgs &a, const float *vals, long long cube, CellView &c) {
    const int S = 1 << a.sub, G = S + 1;
    const long long per_leaf = (long long)S * S * S;
    const long long leaf = cube / per_leaf;
    const int r = (int)(cube - leaf * per_leaf);
    const int x = r % S, y = (r / S) % S, z = r / (S * S);
    const sra_node nd = a.leaves[leaf];
    const int n = (int)nd.level + a.sub;
    const long long R = 1ll << n;
    const float *v = vals + leaf * (long long)G * G * G;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int dx = k & 1, dy = (k >> 1) & 1, dz = (k >> 2) & 1;
        c.f[k] = v[((long long)(z + dz) * G + (y + dy)) * G + (x + dx)];
        mesh_corner(a, nd, x + dx, y + dy, z + dz, c.p[k]);
        const long long gx = ((long long)nd.ix << a.sub) + x + dx, gy = ((long long)nd.iy << a.sub) + y + dy,
                        gz = ((long long)nd.iz << a.sub) + z + dz;
        c.gid[k] = (gz * (R + 1) + gy) * (R + 1) + gx;
    }
}

__device__ __forceinline__ void edge_point(const CellView &c, int u, int w, float *out) {
    if (c.gid[u] > c.gid[w]) { const int t = u; u = w; w = t; }  // lower grid index first
    const float t = c.f[u] / (c.f[u] - c.f[w]);
#pragma unroll
    for (int d = 0; d < 3; ++d) out[d] = c.p[u][d] + t * (c.p[w][d] - c.p[u][d]);
}

__device__ __forceinline__ void put_tri(float *dst, const float *v0, const float *v1, const float *v2,
                                        const float *grad) {
    float e1[3], e2[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) { e1[d] = v1[d] - v0[d]; e2[d] = v2[d] - v0[d]; }
    const float nx = e1[1] * e2[2] - e1[2] * e2[1], ny = e1[2] * e2[0] - e1[0] * e2[2],
                nz = e1[0] * e2[1] - e1[1] * e2[0];
    const bool flip = nx * grad[0] + ny * grad[1] + nz * grad[2] < 0.f;
    const float *b = flip ? v2 : v1, *cc = flip ? v1 : v2;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        dst[d] = v0[d];
        dst[3 + d] = b[d];
        dst[6 + d] = cc[d];
    }
}

__device__ __forceinline__ int cube_triangles(const MeshArgs &a, const float *vals, long long cube) {
    CellView c;
    load_cell(a, vals, cube, c);
    int n = 0;
#pragma unroll
    for (int t = 0; t < 6; ++t) n += tet_triangles(c.f, t);
    return n;
}

__device__ __forceinline__ int block_excl_scan(int v, int &total) {
    __shared__ int ws[32];
    __shared__ int tot;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        ws[lane] = s;
        if (lane == 31) tot = s;
    }
    __syncthreads();
    const int ex = x - v + (w > 0 ? ws[w - 1] : 0);
    total = tot;
    __syncthreads();
    return ex;
}

__global__ void __launch_bounds__(kMeshBlock) mesh_count_kernel(MeshArgs a, const float *vals, long long ncube,
                                                                long long *blk) {
    const long long cube = (long long)blockIdx.x * kMeshBlock + threadIdx.x;
    const int k = cube < ncube ? cube_triangles(a, vals, cube) : 0;
    int total;
    block_excl_scan(k, total);
    if (threadIdx.x == 0) blk[blockIdx.x] = total;
}

// One block: exclusive scan of the block totals after the triangles already
// written (counter[0]); advances the counter.
__global__ void __launch_bounds__(kMeshBlock) mesh_scan_kernel(long long *blk, long long nblk,
                                                               unsigned long long *counter) {
    __shared__ long long carry;
    __shared__ long long ws[32];
    if (threadIdx.x == 0) carry = (long long)counter[0];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (long long b0 = 0; b0 < nblk; b0 += kMeshBlock) {
        const long long b = b0 + threadIdx.x;
        const long long x = b < nblk ? blk[b] : 0;
        long long ix = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, ix, o);
            if (lane >= o) ix += y;
        }
        if (lane == 31) ws[w] = ix;
        __syncthreads();
        if (w == 0) {
            long long s = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            ws[lane] = s;
        }
        __syncthreads();
        const long long ex = carry + (w > 0 ? ws[w - 1] : 0) + ix - x;
        if (b < nblk) blk[b] = ex;
        __syncthreads();
        if (threadIdx.x == kMeshBlock - 1) carry = ex + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) counter[0] = (unsigned long long)carry;
}

__global__ void __launch_bounds__(kMeshBlock) mesh_emit_kernel(MeshArgs a, const float *vals, long long ncube,
                                                               const long long *blk, float *tris, long long cap) {
    const long long cube = (long long)blockIdx.x * kMeshBlock + threadIdx.x;
    CellView c;
    int k = 0;
    if (cube < ncube) {
        load_cell(a, vals, cube, c);
#pragma unroll
        for (int t = 0; t < 6; ++t) k += tet_triangles(c.f, t);
    }
    int total;
    const int ex = block_excl_scan(k, total);
    if (cube >= ncube || k == 0) return;
    long long pos = blk[blockIdx.x] + ex;
    const float h[3] = {c.p[7][0] - c.p[0][0], c.p[7][1] - c.p[0][1], c.p[7][2] - c.p[0][2]};
    for (int t = 0; t < 6; ++t) {
        const unsigned char *v = kKuhnV[t];
        int neg = 0;
        for (int q = 0; q < 4; ++q) neg += c.f[v[q]] < 0.f;
        if (neg == 0 || neg == 4) continue;
        // gradient of the tetrahedron's linear interpolant: one axis per path step
        float grad[3];
        for (int q = 0; q < 3; ++q) grad[kKuhnAxis[t][q]] = (c.f[v[q + 1]] - c.f[v[q]]) / h[kKuhnAxis[t][q]];
        if (neg == 1 || neg == 3) {
            const bool lone_neg = neg == 1;
            int lone = 0;
            for (int q = 0; q < 4; ++q)
                if ((c.f[v[q]] < 0.f) == lone_neg) lone = q;
            float e[3][3];
            int m = 0;
            for (int q = 0; q < 4; ++q)
                if (q != lone) edge_point(c, v[lone], v[q], e[m++]);
            if (pos < cap) put_tri(tris + pos * 9, e[0], e[1], e[2], grad);
            ++pos;
        } else {
            int ng[2], ps[2], a0 = 0, b0 = 0;
            for (int q = 0; q < 4; ++q) {
                if (c.f[v[q]] < 0.f) ng[a0++] = v[q];
                else ps[b0++] = v[q];
            }
            float e[4][3];  // cycle: (n0,p0) (n0,p1) (n1,p1) (n1,p0)
            edge_point(c, ng[0], ps[0], e[0]);
            edge_point(c, ng[0], ps[1], e[1]);
            edge_point(c, ng[1], ps[1], e[2]);
            edge_point(c, ng[1], ps[0], e[3]);
            if (pos < cap) put_tri(tris + pos * 9, e[0], e[1], e[2], grad);
            ++pos;
            if (pos < cap) put_tri(tris + pos * 9, e[0], e[2], e[3], grad);
            ++pos;
        }
    }
}

long long mesh_points(const MeshArgs &a) {
    const long long G = (1 << a.sub) + 1;
    return a.n * G * G * G;
}

cudaError_t launch_mesh_points(const MeshArgs &a, float *pts, cudaStream_t st) {
    const long long np = mesh_points(a);
    if (np == 0) return cudaSuccess;
    mesh_points_kernel<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(a, pts);
    return cudaGetLastError();
}

long long mesh_blocks(const MeshArgs &a) {
    const long long S = 1 << a.sub;
    return (a.n * S * S * S + kMeshBlock - 1) / kMeshBlock;
}

cudaError_t launch_mesh_tris(const MeshArgs &a, const float *vals, long long *blk, unsigned long long *counter,
                             float *tris, long long cap, cudaStream_t st) {
    const long long S = 1 << a.sub, ncube = a.n * S * S * S, nblk = mesh_blocks(a);
    if (nblk == 0) return cudaSuccess;
    mesh_count_kernel<<<(unsigned)nblk, kMeshBlock, 0, st>>>(a, vals, ncube, blk);
    mesh_scan_kernel<<<1, kMeshBlock, 0, st>>>(blk, nblk, counter);
    mesh_emit_kernel<<<(unsigned)nblk, kMeshBlock, 0, st>>>(a, vals, ncube, blk, tris, cap);
    return cudaGetLastError();
}

}  // namespace sra
