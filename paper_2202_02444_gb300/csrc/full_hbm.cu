// Affine-full RangeBound with the noise matrix in device memory (Sec. 3.3,
// "full": every new symbol is kept, so a box's noise matrix gains one column
// per neuron of every nonlinear layer). This is the path for networks whose
// matrix does not fit the shared memory of one CTA: any width up to 512,
// with or without positional encoding. The 3-[256]x8-1 network reaches
// 3 + 8 * 256 = 2051 symbols, 2.1 MB per box in FP32.
//
// A pass takes a chunk of boxes. Box b's state is a row-major matrix
// [rows][LD] in one of two device buffers, columns 1..S holding the S noise
// symbols, and its center, a vector [rows] in FP64 whatever the precision of
// the noise (the center cancels: after a sin layer with large
// pre-activations, for one, a c + b is much smaller than its terms). Per
// linear layer (App. A Table "affine_update_rules"):
//   * full_gemm_kernel: Y = W X for every box of the chunk (one batched GEMM,
//     128 x 128 output tiles, 8 x 8 per thread, K staged through two
//     shared-memory buffers in slices of 8);
//   * full_center_kernel: the center W c + b in FP64 from the FP64 copy of
//     the weights;
//   * full_act_kernel, one warp per row: the range (Eq. def_range: the sum of
//     the row's |noise| entries; x_inf stays zero under "full"), the rule of
//     App. A Table "affine_nonlinearities" (in FP64), the row scaled by its
//     slope, and the row of the new diagonal block (its magnitude gamma on
//     the diagonal, zeros elsewhere) appended after the old symbols.
// The output layer (one row) and Proc. 1's classification run in
// full_out_kernel, one CTA per box. Boxes of a device-side list (the FP64
// re-check) past the list's length are skipped by every kernel.
#include "engine_simt.cuh"
#include "launch.h"

namespace sra {

namespace {

template <typename T> const T *Wt_host(const LayerDev &L);
template <> const float *Wt_host<float>(const LayerDev &L) { return L.Wt; }
template <> const double *Wt_host<double>(const LayerDev &L) { return L.Wt64; }
template <typename T> const T *b_host(const LayerDev &L);
template <> const float *b_host<float>(const LayerDev &L) { return L.b; }
template <> const double *b_host<double>(const LayerDev &L) { return L.b64; }

constexpr int GM = 128;  // GEMM output tile: rows
constexpr int GN = 128;  // GEMM output tile: columns
constexpr int GK = 8;    // GEMM K slice
constexpr int ACT_ROWS = 8;  // rows per CTA of the activation kernel (one warp each)

__device__ __forceinline__ long long boxes_in_chunk(const BoxSrc &src, long long c0, long long nb) {
    const long long n = src.list ? (long long)*src.list_count : src.n;
    const long long left = n - c0;
    return left < nb ? (left > 0 ? left : 0) : nb;
}

__device__ __forceinline__ long long box_index(const BoxSrc &src, long long bidx) {
    return src.list ? (long long)src.list[bidx] : bidx;
}

// The input rows of linear layer 0 for box b: the box (Proc. 1 / App. A:
// center, X = diag(half-widths)) and, with the encoding, its rows
// sin(pi 2^k x_d), cos(pi 2^k x_d) = sin(pi (2^k x_d + 1/2)), each with the
// sin rule (in FP64 from the exact center and radius, as the SIMT engine
// does) and its own new symbol.
template <typename T>
__global__ void full_init_kernel(NetDev net, BoxSrc src, T *X, double *cen, int LD, long long rs, int R,
                                 long long c0, long long nb) {
    const long long nbox = boxes_in_chunk(src, c0, nb);
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    const long long gb = box_index(src, c0 + b);
    T c[3] = {T(0), T(0), T(0)}, h[3] = {T(0), T(0), T(0)};
    if (src.kind == SRC_NODES) {
        node_geometry<T>(src, src.nodes[gb], c, h);
    } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            c[d] = T(src.centers[gb * 3 + d]);
            h[d] = (src.kind == SRC_BOXES) ? T(src.halfw[gb * 3 + d]) : T(0);
        }
    }
    T *Xb = X + b * rs;
    double *cb = cen + b * R;
    const int m = 3 + 6 * net.pe, S0 = m;
    for (int i = 0; i < m; ++i) {
        T *row = Xb + (long long)i * LD;
        for (int k = 0; k <= S0; ++k) row[k] = T(0);
        if (i < 3) {
            cb[i] = (double)c[i];
            row[1 + i] = h[i];
            continue;
        }
        const int q = i - 3, k = q / 6, d = q % 3;
        const T sc = (T)ldexp(1.0, k), sh = (q % 6) >= 3 ? T(0.5) : T(0);
        const T ct = sc * c[d] + sh, at = sc * h[d];
        const double rad = fabs((double)at);
        double a, bb, g;
        linearize_sinpi<double>((double)ct - rad, (double)ct + rad, a, bb, g);
        cb[i] = a * (double)ct + bb;
        row[1 + d] = T(a) * at;
        row[1 + 3 + q] = T(g);
    }
}

// Four consecutive elements from global memory: one 16-byte load when the
// whole run lies inside [0, lim) and `vec` (16-byte alignment of the run),
// else element by element with zero fill.
template <typename T>
__device__ __forceinline__ void gload4(const T *p, long long i, long long lim, bool vec, T *v) {
    if (vec && i + 3 < lim) {
        load4(p + i, v);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = (i + q < lim) ? p[i + q] : T(0);
    }
}

// Y[b] (M x N) = W (M x K) X[b] (K x N) for the boxes of the chunk; W is
// given transposed, Wt [K][M]. CTA tile GM x GN, K slices of GK staged
// through two shared-memory buffers (the next slice's global loads are in
// flight while the current one is multiplied); 256 threads, each 8 x 8
// outputs (rows ty*4 + {0..3} and 64 + ty*4 + {0..3}, columns likewise with
// tx). Every output is summed over k in ascending order.
template <typename T>
__global__ void __launch_bounds__(256) full_gemm_kernel(const T *__restrict__ Wt, int M, int K,
                                                         const T *__restrict__ X, T *__restrict__ Y, int N, int LD,
                                                         long long rs, BoxSrc src, long long c0, long long nb) {
    __shared__ __align__(16) T As[2][GK][GM];  // As[.][k][m] = W[m0 + m][k0 + k]
    __shared__ __align__(16) T Bs[2][GK][GN];  // Bs[.][k][n] = X[k0 + k][n0 + n]
    const long long b = blockIdx.z;
    if (b >= boxes_in_chunk(src, c0, nb)) return;
    const T *Xb = X + b * rs;
    T *Yb = Y + b * rs;
    const int m0 = blockIdx.y * GM, n0 = blockIdx.x * GN;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    // this thread's share of a slice: row lk of the slice, four elements at lc
    const int lk = tid >> 5, lc = (tid & 31) * 4;
    const bool avec = (M & 3) == 0, bvec = (LD & 3) == 0;
    T ra[4], rb[4];
    auto fetch = [&](int k0) {
        const int k = k0 + lk;
        if (k < K) {
            gload4(Wt + (long long)k * M, (long long)(m0 + lc), (long long)M, avec, ra);
            gload4(Xb + (long long)k * LD, (long long)(n0 + lc), (long long)N, bvec, rb);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) ra[q] = rb[q] = T(0);
        }
    };
    auto stash = [&](int buf) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            As[buf][lk][lc + q] = ra[q];
            Bs[buf][lk][lc + q] = rb[q];
        }
    };
    T acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[r][q] = T(0);
    const int nt = (K + GK - 1) / GK;
    fetch(0);
    stash(0);
    __syncthreads();
    for (int t = 0; t < nt; ++t) {
        const int cur = t & 1;
        if (t + 1 < nt) fetch((t + 1) * GK);
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            T a[8], v[8];
            load4(&As[cur][kk][ty * 4], a);
            load4(&As[cur][kk][64 + ty * 4], a + 4);
            load4(&Bs[cur][kk][tx * 4], v);
            load4(&Bs[cur][kk][64 + tx * 4], v + 4);
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[r][q] = fma(a[r], v[q], acc[r][q]);
        }
        if (t + 1 < nt) stash(cur ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int m = m0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + r - 4);
        if (m >= M) continue;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int n = n0 + (q < 4 ? tx * 4 + q : 64 + tx * 4 + q - 4);
            if (n < N) Yb[(long long)m * LD + n] = acc[r][q];
        }
    }
}

// Center of row i: sum_j W_ij c_j + b_i in FP64, in input order (the FP64
// copy of the weights holds the FP32 weights exactly).
__global__ void full_center_kernel(const double *__restrict__ Wt, const double *__restrict__ bias, int M, int K,
                                   const double *__restrict__ cin, double *__restrict__ cout, int R, BoxSrc src,
                                   long long c0, long long nb) {
    const long long b = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= boxes_in_chunk(src, c0, nb) || i >= M) return;
    const double *cb = cin + b * R;
    double s = 0.0;
    for (int j = 0; j < K; ++j) s = fma(__ldg(Wt + (long long)j * M + i), cb[j], s);
    cout[b * R + i] = s + __ldg(bias + i);
}

// Activation of every row of the chunk's boxes (S symbols in columns 1..S);
// appends the M new symbols in columns S+1..S+M.
template <typename T>
__global__ void __launch_bounds__(32 * ACT_ROWS) full_act_kernel(int act, int slope, T *Y, double *cen, int M, int S,
                                                                 int LD, long long rs, int R, BoxSrc src,
                                                                 long long c0, long long nb) {
    const long long b = blockIdx.y;
    const int lane = threadIdx.x & 31, i = blockIdx.x * ACT_ROWS + (threadIdx.x >> 5);
    if (b >= boxes_in_chunk(src, c0, nb) || i >= M) return;
    T *row = Y + b * rs + (long long)i * LD;
    T rad = T(0);
    for (int k = 1 + lane; k <= S; k += 32) rad += fabs(row[k]);
    rad = warp_sum<T>(rad);  // every lane holds the same sum
    // the rule runs in FP64 from the row's FP64 center and its radius (one
    // rule per row is cheap next to the row's share of the GEMM)
    double *cp = cen + b * R + i;
    const double c = *cp, rd = (double)rad;
    double a, bb, g;
    linearize<double>(act, slope, c - rd, c + rd, a, bb, g);
    const T at = T(a);
    for (int k = 1 + lane; k <= S; k += 32) row[k] *= at;
    for (int k = lane; k < M; k += 32) row[1 + S + k] = (k == i) ? T(g) : T(0);
    if (lane == 0) *cp = fma(a, c, bb);
}

// Output layer w . [x0 | X] + b_out (one row) and Proc. 1's class.
template <typename T>
__global__ void __launch_bounds__(256) full_out_kernel(const T *__restrict__ w, const double *__restrict__ w64,
                                                        const double *__restrict__ bout, int K,
                                                        const T *__restrict__ X, const double *__restrict__ cen, int S,
                                                        int LD, long long rs, int R, BoxSrc src, BoundOut out,
                                                        long long c0, long long nb) {
    __shared__ T red[8];
    const long long b = blockIdx.x;
    if (b >= boxes_in_chunk(src, c0, nb)) return;
    const T *Xb = X + b * rs;
    T part = T(0);
    for (int k = 1 + threadIdx.x; k <= S; k += blockDim.x) {
        T y = T(0);
        for (int j = 0; j < K; ++j) y = fma(__ldg(w + j), Xb[(long long)j * LD + k], y);
        part += fabs(y);
    }
    part = warp_sum<T>(part);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x != 0) return;
    T rad = T(0);
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) rad += red[q];
    const double *cb = cen + b * R;
    double s = 0.0;
    for (int j = 0; j < K; ++j) s = fma(__ldg(w64 + j), cb[j], s);
    const T y0 = T(s + __ldg(bout));
    const long long gb = box_index(src, c0 + b);
    const T lo = y0 - rad, hi = y0 + rad;
    const int cls = classify_range(lo, hi);  // Proc. 1
    if (out.lo) out.lo[gb] = (float)lo;
    if (out.hi) out.hi[gb] = (float)hi;
    if (out.cls) out.cls[gb] = (uint8_t)cls;
    if (out.recheck_counter) atomicAdd(out.recheck_counter, 1ull);
    if (out.flag_list) {  // either end of the range near zero: FP64 decides
        const T band = T(out.band) * (fabs(y0) + rad);
        if (fabs(lo) <= band || fabs(hi) <= band) out.flag_list[atomicAdd(out.flag_count, 1)] = (int)gb;
    }
}

template <typename T>
cudaError_t full_hbm_t(const NetDev &net, const FullHbmCfg &fc, const BoxSrc &src, const BoundOut &out,
                       long long n_hint, void *scratch, cudaStream_t st) {
    const long long rs = (long long)fc.rows * fc.LD;
    T *buf[2] = {(T *)scratch, (T *)scratch + rs * fc.chunk};
    double *cen[2] = {(double *)(buf[1] + rs * fc.chunk), nullptr};
    cen[1] = cen[0] + (long long)fc.rows * fc.chunk;
    const int R = fc.rows;
    for (long long c0 = 0; c0 < n_hint; c0 += fc.chunk) {
        const long long nb = n_hint - c0 < fc.chunk ? n_hint - c0 : fc.chunk;
        full_init_kernel<T><<<(unsigned)((nb + 127) / 128), 128, 0, st>>>(net, src, buf[0], cen[0], fc.LD, rs, R,
                                                                            c0, nb);
        int S = 3 + 6 * net.pe, cur = 0;
        for (int l = 0; l + 1 < net.L; ++l) {
            const LayerDev &Ld = net.layer[l];
            const int M = Ld.out, K = Ld.in, N = 1 + S;
            const dim3 gg((unsigned)((N + GN - 1) / GN), (unsigned)((M + GM - 1) / GM), (unsigned)nb);
            full_gemm_kernel<T><<<gg, 256, 0, st>>>(Wt_host<T>(Ld), M, K, buf[cur], buf[cur ^ 1], N, fc.LD, rs, src,
                                                   c0, nb);
            full_center_kernel<<<dim3((unsigned)((M + 127) / 128), (unsigned)nb), 128, 0, st>>>(
                Ld.Wt64, Ld.b64, M, K, cen[cur], cen[cur ^ 1], R, src, c0, nb);
            cur ^= 1;
            if (Ld.act != SRA_ACT_IDENTITY) {
                full_act_kernel<T><<<dim3((unsigned)((M + ACT_ROWS - 1) / ACT_ROWS), (unsigned)nb), 32 * ACT_ROWS,
                                     0, st>>>(Ld.act, fc.slope, buf[cur], cen[cur], M, S, fc.LD, rs, R, src, c0, nb);
                S += M;
            }
        }
        const LayerDev &Lo = net.layer[net.L - 1];
        full_out_kernel<T><<<(unsigned)nb, 256, 0, st>>>(Wt_host<T>(Lo), Lo.Wt64, Lo.b64, Lo.in, buf[cur], cen[cur],
                                                        S, fc.LD, rs, R, src, out, c0, nb);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

sra_status full_hbm_cfg(const NetDev &net, int rows, int slope, int tsize, size_t budget, FullHbmCfg *fc) {
    int S = 3 + 6 * net.pe;
    for (int l = 0; l + 1 < net.L; ++l)
        if (net.layer[l].act != SRA_ACT_IDENTITY) S += net.layer[l].out;
    fc->rows = rows;
    fc->LD = (1 + S + 3) / 4 * 4;
    fc->slope = slope;
    fc->syms = S;
    const size_t per_box = 2 * ((size_t)rows * fc->LD * tsize + (size_t)rows * sizeof(double));
    long long chunk = (long long)(budget / per_box);
    if (chunk < 1) return SRA_EUNSUPPORTED;
    if (chunk > 65535) chunk = 65535;
    fc->chunk = chunk;
    fc->bytes = per_box * (size_t)chunk;
    return SRA_OK;
}

cudaError_t launch_full_hbm(bool fp64, const NetDev &net, const FullHbmCfg &fc, const BoxSrc &src,
                            const BoundOut &out, long long n_hint, void *scratch, cudaStream_t st) {
    return fp64 ? full_hbm_t<double>(net, fc, src, out, n_hint, scratch, st)
                : full_hbm_t<float>(net, fc, src, out, n_hint, scratch, st);
}

}  // namespace sra
