// Affine-full RangeBound beyond the SIMT engine's register row (Sec. 3.3,
// "full": every new symbol is kept, so the noise matrix gains one column per
// neuron of every nonlinear layer; the paper finds it the tightest policy for
// volumetric queries). The 8-layer, 32-wide networks of the paper's
// experiments reach 3 + 7 * 32 = 227 symbols, past the 128 columns a thread
// of the SIMT engine holds in registers.
//
// One CTA per box (grid-stride over boxes). The box's noise matrix X (rows x
// K, row stride KS) lives in shared memory. A dense layer maps every column
// in place: column k of W X depends only on column k of X, so thread t owns
// the columns k = t, t + NT, ... and reads its column into registers before
// overwriting it. The center (compensated sum in FP32, as in the SIMT
// engine) and the independent part x_inf = |W| x_inf go to the second of two
// buffers. The rows' ranges (Eq. def_range) are warp sums over the columns;
// then each row's activation rule (App. A Table "affine_nonlinearities")
// scales its row and the diagonal block of the new symbols is appended.
#include "engine_simt.cuh"
#include "launch.h"

namespace sra {

constexpr int kFullThreads = 128;

template <typename T, int WMAX>
__global__ void __launch_bounds__(kFullThreads) full_bound_kernel(NetDev net, BoxSrc src, BoundOut out, FullCfg fc) {
    extern __shared__ __align__(16) unsigned char fsm[];
    constexpr int NT = kFullThreads, NW = NT / 32;
    const int R = fc.rows, KS = fc.KS;
    T *X = (T *)(fsm + fc.x_off);       // [R][KS]
    T *Ws = (T *)(fsm + fc.w_off);      // [R][R]: W of the current layer, [out][in]
    T *bs = Ws + R * R;                  // [R]
    T *cv = bs + R;                      // [2][R] centers
    T *xv = cv + 2 * R;                  // [2][R] x_inf
    T *alv = xv + 2 * R;                 // [R] slopes
    T *gav = alv + R;                    // [R] new-symbol magnitudes
    T *radv = gav + R;                   // [R] ranges
    T *red = radv + R;                   // [NW] block reduction
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    long long n = src.n;
    if (src.list) n = *src.list_count;
    for (long long bidx = blockIdx.x; bidx < n; bidx += gridDim.x) {
        const long long gb = src.list ? (long long)src.list[bidx] : bidx;
        // Proc. 1 / App. A initialisation: x0 = box center, X = diag(half-widths)
        if (t < 3) {
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
            cv[t] = c[t];
            xv[t] = T(0);
#pragma unroll
            for (int k = 0; k < 3; ++k) X[t * KS + k] = (k == t) ? h[t] : T(0);
        }
        int K = 3, cur = 0;
        __syncthreads();
        for (int l = 0; l + 1 < net.L; ++l) {
            const LayerDev &Ld = net.layer[l];
            const int hin = Ld.in, hout = Ld.out;
            const T *Wt = Wt_of<T>(Ld);  // [in][out]
            for (int e = t; e < hin * hout; e += NT) {
                const int j = e / hout, i = e - j * hout;
                Ws[i * R + j] = __ldg(Wt + e);
            }
            for (int e = t; e < hout; e += NT) bs[e] = __ldg(b_of<T>(Ld) + e);
            __syncthreads();
            // noise columns, in place (Table "affine_update_rules": A' = W A)
            for (int k = t; k < K; k += NT) {
                T x[WMAX];
#pragma unroll
                for (int j = 0; j < WMAX; ++j) x[j] = j < hin ? X[j * KS + k] : T(0);
                for (int i = 0; i < hout; ++i) {
                    const T *wr = Ws + i * R;
                    T y = T(0);
#pragma unroll
                    for (int j = 0; j < WMAX; ++j)
                        if (j < hin) y = fma(wr[j], x[j], y);
                    X[i * KS + k] = y;
                }
            }
            // center c' = W c + b and x_inf' = |W| x_inf, summed in input order
            const T *cin = cv + cur * R, *xin = xv + cur * R;
            T *cout = cv + (cur ^ 1) * R, *xout = xv + (cur ^ 1) * R;
            for (int i = t; i < hout; i += NT) {
                const T *wr = Ws + i * R;
                T xi = T(0);
                if (sizeof(T) == 4) {
                    Dot2<T> cd;
                    for (int j = 0; j < hin; ++j) {
                        cd.add_prod(wr[j], cin[j]);
                        xi = fma(fabs(wr[j]), xin[j], xi);
                    }
                    cd.add(bs[i]);
                    cout[i] = cd.value();
                } else {
                    T c = T(0);
                    for (int j = 0; j < hin; ++j) {
                        c = fma(wr[j], cin[j], c);
                        xi = fma(fabs(wr[j]), xin[j], xi);
                    }
                    cout[i] = c + bs[i];
                }
                xout[i] = xi;
            }
            __syncthreads();
            cur ^= 1;
            if (Ld.act != SRA_ACT_IDENTITY) {
                // ranges (Eq. def_range): sum_k |X_ik| + x_inf_i
                for (int i = warp; i < hout; i += NW) {
                    T s = T(0);
                    for (int k = lane; k < K; k += 32) s += fabs(X[i * KS + k]);
                    s = warp_sum<T>(s);
                    if (lane == 0) radv[i] = s + xv[cur * R + i];
                }
                __syncthreads();
                // linearisation (Eq. affine_func_update)
                for (int i = t; i < hout; i += NT) {
                    const T c = cv[cur * R + i], rad = radv[i];
                    T a, b, g;
                    linearize<T>(Ld.act, fc.slope, c - rad, c + rad, a, b, g);
                    alv[i] = a;
                    gav[i] = g;
                    cv[cur * R + i] = a * c + b;
                    xv[cur * R + i] = fabs(a) * xv[cur * R + i];
                }
                __syncthreads();
                // scale the rows; append the new symbols (one per neuron, full keeps all)
                const int Kn = K + hout;
                for (int e = t; e < hout * Kn; e += NT) {
                    const int i = e / Kn, k = e - i * Kn;
                    T *p = X + i * KS + k;
                    *p = k < K ? alv[i] * *p : (k - K == i ? gav[i] : T(0));
                }
                K = Kn;
                __syncthreads();
            }
        }
        // output layer (1 x in): y_k = w . X[:, k], radius sum_k |y_k| + |w| . x_inf
        const LayerDev &Lo = net.layer[net.L - 1];
        const T *w = Wt_of<T>(Lo);
        const int hin = Lo.in;
        T part = T(0);
        for (int k = t; k < K; k += NT) {
            T y = T(0);
            for (int j = 0; j < hin; ++j) y = fma(__ldg(w + j), X[j * KS + k], y);
            part += fabs(y);
        }
        part = warp_sum<T>(part);
        if (lane == 0) red[warp] = part;
        __syncthreads();
        if (t == 0) {
            T rad = T(0);
            for (int q = 0; q < NW; ++q) rad += red[q];
            T xi = T(0);
            const T *cin = cv + cur * R, *xin = xv + cur * R;
            for (int j = 0; j < hin; ++j) xi = fma(fabs(__ldg(w + j)), xin[j], xi);
            rad += xi;
            T y0;
            if (sizeof(T) == 4) {
                Dot2<T> cd;
                for (int j = 0; j < hin; ++j) cd.add_prod(__ldg(w + j), cin[j]);
                y0 = add_rn(cd.value(), __ldg(b_of<T>(Lo)));
            } else {
                T c = T(0);
                for (int j = 0; j < hin; ++j) c = fma(__ldg(w + j), cin[j], c);
                y0 = c + __ldg(b_of<T>(Lo));
            }
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
        __syncthreads();  // state reuse by the next box
    }
}

sra_status full_cfg(int rows, int total_syms, int slope, int tsize, FullCfg *fc) {
    if (rows > kFullMaxWidth) return SRA_EUNSUPPORTED;
    fc->rows = rows;
    fc->KS = (total_syms + 3) / 4 * 4;
    fc->slope = slope;
    size_t off = 0;
    fc->x_off = 0;
    off = ((size_t)rows * fc->KS * tsize + 15) & ~(size_t)15;
    fc->w_off = (int)off;
    off += ((size_t)rows * rows + 8 * rows + 32) * tsize;
    off = (off + 15) & ~(size_t)15;
    if (off > (size_t)232448) return SRA_EUNSUPPORTED;
    fc->smem = (int)off;
    return SRA_OK;
}

template <typename T, int WMAX>
static cudaError_t launch_full_t(const NetDev &net, const BoxSrc &src, const BoundOut &out, const FullCfg &fc,
                                 long long n_hint, cudaStream_t st) {
    auto k = full_bound_kernel<T, WMAX>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, fc.smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kFullThreads, fc.smem)) != cudaSuccess)
        return e;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long grid = (long long)(per_sm > 0 ? per_sm : 1) * sms * 4;
    if (grid > n_hint) grid = n_hint;
    if (grid < 1) grid = 1;
    k<<<(unsigned)grid, kFullThreads, fc.smem, st>>>(net, src, out, fc);
    return cudaGetLastError();
}

cudaError_t launch_full_bound(bool fp64, const NetDev &net, const BoxSrc &src, const BoundOut &out,
                              const FullCfg &fc, long long n_hint, cudaStream_t st) {
    if (fc.rows <= 32)
        return fp64 ? launch_full_t<double, 32>(net, src, out, fc, n_hint, st)
                    : launch_full_t<float, 32>(net, src, out, fc, n_hint, st);
    return fp64 ? launch_full_t<double, 64>(net, src, out, fc, n_hint, st)
                : launch_full_t<float, 64>(net, src, out, fc, n_hint, st);
}

}  // namespace sra
