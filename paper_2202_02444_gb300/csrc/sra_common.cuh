// Shared device structures and scalar range rules of the CUDA path.
//
// The rules restate App. A, Table "affine_nonlinearities" (Sharp & Jacobson
// 2022) for T = float / double, in the form that stays a valid bound for any
// slope alpha: for a convex activation the largest deviation of
// f(x) - alpha x sits at an endpoint and the smallest at the tangent point
// x* = f'^-1(alpha) clamped to [l, u]; for sin the extremes sit at the
// endpoints or at the extreme critical points of the two families
// +-acos(alpha) + 2 pi k inside [l, u]. With the secant slope these give the
// table's Chebyshev parameters.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sra.h"

namespace sra {

constexpr int kMaxLayers = 24;
constexpr int kMaxWidth = 512;
constexpr int kMaxKdLevels = 64;

// Threads per CTA the SIMT engine kernels are compiled for: the register
// budget of a row of KMAX accumulators (65536 registers per SM).
__host__ __device__ constexpr int engine_max_threads(int tsize, int kmax) {
    return tsize == 4 ? (kmax >= 64 ? 256 : (kmax >= 32 ? 512 : 1024))
                      : (kmax >= 128 ? 128 : (kmax >= 16 ? 256 : (kmax >= 4 ? 512 : 1024)));
}

struct LayerDev {
    const float *Wt;    // [in][out]: transposed, so threads of consecutive
    const float *b;     // output neurons read consecutive words
    const double *Wt64;
    const double *b64;
    int in, out, act;
};

struct NetDev {
    int L;    // linear layers
    int pe;   // positional-encoding octaves (0: none)
    int din;  // widths[0]
    LayerDev layer[kMaxLayers];
};

enum { SRC_BOXES = 0, SRC_NODES = 1, SRC_POINTS = 2 };

// Where a kernel reads its boxes from.
struct BoxSrc {
    int kind;
    const float *centers;   // SRC_BOXES / SRC_POINTS: [n][3]
    const float *halfw;     // SRC_BOXES: [n][3]
    const sra_node *nodes;  // SRC_NODES
    float root_lo[3], root_ext[3];
    int split;
    unsigned char kd_n3[kMaxKdLevels][3];  // per k-d level: halvings per axis
    const int *list;        // if non-null: box b is list[b], count in *list_count
    const int *list_count;
    long long n;            // number of boxes when list == nullptr
};

struct BoundOut {
    float *lo, *hi;
    uint8_t *cls;
    int *flag_list;          // append UNKNOWN boxes whose bound is near zero
    int *flag_count;
    float band;
    unsigned long long *recheck_counter;  // incremented per re-bounded box
};

// Per-launch configuration shared by host and device.
struct RangeCfg {
    int arith, K, slope;
    int H;      // threads per box (multiple of 32, >= every layer width)
    int NB;     // boxes per CTA
    int rows;   // rows of the per-box state matrix (max width)
    int slot_bytes;
    int x_off, score_off, part_off, outv_off, keep_off, src_off, ray_off;
    int threads;  // threads that run the engine on this layout: 0 = the whole
                  // CTA (__syncthreads), else the first `threads` (named barrier 1)
};

// The barrier of the SIMT engine: the whole CTA, or the first cfg.threads
// threads (whole warps) when a CTA runs layouts of several networks.
__device__ __forceinline__ void engine_sync(const RangeCfg &cfg) {
    if (cfg.threads == 0) __syncthreads();
    else asm volatile("bar.sync 1, %0;" ::"r"(cfg.threads) : "memory");
}

// One segment of a batched round over many networks: a network, its
// layout, its nodes and where their classes go.
struct BatchSegDev {
    NetDev net;
    RangeCfg cfg;      // cfg.threads = NB * H engine threads
    BoxSrc src;        // SRC_NODES, this segment's nodes
    BoundOut out;      // classes of this segment's nodes
    long long chunk0;  // first chunk (group of NB nodes) of the segment in its launch
};

// CastRay (Proc. 2) launch parameters and per-slot state. Every per-ray
// array is indexed by the ray's own index.
struct RayParams {
    const float *origins, *dirs, *f0;
    const float *t_start, *sigma_start;  // optional per-ray march state to resume from
    float *t_hit;
    int *iters;
    long long n;
    unsigned long long *next;  // global ray counter
    float delta, t_max, sigma0, eta_plus, eta_minus, safety;
    long long max_iters;
    // optional: march only the rays list[0 .. *list_count) (their indices),
    // adding one to *recheck_counter (if given) per ray taken
    const int *list, *list_count;
    unsigned long long *recheck_counter;
    // optional: append each ray that met a decision near zero (near_zero_step)
    // once, when it ends, to flag_list[atomicAdd(flag_count, 1)]
    int *flag_list, *flag_count;
    float band;
};

// The march state (t, sigma) is kept in the kernel's precision.
template <typename T> struct RaySlotState {
    long long idx;  // ray index, -1 idle
    T t, sigma;
    int f0pos;
    int iters;
    int live;
    int flag;  // a decision of this ray was near zero
};

// Debug builds (-DSRA_DEBUG_BOUNDS) check data-dependent indices of the
// tensor-core kernels before use: an index outside [0, bound) skips the
// access and records `code` (>= 100) in the kernel's status word, which
// sra_sync_status reports, instead of faulting. Release builds compile the
// checks away.
__device__ __forceinline__ bool idx_ok(long long idx, long long bound, int *status, int code) {
#ifdef SRA_DEBUG_BOUNDS
    if (idx >= 0 && idx < bound) return true;
    atomicCAS(status, 0, code);
    return false;
#else
    (void)idx; (void)bound; (void)status; (void)code;
    return true;
#endif
}

// A march step whose decision the FP64 re-check takes again: the segment
// bound [y0 - rad, y0 + rad] has an end within band (|y0| + rad) of zero, the
// case where the rounding of a lower precision can flip the segment's class
// (the rule of the box re-check). A wrong sign of the point value fc near
// zero needs no re-check: a root then lies within about delta of the point,
// which the delta semantics of Proc. 2 accept.
template <typename T>
__device__ __forceinline__ bool near_zero_step(T y0, T rad, float band) {
    const T scale = fabs(y0) + rad, b = (T)band;
    return fabs(y0 - rad) <= b * scale || fabs(y0 + rad) <= b * scale;
}

template <typename T> struct Num;
template <> struct Num<float> {
    static __device__ __forceinline__ float pi() { return 3.14159265358979323846f; }
};
template <> struct Num<double> {
    static __device__ __forceinline__ double pi() { return 3.14159265358979323846; }
};

template <typename T> __device__ __forceinline__ T clampT(T x, T a, T b) {
    return x < a ? a : (x > b ? b : x);
}

template <typename T> __device__ __forceinline__ T act_eval(int act, T x) {
    switch (act) {
    case SRA_ACT_RELU: return x > T(0) ? x : T(0);
    case SRA_ACT_ELU: return x > T(0) ? x : expm1(x);
    case SRA_ACT_SIN: return sin(x);
    default: return x;
    }
}

// Extremes of cos on [l,u], located through multiples of 2 pi (App. A).
template <typename T> __device__ __forceinline__ void cos_extremes(T l, T u, T &lo, T &hi) {
    const T tp = T(2) * Num<T>::pi();
    if (u - l >= tp) { lo = T(-1); hi = T(1); return; }
    T cl = cos(l), cu = cos(u);
    hi = fmax(cl, cu);
    lo = fmin(cl, cu);
    if (tp * ceil(l / tp) <= u) hi = T(1);
    if (tp * ceil((l - Num<T>::pi()) / tp) + Num<T>::pi() <= u) lo = T(-1);
}

template <typename T> __device__ __forceinline__ void sin_extremes(T l, T u, T &lo, T &hi) {
    const T tp = T(2) * Num<T>::pi(), hp = T(0.5) * Num<T>::pi();
    if (u - l >= tp) { lo = T(-1); hi = T(1); return; }
    T sl = sin(l), su = sin(u);
    hi = fmax(sl, su);
    lo = fmin(sl, su);
    if (tp * ceil((l - hp) / tp) + hp <= u) hi = T(1);
    if (tp * ceil((l + hp) / tp) - hp <= u) lo = T(-1);
}

// Interval image of [l,u] (Sec. 3.1): ReLU / ELU / identity are monotone.
template <typename T> __device__ __forceinline__ void interval_image(int act, T l, T u, T &lo, T &hi) {
    if (act == SRA_ACT_SIN) { sin_extremes(l, u, lo, hi); return; }
    lo = act_eval<T>(act, l);
    hi = act_eval<T>(act, u);
}

// phi(t) = expm1(t) - t without cancellation near t = 0 (Taylor series up
// to t^8/8! for |t| < 1/2, where the truncation is below 1e-7 relative).
template <typename T> __device__ __forceinline__ T expm1_minus_id(T t) {
    if (fabs(t) >= T(0.5)) return expm1(t) - t;
    T p = T(1) / T(40320);
    p = fma(p, t, T(1) / T(5040));
    p = fma(p, t, T(1) / T(720));
    p = fma(p, t, T(1) / T(120));
    p = fma(p, t, T(1) / T(24));
    p = fma(p, t, T(1) / T(6));
    p = fma(p, t, T(0.5));
    return p * t * t;
}

// alpha, beta, gamma with |f(x) - alpha x - beta| <= gamma on [l,u]
// (Eq. affine_func_update; App. A Table "affine_nonlinearities").
// gamma is half the spread of g(x) = f(x) - alpha x over [l,u]; it is formed
// from differences g(x) - g(l) written without cancellation (expm1 for ELU,
// sum-to-product for sin), because the plain r_u - r_l loses most digits in
// FP32 when [l,u] is narrow.
template <typename T>
__device__ __forceinline__ void linearize(int act, int slope, T l, T u, T &a, T &b, T &g) {
    a = T(1); b = T(0); g = T(0);
    if (act == SRA_ACT_RELU) {
        if (u <= T(0)) { a = T(0); return; }
        if (l >= T(0)) return;
        if (slope == SRA_SLOPE_MINRANGE) { a = T(0); b = T(0.5) * u; g = b; return; }
        a = u / (u - l);
        b = (T(0) - a * l) / T(2);
        g = b;
        return;
    }
    if (act == SRA_ACT_ELU) {
        if (l >= T(0)) return;
        const T fl = expm1(l);
        // f(u) - f(l) without cancellation
        // (exp(l) expm1(u - l) would be 0 * inf for very wide negative ranges)
        const T df = (u > T(0)) ? (u - fl) : ((u - l < T(30)) ? exp(l) * expm1(u - l) : expm1(u) - fl);
        if (slope == SRA_SLOPE_MINRANGE) {
            a = exp(l);  // smallest derivative: f - a x is non-decreasing on [l,u]
            const T spread = (u > T(0) || u - l >= T(30)) ? (df - a * (u - l)) : a * expm1_minus_id<T>(u - l);
            g = T(0.5) * spread;
            b = (fl - a * l) + g;
            return;
        }
        a = (u > l) ? df / (u - l) : exp(l);
        const T ru = fl - a * l;  // secant intercept: max of f - a x (convex f)
        // min of f - a x at the tangent point x* = ln a (clamped to [l,u])
        T spread;
        const T xs = (a <= T(0)) ? l : (a >= T(1) ? u : clampT<T>(log(a), l, u));
        if (xs > l && xs < u && xs <= T(0)) {
            // g(l) - g(x*) = a (expm1(l - x*) - (l - x*)) since e^{x*} = a
            spread = a * expm1_minus_id<T>(l - xs);
        } else {
            spread = ru - (act_eval<T>(SRA_ACT_ELU, xs) - a * xs);
        }
        if (spread < T(0)) spread = T(0);
        g = T(0.5) * spread;
        b = ru - g;
        return;
    }
    if (act == SRA_ACT_SIN) {
        const T tp = T(2) * Num<T>::pi();
        if (u - l >= tp) { a = T(0); b = T(0); g = T(1); return; }
        T sl, su;
        cos_extremes(l, u, sl, su);
        a = (sl + su) / T(2);
        const T ep = acos(clampT<T>(a, T(-1), T(1)));
        T cand[5];
        cand[0] = u;
        cand[1] = clampT<T>(ep + tp * ceil((l - ep) / tp), l, u);
        cand[2] = clampT<T>(ep + tp * floor((u - ep) / tp), l, u);
        cand[3] = clampT<T>(-ep + tp * ceil((l + ep) / tp), l, u);
        cand[4] = clampT<T>(-ep + tp * floor((u + ep) / tp), l, u);
        // d(x) = g(x) - g(l) = 2 cos((x+l)/2) sin((x-l)/2) - a (x - l)
        T dmax = T(0), dmin = T(0);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const T h = T(0.5) * (cand[q] - l);
            const T d = T(2) * cos(l + h) * sin(h) - a * (cand[q] - l);
            dmax = fmax(dmax, d);
            dmin = fmin(dmin, d);
        }
        g = T(0.5) * (dmax - dmin);
        b = (sin(l) - a * l) + T(0.5) * (dmax + dmin);
        return;
    }
}

__device__ __forceinline__ float sinpi_t(float x) { return sinpif(x); }
__device__ __forceinline__ double sinpi_t(double x) { return sinpi(x); }
__device__ __forceinline__ float cospi_t(float x) { return cospif(x); }
__device__ __forceinline__ double cospi_t(double x) { return cospi(x); }

// The sin rule for y = sin(pi t) on t in [l,u] (t in half-turns), used by the
// positional encoding sin(2^k pi x) = sin(pi * 2^k x): 2^k x is exact, so the
// argument carries no rounding of pi even where 2^k pi x is large. Same rule
// as `linearize` for sin (slope from the cos range, extremes of
// g(t) = sin(pi t) - a t at the ends and at the extreme critical points),
// with the slope a expressed per unit of t.
template <typename T>
__device__ __forceinline__ void linearize_sinpi(T l, T u, T &a, T &b, T &g) {
    if (u - l >= T(2)) { a = T(0); b = T(0); g = T(1); return; }
    // extremes of cos(pi t) on [l,u]: +1 at even integers, -1 at odd ones
    const T cl = cospi_t(l), cu = cospi_t(u);
    T chi = fmax(cl, cu), clo = fmin(cl, cu);
    if (T(2) * ceil(l / T(2)) <= u) chi = T(1);
    if (T(2) * ceil((l - T(1)) / T(2)) + T(1) <= u) clo = T(-1);
    const T az = (clo + chi) / T(2);  // slope per radian
    a = az * Num<T>::pi();            // slope per half-turn
    const T e = acos(clampT<T>(az, T(-1), T(1))) / Num<T>::pi();
    T cand[5];
    cand[0] = u;
    cand[1] = clampT<T>(e + T(2) * ceil((l - e) / T(2)), l, u);
    cand[2] = clampT<T>(e + T(2) * floor((u - e) / T(2)), l, u);
    cand[3] = clampT<T>(-e + T(2) * ceil((l + e) / T(2)), l, u);
    cand[4] = clampT<T>(-e + T(2) * floor((u + e) / T(2)), l, u);
    T dmax = T(0), dmin = T(0);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const T h = T(0.5) * (cand[q] - l);
        const T d = T(2) * cospi_t(l + h) * sinpi_t(h) - a * (cand[q] - l);
        dmax = fmax(dmax, d);
        dmin = fmin(dmin, d);
    }
    g = T(0.5) * (dmax - dmin);
    b = (sinpi_t(l) - a * l) + T(0.5) * (dmax + dmin);
}

// Interval image of sin(pi t) on [l,u].
template <typename T> __device__ __forceinline__ void sinpi_extremes(T l, T u, T &lo, T &hi) {
    if (u - l >= T(2)) { lo = T(-1); hi = T(1); return; }
    const T sl = sinpi_t(l), su = sinpi_t(u);
    hi = fmax(sl, su);
    lo = fmin(sl, su);
    if (T(2) * ceil((l - T(0.5)) / T(2)) + T(0.5) <= u) hi = T(1);
    if (T(2) * ceil((l + T(0.5)) / T(2)) - T(0.5) <= u) lo = T(-1);
}

__device__ __forceinline__ int classify_range(float lo, float hi) {
    return lo > 0.f ? SRA_POSITIVE : (hi < 0.f ? SRA_NEGATIVE : SRA_UNKNOWN);
}
__device__ __forceinline__ int classify_range(double lo, double hi) {
    return lo > 0.0 ? SRA_POSITIVE : (hi < 0.0 ? SRA_NEGATIVE : SRA_UNKNOWN);
}

// Box center / half-widths of tree node nd inside the root box. The same
// sequence of operations as the node geometry of Proc. 3: cell width
// w = extent * 2^-n, lo = root_lo + w * index, hi = lo + w, c = (lo+hi)/2,
// h = hi - c (exact for dyadic roots).
template <typename T>
__device__ __forceinline__ void node_geometry(const BoxSrc &s, const sra_node &nd, T *c, T *h) {
    const int idx[3] = {nd.ix, nd.iy, nd.iz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int lv = nd.level < kMaxKdLevels ? nd.level : kMaxKdLevels - 1;
        int n = (s.split == SRA_SPLIT_OCTREE) ? nd.level : s.kd_n3[lv][d];
        T w = T(s.root_ext[d]) * (T(1) / T(1ull << n));
        T lo = T(s.root_lo[d]) + w * T(idx[d]);
        T hi = lo + w;
        c[d] = T(0.5) * (lo + hi);
        h[d] = hi - c[d];
    }
}

}  // namespace sra
