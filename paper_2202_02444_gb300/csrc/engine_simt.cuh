// SIMT range-analysis engine: the whole MLP for NB boxes per CTA, with the
// per-box affine state resident in shared memory across all layers.
//
// Per box the state is the tuple (x0, X, x_inf) of App. A stored as a
// rows x RS matrix: row i holds [X_i0 .. X_i(KMAX-1), x0_i, xinf_i, p_i, pad]
// where p is an optional plain point value carried through the same weights
// (the CastRay convergence test of Proc. 2). Thread i of a box owns output
// neuron i: it accumulates its row of W [c|A] in registers (Table
// "affine_update_rules", matrix multiplication), linearises its activation
// (Eq. affine_func_update), and the box's threads then condense the noise
// columns together (Sec. 3.3) before the row is written back in place.
//
// Template parameters: T = float (plain FP32 form) or double (FP64 re-check);
// KMAX = compile-time bound on kept noise columns (register row length).
#pragma once

#include "sra_common.cuh"

namespace sra {

template <int KMAX> struct RowStride {
    static constexpr int value = ((KMAX + 3 + 3) / 4) * 4;  // [A.. | c | xinf | p | pad]
};

template <typename T, int KMAX> struct MaxThreads {
    static constexpr int value = engine_max_threads((int)sizeof(T), KMAX);
};

// CTAs per SM the bound kernel is compiled for. FP32 with 33..64 noise
// columns: two 256-thread CTAs (128 registers a thread, some spilled), so
// that a second box's warps hide the shared-memory latency of the row reads
// (measured: 371k against 351k boxes/s on the 3-[256]x8-1 octree frontier).
template <typename T, int KMAX> struct MinBlocks {
    static constexpr int value = (sizeof(T) == 4 && KMAX > 32 && KMAX <= 64) ? 2 : 1;
};

template <typename T> __device__ __forceinline__ const T *Wt_of(const LayerDev &L);
template <> __device__ __forceinline__ const float *Wt_of<float>(const LayerDev &L) { return L.Wt; }
template <> __device__ __forceinline__ const double *Wt_of<double>(const LayerDev &L) { return L.Wt64; }
template <typename T> __device__ __forceinline__ const T *b_of(const LayerDev &L);
template <> __device__ __forceinline__ const float *b_of<float>(const LayerDev &L) { return L.b; }
template <> __device__ __forceinline__ const double *b_of<double>(const LayerDev &L) { return L.b64; }

template <typename T, int KMAX> struct Row {
    T a[KMAX];
    T c, xi, p;
};

// Pointers into one box slot's shared memory.
template <typename T> struct Slot {
    T *X;            // rows x RS
    T *score;        // KMAX + rows candidate scores
    T *part;         // (H/32) x (KMAX+4) per-warp partial column sums
    T *outv;         // KMAX + 4 output-layer column sums
    uint8_t *keep;   // KMAX + rows keep flags
    short *src;      // KMAX source column of each kept position
    char *ray;       // ray slot state (cast_rays only)
};

template <typename T>
__device__ __forceinline__ Slot<T> carve(char *smem, int slot, const RangeCfg &cfg) {
    char *base = smem + (size_t)slot * cfg.slot_bytes;
    Slot<T> s;
    s.X = (T *)(base + cfg.x_off);
    s.score = (T *)(base + cfg.score_off);
    s.part = (T *)(base + cfg.part_off);
    s.outv = (T *)(base + cfg.outv_off);
    s.keep = (uint8_t *)(base + cfg.keep_off);
    s.src = (short *)(base + cfg.src_off);
    s.ray = base + cfg.ray_off;
    return s;
}

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void load4(const float *p, float *v) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void load4(const double *p, double *v) {
    const double2 a = *reinterpret_cast<const double2 *>(p);
    const double2 b = *reinterpret_cast<const double2 *>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// Round-to-nearest add / multiply that the compiler may not fuse into an FMA
// (error-free transformations depend on each operation rounding once).
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// Compensated dot-product accumulator (Ogita, Rump & Oishi 2005, "Accurate
// sum and dot product", Dot2): TwoProduct by FMA, TwoSum for the running sum.
// Used for the FP32 center column, whose sum cancels (|W x0| << |W||x0|).
template <typename T> struct Dot2 {
    T s = T(0), e = T(0);
    __device__ __forceinline__ void add_prod(T a, T b) {
        const T p = mul_rn(a, b);
        const T pe = fma(a, b, -p);
        add(p);
        e = add_rn(e, pe);
    }
    __device__ __forceinline__ void add(T p) {
        const T t = add_rn(s, p);
        const T z = add_rn(t, -s);
        const T te = add_rn(add_rn(s, -add_rn(t, -z)), add_rn(p, -z));
        s = t;
        e = add_rn(e, te);
    }
    __device__ __forceinline__ T value() const { return add_rn(s, e); }
};

// Row i of W [x0|X] + b and |W| x_inf (and W p), summed over inputs in order.
// FP32 box bounds sum the center column with Dot2.
template <typename T, int KMAX, bool PT>
__device__ __forceinline__ void matmul_row(const LayerDev &L, const T *X, int i, Row<T, KMAX> &r) {
    constexpr int RS = RowStride<KMAX>::value;
    constexpr bool COMP = sizeof(T) == 4 && !PT;
    const T *Wt = Wt_of<T>(L);
#pragma unroll
    for (int k = 0; k < KMAX; ++k) r.a[k] = T(0);
    r.c = T(0);
    r.xi = T(0);
    r.p = T(0);
    Dot2<T> cd;
    const int in = L.in, out = L.out;
    auto step = [&](T w, int j) {
        const T aw = fabs(w);
        const T *xr = X + j * RS;  // 16-byte aligned: RS is a multiple of 4
        // broadcast 16-byte loads (every lane of the warp reads the same row)
        constexpr int K4 = (KMAX + 3) / 4;
#pragma unroll
        for (int q = 0; q < K4; ++q) {
            T v[4];
            load4(xr + 4 * q, v);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = 4 * q + e;
                if (k < KMAX) r.a[k] = fma(w, v[e], r.a[k]);
                else if (k == KMAX) { if (COMP) cd.add_prod(w, v[e]); else r.c = fma(w, v[e], r.c); }
                else if (k == KMAX + 1) r.xi = fma(aw, v[e], r.xi);
                else if (k == KMAX + 2) { if (PT) r.p = fma(w, v[e], r.p); }
            }
        }
        if (KMAX % 4 == 0) {  // c, xinf, p sit in the next 16 bytes
            T v[4];
            load4(xr + KMAX, v);
            if (COMP) cd.add_prod(w, v[0]);
            else r.c = fma(w, v[0], r.c);
            r.xi = fma(aw, v[1], r.xi);
            if (PT) r.p = fma(w, v[2], r.p);
        } else if (KMAX % 4 == 1) {  // KMAX == 1: [A0, c, xinf, p] was one load
        }
    };
    // weights of 8 inputs in flight before their FMAs (latency of L2 loads)
    constexpr int U = 8;
    int j = 0;
    for (; j + U <= in; j += U) {
        T w[U];
#pragma unroll
        for (int q = 0; q < U; ++q) w[q] = __ldg(Wt + (size_t)(j + q) * out + i);
#pragma unroll
        for (int q = 0; q < U; ++q) step(w[q], j + q);
    }
    for (; j < in; ++j) step(__ldg(Wt + (size_t)j * out + i), j);
    const T bias = __ldg(b_of<T>(L) + i);
    if (COMP) {
        cd.add(bias);
        r.c = cd.value();
    } else {
        r.c += bias;
    }
    if (PT) r.p += bias;
}

// Activation on one row: interval image (Sec. 3.1) or affine linearisation
// (Eq. affine_func_update). Returns the new symbol's coefficient gamma.
template <typename T, int KMAX, bool PT>
__device__ __forceinline__ T activate_row(int act, const RangeCfg &cfg, Row<T, KMAX> &r) {
    T gamma = T(0);
    if (cfg.arith == SRA_ARITH_INTERVAL) {
        T lo, hi;
        interval_image<T>(act, r.c - r.xi, r.c + r.xi, lo, hi);
        r.c = T(0.5) * (lo + hi);
        r.xi = T(0.5) * (hi - lo);
    } else {
        T rad = T(0);
#pragma unroll
        for (int k = 0; k < KMAX; ++k) rad += fabs(r.a[k]);
        rad += r.xi;
        T a, b;
        linearize<T>(act, cfg.slope, r.c - rad, r.c + rad, a, b, gamma);
#pragma unroll
        for (int k = 0; k < KMAX; ++k) r.a[k] *= a;
        r.c = a * r.c + b;
        r.xi = fabs(a) * r.xi;
    }
    if (PT) r.p = act_eval<T>(act, r.p);
    return gamma;
}

// Condense after a nonlinearity (Sec. 3.3) and write the row back.
// Candidates: the Ncur old columns, then Cnew new symbols (row i's symbol, if
// any, is candidate Ncur + new_idx, holding gamma in row i only). Dropped
// magnitudes go to the row's x_inf. Kept columns stay in candidate order;
// truncate keeps the K largest column L1 norms, lower index first on ties.
// Must be called by every thread of the CTA. Returns the new column count.
template <typename T, int KMAX, bool PT>
__device__ int condense_and_store(Row<T, KMAX> &r, T gamma, bool valid, bool newsym, int new_idx,
                                  int Cnew, int Ncur, const RangeCfg &cfg, const Slot<T> &s, int i) {
    constexpr int RS = RowStride<KMAX>::value;
    if (cfg.arith == SRA_ARITH_INTERVAL || cfg.arith == SRA_ARITH_AFFINE_FIXED || Cnew == 0) {
        if (valid) {
            if (newsym) r.xi += fabs(gamma);
            T *row = s.X + i * RS;
#pragma unroll
            for (int k = 0; k < KMAX; ++k) row[k] = r.a[k];
            row[KMAX] = r.c;
            row[KMAX + 1] = r.xi;
            row[KMAX + 2] = r.p;
        }
        engine_sync(cfg);
        return Ncur;
    }
    const int C = Ncur + Cnew;
    const int Knew = (cfg.arith == SRA_ARITH_AFFINE_FULL) ? C : min(cfg.K, C);
    const bool keep_all = (Knew == C);
    if (!keep_all) {
        const int lane = i & 31, warp = i >> 5, nwarps = cfg.H >> 5;
        // column L1 norms of the old columns over the box's rows
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            T v = warp_sum<T>(valid ? fabs(r.a[k]) : T(0));
            if (lane == 0) s.part[warp * (KMAX + 4) + k] = v;
        }
        if (valid && newsym) s.score[Ncur + new_idx] = fabs(gamma);
        engine_sync(cfg);
        for (int k = i; k < Ncur; k += cfg.H) {
            T v = T(0);
            for (int w = 0; w < nwarps; ++w) v += s.part[w * (KMAX + 4) + k];
            s.score[k] = v;
        }
        engine_sync(cfg);
        for (int c = i; c < C; c += cfg.H) {
            const T sc = s.score[c];
            int rank = 0;
            for (int q = 0; q < C; ++q) {
                const T o = s.score[q];
                rank += (o > sc) || (o == sc && q < c);
            }
            s.keep[c] = rank < Knew;
        }
        engine_sync(cfg);
        if (i < 32) {  // one warp lists kept candidates in order
            int base = 0;
            for (int c0 = 0; c0 < C; c0 += 32) {
                const int c = c0 + i;
                const bool k = (c < C) && s.keep[c];
                const unsigned m = __ballot_sync(0xffffffffu, k);
                if (k) s.src[base + __popc(m & ((1u << i) - 1u))] = (short)c;
                base += __popc(m);
            }
        }
        engine_sync(cfg);
    }
    if (valid) {
        T *row = s.X + i * RS;
#pragma unroll
        for (int k = 0; k < KMAX; ++k) row[k] = r.a[k];
        T dropped = T(0);
        if (!keep_all) {
#pragma unroll
            for (int k = 0; k < KMAX; ++k)
                if (k < Ncur && !s.keep[k]) dropped += fabs(r.a[k]);
            if (newsym && !s.keep[Ncur + new_idx]) dropped += fabs(gamma);
            // in-place forward compaction: src[p] >= p
            for (int p = 0; p < Knew; ++p) {
                const int c = s.src[p];
                row[p] = (c < Ncur) ? row[c] : ((newsym && c - Ncur == new_idx) ? gamma : T(0));
            }
        } else {
            for (int p = Ncur; p < C; ++p) row[p] = (newsym && p - Ncur == new_idx) ? gamma : T(0);
        }
        for (int p = Knew; p < KMAX; ++p) row[p] = T(0);
        row[KMAX] = r.c;
        row[KMAX + 1] = r.xi + dropped;
        row[KMAX + 2] = r.p;
    }
    engine_sync(cfg);
    return Knew;
}

// Positional encoding rows (sin / cos of 2^k pi x) as a nonlinearity layer
// over the 3 input rows: rows 0..2 identity, then per octave 3 sin + 3 cos.
// Each row works on t = 2^k x (+1/2 for cos) in half-turns, which is exact,
// and applies the sin(pi t) rule.
template <typename T, int KMAX, bool PT>
__device__ int posenc_layer(const NetDev &net, const RangeCfg &cfg, const Slot<T> &s, int i, int Ncur) {
    constexpr int RS = RowStride<KMAX>::value;
    const int m = 3 + 6 * net.pe;
    const bool valid = i < m;
    Row<T, KMAX> r;
    T gamma = T(0);
    if (valid) {
        int d = i, k = -1;
        bool is_cos = false;
        if (i >= 3) {
            const int q = i - 3;
            k = q / 6;
            is_cos = (q % 6) >= 3;
            d = q % 3;
        }
        const T sc = (k < 0) ? T(1) : T(1 << k);
        const T sh = is_cos ? T(0.5) : T(0);
        const T *xr = s.X + d * RS;
#pragma unroll
        for (int q = 0; q < KMAX; ++q) r.a[q] = sc * xr[q];
        r.c = sc * xr[KMAX] + sh;
        r.xi = sc * xr[KMAX + 1];
        r.p = sc * xr[KMAX + 2] + sh;
        if (k >= 0) {
            if (cfg.arith == SRA_ARITH_INTERVAL) {
                T lo, hi;
                sinpi_extremes<T>(r.c - r.xi, r.c + r.xi, lo, hi);
                r.c = T(0.5) * (lo + hi);
                r.xi = T(0.5) * (hi - lo);
            } else {
                T rad = T(0);
#pragma unroll
                for (int q = 0; q < KMAX; ++q) rad += fabs(r.a[q]);
                rad += r.xi;
                // The encoding rows are few (6 per octave); their rule runs in
                // FP64 from the exact (c, rad): an FP32 c - rad would lose the
                // width of a narrow range, to which gamma is quadratic.
                double a, b, g;
                linearize_sinpi<double>((double)r.c - (double)rad, (double)r.c + (double)rad, a, b, g);
#pragma unroll
                for (int q = 0; q < KMAX; ++q) r.a[q] *= T(a);
                r.c = T(a * (double)r.c + b);
                r.xi = T(fabs(a)) * r.xi;
                gamma = T(g);
            }
            if (PT) r.p = sinpi_t(r.p);
        }
    }
    engine_sync(cfg);  // every read of the input rows is done
    return condense_and_store<T, KMAX, PT>(r, gamma, valid, i >= 3, i - 3, 6 * net.pe, Ncur, cfg, s, i);
}

// Hidden layers and the output layer. On return (thread 0 of the box) the
// output center, radius and point value are in s.outv[0..2].
template <typename T, int KMAX, bool PT>
__device__ void propagate(const NetDev &net, const RangeCfg &cfg, const Slot<T> &s, int i, int Ncur) {
    constexpr int RS = RowStride<KMAX>::value;
    for (int l = 0; l + 1 < net.L; ++l) {
        const LayerDev &Ld = net.layer[l];
        const bool valid = i < Ld.out;
        Row<T, KMAX> r;
        if (valid) matmul_row<T, KMAX, PT>(Ld, s.X, i, r);
        engine_sync(cfg);  // input rows consumed
        T gamma = T(0);
        if (valid) gamma = activate_row<T, KMAX, PT>(Ld.act, cfg, r);
        const bool nl = Ld.act != SRA_ACT_IDENTITY;
        Ncur = condense_and_store<T, KMAX, PT>(r, gamma, valid, nl, i, nl ? Ld.out : 0, Ncur, cfg, s, i);
    }
    // output layer (1 x in): column sums over input rows, in input order
    const LayerDev &Lo = net.layer[net.L - 1];
    const T *w = Wt_of<T>(Lo);
    constexpr bool COMP = sizeof(T) == 4 && !PT;
    for (int k = i; k < KMAX + 3; k += cfg.H) {
        T acc = T(0);
        const bool is_xi = (k == KMAX + 1);
        if (COMP && k == KMAX) {
            Dot2<T> cd;
            for (int j = 0; j < Lo.in; ++j) cd.add_prod(__ldg(w + j), s.X[j * RS + k]);
            acc = cd.value();
        } else {
            for (int j = 0; j < Lo.in; ++j) {
                const T wj = __ldg(w + j);
                acc = fma(is_xi ? fabs(wj) : wj, s.X[j * RS + k], acc);
            }
        }
        s.outv[k] = acc;
    }
    engine_sync(cfg);
    if (i == 0) {
        const T b0 = __ldg(b_of<T>(Lo));
        T rad = T(0);
        for (int k = 0; k < KMAX; ++k) rad += fabs(s.outv[k]);
        rad += s.outv[KMAX + 1];
        const T y0 = add_rn(s.outv[KMAX], b0);
        const T pv = s.outv[KMAX + 2] + b0;
        s.outv[0] = y0;
        s.outv[1] = rad;
        s.outv[2] = pv;
    }
    engine_sync(cfg);
}

// Initial affine form of a box: x0 = c, X = diag(h), x_inf = 0 (Proc. 1;
// App. A initialisation). Interval arithmetic holds the radius in x_inf.
template <typename T, int KMAX>
__device__ __forceinline__ void init_box_rows(const RangeCfg &cfg, const Slot<T> &s, int i,
                                              const T *c, const T *h, const T *p) {
    constexpr int RS = RowStride<KMAX>::value;
    if (i < 3) {
        T *row = s.X + i * RS;
#pragma unroll
        for (int k = 0; k < KMAX; ++k) row[k] = T(0);
        if (cfg.arith == SRA_ARITH_INTERVAL) row[KMAX + 1] = h[i];
        else {
            row[i] = h[i];
            row[KMAX + 1] = T(0);
        }
        row[KMAX] = c[i];
        row[KMAX + 2] = p ? p[i] : T(0);
    }
}

// ---------------------------------------------------------------------------
// RangeBound (Proc. 1) of group g: boxes g * NB + slot of src, one per slot
// of cfg.H threads. Called by every engine thread of the CTA.
template <typename T, int KMAX>
__device__ __forceinline__ void bound_group(const NetDev &net, const BoxSrc &src, const BoundOut &out,
                                            const RangeCfg &cfg, const Slot<T> &s, int slot, int i,
                                            long long g, long long n) {
    const long long b = g * cfg.NB + slot;
    const bool active = b < n;
    const long long gb = active ? (src.list ? (long long)src.list[b] : b) : 0;

    T c[3] = {T(0), T(0), T(0)}, h[3] = {T(0), T(0), T(0)};
    if (active && i < 3) {
        if (src.kind == SRC_NODES) {
            node_geometry<T>(src, src.nodes[gb], c, h);
        } else {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                c[d] = T(src.centers[gb * 3 + d]);
                h[d] = (src.kind == SRC_BOXES) ? T(src.halfw[gb * 3 + d]) : T(0);
            }
        }
    }
    init_box_rows<T, KMAX>(cfg, s, i, c, h, (const T *)nullptr);
    int Ncur = (cfg.arith == SRA_ARITH_INTERVAL) ? 0 : 3;
    engine_sync(cfg);
    if (net.pe) Ncur = posenc_layer<T, KMAX, false>(net, cfg, s, i, Ncur);
    propagate<T, KMAX, false>(net, cfg, s, i, Ncur);
    if (i == 0 && active) {
        const T y0 = s.outv[0], rad = s.outv[1];
        const T lo = y0 - rad, hi = y0 + rad;
        const int k = classify_range(lo, hi);
        if (out.lo) out.lo[gb] = (float)lo;
        if (out.hi) out.hi[gb] = (float)hi;
        if (out.cls) out.cls[gb] = (uint8_t)k;
        if (out.recheck_counter) atomicAdd(out.recheck_counter, 1ull);
        if (out.flag_list) {  // either end of the range near zero: FP64 decides
            const T band = T(out.band) * (fabs(y0) + rad);
            if (fabs(lo) <= band || fabs(hi) <= band)
                out.flag_list[atomicAdd(out.flag_count, 1)] = (int)gb;
        }
    }
    engine_sync(cfg);  // outv / X reuse by the next group
}

// Bound kernel: RangeBound (Proc. 1) for boxes, tree nodes or points.
template <typename T, int KMAX>
__global__ void __launch_bounds__(MaxThreads<T, KMAX>::value, MinBlocks<T, KMAX>::value)
bound_kernel(NetDev net, BoxSrc src, BoundOut out, RangeCfg cfg) {
    extern __shared__ __align__(16) char smem[];
    const int slot = threadIdx.x / cfg.H, i = threadIdx.x - slot * cfg.H;
    const Slot<T> s = carve<T>(smem, slot, cfg);
    long long n = src.n;
    if (src.list) n = *src.list_count;
    // grid-stride over groups of NB boxes (CTA-uniform trip count)
    for (long long g = blockIdx.x; g * cfg.NB < n; g += gridDim.x)
        bound_group<T, KMAX>(net, src, out, cfg, s, slot, i, g, n);
}

// Persistent RangeBound over the frontiers of many networks (one launch per
// noise-column bound KMAX): each CTA takes the next chunk from a global
// counter, finds its segment and runs that network's layout with the first
// NB * H threads; the others wait for the next chunk. Segments are listed
// heaviest first, so the long chunks start early.
template <typename T, int KMAX>
__global__ void __launch_bounds__(MaxThreads<T, KMAX>::value)
multi_bound_kernel(const BatchSegDev *segs, const int *order, int nseg, long long nchunks,
                   unsigned long long *next) {
    extern __shared__ __align__(16) char smem[];
    __shared__ long long s_chunk;
    for (;;) {
        if (threadIdx.x == 0) s_chunk = (long long)atomicAdd(next, 1ull);
        __syncthreads();
        const long long c = s_chunk;
        __syncthreads();  // read before thread 0 takes the next chunk
        if (c >= nchunks) break;
        int lo = 0, hi = nseg - 1;  // last segment whose first chunk is <= c
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (segs[order[mid]].chunk0 <= c) lo = mid;
            else hi = mid - 1;
        }
        const BatchSegDev &S = segs[order[lo]];
        const RangeCfg cfg = S.cfg;
        if ((int)threadIdx.x < cfg.threads) {
            const int slot = threadIdx.x / cfg.H, i = threadIdx.x - slot * cfg.H;
            const Slot<T> s = carve<T>(smem, slot, cfg);
            bound_group<T, KMAX>(S.net, S.src, S.out, cfg, s, slot, i, c - S.chunk0, S.src.n);
        }
    }
}

// ---------------------------------------------------------------------------
// Ray kernel: CastRay (Proc. 2), persistent over ray slots. Each iteration a
// slot bounds the segment [t, t+sigma] (c = p + (t + sigma/2) r,
// v = (sigma/2) r) and evaluates f(p + (t + delta) r) in the same pass.
// With rp.list the slots take the listed rays only (the FP64 re-check);
// with rp.flag_list a ray that met a near-zero decision is listed when it ends.
template <typename T, int KMAX>
__global__ void __launch_bounds__(MaxThreads<T, KMAX>::value)
ray_kernel(NetDev net, RayParams rp, RangeCfg cfg) {
    extern __shared__ __align__(16) char smem[];
    const int slot = threadIdx.x / cfg.H, i = threadIdx.x - slot * cfg.H;
    const Slot<T> s = carve<T>(smem, slot, cfg);
    RaySlotState<T> *st = (RaySlotState<T> *)s.ray;
    if (i == 0) st->idx = -1;
    __syncthreads();
    for (;;) {
        if (i == 0 && st->idx < 0) {
            const unsigned long long k = atomicAdd(rp.next, 1ull);
            const long long n_rays = rp.list ? (long long)*rp.list_count : rp.n;
            if ((long long)k < n_rays) {
                const long long q = rp.list ? (long long)rp.list[k] : (long long)k;
                st->idx = q;
                st->t = rp.t_start ? T(rp.t_start[q]) : T(0);
                st->sigma = rp.sigma_start ? T(rp.sigma_start[q]) : T(rp.sigma0);
                st->iters = 0;
                st->f0pos = rp.f0[q] >= 0.f;
                st->live = 1;
                st->flag = 0;
                if (rp.recheck_counter) atomicAdd(rp.recheck_counter, 1ull);
            } else {
                st->live = 0;
            }
        }
        __syncthreads();
        const bool live = st->live != 0;
        if (!__syncthreads_or(live)) break;
        T c[3] = {T(0), T(0), T(0)}, h[3] = {T(0), T(0), T(0)}, pc[3] = {T(0), T(0), T(0)};
        if (live && i < 3) {
            const long long q = st->idx;
            const T p = T(rp.origins[q * 3 + i]), r = T(rp.dirs[q * 3 + i]);
            const T t = T(st->t), sg = T(st->sigma);
            c[i] = p + (t + sg / T(2)) * r;
            h[i] = (sg / T(2)) * r;
            pc[i] = p + (t + T(rp.delta)) * r;
        }
        // 1-d box: one symbol whose column is v = (sigma/2) r
        if (i < 3) {
            constexpr int RS = RowStride<KMAX>::value;
            T *row = s.X + i * RS;
#pragma unroll
            for (int k = 0; k < KMAX; ++k) row[k] = T(0);
            if (cfg.arith == SRA_ARITH_INTERVAL) row[KMAX + 1] = fabs(h[i]);
            else {
                row[0] = h[i];
                row[KMAX + 1] = T(0);
            }
            row[KMAX] = c[i];
            row[KMAX + 2] = pc[i];
        }
        int Ncur = (cfg.arith == SRA_ARITH_INTERVAL) ? 0 : 1;
        __syncthreads();
        if (net.pe) Ncur = posenc_layer<T, KMAX, true>(net, cfg, s, i, Ncur);
        propagate<T, KMAX, true>(net, cfg, s, i, Ncur);
        if (i == 0 && live) {
            const T y0 = s.outv[0], rad = s.outv[1], fc = s.outv[2];
            const long long q = st->idx;
            st->iters += 1;
            if (rp.flag_list && near_zero_step<T>(y0, rad, rp.band)) st->flag = 1;
            bool done = false;
            float result = 0.f;
            if ((fc >= T(0)) != (st->f0pos != 0)) {  // DifferentSigns at t + delta
                done = true;
                result = st->t;
            } else {
                const int k = classify_range(y0 - rad, y0 + rad);
                T sstar;
                if (k != SRA_UNKNOWN) { sstar = st->sigma; st->sigma *= T(rp.eta_plus); }
                else { sstar = T(0); st->sigma *= T(rp.eta_minus); }
                st->t += fmax(T(rp.safety) * sstar, T(rp.delta));
                if (!(st->t < T(rp.t_max))) { done = true; result = INFINITY; }
            }
            if (!done && st->iters >= rp.max_iters) { done = true; result = NAN; }
            if (done) {
                rp.t_hit[q] = result;
                if (rp.iters) rp.iters[q] = st->iters;
                if (rp.flag_list && st->flag) rp.flag_list[atomicAdd(rp.flag_count, 1)] = (int)q;
                st->idx = -1;
            }
        }
        __syncthreads();
    }
}

}  // namespace sra
