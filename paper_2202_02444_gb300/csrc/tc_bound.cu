// BF16-sound RangeBound on the tensor cores (tcgen05 + TMEM + TMA).
//
// Network shape served: 3 -> H -> ... -> H -> 1 ReLU MLP (H = 128 or 256),
// affine-truncate with K = 64 kept noise symbols (Sec. 3.3), the dense layers
// of App. A Table "affine_update_rules" on tensor cores. One persistent CTA per
// SM runs the whole network for a tile of NB = 2 boxes with 2H threads: thread
// group g (H threads, one per neuron) owns box g, so the two boxes' SIMT work
// runs concurrently. The per-box affine state never leaves the SM:
//   * operand B of every hidden layer: the 2 x 64 noise columns (BF16) and a
//     16-column chunk holding each box's center as a BF16 hi/lo pair, written
//     by the epilogue threads in the K-major 128-byte-swizzled layout;
//   * operand A: W as BF16 hi + lo (W = W_b + W_r + rho, |rho| <= u_b^2 |W|),
//     streamed per 64-wide K slice by TMA into a two-stage ring;
//   * D = (W_b + W_r) [X | c_hi c_lo] accumulates in TMEM (FP32);
//   * x_inf' >= |W| v is accumulated by the SIMT threads from the resident
//     W_b slice with round-up FMAs (|W| <= |W_b| / (1 - u_b));
//   * epilogue, one thread per neuron (tcgen05.ld of its TMEM row): outward
//     rounded range, the ReLU rule, truncation to the 64 largest columns, and
//     the a-priori rounding radius of every FP operation folded into x_inf.
// The first layer (3 inputs) and the output layer (1 output) run on the SIMT
// cores with directed rounding. Every bounded wait that runs out writes a
// status word and the CTA leaves through its normal exit (TMEM freed).
#include <cuda_bf16.h>

#include "sra_common.cuh"
#include "tc_bound.h"
#include "tc_ptx.cuh"

namespace sra {
namespace tc {

constexpr int NB = 2;        // boxes per tile (one thread group each)
constexpr int KT = 64;       // kept noise symbols per box
constexpr int NA = NB * KT;  // noise columns per tile (MMA N)
constexpr int NCC = 16;      // center-chunk columns (MMA N)
constexpr int NPART = 4;     // partial sums per output-layer dot product
constexpr uint32_t kSpin = 1u << 22;

template <int H> struct Layout {
    static constexpr int MT = H / 128;   // M tiles per layer
    static constexpr int S = H / 64;     // K slices per layer
    static constexpr int TILE = 128 * 128;                  // bytes of one 128 x 64 bf16 tile
    static constexpr int STAGE = 2 * MT * TILE;             // W_b and W_r tiles of one K slice
    static constexpr int W_OFF = 0;
    static constexpr int XA_OFF = 2 * STAGE;
    static constexpr int XA_SLICE = NA * 128;
    static constexpr int XC_OFF = XA_OFF + S * XA_SLICE;
    static constexpr int XC_SLICE = NCC * 128;
    static constexpr int F_OFF = XC_OFF + S * XC_SLICE;
    static constexpr int NCAND = KT + H;
    static constexpr int V_OFF = F_OFF;                              // v[NB][H]
    static constexpr int XR_OFF = V_OFF + NB * H * 4;                // xr[NB][H]
    static constexpr int SC_OFF = XR_OFF + NB * H * 4;               // score[NB][NCAND]
    static constexpr int PART_OFF = SC_OFF + NB * NCAND * 4;         // part[NB][H/32][KT]
    static constexpr int OUT_OFF = PART_OFF + NB * (H / 32) * KT * 4;  // Y,E [NB][NPART][KT+2]
    static constexpr int WOUT_OFF = OUT_OFF + 2 * NB * NPART * (KT + 2) * 4;  // wout[H]
    static constexpr int BOX_OFF = WOUT_OFF + H * 4;                 // box c/h [NB][8]
    static constexpr int HIST_OFF = BOX_OFF + NB * 8 * 4;            // hist[NB][256]
    static constexpr int KEEP_OFF = HIST_OFF + NB * 256 * 4;         // keep[NB][NCAND]
    static constexpr int POS_OFF = ((KEEP_OFF + NB * NCAND) + 15) & ~15;  // pos[NB][NCAND]
    static constexpr int NEW_OFF = ((POS_OFF + NB * NCAND * 2) + 15) & ~15; // newlist[NB][KT]
    static constexpr int BAR_OFF = ((NEW_OFF + NB * KT * 4) + 15) & ~15;   // 5 mbarriers
    static constexpr int MISC_OFF = BAR_OFF + 64;  // tmem slot, abort, nnew[NB], sel[NB][2]
    static constexpr int BYTES = MISC_OFF + 64;
    static constexpr int ALLOC = BYTES + 1024;     // + alignment slack
};

// ---- directed-rounding helpers ----------------------------------------------
__device__ __forceinline__ float ru_add(float a, float b) { return __fadd_ru(a, b); }
__device__ __forceinline__ float rd_add(float a, float b) { return __fadd_rd(a, b); }
__device__ __forceinline__ float ru_mul(float a, float b) { return __fmul_ru(a, b); }
__device__ __forceinline__ float ru_fma(float a, float b, float c) { return __fmaf_ru(a, b, c); }

__device__ __forceinline__ float bf16_ru(float x) {  // smallest bf16 >= x (x >= 0)
    return __bfloat162float(__float2bfloat16_ru(x));
}

// Named barrier of one thread group (ids 1 and 2; 0 is __syncthreads).
__device__ __forceinline__ void group_sync(int g, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(nthreads) : "memory");
}

struct Ctx {
    unsigned char *smem;
    int tid, g, i, wg, lane;  // thread, group (= box), neuron, warp in group, lane
    uint32_t tmem;
    uint64_t *bars;  // [0,1] full, [2,3] empty, [4] acc
    int *abort_flag;
};

__device__ __forceinline__ void fail(const Ctx &x, const TcParams &p, int code) {
    *x.abort_flag = 1;
    atomicExch(p.status, code);
}

// Outward-rounded range of one row, the ReLU rule and its application.
// Scales a in place and returns alpha (the caller may rescale a reloaded row
// bit-identically), gamma, the new center c2 and x_inf.
template <bool SOUND>
__device__ __forceinline__ void relu_apply(float (&a)[KT], float c, float &xinf, float &c2, float &al,
                                           float &ga, float u_b2u) {
    float sa = 0.f;
#pragma unroll
    for (int k = 0; k < KT; ++k) sa = ru_add(sa, fabsf(a[k]));
    const float rad = ru_add(sa, xinf);
    const float lo = rd_add(c, -rad), hi = ru_add(c, rad);
    float be;
    if (hi <= 0.f) { al = 0.f; be = 0.f; ga = 0.f; }
    else if (lo >= 0.f) { al = 1.f; be = 0.f; ga = 0.f; }
    else {
        // any slope in [0,1] is valid: g(x) = ReLU(x) - al x ranges over
        // [0, max(-al lo, hi (1 - al))] on [lo, hi]
        al = fminf(fmaxf(hi / (hi - lo), 0.f), 1.f);
        const float m1 = __fmul_ru(al, -lo);
        const float m2 = __fmul_ru(hi, __fadd_ru(1.f, -al));
        const float M = fmaxf(m1, m2);
        be = 0.5f * M;  // exact halving
        ga = be;
    }
#pragma unroll
    for (int k = 0; k < KT; ++k) a[k] = al * a[k];
    c2 = fmaf(al, c, be);
    // |al| x_inf, the rounding of c2, and of every al * a (and its later bf16
    // rounding) as u_b + 2u relative of sum |a|
    float xi = __fmul_ru(al, xinf);
    if (SOUND) {
        xi = ru_fma(fabsf(c2), 1.1920929e-07f, xi);  // one rounding: <= 2^-23 |c2|
        xi = ru_fma(__fmul_ru(al, sa), u_b2u, xi);
    }
    xinf = xi;
}

// Truncate (Sec. 3.3) the group's box after the activation and write its
// operand rows. Thread i of group g holds the scaled old columns a[0..Ncur)
// of neuron i, its new symbol gamma and x_inf. The column norms consume a;
// `reload` rebuilds it bit-identically for the write-back.
template <int H, bool SOUND, typename Reload>
__device__ void truncate_and_store(const Ctx &x, const TcParams &p, float (&a)[KT], int Ncur, float gamma,
                                   float xinf, float c2, Reload reload) {
    using Lt = Layout<H>;
    const int g = x.g, i = x.i, lane = x.lane, wg = x.wg;
    float *score = (float *)(x.smem + Lt::SC_OFF) + g * Lt::NCAND;
    float *part = (float *)(x.smem + Lt::PART_OFF) + g * (H / 32) * KT;
    uint8_t *keep = x.smem + Lt::KEEP_OFF + g * Lt::NCAND;
    short *pos = (short *)(x.smem + Lt::POS_OFF) + g * Lt::NCAND;
    int *newlist = (int *)(x.smem + Lt::NEW_OFF) + g * KT;
    int *hist = (int *)(x.smem + Lt::HIST_OFF) + g * 256;
    int *nnew_slot = (int *)(x.smem + Lt::MISC_OFF + 16) + g;
    uint32_t *sel = (uint32_t *)(x.smem + Lt::MISC_OFF + 32) + 2 * g;  // [0] prefix, [1] need
    const int C = Ncur + H;
    // column L1 norms of the old columns over the H neurons: butterfly
    // reduce-scatter inside the warp (lane l ends with 2 column sums); a is
    // consumed here
#pragma unroll
    for (int k = 0; k < KT; ++k) a[k] = fabsf(a[k]);
#pragma unroll
    for (int half = KT / 2, o = 16; o >= 1; half >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < half; ++k) {
            const float send = up ? a[k] : a[k + half];
            const float keepv = up ? a[k + half] : a[k];
            a[k] = keepv + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    {
        const int col = ((lane & 16) ? 32 : 0) + ((lane & 8) ? 16 : 0) + ((lane & 4) ? 8 : 0) +
                        ((lane & 2) ? 4 : 0) + ((lane & 1) ? 2 : 0);
        part[wg * KT + col] = a[0];
        part[wg * KT + col + 1] = a[1];
    }
    score[Ncur + i] = gamma;  // the new symbol of neuron i (one nonzero entry)
    if (i == 0) { sel[0] = 0u; sel[1] = KT; }
    group_sync(g, H);
    if (i < Ncur) {
        float v = 0.f;
        for (int w = 0; w < H / 32; ++w) v += part[w * KT + i];
        score[i] = v;
    }
    // exact top-KT by radix select on the score bits (non-negative floats
    // order like their bit patterns), 8 bits per pass
    uint32_t pmask = 0u;
#pragma unroll 1
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int e = i; e < 256; e += H) hist[e] = 0;
        group_sync(g, H);
        const uint32_t prefix = sel[0];
        for (int c = i; c < C; c += H) {
            const uint32_t key = __float_as_uint(score[c]);
            if ((key & pmask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1);
        }
        group_sync(g, H);
        if (wg == 0) {
            // lane l owns digits 255-8l .. 248-8l (descending)
            int cnt[8], tot = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) { cnt[q] = hist[255 - 8 * lane - q]; tot += cnt[q]; }
            int incl = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const int need = (int)sel[1];
            const unsigned hit = __ballot_sync(0xffffffffu, incl >= need);
            const int L = __ffs(hit) - 1;
            if (lane == L) {
                int above = incl - tot, d = 255 - 8 * lane;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (above + cnt[q] >= need) { d = 255 - 8 * lane - q; break; }
                    above += cnt[q];
                }
                sel[0] = prefix | ((uint32_t)d << shift);
                sel[1] = (uint32_t)(need - above);
            }
        }
        pmask |= 255u << shift;
        group_sync(g, H);
    }
    if (wg == 0) {  // keep flags, positions, kept new symbols, in candidate order
        const uint32_t T = sel[0];
        int take_eq = (int)sel[1];
        const unsigned below = (1u << lane) - 1u;
        int base = 0;
        for (int c0 = 0; c0 < C; c0 += 32) {
            const int c = c0 + lane;
            const uint32_t key = (c < C) ? __float_as_uint(score[c]) : 0u;
            const bool gt = (c < C) && key > T, eq = (c < C) && key == T;
            const unsigned meq = __ballot_sync(0xffffffffu, eq);
            const bool k = gt || (eq && __popc(meq & below) < take_eq);
            take_eq -= min(__popc(meq), max(take_eq, 0));
            const unsigned m = __ballot_sync(0xffffffffu, k);
            if (c < C) {
                keep[c] = k;
                pos[c] = k ? (short)(base + __popc(m & below)) : (short)-1;
            }
            base += __popc(m);
        }
        __syncwarp();
        int cnt = 0;  // kept new symbols as (position, neuron)
        for (int c0 = Ncur; c0 < C; c0 += 32) {
            const int c = c0 + lane;
            const bool k = (c < C) && keep[c];
            const unsigned m = __ballot_sync(0xffffffffu, k);
            if (k) newlist[cnt + __popc(m & below)] = (int)pos[c] | ((c - Ncur) << 16);
            cnt += __popc(m);
        }
        if (lane == 0) *nnew_slot = cnt;
    }
    reload(a);  // the scaled old columns again (overlaps the warp-0 listing)
    group_sync(g, H);
    const int nnew = *nnew_slot;
    // dropped magnitudes to x_inf; kept values to operand B (row n = g*KT + pos)
    unsigned char *XA = x.smem + Lt::XA_OFF + (i >> 6) * Lt::XA_SLICE;
    const uint32_t kk = (uint32_t)(i & 63);
    float dropped = 0.f, arow = 0.f;
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        if (k < Ncur) {
            const int pp = pos[k];
            if (pp < 0) {
                dropped = ru_add(dropped, fabsf(a[k]));
            } else {
                const __nv_bfloat16 v = __float2bfloat16_rn(a[k]);
                *(__nv_bfloat16 *)(XA + ptx::sw128_offset((uint32_t)(g * KT + pp), kk)) = v;
                arow = ru_add(arow, fabsf(__bfloat162float(v)));
            }
        }
    }
    if (pos[Ncur + i] < 0) dropped = ru_add(dropped, gamma);
    for (int q = 0; q < nnew; ++q) {
        const int e = newlist[q];
        const int pp = e & 0xffff, neuron = e >> 16;
        float v = 0.f;
        if (neuron == i) {
            v = SOUND ? bf16_ru(gamma) : __bfloat162float(__float2bfloat16_rn(gamma));
            arow = ru_add(arow, v);
        }
        *(__nv_bfloat16 *)(XA + ptx::sw128_offset((uint32_t)(g * KT + pp), kk)) = __float2bfloat16_rn(v);
    }
    xinf = ru_add(xinf, dropped);
    // center as a bf16 hi/lo pair; the residual is exact in fp32
    const __nv_bfloat16 chi = __float2bfloat16_rn(c2);
    const float rem = c2 - __bfloat162float(chi);
    const __nv_bfloat16 clo = __float2bfloat16_rn(rem);
    const float rc = rem - __bfloat162float(clo);
    unsigned char *XC = x.smem + Lt::XC_OFF + (i >> 6) * Lt::XC_SLICE;
    *(__nv_bfloat16 *)(XC + ptx::sw128_offset((uint32_t)(2 * g), kk)) = chi;
    *(__nv_bfloat16 *)(XC + ptx::sw128_offset((uint32_t)(2 * g + 1), kk)) = clo;
    const float xr = SOUND ? ru_add(xinf, fabsf(rc)) : xinf;
    ((float *)(x.smem + Lt::XR_OFF))[g * H + i] = xr;
    if (SOUND) {
        const float mag = ru_add(ru_add(arow, fabsf(__bfloat162float(chi))), fabsf(__bfloat162float(clo)));
        ((float *)(x.smem + Lt::V_OFF))[g * H + i] = ru_fma(p.rho1, mag, xr);
    } else {
        ((float *)(x.smem + Lt::V_OFF))[g * H + i] = xr;
    }
}

template <int H, bool SOUND>
__global__ void __launch_bounds__(2 * H, 1) tc_bound_kernel(const __grid_constant__ TcParams p, BoxSrc src,
                                                            BoundOut out) {
    using Lt = Layout<H>;
    constexpr int NT = 2 * H;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    Ctx x;
    x.smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    x.tid = threadIdx.x;
    x.g = x.tid / H;
    x.i = x.tid - x.g * H;
    x.wg = x.i >> 5;
    x.lane = x.tid & 31;
    x.bars = (uint64_t *)(x.smem + Lt::BAR_OFF);
    uint32_t *tmem_slot = (uint32_t *)(x.smem + Lt::MISC_OFF);
    x.abort_flag = (int *)(x.smem + Lt::MISC_OFF + 4);
    const int tid = x.tid, g = x.g, i = x.i;
    const int warp = tid >> 5;
    if (tid == 0) {
        ptx::mbar_init(&x.bars[0], 1);
        ptx::mbar_init(&x.bars[1], 1);
        ptx::mbar_init(&x.bars[2], 1 + NT / 32);
        ptx::mbar_init(&x.bars[3], 1 + NT / 32);
        ptx::mbar_init(&x.bars[4], 1);
        ptx::fence_mbar_init();
        *x.abort_flag = 0;
    }
    // zero the center chunk once (rows beyond 2*NB stay zero); output weights to smem
    for (int e = tid; e < Lt::S * Lt::XC_SLICE / 4; e += NT) ((uint32_t *)(x.smem + Lt::XC_OFF))[e] = 0u;
    float *wout = (float *)(x.smem + Lt::WOUT_OFF);
    for (int e = tid; e < H; e += NT) wout[e] = p.wout[e];
    if (warp == 0) ptx::tmem_alloc(tmem_slot, 512);
    __syncthreads();
    ptx::tc_fence_after();
    x.tmem = *tmem_slot;
    const uint32_t tl = x.tmem + ((uint32_t)((warp & 3) * 32) << 16);  // this warp's TMEM lanes
    const int m_of_thread = i >> 7;
    float *boxf = (float *)(x.smem + Lt::BOX_OFF);
    const long long n = src.n;
    const long long ntiles = (n + NB - 1) / NB;
    uint32_t gring = 0, accn = 0;

    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        if (*x.abort_flag) break;
        const long long bi = t * NB + g;
        // ---- the group's box ----------------------------------------------
        if (i == 0) {
            float c[3] = {0.f, 0.f, 0.f}, h[3] = {0.f, 0.f, 0.f};
            if (bi < n) {
                if (src.kind == SRC_NODES) node_geometry<float>(src, src.nodes[bi], c, h);
                else
                    for (int d = 0; d < 3; ++d) {
                        c[d] = src.centers[bi * 3 + d];
                        h[d] = src.halfw[bi * 3 + d];
                    }
            }
            for (int d = 0; d < 3; ++d) {
                boxf[g * 8 + d] = c[d];
                boxf[g * 8 + 3 + d] = h[d];
            }
        }
        group_sync(g, H);
        // ---- first layer (3 -> H) on the SIMT cores ----------------------------
        {
            float a[KT];
#pragma unroll
            for (int k = 0; k < KT; ++k) a[k] = 0.f;
            const float w0[3] = {p.W0[i * 3], p.W0[i * 3 + 1], p.W0[i * 3 + 2]};
            const float b0 = p.b[0][i];
            const float hb[3] = {boxf[g * 8 + 3], boxf[g * 8 + 4], boxf[g * 8 + 5]};
            float c = b0, cm = fabsf(b0), am = 0.f;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float cd = boxf[g * 8 + d];
                c = fmaf(w0[d], cd, c);
                cm = ru_fma(fabsf(w0[d]), fabsf(cd), cm);
                a[d] = w0[d] * hb[d];
                am = ru_add(am, fabsf(a[d]));
            }
            float xinf = 0.f;
            if (SOUND) {
                xinf = ru_mul(cm, 2.3841858e-07f);  // 3-FMA sum: gamma_3 < 2^-22
                xinf = ru_fma(am, 1.1920929e-07f, xinf);  // one rounding per product
            }
            float c2, al, ga;
            relu_apply<SOUND>(a, c, xinf, c2, al, ga, p.ub2u);
            truncate_and_store<H, SOUND>(x, p, a, 3, ga, xinf, c2, [&](float (&r)[KT]) {
#pragma unroll
                for (int k = 0; k < KT; ++k) r[k] = 0.f;
#pragma unroll
                for (int d = 0; d < 3; ++d) r[d] = al * (w0[d] * hb[d]);
            });
        }
        // ---- hidden layers on the tensor cores ---------------------------------
        for (int l = 1; l + 1 < p.L; ++l) {
            ptx::fence_proxy_async();  // operand writes -> async proxy
            ptx::tc_fence_before();    // previous TMEM reads done before new MMAs
            __syncthreads();
            if (*x.abort_flag) break;
            float xacc = 0.f;
            const CUtensorMap *mb = &p.wb[l - 1], *mr = &p.wr[l - 1];
            const uint32_t g0 = gring;
            auto load_slice = [&](int s) {  // thread 0
                const uint32_t gg = g0 + (uint32_t)s, st = gg & 1u;
                if (!ptx::mbar_wait(&x.bars[2 + st], ((gg >> 1) & 1u) ^ 1u, kSpin)) { fail(x, p, 3); return; }
                unsigned char *base = x.smem + Lt::W_OFF + st * Lt::STAGE;
                ptx::mbar_arrive_expect_tx(&x.bars[st], Lt::STAGE);
                for (int m = 0; m < Lt::MT; ++m) {
                    ptx::tma_load_2d(base + m * Lt::TILE, mb, s * 64, m * 128, &x.bars[st]);
                    ptx::tma_load_2d(base + (Lt::MT + m) * Lt::TILE, mr, s * 64, m * 128, &x.bars[st]);
                }
            };
            if (tid == 0) {
                load_slice(0);
                if (Lt::S > 1) load_slice(1);
            }
            const float *vg = (const float *)(x.smem + Lt::V_OFF) + g * H;
            for (int s = 0; s < Lt::S; ++s) {
                const uint32_t gg = g0 + (uint32_t)s, st = gg & 1u, par = (gg >> 1) & 1u;
                if (!ptx::mbar_wait(&x.bars[st], par, kSpin)) fail(x, p, 4);
                unsigned char *base = x.smem + Lt::W_OFF + st * Lt::STAGE;
                if (tid == 0 && !*x.abort_flag) {
                    ptx::tc_fence_after();
                    const uint32_t ia = ptx::idesc_bf16(128, NA), ic = ptx::idesc_bf16(128, NCC);
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint32_t acc = (s | ks) ? 1u : 0u;
                        const uint64_t bA =
                            ptx::desc_kmajor_sw128(ptx::smem_u32(x.smem + Lt::XA_OFF + s * Lt::XA_SLICE)) + 2 * ks;
                        const uint64_t bC =
                            ptx::desc_kmajor_sw128(ptx::smem_u32(x.smem + Lt::XC_OFF + s * Lt::XC_SLICE)) + 2 * ks;
                        for (int m = 0; m < Lt::MT; ++m) {
                            const uint64_t aB = ptx::desc_kmajor_sw128(ptx::smem_u32(base + m * Lt::TILE)) + 2 * ks;
                            const uint64_t aR =
                                ptx::desc_kmajor_sw128(ptx::smem_u32(base + (Lt::MT + m) * Lt::TILE)) + 2 * ks;
                            ptx::mma_bf16(x.tmem + m * NA, aB, bA, ia, acc);
                            ptx::mma_bf16(x.tmem + m * NA, aR, bA, ia, 1u);
                            ptx::mma_bf16(x.tmem + Lt::MT * NA + m * NCC, aB, bC, ic, acc);
                            ptx::mma_bf16(x.tmem + Lt::MT * NA + m * NCC, aR, bC, ic, 1u);
                        }
                    }
                    ptx::mma_commit(&x.bars[2 + st]);
                    if (s + 1 == Lt::S) ptx::mma_commit(&x.bars[4]);
                }
                // x_inf' += |W_b| v of the group's box from the resident slice
                {
                    const int r = i & 127;
                    const unsigned char *row = base + m_of_thread * Lt::TILE + r * 128;
#pragma unroll
                    for (int ch = 0; ch < 8; ++ch) {
                        const uint4 q = *(const uint4 *)(row + (((ch ^ (r & 7)) & 7) << 4));
                        const __nv_bfloat162 *w2 = (const __nv_bfloat162 *)&q;
                        const float4 va = *(const float4 *)(vg + s * 64 + ch * 8);
                        const float4 vb = *(const float4 *)(vg + s * 64 + ch * 8 + 4);
                        const float vv[8] = {va.x, va.y, va.z, va.w, vb.x, vb.y, vb.z, vb.w};
#pragma unroll
                        for (int e2 = 0; e2 < 4; ++e2) {
                            const float2 wf = __bfloat1622float2(w2[e2]);
                            xacc = ru_fma(fabsf(wf.x), vv[2 * e2], xacc);
                            xacc = ru_fma(fabsf(wf.y), vv[2 * e2 + 1], xacc);
                        }
                    }
                }
                __syncwarp();
                if (x.lane == 0) ptx::mbar_arrive(&x.bars[2 + st]);
                if (tid == 0 && s + 2 < Lt::S && !*x.abort_flag) load_slice(s + 2);
            }
            gring = g0 + Lt::S;
            if (!ptx::mbar_wait(&x.bars[4], accn & 1u, kSpin)) fail(x, p, 5);
            accn++;
            ptx::tc_fence_after();
            __syncthreads();  // every operand read of this layer is done
            if (*x.abort_flag) break;
            // ---- epilogue of the group's box -------------------------------
            const float bias = p.b[l][i];
            const uint32_t colA = tl + m_of_thread * NA + g * KT;
            float a[KT];
#pragma unroll
            for (int q = 0; q < KT / 16; ++q) ptx::tmem_ld16(colA + q * 16, a + q * 16);
            float cc[2];
            ptx::tmem_ld2(tl + Lt::MT * NA + m_of_thread * NCC + 2 * g, cc);
            ptx::tmem_wait_ld();
            // center: D(c_hi) + D(c_lo) + bias, each add rounded once
            const float c = (cc[0] + cc[1]) + bias;
            float xinf;
            if (SOUND) {
                xinf = ru_mul(xacc, p.kappa);
                // the two adds: u |cc0 + cc1| + u |c| <= 2^-23 (2 |c| + |bias|)
                xinf = ru_fma(ru_add(2.f * fabsf(c), fabsf(bias)), 1.1920929e-07f, xinf);
            } else {
                xinf = xacc;
            }
            float c2, al, ga;
            relu_apply<SOUND>(a, c, xinf, c2, al, ga, p.ub2u);
            truncate_and_store<H, SOUND>(x, p, a, KT, ga, xinf, c2, [&](float (&r)[KT]) {
#pragma unroll
                for (int q = 0; q < KT / 16; ++q) ptx::tmem_ld16(colA + q * 16, r + q * 16);
                ptx::tmem_wait_ld();
#pragma unroll
                for (int k = 0; k < KT; ++k) r[k] = al * r[k];
            });
        }
        __syncthreads();
        if (*x.abort_flag) break;
        // ---- output layer (H -> 1) on the SIMT cores ------------------------------
        {
            float *Y = (float *)(x.smem + Lt::OUT_OFF) + g * NPART * (KT + 2);  // [NPART][KT+2]
            float *E = Y + NB * NPART * (KT + 2);
            // NPART x KT partial dot products of 64 inputs each; thread i
            // takes column k = i % 64 over input slice i / 64
            for (int tt = i; tt < NPART * KT; tt += H) {
                const int k = tt % KT, pp = tt / KT;
                float acc = 0.f, err = 0.f;
                for (int s = pp; s < Lt::S; s += NPART) {
                    const unsigned char *XA = x.smem + Lt::XA_OFF + s * Lt::XA_SLICE;
                    const uint32_t row = (uint32_t)(g * KT + k);
#pragma unroll
                    for (int ch = 0; ch < 8; ++ch) {
                        const uint4 q = *(const uint4 *)(XA + row * 128 + (((ch ^ (row & 7)) & 7) << 4));
                        const __nv_bfloat162 *v2 = (const __nv_bfloat162 *)&q;
#pragma unroll
                        for (int e2 = 0; e2 < 4; ++e2) {
                            const float2 vf = __bfloat1622float2(v2[e2]);
                            const float w0 = wout[s * 64 + ch * 8 + 2 * e2], w1 = wout[s * 64 + ch * 8 + 2 * e2 + 1];
                            acc = fmaf(w0, vf.x, acc);
                            acc = fmaf(w1, vf.y, acc);
                            err = ru_fma(fabsf(w0), fabsf(vf.x), err);
                            err = ru_fma(fabsf(w1), fabsf(vf.y), err);
                        }
                    }
                }
                Y[pp * (KT + 2) + k] = acc;
                E[pp * (KT + 2) + k] = err;
            }
            if (i < 2 * NPART) {  // center (c_hi + c_lo rows) and x_inf parts
                const int pp = i % NPART;
                float acc = 0.f, err = 0.f;
                if (i < NPART) {
                    for (int s = pp; s < Lt::S; s += NPART) {
                        const unsigned char *XC = x.smem + Lt::XC_OFF + s * Lt::XC_SLICE;
                        for (int j = 0; j < 64; ++j) {
                            const float w = wout[s * 64 + j];
                            const float hi = __bfloat162float(
                                *(const __nv_bfloat16 *)(XC + ptx::sw128_offset((uint32_t)(2 * g), (uint32_t)j)));
                            const float lo = __bfloat162float(
                                *(const __nv_bfloat16 *)(XC + ptx::sw128_offset((uint32_t)(2 * g + 1), (uint32_t)j)));
                            acc = fmaf(w, hi, acc);
                            acc = fmaf(w, lo, acc);
                            err = ru_fma(fabsf(w), ru_add(fabsf(hi), fabsf(lo)), err);
                        }
                    }
                    Y[pp * (KT + 2) + KT] = acc;
                    E[pp * (KT + 2) + KT] = err;
                } else {
                    const float *xr = (const float *)(x.smem + Lt::XR_OFF) + g * H;
                    for (int j = pp * (H / NPART); j < (pp + 1) * (H / NPART); ++j) acc = ru_fma(fabsf(wout[j]), xr[j], acc);
                    Y[pp * (KT + 2) + KT + 1] = acc;
                }
            }
            group_sync(g, H);
            if (i == 0 && bi < n) {
                float rad = 0.f, esum = 0.f, y0 = 0.f, ey = 0.f, yinf = 0.f;
                for (int k = 0; k < KT; ++k) {
                    float yk = 0.f, ek = 0.f;
                    for (int pp = 0; pp < NPART; ++pp) {
                        yk += Y[pp * (KT + 2) + k];
                        ek = ru_add(ek, E[pp * (KT + 2) + k]);
                    }
                    rad = ru_add(rad, fabsf(yk));
                    esum = ru_add(esum, ek);
                }
                for (int pp = 0; pp < NPART; ++pp) {
                    y0 += Y[pp * (KT + 2) + KT];
                    ey = ru_add(ey, E[pp * (KT + 2) + KT]);
                    yinf = ru_add(yinf, Y[pp * (KT + 2) + KT + 1]);
                }
                y0 += p.bout;
                ey = ru_add(ey, fabsf(p.bout));
                rad = ru_add(rad, yinf);
                if (SOUND) {
                    rad = ru_fma(esum, p.gam_out, rad);  // noise-column sums (incl. the part adds)
                    rad = ru_fma(ey, p.gam_c_out, rad);  // center sum, part adds and bias add
                }
                const float lo = rd_add(y0, -rad), hi = ru_add(y0, rad);
                const int k = lo > 0.f ? SRA_POSITIVE : (hi < 0.f ? SRA_NEGATIVE : SRA_UNKNOWN);
                if (out.lo) out.lo[bi] = lo;
                if (out.hi) out.hi[bi] = hi;
                if (out.cls) out.cls[bi] = (uint8_t)k;
                if (out.flag_list) {
                    const float band = out.band * (fabsf(y0) + rad);
                    if (fabsf(lo) <= band || fabsf(hi) <= band) out.flag_list[atomicAdd(out.flag_count, 1)] = (int)bi;
                }
            }
        }
        __syncthreads();
    }
    // leave: no MMA may still be writing TMEM; then free it
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 0) ptx::tmem_dealloc(x.tmem, 512);
}

}  // namespace tc

int tc_smem_bytes(int H) {
    return H == 256 ? tc::Layout<256>::ALLOC : (H == 128 ? tc::Layout<128>::ALLOC : 0);
}

template <int H, bool SOUND>
static cudaError_t launch_one(const TcParams &p, const BoxSrc &src, const BoundOut &out, int grid, cudaStream_t st) {
    const int smem = tc_smem_bytes(H);
    cudaError_t e = cudaFuncSetAttribute(tc::tc_bound_kernel<H, SOUND>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    tc::tc_bound_kernel<H, SOUND><<<grid, 2 * H, smem, st>>>(p, src, out);
    return cudaGetLastError();
}

cudaError_t launch_tc_bound(int H, bool sound, const TcParams &p, const BoxSrc &src, const BoundOut &out, int grid,
                            cudaStream_t st) {
    if (H == 256) return sound ? launch_one<256, true>(p, src, out, grid, st) : launch_one<256, false>(p, src, out, grid, st);
    if (H == 128) return sound ? launch_one<128, true>(p, src, out, grid, st) : launch_one<128, false>(p, src, out, grid, st);
    return cudaErrorInvalidValue;
}

}  // namespace sra
