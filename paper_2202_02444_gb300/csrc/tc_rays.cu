// CastRay (Proc. 2) with every layer but the output one on the tensor cores
// (tcgen05, split BF16).
//
// One persistent CTA per SM keeps NR = 16 ray slots in flight and refills a
// slot from a global counter when its ray ends. Every march step bounds each
// slot's segment [t, t+sigma] with affine-fixed arithmetic (the one noise
// symbol v = (sigma/2) r; every new symbol goes to x_inf, Sec. 3.3) and
// evaluates f at p + (t+delta) r in the same pass (Proc. 2).
//
// Linear layer l is two tensor-core products into TMEM (FP32 accumulation):
//   D  = (W_b + W_r) [c_hi c_lo p_hi p_lo A_hi A_lo]     96 operand rows
//   Dx = |W|_ru x_ru                                      16 operand rows
// W = W_b + W_r is the BF16 hi/lo split of the FP32 weights, and the center,
// point and noise values ride as BF16 hi/lo pairs, so each of their products
// keeps about 16 significant bits before the FP32 sums. The independent part
// x_inf is non-negative and only ever multiplied by |W|: both ride rounded up
// to BF16 (|W|_ru >= |W|, x_ru >= x_inf), so Dx bounds |W| x_inf from above
// with one matrix and one operand row per ray. Layer 0 takes the encoded
// input rows (K padded to 64).
//
// The weights stream from L2 by TMA as 16 KB tiles (128 rows x 64 K of one
// matrix) through a ring that runs ahead across layers and march steps. One
// thread issues the copies (it refills a stage once the MMAs that read it
// have completed), another issues the MMAs (one tile = 4 MMAs of K = 16;
// tiles in pairs of consecutive units, their MMAs alternating),
// and the whole CTA then runs the epilogue: per neuron and ray, the range,
// the activation rule (App. A) and the operand rows of the next layer. The
// encoding, the output layer and the march state run on the SIMT cores in
// FP32. Plain arithmetic: no rounding radius.
//
// Every wait is bounded; a wait that runs out sets the status word, the CTA
// drains the copies and MMAs it started (bounded again), frees TMEM and exits.
#include <cuda_bf16.h>

#include "sound_rules.cuh"
#include "sra_common.cuh"
#include "tc_ptx.cuh"
#include "tc_rays.h"

namespace sra {
namespace tcr {

constexpr int NR = 16;      // ray slots per CTA
constexpr int NCOL = 96;    // operand rows of D: 6 per ray
// operand rows of Dx: x_inf of each ray (rounded up), and in the sound form
// also |c| + |A| (rounded up), whose product with |W| bounds the layer's
// rounding errors
template <bool SOUND> constexpr int nxi() { return SOUND ? 32 : 16; }
constexpr int MAXDIN = 64;  // input width (3 + 6 * octaves) bound: layer 0 has one K slice
constexpr int TILE = 128 * 128;
constexpr int kSmemCap = 232448;
constexpr uint32_t kSpin = 1u << 22;
enum { C_HI = 0, C_LO = 16, P_HI = 32, P_LO = 48, A_HI = 64, A_LO = 80 };
enum { X_RU = 0, X_MAG = 16 };

struct RaySlot {
    long long idx;
    float t, sigma;
    int f0pos, iters, live, flag;  // flag: a decision of this ray was near zero
};

constexpr int align1k(int x) { return (x + 1023) & ~1023; }

template <int H, bool SOUND> struct RL {
    static constexpr int MT = H / 128, S = H / 64;
    static constexpr int NXI = nxi<SOUND>();
    static constexpr int NK = SOUND ? 5 : 4;  // output-layer sums per ray
    static constexpr int XB_SLICE = NCOL * 128, XI_SLICE = NXI * 128;
    static constexpr int XB_OFF = 0;
    static constexpr int XI_OFF = XB_OFF + S * XB_SLICE;
    static constexpr int INP_OFF = XI_OFF + S * XI_SLICE;       // segment inputs [NR][12]
    static constexpr int NPART = H / 64;
    static constexpr int OUTP_OFF = INP_OFF + NR * 12 * 4;       // output partial sums [NK NR][NPART]
    static constexpr int WOUT_OFF = OUTP_OFF + NK * NR * NPART * 4;
    static constexpr int RAY_OFF = WOUT_OFF + H * 4;
    static constexpr int BAR_OFF = RAY_OFF + NR * (int)sizeof(RaySlot);
    static constexpr int MISC_OFF = BAR_OFF + 256;
    static constexpr int RING_OFF = align1k(MISC_OFF + 64);
    static constexpr int NSTG_FIT = (kSmemCap - 1024 - RING_OFF) / TILE;
    static constexpr int NSTG = NSTG_FIT >= 8 ? 8 : 4;  // 4 measured faster than 5 at H = 512
    static constexpr int ALLOC = RING_OFF + NSTG * TILE + 1024;
    static constexpr int TCOLS = MT * 128;                       // TMEM: D (96) + Dx (NXI) per M-tile
    static_assert(NCOL + NXI <= 128, "TMEM columns");
    static_assert(NSTG_FIT >= 4, "weight ring");
    static_assert(MT == 1 || MT == 2 || MT == 4, "M tiles");
    static_assert(2 * NSTG + 2 <= 32, "barrier slots");
    static_assert(ALLOC <= kSmemCap, "shared memory");
    static_assert(XI_OFF % 1024 == 0 && XB_SLICE % 1024 == 0 && XI_SLICE % 1024 == 0, "operand alignment");
};

__device__ __forceinline__ void put_pair(unsigned char *slice, int row_hi, int row_lo, uint32_t kk, float v) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    *(__nv_bfloat16 *)(slice + ptx::sw128_offset((uint32_t)row_hi, kk)) = h;
    *(__nv_bfloat16 *)(slice + ptx::sw128_offset((uint32_t)row_lo, kk)) =
        __float2bfloat16_rn(v - __bfloat162float(h));
}

__device__ __forceinline__ float get_pair(const unsigned char *slice, int row_hi, int row_lo, uint32_t kk) {
    return __bfloat162float(*(const __nv_bfloat16 *)(slice + ptx::sw128_offset((uint32_t)row_hi, kk))) +
           __bfloat162float(*(const __nv_bfloat16 *)(slice + ptx::sw128_offset((uint32_t)row_lo, kk)));
}

// Operand rows at K index k (the next layer's input k) for ray slot r. The
// sound form first adds to x_inf the residuals of the centre's and the noise
// entry's BF16 hi/lo pairs (exact in FP32: the stored pair is c_hi + c_lo =
// c - rc), then stores x_inf and |c| + |A| rounded up.
template <int H, bool SOUND>
__device__ __forceinline__ void write_rows(unsigned char *sm, int k, int r, float c, float A, float xi, float p) {
    using L = RL<H, SOUND>;
    const uint32_t kk = (uint32_t)(k & 63);
    unsigned char *xb = sm + L::XB_OFF + (k >> 6) * L::XB_SLICE;
    unsigned char *xs = sm + L::XI_OFF + (k >> 6) * L::XI_SLICE;
    if (SOUND) {
        const float ch = __bfloat162float(__float2bfloat16_rn(c)), ah = __bfloat162float(__float2bfloat16_rn(A));
        const float cr = c - ch, ar = A - ah;  // exact
        const float rc = cr - __bfloat162float(__float2bfloat16_rn(cr)), ra = ar - __bfloat162float(__float2bfloat16_rn(ar));
        const float res = ru_add(fabsf(rc), fabsf(ra));
        xi = ru_add(xi, res);
        const float mag = ru_add(ru_add(fabsf(c), fabsf(A)), res);  // >= |stored c| + |stored A|
        *(__nv_bfloat16 *)(xs + ptx::sw128_offset((uint32_t)(X_MAG + r), kk)) = __float2bfloat16_ru(mag);
    }
    put_pair(xb, C_HI + r, C_LO + r, kk, c);
    put_pair(xb, P_HI + r, P_LO + r, kk, p);
    put_pair(xb, A_HI + r, A_LO + r, kk, A);
    *(__nv_bfloat16 *)(xs + ptx::sw128_offset((uint32_t)(X_RU + r), kk)) = __float2bfloat16_ru(xi);  // xi >= 0
}

// Activation of one neuron for one ray: the affine rule (App. A) on the
// segment form with the new symbol merged into x_inf (affine-fixed), and the
// plain activation on the point value.
__device__ __forceinline__ void activate(int act, int slope, float &c, float &A, float &xi, float &p) {
    if (act == SRA_ACT_IDENTITY) return;
    const float rad = fabsf(A) + xi;
    float a, b, g;
    linearize<float>(act, slope, c - rad, c + rad, a, b, g);
    A = A * a;
    c = a * c + b;
    xi = fabsf(a) * xi + fabsf(g);
    p = act_eval<float>(act, p);
}

// The sound form of `activate` (Chebyshev slope): the rules of
// sound_rules.cuh on the outward-rounded range c +- (|A| + xi); the new
// symbol joins x_inf (affine-fixed), and the FP32 product al * A adds 2^-24
// of its size (its BF16 hi/lo storage is added by write_rows). The point
// value takes the plain activation.
__device__ __forceinline__ void activate_sound(int act, float &c, float &A, float &xi, float &p) {
    if (act == SRA_ACT_IDENTITY) return;
    const float sa = fabsf(A);
    constexpr float kProd = 5.9604645e-08f * 1.001f;
    float al, ga, c2, xo;
    if (act == SRA_ACT_ELU) elu_rule<true>(sa, c, xi, kProd, al, ga, c2, xo);
    else if (act == SRA_ACT_SIN) sin_rule<true>(sa, c, xi, kProd, al, ga, c2, xo);
    else relu_rule<true>(sa, c, xi, kProd, al, ga, c2, xo);
    A = al * A;
    c = c2;
    xi = ru_add(xo, ga);
    p = act_eval<float>(act, p);
}

// A ring unit: one 128 x 64 tile (M tile m, K slice s) of one of the three
// matrices of linear layer `layer` (0 W_b, 1 W_r: into D; 2 |W|_ru: into
// Dx). Within a layer the units run K slice by K slice, M tile by M tile, in
// the order W_b, |W|_ru, W_r, so that two consecutive units feed different
// accumulators (D and Dx of one M tile, or D of two M tiles when there are
// two or more): the MMA thread takes them in pairs and alternates their MMAs.
// Each accumulator D still receives W_b's products before W_r's.
struct Unit {
    int layer, s, m, which;
};

template <int H, bool SOUND> __device__ __forceinline__ Unit unit_of(int layer, int u) {
    using L = RL<H, SOUND>;
    Unit r;
    r.layer = layer;
    const int ms = u / 3, w = u - 3 * ms;
    r.which = w == 0 ? 0 : (w == 1 ? 2 : 1);
    r.m = ms & (L::MT - 1);
    r.s = ms / L::MT;
    return r;
}

template <int H, bool SOUND> __device__ __forceinline__ int units_of(int layer) {
    using L = RL<H, SOUND>;
    return layer == 0 ? 3 * L::MT : 3 * L::MT * L::S;
}

// A position in the weight ring: its stage and the parity of that stage's
// current use (advanced one unit at a time; no division).
struct RingPos {
    int st;
    uint32_t ph;
};

template <int H, bool SOUND> __device__ __forceinline__ void advance(RingPos &r) {
    if (++r.st == RL<H, SOUND>::NSTG) {
        r.st = 0;
        r.ph ^= 1u;
    }
}

// The producer's position in the periodic unit sequence (layer 0, then the
// hidden layers, then layer 0 of the next march step, ...).
struct Cursor {
    uint32_t issued;  // units copied so far (compared modulo 2^32)
    RingPos pos;
    int layer, u;
};

// Issue the copy of the cursor's unit into its stage once the MMAs of that
// stage's previous use have completed; advance the cursor.
template <int H, bool SOUND>
__device__ __forceinline__ bool ring_load(unsigned char *sm, uint64_t *bars, const TcRayParams &p, int NL,
                                          Cursor &c) {
    using L = RL<H, SOUND>;
    const int st = c.pos.st;
    if (!ptx::mbar_wait(&bars[L::NSTG + st], c.pos.ph ^ 1u, kSpin)) return false;
    const Unit u = unit_of<H, SOUND>(c.layer, c.u);
    const TcLayerMaps &mp = u.layer == 0 ? p.first : p.hidden[u.layer - 1];
    const CUtensorMap *map = u.which == 0 ? &mp.wb : (u.which == 1 ? &mp.wr : &mp.wa);
    unsigned char *dst = sm + L::RING_OFF + st * TILE;
    ptx::mbar_arrive_expect_tx(&bars[st], TILE);
    ptx::tma_load_2d(dst, map, u.s * 64, u.m * 128, &bars[st]);
    ++c.issued;
    advance<H, SOUND>(c.pos);
    if (++c.u == units_of<H, SOUND>(c.layer)) {
        c.u = 0;
        c.layer = (c.layer == NL) ? 0 : c.layer + 1;
    }
    return true;
}

template <int H, bool SOUND>
__global__ void __launch_bounds__(H, 1) tc_ray_kernel(const __grid_constant__ TcRayParams p) {
    using L = RL<H, SOUND>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sm = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, i = tid;
    // bars: [0, NSTG) stage full, [NSTG, 2 NSTG) stage empty, then layer done, drain
    uint64_t *bars = (uint64_t *)(sm + L::BAR_OFF);
    uint64_t *acc_bar = &bars[2 * L::NSTG], *drain_bar = &bars[2 * L::NSTG + 1];
    uint32_t *tmem_slot = (uint32_t *)(sm + L::MISC_OFF);
    int *abort_flag = (int *)(sm + L::MISC_OFF + 4);
    uint32_t *consumed = (uint32_t *)(sm + L::MISC_OFF + 8);      // units whose MMAs were issued
    RingPos *issue_pos = (RingPos *)(sm + L::MISC_OFF + 16);      // the MMA thread's ring position
    RaySlot *slots = (RaySlot *)(sm + L::RAY_OFF);
    float *inp = (float *)(sm + L::INP_OFF);
    float *outp = (float *)(sm + L::OUTP_OFF);
    float *wout = (float *)(sm + L::WOUT_OFF);
    const int NL = p.L - 2;  // hidden H -> H layers
    if (tid == 0) {
        for (int k = 0; k < 2 * L::NSTG + 2; ++k) ptx::mbar_init(&bars[k], 1);
        ptx::fence_mbar_init();
        *abort_flag = 0;
        *consumed = 0u;
        issue_pos->st = 0;
        issue_pos->ph = 0u;
    }
    if (tid < NR) {
        slots[tid].idx = -1;
        slots[tid].live = 0;
    }
    wout[tid] = p.wout[tid];
    if (warp == 0) ptx::tmem_alloc(tmem_slot, L::TCOLS);
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int m_of = i >> 7;
    const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(m_of * 128);
    uint32_t gbase = 0;                 // units before the current layer
    Cursor cur = {0u, {0, 0u}, 0, 0};   // producer thread: next unit to copy
    RingPos ipos = {0, 0u};             // MMA thread: next unit to consume
    uint32_t accn = 0;
    auto fail = [&](int code) {
        *abort_flag = 1;
        atomicExch(p.status, code);
    };
    const bool producer = (warp == 0 && lane == 0), issuer = (warp == 1 && lane == 0);

    for (;;) {
        // ---- ray slots: refill, then the segment and point of this step -------
        if (tid < NR) {
            RaySlot &s = slots[tid];
            if (s.idx < 0) {
                const unsigned long long q = atomicAdd(p.next, 1ull);
                if ((long long)q < p.n) {
                    s.idx = (long long)q;
                    s.t = p.t_start ? p.t_start[q] : 0.f;
                    s.sigma = p.sigma_start ? p.sigma_start[q] : p.sigma0;
                    s.iters = 0;
                    s.f0pos = p.f0[q] >= 0.f;
                    s.live = 1;
                    s.flag = 0;
                } else {
                    s.live = 0;
                    s.idx = 0x7fffffffffffffffll;  // the ray list is exhausted for this slot
                }
            }
            float *in = inp + tid * 12;
            if (s.live) {
                const long long q = s.idx;
                for (int d = 0; d < 3; ++d) {
                    const float o = p.origins[q * 3 + d], r = p.dirs[q * 3 + d];
                    in[d] = o + (s.t + s.sigma / 2.f) * r;
                    in[3 + d] = (s.sigma / 2.f) * r;
                    in[6 + d] = o + (s.t + p.delta) * r;
                    if (SOUND) {
                        // the segment's points o + u r, u in [t, t + sigma], lie within
                        // in[9+d] of the box in[d] +- |in[3+d]|: the three roundings of
                        // the centre (the sum t + sigma/2, the product, the add of o)
                        // and the product of the half-width
                        const float m = fabsf((s.t + s.sigma / 2.f) * r);
                        in[9 + d] = ru_fma(ru_add(fabsf(in[d]), 2.f * m), 5.9604645e-08f * 1.001f,
                                           __fmul_ru(fabsf(in[3 + d]), 5.9604645e-08f * 1.001f));
                    }
                }
            } else {
                for (int d = 0; d < 12; ++d) in[d] = 0.f;
            }
        }
        const bool any = __syncthreads_or(tid < NR && slots[tid].live);
        if (!any || *abort_flag) break;
        // ---- layer-0 operand rows: the input and its encoding, sin(pi t), cos(pi t), t = 2^k x
        for (int w = tid; w < MAXDIN * NR; w += H) {
            const int j = w & (MAXDIN - 1), r = w / MAXDIN;
            float c = 0.f, A = 0.f, xi = 0.f, pt = 0.f;
            if (j < p.din) {
                const float *in = inp + r * 12;
                if (j < 3) {
                    c = in[j];
                    A = in[3 + j];
                    if (SOUND) xi = in[9 + j];
                    pt = in[6 + j];
                } else {
                    const int q = j - 3, k = q / 6, d = q % 3;
                    const float sc = (float)(1 << k), sh = ((q % 6) >= 3) ? 0.5f : 0.f;
                    const float ct = sc * in[d] + sh, at = sc * in[3 + d];
                    if (SOUND) {
                        // sc * in[d] and sc * in[3+d] are exact (sc = 2^k); the add of
                        // sh rounds once
                        const float xin = ru_fma(fabsf(ct), 5.9604645e-08f * 1.001f, sc * in[9 + d]);
                        float al, ga, c2, xo;
                        sinpi_rule_sound(fabsf(at), ct, xin, 5.9604645e-08f * 1.001f, al, ga, c2, xo);
                        c = c2;
                        A = at * al;
                        xi = ru_add(xo, ga);
                    } else {
                        const float rad = fabsf(at);
                        float a, b, gm;
                        linearize_sinpi<float>(ct - rad, ct + rad, a, b, gm);
                        c = a * ct + b;
                        A = at * a;
                        xi = fabsf(gm);
                    }
                    pt = sinpi_t(sc * in[6 + d] + sh);
                }
            }
            write_rows<H, SOUND>(sm, j, r, c, A, xi, pt);  // zero rows past din
        }
        // ---- every layer but the output one on the tensor cores --------------
        for (int l = 0; l <= NL; ++l) {
            const uint32_t U = (uint32_t)units_of<H, SOUND>(l);
            ptx::fence_proxy_async();  // operand writes -> async proxy
            ptx::tc_fence_before();    // TMEM reads of the previous layer are done
            __syncthreads();
            if (*abort_flag) break;
            if (producer) {
                bool ok = true;
                // copies run up to NSTG - 1 units past this layer's end
                while (ok && (int32_t)(cur.issued - (gbase + U + (L::NSTG - 1))) < 0)
                    ok = ring_load<H, SOUND>(sm, bars, p, NL, cur);
                if (!ok) fail(6);
            } else if (issuer) {
                bool ok = true;
                const uint32_t iD = ptx::idesc_bf16(128, NCOL), iX = ptx::idesc_bf16(128, L::NXI);
                // two consecutive units at a time (they feed different
                // accumulators): their MMAs alternate; an odd last unit alone
                for (uint32_t k = 0; k < U && ok;) {
                    const int nj = (U - k >= 2u) ? 2 : 1;
                    RingPos pos[2];
                    uint32_t d_col[2], idesc[2];
                    uint64_t a0[2], b0[2];
                    bool first[2];
                    for (int j = 0; j < nj; ++j) {
                        pos[j] = ipos;
                        advance<H, SOUND>(ipos);
                        if (!ptx::mbar_wait(&bars[pos[j].st], pos[j].ph, kSpin)) { ok = false; break; }
                        const Unit u = unit_of<H, SOUND>(l, (int)k + j);
                        const bool dx = u.which == 2;
                        const uint32_t b_addr = dx ? ptx::smem_u32(sm + L::XI_OFF + u.s * L::XI_SLICE)
                                                   : ptx::smem_u32(sm + L::XB_OFF + u.s * L::XB_SLICE);
                        d_col[j] = tmem + (uint32_t)(u.m * 128 + (dx ? NCOL : 0));
                        idesc[j] = dx ? iX : iD;
                        first[j] = u.which != 1 && u.s == 0;  // W_b into D, |W| into Dx: slice 0 starts them
                        a0[j] = ptx::desc_kmajor_sw128(ptx::smem_u32(sm + L::RING_OFF + pos[j].st * TILE));
                        b0[j] = ptx::desc_kmajor_sw128(b_addr);
                    }
                    if (!ok) break;
                    ptx::tc_fence_after();
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks)
                        for (int j = 0; j < nj; ++j)
                            ptx::mma_bf16(d_col[j], a0[j] + 2 * ks, b0[j] + 2 * ks, idesc[j],
                                          (first[j] && ks == 0) ? 0u : 1u);
                    for (int j = 0; j < nj; ++j) ptx::mma_commit(&bars[L::NSTG + pos[j].st]);
                    k += (uint32_t)nj;
                    if (k == U) ptx::mma_commit(acc_bar);
                }
                *consumed += U;  // published once per layer for the exit drain
                *issue_pos = ipos;
                if (!ok) fail(7);
            }
            __syncwarp();
            gbase += U;
            if (!ptx::mbar_wait(acc_bar, accn & 1u, kSpin)) fail(8);
            accn++;
            ptx::tc_fence_after();
            __syncthreads();
            if (*abort_flag) break;
            // epilogue: neuron i of every ray slot (the layer's operands are free)
            const float bias = __ldg(p.b[l] + i);
            const int act = p.act[l];
            // sound form: the FP32 accumulation factor of the Dx sums and the
            // rounding errors of D per unit of |W| (|c| + |A|), by layer depth
            const float kx = l == 0 ? p.kx0 : p.kx, rk = l == 0 ? p.rhok0 : p.rhok;
#pragma unroll 1
            for (int g = 0; g < NR / 8; ++g) {
                float v[64];
                const int r0 = g * 8;
                ptx::tmem_ld8(tl + C_HI + r0, v + 0);
                ptx::tmem_ld8(tl + C_LO + r0, v + 8);
                ptx::tmem_ld8(tl + P_HI + r0, v + 16);
                ptx::tmem_ld8(tl + P_LO + r0, v + 24);
                ptx::tmem_ld8(tl + A_HI + r0, v + 32);
                ptx::tmem_ld8(tl + A_LO + r0, v + 40);
                ptx::tmem_ld8(tl + NCOL + X_RU + r0, v + 48);
                if (SOUND) ptx::tmem_ld8(tl + NCOL + X_MAG + r0, v + 56);
                ptx::tmem_wait_ld();
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    float c = (v[r] + v[8 + r]) + bias;
                    float pp = (v[16 + r] + v[24 + r]) + bias;
                    float A = v[32 + r] + v[40 + r];
                    float xi = v[48 + r];
                    if (SOUND) {
                        // |W| x_inf and the layer's rounding errors from the Dx
                        // sums, each scaled for its FP32 accumulation; the two adds
                        // of the centre and the one of the noise pair
                        xi = ru_fma(v[56 + r], rk, ru_mul(xi, kx));
                        xi = ru_fma(ru_add(2.f * fabsf(c), fabsf(bias)), 5.9604645e-08f * 1.001f, xi);
                        xi = ru_fma(fabsf(A), 5.9604645e-08f * 1.001f, xi);
                        activate_sound(act, c, A, xi, pp);
                    } else {
                        activate(act, p.slope, c, A, xi, pp);
                    }
                    write_rows<H, SOUND>(sm, i, r0 + r, c, A, xi, pp);
                }
            }
        }
        __syncthreads();
        if (*abort_flag) break;
        // ---- output layer (H -> 1): 4 sums per ray (5 in the sound form: also
        // sum |w| (|c| + |A|)), H/64 parts of 64 inputs each
        {
            const int q = tid & 63, part = tid >> 6, r = q >> 2, kind = q & 3;
            float acc = 0.f, accm = 0.f;
            for (int j = part * 64; j < part * 64 + 64; ++j) {
                const uint32_t kk = (uint32_t)(j & 63);
                const unsigned char *xb = sm + L::XB_OFF + (j >> 6) * L::XB_SLICE;
                const unsigned char *xs = sm + L::XI_OFF + (j >> 6) * L::XI_SLICE;
                const float w = wout[j];
                if (kind == 0) acc = fmaf(w, get_pair(xb, C_HI + r, C_LO + r, kk), acc);
                else if (kind == 1) acc = fmaf(w, get_pair(xb, A_HI + r, A_LO + r, kk), acc);
                else if (kind == 2) {
                    acc = fmaf(fabsf(w),
                               __bfloat162float(*(const __nv_bfloat16 *)(xs + ptx::sw128_offset((uint32_t)(X_RU + r), kk))),
                               acc);
                    if (SOUND)
                        accm = fmaf(fabsf(w),
                                    __bfloat162float(
                                        *(const __nv_bfloat16 *)(xs + ptx::sw128_offset((uint32_t)(X_MAG + r), kk))),
                                    accm);
                } else acc = fmaf(w, get_pair(xb, P_HI + r, P_LO + r, kk), acc);
            }
            outp[(r * L::NK + kind) * L::NPART + part] = acc;
            if (SOUND && kind == 2) outp[(r * L::NK + 4) * L::NPART + part] = accm;
        }
        __syncthreads();
        // ---- march step of each live slot (Proc. 2) -------------------------------
        if (tid < NR && slots[tid].live) {
            RaySlot &s = slots[tid];
            float sums[5];
            for (int kind = 0; kind < L::NK; ++kind) {
                float a = 0.f;
                for (int part = 0; part < L::NPART; ++part) a += outp[(tid * L::NK + kind) * L::NPART + part];
                sums[kind] = a;
            }
            const float y0 = sums[0] + p.bout, fc = sums[3] + p.bout;
            float rad = fabsf(sums[1]) + sums[2];
            if (SOUND) {
                // the output sums' FP32 errors: within gam_out of sum |w| (|c| + |A|)
                // (the fifth sum, itself scaled up) and |bout|; the x_inf sum
                // scaled up; the add of the bias
                const float g1 = 1.f + p.gam_out;
                rad = ru_add(fabsf(sums[1]), ru_mul(sums[2], g1));
                rad = ru_fma(ru_fma(sums[4], g1, fabsf(p.bout)), p.gam_out, rad);
                rad = ru_fma(fabsf(y0), 5.9604645e-08f * 1.001f, rad);
            }
            s.iters += 1;
            if (p.flag_list && near_zero_step<float>(y0, rad, p.band)) s.flag = 1;
            bool done = false;
            float result = 0.f;
            if ((fc >= 0.f) != (s.f0pos != 0)) {  // DifferentSigns at t + delta
                done = true;
                result = s.t;
            } else {
                const int k = SOUND ? classify_range(rd_add(y0, -rad), ru_add(y0, rad)) : classify_range(y0 - rad, y0 + rad);
                float sstar;
                if (k != SRA_UNKNOWN) { sstar = s.sigma; s.sigma *= p.eta_plus; }
                else { sstar = 0.f; s.sigma *= p.eta_minus; }
                s.t += fmaxf(p.safety * sstar, p.delta);
                if (!(s.t < p.t_max)) { done = true; result = INFINITY; }
            }
            if (!done && s.iters >= p.max_iters) { done = true; result = NAN; }
            if (done) {
                p.t_hit[s.idx] = result;
                if (p.iters) p.iters[s.idx] = s.iters;
                if (p.flag_list && s.flag) {
                    const int q = atomicAdd(p.flag_count, 1);
                    if (idx_ok(q, p.n, p.status, 106)) p.flag_list[q] = (int)s.idx;
                }
                s.idx = -1;
            }
        }
        __syncthreads();
    }
    // drain: every issued MMA completes and every copy in flight lands before
    // TMEM is freed and the CTA exits
    __syncthreads();
    if (issuer) {
        ptx::mma_commit(drain_bar);
        if (!ptx::mbar_wait(drain_bar, 0u, kSpin)) atomicExch(p.status, 9);
    }
    if (producer) {  // the copies issued but never consumed, from the MMA thread's position on
        RingPos r = *issue_pos;
        for (uint32_t gi = *consumed; (int32_t)(gi - cur.issued) < 0; ++gi) {
            if (!ptx::mbar_wait(&bars[r.st], r.ph, kSpin)) {
                atomicExch(p.status, 10);
                break;
            }
            advance<H, SOUND>(r);
        }
    }
    __syncwarp();
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 0) ptx::tmem_dealloc(tmem, L::TCOLS);
}

}  // namespace tcr

int tc_ray_smem_bytes(int H, bool sound) {
    if (sound)
        return H == 512 ? tcr::RL<512, true>::ALLOC
                        : (H == 256 ? tcr::RL<256, true>::ALLOC : (H == 128 ? tcr::RL<128, true>::ALLOC : 0));
    return H == 512 ? tcr::RL<512, false>::ALLOC
                    : (H == 256 ? tcr::RL<256, false>::ALLOC : (H == 128 ? tcr::RL<128, false>::ALLOC : 0));
}

int tc_ray_max_din() { return tcr::MAXDIN; }

int tc_ray_slots() { return tcr::NR; }

template <int H, bool SOUND> static cudaError_t launch_r(const TcRayParams &p, int grid, cudaStream_t st) {
    const int smem = tcr::RL<H, SOUND>::ALLOC;
    cudaError_t e =
        cudaFuncSetAttribute(tcr::tc_ray_kernel<H, SOUND>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    tcr::tc_ray_kernel<H, SOUND><<<grid, H, smem, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_tc_rays(int H, bool sound, const TcRayParams &p, int grid, cudaStream_t st) {
    if (H == 512) return sound ? launch_r<512, true>(p, grid, st) : launch_r<512, false>(p, grid, st);
    if (H == 256) return sound ? launch_r<256, true>(p, grid, st) : launch_r<256, false>(p, grid, st);
    if (H == 128) return sound ? launch_r<128, true>(p, grid, st) : launch_r<128, false>(p, grid, st);
    return cudaErrorInvalidValue;
}

}  // namespace sra
