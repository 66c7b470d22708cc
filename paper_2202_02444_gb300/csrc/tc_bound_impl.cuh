// Device code of the BF16 tensor-core bound kernel (see tc_bound.cu for
// what it computes); included once per kept-symbol count KT by
// tc_bound.cu (KT = 64), tc_bound_k32.cu and tc_bound_k16.cu, so that the
// instantiations compile in parallel.
#pragma once

#include <cuda_bf16.h>

#include "sra_common.cuh"
#include "tc_bound.h"
#include "sound_rules.cuh"
#include "tc_ptx.cuh"

namespace sra {
namespace tc {

constexpr int NCC = 16;      // center-chunk columns (MMA N)
constexpr int NPART = 4;     // partial sums per output-layer dot product
constexpr uint32_t kSpin = 1u << 22;

// Boxes per tile (one thread group of H threads each) for width H and KT
// kept symbols: two at H = 128 and 256 with KT <= 64, else one (two boxes
// at H = 512, or with KT = 128, would need an MMA N or TMEM columns past
// the limits: N <= 256, 512 columns).
constexpr int boxes_per_tile(int H, int KT) { return (H == 512 || KT > 64) ? 1 : 2; }

template <int H, int KT, int NBV> struct Layout {
    // KT kept noise symbols per box (16, 32 or 64)
    static constexpr int NB = NBV;               // boxes per tile (one thread group each)
    static constexpr int NT = NB * H;            // threads per CTA
    static constexpr int NA = NB * KT;           // noise columns per tile
    static constexpr int MT = H / 128;   // M tiles per layer
    static constexpr int S = H / 64;     // K slices per layer
    // TMEM columns per M tile: NA noise then NCC center accumulators
    static constexpr int TM_STRIDE = (NB == 1 && NA + NCC <= 128) ? 128 : 256;
    static constexpr int TMEM_COLS = MT * TM_STRIDE <= 256 ? 256 : 512;  // allocated (a power of two)
    static constexpr int UPS = (NB == 1 && MT >= 2) ? 2 : 1;  // ring units per K slice
    static constexpr int MPU = MT / UPS;          // M tiles per ring unit
    static constexpr int TILE = 128 * 128;                  // bytes of one 128 x 64 bf16 tile
    static constexpr int STAGE = 2 * MPU * TILE;            // W_b and W_r tiles of one unit
    static constexpr int W_OFF = 0;
    static constexpr int XA_OFF = 2 * STAGE;
    // operand B, per 64-wide K slice: NA noise rows then NCC center rows,
    // so one MMA of N = NA + NCC covers both (slice stride (NA + NCC) x 128 B)
    static constexpr int XA_SLICE = (NA + NCC) * 128;
    static constexpr int XC_OFF = XA_OFF + NA * 128;
    static constexpr int XC_SLICE = XA_SLICE;
    static constexpr int F_OFF = XA_OFF + S * XA_SLICE;
    static constexpr int NCAND = KT + H;
    static constexpr int V_OFF = F_OFF;                              // v[NB][H]
    static constexpr int XR_OFF = V_OFF + NB * H * 4;                // xr[NB][H]
    static constexpr int SC_OFF = XR_OFF + NB * H * 4;               // score[NB][NCAND]
    static constexpr int PART_OFF = SC_OFF + NB * NCAND * 4;         // part[NB][H/32][KT]
    static constexpr int OUT_OFF = PART_OFF + NB * (H / 32) * KT * 4;  // Y,E [NB][NPART][KT+2]
    static constexpr int WOUT_OFF = OUT_OFF + 2 * NB * NPART * (KT + 2) * 4;  // wout[H]
    static constexpr int BOX_OFF = WOUT_OFF + H * 4;                 // box c/h [NB][8]
    static constexpr int XP_OFF = BOX_OFF + NB * 8 * 4;              // |W_b| v partials [NB][H] (two boxes)
    static constexpr int NCH = (KT + H + 31) / 32;                    // candidate chunks of 32
    static constexpr int KMW = NCH <= 16 ? 16 : 32;                  // kept-mask words per box
    static constexpr int KM_OFF = XP_OFF + (NB == 2 ? NB * H * 4 : 0);  // kept masks [NB][KMW]
    static constexpr int NEW_OFF = KM_OFF + NB * KMW * 4;            // newlist[NB][KT]
    static constexpr int BAR_OFF = ((NEW_OFF + NB * KT * 4) + 15) & ~15;   // 5 mbarriers
    static constexpr int MISC_OFF = BAR_OFF + 64;  // tmem slot, abort, nnew[NB], sel[NB][2]
    static constexpr int DUMMY_OFF = MISC_OFF + 64;  // 32 x 16 B sink for dropped columns' stores
    static constexpr int BYTES = DUMMY_OFF + 512;
    static constexpr int ALLOC = BYTES + 1024;     // + alignment slack
    static_assert(MPU >= 1 && MPU * UPS == MT && NA + NCC <= TM_STRIDE && MT * TM_STRIDE <= TMEM_COLS,
                  "TMEM columns");
    static_assert(NCH <= KMW && NB <= 2, "kept masks");
    static_assert(XA_OFF % 1024 == 0 && XA_SLICE % 1024 == 0 && XC_OFF % 1024 == 0, "operand alignment");
    static_assert(ALLOC <= 232448, "shared memory");
};

// Named barrier of one thread group (ids 1 and 2; 0 is __syncthreads).
__device__ __forceinline__ void group_sync(int g, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(nthreads) : "memory");
}

// Warp-wide sum rounded up at every step (every lane gets the same value).
__device__ __forceinline__ float warp_sum_ru(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __fadd_ru(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct Ctx {
    unsigned char *smem;
    int tid, g, i, wg, lane;  // thread, group (= box), neuron, warp in group, lane
    uint32_t tmem;
    uint64_t *bars;  // [0,1] full, [2,3] empty, [4] acc
    int *abort_flag;
    int *status;     // device status word (bounded waits; debug index checks)
};

__device__ __forceinline__ void fail(const Ctx &x, const TcParams &p, int code) {
    *x.abort_flag = 1;
    atomicExch(p.status, code);
}

// The network's activation rule (ReLU, ELU or sin; the same for every
// hidden layer), fixed per kernel instantiation.
template <bool SOUND, int ACT>
__device__ __forceinline__ void act_rule(float sa, float c, float xinf, float u_b2u, float &al, float &ga, float &c2,
                                         float &xi) {
    if constexpr (ACT == SRA_ACT_ELU) elu_rule<SOUND>(sa, c, xinf, u_b2u, al, ga, c2, xi);
    else if constexpr (ACT == SRA_ACT_SIN) sin_rule<SOUND>(sa, c, xinf, u_b2u, al, ga, c2, xi);
    else relu_rule<SOUND>(sa, c, xinf, u_b2u, al, ga, c2, xi);
}

// Upper bound of the summed magnitudes of a neuron's BF16 operand entries
// after truncation: every kept entry is bf16(al * a) (at most (1 + 2^-8)
// |al a| each, kept or not) and the neuron's own new symbol (at most
// (1 + 2^-7) ga).
__device__ __forceinline__ float operand_mag_bound(float al, float sa, float ga) {
    return ru_mul(ru_add(ru_mul(fabsf(al), sa), ga), 1.0078125f);
}

// Top-KT of the group's Ncur + H candidates (Sec. 3.3 truncate), by one
// warp of the group: warp g of group g, so that the two groups' selections
// run on different schedulers. The old columns' scores (L1 norms) are summed
// from the per-warp partials, the new symbols' magnitudes score[Ncur..) were
// written by their neurons; the caller has synchronised the group after
// both. The selection key is the score's top 16 bits (the BF16 truncation of
// a non-negative float: the scores come from BF16 operands and carry their
// 2^-8 relative error, so lower bits are not significant); non-negative
// floats order like their bit patterns. Unless at most KT keys are non-zero
// (then T = 0), the KT-th largest key T is found by a four-way search (three
// warp-wide counts per step) on an interval that starts at [the smallest
// second-largest key of a lane, the largest key]. Ties at T go to the lower
// candidate index, and kept columns stay in candidate order. Writes the kept
// mask of every chunk of 32 candidates, the kept new symbols newlist[q] =
// position | neuron << 16 and nnew to shared memory, valid after the
// caller's next group_sync.
template <int H, int KT, int NBV>
__device__ void select_topk(const Ctx &x, int Ncur) {
    using Lt = Layout<H, KT, NBV>;
    constexpr int NW = H / 32, NCH = Lt::NCH;
    if (x.wg != x.g) return;  // warp g of group g (with two groups warps 0 and H/32 + 1: different schedulers)
    const int g = x.g, lane = x.lane;
    const float *score = (const float *)(x.smem + Lt::SC_OFF) + g * Lt::NCAND;
    const float *part = (const float *)(x.smem + Lt::PART_OFF) + g * NW * KT;
    uint32_t *km = (uint32_t *)(x.smem + Lt::KM_OFF) + g * Lt::KMW;
    int *newlist = (int *)(x.smem + Lt::NEW_OFF) + g * KT;
    int *nnew_slot = (int *)(x.smem + Lt::MISC_OFF + 16) + g;
    const int C = Ncur + H;
    uint32_t key[NCH];
#pragma unroll
    for (int k = 0; k < NCH; ++k) {
        const int c = 32 * k + lane;
        float v = 0.f;
        if (c < Ncur) {
            for (int w = 0; w < NW; ++w) v += part[w * KT + c];
        } else if (c < C) {
            v = score[c];
        }
        key[k] = (32 * k + lane < C) ? __float_as_uint(v) >> 16 : 0u;  // invalid candidates: key 0, never kept below
    }
    uint32_t T = 0u;
    {
        // the lane's two largest keys (four for KT = 128)
        uint32_t nz = 0u, m1 = 0u, m2 = 0u, m3 = 0u, m4 = 0u;
#pragma unroll
        for (int k = 0; k < NCH; ++k) {
            nz += key[k] != 0u ? 1u : 0u;
            const uint32_t v = key[k];
            if constexpr (KT > 64) {
                if (v > m4) {
                    if (v > m3) {
                        m4 = m3;
                        if (v > m2) {
                            m3 = m2;
                            if (v > m1) { m2 = m1; m1 = v; } else m2 = v;
                        } else {
                            m3 = v;
                        }
                    } else {
                        m4 = v;
                    }
                }
            } else {
                m2 = v > m1 ? m1 : (v > m2 ? v : m2);
                m1 = v > m1 ? v : m1;
            }
        }
        if (__reduce_add_sync(0xffffffffu, nz) > (uint32_t)KT) {
            // T is the largest key with at least KT keys >= T. Every lane holds
            // two (four) keys >= its m2 (m4), so 64 >= KT (128 = KT) keys are
            // >= lo; no key exceeds hi.
            uint32_t lo = __reduce_min_sync(0xffffffffu, KT > 64 ? m4 : m2), hi = __reduce_max_sync(0xffffffffu, m1);
            while (lo < hi) {  // invariant: count(>= lo) >= KT, count(> hi) < KT
                const uint32_t w = hi - lo;  // split (lo, hi] at three points
                const uint32_t c1 = lo + (w + 3u) / 4u, c2 = lo + (2u * w + 3u) / 4u, c3 = lo + (3u * w + 3u) / 4u;
                uint32_t n1 = 0u, n2 = 0u, n3 = 0u;
#pragma unroll
                for (int k = 0; k < NCH; ++k) {
                    n1 += key[k] >= c1 ? 1u : 0u;
                    n2 += key[k] >= c2 ? 1u : 0u;
                    n3 += key[k] >= c3 ? 1u : 0u;
                }
                n1 = __reduce_add_sync(0xffffffffu, n1);
                n2 = __reduce_add_sync(0xffffffffu, n2);
                n3 = __reduce_add_sync(0xffffffffu, n3);
                if (n3 >= (uint32_t)KT) lo = c3;
                else if (n2 >= (uint32_t)KT) { lo = c2; hi = c3 - 1u; }
                else if (n1 >= (uint32_t)KT) { lo = c1; hi = c2 - 1u; }
                else hi = c1 - 1u;
            }
            T = lo;
        }
    }
    uint32_t gt = 0u;
#pragma unroll
    for (int k = 0; k < NCH; ++k) gt += key[k] > T ? 1u : 0u;
    const int need = KT - (int)__reduce_add_sync(0xffffffffu, gt);  // ties at T to keep
    const unsigned below = (1u << lane) - 1u;
    int base = 0, eqb = 0, nb = 0;
#pragma unroll
    for (int k = 0; k < NCH; ++k) {
        const int c = 32 * k + lane;
        const bool valid = c < C;
        const bool eq = valid && key[k] == T;
        const unsigned meq = __ballot_sync(0xffffffffu, eq);
        const bool kp = key[k] > T || (eq && eqb + __popc(meq & below) < need);
        const unsigned m = __ballot_sync(0xffffffffu, kp);
        const unsigned mnew = m & __ballot_sync(0xffffffffu, valid && c >= Ncur);
        if (lane == 0) km[k] = m;
        if (kp && c >= Ncur) {
            const int q = nb + __popc(mnew & below);
            if (idx_ok(q, KT, x.status, 101)) newlist[q] = (base + __popc(m & below)) | ((c - Ncur) << 16);
        }
        base += __popc(m);
        eqb += __popc(meq);
        nb += __popc(mnew);
    }
    if (lane == 0) *nnew_slot = nb;
}

// Kept flag of candidate c of the group's box (after select_topk and a group_sync).
template <int H, int KT, int NBV> __device__ __forceinline__ bool cand_kept(const Ctx &x, int c) {
    using Lt = Layout<H, KT, NBV>;
    const uint32_t *km = (const uint32_t *)(x.smem + Lt::KM_OFF) + x.g * Lt::KMW;
    return (km[c >> 5] >> (c & 31)) & 1u;
}

// Operand rows of the kept new symbols (positions KT - nnew .. KT - 1 of the
// group's box): one-hot columns, the neuron's magnitude ga (read back from
// the candidate scores) at its own entry and zeros elsewhere, written as
// 16-byte chunks of eight neurons.
template <int H, bool SOUND, int KT, int NBV>
__device__ __forceinline__ void fill_new_rows(const Ctx &x, int Ncur) {
    using Lt = Layout<H, KT, NBV>;
    const int g = x.g, i = x.i;
    const float *score = (const float *)(x.smem + Lt::SC_OFF) + g * Lt::NCAND;
    const int *newlist = (const int *)(x.smem + Lt::NEW_OFF) + g * KT;
    const int nnew = ((const int *)(x.smem + Lt::MISC_OFF + 16))[g];
    constexpr int CH = H / 8;  // 16-byte chunks per row
    constexpr int QS = H / CH;  // rows per pass of the group
    const int ch = i % CH;
    unsigned char *XA = x.smem + Lt::XA_OFF + (ch >> 3) * Lt::XA_SLICE;
    const uint32_t c16 = (uint32_t)(ch & 7);
    for (int q = i / CH; q < nnew; q += QS) {
        const int ent = newlist[q];
        const uint32_t row = (uint32_t)(g * KT + (ent & 0xffff));
        const int neuron = ent >> 16;
        if (!idx_ok(ent & 0xffff, KT, x.status, 102) || !idx_ok(neuron, H, x.status, 103)) continue;
        uint4 val = make_uint4(0u, 0u, 0u, 0u);
        if ((neuron >> 3) == ch) {
            const float ga = score[Ncur + neuron];
            const __nv_bfloat16 b = SOUND ? __float2bfloat16_ru(ga) : __float2bfloat16_rn(ga);
            const uint32_t bits = (uint32_t)__bfloat16_as_ushort(b);
            const int el = neuron & 7, wi = el >> 1;
            const uint32_t w = (el & 1) ? (bits << 16) : bits;
            val = make_uint4(wi == 0 ? w : 0u, wi == 1 ? w : 0u, wi == 2 ? w : 0u, wi == 3 ? w : 0u);
        }
        *(uint4 *)(XA + row * 128u + ((c16 ^ (row & 7u)) << 4)) = val;
    }
}

// Center (as a BF16 hi/lo pair, operand chunk XC), independent part and the
// sound operand vector v = rho1 |operand| + x_r of neuron n of the group's
// box, for the next layer's MMA and |W_b| v pass.
template <int H, bool SOUND, int KT, int NBV>
__device__ __forceinline__ void store_neuron(const Ctx &x, const TcParams &p, int n, float c2, float xi, float mag) {
    using Lt = Layout<H, KT, NBV>;
    const int g = x.g;
    const uint32_t kk = (uint32_t)(n & 63);
    const __nv_bfloat16 chi = __float2bfloat16_rn(c2);
    const float rem = c2 - __bfloat162float(chi);
    const __nv_bfloat16 clo = __float2bfloat16_rn(rem);
    const float rc = rem - __bfloat162float(clo);  // exact in fp32
    unsigned char *XC = x.smem + Lt::XC_OFF + (n >> 6) * Lt::XC_SLICE;
    *(__nv_bfloat16 *)(XC + ptx::sw128_offset((uint32_t)(2 * g), kk)) = chi;
    *(__nv_bfloat16 *)(XC + ptx::sw128_offset((uint32_t)(2 * g + 1), kk)) = clo;
    const float xr = SOUND ? ru_add(xi, fabsf(rc)) : xi;
    ((float *)(x.smem + Lt::XR_OFF))[g * H + n] = xr;
    if (SOUND) {
        const float m2 = ru_add(ru_add(mag, fabsf(__bfloat162float(chi))), fabsf(__bfloat162float(clo)));
        ((float *)(x.smem + Lt::V_OFF))[g * H + n] = ru_fma(p.rho1, m2, xr);
    } else {
        ((float *)(x.smem + Lt::V_OFF))[g * H + n] = xr;
    }
}

// First layer (3 -> H, SIMT): thread i holds neuron i's three noise entries
// a0 (already scaled by its slope al); truncation over 3 old + H new
// candidates; operand rows written element-wise.
template <int H, bool SOUND, int KT, int NBV>
__device__ void first_layer_store(const Ctx &x, const TcParams &p, const float (&a0)[3], float sa, float al,
                                  float ga, float c2, float xi) {
    using Lt = Layout<H, KT, NBV>;
    const int g = x.g, i = x.i, lane = x.lane, wg = x.wg;
    float *score = (float *)(x.smem + Lt::SC_OFF) + g * Lt::NCAND;
    float *part = (float *)(x.smem + Lt::PART_OFF) + g * (H / 32) * KT;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float s = warp_sum_f(fabsf(a0[k]));
        if (lane == 0) part[wg * KT + k] = s;
    }
    score[3 + i] = ga;
    group_sync(g, H);
    select_topk<H, KT, NBV>(x, 3);
    group_sync(g, H);
    const uint32_t km0 = ((const uint32_t *)(x.smem + Lt::KM_OFF))[g * Lt::KMW];
    unsigned char *XA = x.smem + Lt::XA_OFF + (i >> 6) * Lt::XA_SLICE;
    const uint32_t kk = (uint32_t)(i & 63);
    float dropped = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (!((km0 >> k) & 1u)) {
            dropped = ru_add(dropped, fabsf(a0[k]));
        } else {
            const int pp = __popc(km0 & ((1u << k) - 1u));
            *(__nv_bfloat16 *)(XA + ptx::sw128_offset((uint32_t)(g * KT + pp), kk)) = __float2bfloat16_rn(a0[k]);
        }
    }
    if (!cand_kept<H, KT, NBV>(x, 3 + i)) dropped = ru_add(dropped, ga);
    fill_new_rows<H, SOUND, KT, NBV>(x, 3);
    store_neuron<H, SOUND, KT, NBV>(x, p, i, c2, ru_add(xi, dropped), SOUND ? operand_mag_bound(al, sa, ga) : 0.f);
}

// Sum of N (a power of two) non-negative values, rounded up, as a balanced tree.
template <int N> __device__ __forceinline__ float ru_sum(const float (&t)[N]) {
    float u[N];
#pragma unroll
    for (int k = 0; k < N; ++k) u[k] = t[k];
#pragma unroll
    for (int w = N / 2; w >= 1; w >>= 1)
#pragma unroll
        for (int k = 0; k < w; ++k) u[k] = ru_add(u[2 * k], u[2 * k + 1]);
    return u[0];
}

// Reduce-scatter of four per-slot values over the four lanes of a quad,
// rounded up: lane q of the quad returns the quad's sum of slot q.
__device__ __forceinline__ float quad_scatter_ru(const float (&v)[4], int q) {
    const bool hi2 = (q & 2) != 0;
    const float k0 = hi2 ? v[2] : v[0], k1 = hi2 ? v[3] : v[1];
    const float s0 = hi2 ? v[0] : v[2], s1 = hi2 ? v[1] : v[3];
    const float r0 = ru_add(k0, __shfl_xor_sync(0xffffffffu, s0, 2));
    const float r1 = ru_add(k1, __shfl_xor_sync(0xffffffffu, s1, 2));
    const bool hi1 = (q & 1) != 0;
    return ru_add(hi1 ? r1 : r0, __shfl_xor_sync(0xffffffffu, hi1 ? r0 : r1, 1));
}

// Epilogue of one hidden layer for the group's box. Warp wg holds neurons
// 32 wg .. 32 wg + 31 in the accumulator fragment layout: for half h, lane t
// has neurons nA = 32 wg + 16 h + t/4 and nB = nA + 8 at noise columns
// 8 j + 2(t%4) + e (j < KT/8, e < 2), a[h][j][2 AB + e] with AB = 0 for nA
// and 1 for nB. The four lanes of a quad share their neurons; per-neuron scalars
// are computed redundantly in the quad (bit-identical), and lane t%4 == slot
// stores slot `2h + AB`. Column norms reduce-scatter across the lanes; kept
// columns go to operand B by transposing stmatrix (row = position, 16 bytes
// = eight consecutive neurons).
//
// Thread i's own neuron enters as its two center accumulators (TMEM columns
// ccol, ccol + 1 of its lane), its bias and its |W_b| v sum xacc.
template <int H, bool SOUND, int ACT, int KT, int NBV>
__device__ void hidden_epilogue(const Ctx &x, const TcParams &p, uint32_t tl, int col0, uint32_t ccol, float bias,
                                float xacc) {
    using Lt = Layout<H, KT, NBV>;
    const int g = x.g, lane = x.lane, wg = x.wg;
    float *score = (float *)(x.smem + Lt::SC_OFF) + g * Lt::NCAND;
    float *part = (float *)(x.smem + Lt::PART_OFF) + g * (H / 32) * KT;
    const int quad = lane >> 2, qi = lane & 3;
    constexpr int JJ = KT / 8;  // 8-column chunks of the box's noise columns
    float cc[2], a[2][JJ][4];
    ptx::tmem_ld2(ccol, cc);
#pragma unroll
    for (int h = 0; h < 2; ++h) ptx::tmem_ld16x256_chunks<JJ>(tl + ((uint32_t)(16 * h) << 16) + (uint32_t)col0, &a[h][0][0]);
    ptx::tmem_wait_ld();
    // center: D(c_hi) + D(c_lo) + bias, each add rounded once
    const float c_n = (cc[0] + cc[1]) + bias;
    float xinf_n;
    if (SOUND) {
        xinf_n = ru_mul(xacc, p.kappa);
        // the two adds: u |cc0 + cc1| + u |c| <= 2^-23 (2 |c| + |bias|)
        xinf_n = ru_fma(ru_add(2.f * fabsf(c_n), fabsf(bias)), 1.1920929e-07f, xinf_n);
    } else {
        xinf_n = xacc;
    }
    // lane t%4 == q computes the scalars of slot q (neuron nq)
    const int nq = 32 * wg + 16 * (qi >> 1) + 8 * (qi & 1) + quad;
    const float cq = __shfl_sync(0xffffffffu, c_n, nq & 31);
    const float xq = __shfl_sync(0xffffffffu, xinf_n, nq & 31);
    // range: noise magnitudes per neuron, reduce-scattered over the quad
    // (rounded up): lane q ends with slot q's sum
    float sa;
    {
        float ps[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int h = s >> 1, q0 = 2 * (s & 1);
            float t[2 * JJ];
#pragma unroll
            for (int j = 0; j < JJ; ++j) {
                t[2 * j] = fabsf(a[h][j][q0]);
                t[2 * j + 1] = fabsf(a[h][j][q0 + 1]);
            }
            ps[s] = ru_sum<2 * JJ>(t);
        }
        sa = quad_scatter_ru(ps, qi);
    }
    float al, ga, c2, xi;
    act_rule<SOUND, ACT>(sa, cq, xq, p.ub2u, al, ga, c2, xi);
    score[KT + nq] = ga;
    float als[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) als[s] = __shfl_sync(0xffffffffu, al, (lane & ~3) | s);
    // scale; column L1 norms over the warp's 32 neurons: v[i] (i = 2 j + e,
    // symbol 8 j + 2(t%4) + e) summed over the eight quads by a
    // reduce-scatter on lane bits 4, 3, 2, each step keeping the half of the
    // values that the lane bit selects (bit 4 picks the top bit of i, and so
    // on); with fewer than eight values the last steps are plain sums
    constexpr int NV = 2 * JJ;
    constexpr int LNV = NV == 16 ? 4 : (NV == 8 ? 3 : 2);
    constexpr int NSC = LNV < 3 ? LNV : 3;  // scattering steps
    float v[NV];
#pragma unroll
    for (int j = 0; j < JJ; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            a[0][j][q] *= als[q >> 1];
            a[1][j][q] *= als[2 + (q >> 1)];
        }
#pragma unroll
    for (int j = 0; j < JJ; ++j)
#pragma unroll
        for (int e = 0; e < 2; ++e)
            v[2 * j + e] = (fabsf(a[0][j][e]) + fabsf(a[0][j][2 + e])) + (fabsf(a[1][j][e]) + fabsf(a[1][j][2 + e]));
#pragma unroll
    for (int stp = 0; stp < 3; ++stp) {
        const int o = 16 >> stp;
        if (stp < NSC) {
            const int half = NV >> (stp + 1);
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int k = 0; k < half; ++k) {
                const float send = up ? v[k] : v[k + half];
                const float keepv = up ? v[k + half] : v[k];
                v[k] = keepv + __shfl_xor_sync(0xffffffffu, send, o);
            }
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
        }
    }
    {
        // lane t keeps values i = hi << (LNV - NSC) | k, hi = the lane's NSC
        // bits below bit 5; lanes that differ only below them hold copies
        constexpr int KEEP = NV >> NSC;
        const int hi = (lane >> (5 - NSC)) & ((1 << NSC) - 1);
        if (((lane >> 2) & ((1 << (3 - NSC)) - 1)) == 0) {
#pragma unroll
            for (int k = 0; k < KEEP; ++k) {
                const int iv = (hi << (LNV - NSC)) | k;
                part[wg * KT + 8 * (iv >> 1) + 2 * qi + (iv & 1)] = v[k];
            }
        }
    }
    group_sync(g, H);
    select_topk<H, KT, NBV>(x, KT);
    group_sync(g, H);
    const uint32_t *kmw = (const uint32_t *)(x.smem + Lt::KM_OFF) + g * Lt::KMW;
    // kept flags of the KT old columns (candidates 0 .. KT-1; the bits above
    // belong to new symbols)
    constexpr unsigned long long KMASK = KT == 64 ? ~0ull : ((1ull << KT) - 1ull);
    const unsigned long long kept = (((unsigned long long)kmw[1] << 32) | kmw[0]) & KMASK;
    // dropped magnitudes per neuron (reduce-scattered over the quad, rounded
    // up) to x_inf: 0/1 masks times |a|, exact products
    {
        const unsigned long long mine = ~kept >> (2 * qi);
        float mf[2 * JJ];
#pragma unroll
        for (int j = 0; j < JJ; ++j)
#pragma unroll
            for (int e = 0; e < 2; ++e) mf[2 * j + e] = ((mine >> (8 * j + e)) & 1ull) ? 1.f : 0.f;
        float pd[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int h = s >> 1, q0 = 2 * (s & 1);
            float d0 = 0.f, d1 = 0.f;
#pragma unroll
            for (int j = 0; j < JJ; ++j) {
                d0 = ru_fma(mf[2 * j], fabsf(a[h][j][q0]), d0);
                d1 = ru_fma(mf[2 * j + 1], fabsf(a[h][j][q0 + 1]), d1);
            }
            pd[s] = ru_add(d0, d1);
        }
        xi = ru_add(xi, quad_scatter_ru(pd, qi));
    }
    // kept old columns -> operand B rows g*KT + pos (dropped rows to a dummy
    // area); pos counts the kept symbols below 8 j + r: whole bytes of the
    // mask, then the low r bits of byte j
    {
        const int mi = lane >> 3, r = lane & 7;
        const int nb = 32 * wg + 8 * mi;
        const uint32_t xa = ptx::smem_u32(x.smem + Lt::XA_OFF + (nb >> 6) * Lt::XA_SLICE);
        const uint32_t c16 = (uint32_t)((nb & 63) >> 3);
        const uint32_t dummy = ptx::smem_u32(x.smem + Lt::DUMMY_OFF) + 16u * (uint32_t)lane;
        const uint32_t below_r = (1u << r) - 1u;
        uint32_t pre = 0u;
#pragma unroll
        for (int j = 0; j < JJ; ++j) {
            const uint32_t byte = (uint32_t)(kept >> (8 * j)) & 0xffu;
            const bool k = (byte >> r) & 1u;
            const uint32_t row = (uint32_t)(g * KT) + pre + (uint32_t)__popc(byte & below_r);
            pre += (uint32_t)__popc(byte);
            const bool in = idx_ok((long long)row - g * KT, KT, x.status, 104);
            const uint32_t addr = (k && in) ? xa + row * 128u + ((c16 ^ (row & 7u)) << 4) : dummy;
            uint32_t R[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const __nv_bfloat162 b = __floats2bfloat162_rn(a[m >> 1][j][2 * (m & 1)], a[m >> 1][j][2 * (m & 1) + 1]);
                R[m] = *(const uint32_t *)&b;
            }
            ptx::stmatrix_x4_trans(addr, R[0], R[1], R[2], R[3]);
        }
    }
    if (!cand_kept<H, KT, NBV>(x, KT + nq)) xi = ru_add(xi, ga);
    fill_new_rows<H, SOUND, KT, NBV>(x, KT);
    store_neuron<H, SOUND, KT, NBV>(x, p, nq, c2, xi, SOUND ? operand_mag_bound(al, sa, ga) : 0.f);
}

// Epilogue of one hidden layer with K = 128 kept symbols: the steps of
// hidden_epilogue over the box's 128 noise columns in two halves of 64 (a
// thread cannot hold both halves' accumulators): the range sums over both
// halves (each rounded up), then per half the scaled columns' L1 norms; the
// selection over the 128 + H candidates; then per half the dropped
// magnitudes and the write-back of the kept columns, whose positions
// continue from the first half into the second. Each half is read from TMEM
// again where it is needed.
template <int H, bool SOUND, int ACT, int NBV>
__device__ void hidden_epilogue_wide(const Ctx &x, const TcParams &p, uint32_t tl, int col0, uint32_t ccol,
                                     float bias, float xacc) {
    constexpr int KT = 128;
    using Lt = Layout<H, KT, NBV>;
    const int g = x.g, lane = x.lane, wg = x.wg;
    float *score = (float *)(x.smem + Lt::SC_OFF) + g * Lt::NCAND;
    float *part = (float *)(x.smem + Lt::PART_OFF) + g * (H / 32) * KT;
    const int quad = lane >> 2, qi = lane & 3;
    float cc[2], a[2][8][4];
    auto load_half = [&](int hf) {
#pragma unroll
        for (int h = 0; h < 2; ++h)
            ptx::tmem_ld16x256_x8(tl + ((uint32_t)(16 * h) << 16) + (uint32_t)(col0 + 64 * hf), &a[h][0][0]);
        ptx::tmem_wait_ld();
    };
    ptx::tmem_ld2(ccol, cc);
    load_half(0);
    const float c_n = (cc[0] + cc[1]) + bias;
    float xinf_n;
    if (SOUND) {
        xinf_n = ru_mul(xacc, p.kappa);
        xinf_n = ru_fma(ru_add(2.f * fabsf(c_n), fabsf(bias)), 1.1920929e-07f, xinf_n);
    } else {
        xinf_n = xacc;
    }
    const int nq = 32 * wg + 16 * (qi >> 1) + 8 * (qi & 1) + quad;
    const float cq = __shfl_sync(0xffffffffu, c_n, nq & 31);
    const float xq = __shfl_sync(0xffffffffu, xinf_n, nq & 31);
    float sa;
    {
        float ps[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
        for (int hf = 0; hf < 2; ++hf) {
            if (hf == 1) load_half(1);
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const int h = s >> 1, q0 = 2 * (s & 1);
                float t[16];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    t[2 * j] = fabsf(a[h][j][q0]);
                    t[2 * j + 1] = fabsf(a[h][j][q0 + 1]);
                }
                ps[s] = ru_add(ps[s], ru_sum<16>(t));
            }
        }
        sa = quad_scatter_ru(ps, qi);
    }
    float al, ga, c2, xi;
    act_rule<SOUND, ACT>(sa, cq, xq, p.ub2u, al, ga, c2, xi);
    score[KT + nq] = ga;
    float als[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) als[s] = __shfl_sync(0xffffffffu, al, (lane & ~3) | s);
    auto scale = [&]() {
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[0][j][q] *= als[q >> 1];
                a[1][j][q] *= als[2 + (q >> 1)];
            }
    };
    // column L1 norms of each half (the reduce-scatter of hidden_epilogue):
    // half 1 first, which the range sums left in the registers; half 0 then
    // stays there, scaled, for the write-back below
#pragma unroll 1
    for (int hf = 1; hf >= 0; --hf) {
        if (hf == 0) load_half(0);
        scale();
        float v[16];
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int e = 0; e < 2; ++e)
                v[2 * j + e] = (fabsf(a[0][j][e]) + fabsf(a[0][j][2 + e])) + (fabsf(a[1][j][e]) + fabsf(a[1][j][2 + e]));
#pragma unroll
        for (int half = 8, o = 16; o >= 4; half >>= 1, o >>= 1) {
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int k = 0; k < half; ++k) {
                const float send = up ? v[k] : v[k + half];
                const float keepv = up ? v[k + half] : v[k];
                v[k] = keepv + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
        part[wg * KT + 64 * hf + 8 * quad + 2 * qi] = v[0];
        part[wg * KT + 64 * hf + 8 * quad + 2 * qi + 1] = v[1];
    }
    group_sync(g, H);
    select_topk<H, KT, NBV>(x, KT);
    group_sync(g, H);
    const uint32_t *kmw = (const uint32_t *)(x.smem + Lt::KM_OFF) + g * Lt::KMW;
    const int mi = lane >> 3, r = lane & 7;
    const int nb = 32 * wg + 8 * mi;
    const uint32_t xa = ptx::smem_u32(x.smem + Lt::XA_OFF + (nb >> 6) * Lt::XA_SLICE);
    const uint32_t c16 = (uint32_t)((nb & 63) >> 3);
    const uint32_t dummy = ptx::smem_u32(x.smem + Lt::DUMMY_OFF) + 16u * (uint32_t)lane;
    const uint32_t below_r = (1u << r) - 1u;
    uint32_t pre = 0u;  // kept old columns below the current byte, over both halves
#pragma unroll 1
    for (int hf = 0; hf < 2; ++hf) {
        if (hf == 1) {
            load_half(1);
            scale();
        }
        const unsigned long long kept = ((unsigned long long)kmw[2 * hf + 1] << 32) | kmw[2 * hf];
        {
            const unsigned long long mine = ~kept >> (2 * qi);
            float mf[16];
#pragma unroll
            for (int j = 0; j < 8; ++j)
#pragma unroll
                for (int e = 0; e < 2; ++e) mf[2 * j + e] = ((mine >> (8 * j + e)) & 1ull) ? 1.f : 0.f;
            float pd[4];
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const int h = s >> 1, q0 = 2 * (s & 1);
                float d0 = 0.f, d1 = 0.f;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    d0 = ru_fma(mf[2 * j], fabsf(a[h][j][q0]), d0);
                    d1 = ru_fma(mf[2 * j + 1], fabsf(a[h][j][q0 + 1]), d1);
                }
                pd[s] = ru_add(d0, d1);
            }
            xi = ru_add(xi, quad_scatter_ru(pd, qi));
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t byte = (uint32_t)(kept >> (8 * j)) & 0xffu;
            const bool k = (byte >> r) & 1u;
            const uint32_t row = (uint32_t)(g * KT) + pre + (uint32_t)__popc(byte & below_r);
            pre += (uint32_t)__popc(byte);
            const bool in = idx_ok((long long)row - g * KT, KT, x.status, 104);
            const uint32_t addr = (k && in) ? xa + row * 128u + ((c16 ^ (row & 7u)) << 4) : dummy;
            uint32_t R[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const __nv_bfloat162 b = __floats2bfloat162_rn(a[m >> 1][j][2 * (m & 1)], a[m >> 1][j][2 * (m & 1) + 1]);
                R[m] = *(const uint32_t *)&b;
            }
            ptx::stmatrix_x4_trans(addr, R[0], R[1], R[2], R[3]);
        }
    }
    if (!cand_kept<H, KT, NBV>(x, KT + nq)) xi = ru_add(xi, ga);
    fill_new_rows<H, SOUND, KT, NBV>(x, KT);
    store_neuron<H, SOUND, KT, NBV>(x, p, nq, c2, xi, SOUND ? operand_mag_bound(al, sa, ga) : 0.f);
}

template <int H, bool SOUND, int ACT, int KT, int NBV>
__global__ void __launch_bounds__(Layout<H, KT, NBV>::NT, 1) tc_bound_kernel(const __grid_constant__ TcParams p, BoxSrc src,
                                                                    BoundOut out) {
    using Lt = Layout<H, KT, NBV>;
    constexpr int NT = Lt::NT, NB = Lt::NB, NA = Lt::NA, TM_STRIDE = Lt::TM_STRIDE;
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
    x.status = p.status;
    const int tid = x.tid, g = x.g, i = x.i;
    const int warp = tid >> 5;
    // M tile m's MMAs are issued by one thread: with two groups lane 0 of
    // warp m of group m (warps 0 and 9: two different schedulers), with one
    // group lane 0 of warp m; each issuer commits to the stage barrier of
    // every ring unit holding its tile and to the accumulator barrier
    constexpr int ISSUERS = Lt::MT;
    const int my_m = NB == 2 ? g : (i >> 5);
    const bool issuer = NB == 2 ? (i == 32 * g && g < ISSUERS) : (x.lane == 0 && my_m < ISSUERS);
    // a stage is free once the issuers of its unit's M tiles have committed
    // and every warp that reads the unit's W_b tiles (for |W_b| v) has arrived
    constexpr int STAGE_ARRIVALS = Lt::MPU + NT / 32 / Lt::UPS;
    if (tid == 0) {
        ptx::mbar_init(&x.bars[0], 1);
        ptx::mbar_init(&x.bars[1], 1);
        ptx::mbar_init(&x.bars[2], STAGE_ARRIVALS);
        ptx::mbar_init(&x.bars[3], STAGE_ARRIVALS);
        ptx::mbar_init(&x.bars[4], ISSUERS);
        ptx::fence_mbar_init();
        *x.abort_flag = 0;
        uint32_t *sel = (uint32_t *)(x.smem + Lt::MISC_OFF + 32);
        for (int gg = 0; gg < NB; ++gg) { sel[2 * gg] = 0u; sel[2 * gg + 1] = KT; }
    }
    // zero the center chunk once (rows beyond 2*NB stay zero); output weights to smem
    for (int e = tid; e < Lt::S * NCC * 32; e += NT)
        ((uint32_t *)(x.smem + Lt::XC_OFF + (e / (NCC * 32)) * Lt::XC_SLICE))[e % (NCC * 32)] = 0u;
    float *wout = (float *)(x.smem + Lt::WOUT_OFF);
    for (int e = tid; e < H; e += NT) wout[e] = p.wout[e];
    if (warp == 0) ptx::tmem_alloc(tmem_slot, Lt::TMEM_COLS);
    __syncthreads();
    ptx::tc_fence_after();
    x.tmem = *tmem_slot;
    const uint32_t tl = x.tmem + ((uint32_t)((warp & 3) * 32) << 16);  // this warp's TMEM lanes
    const int m_of_thread = i >> 7;
    float *boxf = (float *)(x.smem + Lt::BOX_OFF);
    const long long n = src.n;
    const long long ntiles = (n + NB - 1) / NB;
    uint32_t gring = 0, accn = 0;
    // weight units (a K slice, or at H = 512 half of its M tiles) stream
    // through the ring in one global order (layer 1..L-2 of every tile this
    // CTA takes); the producer thread issues them up to two ahead of the
    // consumers, across layer and tile boundaries, and never past the CTA's
    // last unit
    const int NL = p.L - 2;
    const long long my_tiles = ntiles > (long long)blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const uint32_t total_units = (uint32_t)(my_tiles * NL * Lt::S * Lt::UPS);
    // the copies are issued by lane 0 of the last warp, so that a refill,
    // which waits for the MMAs that read the stage, never holds up the
    // issue of the next slice's MMAs
    constexpr int PRODUCER = NT - 32;
    uint32_t gload = 0;
    int ld_layer = 1, ld_slice = 0, ld_half = 0;
    // bounded-wait budget; a test setting (p.test_stall > 0) also switches the
    // copies off, so that every wait on a full stage runs out with nothing in
    // flight (no copy, no MMA) and the CTA leaves through its normal exit
    const uint32_t spins = p.test_stall > 0 ? (uint32_t)p.test_stall : kSpin;
    auto issue_upto = [&](uint32_t target) {  // the producer thread
        if (p.test_stall > 0) return;
        while (gload < target && gload < total_units && !*x.abort_flag) {
            const uint32_t gg = gload, st = gg & 1u;
            if (!ptx::mbar_wait(&x.bars[2 + st], ((gg >> 1) & 1u) ^ 1u, spins)) { fail(x, p, 3); return; }
            unsigned char *base = x.smem + Lt::W_OFF + st * Lt::STAGE;
            ptx::mbar_arrive_expect_tx(&x.bars[st], Lt::STAGE);
            const CUtensorMap *mb = &p.wb[ld_layer - 1], *mr = &p.wr[ld_layer - 1];
            for (int mm = 0; mm < Lt::MPU; ++mm) {
                const int m = ld_half * Lt::MPU + mm;
                ptx::tma_load_2d(base + mm * Lt::TILE, mb, ld_slice * 64, m * 128, &x.bars[st]);
                ptx::tma_load_2d(base + (Lt::MPU + mm) * Lt::TILE, mr, ld_slice * 64, m * 128, &x.bars[st]);
            }
            ++gload;
            if (++ld_half == Lt::UPS) {
                ld_half = 0;
                if (++ld_slice == Lt::S) {
                    ld_slice = 0;
                    if (++ld_layer > NL) ld_layer = 1;
                }
            }
        }
    };

    // every abort decision is taken on a barrier that ORs the threads' flags,
    // so the whole CTA leaves together even if a wait ran out just after it
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        if (__syncthreads_or(*x.abort_flag != 0)) break;
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
            const float w0[3] = {p.W0[i * 3], p.W0[i * 3 + 1], p.W0[i * 3 + 2]};
            const float b0 = p.b[0][i];
            float a0[3];
            float c = b0, cm = fabsf(b0), am = 0.f;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float cd = boxf[g * 8 + d];
                c = fmaf(w0[d], cd, c);
                cm = ru_fma(fabsf(w0[d]), fabsf(cd), cm);
                a0[d] = w0[d] * boxf[g * 8 + 3 + d];
                am = ru_add(am, fabsf(a0[d]));
            }
            float xinf = 0.f;
            if (SOUND) {
                xinf = ru_mul(cm, 2.3841858e-07f);  // 3-FMA sum: gamma_3 < 2^-22
                xinf = ru_fma(am, 1.1920929e-07f, xinf);  // one rounding per product
            }
            float al, ga, c2, xi;
            act_rule<SOUND, ACT>(am, c, xinf, p.ub2u, al, ga, c2, xi);
#pragma unroll
            for (int d = 0; d < 3; ++d) a0[d] *= al;
            first_layer_store<H, SOUND, KT, NBV>(x, p, a0, am, al, ga, c2, xi);
        }
        // ---- hidden layers on the tensor cores ---------------------------------
        for (int l = 1; l + 1 < p.L; ++l) {
            ptx::fence_proxy_async();  // operand writes -> async proxy
            ptx::tc_fence_before();    // previous TMEM reads done before new MMAs
            if (__syncthreads_or(*x.abort_flag != 0)) break;
            const float bias = p.b[l][i];  // read early: its latency hides under the MMA phase
            float xa0 = 0.f, xa1 = 0.f, xb0 = 0.f, xb1 = 0.f;  // rounded-up |W_b| v partials, boxes 0 and 1
            const uint32_t g0 = gring;
            if (tid == PRODUCER) issue_upto(g0 + 2);  // no-op when prefetched during the last epilogue
            for (int s = 0; s < Lt::S; ++s) {
#pragma unroll
                for (int hf = 0; hf < Lt::UPS; ++hf) {
                    const uint32_t gg = g0 + (uint32_t)(s * Lt::UPS + hf), st = gg & 1u, par = (gg >> 1) & 1u;
                    // this thread reads the unit's W_b tile of its M tile; it issues the unit's MMAs of its tile
                    const bool mine = Lt::UPS == 1 || m_of_thread / Lt::MPU == hf;
                    const bool my_mma = issuer && my_m / Lt::MPU == hf;
                    if (mine || my_mma)
                        if (!ptx::mbar_wait(&x.bars[st], par, spins)) fail(x, p, 4);
                    unsigned char *base = x.smem + Lt::W_OFF + st * Lt::STAGE;
                    if (my_mma && !*x.abort_flag) {
                        ptx::tc_fence_after();
                        const uint32_t ia = ptx::idesc_bf16(128, NA + NCC);
                        const int mm = my_m - hf * Lt::MPU;  // the tile's place in the unit
                        for (int ks = 0; ks < 4; ++ks) {
                            const uint32_t acc = (s | ks) ? 1u : 0u;
                            const uint64_t bA =
                                ptx::desc_kmajor_sw128(ptx::smem_u32(x.smem + Lt::XA_OFF + s * Lt::XA_SLICE)) + 2 * ks;
                            const uint64_t aB = ptx::desc_kmajor_sw128(ptx::smem_u32(base + mm * Lt::TILE)) + 2 * ks;
                            const uint64_t aR =
                                ptx::desc_kmajor_sw128(ptx::smem_u32(base + (Lt::MPU + mm) * Lt::TILE)) + 2 * ks;
                            ptx::mma_bf16(x.tmem + my_m * TM_STRIDE, aB, bA, ia, acc);
                            ptx::mma_bf16(x.tmem + my_m * TM_STRIDE, aR, bA, ia, 1u);
                        }
                        ptx::mma_commit(&x.bars[2 + st]);
                        if (s + 1 == Lt::S) ptx::mma_commit(&x.bars[4]);
                    }
                    if constexpr (NB == 2) {
                        // x_inf' += |W_b| v from the resident slice: thread (g, i) takes
                        // row i over inputs 32 g .. 32 g + 31 of the slice for both boxes
                        // (one read and unpack of each weight), in four 8-input chunks
                        const int r = i & 127;
                        const unsigned char *row = base + m_of_thread * Lt::TILE + r * 128;
                        const float *v0 = (const float *)(x.smem + Lt::V_OFF) + s * 64;
                        const float *v1 = v0 + H;
                        // the MMA-issuing warps leave their last chunk to the other
                        // group's warp over the same rows, which sums it into the
                        // same row's partials (every partial rounded up)
                        const bool light = x.wg == g && g < ISSUERS;
                        const bool heavy = x.wg == 1 - g && 1 - g < ISSUERS;
#pragma unroll
                        for (int cc = 0; cc < 5; ++cc) {
                            if ((cc == 3 && light) || (cc == 4 && !heavy)) continue;
                            const int ch = cc < 4 ? 4 * g + cc : 4 * (1 - g) + 3;
                            const uint4 q = *(const uint4 *)(row + (((ch ^ (r & 7)) & 7) << 4));
                            const float4 a0 = *(const float4 *)(v0 + ch * 8), a1 = *(const float4 *)(v0 + ch * 8 + 4);
                            const float4 b0 = *(const float4 *)(v1 + ch * 8), b1 = *(const float4 *)(v1 + ch * 8 + 4);
                            const uint32_t wq[4] = {q.x, q.y, q.z, q.w};
                            const float va[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                            const float vb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                            for (int e2 = 0; e2 < 4; ++e2) {
                                // |w| of the pair as floats (bf16 bits in the high half)
                                const float wlo = __uint_as_float((wq[e2] & 0x7fffu) << 16);
                                const float whi = __uint_as_float(wq[e2] & 0x7fff0000u);
                                xa0 = ru_fma(wlo, va[2 * e2], xa0);
                                xa1 = ru_fma(whi, va[2 * e2 + 1], xa1);
                                xb0 = ru_fma(wlo, vb[2 * e2], xb0);
                                xb1 = ru_fma(whi, vb[2 * e2 + 1], xb1);
                            }
                        }
                    } else if (mine) {
                        // one box: thread i takes row i over the slice's 64 inputs
                        const int r = i & 127;
                        const unsigned char *row = base + (m_of_thread - hf * Lt::MPU) * Lt::TILE + r * 128;
                        const float *v0 = (const float *)(x.smem + Lt::V_OFF) + s * 64;
#pragma unroll
                        for (int ch = 0; ch < 8; ++ch) {
                            const uint4 q = *(const uint4 *)(row + (((ch ^ (r & 7)) & 7) << 4));
                            const float4 a0 = *(const float4 *)(v0 + ch * 8), a1 = *(const float4 *)(v0 + ch * 8 + 4);
                            const uint32_t wq[4] = {q.x, q.y, q.z, q.w};
                            const float va[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
                            for (int e2 = 0; e2 < 4; ++e2) {
                                const float wlo = __uint_as_float((wq[e2] & 0x7fffu) << 16);
                                const float whi = __uint_as_float(wq[e2] & 0x7fff0000u);
                                xa0 = ru_fma(wlo, va[2 * e2], xa0);
                                xa1 = ru_fma(whi, va[2 * e2 + 1], xa1);
                            }
                        }
                    }
                    __syncwarp();
                    if (mine && x.lane == 0) ptx::mbar_arrive(&x.bars[2 + st]);
                    if (tid == PRODUCER) issue_upto(gg + 3);
                }
            }
            gring = g0 + Lt::S * Lt::UPS;
            if (!ptx::mbar_wait(&x.bars[4], accn & 1u, spins)) fail(x, p, 5);
            accn++;
            if (tid == PRODUCER) issue_upto(gring + 2);  // next layer's (or tile's) first units, during the epilogue
            float xown;
            if constexpr (NB == 2) {
                // the other group's box: hand over this thread's half of its |W_b| v
                float *xp = (float *)(x.smem + Lt::XP_OFF);
                xown = ru_add(g == 0 ? xa0 : xb0, g == 0 ? xa1 : xb1);
                xp[(1 - g) * H + i] = ru_add(g == 0 ? xb0 : xa0, g == 0 ? xb1 : xa1);
            } else {
                xown = ru_add(xa0, xa1);
            }
            ptx::tc_fence_after();
            if (__syncthreads_or(*x.abort_flag != 0)) break;  // every operand read of this layer is done
            // ---- epilogue of the group's box -------------------------------
            const float xacc = NB == 2 ? ru_add(xown, ((const float *)(x.smem + Lt::XP_OFF))[g * H + i]) : xown;
            if constexpr (KT > 64)
                hidden_epilogue_wide<H, SOUND, ACT, NBV>(x, p, tl, m_of_thread * TM_STRIDE + g * KT,
                                                         tl + (uint32_t)(m_of_thread * TM_STRIDE + NA + 2 * g), bias,
                                                         xacc);
            else
                hidden_epilogue<H, SOUND, ACT, KT, NBV>(x, p, tl, m_of_thread * TM_STRIDE + g * KT,
                                                        tl + (uint32_t)(m_of_thread * TM_STRIDE + NA + 2 * g), bias,
                                                        xacc);
        }
        if (__syncthreads_or(*x.abort_flag != 0)) break;
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
            // center (c_hi + c_lo rows) and x_inf parts: warp wg < NPART takes
            // part wg, its lanes split the inputs, warp reductions (rounded up
            // for the error and x_inf sums)
            if (x.wg < NPART) {
                const int pp = x.wg, lane = x.lane;
                float acc = 0.f, err = 0.f, xacc = 0.f;
                for (int s = pp; s < Lt::S; s += NPART) {
                    const unsigned char *XC = x.smem + Lt::XC_OFF + s * Lt::XC_SLICE;
#pragma unroll
                    for (int jj = 0; jj < 2; ++jj) {
                        const int j = lane + 32 * jj;
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
                const float *xr = (const float *)(x.smem + Lt::XR_OFF) + g * H;
                for (int j = pp * (H / NPART) + lane; j < (pp + 1) * (H / NPART); j += 32)
                    xacc = ru_fma(fabsf(wout[j]), xr[j], xacc);
                acc = warp_sum_f(acc);
                err = warp_sum_ru(err);
                xacc = warp_sum_ru(xacc);
                if (lane == 0) {
                    Y[pp * (KT + 2) + KT] = acc;
                    E[pp * (KT + 2) + KT] = err;
                    Y[pp * (KT + 2) + KT + 1] = xacc;
                }
            }
            group_sync(g, H);
            // final sums by warp g of the group (with two groups warps 0 and H/32 + 1), two noise
            // columns per lane; the radius and error sums are rounded up in
            // any order, and the FP32 error factors gam_out / gam_c_out bound
            // sequential summation, hence every other order too
            if (x.wg == g && bi < n) {
                float rad = 0.f, esum = 0.f, y0 = 0.f, ey = 0.f, yinf = 0.f;
                for (int k = x.lane; k < KT; k += 32) {
                    float yk = 0.f, ek = 0.f;
#pragma unroll
                    for (int pp = 0; pp < NPART; ++pp) {
                        yk += Y[pp * (KT + 2) + k];
                        ek = ru_add(ek, E[pp * (KT + 2) + k]);
                    }
                    rad = ru_add(rad, fabsf(yk));
                    esum = ru_add(esum, ek);
                }
                rad = warp_sum_ru(rad);
                esum = warp_sum_ru(esum);
                if (x.lane == 0) {
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
                        if (fabsf(lo) <= band || fabsf(hi) <= band) {
                            const int q = atomicAdd(out.flag_count, 1);
                            if (idx_ok(q, n, x.status, 105)) out.flag_list[q] = (int)bi;
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
    // leave: no MMA may still be writing TMEM; then free it
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 0) ptx::tmem_dealloc(x.tmem, Lt::TMEM_COLS);
}

}  // namespace tc

// Launch of one instantiation; the dispatch over the width, the precision
// form and the activation rule for one kept-symbol count KT.
template <int H, bool SOUND, int ACT, int KT>
static cudaError_t launch_one(const TcParams &p, const BoxSrc &src, const BoundOut &out, int grid, cudaStream_t st) {
    constexpr int NBV = tc::boxes_per_tile(H, KT);
    using Lt = tc::Layout<H, KT, NBV>;
    const int smem = Lt::ALLOC;
    cudaError_t e = cudaFuncSetAttribute(tc::tc_bound_kernel<H, SOUND, ACT, KT, NBV>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    tc::tc_bound_kernel<H, SOUND, ACT, KT, NBV><<<grid, Lt::NT, smem, st>>>(p, src, out);
    return cudaGetLastError();
}

template <int H, int ACT, int KT>
static cudaError_t launch_act(bool sound, const TcParams &p, const BoxSrc &src, const BoundOut &out, int grid,
                              cudaStream_t st) {
    return sound ? launch_one<H, true, ACT, KT>(p, src, out, grid, st)
                 : launch_one<H, false, ACT, KT>(p, src, out, grid, st);
}

template <int H, int KT>
static cudaError_t launch_h(bool sound, const TcParams &p, const BoxSrc &src, const BoundOut &out, int grid,
                            cudaStream_t st) {
    switch (p.act) {
        case SRA_ACT_RELU: return launch_act<H, SRA_ACT_RELU, KT>(sound, p, src, out, grid, st);
        case SRA_ACT_ELU: return launch_act<H, SRA_ACT_ELU, KT>(sound, p, src, out, grid, st);
        case SRA_ACT_SIN: return launch_act<H, SRA_ACT_SIN, KT>(sound, p, src, out, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int KT>
cudaError_t launch_tc_bound_kt(int H, bool sound, const TcParams &p, const BoxSrc &src, const BoundOut &out,
                               int grid, cudaStream_t st) {
    if (H == 512) {
        if constexpr (KT <= 64) return launch_h<512, KT>(sound, p, src, out, grid, st);
        else return cudaErrorInvalidValue;  // 4 M tiles x (128 + 16) columns exceed TMEM
    }
    if (H == 256) return launch_h<256, KT>(sound, p, src, out, grid, st);
    if (H == 128) return launch_h<128, KT>(sound, p, src, out, grid, st);
    return cudaErrorInvalidValue;
}

}  // namespace sra
