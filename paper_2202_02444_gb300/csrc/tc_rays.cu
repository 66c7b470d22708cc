// CastRay (Proc. 2) with the hidden layers on the tensor cores (tcgen05, BF16).
//
// One persistent CTA per SM keeps NR = 8 ray slots in flight and refills a
// slot from a global counter when its ray ends. Every march step bounds each
// slot's segment [t, t+sigma] with affine-fixed arithmetic (the one noise
// symbol v = (sigma/2) r; every new symbol goes to x_inf, Sec. 3.3) and
// evaluates f at p + (t+delta) r in the same pass (Proc. 2).
//
// Hidden layer l as two tensor-core products into TMEM (FP32 accumulation):
//   D  = (W_b + W_r) [c_hi c_lo p_hi p_lo A_hi A_lo]     48 operand rows
//   Dx = (|W_b| + sign(W_b) W_r) [x_hi x_lo]              16 operand rows
// W = W_b + W_r is the BF16 hi/lo split of the FP32 weights (|W_b + W_r| =
// |W_b| + sign(W_b) W_r, since |W_r| <= 2^-8 |W_b|) and every operand value
// rides as a BF16 hi/lo pair, so each product keeps about 16 significant bits
// before the FP32 sums. The weights stream from L2 by TMA in 32 KB stages of
// (128-row tile, 64-wide K slice) pairs through a four-stage ring, running
// ahead across layers and march steps. The positional encoding, the first
// layer, the activation rules (App. A), the output layer and the march state
// run on the SIMT cores in FP32. Plain arithmetic: no rounding radius.
//
// Every wait is bounded; a wait that runs out sets the status word, the CTA
// drains the copies it started (bounded again), frees TMEM and exits.
#include <cuda_bf16.h>

#include "sra_common.cuh"
#include "tc_ptx.cuh"
#include "tc_rays.h"

namespace sra {
namespace tcr {

constexpr int NR = 8;       // ray slots per CTA
constexpr int NCOL = 48;    // operand rows of D: 6 per ray
constexpr int NXI = 16;     // operand rows of Dx: 2 per ray
constexpr int MAXDIN = 64;  // network input width (3 + 6 * octaves) bound
constexpr int NSTG = 4;     // weight ring stages
constexpr int LA = NSTG - 1;
constexpr uint32_t kSpin = 1u << 22;
enum { C_HI = 0, C_LO = 8, P_HI = 16, P_LO = 24, A_HI = 32, A_LO = 40 };
enum { X_HI = 0, X_LO = 8 };

struct RaySlot {
    long long idx;
    float t, sigma;
    int f0pos, iters, live, pad;
};

template <int H> struct RL {
    static constexpr int MT = H / 128, S = H / 64;
    static constexpr int TILE = 128 * 128;                // one 128 x 64 BF16 tile
    static constexpr int STAGE = 2 * TILE;                // a pair of tiles
    static constexpr int UNITS = 2 * S * MT;              // stages per hidden layer
    static constexpr int W_OFF = 0;
    static constexpr int XB_OFF = NSTG * STAGE;
    static constexpr int XB_SLICE = NCOL * 128;
    static constexpr int XI_OFF = XB_OFF + S * XB_SLICE;
    static constexpr int XI_SLICE = NXI * 128;
    static constexpr int PE_OFF = XI_OFF + S * XI_SLICE;  // pe[MAXDIN][NR] float4 (c, A, x_inf, p)
    static constexpr int INP_OFF = PE_OFF + MAXDIN * NR * 16;  // segment inputs [NR][12]
    static constexpr int NPART = H / 32;
    static constexpr int OUTP_OFF = INP_OFF + NR * 12 * 4;     // output partial sums [4 NR][NPART]
    static constexpr int WOUT_OFF = OUTP_OFF + 4 * NR * NPART * 4;
    static constexpr int RAY_OFF = WOUT_OFF + H * 4;
    static constexpr int BAR_OFF = RAY_OFF + NR * (int)sizeof(RaySlot);
    static constexpr int MISC_OFF = BAR_OFF + 128;
    static constexpr int BYTES = MISC_OFF + 64;
    static constexpr int ALLOC = BYTES + 1024;
    static_assert(XB_OFF % 1024 == 0 && XB_SLICE % 1024 == 0 && XI_SLICE % 1024 == 0, "operand alignment");
    static_assert(ALLOC <= 232448, "shared memory");
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

// Operand rows of neuron i (the next layer's K index) for ray slot r.
template <int H>
__device__ __forceinline__ void write_rows(unsigned char *sm, int i, int r, float c, float A, float xi, float p) {
    using L = RL<H>;
    const uint32_t kk = (uint32_t)(i & 63);
    unsigned char *xb = sm + L::XB_OFF + (i >> 6) * L::XB_SLICE;
    unsigned char *xs = sm + L::XI_OFF + (i >> 6) * L::XI_SLICE;
    put_pair(xb, C_HI + r, C_LO + r, kk, c);
    put_pair(xb, P_HI + r, P_LO + r, kk, p);
    put_pair(xb, A_HI + r, A_LO + r, kk, A);
    put_pair(xs, X_HI + r, X_LO + r, kk, xi);
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

struct Ring {  // producer / MMA state, held by thread 0
    uint32_t ld_next, mma_next;
};

// Issue the TMA copies of ring unit gi into stage gi % NSTG once the MMAs of
// that stage's previous use have completed.
template <int H>
__device__ __forceinline__ bool ring_load(unsigned char *sm, uint64_t *bars, const TcRayParams &p, int NL,
                                          uint32_t gi) {
    using L = RL<H>;
    const uint32_t st = gi % NSTG, use = gi / NSTG;
    if (!ptx::mbar_wait(&bars[NSTG + st], (use & 1u) ^ 1u, kSpin)) return false;
    const uint32_t u = gi % L::UNITS;
    const int layer = (int)((gi / L::UNITS) % (uint32_t)NL);
    const int pair = (int)(u & 1u), ms = (int)(u >> 1);
    const int s = ms / L::MT, m = ms % L::MT;
    const CUtensorMap *m0 = pair ? &p.wa[layer] : &p.wb[layer];
    const CUtensorMap *m1 = pair ? &p.ws[layer] : &p.wr[layer];
    unsigned char *base = sm + L::W_OFF + st * L::STAGE;
    ptx::mbar_arrive_expect_tx(&bars[st], L::STAGE);
    ptx::tma_load_2d(base, m0, s * 64, m * 128, &bars[st]);
    ptx::tma_load_2d(base + L::TILE, m1, s * 64, m * 128, &bars[st]);
    return true;
}

template <int H>
__global__ void __launch_bounds__(H, 1) tc_ray_kernel(const __grid_constant__ TcRayParams p) {
    using L = RL<H>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sm = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, i = tid;
    // bars: [0, NSTG) stage full, [NSTG, 2 NSTG) stage empty, then layer done, drain
    uint64_t *bars = (uint64_t *)(sm + L::BAR_OFF);
    uint64_t *acc_bar = &bars[2 * NSTG], *drain_bar = &bars[2 * NSTG + 1];
    uint32_t *tmem_slot = (uint32_t *)(sm + L::MISC_OFF);
    int *abort_flag = (int *)(sm + L::MISC_OFF + 4);
    RaySlot *slots = (RaySlot *)(sm + L::RAY_OFF);
    float4 *pe = (float4 *)(sm + L::PE_OFF);
    float *inp = (float *)(sm + L::INP_OFF);
    float *outp = (float *)(sm + L::OUTP_OFF);
    float *wout = (float *)(sm + L::WOUT_OFF);
    const int NL = p.L - 2;  // hidden H -> H layers
    if (tid == 0) {
        for (int k = 0; k < 2 * NSTG + 2; ++k) ptx::mbar_init(&bars[k], 1);
        ptx::fence_mbar_init();
        *abort_flag = 0;
    }
    if (tid < NR) {
        slots[tid].idx = -1;
        slots[tid].live = 0;
    }
    for (int e = tid; e < (L::S * (L::XB_SLICE + L::XI_SLICE)) / 4; e += H)
        ((uint32_t *)(sm + L::XB_OFF))[e] = 0u;
    wout[tid] = p.wout[tid];
    if (warp == 0) ptx::tmem_alloc(tmem_slot, 256);
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int m_of = i >> 7;
    const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(m_of * 64);
    Ring ring = {0u, 0u};
    uint32_t accn = 0;
    auto fail = [&](int code) {
        *abort_flag = 1;
        atomicExch(p.status, code);
    };

    for (;;) {
        // ---- ray slots: refill, then the segment and point of this step -------
        if (tid < NR) {
            RaySlot &s = slots[tid];
            if (s.idx < 0) {
                const unsigned long long q = atomicAdd(p.next, 1ull);
                if ((long long)q < p.n) {
                    s.idx = (long long)q;
                    s.t = 0.f;
                    s.sigma = p.sigma0;
                    s.iters = 0;
                    s.f0pos = p.f0[q] >= 0.f;
                    s.live = 1;
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
                }
            } else {
                for (int d = 0; d < 9; ++d) in[d] = 0.f;
            }
        }
        const bool any = __syncthreads_or(tid < NR && slots[tid].live);
        if (!any || *abort_flag) break;
        // ---- input rows and positional encoding: sin(pi t), cos(pi t), t = 2^k x
        if (i < p.din) {
            int d = i, k = -1;
            bool is_cos = false;
            if (i >= 3) {
                const int q = i - 3;
                k = q / 6;
                is_cos = (q % 6) >= 3;
                d = q % 3;
            }
            for (int r = 0; r < NR; ++r) {
                const float *in = inp + r * 12;
                if (k < 0) {
                    pe[i * NR + r] = make_float4(in[d], in[3 + d], 0.f, in[6 + d]);
                } else {
                    const float sc = (float)(1 << k), sh = is_cos ? 0.5f : 0.f;
                    const float ct = sc * in[d] + sh, at = sc * in[3 + d];
                    const float rad = fabsf(at);
                    float a, b, gm;
                    linearize_sinpi<float>(ct - rad, ct + rad, a, b, gm);
                    pe[i * NR + r] = make_float4(a * ct + b, at * a, fabsf(gm), sinpi_t(sc * in[6 + d] + sh));
                }
            }
        }
        __syncthreads();
        // ---- first layer (din -> H) on the SIMT cores -------------------------
        {
            float ac[NR], aa[NR], ax[NR], ap[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) ac[r] = aa[r] = ax[r] = ap[r] = 0.f;
            for (int j = 0; j < p.din; ++j) {
                const float w = __ldg(p.W0t + (size_t)j * H + i), aw = fabsf(w);
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const float4 v = pe[j * NR + r];
                    ac[r] = fmaf(w, v.x, ac[r]);
                    aa[r] = fmaf(w, v.y, aa[r]);
                    ax[r] = fmaf(aw, v.z, ax[r]);
                    ap[r] = fmaf(w, v.w, ap[r]);
                }
            }
            const float b0 = __ldg(p.b[0] + i);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                float c = ac[r] + b0, A = aa[r], xi = ax[r], pp = ap[r] + b0;
                activate(p.act[0], p.slope, c, A, xi, pp);
                write_rows<H>(sm, i, r, c, A, xi, pp);
            }
        }
        // ---- hidden layers on the tensor cores ----------------------------------
        for (int l = 1; l <= NL; ++l) {
            ptx::fence_proxy_async();  // operand writes -> async proxy
            ptx::tc_fence_before();    // TMEM reads of the previous layer are done
            __syncthreads();
            if (*abort_flag) break;
            if (tid == 0) {
                bool ok = true;
                while (ok && ring.ld_next < ring.mma_next + LA) {
                    ok = ring_load<H>(sm, bars, p, NL, ring.ld_next);
                    if (ok) ++ring.ld_next;
                }
                const uint32_t id = ptx::idesc_bf16(128, NCOL), ix = ptx::idesc_bf16(128, NXI);
                for (int u = 0; u < L::UNITS && ok; ++u) {
                    const uint32_t gi = ring.mma_next, st = gi % NSTG;
                    if (!ptx::mbar_wait(&bars[st], (gi / NSTG) & 1u, kSpin)) { ok = false; break; }
                    ptx::tc_fence_after();
                    const int pair = u & 1, ms = u >> 1, s = ms / L::MT, m = ms % L::MT;
                    unsigned char *base = sm + L::W_OFF + st * L::STAGE;
                    const uint32_t b_addr = pair ? ptx::smem_u32(sm + L::XI_OFF + s * L::XI_SLICE)
                                                 : ptx::smem_u32(sm + L::XB_OFF + s * L::XB_SLICE);
                    const uint32_t d_col = tmem + (uint32_t)(m * 64 + (pair ? NCOL : 0));
                    const uint32_t idesc = pair ? ix : id;
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint64_t bd = ptx::desc_kmajor_sw128(b_addr) + 2 * ks;
                        const uint64_t a0 = ptx::desc_kmajor_sw128(ptx::smem_u32(base)) + 2 * ks;
                        const uint64_t a1 = ptx::desc_kmajor_sw128(ptx::smem_u32(base + L::TILE)) + 2 * ks;
                        ptx::mma_bf16(d_col, a0, bd, idesc, (s | ks) ? 1u : 0u);
                        ptx::mma_bf16(d_col, a1, bd, idesc, 1u);
                    }
                    ptx::mma_commit(&bars[NSTG + st]);
                    if (u + 1 == L::UNITS) ptx::mma_commit(acc_bar);
                    ++ring.mma_next;
                    while (ok && ring.ld_next < ring.mma_next + LA) {
                        ok = ring_load<H>(sm, bars, p, NL, ring.ld_next);
                        if (ok) ++ring.ld_next;
                    }
                }
                if (!ok) fail(6);
            }
            __syncthreads();
            if (*abort_flag) break;
            if (!ptx::mbar_wait(acc_bar, accn & 1u, kSpin)) fail(7);
            accn++;
            ptx::tc_fence_after();
            __syncthreads();
            if (*abort_flag) break;
            // epilogue: neuron i of every ray slot; the layer's operands are free
            float v[64];
#pragma unroll
            for (int q = 0; q < 4; ++q) ptx::tmem_ld16(tl + q * 16, v + q * 16);
            ptx::tmem_wait_ld();
            const float bias = __ldg(p.b[l] + i);
            const int act = p.act[l];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                float c = (v[C_HI + r] + v[C_LO + r]) + bias;
                float pp = (v[P_HI + r] + v[P_LO + r]) + bias;
                float A = v[A_HI + r] + v[A_LO + r];
                float xi = v[NCOL + X_HI + r] + v[NCOL + X_LO + r];
                activate(act, p.slope, c, A, xi, pp);
                write_rows<H>(sm, i, r, c, A, xi, pp);
            }
        }
        __syncthreads();
        if (*abort_flag) break;
        // ---- output layer (H -> 1): 4 sums per ray, H/32 parts of 32 inputs each
        {
            const int q = tid & 31, part = tid >> 5, r = q >> 2, kind = q & 3;
            float acc = 0.f;
            for (int j = part * 32; j < part * 32 + 32; ++j) {
                const uint32_t kk = (uint32_t)(j & 63);
                const unsigned char *xb = sm + L::XB_OFF + (j >> 6) * L::XB_SLICE;
                const unsigned char *xs = sm + L::XI_OFF + (j >> 6) * L::XI_SLICE;
                const float w = wout[j];
                if (kind == 0) acc = fmaf(w, get_pair(xb, C_HI + r, C_LO + r, kk), acc);
                else if (kind == 1) acc = fmaf(w, get_pair(xb, A_HI + r, A_LO + r, kk), acc);
                else if (kind == 2) acc = fmaf(fabsf(w), get_pair(xs, X_HI + r, X_LO + r, kk), acc);
                else acc = fmaf(w, get_pair(xb, P_HI + r, P_LO + r, kk), acc);
            }
            outp[q * L::NPART + part] = acc;
        }
        __syncthreads();
        // ---- march step of each live slot (Proc. 2) -------------------------------
        if (tid < NR && slots[tid].live) {
            RaySlot &s = slots[tid];
            float sums[4];
            for (int kind = 0; kind < 4; ++kind) {
                float a = 0.f;
                for (int part = 0; part < L::NPART; ++part) a += outp[(tid * 4 + kind) * L::NPART + part];
                sums[kind] = a;
            }
            const float y0 = sums[0] + p.bout, rad = fabsf(sums[1]) + sums[2], fc = sums[3] + p.bout;
            s.iters += 1;
            bool done = false;
            float result = 0.f;
            if ((fc >= 0.f) != (s.f0pos != 0)) {  // DifferentSigns at t + delta
                done = true;
                result = s.t;
            } else {
                const int k = classify_range(y0 - rad, y0 + rad);
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
                s.idx = -1;
            }
        }
        __syncthreads();
    }
    // drain: the copies still in flight land before the CTA exits, and every
    // MMA issued (also after an abort) completes before TMEM is freed
    if (tid == 0) {
        for (uint32_t gi = ring.mma_next; gi < ring.ld_next; ++gi)
            if (!ptx::mbar_wait(&bars[gi % NSTG], (gi / NSTG) & 1u, kSpin)) {
                atomicExch(p.status, 8);
                break;
            }
        ptx::mma_commit(drain_bar);
        if (!ptx::mbar_wait(drain_bar, 0u, kSpin)) atomicExch(p.status, 9);
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 0) ptx::tmem_dealloc(tmem, 256);
}

}  // namespace tcr

int tc_ray_smem_bytes(int H) {
    return H == 512 ? tcr::RL<512>::ALLOC : (H == 256 ? tcr::RL<256>::ALLOC : (H == 128 ? tcr::RL<128>::ALLOC : 0));
}

int tc_ray_max_din() { return tcr::MAXDIN; }

template <int H> static cudaError_t launch_r(const TcRayParams &p, int grid, cudaStream_t st) {
    const int smem = tc_ray_smem_bytes(H);
    cudaError_t e = cudaFuncSetAttribute(tcr::tc_ray_kernel<H>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    tcr::tc_ray_kernel<H><<<grid, H, smem, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_tc_rays(int H, const TcRayParams &p, int grid, cudaStream_t st) {
    if (H == 512) return launch_r<512>(p, grid, st);
    if (H == 256) return launch_r<256>(p, grid, st);
    if (H == 128) return launch_r<128>(p, grid, st);
    return cudaErrorInvalidValue;
}

}  // namespace sra
