// Directed-rounding helpers and the activation rules of App. A Table
// "affine_nonlinearities" (ReLU, ELU, sin) in FP32 for one neuron, plain or
// sound (outward-rounded ranges, padded transcendentals, every rounding of
// the new centre and independent part accounted for), shared by the
// tensor-core bound and ray kernels.
#pragma once

#include <cuda_bf16.h>

#include "sra_common.cuh"

namespace sra {

// ---- directed-rounding helpers ----------------------------------------------
__device__ __forceinline__ float ru_add(float a, float b) { return __fadd_ru(a, b); }
__device__ __forceinline__ float rd_add(float a, float b) { return __fadd_rd(a, b); }
__device__ __forceinline__ float ru_mul(float a, float b) { return __fmul_ru(a, b); }
__device__ __forceinline__ float ru_fma(float a, float b, float c) { return __fmaf_ru(a, b, c); }

__device__ __forceinline__ float bf16_ru(float x) {  // smallest bf16 >= x (x >= 0)
    return __bfloat162float(__float2bfloat16_ru(x));
}

// The ReLU rule of App. A Table "affine_nonlinearities" for one neuron whose
// noise magnitudes sum to sa (rounded up), center c and independent part
// xinf: outward-rounded range, slope al, new-symbol magnitude ga, new center
// c2 and the new independent part xi. The sound form adds the rounding of c2
// and of every al * a entry (and its later BF16 rounding) to xi.
template <bool SOUND>
__device__ __forceinline__ void relu_rule(float sa, float c, float xinf, float u_b2u, float &al, float &ga, float &c2,
                                          float &xi) {
    const float rad = ru_add(sa, xinf);
    const float lo = rd_add(c, -rad), hi = ru_add(c, rad);
    float be;
    if (hi <= 0.f) { al = 0.f; be = 0.f; ga = 0.f; }
    else if (lo >= 0.f) { al = 1.f; be = 0.f; ga = 0.f; }
    else {
        // any slope in [0,1] is valid: g(x) = ReLU(x) - al x ranges over
        // [0, max(-al lo, hi (1 - al))] on [lo, hi], so the Chebyshev slope
        // hi / (hi - lo) may be approximate (fast division)
        al = fminf(fmaxf(__fdividef(hi, hi - lo), 0.f), 1.f);
        const float m1 = __fmul_ru(al, -lo);
        const float m2 = __fmul_ru(hi, __fadd_ru(1.f, -al));
        const float M = fmaxf(m1, m2);
        be = 0.5f * M;  // exact halving
        ga = be;
    }
    c2 = fmaf(al, c, be);
    xi = __fmul_ru(al, xinf);
    if (SOUND) {
        xi = ru_fma(fabsf(c2), 1.1920929e-07f, xi);  // one rounding: <= 2^-23 |c2|
        xi = ru_fma(__fmul_ru(al, sa), u_b2u, xi);
    }
}

// ELU(x) = x for x >= 0, else e^x - 1, bounded from above and below in FP32.
// expm1f is within 1 ulp of e^x - 1 (CUDA's documented maximum error), i.e.
// within 2^-23 of its result's magnitude; the bounds pad by 2^-22 of it plus
// the smallest normal float.
__device__ __forceinline__ float elu_pad(float e) { return ru_fma(fabsf(e), 2.3841858e-07f, 1.17549435e-38f); }
__device__ __forceinline__ float elu_up(float x) {
    if (x >= 0.f) return x;
    const float e = expm1f(x);
    return ru_add(e, elu_pad(e));
}
__device__ __forceinline__ float elu_dn(float x) {
    if (x >= 0.f) return x;
    const float e = expm1f(x);
    return rd_add(e, -elu_pad(e));
}

// The ELU rule of App. A Table "affine_nonlinearities" (reading R2) for one
// neuron, with the outputs of relu_rule. The slope is the FP32 Chebyshev
// (secant) slope; in the sound form any slope in [0, 1] is valid because the
// extremes of g(x) = ELU(x) - al x on the outward-rounded [lo, hi] are
// bounded directly: g is convex, so its maximum sits at an end (each end
// evaluated rounded up), and at any point x0 (here clamp(ln al, lo, hi)) the
// tangent gives min g >= g(x0) - |g'(x0)| max(x0 - lo, hi - x0), every term
// rounded outward (expf within 2 ulp, padded by 2^-21), and min g >= -1 - al
// hi. Then
// be = (r_u + r_l) / 2 and ga = max(r_u - be, be - r_l), rounded up.
template <bool SOUND>
__device__ __forceinline__ void elu_rule(float sa, float c, float xinf, float u_b2u, float &al, float &ga, float &c2,
                                         float &xi) {
    const float rad = ru_add(sa, xinf);
    const float lo = rd_add(c, -rad), hi = ru_add(c, rad);
    float be;
    if (lo >= 0.f) {
        al = 1.f; be = 0.f; ga = 0.f;
    } else if (!SOUND) {
        linearize<float>(SRA_ACT_ELU, SRA_SLOPE_CHEBYSHEV, lo, hi, al, be, ga);
    } else {
        float b0, g0;
        linearize<float>(SRA_ACT_ELU, SRA_SLOPE_CHEBYSHEV, lo, hi, al, b0, g0);
        al = fminf(fmaxf(al, 0.f), 1.f);
        const float r_u = fmaxf(ru_add(elu_up(lo), -__fmul_rd(al, lo)), ru_add(elu_up(hi), -__fmul_rd(al, hi)));
        const float x0 = al > 0.f ? fminf(fmaxf(logf(al), lo), hi) : lo;
        const float g_x0 = rd_add(elu_dn(x0), -__fmul_ru(al, x0));
        float slope_up;  // |ELU'(x0) - al|, rounded up
        if (x0 >= 0.f) {
            slope_up = ru_add(1.f, -al);
        } else {
            const float ex = expf(x0);
            slope_up = ru_fma(ex, 4.7683716e-07f, fmaxf(ru_add(ex, -al), ru_add(al, -ex)));
        }
        const float span = fmaxf(ru_add(x0, -lo), ru_add(hi, -x0));
        // also g >= -1 - al hi on [lo, hi] (ELU >= -1, al >= 0): the bound that
        // stays finite when the span overflows (fmaxf drops a NaN operand)
        const float r_l = fmaxf(rd_add(g_x0, -ru_mul(slope_up, span)), rd_add(-1.f, -__fmul_ru(al, hi)));
        be = 0.5f * (r_u + r_l);
        ga = fmaxf(ru_add(r_u, -be), ru_add(be, -r_l));
    }
    c2 = fmaf(al, c, be);
    xi = __fmul_ru(al, xinf);
    if (SOUND) {
        xi = ru_fma(fabsf(c2), 1.1920929e-07f, xi);  // one rounding: <= 2^-23 |c2|
        xi = ru_fma(__fmul_ru(al, sa), u_b2u, xi);
    }
}

// Bounds of al * (x - c) for floats x, c: the difference is bracketed by its
// two directed roundings, each product rounded outward.
__device__ __forceinline__ void slope_times_offset(float al, float x, float c, float &p_dn, float &p_up) {
    const float t0 = rd_add(x, -c), t1 = ru_add(x, -c);
    p_dn = fminf(__fmul_rd(al, t0), __fmul_rd(al, t1));
    p_up = fmaxf(__fmul_ru(al, t0), __fmul_ru(al, t1));
}

// The sin rule of App. A Table "affine_nonlinearities" (reading R3) for one
// neuron, with the outputs of relu_rule. The slope is the FP32 one of the
// table (from the cos range). The sound form bounds h(x) = sin(x) - al (x - c)
// on the outward-rounded [lo, hi] (the output is al (y - c) + c2 +- ga for
// the input form y of centre c, so c2 is the mid-point of that bound and
// carries no rounding of its own; measuring x from c keeps the products small
// when |c| is large, as on SIREN layers). Any slope is valid: the extremes of
// h lie at the ends or at the critical points +-acos(al) + 2 pi k inside
// [lo, hi], and each of those is within dx of one of the computed candidates
// (per family the first point >= lo and the last point <= hi, clamped to
// [lo, hi]), where dx = 2^-20 (|x| + 8) covers the FP32 error of acos, of
// 2 pi k and of the sums. Since |h''| <= 1 and h' vanishes at a true critical
// point x*, |h'| <= dx between x* and its candidate, so h(x*) is within dx^2
// of h at the candidate. The ends are exact floats; sinf is within 2 ulp
// (padded by 4 ulp of its result plus the smallest normal float). A range of
// 2 pi or more gives al = 0, c2 = 0, ga = 1.
template <bool SOUND>
__device__ __forceinline__ void sin_rule(float sa, float c, float xinf, float u_b2u, float &al, float &ga, float &c2,
                                         float &xi) {
    const float rad = ru_add(sa, xinf);
    const float lo = rd_add(c, -rad), hi = ru_add(c, rad);
    const float two_pi = 6.2831853f;
    if (!SOUND) {
        float be;
        linearize<float>(SRA_ACT_SIN, SRA_SLOPE_CHEBYSHEV, lo, hi, al, be, ga);
        c2 = fmaf(al, c, be);
    } else if (!(ru_add(hi, -lo) < two_pi)) {
        al = 0.f; c2 = 0.f; ga = 1.f;
    } else {
        float b0, g0;
        linearize<float>(SRA_ACT_SIN, SRA_SLOPE_CHEBYSHEV, lo, hi, al, b0, g0);
        al = fminf(fmaxf(al, -1.f), 1.f);
        const float ep = acosf(al);
        float cand[6];
        cand[0] = lo;
        cand[1] = hi;
        cand[2] = fminf(fmaxf(ep + two_pi * ceilf((lo - ep) / two_pi), lo), hi);
        cand[3] = fminf(fmaxf(ep + two_pi * floorf((hi - ep) / two_pi), lo), hi);
        cand[4] = fminf(fmaxf(-ep + two_pi * ceilf((lo + ep) / two_pi), lo), hi);
        cand[5] = fminf(fmaxf(-ep + two_pi * floorf((hi + ep) / two_pi), lo), hi);
        float r_u = -INFINITY, r_l = INFINITY, end_dn = INFINITY, end_up = -INFINITY;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const float x = cand[q];
            const float sv = sinf(x);
            float margin = ru_fma(fabsf(sv), 4.7683716e-07f, 1.17549435e-38f);
            if (q >= 2) {
                const float dx = ru_mul(ru_add(fabsf(x), 8.f), 9.5367432e-07f);
                margin = ru_fma(dx, dx, margin);
            }
            float p_dn, p_up;
            slope_times_offset(al, x, c, p_dn, p_up);
            if (q < 2) { end_dn = fminf(end_dn, p_dn); end_up = fmaxf(end_up, p_up); }
            r_u = fmaxf(r_u, ru_add(ru_add(sv, -p_dn), margin));
            r_l = fminf(r_l, rd_add(rd_add(sv, -p_up), -margin));
        }
        // al (x - c) is linear in x, so its range on [lo, hi] is that of the
        // ends, and h lies in [-1 - al (x - c), 1 - al (x - c)]
        r_u = fminf(r_u, ru_add(1.f, -end_dn));
        r_l = fmaxf(r_l, rd_add(-1.f, -end_up));
        c2 = 0.5f * (r_u + r_l);
        ga = fmaxf(ru_add(r_u, -c2), ru_add(c2, -r_l));
    }
    xi = __fmul_ru(fabsf(al), xinf);
    if (SOUND) xi = ru_fma(__fmul_ru(fabsf(al), sa), u_b2u, xi);
}

// The half-turn sin rule (y = sin(pi t), t in half-turns) of the positional
// encoding, with the outputs of relu_rule, sound: linearize_sinpi gives the
// slope al (per half-turn); h(t) = sinpi(t) - al (t - c) is bounded on the
// outward-rounded [lo, hi] at the ends and at the candidates of its critical
// points +-e + 2k, e = acos(al / pi) / pi. A candidate is within dt of its
// critical point, dt = 2^-10 + 2^-18 (|t| + 8): the computed al / pi is
// within 2^-21 of the exact one, which moves acos by at most sqrt(2^-20)
// even where acos is steepest, and acos, the division and the sums add
// less than 2^-18 (|t| + 8). With |h''| <= pi^2 and h' = 0 at the critical
// point, h there is within pi^2 dt^2 of h at its candidate. sinpif is padded
// by 4 ulp of its result plus the smallest normal float; the products
// al (t - c) bracket the rounded difference. A range of two half-turns or
// more gives al = 0, c2 = 0, ga = 1.
__device__ __forceinline__ void sinpi_rule_sound(float sa, float c, float xinf, float u_b2u, float &al, float &ga,
                                                 float &c2, float &xi) {
    const float rad = ru_add(sa, xinf);
    const float lo = rd_add(c, -rad), hi = ru_add(c, rad);
    if (!(ru_add(hi, -lo) < 2.f)) {
        al = 0.f; c2 = 0.f; ga = 1.f;
    } else {
        float b0, g0;
        linearize_sinpi<float>(lo, hi, al, b0, g0);
        const float az = fminf(fmaxf(al / 3.14159265f, -1.f), 1.f);
        const float e = acosf(az) / 3.14159265f;
        float cand[6];
        cand[0] = lo;
        cand[1] = hi;
        cand[2] = fminf(fmaxf(e + 2.f * ceilf((lo - e) / 2.f), lo), hi);
        cand[3] = fminf(fmaxf(e + 2.f * floorf((hi - e) / 2.f), lo), hi);
        cand[4] = fminf(fmaxf(-e + 2.f * ceilf((lo + e) / 2.f), lo), hi);
        cand[5] = fminf(fmaxf(-e + 2.f * floorf((hi + e) / 2.f), lo), hi);
        float r_u = -INFINITY, r_l = INFINITY, end_dn = INFINITY, end_up = -INFINITY;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const float x = cand[q];
            const float sv = sinpif(x);
            float margin = ru_fma(fabsf(sv), 4.7683716e-07f, 1.17549435e-38f);
            if (q >= 2) {
                const float dt = ru_fma(ru_add(fabsf(x), 8.f), 3.8146973e-06f, 9.765625e-04f);
                margin = ru_fma(9.8697f, ru_mul(dt, dt), margin);
            }
            float p_dn, p_up;
            slope_times_offset(al, x, c, p_dn, p_up);
            if (q < 2) { end_dn = fminf(end_dn, p_dn); end_up = fmaxf(end_up, p_up); }
            r_u = fmaxf(r_u, ru_add(ru_add(sv, -p_dn), margin));
            r_l = fminf(r_l, rd_add(rd_add(sv, -p_up), -margin));
        }
        r_u = fminf(r_u, ru_add(1.f, -end_dn));
        r_l = fmaxf(r_l, rd_add(-1.f, -end_up));
        c2 = 0.5f * (r_u + r_l);
        ga = fmaxf(ru_add(r_u, -c2), ru_add(c2, -r_l));
    }
    xi = __fmul_ru(fabsf(al), xinf);
    xi = ru_fma(__fmul_ru(fabsf(al), sa), u_b2u, xi);
}

}  // namespace sra
