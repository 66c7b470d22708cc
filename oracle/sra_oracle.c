/* FP64 oracle for range analysis of MLP implicit functions
 * (Sharp & Jacobson, "Spelunking the Deep", SIGGRAPH 2022).
 *
 * TEST INFRASTRUCTURE: used only by the tests, the smoke check and the CPU
 * baseline leg of the benchmark. No code, header, table or constant is shared
 * with the CUDA path.
 *
 * What each part follows:
 *   - interval arithmetic:                 Sec. 3.1
 *   - affine form, range, exact ops:       Sec. 3.2, Eq. (affine_def),
 *                                          Eq. (def_range), App. A Table
 *                                          "affine_update_rules"
 *   - nonlinearity update:                 Eq. (affine_func_update), App. A
 *                                          Table "affine_nonlinearities"
 *   - condensation policies:               Sec. 3.3 (full / fixed / truncate)
 *   - the distinguished x_inf coefficient: App. A (vector notation paragraph)
 *   - box initialisation:                  Proc. 1 and App. A
 *   - RangeBound:                          Proc. 1
 *   - CastRay:                             Proc. 2, App. B "Ray Casting"
 *   - BuildSpatialTree (fixed depth):      Proc. 3, Sec. 4.5, Sec. 4.7
 *
 * Readings taken where the paper is garbled or silent:
 *   R1 ReLU table: the third line's "delta" is gamma; u<=0 gives the zero map,
 *      l>=0 the identity.
 *   R2 ELU table: "x_l > 0" means l >= 0; r_l is the tangent intercept
 *      (alpha-1) - alpha*ln(alpha) at x* = ln(alpha); gamma = r_u - beta;
 *      l == u uses the derivative exp(l) as slope.
 *   R3 sin table: the second "max" is a "min"; the critical-point candidates
 *      are the first point >= l and the last point <= u of each family
 *      +-acos(alpha) + 2 pi k (the printed floor terms use l instead of u).
 *   R4 x_inf holds one independent coefficient per vector component; condensed
 *      magnitudes are added to it row by row.
 *   R5 truncate scores a column by its L1 norm over the vector's components,
 *      runs after every nonlinearity over the K old and the new columns,
 *      breaks ties by lower candidate index (old columns before new ones), and
 *      keeps the surviving columns in candidate order. K excludes x_inf.
 *   R6 classification is strict: lo > 0 is POSITIVE, hi < 0 is NEGATIVE.
 *   R7 Proc. 3 splits at the midpoint of the widest axis (the printed split
 *      vector holds the full width); ties go to the lowest axis.
 *   R8 positional encoding: [x, then per octave k: sin(2^k pi x_{0,1,2}),
 *      cos(2^k pi x_{0,1,2})], cos(z) = sin(z + pi/2); each sin row is a
 *      nonlinearity with its own new symbol; identity rows add none.
 *   R9 CastRay: a value f >= 0 counts as positive in DifferentSigns; the step
 *      is max(safety * sigma*, delta) (App. B uses safety 0.98).
 */
#include "sra_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TWO_PI (2.0 * M_PI)

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- scalars */

static double act_eval(int act, double x) {
    switch (act) {
    case ORC_ACT_RELU: return x > 0.0 ? x : 0.0;
    case ORC_ACT_ELU: return x > 0.0 ? x : expm1(x);
    case ORC_ACT_SIN: return sin(x);
    default: return x;
    }
}

/* Range of cos on [l,u], located through multiples of 2 pi (App. A). */
static void cos_range(double l, double u, double *lo, double *hi) {
    if (u - l >= TWO_PI) { *lo = -1.0; *hi = 1.0; return; }
    double cl = cos(l), cu = cos(u);
    *hi = cl > cu ? cl : cu;
    *lo = cl < cu ? cl : cu;
    /* a maximum 2 pi k inside [l,u] */
    if (TWO_PI * ceil(l / TWO_PI) <= u) *hi = 1.0;
    /* a minimum pi + 2 pi k inside [l,u] */
    if (TWO_PI * ceil((l - M_PI) / TWO_PI) + M_PI <= u) *lo = -1.0;
}

/* Range of sin on [l,u]: sin(x) = cos(x - pi/2). */
static void sin_range(double l, double u, double *lo, double *hi) {
    if (u - l >= TWO_PI) { *lo = -1.0; *hi = 1.0; return; }
    double sl = sin(l), su = sin(u);
    *hi = sl > su ? sl : su;
    *lo = sl < su ? sl : su;
    if (TWO_PI * ceil((l - M_PI / 2) / TWO_PI) + M_PI / 2 <= u) *hi = 1.0;
    if (TWO_PI * ceil((l + M_PI / 2) / TWO_PI) - M_PI / 2 <= u) *lo = -1.0;
}

void orc_interval_act(int act, double l, double u, double *lo, double *hi) {
    if (act == ORC_ACT_SIN) { sin_range(l, u, lo, hi); return; }
    /* ReLU, ELU and identity are monotone non-decreasing (Sec. 3.1 rules) */
    *lo = act_eval(act, l);
    *hi = act_eval(act, u);
}

static double clampd(double x, double a, double b) { return x < a ? a : (x > b ? b : x); }

/* App. A Table "affine_nonlinearities". */
void orc_linearize(int act, int slope, double l, double u, double *alpha,
                   double *beta, double *gamma) {
    double a = 1.0, b = 0.0, g = 0.0;
    if (act == ORC_ACT_RELU) {
        if (u <= 0.0) { a = 0.0; b = 0.0; g = 0.0; }
        else if (l >= 0.0) { a = 1.0; b = 0.0; g = 0.0; }
        else if (slope == ORC_SLOPE_MINRANGE) {
            /* smallest slope on [l,u]: the affine image spans exactly [0,u] */
            a = 0.0; b = 0.5 * u; g = 0.5 * u;
        } else {
            /* Chebyshev: alpha = secant slope, beta = gamma = (ReLU(l) - alpha l)/2 (R1) */
            a = u / (u - l);
            b = (0.0 - a * l) / 2.0;
            g = b;
        }
    } else if (act == ORC_ACT_ELU) {
        if (l >= 0.0) { a = 1.0; b = 0.0; g = 0.0; }
        else if (slope == ORC_SLOPE_MINRANGE) {
            /* ELU is convex and increasing: slope exp(l) = min derivative;
             * f(x) - a x is then non-decreasing on [l,u] */
            a = exp(l);
            double gl = act_eval(ORC_ACT_ELU, l) - a * l;
            double gu = act_eval(ORC_ACT_ELU, u) - a * u;
            b = 0.5 * (gu + gl);
            g = 0.5 * (gu - gl);
        } else {
            /* Chebyshev for a convex function (R2) */
            if (u > l) a = (act_eval(ORC_ACT_ELU, u) - act_eval(ORC_ACT_ELU, l)) / (u - l);
            else a = exp(l);
            double ru = act_eval(ORC_ACT_ELU, l) - a * l; /* secant intercept */
            double rl;                                    /* tangent intercept at x* = ln a */
            if (a > 0.0) rl = (a - 1.0) - a * log(a);
            else rl = -1.0;                               /* a ln a -> 0 as a -> 0 */
            b = (ru + rl) / 2.0;
            g = ru - b;
        }
    } else if (act == ORC_ACT_SIN) {
        /* R3: alpha from the cos range, extrema of sin(x) - alpha x over the
         * endpoints and the extreme critical points of both families */
        double sl, su;
        cos_range(l, u, &sl, &su);
        a = (sl + su) / 2.0;
        double ep = acos(clampd(a, -1.0, 1.0));
        double cand[6];
        int nc = 0;
        cand[nc++] = l;
        cand[nc++] = u;
        const double fam[2] = {ep, -ep};
        for (int f = 0; f < 2; ++f) {
            double c = fam[f];
            cand[nc++] = clampd(c + TWO_PI * ceil((l - c) / TWO_PI), l, u);
            cand[nc++] = clampd(c + TWO_PI * floor((u - c) / TWO_PI), l, u);
        }
        double ru = -INFINITY, rl = INFINITY;
        for (int i = 0; i < nc; ++i) {
            double v = sin(cand[i]) - a * cand[i];
            if (v > ru) ru = v;
            if (v < rl) rl = v;
        }
        b = (ru + rl) / 2.0;
        g = ru - b;
    }
    *alpha = a;
    *beta = b;
    *gamma = g;
}

/* ------------------------------------------------------------ affine forms */

/* (x0, X, x_inf) of App. A: m components, N shared noise symbols. */
typedef struct {
    int m, N;
    double *c;  /* m        base values x0 */
    double *A;  /* m x N    coefficients, row-major */
    double *xi; /* m        distinguished coefficient x_inf (R4) */
} aform;

static aform af_new(int m, int N) {
    aform f;
    f.m = m;
    f.N = N;
    f.c = (double *)calloc((size_t)m, sizeof(double));
    f.A = (double *)calloc((size_t)m * (N > 0 ? N : 1), sizeof(double));
    f.xi = (double *)calloc((size_t)m, sizeof(double));
    return f;
}

static void af_free(aform *f) {
    free(f->c);
    free(f->A);
    free(f->xi);
    f->c = f->A = f->xi = NULL;
}

/* Table "affine_update_rules": matrix multiplication then constant addition.
 * z0 = W x0 + b, Z = W X, z_inf = |W| x_inf. */
static aform af_linear(const aform *x, const double *W, const double *b, int out) {
    aform z = af_new(out, x->N);
    for (int i = 0; i < out; ++i) {
        const double *w = W + (size_t)i * x->m;
        double s0 = 0.0, si = 0.0;
        double *zr = z.A + (size_t)i * x->N;
        for (int j = 0; j < x->m; ++j) {
            s0 += w[j] * x->c[j];
            si += fabs(w[j]) * x->xi[j];
            const double *xr = x->A + (size_t)j * x->N;
            for (int k = 0; k < x->N; ++k) zr[k] += w[j] * xr[k];
        }
        z.c[i] = s0 + b[i];
        z.xi[i] = si;
    }
    return z;
}

/* Eq. (def_range) with the x_inf term: r_i = sum_k |X_ik| + x_inf_i. */
static double af_radius(const aform *f, int i) {
    double r = 0.0;
    const double *row = f->A + (size_t)i * f->N;
    for (int k = 0; k < f->N; ++k) r += fabs(row[k]);
    return r + f->xi[i];
}

typedef struct {
    double score;
    int idx;
} cand_t;

/* Test diagnostic: smallest relative gap between the last kept and the first
 * dropped truncate score seen since the last reset (per thread). A GPU that
 * sums scores in another order may keep the other column when this is tiny. */
static _Thread_local double t_sel_gap = INFINITY;

static int cand_cmp(const void *pa, const void *pb) {
    const cand_t *a = (const cand_t *)pa, *b = (const cand_t *)pb;
    if (a->score > b->score) return -1;
    if (a->score < b->score) return 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx ? 1 : 0);
}

/* Apply per-row linearisations (alpha, beta, gamma) as in
 * Eq. (affine_func_update) / Table "affine_update_rules" (nonlinearities row):
 * z0 = alpha x0 + beta, Z = [alpha X ; diag(gamma)], z_inf = |alpha| x_inf.
 * Only rows with newsym[i] != 0 introduce a new symbol. Then condense the
 * result with the policy of Sec. 3.3. Consumes f. */
static aform af_nonlinear(aform *f, const double *alpha, const double *beta,
                          const double *gamma, const unsigned char *newsym,
                          const orc_opts *o) {
    const int m = f->m, N = f->N;
    /* the new symbols, one per flagged row, in row order */
    int nnew = 0;
    int *newrow = (int *)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
    for (int i = 0; i < m; ++i)
        if (newsym[i]) newrow[nnew++] = i;
    const int ncand = N + nnew;

    /* candidate matrix [alpha X | diag(gamma)] and scaled base terms */
    const size_t mrows = (size_t)(m > 0 ? m : 1), ncols = (size_t)(ncand > 0 ? ncand : 1);
    double *cand = (double *)calloc(mrows * ncols, sizeof(double));
    aform z;
    z.m = m;
    z.c = (double *)malloc(sizeof(double) * (size_t)m);
    z.xi = (double *)malloc(sizeof(double) * (size_t)m);
    for (int i = 0; i < m; ++i) {
        z.c[i] = alpha[i] * f->c[i] + beta[i];
        z.xi[i] = fabs(alpha[i]) * f->xi[i];
        const double *xr = f->A + (size_t)i * N;
        double *cr = cand + (size_t)i * ncand;
        for (int k = 0; k < N; ++k) cr[k] = alpha[i] * xr[k];
    }
    for (int q = 0; q < nnew; ++q) cand[(size_t)newrow[q] * ncand + N + q] = gamma[newrow[q]];

    /* which candidate columns survive (Sec. 3.3) */
    unsigned char *keep = (unsigned char *)calloc((size_t)(ncand > 0 ? ncand : 1), 1);
    if (o->arith == ORC_AFFINE_FULL) {
        for (int k = 0; k < ncand; ++k) keep[k] = 1;
    } else if (o->arith == ORC_AFFINE_FIXED) {
        /* only symbols of the original input domain survive; every new symbol
         * is condensed immediately */
        for (int k = 0; k < N; ++k) keep[k] = 1;
    } else { /* ORC_AFFINE_TRUNCATE (R5) */
        cand_t *cs = (cand_t *)malloc(sizeof(cand_t) * (size_t)(ncand > 0 ? ncand : 1));
        for (int k = 0; k < ncand; ++k) {
            double s = 0.0;
            for (int i = 0; i < m; ++i) s += fabs(cand[(size_t)i * ncand + k]);
            cs[k].score = s;
            cs[k].idx = k;
        }
        qsort(cs, (size_t)ncand, sizeof(cand_t), cand_cmp);
        int nk = o->K < ncand ? o->K : ncand;
        for (int q = 0; q < nk; ++q) keep[cs[q].idx] = 1;
        if (nk > 0 && nk < ncand) {
            /* equal zero scores are exact on any machine: no ambiguity */
            double top = cs[nk - 1].score;
            double g = (top > 0.0) ? (top - cs[nk].score) / top : INFINITY;
            if (g < t_sel_gap) t_sel_gap = g;
        }
        free(cs);
    }
    int nkeep = 0;
    for (int k = 0; k < ncand; ++k) nkeep += keep[k];

    /* condense: dropped magnitudes go to x_inf row by row (R4) */
    z.N = nkeep;
    z.A = (double *)calloc((size_t)m * (nkeep > 0 ? nkeep : 1), sizeof(double));
    for (int i = 0; i < m; ++i) {
        const double *cr = cand + (size_t)i * ncand;
        double *zr = z.A + (size_t)i * nkeep;
        int p = 0;
        double dropped = 0.0;
        for (int k = 0; k < ncand; ++k) {
            if (keep[k]) zr[p++] = cr[k];
            else dropped += fabs(cr[k]);
        }
        z.xi[i] += dropped;
    }
    free(keep);
    free(cand);
    free(newrow);
    af_free(f);
    return z;
}

/* Activation layer on an affine vector. */
static aform af_activation(aform *f, int act, const orc_opts *o) {
    if (act == ORC_ACT_IDENTITY) return *f; /* exact; no new symbol */
    const int m = f->m;
    double *al = (double *)malloc(sizeof(double) * (size_t)m);
    double *be = (double *)malloc(sizeof(double) * (size_t)m);
    double *ga = (double *)malloc(sizeof(double) * (size_t)m);
    unsigned char *ns = (unsigned char *)malloc((size_t)m);
    for (int i = 0; i < m; ++i) {
        double r = af_radius(f, i);
        orc_linearize(act, o->slope, f->c[i] - r, f->c[i] + r, &al[i], &be[i], &ga[i]);
        ns[i] = 1;
    }
    aform z = af_nonlinear(f, al, be, ga, ns, o);
    free(al);
    free(be);
    free(ga);
    free(ns);
    return z;
}

/* Positional encoding on an affine input (R8): 3 identity rows, then per
 * octave k the rows sin(2^k pi x_d) and cos(2^k pi x_d) = sin(2^k pi x_d + pi/2). */
static aform af_posenc(aform *x, int octaves, const orc_opts *o) {
    const int m = 3 + 6 * octaves, N = x->N;
    aform pre = af_new(m, N);
    double *al = (double *)malloc(sizeof(double) * (size_t)m);
    double *be = (double *)malloc(sizeof(double) * (size_t)m);
    double *ga = (double *)malloc(sizeof(double) * (size_t)m);
    unsigned char *ns = (unsigned char *)malloc((size_t)m);
    for (int i = 0; i < m; ++i) {
        int d, k = -1, is_cos = 0;
        if (i < 3) d = i;
        else {
            int q = i - 3;
            k = q / 6;
            is_cos = (q % 6) >= 3;
            d = q % 3;
        }
        double s = (k < 0) ? 1.0 : ldexp(M_PI, k);
        double shift = is_cos ? M_PI / 2 : 0.0;
        /* constant multiplication and constant addition rules */
        pre.c[i] = s * x->c[d] + shift;
        for (int j = 0; j < N; ++j) pre.A[(size_t)i * N + j] = s * x->A[(size_t)d * N + j];
        pre.xi[i] = fabs(s) * x->xi[d];
        if (k < 0) {
            al[i] = 1.0; be[i] = 0.0; ga[i] = 0.0; ns[i] = 0;
        } else {
            double r = af_radius(&pre, i);
            orc_linearize(ORC_ACT_SIN, o->slope, pre.c[i] - r, pre.c[i] + r, &al[i], &be[i], &ga[i]);
            ns[i] = 1;
        }
    }
    af_free(x);
    aform z = af_nonlinear(&pre, al, be, ga, ns, o);
    free(al);
    free(be);
    free(ga);
    free(ns);
    return z;
}

static const double *layer_W(const orc_net *net, int l) {
    size_t off = 0;
    for (int k = 0; k < l; ++k)
        off += (size_t)net->widths[k + 1] * net->widths[k] + net->widths[k + 1];
    return net->params + off;
}

static const double *layer_b(const orc_net *net, int l) {
    return layer_W(net, l) + (size_t)net->widths[l + 1] * net->widths[l];
}

static int classify(double lo, double hi) {
    if (lo > 0.0) return ORC_POSITIVE; /* R6 */
    if (hi < 0.0) return ORC_NEGATIVE;
    return ORC_UNKNOWN;
}

/* ---------------------------------------------------------- plain forward */

double orc_eval(const orc_net *net, const double *x) {
    int maxw = 3 + 6 * net->pe_octaves;
    for (int l = 0; l <= net->n_layers; ++l)
        if (net->widths[l] > maxw) maxw = net->widths[l];
    double *a = (double *)malloc(sizeof(double) * (size_t)maxw);
    double *b = (double *)malloc(sizeof(double) * (size_t)maxw);
    int m = 3;
    for (int d = 0; d < 3; ++d) a[d] = x[d];
    if (net->pe_octaves > 0) {
        for (int k = 0; k < net->pe_octaves; ++k)
            for (int q = 0; q < 6; ++q) {
                double z = ldexp(M_PI, k) * x[q % 3] + ((q >= 3) ? M_PI / 2 : 0.0);
                a[3 + 6 * k + q] = sin(z);
            }
        m = 3 + 6 * net->pe_octaves;
    }
    for (int l = 0; l < net->n_layers; ++l) {
        const double *W = layer_W(net, l), *bb = layer_b(net, l);
        int out = net->widths[l + 1];
        for (int i = 0; i < out; ++i) {
            double s = 0.0;
            for (int j = 0; j < m; ++j) s += W[(size_t)i * m + j] * a[j];
            s += bb[i];
            b[i] = (l < net->n_layers - 1) ? act_eval(net->acts[l], s) : s;
        }
        double *t = a; a = b; b = t;
        m = out;
    }
    double y = a[0];
    free(a);
    free(b);
    return y;
}

void orc_eval_batch(const orc_net *net, int64_t n, const double *x, double *out, int nthreads) {
    if (nthreads <= 0) nthreads = orc_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
    for (int64_t i = 0; i < n; ++i) out[i] = orc_eval(net, x + 3 * i);
}

/* ------------------------------------------------------------- RangeBound */

static int range_interval(const orc_net *net, const double *c, const double *axes, int s,
                          double *lo, double *hi) {
    int maxw = 3 + 6 * net->pe_octaves;
    for (int l = 0; l <= net->n_layers; ++l)
        if (net->widths[l] > maxw) maxw = net->widths[l];
    double *L0 = (double *)malloc(sizeof(double) * (size_t)maxw);
    double *U0 = (double *)malloc(sizeof(double) * (size_t)maxw);
    double *L1 = (double *)malloc(sizeof(double) * (size_t)maxw);
    double *U1 = (double *)malloc(sizeof(double) * (size_t)maxw);
    /* interval hull of the box */
    for (int d = 0; d < 3; ++d) {
        double r = 0.0;
        for (int k = 0; k < s; ++k) r += fabs(axes[k * 3 + d]);
        L0[d] = c[d] - r;
        U0[d] = c[d] + r;
    }
    int m = 3;
    if (net->pe_octaves > 0) {
        for (int k = 0; k < net->pe_octaves; ++k)
            for (int q = 0; q < 6; ++q) {
                double sc = ldexp(M_PI, k), sh = (q >= 3) ? M_PI / 2 : 0.0;
                int d = q % 3;
                sin_range(sc * L0[d] + sh, sc * U0[d] + sh, &L0[3 + 6 * k + q], &U0[3 + 6 * k + q]);
            }
        m = 3 + 6 * net->pe_octaves;
    }
    for (int l = 0; l < net->n_layers; ++l) {
        const double *W = layer_W(net, l), *bb = layer_b(net, l);
        int out = net->widths[l + 1];
        for (int i = 0; i < out; ++i) {
            /* sum of scaled intervals plus a constant (Sec. 3.1 rules) */
            double sl = bb[i], su = bb[i];
            for (int j = 0; j < m; ++j) {
                double w = W[(size_t)i * m + j];
                double p = w * L0[j], q = w * U0[j];
                sl += p < q ? p : q;
                su += p < q ? q : p;
            }
            if (l < net->n_layers - 1) orc_interval_act(net->acts[l], sl, su, &L1[i], &U1[i]);
            else { L1[i] = sl; U1[i] = su; }
        }
        double *t;
        t = L0; L0 = L1; L1 = t;
        t = U0; U0 = U1; U1 = t;
        m = out;
    }
    *lo = L0[0];
    *hi = U0[0];
    free(L0); free(U0); free(L1); free(U1);
    return classify(*lo, *hi);
}

int orc_range_bound(const orc_net *net, const orc_opts *o, const double *c,
                    const double *axes, int s, double *lo, double *hi,
                    double *y0, double *rad) {
    if (o->arith == ORC_INTERVAL) {
        int cls = range_interval(net, c, axes, s, lo, hi);
        *y0 = 0.5 * (*lo + *hi);
        *rad = 0.5 * (*hi - *lo);
        return cls;
    }
    /* Proc. 1 line 1 and App. A: x0 = c, X = [v_0 .. v_{s-1}], x_inf = 0 */
    aform f = af_new(3, s);
    for (int d = 0; d < 3; ++d) {
        f.c[d] = c[d];
        for (int k = 0; k < s; ++k) f.A[(size_t)d * s + k] = axes[k * 3 + d];
    }
    if (net->pe_octaves > 0) f = af_posenc(&f, net->pe_octaves, o);
    /* Proc. 1 line 2: propagate through the MLP */
    for (int l = 0; l < net->n_layers; ++l) {
        aform z = af_linear(&f, layer_W(net, l), layer_b(net, l), net->widths[l + 1]);
        af_free(&f);
        if (l < net->n_layers - 1) z = af_activation(&z, net->acts[l], o);
        f = z;
    }
    /* Proc. 1 line 3: bound the output */
    double r = af_radius(&f, 0);
    *y0 = f.c[0];
    *rad = r;
    *lo = f.c[0] - r;
    *hi = f.c[0] + r;
    af_free(&f);
    return classify(*lo, *hi);
}

void orc_bound_boxes(const orc_net *net, const orc_opts *o, int64_t n,
                     const double *centers, const double *halfw, double *lo,
                     double *hi, double *y0, double *rad, int32_t *cls,
                     double *sel_gap, int nthreads) {
    if (nthreads <= 0) nthreads = orc_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (int64_t i = 0; i < n; ++i) {
        double axes[9] = {0};
        for (int d = 0; d < 3; ++d) axes[d * 3 + d] = halfw[3 * i + d];
        double l, h, c0, r;
        t_sel_gap = INFINITY;
        int k = orc_range_bound(net, o, centers + 3 * i, axes, 3, &l, &h, &c0, &r);
        if (sel_gap) sel_gap[i] = t_sel_gap;
        if (lo) lo[i] = l;
        if (hi) hi[i] = h;
        if (y0) y0[i] = c0;
        if (rad) rad[i] = r;
        if (cls) cls[i] = k;
    }
}

/* ------------------------------------------------------- BuildSpatialTree */

/* Number of halvings of each axis at a k-d level: replay the widest-axis
 * rule of Proc. 3 from the root extents (R7). */
static void kd_counts(const double *xl, const double *xu, int level, int *n3) {
    double e[3] = {xu[0] - xl[0], xu[1] - xl[1], xu[2] - xl[2]};
    n3[0] = n3[1] = n3[2] = 0;
    for (int k = 0; k < level; ++k) {
        int a = 0;
        if (e[1] > e[a]) a = 1;
        if (e[2] > e[a]) a = 2;
        e[a] *= 0.5;
        n3[a]++;
    }
}

static void node_box(const double *xl, const double *xu, int split, const orc_node *nd,
                     double *lo, double *hi) {
    int n3[3];
    if (split == ORC_SPLIT_OCTREE) n3[0] = n3[1] = n3[2] = nd->level;
    else kd_counts(xl, xu, nd->level, n3);
    const int idx[3] = {nd->ix, nd->iy, nd->iz};
    for (int d = 0; d < 3; ++d) {
        double w = ldexp(xu[d] - xl[d], -n3[d]);
        lo[d] = xl[d] + w * idx[d];
        hi[d] = lo[d] + w;
    }
}

typedef struct {
    const orc_net *net;
    const orc_opts *o;
    const double *xl, *xu;
    int max_level, split;
    orc_node *out;
    int64_t cap, n;
    int64_t counts[5];
    double delta;  /* > 0: the convergence test of Proc. 3 for small nodes */
} tree_ctx;

static void tree_emit(tree_ctx *t, orc_node nd, int cls) {
    nd.cls = cls;
    if (t->n < t->cap) t->out[t->n] = nd;
    t->n++;
    t->counts[cls == ORC_POSITIVE ? 0 : (cls == ORC_NEGATIVE ? 1 : 2)]++;
}

static void tree_rec(tree_ctx *t, orc_node nd) {
    double lo[3], hi[3];
    node_box(t->xl, t->xu, t->split, &nd, lo, hi);
    /* Proc. 3: center and diagonal axes from the node bounds */
    double c[3], axes[9] = {0};
    for (int d = 0; d < 3; ++d) {
        c[d] = 0.5 * (lo[d] + hi[d]);
        axes[d * 3 + d] = hi[d] - c[d];
    }
    double l, h, y0, r;
    int cls = orc_range_bound(t->net, t->o, c, axes, 3, &l, &h, &y0, &r);
    t->counts[3]++;
    if (cls != ORC_UNKNOWN) { tree_emit(t, nd, cls); return; }
    /* convergence of Proc. 3: a node narrower than delta / sqrt(3) whose
       sample points, one per face (the face centres), take both signs lies
       within delta of the level set and is returned as it is */
    if (t->delta > 0.0) {
        double wmax = 0.0;
        for (int d = 0; d < 3; ++d)
            if (hi[d] - lo[d] > wmax) wmax = hi[d] - lo[d];
        if (wmax < t->delta / sqrt(3.0)) {
            int neg = 0, pos = 0;
            for (int d = 0; d < 3; ++d)
                for (int side = 0; side < 2; ++side) {
                    double pf[3] = {c[0], c[1], c[2]};
                    pf[d] = side ? hi[d] : lo[d];
                    const double f = orc_eval(t->net, pf);
                    neg |= f < 0.0;
                    pos |= f > 0.0;
                }
            if (neg && pos) {
                t->counts[4]++;
                tree_emit(t, nd, ORC_UNKNOWN);
                return;
            }
        }
    }
    /* fixed-depth stop (the alternative named in Proc. 3 and used by Sec. 4.7) */
    if (nd.level >= t->max_level) { tree_emit(t, nd, ORC_UNKNOWN); return; }
    if (t->split == ORC_SPLIT_OCTREE) {
        for (int q = 0; q < 8; ++q) {
            orc_node ch = nd;
            ch.level = (uint16_t)(nd.level + 1);
            ch.ix = (uint16_t)(2 * nd.ix + (q & 1));
            ch.iy = (uint16_t)(2 * nd.iy + ((q >> 1) & 1));
            ch.iz = (uint16_t)(2 * nd.iz + ((q >> 2) & 1));
            tree_rec(t, ch);
        }
    } else {
        /* widest dimension, lowest axis on ties (R7) */
        double e[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
        int a = 0;
        if (e[1] > e[a]) a = 1;
        if (e[2] > e[a]) a = 2;
        for (int q = 0; q < 2; ++q) {
            orc_node ch = nd;
            ch.level = (uint16_t)(nd.level + 1);
            if (a == 0) ch.ix = (uint16_t)(2 * nd.ix + q);
            if (a == 1) ch.iy = (uint16_t)(2 * nd.iy + q);
            if (a == 2) ch.iz = (uint16_t)(2 * nd.iz + q);
            tree_rec(t, ch);
        }
    }
}

int64_t orc_build_tree(const orc_net *net, const orc_opts *o, const double *xl,
                       const double *xu, int max_level, int split,
                       orc_node *out, int64_t cap, int64_t *counts) {
    tree_ctx t;
    memset(&t, 0, sizeof(t));
    t.net = net; t.o = o; t.xl = xl; t.xu = xu;
    t.max_level = max_level; t.split = split;
    t.out = out; t.cap = cap;
    orc_node root = {0, 0, 0, 0, 0};
    tree_rec(&t, root);
    if (counts)
        for (int k = 0; k < 4; ++k) counts[k] = t.counts[k];
    return t.n;
}

int64_t orc_build_tree_conv(const orc_net *net, const orc_opts *o, const double *xl,
                            const double *xu, int max_level, int split, double delta,
                            orc_node *out, int64_t cap, int64_t *counts) {
    tree_ctx t;
    memset(&t, 0, sizeof(t));
    t.net = net; t.o = o; t.xl = xl; t.xu = xu;
    t.max_level = max_level; t.split = split;
    t.out = out; t.cap = cap;
    t.delta = delta;
    orc_node root = {0, 0, 0, 0, 0};
    tree_rec(&t, root);
    if (counts)
        for (int k = 0; k < 5; ++k) counts[k] = t.counts[k];
    return t.n;
}

void orc_classify_nodes(const orc_net *net, const orc_opts *o, const double *xl,
                        const double *xu, int split, int64_t n,
                        const orc_node *nodes, int32_t *cls, double *lo,
                        double *hi, double *sel_gap, int nthreads) {
    if (nthreads <= 0) nthreads = orc_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (int64_t i = 0; i < n; ++i) {
        double bl[3], bh[3], c[3], axes[9] = {0};
        node_box(xl, xu, split, &nodes[i], bl, bh);
        for (int d = 0; d < 3; ++d) {
            c[d] = 0.5 * (bl[d] + bh[d]);
            axes[d * 3 + d] = bh[d] - c[d];
        }
        double l, h, y0, r;
        t_sel_gap = INFINITY;
        int k = orc_range_bound(net, o, c, axes, 3, &l, &h, &y0, &r);
        if (sel_gap) sel_gap[i] = t_sel_gap;
        if (cls) cls[i] = k;
        if (lo) lo[i] = l;
        if (hi) hi[i] = h;
    }
}

/* ---------------------------------------------------------------- CastRay */

int orc_cast_ray(const orc_net *net, const orc_opts *o, const orc_ray_opts *ro,
                 const double *p, const double *r, double *t_out,
                 int64_t *iters_out, double *margin_out) {
    double sigma = ro->sigma0, t = 0.0;
    double f0 = orc_eval(net, p);
    double margin = fabs(f0);
    int64_t it = 0;
    int status = 0;
    *t_out = INFINITY;
    while (t < ro->t_max) {
        if (it >= ro->max_iters) { status = 2; break; }
        ++it;
        /* convergence test at t + delta */
        double pc[3];
        for (int d = 0; d < 3; ++d) pc[d] = p[d] + (t + ro->delta) * r[d];
        double fc = orc_eval(net, pc);
        if (fabs(fc) < margin) margin = fabs(fc);
        if ((f0 >= 0.0) != (fc >= 0.0)) { /* DifferentSigns (R9) */
            *t_out = t;
            status = 1;
            break;
        }
        /* 1-d query box over [t, t + sigma] */
        double c[3], v[3];
        for (int d = 0; d < 3; ++d) {
            c[d] = p[d] + (t + sigma / 2.0) * r[d];
            v[d] = (sigma / 2.0) * r[d];
        }
        double lo, hi, y0, rad;
        int cls = orc_range_bound(net, o, c, v, 1, &lo, &hi, &y0, &rad);
        if (fabs(lo) < margin) margin = fabs(lo);
        if (fabs(hi) < margin) margin = fabs(hi);
        double sigma_star;
        if (cls != ORC_UNKNOWN) { sigma_star = sigma; sigma = sigma * ro->eta_plus; }
        else { sigma_star = 0.0; sigma = sigma * ro->eta_minus; }
        double step = ro->safety * sigma_star;
        t = t + (step > ro->delta ? step : ro->delta);
    }
    *iters_out = it;
    *margin_out = margin;
    return status;
}

void orc_cast_rays(const orc_net *net, const orc_opts *o, const orc_ray_opts *ro,
                   int64_t n, const double *p, const double *r, double *t,
                   int64_t *iters, int32_t *status, double *margin, int nthreads) {
    if (nthreads <= 0) nthreads = orc_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (int64_t i = 0; i < n; ++i) {
        double tt, mg;
        int64_t it;
        int st = orc_cast_ray(net, o, ro, p + 3 * i, r + 3 * i, &tt, &it, &mg);
        t[i] = tt;
        iters[i] = it;
        status[i] = st;
        margin[i] = mg;
    }
}
