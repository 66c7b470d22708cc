/* FP64 oracle for range analysis of MLP implicit functions
 * (Sharp & Jacobson, "Spelunking the Deep", SIGGRAPH 2022).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark use this library. It shares no code, header
 * or constant with the CUDA path; the product library never links it.
 *
 * Everything here is plain double-precision C: slow, direct, and written to be
 * checked against the paper by eye. Parallelism is over independent boxes or
 * rays only (OpenMP); the arithmetic of each query is sequential.
 */
#ifndef SRA_ORACLE_H
#define SRA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_ACT_IDENTITY = 0, ORC_ACT_RELU = 1, ORC_ACT_ELU = 2, ORC_ACT_SIN = 3 };
enum { ORC_INTERVAL = 0, ORC_AFFINE_FIXED = 1, ORC_AFFINE_TRUNCATE = 2, ORC_AFFINE_FULL = 3 };
enum { ORC_SLOPE_CHEBYSHEV = 0, ORC_SLOPE_MINRANGE = 1 };
enum { ORC_UNKNOWN = 0, ORC_POSITIVE = 1, ORC_NEGATIVE = 2 };
enum { ORC_SPLIT_OCTREE = 0, ORC_SPLIT_KD = 1 };

/* A scalar MLP f: R^3 -> R. widths[0] is the first linear layer's input
 * width (3, or 3 + 6*pe_octaves), widths[n_layers] == 1. acts[l] follows
 * linear layer l for l < n_layers-1. params packs, per layer, the row-major
 * W_l (widths[l+1] x widths[l]) then b_l. */
typedef struct {
    int n_layers;
    const int *widths;
    const int *acts;
    const double *params;
    int pe_octaves;
} orc_net;

typedef struct {
    int arith; /* ORC_INTERVAL / ORC_AFFINE_* */
    int K;     /* kept noise symbols for affine-truncate */
    int slope; /* ORC_SLOPE_* (ReLU and ELU; sin always uses its own rule) */
} orc_opts;

typedef struct {
    uint16_t ix, iy, iz, level;
    int32_t cls;
} orc_node;

/* Linearisation rules of App. A (Table "affine_nonlinearities"), exposed for
 * unit tests: on input range [l,u] returns alpha, beta, gamma such that
 * |f(x) - alpha x - beta| <= gamma on [l,u]. act is ORC_ACT_*. */
void orc_linearize(int act, int slope, double l, double u,
                   double *alpha, double *beta, double *gamma);
/* Interval image of [l,u] under the activation (Sec. 3.1). */
void orc_interval_act(int act, double l, double u, double *lo, double *hi);

/* Plain forward evaluation f(x). */
double orc_eval(const orc_net *net, const double *x);
void orc_eval_batch(const orc_net *net, int64_t n, const double *x, double *out, int nthreads);

/* Proc. 1 (RangeBound) on a box with center c (3) and s axis vectors
 * axes[s][3]: writes the output range [lo,hi], its center y0 and radius rad
 * (for interval arithmetic y0 = (lo+hi)/2, rad = (hi-lo)/2). Returns the
 * class ORC_POSITIVE / ORC_NEGATIVE / ORC_UNKNOWN. */
int orc_range_bound(const orc_net *net, const orc_opts *o, const double *c,
                    const double *axes, int s, double *lo, double *hi,
                    double *y0, double *rad);

/* Batch of axis-aligned boxes (center, half-width per axis). sel_gap (may be
 * NULL) receives, per box, the smallest relative gap between the last kept
 * and the first dropped affine-truncate column score (+inf if none). */
void orc_bound_boxes(const orc_net *net, const orc_opts *o, int64_t n,
                     const double *centers, const double *halfw, double *lo,
                     double *hi, double *y0, double *rad, int32_t *cls,
                     double *sel_gap, int nthreads);

/* Proc. 3 (BuildSpatialTree) stopped at a fixed depth, over the root box
 * [xl,xu]. split = ORC_SPLIT_OCTREE classifies cubes and splits all three
 * axes at once (level = octree level); ORC_SPLIT_KD splits the widest
 * dimension as in Proc. 3 (level = k-d level). Writes every returned node
 * (decided nodes and UNKNOWN nodes at max_level) in depth-first order; returns
 * the node count (may exceed cap, in which case only cap were written).
 * counts[0..2] receive the number of POSITIVE, NEGATIVE and UNKNOWN nodes
 * returned; counts[3] the number of RangeBound calls. */
int64_t orc_build_tree(const orc_net *net, const orc_opts *o, const double *xl,
                       const double *xu, int max_level, int split,
                       orc_node *out, int64_t cap, int64_t *counts);

/* orc_build_tree with the convergence test of Proc. 3 as well: an UNKNOWN
 * node narrower than delta / sqrt(3) (widest side) whose six face centres
 * take both signs (some f < 0 and some f > 0) is returned as an UNKNOWN
 * leaf; other nodes continue to max_level. counts[4] receives the number of
 * nodes returned by that test. */
int64_t orc_build_tree_conv(const orc_net *net, const orc_opts *o, const double *xl,
                            const double *xu, int max_level, int split, double delta,
                            orc_node *out, int64_t cap, int64_t *counts);

/* RangeBound for a list of tree nodes (the per-node step of Proc. 3). */
void orc_classify_nodes(const orc_net *net, const orc_opts *o, const double *xl,
                        const double *xu, int split, int64_t n,
                        const orc_node *nodes, int32_t *cls, double *lo,
                        double *hi, double *sel_gap, int nthreads);

typedef struct {
    double delta, t_max, sigma0, eta_plus, eta_minus, safety;
    int64_t max_iters;
} orc_ray_opts;

/* Proc. 2 (CastRay). Returns 1 on hit (t_out = t), 0 on miss (t_out = +inf),
 * 2 when max_iters was reached first. iters_out counts loop iterations;
 * margin_out is the smallest |f_c|, |lo| or |hi| met along the way. */
int orc_cast_ray(const orc_net *net, const orc_opts *o, const orc_ray_opts *ro,
                 const double *p, const double *r, double *t_out,
                 int64_t *iters_out, double *margin_out);
void orc_cast_rays(const orc_net *net, const orc_opts *o, const orc_ray_opts *ro,
                   int64_t n, const double *p, const double *r, double *t,
                   int64_t *iters, int32_t *status, double *margin, int nthreads);

int orc_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
