/* sra.h — sound range analysis of MLP implicit functions on GB300 (sm_103a).
 *
 * C ABI of the library libsra.so. It bounds a scalar MLP f: R^3 -> R over
 * many boxes and ray segments with affine (or interval) arithmetic and uses
 * the bounds to classify octree nodes and to cast rays. Method: Sharp &
 * Jacobson, "Spelunking the Deep: Guaranteed Queries on General Neural
 * Implicit Surfaces via Range Analysis", SIGGRAPH 2022 (arXiv 2202.02444).
 *
 * Conventions for every entry point:
 *   - Array arguments marked "device" are caller-owned device pointers
 *     (e.g. torch tensors' data_ptr()); "host" marks host pointers. The
 *     library owns only the network copy made by sra_load_mlp and transient
 *     scratch it allocates stream-ordered (cudaMallocAsync) on the call's
 *     stream.
 *   - Calls enqueue work on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and return without synchronising unless stated. Launch and
 *     argument errors are returned at once; nothing aborts the process.
 *   - On an error the function returns a non-zero sra_status and
 *     sra_last_error() describes it (thread-local string).
 *   - Calls on distinct streams may run concurrently on one network.
 */
#ifndef SRA_H
#define SRA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sra_net sra_net; /* opaque; owns device copies of the weights */

typedef enum {
    SRA_OK = 0,
    SRA_EINVAL = 1,        /* bad argument (null pointer, size, option) */
    SRA_ENOMEM = 2,        /* device or host allocation failed */
    SRA_ECUDA = 3,         /* a CUDA call failed; see sra_last_error() */
    SRA_ETIMEOUT = 4,      /* a bounded device wait ran out */
    SRA_ECAPACITY = 5,     /* an output buffer was too small; needed size reported */
    SRA_EUNSUPPORTED = 6   /* network shape / option not supported by a kernel */
} sra_status;

/* uint8 box classes (Proc. 1 "RangeBound"). */
enum { SRA_UNKNOWN = 0, SRA_POSITIVE = 1, SRA_NEGATIVE = 2 };

/* Activations (App. A Table "affine_nonlinearities"). */
enum { SRA_ACT_IDENTITY = 0, SRA_ACT_RELU = 1, SRA_ACT_ELU = 2, SRA_ACT_SIN = 3 };

/* Range arithmetic (Sec. 3.1 interval; Sec. 3.3 affine condensation policies). */
enum {
    SRA_ARITH_INTERVAL = 0,
    SRA_ARITH_AFFINE_FIXED = 1,    /* keep only the input-domain symbols */
    SRA_ARITH_AFFINE_TRUNCATE = 2, /* keep the K largest symbols (column L1 norm) */
    SRA_ARITH_AFFINE_FULL = 3      /* keep every symbol: up to 128 symbols on every kernel; past
                                      that, box bounds only (sra_bound_boxes, sra_classify_and_split
                                      and the entry points built on them): networks of width <= 64
                                      without positional encoding whose state fits in shared memory
                                      run one CTA per box (e.g. 8-layer 32-wide: 227 symbols); any
                                      other network keeps each box's noise matrix in device memory
                                      (stream-ordered scratch of up to 1 GiB per call, 2 * width *
                                      (symbols + 1) floats per box; 3-[256]x8-1: 2051 symbols,
                                      4.2 MB per box in FP32), the boxes taken in passes that fit */
};

/* Slope of the activation linearisation: Chebyshev (App. A) or min-range. */
enum { SRA_SLOPE_CHEBYSHEV = 0, SRA_SLOPE_MINRANGE = 1 };

/* Arithmetic the bound is computed in.
 *   FP32:       plain single precision, no rounding control (the paper's form;
 *               Sec. 3.4 reports that none was needed in practice).
 *   FP64:       plain double precision.
 *   BF16_SOUND: the dense layers on BF16 tensor cores with FP32 accumulation
 *               (weights split into a BF16 hi/lo pair, centers as a BF16
 *               hi/lo pair), and an a-priori rounding radius of every FP
 *               operation folded into x_inf with outward rounding, so the
 *               range is guaranteed to contain f over the box. The radius
 *               sits in x_inf, which every later layer widens by the row sums
 *               of |W|: on deep wide networks the bound is much wider than the
 *               exact-arithmetic affine bound.
 *   BF16:       the same tensor-core computation without the rounding radius
 *               (plain, like FP32; results differ from FP64 by BF16 operand
 *               rounding of the noise columns).
 * BF16_SOUND and BF16 serve networks with 3 inputs (no positional
 * encoding), 2 to 13 hidden layers of widths up to 512, all ReLU, all ELU or
 * all sin, and a scalar output, with affine-truncate K = 16, 32, 64 or
 * (H <= 256) 128 and the Chebyshev slope. The kernel runs at the width
 * H in {128, 256, 512} that holds every hidden layer; a narrower layer runs
 * on weights padded with zeros (the padded neurons stay exactly zero; their
 * sums count in the rounding radius, as if the network were H wide). Other
 * shapes and options return SRA_EUNSUPPORTED. */
enum { SRA_PREC_FP32 = 0, SRA_PREC_FP64 = 1, SRA_PREC_BF16_SOUND = 2, SRA_PREC_BF16 = 3 };

/* Tree refinement: 8-way octree (one level = 3 k-d levels on a cube) or the
 * widest-axis binary split of Proc. 3 ("BuildSpatialTree"). */
enum { SRA_SPLIT_OCTREE = 0, SRA_SPLIT_KD = 1 };

/* Network description (host memory, read during sra_load_mlp only).
 * widths[0] is the first linear layer's input width: 3, or 3 + 6*pe_octaves
 * when the input x in R^3 is encoded as [x, then per octave k:
 * sin(2^k pi x_0..2), cos(2^k pi x_0..2)]. widths[n_layers] must be 1.
 * acts[l] (l < n_layers-1) follows linear layer l; the last layer is linear.
 * params packs, for each layer l, the row-major W_l (widths[l+1] x widths[l])
 * followed by b_l (widths[l+1]), as float32. */
typedef struct {
    int32_t n_layers;
    const int32_t *widths;
    const int32_t *acts;
    const float *params;
    int32_t pe_octaves;
} sra_mlp_desc;

/* Query options; sra_default_opts() fills the paper's defaults. */
typedef struct {
    int32_t arith;       /* SRA_ARITH_* */
    int32_t K;           /* kept noise symbols for affine-truncate (excl. x_inf) */
    int32_t slope;       /* SRA_SLOPE_* */
    int32_t precision;   /* SRA_PREC_* */
    int32_t recheck;     /* 1: re-bound in FP64 every box whose lo or hi lies
                            within the band of zero, and keep the FP64 result;
                            sra_cast_rays: march again in FP64 every ray with a
                            step whose segment bound has an end within the
                            band of zero */
    float recheck_band;  /* band half-width relative to |center| + radius */
    int32_t split;       /* SRA_SPLIT_* */
    float delta;         /* convergence tolerance (Sec. 4.1), > 0 */
    float t_max;         /* ray miss distance (Sec. 4.2) */
    float sigma0;        /* initial ray step (Sec. 4.2: t_max / 10) */
    float eta_plus;      /* step growth on success (1.5) */
    float eta_minus;     /* step shrink on failure (0.5) */
    float safety;        /* step fraction taken (App. B: 0.98) */
    int64_t max_iters;   /* per-ray iteration cap; the ray then reports NaN */
    int32_t block_threads; /* SIMT bound kernels: threads per CTA (boxes per CTA
                              = block_threads / padded width); 0 = 256. A
                              multiple of 32 in [32, 1024], capped by what the
                              noise-column count allows (the tile shape the
                              autotuner chooses) */
    int32_t converge;    /* sra_classify_and_split / sra_extract_leaves: 1 = also the
                            convergence test of Proc. 3: an UNKNOWN node narrower than
                            delta / sqrt(3) whose six face centres take both signs is
                            returned as a leaf (counts[SRA_CNT_CONVERGED]); 0 = fixed
                            depth only */
    int64_t *recheck_count; /* optional device int64 (NULL: not counted):
                            sra_bound_boxes and sra_cast_rays add the number of
                            boxes / rays their FP64 re-check took again */
} sra_opts;

/* Octree / k-d node: integer cell coordinates at `level` inside the root box
 * given with each call. Octree: 2^level cells per axis. k-d: the per-axis
 * number of halvings follows the widest-axis rule of Proc. 3 from the root
 * extents (lowest axis on ties). */
typedef struct {
    uint16_t ix, iy, iz, level;
} sra_node;

/* Indices into the int64 counts array of sra_classify_and_split. */
enum {
    SRA_CNT_CHILDREN = 0, /* children appended to frontier_out (total, may exceed cap) */
    SRA_CNT_LEAVES = 1,   /* UNKNOWN leaves at max_level appended (may exceed cap) */
    SRA_CNT_POSITIVE = 2, /* nodes classified POSITIVE */
    SRA_CNT_NEGATIVE = 3, /* nodes classified NEGATIVE */
    SRA_CNT_UNKNOWN = 4,  /* nodes classified UNKNOWN */
    SRA_CNT_RECHECKED = 5,/* nodes re-bounded in FP64 */
    SRA_CNT_CONVERGED = 6,/* UNKNOWN nodes returned by the convergence test (opts->converge) */
    SRA_CNT_N = 8
};

/* Fill *o with the defaults: affine-fixed, Chebyshev, FP32, no re-check,
 * band 1e-5, octree, delta 1e-3, t_max 10, sigma0 1, eta 1.5 / 0.5,
 * safety 0.98, max_iters 1<<20 (Sec. 4.1, Sec. 4.2, App. B). */
void sra_default_opts(sra_opts *o);

/* Copy a network to the current device (App. A: the MLP f whose affine
 * propagation all queries use). Host `desc` may be freed after the call.
 * Errors: SRA_EINVAL (shape), SRA_EUNSUPPORTED (more than 24 layers or a
 * width above 512), SRA_ENOMEM, SRA_ECUDA. Synchronous. */
sra_status sra_load_mlp(const sra_mlp_desc *desc, sra_net **out);

/* Free a network (synchronises the device first). NULL is accepted. */
sra_status sra_free_mlp(sra_net *net);

/* Proc. 1 (RangeBound) on n axis-aligned boxes: box i is
 * centers[i] +- halfw[i] (device float[n][3] each). Writes the output range
 * lo[i], hi[i] (device float[n]) and the class cls[i] (device uint8[n]):
 * POSITIVE iff lo > 0, NEGATIVE iff hi < 0, else UNKNOWN. lo/hi may be NULL.
 * With opts->recheck the boxes whose lo or hi lies within the band of zero
 * are re-bounded in FP64 on the GPU and their lo/hi/cls replaced;
 * opts->recheck_count, if given, counts them.
 * n == 0 is a no-op.
 * Errors: SRA_EINVAL, SRA_EUNSUPPORTED (K / width beyond the kernels' limits),
 * SRA_ECUDA. Asynchronous on `stream`. */
sra_status sra_bound_boxes(const sra_net *net, const sra_opts *opts, const float *centers,
                           const float *halfw, int64_t n, float *lo, float *hi,
                           uint8_t *cls, void *stream);

/* One batched round of Proc. 3 (Sec. 4.5 builds the tree level by level in batches)
 * at a fixed depth (Sec. 4.7). For each node of frontier_in (device
 * sra_node[n_in]) inside the root box [root_lo, root_hi] (host float[3]):
 * bound it; if UNKNOWN and level < max_level append its children (8 for the
 * octree, 2 for k-d) to frontier_out; if UNKNOWN and level == max_level
 * append it to leaves_out. Output positions start at the values already in
 * counts[SRA_CNT_CHILDREN] / counts[SRA_CNT_LEAVES] (device int64[8]; zero
 * it before the first call of a level, so chunked calls append) and follow
 * the input order (deterministic). Records beyond cap_out / cap_leaves are
 * not written but still counted, so a caller detects overflow after the
 * stream syncs by counts[...] > cap. counts[2..5] accumulate per-class and
 * re-check tallies. Uses stream-ordered scratch of about n_in * 9 bytes.
 * Errors: SRA_EINVAL, SRA_EUNSUPPORTED, SRA_ENOMEM, SRA_ECUDA. Asynchronous. */
sra_status sra_classify_and_split(const sra_net *net, const sra_opts *opts,
                                  const float *root_lo, const float *root_hi,
                                  const sra_node *frontier_in, int64_t n_in, int32_t max_level,
                                  sra_node *frontier_out, int64_t cap_out,
                                  sra_node *leaves_out, int64_t cap_leaves,
                                  int64_t *counts, void *stream);

/* One segment of a batched round (sra_classify_and_split_batch): the
 * frontier of one network. */
typedef struct {
    int32_t net;          /* index into nets[] and opts[] */
    int32_t max_level;    /* octree (k-d) depth of this network's tree */
    int64_t first, n;     /* its nodes: frontier_in[first, first + n) */
    int64_t out_first;    /* children go to frontier_out[out_first, out_first + cap_out) */
    int64_t cap_out;
    int64_t leaf_first;   /* UNKNOWN nodes at max_level go to leaves_out[leaf_first, + cap_leaves) */
    int64_t cap_leaves;
} sra_batch_seg;

/* One round of Proc. 3 over the frontiers of many networks at once: the
 * batched form of sra_classify_and_split for uneven workloads. Every
 * segment's results (classes, children, leaves, counters) equal those of a
 * lone sra_classify_and_split call on that segment (root box [root_lo,
 * root_hi] for all). The bounds of all segments whose option sets need the
 * same noise-column bound run in one persistent launch (a chunk queue that
 * hands each CTA groups of nodes of one network, heaviest networks first),
 * and one segmented compaction serves every segment. counts: device
 * int64[n_segs][SRA_CNT_N], zeroed by the caller (or holding earlier
 * chunks' totals, which are appended after). Precision FP32 (the SIMT
 * launches above) or, for networks with the tensor-core path (3 -> H x L -> 1
 * ReLU, ELU or sin, hidden widths up to 512, run at H = 128, 256 or 512) and affine-truncate K = 16, 32, 64 or (H <= 256) 128,
 * SRA_PREC_BF16 /
 * SRA_PREC_BF16_SOUND: each such segment runs one tensor-core launch beside
 * the SIMT launches (check sra_sync_status on its network for a timed-out
 * wait). recheck and converge must be 0; FP64 is not batched; otherwise
 * SRA_EUNSUPPORTED. Segments must not overlap in frontier_out or leaves_out.
 * Uses stream-ordered scratch of about 2 KB per segment plus one byte per
 * node. Asynchronous. The segment tables reach the device as kernel
 * parameters (no host memory is read after the call returns), so the round
 * can be captured into a CUDA graph and replayed with new nodes written into
 * the same buffers, for the same segments; counts must be zeroed inside the
 * graph if each replay should start from zero. The library's pool of
 * streams is created by the first batched call that runs more than one
 * launch: make one eager call with the same segments before a capture. */
sra_status sra_classify_and_split_batch(const sra_net *const *nets, const sra_opts *opts,
                                        int32_t n_nets, const float *root_lo, const float *root_hi,
                                        const sra_node *frontier_in, const sra_batch_seg *segs,
                                        int32_t n_segs, sra_node *frontier_out, sra_node *leaves_out,
                                        int64_t *counts, void *stream);

/* Proc. 2 (CastRay) for n rays p = origins[i], r = dirs[i] (device
 * float[n][3]; r need not be unit length; t is in units of r). Writes
 * t_hit[i] (device float[n]): the returned t on a hit, +inf for NO_HIT, NaN
 * when opts->max_iters ran out; and iters[i] (device int32[n], may be NULL):
 * loop iterations taken. One persistent launch refills finished ray slots.
 * opts->precision: SRA_PREC_FP32 (and SRA_PREC_FP64) runs every step on the
 * SIMT cores in FP32 (FP64), any arithmetic; SRA_PREC_BF16 runs every layer
 * but the output one on the tensor cores (tcgen05) with the weights and the
 * center, point and noise operands split into BF16 hi/lo pairs and FP32
 * accumulation (about 16 significant bits per product), and |W| x_inf from
 * |W| and x_inf rounded up to BF16 (an upper bound of that term); plain
 * arithmetic otherwise, no rounding radius. SRA_PREC_BF16_SOUND is the same
 * computation with every segment bound guaranteed: the rounding of the
 * segment box and of the encoding, the products' and FP32 sums' errors
 * (a-priori, from |W| (|c| + |A|) on the tensor cores) and the operands'
 * BF16 storage go to x_inf, the activation rules are the outward-rounded
 * ones (Chebyshev slope only), and the segment's range is rounded outward;
 * the point test f(t + delta) stays a plain evaluation. Both BF16 forms
 * need affine-fixed arithmetic and a network with hidden widths up to 512,
 * 1 to 8 hidden-to-hidden layers and an input width (after the encoding) of
 * at most 64 (the kernel runs at the width H in {128, 256, 512} that holds
 * every hidden layer, narrower layers on weights padded with zeros);
 * otherwise SRA_EUNSUPPORTED. A
 * bounded wait of that kernel that runs out is reported by sra_sync_status as
 * SRA_ETIMEOUT. With opts->recheck (FP32 or BF16) a ray that took a step
 * whose segment bound [y0 - rad, y0 + rad] has an end within
 * recheck_band (|y0| + rad) of zero is marched again from its start in FP64
 * (its origin's sign too) and its t_hit and iters are the FP64 ones;
 * opts->recheck_count, if given, counts those rays. n is at most 2^31 - 1.
 * Uses stream-ordered scratch of 4 bytes per ray (8 with recheck).
 * Errors: SRA_EINVAL (delta <= 0, bad steps, n > 2^31 - 1), SRA_EUNSUPPORTED,
 * SRA_ENOMEM (scratch), SRA_ECUDA. Asynchronous. */
sra_status sra_cast_rays(const sra_net *net, const sra_opts *opts, const float *origins,
                         const float *dirs, int64_t n, float *t_hit, int32_t *iters,
                         void *stream);

/* Frustum ray casting (Sec. 4.3) for a pinhole image: width x height pixel
 * rays from one eye (host float[3]) along unit directions dirs (device
 * float[height * width][3], row-major, the rays of a pinhole camera: each
 * pixel's direction a positive combination of its rectangle's corner
 * directions). A grid x grid set of coarse frusta marches like Proc. 2: each
 * frustum bounds its segment [t, t + sigma] by one box that contains every
 * pixel ray's points (the truncated pyramid of its corner rays, far face
 * pushed out by 1 / cos of the widest corner angle), advances on POSITIVE or
 * NEGATIVE, shrinks sigma on UNKNOWN, splits its longer pixel side when that
 * side is wider than 2 sigma at the far face, and hands single pixels to the
 * ray kernel of opts->precision, which resumes Proc. 2 from the frustum's
 * (t, sigma). Frustum boxes are bounded in FP32 (with opts->recheck, FP64
 * near zero). Writes t_hit (device float[height * width]: t, +inf for
 * NO_HIT, NaN at the iteration cap) and, if not NULL, iters (device
 * int32[height * width]: ray iterations after the hand-over). stats (host
 * int64[4], may be NULL): frustum rounds, frustum boxes bounded, pixels
 * handed to rays, 0. Synchronises once per round. Errors as sra_cast_rays;
 * SRA_EUNSUPPORTED on a stream that is being captured into a CUDA graph. */
sra_status sra_cast_frustum(const sra_net *net, const sra_opts *opts, const float *eye, const float *dirs,
                            int32_t width, int32_t height, int32_t grid, float *t_hit, int32_t *iters,
                            int64_t *stats, void *stream);

/* Proc. 3 to a fixed depth from the root box [xl, xu] (host float[3]): runs
 * sra_classify_and_split level by level and writes the UNKNOWN nodes at
 * `depth` to leaves_out (device sra_node[cap]) in level-order; these are the
 * cells that hierarchical mesh extraction (Sec. 4.7) visits. *n_leaves
 * (host) receives the leaf count. Per-level POSITIVE/NEGATIVE/UNKNOWN counts
 * are written to level_counts (host int64[(depth+1)*3], may be NULL).
 * Synchronises the stream once per level. Errors: SRA_ECAPACITY when the
 * leaves exceed cap (*n_leaves holds the needed count, the first cap are
 * written), SRA_EINVAL, SRA_EUNSUPPORTED (also on a stream that is being
 * captured into a CUDA graph), SRA_ENOMEM, SRA_ECUDA. */
sra_status sra_extract_leaves(const sra_net *net, const sra_opts *opts, const float *xl,
                              const float *xu, int32_t depth, sra_node *leaves_out,
                              int64_t cap, int64_t *n_leaves, int64_t *level_counts,
                              void *stream);

/* Mesh of the zero level set inside octree leaves: the dense bottom of
 * hierarchical mesh extraction (Sec. 4.7). Each leaf (device sra_node[n],
 * e.g. the UNKNOWN leaves of sra_extract_leaves) is split into 2^sub_levels
 * cells per axis (0 <= sub_levels <= 5); f is evaluated at the cell corners
 * (FP32 forward pass) and every cell is cut into the six tetrahedra around
 * its main diagonal, each meshed by marching tetrahedra (linear
 * interpolation of f along the crossing edges). Leaves of one level give a
 * closed, crack-free surface; a shared grid edge yields bit-identical
 * vertices from every cell around it. Triangles face the f >= 0 side.
 * tris_out (device float[cap][3][3]) is written in leaf, cell (x fastest),
 * tetrahedron order; *n_tris (host) receives the triangle count. Errors:
 * SRA_ECAPACITY when the count exceeds cap (the first cap are written),
 * SRA_EINVAL, SRA_ENOMEM, SRA_ECUDA, SRA_EUNSUPPORTED on a stream that is
 * being captured into a CUDA graph. Synchronises the stream once. */
sra_status sra_mesh_leaves(const sra_net *net, const float *root_lo, const float *root_hi,
                           const sra_node *leaves, int64_t n_leaves, int32_t sub_levels,
                           float *tris_out, int64_t cap, int64_t *n_tris, void *stream);

/* Empty-sphere queries (Sec. 4.4). For every point p (device float[n][3])
 * writes radius_out[i] (device float[n]): the largest r = r_max * 2^-k,
 * 0 <= k < levels, whose box [p - r, p + r] range analysis classifies
 * POSITIVE or NEGATIVE (Proc. 1 with opts), else 0. The box of half-width r
 * contains the ball of radius r, so that ball does not meet f = 0. Runs
 * `levels` rounds over the points still open (no host synchronisation).
 * Precision FP32 or FP64; opts->recheck re-bounds near-zero FP32 results in
 * FP64. Uses stream-ordered scratch of about 30 bytes per point. Errors:
 * SRA_EINVAL (r_max <= 0, levels outside [1, 30], n > 2^31 - 1),
 * SRA_EUNSUPPORTED (BF16 precisions), SRA_ENOMEM, SRA_ECUDA. Asynchronous. */
sra_status sra_empty_spheres(const sra_net *net, const sra_opts *opts, const float *points, int64_t n,
                             float r_max, int32_t levels, float *radius_out, void *stream);

/* Plain forward evaluation f(x) for n points (device float[n][3] -> device
 * float[n]) in the network's FP32 weights. Asynchronous. */
sra_status sra_eval(const sra_net *net, const float *x, int64_t n, float *out, void *stream);

/* Allocation-free variant of sra_classify_and_split (same arguments, same
 * results for the options it accepts). The paper has no counterpart: it
 * exists for callers that cannot allocate device memory at all, such as
 * real-time loops that forbid allocator calls and their implicit
 * synchronisation on the hot path, or hosts that give this library a
 * pre-partitioned device without an allocator. The round's scratch lives in
 * a fixed file-scope device array of SRA_NOALLOC_SCRATCH_BYTES that every GPU
 * loading the library holds until the process exits; the call itself
 * allocates nothing.
 * Limits: n_in <= SRA_NOALLOC_MAX_NODES, else SRA_EINVAL (nothing queued).
 * Unsupported options, each SRA_EUNSUPPORTED (nothing queued): precision
 * SRA_PREC_BF16_SOUND or SRA_PREC_BF16 (FP32 and FP64 only),
 * opts->converge (the convergence test of Proc. 3), and affine-full on a
 * network whose noise matrix does not fit shared memory (positional
 * encoding, or widths past 64: that form keeps its state in device memory).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for the rest of the process. The
 * address is not looked up again,
 * so after cudaDeviceReset (or any teardown of the device's primary context)
 * this entry point must not be used in the same process. All calls share
 * the array, which keeps the previous call's contents (each call clears what
 * must start at zero): calls whose device work overlaps (other streams or
 * host threads) race on it, so serialise them. Asynchronous on `stream`. */
#define SRA_NOALLOC_MAX_NODES 524288
#define SRA_NOALLOC_SCRATCH_BYTES (5u << 20)
sra_status sra_classify_and_split_noalloc(const sra_net *net, const sra_opts *opts,
                                          const float *root_lo, const float *root_hi,
                                          const sra_node *frontier_in, int64_t n_in,
                                          int32_t max_level, sra_node *frontier_out,
                                          int64_t cap_out, sra_node *leaves_out,
                                          int64_t cap_leaves, int64_t *counts, void *stream);

/* Diagnostics: self-test of the tensor-core building blocks used by
 * SRA_PREC_BF16_SOUND (TMA-loaded 128-byte-swizzled K-major weight tiles,
 * thread-written operand tiles, tcgen05.mma into TMEM, tcgen05.ld). Computes
 * D[256][144] = W[256][256] * X[144][256]^T with W, X device bf16 row-major
 * and D device float; *status (device int, zero it first) becomes non-zero if
 * a bounded wait ran out. Asynchronous; one CTA. */
sra_status sra_selftest_tc_gemm(const void *W, const void *X, float *D, int *status, void *stream);

/* Synchronise `stream` and report kernel-side failures recorded for this
 * network since the last call: SRA_ETIMEOUT if a bounded device wait of the
 * tensor-core path ran out (the kernel then left without finishing its boxes;
 * their outputs are undefined). The record is cleared. */
sra_status sra_sync_status(const sra_net *net, void *stream);

/* ---- Serving: continuous batching over resident networks ----------------
 * Not a procedure of the paper: a request loop around Proc. 1-3 for many
 * concurrent queries. sra_serve runs a whole request trace. Requests become
 * eligible at their arrival time; the loop admits them first come, first
 * served, each into a free slot (one CUDA stream per slot) when the device
 * memory it reserves fits in the frontier budget, and drives every admitted
 * request on its slot's stream while others run, so the work of several
 * requests overlaps on the device. A leaf job (Proc. 3) is stepped one chunk
 * of one level's frontier at a time; between its chunks the loop serves
 * other slots. It walks the tree depth-first over chunks: the next chunk is
 * always the front of the deepest level that still has unprocessed nodes,
 * at most cap / 8 nodes (cap / 2 for the k-d split), so every level's
 * frontier fits a buffer of cap nodes however large the tree grows.
 *
 * Memory: the loop allocates one device arena of cfg->frontier_bytes and
 * one stream per slot when it starts and frees them before it returns. A
 * leaf job takes one frontier buffer per level 0..depth
 * ((depth + 1) * cap * sizeof(sra_node), each rounded up to 256 bytes) and
 * its counters from the arena, fixed for the job's lifetime; ray and box
 * requests reserve their stream-ordered scratch size (16 bytes per ray /
 * box) from the same budget. A request whose reservation exceeds the whole
 * budget ends at once with SRA_ENOMEM.
 *
 * Results are the same as a lone call of the entry point each kind uses
 * (sra_cast_rays, sra_bound_boxes, sra_extract_leaves): a leaf job's leaves
 * come out in the order of a level-by-level build, because chunks are taken
 * from the front of their level. (With opts->converge the converged leaves
 * of shallower levels are the same set, but they interleave with deeper
 * leaves in the order the chunks ran.)
 */
enum { SRA_REQ_RAYS = 0, SRA_REQ_BOXES = 1, SRA_REQ_LEAVES = 2 };

typedef struct {
    int32_t kind;          /* SRA_REQ_* */
    int32_t net;           /* index into nets[] */
    int32_t form;          /* index into forms[] (the sra_opts of this request) */
    int32_t depth;         /* LEAVES: octree depth (root box [-1,1]^3 is level 0) */
    double arrival;        /* seconds after the trace starts; non-decreasing */
    int64_t n;             /* RAYS: rays; BOXES: boxes */
    const float *a, *b;    /* RAYS: origins, dirs; BOXES: centers, half-widths
                              (device float[n][3]) */
    float *lo, *hi;        /* RAYS: lo = t_hit (device float[n]), hi unused;
                              BOXES: range bounds (device float[n]) */
    int32_t *iters;        /* RAYS: iterations per ray (device int32[n]; may be NULL) */
    uint8_t *cls;          /* BOXES: classes (device uint8[n]; may be NULL) */
    sra_node *leaves;      /* LEAVES: UNKNOWN nodes at `depth` (device sra_node[cap]) */
    int64_t cap;           /* LEAVES: capacity of leaves and of each level's frontier
                              buffer (the chunk size is cap / 8, octree) */
    /* written by sra_serve */
    int64_t n_out;         /* LEAVES: leaves found. On SRA_ECAPACITY: the leaves found
                              when the job stopped (more than cap; the tree may hold
                              more), or, if cap is below the fan-out, the children of
                              one node */
    int32_t status;        /* sra_status of this request */
    int32_t slot;          /* slot that ran it (-1: never admitted) */
    int32_t levels;        /* LEAVES: levels reached (deepest level with nodes + 1) */
    int32_t pad;
    double t_admit, t_done;/* seconds after the trace starts */
} sra_request;

typedef struct {
    int32_t slots;          /* concurrent requests, 1..64 */
    int32_t realtime;       /* 1: a request is eligible at its arrival time;
                               0: every request is eligible at once */
    int64_t frontier_bytes; /* device memory budget of admitted requests */
} sra_serve_cfg;

/* Runs the trace reqs[0..n_req) against nets[0..n_nets) (all loaded on the
 * current device) with the option sets forms[0..n_forms). Returns SRA_OK
 * when every request has ended (each request's own outcome is in its
 * `status`); SRA_EINVAL for bad arguments (a net or form index out of range,
 * arrivals out of order); SRA_ENOMEM / SRA_ECUDA if the arena, a stream or a
 * CUDA call of the loop itself fails. Synchronous: returns after all device
 * work of the trace has finished. */
sra_status sra_serve(const sra_net *const *nets, int32_t n_nets, const sra_opts *forms,
                     int32_t n_forms, const sra_serve_cfg *cfg, sra_request *reqs, int64_t n_req);

/* Description of the last error on this thread ("" if none). */
const char *sra_last_error(void);

/* Fault injection for tests (the paper has no counterpart): the next n
 * device allocations made by the entry points (stream-ordered scratch and
 * network buffers) fail as if the device were out of memory, so the calls
 * that need them return SRA_ENOMEM after releasing what they had taken.
 * Host-side only: no GPU work is involved. n = 0 cancels the injection.
 * Errors: SRA_EINVAL for n < 0. */
sra_status sra_test_fail_allocs(int32_t n);

/* Failure detection test (the paper has no counterpart): while spins > 0,
 * every launch of the tensor-core bound kernel (SRA_PREC_BF16_SOUND /
 * SRA_PREC_BF16 box bounds) runs with its weight copies switched off and a
 * budget of `spins` iterations for each bounded mbarrier wait. Every wait on
 * a weight stage then runs out with no copy and no MMA in flight; the kernel
 * records the timeout, frees its TMEM and leaves without writing its boxes'
 * results, and sra_sync_status reports SRA_ETIMEOUT. spins = 0 restores
 * normal operation (the default). Host-side setting; no GPU fault involved.
 * Errors: SRA_EINVAL for spins outside [0, 2^20]. */
sra_status sra_test_tc_stall(int32_t spins);

/* Diagnostics (the paper has no counterpart): y[i] = f(x[i]) on the device
 * for the FP32 math functions whose errors the sound activation rules pad:
 * fn 0 sinf, 1 cosf, 2 sinpif, 3 acosf, 4 expm1f, 5 expf, 6 logf. x, y:
 * device float[n]. Asynchronous on `stream`. Errors: SRA_EINVAL (unknown fn,
 * n < 0, null pointers with n > 0), SRA_ECUDA. */
#define SRA_MATH_N 7
sra_status sra_test_math_f32(int32_t fn, const float *x, int64_t n, float *y, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SRA_H */
