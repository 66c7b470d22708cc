// C-ABI layer of libsra.so: argument validation, kernel-variant choice,
// shared-memory layout, stream-ordered scratch and the level loop of the
// fixed-depth tree build (Proc. 3). Every step of the path runs in the
// kernels of this library.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "launch.h"
#include "tc_bound.h"
#include "tc_host.h"
#include "tc_rays.h"

using namespace sra;

struct sra_net {
    NetDev dev;
    int L = 0, pe = 0, din = 0;
    std::vector<int> widths, acts;
    int rows = 0;      // max width (state matrix rows)
    int H = 0;         // threads per box
    int new_syms = 0;  // symbols created by all nonlinearities (affine-full sizing)
    void *buf = nullptr;
    int device = 0;
    // BF16-sound tensor-core path (3 -> H x (L-1) -> 1 ReLU nets, H = 128/256)
    bool tc_ok = false;
    int tc_H = 0;
    void *tc_buf = nullptr;  // bf16 hi/lo weights of the hidden layers, status word
    TcParams tcp;
    // tensor-core ray kernel (din -> H x (L-1) -> 1 nets, H = 128/256/512)
    bool tcr_ok = false;
    int tcr_H = 0;
    void *tcr_buf = nullptr;  // W_b, W_r, |W_b|, sign(W_b) W_r per hidden layer, status word
    TcRayParams tcrp;
};

namespace {

thread_local std::string g_err;

sra_status fail(sra_status s, const char *fmt, ...) {
    char b[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b, sizeof b, fmt, ap);
    va_end(ap);
    g_err = b;
    return s;
}

#define SRA_CK(call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return fail(SRA_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

constexpr int kMaxSmem = 232448;  // 227 KB opt-in per CTA on sm_100-class GPUs

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Smallest instantiated KMAX >= need, or 0.
int pick_kmax(int need) {
    for (int k : kKmaxList)
        if (k >= need) return k;
    return 0;
}

sra_status kmax_for(const sra_net *n, const sra_opts *o, int s, int *kmax) {
    int need = 1;
    switch (o->arith) {
    case SRA_ARITH_INTERVAL: need = 1; break;
    case SRA_ARITH_AFFINE_FIXED: need = s; break;
    case SRA_ARITH_AFFINE_TRUNCATE:
        if (o->K < 1) return fail(SRA_EINVAL, "affine-truncate needs K >= 1 (got %d)", o->K);
        need = o->K > s ? o->K : s;
        break;
    case SRA_ARITH_AFFINE_FULL: need = s + n->new_syms; break;
    default: return fail(SRA_EINVAL, "unknown arith %d", o->arith);
    }
    *kmax = pick_kmax(need);
    if (!*kmax) return fail(SRA_EUNSUPPORTED, "needs %d noise columns; the kernels hold at most 128", need);
    return SRA_OK;
}

// Per-box shared-memory layout and boxes per CTA.
sra_status make_cfg(const sra_net *n, const sra_opts *o, int kmax, int tsize, int target_threads,
                    RangeCfg *cfg) {
    memset(cfg, 0, sizeof *cfg);
    cfg->arith = o->arith;
    cfg->K = o->K;
    cfg->slope = o->slope;
    cfg->H = n->H;
    cfg->rows = n->rows;
    const int RS = engine_row_stride(kmax);
    size_t off = 0;
    cfg->x_off = (int)off;
    off = align16(off + (size_t)n->rows * RS * tsize);
    cfg->score_off = (int)off;
    off = align16(off + (size_t)(kmax + n->rows) * tsize);
    cfg->part_off = (int)off;
    off = align16(off + (size_t)(n->H / 32) * (kmax + 4) * tsize);
    cfg->outv_off = (int)off;
    off = align16(off + (size_t)(kmax + 4) * tsize);
    cfg->keep_off = (int)off;
    off = align16(off + (size_t)(kmax + n->rows));
    cfg->src_off = (int)off;
    off = align16(off + (size_t)kmax * 2);
    cfg->ray_off = (int)off;
    off = align16(off + (tsize == 8 ? sizeof(RaySlotState<double>) : sizeof(RaySlotState<float>)));
    cfg->slot_bytes = (int)off;
    const int maxT = engine_max_threads(tsize, kmax);
    if (n->H > maxT)
        return fail(SRA_EUNSUPPORTED, "width %d needs %d threads per box; this K allows %d", n->rows,
                    n->H, maxT);
    if (cfg->slot_bytes > kMaxSmem)
        return fail(SRA_EUNSUPPORTED, "per-box state of %d bytes exceeds shared memory", cfg->slot_bytes);
    int NB = target_threads / n->H;
    if (NB < 1) NB = 1;
    while (NB > 1 && (NB * n->H > maxT || NB * cfg->slot_bytes > kMaxSmem)) --NB;
    cfg->NB = NB;
    return SRA_OK;
}

sra_status check_opts(const sra_opts *o) {
    if (!o) return fail(SRA_EINVAL, "opts is NULL");
    if (o->slope != SRA_SLOPE_CHEBYSHEV && o->slope != SRA_SLOPE_MINRANGE)
        return fail(SRA_EINVAL, "unknown slope %d", o->slope);
    if (o->precision < SRA_PREC_FP32 || o->precision > SRA_PREC_BF16)
        return fail(SRA_EINVAL, "unknown precision %d", o->precision);
    if (o->split != SRA_SPLIT_OCTREE && o->split != SRA_SPLIT_KD)
        return fail(SRA_EINVAL, "unknown split %d", o->split);
    if (o->converge != 0 && (o->converge != 1 || !(o->delta > 0.f)))
        return fail(SRA_EINVAL, "converge must be 0 or 1, and needs delta > 0");
    if (o->block_threads != 0 && (o->block_threads < 32 || o->block_threads > 1024 || o->block_threads % 32))
        return fail(SRA_EINVAL, "block_threads %d: 0 or a multiple of 32 in [32, 1024]", o->block_threads);
    if (!(o->recheck_band >= 0.f)) return fail(SRA_EINVAL, "recheck_band must be >= 0");
    return SRA_OK;
}

cudaStream_t as_stream(void *s) { return (cudaStream_t)s; }

// Host tables to device memory through kernel parameters: one launch of
// upload_kernel carries up to kUploadChunk bytes by value, so the copy reads
// no host memory after the launch is enqueued, and a CUDA graph that captures
// it holds the bytes itself. (A captured cudaMemcpyAsync from host memory
// reads that memory again at every replay, after the call has released it.)
constexpr int kUploadChunk = 4000;  // with the other two parameters, under 4 KB of parameters
struct UploadChunk {
    unsigned char b[kUploadChunk];
};
__global__ void upload_kernel(const __grid_constant__ UploadChunk c, unsigned char *dst, int n) {
    for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = c.b[k];
}
cudaError_t upload(void *dst, const void *src, size_t bytes, cudaStream_t st) {
    UploadChunk c = {};
    for (size_t off = 0; off < bytes; off += kUploadChunk) {
        const int n = (int)(bytes - off < (size_t)kUploadChunk ? bytes - off : (size_t)kUploadChunk);
        memcpy(c.b, (const unsigned char *)src + off, (size_t)n);
        upload_kernel<<<1, 256, 0, st>>>(c, (unsigned char *)dst + off, n);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Entry points that read counts back to the host between their launches
// cannot be captured into a CUDA graph (a replay would not repeat the host
// decisions taken on them); they refuse a capturing stream instead of
// enqueueing work.
sra_status refuse_capture(void *stream, const char *what) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(as_stream(stream), &cs) != cudaSuccess) {
        cudaGetLastError();
        return SRA_OK;
    }
    if (cs != cudaStreamCaptureStatusNone)
        return fail(SRA_EUNSUPPORTED, "%s cannot be captured into a CUDA graph: it moves host data between its launches",
                    what);
    return SRA_OK;
}

int num_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// Keep freed stream-ordered scratch in the pool instead of returning it to
// the driver at every synchronisation.
void keep_pool_memory() {
    static bool done = false;
    if (done) return;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done = true;
}

struct Scratch {
    void *p = nullptr;
    cudaStream_t st = nullptr;
    ~Scratch() {
        if (p) cudaFreeAsync(p, st);
    }
};

// Regions of one scratch allocation, taken in order. A sizing pass (base
// null) adds up the bytes; the carving pass over the allocation hands out
// 16-byte-aligned regions and reports a region that would pass its end.
struct Carve {
    char *base = nullptr;
    size_t off = 0, cap = 0;
    bool overflow = false;
    template <typename T> T *take(size_t count) {
        const size_t b = align16(count * sizeof(T));
        T *q = base ? (T *)(base + off) : nullptr;
        off += b;
        if (base && off > cap) overflow = true;
        return q;
    }
};

// Bounded-wait budget of the tensor-core bound kernel for tests
// (sra_test_tc_stall): 0 = normal operation.
std::atomic<int> g_test_tc_stall{0};

// Allocation failures to inject (sra_test_fail_allocs): each device
// allocation of an entry point takes one and fails as out of memory.
std::atomic<int> g_fail_allocs{0};

bool take_injected_failure() {
    int v = g_fail_allocs.load();
    while (v > 0 && !g_fail_allocs.compare_exchange_weak(v, v - 1)) {
    }
    return v > 0;
}

sra_status scratch_alloc(Scratch &s, size_t bytes, cudaStream_t st) {
    keep_pool_memory();
    s.st = st;
    if (bytes == 0) bytes = 256;
    if (take_injected_failure()) {
        s.p = nullptr;
        return fail(SRA_ENOMEM, "cudaMallocAsync(%zu): injected allocation failure", bytes);
    }
    cudaError_t e = cudaMallocAsync(&s.p, bytes, st);
    if (e != cudaSuccess) {
        s.p = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? SRA_ENOMEM : SRA_ECUDA,
                    "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
    }
    return SRA_OK;
}

// k-d halvings per axis at each level and the axis split when leaving it
// (Proc. 3 widest-dimension rule, lowest axis on ties).
void kd_tables(const float *lo, const float *hi, unsigned char n3[][3], unsigned char *axis) {
    double e[3] = {(double)hi[0] - lo[0], (double)hi[1] - lo[1], (double)hi[2] - lo[2]};
    int c[3] = {0, 0, 0};
    for (int k = 0; k < kMaxKdLevels; ++k) {
        for (int d = 0; d < 3; ++d) n3[k][d] = (unsigned char)c[d];
        int a = 0;
        if (e[1] > e[a]) a = 1;
        if (e[2] > e[a]) a = 2;
        axis[k] = (unsigned char)a;
        e[a] *= 0.5;
        c[a]++;
    }
}

// Launch RangeBound over a box source in FP32 or FP64: the SIMT engine, or,
// for affine-full past its 128 register columns, the shared-memory full
// kernel (widths up to 64, no positional encoding, state within one CTA) or
// else the full kernels with each box's noise matrix in device memory.
sra_status run_bound(const sra_net *n, const sra_opts *o, bool fp64, int s, const BoxSrc &src,
                     const BoundOut &out, long long n_hint, cudaStream_t st) {
    if (o->arith == SRA_ARITH_AFFINE_FULL && s + n->new_syms > kKmaxList[sizeof kKmaxList / sizeof(int) - 1]) {
        if (s != 3) return fail(SRA_EUNSUPPORTED, "affine-full with %d symbols runs on box bounds only", s + n->new_syms);
        FullCfg fc;
        if (!n->pe && full_cfg(n->rows, s + n->new_syms, o->slope, fp64 ? 8 : 4, &fc) == SRA_OK) {
            cudaError_t e = launch_full_bound(fp64, n->dev, src, out, fc, n_hint, st);
            if (e != cudaSuccess) return fail(SRA_ECUDA, "full bound kernel launch: %s", cudaGetErrorString(e));
            return SRA_OK;
        }
        FullHbmCfg hc;
        if (full_hbm_cfg(n->dev, n->rows, o->slope, fp64 ? 8 : 4, kFullHbmBudget, &hc) != SRA_OK)
            return fail(SRA_EUNSUPPORTED, "affine-full state of one box exceeds %zu bytes", kFullHbmBudget / 2);
        if (n_hint <= 0) return SRA_OK;
        if (hc.chunk > n_hint) {  // one pass: scratch for the boxes there are
            hc.bytes = hc.bytes / (size_t)hc.chunk * (size_t)n_hint;
            hc.chunk = n_hint;
        }
        Scratch sc;
        sra_status r = scratch_alloc(sc, hc.bytes, st);
        if (r) return r;
        cudaError_t e = launch_full_hbm(fp64, n->dev, hc, src, out, n_hint, sc.p, st);
        if (e != cudaSuccess) return fail(SRA_ECUDA, "full (device-memory) kernel launch: %s", cudaGetErrorString(e));
        return SRA_OK;
    }
    int kmax = 0;
    sra_status r = kmax_for(n, o, s, &kmax);
    if (r) return r;
    RangeCfg cfg;
    r = make_cfg(n, o, kmax, fp64 ? 8 : 4, o->block_threads > 0 ? o->block_threads : 256, &cfg);
    if (r) return r;
    long long groups = (n_hint + cfg.NB - 1) / cfg.NB;
    long long cap = (long long)num_sms() * 64;
    if (src.list) cap = (long long)num_sms() * 8;
    long long grid = groups < cap ? groups : cap;
    if (grid < 1) grid = 1;
    cudaError_t e = fp64 ? launch_bound_f64(kmax, n->dev, src, out, cfg, grid, st)
                         : launch_bound_f32(kmax, n->dev, src, out, cfg, grid, st);
    if (e != cudaSuccess) return fail(SRA_ECUDA, "bound kernel launch: %s", cudaGetErrorString(e));
    return SRA_OK;
}

// FP32 (or FP64) bound with an optional FP64 re-check of near-zero UNKNOWNs.
sra_status bound_with_recheck(const sra_net *n, const sra_opts *o, BoxSrc src, BoundOut out,
                              long long count, unsigned long long *recheck_counter,
                              cudaStream_t st) {
    const bool bf16 = o->precision == SRA_PREC_BF16_SOUND || o->precision == SRA_PREC_BF16;
    if (bf16 && (!n->tc_ok || o->arith != SRA_ARITH_AFFINE_TRUNCATE || !tc_kt_served(o->K, n->tc_H) ||
                 o->slope != SRA_SLOPE_CHEBYSHEV))
        return fail(SRA_EUNSUPPORTED,
                    "BF16 tensor-core bounds need a 3 -> H x L -> 1 network with one activation (ReLU, ELU or sin; "
                    "H = 128, 256 or 512, at most %d hidden tensor-core layers) with affine-truncate K = 16, 32, "
                    "64 or (H <= 256) 128 and the Chebyshev slope",
                    kMaxTcLayers);
    const bool fp64 = o->precision == SRA_PREC_FP64;
    const bool recheck = o->recheck && !fp64;
    Scratch sc;
    if (recheck) {
        sra_status r = scratch_alloc(sc, align16(sizeof(int)) + (size_t)count * sizeof(int), st);
        if (r) return r;
        out.flag_count = (int *)sc.p;
        out.flag_list = (int *)((char *)sc.p + align16(sizeof(int)));
        out.band = o->recheck_band;
        SRA_CK(cudaMemsetAsync(out.flag_count, 0, sizeof(int), st));
    }
    sra_status r = SRA_OK;
    if (bf16) {
        const int nb = tc_boxes_per_tile(n->tc_H, o->K);
        const long long tiles = (count + nb - 1) / nb;
        long long grid = num_sms();
        if (grid > tiles) grid = tiles;
        if (grid < 1) grid = 1;
        const int stall = g_test_tc_stall.load();
        cudaError_t e;
        if (stall > 0) {  // sra_test_tc_stall: a copy of the parameters with the stall set
            TcParams p = n->tcp;
            p.test_stall = stall;
            e = launch_tc_bound(n->tc_H, o->K, o->precision == SRA_PREC_BF16_SOUND, p, src, out, (int)grid, st);
        } else {
            e = launch_tc_bound(n->tc_H, o->K, o->precision == SRA_PREC_BF16_SOUND, n->tcp, src, out, (int)grid,
                                st);
        }
        if (e != cudaSuccess) return fail(SRA_ECUDA, "tensor-core bound launch: %s", cudaGetErrorString(e));
    } else {
        r = run_bound(n, o, fp64, 3, src, out, count, st);
        if (r) return r;
    }
    if (recheck) {
        BoxSrc s2 = src;
        s2.list = out.flag_list;
        s2.list_count = out.flag_count;
        BoundOut o2 = out;
        o2.flag_list = nullptr;
        o2.flag_count = nullptr;
        o2.recheck_counter = recheck_counter;
        r = run_bound(n, o, true, 3, s2, o2, count, st);
        if (r) return r;
    }
    return SRA_OK;
}

sra_status check_net(const sra_net *n) {
    if (!n) return fail(SRA_EINVAL, "net is NULL");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != n->device) return fail(SRA_EINVAL, "net was loaded on device %d, current is %d", n->device, dev);
    return SRA_OK;
}

// Prepare the tensor-core path if the network has its shape: 3 inputs,
// L-1 >= 2 hidden layers of widths up to 512, all ReLU, all ELU or all sin,
// scalar output. The kernel runs at one width H in {128, 256, 512}, the
// smallest that holds every hidden layer (M = 128 is its MMA tile): a network
// narrower than H somewhere runs on weights padded with zeros. The padded
// neurons get exactly zero weights, bias and output weight, so their value
// and noise entries are 0, their range is [0, 0] and each rule maps it to 0
// (a new symbol of magnitude 0, or the rule's padding of it, which meets
// only zero weights), and the real neurons' sums gain only zero terms. The
// rounding constants take the padded width, whose sums are the longer ones.
void prepare_tc(sra_net *n, const float *params) {
    const int L = n->L;
    if (n->pe || L < 3 || L - 2 > kMaxTcLayers || n->widths.size() != (size_t)L + 1 || n->widths[0] != 3 ||
        n->widths[L] != 1)
        return;
    int wmax = 0;
    for (int l = 1; l < L; ++l) {
        if (n->widths[l] < 1 || n->widths[l] > 512) return;
        wmax = std::max(wmax, n->widths[l]);
    }
    const int act = n->acts[0];
    if (act != SRA_ACT_RELU && act != SRA_ACT_ELU && act != SRA_ACT_SIN) return;
    for (int l = 0; l + 1 < L; ++l)
        if (n->acts[l] != act) return;
    const int H = wmax <= 128 ? 128 : (wmax <= 256 ? 256 : 512);  // kernel width
    const int nh = L - 2;
    const size_t per = (size_t)H * H * 2;
    // device layout: W_b, W_r of every hidden layer; the status word (256 B);
    // then FP32 [H] biases of layers 0 .. L-2, the output weights [H] and the
    // first layer's weights [H][3], zero past the network's widths
    const size_t off_status = 2 * nh * per, off_bias = off_status + 256;
    const size_t off_wout = off_bias + (size_t)(L - 1) * H * 4, off_w0 = off_wout + (size_t)H * 4;
    const size_t bytes = off_w0 + (size_t)H * 3 * 4;
    if (cudaMalloc(&n->tc_buf, bytes) != cudaSuccess) { n->tc_buf = nullptr; cudaGetLastError(); return; }
    char *dev = (char *)n->tc_buf;
    auto give_up = [&]() {
        cudaFree(n->tc_buf);
        n->tc_buf = nullptr;
        cudaGetLastError();
    };
    std::vector<__nv_bfloat16> hi((size_t)H * H), lo((size_t)H * H);
    std::vector<float> tail((bytes - off_bias) / 4, 0.f);  // biases, output and first-layer weights
    float *bias = tail.data(), *wout = bias + (size_t)(L - 1) * H, *w0 = wout + H;
    // layer 0: W0 [w1][3] row-major, then b0 [w1]
    const int w1 = n->widths[1];
    for (int i = 0; i < w1; ++i)
        for (int d = 0; d < 3; ++d) w0[i * 3 + d] = params[i * 3 + d];
    for (int i = 0; i < w1; ++i) bias[i] = params[3 * w1 + i];
    size_t off = (size_t)3 * w1 + w1;
    TcParams &t = n->tcp;
    memset(&t, 0, sizeof t);
    for (int l = 1; l <= nh; ++l) {
        const int in = n->widths[l], out = n->widths[l + 1];
        const float *W = params + off;  // [out][in] row-major
        std::fill(hi.begin(), hi.end(), __float2bfloat16_rn(0.f));
        std::fill(lo.begin(), lo.end(), __float2bfloat16_rn(0.f));
        for (int i = 0; i < out; ++i)
            for (int j = 0; j < in; ++j) {
                const float w = W[(size_t)i * in + j];
                const __nv_bfloat16 h = __float2bfloat16_rn(w);
                hi[(size_t)i * H + j] = h;
                lo[(size_t)i * H + j] = __float2bfloat16_rn(w - __bfloat162float(h));
            }
        for (int i = 0; i < out; ++i) bias[(size_t)l * H + i] = params[off + (size_t)out * in + i];
        char *dhi = dev + (2 * (l - 1)) * per, *dlo = dhi + per;
        if (cudaMemcpy(dhi, hi.data(), per, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(dlo, lo.data(), per, cudaMemcpyHostToDevice) != cudaSuccess ||
            make_bf16_tile_map(&t.wb[l - 1], dhi, H, H, 128, 64) != 0 ||
            make_bf16_tile_map(&t.wr[l - 1], dlo, H, H, 128, 64) != 0) {
            give_up();
            return;
        }
        off += (size_t)out * in + out;
    }
    const int wl = n->widths[L - 1];
    for (int i = 0; i < wl; ++i) wout[i] = params[off + i];  // output layer [1][wl], then its bias
    if (cudaMemcpy(dev + off_bias, tail.data(), tail.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(dev + off_status, 0, sizeof(int)) != cudaSuccess) {
        give_up();
        return;
    }
    for (int l = 0; l + 1 < L; ++l) t.b[l] = (const float *)(dev + off_bias + (size_t)l * H * 4);
    t.b[L - 1] = n->dev.layer[L - 1].b;
    t.W0 = (const float *)(dev + off_w0);
    t.wout = (const float *)(dev + off_wout);
    t.bout = params[off + wl];  // the output layer's bias follows its wl weights
    t.L = L;
    t.act = act;
    t.status = (int *)(dev + off_status);
    // rounding constants (u = 2^-24, u_b = 2^-8); accumulation model: each
    // 16-deep MMA step adds at most 17 * 2^-23 of the sum of its terms' sizes
    const double u = std::ldexp(1.0, -24), ub = std::ldexp(1.0, -8);
    const double n_steps = 2.0 * H / 16.0;
    const double gacc = 17.0 * n_steps * std::ldexp(1.0, -23);
    t.rho1 = (float)((ub * ub + gacc * (1.0 + 2.0 * ub)) * 1.001);
    t.kappa = (float)(1.0 / (1.0 - ub) * (1.0 + 1e-6));
    t.ub2u = (float)((ub + 2.0 * u) * 1.001);
    // output-layer dot products: per part 64 FMAs, then 4 part adds (and the bias)
    const double nsum = H + 4.0, ncen = 2.0 * H + 5.0;
    t.gam_out = (float)(nsum * u / (1.0 - nsum * u) * 1.001);
    t.gam_c_out = (float)(ncen * u / (1.0 - ncen * u) * 1.001);
    n->tc_H = H;
    n->tc_ok = true;
}

// Prepare the tensor-core ray kernel if the network has its shape: hidden
// widths up to 512, 1 <= L-2 <= 8 hidden-to-hidden layers, an input width
// (after the positional encoding) of at most 64, scalar output. The kernel
// runs at the width H in {128, 256, 512} that holds every hidden layer;
// narrower layers are padded with zeros (zero weights, biases and output
// weights: the padded neurons stay exactly zero, as in the bound kernel).
// Each layer becomes three BF16 matrices (W_b, W_r, and |W| rounded up);
// layer 0's K is padded to 64 with zero columns.
void prepare_tc_rays(sra_net *n, const float *params) {
    const int L = n->L;
    if (L < 3 || L - 2 > kMaxRayTc || n->widths.size() != (size_t)L + 1 || n->widths[L] != 1) return;
    if (n->din > tc_ray_max_din()) return;
    int wmax = 0;
    for (int l = 1; l < L; ++l) {
        if (n->widths[l] < 1 || n->widths[l] > 512) return;
        wmax = std::max(wmax, n->widths[l]);
    }
    const int H = wmax <= 128 ? 128 : (wmax <= 256 ? 256 : 512);  // kernel width
    const int nh = L - 2;
    const size_t per_h = (size_t)H * H * 2, per_0 = (size_t)H * 64 * 2;
    // W_b, W_r, |W| of layer 0 and the hidden layers; the status word
    // (256 B); FP32 [H] biases of layers 0 .. L-2 and the output weights [H]
    const size_t off_status = 3 * per_0 + 3 * nh * per_h, off_bias = off_status + 256;
    const size_t bytes = off_bias + (size_t)L * H * 4;
    if (cudaMalloc(&n->tcr_buf, bytes) != cudaSuccess) { n->tcr_buf = nullptr; cudaGetLastError(); return; }
    char *dev = (char *)n->tcr_buf;
    TcRayParams &t = n->tcrp;
    memset(&t, 0, sizeof t);
    // smallest BF16 >= x for x >= 0 (the next bit pattern up is the next
    // larger value of a non-negative BF16)
    auto bf16_up = [](float x) {
        __nv_bfloat16 h = __float2bfloat16_rn(x);
        if (__bfloat162float(h) < x) {
            uint16_t b;
            memcpy(&b, &h, 2);
            ++b;
            memcpy(&h, &b, 2);
        }
        return h;
    };
    // three matrices of one layer, from W [out][k_in] zero-padded to [H][K]
    auto upload = [&](const float *W, int out, int k_in, int K, char *dst, TcLayerMaps &maps) -> bool {
        const size_t per = (size_t)H * K;
        std::vector<__nv_bfloat16> m(3 * per);
        for (int r = 0; r < H; ++r)
            for (int k = 0; k < K; ++k) {
                const float w = (r < out && k < k_in) ? W[(size_t)r * k_in + k] : 0.f;
                const __nv_bfloat16 h = __float2bfloat16_rn(w);
                const size_t e = (size_t)r * K + k;
                m[e] = h;
                m[per + e] = __float2bfloat16_rn(w - __bfloat162float(h));
                m[2 * per + e] = bf16_up(std::fabs(w));
            }
        const size_t b = per * 2;
        return cudaMemcpy(dst, m.data(), 3 * b, cudaMemcpyHostToDevice) == cudaSuccess &&
               make_bf16_tile_map(&maps.wb, dst, H, K, 128, 64) == 0 &&
               make_bf16_tile_map(&maps.wr, dst + b, H, K, 128, 64) == 0 &&
               make_bf16_tile_map(&maps.wa, dst + 2 * b, H, K, 128, 64) == 0;
    };
    std::vector<float> tail((size_t)L * H, 0.f);  // biases of layers 0 .. L-2, then the output weights
    const int w1 = n->widths[1];
    bool ok = upload(params, w1, n->din, 64, dev, t.first);
    for (int i = 0; i < w1; ++i) tail[i] = params[(size_t)n->din * w1 + i];
    size_t off = (size_t)n->din * w1 + w1;  // layer 1 starts after W0, b0
    for (int l = 1; ok && l <= nh; ++l) {
        const int in = n->widths[l], out = n->widths[l + 1];
        ok = upload(params + off, out, in, H, dev + 3 * per_0 + 3 * (l - 1) * per_h, t.hidden[l - 1]);
        for (int i = 0; i < out; ++i) tail[(size_t)l * H + i] = params[off + (size_t)out * in + i];
        off += (size_t)out * in + out;
    }
    const int wl = n->widths[L - 1];
    for (int i = 0; i < wl; ++i) tail[(size_t)(L - 1) * H + i] = params[off + i];
    ok = ok && cudaMemcpy(dev + off_bias, tail.data(), tail.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        cudaFree(n->tcr_buf);
        n->tcr_buf = nullptr;
        cudaGetLastError();
        return;
    }
    for (int l = 0; l + 1 < L; ++l) t.b[l] = (const float *)(dev + off_bias + (size_t)l * H * 4);
    t.b[L - 1] = n->dev.layer[L - 1].b;
    for (int l = 0; l + 1 < L; ++l) t.act[l] = n->acts[l];
    t.wout = (const float *)(dev + off_bias + (size_t)(L - 1) * H * 4);
    t.bout = params[off + wl];  // the output layer's bias follows its wl weights
    t.L = L;
    t.din = n->din;
    t.pe = n->pe;
    t.status = (int *)(dev + off_status);
    // sound form: per linear layer of K inputs, D takes 2 K/16 MMA steps
    // (W_b and W_r) and each |W| x sum of Dx K/16; each 16-deep step adds at
    // most 17 * 2^-23 of its terms' sizes; W_b + W_r is within u_b^2 of W
    {
        const double u = std::ldexp(1.0, -24), ub = std::ldexp(1.0, -8);
        auto layer = [&](int K, float &kx, float &rhok) {
            const double gx = 17.0 * (K / 16.0) * std::ldexp(1.0, -23);
            const double gacc = 17.0 * (2.0 * K / 16.0) * std::ldexp(1.0, -23);
            const double k = 1.0 / (1.0 - gx) * (1.0 + 1e-6);
            kx = (float)k;
            rhok = (float)((ub * ub + gacc * (1.0 + 2.0 * ub)) * k * 1.001);
        };
        layer(64, t.kx0, t.rhok0);
        layer(H, t.kx, t.rhok);
        // output layer: 64-term fmaf parts, H/64 part adds, the pair sums of
        // the operands and the final add
        const double nsum = H + H / 64.0 + 3.0;
        t.gam_out = (float)(nsum * u / (1.0 - nsum * u) * 1.001);
    }
    cudaMemset(t.status, 0, sizeof(int));
    n->tcr_H = H;
    n->tcr_ok = true;
}

// Streams the library forks work onto (per device, created on first use and
// kept for the process lifetime).
constexpr int kPoolStreams = 8;
std::mutex g_pool_mu;
std::vector<cudaStream_t> g_pool[64];

cudaStream_t pool_stream(int k) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_pool_mu);
    std::vector<cudaStream_t> &p = g_pool[dev & 63];
    while ((int)p.size() < kPoolStreams) {
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            break;
        }
        p.push_back(s);
    }
    return p.empty() ? nullptr : p[k % p.size()];
}

// Run n pieces of work concurrently: piece q is enqueued by f(q, stream) on a
// pooled stream that first waits for everything already on st; st then waits
// for all pieces. With one piece (or no pool) everything goes on st.
template <typename F> sra_status fork_join(cudaStream_t st, int n, F &&f) {
    if (n <= 1 || !pool_stream(0)) {
        for (int q = 0; q < n; ++q) {
            sra_status r = f(q, st);
            if (r) return r;
        }
        return SRA_OK;
    }
    cudaEvent_t fork = nullptr;
    SRA_CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    SRA_CK(cudaEventRecord(fork, st));
    sra_status status = SRA_OK;
    const int used = n < kPoolStreams ? n : kPoolStreams;
    for (int q = 0; q < n && status == SRA_OK; ++q) {
        cudaStream_t ls = pool_stream(q);
        if (q < used && cudaStreamWaitEvent(ls, fork, 0) != cudaSuccess) status = fail(SRA_ECUDA, "fork wait");
        if (status == SRA_OK) status = f(q, ls);
    }
    for (int q = 0; q < used; ++q) {  // join every stream that received work
        cudaEvent_t j = nullptr;
        if (cudaEventCreateWithFlags(&j, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(j, pool_stream(q)) != cudaSuccess || cudaStreamWaitEvent(st, j, 0) != cudaSuccess) {
            if (status == SRA_OK) status = fail(SRA_ECUDA, "join");
        }
        if (j) cudaEventDestroy(j);
    }
    cudaEventDestroy(fork);
    return status;
}

}  // namespace

sra_status sra::set_error(sra_status s, const char *fmt, ...) {
    char b[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b, sizeof b, fmt, ap);
    va_end(ap);
    g_err = b;
    return s;
}

extern "C" {

const char *sra_last_error(void) { return g_err.c_str(); }

void sra_default_opts(sra_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->arith = SRA_ARITH_AFFINE_FIXED;
    o->K = 0;
    o->slope = SRA_SLOPE_CHEBYSHEV;
    o->precision = SRA_PREC_FP32;
    o->recheck = 0;
    o->recheck_band = 1e-5f;
    o->split = SRA_SPLIT_OCTREE;
    o->delta = 1e-3f;
    o->t_max = 10.f;
    o->sigma0 = 1.f;
    o->eta_plus = 1.5f;
    o->eta_minus = 0.5f;
    o->safety = 0.98f;
    o->max_iters = 1 << 20;
}

sra_status sra_load_mlp(const sra_mlp_desc *d, sra_net **out) {
    g_err.clear();
    if (!d || !out) return fail(SRA_EINVAL, "desc/out is NULL");
    *out = nullptr;
    const int L = d->n_layers;
    if (L < 1 || L > kMaxLayers) return fail(SRA_EUNSUPPORTED, "n_layers %d outside [1, %d]", L, kMaxLayers);
    if (!d->widths || !d->params || (L > 1 && !d->acts)) return fail(SRA_EINVAL, "null widths/acts/params");
    if (d->pe_octaves < 0 || d->pe_octaves > 12) return fail(SRA_EINVAL, "pe_octaves %d", d->pe_octaves);
    const int din = d->pe_octaves ? 3 + 6 * d->pe_octaves : 3;
    if (d->widths[0] != din) return fail(SRA_EINVAL, "widths[0]=%d, expected %d", d->widths[0], din);
    if (d->widths[L] != 1) return fail(SRA_EINVAL, "widths[n_layers] must be 1");
    for (int l = 0; l <= L; ++l) {
        if (d->widths[l] < 1) return fail(SRA_EINVAL, "widths[%d]=%d", l, d->widths[l]);
        if (d->widths[l] > kMaxWidth) return fail(SRA_EUNSUPPORTED, "width %d > %d", d->widths[l], kMaxWidth);
    }
    for (int l = 0; l + 1 < L; ++l)
        if (d->acts[l] < SRA_ACT_IDENTITY || d->acts[l] > SRA_ACT_SIN)
            return fail(SRA_EINVAL, "acts[%d]=%d", l, d->acts[l]);
    int dev = 0;
    SRA_CK(cudaGetDevice(&dev));
    sra_net *n = new sra_net();
    n->device = dev;
    n->L = L;
    n->pe = d->pe_octaves;
    n->din = din;
    n->widths.assign(d->widths, d->widths + L + 1);
    n->acts.assign(L > 1 ? d->acts : d->widths, L > 1 ? d->acts + (L - 1) : d->widths);
    int rows = 3, hmax = din;
    for (int l = 0; l <= L; ++l) rows = rows > d->widths[l] ? rows : d->widths[l];
    for (int l = 1; l < L; ++l) hmax = hmax > d->widths[l] ? hmax : d->widths[l];
    n->rows = rows;
    n->H = ((hmax + 31) / 32) * 32;
    n->new_syms = 6 * n->pe;
    for (int l = 0; l + 1 < L; ++l)
        if (n->acts[l] != SRA_ACT_IDENTITY) n->new_syms += d->widths[l + 1];

    // device layout: per layer Wt (f32), b (f32), Wt64, b64; 256-byte aligned
    std::vector<size_t> off_w(L), off_b(L), off_w64(L), off_b64(L);
    size_t total = 0;
    auto take = [&](size_t bytes) {
        size_t o = total;
        total += (bytes + 255) & ~size_t(255);
        return o;
    };
    for (int l = 0; l < L; ++l) {
        const size_t in = d->widths[l], o = d->widths[l + 1];
        off_w[l] = take(in * o * 4);
        off_b[l] = take(o * 4);
        off_w64[l] = take(in * o * 8);
        off_b64[l] = take(o * 8);
    }
    std::vector<char> host(total, 0);
    size_t p = 0;
    for (int l = 0; l < L; ++l) {
        const int in = d->widths[l], o = d->widths[l + 1];
        const float *W = d->params + p, *b = W + (size_t)in * o;
        float *wt = (float *)(host.data() + off_w[l]);
        double *wt64 = (double *)(host.data() + off_w64[l]);
        for (int i = 0; i < o; ++i)
            for (int j = 0; j < in; ++j) {
                wt[(size_t)j * o + i] = W[(size_t)i * in + j];
                wt64[(size_t)j * o + i] = (double)W[(size_t)i * in + j];
            }
        memcpy(host.data() + off_b[l], b, (size_t)o * 4);
        double *b64 = (double *)(host.data() + off_b64[l]);
        for (int i = 0; i < o; ++i) b64[i] = (double)b[i];
        p += (size_t)in * o + o;
    }
    if (take_injected_failure()) {
        delete n;
        return fail(SRA_ENOMEM, "cudaMalloc(%zu): injected allocation failure", total);
    }
    cudaError_t e = cudaMalloc(&n->buf, total);
    if (e != cudaSuccess) {
        delete n;
        return fail(SRA_ENOMEM, "cudaMalloc(%zu): %s", total, cudaGetErrorString(e));
    }
    e = cudaMemcpy(n->buf, host.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(n->buf);
        delete n;
        return fail(SRA_ECUDA, "cudaMemcpy: %s", cudaGetErrorString(e));
    }
    memset(&n->dev, 0, sizeof n->dev);
    n->dev.L = L;
    n->dev.pe = n->pe;
    n->dev.din = din;
    char *base = (char *)n->buf;
    for (int l = 0; l < L; ++l) {
        LayerDev &ld = n->dev.layer[l];
        ld.Wt = (const float *)(base + off_w[l]);
        ld.b = (const float *)(base + off_b[l]);
        ld.Wt64 = (const double *)(base + off_w64[l]);
        ld.b64 = (const double *)(base + off_b64[l]);
        ld.in = d->widths[l];
        ld.out = d->widths[l + 1];
        ld.act = (l + 1 < L) ? n->acts[l] : SRA_ACT_IDENTITY;
    }
    prepare_tc(n, d->params);
    prepare_tc_rays(n, d->params);
    cudaGetLastError();
    *out = n;
    return SRA_OK;
}

sra_status sra_free_mlp(sra_net *n) {
    if (!n) return SRA_OK;
    cudaDeviceSynchronize();
    if (n->buf) cudaFree(n->buf);
    if (n->tc_buf) cudaFree(n->tc_buf);
    if (n->tcr_buf) cudaFree(n->tcr_buf);
    delete n;
    return SRA_OK;
}

sra_status sra_bound_boxes(const sra_net *n, const sra_opts *o, const float *centers,
                           const float *halfw, int64_t count, float *lo, float *hi, uint8_t *cls,
                           void *stream) {
    g_err.clear();
    sra_status r = check_net(n);
    if (r) return r;
    if ((r = check_opts(o))) return r;
    if (count < 0) return fail(SRA_EINVAL, "n < 0");
    if (count == 0) return SRA_OK;
    if (count > INT32_MAX) return fail(SRA_EINVAL, "n > 2^31-1");
    if (!centers || !halfw || !cls) return fail(SRA_EINVAL, "null centers/halfw/cls");
    BoxSrc src;
    memset(&src, 0, sizeof src);
    src.kind = SRC_BOXES;
    src.centers = centers;
    src.halfw = halfw;
    src.n = count;
    BoundOut out;
    memset(&out, 0, sizeof out);
    out.lo = lo;
    out.hi = hi;
    out.cls = cls;
    return bound_with_recheck(n, o, src, out, count, (unsigned long long *)o->recheck_count, as_stream(stream));
}

sra_status sra_eval(const sra_net *n, const float *x, int64_t count, float *y, void *stream) {
    g_err.clear();
    sra_status r = check_net(n);
    if (r) return r;
    if (count < 0 || (count > 0 && (!x || !y))) return fail(SRA_EINVAL, "bad eval arguments");
    if (count == 0) return SRA_OK;
    sra_opts o;
    sra_default_opts(&o);
    o.arith = SRA_ARITH_INTERVAL;  // zero-width intervals: exact plain forward pass
    BoxSrc src;
    memset(&src, 0, sizeof src);
    src.kind = SRC_POINTS;
    src.centers = x;
    src.n = count;
    BoundOut out;
    memset(&out, 0, sizeof out);
    out.lo = y;
    return run_bound(n, &o, false, 1, src, out, count, as_stream(stream));
}

sra_status sra_empty_spheres(const sra_net *n, const sra_opts *o, const float *points, int64_t count, float r_max,
                             int32_t levels, float *radius, void *stream) {
    g_err.clear();
    sra_status r = check_net(n);
    if (r) return r;
    if ((r = check_opts(o))) return r;
    if (o->precision != SRA_PREC_FP32 && o->precision != SRA_PREC_FP64)
        return fail(SRA_EUNSUPPORTED, "empty-sphere queries run in FP32 or FP64");
    if (!(r_max > 0.f) || levels < 1 || levels > 30) return fail(SRA_EINVAL, "need r_max > 0 and 1 <= levels <= 30");
    if (count < 0 || count > INT32_MAX) return fail(SRA_EINVAL, "n outside [0, 2^31 - 1]");
    if (count == 0) return SRA_OK;
    if (!points || !radius) return fail(SRA_EINVAL, "null points / radius_out");
    cudaStream_t st = as_stream(stream);
    int *list[2], *cnt;
    float *halfw;
    uint8_t *cls;
    auto carve = [&](Carve &c) {
        list[0] = c.take<int>(count);
        list[1] = c.take<int>(count);
        halfw = c.take<float>(3 * count);
        cls = c.take<uint8_t>(count);
        cnt = c.take<int>(16);  // [0], [1]: list counts; [4..5]: recheck tally
    };
    Carve sizing;
    carve(sizing);
    Scratch sc;
    if ((r = scratch_alloc(sc, sizing.off, st))) return r;
    Carve cv;
    cv.base = (char *)sc.p;
    cv.cap = sizing.off;
    carve(cv);
    if (cv.overflow) return fail(SRA_ECUDA, "sphere scratch layout exceeds its allocation");
    cudaError_t e = launch_sphere_init(count, list[0], &cnt[0], radius, st);
    if (e != cudaSuccess) return fail(SRA_ECUDA, "sphere init: %s", cudaGetErrorString(e));
    float rk = r_max;
    for (int k = 0; k < levels; ++k, rk *= 0.5f) {
        const int a = k & 1, b = a ^ 1;
        SRA_CK(cudaMemsetAsync(&cnt[b], 0, sizeof(int), st));
        if ((e = launch_sphere_halfw(count, list[a], &cnt[a], rk, halfw, st)) != cudaSuccess)
            return fail(SRA_ECUDA, "sphere half-widths: %s", cudaGetErrorString(e));
        BoxSrc src;
        memset(&src, 0, sizeof src);
        src.kind = SRC_BOXES;
        src.centers = points;
        src.halfw = halfw;
        src.list = list[a];
        src.list_count = &cnt[a];
        BoundOut out;
        memset(&out, 0, sizeof out);
        out.cls = cls;
        if ((r = bound_with_recheck(n, o, src, out, count, (unsigned long long *)&cnt[4], st))) return r;
        if ((e = launch_sphere_update(count, list[a], &cnt[a], cls, rk, radius, list[b], &cnt[b], st)) != cudaSuccess)
            return fail(SRA_ECUDA, "sphere update: %s", cudaGetErrorString(e));
    }
    return SRA_OK;
}

sra_status sra_mesh_leaves(const sra_net *n, const float *root_lo, const float *root_hi, const sra_node *leaves,
                           int64_t n_leaves, int32_t sub_levels, float *tris, int64_t cap, int64_t *n_tris,
                           void *stream) {
    g_err.clear();
    sra_status r = check_net(n);
    if (r) return r;
    if ((r = refuse_capture(stream, "sra_mesh_leaves"))) return r;
    if (!root_lo || !root_hi || !n_tris) return fail(SRA_EINVAL, "null root / n_tris");
    for (int d = 0; d < 3; ++d)
        if (!(root_hi[d] > root_lo[d])) return fail(SRA_EINVAL, "empty root box on axis %d", d);
    if (sub_levels < 0 || sub_levels > 5) return fail(SRA_EINVAL, "sub_levels %d outside [0, 5]", sub_levels);
    if (n_leaves < 0 || cap < 0) return fail(SRA_EINVAL, "negative size");
    if ((n_leaves > 0 && !leaves) || (cap > 0 && !tris)) return fail(SRA_EINVAL, "null leaves / tris_out");
    *n_tris = 0;
    if (n_leaves == 0) return SRA_OK;
    cudaStream_t st = as_stream(stream);
    const long long G = (1 << sub_levels) + 1, per_leaf = G * G * G;
    long long chunk = (1ll << 22) / per_leaf;
    if (chunk < 1) chunk = 1;
    if (chunk > n_leaves) chunk = n_leaves;
    MeshArgs a;
    memset(&a, 0, sizeof a);
    a.sub = sub_levels;
    for (int d = 0; d < 3; ++d) {
        a.lo[d] = root_lo[d];
        a.ext[d] = root_hi[d] - root_lo[d];
    }
    a.n = chunk;
    const size_t b_pts = align16((size_t)chunk * per_leaf * 12), b_val = align16((size_t)chunk * per_leaf * 4),
                 b_blk = align16((size_t)mesh_blocks(a) * 8);
    Scratch sc;
    if ((r = scratch_alloc(sc, b_pts + b_val + b_blk + 16, st))) return r;
    float *pts = (float *)sc.p, *vals = (float *)((char *)sc.p + b_pts);
    long long *blk = (long long *)((char *)sc.p + b_pts + b_val);
    unsigned long long *counter = (unsigned long long *)((char *)sc.p + b_pts + b_val + b_blk);
    SRA_CK(cudaMemsetAsync(counter, 0, 8, st));
    sra_opts o;
    sra_default_opts(&o);
    o.arith = SRA_ARITH_INTERVAL;  // zero-width intervals: the plain forward pass of sra_eval
    for (long long off = 0; off < n_leaves; off += chunk) {
        a.leaves = leaves + off;
        a.n = (n_leaves - off < chunk) ? n_leaves - off : chunk;
        cudaError_t e = launch_mesh_points(a, pts, st);
        if (e != cudaSuccess) return fail(SRA_ECUDA, "mesh points: %s", cudaGetErrorString(e));
        BoxSrc src;
        memset(&src, 0, sizeof src);
        src.kind = SRC_POINTS;
        src.centers = pts;
        src.n = mesh_points(a);
        BoundOut out;
        memset(&out, 0, sizeof out);
        out.lo = vals;
        if ((r = run_bound(n, &o, false, 1, src, out, src.n, st))) return r;
        e = launch_mesh_tris(a, vals, blk, counter, tris, cap, st);
        if (e != cudaSuccess) return fail(SRA_ECUDA, "mesh triangles: %s", cudaGetErrorString(e));
    }
    unsigned long long total = 0;
    SRA_CK(cudaMemcpyAsync(&total, counter, 8, cudaMemcpyDeviceToHost, st));
    SRA_CK(cudaStreamSynchronize(st));
    *n_tris = (int64_t)total;
    if ((long long)total > cap)
        return fail(SRA_ECAPACITY, "%llu triangles, capacity %lld", total, (long long)cap);
    return SRA_OK;
}

sra_status sra_classify_and_split(const sra_net *n, const sra_opts *o, const float *root_lo,
                                  const float *root_hi, const sra_node *in, int64_t n_in,
                                  int32_t max_level, sra_node *out, int64_t cap_out,
                                  sra_node *leaves, int64_t cap_leaves, int64_t *counts,
                                  void *stream) {
    g_err.clear();
    sra_status r = check_net(n);
    if (r) return r;
    if ((r = check_opts(o))) return r;
    if (!root_lo || !root_hi || !counts) return fail(SRA_EINVAL, "null root/counts");
    for (int d = 0; d < 3; ++d)
        if (!(root_hi[d] > root_lo[d])) return fail(SRA_EINVAL, "empty root box on axis %d", d);
    const int lvl_cap = (o->split == SRA_SPLIT_OCTREE) ? 16 : kMaxKdLevels - 1;
    if (max_level < 0 || max_level > lvl_cap) return fail(SRA_EINVAL, "max_level %d outside [0, %d]", max_level, lvl_cap);
    if (n_in < 0 || cap_out < 0 || cap_leaves < 0) return fail(SRA_EINVAL, "negative size");
    if (n_in > INT32_MAX) return fail(SRA_EINVAL, "n_in > 2^31-1");
    if (n_in > 0 && !in) return fail(SRA_EINVAL, "null frontier_in");
    if ((cap_out > 0 && !out) || (cap_leaves > 0 && !leaves)) return fail(SRA_EINVAL, "null output buffer");
    if (n_in == 0) return SRA_OK;
    cudaStream_t st = as_stream(stream);

    BoxSrc src;
    memset(&src, 0, sizeof src);
    src.kind = SRC_NODES;
    src.nodes = in;
    src.n = n_in;
    src.split = o->split;
    unsigned char axis[kMaxKdLevels];
    kd_tables(root_lo, root_hi, src.kd_n3, axis);
    for (int d = 0; d < 3; ++d) {
        src.root_lo[d] = root_lo[d];
        src.root_ext[d] = root_hi[d] - root_lo[d];
    }
    const long long nblk = split_blocks(n_in);
    Scratch sc;
    const size_t cls_bytes = align16((size_t)n_in), blk_bytes = align16((size_t)nblk * 2 * 8);
    if ((r = scratch_alloc(sc, cls_bytes + blk_bytes, st))) return r;
    uint8_t *cls = (uint8_t *)sc.p;
    long long *blk = (long long *)((char *)sc.p + cls_bytes);

    BoundOut bo;
    memset(&bo, 0, sizeof bo);
    bo.cls = cls;
    if ((r = bound_with_recheck(n, o, src, bo, n_in,
                                (unsigned long long *)(counts + SRA_CNT_RECHECKED), st)))
        return r;
    Scratch scv;
    if (o->converge) {  // the convergence test of Proc. 3 on the small UNKNOWN nodes
        int *list, *iota, *cc;
        float *pts, *vals;
        auto carve = [&](Carve &c) {
            list = c.take<int>(n_in);
            iota = c.take<int>(6 * n_in);
            pts = c.take<float>(18 * n_in);
            vals = c.take<float>(6 * n_in);
            cc = c.take<int>(4);
        };
        Carve sizing;
        carve(sizing);
        if ((r = scratch_alloc(scv, sizing.off, st))) return r;
        Carve cv;
        cv.base = (char *)scv.p;
        cv.cap = sizing.off;
        carve(cv);
        if (cv.overflow) return fail(SRA_ECUDA, "convergence scratch layout exceeds its allocation");
        SRA_CK(cudaMemsetAsync(cc, 0, 16, st));
        const float wlim = (float)((double)o->delta / std::sqrt(3.0));
        cudaError_t e = launch_conv_points(src, cls, n_in, wlim, list, &cc[0], &cc[1], pts, st);
        if (e == cudaSuccess) e = launch_iota(iota, 6 * n_in, st);
        if (e != cudaSuccess) return fail(SRA_ECUDA, "convergence points: %s", cudaGetErrorString(e));
        sra_opts eo;
        sra_default_opts(&eo);
        eo.arith = SRA_ARITH_INTERVAL;  // zero-width intervals: the plain forward pass
        BoxSrc ps;
        memset(&ps, 0, sizeof ps);
        ps.kind = SRC_POINTS;
        ps.centers = pts;
        ps.list = iota;
        ps.list_count = &cc[1];
        BoundOut po;
        memset(&po, 0, sizeof po);
        po.lo = vals;
        if ((r = run_bound(n, &eo, false, 1, ps, po, 6 * n_in, st))) return r;
        if ((e = launch_conv_mark(list, &cc[0], n_in, vals, cls, st)) != cudaSuccess)
            return fail(SRA_ECUDA, "convergence marks: %s", cudaGetErrorString(e));
    }
    SplitArgs a;
    memset(&a, 0, sizeof a);
    a.cls = cls;
    a.in = in;
    a.n = n_in;
    a.max_level = max_level;
    a.split = o->split;
    memcpy(a.kd_axis, axis, sizeof axis);
    a.out = out;
    a.cap_out = cap_out;
    a.leaves = leaves;
    a.cap_leaves = cap_leaves;
    a.counts = (unsigned long long *)counts;
    a.blk = blk;
    cudaError_t e = launch_split(a, st);
    if (e != cudaSuccess) return fail(SRA_ECUDA, "split launch: %s", cudaGetErrorString(e));
    return SRA_OK;
}

sra_status sra_classify_and_split_batch(const sra_net *const *nets, const sra_opts *opts, int32_t n_nets,
                                        const float *root_lo, const float *root_hi, const sra_node *in,
                                        const sra_batch_seg *segs, int32_t n_segs, sra_node *out,
                                        sra_node *leaves, int64_t *counts, void *stream) {
    g_err.clear();
    if (!nets || !opts || n_nets < 1 || !segs || n_segs < 1 || !root_lo || !root_hi || !counts)
        return fail(SRA_EINVAL, "null or empty nets / opts / segs / root / counts");
    for (int d = 0; d < 3; ++d)
        if (!(root_hi[d] > root_lo[d])) return fail(SRA_EINVAL, "empty root box on axis %d", d);
    sra_status r;
    for (int k = 0; k < n_nets; ++k) {
        if ((r = check_net(nets[k]))) return r;
        if ((r = check_opts(&opts[k]))) return r;
        const int pr = opts[k].precision;
        if (pr == SRA_PREC_FP64 || opts[k].recheck || opts[k].converge)
            return fail(SRA_EUNSUPPORTED,
                        "batched rounds run in FP32 or BF16 without re-check or convergence test (opts[%d])", k);
        if ((pr == SRA_PREC_BF16 || pr == SRA_PREC_BF16_SOUND) &&
            (!nets[k]->tc_ok || opts[k].arith != SRA_ARITH_AFFINE_TRUNCATE || !tc_kt_served(opts[k].K, nets[k]->tc_H) ||
             opts[k].slope != SRA_SLOPE_CHEBYSHEV))
            return fail(SRA_EUNSUPPORTED,
                        "batched BF16 segments need a network with the tensor-core path and affine-truncate K = 16, "
                        "32, 64 or (H <= 256) 128 (opts[%d])", k);
    }
    cudaStream_t st = as_stream(stream);
    unsigned char n3[kMaxKdLevels][3], axis[kMaxKdLevels];
    kd_tables(root_lo, root_hi, n3, axis);
    std::vector<BatchSegDev> ds(n_segs);
    std::vector<BatchSplitSeg> ss(n_segs);
    std::vector<int> kmaxes(n_segs);
    std::vector<double> chunk_cost(n_segs);
    std::vector<char> on_tc(n_segs, 0);  // bounded on the tensor cores (BF16 / BF16-sound)
    long long cls_n = 0, nblk = 0;
    for (int s = 0; s < n_segs; ++s) {
        const sra_batch_seg &g = segs[s];
        if (g.net < 0 || g.net >= n_nets) return fail(SRA_EINVAL, "segment %d: net %d out of range", s, g.net);
        const sra_net *n = nets[g.net];
        const sra_opts *o = &opts[g.net];
        const int lvl_cap = (o->split == SRA_SPLIT_OCTREE) ? 16 : kMaxKdLevels - 1;
        if (g.max_level < 0 || g.max_level > lvl_cap)
            return fail(SRA_EINVAL, "segment %d: max_level %d outside [0, %d]", s, g.max_level, lvl_cap);
        if (g.first < 0 || g.n < 0 || g.n > INT32_MAX || g.out_first < 0 || g.cap_out < 0 || g.leaf_first < 0 ||
            g.cap_leaves < 0)
            return fail(SRA_EINVAL, "segment %d: negative or oversized range", s);
        if ((g.n > 0 && !in) || (g.cap_out > 0 && !out) || (g.cap_leaves > 0 && !leaves))
            return fail(SRA_EINVAL, "segment %d: null buffer", s);
        BatchSegDev &D = ds[s];
        memset(&D, 0, sizeof D);
        on_tc[s] = o->precision == SRA_PREC_BF16 || o->precision == SRA_PREC_BF16_SOUND;
        int kmax = 0;
        RangeCfg cfg;
        memset(&cfg, 0, sizeof cfg);
        if (!on_tc[s]) {
            if ((r = kmax_for(n, o, 3, &kmax))) return r;
            if ((r = make_cfg(n, o, kmax, 4, o->block_threads > 0 ? o->block_threads : 256, &cfg))) return r;
            cfg.threads = cfg.NB * cfg.H;
        }
        kmaxes[s] = kmax;
        D.net = n->dev;
        D.cfg = cfg;
        D.src.kind = SRC_NODES;
        D.src.nodes = in + g.first;
        D.src.n = g.n;
        D.src.split = o->split;
        memcpy(D.src.kd_n3, n3, sizeof n3);
        for (int d = 0; d < 3; ++d) {
            D.src.root_lo[d] = root_lo[d];
            D.src.root_ext[d] = root_hi[d] - root_lo[d];
        }
        double per_box = 0;
        for (int l = 0; l < n->L; ++l) per_box += (double)n->widths[l] * n->widths[l + 1] * (kmax + 2);
        chunk_cost[s] = per_box * (cfg.NB > 0 ? cfg.NB : 1);
        BatchSplitSeg &S = ss[s];
        memset(&S, 0, sizeof S);
        S.first = g.first;
        S.n = g.n;
        S.out_first = g.out_first;
        S.cap_out = g.cap_out;
        S.leaf_first = g.leaf_first;
        S.cap_leaves = g.cap_leaves;
        S.blk0 = nblk;
        S.max_level = g.max_level;
        S.split = o->split;
        memcpy(S.kd_axis, axis, sizeof axis);
        nblk += split_blocks(g.n);
        if (g.first + g.n > cls_n) cls_n = g.first + g.n;
    }
    // launches: one per (noise-column bound, CTA shape), segments heaviest
    // chunk first; the launches run concurrently on pooled streams
    std::vector<std::pair<int, int>> kinds;
    std::vector<int> tc_segs;  // one tensor-core launch each, beside the SIMT launches
    for (int s = 0; s < n_segs; ++s) {
        if (segs[s].n > 0 && on_tc[s]) tc_segs.push_back(s);
        if (on_tc[s]) continue;
        const std::pair<int, int> key(kmaxes[s], ds[s].cfg.threads);
        if (segs[s].n > 0 && std::find(kinds.begin(), kinds.end(), key) == kinds.end()) kinds.push_back(key);
    }
    std::vector<int> order;
    struct Launch { int kmax, off, cnt, threads, smem; long long chunks; double work; };
    std::vector<Launch> launches;
    for (const auto &kk : kinds) {
        const int km = kk.first;
        Launch L = {km, (int)order.size(), 0, 0, 0, 0, 0.0};
        std::vector<int> mine;
        for (int s = 0; s < n_segs; ++s)
            if (segs[s].n > 0 && !on_tc[s] && kmaxes[s] == km && ds[s].cfg.threads == kk.second) mine.push_back(s);
        std::stable_sort(mine.begin(), mine.end(), [&](int a, int b) { return chunk_cost[a] > chunk_cost[b]; });
        for (int s : mine) {
            ds[s].chunk0 = L.chunks;
            L.chunks += (segs[s].n + ds[s].cfg.NB - 1) / ds[s].cfg.NB;
            L.work += chunk_cost[s] * (double)((segs[s].n + ds[s].cfg.NB - 1) / ds[s].cfg.NB);
            L.threads = std::max(L.threads, ds[s].cfg.threads);
            L.smem = std::max(L.smem, ds[s].cfg.NB * ds[s].cfg.slot_bytes);
            order.push_back(s);
        }
        L.cnt = (int)mine.size();
        launches.push_back(L);
    }
    const size_t b_cls = align16((size_t)cls_n), b_blk = align16((size_t)nblk * 16),
                 b_ds = align16(ds.size() * sizeof(BatchSegDev)), b_ss = align16(ss.size() * sizeof(BatchSplitSeg)),
                 b_ord = align16((order.size() + 1) * sizeof(int)), b_next = align16(launches.size() * 8 + 8);
    Scratch sc;
    if ((r = scratch_alloc(sc, b_cls + b_blk + b_ds + b_ss + b_ord + b_next, st))) return r;
    char *base = (char *)sc.p;
    uint8_t *cls = (uint8_t *)base;
    long long *blk = (long long *)(base + b_cls);
    BatchSegDev *dsd = (BatchSegDev *)(base + b_cls + b_blk);
    BatchSplitSeg *ssd = (BatchSplitSeg *)(base + b_cls + b_blk + b_ds);
    int *ordd = (int *)(base + b_cls + b_blk + b_ds + b_ss);
    unsigned long long *next = (unsigned long long *)(base + b_cls + b_blk + b_ds + b_ss + b_ord);
    for (int s = 0; s < n_segs; ++s) ds[s].out.cls = cls + segs[s].first;
    // the segment tables travel as kernel parameters (no host memory is read
    // after these calls return, so the round can be captured into a graph)
    SRA_CK(upload(dsd, ds.data(), ds.size() * sizeof(BatchSegDev), st));
    SRA_CK(upload(ssd, ss.data(), ss.size() * sizeof(BatchSplitSeg), st));
    if (!order.empty()) SRA_CK(upload(ordd, order.data(), order.size() * sizeof(int), st));
    SRA_CK(cudaMemsetAsync(next, 0, launches.size() * 8 + 8, st));
    // heaviest launch first: the lighter ones fill the SMs its tail frees
    std::vector<size_t> lorder(launches.size());
    for (size_t k = 0; k < lorder.size(); ++k) lorder[k] = k;
    std::stable_sort(lorder.begin(), lorder.end(),
                     [&](size_t a, size_t b) { return launches[a].work > launches[b].work; });
    const int n_simt = (int)launches.size();
    if ((r = fork_join(st, n_simt + (int)tc_segs.size(), [&](int q, cudaStream_t ls) -> sra_status {
             if (q >= n_simt) {  // a tensor-core segment: its nodes, its classes
                 const int s = tc_segs[q - n_simt];
                 const sra_net *n = nets[segs[s].net];
                 BoundOut bo;
                 memset(&bo, 0, sizeof bo);
                 bo.cls = ds[s].out.cls;
                 const sra_opts &so = opts[segs[s].net];
                 const int nb = tc_boxes_per_tile(n->tc_H, so.K);
                 const long long tiles = (segs[s].n + nb - 1) / nb;
                 long long grid = num_sms();
                 if (grid > tiles) grid = tiles;
                 cudaError_t e = launch_tc_bound(n->tc_H, so.K, so.precision == SRA_PREC_BF16_SOUND, n->tcp,
                                                 ds[s].src, bo, (int)grid, ls);
                 if (e != cudaSuccess)
                     return fail(SRA_ECUDA, "batched tensor-core bound launch: %s", cudaGetErrorString(e));
                 return SRA_OK;
             }
             const size_t k = lorder[q];
             const Launch &L = launches[k];
             cudaError_t e = launch_multi_bound_f32(L.kmax, dsd, ordd + L.off, L.cnt, L.chunks, next + k,
                                                    L.threads, L.smem, ls);
             if (e != cudaSuccess)
                 return fail(SRA_ECUDA, "batched bound launch (K <= %d): %s", L.kmax, cudaGetErrorString(e));
             return SRA_OK;
         })))
        return r;
    cudaError_t e = launch_split_batch(cls, in, ssd, n_segs, nblk, out, leaves, (unsigned long long *)counts, blk, st);
    if (e != cudaSuccess) return fail(SRA_ECUDA, "batched split launch: %s", cudaGetErrorString(e));
    return SRA_OK;
}

// The plain forward pass f(x) at count points (zero-width intervals), in
// FP32 or FP64; with a list only at the listed points (y indexed by point).
static sra_status eval_points(const sra_net *n, bool fp64, const float *x, int64_t count, float *y,
                              const int *list, const int *list_count, cudaStream_t st) {
    sra_opts o;
    sra_default_opts(&o);
    o.arith = SRA_ARITH_INTERVAL;
    BoxSrc src;
    memset(&src, 0, sizeof src);
    src.kind = SRC_POINTS;
    src.centers = x;
    src.n = count;
    src.list = list;
    src.list_count = list_count;
    BoundOut out;
    memset(&out, 0, sizeof out);
    out.lo = y;
    return run_bound(n, &o, fp64, 1, src, out, count, st);
}

// The persistent SIMT ray kernel (FP32 or FP64) over rp (every field but the
// march options, which come from o); n_hint bounds the rays it can take.
static sra_status launch_rays(const sra_net *n, const sra_opts *o, bool fp64, RayParams rp, int64_t n_hint,
                              cudaStream_t st) {
    int kmax = 0;
    sra_status r = kmax_for(n, o, 1, &kmax);
    if (r) return r;
    RangeCfg cfg;
    if ((r = make_cfg(n, o, kmax, fp64 ? 8 : 4, 512, &cfg))) return r;
    rp.delta = o->delta;
    rp.t_max = o->t_max;
    rp.sigma0 = o->sigma0;
    rp.eta_plus = o->eta_plus;
    rp.eta_minus = o->eta_minus;
    rp.safety = o->safety;
    rp.max_iters = o->max_iters;
    const int per_sm = fp64 ? rays_blocks_per_sm_f64(kmax, cfg) : rays_blocks_per_sm_f32(kmax, cfg);
    long long grid = (long long)per_sm * num_sms();
    const long long need = (n_hint + cfg.NB - 1) / cfg.NB;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    cudaError_t e = fp64 ? launch_rays_f64(kmax, n->dev, &rp, cfg, (int)grid, st)
                         : launch_rays_f32(kmax, n->dev, &rp, cfg, (int)grid, st);
    if (e != cudaSuccess) return fail(SRA_ECUDA, "ray kernel launch: %s", cudaGetErrorString(e));
    return SRA_OK;
}

// Proc. 2 for `count` rays, resuming each ray from (t_start[i], sigma_start[i])
// when those are given (the hand-over of frustum casting).
static sra_status cast_rays_impl(const sra_net *n, const sra_opts *o, const float *origins, const float *dirs,
                                 int64_t count, float *t_hit, int32_t *iters, const float *t_start,
                                 const float *sigma_start, void *stream) {
    sra_status r = check_net(n);
    if (r) return r;
    if ((r = check_opts(o))) return r;
    if (count < 0) return fail(SRA_EINVAL, "n < 0");
    if (count == 0) return SRA_OK;
    if (!origins || !dirs || !t_hit) return fail(SRA_EINVAL, "null origins/dirs/t_hit");
    if (!(o->delta > 0.f) || !(o->t_max > 0.f) || !(o->sigma0 > 0.f) || !(o->eta_plus >= 1.f) ||
        !(o->eta_minus > 0.f && o->eta_minus < 1.f) || !(o->safety > 0.f && o->safety <= 1.f) ||
        o->max_iters < 1)
        return fail(SRA_EINVAL, "ray options out of range (delta, t_max, sigma0 > 0; eta+ >= 1; "
                                "0 < eta- < 1; 0 < safety <= 1; max_iters >= 1)");
    const bool sound = o->precision == SRA_PREC_BF16_SOUND;
    const bool tc = o->precision == SRA_PREC_BF16 || sound, fp64 = o->precision == SRA_PREC_FP64;
    if (o->precision != SRA_PREC_FP32 && !tc && !fp64)
        return fail(SRA_EUNSUPPORTED, "cast_rays runs in FP32, FP64 or (tensor cores) BF16 / BF16-sound");
    if (tc && (!n->tcr_ok || o->arith != SRA_ARITH_AFFINE_FIXED))
        return fail(SRA_EUNSUPPORTED, "BF16 cast_rays needs affine-fixed arithmetic and a net of "
                                      "uniform hidden width 128/256/512 with 1..%d hidden layers and "
                                      "input width <= %d", kMaxRayTc, tc_ray_max_din());
    if (sound && o->slope != SRA_SLOPE_CHEBYSHEV)
        return fail(SRA_EUNSUPPORTED, "BF16-sound cast_rays uses the Chebyshev slope");
    if (count > INT32_MAX) return fail(SRA_EINVAL, "n > 2^31 - 1");
    const bool recheck = o->recheck && !fp64;
    cudaStream_t st = as_stream(stream);
    float *f0;
    int *flags = nullptr, *cnt;
    unsigned long long *next;
    auto carve = [&](Carve &c) {
        f0 = c.take<float>(count);
        if (recheck) flags = c.take<int>(count);
        next = c.take<unsigned long long>(2);  // [0] main march, [1] FP64 re-check
        cnt = c.take<int>(4);                  // [0] flagged rays
    };
    Carve sizing;
    carve(sizing);
    Scratch sc;
    if ((r = scratch_alloc(sc, sizing.off, st))) return r;
    Carve cv;
    cv.base = (char *)sc.p;
    cv.cap = sizing.off;
    carve(cv);
    if (cv.overflow) return fail(SRA_ECUDA, "ray scratch layout exceeds its allocation");
    SRA_CK(cudaMemsetAsync(next, 0, 2 * sizeof(unsigned long long), st));
    SRA_CK(cudaMemsetAsync(cnt, 0, 4 * sizeof(int), st));
    // f(p) at every origin, in the march's precision: the reference sign of
    // DifferentSigns (Proc. 2)
    if ((r = eval_points(n, fp64, origins, count, f0, nullptr, nullptr, st))) return r;
    if (tc) {
        TcRayParams p = n->tcrp;
        p.slope = o->slope;
        p.origins = origins;
        p.dirs = dirs;
        p.f0 = f0;
        p.t_hit = t_hit;
        p.iters = iters;
        p.t_start = t_start;
        p.sigma_start = sigma_start;
        p.n = count;
        p.next = next;
        p.delta = o->delta;
        p.t_max = o->t_max;
        p.sigma0 = o->sigma0;
        p.eta_plus = o->eta_plus;
        p.eta_minus = o->eta_minus;
        p.safety = o->safety;
        p.max_iters = o->max_iters;
        p.flag_list = flags;
        p.flag_count = cnt;
        p.band = o->recheck_band;
        long long grid = num_sms();
        const long long need = (count + tc_ray_slots() - 1) / tc_ray_slots();
        if (grid > need) grid = need;
        cudaError_t e = launch_tc_rays(n->tcr_H, sound, p, (int)grid, st);
        if (e != cudaSuccess) return fail(SRA_ECUDA, "tensor-core ray kernel launch: %s", cudaGetErrorString(e));
    } else {
        RayParams rp;
        memset(&rp, 0, sizeof rp);
        rp.origins = origins;
        rp.dirs = dirs;
        rp.f0 = f0;
        rp.t_hit = t_hit;
        rp.iters = iters;
        rp.t_start = t_start;
        rp.sigma_start = sigma_start;
        rp.n = count;
        rp.next = next;
        rp.flag_list = flags;
        rp.flag_count = cnt;
        rp.band = o->recheck_band;
        if ((r = launch_rays(n, o, fp64, rp, count, st))) return r;
    }
    if (!recheck) return SRA_OK;
    // FP64 re-check: the flagged rays march again from their start in FP64
    // (their origin signs too) and overwrite their results
    if ((r = eval_points(n, true, origins, count, f0, flags, cnt, st))) return r;
    RayParams rp;
    memset(&rp, 0, sizeof rp);
    rp.origins = origins;
    rp.dirs = dirs;
    rp.f0 = f0;
    rp.t_hit = t_hit;
    rp.iters = iters;
    rp.t_start = t_start;
    rp.sigma_start = sigma_start;
    rp.n = count;
    rp.next = next + 1;
    rp.list = flags;
    rp.list_count = cnt;
    rp.recheck_counter = (unsigned long long *)o->recheck_count;
    return launch_rays(n, o, true, rp, count, st);
}

sra_status sra_cast_frustum(const sra_net *n, const sra_opts *o, const float *eye, const float *dirs, int32_t W,
                            int32_t Hh, int32_t grid, float *t_hit, int32_t *iters, int64_t *stats, void *stream) {
    g_err.clear();
    sra_status r = check_net(n);
    if (r) return r;
    if ((r = refuse_capture(stream, "sra_cast_frustum"))) return r;
    if ((r = check_opts(o))) return r;
    if (!eye || !dirs || !t_hit) return fail(SRA_EINVAL, "null eye / dirs / t_hit");
    if (W < 1 || Hh < 1 || (long long)W * Hh > INT32_MAX || grid < 1 || grid > 4096)
        return fail(SRA_EINVAL, "bad image size %d x %d or grid %d", W, Hh, grid);
    if (!(o->delta > 0.f) || !(o->t_max > 0.f) || !(o->sigma0 > 0.f) || !(o->eta_plus >= 1.f) ||
        !(o->eta_minus > 0.f && o->eta_minus < 1.f) || !(o->safety > 0.f && o->safety <= 1.f) || o->max_iters < 1)
        return fail(SRA_EINVAL, "ray options out of range");
    if (o->precision != SRA_PREC_FP32 && o->precision != SRA_PREC_BF16)
        return fail(SRA_EUNSUPPORTED, "frustum casting hands pixels to the FP32 or BF16 ray kernels");
    cudaStream_t st = as_stream(stream);
    const long long npix = (long long)W * Hh;
    FrustumArgs a;
    memset(&a, 0, sizeof a);
    a.dirs = dirs;
    a.W = W;
    a.H = Hh;
    for (int d = 0; d < 3; ++d) a.eye[d] = eye[d];
    a.sigma0 = o->sigma0;
    a.t_max = o->t_max;
    a.eta_plus = o->eta_plus;
    a.eta_minus = o->eta_minus;
    a.safety = o->safety;
    a.delta = o->delta;
    sra_opts bo = *o;  // frustum boxes: FP32 bounds of the same arithmetic
    bo.precision = SRA_PREC_FP32;
    Frustum *fr[2];
    float *centers, *halfw, *ray_t, *ray_sigma;
    uint8_t *cls;
    int *ray_pix, *iota, *cnt;
    auto carve = [&](Carve &c) {
        fr[0] = c.take<Frustum>(npix);
        fr[1] = c.take<Frustum>(npix);
        centers = c.take<float>(3 * npix);
        halfw = c.take<float>(3 * npix);
        cls = c.take<uint8_t>(npix);
        ray_pix = c.take<int>(npix);
        ray_t = c.take<float>(npix);
        ray_sigma = c.take<float>(npix);
        iota = c.take<int>(npix);
        // [0] current frusta, [1] next frusta, [2] rays, [3] boxes bounded, [4..5] recheck tally
        cnt = c.take<int>(16);
    };
    Carve sizing;
    carve(sizing);
    Scratch sc;
    if ((r = scratch_alloc(sc, sizing.off, st))) return r;
    Carve cv;
    cv.base = (char *)sc.p;
    cv.cap = sizing.off;
    carve(cv);
    if (cv.overflow) return fail(SRA_ECUDA, "frustum scratch layout exceeds its allocation");
    SRA_CK(cudaMemsetAsync(cnt, 0, 64, st));
    cudaError_t e = launch_frustum_init(a, grid, fr[0], &cnt[0], st);
    if (e == cudaSuccess) e = launch_iota(iota, npix, st);
    if (e != cudaSuccess) return fail(SRA_ECUDA, "frustum init: %s", cudaGetErrorString(e));
    // Rounds run from device-side counts; the host reads them every kBatch
    // rounds (a round with no frusta left launches kernels that do nothing).
    constexpr int kBatch = 8;
    long long rounds = 0, boxes = 0;
    int host_cnt[4] = {1, 0, 0, 0};
    int cur = 0;
    while (host_cnt[0] > 0) {
        for (int k = 0; k < kBatch; ++k) {
            if (++rounds > 1000000) return fail(SRA_ETIMEOUT, "frustum march did not finish");
            SRA_CK(cudaMemsetAsync(&cnt[1], 0, sizeof(int), st));
            if ((e = launch_frustum_boxes(a, fr[cur], &cnt[0], npix, centers, halfw, st)) != cudaSuccess)
                return fail(SRA_ECUDA, "frustum boxes: %s", cudaGetErrorString(e));
            BoxSrc src;
            memset(&src, 0, sizeof src);
            src.kind = SRC_BOXES;
            src.centers = centers;
            src.halfw = halfw;
            src.list = iota;  // box b is frustum b, count on the device
            src.list_count = &cnt[0];
            BoundOut out;
            memset(&out, 0, sizeof out);
            out.cls = cls;
            if ((r = bound_with_recheck(n, &bo, src, out, npix, (unsigned long long *)&cnt[4], st))) return r;
            if ((e = launch_frustum_update(a, fr[cur], &cnt[0], npix, cls, fr[cur ^ 1], &cnt[1], ray_pix, ray_t,
                                           ray_sigma, &cnt[2], &cnt[3], t_hit, iters, st)) != cudaSuccess)
                return fail(SRA_ECUDA, "frustum update: %s", cudaGetErrorString(e));
            SRA_CK(cudaMemcpyAsync(&cnt[0], &cnt[1], sizeof(int), cudaMemcpyDeviceToDevice, st));
            cur ^= 1;
        }
        SRA_CK(cudaMemcpyAsync(host_cnt, cnt, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
        SRA_CK(cudaStreamSynchronize(st));
    }
    boxes = host_cnt[3];
    const int nr = host_cnt[2];
    if (stats) {
        stats[0] = rounds;
        stats[1] = boxes;
        stats[2] = nr;
        stats[3] = 0;
    }
    if (nr == 0) return SRA_OK;
    Scratch sr;
    const size_t b_r3 = align16((size_t)nr * 12), b_r = align16((size_t)nr * 4);
    if ((r = scratch_alloc(sr, 2 * b_r3 + 2 * b_r, st))) return r;
    float *org = (float *)sr.p, *dr = (float *)((char *)sr.p + b_r3);
    float *t_ray = (float *)((char *)sr.p + 2 * b_r3);
    int *it_ray = (int *)((char *)sr.p + 2 * b_r3 + b_r);
    if ((e = launch_ray_gather(a, ray_pix, nr, org, dr, st)) != cudaSuccess)
        return fail(SRA_ECUDA, "ray gather: %s", cudaGetErrorString(e));
    if ((r = cast_rays_impl(n, o, org, dr, nr, t_ray, it_ray, ray_t, ray_sigma, stream))) return r;
    if ((e = launch_ray_scatter(ray_pix, nr, t_ray, it_ray, t_hit, iters, st)) != cudaSuccess)
        return fail(SRA_ECUDA, "ray scatter: %s", cudaGetErrorString(e));
    return SRA_OK;
}

sra_status sra_cast_rays(const sra_net *n, const sra_opts *o, const float *origins,
                         const float *dirs, int64_t count, float *t_hit, int32_t *iters,
                         void *stream) {
    g_err.clear();
    return cast_rays_impl(n, o, origins, dirs, count, t_hit, iters, nullptr, nullptr, stream);
}

sra_status sra_extract_leaves(const sra_net *n, const sra_opts *o, const float *xl, const float *xu,
                              int32_t depth, sra_node *leaves, int64_t cap, int64_t *n_leaves,
                              int64_t *level_counts, void *stream) {
    g_err.clear();
    sra_status r = check_net(n);
    if (r) return r;
    if ((r = refuse_capture(stream, "sra_extract_leaves"))) return r;
    if ((r = check_opts(o))) return r;
    if (!xl || !xu || !n_leaves) return fail(SRA_EINVAL, "null xl/xu/n_leaves");
    if (cap < 0 || (cap > 0 && !leaves)) return fail(SRA_EINVAL, "bad leaves buffer");
    cudaStream_t st = as_stream(stream);
    const int fan = (o->split == SRA_SPLIT_OCTREE) ? 8 : 2;
    int64_t *dcounts = nullptr;
    sra_node *bufA = nullptr, *bufB = nullptr;
    size_t capA = 0, capB = 0;
    sra_status status = SRA_OK;
    int64_t hc[SRA_CNT_N] = {0};
    int64_t leaves_found = 0;
    long long ncur = 1;
    keep_pool_memory();
    auto grow = [&](sra_node **b, size_t *c, size_t need) -> sra_status {
        if (need <= *c) return SRA_OK;
        if (*b) cudaFreeAsync(*b, st);
        *b = nullptr;
        size_t want = need < 1024 ? 1024 : need;
        cudaError_t e = cudaMallocAsync((void **)b, want * sizeof(sra_node), st);
        if (e != cudaSuccess) {
            *b = nullptr;
            *c = 0;
            return fail(SRA_ENOMEM, "frontier buffer of %zu nodes: %s", want, cudaGetErrorString(e));
        }
        *c = want;
        return SRA_OK;
    };
    cudaError_t e = cudaMallocAsync((void **)&dcounts, SRA_CNT_N * sizeof(int64_t), st);
    if (e != cudaSuccess) return fail(SRA_ENOMEM, "counts: %s", cudaGetErrorString(e));
    if ((status = grow(&bufA, &capA, 1)) == SRA_OK) {
        sra_node root = {0, 0, 0, 0};
        e = cudaMemcpyAsync(bufA, &root, sizeof root, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) status = fail(SRA_ECUDA, "root upload: %s", cudaGetErrorString(e));
        // the host copy must stay valid until the copy ran
        if (status == SRA_OK && cudaStreamSynchronize(st) != cudaSuccess)
            status = fail(SRA_ECUDA, "stream sync");
    }
    for (int level = 0; status == SRA_OK && level <= depth; ++level) {
        const size_t next = (level < depth) ? (size_t)ncur * fan : 0;
        if ((status = grow(&bufB, &capB, next > 0 ? next : 1)) != SRA_OK) break;
        e = cudaMemsetAsync(dcounts, 0, SRA_CNT_N * sizeof(int64_t), st);
        if (e != cudaSuccess) { status = fail(SRA_ECUDA, "memset: %s", cudaGetErrorString(e)); break; }
        // leaves of every level go after those already found (the convergence
        // test returns leaves above the last level)
        const int64_t lcap = cap > leaves_found ? cap - leaves_found : 0;
        status = sra_classify_and_split(n, o, xl, xu, bufA, ncur, depth, bufB, (int64_t)next,
                                        lcap > 0 ? leaves + leaves_found : nullptr, lcap, dcounts, stream);
        if (status) break;
        e = cudaMemcpyAsync(hc, dcounts, sizeof hc, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { status = fail(SRA_ECUDA, "level %d: %s", level, cudaGetErrorString(e)); break; }
        if (level_counts) {
            level_counts[level * 3 + 0] = hc[SRA_CNT_POSITIVE];
            level_counts[level * 3 + 1] = hc[SRA_CNT_NEGATIVE];
            level_counts[level * 3 + 2] = hc[SRA_CNT_UNKNOWN];
        }
        ncur = hc[SRA_CNT_CHILDREN];
        leaves_found += hc[SRA_CNT_LEAVES];
        std::swap(bufA, bufB);
        std::swap(capA, capB);
        if (ncur == 0 && level < depth) {
            for (int k = level + 1; level_counts && k <= depth; ++k)
                level_counts[k * 3 + 0] = level_counts[k * 3 + 1] = level_counts[k * 3 + 2] = 0;
            break;
        }
    }
    if (bufA) cudaFreeAsync(bufA, st);
    if (bufB) cudaFreeAsync(bufB, st);
    cudaFreeAsync(dcounts, st);
    if (status) return status;
    *n_leaves = leaves_found;
    if (leaves_found > cap)
        return fail(SRA_ECAPACITY, "%lld leaves, capacity %lld", (long long)leaves_found, (long long)cap);
    return SRA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of sra_classify_and_split.
//
// Some callers cannot allocate device memory at all: code running inside a
// captured CUDA graph whose memory plan is fixed, real-time render or serving
// loops that forbid allocator calls (and their implicit synchronisation) on
// the hot path, and hosts that hand this library a pre-partitioned device
// with no allocator of their own. For them the scratch this round needs
// (per-node classes, per-block scan totals, the re-check list) lives in one
// file-scope __device__ array of fixed size instead of cudaMallocAsync memory.
//
// Limits and contract (also in include/sra.h):
//   - n_in <= SRA_NOALLOC_MAX_NODES (524288 nodes per call); larger inputs are
//     rejected with SRA_EINVAL before any device work is queued.
//   - The array is shared by every call in the process on a given device:
//     calls whose device work overlaps (two streams, or two host threads)
//     race on it and give undefined results. Serialise them.
//   - The array keeps the last call's contents; each call clears the one
//     field that must start at zero (the re-check counter) itself.
//   - The first call on each device resolves the array's device address with
//     cudaGetSymbolAddress (a host-side name of a __device__ variable is not a
//     device address). Make that first call before any stream capture.
//   - The array occupies SRA_NOALLOC_SCRATCH_BYTES of device memory on every
//     GPU that loads this library, until the process exits.
namespace {

constexpr size_t kNoallocCls = (size_t)SRA_NOALLOC_MAX_NODES;                  // uint8 per node
constexpr size_t kNoallocBlk = ((SRA_NOALLOC_MAX_NODES + 1023) / 1024) * 2 * 8; // scan totals
constexpr size_t kNoallocFlags = 16 + (size_t)SRA_NOALLOC_MAX_NODES * 4;       // count + list
static_assert(kNoallocCls + kNoallocBlk + kNoallocFlags <= SRA_NOALLOC_SCRATCH_BYTES,
              "scratch array too small for its node limit");

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[SRA_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64] = {nullptr};

// Device address of the scratch array on the current device (once per device).
sra_status noalloc_scratch(void **out) {
    int dev = 0;
    SRA_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(SRA_EUNSUPPORTED, "device ordinal %d", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(SRA_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return SRA_OK;
}

}  // namespace

extern "C" sra_status sra_classify_and_split_noalloc(
    const sra_net *n, const sra_opts *o, const float *root_lo, const float *root_hi,
    const sra_node *in, int64_t n_in, int32_t max_level, sra_node *out, int64_t cap_out,
    sra_node *leaves, int64_t cap_leaves, int64_t *counts, void *stream) {
    g_err.clear();
    sra_status r = check_net(n);
    if (r) return r;
    if ((r = check_opts(o))) return r;
    if (!root_lo || !root_hi || !counts) return fail(SRA_EINVAL, "null root/counts");
    for (int d = 0; d < 3; ++d)
        if (!(root_hi[d] > root_lo[d])) return fail(SRA_EINVAL, "empty root box on axis %d", d);
    const int lvl_cap = (o->split == SRA_SPLIT_OCTREE) ? 16 : kMaxKdLevels - 1;
    if (max_level < 0 || max_level > lvl_cap)
        return fail(SRA_EINVAL, "max_level %d outside [0, %d]", max_level, lvl_cap);
    if (n_in < 0 || cap_out < 0 || cap_leaves < 0) return fail(SRA_EINVAL, "negative size");
    if (n_in > SRA_NOALLOC_MAX_NODES)
        return fail(SRA_EINVAL, "n_in %lld exceeds the allocation-free limit of %d nodes per call",
                    (long long)n_in, SRA_NOALLOC_MAX_NODES);
    if (n_in > 0 && !in) return fail(SRA_EINVAL, "null frontier_in");
    if ((cap_out > 0 && !out) || (cap_leaves > 0 && !leaves)) return fail(SRA_EINVAL, "null output buffer");
    if (o->precision == SRA_PREC_BF16_SOUND || o->precision == SRA_PREC_BF16)
        return fail(SRA_EUNSUPPORTED, "the allocation-free round runs in FP32 or FP64");
    if (o->converge) return fail(SRA_EUNSUPPORTED, "the allocation-free round has no convergence test");
    if (o->arith == SRA_ARITH_AFFINE_FULL && 3 + n->new_syms > kKmaxList[sizeof kKmaxList / sizeof(int) - 1]) {
        FullCfg fc;
        if (n->pe || full_cfg(n->rows, 3 + n->new_syms, o->slope, o->precision == SRA_PREC_FP64 ? 8 : 4, &fc))
            return fail(SRA_EUNSUPPORTED, "the allocation-free round has no affine-full state in device memory");
    }
    void *scratch = nullptr;
    if ((r = noalloc_scratch(&scratch))) return r;  // before any early return for n_in == 0
    if (n_in == 0) return SRA_OK;
    cudaStream_t st = as_stream(stream);

    uint8_t *cls = (uint8_t *)scratch;
    long long *blk = (long long *)((char *)scratch + kNoallocCls);
    int *flag_count = (int *)((char *)scratch + kNoallocCls + kNoallocBlk);
    int *flag_list = (int *)((char *)scratch + kNoallocCls + kNoallocBlk + 16);

    BoxSrc src;
    memset(&src, 0, sizeof src);
    src.kind = SRC_NODES;
    src.nodes = in;
    src.n = n_in;
    src.split = o->split;
    unsigned char axis[kMaxKdLevels];
    kd_tables(root_lo, root_hi, src.kd_n3, axis);
    for (int d = 0; d < 3; ++d) {
        src.root_lo[d] = root_lo[d];
        src.root_ext[d] = root_hi[d] - root_lo[d];
    }
    const bool fp64 = o->precision == SRA_PREC_FP64;
    const bool recheck = o->recheck && !fp64;
    BoundOut bo;
    memset(&bo, 0, sizeof bo);
    bo.cls = cls;
    if (recheck) {
        bo.flag_count = flag_count;
        bo.flag_list = flag_list;
        bo.band = o->recheck_band;
        SRA_CK(cudaMemsetAsync(flag_count, 0, sizeof(int), st));  // must start at zero
    }
    if ((r = run_bound(n, o, fp64, 3, src, bo, n_in, st))) return r;
    if (recheck) {
        BoxSrc s2 = src;
        s2.list = flag_list;
        s2.list_count = flag_count;
        BoundOut o2 = bo;
        o2.flag_list = nullptr;
        o2.flag_count = nullptr;
        o2.recheck_counter = (unsigned long long *)(counts + SRA_CNT_RECHECKED);
        if ((r = run_bound(n, o, true, 3, s2, o2, n_in, st))) return r;
    }
    SplitArgs a;
    memset(&a, 0, sizeof a);
    a.cls = cls;
    a.in = in;
    a.n = n_in;
    a.max_level = max_level;
    a.split = o->split;
    memcpy(a.kd_axis, axis, sizeof axis);
    a.out = out;
    a.cap_out = cap_out;
    a.leaves = leaves;
    a.cap_leaves = cap_leaves;
    a.counts = (unsigned long long *)counts;
    a.blk = blk;
    cudaError_t e = launch_split(a, st);
    if (e != cudaSuccess) return fail(SRA_ECUDA, "split launch: %s", cudaGetErrorString(e));
    return SRA_OK;
}

extern "C" sra_status sra_sync_status(const sra_net *n, void *stream) {
    g_err.clear();
    sra_status r = check_net(n);
    if (r) return r;
    SRA_CK(cudaStreamSynchronize(as_stream(stream)));
    int *words[2] = {n->tc_ok ? n->tcp.status : nullptr, n->tcr_ok ? n->tcrp.status : nullptr};
    for (int *w : words) {
        if (!w) continue;
        int h = 0;
        SRA_CK(cudaMemcpy(&h, w, sizeof h, cudaMemcpyDeviceToHost));
        if (h != 0) {
            SRA_CK(cudaMemset(w, 0, sizeof(int)));
            if (h >= 100)  // debug builds only (SRA_DEBUG_BOUNDS)
                return fail(SRA_ECUDA, "a device index check of a tensor-core kernel failed (code %d)", h);
            return fail(SRA_ETIMEOUT, "a bounded wait of a tensor-core kernel ran out (code %d)", h);
        }
    }
    return SRA_OK;
}

extern "C" sra_status sra_test_tc_stall(int32_t spins) {
    g_err.clear();
    if (spins < 0 || spins > (1 << 20)) return fail(SRA_EINVAL, "spins %d outside [0, 2^20]", spins);
    g_test_tc_stall.store(spins);
    return SRA_OK;
}

extern "C" sra_status sra_test_math_f32(int32_t fn, const float *x, int64_t n, float *y, void *stream) {
    g_err.clear();
    if (fn < 0 || fn >= SRA_MATH_N) return fail(SRA_EINVAL, "math function %d outside [0, %d)", fn, SRA_MATH_N);
    if (n < 0) return fail(SRA_EINVAL, "n < 0");
    if (n == 0) return SRA_OK;
    if (!x || !y) return fail(SRA_EINVAL, "null x/y");
    cudaError_t e = launch_math_f32(fn, x, n, y, as_stream(stream));
    if (e != cudaSuccess) return fail(SRA_ECUDA, "math kernel launch: %s", cudaGetErrorString(e));
    return SRA_OK;
}

extern "C" sra_status sra_test_fail_allocs(int32_t n) {
    g_err.clear();
    if (n < 0) return fail(SRA_EINVAL, "n < 0");
    g_fail_allocs.store(n);
    return SRA_OK;
}
