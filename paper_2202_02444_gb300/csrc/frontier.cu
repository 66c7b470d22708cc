// Frontier stream compaction and octree / k-d split: one batched round of
// Proc. 3 (BuildSpatialTree); Sec. 4.5 builds the tree breadth-first in such
// rounds instead of recursing.
//
// Deterministic: children and leaves are written in input order through a
// two-level exclusive scan (per-block totals, one-block scan of the totals,
// per-block local scan + scatter), appended after the positions already held
// in counts[CHILDREN] / counts[LEAVES]. HBM-bound: per node it reads 9 bytes
// (record + class) and writes 8 bytes per emitted record.
#include "launch.h"

namespace sra {

constexpr int kSplitBlock = 1024;

long long split_blocks(long long n) { return (n + kSplitBlock - 1) / kSplitBlock; }

__device__ __forceinline__ void emit_counts(const SplitArgs &a, long long i, int &ch, int &lf,
                                            int &pos, int &neg, int &unk) {
    ch = lf = pos = neg = unk = 0;
    if (i >= a.n) return;
    const int k = a.cls[i];
    if (k == SRA_POSITIVE) pos = 1;
    else if (k == SRA_NEGATIVE) neg = 1;
    else {
        unk = 1;
        // a node of the convergence test is a leaf at any level
        if (k != kClsConverged && (int)a.in[i].level < a.max_level) ch = (a.split == SRA_SPLIT_OCTREE) ? 8 : 2;
        else lf = 1;
    }
}

template <typename V> __device__ __forceinline__ V warp_incl_scan(V v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        V t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Block-wide exclusive scan of two ints (1024 threads); returns totals.
__device__ __forceinline__ void block_scan2(int a, int b, int &ea, int &eb, int &ta, int &tb) {
    __shared__ int wa[32], wb[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int ia = warp_incl_scan(a, lane), ib = warp_incl_scan(b, lane);
    if (lane == 31) { wa[w] = ia; wb[w] = ib; }
    __syncthreads();
    if (w == 0) {
        int x = wa[lane], y = wb[lane];
        int sx = warp_incl_scan(x, lane), sy = warp_incl_scan(y, lane);
        wa[lane] = sx - x;
        wb[lane] = sy - y;
        ta = __shfl_sync(0xffffffffu, sx, 31);
        tb = __shfl_sync(0xffffffffu, sy, 31);
    }
    __syncthreads();
    ea = wa[w] + ia - a;
    eb = wb[w] + ib - b;
    __shared__ int tot[2];
    if (threadIdx.x == 0) { tot[0] = ta; tot[1] = tb; }
    __syncthreads();
    ta = tot[0];
    tb = tot[1];
}

__global__ void __launch_bounds__(kSplitBlock) split_count_kernel(SplitArgs a) {
    const long long i = (long long)blockIdx.x * kSplitBlock + threadIdx.x;
    int ch, lf, pos, neg, unk;
    emit_counts(a, i, ch, lf, pos, neg, unk);
    int ea, eb, ta = 0, tb = 0;
    block_scan2(ch, lf, ea, eb, ta, tb);
    // per-class tallies (sums; order does not matter)
    const int lane = threadIdx.x & 31;
    int p = pos, q = neg, u = unk, cv = (i < a.n && a.cls[i] == kClsConverged) ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        p += __shfl_xor_sync(0xffffffffu, p, o);
        q += __shfl_xor_sync(0xffffffffu, q, o);
        u += __shfl_xor_sync(0xffffffffu, u, o);
        cv += __shfl_xor_sync(0xffffffffu, cv, o);
    }
    if (lane == 0) {
        if (p) atomicAdd(&a.counts[SRA_CNT_POSITIVE], (unsigned long long)p);
        if (q) atomicAdd(&a.counts[SRA_CNT_NEGATIVE], (unsigned long long)q);
        if (u) atomicAdd(&a.counts[SRA_CNT_UNKNOWN], (unsigned long long)u);
        if (cv) atomicAdd(&a.counts[SRA_CNT_CONVERGED], (unsigned long long)cv);
    }
    if (threadIdx.x == 0) {
        a.blk[2 * blockIdx.x] = ta;
        a.blk[2 * blockIdx.x + 1] = tb;
    }
}

// One block: exclusive scan of the per-block totals, offset by the counts
// already present; then advance the counts by the totals.
__global__ void __launch_bounds__(kSplitBlock) split_scan_kernel(SplitArgs a, long long nblk) {
    __shared__ long long carry[2];
    __shared__ long long ws[2][32];
    if (threadIdx.x == 0) {
        carry[0] = (long long)a.counts[SRA_CNT_CHILDREN];
        carry[1] = (long long)a.counts[SRA_CNT_LEAVES];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (long long b0 = 0; b0 < nblk; b0 += kSplitBlock) {
        const long long b = b0 + threadIdx.x;
        long long x = (b < nblk) ? a.blk[2 * b] : 0, y = (b < nblk) ? a.blk[2 * b + 1] : 0;
        long long ix = warp_incl_scan(x, lane), iy = warp_incl_scan(y, lane);
        if (lane == 31) { ws[0][w] = ix; ws[1][w] = iy; }
        __syncthreads();
        if (w == 0) {
            long long u = ws[0][lane], v = ws[1][lane];
            long long su = warp_incl_scan(u, lane), sv = warp_incl_scan(v, lane);
            ws[0][lane] = su - u;
            ws[1][lane] = sv - v;
        }
        __syncthreads();
        const long long ex = carry[0] + ws[0][w] + ix - x, ey = carry[1] + ws[1][w] + iy - y;
        if (b < nblk) { a.blk[2 * b] = ex; a.blk[2 * b + 1] = ey; }
        __syncthreads();
        if (threadIdx.x == kSplitBlock - 1) { carry[0] = ex + x; carry[1] = ey + y; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.counts[SRA_CNT_CHILDREN] = (unsigned long long)carry[0];
        a.counts[SRA_CNT_LEAVES] = (unsigned long long)carry[1];
    }
}

__global__ void __launch_bounds__(kSplitBlock) split_scatter_kernel(SplitArgs a) {
    const long long i = (long long)blockIdx.x * kSplitBlock + threadIdx.x;
    int ch, lf, pos, neg, unk;
    emit_counts(a, i, ch, lf, pos, neg, unk);
    int ea, eb, ta, tb;
    block_scan2(ch, lf, ea, eb, ta, tb);
    if (i >= a.n) return;
    const long long base_c = a.blk[2 * blockIdx.x] + ea, base_l = a.blk[2 * blockIdx.x + 1] + eb;
    const sra_node nd = a.in[i];
    if (ch) {
        if (a.split == SRA_SPLIT_OCTREE) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const long long p = base_c + q;
                if (p < a.cap_out) {
                    sra_node c;
                    c.ix = (uint16_t)(2 * nd.ix + (q & 1));
                    c.iy = (uint16_t)(2 * nd.iy + ((q >> 1) & 1));
                    c.iz = (uint16_t)(2 * nd.iz + ((q >> 2) & 1));
                    c.level = (uint16_t)(nd.level + 1);
                    a.out[p] = c;
                }
            }
        } else {
            const int ax = a.kd_axis[nd.level < kMaxKdLevels ? nd.level : kMaxKdLevels - 1];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const long long p = base_c + q;
                if (p < a.cap_out) {
                    sra_node c = nd;
                    if (ax == 0) c.ix = (uint16_t)(2 * nd.ix + q);
                    if (ax == 1) c.iy = (uint16_t)(2 * nd.iy + q);
                    if (ax == 2) c.iz = (uint16_t)(2 * nd.iz + q);
                    c.level = (uint16_t)(nd.level + 1);
                    a.out[p] = c;
                }
            }
        }
    }
    if (lf && base_l < a.cap_leaves) a.leaves[base_l] = nd;
}

// ---- segmented split: the frontiers of many networks in one round ----------
// Segment s owns the split blocks [blk0, blk0 + ceil(n / kSplitBlock)), so no
// block straddles two segments; each segment scans and scatters into its own
// output ranges and counters exactly as a lone round would.
__device__ __forceinline__ int seg_of_block(const BatchSplitSeg *segs, int nseg, long long b) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segs[mid].blk0 <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void emit_counts_seg(const BatchSplitSeg &S, const uint8_t *cls, const sra_node *in,
                                                long long j, int &ch, int &lf, int &pos, int &neg, int &unk) {
    ch = lf = pos = neg = unk = 0;
    if (j >= S.n) return;
    const int k = cls[S.first + j];
    if (k == SRA_POSITIVE) pos = 1;
    else if (k == SRA_NEGATIVE) neg = 1;
    else {
        unk = 1;
        if ((int)in[S.first + j].level < S.max_level) ch = (S.split == SRA_SPLIT_OCTREE) ? 8 : 2;
        else lf = 1;
    }
}

__global__ void __launch_bounds__(kSplitBlock)
split_count_batch(const uint8_t *cls, const sra_node *in, const BatchSplitSeg *segs, int nseg,
                  unsigned long long *counts, long long *blk) {
    const long long b = blockIdx.x;
    const int s = seg_of_block(segs, nseg, b);
    const BatchSplitSeg &S = segs[s];
    const long long j = (b - S.blk0) * kSplitBlock + threadIdx.x;
    int ch, lf, pos, neg, unk;
    emit_counts_seg(S, cls, in, j, ch, lf, pos, neg, unk);
    int ea, eb, ta = 0, tb = 0;
    block_scan2(ch, lf, ea, eb, ta, tb);
    const int lane = threadIdx.x & 31;
    int p = pos, q = neg, u = unk;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        p += __shfl_xor_sync(0xffffffffu, p, o);
        q += __shfl_xor_sync(0xffffffffu, q, o);
        u += __shfl_xor_sync(0xffffffffu, u, o);
    }
    unsigned long long *c = counts + (size_t)s * SRA_CNT_N;
    if (lane == 0) {
        if (p) atomicAdd(&c[SRA_CNT_POSITIVE], (unsigned long long)p);
        if (q) atomicAdd(&c[SRA_CNT_NEGATIVE], (unsigned long long)q);
        if (u) atomicAdd(&c[SRA_CNT_UNKNOWN], (unsigned long long)u);
    }
    if (threadIdx.x == 0) {
        blk[2 * b] = ta;
        blk[2 * b + 1] = tb;
    }
}

// One block per segment: exclusive scan of its block totals after the
// positions already counted, then advance its counters.
__global__ void __launch_bounds__(kSplitBlock)
split_scan_batch(const BatchSplitSeg *segs, unsigned long long *counts, long long *blk) {
    __shared__ long long carry[2];
    __shared__ long long ws[2][32];
    const BatchSplitSeg &S = segs[blockIdx.x];
    unsigned long long *c = counts + (size_t)blockIdx.x * SRA_CNT_N;
    const long long nb = (S.n + kSplitBlock - 1) / kSplitBlock;
    if (threadIdx.x == 0) {
        carry[0] = (long long)c[SRA_CNT_CHILDREN];
        carry[1] = (long long)c[SRA_CNT_LEAVES];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (long long b0 = 0; b0 < nb; b0 += kSplitBlock) {
        const long long bl = b0 + threadIdx.x, b = S.blk0 + bl;
        long long x = (bl < nb) ? blk[2 * b] : 0, y = (bl < nb) ? blk[2 * b + 1] : 0;
        long long ix = warp_incl_scan(x, lane), iy = warp_incl_scan(y, lane);
        if (lane == 31) { ws[0][w] = ix; ws[1][w] = iy; }
        __syncthreads();
        if (w == 0) {
            long long u = ws[0][lane], v = ws[1][lane];
            long long su = warp_incl_scan(u, lane), sv = warp_incl_scan(v, lane);
            ws[0][lane] = su - u;
            ws[1][lane] = sv - v;
        }
        __syncthreads();
        const long long ex = carry[0] + ws[0][w] + ix - x, ey = carry[1] + ws[1][w] + iy - y;
        if (bl < nb) { blk[2 * b] = ex; blk[2 * b + 1] = ey; }
        __syncthreads();
        if (threadIdx.x == kSplitBlock - 1) { carry[0] = ex + x; carry[1] = ey + y; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        c[SRA_CNT_CHILDREN] = (unsigned long long)carry[0];
        c[SRA_CNT_LEAVES] = (unsigned long long)carry[1];
    }
}

__global__ void __launch_bounds__(kSplitBlock)
split_scatter_batch(const uint8_t *cls, const sra_node *in, const BatchSplitSeg *segs, int nseg,
                    sra_node *out, sra_node *leaves, const long long *blk) {
    const long long b = blockIdx.x;
    const int s = seg_of_block(segs, nseg, b);
    const BatchSplitSeg &S = segs[s];
    const long long j = (b - S.blk0) * kSplitBlock + threadIdx.x;
    int ch, lf, pos, neg, unk;
    emit_counts_seg(S, cls, in, j, ch, lf, pos, neg, unk);
    int ea, eb, ta, tb;
    block_scan2(ch, lf, ea, eb, ta, tb);
    if (j >= S.n) return;
    const long long base_c = blk[2 * b] + ea, base_l = blk[2 * b + 1] + eb;
    const sra_node nd = in[S.first + j];
    if (ch) {
        const int ax = (S.split == SRA_SPLIT_OCTREE)
                           ? -1 : S.kd_axis[nd.level < kMaxKdLevels ? nd.level : kMaxKdLevels - 1];
        for (int q = 0; q < ch; ++q) {
            const long long p = base_c + q;
            if (p >= S.cap_out) break;
            sra_node c = nd;
            if (ax < 0) {
                c.ix = (uint16_t)(2 * nd.ix + (q & 1));
                c.iy = (uint16_t)(2 * nd.iy + ((q >> 1) & 1));
                c.iz = (uint16_t)(2 * nd.iz + ((q >> 2) & 1));
            } else {
                if (ax == 0) c.ix = (uint16_t)(2 * nd.ix + q);
                if (ax == 1) c.iy = (uint16_t)(2 * nd.iy + q);
                if (ax == 2) c.iz = (uint16_t)(2 * nd.iz + q);
            }
            c.level = (uint16_t)(nd.level + 1);
            out[S.out_first + p] = c;
        }
    }
    if (lf && base_l < S.cap_leaves) leaves[S.leaf_first + base_l] = nd;
}

cudaError_t launch_split_batch(const uint8_t *cls, const sra_node *in, const BatchSplitSeg *segs, int nseg,
                               long long nblk, sra_node *out, sra_node *leaves, unsigned long long *counts,
                               long long *blk, cudaStream_t st) {
    if (nblk == 0 || nseg == 0) return cudaSuccess;
    split_count_batch<<<(unsigned)nblk, kSplitBlock, 0, st>>>(cls, in, segs, nseg, counts, blk);
    split_scan_batch<<<(unsigned)nseg, kSplitBlock, 0, st>>>(segs, counts, blk);
    split_scatter_batch<<<(unsigned)nblk, kSplitBlock, 0, st>>>(cls, in, segs, nseg, out, leaves, blk);
    return cudaGetLastError();
}

cudaError_t launch_split(const SplitArgs &a, cudaStream_t st) {
    const long long nblk = split_blocks(a.n);
    if (nblk == 0) return cudaSuccess;
    split_count_kernel<<<(unsigned)nblk, kSplitBlock, 0, st>>>(a);
    split_scan_kernel<<<1, kSplitBlock, 0, st>>>(a, nblk);
    split_scatter_kernel<<<(unsigned)nblk, kSplitBlock, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace sra
