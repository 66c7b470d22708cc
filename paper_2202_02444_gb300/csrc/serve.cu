// Request loop for concurrent range-analysis queries (sra_serve): continuous
// batching over resident networks.
//
// One host thread drives a fixed set of slots, each owning a CUDA stream, an
// event and a pinned counter buffer. Requests become eligible at their
// arrival time and are admitted first come, first served when a slot is free
// and their device-memory reservation fits in an arena of fixed size (the
// frontier budget). An admitted request is a short state machine on its
// slot's stream: a ray tile or a box batch is one call of the entry point it
// uses; a leaf job (Proc. 3) is a sequence of sra_classify_and_split calls,
// each over a chunk of one level's frontier, with the chunk's counters copied
// to pinned memory behind an event. The loop polls the events; a finished
// step either ends the request or launches its next chunk, so the device
// always holds work of several requests at once and a long leaf job never
// blocks the others between its chunks.
//
// A leaf job walks its tree depth-first over chunks, so its frontier memory
// is fixed by its capacity and depth, whatever the size of the tree: one
// buffer of `cap` nodes per level. The next chunk always comes from the
// deepest level that still has unprocessed nodes, taken from the front of
// that level, at most cap / fanout nodes (fanout 8 for the octree, 2 for the
// k-d split), so its children fit the next level's buffer, which is empty at
// that point. Taking chunks from the front keeps the level-by-level order:
// the descendants of earlier nodes of a level come first at every deeper
// level, so the leaves come out in the order of a breadth-first build
// (sra_extract_leaves). The buffers live in the arena and stay on the device
// for the job's lifetime.
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <thread>
#include <vector>

#include "launch.h"

namespace sra {
namespace {

constexpr int kMaxServeDepth = 15;

// First-fit allocator over one device buffer; host-side bookkeeping only.
// Blocks are 256-byte aligned; freed blocks merge with free neighbours.
class Arena {
  public:
    void reset(size_t total) {
        free_.clear();
        if (total) free_[0] = total;
        total_ = total;
    }
    size_t total() const { return total_; }
    static size_t round(size_t b) { return ((b ? b : 1) + 255) & ~size_t(255); }
    bool take(size_t bytes, size_t *off) {
        bytes = round(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes, at = it->first + bytes;
            free_.erase(it);
            if (rest) free_[at] = rest;
            return true;
        }
        return false;
    }
    void give(size_t off, size_t bytes) {
        bytes = round(bytes);
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && off + bytes == nx->first) {  // merge with the next block
            bytes += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {  // merge with the previous block
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                pv->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }

  private:
    std::map<size_t, size_t> free_;  // offset -> size
    size_t total_ = 0;
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    int64_t *hcounts = nullptr;  // pinned, SRA_CNT_N entries
    int64_t req = -1;            // active request, -1 = free
    size_t off = 0, bytes = 0;   // arena reservation
    // leaf job state: one frontier buffer per level 0..depth, with the
    // level's node count and the read position of its next chunk
    sra_node *levels = nullptr;
    size_t level_bytes = 0;
    int level = 0;        // level of the chunk in flight
    int64_t chunk = 0;    // nodes in the chunk in flight
    int64_t n[kMaxServeDepth + 1] = {}, next[kMaxServeDepth + 1] = {};
    int deepest = 0;      // deepest level reached
    int64_t leaves_found = 0;
    int64_t *dcounts = nullptr;
    sra_node *buf(int l) const { return (sra_node *)((char *)levels + (size_t)l * level_bytes); }
};

size_t level_buffer_bytes(const sra_request &q) {
    return Arena::round((size_t)(q.cap > 0 ? q.cap : 1) * sizeof(sra_node));
}

size_t reservation(const sra_request &q) {
    if (q.kind == SRA_REQ_LEAVES) return (size_t)(q.depth + 1) * level_buffer_bytes(q) + 256;
    return (size_t)(q.n > 0 ? q.n : 1) * 16;
}

const float kRootLo[3] = {-1.f, -1.f, -1.f}, kRootHi[3] = {1.f, 1.f, 1.f};

}  // namespace
}  // namespace sra

using namespace sra;

extern "C" sra_status sra_serve(const sra_net *const *nets, int32_t n_nets, const sra_opts *forms,
                                int32_t n_forms, const sra_serve_cfg *cfg, sra_request *reqs,
                                int64_t n_req) {
    if (!nets || n_nets < 1 || !forms || n_forms < 1 || !cfg || (n_req > 0 && !reqs) || n_req < 0)
        return set_error(SRA_EINVAL, "sra_serve: null or empty nets / forms / cfg / requests");
    if (cfg->slots < 1 || cfg->slots > 64) return set_error(SRA_EINVAL, "slots %d outside [1, 64]", cfg->slots);
    if (cfg->frontier_bytes < 0) return set_error(SRA_EINVAL, "frontier_bytes < 0");
    for (int32_t k = 0; k < n_nets; ++k)
        if (!nets[k]) return set_error(SRA_EINVAL, "nets[%d] is NULL", k);
    for (int64_t i = 0; i < n_req; ++i) {
        const sra_request &q = reqs[i];
        if (q.net < 0 || q.net >= n_nets || q.form < 0 || q.form >= n_forms)
            return set_error(SRA_EINVAL, "request %lld: net %d / form %d out of range", (long long)i, q.net, q.form);
        if (q.kind < SRA_REQ_RAYS || q.kind > SRA_REQ_LEAVES)
            return set_error(SRA_EINVAL, "request %lld: kind %d", (long long)i, q.kind);
        if (i > 0 && q.arrival < reqs[i - 1].arrival)
            return set_error(SRA_EINVAL, "request %lld arrives before request %lld", (long long)i, (long long)i - 1);
        if (q.kind == SRA_REQ_LEAVES && (q.depth < 0 || q.depth > kMaxServeDepth || q.cap < 1 || !q.leaves))
            return set_error(SRA_EINVAL, "request %lld: leaf job needs 0 <= depth <= 15, cap >= 1, leaves", (long long)i);
    }
    for (int64_t i = 0; i < n_req; ++i) {
        reqs[i].status = -1;
        reqs[i].slot = -1;
        reqs[i].levels = 0;
        reqs[i].n_out = 0;
        reqs[i].t_admit = reqs[i].t_done = -1.0;
    }

    // ---- resources of the loop ------------------------------------------------
    std::vector<Slot> slots(cfg->slots);
    void *arena_mem = nullptr;
    Arena arena;
    sra_status result = SRA_OK;
    auto release_all = [&]() {
        for (Slot &s : slots) {
            if (s.st) cudaStreamSynchronize(s.st);
        }
        for (Slot &s : slots) {
            if (s.ev) cudaEventDestroy(s.ev);
            if (s.st) cudaStreamDestroy(s.st);
            if (s.hcounts) cudaFreeHost(s.hcounts);
        }
        if (arena_mem) cudaFree(arena_mem);
    };
    if (cfg->frontier_bytes > 0) {
        cudaError_t e = cudaMalloc(&arena_mem, (size_t)cfg->frontier_bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(SRA_ENOMEM, "frontier arena of %lld bytes: %s", (long long)cfg->frontier_bytes,
                             cudaGetErrorString(e));
        }
    }
    arena.reset((size_t)cfg->frontier_bytes);
    for (Slot &s : slots) {
        if (cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost((void **)&s.hcounts, SRA_CNT_N * sizeof(int64_t)) != cudaSuccess) {
            cudaGetLastError();
            release_all();
            return set_error(SRA_ECUDA, "slot streams / events / pinned counters");
        }
    }

    const auto t0 = std::chrono::steady_clock::now();
    auto elapsed = [&]() {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    };
    int64_t ended = 0;
    auto finish = [&](Slot &s, sra_status st) {
        sra_request &q = reqs[s.req];
        q.status = st;
        q.t_done = elapsed();
        arena.give(s.off, s.bytes);
        s.req = -1;
        ++ended;
    };
    // Enqueue the next chunk of a leaf job (from the front of level s.level):
    // classify and split it into the (empty) buffer of the next level, copy
    // the chunk's counters to pinned memory, record the event.
    auto launch_chunk = [&](Slot &s) -> sra_status {
        const sra_request &q = reqs[s.req];
        const sra_opts &o = forms[q.form];
        const int64_t fan = o.split == SRA_SPLIT_OCTREE ? 8 : 2;
        const int l = s.level;
        const int64_t room = q.cap / fan > 0 ? q.cap / fan : 1;
        s.chunk = s.n[l] - s.next[l] < room ? s.n[l] - s.next[l] : room;
        if (cudaMemsetAsync(s.dcounts, 0, SRA_CNT_N * sizeof(int64_t), s.st) != cudaSuccess)
            return SRA_ECUDA;
        const int64_t lcap = q.cap > s.leaves_found ? q.cap - s.leaves_found : 0;
        const bool last = l == q.depth;
        sra_status r = sra_classify_and_split(nets[q.net], &o, kRootLo, kRootHi, s.buf(l) + s.next[l], s.chunk,
                                              q.depth, last ? nullptr : s.buf(l + 1), last ? 0 : q.cap,
                                              lcap > 0 ? q.leaves + s.leaves_found : nullptr, lcap, s.dcounts, s.st);
        if (r) return r;
        if (cudaMemcpyAsync(s.hcounts, s.dcounts, SRA_CNT_N * sizeof(int64_t), cudaMemcpyDeviceToHost, s.st) !=
                cudaSuccess ||
            cudaEventRecord(s.ev, s.st) != cudaSuccess)
            return SRA_ECUDA;
        return SRA_OK;
    };
    auto start = [&](Slot &s, int64_t qi, size_t off, size_t bytes) {
        sra_request &q = reqs[qi];
        s.req = qi;
        s.off = off;
        s.bytes = bytes;
        q.slot = (int32_t)(&s - slots.data());
        q.t_admit = elapsed();
        sra_status r = SRA_OK;
        const sra_net *net = nets[q.net];
        const sra_opts *o = &forms[q.form];
        if (q.kind == SRA_REQ_RAYS) {
            r = sra_cast_rays(net, o, q.a, q.b, q.n, q.lo, q.iters, s.st);
        } else if (q.kind == SRA_REQ_BOXES) {
            r = sra_bound_boxes(net, o, q.a, q.b, q.n, q.lo, q.hi, q.cls, s.st);
        } else {
            s.levels = (sra_node *)((char *)arena_mem + off);
            s.level_bytes = level_buffer_bytes(q);
            s.dcounts = (int64_t *)((char *)arena_mem + off + (size_t)(q.depth + 1) * s.level_bytes);
            for (int l = 0; l <= kMaxServeDepth; ++l) s.n[l] = s.next[l] = 0;
            s.level = s.deepest = 0;
            s.n[0] = 1;
            s.leaves_found = 0;
            // the root node (level 0, index 0) is all zero bytes
            r = cudaMemsetAsync(s.buf(0), 0, sizeof(sra_node), s.st) == cudaSuccess ? SRA_OK : SRA_ECUDA;
            if (!r) r = launch_chunk(s);
        }
        if (!r && q.kind != SRA_REQ_LEAVES && cudaEventRecord(s.ev, s.st) != cudaSuccess) r = SRA_ECUDA;
        if (r) finish(s, r);
    };
    // A finished step: end the request or launch the leaf job's next chunk.
    auto advance = [&](Slot &s) {
        sra_request &q = reqs[s.req];
        if (q.kind != SRA_REQ_LEAVES) {
            finish(s, SRA_OK);
            return;
        }
        const int64_t *hc = s.hcounts;
        const int l = s.level;
        s.next[l] += s.chunk;
        s.leaves_found += hc[SRA_CNT_LEAVES];
        if (s.leaves_found > q.cap) {  // the leaves do not fit: stop (n_out is a lower bound)
            q.n_out = s.leaves_found;
            finish(s, SRA_ECAPACITY);
            return;
        }
        if (l < q.depth) {
            const int64_t children = hc[SRA_CNT_CHILDREN];
            if (children > q.cap) {  // only when cap < fanout: one node's children do not fit
                q.n_out = children;
                finish(s, SRA_ECAPACITY);
                return;
            }
            s.n[l + 1] = children;
            s.next[l + 1] = 0;
            if (children > 0 && l + 1 > s.deepest) s.deepest = l + 1;
        }
        q.levels = s.deepest + 1;
        // the deepest level with unprocessed nodes
        int d = l < q.depth ? l + 1 : l;
        while (d >= 0 && s.next[d] >= s.n[d]) --d;
        if (d < 0) {
            q.n_out = s.leaves_found;
            finish(s, SRA_OK);
            return;
        }
        s.level = d;
        sra_status r = launch_chunk(s);
        if (r) finish(s, r);
    };

    std::deque<int64_t> queue;
    int64_t next = 0;
    while (ended < n_req) {
        const double now = elapsed();
        while (next < n_req && (!cfg->realtime || reqs[next].arrival <= now)) queue.push_back(next++);
        bool progressed = false;
        // admission: first come, first served
        while (!queue.empty()) {
            const int64_t qi = queue.front();
            const size_t need = reservation(reqs[qi]);
            if (need > arena.total()) {  // can never fit
                reqs[qi].t_admit = reqs[qi].t_done = elapsed();
                reqs[qi].status = SRA_ENOMEM;
                queue.pop_front();
                ++ended;
                progressed = true;
                continue;
            }
            Slot *free_slot = nullptr;
            for (Slot &s : slots)
                if (s.req < 0) { free_slot = &s; break; }
            if (!free_slot) break;
            size_t off = 0;
            if (!arena.take(need, &off)) break;  // wait until admitted work frees memory
            queue.pop_front();
            start(*free_slot, qi, off, need);
            progressed = true;
        }
        // progress of admitted requests
        for (Slot &s : slots) {
            if (s.req < 0) continue;
            const cudaError_t e = cudaEventQuery(s.ev);
            if (e == cudaSuccess) {
                advance(s);
                progressed = true;
            } else if (e != cudaErrorNotReady) {
                cudaGetLastError();
                finish(s, SRA_ECUDA);
                result = set_error(SRA_ECUDA, "request %lld: %s", (long long)s.req, cudaGetErrorString(e));
                progressed = true;
            }
        }
        if (!progressed) {
            bool idle = queue.empty();
            for (const Slot &s : slots) idle = idle && s.req < 0;
            if (idle && next < n_req && cfg->realtime) {
                const double wait = reqs[next].arrival - elapsed();
                if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(wait < 1e-3 ? wait : 1e-3));
            } else {
                std::this_thread::sleep_for(std::chrono::microseconds(20));
            }
        }
    }
    release_all();
    return result;
}
