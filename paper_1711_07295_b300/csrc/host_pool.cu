// host_pool.cu -- page-locked host blocks reused between calls.
//
// Pinning pages costs about as much time per byte as copying them over the
// link, so a pair list returned in page-locked memory goes back to this pool
// when it is freed and the next call with a result of similar size takes it
// again instead of asking the CUDA driver.  Blocks in use are never handed out; the
// pool keeps at most kMaxFree idle blocks and kMaxFreeBytes idle bytes and
// gives the oldest idle blocks back to the CUDA driver beyond that.
#include <mutex>
#include <unordered_map>
#include <vector>

#include "bmj_internal.cuh"

namespace bmj {
namespace {

constexpr size_t kGranule = size_t(2) << 20;        // block sizes are rounded up to 2 MiB
constexpr size_t kMaxFree = 8;                      // idle blocks kept
constexpr size_t kMaxFreeBytes = size_t(4) << 30;   // idle bytes kept

struct Block {
    void *ptr;
    size_t cap;
};

struct Pool {
    std::mutex mu;
    std::unordered_map<void *, size_t> live;  // handed out: base -> capacity
    std::vector<Block> idle;                  // oldest first
    size_t idle_bytes = 0;
};

// Never destroyed: at process exit the CUDA driver reclaims the pages, and a
// destructor running after the CUDA runtime has shut down must not free them.
Pool &pool() {
    static Pool *p = new Pool();
    return *p;
}

}  // namespace

void *pinned_alloc(size_t bytes) {
    if (bytes == 0) bytes = 1;
    Pool &P = pool();
    {
        std::lock_guard<std::mutex> g(P.mu);
        // smallest idle block that fits and wastes at most half of itself; among
        // equal ones the most recently returned (its pages are the warmest)
        int best = -1;
        for (size_t k = 0; k < P.idle.size(); k++) {
            const size_t c = P.idle[k].cap;
            if (c >= bytes && c / 2 <= bytes + kGranule &&
                (best < 0 || c <= P.idle[best].cap))
                best = (int)k;
        }
        if (best >= 0) {
            Block b = P.idle[best];
            P.idle.erase(P.idle.begin() + best);
            P.idle_bytes -= b.cap;
            P.live[b.ptr] = b.cap;
            return b.ptr;
        }
    }
    const size_t cap = (bytes + kGranule - 1) / kGranule * kGranule;
    void *p = nullptr;
    if (cudaMallocHost(&p, cap) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> g(P.mu);
    P.live[p] = cap;
    return p;
}

bool pinned_release(void *p) {
    if (!p) return false;
    Pool &P = pool();
    std::vector<void *> drop;
    {
        std::lock_guard<std::mutex> g(P.mu);
        auto it = P.live.find(p);
        if (it == P.live.end()) return false;
        P.idle.push_back(Block{p, it->second});
        P.idle_bytes += it->second;
        P.live.erase(it);
        while (P.idle.size() > kMaxFree || P.idle_bytes > kMaxFreeBytes) {
            drop.push_back(P.idle.front().ptr);
            P.idle_bytes -= P.idle.front().cap;
            P.idle.erase(P.idle.begin());
        }
    }
    for (void *d : drop) cudaFreeHost(d);
    return true;
}

}  // namespace bmj

extern "C" int64_t bmj_host_pool_trim(void) {
    bmj::Pool &P = bmj::pool();
    std::vector<bmj::Block> drop;
    {
        std::lock_guard<std::mutex> g(P.mu);
        drop.swap(P.idle);
        P.idle_bytes = 0;
    }
    int64_t bytes = 0;
    for (const auto &b : drop) {
        cudaFreeHost(b.ptr);
        bytes += (int64_t)b.cap;
    }
    return bytes;
}
