// serve.cu -- a resident index and probe queries with continuous batching.
//
// bmj_index_create keeps one collection resident on the device in size order
// (sizes, sorted CSR, bitmaps).  A probe set x with threshold p/q is an
// RS-join with |R| = 1 (Eq. 1): its candidates are the resident sets inside
// both sides of the length window (Table 2: ceil(p|x|/q) <= |s| <= floor(q|x|/p)),
// filtered by the Eq. 2 bound and verified exactly.
//
// A batch of probes runs as:
//   probe bitmaps + windows -> work items (probe, column chunk) -> filter ->
//   verification -> sort by (probe, id) -> per-probe id lists.
// The counters and the first 2048 result keys come back together; a batch
// with no more results than that is sorted on the host (one round trip), a
// larger one is radix-sorted on the device in a second phase.
// Every batch has its own slot (stream, pinned staging, fixed device buffers),
// so several batches are in flight at once and overlap on the device.
//
// bmj_serve runs an arrival stream through the slots: queries that have
// arrived are admitted into a free slot while the batch's exact window-pair
// count (from a host histogram of resident sizes) fits the slot's buffers,
// which bounds every buffer of the batch (survivors and results cannot
// exceed window pairs).  Latency of a query = completion - arrival.
//
// bmj_serve_open / _submit / _poll / _close run the same slots live: a
// server owns a host thread that admits the queries submitted so far (from
// any thread, while other batches are on the device) into free slots by the
// same window-pair budget, completes batches as their events fire and files
// every result under its ticket until it is polled.  Latency of a query =
// completion - submission.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "filter_core.cuh"
#include "host_util.cuh"

struct bmj_index {
    int device = 0;
    int b = 64, W = 1, method = BMJ_XOR, sim = BMJ_JACCARD;
    int64_t n = 0;
    int max_size = 0;
    uint32_t *ssz = nullptr;  // n + 4
    uint32_t *perm = nullptr;
    int64_t *soff = nullptr;  // n + 1
    int32_t *stok = nullptr;
    uint64_t *bm = nullptr;   // (n + 4) * W
    std::vector<int64_t> size_cum;  // size_cum[s] = resident sets with size < s
    int64_t *d_size_cum = nullptr;  // the same on the device (max_size + 2 entries)
    int sticky = 0;  // a CUDA runtime or timeout failure of an earlier call (then every call fails)
};

namespace bmj {
namespace {

constexpr unsigned kFullQ = 0xffffffffu;
// Columns per work item of the query filter: kQueryChunk, halved down to
// kQueryChunkMin while a batch has fewer items than the GPU has warp slots
// (a single probe's window then spreads over many warps).
constexpr int kQueryChunk = 1024;
constexpr int kQueryChunkMin = 64;
// Result keys copied back with a batch's counters (16 KB).
constexpr int64_t kEagerKeys = 2048;

// First resident position with a size >= v: size_cum[v] = the resident sets
// of size below v (max_size + 2 entries, the last equal to n).
__device__ __forceinline__ int64_t lb_sizes(const int64_t *size_cum, int max_size, int64_t n,
                                            uint64_t v) {
    return v > (uint64_t)max_size ? n : size_cum[v];
}

// Per probe x: its window [lo, hi) of resident sorted positions (Table 2, both
// bounds) and its number of column chunks.
__device__ __forceinline__ int64_t probe_window(const int64_t *poff, const uint32_t *pp,
                                                const uint32_t *pq, const int64_t *size_cum,
                                                int max_size, int64_t n, int sim, int chunk,
                                                int64_t x, int64_t *lo, int64_t *hi) {
    const uint64_t sx = (uint64_t)(poff[x + 1] - poff[x]);
    const SimWindow w = sim_window(sim, pp[x], pq[x]);
    const uint64_t low = window_low(sx, w);     // e.g. Jaccard: ceil(p|x|/q)
    const uint64_t high = window_high(sx, w);   // e.g. Jaccard: floor(q|x|/p); ~0: none
    *lo = lb_sizes(size_cum, max_size, n, low);
    *hi = high == ~0ull ? n : lb_sizes(size_cum, max_size, n, high + 1);
    return *hi > *lo ? (*hi - *lo + chunk - 1) / chunk : 0;
}

// Per probe: its window and its number of column chunks (items[x]).
__global__ void k_probe_windows(const int64_t *__restrict__ poff, int64_t nq,
                                const uint32_t *__restrict__ pp, const uint32_t *__restrict__ pq,
                                const int64_t *__restrict__ size_cum, int max_size, int64_t n,
                                int64_t *__restrict__ wlo, int64_t *__restrict__ whi,
                                int64_t *__restrict__ items, int sim, int chunk) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nq; x += stride)
        items[x] = probe_window(poff, pp, pq, size_cum, max_size, n, sim, chunk, x, &wlo[x],
                                &whi[x]);
}

// The same for a batch of at most kScanProbes probes in one block, with the
// exclusive scan of the chunk counts (items[nq] = their total) done in place.
// With bw > 0 (b = 64 bw, a power of two up to 256; Xor or Set; at most
// kFuseProbes probes) warp w also writes probe w's bitmap (Alg. 3b / 3a,
// h(t) = t mod b), which saves the bitmap launch for small batches.
constexpr int kScanProbes = 1024;
constexpr int kFuseProbes = 16;
// window pairs of a small batch up to which its survivors are verified in the
// filter's lanes (about two probes of the typical size against 2,000,000 sets)
constexpr int64_t kInlineVerifyWindow = int64_t(1) << 22;
static_assert(kFuseProbes <= kScanProbes / 32, "a warp per fused probe");
__global__ void __launch_bounds__(kScanProbes)
    k_probe_windows_scan(const int64_t *__restrict__ poff, int64_t nq,
                         const uint32_t *__restrict__ pp, const uint32_t *__restrict__ pq,
                         const int64_t *__restrict__ size_cum, int max_size, int64_t n,
                         int64_t *__restrict__ wlo, int64_t *__restrict__ whi,
                         int64_t *__restrict__ items, int sim, int chunk,
                         unsigned long long *__restrict__ ctr, const int32_t *__restrict__ ptok,
                         uint64_t *__restrict__ pbm, int bw, int xor_method) {
    __shared__ int64_t warp_sum[kScanProbes / 32];
    const int x = threadIdx.x, lane = x & 31, w = x >> 5;
    if (x < 2) ctr[x] = 0;  // the batch's survivor and result counters
    if (bw > 0 && w < nq) {  // warp w builds probe w's bitmap (nq <= kFuseProbes < 32 warps)
        uint64_t m0 = 0, m1 = 0, m2 = 0, m3 = 0;
        const uint32_t hmask = 64u * (uint32_t)bw - 1u;
        for (int64_t k = poff[w] + lane; k < poff[w + 1]; k += 32) {
            const uint32_t h = (uint32_t)ptok[k] & hmask;
            const uint64_t bit = 1ull << (h & 63);
            const uint32_t word = h >> 6;
            if (xor_method) {
                m0 ^= word == 0 ? bit : 0ull;
                m1 ^= word == 1 ? bit : 0ull;
                m2 ^= word == 2 ? bit : 0ull;
                m3 ^= word == 3 ? bit : 0ull;
            } else {
                m0 |= word == 0 ? bit : 0ull;
                m1 |= word == 1 ? bit : 0ull;
                m2 |= word == 2 ? bit : 0ull;
                m3 |= word == 3 ? bit : 0ull;
            }
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {  // Xor (Alg. 3b) and Or (Alg. 3a) are associative
            const uint64_t o0 = __shfl_xor_sync(0xffffffffu, m0, d);
            const uint64_t o1 = __shfl_xor_sync(0xffffffffu, m1, d);
            const uint64_t o2 = __shfl_xor_sync(0xffffffffu, m2, d);
            const uint64_t o3 = __shfl_xor_sync(0xffffffffu, m3, d);
            if (xor_method) {
                m0 ^= o0; m1 ^= o1; m2 ^= o2; m3 ^= o3;
            } else {
                m0 |= o0; m1 |= o1; m2 |= o2; m3 |= o3;
            }
        }
        if (lane == 0) {
            uint64_t *dst = pbm + (int64_t)w * bw;
            dst[0] = m0;
            if (bw > 1) dst[1] = m1;
            if (bw > 2) {
                dst[2] = m2;
                dst[3] = m3;
            }
        }
    }
    int64_t c = 0;
    if (x < nq)
        c = probe_window(poff, pp, pq, size_cum, max_size, n, sim, chunk, x, &wlo[x], &whi[x]);
    int64_t incl = c;  // inclusive scan within the warp
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t v = __shfl_up_sync(kFullQ, incl, d);
        if (lane >= d) incl += v;
    }
    if (lane == 31) warp_sum[w] = incl;
    __syncthreads();
    if (w == 0) {  // scan of the warp totals
        int64_t t = lane < kScanProbes / 32 ? warp_sum[lane] : 0;
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t v = __shfl_up_sync(kFullQ, t, d);
            if (lane >= d) t += v;
        }
        warp_sum[lane] = t;  // inclusive totals up to warp `lane`
    }
    __syncthreads();
    const int64_t excl = incl - c + (w > 0 ? warp_sum[w - 1] : 0);
    if (x < nq) items[x] = excl;
    if (x == 0) items[nq] = warp_sum[kScanProbes / 32 - 1];
}

// One warp per work item (probe, chunk of columns); lanes take consecutive
// columns.  Survive iff floor((S - h)/2) * (p+q) >= p * S (Eq. 2, Table 1).
// kW > 0: the probe's bitmap of kW words stays in registers and every lane
// takes four columns per step, their loads issued together; kW = 0: any width,
// one column per lane and step.  A lane recomputes the smallest passing overlap
// only when its column's size changes (sizes ascend along the window).
// kV: a survivor is verified at once by its lane (the merge of k_query_verify)
// and only similar pairs leave the kernel, as keys; the survivor queue is not
// written (small batches, which then skip the verification launch).
template <int kW, bool kV>
__global__ void __launch_bounds__(256)
    k_query_filter(const uint64_t *__restrict__ pbm, const int64_t *__restrict__ poff,
                   const uint32_t *__restrict__ pp, const uint32_t *__restrict__ pq,
                   const int64_t *__restrict__ wlo, const int64_t *__restrict__ whi,
                   const int64_t *__restrict__ item_off, int64_t nq,
                   const uint64_t *__restrict__ bm, const uint32_t *__restrict__ ssz, int W,
                   uint2 *__restrict__ queue, unsigned long long *__restrict__ qcount, int64_t qcap,
                   int sim, int chunk, const int32_t *__restrict__ ptok,
                   const int64_t *__restrict__ soff, const int32_t *__restrict__ stok,
                   const uint32_t *__restrict__ perm, uint64_t *__restrict__ keys,
                   unsigned long long *__restrict__ rcount) {
    constexpr int U = kW > 0 ? 4 : 1;  // columns per lane and step
    const int lane = threadIdx.x & 31;
    const int64_t n_items = item_off[nq];
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); item < n_items;
         item += warps) {
        int64_t lo = 0, hi = nq;  // probe x with item_off[x] <= item < item_off[x+1]
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (item_off[mid] <= item) lo = mid;
            else hi = mid;
        }
        const int64_t x = lo;
        const int64_t c0 = wlo[x] + (item - item_off[x]) * chunk;
        const int64_t c1 = min(c0 + (int64_t)chunk, whi[x]);
        const uint64_t sx = (uint64_t)(poff[x + 1] - poff[x]);
        const uint32_t p = pp[x], q = pq[x];
        uint64_t pb[kW > 0 ? kW : 1];
#pragma unroll
        for (int w = 0; w < kW; w++) pb[w] = pbm[x * kW + w];
        uint32_t last_s = 0xffffffffu;
        int64_t last_need = 0;
        for (int64_t j0 = c0; j0 < c1; j0 += 32 * U) {
            uint32_t cs[U];
            uint64_t cb[U][kW > 0 ? kW : 1];
#pragma unroll
            for (int u = 0; u < U; u++) {  // all loads of the step first
                const int64_t j = j0 + u * 32 + lane;
                cs[u] = j < c1 ? ssz[j] : 0u;
                if constexpr (kW == 2 || kW == 4) {  // 16-byte loads (a bitmap row is 16 or 32 bytes)
                    const ulonglong2 *b2 = reinterpret_cast<const ulonglong2 *>(bm) + j * (kW / 2);
#pragma unroll
                    for (int w = 0; w < kW / 2; w++) {
                        const ulonglong2 v = j < c1 ? b2[w] : make_ulonglong2(0ull, 0ull);
                        cb[u][2 * w] = v.x;
                        cb[u][2 * w + 1] = v.y;
                    }
                } else {
#pragma unroll
                    for (int w = 0; w < kW; w++) cb[u][w] = j < c1 ? bm[j * kW + w] : 0ull;
                }
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int64_t j = j0 + u * 32 + lane;
                bool sv = false;
                if (j < c1) {
                    int h = 0;
                    if constexpr (kW == 2 || kW == 4) {
                        // the carry-save popcount of the join's filter (3 or 4 POPC
                        // for 4 or 8 words instead of 4 or 8)
                        uint32_t xw[2 * kW];
#pragma unroll
                        for (int w = 0; w < kW; w++) {
                            const uint64_t d = pb[w] ^ cb[u][w];
                            xw[2 * w] = (uint32_t)d;
                            xw[2 * w + 1] = (uint32_t)(d >> 32);
                        }
                        h = PopcHS<kW>::h(xw);
                    } else if (kW > 0) {
#pragma unroll
                        for (int w = 0; w < kW; w++) h += __popcll(pb[w] ^ cb[u][w]);
                    } else {
                        for (int w = 0; w < W; w++) h += __popcll(pbm[x * W + w] ^ bm[j * W + w]);
                    }
                    if (cs[u] != last_s) {
                        last_s = cs[u];
                        last_need = sim_need(sim, p, q, (int64_t)sx, (int64_t)cs[u]);
                    }
                    const uint64_t S = sx + cs[u];
                    const int64_t ub = (int64_t)((S - (uint64_t)h) >> 1);   // Eq. 2
                    sv = ub >= last_need;
                }
                const unsigned ball = __ballot_sync(kFullQ, sv);
                if (ball) {
                    unsigned long long base = 0;
                    if (lane == 0) base = atomicAdd(qcount, (unsigned long long)__popc(ball));
                    base = __shfl_sync(kFullQ, base, 0);
                    const unsigned long long pos = base + __popc(ball & ((1u << lane) - 1u));
                    if (!kV && sv && pos < (unsigned long long)qcap)
                        queue[pos] = make_uint2((uint32_t)x, (uint32_t)j);
                    if (kV) {
                        bool similar = false;
                        uint64_t key = 0;
                        if (sv) {
                            const int32_t *xt = ptok + poff[x];
                            const int32_t *yt = stok + soff[j];
                            const int na = (int)sx, nb = (int)cs[u], nd = (int)last_need;
                            int a = 0, b = 0, o = 0;
                            while (a < na && b < nb) {
                                if (o + min(na - a, nb - b) < nd) break;
                                const int32_t xa = xt[a], yb = yt[b];
                                o += (xa == yb);
                                a += (xa <= yb);
                                b += (yb <= xa);
                                if (o >= nd) break;
                            }
                            similar = o >= nd;
                            if (similar) key = ((uint64_t)x << 32) | perm[j];
                        }
                        const unsigned rb = __ballot_sync(kFullQ, similar);
                        if (rb) {
                            unsigned long long rbase = 0;
                            if (lane == 0) rbase = atomicAdd(rcount, (unsigned long long)__popc(rb));
                            rbase = __shfl_sync(kFullQ, rbase, 0);
                            const unsigned long long rpos = rbase + __popc(rb & ((1u << lane) - 1u));
                            if (similar && rpos < (unsigned long long)qcap) keys[rpos] = key;
                        }
                    }
                }
            }
        }
    }
}

// Exact verification; similar pairs become keys (probe << 32) | original id.
__global__ void __launch_bounds__(256)
    k_query_verify(const uint2 *__restrict__ queue, const unsigned long long *__restrict__ qcount,
                   int64_t qcap, const int64_t *__restrict__ poff, const int32_t *__restrict__ ptok,
                   const uint32_t *__restrict__ pp, const uint32_t *__restrict__ pq,
                   const int64_t *__restrict__ soff, const int32_t *__restrict__ stok,
                   const uint32_t *__restrict__ ssz, const uint32_t *__restrict__ perm,
                   uint64_t *__restrict__ keys, unsigned long long *__restrict__ rcount, int sim) {
    const int lane = threadIdx.x & 31;
    const int64_t n_surv = min((int64_t)*qcount, qcap);
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (int64_t base = gw * 32; base < n_surv; base += warps * 32) {
        const int64_t idx = base + lane;
        bool similar = false;
        uint64_t key = 0;
        if (idx < n_surv) {
            const uint2 pr = queue[idx];
            const int32_t *x = ptok + poff[pr.x];
            const int na = (int)(poff[pr.x + 1] - poff[pr.x]);
            const int32_t *y = stok + soff[pr.y];
            const int nb = (int)ssz[pr.y];
            const int nd = (int)sim_need(sim, pp[pr.x], pq[pr.x], na, nb);
            int a = 0, b = 0, o = 0;
            while (a < na && b < nb) {
                if (o + min(na - a, nb - b) < nd) break;
                const int32_t xa = x[a], yb = y[b];
                o += (xa == yb);
                a += (xa <= yb);
                b += (yb <= xa);
                if (o >= nd) break;
            }
            similar = o >= nd;
            if (similar) key = ((uint64_t)pr.x << 32) | perm[pr.y];
        }
        const unsigned ball = __ballot_sync(kFullQ, similar);
        if (ball) {
            unsigned long long off = 0;
            if (lane == 0) off = atomicAdd(rcount, (unsigned long long)__popc(ball));
            off = __shfl_sync(kFullQ, off, 0);
            if (similar) keys[off + __popc(ball & ((1u << lane) - 1u))] = key;
        }
    }
}

__global__ void k_query_bounds(const uint64_t *__restrict__ keys, int64_t n, int64_t nq,
                               int64_t *__restrict__ bounds) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x <= nq; x += stride) {
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)(keys[mid] >> 32) < x) lo = mid + 1;
            else hi = mid;
        }
        bounds[x] = lo;
    }
}

unsigned grid_q(int64_t n, int threads, int64_t cap = 148 * 16) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

// ----------------------------------------------------------------------------
// A slot: everything one in-flight batch needs, allocated once.
// ----------------------------------------------------------------------------
struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    int64_t q_cap = 0, tok_cap = 0, pair_cap = 0;
    // pinned host staging: a batch's offsets, thresholds and tokens packed
    // into h_in, copied to d_in in one transfer (the pointers below point into
    // them, laid out for the batch by stage)
    unsigned char *h_in = nullptr, *d_in = nullptr;
    int64_t in_bytes = 0;
    int64_t *h_off = nullptr;
    int32_t *h_tok = nullptr;
    uint32_t *h_p = nullptr, *h_q = nullptr;
    unsigned long long *h_ctr = nullptr;  // [0] survivors, [1] results
    uint64_t *h_keys = nullptr;
    int64_t *h_bounds = nullptr;
    // device
    int64_t *d_off = nullptr;
    int32_t *d_tok = nullptr;
    uint32_t *d_p = nullptr, *d_q = nullptr;
    uint64_t *d_pbm = nullptr;
    int64_t *d_lo = nullptr, *d_hi = nullptr, *d_items = nullptr;
    uint2 *d_queue = nullptr;
    uint64_t *d_keys = nullptr, *d_sorted = nullptr;
    int64_t *d_bounds = nullptr;
    unsigned long long *d_ctr = nullptr;
    // in flight
    int phase = 0;  // 0 free, 1 filter+verify running, 2 sort+copy running
    int64_t win = 0;  // window pairs of the batch (exact, from the host size histogram)
    std::vector<int64_t> ids;  // query ids of the batch
    int64_t nq = 0, ntok = 0;
};

void free_slot(Slot &s) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    cudaFreeHost(s.h_in);
    cudaFreeHost(s.h_ctr);  // (h_keys lives in the same block)
    cudaFreeHost(s.h_bounds);
    cudaFree(s.d_in);
    cudaFree(s.d_pbm);
    cudaFree(s.d_lo);
    cudaFree(s.d_hi);
    cudaFree(s.d_items);
    cudaFree(s.d_queue);
    cudaFree(s.d_ctr);  // (d_keys lives in the same block)
    cudaFree(s.d_sorted);
    cudaFree(s.d_bounds);
    if (s.done) cudaEventDestroy(s.done);
    if (s.stream) cudaStreamDestroy(s.stream);
    cudaGetLastError();
    s = Slot();
}

int alloc_slot(Slot &s, int64_t q_cap, int64_t tok_cap, int64_t pair_cap, int W) {
    s.q_cap = q_cap;
    s.tok_cap = tok_cap;
    s.pair_cap = pair_cap;
    const size_t in_cap = (size_t)(q_cap + 1) * sizeof(int64_t) + 2 * (size_t)q_cap * sizeof(uint32_t) +
                          (size_t)std::max<int64_t>(tok_cap, 1) * sizeof(int32_t);
    bool ok = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) == cudaSuccess &&
              cudaMallocHost(&s.h_in, in_cap) == cudaSuccess &&
              cudaMallocHost(&s.h_ctr, (2 + pair_cap) * sizeof(uint64_t)) == cudaSuccess &&
              cudaMallocHost(&s.h_bounds, (q_cap + 1) * sizeof(int64_t)) == cudaSuccess &&
              cudaMalloc(&s.d_in, in_cap) == cudaSuccess &&
              cudaMalloc(&s.d_pbm, q_cap * W * sizeof(uint64_t)) == cudaSuccess &&
              cudaMalloc(&s.d_lo, q_cap * sizeof(int64_t)) == cudaSuccess &&
              cudaMalloc(&s.d_hi, q_cap * sizeof(int64_t)) == cudaSuccess &&
              cudaMalloc(&s.d_items, (q_cap + 1) * sizeof(int64_t)) == cudaSuccess &&
              cudaMalloc(&s.d_queue, pair_cap * sizeof(uint2)) == cudaSuccess &&
              cudaMalloc(&s.d_ctr, (2 + pair_cap) * sizeof(uint64_t)) == cudaSuccess &&
              cudaMalloc(&s.d_sorted, pair_cap * sizeof(uint64_t)) == cudaSuccess &&
              cudaMalloc(&s.d_bounds, (q_cap + 1) * sizeof(int64_t)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_slot(s);
        return BMJ_ERR_OOM;
    }
    // the result keys follow the two counters in the same block, host and device
    s.h_keys = reinterpret_cast<uint64_t *>(s.h_ctr + 2);
    s.d_keys = reinterpret_cast<uint64_t *>(s.d_ctr + 2);
    return BMJ_OK;
}

// Exact number of resident sets inside the window of a probe of size sx.
int64_t window_of(const bmj_index *idx, int64_t sx, uint32_t p, uint32_t q) {
    const SimWindow w = sim_window(idx->sim, p, q);
    const uint64_t lo_u = window_low((uint64_t)sx, w), hi_u = window_high((uint64_t)sx, w);
    const int64_t ms = (int64_t)idx->size_cum.size() - 1;
    const int64_t low = (int64_t)std::min<uint64_t>(lo_u, (uint64_t)ms);
    const int64_t high = (int64_t)std::min<uint64_t>(hi_u, (uint64_t)ms);
    auto cum = [&](int64_t s) { return idx->size_cum[(size_t)std::min(std::max<int64_t>(s, 0), ms)]; };
    return std::max<int64_t>(0, cum(high + 1) - cum(low));
}

// Phase 1 of a staged batch: copy in, bitmaps, windows, filter, verification,
// result count back to pinned memory.
int launch_phase1(const bmj_index *idx, Slot &s, int sms) {
    NvtxRange nv("bmj.serve_batch");
    cudaStream_t st = s.stream;
    const int64_t nq = s.nq;
    BMJ_CHECK(cudaMemcpyAsync(s.d_in, s.h_in, s.in_bytes, cudaMemcpyHostToDevice, st));
    if (nq > kScanProbes)  // (the one-block window kernel clears them otherwise)
        BMJ_CHECK(cudaMemsetAsync(s.d_ctr, 0, 2 * sizeof(unsigned long long), st));
    // the bitmaps of small batches (Xor/Set, up to 256 bits) are built in the
    // window kernel, a warp per probe: one launch fewer (p50 0.049 -> 0.043 ms
    // at 20,000 q/s); larger batches keep the separate warp-per-probe kernel
    const bool fuse = nq <= kFuseProbes && (idx->method == BMJ_XOR || idx->method == BMJ_SET) &&
                      (idx->b == 64 || idx->b == 128 || idx->b == 256);
    int rc = BMJ_OK;
    if (!fuse)
        rc = launch_gather_build(nullptr, s.d_off, s.d_tok, nullptr, nullptr, s.d_pbm, nq, idx->b,
                                 idx->method, st);
    if (rc) return rc;
    Arena A(st);
    int chunk = kQueryChunk;
    while (chunk > kQueryChunkMin && s.win / chunk < (int64_t)sms * 32) chunk >>= 1;
    if (nq <= kScanProbes) {  // windows and their scan in one launch
        BMJ_LAUNCH(k_probe_windows_scan, 1, kScanProbes, 0, st, s.d_off, nq, s.d_p, s.d_q,
                   idx->d_size_cum, idx->max_size, idx->n, s.d_lo, s.d_hi, s.d_items, idx->sim,
                   chunk, s.d_ctr, s.d_tok, s.d_pbm, fuse ? idx->b / 64 : 0,
                   idx->method == BMJ_XOR ? 1 : 0);
    } else {
        BMJ_LAUNCH(k_probe_windows, grid_q(nq, 128), 128, 0, st, s.d_off, nq, s.d_p, s.d_q,
                   idx->d_size_cum, idx->max_size, idx->n, s.d_lo, s.d_hi, s.d_items, idx->sim,
                   chunk);
        rc = exclusive_scan_i64(s.d_items, s.d_items, nq, s.d_items + nq, A, st);
        if (rc) return rc;
    }
    // grids no larger than the batch's work: a probe's window of w sets is
    // ceil(w / chunk) work items, and every survivor is a window pair
    const int64_t items_ub = s.win / chunk + nq;
    const unsigned fblocks =
        (unsigned)std::min<int64_t>((int64_t)sms * 8, std::max<int64_t>(1, (items_ub + 7) / 8));
    const unsigned vblocks =
        (unsigned)std::min<int64_t>((int64_t)sms * 4, std::max<int64_t>(1, (s.win + 255) / 256));
    // a batch of at most kFuseProbes probes whose windows hold at most
    // kInlineVerifyWindow pairs verifies its survivors inside the filter (one
    // launch fewer): a lane merges the survivors it found while the rest of
    // its warp waits, which is cheap while survivors are few per warp; larger
    // batches and wide windows (many survivors at low thresholds) keep the
    // thread-per-survivor kernel
    const bool inline_verify = nq <= kFuseProbes && s.win <= kInlineVerifyWindow;
#define BMJ_QUERY_FILTER(KW, KV)                                                               \
    BMJ_LAUNCH((k_query_filter<KW, KV>), fblocks, 256, 0, st, s.d_pbm, s.d_off, s.d_p, s.d_q,   \
               s.d_lo, s.d_hi, s.d_items, nq, idx->bm, idx->ssz, idx->W, s.d_queue, &s.d_ctr[0],  \
               s.pair_cap, idx->sim, chunk, s.d_tok, idx->soff, idx->stok, idx->perm, s.d_keys,   \
               &s.d_ctr[1])
    switch (idx->W * 2 + (inline_verify ? 1 : 0)) {
        case 2: BMJ_QUERY_FILTER(1, false); break;
        case 3: BMJ_QUERY_FILTER(1, true); break;
        case 4: BMJ_QUERY_FILTER(2, false); break;
        case 5: BMJ_QUERY_FILTER(2, true); break;
        case 8: BMJ_QUERY_FILTER(4, false); break;
        case 9: BMJ_QUERY_FILTER(4, true); break;
        default:
            if (inline_verify) BMJ_QUERY_FILTER(0, true);
            else BMJ_QUERY_FILTER(0, false);
            break;
    }
#undef BMJ_QUERY_FILTER
    if (!inline_verify)
        BMJ_LAUNCH(k_query_verify, vblocks, 256, 0, st, s.d_queue, &s.d_ctr[0], s.pair_cap,
                   s.d_off, s.d_tok, s.d_p, s.d_q, idx->soff, idx->stok, idx->ssz, idx->perm,
                   s.d_keys, &s.d_ctr[1], idx->sim);
    // the counters and the first result keys, adjacent on both sides, come back in
    // one copy: a batch with few results then finishes on the host without a
    // second round trip (finish_on_host)
    BMJ_CHECK(cudaMemcpyAsync(s.h_ctr, s.d_ctr,
                              (2 + std::min(s.pair_cap, kEagerKeys)) * sizeof(uint64_t),
                              cudaMemcpyDeviceToHost, st));
    BMJ_CHECK(cudaEventRecord(s.done, st));
    A.release();
    return BMJ_OK;
}

// After phase 1: a batch whose results all came back with its counters is
// sorted by (probe, id) on the host and gets its per-probe bounds there.
// Returns false when the batch has more results than that (phase 2 sorts them
// on the device).
bool finish_on_host(Slot &s) {
    const int64_t nres = (int64_t)s.h_ctr[1];
    if (nres > std::min(s.pair_cap, kEagerKeys)) return false;
    std::sort(s.h_keys, s.h_keys + nres);
    int64_t r = 0;
    for (int64_t k = 0; k <= s.nq; k++) {
        while (r < nres && (int64_t)(s.h_keys[r] >> 32) < k) r++;
        s.h_bounds[k] = r;
    }
    return true;
}

// Phase 2: sort the results by (probe, id), per-probe bounds, copy out.
int launch_phase2(Slot &s) {
    cudaStream_t st = s.stream;
    const int64_t nres = (int64_t)s.h_ctr[1];
    const int64_t nq = s.nq;
    Arena A(st);
    if (nres > 0) {
        const int pbits = nq > 1 ? bit_length((uint64_t)(nq - 1)) : 1;
        int rc = radix_sort_u64(s.d_keys, s.d_sorted, nres, 32 + pbits, A, st);
        if (rc) return rc;
        BMJ_LAUNCH(k_query_bounds, grid_q(nq + 1, 128), 128, 0, st, s.d_sorted, nres, nq, s.d_bounds);
        BMJ_CHECK(cudaMemcpyAsync(s.h_keys, s.d_sorted, nres * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
        BMJ_CHECK(cudaMemcpyAsync(s.h_bounds, s.d_bounds, (nq + 1) * sizeof(int64_t),
                                  cudaMemcpyDeviceToHost, st));
    } else {
        memset(s.h_bounds, 0, (nq + 1) * sizeof(int64_t));
    }
    BMJ_CHECK(cudaEventRecord(s.done, st));
    A.release();
    return BMJ_OK;
}

// Stages m queries into a slot.  get(k, &tokens, &n_tokens, &p, &q) gives
// the k-th query of the batch.
template <class Get>
void stage_with(Slot &s, int64_t m, Get get) {
    s.nq = m;
    // packed layout: offsets (m + 1 int64), p (m), q (m), then the tokens
    const size_t o_p = (size_t)(m + 1) * sizeof(int64_t), o_q = o_p + m * sizeof(uint32_t),
                 o_t = o_q + m * sizeof(uint32_t);
    s.h_off = reinterpret_cast<int64_t *>(s.h_in);
    s.h_p = reinterpret_cast<uint32_t *>(s.h_in + o_p);
    s.h_q = reinterpret_cast<uint32_t *>(s.h_in + o_q);
    s.h_tok = reinterpret_cast<int32_t *>(s.h_in + o_t);
    s.d_off = reinterpret_cast<int64_t *>(s.d_in);
    s.d_p = reinterpret_cast<uint32_t *>(s.d_in + o_p);
    s.d_q = reinterpret_cast<uint32_t *>(s.d_in + o_q);
    s.d_tok = reinterpret_cast<int32_t *>(s.d_in + o_t);
    s.h_off[0] = 0;
    int64_t t = 0;
    for (int64_t k = 0; k < m; k++) {
        const int32_t *tk = nullptr;
        int64_t nt = 0;
        get(k, &tk, &nt, &s.h_p[k], &s.h_q[k]);
        memcpy(s.h_tok + t, tk, nt * sizeof(int32_t));
        t += nt;
        s.h_off[k + 1] = t;
    }
    s.ntok = t;
    s.in_bytes = (int64_t)(o_t + t * sizeof(int32_t));
}

// Stages queries ids[0..m) of a host query collection into a slot.
void stage(Slot &s, const bmj_collection *qc, const uint32_t *p, const uint32_t *q,
           const int64_t *ids, int64_t m) {
    s.ids.assign(ids, ids + m);
    stage_with(s, m, [&](int64_t k, const int32_t **tk, int64_t *nt, uint32_t *pk, uint32_t *qk) {
        const int64_t x = ids[k];
        *tk = qc->tokens + qc->offsets[x];
        *nt = qc->offsets[x + 1] - qc->offsets[x];
        *pk = p[x];
        *qk = q[x];
    });
}

}  // namespace
}  // namespace bmj

// ============================================================================
// C ABI
// ============================================================================
using namespace bmj;

extern "C" int bmj_index_create(const bmj_collection *coll, const bmj_options *opt,
                                bmj_index **out) {
    if (!out) return BMJ_ERR_INVALID_ARG;
    *out = nullptr;
    if (!coll || coll->n_sets < 0 || !coll->offsets || (coll->n_sets > 0 && !coll->tokens))
        return BMJ_ERR_INVALID_ARG;
    if (coll->n_sets > 0x7fffffffLL) return BMJ_ERR_TOO_LARGE;
    bmj_options o;
    if (opt) o = *opt;
    else bmj_default_options(&o);
    if (!valid_b(o.b)) return BMJ_ERR_INVALID_ARG;
    if (o.method != BMJ_XOR && o.method != BMJ_SET && o.method != BMJ_NEXT) return BMJ_ERR_INVALID_ARG;
    if (o.sim < BMJ_JACCARD || o.sim > BMJ_OVERLAP) return BMJ_ERR_INVALID_ARG;
    bmj_index *idx = new (std::nothrow) bmj_index();
    if (!idx) return BMJ_ERR_OOM;
    cudaStream_t s = (cudaStream_t)o.stream;
    int st = BMJ_OK;
    {
        Arena A(s);
        DevColl d;
        st = stage_collection(coll, A, s, &d);
        uint32_t *sizes = nullptr, *ids = nullptr;
        int max_size = 0;
        if (!st && d.n > 0) st = validate(d, o.validate != 0, A, s, &sizes, &ids, &max_size);
        if (!st) {
            cudaGetDevice(&idx->device);
            idx->b = o.b;
            idx->W = o.b / 64;
            idx->method = o.method;
            idx->sim = o.sim;
            idx->n = d.n;
            idx->max_size = max_size;
            const int64_t n = d.n;
            bool ok = cudaMalloc(&idx->ssz, (n + 4) * sizeof(uint32_t)) == cudaSuccess &&
                      cudaMalloc(&idx->perm, std::max<int64_t>(n, 1) * sizeof(uint32_t)) == cudaSuccess &&
                      cudaMalloc(&idx->soff, (n + 1) * sizeof(int64_t)) == cudaSuccess &&
                      cudaMalloc(&idx->stok, std::max<int64_t>(d.ntok, 1) * sizeof(int32_t)) == cudaSuccess &&
                      cudaMalloc(&idx->bm, (n + 4) * idx->W * sizeof(uint64_t)) == cudaSuccess;
            if (!ok) {
                cudaGetLastError();
                st = BMJ_ERR_OOM;
            }
            if (!st && n > 0) {
                if (cudaMemsetAsync(idx->ssz + n, 0, 4 * sizeof(uint32_t), s) != cudaSuccess)
                    st = BMJ_ERR_CUDA;
                if (!st) st = radix_sort_u32_pairs(sizes, ids, idx->ssz, idx->perm, n,
                                          std::max(1, bit_length((uint64_t)max_size)), A, s);
                if (!st) st = launch_widen(idx->ssz, idx->soff, n, s);
                if (!st) st = exclusive_scan_i64(idx->soff, idx->soff, n, idx->soff + n, A, s);
                if (!st)
                    st = launch_gather_build(idx->perm, d.off, d.tok, idx->soff, idx->stok, idx->bm,
                                             n, idx->b, idx->method, s);
                if (!st) {
                    std::vector<uint32_t> h(n);
                    if (cudaMemcpyAsync(h.data(), idx->ssz, n * sizeof(uint32_t),
                                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                        cudaStreamSynchronize(s) != cudaSuccess) {
                        st = BMJ_ERR_CUDA;
                    } else {
                        idx->size_cum.assign((size_t)max_size + 2, 0);
                        for (int64_t i = 0; i < n; i++) idx->size_cum[h[i] + 1]++;
                        for (size_t k = 1; k < idx->size_cum.size(); k++)
                            idx->size_cum[k] += idx->size_cum[k - 1];
                    }
                }
            } else if (!st) {
                idx->size_cum.assign(2, 0);
                cudaMemsetAsync(idx->soff, 0, sizeof(int64_t), s);
            }
            if (!st) {  // the window lookup table on the device
                const size_t bytes = idx->size_cum.size() * sizeof(int64_t);
                if (cudaMalloc(&idx->d_size_cum, bytes) != cudaSuccess) {
                    cudaGetLastError();
                    st = BMJ_ERR_OOM;
                } else if (cudaMemcpyAsync(idx->d_size_cum, idx->size_cum.data(), bytes,
                                           cudaMemcpyHostToDevice, s) != cudaSuccess) {
                    st = BMJ_ERR_CUDA;
                }
            }
        }
        A.release();
        if (cudaStreamSynchronize(s) != cudaSuccess && !st) st = BMJ_ERR_CUDA;
    }
    if (st) {
        bmj_index_destroy(idx);
        cudaGetLastError();
        return st;
    }
    *out = idx;
    return BMJ_OK;
}

extern "C" void bmj_index_destroy(bmj_index *idx) {
    if (!idx) return;
    cudaFree(idx->ssz);
    cudaFree(idx->perm);
    cudaFree(idx->soff);
    cudaFree(idx->stok);
    cudaFree(idx->bm);
    cudaFree(idx->d_size_cum);
    cudaGetLastError();
    delete idx;
}

extern "C" int64_t bmj_index_size(const bmj_index *idx) { return idx ? idx->n : -1; }

static int check_queries(const bmj_index *idx, const bmj_collection *qc, const uint32_t *p,
                         const uint32_t *q) {
    if (!qc || qc->on_device || qc->n_sets < 0 || !qc->offsets || (qc->n_sets > 0 && (!qc->tokens || !p || !q)))
        return BMJ_ERR_INVALID_ARG;
    if (qc->offsets[0] != 0) return BMJ_ERR_UNSORTED;
    for (int64_t x = 0; x < qc->n_sets; x++) {
        if (!sim_valid(idx->sim, p[x], q[x])) return BMJ_ERR_INVALID_ARG;
        const int64_t a = qc->offsets[x], b = qc->offsets[x + 1];
        if (b < a) return BMJ_ERR_UNSORTED;
        if (b == a) return BMJ_ERR_EMPTY_SET;
        if (qc->tokens[a] < 0) return BMJ_ERR_NEG_TOKEN;
        for (int64_t k = a + 1; k < b; k++)
            if (qc->tokens[k] <= qc->tokens[k - 1]) return BMJ_ERR_UNSORTED;
    }
    return BMJ_OK;
}

static void id_lists_free_impl(bmj_id_lists *l) {
    if (!l) return;
    free(l->offsets);
    free(l->ids);
    l->offsets = nullptr;
    l->ids = nullptr;
    l->n_queries = 0;
}

extern "C" void bmj_id_lists_free(bmj_id_lists *lists) { id_lists_free_impl(lists); }

// Runs queries through the slots.  arrival_s == NULL: everything is available
// at once (a plain batched query).  Results are written into *out (optional)
// and per-query latency into latency_ms (optional).
static int serve_impl(bmj_index *idx, const bmj_collection *qc, const double *arrival_s,
                      const uint32_t *p, const uint32_t *q, const bmj_serve_options &so,
                      bmj_id_lists *out, double *latency_ms, bmj_serve_stats *stats) {
    using clk = std::chrono::steady_clock;
    const int64_t Q = qc->n_sets;
    int dev = 0;
    BMJ_CHECK(cudaGetDevice(&dev));
    const int sms = num_sms(dev);
    const int n_slots = std::max(1, so.n_slots);
    int64_t max_q = so.max_batch_queries > 0 ? so.max_batch_queries : 4096;
    int64_t pair_budget = so.max_batch_window_pairs > 0 ? so.max_batch_window_pairs : ((int64_t)1 << 25);
    int64_t max_tok = 0, max_win = 0;
    std::vector<int64_t> win(Q);
    for (int64_t x = 0; x < Q; x++) {
        const int64_t sx = qc->offsets[x + 1] - qc->offsets[x];
        max_tok = std::max(max_tok, sx);
        win[x] = window_of(idx, sx, p[x], q[x]);
        max_win = std::max(max_win, win[x]);
    }
    // A single query always fits a slot on its own.
    pair_budget = std::max(pair_budget, std::max<int64_t>(max_win, 1));
    const int64_t tok_cap = max_q * std::max<int64_t>(max_tok, 1);
    std::vector<Slot> slots(n_slots);
    for (auto &s : slots) {
        int rc = alloc_slot(s, max_q, tok_cap, pair_budget, idx->W);
        if (rc) {
            for (auto &t : slots) free_slot(t);
            return rc;
        }
    }
    std::vector<int64_t> counts(Q, 0);
    std::vector<std::vector<int64_t>> per_q(out ? Q : 0);
    std::vector<double> lat(Q, 0.0);
    int64_t next = 0, completed = 0, batches = 0, total_window = 0, total_surv = 0, total_res = 0;
    std::vector<int64_t> pending;
    size_t pend_head = 0;
    int rc = BMJ_OK;
    const auto t0 = clk::now();
    auto now_s = [&]() { return std::chrono::duration<double>(clk::now() - t0).count(); };
    while (completed < Q && !rc) {
        const double now = now_s();
        while (next < Q && (!arrival_s || arrival_s[next] <= now)) pending.push_back(next++);
        bool progressed = false;
        // 1. finished phases
        for (auto &s : slots) {
            if (s.phase == 0) continue;
            const cudaError_t e = cudaEventQuery(s.done);
            if (e == cudaErrorNotReady) continue;
            if (e != cudaSuccess) {
                rc = status_of(e);
                break;
            }
            progressed = true;
            bool finished = s.phase == 2;
            if (s.phase == 1) {
                total_surv += (int64_t)s.h_ctr[0];
                total_res += (int64_t)s.h_ctr[1];
                if (finish_on_host(s)) {
                    finished = true;
                } else {
                    rc = launch_phase2(s);
                    s.phase = 2;
                }
            }
            if (finished) {
                const double t_done = now_s();
                for (int64_t k = 0; k < s.nq; k++) {
                    const int64_t x = s.ids[k];
                    lat[x] = (t_done - (arrival_s ? arrival_s[x] : 0.0)) * 1e3;
                    const int64_t lo = s.h_bounds[k], hi = s.h_bounds[k + 1];
                    counts[x] = hi - lo;
                    if (out) {
                        per_q[x].resize(hi - lo);
                        for (int64_t r = lo; r < hi; r++)
                            per_q[x][r - lo] = (int64_t)(s.h_keys[r] & 0xffffffffu);
                    }
                }
                completed += s.nq;
                s.phase = 0;
            }
        }
        if (rc) break;
        // 2. admission: arrived queries into free slots, bounded by the slot's
        //    query, token and window-pair capacities.
        for (auto &s : slots) {
            if (pend_head >= pending.size()) break;
            if (s.phase != 0) continue;
            std::vector<int64_t> take;
            int64_t w = 0, t = 0;
            while (pend_head < pending.size() && (int64_t)take.size() < max_q) {
                const int64_t x = pending[pend_head];
                const int64_t sx = qc->offsets[x + 1] - qc->offsets[x];
                if (!take.empty() && (w + win[x] > pair_budget || t + sx > tok_cap)) break;
                take.push_back(x);
                w += win[x];
                t += sx;
                pend_head++;
            }
            stage(s, qc, p, q, take.data(), (int64_t)take.size());
            s.win = w;
            total_window += w;
            rc = launch_phase1(idx, s, sms);
            if (rc) break;
            s.phase = 1;
            batches++;
            progressed = true;
        }
        if (!progressed) {
            // sleep only through long gaps (the wake-up can come tens of
            // microseconds late); otherwise keep polling arrivals and events
            const double wait = (pend_head >= pending.size() && next < Q && arrival_s)
                                    ? arrival_s[next] - now_s()
                                    : 0.0;
            if (wait > 1e-3)
                std::this_thread::sleep_for(std::chrono::microseconds((int64_t)((wait - 5e-4) * 1e6)));
            else
                std::this_thread::yield();
        }
    }
    const double wall = now_s();
    for (auto &s : slots) free_slot(s);
    if (rc) return rc;
    if (out) {
        out->n_queries = Q;
        out->offsets = (int64_t *)malloc((Q + 1) * sizeof(int64_t));
        int64_t tot = 0;
        for (int64_t x = 0; x < Q; x++) tot += counts[x];
        out->ids = (int64_t *)malloc(std::max<int64_t>(tot, 1) * sizeof(int64_t));
        if (!out->offsets || !out->ids) {
            id_lists_free_impl(out);
            return BMJ_ERR_OOM;
        }
        out->offsets[0] = 0;
        for (int64_t x = 0; x < Q; x++) {
            out->offsets[x + 1] = out->offsets[x] + counts[x];
            if (counts[x])
                memcpy(out->ids + out->offsets[x], per_q[x].data(), counts[x] * sizeof(int64_t));
        }
    }
    if (latency_ms) memcpy(latency_ms, lat.data(), Q * sizeof(double));
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->n_queries = Q;
        stats->batches = batches;
        stats->window_pairs = total_window;
        stats->survivors = total_surv;
        stats->results = total_res;
        stats->wall_s = wall;
        std::vector<double> sorted = lat;
        std::sort(sorted.begin(), sorted.end());
        auto pct = [&](double f) {
            if (sorted.empty()) return 0.0;
            size_t k = (size_t)std::min<double>((double)sorted.size() - 1, f * (double)sorted.size());
            return sorted[k];
        };
        stats->p50_ms = pct(0.50);
        stats->p99_ms = pct(0.99);
        stats->max_ms = sorted.empty() ? 0.0 : sorted.back();
        stats->qps = wall > 0 ? (double)Q / wall : 0.0;
    }
    return BMJ_OK;
}

extern "C" void bmj_default_serve_options(bmj_serve_options *so) {
    if (!so) return;
    memset(so, 0, sizeof(*so));
    so->n_slots = 4;
    so->max_batch_queries = 4096;
    so->max_batch_window_pairs = (int64_t)1 << 25;
    so->max_probe_tokens = 4096;
}

// A device-level failure (CUDA runtime error, bounded wait given up) leaves the
// index's device state in doubt: it sticks to the handle.  Argument errors and
// out-of-memory do not.
static int stick(bmj_index *idx, int st) {
    if (st == BMJ_ERR_CUDA || st == BMJ_ERR_TIMEOUT) idx->sticky = st;
    return st;
}

extern "C" int bmj_index_status(const bmj_index *idx) {
    return idx ? idx->sticky : BMJ_ERR_INVALID_ARG;
}

extern "C" int bmj_index_query(bmj_index *idx, const bmj_collection *probes, const uint32_t *p,
                               const uint32_t *q, bmj_id_lists *out, bmj_serve_stats *stats) {
    if (!idx || !out) return BMJ_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    if (idx->sticky) return idx->sticky;
    int st = check_queries(idx, probes, p, q);
    if (st) return st;
    if (bmj::read_fault_plan().serve) return stick(idx, BMJ_ERR_CUDA);
    bmj_serve_options so;
    bmj_default_serve_options(&so);
    so.n_slots = 1;
    so.max_batch_queries = std::max<int64_t>(1, std::min<int64_t>(probes->n_sets, 1 << 16));
    try {
        st = serve_impl(idx, probes, nullptr, p, q, so, out, nullptr, stats);
    } catch (...) {
        st = BMJ_ERR_OOM;
    }
    if (st) {
        id_lists_free_impl(out);
        cudaGetLastError();
    }
    return stick(idx, st);
}

extern "C" int bmj_serve(bmj_index *idx, const bmj_collection *queries, const double *arrival_s,
                         const uint32_t *p, const uint32_t *q, const bmj_serve_options *opt,
                         bmj_id_lists *out, double *latency_ms, bmj_serve_stats *stats) {
    if (!idx || !arrival_s) return BMJ_ERR_INVALID_ARG;
    if (out) memset(out, 0, sizeof(*out));
    if (idx->sticky) return idx->sticky;
    int st = check_queries(idx, queries, p, q);
    if (st) return st;
    if (bmj::read_fault_plan().serve) return stick(idx, BMJ_ERR_CUDA);
    for (int64_t x = 1; x < queries->n_sets; x++)
        if (arrival_s[x] < arrival_s[x - 1]) return BMJ_ERR_INVALID_ARG;
    bmj_serve_options so;
    if (opt) so = *opt;
    else bmj_default_serve_options(&so);
    if (so.n_slots < 1 || so.max_batch_queries < 0 || so.max_batch_window_pairs < 0)
        return BMJ_ERR_INVALID_ARG;
    try {
        st = serve_impl(idx, queries, arrival_s, p, q, so, out, latency_ms, stats);
    } catch (...) {
        st = BMJ_ERR_OOM;
    }
    if (st) {
        if (out) id_lists_free_impl(out);
        cudaGetLastError();
    }
    return stick(idx, st);
}

// ============================================================================
// Live serving: a request loop that accepts queries while batches run.
// ============================================================================
namespace {

struct LiveQuery {
    std::vector<int32_t> tok;
    uint32_t p = 0, q = 0;
    int64_t win = 0;
    std::chrono::steady_clock::time_point t_submit;
};

struct LiveResult {
    int status = BMJ_OK;
    std::vector<int64_t> ids;
    double latency_ms = 0.0;
};

}  // namespace

struct bmj_server {
    bmj_index *idx = nullptr;
    int64_t max_q = 0, tok_cap = 0, pair_budget = 0, max_probe = 0;
    std::vector<bmj::Slot> slots;
    std::thread loop;
    std::mutex mu;
    std::condition_variable cv_work;   // the loop waits here for submissions
    std::condition_variable cv_done;   // pollers wait here for results
    std::deque<int64_t> pending;       // submitted, not yet in a batch (ticket order)
    std::atomic<int64_t> n_pending{0}; // its length, read by the loop without the lock
    std::atomic<bool> closing_flag{false};
    std::unordered_map<int64_t, LiveQuery> queries;   // submitted, not yet completed
    std::unordered_map<int64_t, LiveResult> results;  // completed, not yet polled
    int64_t next_ticket = 0;
    bool closing = false;
    bool fault_serve = false;  // host fault injection: the first batch fails as a CUDA error would
    int error = BMJ_OK;
    // totals (written by the loop under mu)
    std::vector<double> latencies;
    int64_t batches = 0, window_pairs = 0, survivors = 0, n_results = 0;
    std::chrono::steady_clock::time_point t_open, t_last;
};

namespace {

// The request loop of a live server (its own host thread, the index's device
// current).  Slots are touched by this thread only; the queues and result
// table are shared with submitters and pollers under srv->mu.
void live_loop(bmj_server *srv) {
    using clk = std::chrono::steady_clock;
    bmj_index *idx = srv->idx;
    // a device that cannot be made current fails every query (below)
    int rc = cudaSetDevice(idx->device) == cudaSuccess ? BMJ_OK : BMJ_ERR_CUDA;
    const int sms = bmj::num_sms(idx->device);
    // per slot: the queries of its batch (pointers stay valid: node-based map,
    // entries erased by this thread only)
    std::vector<std::vector<const LiveQuery *>> batch_q(srv->slots.size());
    auto last_activity = clk::now();
    while (!rc) {
        bool progressed = false;
        bool in_flight = false;
        // 1. finished phases
        for (size_t si = 0; si < srv->slots.size() && !rc; si++) {
            bmj::Slot &s = srv->slots[si];
            if (s.phase == 0) continue;
            const cudaError_t e = cudaEventQuery(s.done);
            if (e == cudaErrorNotReady) {
                in_flight = true;
                continue;
            }
            if (e != cudaSuccess) {
                rc = bmj::status_of(e);
                break;
            }
            progressed = true;
            bool finished = s.phase == 2;
            if (s.phase == 1) {
                if (bmj::finish_on_host(s)) {
                    finished = true;
                } else {
                    rc = bmj::launch_phase2(s);
                    s.phase = 2;
                    in_flight = true;
                }
            }
            if (finished) {
                const auto t_done = clk::now();
                std::vector<LiveResult> out(s.nq);
                for (int64_t k = 0; k < s.nq; k++) {
                    const int64_t lo = s.h_bounds[k], hi = s.h_bounds[k + 1];
                    out[k].ids.resize(hi - lo);
                    for (int64_t r = lo; r < hi; r++)
                        out[k].ids[r - lo] = (int64_t)(s.h_keys[r] & 0xffffffffu);
                    out[k].latency_ms = std::chrono::duration<double, std::milli>(
                                            t_done - batch_q[si][k]->t_submit).count();
                }
                {
                    std::lock_guard<std::mutex> g(srv->mu);
                    srv->survivors += (int64_t)s.h_ctr[0];
                    srv->n_results += (int64_t)s.h_ctr[1];
                    for (int64_t k = 0; k < s.nq; k++) {
                        srv->latencies.push_back(out[k].latency_ms);
                        srv->results[s.ids[k]] = std::move(out[k]);
                        srv->queries.erase(s.ids[k]);
                    }
                    srv->t_last = t_done;
                }
                srv->cv_done.notify_all();
                batch_q[si].clear();
                s.phase = 0;
            }
        }
        if (rc) break;
        // 2. admission: submitted queries into free slots, bounded by the slot's
        //    query, token and window-pair capacities
        bool closing = false, waiting = false;
        for (size_t si = 0; si < srv->slots.size() && !rc; si++) {
            bmj::Slot &s = srv->slots[si];
            if (s.phase != 0) continue;
            std::vector<int64_t> take;
            std::vector<const LiveQuery *> qs;
            int64_t w = 0, t = 0;
            if (srv->n_pending.load(std::memory_order_acquire) == 0) break;
            {
                std::lock_guard<std::mutex> g(srv->mu);
                while (!srv->pending.empty() && (int64_t)take.size() < srv->max_q) {
                    const int64_t x = srv->pending.front();
                    const LiveQuery &lq = srv->queries.at(x);
                    const int64_t sx = (int64_t)lq.tok.size();
                    if (!take.empty() && (w + lq.win > srv->pair_budget || t + sx > srv->tok_cap))
                        break;
                    take.push_back(x);
                    qs.push_back(&lq);
                    w += lq.win;
                    t += sx;
                    srv->pending.pop_front();
                }
                srv->n_pending.fetch_sub((int64_t)take.size(), std::memory_order_release);
                if (!take.empty()) {
                    srv->batches++;
                    srv->window_pairs += w;
                }
            }
            if (take.empty()) break;
            s.ids = take;
            bmj::stage_with(s, (int64_t)take.size(),
                            [&](int64_t k, const int32_t **tk, int64_t *nt, uint32_t *pk,
                                uint32_t *qk) {
                                *tk = qs[k]->tok.data();
                                *nt = (int64_t)qs[k]->tok.size();
                                *pk = qs[k]->p;
                                *qk = qs[k]->q;
                            });
            s.win = w;
            batch_q[si] = std::move(qs);
            if (srv->fault_serve) {  // (BMJ_FAULT=serve at open: nothing is launched)
                rc = BMJ_ERR_CUDA;
                break;
            }
            rc = bmj::launch_phase1(idx, s, sms);
            if (rc) break;
            s.phase = 1;
            in_flight = true;
            progressed = true;
        }
        if (rc) break;
        closing = srv->closing_flag.load(std::memory_order_acquire);
        waiting = srv->n_pending.load(std::memory_order_acquire) > 0;
        if (!in_flight && !waiting && closing) break;  // drained
        if (progressed) {
            last_activity = clk::now();
        } else if (!in_flight && !waiting) {
            // idle: poll for a millisecond (a wake-up from a sleep can come tens of
            // microseconds late), then block until a submission or close
            if (clk::now() - last_activity < std::chrono::milliseconds(1)) {
                std::this_thread::yield();
            } else {
                std::unique_lock<std::mutex> lk(srv->mu);
                srv->cv_work.wait(lk, [&] { return srv->closing || !srv->pending.empty(); });
                last_activity = clk::now();
            }
        } else {
            std::this_thread::yield();
        }
    }
    if (rc) {
        // a device-level failure: every query not yet completed fails with it
        for (auto &s : srv->slots)
            if (s.stream) cudaStreamSynchronize(s.stream);
        cudaGetLastError();
        std::lock_guard<std::mutex> g(srv->mu);
        srv->error = rc;
        for (auto &kv : srv->queries) {
            LiveResult r;
            r.status = rc;
            srv->results[kv.first] = std::move(r);
        }
        srv->queries.clear();
        srv->pending.clear();
        srv->n_pending.store(0);
        if (rc == BMJ_ERR_CUDA || rc == BMJ_ERR_TIMEOUT) idx->sticky = rc;
    }
    srv->cv_done.notify_all();
}

void destroy_server(bmj_server *srv) {
    for (auto &s : srv->slots) bmj::free_slot(s);
    delete srv;
}

}  // namespace

extern "C" int bmj_serve_open(bmj_index *idx, const bmj_serve_options *opt, bmj_server **out) {
    if (!out) return BMJ_ERR_INVALID_ARG;
    *out = nullptr;
    if (!idx) return BMJ_ERR_INVALID_ARG;
    if (idx->sticky) return idx->sticky;
    bmj_serve_options so;
    if (opt) so = *opt;
    else bmj_default_serve_options(&so);
    if (so.n_slots < 1 || so.max_batch_queries < 0 || so.max_batch_window_pairs < 0 ||
        so.max_probe_tokens < 0)
        return BMJ_ERR_INVALID_ARG;
    bmj_server *srv = new (std::nothrow) bmj_server();
    if (!srv) return BMJ_ERR_OOM;
    srv->idx = idx;
    srv->fault_serve = bmj::read_fault_plan().serve;
    srv->max_q = so.max_batch_queries > 0 ? so.max_batch_queries : 4096;
    srv->max_probe = so.max_probe_tokens > 0 ? so.max_probe_tokens : 4096;
    srv->tok_cap = std::max<int64_t>(srv->max_probe,
                                     std::min<int64_t>(srv->max_q * srv->max_probe, (int64_t)1 << 22));
    // a single query's window holds at most every resident set: it always fits a slot
    srv->pair_budget = std::max<int64_t>(
        so.max_batch_window_pairs > 0 ? so.max_batch_window_pairs : ((int64_t)1 << 25),
        std::max<int64_t>(idx->n, 1));
    int dev_prev = 0;
    cudaGetDevice(&dev_prev);
    if (cudaSetDevice(idx->device) != cudaSuccess) {
        cudaGetLastError();
        delete srv;
        return BMJ_ERR_CUDA;
    }
    srv->slots.resize(so.n_slots);
    int rc = BMJ_OK;
    for (auto &s : srv->slots) {
        rc = bmj::alloc_slot(s, srv->max_q, srv->tok_cap, srv->pair_budget, idx->W);
        if (rc) break;
    }
    cudaSetDevice(dev_prev);
    if (rc) {
        destroy_server(srv);
        return rc;
    }
    srv->t_open = srv->t_last = std::chrono::steady_clock::now();
    try {
        srv->loop = std::thread(live_loop, srv);
    } catch (...) {
        destroy_server(srv);
        return BMJ_ERR_OOM;
    }
    *out = srv;
    return BMJ_OK;
}

extern "C" int bmj_serve_submit(bmj_server *srv, const int32_t *tokens, int64_t n_tokens,
                                uint32_t p, uint32_t q, int64_t *ticket) {
    if (!srv || !ticket || n_tokens < 0 || (n_tokens > 0 && !tokens)) return BMJ_ERR_INVALID_ARG;
    *ticket = -1;
    if (!sim_valid(srv->idx->sim, p, q)) return BMJ_ERR_INVALID_ARG;
    if (n_tokens == 0) return BMJ_ERR_EMPTY_SET;
    if (n_tokens > srv->max_probe) return BMJ_ERR_TOO_LARGE;
    if (tokens[0] < 0) return BMJ_ERR_NEG_TOKEN;
    for (int64_t k = 1; k < n_tokens; k++)
        if (tokens[k] <= tokens[k - 1]) return BMJ_ERR_UNSORTED;
    LiveQuery lq;
    try {
        lq.tok.assign(tokens, tokens + n_tokens);
    } catch (...) {
        return BMJ_ERR_OOM;
    }
    lq.p = p;
    lq.q = q;
    lq.win = window_of(srv->idx, n_tokens, p, q);
    {
        std::lock_guard<std::mutex> g(srv->mu);
        if (srv->error) return srv->error;
        if (srv->closing) return BMJ_ERR_INVALID_ARG;
        lq.t_submit = std::chrono::steady_clock::now();
        const int64_t t = srv->next_ticket++;
        try {
            srv->queries.emplace(t, std::move(lq));
            srv->pending.push_back(t);
            srv->n_pending.fetch_add(1, std::memory_order_release);
        } catch (...) {
            srv->queries.erase(t);
            return BMJ_ERR_OOM;
        }
        *ticket = t;
    }
    srv->cv_work.notify_one();
    return BMJ_OK;
}

extern "C" int bmj_serve_poll(bmj_server *srv, int64_t ticket, int32_t wait_ms,
                              bmj_id_lists *out, double *latency_ms) {
    if (!srv || !out) return BMJ_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    std::unique_lock<std::mutex> lk(srv->mu);
    const auto deadline = std::chrono::steady_clock::now() +
                          std::chrono::milliseconds(std::max<int32_t>(wait_ms, 0));
    for (;;) {
        auto it = srv->results.find(ticket);
        if (it != srv->results.end()) {
            LiveResult r = std::move(it->second);
            srv->results.erase(it);
            lk.unlock();
            if (r.status) return r.status;
            out->n_queries = 1;
            out->offsets = (int64_t *)malloc(2 * sizeof(int64_t));
            out->ids = (int64_t *)malloc(std::max<size_t>(r.ids.size(), 1) * sizeof(int64_t));
            if (!out->offsets || !out->ids) {
                id_lists_free_impl(out);
                return BMJ_ERR_OOM;
            }
            out->offsets[0] = 0;
            out->offsets[1] = (int64_t)r.ids.size();
            if (!r.ids.empty()) memcpy(out->ids, r.ids.data(), r.ids.size() * sizeof(int64_t));
            if (latency_ms) *latency_ms = r.latency_ms;
            return BMJ_OK;
        }
        if (srv->queries.find(ticket) == srv->queries.end())
            return BMJ_ERR_INVALID_ARG;  // never submitted, or already polled
        if (wait_ms <= 0) return BMJ_PENDING;
        if (srv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout &&
            srv->results.find(ticket) == srv->results.end())
            return BMJ_PENDING;
    }
}

extern "C" int bmj_serve_close(bmj_server *srv, bmj_serve_stats *stats) {
    if (!srv) return BMJ_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        srv->closing = true;
        srv->closing_flag.store(true, std::memory_order_release);
    }
    srv->cv_work.notify_all();
    if (srv->loop.joinable()) srv->loop.join();
    const int err = srv->error;
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        std::vector<double> lat = srv->latencies;
        std::sort(lat.begin(), lat.end());
        auto pct = [&](double f) {
            if (lat.empty()) return 0.0;
            size_t k = (size_t)std::min<double>((double)lat.size() - 1, f * (double)lat.size());
            return lat[k];
        };
        stats->n_queries = (int64_t)lat.size();
        stats->batches = srv->batches;
        stats->window_pairs = srv->window_pairs;
        stats->survivors = srv->survivors;
        stats->results = srv->n_results;
        stats->wall_s = std::chrono::duration<double>(srv->t_last - srv->t_open).count();
        stats->qps = stats->wall_s > 0 ? (double)lat.size() / stats->wall_s : 0.0;
        stats->p50_ms = pct(0.50);
        stats->p99_ms = pct(0.99);
        stats->max_ms = lat.empty() ? 0.0 : lat.back();
    }
    int dev_prev = 0;
    cudaGetDevice(&dev_prev);
    cudaSetDevice(srv->idx->device);
    destroy_server(srv);
    cudaSetDevice(dev_prev);
    cudaGetLastError();
    return err;
}
