// batch.cu -- many independent self-joins in one pass over the GPU.
//
// The jobs arrive as one concatenated CSR collection with job boundaries.
// Every stage runs once for all jobs:
//   validate -> one radix sort by (job, size) -> sorted CSR + bitmaps for each
//   bitmap width in use -> per-job thresholds -> tiles of every job ->
//   ONE persistent Bitmap Filter launch over the work items of all jobs ->
//   ONE verification launch over all survivors -> one result sort.
// Per-job parameters (threshold p/q, bitmap width b, generation method, tile
// shape) live in a device table that the kernels index by job.
//
// b per job is picked by a sampling autotuner (when the caller passes b = 0):
// up to four blocks of 128 rows of every job are filtered at b = 64, 128 and
// 256 with the survivors only counted, and per job
//     cost(b) = window_pairs * t_filter(b) + survivors(b) * t_verify(mean size)
// with survivors(b) scaled from the sample and fixed cost ratios measured on
// a B300 (so the choice is deterministic).  The choice trades filter work
// (growing with b) against verification work (the survivors that a wider
// bitmap removes): the filter/verify split.
//
// The execute stage (filter + verification) enqueues no allocation and no
// host read, so it can be captured into a CUDA graph (opt.use_graph).
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "filter_core.cuh"
#include "host_util.cuh"

namespace bmj {
namespace {

constexpr unsigned kFullMask = 0xffffffffu;

// Rows per lane of the small row tile of each width (the default tile is the
// single join's at b = 64 and 256, kTmaR1 and kTmaR4, and 4 rows at b = 128,
// the batch's measured configuration), the tile classes (three widths, two
// tiles each, every other width, then b = 128 default tiles with the folded
// test) and the counters of a plan.
constexpr int kSmallR1 = 2, kSmallR2 = 1, kSmallR4 = 1;
constexpr int kBatchR2 = 4;
constexpr int kClasses = 8;
constexpr int kCounters = 3 + kClasses;
#ifndef BMJ_SMALL_COST1
#define BMJ_SMALL_COST1 1.3
#endif
#ifndef BMJ_SMALL_COST2
#define BMJ_SMALL_COST2 1.3
#endif
#ifndef BMJ_SMALL_COST4
#define BMJ_SMALL_COST4 1.3
#endif
constexpr double kSmallCost1 = BMJ_SMALL_COST1, kSmallCost2 = BMJ_SMALL_COST2,
                 kSmallCost4 = BMJ_SMALL_COST4;

struct JobDesc {
    const uint64_t *bm;  // bitmap array of the job's width (indexed by global sorted position)
    const uint64_t *bm2; // cascade bitmaps (256 bits) checked before a merge, or null
    int64_t base;        // first sorted position of the job
    int64_t end;         // one past its last sorted position
    int64_t id_base;     // first input position of the job (output ids are local to it)
    int64_t lim_off;     // offset of the job's need/lim tables
    uint32_t p, q;
    int32_t W;
    int32_t tile_rows;
    int32_t chunk_cols;
    int32_t sim;         // similarity function of the threshold p/q
    SimWindow win;       // its length window (Table 2)
    int32_t fold;        // b = 128: the folded 64-bit test before the 128-bit one
};

__device__ __forceinline__ int64_t lower_bound_range(const uint32_t *a, int64_t lo, int64_t hi,
                                                     uint64_t v) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((uint64_t)a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Last k in [0, n) with a[k] <= v.
__device__ __forceinline__ int64_t last_le(const int64_t *a, int64_t n, int64_t v) {
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] <= v) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Sort key of input set x: (job << sbits) | size (jbits + sbits <= 32).
__global__ void k_batch_keys(const uint32_t *__restrict__ sizes, int64_t n,
                             const int64_t *__restrict__ job_sets, int64_t n_jobs, int sbits,
                             uint32_t *__restrict__ keys) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        const int64_t k = last_le(job_sets, n_jobs, x);
        keys[x] = ((uint32_t)k << sbits) | sizes[x];
    }
}

__global__ void k_split_keys(const uint32_t *__restrict__ skey, int64_t n, int sbits,
                             uint32_t *__restrict__ ssz, uint32_t *__restrict__ sjob) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const uint32_t mask = (sbits >= 32) ? 0xffffffffu : ((1u << sbits) - 1u);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        ssz[i] = skey[i] & mask;
        sjob[i] = sbits >= 32 ? 0u : (skey[i] >> sbits);
    }
}

// Output pairs from keys (job << 2*nbits) | (lo << nbits) | hi.
// out[k] = src[idx[k]] for k < m.
__global__ void k_gather_at(const int64_t *__restrict__ src, const int64_t *__restrict__ idx,
                            int64_t m, int64_t *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += stride)
        out[k] = src[idx[k]];
}

__global__ void k_unpack_local(const uint64_t *__restrict__ keys, int64_t n, int nbits,
                               uint32_t *__restrict__ a, uint32_t *__restrict__ b) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const uint64_t mask = (1ull << nbits) - 1ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t k = keys[i];
        a[i] = (uint32_t)((k >> nbits) & mask);
        b[i] = (uint32_t)(k & mask);
    }
}

__global__ void k_batch_tables(int32_t *__restrict__ need, int32_t *__restrict__ lim, int64_t n_s,
                               const uint32_t *__restrict__ jp, const uint32_t *__restrict__ jq,
                               int64_t n_jobs, int sim) {
    const int64_t total = n_s * n_jobs;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += stride) {
        const int64_t k = x / n_s, S = x - k * n_s;
        // e.g. Jaccard: ceil(p*S/(p+q)) (Table 1); Cosine computes it per pair
        const int64_t nd = sim == BMJ_COSINE ? 0 : need_of_sum(sim, jp[k], jq[k], S);
        need[x] = (int32_t)nd;
        lim[x] = (int32_t)(S - 2 * nd);   // Eq. 2 with its floor
    }
}

// Window pairs per job: sum over its sorted rows of (i - j0(i)).
__global__ void k_batch_window(const uint32_t *__restrict__ ssz, const uint32_t *__restrict__ sjob,
                               int64_t n, const JobDesc *__restrict__ jobs,
                               unsigned long long *__restrict__ job_win) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t i = base + threadIdx.x;
        unsigned long long v = 0;
        uint32_t k = 0xffffffffu;
        if (i < n) {
            k = sjob[i];
            const JobDesc &jd = jobs[k];
            const uint64_t low = window_low(ssz[i], jd.win);
            const int64_t j0 = lower_bound_range(ssz, jd.base, i, low);
            v = (unsigned long long)(i - j0);
        }
        const uint32_t k0 = __shfl_sync(kFullMask, k, 0);
        if (__all_sync(kFullMask, k == k0)) {
            for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFullMask, v, d);
            if (lane == 0 && k0 != 0xffffffffu && v) atomicAdd(&job_win[k0], v);
        } else if (k != 0xffffffffu && v) {
            atomicAdd(&job_win[k], v);
        }
    }
}

// Tile descriptors from (job, local tile) pairs.
__global__ void k_batch_tiles(const uint32_t *__restrict__ ssz, const JobDesc *__restrict__ jobs,
                              const int32_t *__restrict__ tl_job, const int64_t *__restrict__ tl_local,
                              int64_t n_tiles, int64_t *__restrict__ tile_i0,
                              int64_t *__restrict__ tile_c0, int64_t *__restrict__ tile_items,
                              unsigned long long *__restrict__ tile_win) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += stride) {
        const JobDesc &jd = jobs[tl_job[t]];
        const int64_t i0 = jd.base + tl_local[t] * jd.tile_rows;
        const uint64_t low = window_low(ssz[i0], jd.win);
        const int64_t c0 = lower_bound_range(ssz, jd.base, jd.end, low);  // j0 of the first row
        const int64_t i_end = min(i0 + (int64_t)jd.tile_rows, jd.end);
        const int64_t c_end = i_end - 1;
        const int64_t cols = c_end - c0;
        tile_i0[t] = i0;
        tile_c0[t] = c0;
        tile_items[t] = cols > 0 ? (cols + jd.chunk_cols - 1) / jd.chunk_cols : 0;
        if (tile_win) {
            unsigned long long w = 0;
            for (int64_t i = i0; i < i_end; i++) {
                const uint64_t li = window_low(ssz[i], jd.win);
                w += (unsigned long long)(i - lower_bound_range(ssz, jd.base, i, li));
            }
            tile_win[t] = w;
        }
    }
}

// (job, local tile) of every tile of every job, jobs taken in the order
// `order` (grouped by bitmap width) with first tiles job_tile0 in that order.
__global__ void k_enumerate_tiles(const int64_t *__restrict__ job_tile0,
                                  const int32_t *__restrict__ order, int64_t n_jobs,
                                  int64_t n_tiles, int32_t *__restrict__ tl_job,
                                  int64_t *__restrict__ tl_local) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += stride) {
        const int64_t pos = last_le(job_tile0, n_jobs, t);
        tl_job[t] = order[pos];
        tl_local[t] = t - job_tile0[pos];
    }
}

struct BatchFilterArgs {
    const JobDesc *jobs;
    const uint32_t *ssz;
    const int32_t *lim;
    const int32_t *tile_job;
    const int64_t *tile_i0;
    const int64_t *tile_c0;
    const int64_t *tile_item_off;  // [n_tiles + 1]
    int64_t n_tiles;
    uint2 *queue;
    unsigned long long *qcount;
    unsigned long long *job_surv;  // per-job survivor counters
    int64_t qcap;
    int *err;                      // set when a bounded wait on a copy gave up
    int sim;                       // similarity function of every job
};

// The Bitmap Filter over the work items of every job of one bitmap width:
// tiles [t0, t1) (the jobs of that width are contiguous in the tile list),
// items pulled from a per-class counter.  Columns are staged by TMA.
// Rows per lane that take the width's second popcount form in the batched
// filter, as in the single join: one row in eight counted on the ALU at b = 64
// (249.7 against 251.6 ms for the 512-job batch), two rows in four reduced to
// 5 POPC at b = 256 (242.8 against 243.3 ms); in tiles of the default height
// only (a small tile keeps every row on the first form).
template <int W, int R>
constexpr int kBatchAltR = (W == 1 && R >= 8) || (W == 4 && R >= 4) ? kAltRows<W> : 0;

// Resident 4-warp blocks per SM of the batched filter at b = 64: eight (64
// registers, 8 bytes spilled) ran the 512-job execute stage in 248.2 ms against
// 249.6 ms with seven.  At b = 256 seven (72 registers): eight, within 64
// registers, took it from 242.8 to 250.1 ms.
// The batched b = 128 filter takes the folded test (as the single join does) in
// jobs whose sampled 64-bit survivor rate is at most this (from the autotuner;
// every b = 128 job of default-height tiles when the width is given).
#ifndef BMJ_BATCH_FOLD_RATE
#define BMJ_BATCH_FOLD_RATE 2e-3
#endif
constexpr double kBatchFoldMaxRate64 = BMJ_BATCH_FOLD_RATE;

#ifndef BMJ_BATCH_W1_BLOCKS
#define BMJ_BATCH_W1_BLOCKS 8
#endif
#ifndef BMJ_BATCH_W4_BLOCKS
#define BMJ_BATCH_W4_BLOCKS 7
#endif

template <int W, int R, int CS, bool kCos, bool kFold>
__global__ void __launch_bounds__(128, kCos ? 6 : W == 1 ? BMJ_BATCH_W1_BLOCKS : W == 4 ? BMJ_BATCH_W4_BLOCKS : 7)
    k_filter_batch_w(const BatchFilterArgs a, int64_t t0, int64_t t1,
                     unsigned long long *counter) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    StageState stg;
    init_stage(stg, smem + (threadIdx.x >> 5) * ColStage<W, CS>::kWarpBytes,
               ColStage<W, CS>::kStageOff);  // default bounded waits
    const int64_t ibase = a.tile_item_off[t0], iend = a.tile_item_off[t1];
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = (unsigned long long)ibase + atomicAdd(counter, 1ull);
        item = __shfl_sync(kFullMask, item, 0);
        if ((int64_t)item >= iend) return;
        const int64_t t = t0 + find_tile(a.tile_item_off + t0, t1 - t0, item);
        const int32_t k = a.tile_job[t];
        const JobDesc jd = a.jobs[k];
        const int64_t chunk = (int64_t)item - a.tile_item_off[t];
        const int64_t i0 = a.tile_i0[t];
        const int64_t c0 = a.tile_c0[t] + chunk * jd.chunk_cols;
        const int64_t c_end = min(i0 + (int64_t)jd.tile_rows, jd.end) - 1;
        const int64_t c1 = min(c0 + (int64_t)jd.chunk_cols, c_end);
        const SurvivorSink sink{a.queue, a.qcount, a.job_surv ? &a.job_surv[k] : nullptr, a.qcap};
        const SimArgs sa{jd.win, jd.p, jd.q};
        filter_item_tma<W, R, CS, kBatchAltR<W, R>, kCos, false, kFold>(
            jd.bm, a.ssz, a.lim + jd.lim_off, jd.end, i0, c0, c1, sa, sink, stg);
        if (!stg.ok) {
            drain_stage(stg);
            if (lane == 0) atomicOr(a.err, 1);
            return;
        }
    }
}

// Other widths: one row per lane, columns read from memory.
__global__ void __launch_bounds__(256) k_filter_batch_generic(const BatchFilterArgs a, int64_t t0,
                                                               int64_t t1,
                                                               unsigned long long *counter) {
    const int lane = threadIdx.x & 31;
    const int64_t ibase = a.tile_item_off[t0], iend = a.tile_item_off[t1];
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = (unsigned long long)ibase + atomicAdd(counter, 1ull);
        item = __shfl_sync(kFullMask, item, 0);
        if ((int64_t)item >= iend) return;
        const int64_t t = t0 + find_tile(a.tile_item_off + t0, t1 - t0, item);
        const int32_t k = a.tile_job[t];
        const JobDesc jd = a.jobs[k];
        const int64_t chunk = (int64_t)item - a.tile_item_off[t];
        const int64_t i0 = a.tile_i0[t];
        const int64_t c0 = a.tile_c0[t] + chunk * jd.chunk_cols;
        const int64_t c_end = min(i0 + (int64_t)jd.tile_rows, jd.end) - 1;
        const int64_t c1 = min(c0 + (int64_t)jd.chunk_cols, c_end);
        const SurvivorSink sink{a.queue, a.qcount, a.job_surv ? &a.job_surv[k] : nullptr, a.qcap};
        const SimArgs sa{jd.win, jd.p, jd.q};
        if (jd.sim == BMJ_COSINE)
            filter_item_generic<true>(jd.bm, a.ssz, a.lim + jd.lim_off, jd.end, i0, c0, c1, sa,
                                      jd.W, sink);
        else
            filter_item_generic<false>(jd.bm, a.ssz, a.lim + jd.lim_off, jd.end, i0, c0, c1, sa,
                                       jd.W, sink);
    }
}

// Verification of all survivors (count read on the device); similar pairs
// become keys (job << 2*nbits) | (lo << nbits) | hi in job-local ids.
__global__ void __launch_bounds__(256)
    k_verify_batch(const uint2 *__restrict__ queue, const unsigned long long *__restrict__ n_surv_dev,
                   int64_t cap, const int64_t *__restrict__ soff, const int32_t *__restrict__ stok,
                   const uint32_t *__restrict__ ssz, const uint32_t *__restrict__ sjob,
                   const uint32_t *__restrict__ perm, const JobDesc *__restrict__ jobs,
                   const int32_t *__restrict__ need, const int32_t *__restrict__ lim,
                   uint64_t *__restrict__ keys, unsigned long long *__restrict__ rcount, int nbits) {
    const int lane = threadIdx.x & 31;
    const int64_t n_surv = min((int64_t)*n_surv_dev, cap);
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (int64_t base = gw * 32; base < n_surv; base += warps * 32) {
        const int64_t idx = base + lane;
        bool similar = false;
        uint64_t key = 0;
        if (idx < n_surv) {
            const uint2 pr = queue[idx];
            const uint32_t k = sjob[pr.x];
            const JobDesc &jd = jobs[k];
            const uint32_t si = ssz[pr.x], sj = ssz[pr.y];
            const bool cosine = jd.sim == BMJ_COSINE;
            int nd = cosine ? (int)cosine_need(jd.p, jd.q, si, sj) : need[jd.lim_off + si + sj];
            if (jd.bm2) {  // cascade: Eq. 2 again with the 256-bit bitmaps (sound for any b)
                const uint64_t *r2 = jd.bm2 + (int64_t)pr.x * 4;
                const uint64_t *c2 = jd.bm2 + (int64_t)pr.y * 4;
                int h2 = 0;
#pragma unroll
                for (int w = 0; w < 4; w++) h2 += __popcll(r2[w] ^ c2[w]);
                const int l2 = cosine ? (int)si + (int)sj - 2 * nd : lim[jd.lim_off + si + sj];
                if (h2 > l2) nd = 0x7fffffff;  // cannot reach the threshold
            }
            const int32_t *x = stok + soff[pr.x];
            const int32_t *y = stok + soff[pr.y];
            int a = 0, b = 0, o = 0;
            const int na = (int)si, nb = (int)sj;
            while (a < na && b < nb) {
                if (o + min(na - a, nb - b) < nd) break;
                const int32_t xa = x[a], yb = y[b];
                o += (xa == yb);
                a += (xa <= yb);
                b += (yb <= xa);
                if (o >= nd) break;
            }
            similar = o >= nd;
            if (similar) {
                const uint64_t u = (uint64_t)((int64_t)perm[pr.x] - jd.id_base);
                const uint64_t v = (uint64_t)((int64_t)perm[pr.y] - jd.id_base);
                const uint64_t lo = u < v ? u : v, hi = u < v ? v : u;
                key = ((uint64_t)k << (2 * nbits)) | (lo << nbits) | hi;
            }
        }
        const unsigned ball = __ballot_sync(kFullMask, similar);
        if (ball) {
            unsigned long long off = 0;
            if (lane == 0) off = atomicAdd(rcount, (unsigned long long)__popc(ball));
            off = __shfl_sync(kFullMask, off, 0);
            if (similar) keys[off + __popc(ball & ((1u << lane) - 1u))] = key;
        }
    }
}

// First result of every job in the sorted keys.
__global__ void k_job_bounds(const uint64_t *__restrict__ keys, int64_t n, int64_t n_jobs,
                             int shift, int64_t *__restrict__ bounds) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= n_jobs; k += stride) {
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)(keys[mid] >> shift) < k) lo = mid + 1;
            else hi = mid;
        }
        bounds[k] = lo;
    }
}

unsigned grid_of(int64_t n, int threads, int64_t cap = 148 * 32) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

// ----------------------------------------------------------------------------
// Host side
// ----------------------------------------------------------------------------
struct Plan {
    // sorted collection
    int64_t n = 0, n_jobs = 0;
    uint32_t *ssz = nullptr, *sjob = nullptr, *perm = nullptr;
    int64_t *soff = nullptr;
    int32_t *stok = nullptr;
    int64_t n_s = 0;
    int sim = BMJ_JACCARD;
    int32_t *need = nullptr, *lim = nullptr;
    JobDesc *jobs_dev = nullptr;
    std::vector<JobDesc> jobs;
    // tiles / items
    int64_t n_tiles = 0;
    int32_t *tile_job = nullptr;
    int64_t *tile_i0 = nullptr, *tile_c0 = nullptr, *tile_off = nullptr;
    // tile ranges of the tile classes (tile_class: b = 64, 128, 256 each with its
    // default and its small row tile, then other widths), in tile order
    int64_t class_t0[kClasses] = {0}, class_t1[kClasses] = {0};
    // counters: [1] survivors, [2] results, [3 + c] item counter of class c
    unsigned long long *ctr = nullptr;
    unsigned long long *job_surv = nullptr;
    int *err = nullptr;
    uint2 *queue = nullptr;
    int64_t qcap = 0;
    uint64_t *keys = nullptr;
    int nbits = 1;
};

int build_tiles(Plan &P, const std::vector<int32_t> &h_job, const std::vector<int64_t> &h_local,
                bool enumerate_all, const std::vector<int64_t> &job_tile0,
                const std::vector<int32_t> &order, Arena &A, cudaStream_t s,
                unsigned long long **tile_win_out) {
    const int64_t T = enumerate_all ? job_tile0.back() : (int64_t)h_job.size();
    P.n_tiles = T;
    int32_t *tl_job = nullptr;
    int64_t *tl_local = nullptr;
    int st = A.alloc(&tl_job, (size_t)std::max<int64_t>(T, 1));
    if (!st) st = A.alloc(&tl_local, (size_t)std::max<int64_t>(T, 1));
    if (!st) st = A.alloc(&P.tile_i0, (size_t)std::max<int64_t>(T, 1));
    if (!st) st = A.alloc(&P.tile_c0, (size_t)std::max<int64_t>(T, 1));
    if (!st) st = A.alloc(&P.tile_off, (size_t)T + 1);
    if (st) return st;
    if (T == 0) {
        BMJ_CHECK(cudaMemsetAsync(P.tile_off, 0, sizeof(int64_t), s));
        P.tile_job = tl_job;
        return BMJ_OK;
    }
    if (enumerate_all) {
        int64_t *jt0 = nullptr;
        int32_t *ord = nullptr;
        st = A.alloc(&jt0, job_tile0.size());
        if (!st) st = A.alloc(&ord, order.size());
        if (st) return st;
        BMJ_CHECK(cudaMemcpyAsync(jt0, job_tile0.data(), job_tile0.size() * sizeof(int64_t),
                                  cudaMemcpyHostToDevice, s));
        BMJ_CHECK(cudaMemcpyAsync(ord, order.data(), order.size() * sizeof(int32_t),
                                  cudaMemcpyHostToDevice, s));
        BMJ_LAUNCH(k_enumerate_tiles, grid_of(T, 256), 256, 0, s, jt0, ord,
                   (int64_t)job_tile0.size() - 1, T, tl_job, tl_local);
    } else {
        BMJ_CHECK(cudaMemcpyAsync(tl_job, h_job.data(), T * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        BMJ_CHECK(cudaMemcpyAsync(tl_local, h_local.data(), T * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    }
    unsigned long long *tile_win = nullptr;
    if (tile_win_out) {
        st = A.alloc(&tile_win, (size_t)T);
        if (st) return st;
        *tile_win_out = tile_win;
    }
    BMJ_LAUNCH(k_batch_tiles, grid_of(T, 128), 128, 0, s, P.ssz, P.jobs_dev, tl_job, tl_local, T,
               P.tile_i0, P.tile_c0, P.tile_off, tile_win);
    st = exclusive_scan_i64(P.tile_off, P.tile_off, T, P.tile_off + T, A, s);
    P.tile_job = tl_job;
    return st;
}

int upload_jobs(Plan &P, Arena &A, cudaStream_t s) {
    if (!P.jobs_dev) {
        int st = A.alloc(&P.jobs_dev, (size_t)P.n_jobs);
        if (st) return st;
    }
    BMJ_CHECK(cudaMemcpyAsync(P.jobs_dev, P.jobs.data(), P.n_jobs * sizeof(JobDesc),
                              cudaMemcpyHostToDevice, s));
    return BMJ_OK;
}

// Tile class of a job: its width and its rows per lane (the default of the
// single join, or the small tile for jobs whose diagonal tiles would waste a
// large share of their window; see the tuner).
int tile_class(int W, int tile_rows, int fold = 0) {
    switch (W) {
        case 1: return tile_rows == 32 * kTmaR1 ? 0 : 1;
        case 2: return tile_rows == 32 * kBatchR2 ? (fold ? 7 : 2) : 3;
        case 4: return tile_rows == 32 * kTmaR4 ? 4 : 5;
        default: return 6;
    }
}
int default_tile_rows(int W) {
    return W == 1 ? 32 * kTmaR1 : W == 2 ? 32 * kBatchR2 : W == 4 ? 32 * kTmaR4 : 32;
}
int small_tile_rows(int W) {
    return W == 1 ? 32 * kSmallR1 : W == 2 ? 32 * kSmallR2 : W == 4 ? 32 * kSmallR4 : 32;
}
// Filter time per evaluated pair in the small tile relative to the default
// tile of the width (measured on a B300 with large jobs forced to each tile).
double small_tile_cost(int W) { return W == 1 ? kSmallCost1 : W == 2 ? kSmallCost2 : kSmallCost4; }

template <int W, int R, int CS, bool kCos, bool kFold>
int launch_class_c(const BatchFilterArgs &fa, int64_t t0, int64_t t1, unsigned long long *counter,
                   int sms, cudaStream_t s) {
    const int smem = 4 * ColStage<W, CS>::kWarpBytes;
    int per_sm = 0;
    BMJ_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, k_filter_batch_w<W, R, CS, kCos, kFold>, 128, smem));
    if (per_sm < 1) per_sm = 1;
    BMJ_LAUNCH((k_filter_batch_w<W, R, CS, kCos, kFold>), (unsigned)(sms * per_sm), 128, smem, s,
               fa, t0, t1, counter);
    return BMJ_OK;
}

template <int W, int R, int CS, bool kFold = false>
int launch_class(const BatchFilterArgs &fa, int64_t t0, int64_t t1, unsigned long long *counter,
                 int sms, cudaStream_t s) {
    return fa.sim == BMJ_COSINE ? launch_class_c<W, R, CS, true, kFold>(fa, t0, t1, counter, sms, s)
                                : launch_class_c<W, R, CS, false, kFold>(fa, t0, t1, counter, sms, s);
}

// Filter over the planned items into the plan's queue (cap may be 0: count
// only): one persistent launch per width class present.
int enqueue_filter(const Plan &P, int sms, cudaStream_t s) {
    BatchFilterArgs fa;
    fa.sim = P.sim;
    fa.jobs = P.jobs_dev;
    fa.ssz = P.ssz;
    fa.lim = P.lim;
    fa.tile_job = P.tile_job;
    fa.tile_i0 = P.tile_i0;
    fa.tile_c0 = P.tile_c0;
    fa.tile_item_off = P.tile_off;
    fa.n_tiles = P.n_tiles;
    fa.queue = P.queue;
    fa.qcount = &P.ctr[1];
    fa.job_surv = P.job_surv;
    fa.qcap = P.qcap;
    fa.err = P.err;
    for (int c = 0; c < kClasses; c++) {
        const int64_t t0 = P.class_t0[c], t1 = P.class_t1[c];
        if (t1 <= t0) continue;
        unsigned long long *counter = &P.ctr[3 + c];
        int st = BMJ_OK;
        switch (c) {
            case 0: st = launch_class<1, kTmaR1, kTmaCS1>(fa, t0, t1, counter, sms, s); break;
            case 1: st = launch_class<1, kSmallR1, kTmaCS1>(fa, t0, t1, counter, sms, s); break;
            case 2: st = launch_class<2, kBatchR2, kTmaCS2>(fa, t0, t1, counter, sms, s); break;
            case 3: st = launch_class<2, kSmallR2, kTmaCS2>(fa, t0, t1, counter, sms, s); break;
            case 4: st = launch_class<4, kTmaR4, kTmaCS4>(fa, t0, t1, counter, sms, s); break;
            case 5: st = launch_class<4, kSmallR4, kTmaCS4>(fa, t0, t1, counter, sms, s); break;
            case 7: st = launch_class<2, kBatchR2, kTmaCS2, true>(fa, t0, t1, counter, sms, s); break;
            default: {
                int per_sm = 0;
                BMJ_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_filter_batch_generic,
                                                                        256, 0));
                if (per_sm < 1) per_sm = 1;
                BMJ_LAUNCH(k_filter_batch_generic, (unsigned)(sms * per_sm), 256, 0, s, fa, t0, t1,
                           counter);
            }
        }
        if (st) return st;
    }
    return BMJ_OK;
}

// The execute stage: clear counters, filter every job, verify every survivor.
// No allocation and no host read: capturable into a CUDA graph.
int enqueue_execute(const Plan &P, int sms, cudaStream_t s) {
    BMJ_CHECK(cudaMemsetAsync(P.ctr, 0, kCounters * sizeof(unsigned long long), s));
    BMJ_CHECK(cudaMemsetAsync(P.job_surv, 0, P.n_jobs * sizeof(unsigned long long), s));
    int st = enqueue_filter(P, sms, s);
    if (st) return st;
    BMJ_LAUNCH(k_verify_batch, (unsigned)(sms * 8), 256, 0, s, P.queue, &P.ctr[1], P.qcap, P.soff,
               P.stok, P.ssz, P.sjob, P.perm, P.jobs_dev, P.need, P.lim, P.keys, &P.ctr[2], P.nbits);
    return BMJ_OK;
}

int run_execute(const Plan &P, int sms, cudaStream_t s, bool use_graph, int *graphed) {
    NvtxRange nv("bmj.batch_execute");
    *graphed = 0;
    if (!use_graph) return enqueue_execute(P, sms, s);
    cudaStream_t cs = nullptr;
    BMJ_CHECK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    int st = BMJ_OK;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        st = enqueue_execute(P, sms, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (!st && e2 != cudaSuccess) st = status_of(e2);
    } else {
        st = status_of(e);
    }
    if (!st && cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) st = BMJ_ERR_CUDA;
    if (!st) {
        // The graph runs on the caller's stream, ordered after the planning work.
        if (cudaGraphLaunch(ge, s) != cudaSuccess) st = BMJ_ERR_CUDA;
    }
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    cudaGetLastError();
    if (!st) *graphed = 1;
    return st;
}

int batch_impl(const bmj_collection *coll, int64_t n_jobs, const int64_t *job_sets, int sim,
               const uint32_t *hp, const uint32_t *hq, const bmj_options &o, bmj_pairs *outs,
               bmj_stats *job_stats, bmj_batch_stats *bst) {
    NvtxRange nv_call("bmj_self_join_batch");
    cudaStream_t s = (cudaStream_t)o.stream;
    const int64_t launches0 = launches();
    int dev = 0;
    BMJ_CHECK(cudaGetDevice(&dev));
    retain_pool_memory(dev);
    const int sms = num_sms(dev);
    bmj_batch_stats bs;
    memset(&bs, 0, sizeof(bs));
    bs.n_jobs = n_jobs;
    Events ev;
    int st = ev.init();
    if (st) return st;
    Arena A(s);
    BMJ_CHECK(cudaEventRecord(ev.e[0], s));
    DevColl d;
    st = stage_collection(coll, A, s, &d);
    if (st) return st;
    Plan P;
    P.n = d.n;
    P.n_jobs = n_jobs;
    P.sim = sim;
    const int64_t n = d.n;
    std::vector<int64_t> result_bounds(n_jobs + 1, 0);
    std::vector<uint32_t> res_a, res_b;
    std::vector<int> job_b(n_jobs, o.b > 0 ? o.b : 64), job_method(n_jobs, o.method);
    std::vector<char> job_small(n_jobs, 0);  // 1: the job's tiles are the small row tile
    std::vector<char> job_fold(n_jobs, 1);   // b = 128 jobs: 1 = the folded test first
    for (int64_t k = 0; k < n_jobs; k++)
        if (o.method == BMJ_COMBINED) job_method[k] = combined_method(sim, hp[k], hq[k]);
    std::vector<unsigned long long> job_win(n_jobs, 0), job_sv(n_jobs, 0);
    int64_t max_job = 0;
    for (int64_t k = 0; k < n_jobs; k++) max_job = std::max(max_job, job_sets[k + 1] - job_sets[k]);
    P.nbits = max_job > 1 ? bit_length((uint64_t)(max_job - 1)) : 1;
    const int jbits = n_jobs > 1 ? bit_length((uint64_t)(n_jobs - 1)) : 1;
    if (jbits + 2 * P.nbits > 64) return BMJ_ERR_TOO_LARGE;

    if (n >= 2) {
        uint32_t *sizes = nullptr, *ids = nullptr;
        int max_size = 0;
        st = validate(d, o.validate != 0, A, s, &sizes, &ids, &max_size);
        if (st) return st;
        // ---- one sort by (job, size), ties by input position ----
        const int sbits = std::max(1, bit_length((uint64_t)max_size));
        if (sbits + jbits > 32) return BMJ_ERR_TOO_LARGE;
        int64_t *js_dev = nullptr;
        uint32_t *keys_in = nullptr, *skey = nullptr;
        st = A.alloc(&js_dev, (size_t)n_jobs + 1);
        if (!st) st = A.alloc(&keys_in, (size_t)n);
        if (!st) st = A.alloc(&skey, (size_t)n);
        if (!st) st = A.alloc(&P.ssz, (size_t)n + 4);  // padded: TMA chunks may read 3 past the end
        if (!st) st = A.alloc(&P.sjob, (size_t)n);
        if (!st) st = A.alloc(&P.perm, (size_t)n);
        if (!st) st = A.alloc(&P.soff, (size_t)n + 1);
        if (!st) st = A.alloc(&P.stok, (size_t)d.ntok);
        if (st) return st;
        BMJ_CHECK(cudaMemcpyAsync(js_dev, job_sets, (n_jobs + 1) * sizeof(int64_t),
                                  cudaMemcpyHostToDevice, s));
        BMJ_LAUNCH(k_batch_keys, grid_of(n, 256), 256, 0, s, sizes, n, js_dev, n_jobs, sbits, keys_in);
        st = radix_sort_u32_pairs(keys_in, ids, skey, P.perm, n, jbits + sbits, A, s);
        if (st) return st;
        BMJ_LAUNCH(k_split_keys, grid_of(n, 256), 256, 0, s, skey, n, sbits, P.ssz, P.sjob);
        BMJ_CHECK(cudaMemsetAsync(P.ssz + n, 0, 4 * sizeof(uint32_t), s));
        st = launch_widen(P.ssz, P.soff, n, s);
        if (!st) st = exclusive_scan_i64(P.soff, P.soff, n, P.soff + n, A, s);
        if (st) return st;

        // ---- thresholds per job ----
        P.n_s = 2 * (int64_t)max_size + 1;
        uint32_t *jp = nullptr, *jq = nullptr;
        st = A.alloc(&P.need, (size_t)(P.n_s * n_jobs));
        if (!st) st = A.alloc(&P.lim, (size_t)(P.n_s * n_jobs));
        if (!st) st = A.alloc(&jp, (size_t)n_jobs);
        if (!st) st = A.alloc(&jq, (size_t)n_jobs);
        if (!st) st = A.alloc(&P.ctr, kCounters);
        if (!st) st = A.alloc(&P.job_surv, (size_t)n_jobs);
        if (!st) st = A.alloc(&P.err, 1);
        if (st) return st;
        BMJ_CHECK(cudaMemsetAsync(P.err, 0, sizeof(int), s));
        BMJ_CHECK(cudaMemcpyAsync(jp, hp, n_jobs * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
        BMJ_CHECK(cudaMemcpyAsync(jq, hq, n_jobs * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
        BMJ_LAUNCH(k_batch_tables, grid_of(P.n_s * n_jobs, 256), 256, 0, s, P.need, P.lim, P.n_s, jp,
                   jq, n_jobs, sim);

        // ---- bitmaps: one array per (b, method) in use ----
        const bool tune = o.b <= 0;
        const bool cascade = o.cascade_b != -1;
        std::vector<int> widths = tune ? std::vector<int>{64, 128, 256} : std::vector<int>{o.b};
        if (cascade && !tune && o.b < 256) widths.push_back(256);
        std::vector<int> methods;
        for (int64_t k = 0; k < n_jobs; k++)
            if (std::find(methods.begin(), methods.end(), job_method[k]) == methods.end())
                methods.push_back(job_method[k]);
        uint64_t *bms[3][4] = {{nullptr}};
        for (size_t wi = 0; wi < widths.size(); wi++)
            for (int m : methods) {
                const int W = widths[wi] / 64;
                st = A.alloc(&bms[wi][m], (size_t)(n + 4) * W);
                if (st) return st;
                BMJ_CHECK(cudaMemsetAsync(bms[wi][m] + (size_t)n * W, 0, 4 * W * sizeof(uint64_t), s));
            }
        bool gathered = false;
        for (int m : methods) {
            uint64_t *w64 = nullptr, *w128 = nullptr, *w256 = nullptr;
            for (size_t wi = 0; wi < widths.size(); wi++) {
                if (widths[wi] == 64) w64 = bms[wi][m];
                else if (widths[wi] == 128) w128 = bms[wi][m];
                else if (widths[wi] == 256) w256 = bms[wi][m];
            }
            if ((m == BMJ_XOR || m == BMJ_SET) && (w64 || w128 || w256)) {
                // one pass over the tokens for every power-of-two width up to 256
                st = gathered ? launch_build_multi(nullptr, P.soff, P.stok, nullptr, nullptr, n, m,
                                                   w64, w128, w256, s)
                              : launch_build_multi(P.perm, d.off, d.tok, P.soff, P.stok, n, m, w64,
                                                   w128, w256, s);
                if (st) return st;
                gathered = true;
            }
            for (size_t wi = 0; wi < widths.size(); wi++) {
                const bool done = (m == BMJ_XOR || m == BMJ_SET) &&
                                  (widths[wi] == 64 || widths[wi] == 128 || widths[wi] == 256);
                if (done) continue;
                st = gathered ? launch_gather_build(nullptr, P.soff, P.stok, nullptr, nullptr,
                                                    bms[wi][m], n, widths[wi], m, s)
                              : launch_gather_build(P.perm, d.off, d.tok, P.soff, P.stok, bms[wi][m],
                                                    n, widths[wi], m, s);
                if (st) return st;
                gathered = true;
            }
        }

        // ---- job table ----
        P.jobs.assign(n_jobs, JobDesc());
        auto set_jobs = [&](const std::vector<int> &jb) {
            for (int64_t k = 0; k < n_jobs; k++) {
                JobDesc &jd = P.jobs[k];
                size_t wi = 0;
                while (widths[wi] != jb[k]) wi++;
                jd.bm = bms[wi][job_method[k]];
                jd.bm2 = nullptr;
                if (cascade && jb[k] < 256) {
                    size_t w2 = 0;
                    while (widths[w2] != 256) w2++;
                    jd.bm2 = bms[w2][job_method[k]];
                }
                jd.base = job_sets[k];
                jd.end = job_sets[k + 1];
                jd.id_base = job_sets[k];
                jd.lim_off = k * P.n_s;
                jd.p = hp[k];
                jd.q = hq[k];
                jd.sim = sim;
                jd.win = sim_window(sim, hp[k], hq[k]);
                jd.W = jb[k] / 64;
                jd.tile_rows = job_small[k] ? small_tile_rows(jd.W) : default_tile_rows(jd.W);
                jd.chunk_cols = 4096;
                jd.fold = jd.W == 2 && !job_small[k] && job_fold[k] ? 1 : 0;
            }
        };
        set_jobs(job_b);
        st = upload_jobs(P, A, s);
        if (st) return st;
        {
            unsigned long long *jw = nullptr;
            st = A.alloc(&jw, (size_t)n_jobs);
            if (st) return st;
            BMJ_CHECK(cudaMemsetAsync(jw, 0, n_jobs * sizeof(unsigned long long), s));
            BMJ_LAUNCH(k_batch_window, grid_of(n, 256), 256, 0, s, P.ssz, P.sjob, n, P.jobs_dev, jw);
            BMJ_CHECK(cudaMemcpyAsync(job_win.data(), jw, n_jobs * sizeof(unsigned long long),
                                      cudaMemcpyDeviceToHost, s));
        }
        BMJ_CHECK(cudaStreamSynchronize(s));
        BMJ_CHECK(cudaEventRecord(ev.e[1], s));
        unsigned long long total_win = 0;
        for (auto w : job_win) total_win += w;
        double est_surv = -1.0;

        // ---- autotuner: sampled filter at each width ----
        // The sample is up to 4 blocks of 128 rows per job (evenly spaced),
        // covered by the tiles of each width, so every width sees the same pairs.
        if (tune && total_win > 0) {
            bs.tuned = 1;
            std::vector<int64_t> s_rows_job, s_rows_r0;
            for (int64_t k = 0; k < n_jobs; k++) {
                const int64_t nk = job_sets[k + 1] - job_sets[k];
                if (nk < 2) continue;
                const int64_t blocks = (nk + 127) / 128;
                const int64_t pick = std::min<int64_t>(blocks, 4);
                for (int64_t j = 0; j < pick; j++) {
                    s_rows_job.push_back(k);
                    s_rows_r0.push_back(128 * (((2 * j + 1) * blocks) / (2 * pick)));
                }
            }
            auto sample_tiles = [&](int width, std::vector<int32_t> &tj, std::vector<int64_t> &tl) {
                const int wq = width / 64;
                const int tr = default_tile_rows(wq);
                tj.clear();
                tl.clear();
                for (size_t r = 0; r < s_rows_job.size(); r++) {
                    const int64_t k = s_rows_job[r];
                    const int64_t nk = job_sets[k + 1] - job_sets[k];
                    int64_t last = -1;
                    for (int64_t row = s_rows_r0[r]; row < s_rows_r0[r] + 128 && row < nk; row++) {
                        if (row / tr == last) continue;
                        last = row / tr;
                        tj.push_back((int32_t)k);
                        tl.push_back(last);
                    }
                }
            };
            std::vector<std::vector<double>> samp_win(widths.size(), std::vector<double>(n_jobs, 0.0));
            std::vector<std::vector<unsigned long long>> samp_surv(widths.size(),
                                                                   std::vector<unsigned long long>(n_jobs));
            P.queue = nullptr;
            P.qcap = 0;
            std::vector<int32_t> tj;
            std::vector<int64_t> tl;
            for (size_t wi = 0; wi < widths.size(); wi++) {
                std::vector<int> jb(n_jobs, widths[wi]);
                set_jobs(jb);
                st = upload_jobs(P, A, s);
                if (st) return st;
                sample_tiles(widths[wi], tj, tl);
                unsigned long long *twin = nullptr;
                st = build_tiles(P, tj, tl, false, {}, {}, A, s, &twin);
                for (int c = 0; c < kClasses; c++) P.class_t0[c] = P.class_t1[c] = 0;
                P.class_t1[tile_class(widths[wi] / 64, default_tile_rows(widths[wi] / 64))] =
                    P.n_tiles;
                if (st) return st;
                std::vector<unsigned long long> h_twin(P.n_tiles);
                BMJ_CHECK(cudaMemcpyAsync(h_twin.data(), twin, P.n_tiles * sizeof(unsigned long long),
                                          cudaMemcpyDeviceToHost, s));
                BMJ_CHECK(cudaMemsetAsync(P.ctr, 0, kCounters * sizeof(unsigned long long), s));
                BMJ_CHECK(cudaMemsetAsync(P.job_surv, 0, n_jobs * sizeof(unsigned long long), s));
                st = enqueue_filter(P, sms, s);
                if (st) return st;
                BMJ_CHECK(cudaMemcpyAsync(samp_surv[wi].data(), P.job_surv,
                                          n_jobs * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
                BMJ_CHECK(cudaStreamSynchronize(s));
                for (int64_t t = 0; t < P.n_tiles; t++) samp_win[wi][tj[t]] += (double)h_twin[t];
            }
            // Deterministic cost model (the sampled survivor counts are exact
            // counts; the costs below are fixed ratios measured on a B300):
            //   filter, per window pair, relative to b = 64:  1, 1.55, 2.55
            //   verification, per survivor: 57 window-pair units at a mean
            //   set size of 12, growing with the merge length (mean size).
            std::vector<double> mean_size(n_jobs, 0.0);
            {
                // each job's first token position in the sorted CSR, gathered at once
                std::vector<int64_t> h_soff(n_jobs + 1);
                int64_t *jsd = nullptr, *jso = nullptr;
                st = A.alloc(&jsd, (size_t)n_jobs + 1);
                if (!st) st = A.alloc(&jso, (size_t)n_jobs + 1);
                if (st) return st;
                BMJ_CHECK(cudaMemcpyAsync(jsd, job_sets, (n_jobs + 1) * sizeof(int64_t),
                                          cudaMemcpyHostToDevice, s));
                BMJ_LAUNCH(k_gather_at, grid_of(n_jobs + 1, 256), 256, 0, s, P.soff, jsd,
                           n_jobs + 1, jso);
                BMJ_CHECK(cudaMemcpyAsync(h_soff.data(), jso, (n_jobs + 1) * sizeof(int64_t),
                                          cudaMemcpyDeviceToHost, s));
                BMJ_CHECK(cudaStreamSynchronize(s));
                for (int64_t k = 0; k < n_jobs; k++) {
                    const int64_t nk = job_sets[k + 1] - job_sets[k];
                    mean_size[k] = nk > 0 ? (double)(h_soff[k + 1] - h_soff[k]) / (double)nk : 0.0;
                }
            }
            auto filter_cost = [](int width) { return width == 64 ? 1.0 : width == 128 ? 1.55 : 2.55; };
            // with the cascade, a survivor of a narrower filter costs one 256-bit
            // check (28 pair-units) and is merged only if it passes that too
            // (about as often as a survivor of the 256-bit filter itself)
            const size_t w256 = widths.size() - 1;
            est_surv = 0.0;
            for (int64_t k = 0; k < n_jobs; k++) {
                double best = 1e300;
                double best_surv = 0.0;
                const double verify_cost = 57.0 * std::max(1.0, mean_size[k] / 12.0);
                const double s256 = samp_win[w256][k] > 0
                                        ? (double)samp_surv[w256][k] * (double)job_win[k] / samp_win[w256][k]
                                        : 0.0;
                for (size_t wi = 0; wi < widths.size(); wi++) {
                    const double scale =
                        samp_win[wi][k] > 0 ? (double)job_win[k] / samp_win[wi][k] : 0.0;
                    const double surv = (double)samp_surv[wi][k] * scale;
                    const bool casc = cascade && widths[wi] < 256;
                    const double cost = (double)job_win[k] * filter_cost(widths[wi]) +
                                        (casc ? surv * 28.0 + std::min(surv, s256) * verify_cost
                                              : surv * verify_cost);
                    if (cost < best) {
                        best = cost;
                        best_surv = surv;
                        job_b[k] = widths[wi];
                    }
                }
                est_surv += best_surv;
                // the folded test pays where few pairs pass the 64-bit filter (a column
                // step of 128 pairs then rarely needs the 128-bit test)
                const double r64 = samp_win[0][k] > 0 ? (double)samp_surv[0][k] / samp_win[0][k] : 0.0;
                job_fold[k] = widths[0] == 64 && r64 > kBatchFoldMaxRate64 ? 0 : 1;
            }
            set_jobs(job_b);
            st = upload_jobs(P, A, s);
            if (st) return st;
        }
        BMJ_CHECK(cudaEventRecord(ev.e[4], s));

        // ---- row tile per job ----
        // A tile of T rows evaluates every pair of its column range, also the
        // T(T-1)/2 pairs at or above the diagonal (masked out), so a job of N
        // sets in tiles of T rows evaluates about its window plus N*T/2 pairs.
        // The small tile wastes less of a small job's window but costs more
        // per evaluated pair (fewer rows share each staged column); per job the
        // cheaper of the two is taken, or the caller's choice.
        for (int64_t k = 0; k < n_jobs; k++) {
            const int W = job_b[k] / 64;
            const double nk = (double)(job_sets[k + 1] - job_sets[k]);
            const double cost_d = (double)job_win[k] + nk * default_tile_rows(W) / 2.0;
            const double cost_s =
                ((double)job_win[k] + nk * small_tile_rows(W) / 2.0) * small_tile_cost(W);
            if (o.rows_per_thread > 0)
                job_small[k] = o.rows_per_thread * 32 < default_tile_rows(W) ? 1 : 0;
            else
                job_small[k] = (W == 1 || W == 2 || W == 4) && cost_s < cost_d ? 1 : 0;
        }
        set_jobs(job_b);
        st = upload_jobs(P, A, s);
        if (st) return st;

        // ---- tiles of every job ----
        // jobs grouped by tile class, so that each class is one tile range
        std::vector<int32_t> order(n_jobs);
        for (int64_t k = 0; k < n_jobs; k++) order[k] = (int32_t)k;
        std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t c) {
            return tile_class(P.jobs[a].W, P.jobs[a].tile_rows, P.jobs[a].fold) <
                   tile_class(P.jobs[c].W, P.jobs[c].tile_rows, P.jobs[c].fold);
        });
        std::vector<int64_t> job_tile0(n_jobs + 1, 0);
        for (int c = 0; c < kClasses; c++) P.class_t0[c] = P.class_t1[c] = 0;
        for (int64_t pos = 0; pos < n_jobs; pos++) {
            const int64_t k = order[pos];
            const int64_t nk = job_sets[k + 1] - job_sets[k];
            job_tile0[pos + 1] =
                job_tile0[pos] + (nk >= 2 ? (nk + P.jobs[k].tile_rows - 1) / P.jobs[k].tile_rows : 0);
        }
        for (int c = 0; c < kClasses; c++) {
            int64_t lo = -1, hi = -1;
            for (int64_t pos = 0; pos < n_jobs; pos++)
                if (tile_class(P.jobs[order[pos]].W, P.jobs[order[pos]].tile_rows,
                               P.jobs[order[pos]].fold) == c) {
                    if (lo < 0) lo = job_tile0[pos];
                    hi = job_tile0[pos + 1];
                }
            if (lo >= 0) {
                P.class_t0[c] = lo;
                P.class_t1[c] = hi;
            }
        }
        st = build_tiles(P, {}, {}, true, job_tile0, order, A, s, nullptr);
        if (st) return st;

        // ---- execute (filter + verification of all jobs) ----
        // The sampled estimate can miss clustered survivors (duplicate-heavy rows),
        // and an overflow reruns the whole filter: size the queue generously
        // (4x the estimate + 16M entries, at most a quarter of free memory).
        int64_t qcap = o.queue_cap > 0
                           ? o.queue_cap
                           : (est_surv >= 0 ? (int64_t)(4.0 * est_surv) + ((int64_t)1 << 24)
                                            : std::max<int64_t>((int64_t)(total_win / 128),
                                                                (int64_t)1 << 24));
        {
            size_t free_b = 0, total_b = 0;
            if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess)
                qcap = std::min<int64_t>(qcap, (int64_t)(free_b / 4 / (sizeof(uint2) + sizeof(uint64_t))));
            cudaGetLastError();
            qcap = std::max<int64_t>(qcap, 1);
        }
        int64_t n_surv = 0;
        unsigned long long hc[3] = {0, 0, 0};
        for (int pass = 0; pass < 2; pass++) {
            st = A.alloc(&P.queue, (size_t)qcap);
            if (!st) st = A.alloc(&P.keys, (size_t)qcap);
            if (st) return st;
            P.qcap = qcap;
            BMJ_CHECK(cudaEventRecord(ev.e[5], s));
            int graphed = 0;
            st = run_execute(P, sms, s, o.use_graph != 0, &graphed);
            if (st) return st;
            bs.graph = graphed;
            BMJ_CHECK(cudaEventRecord(ev.e[6], s));
            BMJ_CHECK(cudaMemcpyAsync(hc, P.ctr, sizeof(hc), cudaMemcpyDeviceToHost, s));
        {
            int herr = 0;
            BMJ_CHECK(cudaMemcpyAsync(&herr, P.err, sizeof(int), cudaMemcpyDeviceToHost, s));
            BMJ_CHECK(cudaStreamSynchronize(s));
            if (herr) return BMJ_ERR_TIMEOUT;
        }
            BMJ_CHECK(cudaStreamSynchronize(s));
            bs.filter_passes++;
            bs.ms_execute += ev.ms(5, 6);
            n_surv = (int64_t)hc[1];
            if (n_surv <= qcap) break;
            A.free_one(P.queue);
            A.free_one(P.keys);
            qcap = n_surv;  // every survivor was counted: rerun once with exact room
        }
        BMJ_CHECK(cudaMemcpyAsync(job_sv.data(), P.job_surv, n_jobs * sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, s));
        const int64_t n_res = (int64_t)hc[2];
        bs.survivors = n_surv;
        bs.results = n_res;
        bs.window_pairs = (int64_t)total_win;
        bs.ms_prepare = ev.ms(0, 1);
        bs.ms_tune = ev.ms(1, 4);

        // ---- canonical order and per-job split ----
        if (n_res > 0) {
            uint64_t *sk = nullptr;
            int64_t *bounds = nullptr;
            uint32_t *da = nullptr, *db = nullptr;
            st = A.alloc(&sk, (size_t)n_res);
            if (!st) st = A.alloc(&bounds, (size_t)n_jobs + 1);
            if (!st) st = A.alloc(&da, (size_t)n_res);
            if (!st) st = A.alloc(&db, (size_t)n_res);
            if (st) return st;
            st = radix_sort_u64(P.keys, sk, n_res, jbits + 2 * P.nbits, A, s);
            if (st) return st;
            BMJ_LAUNCH(k_job_bounds, grid_of(n_jobs + 1, 256), 256, 0, s, sk, n_res, n_jobs,
                       2 * P.nbits, bounds);
            BMJ_LAUNCH(k_unpack_local, grid_of(n_res, 256), 256, 0, s, sk, n_res, P.nbits, da, db);
            res_a.resize(n_res);
            res_b.resize(n_res);
            BMJ_CHECK(cudaMemcpyAsync(result_bounds.data(), bounds, (n_jobs + 1) * sizeof(int64_t),
                                      cudaMemcpyDeviceToHost, s));
            BMJ_CHECK(cudaMemcpyAsync(res_a.data(), da, n_res * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
            BMJ_CHECK(cudaMemcpyAsync(res_b.data(), db, n_res * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        }
    }
    BMJ_CHECK(cudaEventRecord(ev.e[7], s));
    A.release();
    BMJ_CHECK(cudaStreamSynchronize(s));
    bs.ms_output = 0.f;
    bs.ms_total = ev.ms(0, 7);

    // ---- outputs ----
    for (int64_t k = 0; k < n_jobs; k++) memset(&outs[k], 0, sizeof(bmj_pairs));
    for (int64_t k = 0; k < n_jobs; k++) {
        const int64_t lo = result_bounds[k], hi = result_bounds[k + 1];
        const int64_t m = res_a.empty() ? 0 : hi - lo;
        bmj_pairs &op = outs[k];
        op.on_device = o.output_on_device ? 1 : 0;
        if (m > 0) {
            if (o.output_on_device) {
                if (cudaMalloc(&op.a, m * sizeof(uint32_t)) != cudaSuccess ||
                    cudaMalloc(&op.b, m * sizeof(uint32_t)) != cudaSuccess) {
                    cudaGetLastError();
                    for (int64_t j = 0; j <= k; j++) bmj_pairs_free(&outs[j]);
                    return BMJ_ERR_OOM;
                }
                cudaMemcpy(op.a, res_a.data() + lo, m * sizeof(uint32_t), cudaMemcpyHostToDevice);
                cudaMemcpy(op.b, res_b.data() + lo, m * sizeof(uint32_t), cudaMemcpyHostToDevice);
            } else {
                op.a = (uint32_t *)malloc(m * sizeof(uint32_t));
                op.b = (uint32_t *)malloc(m * sizeof(uint32_t));
                if (!op.a || !op.b) {
                    for (int64_t j = 0; j <= k; j++) bmj_pairs_free(&outs[j]);
                    return BMJ_ERR_OOM;
                }
                memcpy(op.a, res_a.data() + lo, m * sizeof(uint32_t));
                memcpy(op.b, res_b.data() + lo, m * sizeof(uint32_t));
            }
            op.n = m;
        }
        if (job_stats) {
            bmj_stats &js = job_stats[k];
            memset(&js, 0, sizeof(js));
            js.window_pairs = (int64_t)job_win[k];
            js.survivors = (int64_t)job_sv[k];
            js.results = m;
            js.filter_passes = bs.filter_passes;
            js.b = job_b[k];
            js.method = job_method[k];
            js.tile_rows = P.jobs.empty() ? 0 : P.jobs[k].tile_rows;
            js.chunk_cols = P.jobs.empty() ? 0 : P.jobs[k].chunk_cols;
        }
    }
    bs.n_launches = (int32_t)(launches() - launches0);
    if (bst) *bst = bs;
    return BMJ_OK;
}

}  // namespace
}  // namespace bmj

namespace bmj {
namespace {

__global__ void k_rebase(const int64_t *__restrict__ in, int64_t n, int64_t base,
                         int64_t *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = in[i] - base;
}

void add_batch_stats(bmj_batch_stats &t, const bmj_batch_stats &u) {
    t.n_jobs += u.n_jobs;
    t.window_pairs += u.window_pairs;
    t.survivors += u.survivors;
    t.results += u.results;
    t.n_launches += u.n_launches;
    t.filter_passes += u.filter_passes;
    t.graph = t.graph || u.graph;
    t.tuned = t.tuned || u.tuned;
    t.ms_prepare += u.ms_prepare;
    t.ms_tune += u.ms_tune;
    t.ms_execute += u.ms_execute;
    t.ms_output += u.ms_output;
    t.ms_total += u.ms_total;
}

// Jobs [k0, k1) of the batch as a collection of their own: offsets rebased to
// start at 0 (a device copy for a device collection), tokens borrowed.
struct SubColl {
    bmj_collection c{};
    std::vector<int64_t> host_off;
    int64_t *dev_off = nullptr;
    cudaStream_t s = nullptr;
    ~SubColl() {
        if (dev_off) cudaFreeAsync(dev_off, s);
    }
};

int make_sub(const bmj_collection *coll, int64_t s0, int64_t s1, cudaStream_t s, SubColl &sub) {
    sub.s = s;
    const int64_t m = s1 - s0;
    int64_t base = 0;
    if (coll->on_device) {
        BMJ_CHECK(cudaMemcpyAsync(&base, coll->offsets + s0, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        BMJ_CHECK(cudaStreamSynchronize(s));
        BMJ_CHECK(cudaMallocAsync(&sub.dev_off, (m + 1) * sizeof(int64_t), s));
        k_rebase<<<(unsigned)std::min<int64_t>((m + 256) / 256, 148 * 8), 256, 0, s>>>(
            coll->offsets + s0, m + 1, base, sub.dev_off);
        count_launch();
        BMJ_CHECK(cudaGetLastError());
        sub.c.offsets = sub.dev_off;
    } else {
        base = coll->offsets[s0];
        sub.host_off.resize(m + 1);
        for (int64_t i = 0; i <= m; i++) sub.host_off[i] = coll->offsets[s0 + i] - base;
        sub.c.offsets = sub.host_off.data();
    }
    sub.c.n_sets = m;
    sub.c.tokens = coll->tokens + base;
    sub.c.on_device = coll->on_device;
    return BMJ_OK;
}

// After an out-of-memory batch: the jobs run in two halves (recursively); a
// single job that still does not fit runs as bmj_self_join, whose survivor
// handling never needs all survivors in memory at once.
int batch_in_parts(const bmj_collection *coll, int64_t n_jobs, const int64_t *job_sets, int sim,
                   const uint32_t *hp, const uint32_t *hq, const bmj_options &o, bmj_pairs *outs,
                   bmj_stats *job_stats, bmj_batch_stats *bst) {
    cudaStream_t s = (cudaStream_t)o.stream;
    if (n_jobs == 1) {
        SubColl sub;
        int st = make_sub(coll, job_sets[0], job_sets[1], s, sub);
        if (st) return st;
        bmj_options so = o;
        if (so.b == 0) so.b = 256;  // the widest tuned width leaves the fewest survivors
        so.use_graph = 0;
        bmj_stats js;
        memset(&js, 0, sizeof(js));
        st = bmj_self_join(&sub.c, sim, hp[0], hq[0], &so, &outs[0], &js);
        if (st) return st;
        if (job_stats) job_stats[0] = js;
        bmj_batch_stats u;
        memset(&u, 0, sizeof(u));
        u.n_jobs = 1;
        u.window_pairs = js.window_pairs;
        u.survivors = js.survivors;
        u.results = js.results;
        u.n_launches = js.n_launches;
        u.filter_passes = (int32_t)js.filter_passes;
        u.ms_prepare = js.ms_prepare;
        u.ms_execute = js.ms_filter + js.ms_verify;
        u.ms_output = js.ms_output;
        u.ms_total = js.ms_total;
        add_batch_stats(*bst, u);
        return BMJ_OK;
    }
    const int64_t half = n_jobs / 2;
    for (int part = 0; part < 2; part++) {
        const int64_t k0 = part ? half : 0, k1 = part ? n_jobs : half;
        SubColl sub;
        int st = make_sub(coll, job_sets[k0], job_sets[k1], s, sub);
        if (st) return st;
        std::vector<int64_t> js(k1 - k0 + 1);
        for (int64_t k = k0; k <= k1; k++) js[k - k0] = job_sets[k] - job_sets[k0];
        bmj_batch_stats u;
        memset(&u, 0, sizeof(u));
        try {
            st = batch_impl(&sub.c, k1 - k0, js.data(), sim, hp + k0, hq + k0, o, outs + k0,
                            job_stats ? job_stats + k0 : nullptr, &u);
        } catch (...) {
            st = BMJ_ERR_OOM;
        }
        if (st == BMJ_ERR_OOM) {
            for (int64_t k = k0; k < k1; k++) bmj_pairs_free(&outs[k]);
            cudaGetLastError();
            memset(&u, 0, sizeof(u));
            st = batch_in_parts(&sub.c, k1 - k0, js.data(), sim, hp + k0, hq + k0, o, outs + k0,
                                job_stats ? job_stats + k0 : nullptr, &u);
        }
        if (st) return st;
        add_batch_stats(*bst, u);
    }
    return BMJ_OK;
}

}  // namespace
}  // namespace bmj

extern "C" int bmj_self_join_batch(const bmj_collection *coll, int64_t n_jobs,
                                   const int64_t *job_sets, int sim, const uint32_t *p,
                                   const uint32_t *q, const bmj_options *opt, bmj_pairs *outs,
                                   bmj_stats *job_stats, bmj_batch_stats *batch_stats) {
    if (batch_stats) memset(batch_stats, 0, sizeof(*batch_stats));
    if (!coll || !job_sets || !outs || n_jobs <= 0 || !p || !q) return BMJ_ERR_INVALID_ARG;
    for (int64_t k = 0; k < n_jobs; k++) memset(&outs[k], 0, sizeof(bmj_pairs));
    if (sim < BMJ_JACCARD || sim > BMJ_OVERLAP) return BMJ_ERR_INVALID_ARG;
    if (coll->n_sets < 0 || !coll->offsets || (coll->n_sets > 0 && !coll->tokens))
        return BMJ_ERR_INVALID_ARG;
    if (coll->n_sets > 0x7fffffffLL || n_jobs > 0x7fffffffLL) return BMJ_ERR_TOO_LARGE;
    if (job_sets[0] != 0 || job_sets[n_jobs] != coll->n_sets) return BMJ_ERR_INVALID_ARG;
    for (int64_t k = 0; k < n_jobs; k++) {
        if (job_sets[k + 1] < job_sets[k]) return BMJ_ERR_INVALID_ARG;
        if (!bmj::sim_valid(sim, p[k], q[k])) return BMJ_ERR_INVALID_ARG;
    }
    bmj_options o;
    if (opt) o = *opt;
    else bmj_default_options(&o);
    if (o.b != 0 && !bmj::valid_b(o.b)) return BMJ_ERR_INVALID_ARG;
    if (o.method < BMJ_XOR || o.method > BMJ_COMBINED) return BMJ_ERR_INVALID_ARG;
    if (o.queue_cap < 0) return BMJ_ERR_INVALID_ARG;
    if (o.cascade_b != 0 && o.cascade_b != -1 && o.cascade_b != 256) return BMJ_ERR_INVALID_ARG;
    if (o.row_begin != 0 || o.row_end != 0 || o.candidates != BMJ_CAND_WINDOW || o.cutoff != 0)
        return BMJ_ERR_INVALID_ARG;  // options of the single join only
    int st;
    bmj_batch_stats bs;
    memset(&bs, 0, sizeof(bs));
    bmj::arm_alloc_fault(bmj::read_fault_plan().alloc_at);  // tests: BMJ_FAULT=alloc:K
    try {
        st = bmj::batch_impl(coll, n_jobs, job_sets, sim, p, q, o, outs, job_stats, &bs);
    } catch (...) {
        st = BMJ_ERR_OOM;
    }
    bmj::arm_alloc_fault(0);
    if (st == BMJ_ERR_OOM) {  // retry in parts: halves of the job list, then single joins
        for (int64_t k = 0; k < n_jobs; k++) bmj_pairs_free(&outs[k]);
        cudaGetLastError();
        memset(&bs, 0, sizeof(bs));
        try {
            st = bmj::batch_in_parts(coll, n_jobs, job_sets, sim, p, q, o, outs, job_stats, &bs);
        } catch (...) {
            st = BMJ_ERR_OOM;
        }
    }
    if (!st && batch_stats) *batch_stats = bs;
    if (st) {
        for (int64_t k = 0; k < n_jobs; k++) bmj_pairs_free(&outs[k]);
        cudaGetLastError();
    }
    return st;
}
