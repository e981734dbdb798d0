// filter.cu -- the Bitmap Filter kernels (Alg. 5/6, Eq. 2 against the Table 1
// overlap threshold) and their launchers.  The per-item bodies are in
// filter_core.cuh; preparation kernels are in kernels.cu.
//   k_filter          columns broadcast by warp shuffles (any b)
//   k_filter_tma      columns staged in shared memory by TMA bulk copies
//                     (b = 64, 128, 256)
#include "kernels.cuh"
#include "filter_core.cuh"

namespace bmj {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// ----------------------------------------------------------------------------
// Bitmap Filter (per-item body in filter_core.cuh).  Warps pull work items
// (row tile, column chunk) from a global counter: a persistent grid that
// balances the uneven band of the size-sorted triangle.
template <int W, int R, bool kCos>
__global__ void __launch_bounds__(256) k_filter(const FilterArgs a) {
    const int lane = threadIdx.x & 31;
    const SurvivorSink sink{a.queue, a.qcount, nullptr, a.qcap};
    const SimArgs sa{sim_window(a.sim, a.p, a.q), a.p, a.q, a.cut};
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(a.item_counter, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if ((int64_t)item >= a.n_items) return;
        const int64_t t = find_tile(a.tile_item_off, a.n_tiles, item);
        const int64_t chunk = (int64_t)item - a.tile_item_off[t];
        const int64_t row_end = a.row_end < 0 ? a.n : a.row_end;
        const int64_t i0 = a.row0 + t * a.tile_rows;
        const int64_t c0 = (int64_t)a.tile_c0[t] + chunk * a.chunk_cols;
        const int64_t c_end =
            a.tile_c1 ? (int64_t)a.tile_c1[t] : min(i0 + (int64_t)a.tile_rows, row_end) - 1;
        const int64_t c1 = min(c0 + (int64_t)a.chunk_cols, c_end);
        filter_item<W, R, kCos>(a.bm, a.ssz, a.lim, row_end, i0, c0, c1, sa, sink);
    }
}

__global__ void __launch_bounds__(256) k_filter_generic(const FilterArgs a, int W) {
    const int lane = threadIdx.x & 31;
    const SurvivorSink sink{a.queue, a.qcount, nullptr, a.qcap};
    const SimArgs sa{sim_window(a.sim, a.p, a.q), a.p, a.q, a.cut};
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(a.item_counter, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if ((int64_t)item >= a.n_items) return;
        const int64_t t = find_tile(a.tile_item_off, a.n_tiles, item);
        const int64_t chunk = (int64_t)item - a.tile_item_off[t];
        const int64_t row_end = a.row_end < 0 ? a.n : a.row_end;
        const int64_t i0 = a.row0 + t * a.tile_rows;
        const int64_t c0 = (int64_t)a.tile_c0[t] + chunk * a.chunk_cols;
        const int64_t c_end =
            a.tile_c1 ? (int64_t)a.tile_c1[t] : min(i0 + (int64_t)a.tile_rows, row_end) - 1;
        const int64_t c1 = min(c0 + (int64_t)a.chunk_cols, c_end);
        if (a.sim == BMJ_COSINE)
            filter_item_generic<true>(a.bm, a.ssz, a.lim, row_end, i0, c0, c1, sa, W, sink);
        else
            filter_item_generic<false>(a.bm, a.ssz, a.lim, row_end, i0, c0, c1, sa, W, sink);
    }
}

// Bitmap Filter with TMA-staged columns (filter_item_tma).  Each warp owns a
// double buffer of column chunks in dynamic shared memory and its two
// mbarriers; a wait that gives up sets *err and stops the warp.
// Eight 4-warp blocks per SM (64 registers) for the production variants; the
// Cosine variant's per-pair limit needs more registers.  kCut: pairs whose
// larger set is above the cutoff point skip Eq. 2 (Section 3.5).
// Resident blocks per SM at b = 128 (the register bound follows: 56 at nine).
#ifndef BMJ_TMA_MINB2
#define BMJ_TMA_MINB2 9
#endif
template <int W, int R, int CS, bool kFault, bool kCos, bool kCut>
__global__ void __launch_bounds__(128, kCos ? 6 : W == 2 ? BMJ_TMA_MINB2 : 8)
    k_filter_tma(const FilterArgs a, int *err) {
    extern __shared__ __align__(128) unsigned char smem[];
    using L = ColStage<W, CS>;
    const int lane = threadIdx.x & 31;
    StageState st;
    init_stage(st, smem + (threadIdx.x >> 5) * L::kWarpBytes, L::kStageOff);
    if (kFault) {  // fault injection: the first warp skips its first copy; short waits
        st.wait_limit = a.wait_limit;
        st.skip_copy = (blockIdx.x == 0 && threadIdx.x < 32) ? 1 : 0;
    }
    const SurvivorSink sink{a.queue, a.qcount, nullptr, a.qcap};
    const SimArgs sa{sim_window(a.sim, a.p, a.q), a.p, a.q, a.cut};
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(a.item_counter, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if ((int64_t)item >= a.n_items) break;
        const int64_t t = find_tile(a.tile_item_off, a.n_tiles, item);
        const int64_t chunk = (int64_t)item - a.tile_item_off[t];
        const int64_t row_end = a.row_end < 0 ? a.n : a.row_end;
        const int64_t i0 = a.row0 + t * a.tile_rows;
        const int64_t c0 = (int64_t)a.tile_c0[t] + chunk * a.chunk_cols;
        const int64_t c_end =
            a.tile_c1 ? (int64_t)a.tile_c1[t] : min(i0 + (int64_t)a.tile_rows, row_end) - 1;
        const int64_t c1 = min(c0 + (int64_t)a.chunk_cols, c_end);
        filter_item_tma<W, R, CS, kAltRows<W>, kCos, kCut, kFoldW<W>>(a.bm, a.ssz, a.lim, row_end,
                                                                       i0, c0, c1, sa, sink, st);
        if (kFoldW<W> && a.steps && lane == 0 && c1 > c0) {
            atomicAdd(&a.steps[0], (unsigned long long)(c1 - c0));
            atomicAdd(&a.steps[1], (unsigned long long)st.n_full);
        }
        if (!st.ok) {
            drain_stage(st);
            if (lane == 0) atomicOr(err, 1);
            break;
        }
    }
}

template <int W, int R, bool kCos>
int launch_filter_c(const FilterArgs &a, int num_sms, cudaStream_t s) {
    int per_sm = 0;
    BMJ_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_filter<W, R, kCos>, 256, 0));
    if (per_sm < 1) per_sm = 1;
    int64_t warps_needed = a.n_items;
    int64_t blocks = (int64_t)num_sms * per_sm;
    const int64_t need_blocks = (warps_needed + 7) / 8;
    if (need_blocks < blocks) blocks = need_blocks;
    if (blocks < 1) blocks = 1;
    BMJ_LAUNCH((k_filter<W, R, kCos>), (unsigned)blocks, 256, 0, s, a);
    return BMJ_OK;
}

template <int W, int R>
int launch_filter_t(const FilterArgs &a, int num_sms, cudaStream_t s) {
    return a.sim == BMJ_COSINE ? launch_filter_c<W, R, true>(a, num_sms, s)
                               : launch_filter_c<W, R, false>(a, num_sms, s);
}

}  // namespace

int filter_tile_rows(int W) {
    switch (W) {
        case 1: case 2: case 4: return 32 * 4;
        case 8: return 32 * 2;
        default: return 32;
    }
}

int launch_filter(const FilterArgs &a, int W, int num_sms, cudaStream_t s) {
    if (a.n_items <= 0) return BMJ_OK;
    switch (W) {
        case 1: return launch_filter_t<1, 4>(a, num_sms, s);
        case 2: return launch_filter_t<2, 4>(a, num_sms, s);
        case 4: return launch_filter_t<4, 4>(a, num_sms, s);
        case 8: return launch_filter_t<8, 2>(a, num_sms, s);
        default: {
            int per_sm = 0;
            BMJ_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_filter_generic, 256, 0));
            if (per_sm < 1) per_sm = 1;
            int64_t blocks = (int64_t)num_sms * per_sm;
            const int64_t need_blocks = (a.n_items + 7) / 8;
            if (need_blocks < blocks) blocks = need_blocks;
            if (blocks < 1) blocks = 1;
            BMJ_LAUNCH(k_filter_generic, (unsigned)blocks, 256, 0, s, a, W);
            return BMJ_OK;
        }
    }
}

template <int W, int R, int CS, bool kFault, bool kCos, bool kCut>
int launch_filter_tma_k(const FilterArgs &a, int *err, int num_sms, cudaStream_t s) {
    using L = ColStage<W, CS>;
    const int smem = 4 * L::kWarpBytes;
    int per_sm = 0;
    BMJ_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, k_filter_tma<W, R, CS, kFault, kCos, kCut>, 128, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (int64_t)num_sms * per_sm;
    const int64_t need_blocks = (a.n_items + 3) / 4;
    if (need_blocks < blocks) blocks = need_blocks;
    if (blocks < 1) blocks = 1;
    BMJ_LAUNCH((k_filter_tma<W, R, CS, kFault, kCos, kCut>), (unsigned)blocks, 128, smem, s, a,
               err);
    return BMJ_OK;
}

template <int W, int R, int CS>
int launch_filter_tma_t(const FilterArgs &a, int *err, int num_sms, cudaStream_t s) {
    const bool cut = a.cut != 0xffffffffu;
    if (a.sim == BMJ_COSINE)  // (fault injection is exercised with the other functions)
        return cut ? launch_filter_tma_k<W, R, CS, false, true, true>(a, err, num_sms, s)
                   : launch_filter_tma_k<W, R, CS, false, true, false>(a, err, num_sms, s);
    if (cut) return launch_filter_tma_k<W, R, CS, false, false, true>(a, err, num_sms, s);
    return a.fault_skip_copy ? launch_filter_tma_k<W, R, CS, true, false, false>(a, err, num_sms, s)
                             : launch_filter_tma_k<W, R, CS, false, false, false>(a, err, num_sms, s);
}

int filter_tma_tile_rows(int W) {
    switch (W) {
        case 1: return 32 * kTmaR1;
        case 2: return 32 * kTmaR2;
        case 4: return 32 * kTmaR4;
        default: return filter_tile_rows(W);
    }
}

int launch_filter_tma(const FilterArgs &a, int W, int *err, int num_sms, cudaStream_t s) {
    if (a.n_items <= 0) return BMJ_OK;
    switch (W) {
        case 1: return launch_filter_tma_t<1, kTmaR1, kTmaCS1>(a, err, num_sms, s);
        case 2: return launch_filter_tma_t<2, kTmaR2, kTmaCS2>(a, err, num_sms, s);
        case 4: return launch_filter_tma_t<4, kTmaR4, kTmaCS4>(a, err, num_sms, s);
        default: return launch_filter(a, W, num_sms, s);
    }
}

}  // namespace bmj
