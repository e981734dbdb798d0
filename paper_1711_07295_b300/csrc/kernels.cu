// kernels.cu -- device kernels of the Bitmap Filter self-join.
//
// Stages (each cited where it is defined in the paper):
//   k_validate       CSR invariants; sizes and ids for the size sort (Section 5
//                    preprocessing: sets ordered by size)
//   k_gather_build   sorted CSR gather + b-bit bitmaps (Section 3.2, Alg. 3a/3b/3c,
//                    h(t) = t mod b as in Section 5.1)
//   k_tables         need[S] / lim[S]: Jaccard as an overlap threshold (Table 1)
//                    folded into the Eq. 2 test
//   k_tiles,
//   k_window_count   the length filter window j in [j0(i), i) (Table 2; Alg. 6)
//   k_filter         the Bitmap Filter over every window pair (Alg. 5/6, Eq. 2)
// Verification and the output kernels are in verify.cu.
#include "kernels.cuh"
#include "filter_core.cuh"

namespace bmj {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// First index j in [0, n) with ssz[j] >= v (n if none).
__device__ __forceinline__ int64_t lower_bound_u32(const uint32_t *a, int64_t n, uint64_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((uint64_t)a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Smallest size s' with q*s' >= p*s, i.e. ceil(p*s/q) (Table 2, Jaccard row, integer form).
__device__ __forceinline__ uint64_t window_low(uint64_t s, uint32_t p, uint32_t q) {
    return (s * p + q - 1) / q;
}

// ----------------------------------------------------------------------------
__global__ void k_validate(const int64_t *__restrict__ off, const int32_t *__restrict__ tok,
                           int64_t n, int64_t ntok, int check_tokens, uint32_t *__restrict__ sizes,
                           uint32_t *__restrict__ ids, int *__restrict__ info) {
    int flags = 0;
    uint32_t mx = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        const int64_t lo = off[x], hi = off[x + 1];
        int64_t sz = hi - lo;
        if (x == 0 && lo != 0) flags |= kFlagUnsorted;
        if (lo < 0 || hi > ntok || sz < 0) {
            flags |= kFlagUnsorted;
            sz = 0;
        } else if (sz == 0) {
            flags |= kFlagEmpty;
        } else if (sz > kMaxSetSize) {
            flags |= kFlagTooLarge;
            sz = 0;
        } else if (check_tokens) {
            int32_t prev = tok[lo];
            if (prev < 0) flags |= kFlagNegative;
            for (int64_t k = lo + 1; k < hi; k++) {
                const int32_t t = tok[k];
                if (t <= prev) flags |= kFlagUnsorted;
                if (t < 0) flags |= kFlagNegative;
                prev = t;
            }
        }
        sizes[x] = (uint32_t)sz;
        ids[x] = (uint32_t)x;
        mx = max(mx, (uint32_t)sz);
    }
    flags = __reduce_or_sync(kFull, flags);
    mx = __reduce_max_sync(kFull, mx);
    if ((threadIdx.x & 31) == 0) {
        if (flags) atomicOr(&info[0], flags);
        atomicMax(&info[1], (int)mx);
    }
}

__global__ void k_widen(const uint32_t *__restrict__ in, int64_t *__restrict__ out, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = in[i];
}

// One warp per set.  The bitmap is assembled in shared memory (one 64-word
// slot per warp, enough for b <= 4096) and written out as whole words.
constexpr int kBuildWarps = 8;

__global__ void __launch_bounds__(kBuildWarps * 32)
    k_gather_build(const uint32_t *__restrict__ perm, const int64_t *__restrict__ off,
                   const int32_t *__restrict__ tok, const int64_t *__restrict__ soff,
                   int32_t *__restrict__ stok, uint64_t *__restrict__ bm, int64_t n, int b,
                   int method) {
    __shared__ unsigned long long sbm[kBuildWarps][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int W = b >> 6;
    const bool pow2 = (b & (b - 1)) == 0;
    unsigned long long *mine = sbm[warp];
    for (int64_t i = (int64_t)blockIdx.x * kBuildWarps + warp; i < n;
         i += (int64_t)gridDim.x * kBuildWarps) {
        const int64_t src = perm ? (int64_t)perm[i] : i;
        const int64_t lo = off[src];
        const int64_t cnt = off[src + 1] - lo;
        const int32_t *x = tok + lo;
        for (int w = lane; w < W; w += 32) mine[w] = 0ull;
        __syncwarp();
        if (stok) {
            int32_t *y = stok + soff[i];
            for (int64_t k = lane; k < cnt; k += 32) y[k] = x[k];
        }
        if (method == BMJ_NEXT) {
            if (cnt >= b) {
                for (int w = lane; w < W; w += 32) mine[w] = ~0ull;
            } else if (lane == 0) {
                // Alg. 3c: linear probing to the first unset bit at or after
                // h(t), wrapping around; cnt < b guarantees a free bit, so the
                // scan ends within W + 1 words.
                for (int64_t k = 0; k < cnt; k++) {
                    const uint32_t t = (uint32_t)x[k];
                    const uint32_t h = pow2 ? (t & (uint32_t)(b - 1)) : (t % (uint32_t)b);
                    int w = (int)(h >> 6);
                    unsigned long long m = ~mine[w] & (~0ull << (h & 63));
                    for (int guard = 0; m == 0ull && guard <= W; guard++) {
                        w = (w + 1 == W) ? 0 : w + 1;
                        m = ~mine[w];
                    }
                    mine[w] |= m & (~m + 1ull);
                }
            }
        } else {
            for (int64_t k = lane; k < cnt; k += 32) {
                const uint32_t t = (uint32_t)x[k];
                const uint32_t h = pow2 ? (t & (uint32_t)(b - 1)) : (t % (uint32_t)b);
                const unsigned long long bit = 1ull << (h & 63);
                if (method == BMJ_XOR) atomicXor(&mine[h >> 6], bit);  // Alg. 3b
                else atomicOr(&mine[h >> 6], bit);                     // Alg. 3a
            }
        }
        __syncwarp();
        uint64_t *dst = bm + i * W;
        for (int w = lane; w < W; w += 32) dst[w] = mine[w];
        __syncwarp();
    }
}

// One thread per set: gathers the set's tokens into the sorted CSR (when stok
// is given) and writes its Xor (Alg. 3b) or Set (Alg. 3a) bitmaps for up to
// three widths at once (64, 128, 256 bits; a null output skips a width).
// With b a power of two, h(t) = t mod b selects word (t mod b) / 64 and bit
// t mod 64 for all three widths.
__global__ void __launch_bounds__(256)
    k_build_multi(const uint32_t *__restrict__ perm, const int64_t *__restrict__ off,
                  const int32_t *__restrict__ tok, const int64_t *__restrict__ soff,
                  int32_t *__restrict__ stok, int64_t n, int method, uint64_t *__restrict__ bm64,
                  uint64_t *__restrict__ bm128, uint64_t *__restrict__ bm256) {
    const bool xr = method == BMJ_XOR;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t src = perm ? (int64_t)perm[i] : i;
        const int64_t lo = off[src];
        const int64_t cnt = off[src + 1] - lo;
        const int32_t *x = tok + lo;
        int32_t *y = stok ? stok + soff[i] : nullptr;
        uint64_t a = 0, b0 = 0, b1 = 0, c0 = 0, c1 = 0, c2 = 0, c3 = 0;
        for (int64_t k = 0; k < cnt; k++) {
            const uint32_t t = (uint32_t)x[k];
            if (y) y[k] = (int32_t)t;
            const uint64_t bit = 1ull << (t & 63u);
            const uint32_t w2 = (t >> 6) & 1u, w4 = (t >> 6) & 3u;
            if (xr) {
                a ^= bit;
                b0 ^= w2 == 0 ? bit : 0ull;
                b1 ^= w2 == 1 ? bit : 0ull;
                c0 ^= w4 == 0 ? bit : 0ull;
                c1 ^= w4 == 1 ? bit : 0ull;
                c2 ^= w4 == 2 ? bit : 0ull;
                c3 ^= w4 == 3 ? bit : 0ull;
            } else {
                a |= bit;
                b0 |= w2 == 0 ? bit : 0ull;
                b1 |= w2 == 1 ? bit : 0ull;
                c0 |= w4 == 0 ? bit : 0ull;
                c1 |= w4 == 1 ? bit : 0ull;
                c2 |= w4 == 2 ? bit : 0ull;
                c3 |= w4 == 3 ? bit : 0ull;
            }
        }
        if (bm64) bm64[i] = a;
        if (bm128) {
            bm128[2 * i] = b0;
            bm128[2 * i + 1] = b1;
        }
        if (bm256) {
            bm256[4 * i] = c0;
            bm256[4 * i + 1] = c1;
            bm256[4 * i + 2] = c2;
            bm256[4 * i + 3] = c3;
        }
    }
}

__global__ void k_tables(int32_t *__restrict__ need, int32_t *__restrict__ lim, int64_t n_s,
                         uint32_t p, uint32_t q) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const uint64_t d = (uint64_t)p + q;
    for (int64_t S = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; S < n_s; S += stride) {
        // Jaccard >= p/q  <=>  o*(p+q) >= p*S  <=>  o >= ceil(p*S/(p+q)) (Table 1).
        const uint64_t nd = ((uint64_t)S * p + d - 1) / d;
        need[S] = (int32_t)nd;
        // floor((S - h)/2) >= nd  <=>  h <= S - 2*nd (Eq. 2 with its floor).
        lim[S] = (int32_t)((int64_t)S - 2 * (int64_t)nd);
    }
}

__global__ void k_tiles(const uint32_t *__restrict__ ssz, int64_t n, uint32_t p, uint32_t q,
                        int tile_rows, int chunk_cols, int64_t n_tiles,
                        int32_t *__restrict__ tile_c0, int64_t *__restrict__ tile_items,
                        int64_t row0, int64_t row_end) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += stride) {
        const int64_t i0 = row0 + t * tile_rows;
        const int64_t j0 = lower_bound_u32(ssz, n, window_low(ssz[i0], p, q));
        const int64_t c0 = j0 & ~(int64_t)3;
        const int64_t c_end = min(i0 + (int64_t)tile_rows, row_end) - 1;  // columns j < i <= c_end
        const int64_t cols = c_end - c0;
        tile_c0[t] = (int32_t)c0;
        tile_items[t] = cols > 0 ? (cols + chunk_cols - 1) / chunk_cols : 0;
    }
}

__global__ void k_window_count(const uint32_t *__restrict__ ssz, int64_t n, uint32_t p,
                               uint32_t q, unsigned long long *__restrict__ out, int64_t row0,
                               int64_t row_end) {
    unsigned long long acc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = row0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < row_end; i += stride) {
        const int64_t j0 = lower_bound_u32(ssz, n, window_low(ssz[i], p, q));
        if (j0 < i) acc += (unsigned long long)(i - j0);
    }
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(kFull, acc, d);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

// ----------------------------------------------------------------------------
// Bitmap Filter (per-item body in filter_core.cuh).  Warps pull work items
// (row tile, column chunk) from a global counter: a persistent grid that
// balances the uneven band of the size-sorted triangle.
template <int W, int R>
__global__ void __launch_bounds__(256) k_filter(const FilterArgs a) {
    const int lane = threadIdx.x & 31;
    const SurvivorSink sink{a.queue, a.qcount, nullptr, a.qcap};
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
        const int64_t c_end = min(i0 + (int64_t)a.tile_rows, row_end) - 1;
        const int64_t c1 = min(c0 + (int64_t)a.chunk_cols, c_end);
        filter_item<W, R>(a.bm, a.ssz, a.lim, row_end, i0, c0, c1, a.p, a.q, sink);
    }
}

__global__ void __launch_bounds__(256) k_filter_generic(const FilterArgs a, int W) {
    const int lane = threadIdx.x & 31;
    const SurvivorSink sink{a.queue, a.qcount, nullptr, a.qcap};
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
        const int64_t c_end = min(i0 + (int64_t)a.tile_rows, row_end) - 1;
        const int64_t c1 = min(c0 + (int64_t)a.chunk_cols, c_end);
        filter_item_generic(a.bm, a.ssz, a.lim, row_end, i0, c0, c1, a.p, a.q, W, sink);
    }
}

// Bitmap Filter with TMA-staged columns (filter_item_tma).  Each warp owns a
// double buffer of column chunks in dynamic shared memory and its two
// mbarriers; a wait that gives up sets *err and stops the warp.
template <int W, int R, int CS, bool kFault>
__global__ void __launch_bounds__(128) k_filter_tma(const FilterArgs a, int *err) {
    extern __shared__ __align__(128) unsigned char smem[];
    using L = ColStage<W, CS>;
    const int lane = threadIdx.x & 31;
    StageState st;
    init_stage(st, smem + (threadIdx.x >> 5) * L::kWarpBytes);
    if (kFault) {  // fault injection: the first warp skips its first copy; short waits
        st.wait_limit = a.wait_limit;
        st.skip_copy = (blockIdx.x == 0 && threadIdx.x < 32) ? 1 : 0;
    }
    const SurvivorSink sink{a.queue, a.qcount, nullptr, a.qcap};
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
        const int64_t c_end = min(i0 + (int64_t)a.tile_rows, row_end) - 1;
        const int64_t c1 = min(c0 + (int64_t)a.chunk_cols, c_end);
        filter_item_tma<W, R, CS, (W == 1 ? kAluRowsW1 : 0)>(a.bm, a.ssz, a.lim, row_end, i0, c0, c1,
                                                             a.p, a.q, sink, st);
        if (!st.ok) {
            drain_stage(st);
            if (lane == 0) atomicOr(err, 1);
            break;
        }
    }
}

unsigned grid_for(int64_t n, int threads, int64_t cap = 148 * 32) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

template <int W, int R>
int launch_filter_t(const FilterArgs &a, int num_sms, cudaStream_t s) {
    int per_sm = 0;
    BMJ_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_filter<W, R>, 256, 0));
    if (per_sm < 1) per_sm = 1;
    int64_t warps_needed = a.n_items;
    int64_t blocks = (int64_t)num_sms * per_sm;
    const int64_t need_blocks = (warps_needed + 7) / 8;
    if (need_blocks < blocks) blocks = need_blocks;
    if (blocks < 1) blocks = 1;
    BMJ_LAUNCH((k_filter<W, R>), (unsigned)blocks, 256, 0, s, a);
    return BMJ_OK;
}

}  // namespace

int launch_validate(const int64_t *off, const int32_t *tok, int64_t n, int64_t ntok,
                    int check_tokens, uint32_t *sizes, uint32_t *ids, int *info, cudaStream_t s) {
    if (n <= 0) return BMJ_OK;
    BMJ_LAUNCH(k_validate, grid_for(n, 256), 256, 0, s, off, tok, n, ntok, check_tokens, sizes,
               ids, info);
    return BMJ_OK;
}

int launch_widen(const uint32_t *in, int64_t *out, int64_t n, cudaStream_t s) {
    if (n <= 0) return BMJ_OK;
    BMJ_LAUNCH(k_widen, grid_for(n, 256), 256, 0, s, in, out, n);
    return BMJ_OK;
}

int launch_gather_build(const uint32_t *perm, const int64_t *off, const int32_t *tok,
                        const int64_t *soff, int32_t *stok, uint64_t *bm, int64_t n, int b,
                        int method, cudaStream_t s) {
    if (n <= 0) return BMJ_OK;
    BMJ_LAUNCH(k_gather_build, grid_for(n, kBuildWarps, 148 * 64), kBuildWarps * 32, 0, s, perm,
               off, tok, soff, stok, bm, n, b, method);
    return BMJ_OK;
}

int launch_build_multi(const uint32_t *perm, const int64_t *off, const int32_t *tok,
                       const int64_t *soff, int32_t *stok, int64_t n, int method, uint64_t *bm64,
                       uint64_t *bm128, uint64_t *bm256, cudaStream_t s) {
    if (n <= 0) return BMJ_OK;
    BMJ_LAUNCH(k_build_multi, grid_for(n, 256, 148 * 16), 256, 0, s, perm, off, tok, soff, stok, n,
               method, bm64, bm128, bm256);
    return BMJ_OK;
}

int launch_tables(int32_t *need, int32_t *lim, int64_t n_s, uint32_t p, uint32_t q,
                  cudaStream_t s) {
    BMJ_LAUNCH(k_tables, grid_for(n_s, 256), 256, 0, s, need, lim, n_s, p, q);
    return BMJ_OK;
}

int launch_tiles(const uint32_t *ssz, int64_t n, uint32_t p, uint32_t q, int tile_rows,
                 int chunk_cols, int64_t n_tiles, int32_t *tile_c0, int64_t *tile_items,
                 cudaStream_t s, int64_t row0, int64_t row_end) {
    if (n_tiles <= 0) return BMJ_OK;
    BMJ_LAUNCH(k_tiles, grid_for(n_tiles, 256), 256, 0, s, ssz, n, p, q, tile_rows, chunk_cols,
               n_tiles, tile_c0, tile_items, row0, row_end < 0 ? n : row_end);
    return BMJ_OK;
}

int launch_window_count(const uint32_t *ssz, int64_t n, uint32_t p, uint32_t q,
                        unsigned long long *out, cudaStream_t s, int64_t row0, int64_t row_end) {
    if (row_end < 0) row_end = n;
    if (row_end <= row0) return BMJ_OK;
    BMJ_LAUNCH(k_window_count, grid_for(row_end - row0, 256), 256, 0, s, ssz, n, p, q, out, row0,
               row_end);
    return BMJ_OK;
}

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

template <int W, int R, int CS, bool kFault>
int launch_filter_tma_k(const FilterArgs &a, int *err, int num_sms, cudaStream_t s) {
    using L = ColStage<W, CS>;
    const int smem = 4 * L::kWarpBytes;
    int per_sm = 0;
    BMJ_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_filter_tma<W, R, CS, kFault>,
                                                            128, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (int64_t)num_sms * per_sm;
    const int64_t need_blocks = (a.n_items + 3) / 4;
    if (need_blocks < blocks) blocks = need_blocks;
    if (blocks < 1) blocks = 1;
    BMJ_LAUNCH((k_filter_tma<W, R, CS, kFault>), (unsigned)blocks, 128, smem, s, a, err);
    return BMJ_OK;
}

template <int W, int R, int CS>
int launch_filter_tma_t(const FilterArgs &a, int *err, int num_sms, cudaStream_t s) {
    return a.fault_skip_copy ? launch_filter_tma_k<W, R, CS, true>(a, err, num_sms, s)
                             : launch_filter_tma_k<W, R, CS, false>(a, err, num_sms, s);
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
        case 1: return launch_filter_tma_t<1, kTmaR1, 256>(a, err, num_sms, s);
        case 2: return launch_filter_tma_t<2, kTmaR2, 256>(a, err, num_sms, s);
        case 4: return launch_filter_tma_t<4, kTmaR4, 128>(a, err, num_sms, s);
        default: return launch_filter(a, W, num_sms, s);
    }
}

}  // namespace bmj
