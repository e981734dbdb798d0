// scan_sort.cu -- device-wide exclusive scan and stable LSD radix sort.
//
// Used for the size sort of the collection (sets ordered by size, ties by
// original id: the preprocessing of Section 5) and for the canonical order of
// the result pairs.  Both are plain, deterministic building blocks:
//   scan:  tile-local scans (4096 items per 256-thread block), a recursive
//          scan of the tile totals, then a pass that adds the tile offsets;
//   sort:  per pass an 8-bit digit histogram per tile, an exclusive scan of
//          the digit-major histogram, then a stable scatter in which every
//          warp ranks its items by ballots over the digit bits and a per-warp
//          histogram in shared memory.
#include "bmj_internal.cuh"

namespace bmj {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;  // 4096
constexpr int kWarps = kThreads / 32;

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += u;
    }
    return v;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_scan_tiles(const T *in, T *out, int64_t n,
                                                         T *tile_sums) {
    __shared__ T s[kTile];
    __shared__ T warp_tot[kWarps];
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int k = threadIdx.x; k < kTile; k += kThreads) {
        int64_t i = base + k;
        s[k] = i < n ? in[i] : T(0);
    }
    __syncthreads();
    T local[kItems];
    T sum = 0;
#pragma unroll
    for (int k = 0; k < kItems; k++) {
        local[k] = s[threadIdx.x * kItems + k];
        sum += local[k];
    }
    T incl = warp_inclusive_scan(sum);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    T woff = 0;
    for (int w = 0; w < warp; w++) woff += warp_tot[w];
    T run = incl - sum + woff;
#pragma unroll
    for (int k = 0; k < kItems; k++) {
        s[threadIdx.x * kItems + k] = run;
        run += local[k];
    }
    if (threadIdx.x == kThreads - 1) tile_sums[blockIdx.x] = run;
    __syncthreads();
    for (int k = threadIdx.x; k < kTile; k += kThreads) {
        int64_t i = base + k;
        if (i < n) out[i] = s[k];
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_add_tile_offsets(T *out, int64_t n,
                                                               const T *tile_offsets) {
    const int64_t base = (int64_t)blockIdx.x * kTile;
    const T add = tile_offsets[blockIdx.x];
    for (int k = threadIdx.x; k < kTile; k += kThreads) {
        int64_t i = base + k;
        if (i < n) out[i] += add;
    }
}

template <typename T>
int scan_impl(const T *in, T *out, int64_t n, T *total_dev, Arena &arena, cudaStream_t s) {
    if (n <= 0) {
        if (total_dev) BMJ_CHECK(cudaMemsetAsync(total_dev, 0, sizeof(T), s));
        return BMJ_OK;
    }
    const int64_t tiles = (n + kTile - 1) / kTile;
    T *sums = nullptr;
    int st = arena.alloc(&sums, (size_t)tiles);
    if (st) return st;
    BMJ_LAUNCH(k_scan_tiles<T>, (unsigned)tiles, kThreads, 0, s, in, out, n, sums);
    if (tiles == 1) {
        if (total_dev)
            BMJ_CHECK(cudaMemcpyAsync(total_dev, sums, sizeof(T), cudaMemcpyDeviceToDevice, s));
        return BMJ_OK;
    }
    st = scan_impl<T>(sums, sums, tiles, total_dev, arena, s);
    if (st) return st;
    BMJ_LAUNCH(k_add_tile_offsets<T>, (unsigned)tiles, kThreads, 0, s, out, n, sums);
    return BMJ_OK;
}

// ---------------------------------------------------------------------------
// Radix sort
// ---------------------------------------------------------------------------
template <typename K>
__global__ void __launch_bounds__(kThreads) k_radix_hist(const K *keys, int64_t n, int shift,
                                                         uint32_t *hist) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int k = threadIdx.x; k < kTile; k += kThreads) {
        int64_t i = base + k;
        if (i < n) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one 8-bit digit.  Warp w of a block owns the contiguous
// items [tile + w*512, tile + (w+1)*512); iteration `it` covers 32 of them in
// lane order, so ranks follow the input order inside the tile.
template <typename K, typename V, bool kHasVals>
__global__ void __launch_bounds__(kThreads) k_radix_scatter(const K *keys_in, const V *vals_in,
                                                            K *keys_out, V *vals_out, int64_t n,
                                                            int shift,
                                                            const uint32_t *digit_offsets,
                                                            const uint32_t *chunk_offsets) {
    __shared__ uint32_t warp_hist[kWarps][257];
    __shared__ uint32_t block_base[256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = threadIdx.x; k < kWarps * 257; k += kThreads) (&warp_hist[0][0])[k] = 0;
    {  // this block's start for its digit: the chunk-local scan plus its chunk's offset
        const int64_t h = (int64_t)threadIdx.x * gridDim.x + blockIdx.x;
        block_base[threadIdx.x] = digit_offsets[h] + (chunk_offsets ? chunk_offsets[h / kTile] : 0u);
    }
    __syncthreads();
    const int64_t wbase = (int64_t)blockIdx.x * kTile + (int64_t)warp * 32 * kItems;
    const uint32_t lt_mask = (1u << lane) - 1u;
    K key[kItems];
    V val[kItems];
    uint32_t rank[kItems];
#pragma unroll
    for (int it = 0; it < kItems; it++) {
        const int64_t i = wbase + it * 32 + lane;
        const bool valid = i < n;
        uint32_t d = 256;  // invalid lanes form their own group
        if (valid) {
            key[it] = keys_in[i];
            if (kHasVals) val[it] = vals_in[i];
            d = (uint32_t)(key[it] >> shift) & 255u;
        }
        // the lanes holding the same digit: one ballot per digit bit (a little
        // faster than __match_any_sync here); an invalid lane is a group alone
        uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
        for (int bit = 0; bit < 8; bit++) {
            const unsigned bal = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
            peers &= ((d >> bit) & 1u) ? bal : ~bal;
        }
        if (!valid) peers = 1u << lane;
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (lane == leader) {
            base = warp_hist[warp][d];
            warp_hist[warp][d] = base + __popc(peers);
        }
        base = __shfl_sync(0xffffffffu, base, leader);
        rank[it] = (base + __popc(peers & lt_mask)) | (d << 20);  // rank < 512 fits below bit 20
        __syncwarp();
    }
    __syncthreads();
    // Exclusive prefix over warps, per digit.
    {
        const int d = threadIdx.x;
        uint32_t sum = 0;
        for (int w = 0; w < kWarps; w++) {
            uint32_t t = warp_hist[w][d];
            warp_hist[w][d] = sum;
            sum += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kItems; it++) {
        const int64_t i = wbase + it * 32 + lane;
        if (i < n) {
            const uint32_t d = rank[it] >> 20;
            const uint32_t r = rank[it] & 0xfffffu;
            const int64_t pos = (int64_t)block_base[d] + warp_hist[warp][d] + r;
            keys_out[pos] = key[it];
            if (kHasVals) vals_out[pos] = val[it];
        }
    }
}

template <typename K, typename V, bool kHasVals>
int radix_impl(const K *keys_in, const V *vals_in, K *keys_out, V *vals_out, int64_t n,
               int key_bits, Arena &arena, cudaStream_t s) {
    if (n <= 0) return BMJ_OK;
    const int passes = (key_bits + 7) / 8;
    if (passes == 0 || n == 1) {
        if (keys_out != keys_in)
            BMJ_CHECK(cudaMemcpyAsync(keys_out, keys_in, n * sizeof(K), cudaMemcpyDeviceToDevice, s));
        if (kHasVals && vals_out != vals_in)
            BMJ_CHECK(cudaMemcpyAsync(vals_out, vals_in, n * sizeof(V), cudaMemcpyDeviceToDevice, s));
        return BMJ_OK;
    }
    const int64_t tiles = (n + kTile - 1) / kTile;
    if (tiles > 0x7fffffff) return BMJ_ERR_TOO_LARGE;
    K *tk = nullptr;
    V *tv = nullptr;
    uint32_t *hist = nullptr;
    int st = arena.alloc(&tk, (size_t)n);
    if (!st && kHasVals) st = arena.alloc(&tv, (size_t)n);
    if (!st) st = arena.alloc(&hist, (size_t)tiles * 256);
    uint32_t *csum = nullptr;  // totals of the histogram's scan chunks
    if (!st) st = arena.alloc(&csum, (size_t)((tiles * 256 + kTile - 1) / kTile));
    if (st) return st;
    const K *src_k = keys_in;
    const V *src_v = vals_in;
    for (int pass = 0; pass < passes; pass++) {
        // The last pass must land in keys_out.
        const bool to_out = ((passes - 1 - pass) % 2) == 0;
        K *dst_k = to_out ? keys_out : tk;
        V *dst_v = to_out ? vals_out : tv;
        const int shift = 8 * pass;
        BMJ_LAUNCH(k_radix_hist<K>, (unsigned)tiles, kThreads, 0, s, src_k, n, shift, hist);
        // The digit-major histogram is scanned in chunks of kTile entries; the
        // chunk totals are scanned on their own, and the scatter adds a chunk's
        // offset itself (one launch fewer per pass than a full scan).
        const int64_t m = tiles * 256;
        if (m <= kTile) {
            BMJ_LAUNCH(k_scan_tiles<uint32_t>, 1u, kThreads, 0, s, hist, hist, m, csum);
        } else {
            BMJ_LAUNCH(k_scan_tiles<uint32_t>, (unsigned)((m + kTile - 1) / kTile), kThreads, 0, s,
                       hist, hist, m, csum);
            st = scan_impl<uint32_t>(csum, csum, (m + kTile - 1) / kTile, nullptr, arena, s);
            if (st) return st;
        }
        BMJ_LAUNCH((k_radix_scatter<K, V, kHasVals>), (unsigned)tiles, kThreads, 0, s, src_k,
                   src_v, dst_k, dst_v, n, shift, hist, m <= kTile ? nullptr : csum);
        src_k = dst_k;
        src_v = dst_v;
    }
    return BMJ_OK;
}

}  // namespace

int exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total_dev,
                       Arena &arena, cudaStream_t s) {
    return scan_impl<int64_t>(in, out, n, total_dev, arena, s);
}

int exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, Arena &arena,
                       cudaStream_t s) {
    return scan_impl<uint32_t>(in, out, n, nullptr, arena, s);
}

int radix_sort_u32_pairs(const uint32_t *keys_in, const uint32_t *vals_in, uint32_t *keys_out,
                         uint32_t *vals_out, int64_t n, int key_bits, Arena &arena,
                         cudaStream_t s) {
    return radix_impl<uint32_t, uint32_t, true>(keys_in, vals_in, keys_out, vals_out, n, key_bits,
                                                arena, s);
}

int radix_sort_u32(const uint32_t *keys_in, uint32_t *keys_out, int64_t n, int key_bits,
                   Arena &arena, cudaStream_t s) {
    return radix_impl<uint32_t, uint32_t, false>(keys_in, nullptr, keys_out, nullptr, n, key_bits,
                                                 arena, s);
}

int radix_sort_u64(const uint64_t *keys_in, uint64_t *keys_out, int64_t n, int key_bits,
                   Arena &arena, cudaStream_t s) {
    return radix_impl<uint64_t, uint32_t, false>(keys_in, nullptr, keys_out, nullptr, n, key_bits,
                                                 arena, s);
}

}  // namespace bmj
