// noalloc.cu -- the Bitmap Filter for callers that cannot allocate device memory.
//
// bmj_bitmap_filter_noalloc runs the same filter kernel as bmj_self_join, but
// every piece of scratch it needs (the window tile table, the per-|x|+|y|
// threshold table and the work/survivor counters) lives in one file-scope
// device array of fixed size instead of coming from cudaMalloc.  The caller
// passes the inputs (size-sorted bitmaps and sizes) and the output buffer.
//
// The array exists once per device that loads this library and stays
// allocated until the process exits.  Its device address is looked up once
// per device (cudaGetSymbolAddress, with that device current) on the first
// call made on that device.  All calls share the array, so calls that overlap
// on the GPU (other streams, other host threads) race on it.
#include <mutex>

#include "kernels.cuh"

namespace bmj {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[BMJ_NOALLOC_SCRATCH_BYTES];

constexpr int kSetupThreads = 1024;

__device__ __forceinline__ int64_t lower_bound_sizes(const uint32_t *a, int64_t n, uint64_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((uint64_t)a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// One block: clears the counters, checks that sizes are >= 1 and
// nondecreasing, fills lim[S] for S < n_s, and builds the tile table (first
// window column per tile and the exclusive prefix of column chunks per tile),
// exactly as the allocating path does.
__global__ void __launch_bounds__(kSetupThreads)
    k_noalloc_setup(const uint32_t *__restrict__ sizes, int64_t n, uint32_t p, uint32_t q,
                    int tile_rows, int chunk_cols, int64_t n_tiles, int64_t n_s,
                    unsigned long long *__restrict__ ctr, int32_t *__restrict__ lim,
                    int32_t *__restrict__ tile_c0, int64_t *__restrict__ tile_off) {
    __shared__ int64_t warp_sums[kSetupThreads / 32];
    __shared__ int64_t running;
    __shared__ int flags;
    if (threadIdx.x == 0) {
        running = 0;
        flags = 0;
        ctr[0] = 0;  // work-item counter
        ctr[1] = 0;  // survivor counter
    }
    __syncthreads();
    int f = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const uint32_t s = sizes[i];
        if (s == 0) f |= kFlagEmpty;
        if (i > 0 && s < sizes[i - 1]) f |= kFlagUnsorted;
    }
    if (f) atomicOr(&flags, f);
    const uint64_t d = (uint64_t)p + q;
    for (int64_t S = threadIdx.x; S < n_s; S += blockDim.x) {
        const uint64_t nd = ((uint64_t)S * p + d - 1) / d;     // ceil(p*S/(p+q))
        lim[S] = (int32_t)((int64_t)S - 2 * (int64_t)nd);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = 0; base < n_tiles; base += blockDim.x) {
        const int64_t t = base + threadIdx.x;
        int64_t items = 0;
        if (t < n_tiles) {
            const int64_t i0 = t * tile_rows;
            const uint64_t low = ((uint64_t)sizes[i0] * p + q - 1) / q;
            const int64_t c0 = lower_bound_sizes(sizes, n, low) & ~(int64_t)3;
            const int64_t c_end = min(i0 + (int64_t)tile_rows, n) - 1;
            const int64_t cols = c_end - c0;
            items = cols > 0 ? (cols + chunk_cols - 1) / chunk_cols : 0;
            tile_c0[t] = (int32_t)c0;
        }
        int64_t v = items;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (lane == 31) warp_sums[warp] = v;
        __syncthreads();
        int64_t woff = 0;
        for (int w = 0; w < warp; w++) woff += warp_sums[w];
        if (t < n_tiles) tile_off[t] = running + woff + v - items;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) running += woff + v;
        __syncthreads();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        tile_off[n_tiles] = running;
        ctr[3] = (unsigned long long)flags;
    }
}

std::mutex g_scratch_mu;
unsigned char *g_scratch_addr[128] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
int scratch_address(unsigned char **out) {
    int dev = 0;
    BMJ_CHECK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) return BMJ_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return status_of(e);
        }
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[dev];
    return BMJ_OK;
}

inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

int filter_noalloc_impl(const uint64_t *bitmaps, const uint32_t *sizes, int64_t n, int b,
                        uint32_t p, uint32_t q, uint32_t *out_pairs, int64_t out_cap,
                        int64_t *out_count, cudaStream_t s) {
    *out_count = 0;
    if (n < 2) return BMJ_OK;
    unsigned char *scratch = nullptr;
    int st = scratch_address(&scratch);
    if (st) return st;
    // The largest size is the last one when sizes are sorted (checked below
    // before any table is indexed with it).
    uint32_t max_size = 0;
    BMJ_CHECK(cudaMemcpyAsync(&max_size, sizes + (n - 1), sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    BMJ_CHECK(cudaStreamSynchronize(s));
    if (max_size > (uint32_t)kMaxSetSize) return BMJ_ERR_TOO_LARGE;
    const int W = b / 64;
    const int tile_rows = filter_tile_rows(W);
    const int chunk_cols = W <= 4 ? 4096 : 2048;
    const int64_t n_tiles = (n + tile_rows - 1) / tile_rows;
    const int64_t n_s = 2 * (int64_t)max_size + 1;
    const size_t off_lim = 256;
    const size_t off_c0 = align256(off_lim + (size_t)n_s * sizeof(int32_t));
    const size_t off_to = align256(off_c0 + (size_t)n_tiles * sizeof(int32_t));
    const size_t need = off_to + (size_t)(n_tiles + 1) * sizeof(int64_t);
    if (need > (size_t)BMJ_NOALLOC_SCRATCH_BYTES) return BMJ_ERR_TOO_LARGE;
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(scratch);
    int32_t *lim = reinterpret_cast<int32_t *>(scratch + off_lim);
    int32_t *tile_c0 = reinterpret_cast<int32_t *>(scratch + off_c0);
    int64_t *tile_off = reinterpret_cast<int64_t *>(scratch + off_to);

    BMJ_LAUNCH(k_noalloc_setup, 1, kSetupThreads, 0, s, sizes, n, p, q, tile_rows, chunk_cols,
               n_tiles, n_s, ctr, lim, tile_c0, tile_off);
    unsigned long long h[2] = {0, 0};
    BMJ_CHECK(cudaMemcpyAsync(&h[0], &ctr[3], sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    BMJ_CHECK(cudaMemcpyAsync(&h[1], &tile_off[n_tiles], sizeof(unsigned long long),
                              cudaMemcpyDeviceToHost, s));
    BMJ_CHECK(cudaStreamSynchronize(s));
    if (h[0] & kFlagUnsorted) return BMJ_ERR_UNSORTED;
    if (h[0] & kFlagEmpty) return BMJ_ERR_EMPTY_SET;

    int dev = 0, sms = 0;
    BMJ_CHECK(cudaGetDevice(&dev));
    BMJ_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    FilterArgs fa;
    fa.bm = bitmaps;
    fa.ssz = sizes;
    fa.lim = lim;
    fa.n = n;
    fa.p = p;
    fa.q = q;
    fa.tile_item_off = tile_off;
    fa.tile_c0 = tile_c0;
    fa.n_tiles = n_tiles;
    fa.n_items = (int64_t)h[1];
    fa.tile_rows = tile_rows;
    fa.chunk_cols = chunk_cols;
    fa.queue = reinterpret_cast<uint2 *>(out_pairs);
    fa.qcount = &ctr[1];
    fa.qcap = out_cap;
    fa.item_counter = &ctr[0];
    st = launch_filter(fa, W, sms, s);
    if (st) return st;
    unsigned long long cnt = 0;
    BMJ_CHECK(cudaMemcpyAsync(&cnt, &ctr[1], sizeof(cnt), cudaMemcpyDeviceToHost, s));
    BMJ_CHECK(cudaStreamSynchronize(s));
    *out_count = (int64_t)cnt;
    return (int64_t)cnt > out_cap ? BMJ_ERR_OUTPUT_OVERFLOW : BMJ_OK;
}

}  // namespace
}  // namespace bmj

extern "C" int bmj_bitmap_filter_noalloc(const uint64_t *bitmaps, const uint32_t *sizes,
                                         int64_t n_sets, int b, uint32_t p, uint32_t q,
                                         uint32_t *out_pairs, int64_t out_cap,
                                         int64_t *out_count, void *stream) {
    if (!out_count) return BMJ_ERR_INVALID_ARG;
    *out_count = 0;
    if (n_sets < 0 || out_cap < 0) return BMJ_ERR_INVALID_ARG;
    if (n_sets > 0x7fffffffLL) return BMJ_ERR_TOO_LARGE;
    if (b < 64 || b > 4096 || (b % 64) != 0) return BMJ_ERR_INVALID_ARG;
    if (p == 0 || q == 0 || p > q) return BMJ_ERR_INVALID_ARG;
    if (n_sets > 0 && (!bitmaps || !sizes)) return BMJ_ERR_INVALID_ARG;
    if (out_cap > 0 && (!out_pairs || (reinterpret_cast<uintptr_t>(out_pairs) & 7) != 0))
        return BMJ_ERR_INVALID_ARG;
    int st = bmj::filter_noalloc_impl(bitmaps, sizes, n_sets, b, p, q, out_pairs, out_cap,
                                      out_count, static_cast<cudaStream_t>(stream));
    if (st != BMJ_OK && st != BMJ_ERR_OUTPUT_OVERFLOW) cudaGetLastError();
    return st;
}
