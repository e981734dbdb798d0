// kernels.cu -- preparation kernels of the Bitmap Filter self-join.
//
// Stages (each cited where it is defined in the paper):
//   k_validate       CSR invariants; sizes and ids for the size sort (Section 5
//                    preprocessing: sets ordered by size)
//   k_gather_build   sorted CSR gather + b-bit bitmaps (Section 3.2, Alg. 3a/3b/3c,
//                    h(t) = t mod b as in Section 5.1)
//   k_tables         need[S] / lim[S]: Jaccard as an overlap threshold (Table 1)
//                    folded into the Eq. 2 test
//   k_build_multi    the same for 64-, 128- and 256-bit Xor/Set bitmaps in one pass
//   k_tiles,
//   k_window_count   the length filter window j in [j0(i), i) (Table 2; Alg. 6)
//   k_rs_tiles,
//   k_rs_window_count  the same for an RS-join: the columns of S in a row's
//                    window (both bounds of Table 2)
// The Bitmap Filter is in filter.cu, verification and output in verify.cu.
#include "kernels.cuh"

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

// One thread per set: writes its Xor (Alg. 3b) or Set (Alg. 3a) bitmaps for
// up to three widths at once (64, 128, 256 bits; a null output skips a
// width).  With b a power of two, h(t) = t mod b selects word (t mod b) / 64
// and bit t mod 64 for all three widths.  When stok is given the warp then
// gathers its 32 sets' tokens into the sorted CSR together, one set at a
// time with consecutive lanes on consecutive tokens, so that the writes are
// whole sectors (per-thread writes left partial sectors that DRAM had to
// merge, doubling the traffic).
__global__ void __launch_bounds__(256)
    k_build_multi(const uint32_t *__restrict__ perm, const int64_t *__restrict__ off,
                  const int32_t *__restrict__ tok, const int64_t *__restrict__ soff,
                  int32_t *__restrict__ stok, int64_t n, int method, uint64_t *__restrict__ bm64,
                  uint64_t *__restrict__ bm128, uint64_t *__restrict__ bm256) {
    const bool xr = method == BMJ_XOR;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // whole warps iterate together (the gather below is warp-wide)
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < n; i0 += stride) {
        const int64_t i = i0 + lane;
        const bool live = i < n;
        const int64_t src = live ? (perm ? (int64_t)perm[i] : i) : 0;
        const int64_t lo = live ? off[src] : 0;
        const int64_t cnt = live ? off[src + 1] - lo : 0;
        const int32_t *x = tok + lo;
        uint64_t a = 0, b0 = 0, b1 = 0, c0 = 0, c1 = 0, c2 = 0, c3 = 0;
        for (int64_t k = 0; k < cnt; k++) {
            const uint32_t t = (uint32_t)x[k];
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
        if (live) {
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
        if (stok) {
            const int64_t dst = live ? soff[i] : 0;
            const int nl = (int)min((int64_t)32, n - i0);
            for (int l = 0; l < nl; l++) {
                const int64_t lo_l = __shfl_sync(kFull, lo, l);
                const int64_t cnt_l = __shfl_sync(kFull, cnt, l);
                const int64_t dst_l = __shfl_sync(kFull, dst, l);
                for (int64_t k = lane; k < cnt_l; k += 32) stok[dst_l + k] = tok[lo_l + k];
            }
        }
    }
}

// need[S] / lim[S] for the functions whose smallest passing overlap depends on
// S = |x|+|y| alone (Jaccard, Dice, Overlap; Cosine computes them per pair).
__global__ void k_tables(int32_t *__restrict__ need, int32_t *__restrict__ lim, int64_t n_s,
                         int sim, uint32_t p, uint32_t q) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t S = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; S < n_s; S += stride) {
        // e.g. Jaccard >= p/q  <=>  o*(p+q) >= p*S  <=>  o >= ceil(p*S/(p+q)) (Table 1).
        const int64_t nd = sim == BMJ_COSINE ? 0 : need_of_sum(sim, p, q, S);
        need[S] = (int32_t)nd;
        // floor((S - h)/2) >= nd  <=>  h <= S - 2*nd (Eq. 2 with its floor).
        lim[S] = (int32_t)(S - 2 * nd);
    }
}

__global__ void k_tiles(const uint32_t *__restrict__ ssz, int64_t n, SimWindow win,
                        int tile_rows, int chunk_cols, int64_t n_tiles,
                        int32_t *__restrict__ tile_c0, int64_t *__restrict__ tile_items,
                        int64_t row0, int64_t row_end) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += stride) {
        const int64_t i0 = row0 + t * tile_rows;
        const int64_t j0 = lower_bound_u32(ssz, n, window_low(ssz[i0], win));
        const int64_t c0 = j0 & ~(int64_t)3;
        const int64_t c_end = min(i0 + (int64_t)tile_rows, row_end) - 1;  // columns j < i <= c_end
        const int64_t cols = c_end - c0;
        tile_c0[t] = (int32_t)c0;
        tile_items[t] = cols > 0 ? (cols + chunk_cols - 1) / chunk_cols : 0;
    }
}

__global__ void k_window_count(const uint32_t *__restrict__ ssz, int64_t n, SimWindow win,
                               unsigned long long *__restrict__ out, int64_t row0,
                               int64_t row_end) {
    unsigned long long acc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = row0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < row_end; i += stride) {
        const int64_t j0 = lower_bound_u32(ssz, n, window_low(ssz[i], win));
        if (j0 < i) acc += (unsigned long long)(i - j0);
    }
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(kFull, acc, d);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

// ---- RS-join (R and S in one size-sorted array: S at [0, n_cols), R after) ----
// The columns of S inside the window of a row of size x: sizes in
// [window_low(x), window_high(x)], a contiguous range [lo, hi) of the sorted S.
__device__ __forceinline__ void rs_cols(const uint32_t *__restrict__ ssz, int64_t n_cols,
                                        uint64_t x_lo, uint64_t x_hi, SimWindow win, int64_t *lo,
                                        int64_t *hi) {
    *lo = lower_bound_u32(ssz, n_cols, window_low(x_lo, win));
    const uint64_t top = window_high(x_hi, win);
    *hi = top == ~0ull ? n_cols : lower_bound_u32(ssz, n_cols, top + 1);
}

__global__ void k_rs_tiles(const uint32_t *__restrict__ ssz, int64_t n_cols, SimWindow win,
                           int tile_rows, int chunk_cols, int64_t n_tiles,
                           int32_t *__restrict__ tile_c0, int32_t *__restrict__ tile_c1,
                           int64_t *__restrict__ tile_items, int64_t row0, int64_t row_end) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += stride) {
        const int64_t i0 = row0 + t * tile_rows;
        const int64_t i1 = min(i0 + (int64_t)tile_rows, row_end) - 1;
        int64_t lo, hi;
        rs_cols(ssz, n_cols, ssz[i0], ssz[i1], win, &lo, &hi);  // union of the rows' windows
        const int64_t c0 = lo & ~(int64_t)3;
        const int64_t cols = hi - c0;
        tile_c0[t] = (int32_t)c0;
        tile_c1[t] = (int32_t)(hi > c0 ? hi : c0);
        tile_items[t] = (hi > lo && cols > 0) ? (cols + chunk_cols - 1) / chunk_cols : 0;
    }
}

__global__ void k_rs_window_count(const uint32_t *__restrict__ ssz, int64_t n_cols, SimWindow win,
                                  unsigned long long *__restrict__ out, int64_t row0,
                                  int64_t row_end) {
    unsigned long long acc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = row0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < row_end; i += stride) {
        int64_t lo, hi;
        rs_cols(ssz, n_cols, ssz[i], ssz[i], win, &lo, &hi);
        if (hi > lo) acc += (unsigned long long)(hi - lo);
    }
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(kFull, acc, d);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

// v[i] |= bit for i in [0, n) (marks the sort keys of R so that R sorts after S).
__global__ void k_or_bits(uint32_t *__restrict__ v, int64_t n, uint32_t bit) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) v[i] |= bit;
}

__global__ void k_and_bits(uint32_t *__restrict__ v, int64_t n, uint32_t mask) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) v[i] &= mask;
}

__global__ void k_add_i64(int64_t *__restrict__ v, int64_t n, int64_t add) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) v[i] += add;
}

unsigned grid_for(int64_t n, int threads, int64_t cap = 148 * 32) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
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

int launch_tables(int32_t *need, int32_t *lim, int64_t n_s, int sim, uint32_t p, uint32_t q,
                  cudaStream_t s) {
    BMJ_LAUNCH(k_tables, grid_for(n_s, 256), 256, 0, s, need, lim, n_s, sim, p, q);
    return BMJ_OK;
}

int launch_tiles(const uint32_t *ssz, int64_t n, SimWindow win, int tile_rows,
                 int chunk_cols, int64_t n_tiles, int32_t *tile_c0, int64_t *tile_items,
                 cudaStream_t s, int64_t row0, int64_t row_end) {
    if (n_tiles <= 0) return BMJ_OK;
    BMJ_LAUNCH(k_tiles, grid_for(n_tiles, 256), 256, 0, s, ssz, n, win, tile_rows, chunk_cols,
               n_tiles, tile_c0, tile_items, row0, row_end < 0 ? n : row_end);
    return BMJ_OK;
}

int launch_window_count(const uint32_t *ssz, int64_t n, SimWindow win,
                        unsigned long long *out, cudaStream_t s, int64_t row0, int64_t row_end) {
    if (row_end < 0) row_end = n;
    if (row_end <= row0) return BMJ_OK;
    BMJ_LAUNCH(k_window_count, grid_for(row_end - row0, 256), 256, 0, s, ssz, n, win, out, row0,
               row_end);
    return BMJ_OK;
}

int launch_rs_tiles(const uint32_t *ssz, int64_t n_cols, SimWindow win, int tile_rows,
                    int chunk_cols, int64_t n_tiles, int32_t *tile_c0, int32_t *tile_c1,
                    int64_t *tile_items, int64_t row0, int64_t row_end, cudaStream_t s) {
    if (n_tiles <= 0) return BMJ_OK;
    BMJ_LAUNCH(k_rs_tiles, grid_for(n_tiles, 256), 256, 0, s, ssz, n_cols, win, tile_rows,
               chunk_cols, n_tiles, tile_c0, tile_c1, tile_items, row0, row_end);
    return BMJ_OK;
}

int launch_rs_window_count(const uint32_t *ssz, int64_t n_cols, SimWindow win,
                           unsigned long long *out, int64_t row0, int64_t row_end,
                           cudaStream_t s) {
    if (row_end <= row0) return BMJ_OK;
    BMJ_LAUNCH(k_rs_window_count, grid_for(row_end - row0, 256), 256, 0, s, ssz, n_cols, win, out,
               row0, row_end);
    return BMJ_OK;
}

int launch_or_bits(uint32_t *v, int64_t n, uint32_t bit, cudaStream_t s) {
    if (n <= 0) return BMJ_OK;
    BMJ_LAUNCH(k_or_bits, grid_for(n, 256), 256, 0, s, v, n, bit);
    return BMJ_OK;
}

int launch_and_bits(uint32_t *v, int64_t n, uint32_t mask, cudaStream_t s) {
    if (n <= 0) return BMJ_OK;
    BMJ_LAUNCH(k_and_bits, grid_for(n, 256), 256, 0, s, v, n, mask);
    return BMJ_OK;
}

int launch_add_i64(int64_t *v, int64_t n, int64_t add, cudaStream_t s) {
    if (n <= 0) return BMJ_OK;
    BMJ_LAUNCH(k_add_i64, grid_for(n, 256), 256, 0, s, v, n, add);
    return BMJ_OK;
}

}  // namespace bmj
