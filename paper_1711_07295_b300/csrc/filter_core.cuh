// filter_core.cuh -- the Bitmap Filter over one work item, shared by the
// single-join and the batched kernels.
//
// A work item is a tile of 32*R consecutive size-sorted rows [i0, i0+32R)
// against the columns [c0, c1) of its length window.  Lane l owns rows
// i0 + l + 32k (k < R) with their bitmaps in registers.  Each group of 32
// columns is loaded coalesced (one column per lane) and broadcast with
// __shfl_sync, so one load serves 32*R pairs.
//
// For a pair (i, j), with S = |R[i]| + |R[j]| and h = popcount(b_i ^ b_j):
//   in window  <=>  q*min(|R[i]|,|R[j]|) >= p*max(...)   (Table 2)
//   survives   <=>  floor((S - h)/2) >= ceil(p*S/(p+q))  (Eq. 2 vs Table 1)
//              <=>  h <= lim[S]
// Each row keeps lim (or -1 outside the window) for the current column size,
// refreshed only when the warp-uniform column size changes.  Pairs with
// j >= i (diagonal part of a tile) and rows past row_end are excluded.
// Survivors of a 32-column group are reserved with one atomicAdd per warp
// (plus one on the per-job counter when given) and written as (i, j).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bmj {

__device__ __forceinline__ int warp_excl_scan_i(int v) {
    const int lane = threadIdx.x & 31;
    int x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += u;
    }
    return x - v;
}

// Survivor sink: global queue with a capacity (the count runs past it so an
// overflow is detected exactly) and an optional second counter (per job).
struct SurvivorSink {
    uint2 *queue;
    unsigned long long *count;
    unsigned long long *job_count;  // may be null
    int64_t cap;
};

template <int W, int R>
__device__ __forceinline__ void filter_item(const uint64_t *__restrict__ bm,
                                            const uint32_t *__restrict__ ssz,
                                            const int32_t *__restrict__ lim_tab, int64_t row_end,
                                            int64_t i0, int64_t c0, int64_t c1, uint32_t p,
                                            uint32_t q, const SurvivorSink &sink) {
    constexpr unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    uint64_t rb[R][W];
    uint32_t rs[R];
    int64_t ri[R];
#pragma unroll
    for (int k = 0; k < R; k++) {
        const int64_t i = i0 + k * 32 + lane;
        ri[k] = i;
        if (i < row_end) {
            rs[k] = ssz[i];
#pragma unroll
            for (int w = 0; w < W; w++) rb[k][w] = bm[i * W + w];
        } else {
            rs[k] = 0;
#pragma unroll
            for (int w = 0; w < W; w++) rb[k][w] = 0;
        }
    }
    int lim[R];
    uint32_t prev_cs = 0xffffffffu;
#pragma unroll
    for (int k = 0; k < R; k++) lim[k] = -1;

    for (int64_t j = c0; j < c1; j += 32) {
        const int gj = (int)min((int64_t)32, c1 - j);
        uint64_t cb[W];
        uint32_t cs = 0;
        if (lane < gj) {
            cs = ssz[j + lane];
#pragma unroll
            for (int w = 0; w < W; w++) cb[w] = bm[(j + lane) * W + w];
        } else {
#pragma unroll
            for (int w = 0; w < W; w++) cb[w] = 0;
        }
        const bool diag = (j + gj - 1) >= i0;
        uint32_t mask[R];
#pragma unroll
        for (int k = 0; k < R; k++) mask[k] = 0;
        uint32_t bit = 1u;
        for (int cc = 0; cc < gj; cc++, bit <<= 1) {
            const uint32_t s = __shfl_sync(kFull, cs, cc);
            uint64_t c[W];
#pragma unroll
            for (int w = 0; w < W; w++) c[w] = __shfl_sync(kFull, cb[w], cc);
            if (s != prev_cs) {  // warp-uniform
                prev_cs = s;
#pragma unroll
                for (int k = 0; k < R; k++) {
                    const uint32_t mn = min(rs[k], s), mx = max(rs[k], s);
                    const bool in_win = rs[k] != 0 && (uint64_t)q * mn >= (uint64_t)p * mx;
                    lim[k] = in_win ? lim_tab[rs[k] + s] : -1;
                }
            }
#pragma unroll
            for (int k = 0; k < R; k++) {
                int h = 0;
#pragma unroll
                for (int w = 0; w < W; w++) h += __popcll(rb[k][w] ^ c[w]);
                bool sv = h <= lim[k];
                if (diag) sv = sv && (j + cc < ri[k]);
                if (sv) mask[k] |= bit;
            }
        }
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < R; k++) cnt += __popc(mask[k]);
        const int total = __reduce_add_sync(kFull, cnt);
        if (total) {
            const int excl = warp_excl_scan_i(cnt);
            unsigned long long base = 0;
            if (lane == 0) {
                base = atomicAdd(sink.count, (unsigned long long)total);
                if (sink.job_count) atomicAdd(sink.job_count, (unsigned long long)total);
            }
            base = __shfl_sync(kFull, base, 0);
            unsigned long long pos = base + excl;
#pragma unroll
            for (int k = 0; k < R; k++) {
                uint32_t m = mask[k];
                while (m) {
                    const int bpos = __ffs(m) - 1;
                    m &= m - 1;
                    if (pos < (unsigned long long)sink.cap)
                        sink.queue[pos] = make_uint2((uint32_t)ri[k], (uint32_t)(j + bpos));
                    pos++;
                }
            }
        }
    }
}

// Generic width (b not in {64,128,256,512}): one row per lane, bitmaps read
// word by word from memory.
__device__ __forceinline__ void filter_item_generic(const uint64_t *__restrict__ bm,
                                                    const uint32_t *__restrict__ ssz,
                                                    const int32_t *__restrict__ lim_tab,
                                                    int64_t row_end, int64_t i0, int64_t c0,
                                                    int64_t c1, uint32_t p, uint32_t q, int W,
                                                    const SurvivorSink &sink) {
    constexpr unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t i = i0 + lane;
    const uint32_t rs = i < row_end ? ssz[i] : 0u;
    const uint64_t *rowp = bm + (i < row_end ? i : i0) * W;
    for (int64_t j = c0; j < c1; j += 32) {
        const int gj = (int)min((int64_t)32, c1 - j);
        uint32_t mask = 0;
        for (int cc = 0; cc < gj; cc++) {
            const int64_t jj = j + cc;
            const uint32_t s = ssz[jj];
            const uint32_t mn = min(rs, s), mx = max(rs, s);
            const bool in_win = rs != 0 && (uint64_t)q * mn >= (uint64_t)p * mx;
            if (!in_win || jj >= i) continue;
            const uint64_t *colp = bm + jj * W;
            int h = 0;
            for (int w = 0; w < W; w++) h += __popcll(rowp[w] ^ colp[w]);
            if (h <= lim_tab[rs + s]) mask |= 1u << cc;
        }
        const int cnt = __popc(mask);
        const int total = __reduce_add_sync(kFull, cnt);
        if (total) {
            const int excl = warp_excl_scan_i(cnt);
            unsigned long long base = 0;
            if (lane == 0) {
                base = atomicAdd(sink.count, (unsigned long long)total);
                if (sink.job_count) atomicAdd(sink.job_count, (unsigned long long)total);
            }
            base = __shfl_sync(kFull, base, 0);
            unsigned long long pos = base + excl;
            uint32_t m = mask;
            while (m) {
                const int bpos = __ffs(m) - 1;
                m &= m - 1;
                if (pos < (unsigned long long)sink.cap)
                    sink.queue[pos] = make_uint2((uint32_t)i, (uint32_t)(j + bpos));
                pos++;
            }
        }
    }
}

// Largest t in [0, n_tiles) with tile_item_off[t] <= item (tile_item_off has
// n_tiles + 1 entries and tile_item_off[n_tiles] > item).
__device__ __forceinline__ int64_t find_tile(const int64_t *__restrict__ tile_item_off,
                                             int64_t n_tiles, unsigned long long item) {
    int64_t lo = 0, hi = n_tiles;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if ((unsigned long long)tile_item_off[mid] <= item) lo = mid;
        else hi = mid;
    }
    return lo;
}

}  // namespace bmj
