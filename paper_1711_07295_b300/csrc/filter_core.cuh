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

#include "sim.cuh"

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

// The similarity function's window (Table 2) and threshold.
struct SimArgs {
    SimWindow win;
    uint32_t p, q;
    uint32_t cut = 0xffffffffu;  // cutoff point: a pair whose larger size exceeds it skips Eq. 2
};

// Eq. 2 limit of a pair of sizes: from the table indexed by |x|+|y| (Jaccard,
// Dice, Overlap), or computed (Cosine, whose limit depends on |x|*|y|).
template <bool kCos>
__device__ __forceinline__ int32_t pair_lim(const int32_t *__restrict__ lim_tab, uint32_t x,
                                            uint32_t y, const SimArgs &sa) {
    if (kCos) return (int32_t)sim_lim(BMJ_COSINE, sa.p, sa.q, x, y);
    return lim_tab[x + y];
}

template <int W, int R, bool kCos = false>
__device__ __forceinline__ void filter_item(const uint64_t *__restrict__ bm,
                                            const uint32_t *__restrict__ ssz,
                                            const int32_t *__restrict__ lim_tab, int64_t row_end,
                                            int64_t i0, int64_t c0, int64_t c1, const SimArgs &sa,
                                            const SurvivorSink &sink) {
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
                    const bool in_win = rs[k] != 0 && in_window(mn, mx, sa.win);
                    lim[k] = !in_win ? -1 : mx > sa.cut ? (1 << 30) : pair_lim<kCos>(lim_tab, rs[k], s, sa);
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
template <bool kCos = false>
__device__ __forceinline__ void filter_item_generic(const uint64_t *__restrict__ bm,
                                                    const uint32_t *__restrict__ ssz,
                                                    const int32_t *__restrict__ lim_tab,
                                                    int64_t row_end, int64_t i0, int64_t c0,
                                                    int64_t c1, const SimArgs &sa, int W,
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
            const bool in_win = rs != 0 && in_window(mn, mx, sa.win);
            if (!in_win || jj >= i) continue;
            const uint64_t *colp = bm + jj * W;
            int h = 0;
            for (int w = 0; w < W; w++) h += __popcll(rowp[w] ^ colp[w]);
            if (mx > sa.cut || h <= pair_lim<kCos>(lim_tab, rs, s, sa)) mask |= 1u << cc;
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


// ============================================================================
// Filter with TMA-staged columns.
//
// Each warp owns a double buffer in shared memory.  Column chunks (bitmaps and
// sizes of up to CS consecutive sorted sets) are copied in by one-dimensional
// bulk copies (cp.async.bulk, completion on an mbarrier), one chunk ahead of
// the compute.  Every column is then read by all lanes from shared memory (a
// broadcast), so the per-pair work is: xor, popcount, one IADD3 and one funnel
// shift that appends the survive bit to the row's 32-column mask.
//
// Survive test: h <= lim  <=>  h + (-(lim + 1)) < 0, so the sign bit of
// t = h + nlim (nlim = -(lim+1); nlim = 0 outside the window, where lim = -1)
// is the survive bit.
//
// For b >= 128 the popcount of the xor words uses carry-save adders
// (Harley-Seal): three words a, b, c become sum = a^b^c and carry =
// maj(a,b,c) with popc(a)+popc(b)+popc(c) = popc(sum) + 2*popc(carry), which
// trades POPC (16 per clock per SM) for LOP3 (64 per clock per SM).
// ============================================================================

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Waits for the phase `parity` of bar, giving up after `limit` polls
// (returns false then).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int limit) {
    const uint32_t addr = smem_u32(bar);
    for (int it = 0; it < limit; it++) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(addr), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Population count of a 64-bit word (lo, hi) with ALU operations only:
// pairwise bit sums (2-bit fields), then 4-bit fields, the two halves added,
// then byte fields summed by a multiply.  Used for one row in eight so that
// part of the popcount work runs on the ALU and FMA pipes instead of POPC.
__device__ __forceinline__ int popc64_alu(uint32_t lo, uint32_t hi) {
    lo = lo - ((lo >> 1) & 0x55555555u);
    hi = hi - ((hi >> 1) & 0x55555555u);
    lo = (lo & 0x33333333u) + ((lo >> 2) & 0x33333333u);
    hi = (hi & 0x33333333u) + ((hi >> 2) & 0x33333333u);
    uint32_t v = lo + hi;                                      // 4-bit fields, each <= 8
    v = (v & 0x0F0F0F0Fu) + ((v >> 4) & 0x0F0F0F0Fu);          // byte fields, each <= 16
    return (int)((v * 0x01010101u) >> 24);                     // sum of the four bytes (<= 64)
}

template <int W>
struct PopcHS;

template <>
struct PopcHS<1> {
    __device__ __forceinline__ static int h(const uint32_t *x) {
        return __popc(x[0]) + __popc(x[1]);
    }
};

template <>
struct PopcHS<2> {
    // 4 words: one carry-save adder on 3 of them -> 3 POPC.
    __device__ __forceinline__ static int h(const uint32_t *x) {
        const uint32_t s = x[0] ^ x[1] ^ x[2];
        const uint32_t c = (x[0] & x[1]) | (x[2] & (x[0] ^ x[1]));
        return __popc(s) + __popc(x[3]) + 2 * __popc(c);
    }
};

template <>
struct PopcHS<4> {
    // 8 words: four carry-save adders -> 4 POPC.
    __device__ __forceinline__ static int h(const uint32_t *x) {
        const uint32_t s1 = x[0] ^ x[1] ^ x[2];
        const uint32_t c1 = (x[0] & x[1]) | (x[2] & (x[0] ^ x[1]));
        const uint32_t s2 = x[3] ^ x[4] ^ x[5];
        const uint32_t c2 = (x[3] & x[4]) | (x[5] & (x[3] ^ x[4]));
        const uint32_t s3 = s1 ^ s2 ^ x[6];
        const uint32_t c3 = (s1 & s2) | (x[6] & (s1 ^ s2));
        const uint32_t s4 = c1 ^ c2 ^ c3;
        const uint32_t c4 = (c1 & c2) | (c3 & (c1 ^ c2));
        return __popc(s3) + __popc(x[7]) + 2 * __popc(s4) + 4 * __popc(c4);
    }
};

// The second form at b = 256, used for some rows so that part of the work
// moves from the ALU to POPC: three carry-save adders and 5 POPC (one POPC
// more and two LOP3 fewer than PopcHS<4>).
struct PopcAlt4 {
    __device__ __forceinline__ static int h(const uint32_t *x) {
        const uint32_t s1 = x[0] ^ x[1] ^ x[2];
        const uint32_t c1 = (x[0] & x[1]) | (x[2] & (x[0] ^ x[1]));
        const uint32_t s2 = x[3] ^ x[4] ^ x[5];
        const uint32_t c2 = (x[3] & x[4]) | (x[5] & (x[3] ^ x[4]));
        const uint32_t s3 = s1 ^ s2 ^ x[6];
        const uint32_t c3 = (s1 & s2) | (x[6] & (s1 ^ s2));
        return __popc(s3) + __popc(x[7]) + 2 * (__popc(c1) + __popc(c2) + __popc(c3));
    }
};

// Shared-memory layout of one warp's column buffers.
template <int W, int CS>
struct ColStage {
    static constexpr int kCols = CS + 4;  // room for the 16-byte alignment of a chunk start
    static constexpr int kBufBytes = kCols * (8 * W + 4);
    static constexpr int kStage = 64;     // survivor masks staged per round (see flush_masks)
    static constexpr int kStageOff = 16 + 2 * kBufBytes;
    // two mbarriers, two column buffers, then the survivor-mask staging area
    static constexpr int kWarpBytes = kStageOff + kStage * 8;
};

// Per-warp pipeline state, kept across work items.  A warp's shared-memory
// region holds its two mbarriers first (their place does not depend on the
// bitmap width) and then its two column buffers.
struct StageState {
    uint2 *stage;         // kStage (row offset, mask) entries: survivor masks of one group
    unsigned char *buf;   // two buffers of kBufBytes (of the width in use)
    uint64_t *bar;        // two mbarriers
    uint32_t phase;       // bit k: parity to wait for on buffer k
    bool ok;              // false once a wait gave up
    int pending;          // after a failed wait: 1 + slot of a copy still in flight, or 0
    int wait_limit;       // polls before a wait gives up
    int skip_copy;        // fault injection: issue no copy for the next fill (then 0)
    uint32_t n_full;      // filter_item_tma with kFold: column steps of the last item that
                          // took the full-width test
};

// After a failed wait: waits (bounded) for the copy still in flight, so that
// no copy targets the warp's shared memory after it stops.
__device__ __forceinline__ void drain_stage(StageState &st) {
    if (st.pending) {
        const int slot = st.pending - 1;
        mbar_wait(&st.bar[slot], (st.phase >> slot) & 1u, st.wait_limit);
        st.pending = 0;
    }
}

__device__ __forceinline__ void init_stage(StageState &st, unsigned char *region, int stage_off) {
    st.stage = reinterpret_cast<uint2 *>(region + stage_off);
    st.bar = reinterpret_cast<uint64_t *>(region);
    st.buf = region + 16;
    st.phase = 0;
    st.ok = true;
    st.pending = 0;
    st.wait_limit = 1 << 22;
    st.skip_copy = 0;
    st.n_full = 0;
    if ((threadIdx.x & 31) == 0) {
        mbar_init(&st.bar[0], 1);
        mbar_init(&st.bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_shared();
    }
    __syncwarp();
}

template <int W, int CS>
__device__ __forceinline__ void stage_issue(StageState &st, int slot,
                                            const uint64_t *__restrict__ bm,
                                            const uint32_t *__restrict__ ssz, int64_t c_al,
                                            int ncols) {
    using L = ColStage<W, CS>;
    unsigned char *b = st.buf + slot * L::kBufBytes;
    const uint32_t bm_bytes = (uint32_t)ncols * 8u * W;
    const uint32_t sz_bytes = (uint32_t)ncols * 4u;
    fence_async_shared();
    mbar_expect_tx(&st.bar[slot], bm_bytes + sz_bytes);
    if (st.skip_copy) {  // fault injection: the bytes the barrier expects never arrive
        st.skip_copy = 0;
        return;
    }
    tma_load_1d(b, bm + c_al * W, bm_bytes, &st.bar[slot]);
    tma_load_1d(b + L::kCols * 8 * W, ssz + c_al, sz_bytes, &st.bar[slot]);
}

// Writes the survivors of one 32-column group to the queue.  A lane's masks are
// sparse (at threshold 1/2 about one survivor per lane and group), so looping
// over each lane's own bits leaves most lanes idle for most iterations.
// Instead the warp stages its nonzero masks (row offset, mask) in shared memory,
// kStage per round, and each lane expands two of them: the loop runs for the
// largest number of bits in two masks, not the largest over eight.  Bit b of a
// mask is column col_hi - b.  One atomicAdd per round reserves the queue slots.
template <int R, int kStage>
__device__ __forceinline__ void flush_masks(const uint32_t (&mask)[R], const int32_t (&rd)[R], int nz,
                                            int n_masks, int64_t i0, int64_t col_hi,
                                            const SurvivorSink &sink, uint2 *stage) {
    static_assert(kStage == 64, "two staged masks per lane");
    constexpr unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int first = warp_excl_scan_i(nz);  // index of this lane's first nonzero mask
    for (int base = 0; base < n_masks; base += kStage) {  // warp-uniform; one round usually
        int e = first;
#pragma unroll
        for (int k = 0; k < R; k++) {
            if (mask[k]) {
                if (e >= base && e < base + kStage)
                    stage[e - base] = make_uint2((uint32_t)rd[k], mask[k]);
                e++;
            }
        }
        __syncwarp();
        const int n_e = min(kStage, n_masks - base);
        const uint2 ea = lane < n_e ? stage[lane] : make_uint2(0u, 0u);
        const uint2 eb = lane + 32 < n_e ? stage[lane + 32] : make_uint2(0u, 0u);
        __syncwarp();  // the staging area may be rewritten in the next round
        const int c = __popc(ea.y) + __popc(eb.y);
        const int total = __reduce_add_sync(kFull, c);
        const int excl = warp_excl_scan_i(c);
        unsigned long long pos0 = 0;
        if (lane == 0) {
            pos0 = atomicAdd(sink.count, (unsigned long long)total);
            if (sink.job_count) atomicAdd(sink.job_count, (unsigned long long)total);
        }
        pos0 = __shfl_sync(kFull, pos0, 0);
        unsigned long long pos = pos0 + excl;
        uint32_t m = ea.y;
        uint32_t row = (uint32_t)(i0 + ea.x);
        while (m) {
            const int bpos = __ffs(m) - 1;
            m &= m - 1;
            if (pos < (unsigned long long)sink.cap)
                sink.queue[pos] = make_uint2(row, (uint32_t)(col_hi - bpos));
            pos++;
        }
        m = eb.y;
        row = (uint32_t)(i0 + eb.x);
        while (m) {
            const int bpos = __ffs(m) - 1;
            m &= m - 1;
            if (pos < (unsigned long long)sink.cap)
                sink.queue[pos] = make_uint2(row, (uint32_t)(col_hi - bpos));
            pos++;
        }
    }
}

// Filter over one work item with TMA-staged columns.  The bitmap and size
// arrays must be readable up to 3 entries past the last column (padded).
// kFold (b = 128 and 256): every pair first meets Eq. 2 with the two halves of
// the xor folded onto each other (64 or 128 bits); popc(x0 ^ x1) <= popc(x0) +
// popc(x1), so a pair that fails this test fails the full-width one too, and a
// warp runs the full-width test on a column only when one of its 32 x R pairs
// passes the folded one (the survivors are the same).
template <int W, int R, int CS, int kAltRows = 0, bool kCos = false, bool kCut = false,
          bool kFold = false>
__device__ __forceinline__ void filter_item_tma(const uint64_t *__restrict__ bm,
                                                const uint32_t *__restrict__ ssz,
                                                const int32_t *__restrict__ lim_tab,
                                                int64_t row_end, int64_t i0, int64_t c0, int64_t c1,
                                                const SimArgs &sa, const SurvivorSink &sink,
                                                StageState &st) {
    using L = ColStage<W, CS>;
    constexpr unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    st.n_full = 0;
    if (c1 <= c0) return;
    // rows in registers, as 32-bit words
    uint32_t rb[R][2 * W];
    uint32_t rs[R];
    int32_t rd[R];  // row index - i0 (for the diagonal mask)
#pragma unroll
    for (int k = 0; k < R; k++) {
        const int64_t i = i0 + k * 32 + lane;
        rd[k] = k * 32 + lane;
        if (i < row_end) {
            rs[k] = ssz[i];
#pragma unroll
            for (int w = 0; w < W; w++) {
                const uint64_t v = bm[i * W + w];
                rb[k][2 * w] = (uint32_t)v;
                rb[k][2 * w + 1] = (uint32_t)(v >> 32);
            }
        } else {
            rs[k] = 0;
#pragma unroll
            for (int w = 0; w < 2 * W; w++) rb[k][w] = 0;
        }
    }
    static_assert(!kFold || W == 2 || W == 4, "the folded test is for b = 128 and 256");
    uint32_t n_full = 0;  // kFold: column steps that took the full-width test (left in st.n_full)
    int nlim[R];
#pragma unroll
    for (int k = 0; k < R; k++) nlim[k] = 0;
    uint32_t prev_cs = 0xffffffffu;

    const int64_t n_chunks = (c1 - c0 + CS - 1) / CS;
    // prefetch chunk 0 into slot 0
    if (lane == 0) {
        const int64_t cs_ = c0, ce_ = min(c0 + (int64_t)CS, c1);
        const int64_t c_al = cs_ & ~(int64_t)3;
        stage_issue<W, CS>(st, 0, bm, ssz, c_al, (int)(((ce_ - c_al) + 3) & ~(int64_t)3));
    }
    for (int64_t ch = 0; ch < n_chunks; ch++) {
        const int slot = (int)(ch & 1);
        if (ch + 1 < n_chunks && lane == 0) {
            const int64_t cs_ = c0 + (ch + 1) * CS, ce_ = min(cs_ + (int64_t)CS, c1);
            const int64_t c_al = cs_ & ~(int64_t)3;
            stage_issue<W, CS>(st, slot ^ 1, bm, ssz, c_al, (int)(((ce_ - c_al) + 3) & ~(int64_t)3));
        }
        const bool got = mbar_wait(&st.bar[slot], (st.phase >> slot) & 1u, st.wait_limit);
        st.phase ^= 1u << slot;
        if (!__all_sync(kFull, got)) {
            // give up; the copy into the other buffer (if any) is drained by the caller
            st.ok = false;
            st.pending = (ch + 1 < n_chunks) ? (slot ^ 1) + 1 : 0;
            return;
        }
        const int64_t cs = c0 + ch * CS, ce = min(cs + (int64_t)CS, c1);
        const int64_t c_al = cs & ~(int64_t)3;
        const unsigned char *b = st.buf + slot * L::kBufBytes;
        const uint32_t *colw = reinterpret_cast<const uint32_t *>(b);
        const uint32_t *cols = reinterpret_cast<const uint32_t *>(b + L::kCols * 8 * W);
        for (int64_t g = cs; g < ce; g += 32) {
            const int gj = (int)min((int64_t)32, ce - g);
            const int base = (int)(g - c_al);
            uint32_t mask[R];
#pragma unroll
            for (int k = 0; k < R; k++) mask[k] = 0;
            for (int cc = 0; cc < gj; cc++) {
                const int col = base + cc;
                const uint32_t s = cols[col];
                if (s != prev_cs) {  // warp-uniform
                    prev_cs = s;
#pragma unroll
                    for (int k = 0; k < R; k++) {
                        const uint32_t mn = min(rs[k], s), mx = max(rs[k], s);
                        const bool in_win = rs[k] != 0 && in_window(mn, mx, sa.win);
                        if (kCut && in_win && mx > sa.cut) nlim[k] = -(1 << 30);  // skips Eq. 2
                        else nlim[k] = in_win ? -(pair_lim<kCos>(lim_tab, rs[k], s, sa) + 1) : 0;
                    }
                }
                uint32_t cw[2 * W];
#pragma unroll
                for (int w = 0; w < 2 * W; w++) cw[w] = colw[col * 2 * W + w];
                if constexpr (kFold) {
                    // the column's fold (its 32-bit word w xored with word w + W);
                    // each row's fold is taken inside the same three-input xor
                    uint32_t f[W];
#pragma unroll
                    for (int w = 0; w < W; w++) f[w] = cw[w] ^ cw[w + W];
                    int any = 0;  // sign bit: some row passes the folded test
#pragma unroll
                    for (int k = 0; k < R; k++) {
                        uint32_t y[W];
#pragma unroll
                        for (int w = 0; w < W; w++) y[w] = rb[k][w] ^ rb[k][w + W] ^ f[w];
                        any |= PopcHS<W / 2>::h(y) + nlim[k];
                    }
                    if (__builtin_expect(__any_sync(kFull, any < 0), 0)) {
                        n_full++;
                        const int sh = gj - 1 - cc;  // bit of this column in the masks
#pragma unroll
                        for (int k = 0; k < R; k++) {
                            uint32_t x[2 * W];
#pragma unroll
                            for (int w = 0; w < 2 * W; w++) x[w] = rb[k][w] ^ cw[w];
                            const bool alt = W == 4 && kAltRows > 0 && k >= R - kAltRows;
                            int h;
                            if constexpr (W == 4) h = alt ? PopcAlt4::h(x) : PopcHS<4>::h(x);
                            else h = PopcHS<W>::h(x);
                            const int t = h + nlim[k];
                            mask[k] |= ((uint32_t)t >> 31) << sh;
                        }
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < R; k++) {
                        uint32_t x[2 * W];
#pragma unroll
                        for (int w = 0; w < 2 * W; w++) x[w] = rb[k][w] ^ cw[w];
                        // rows R - kAltRows .. R - 1 take the width's second form
                        const bool alt = kAltRows > 0 && k >= R - kAltRows;
                        int h;
                        if constexpr (W == 1) h = alt ? popc64_alu(x[0], x[1]) : PopcHS<1>::h(x);
                        else if constexpr (W == 4) h = alt ? PopcAlt4::h(x) : PopcHS<4>::h(x);
                        else h = PopcHS<W>::h(x);
                        const int t = h + nlim[k];
                        mask[k] = __funnelshift_l((uint32_t)t, mask[k], 1);
                    }
                }
            }
            // bit (gj-1-cc) of mask[k] is column g+cc; keep only columns j < i
            const int64_t dg = i0 - g;
            int nz = 0;
#pragma unroll
            for (int k = 0; k < R; k++) {
                const int64_t d = dg + rd[k];  // i - g
                if (d < gj) mask[k] = d <= 0 ? 0u : (mask[k] & (~0u << (gj - (int)d)));
                nz += mask[k] != 0u;
            }
            const int n_masks = __reduce_add_sync(kFull, nz);
            if (n_masks) flush_masks<R, L::kStage>(mask, rd, nz, n_masks, i0, g + gj - 1, sink, st.stage);
        }
        __syncwarp();  // every lane is done with this slot before it is refilled
    }
    st.n_full = n_full;
}

}  // namespace bmj
