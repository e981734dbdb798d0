// prefix.cu -- the prefix filter (Section 2.2) as a candidate generator for
// the Bitmap Filter: instead of every pair inside the length window, only the
// window pairs whose prefixes share a token go on to the Eq. 2 test and the
// merge.
//
// Tokens are ranked by (frequency, id), rarest first.  The prefix of a set of
// size x holds its x - low(x) + 1 lowest-ranked tokens, low(x) being the
// smallest partner size inside the window (Table 2), which is also the smallest
// overlap a similar partner can have: two similar sets therefore share a prefix
// token.  A pair sharing several prefix tokens is emitted once, at the lowest
// shared rank.
//
// Steps (all on the device, in size order):
//   rank the distinct tokens        sort the token occurrences, run lengths,
//                                   sort (count, token index)
//   every set's prefix by rank      one thread per set selects it (sets of up
//                                   to 32 tokens); one warp per set ranks its
//                                   tokens by counting in shared memory (up to
//                                   2048); a sort of (set, rank) keys beyond
//   index the prefixes              sort (rank, set) entries of every prefix
//   count and expand candidates     per index entry, the earlier sets of its
//                                   rank's list inside the window (its slots);
//                                   a slot is kept when the entry's rank is the
//                                   pair's lowest shared one.  The slots are
//                                   expanded in ranges (prefix_expand), so that
//                                   any number of them goes through a buffer of
//                                   fixed size, a range at a time
#include <algorithm>

#include "host_util.cuh"
#include "prefix.cuh"

namespace bmj {
namespace {

constexpr unsigned kFullP = 0xffffffffu;

unsigned grid_p(int64_t n, int threads, int64_t cap = 148 * 32) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

// Sets of up to kThreadSetMax tokens have their prefix selected by one thread,
// sets of up to kWarpSetMax tokens by one warp in shared memory; larger ones
// by a sort.
constexpr int kThreadSetMax = 32;
constexpr int kWarpSetMax = 2048;
constexpr int kPrefWarps = 4;

// Token values as sort keys, and their maximum (for the number of key bits).
__global__ void k_tok_keys(const int32_t *__restrict__ tok, int64_t T, uint32_t *__restrict__ out,
                           unsigned int *__restrict__ max_tok) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned int m = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < T; k += stride) {
        out[k] = (uint32_t)tok[k];
        m = max(m, (unsigned int)tok[k]);
    }
    m = __reduce_max_sync(kFullP, m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(max_tok, m);
}

// 1 where a run of equal sorted tokens starts.
__device__ __forceinline__ bool run_head(const uint32_t *st, int64_t k) {
    return k == 0 || st[k] != st[k - 1];
}

__global__ void k_run_heads(const uint32_t *__restrict__ st, int64_t T, uint32_t *__restrict__ flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < T; k += stride)
        flag[k] = run_head(st, k) ? 1u : 0u;
}

// The number of runs, from the exclusive scan of the head flags (one thread).
__global__ void k_run_total(const uint32_t *__restrict__ st, const uint32_t *__restrict__ pos,
                            int64_t T, int64_t *__restrict__ total) {
    total[0] = (int64_t)pos[T - 1] + (run_head(st, T - 1) ? 1 : 0);
}

// Distinct tokens (ascending) and the start of each run; pos is the exclusive
// scan of the head flags.
__global__ void k_run_write(const uint32_t *__restrict__ st, int64_t T,
                            const uint32_t *__restrict__ pos, uint32_t *__restrict__ utok,
                            int64_t *__restrict__ ustart) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < T; k += stride)
        if (run_head(st, k)) {
            utok[pos[k]] = st[k];
            ustart[pos[k]] = k;
        }
}

// (distinct-token index << cshift) | count, in index order: a stable sort by
// the count digits (the low cshift bits, a whole number of 8-bit radix digits)
// leaves equal counts in index order, which is the rank order.  Keys pack their
// fields into as few digits as the sizes need, and sorts touch only the digits
// they order by, which saves radix-sort passes.
__global__ void k_rank_keys(const int64_t *__restrict__ ustart, int64_t nu, int cshift,
                            uint64_t *__restrict__ key) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nu; u += stride)
        key[u] = ((uint64_t)u << cshift) | (uint64_t)(ustart[u + 1] - ustart[u]);
}

__global__ void k_rank_scatter(const uint64_t *__restrict__ skey, int64_t nu, int cshift,
                               uint32_t *__restrict__ rank_of) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nu; r += stride)
        rank_of[skey[r] >> cshift] = (uint32_t)r;
}

__device__ __forceinline__ int64_t lb_u32(const uint32_t *a, int64_t n, uint32_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// rank_map[token] = rank, for token values small enough to index directly.
__global__ void k_rank_map(const uint32_t *__restrict__ utok, const uint32_t *__restrict__ rank_of,
                           int64_t nu, uint32_t *__restrict__ rank_map) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nu; u += stride)
        rank_map[utok[u]] = rank_of[u];
}

// The rank of a token value: a direct map (token values below 2^26), else a
// binary search of the distinct tokens.
struct RankLookup {
    const uint32_t *map;
    const uint32_t *utok, *rank_of;
    int64_t nu;
    __device__ __forceinline__ uint32_t operator()(uint32_t t) const {
        return map ? map[t] : rank_of[lb_u32(utok, nu, t)];
    }
};

__device__ __forceinline__ int64_t prefix_len(uint32_t x, SimWindow win) {
    const uint64_t low = window_low(x, win);
    return low > x ? 0 : (int64_t)(x - low + 1);
}

// Within the size-ordered sets [i0, i1): the first set with more than
// kThreadSetMax tokens, the first with more than kWarpSetMax, the position of
// the latter's first token and the end of the range's tokens (one thread).
__global__ void k_size_bounds(const uint32_t *__restrict__ ssz, const int64_t *__restrict__ soff,
                              int64_t i0, int64_t i1, int64_t n, int64_t ntok,
                              int64_t *__restrict__ out) {
    const uint32_t lim[2] = {(uint32_t)kThreadSetMax, (uint32_t)kWarpSetMax};
    for (int k = 0; k < 2; k++) {
        int64_t lo = i0, hi = i1;
        while (lo < hi) {
            const int64_t m = (lo + hi) >> 1;
            if (ssz[m] <= lim[k]) lo = m + 1;
            else hi = m;
        }
        out[k] = lo;
    }
    out[2] = out[1] < n ? soff[out[1]] : ntok;
    out[3] = i1 < n ? soff[i1] : ntok;
}

// The prefix of every set of at most kThreadSetMax tokens, in rank order: one
// thread per set keeps its ranks in a local array and selects the smallest,
// the next smallest, and so on, prefix-length times (ranks are distinct within
// a set).
__global__ void k_prefix_small(const uint32_t *__restrict__ ssz, const int64_t *__restrict__ soff,
                               const int32_t *__restrict__ stok, int64_t i0, int64_t n1,
                               SimWindow win, const int64_t *__restrict__ pofs,
                               const RankLookup rl, uint32_t *__restrict__ pref) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = i0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n1; i += stride) {
        const int x = (int)ssz[i];
        const int L = (int)prefix_len((uint32_t)x, win);
        if (L == 0) continue;
        uint32_t r[kThreadSetMax];
        const int64_t o = soff[i];
        for (int e = 0; e < x; e++) r[e] = rl((uint32_t)stok[o + e]);
        uint32_t *dst = pref + pofs[i];
        int64_t prev = -1;
        for (int k = 0; k < L; k++) {
            uint32_t m = 0xffffffffu;
            for (int e = 0; e < x; e++)
                if ((int64_t)r[e] > prev && r[e] < m) m = r[e];
            dst[k] = m;
            prev = m;
        }
    }
}

// The prefix of every set of kThreadSetMax + 1 to kWarpSetMax tokens (sets
// [n1, n2) in size order), in rank order: one warp per set loads its tokens' ranks into shared memory; a rank's position
// in the set is the number of smaller ranks (ranks are distinct within a set),
// and the positions below the prefix length are written to pref[pofs[i] ..].
__global__ void __launch_bounds__(32 * kPrefWarps)
    k_prefix_rank(const uint32_t *__restrict__ ssz, const int64_t *__restrict__ soff,
                  const int32_t *__restrict__ stok, int64_t n1, int64_t n2, SimWindow win,
                  const int64_t *__restrict__ pofs, const RankLookup rl,
                  uint32_t *__restrict__ pref) {
    __shared__ uint32_t buf[kPrefWarps][kWarpSetMax];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t *b = buf[w];
    const int64_t warps = (int64_t)gridDim.x * kPrefWarps;
    for (int64_t i = n1 + (int64_t)blockIdx.x * kPrefWarps + w; i < n2; i += warps) {
        const int x = (int)ssz[i];
        const int L = (int)prefix_len((uint32_t)x, win);
        if (L == 0) continue;  // warp-uniform
        const int64_t o = soff[i];
        for (int e = lane; e < x; e += 32) b[e] = rl((uint32_t)stok[o + e]);
        __syncwarp();
        uint32_t *dst = pref + pofs[i];
        for (int e = lane; e < x; e += 32) {
            const uint32_t re = b[e];
            int c = 0;
            for (int f = 0; f < x && c < L; f++) c += b[f] < re;
            if (c < L) dst[c] = re;
        }
        __syncwarp();  // the buffer is reused for the next set
    }
}

// (set - i0) << ubits | rank for the tokens of the sets [i0, i1) (their tokens
// are contiguous in the sorted CSR from soff[i0] = t0); one thread per set.
__global__ void k_set_keys(const uint32_t *__restrict__ ssz, const int64_t *__restrict__ soff,
                           const int32_t *__restrict__ stok, int64_t i0, int64_t i1, int64_t t0,
                           const RankLookup rl, int ubits, uint64_t *__restrict__ keys) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = i0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < i1; i += stride) {
        const int64_t o = soff[i];
        for (uint32_t k = 0; k < ssz[i]; k++)
            keys[o - t0 + k] = ((uint64_t)(i - i0) << ubits) | rl((uint32_t)stok[o + k]);
    }
}

// The prefixes of the sets [i0, i1) from their (set, rank) keys sorted.
__global__ void k_prefix_big(const uint32_t *__restrict__ ssz, const int64_t *__restrict__ soff,
                             const uint64_t *__restrict__ sorted, int64_t i0, int64_t i1,
                             int64_t t0, SimWindow win, const int64_t *__restrict__ pofs,
                             int ubits, uint32_t *__restrict__ pref) {
    const uint64_t umask = (1ull << ubits) - 1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = i0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < i1; i += stride) {
        const int64_t len = prefix_len(ssz[i], win);
        for (int64_t k = 0; k < len; k++)
            pref[pofs[i] + k] = (uint32_t)(sorted[soff[i] - t0 + k] & umask);
    }
}

__global__ void k_prefix_len(const uint32_t *__restrict__ ssz, int64_t n, SimWindow win,
                             int64_t *__restrict__ plen) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        plen[i] = prefix_len(ssz[i], win);
}

// (set << rshift) | rank for the prefix tokens of every set, in set order; a
// stable sort by the rank digits (the low rshift bits) then gives every rank's
// list in size order.
__global__ void k_prefix_emit(const uint32_t *__restrict__ ssz, const uint32_t *__restrict__ pref,
                              int64_t n, SimWindow win, const int64_t *__restrict__ pofs, int rshift,
                              uint64_t *__restrict__ idx) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t len = prefix_len(ssz[i], win), o = pofs[i];
        for (int64_t k = 0; k < len; k++) idx[o + k] = ((uint64_t)i << rshift) | pref[o + k];
    }
}

// Per index entry k = (rank r, set i): the entries of r's list before k (earlier
// sets in size order) whose size is inside i's window form [lo, k).  RS-join
// (n_cols > 0: S holds positions [0, n_cols), R the rest): an entry of S owns
// no candidates; an entry of R owns the entries of S in its rank's list whose
// size lies between i's window bounds (S's sets precede R's in every list).
__global__ void k_cand_count(const uint64_t *__restrict__ idx, int64_t P,
                             const uint32_t *__restrict__ ssz, SimWindow win, int rshift,
                             int64_t n_cols, int64_t *__restrict__ lo_out,
                             int64_t *__restrict__ cnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const uint64_t umask = (1ull << rshift) - 1;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < P; k += stride) {
        const uint64_t key = idx[k];
        const uint64_t r = key & umask;
        const int64_t i = (int64_t)(key >> rshift);
        if (n_cols > 0 && i < n_cols) {
            lo_out[k] = k;
            cnt[k] = 0;
            continue;
        }
        int64_t a = 0, b = k;  // first entry of the rank's list
        while (a < b) {
            const int64_t m = (a + b) >> 1;
            if ((idx[m] & umask) < r) a = m + 1;
            else b = m;
        }
        int64_t e = k;  // end of the candidate partners: k, or (RS) the first entry of R
        if (n_cols > 0) {
            int64_t c = a;
            while (c < e) {
                const int64_t m = (c + e) >> 1;
                if ((int64_t)(idx[m] >> rshift) < n_cols) c = m + 1;
                else e = m;
            }
        }
        const uint64_t low = window_low(ssz[i], win);
        b = e;  // first entry with a size inside the window
        while (a < b) {
            const int64_t m = (a + b) >> 1;
            if (ssz[idx[m] >> rshift] < low) a = m + 1;
            else b = m;
        }
        if (n_cols > 0) {  // (RS) past the last entry with a size below the upper bound
            const uint64_t high = window_high(ssz[i], win);
            if (high != ~0ull) {
                int64_t c = a, d = e;
                while (c < d) {
                    const int64_t m = (c + d) >> 1;
                    if ((uint64_t)ssz[idx[m] >> rshift] <= high) c = m + 1;
                    else d = m;
                }
                e = c;
            }
        }
        lo_out[k] = a;
        cnt[k] = e > a ? e - a : 0;
    }
}

// Candidate slots [o0, o1) in tiles of 32 * kExpandPerLane consecutive slots
// per warp.  The warp finds the entries owning its tile's first and last slots
// (binary searches of cand_off over all entries), then each slot's entry by a
// binary search between those two.  The pair (i, j) of a slot is kept when no
// rank below the entry's is in both prefixes (sorted ranks of a prefix:
// pref[pofs[x] ..]), so that a pair sharing several prefix tokens comes out
// once.  With W > 0 the pair then meets Eq. 2 with its W-word bitmaps.  The
// pairs kept in a tile are appended with one atomicAdd per warp and tile; the
// candidates are counted with one atomicAdd per warp.
constexpr int kExpandPerLane = 8;

__device__ __forceinline__ int64_t owner_of(const int64_t *__restrict__ cand_off, int64_t a,
                                            int64_t b, int64_t o) {
    // last k in [a, b) with cand_off[k] <= o (cand_off[a] <= o holds)
    while (b - a > 1) {
        const int64_t m = (a + b) >> 1;
        if (cand_off[m] <= o) a = m;
        else b = m;
    }
    return a;
}

// One candidate slot of the expansion: its entry and pair (fetch), the
// partner data (load: sizes, prefix offsets and, with W > 0, bitmaps), the
// prefix test (lowest_shared: no rank below the entry's in both prefixes) and
// Eq. 2 (passes).
// 64-bit words of a set's record for the expansion: its size, its prefix
// offset and its W bitmap words, padded to 16, 32 or 64 bytes.
__host__ __device__ constexpr int rec_words(int W) { return W == 0 ? 2 : W <= 2 ? 4 : 8; }

__global__ void k_pack_records(const uint32_t *__restrict__ ssz, const int64_t *__restrict__ pofs,
                               const uint64_t *__restrict__ bm, int W, int K, int64_t n,
                               uint64_t *__restrict__ rec) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        uint64_t *r = rec + (size_t)x * K;
        r[0] = ssz[x];
        r[1] = (uint64_t)pofs[x];
        for (int w = 0; w < W; w++) r[2 + w] = bm[(size_t)x * W + w];
        for (int w = 2 + W; w < K; w++) r[w] = 0;
    }
}

template <int W>
struct SlotLoad {
    bool valid = false;
    uint32_t i = 0, j = 0, r = 0, si = 0, sj = 0;
    int64_t poi = 0, poj = 0;
    uint64_t bwi[W > 0 ? W : 1], bwj[W > 0 ? W : 1];

    __device__ __forceinline__ void fetch(int64_t o, int64_t t1, int64_t ka, int64_t kz,
                                          const uint64_t *__restrict__ idx,
                                          const int64_t *__restrict__ cand_off,
                                          const int64_t *__restrict__ lo, uint64_t umask,
                                          int rshift) {
        valid = o < t1;
        if (!valid) return;
        const int64_t k = owner_of(cand_off, ka, kz, o);
        const uint64_t key = idx[k];
        r = (uint32_t)(key & umask);
        i = (uint32_t)(key >> rshift);
        j = (uint32_t)(idx[lo[k] + (o - cand_off[k])] >> rshift);
    }
    // the two sets' records (size, prefix offset, bitmap): one or two aligned
    // 16-byte loads per record, so a partner costs one random sector or two
    __device__ __forceinline__ void load(const uint64_t *__restrict__ rec) {
        if (!valid) return;
        constexpr int K = rec_words(W);
        uint64_t a[K], b[K];
        const ulonglong2 *ra = reinterpret_cast<const ulonglong2 *>(rec + (size_t)i * K);
        const ulonglong2 *rb = reinterpret_cast<const ulonglong2 *>(rec + (size_t)j * K);
#pragma unroll
        for (int v = 0; v < K / 2; v++) {
            const ulonglong2 x = ra[v], y = rb[v];
            a[2 * v] = x.x;
            a[2 * v + 1] = x.y;
            b[2 * v] = y.x;
            b[2 * v + 1] = y.y;
        }
        si = (uint32_t)a[0];
        sj = (uint32_t)b[0];
        poi = (int64_t)a[1];
        poj = (int64_t)b[1];
#pragma unroll
        for (int w = 0; w < W; w++) {
            bwi[w] = a[2 + w];
            bwj[w] = b[2 + w];
        }
    }
    __device__ __forceinline__ bool lowest_shared(const uint32_t *__restrict__ pref,
                                                  SimWindow win) const {
        const uint32_t *pi = pref + poi;
        const uint32_t *pj = pref + poj;
        const int64_t ni = prefix_len(si, win), nj = prefix_len(sj, win);
        int64_t x = 0, y = 0;
        while (x < ni && y < nj) {
            const uint32_t rx = pi[x], ry = pj[y];
            if (rx >= r || ry >= r) break;
            if (rx == ry) return false;
            if (rx < ry) x++;
            else y++;
        }
        return true;
    }
    __device__ __forceinline__ bool passes(const int32_t *__restrict__ lim) const {
        if (W == 0) return true;
        int h = 0;
#pragma unroll
        for (int w = 0; w < W; w++) h += __popcll(bwi[w] ^ bwj[w]);
        return h <= lim[si + sj];
    }
};

template <int W>
__global__ void k_cand_expand(const uint64_t *__restrict__ idx, int64_t P,
                              const int64_t *__restrict__ cand_off, const int64_t *__restrict__ lo,
                              int64_t o0, int64_t o1, const uint64_t *__restrict__ rec,
                              const uint32_t *__restrict__ pref, SimWindow win, int rshift,
                              const int32_t *__restrict__ lim, uint2 *__restrict__ out,
                              unsigned long long *__restrict__ count,
                              unsigned long long *__restrict__ n_cand) {
    constexpr int64_t kTile = 32 * kExpandPerLane;
    const int lane = threadIdx.x & 31;
    const uint64_t umask = (1ull << rshift) - 1;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    unsigned n_keep = 0;  // this lane's candidates (fewer than 2^32 per lane)
    for (int64_t t0 = o0 + gw * kTile; t0 < o1; t0 += warps * kTile) {
        const int64_t t1 = min(t0 + kTile, o1);
        // lane 0: the first slot's entry, lane 1: the last slot's
        int64_t kb = 0;
        if (lane < 2) kb = owner_of(cand_off, 0, P, lane == 0 ? t0 : t1 - 1);
        const int64_t ka = __shfl_sync(kFullP, kb, 0);
        const int64_t kz = __shfl_sync(kFullP, kb, 1) + 1;
        // every round's kept pairs stay in registers; the tile reserves its
        // output slots with one atomicAdd (same-address atomics per round were
        // the bottleneck with billions of candidates)
        uint32_t ii[kExpandPerLane], jj[kExpandPerLane];
        uint32_t pmask = 0;
        // two slots per lane in flight: every load of both is issued before
        // either prefix merge, so that their latencies overlap
#pragma unroll
        for (int m = 0; m < kExpandPerLane; m += 2) {
            SlotLoad<W> a, b;
            a.fetch(t0 + m * 32 + lane, t1, ka, kz, idx, cand_off, lo, umask, rshift);
            b.fetch(t0 + (m + 1) * 32 + lane, t1, ka, kz, idx, cand_off, lo, umask, rshift);
            a.load(rec);
            b.load(rec);
            const bool ka_ = a.valid && a.lowest_shared(pref, win);
            const bool kb_ = b.valid && b.lowest_shared(pref, win);
            // the Bitmap Filter (Eq. 2) on the candidate, inside the window by construction
            const bool pa = ka_ && a.passes(lim);
            const bool pb = kb_ && b.passes(lim);
            n_keep += (ka_ ? 1u : 0u) + (kb_ ? 1u : 0u);
            ii[m] = a.i;
            jj[m] = a.j;
            ii[m + 1] = b.i;
            jj[m + 1] = b.j;
            pmask |= (pa ? (1u << m) : 0u) | (pb ? (2u << m) : 0u);
        }
        const int c = __popc(pmask);
        const int total = __reduce_add_sync(kFullP, c);
        if (total) {
            int excl = c;  // exclusive scan of c over the lanes
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int u = __shfl_up_sync(kFullP, excl, d);
                if (lane >= d) excl += u;
            }
            excl -= c;
            unsigned long long pos = 0;
            if (lane == 0) pos = atomicAdd(count, (unsigned long long)total);
            pos = __shfl_sync(kFullP, pos, 0) + excl;
#pragma unroll
            for (int m = 0; m < kExpandPerLane; m++)
                if (pmask & (1u << m)) out[pos++] = make_uint2(ii[m], jj[m]);
        }
    }
    // candidates: one atomicAdd per warp for its whole share
    const unsigned tot_keep = __reduce_add_sync(kFullP, n_keep);
    if (lane == 0 && tot_keep) atomicAdd(n_cand, (unsigned long long)tot_keep);
}

}  // namespace

int prefix_index(const uint32_t *ssz, const int64_t *soff, const int32_t *stok, int64_t n,
                 int64_t ntok, int64_t n_cols, SimWindow win, Arena &A, cudaStream_t s,
                 PrefixIndex *out) {
    *out = PrefixIndex{};
    out->ssz = ssz;
    out->win = win;
    if (n < 2 || ntok <= 0) return BMJ_OK;
    if (ntok >= ((int64_t)1 << 32)) return BMJ_ERR_TOO_LARGE;  // counts and ranks are 32-bit
    // ---- rank the distinct tokens: (occurrences, token value), rarest first ----
    // Sort the occurrences; run lengths give each distinct token's count; sort
    // the (count, token index) pairs.
    unsigned int *max_tok = nullptr;
    int64_t *tot = nullptr;
    uint32_t *tk = nullptr, *st = nullptr;
    uint32_t *pos = nullptr;
    int64_t *ustart = nullptr;
    int rc = A.alloc(&max_tok, 1);
    if (!rc) rc = A.alloc(&tot, 2);
    if (!rc) rc = A.alloc(&tk, (size_t)ntok);
    if (!rc) rc = A.alloc(&st, (size_t)ntok);
    if (!rc) rc = A.alloc(&pos, (size_t)ntok);
    if (rc) return rc;
    BMJ_CHECK(cudaMemsetAsync(max_tok, 0, sizeof(unsigned int), s));
    BMJ_LAUNCH(k_tok_keys, grid_p(ntok, 256), 256, 0, s, stok, ntok, tk, max_tok);
    unsigned int hmax = 0;
    BMJ_CHECK(cudaMemcpyAsync(&hmax, max_tok, sizeof(hmax), cudaMemcpyDeviceToHost, s));
    BMJ_CHECK(cudaStreamSynchronize(s));
    rc = radix_sort_u32(tk, st, ntok, std::max(1, bit_length((uint64_t)hmax)), A, s);
    if (rc) return rc;
    BMJ_LAUNCH(k_run_heads, grid_p(ntok, 256), 256, 0, s, st, ntok, pos);
    rc = exclusive_scan_u32(pos, pos, ntok, A, s);  // (ntok < 2^32)
    if (rc) return rc;
    BMJ_LAUNCH(k_run_total, 1, 1, 0, s, st, pos, ntok, tot);
    int64_t nu = 0;
    BMJ_CHECK(cudaMemcpyAsync(&nu, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    BMJ_CHECK(cudaStreamSynchronize(s));
    uint32_t *utok = nullptr, *rank_of = nullptr;
    uint64_t *rkey = nullptr, *rkey_s = nullptr;
    rc = A.alloc(&utok, (size_t)nu);
    if (!rc) rc = A.alloc(&ustart, (size_t)nu + 1);
    if (!rc) rc = A.alloc(&rank_of, (size_t)nu);
    if (!rc) rc = A.alloc(&rkey, (size_t)nu);
    if (!rc) rc = A.alloc(&rkey_s, (size_t)nu);
    if (rc) return rc;
    BMJ_LAUNCH(k_run_write, grid_p(ntok, 256), 256, 0, s, st, ntok, pos, utok, ustart);
    BMJ_CHECK(cudaMemcpyAsync(ustart + nu, &ntok, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    const int ubits = std::max(1, bit_length((uint64_t)(nu - 1)));
    const int cbits = std::max(1, bit_length((uint64_t)n));  // a token occurs at most once per set
    const int cshift = 8 * ((cbits + 7) / 8);  // the count in whole radix digits
    BMJ_LAUNCH(k_rank_keys, grid_p(nu, 256), 256, 0, s, ustart, nu, cshift, rkey);
    rc = radix_sort_u64(rkey, rkey_s, nu, cshift, A, s);  // by count; ties stay in token order
    if (rc) return rc;
    BMJ_LAUNCH(k_rank_scatter, grid_p(nu, 256), 256, 0, s, rkey_s, nu, cshift, rank_of);
    A.free_one(tk);
    A.free_one(st);
    A.free_one(pos);
    A.free_one(rkey);
    A.free_one(rkey_s);
    RankLookup rl{nullptr, utok, rank_of, nu};
    if (hmax < (1u << 26)) {  // a direct map of at most 256 MB
        uint32_t *rank_map = nullptr;
        rc = A.alloc(&rank_map, (size_t)hmax + 1);
        if (rc) return rc;
        BMJ_LAUNCH(k_rank_map, grid_p(nu, 256), 256, 0, s, utok, rank_of, nu, rank_map);
        rl.map = rank_map;
    }
    // ---- prefix lengths and offsets ----
    int64_t *pofs = nullptr, *bounds = nullptr;
    rc = A.alloc(&pofs, (size_t)n);
    if (!rc) rc = A.alloc(&bounds, 4);
    if (rc) return rc;
    BMJ_LAUNCH(k_prefix_len, grid_p(n, 256), 256, 0, s, ssz, n, win, pofs);
    rc = exclusive_scan_i64(pofs, pofs, n, tot, A, s);  // pofs: the prefix offsets
    if (rc) return rc;
    const int64_t run0_end = n_cols > 0 ? n_cols : n;
    BMJ_LAUNCH(k_size_bounds, 1, 1, 0, s, ssz, soff, (int64_t)0, run0_end, n, ntok, bounds);
    int64_t hv[5] = {0, 0, 0, 0, 0};  // P, then the first run's size-class bounds
    BMJ_CHECK(cudaMemcpyAsync(&hv[0], tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    BMJ_CHECK(cudaMemcpyAsync(&hv[1], bounds, 4 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    BMJ_CHECK(cudaStreamSynchronize(s));
    const int64_t P = hv[0];
    if (P == 0) return BMJ_OK;  // (no set has a prefix: no candidate)
    // ---- every set's prefix in rank order, per run of sets in size order (one
    //      run for a self-join; S's run and R's run for an RS-join) ----
    uint32_t *pref = nullptr;
    rc = A.alloc(&pref, (size_t)P);
    if (rc) return rc;
    // hb: the run's first set above one thread, above one warp, its first token,
    // the run's end token (read back with P for the first run)
    auto prefix_run = [&](int64_t i0, int64_t i1, const int64_t *known) -> int {
        if (i1 <= i0) return BMJ_OK;
        int64_t hb[4] = {0, 0, 0, 0};
        if (known) {
            for (int k = 0; k < 4; k++) hb[k] = known[k];
        } else {
            BMJ_LAUNCH(k_size_bounds, 1, 1, 0, s, ssz, soff, i0, i1, n, ntok, bounds);
            BMJ_CHECK(cudaMemcpyAsync(hb, bounds, 4 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            BMJ_CHECK(cudaStreamSynchronize(s));
        }
        const int64_t n1 = hb[0], n2 = hb[1], t0 = hb[2], t1 = hb[3];
        if (n1 > i0)
            BMJ_LAUNCH(k_prefix_small, grid_p(n1 - i0, 128, 148 * 64), 128, 0, s, ssz, soff, stok, i0,
                       n1, win, pofs, rl, pref);
        if (n2 > n1)
            BMJ_LAUNCH(k_prefix_rank, grid_p(n2 - n1, kPrefWarps, 148 * 16), 32 * kPrefWarps, 0, s,
                       ssz, soff, stok, n1, n2, win, pofs, rl, pref);
        if (n2 < i1) {  // sets of more than kWarpSetMax tokens: sort their (set, rank) keys
            const int64_t tb = t1 - t0;
            const int bbits = std::max(1, bit_length((uint64_t)(i1 - n2 - 1)));
            uint64_t *bk = nullptr, *bs = nullptr;
            int r2 = A.alloc(&bk, (size_t)tb);
            if (!r2) r2 = A.alloc(&bs, (size_t)tb);
            if (r2) return r2;
            BMJ_LAUNCH(k_set_keys, grid_p(i1 - n2, 128), 128, 0, s, ssz, soff, stok, n2, i1, t0, rl,
                       ubits, bk);
            r2 = radix_sort_u64(bk, bs, tb, ubits + bbits, A, s);
            if (r2) return r2;
            BMJ_LAUNCH(k_prefix_big, grid_p(i1 - n2, 128), 128, 0, s, ssz, soff, bs, n2, i1, t0, win,
                       pofs, ubits, pref);
            A.free_one(bk);
            A.free_one(bs);
        }
        return BMJ_OK;
    };
    rc = prefix_run(0, run0_end, &hv[1]);
    if (!rc && n_cols > 0) rc = prefix_run(n_cols, n, nullptr);
    if (rc) return rc;
    // ---- index the prefixes by (rank, set) ----
    uint64_t *ix = nullptr, *idx = nullptr;
    rc = A.alloc(&ix, (size_t)P);
    if (!rc) rc = A.alloc(&idx, (size_t)P);
    if (rc) return rc;
    const int rshift = 8 * ((ubits + 7) / 8);  // the rank in whole radix digits
    BMJ_LAUNCH(k_prefix_emit, grid_p(n, 256), 256, 0, s, ssz, pref, n, win, pofs, rshift, ix);
    rc = radix_sort_u64(ix, idx, P, rshift, A, s);  // by rank; each list stays in size order
    if (rc) return rc;
    A.free_one(ix);
    // ---- count, then expand the candidates ----
    int64_t *lo = nullptr, *coff = nullptr;
    rc = A.alloc(&lo, (size_t)P);
    if (!rc) rc = A.alloc(&coff, (size_t)P + 1);
    if (rc) return rc;
    BMJ_LAUNCH(k_cand_count, grid_p(P, 256), 256, 0, s, idx, P, ssz, win, rshift, n_cols, lo,
               coff);
    rc = exclusive_scan_i64(coff, coff, P, coff + P, A, s);
    if (rc) return rc;
    int64_t C = 0;
    BMJ_CHECK(cudaMemcpyAsync(&C, coff + P, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    BMJ_CHECK(cudaStreamSynchronize(s));
    out->n = n;
    out->idx = idx;
    out->lo = lo;
    out->cand_off = coff;
    out->pofs = pofs;
    out->pref = pref;
    out->P = P;
    out->slots = C;
    out->rshift = rshift;
    return BMJ_OK;
}

int prefix_records(const PrefixIndex &ix, PrefixTest &test, Arena &A, cudaStream_t s) {
    test.rec = nullptr;
    if (ix.P == 0) return BMJ_OK;
    const int W = test.bm ? test.W : 0;
    const int K = rec_words(W);
    const int64_t n = ix.n;
    uint64_t *rec = nullptr;
    int rc = A.alloc(&rec, (size_t)std::max<int64_t>(n, 1) * K);
    if (rc) return rc;
    BMJ_LAUNCH(k_pack_records, grid_p(n, 256), 256, 0, s, ix.ssz, ix.pofs, test.bm, W, K, n, rec);
    test.rec = rec;
    return BMJ_OK;
}

int prefix_expand(const PrefixIndex &ix, int64_t o0, int64_t o1, const PrefixTest &test,
                  uint2 *out, unsigned long long *count, unsigned long long *n_cand,
                  cudaStream_t s) {
    if (o1 <= o0 || ix.P == 0) return BMJ_OK;
    if (!test.rec) return BMJ_ERR_INVALID_ARG;  // prefix_records first
    constexpr int64_t kTile = 32 * kExpandPerLane;
    const unsigned grid = grid_p((o1 - o0 + kTile - 1) / kTile, 8, 148 * 64);
#define BMJ_EXPAND(KW)                                                                            \
    BMJ_LAUNCH(k_cand_expand<KW>, grid, 256, 0, s, ix.idx, ix.P, ix.cand_off, ix.lo, o0, o1,       \
               test.rec, ix.pref, ix.win, ix.rshift, test.lim, out, count, n_cand)
    switch (test.bm ? test.W : 0) {
        case 1: BMJ_EXPAND(1); break;
        case 2: BMJ_EXPAND(2); break;
        case 4: BMJ_EXPAND(4); break;
        default: BMJ_EXPAND(0); break;
    }
#undef BMJ_EXPAND
    return BMJ_OK;
}

}  // namespace bmj
