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
//   order each set by rank          sort (set, rank) keys
//   index the prefixes              sort (rank, set) entries of every prefix
//   count and expand candidates     per index entry, the earlier sets of its
//                                   rank's list inside the window; one thread
//                                   per candidate slot, kept when the entry's
//                                   rank is the pair's lowest shared one
#include <algorithm>

#include "host_util.cuh"

namespace bmj {
namespace {

constexpr unsigned kFullP = 0xffffffffu;

unsigned grid_p(int64_t n, int threads, int64_t cap = 148 * 32) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

// Token values as sort keys, and their maximum (for the number of key bits).
__global__ void k_tok_keys(const int32_t *__restrict__ tok, int64_t T, uint64_t *__restrict__ out,
                           unsigned int *__restrict__ max_tok) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned int m = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < T; k += stride) {
        out[k] = (uint64_t)(uint32_t)tok[k];
        m = max(m, (unsigned int)tok[k]);
    }
    m = __reduce_max_sync(kFullP, m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(max_tok, m);
}

// 1 where a run of equal sorted tokens starts.
__global__ void k_run_heads(const uint64_t *__restrict__ st, int64_t T, int64_t *__restrict__ flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < T; k += stride)
        flag[k] = (k == 0 || st[k] != st[k - 1]) ? 1 : 0;
}

// Distinct tokens (ascending) and the start of each run; pos is the exclusive
// scan of the head flags, recomputed here from the flags.
__global__ void k_run_write(const uint64_t *__restrict__ st, int64_t T,
                            const int64_t *__restrict__ flag, const int64_t *__restrict__ pos,
                            uint32_t *__restrict__ utok, int64_t *__restrict__ ustart) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < T; k += stride)
        if (flag[k]) {
            utok[pos[k]] = (uint32_t)st[k];
            ustart[pos[k]] = k;
        }
}

// (count << ubits) | distinct-token index: sorted, this is the rank order.
// Keys pack their fields into as few bits as the sizes need, which saves
// radix-sort passes (ubits = bits of a distinct-token index or rank, sbits =
// bits of a set position).
__global__ void k_rank_keys(const int64_t *__restrict__ ustart, int64_t nu, int ubits,
                            uint64_t *__restrict__ key) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nu; u += stride)
        key[u] = ((uint64_t)(ustart[u + 1] - ustart[u]) << ubits) | (uint64_t)u;
}

__global__ void k_rank_scatter(const uint64_t *__restrict__ skey, int64_t nu, int ubits,
                               uint32_t *__restrict__ rank_of) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const uint64_t umask = (1ull << ubits) - 1;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nu; r += stride)
        rank_of[skey[r] & umask] = (uint32_t)r;
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

// Rank of every token value, for token universes small enough to index
// directly (rank_map[token]); larger ones search the distinct tokens instead.
__global__ void k_rank_map(const uint32_t *__restrict__ utok, const uint32_t *__restrict__ rank_of,
                           int64_t nu, uint32_t *__restrict__ rank_map) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nu; u += stride)
        rank_map[utok[u]] = rank_of[u];
}

// (set << ubits) | rank for every token occurrence of the sorted CSR; one
// thread per set (its keys are contiguous at soff[i]).
__global__ void k_set_keys(const uint32_t *__restrict__ ssz, const int64_t *__restrict__ soff,
                           const int32_t *__restrict__ stok, int64_t n,
                           const uint32_t *__restrict__ utok, int64_t nu,
                           const uint32_t *__restrict__ rank_of,
                           const uint32_t *__restrict__ rank_map, int ubits,
                           uint64_t *__restrict__ keys) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t o = soff[i];
        for (uint32_t k = 0; k < ssz[i]; k++) {
            const uint32_t t = (uint32_t)stok[o + k];
            const uint32_t r = rank_map ? rank_map[t] : rank_of[lb_u32(utok, nu, t)];
            keys[o + k] = ((uint64_t)i << ubits) | r;
        }
    }
}

__device__ __forceinline__ int64_t prefix_len(uint32_t x, SimWindow win) {
    const uint64_t low = window_low(x, win);
    return low > x ? 0 : (int64_t)(x - low + 1);
}

__global__ void k_prefix_len(const uint32_t *__restrict__ ssz, int64_t n, SimWindow win,
                             int64_t *__restrict__ plen) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        plen[i] = prefix_len(ssz[i], win);
}

// (rank << sbits) | set for the prefix tokens of every set.
__global__ void k_prefix_emit(const uint32_t *__restrict__ ssz, const int64_t *__restrict__ soff,
                              const uint64_t *__restrict__ srank, int64_t n, SimWindow win,
                              const int64_t *__restrict__ pofs, int ubits, int sbits,
                              uint64_t *__restrict__ idx) {
    const uint64_t umask = (1ull << ubits) - 1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t len = prefix_len(ssz[i], win);
        for (int64_t k = 0; k < len; k++)
            idx[pofs[i] + k] = ((srank[soff[i] + k] & umask) << sbits) | (uint64_t)i;
    }
}

// Per index entry k = (rank r, set i): the entries of r's list before k (earlier
// sets in size order) whose size is inside i's window form [lo, k).
__global__ void k_cand_count(const uint64_t *__restrict__ idx, int64_t P,
                             const uint32_t *__restrict__ ssz, SimWindow win, int sbits,
                             int64_t *__restrict__ lo_out, int64_t *__restrict__ cnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const uint64_t smask = (1ull << sbits) - 1;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < P; k += stride) {
        const uint64_t key = idx[k];
        const uint64_t head = key & ~smask;
        int64_t a = 0, b = k;  // first entry of the rank's list
        while (a < b) {
            const int64_t m = (a + b) >> 1;
            if (idx[m] < head) a = m + 1;
            else b = m;
        }
        const uint64_t low = window_low(ssz[key & smask], win);
        b = k;  // first entry of the list with a size inside the window
        while (a < b) {
            const int64_t m = (a + b) >> 1;
            if (ssz[idx[m] & smask] < low) a = m + 1;
            else b = m;
        }
        lo_out[k] = a;
        cnt[k] = k - a;
    }
}

// One candidate slot per thread: slot o belongs to entry k (cand_off[k] <= o <
// cand_off[k+1]); the pair (i, j) is kept when no rank below the entry's is in
// both prefixes (sorted ranks of a prefix: srank[soff[x] ..]).  Kept pairs are
// appended with one atomicAdd per warp.
__global__ void k_cand_expand(const uint64_t *__restrict__ idx, int64_t P,
                              const int64_t *__restrict__ cand_off, const int64_t *__restrict__ lo,
                              int64_t C, const uint32_t *__restrict__ ssz,
                              const int64_t *__restrict__ soff, const uint64_t *__restrict__ srank,
                              SimWindow win, int ubits, int sbits, uint2 *__restrict__ out,
                              unsigned long long *__restrict__ count) {
    const int lane = threadIdx.x & 31;
    const uint64_t umask = (1ull << ubits) - 1, smask = (1ull << sbits) - 1;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (int64_t base = gw * 32; base < C; base += warps * 32) {
        const int64_t o = base + lane;
        bool keep = false;
        uint32_t i = 0, j = 0;
        if (o < C) {
            int64_t a = 0, b = P;  // last k with cand_off[k] <= o
            while (b - a > 1) {
                const int64_t m = (a + b) >> 1;
                if (cand_off[m] <= o) a = m;
                else b = m;
            }
            const int64_t k = a;
            const uint64_t key = idx[k];
            const uint32_t r = (uint32_t)(key >> sbits);
            i = (uint32_t)(key & smask);
            j = (uint32_t)(idx[lo[k] + (o - cand_off[k])] & smask);
            const uint64_t *pi = srank + soff[i];
            const uint64_t *pj = srank + soff[j];
            const int64_t ni = prefix_len(ssz[i], win), nj = prefix_len(ssz[j], win);
            int64_t x = 0, y = 0;
            keep = true;
            while (x < ni && y < nj) {
                const uint32_t rx = (uint32_t)(pi[x] & umask), ry = (uint32_t)(pj[y] & umask);
                if (rx >= r || ry >= r) break;
                if (rx == ry) {
                    keep = false;
                    break;
                }
                if (rx < ry) x++;
                else y++;
            }
        }
        const unsigned ball = __ballot_sync(kFullP, keep);
        if (ball) {
            unsigned long long pos = 0;
            if (lane == 0) pos = atomicAdd(count, (unsigned long long)__popc(ball));
            pos = __shfl_sync(kFullP, pos, 0);
            if (keep) out[pos + __popc(ball & ((1u << lane) - 1u))] = make_uint2(i, j);
        }
    }
}

}  // namespace

int prefix_candidates(const uint32_t *ssz, const int64_t *soff, const int32_t *stok, int64_t n,
                      int64_t ntok, SimWindow win, int64_t max_cand, Arena &A, cudaStream_t s,
                      uint2 **cand, int64_t *n_cand, int64_t *n_slots) {
    *cand = nullptr;
    *n_cand = 0;
    *n_slots = 0;
    if (n < 2 || ntok <= 0) return BMJ_OK;
    if (ntok >= ((int64_t)1 << 32)) return BMJ_ERR_TOO_LARGE;  // counts and ranks are 32-bit
    const int nbits_set = std::max(1, bit_length((uint64_t)(n - 1)));
    // ---- rank the distinct tokens ----
    uint64_t *tk = nullptr, *st = nullptr;
    int64_t *flag = nullptr, *pos = nullptr, *ustart = nullptr, *tot = nullptr;
    unsigned int *max_tok = nullptr;
    int rc = A.alloc(&tk, (size_t)ntok);
    if (!rc) rc = A.alloc(&st, (size_t)ntok);
    if (!rc) rc = A.alloc(&flag, (size_t)ntok);
    if (!rc) rc = A.alloc(&pos, (size_t)ntok);
    if (!rc) rc = A.alloc(&tot, 2);
    if (!rc) rc = A.alloc(&max_tok, 1);
    if (rc) return rc;
    BMJ_CHECK(cudaMemsetAsync(max_tok, 0, sizeof(unsigned int), s));
    BMJ_LAUNCH(k_tok_keys, grid_p(ntok, 256), 256, 0, s, stok, ntok, tk, max_tok);
    unsigned int hmax = 0;
    BMJ_CHECK(cudaMemcpyAsync(&hmax, max_tok, sizeof(hmax), cudaMemcpyDeviceToHost, s));
    BMJ_CHECK(cudaStreamSynchronize(s));
    rc = radix_sort_u64(tk, st, ntok, std::max(1, bit_length((uint64_t)hmax)), A, s);
    if (rc) return rc;
    BMJ_LAUNCH(k_run_heads, grid_p(ntok, 256), 256, 0, s, st, ntok, flag);
    rc = exclusive_scan_i64(flag, pos, ntok, tot, A, s);
    if (rc) return rc;
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
    BMJ_LAUNCH(k_run_write, grid_p(ntok, 256), 256, 0, s, st, ntok, flag, pos, utok, ustart);
    BMJ_CHECK(cudaMemcpyAsync(ustart + nu, &ntok, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    const int ubits = std::max(1, bit_length((uint64_t)(nu - 1)));
    const int cbits = std::max(1, bit_length((uint64_t)ntok));
    BMJ_LAUNCH(k_rank_keys, grid_p(nu, 256), 256, 0, s, ustart, nu, ubits, rkey);
    rc = radix_sort_u64(rkey, rkey_s, nu, cbits + ubits, A, s);
    if (rc) return rc;
    BMJ_LAUNCH(k_rank_scatter, grid_p(nu, 256), 256, 0, s, rkey_s, nu, ubits, rank_of);
    A.free_one(flag);
    A.free_one(pos);
    A.free_one(rkey);
    A.free_one(rkey_s);
    // ---- order every set by rank ----
    uint32_t *rank_map = nullptr;
    if (hmax < (1u << 26)) {  // a direct map of at most 256 MB
        rc = A.alloc(&rank_map, (size_t)hmax + 1);
        if (rc) return rc;
        BMJ_LAUNCH(k_rank_map, grid_p(nu, 256), 256, 0, s, utok, rank_of, nu, rank_map);
    }
    BMJ_LAUNCH(k_set_keys, grid_p(n, 256), 256, 0, s, ssz, soff, stok, n, utok, nu, rank_of,
               rank_map, ubits, tk);
    rc = radix_sort_u64(tk, st, ntok, ubits + nbits_set, A, s);  // st: (set, rank) in order
    if (rc) return rc;
    A.free_one(tk);
    // ---- index the prefixes by rank ----
    int64_t *plen = nullptr;
    rc = A.alloc(&plen, (size_t)n);
    if (rc) return rc;
    BMJ_LAUNCH(k_prefix_len, grid_p(n, 256), 256, 0, s, ssz, n, win, plen);
    rc = exclusive_scan_i64(plen, plen, n, tot, A, s);  // plen becomes the prefix offsets
    if (rc) return rc;
    int64_t P = 0;
    BMJ_CHECK(cudaMemcpyAsync(&P, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    BMJ_CHECK(cudaStreamSynchronize(s));
    if (P == 0) return BMJ_OK;
    uint64_t *ix = nullptr, *idx = nullptr;
    rc = A.alloc(&ix, (size_t)P);
    if (!rc) rc = A.alloc(&idx, (size_t)P);
    if (rc) return rc;
    BMJ_LAUNCH(k_prefix_emit, grid_p(n, 256), 256, 0, s, ssz, soff, st, n, win, plen, ubits,
               nbits_set, ix);
    rc = radix_sort_u64(ix, idx, P, ubits + nbits_set, A, s);
    if (rc) return rc;
    A.free_one(ix);
    // ---- count, then expand the candidates ----
    int64_t *lo = nullptr, *coff = nullptr;
    rc = A.alloc(&lo, (size_t)P);
    if (!rc) rc = A.alloc(&coff, (size_t)P + 1);
    if (rc) return rc;
    BMJ_LAUNCH(k_cand_count, grid_p(P, 256), 256, 0, s, idx, P, ssz, win, nbits_set, lo, coff);
    rc = exclusive_scan_i64(coff, coff, P, coff + P, A, s);
    if (rc) return rc;
    int64_t C = 0;
    BMJ_CHECK(cudaMemcpyAsync(&C, coff + P, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    BMJ_CHECK(cudaStreamSynchronize(s));
    *n_slots = C;
    if (C == 0) return BMJ_OK;
    if (max_cand > 0 && C > max_cand) return BMJ_ERR_OOM;  // more slots than the caller allows
    uint2 *out = nullptr;
    unsigned long long *cnt = nullptr;
    rc = A.alloc(&out, (size_t)C);
    if (!rc) rc = A.alloc(&cnt, 1);
    if (rc) return rc;
    BMJ_CHECK(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
    BMJ_LAUNCH(k_cand_expand, grid_p(C, 256, 148 * 16), 256, 0, s, idx, P, coff, lo, C, ssz, soff,
               st, win, ubits, nbits_set, out, cnt);
    unsigned long long nc = 0;
    BMJ_CHECK(cudaMemcpyAsync(&nc, cnt, sizeof(nc), cudaMemcpyDeviceToHost, s));
    BMJ_CHECK(cudaStreamSynchronize(s));
    *cand = out;
    *n_cand = (int64_t)nc;
    return BMJ_OK;
}

}  // namespace bmj
