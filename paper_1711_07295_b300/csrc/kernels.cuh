// kernels.cuh -- device kernels of the self-join path and their launch helpers.
#pragma once

#include "bmj_internal.cuh"
#include "sim.cuh"

namespace bmj {

// Validation flags (bit set on the device, read by the host).
enum : int {
    kFlagEmpty = 1,
    kFlagNegative = 2,
    kFlagUnsorted = 4,
    kFlagTooLarge = 8,
};

constexpr int kMaxSetSize = (1 << 24) - 1;

// Checks the CSR invariants of a collection, writes each set's size (as the
// sort key) and its id (the sort value), and the maximum size.
//   info[0] |= flags, info[1] = max size (atomicMax)
int launch_validate(const int64_t *off, const int32_t *tok, int64_t n, int64_t ntok,
                    int check_tokens, uint32_t *sizes, uint32_t *ids, int *info, cudaStream_t s);

// Widens sorted uint32 sizes into int64 (input of the offsets scan).
int launch_widen(const uint32_t *in, int64_t *out, int64_t n, cudaStream_t s);

// Per set (in sorted order when perm != nullptr): gathers its tokens into the
// sorted CSR (when stok != nullptr) and writes its b-bit bitmap to
// bm[i*(b/64) ..] (Alg. 3a/3b/3c, h(t) = t mod b).
int launch_gather_build(const uint32_t *perm, const int64_t *off, const int32_t *tok,
                        const int64_t *soff, int32_t *stok, uint64_t *bm, int64_t n, int b,
                        int method, cudaStream_t s);

// Xor or Set bitmaps (method BMJ_XOR / BMJ_SET) of up to three widths at once,
// one thread per set, with the sorted-CSR gather fused as in
// launch_gather_build; bm64 / bm128 / bm256 may be null.
int launch_build_multi(const uint32_t *perm, const int64_t *off, const int32_t *tok,
                       const int64_t *soff, int32_t *stok, int64_t n, int method, uint64_t *bm64,
                       uint64_t *bm128, uint64_t *bm256, cudaStream_t s);

// need[S] = ceil(p*S/(p+q)) (the smallest overlap with Jaccard >= p/q when
// |x|+|y| = S) and lim[S] = S - 2*need[S] (the largest Hamming distance
// whose Eq. 2 bound still reaches need[S]), for S in [0, n_s).
int launch_tables(int32_t *need, int32_t *lim, int64_t n_s, int sim, uint32_t p, uint32_t q,
                  cudaStream_t s);

// Row tiles of `tile_rows` sorted rows: first window column (j0 of the tile's
// first row, rounded down to a multiple of 4) and the number of column chunks
// of `chunk_cols` columns.
int launch_tiles(const uint32_t *ssz, int64_t n, SimWindow win, int tile_rows,
                 int chunk_cols, int64_t n_tiles, int32_t *tile_c0, int64_t *tile_items,
                 cudaStream_t s, int64_t row0 = 0, int64_t row_end = -1);

// Sum over sorted rows i of (i - j0(i)): the pairs inside the length window.
int launch_window_count(const uint32_t *ssz, int64_t n, SimWindow win,
                        unsigned long long *out, cudaStream_t s, int64_t row0 = 0,
                        int64_t row_end = -1);

// RS-join: R and S share one size-sorted array, S at [0, n_cols) and R at
// [row0, row_end).  Per tile of tile_rows rows of R, the columns of S inside
// the union of its rows' windows, [tile_c0 (rounded down to a multiple of 4),
// tile_c1), and their number of chunks.
int launch_rs_tiles(const uint32_t *ssz, int64_t n_cols, SimWindow win, int tile_rows,
                    int chunk_cols, int64_t n_tiles, int32_t *tile_c0, int32_t *tile_c1,
                    int64_t *tile_items, int64_t row0, int64_t row_end, cudaStream_t s);
// Sum over rows of R of the columns of S inside the row's window.
int launch_rs_window_count(const uint32_t *ssz, int64_t n_cols, SimWindow win,
                           unsigned long long *out, int64_t row0, int64_t row_end,
                           cudaStream_t s);
// v[i] |= bit, v[i] &= mask, v[i] += add over [0, n).
int launch_or_bits(uint32_t *v, int64_t n, uint32_t bit, cudaStream_t s);
int launch_and_bits(uint32_t *v, int64_t n, uint32_t mask, cudaStream_t s);
int launch_add_i64(int64_t *v, int64_t n, int64_t add, cudaStream_t s);

struct FilterArgs {
    const uint64_t *bm;
    const uint32_t *ssz;
    const int32_t *lim;
    int64_t n;
    int64_t row0 = 0;       // rows (size-order positions) [row0, row_end) are joined
    int64_t row_end = -1;   // -1: n
    int wait_limit = 0;     // TMA filter: polls before a copy wait gives up (0: default)
    int fault_skip_copy = 0;  // fault injection: one warp skips one copy (the wait runs out)
    uint32_t p, q;
    int sim = BMJ_JACCARD;  // similarity function of the threshold p/q
    uint32_t cut = 0xffffffffu;  // cutoff point (Section 3.5); all ones: none
    const int64_t *tile_item_off;  // [n_tiles + 1], exclusive scan of items per tile
    const int32_t *tile_c0;
    const int32_t *tile_c1 = nullptr;  // RS-join: end of each tile's columns (else the diagonal)
    int64_t n_tiles;
    int64_t n_items;
    int tile_rows;
    int chunk_cols;
    uint2 *queue;
    unsigned long long *qcount;
    int64_t qcap;
    unsigned long long *item_counter;
    // [2] (may be null): with the folded test (b = 128, and 256 where built),
    // warp column steps of the folded test and those that took the full-width one
    unsigned long long *steps = nullptr;
};

// The Bitmap Filter over every window pair (persistent, warp-level work items;
// columns broadcast by shuffles).  Reads no column past the window.
int launch_filter(const FilterArgs &a, int W, int num_sms, cudaStream_t s);
int filter_tile_rows(int W);

// Rows per lane of the TMA-staged filter, per bitmap width.
#ifndef BMJ_TMA_R1
#define BMJ_TMA_R1 8
#endif
// At b = 128, with the folded test, 5 rows per lane and nine blocks per SM
// (56 registers) ran 4M sets of the 10M shape at 2.071 / 2.191e12 pairs/s
// (3/5, 9/10) against 1.962 / 2.058 with 4 rows and eight blocks, 2.039 / 2.140
// with 4 rows and nine, 2.044 / 2.176 with 6 rows and eight, 2.013 / 2.144 with
// 6 rows and nine (spilling); 8 rows spill.
#ifndef BMJ_TMA_R2
#define BMJ_TMA_R2 5
#endif
// Chunks of 128 columns at b = 128 and 64 at b = 256 (half the shared memory of
// 256 and 128: more resident warps) measured 3.4% faster each; 128 at b = 64
// and 64 at b = 128 were slower, as were 3 rows per lane at b = 128 and 2 at
// b = 256 (1M workload and 2M sets of the 10M shape).
#ifndef BMJ_TMA_CS2
#define BMJ_TMA_CS2 128
#endif
#ifndef BMJ_TMA_CS1
#define BMJ_TMA_CS1 256
#endif
#ifndef BMJ_TMA_CS4
#define BMJ_TMA_CS4 64
#endif
#ifndef BMJ_TMA_R4
#define BMJ_TMA_R4 4
#endif
constexpr int kTmaR1 = BMJ_TMA_R1, kTmaR2 = BMJ_TMA_R2, kTmaR4 = BMJ_TMA_R4;
// Columns per staged chunk (one TMA bulk copy of bitmaps, one of sizes) per width.
constexpr int kTmaCS1 = BMJ_TMA_CS1, kTmaCS2 = BMJ_TMA_CS2, kTmaCS4 = BMJ_TMA_CS4;
// At b = 64, rows per lane whose popcount runs on the ALU instead of POPC.
#ifndef BMJ_ALU_ROWS_W1
#define BMJ_ALU_ROWS_W1 1
#endif
constexpr int kAluRowsW1 = BMJ_ALU_ROWS_W1;
// At b = 256, rows per lane (of four) reduced by three carry-save adders and
// 5 POPC (PopcAlt4) instead of four and 4 POPC: two rows took the 1M-set
// filter from 0.874 to 0.882e12 pairs/s (one or three rows within 0.3% of two).
#ifndef BMJ_ALT_ROWS_W4
#define BMJ_ALT_ROWS_W4 2
#endif
// At b = 128 and 256, the folded test (64 and 128 bits) before the full-width one
// (filter_item_tma's kFold).  Off at b = 256: it took the 1M joins from 0.882 to
// 1.157e12 pairs/s, but one join per call of the 512 batched jobs from 650-742 to
// 865 ms, where the 128-bit filter passes many pairs and the folded test rarely
// spares the full one.
#ifndef BMJ_FOLD_W2
#define BMJ_FOLD_W2 1
#endif
#ifndef BMJ_FOLD_W4
#define BMJ_FOLD_W4 0
#endif
template <int W>
constexpr bool kFoldW = (W == 2 && BMJ_FOLD_W2) || (W == 4 && BMJ_FOLD_W4);
// Rows per lane that take the second popcount form of width W (popc64_alu at
// b = 64, PopcAlt4 at b = 256).
template <int W>
constexpr int kAltRows = W == 1 ? kAluRowsW1 : W == 4 ? BMJ_ALT_ROWS_W4 : 0;

// The Bitmap Filter with column chunks staged in shared memory by TMA bulk
// copies (b in {64, 128, 256}; other widths fall back to launch_filter).  The
// bitmap and size arrays must stay readable 4 entries past the last set.
// *err becomes nonzero if a bounded wait on a copy gave up.
int launch_filter_tma(const FilterArgs &a, int W, int *err, int num_sms, cudaStream_t s);
int filter_tma_tile_rows(int W);

// Exact verification of the survivors; similar pairs are written as packed
// keys (min_id << nbits) | max_id in original ids.  With bm2 (W2 words per
// set, size order) a survivor first meets the Eq. 2 bound with those wider
// bitmaps (lim[S] as in the filter); *ccount (optional) counts the survivors
// that pass it.
int launch_verify(const uint2 *queue, int64_t n_surv, const int64_t *soff, const int32_t *stok,
                  const uint32_t *ssz, const uint32_t *perm, const int32_t *need,
                  const int32_t *lim, const uint64_t *bm2, int W2, uint64_t *keys,
                  unsigned long long *rcount, unsigned long long *ccount, int nbits, int num_sms,
                  cudaStream_t s, int sim = BMJ_JACCARD, uint32_t p = 0, uint32_t q = 0);

// Splits packed keys into the (a, b) arrays of the output; b_sub is taken off
// every b (an RS-join's S ids follow R's in its packed keys).
int launch_unpack(const uint64_t *keys, int64_t n, int nbits, uint32_t *a, uint32_t *b,
                  cudaStream_t s, uint32_t b_sub = 0);

}  // namespace bmj
