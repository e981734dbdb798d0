// prefix.cuh -- the prefix filter (Section 2.2) as a candidate generator for
// the Bitmap Filter (prefix.cu).
#pragma once

#include "kernels.cuh"

namespace bmj {

// The prefix index of a size-sorted collection: every set's prefix (its
// lowest-ranked tokens, tokens ranked by (frequency, value)), the (rank, set)
// entries of all prefixes sorted by rank (each rank's list in size order), and
// per entry the run of earlier entries of its list inside the set's window.
// Candidate slot o belongs to entry k when cand_off[k] <= o < cand_off[k+1];
// its pair is (the entry's set, the (o - cand_off[k])-th set of that run).
// The buffers live in the Arena given to prefix_index.
struct PrefixIndex {
    const uint64_t *idx = nullptr;      // P entries: (set << rshift) | rank, sorted by rank
    const int64_t *lo = nullptr;        // per entry: first entry of its run of partners
    const int64_t *cand_off = nullptr;  // P + 1: exclusive scan of the run lengths
    const int64_t *pofs = nullptr;      // per set: offset of its prefix in pref
    const uint32_t *pref = nullptr;     // every prefix, ranks ascending
    const uint32_t *ssz = nullptr;      // set sizes in size order
    int64_t n = 0;                      // sets
    int64_t P = 0;                      // index entries
    int64_t slots = 0;                  // candidate slots, = cand_off[P]
    int rshift = 0;
    SimWindow win{};
};

// Builds the index on the size-sorted collection (sizes, sorted CSR).
// RS-join (n_cols > 0): S's sets at positions [0, n_cols) and R's after them,
// each run in size order; an entry of R owns the entries of S in its rank's
// list inside both window bounds, an entry of S owns none.
int prefix_index(const uint32_t *ssz, const int64_t *soff, const int32_t *stok, int64_t n,
                 int64_t ntok, int64_t n_cols, SimWindow win, Arena &A, cudaStream_t s,
                 PrefixIndex *out);

// The Bitmap Filter applied to the candidates as they are expanded: W words
// per set (1, 2 or 4) in size order, and lim[|x|+|y|] of Eq. 2 against the
// threshold (for the functions whose limit depends on the size sum alone).
// W = 0: no test, every candidate is emitted.
struct PrefixTest {
    const uint64_t *bm = nullptr;
    const int32_t *lim = nullptr;
    int W = 0;
    const uint64_t *rec = nullptr;  // per set: size, prefix offset, bitmap (prefix_records)
};

// Packs every set's size, prefix offset and (with a test) bitmap into one
// aligned record, so that the expansion reads a random partner in one or two
// sectors instead of three separate arrays; sets test.rec (memory from A).
int prefix_records(const PrefixIndex &ix, PrefixTest &test, Arena &A, cudaStream_t s);

// Candidates of the slots [o0, o1): the pairs (i, j), j < i in size order
// (RS: i in R, j in S) inside the window whose prefixes share a token, kept
// at the slot of their lowest shared rank so that every pair appears once over
// all slots.  Adds their number to *n_cand (device); appends to out (room for
// o1 - o0 pairs) those that pass the test (all of them when test.W = 0) and
// adds their number to *count (device).  test.rec must come from prefix_records.
int prefix_expand(const PrefixIndex &ix, int64_t o0, int64_t o1, const PrefixTest &test,
                  uint2 *out, unsigned long long *count, unsigned long long *n_cand,
                  cudaStream_t s);

}  // namespace bmj
