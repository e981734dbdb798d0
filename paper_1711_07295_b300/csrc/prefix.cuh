// prefix.cuh -- the prefix filter (Section 2.2) as a candidate generator for
// the Bitmap Filter (prefix.cu).
#pragma once

#include "kernels.cuh"

namespace bmj {

// Candidates of the prefix filter (Section 2.2, prefix.cu): the pairs (i, j),
// j < i in size order inside the window, whose prefixes share a token, each
// once.  On the size-sorted collection (sizes, sorted CSR).  RS-join
// (n_cols > 0): S's sets at positions [0, n_cols) and R's after them, each run
// in size order; the pairs are (i in R, j in S) inside both window bounds.
// *n_slots is the number of (rank, pair) slots examined; BMJ_ERR_OOM when they
// exceed max_cand (> 0) or do not fit.
int prefix_candidates(const uint32_t *ssz, const int64_t *soff, const int32_t *stok, int64_t n,
                      int64_t ntok, int64_t n_cols, SimWindow win, int64_t max_cand, Arena &A,
                      cudaStream_t s, uint2 **cand, int64_t *n_cand, int64_t *n_slots);

}  // namespace bmj
