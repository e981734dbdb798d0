/*
 * bmj.h -- C ABI of the Bitmap Filter set-similarity self-join on B300 (sm_103a).
 *
 * Method: Sandes, Teodoro & Melo, "Bitmap Filter: Speeding up Exact Set
 * Similarity Joins with Bitwise Operations".  A self-join returns every pair
 * of sets whose similarity (Jaccard by default; Cosine, Dice, Overlap,
 * Table 1) reaches the threshold (Section 2.1, Eq. 1); an RS-join every pair
 * of two collections.  The library computes them exactly, on the GPU, in
 * four stages:
 *   1. one b-bit bitmap per set from hashed tokens (Section 3.2, Alg. 3a-3c,
 *      hash h(t) = t mod b, Section 5.1);
 *   2. for every pair inside the length-filter window (Section 2.3.2,
 *      Table 2) the xor+popcount bound of Theorem 1 (Eq. 2) -- the Bitmap
 *      Filter -- discards pairs that cannot reach the threshold;
 *   3. the surviving pairs are verified exactly by merge intersection of
 *      their sorted token arrays;
 *   4. the similar pairs are returned as original ids (a < b), sorted.
 *
 * Conventions for every entry point:
 *   - Return value: BMJ_OK (0) or a negative BMJ_ERR_* code; bmj_strerror()
 *     names it.  No C++ exception crosses this ABI.  On error, outputs are
 *     left empty (pairs: n = 0, pointers NULL) and nothing is leaked.
 *   - Collections are borrowed, read-only, and must stay valid until the
 *     call returns.  Tokens of a set must be non-negative and strictly
 *     increasing (a set has no repeated element; Bitmap-Xor would cancel a
 *     repeated token), and no set may be empty (Jaccard of two empty sets is
 *     undefined).  Violations are detected on the device and reported as
 *     BMJ_ERR_UNSORTED / BMJ_ERR_NEG_TOKEN / BMJ_ERR_EMPTY_SET.
 *   - Thresholds are exact rationals p/q (0 < p <= q; Overlap counts tokens
 *     and allows p > q); "similar" means sim(x, y) >= p/q, decided in
 *     integers, e.g. Jaccard as |x&y|*(p+q) >= p*(|x|+|y|) (Table 1).  Only
 *     Cosine's smallest passing overlap starts from a floating-point estimate,
 *     which exact 128-bit integer arithmetic then corrects, so every decision
 *     is exact.
 *   - Bitmaps have b bits, b a multiple of 64 in [64, 4096]; bit k of a set's
 *     bitmap is bit (k % 64) of 64-bit word k / 64.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Calls are stream-ordered on that stream; entry points that
 *     return host-visible results synchronise it before returning.
 *   - Device memory for temporaries comes from the CUDA stream-ordered
 *     allocator of the current device; the calling thread's current device
 *     must be the one that holds device-resident inputs.
 */
#ifndef BMJ_H
#define BMJ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define BMJ_OK                   0
#define BMJ_ERR_INVALID_ARG     (-1)  /* NULL pointer, q == 0, p == 0, p > q, bad b/method, n < 0 */
#define BMJ_ERR_UNSORTED        (-2)  /* tokens of a set not strictly increasing, or offsets decreasing */
#define BMJ_ERR_EMPTY_SET       (-3)  /* a set with no token */
#define BMJ_ERR_NEG_TOKEN       (-4)  /* a negative token id */
#define BMJ_ERR_OOM             (-5)  /* device or host allocation failed */
#define BMJ_ERR_OUTPUT_OVERFLOW (-6)  /* a caller-provided output is too small */
#define BMJ_ERR_TIMEOUT         (-7)  /* a bounded device-side wait gave up */
#define BMJ_ERR_CUDA            (-8)  /* a CUDA runtime call failed */
#define BMJ_ERR_TOO_LARGE       (-9)  /* more than 2^31 - 1 sets, or a set of 2^24 tokens or more */
#define BMJ_PENDING              1    /* bmj_serve_poll: not completed yet (not an error) */

/* ---- bitmap generation methods (Section 3.2) ---------------------------- */
#define BMJ_XOR      0   /* Alg. 3b: toggle bit h(t); the paper's GPU default */
#define BMJ_SET      1   /* Alg. 3a: set bit h(t) */
#define BMJ_NEXT     2   /* Alg. 3c: set the first unset bit at or after h(t), circularly; all ones if n >= b */
#define BMJ_COMBINED 3   /* Alg. 4: Next / Set / Xor chosen from the threshold (switch points on 2p/(p+q)) */

/* ---- similarity functions (Table 1) ------------------------------------- */
/* A threshold is p/q; every test is exact in integers:
 *   BMJ_JACCARD  |x&y| / |x|y|          >= p/q   (0 < p <= q)
 *   BMJ_COSINE   |x&y| / sqrt(|x||y|)   >= p/q   (0 < p <= q <= 65535)
 *   BMJ_DICE     2|x&y| / (|x|+|y|)     >= p/q   (0 < p <= q)
 *   BMJ_OVERLAP  |x&y|                  >= p/q   (p, q >= 1; p/q counts tokens)
 * p, q < 2^31.  The length window of each function is the one of Table 2. */
#define BMJ_JACCARD  0
#define BMJ_COSINE   1
#define BMJ_DICE     2
#define BMJ_OVERLAP  3

/* A collection of n_sets sets in CSR form: set x holds
 * tokens[offsets[x] .. offsets[x+1]-1].  offsets has n_sets+1 entries and
 * offsets[0] == 0.  on_device != 0 means both arrays live in device memory;
 * otherwise they are host memory (pinned or pageable) and are copied in. */
typedef struct {
    int64_t        n_sets;
    const int64_t *offsets;
    const int32_t *tokens;
    int32_t        on_device;
    int32_t        reserved;
} bmj_collection;

/* A pair list owned by the library until bmj_pairs_free().  Pair k is
 * (a[k], b[k]) in original 0-based set ids with a[k] < b[k]; pairs are sorted
 * by (a, b) and unique.  on_device says where a and b live; host lists of
 * bmj_self_join are page-locked when possible (host_pinned = 1): then a and b
 * share one block that bmj_pairs_free returns to a reuse pool of the library
 * (at most 8 idle blocks and 4 GiB are kept), so that the next call does not
 * pin pages again. */
typedef struct {
    int64_t   n;
    uint32_t *a;
    uint32_t *b;
    int32_t   on_device;
    int32_t   host_pinned;   /* set by the library; leave it as returned */
} bmj_pairs;

/* Tuning and placement options; bmj_default_options() fills the defaults. */
typedef struct {
    int32_t b;                 /* bitmap bits (default 64) */
    int32_t method;            /* BMJ_XOR (default) / SET / NEXT / COMBINED */
    int32_t output_on_device;  /* 1: pairs returned in device memory; 0 (default): host memory */
    int32_t validate;          /* 1 (default): check the collection invariants on the device */
    int64_t queue_cap;         /* survivor-queue capacity in pairs; 0 (default) = automatic.
                                  bmj_self_join and bmj_rs_join never drop a survivor: when
                                  they exceed the queue, an automatic queue is regrown to the
                                  exact count if that fits in a quarter of free memory;
                                  otherwise (and always for a caller-given capacity) the
                                  filter's work items run in consecutive ranges whose
                                  survivors fit, each verified before the next
                                  (stats.filter_passes counts the passes) */
    void   *stream;            /* cudaStream_t; NULL = legacy default stream */
    int32_t rows_per_thread;   /* bmj_self_join_batch: rows per lane of the filter's row tile.
                                  0 (default) = per job, the width's default tile (as in
                                  bmj_self_join) or a small one (a quarter or fewer of the
                                  rows) where the default tile's diagonal would waste a large
                                  share of a small job's window (cost model in the tuner);
                                  a value below the width's default forces the small tile,
                                  any other value the default */
    int32_t use_graph;         /* bmj_self_join_batch: run the execute stage as a CUDA graph */
    int32_t cascade_b;         /* bmj_self_join, bmj_rs_join: width of a second Bitmap Filter
                                  applied to the survivors before merging (0 = automatic: 256
                                  when b < 256; -1 = none; otherwise a valid b larger than b) */
    int32_t sim;               /* bmj_index_create: similarity function of every query on the
                                  index (default BMJ_JACCARD); bmj_self_join, bmj_rs_join and
                                  bmj_self_join_batch take it as an argument instead */
    int64_t row_begin;         /* bmj_self_join: join only the pairs whose later set in size order
                                  (sets ordered by size, ties by id) has its position in */
    int64_t row_end;           /*   [row_begin, row_end); 0, 0 = every pair.  Bands that cover
                                  [0, n) give disjoint pair lists whose union is the full join. */
    int32_t candidates;        /* bmj_self_join, bmj_rs_join: BMJ_CAND_WINDOW (default) filters
                                  every pair of the length window; BMJ_CAND_PREFIX filters only the window
                                  pairs whose prefixes share a token (prefix filter, Section 2.2)
                                  -- fewer pairs at high thresholds, same result.  Its candidates
                                  are expanded in ranges of at most queue_cap slots (0: a quarter
                                  of the free device memory), each filtered and verified before
                                  the next, so any number of them fits; it falls back to the
                                  window only when the prefix index itself does not fit.
                                  BMJ_CAND_AUTO builds the prefix index and takes the prefix
                                  filter or the window, whichever its slot count says is faster.
                                  Both need row_begin = row_end = 0 and cutoff = 0 */
    int32_t cutoff;            /* bmj_self_join, bmj_rs_join: the cutoff point of Section 3.5.
                                  0 (default) = none, every window pair meets the Bitmap Filter
                                  (the paper's GPU setting); n > 0 = a pair whose larger set has
                                  more than n tokens skips the filter and is verified directly;
                                  BMJ_CUTOFF_AUTO = n from Eq. 4-6 for b, the method used and the
                                  normalised threshold (Jaccard 2p/(p+q), Dice and Cosine p/q;
                                  none for Overlap).  With BMJ_CAND_PREFIX or AUTO it must be 0. */
} bmj_options;

#define BMJ_CUTOFF_AUTO (-1)
#define BMJ_CAND_WINDOW 0
#define BMJ_CAND_PREFIX 1
#define BMJ_CAND_AUTO   2   /* the prefix filter when its candidate slots are few enough for the
                               expansion to beat the whole window (a per-width cost ratio
                               measured on a B300), else the window */

/* Counters and stage times of one join.  Pair counts are exact and do not
 * depend on the launch configuration. */
typedef struct {
    int64_t window_pairs;   /* pairs (i, j) inside the length-filter window = pairs the Bitmap Filter evaluated */
    int64_t survivors;      /* pairs that passed the Bitmap Filter (verified exactly) */
    int64_t results;        /* similar pairs returned */
    int64_t filter_passes;  /* filter launches over the whole window (1 unless the survivor queue had to grow) */
    int64_t verified;       /* survivors that passed the cascade bound and were merged (= survivors without cascade) */
    int32_t n_launches;     /* CUDA kernels launched by this call */
    int32_t b;              /* bitmap bits used */
    int32_t method;         /* generation method used (COMBINED resolved) */
    int32_t max_set_size;
    int32_t cascade_b;      /* width of the cascade bitmaps, 0 = none */
    int32_t cutoff;         /* cutoff point applied (set size), 0 = none */
    float   ms_prepare;     /* validation, size sort, sorted-CSR gather and bitmap build */
    float   ms_filter;      /* Bitmap Filter kernel(s) */
    float   ms_verify;      /* verification kernel(s) */
    float   ms_output;      /* result sort, id mapping and output copy */
    float   ms_total;       /* whole call, device time on the stream */
    float   reserved_f;
    int64_t candidates;     /* BMJ_CAND_PREFIX: distinct prefix-filter candidates, which the
                               Bitmap Filter then evaluated (survivors counts those passing it);
                               0 in window mode; -1 when prefix mode fell back to the window
                               (only when the prefix index itself does not fit in memory); -2
                               when BMJ_CAND_AUTO chose the window */
    int64_t candidate_slots;/* BMJ_CAND_PREFIX / AUTO: (rank, pair) slots the candidates were expanded
                               from (a pair sharing k prefix tokens has k slots); they go
                               through a buffer of fixed size in filter_passes ranges */
    int32_t tile_rows;      /* rows of the filter's tile (32 x rows per lane), of the job's tile in
                               bmj_self_join_batch job stats */
    int32_t chunk_cols;     /* ... and columns per filter work item */
    int64_t fold_steps;     /* b = 128 and 256: warp column steps of the filter (the tile_rows
                               rows of a warp's tile against one column each), every one first
                               tested with the two halves of the xor folded onto each other
                               (64 or 128 bits; no more differing bits than the full xor, so a
                               pair that fails it fails Eq. 2); counted over the first filter
                               pass, 0 at other widths */
    int64_t fold_full_steps;/* ... those in which some pair passed the folded test, so that the
                               warp ran the full-width test */
} bmj_stats;

/* Counters and stage times of one bmj_self_join_batch call. */
typedef struct {
    int64_t n_jobs;
    int64_t window_pairs;   /* summed over the jobs */
    int64_t survivors;
    int64_t results;
    int32_t n_launches;     /* CUDA kernels launched (kernels inside a graph counted once) */
    int32_t filter_passes;  /* 1 unless the survivor queue had to grow */
    int32_t graph;          /* 1 when the execute stage ran as a CUDA graph */
    int32_t tuned;          /* 1 when b was chosen per job by the autotuner */
    float   ms_prepare;     /* validation, sort, sorted CSR, bitmaps, thresholds, window sizes */
    float   ms_tune;        /* autotuner sampling */
    float   ms_execute;     /* Bitmap Filter + verification of every job */
    float   ms_output;
    float   ms_total;       /* whole call, device time on the stream */
    float   reserved_f[3];
} bmj_batch_stats;

/* Fills *opt with the defaults listed above.  Never fails. */
void bmj_default_options(bmj_options *opt);

/* Human-readable name of a status code (static storage; never NULL). */
const char *bmj_strerror(int status);

/*
 * Per-set bitmaps (Section 3.2; Alg. 5 initialisation).
 *   coll    collection (host or device, see bmj_collection)
 *   b       bitmap bits, a multiple of 64 in [64, 4096]
 *   method  BMJ_XOR, BMJ_SET or BMJ_NEXT (BMJ_COMBINED needs a threshold:
 *           BMJ_ERR_INVALID_ARG)
 *   out     caller-owned array of n_sets * (b/64) uint64 words, set x at
 *           out[x*(b/64) .. x*(b/64)+b/64-1], in original set order; it is
 *           device memory iff coll->on_device, otherwise host memory
 *   stream  cudaStream_t as void* (NULL = legacy default stream)
 * The call validates the collection, writes every word of out and, for host
 * output, synchronises the stream before returning.
 */
int bmj_build_bitmaps(const bmj_collection *coll, int b, int method, uint64_t *out,
                      void *stream);

/*
 * Exact self-join with the Bitmap Filter (Section 4.2, Alg. 6, with the
 * verification moved onto the GPU).
 *   coll    collection (host or device)
 *   sim     BMJ_JACCARD, BMJ_COSINE, BMJ_DICE or BMJ_OVERLAP
 *   p, q    threshold p/q (ranges above; BMJ_ERR_INVALID_ARG outside them)
 *   opt     options (NULL = defaults)
 *   out     receives the library-owned, canonical pair list (free it with
 *           bmj_pairs_free); on error it is left empty
 *   stats   optional (NULL allowed): counters and stage times
 * The stream in opt is synchronised before the call returns.
 */
int bmj_self_join(const bmj_collection *coll, int sim, uint32_t p, uint32_t q,
                  const bmj_options *opt, bmj_pairs *out, bmj_stats *stats);

/*
 * Exact RS-join (Section 2.1, Eq. 1 with R and S two collections): every pair
 * (r, s) of R x S with sim(r, s) >= p/q, by the algorithm of bmj_self_join
 * (length window of Table 2 with both of its bounds, Bitmap Filter, exact
 * verification).
 *   r, s    the two collections (host or device, independently); each must
 *           start at offset 0; r->n_sets + s->n_sets < 2^31
 *           (BMJ_ERR_TOO_LARGE otherwise)
 *   sim, p, q, opt, stats  as for bmj_self_join; opt->row_begin / row_end
 *           must be 0 (BMJ_ERR_INVALID_ARG otherwise); with
 *           opt->candidates = BMJ_CAND_PREFIX the candidates are the window
 *           pairs whose prefixes share a token, tokens ranked by their
 *           frequency over R and S together
 *   out     library-owned pairs (free with bmj_pairs_free): a = id in R, b = id
 *           in S, sorted by (a, b); every pair appears once
 * Either collection empty gives an empty result.  The stream in opt is
 * synchronised before the call returns.
 */
int bmj_rs_join(const bmj_collection *r, const bmj_collection *s, int sim, uint32_t p, uint32_t q,
                const bmj_options *opt, bmj_pairs *out, bmj_stats *stats);

/*
 * Many independent exact self-joins in one pass over the GPU (no counterpart
 * in the paper, which joins one collection per run; the arithmetic of every
 * job is the one of bmj_self_join).
 *   coll      all jobs' sets concatenated into one collection (host or device)
 *   n_jobs    number of jobs (>= 1)
 *   job_sets  host int64[n_jobs+1]: job k is sets [job_sets[k], job_sets[k+1])
 *             of coll; job_sets[0] = 0, job_sets[n_jobs] = coll->n_sets,
 *             nondecreasing (empty jobs allowed)
 *   sim       BMJ_JACCARD
 *   p, q      host uint32[n_jobs]: threshold p[k]/q[k] of job k (0 < p <= q)
 *   opt       options (NULL = defaults).  opt->b = 0 lets a sampling
 *             autotuner pick b in {64, 128, 256} per job (cost = window pairs
 *             x measured filter time per pair + estimated survivors x measured
 *             verification time per survivor); BMJ_COMBINED resolves the
 *             method per job; opt->use_graph runs the filter + verification
 *             stage as a CUDA graph; opt->cascade_b is 0 (jobs with b < 256 get
 *             the 256-bit check before merging, and the autotuner counts it),
 *             -1 (none) or 256; row_begin, row_end, candidates and cutoff must
 *             be 0 (BMJ_ERR_INVALID_ARG otherwise).
 *   outs      n_jobs pair lists (library-owned; free each with
 *             bmj_pairs_free), in job-local ids (0 = the job's first set),
 *             sorted and unique as for bmj_self_join
 *   job_stats optional n_jobs entries: window_pairs, survivors, results, b,
 *             method per job
 *   batch_stats optional totals and stage times
 * Errors as for bmj_self_join; BMJ_ERR_TOO_LARGE also when
 * bits(n_jobs - 1) + bits(max set size) > 32 or
 * bits(n_jobs - 1) + 2 * bits(largest job - 1) > 64.
 */
int bmj_self_join_batch(const bmj_collection *coll, int64_t n_jobs, const int64_t *job_sets,
                        int sim, const uint32_t *p, const uint32_t *q, const bmj_options *opt,
                        bmj_pairs *outs, bmj_stats *job_stats, bmj_batch_stats *batch_stats);

/* ---- resident index and served queries --------------------------------- */

/* A collection kept resident on the device in size order (sizes, sorted CSR,
 * b-bit bitmaps), built once and probed many times. */
typedef struct bmj_index bmj_index;

/* Result of a query batch: the ids of query x are
 * ids[offsets[x] .. offsets[x+1]-1] (original resident ids, ascending).
 * Library-owned host memory; free with bmj_id_lists_free. */
typedef struct {
    int64_t  n_queries;
    int64_t *offsets;   /* n_queries + 1 */
    int64_t *ids;
} bmj_id_lists;

typedef struct {
    int32_t n_slots;               /* batches in flight at once (default 4) */
    int32_t reserved0;
    int64_t max_batch_queries;     /* queries per batch (default 4096) */
    int64_t max_batch_window_pairs;/* memory admission: window pairs per batch (default 2^25);
                                      raised to the largest single query's window */
    int64_t max_probe_tokens;      /* bmj_serve_open: largest probe a submission may hold
                                      (default 4096); bmj_serve sizes it from its queries */
    int64_t reserved[3];
} bmj_serve_options;

typedef struct {
    int64_t n_queries;
    int64_t batches;
    int64_t window_pairs;   /* pairs the Bitmap Filter evaluated */
    int64_t survivors;
    int64_t results;
    double  wall_s;         /* from the first arrival slot to the last completion */
    double  qps;
    double  p50_ms, p99_ms, max_ms;  /* latency = completion - arrival */
    double  reserved[4];
} bmj_serve_stats;

/*
 * Builds a resident index of coll (host or device; copied, so the caller may
 * free coll afterwards) with opt->b and opt->method (BMJ_XOR, BMJ_SET or
 * BMJ_NEXT; NULL = defaults).  The index is bound to the current device.
 * Errors as for bmj_self_join.  No counterpart in the paper beyond Alg. 5's
 * initialisation (bitmaps of every set built once).
 */
int bmj_index_create(const bmj_collection *coll, const bmj_options *opt, bmj_index **out);
void bmj_index_destroy(bmj_index *idx);
int64_t bmj_index_size(const bmj_index *idx);

/*
 * Errors stick to an index: once a call on it fails with BMJ_ERR_CUDA or
 * BMJ_ERR_TIMEOUT (its device state is then in doubt), every later
 * bmj_index_query / bmj_serve on it returns that status without running, and
 * only bmj_index_destroy remains useful.  Argument errors and BMJ_ERR_OOM do
 * not stick.  bmj_index_status returns the sticky status (BMJ_OK while the
 * index is usable; BMJ_ERR_INVALID_ARG for NULL).
 */
int bmj_index_status(const bmj_index *idx);

/* Fills *opt with the serving defaults listed above. */
void bmj_default_serve_options(bmj_serve_options *opt);

/*
 * Probe queries against the index: for every probe set x (host collection,
 * tokens strictly increasing) the resident sets s with
 * sim(x, s) >= p[x]/q[x] (an RS-join with |R| = 1, Eq. 1), sim being the
 * index's function (bmj_options.sim at creation; thresholds outside its range
 * give BMJ_ERR_INVALID_ARG).  Candidates
 * are the resident sets inside both sides of the length window (Table 2),
 * filtered by the Eq. 2 bound and verified exactly.  Runs as one batch and
 * returns when done.  out is filled (free with bmj_id_lists_free); stats
 * optional.
 */
int bmj_index_query(bmj_index *idx, const bmj_collection *probes, const uint32_t *p,
                    const uint32_t *q, bmj_id_lists *out, bmj_serve_stats *stats);

/*
 * Serves an arrival stream with continuous batching: query x becomes
 * available at arrival_s[x] seconds after the call starts (nondecreasing).
 * Arrived queries are admitted into a free slot (stream + fixed buffers) up
 * to opt->max_batch_queries and while the batch's exact window-pair count
 * stays within opt->max_batch_window_pairs (this bounds every buffer of the
 * batch); up to opt->n_slots batches are in flight and overlap on the device.
 * Results go to *out (optional), per-query latency in milliseconds to
 * latency_ms[x] (optional), totals and p50/p99 to *stats (optional).  Each
 * query's result does not depend on how it was batched.
 */
int bmj_serve(bmj_index *idx, const bmj_collection *queries, const double *arrival_s,
              const uint32_t *p, const uint32_t *q, const bmj_serve_options *opt,
              bmj_id_lists *out, double *latency_ms, bmj_serve_stats *stats);

/* ---- live serving: queries submitted while other batches run ------------ */

/* A request loop over an index (its own host thread and stream slots). */
typedef struct bmj_server bmj_server;

/*
 * Opens a live server on idx (no counterpart in the paper; the arithmetic of
 * every query is the one of bmj_index_query).  opt as for bmj_serve (NULL =
 * defaults): n_slots batches in flight, at most max_batch_queries queries and
 * max_batch_window_pairs window pairs per batch (raised to the index's size,
 * the largest window a single query can have), probes of at most
 * max_probe_tokens tokens.  The server allocates its slots (stream, pinned and
 * device buffers) once, here, and starts its loop thread: queries submitted
 * from any thread are admitted into free slots by the exact window-pair count
 * of the batch (memory admission) while earlier batches are on the device,
 * and several batches overlap.  idx must outlive the server.
 * Errors: BMJ_ERR_INVALID_ARG, BMJ_ERR_OOM, BMJ_ERR_CUDA, or the index's
 * sticky status.
 */
int bmj_serve_open(bmj_index *idx, const bmj_serve_options *opt, bmj_server **out);

/*
 * Submits one probe set: tokens[0 .. n_tokens-1] (host memory, strictly
 * increasing, non-negative; copied, so the caller may reuse the buffer) with
 * threshold p/q for the index's similarity function.  *ticket receives the
 * query's ticket (0, 1, 2, ... in submission order).  Thread-safe.
 * Errors: BMJ_ERR_INVALID_ARG (NULL, bad threshold, or after
 * bmj_serve_close began), BMJ_ERR_EMPTY_SET, BMJ_ERR_UNSORTED,
 * BMJ_ERR_NEG_TOKEN, BMJ_ERR_TOO_LARGE (more than max_probe_tokens), or a
 * device failure of the server's loop (sticky).
 */
int bmj_serve_submit(bmj_server *srv, const int32_t *tokens, int64_t n_tokens, uint32_t p,
                     uint32_t q, int64_t *ticket);

/*
 * The result of a submitted query: BMJ_OK with out filled (one list: the
 * resident ids s with sim(x, s) >= p/q, ascending; free with
 * bmj_id_lists_free) and *latency_ms (optional) = completion - submission;
 * BMJ_PENDING when the query has not completed within wait_ms milliseconds
 * (0 = do not wait); a negative status when its batch failed.  A result is
 * handed out once: a second poll of the same ticket, like an unknown ticket,
 * gives BMJ_ERR_INVALID_ARG.  Thread-safe.
 */
int bmj_serve_poll(bmj_server *srv, int64_t ticket, int32_t wait_ms, bmj_id_lists *out,
                   double *latency_ms);

/*
 * Finishes every submitted query, stops the loop and frees the server;
 * results not yet polled are dropped.  stats (optional): the queries
 * completed, batches, window pairs, survivors, results, p50/p99/max latency
 * (completion - submission) and qps over the time from open to the last
 * completion.  Returns the loop's device failure, if any (BMJ_OK otherwise).
 */
int bmj_serve_close(bmj_server *srv, bmj_serve_stats *stats);

void bmj_id_lists_free(bmj_id_lists *lists);

/* Releases a pair list returned by the library and empties *pairs.
 * Safe on an empty or already freed list. */
void bmj_pairs_free(bmj_pairs *pairs);

/* Gives every idle page-locked block of the library's reuse pool back to the
 * CUDA driver and returns the number of bytes released.  Lists still held by
 * the caller are untouched (they return to the pool when freed).  Calls no
 * CUDA function when the pool is empty. */
int64_t bmj_host_pool_trim(void);

/* Number of CUDA kernels this library has launched in this process (a
 * monotone counter, for accounting in benchmarks). */
int64_t bmj_kernel_launches(void);

/* Measures the device's 32-bit population-count throughput (popcounts per
 * second over all SMs, a 65,536-iteration loop of independent popcounts on
 * every resident thread; about 40 ms on a B300) on `stream` (cudaStream_t,
 * NULL = legacy default stream).  This is the peak of the Bitmap Filter's
 * roofline, which needs b/32 popcounts per window pair.  Returns a BMJ status;
 * *popc_per_s is 0 on error. */
int bmj_measure_popc_rate(void *stream, double *popc_per_s);

/* Size of the device scratch array used by bmj_bitmap_filter_noalloc. */
#define BMJ_NOALLOC_SCRATCH_BYTES (8u << 20)

/*
 * bmj_bitmap_filter_noalloc -- the Bitmap Filter alone, without allocating.
 * The paper has no counterpart to this entry point; it exists for callers
 * that must not allocate device memory while they run: code inside a fixed
 * memory budget owned by another framework's pool, latency-critical serving
 * loops where cudaMalloc/cudaFree (which can synchronise the device) are not
 * allowed, and sandboxes that forbid allocator calls altogether.  It calls
 * no cudaMalloc, cudaFree or allocating library routine.
 *
 * Inputs describe a collection already ordered by set size (the order
 * bmj_self_join uses internally):
 *   bitmaps    device, n_sets * (b/64) uint64 words; row i is the bitmap of
 *              the set at sorted position i (e.g. bmj_build_bitmaps run on
 *              the size-sorted collection)
 *   sizes      device, n_sets uint32 set sizes, each >= 1, nondecreasing
 *   b, p, q    bitmap bits (multiple of 64 in [64, 4096]) and Jaccard threshold p/q
 * Output (caller-owned):
 *   out_pairs  device, 2*out_cap uint32, 8-byte aligned: the surviving pairs
 *              as (i, j) with j < i in sorted positions, in no particular
 *              order -- every pair inside the length window whose Eq. 2
 *              bound reaches the threshold, the same set of pairs that
 *              bmj_self_join verifies (its stats.survivors counts them)
 *   out_count  host: the number of survivors.  If it exceeds out_cap, the
 *              call returns BMJ_ERR_OUTPUT_OVERFLOW, out_count still holds
 *              the full count and out_pairs holds out_cap of the survivors.
 * Scratch: one file-scope device array of BMJ_NOALLOC_SCRATCH_BYTES (8 MiB)
 *   per device that loads the library, held until the process exits.  It
 *   holds 32 bytes of counters, 4*(2*max_size+1) bytes of thresholds and
 *   about 12 bytes per 128 sets (per 64 sets when b = 512, per 32 sets for
 *   other b beyond 256) of window tiles; a collection needing more returns
 *   BMJ_ERR_TOO_LARGE before any launch.  The counters are cleared on every
 *   call.  Every call shares the array: calls that overlap on the GPU (other
 *   streams or host threads) race and must be serialised by the caller.
 * Set-up: the first call on a device looks up the array's device address
 *   with that device current (cudaGetSymbolAddress).
 * Synchronisation: every call copies the counters back and synchronises
 *   `stream` before it returns, so it must not be called while a stream is
 *   being captured into a CUDA graph.
 * Errors: BMJ_ERR_INVALID_ARG (NULL or misaligned pointers, bad b, p, q),
 *   BMJ_ERR_UNSORTED (sizes decrease), BMJ_ERR_EMPTY_SET (a size of 0),
 *   BMJ_ERR_TOO_LARGE, BMJ_ERR_OUTPUT_OVERFLOW, BMJ_ERR_CUDA.  The stream is
 *   synchronised before the call returns.
 */
int bmj_bitmap_filter_noalloc(const uint64_t *bitmaps, const uint32_t *sizes, int64_t n_sets,
                              int b, uint32_t p, uint32_t q, uint32_t *out_pairs,
                              int64_t out_cap, int64_t *out_count, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BMJ_H */
