/*
 * oracle.c -- plain CPU oracle for exact set-similarity self-joins and the
 * Bitmap Filter (Sandes, Teodoro & Melo, "Bitmap Filter: Speeding up Exact
 * Set Similarity Joins with Bitwise Operations").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may call, link or
 * include this file; only the tests, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header or table with the CUDA
 * path.  Every function is written as plainly as the definition allows, in
 * 64-bit integer arithmetic (the method is exact integer work: there is no
 * floating point anywhere in this file).
 *
 * Conventions shared with the paper:
 *   - a collection is N sets in CSR form: set x holds tokens
 *     tok[off[x] .. off[x+1]-1], strictly increasing, non-negative
 *     (sets have no repeated elements, Section 2.1);
 *   - Jaccard J(x,y) = |x & y| / |x | y| (Table 1); the threshold is the
 *     rational p/q, and "similar" means J >= p/q (Eq. 1 uses >=).  Since
 *     |x | y| = |x| + |y| - |x & y|, J >= p/q  <=>  o*(p+q) >= p*(|x|+|y|)
 *     with o = |x & y|; both sides are exact in int64;
 *   - bitmaps have b bits, b a multiple of 64, stored as b/64 uint64 words;
 *     bit k lives in word k/64 at bit position k%64; the hash is
 *     h(t) = t mod b (Section 5.1).
 *
 * Functions:
 *   oracle_overlap        |x & y| by a plain two-pointer merge (Alg. 1 verify)
 *   oracle_similar        the integer Jaccard test above
 *   oracle_similar_sim    the same for Jaccard, Cosine, Dice and Overlap (Table 1)
 *   oracle_in_window      the length filter of Table 2 for any of them
 *   oracle_self_join      Alg. 1 over all pairs a<b, no filter at all
 *   oracle_join_rows      Alg. 1 restricted to pairs touching sampled rows
 *   oracle_join_rows_window  the same with the length filter of Table 2
 *   oracle_search         one probe set against every set of a collection
 *   oracle_bitmap         Alg. 3a (Set), 3b (Xor), 3c (Next), literally
 *   oracle_filter_counts  the GPU algorithm (Alg. 6): size order, length
 *                         window, Eq. 2 bound, then verification -- counted
 *   oracle_window_pairs_hist  the window count of oracle_filter_counts from the
 *                         size histogram alone (Table 2)
 *   oracle_rs_window_pairs_hist  the same for the pairs of R x S
 *   oracle_prefix_counts  the same with the prefix filter (Section 2.2)
 *                         choosing the candidates inside the window
 *   oracle_rs_join        Eq. 1 between two collections R and S (an RS-join,
 *                         Section 2.1): every pair (r, s) verified
 *   oracle_rs_filter_counts  window pairs, Bitmap Filter survivors and
 *                         results of an RS-join (length window of Table 2,
 *                         Eq. 2), counted over every pair of R x S
 *   oracle_rs_prefix_counts  the same with the prefix filter choosing the
 *                         candidates among the window pairs of R x S
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_XOR = 0, OR_SET = 1, OR_NEXT = 2, OR_COMBINED = 3 };
enum { OR_JACCARD = 0, OR_COSINE = 1, OR_DICE = 2, OR_OVERLAP = 3 };

/* |x & y| for two strictly increasing token arrays (plain merge). */
int64_t oracle_overlap(const int32_t *x, int64_t nx, const int32_t *y, int64_t ny)
{
    int64_t i = 0, j = 0, o = 0;
    while (i < nx && j < ny) {
        if (x[i] == y[j]) { o++; i++; j++; }
        else if (x[i] < y[j]) i++;
        else j++;
    }
    return o;
}

/* Jaccard(x,y) >= p/q, as o*(p+q) >= p*(|x|+|y|) (Table 1, Eq. 1). */
int oracle_similar(int64_t o, int64_t nx, int64_t ny, int64_t p, int64_t q)
{
    return o * (p + q) >= p * (nx + ny);
}

/*
 * sim(x,y) >= p/q for the four functions of Table 1, each cleared of its
 * fraction (and of the square root for Cosine) so that the test is exact in
 * integers (128-bit where a product of four 32-bit factors can occur):
 *   Jaccard  o / (|x|+|y|-o) >= p/q   <=>  o*(p+q)     >= p*(|x|+|y|)
 *   Cosine   o / sqrt(|x||y|) >= p/q  <=>  o^2*q^2     >= p^2*|x|*|y|
 *   Dice     2o / (|x|+|y|) >= p/q    <=>  2*o*q       >= p*(|x|+|y|)
 *   Overlap  o >= p/q                 <=>  o*q         >= p
 */
int oracle_similar_sim(int sim, int64_t o, int64_t nx, int64_t ny, int64_t p, int64_t q)
{
    switch (sim) {
    case OR_JACCARD: return oracle_similar(o, nx, ny, p, q);
    case OR_COSINE: {
        __int128 lhs = (__int128)o * o * q * q;
        __int128 rhs = (__int128)p * p * nx * ny;
        return lhs >= rhs;
    }
    case OR_DICE: return 2 * o * q >= p * (nx + ny);
    case OR_OVERLAP: return o * q >= p;
    }
    return 0;
}

/*
 * The length filter of Table 2 for sizes a <= b: a pair of sizes (a, b) can
 * reach the threshold only if the overlap min(a,b) = a does, i.e. if
 * sim(a, b) with o = a passes.  Returns 1 when (a, b) is inside the window.
 */
int oracle_in_window(int sim, int64_t a, int64_t b, int64_t p, int64_t q)
{
    return oracle_similar_sim(sim, a, a, b, p, q);
}

/* Growable pair buffer. */
typedef struct { uint32_t *a, *b; int64_t n, cap; } pairbuf;

static int pb_push(pairbuf *pb, uint32_t a, uint32_t b)
{
    if (pb->n == pb->cap) {
        int64_t nc = pb->cap ? 2 * pb->cap : 64;
        uint32_t *na = (uint32_t *)realloc(pb->a, (size_t)nc * sizeof(uint32_t));
        if (!na) return -1;
        pb->a = na;
        uint32_t *nb = (uint32_t *)realloc(pb->b, (size_t)nc * sizeof(uint32_t));
        if (!nb) return -1;
        pb->b = nb;
        pb->cap = nc;
    }
    pb->a[pb->n] = a;
    pb->b[pb->n] = b;
    pb->n++;
    return 0;
}

void oracle_free(void *p) { free(p); }

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Alg. 1 (naive algorithm) for a self-join: every pair a < b of original
 * ids is verified; the output is every similar pair, in (a, b) order.
 * Rows are independent, so they are spread over threads (dynamic
 * schedule); each row's pairs are collected separately and concatenated in
 * row order, so the output order is the sequential order.
 * Returns the pair count, or -1 on allocation failure.  *out_a / *out_b are
 * malloc'd (free with oracle_free); both are NULL when the count is 0.
 */
int64_t oracle_self_join(int64_t n, const int64_t *off, const int32_t *tok, int sim,
                         int64_t p, int64_t q, uint32_t **out_a, uint32_t **out_b)
{
    *out_a = NULL;
    *out_b = NULL;
    if (n <= 1) return 0;
    pairbuf *rows = (pairbuf *)calloc((size_t)n, sizeof(pairbuf));
    if (!rows) return -1;
    int failed = 0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t a = 0; a < n; a++) {
        const int32_t *xa = tok + off[a];
        int64_t na = off[a + 1] - off[a];
        for (int64_t b = a + 1; b < n; b++) {
            const int32_t *xb = tok + off[b];
            int64_t nb = off[b + 1] - off[b];
            int64_t o = oracle_overlap(xa, na, xb, nb);
            if (oracle_similar_sim(sim, o, na, nb, p, q))
                if (pb_push(&rows[a], (uint32_t)a, (uint32_t)b)) failed = 1;
        }
    }
    int64_t total = 0;
    for (int64_t a = 0; a < n; a++) total += rows[a].n;
    uint32_t *A = NULL, *B = NULL;
    if (!failed && total > 0) {
        A = (uint32_t *)malloc((size_t)total * sizeof(uint32_t));
        B = (uint32_t *)malloc((size_t)total * sizeof(uint32_t));
        if (!A || !B) failed = 1;
    }
    int64_t k = 0;
    for (int64_t a = 0; a < n; a++) {
        if (!failed && rows[a].n) {
            memcpy(A + k, rows[a].a, (size_t)rows[a].n * sizeof(uint32_t));
            memcpy(B + k, rows[a].b, (size_t)rows[a].n * sizeof(uint32_t));
            k += rows[a].n;
        }
        free(rows[a].a);
        free(rows[a].b);
    }
    free(rows);
    if (failed) { free(A); free(B); return -1; }
    *out_a = A;
    *out_b = B;
    return total;
}

/*
 * Alg. 1 restricted to the pairs that touch a row in rows[0..k-1] (original
 * ids, any order, duplicates allowed): for each sampled row r, every other
 * set s is verified and a similar pair is emitted as (min(r,s), max(r,s)).
 * The output is sorted by (a, b) with duplicates removed (a pair whose two
 * ends are both sampled is found twice).  This gives exact parity for a
 * sample of rows of a join too large for Alg. 1 in full.
 */
static int cmp_pair64(const void *x, const void *y)
{
    uint64_t u = *(const uint64_t *)x, v = *(const uint64_t *)y;
    return (u > v) - (u < v);
}

int64_t oracle_join_rows(int64_t n, const int64_t *off, const int32_t *tok, int sim,
                         int64_t p, int64_t q, const int64_t *rows, int64_t k,
                         uint32_t **out_a, uint32_t **out_b)
{
    *out_a = NULL;
    *out_b = NULL;
    if (k <= 0 || n <= 1) return 0;
    pairbuf *per = (pairbuf *)calloc((size_t)k, sizeof(pairbuf));
    if (!per) return -1;
    int failed = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < k; t++) {
        int64_t r = rows[t];
        const int32_t *xr = tok + off[r];
        int64_t nr = off[r + 1] - off[r];
        for (int64_t s = 0; s < n; s++) {
            if (s == r) continue;
            int64_t ns = off[s + 1] - off[s];
            int64_t o = oracle_overlap(xr, nr, tok + off[s], ns);
            if (oracle_similar_sim(sim, o, nr, ns, p, q)) {
                uint32_t a = (uint32_t)(r < s ? r : s), b = (uint32_t)(r < s ? s : r);
                if (pb_push(&per[t], a, b)) failed = 1;
            }
        }
    }
    int64_t total = 0;
    for (int64_t t = 0; t < k; t++) total += per[t].n;
    uint64_t *keys = NULL;
    if (!failed && total > 0) {
        keys = (uint64_t *)malloc((size_t)total * sizeof(uint64_t));
        if (!keys) failed = 1;
    }
    int64_t m = 0;
    for (int64_t t = 0; t < k; t++) {
        for (int64_t i = 0; !failed && i < per[t].n; i++)
            keys[m++] = ((uint64_t)per[t].a[i] << 32) | per[t].b[i];
        free(per[t].a);
        free(per[t].b);
    }
    free(per);
    if (failed) { free(keys); return -1; }
    if (total == 0) return 0;
    qsort(keys, (size_t)total, sizeof(uint64_t), cmp_pair64);
    int64_t u = 0;
    for (int64_t i = 0; i < total; i++)
        if (i == 0 || keys[i] != keys[i - 1]) keys[u++] = keys[i];
    uint32_t *A = (uint32_t *)malloc((size_t)u * sizeof(uint32_t));
    uint32_t *B = (uint32_t *)malloc((size_t)u * sizeof(uint32_t));
    if (!A || !B) { free(A); free(B); free(keys); return -1; }
    for (int64_t i = 0; i < u; i++) {
        A[i] = (uint32_t)(keys[i] >> 32);
        B[i] = (uint32_t)(keys[i] & 0xffffffffu);
    }
    free(keys);
    *out_a = A;
    *out_b = B;
    return u;
}

/*
 * oracle_join_rows with the length filter (Section 2.3.2, Table 2): a sampled
 * row r is verified only against the sets s whose size is inside its window
 * (oracle_in_window; for Jaccard [ceil(p|r|/q), floor(q|r|/p)]) -- outside it
 * sim(r,s) < p/q for any contents, so the output equals oracle_join_rows'.
 * The sets are visited through size buckets built once per call (a counting
 * sort of the ids by size).  It exists to time the plain join with the
 * paper's cheapest filter beside the plain definition.
 */
int64_t oracle_join_rows_window(int64_t n, const int64_t *off, const int32_t *tok, int sim,
                                int64_t p, int64_t q, const int64_t *rows, int64_t k,
                                uint32_t **out_a, uint32_t **out_b)
{
    *out_a = NULL;
    *out_b = NULL;
    if (k <= 0 || n <= 1) return 0;
    int64_t max_size = 0;
    for (int64_t s = 0; s < n; s++)
        if (off[s + 1] - off[s] > max_size) max_size = off[s + 1] - off[s];
    /* bucket[z] .. bucket[z+1]-1: positions in by_size of the sets of size z */
    int64_t *bucket = (int64_t *)calloc((size_t)max_size + 2, sizeof(int64_t));
    int64_t *by_size = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    pairbuf *per = (pairbuf *)calloc((size_t)k, sizeof(pairbuf));
    if (!bucket || !by_size || !per) { free(bucket); free(by_size); free(per); return -1; }
    for (int64_t s = 0; s < n; s++) bucket[off[s + 1] - off[s] + 1]++;
    for (int64_t z = 0; z <= max_size; z++) bucket[z + 1] += bucket[z];
    {
        int64_t *fill = (int64_t *)malloc((size_t)(max_size + 1) * sizeof(int64_t));
        if (!fill) { free(bucket); free(by_size); free(per); return -1; }
        memcpy(fill, bucket, (size_t)(max_size + 1) * sizeof(int64_t));
        for (int64_t s = 0; s < n; s++) by_size[fill[off[s + 1] - off[s]]++] = s;
        free(fill);
    }
    int failed = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < k; t++) {
        int64_t r = rows[t];
        const int32_t *xr = tok + off[r];
        int64_t nr = off[r + 1] - off[r];
        for (int64_t z = 0; z <= max_size; z++) {
            if (bucket[z] == bucket[z + 1]) continue;
            if (!oracle_in_window(sim, z < nr ? z : nr, z < nr ? nr : z, p, q)) continue;
            for (int64_t x = bucket[z]; x < bucket[z + 1]; x++) {
                int64_t s = by_size[x];
                if (s == r) continue;
                int64_t o = oracle_overlap(xr, nr, tok + off[s], z);
                if (oracle_similar_sim(sim, o, nr, z, p, q)) {
                    uint32_t a = (uint32_t)(r < s ? r : s), b = (uint32_t)(r < s ? s : r);
                    if (pb_push(&per[t], a, b)) failed = 1;
                }
            }
        }
    }
    free(bucket);
    free(by_size);
    int64_t total = 0;
    for (int64_t t = 0; t < k; t++) total += per[t].n;
    uint64_t *keys = NULL;
    if (!failed && total > 0) {
        keys = (uint64_t *)malloc((size_t)total * sizeof(uint64_t));
        if (!keys) failed = 1;
    }
    int64_t m = 0;
    for (int64_t t = 0; t < k; t++) {
        for (int64_t i = 0; !failed && i < per[t].n; i++)
            keys[m++] = ((uint64_t)per[t].a[i] << 32) | per[t].b[i];
        free(per[t].a);
        free(per[t].b);
    }
    free(per);
    if (failed) { free(keys); return -1; }
    if (total == 0) return 0;
    qsort(keys, (size_t)total, sizeof(uint64_t), cmp_pair64);
    int64_t u = 0;
    for (int64_t i = 0; i < total; i++)
        if (i == 0 || keys[i] != keys[i - 1]) keys[u++] = keys[i];
    uint32_t *A = (uint32_t *)malloc((size_t)u * sizeof(uint32_t));
    uint32_t *B = (uint32_t *)malloc((size_t)u * sizeof(uint32_t));
    if (!A || !B) { free(A); free(B); free(keys); return -1; }
    for (int64_t i = 0; i < u; i++) {
        A[i] = (uint32_t)(keys[i] >> 32);
        B[i] = (uint32_t)(keys[i] & 0xffffffffu);
    }
    free(keys);
    *out_a = A;
    *out_b = B;
    return u;
}

/*
 * One probe set x against every set of the collection (an RS-join with
 * |R| = 1, Eq. 1): the ids s with J(x, s) >= p/q, ascending.
 */
int64_t oracle_search(const int32_t *x, int64_t nx, int64_t n, const int64_t *off,
                      const int32_t *tok, int sim, int64_t p, int64_t q, int64_t **out_ids)
{
    *out_ids = NULL;
    int64_t cnt = 0, cap = 0;
    int64_t *ids = NULL;
    for (int64_t s = 0; s < n; s++) {
        int64_t ns = off[s + 1] - off[s];
        int64_t o = oracle_overlap(x, nx, tok + off[s], ns);
        if (oracle_similar_sim(sim, o, nx, ns, p, q)) {
            if (cnt == cap) {
                cap = cap ? 2 * cap : 64;
                int64_t *ni = (int64_t *)realloc(ids, (size_t)cap * sizeof(int64_t));
                if (!ni) { free(ids); return -1; }
                ids = ni;
            }
            ids[cnt++] = s;
        }
    }
    *out_ids = ids;
    return cnt;
}

/* ------------------------------------------------------------------------
 * Bitmaps (Section 3.2).  Bit k of a b-bit bitmap is word k/64, bit k%64.
 * ---------------------------------------------------------------------- */
static int get_bit(const uint64_t *w, int64_t k) { return (int)((w[k / 64] >> (k % 64)) & 1u); }
static void set_bit(uint64_t *w, int64_t k) { w[k / 64] |= (uint64_t)1 << (k % 64); }
static void flip_bit(uint64_t *w, int64_t k) { w[k / 64] ^= (uint64_t)1 << (k % 64); }

/*
 * Alg. 4 (Bitmap-Combined) picks the generation method from the threshold.
 * The paper's switch points 0.56 and 0.73 are read on the normalised overlap
 * 2*tj/(1+tj) (the scale of its Figs. 6-7), i.e. 2p/(p+q) for tj = p/q:
 *   2p/(p+q) <= 0.56 -> Next;  2p/(p+q) >= 0.73 -> Xor;  otherwise Set.
 */
int oracle_combined_method(int64_t p, int64_t q)
{
    if (2 * p * 100 <= 56 * (p + q)) return OR_NEXT;
    if (2 * p * 100 >= 73 * (p + q)) return OR_XOR;
    return OR_SET;
}

/* Alg. 4 for the other functions: the normalised overlap at the threshold of
 * two sets of equal size n is tau*n/n = p/q for Dice and Cosine; an Overlap
 * threshold counts tokens, so it keeps Xor (the paper's GPU choice). */
int oracle_combined_method_sim(int sim, int64_t p, int64_t q)
{
    if (sim == OR_JACCARD) return oracle_combined_method(p, q);
    if (sim == OR_OVERLAP) return OR_XOR;
    if (p * 100 <= 56 * q) return OR_NEXT;
    if (p * 100 >= 73 * q) return OR_XOR;
    return OR_SET;
}

/*
 * Bitmap of one set x (n tokens) with b bits, written to out[0..b/64-1].
 *   Set  (Alg. 3a): bit h(t) <- 1 for every token t.
 *   Xor  (Alg. 3b): bit h(t) <- bit h(t) xor 1 for every token t.
 *   Next (Alg. 3c): if n >= b all bits are 1; otherwise for every token,
 *                   starting at i = h(t), step i <- (i+1) mod b while bit i
 *                   is 1, then set bit i.
 * method OR_COMBINED is resolved by the caller (it needs the threshold).
 */
void oracle_bitmap(const int32_t *x, int64_t n, int b, int method, uint64_t *out)
{
    int W = b / 64;
    for (int w = 0; w < W; w++) out[w] = 0;
    if (method == OR_SET) {
        for (int64_t k = 0; k < n; k++) set_bit(out, (int64_t)x[k] % b);
    } else if (method == OR_XOR) {
        for (int64_t k = 0; k < n; k++) flip_bit(out, (int64_t)x[k] % b);
    } else if (method == OR_NEXT) {
        if (n >= b) {
            for (int w = 0; w < W; w++) out[w] = ~(uint64_t)0;
        } else {
            for (int64_t k = 0; k < n; k++) {
                int64_t i = (int64_t)x[k] % b;
                while (get_bit(out, i)) i = (i + 1) % b;
                set_bit(out, i);
            }
        }
    }
}

/* Bitmaps of a whole collection, in original set order: out[x*W + w]. */
void oracle_bitmaps(int64_t n, const int64_t *off, const int32_t *tok, int b, int method,
                    uint64_t *out)
{
    int W = b / 64;
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < n; x++)
        oracle_bitmap(tok + off[x], off[x + 1] - off[x], b, method, out + x * W);
}

static int64_t popcount64(uint64_t v)
{
    int64_t c = 0;
    while (v) { c += (int64_t)(v & 1u); v >>= 1; }
    return c;
}

/* Hamming distance popcount(br xor bs) of two b-bit bitmaps. */
int64_t oracle_hamming(const uint64_t *br, const uint64_t *bs, int b)
{
    int64_t h = 0;
    for (int w = 0; w < b / 64; w++) h += popcount64(br[w] ^ bs[w]);
    return h;
}

/* Theorem 1, Eq. 2: |r & s| <= floor((|r| + |s| - popcount(br xor bs)) / 2). */
int64_t oracle_upper_bound(int64_t nr, int64_t ns, int64_t hamming)
{
    int64_t v = nr + ns - hamming;
    /* v >= 0 always holds (hamming <= |r| + |s|); floor of a non-negative. */
    return v / 2;
}

/*
 * Counts of the GPU algorithm (Alg. 6) with verification (its host code):
 *   1. order the sets by size, ties by original id (stable);
 *   2. for sorted index i, j0 = the first sorted index whose size s satisfies
 *      q*s >= p*|R[i]| (the length filter of Table 2, integer form of
 *      |R[j]| >= tj*|R[i]|); the window is j in [j0, i);
 *   3. for every window pair: UB by Eq. 2, the pair survives the Bitmap
 *      Filter iff UB*(p+q) >= p*(|R[i]|+|R[j]|) (UB reaches the Jaccard
 *      overlap threshold of Table 1); no cutoff point (the GPU algorithm
 *      runs without it);
 *   4. a survivor is a result iff it passes oracle_similar.
 * method selects the bitmap generation (OR_COMBINED resolved from p/q).
 * cutoff > 0 is the cutoff point of Section 3.5: a pair whose larger set has
 * more than cutoff tokens skips the bound (Alg. 5) and is a survivor as it is;
 * cutoff <= 0 applies the bound to every pair (the GPU algorithm's setting).
 * Writes window pairs, survivors and results to counts[0..2].  The sort is a
 * plain insertion of (size, id) keys through qsort of packed keys.
 */
void oracle_filter_counts(int64_t n, const int64_t *off, const int32_t *tok, int sim, int64_t p,
                          int64_t q, int b, int method, int64_t cutoff, int64_t *counts)
{
    counts[0] = counts[1] = counts[2] = 0;
    if (n <= 1) return;
    if (method == OR_COMBINED) method = oracle_combined_method(p, q);
    int W = b / 64;
    uint64_t *keys = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    int64_t *ord = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *sz = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    uint64_t *bm = (uint64_t *)malloc((size_t)n * (size_t)W * sizeof(uint64_t));
    if (!keys || !ord || !sz || !bm) {
        counts[0] = counts[1] = counts[2] = -1;
        free(keys); free(ord); free(sz); free(bm);
        return;
    }
    for (int64_t x = 0; x < n; x++)
        keys[x] = ((uint64_t)(off[x + 1] - off[x]) << 32) | (uint64_t)x;
    qsort(keys, (size_t)n, sizeof(uint64_t), cmp_pair64);
    for (int64_t i = 0; i < n; i++) {
        ord[i] = (int64_t)(keys[i] & 0xffffffffu);
        sz[i] = (int64_t)(keys[i] >> 32);
        oracle_bitmap(tok + off[ord[i]], sz[i], b, method, bm + i * W);
    }
    free(keys);
    int64_t win = 0, surv = 0, res = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : win, surv, res)
    for (int64_t i = 0; i < n; i++) {
        int64_t j0 = 0;
        while (j0 < i && !oracle_in_window(sim, sz[j0], sz[i], p, q)) j0++;
        for (int64_t j = j0; j < i; j++) {
            win++;
            int64_t h = oracle_hamming(bm + i * W, bm + j * W, b);
            int64_t ub = oracle_upper_bound(sz[i], sz[j], h);
            /* the bound passes iff the similarity of an overlap of ub passes;
               sz[i] >= sz[j] is the larger size (size order) */
            int skip = cutoff > 0 && sz[i] > cutoff;
            if (skip || oracle_similar_sim(sim, ub, sz[i], sz[j], p, q)) {
                surv++;
                int64_t o = oracle_overlap(tok + off[ord[i]], sz[i], tok + off[ord[j]], sz[j]);
                if (oracle_similar_sim(sim, o, sz[i], sz[j], p, q)) res++;
            }
        }
    }
    counts[0] = win;
    counts[1] = surv;
    counts[2] = res;
    free(ord); free(sz); free(bm);
}

/*
 * Window pairs of a self-join from its size histogram alone (the count of
 * step 2 of oracle_filter_counts, Alg. 6's inner loop, without the sets):
 * hist[s] sets have size s (0 <= s < n_sizes).  Two sets of sizes t <= s form
 * a window pair iff oracle_in_window(t, s) (Table 2); sets of equal size pair
 * C(hist[s], 2) times when the size is in its own window, sets of different
 * sizes hist[t] * hist[s] times.  Returns -1 on a negative count.
 */
int64_t oracle_window_pairs_hist(const int64_t *hist, int64_t n_sizes, int sim, int64_t p,
                                 int64_t q)
{
    int64_t total = 0;
    for (int64_t s = 1; s < n_sizes; s++) {
        if (hist[s] < 0) return -1;
        if (hist[s] == 0) continue;
        if (oracle_in_window(sim, s, s, p, q)) total += hist[s] * (hist[s] - 1) / 2;
        for (int64_t t = 1; t < s; t++)
            if (hist[t] > 0 && oracle_in_window(sim, t, s, p, q)) total += hist[t] * hist[s];
    }
    return total;
}

/*
 * Window pairs of an RS-join (or of probe queries against a collection) from
 * the two size histograms: hist_r[a] sets of R and hist_s[c] sets of S have
 * sizes a and c; every pair of sizes inside the window of Table 2
 * (oracle_in_window of the smaller and the larger size) gives
 * hist_r[a] * hist_s[c] pairs.  Returns -1 on a negative count.
 */
int64_t oracle_rs_window_pairs_hist(const int64_t *hist_r, int64_t nr, const int64_t *hist_s,
                                    int64_t ns, int sim, int64_t p, int64_t q)
{
    int64_t total = 0;
    for (int64_t a = 1; a < nr; a++) {
        if (hist_r[a] < 0) return -1;
        if (hist_r[a] == 0) continue;
        for (int64_t c = 1; c < ns; c++) {
            if (hist_s[c] < 0) return -1;
            if (hist_s[c] == 0) continue;
            int64_t lo = a < c ? a : c, hi = a < c ? c : a;
            if (oracle_in_window(sim, lo, hi, p, q)) total += hist_r[a] * hist_s[c];
        }
    }
    return total;
}

/*
 * The prefix filter (Section 2.2) as a candidate generator for the Bitmap
 * Filter.  Tokens are ordered globally by frequency (rarest first, ties by
 * token id); the prefix of a set of size x is its x - low(x) + 1 first tokens
 * in that order, where low(x) is the smallest partner size inside the length
 * window (oracle_in_window), which is also the smallest overlap any similar
 * partner can have.  Two similar sets share a prefix token, so the pairs of the
 * window whose prefixes intersect (the candidates) contain every result.
 * counts[0] = candidates (pairs j < i in size order inside the window with
 * intersecting prefixes), counts[1] = candidates passing Eq. 2 with the
 * b-bit bitmaps of `method`, counts[2] = results among them.
 */
static int cmp_i64(const void *x, const void *y)
{
    int64_t u = *(const int64_t *)x, v = *(const int64_t *)y;
    return (u > v) - (u < v);
}

void oracle_prefix_counts(int64_t n, const int64_t *off, const int32_t *tok, int sim, int64_t p,
                          int64_t q, int b, int method, int64_t *counts)
{
    counts[0] = counts[1] = counts[2] = 0;
    if (n <= 1) return;
    if (method == OR_COMBINED) method = oracle_combined_method_sim(sim, p, q);
    const int64_t ntok = off[n];
    const int W = b / 64;
    /* global token order: distinct tokens with their counts, sorted by (count, token) */
    int64_t *all = (int64_t *)malloc((size_t)(ntok > 0 ? ntok : 1) * sizeof(int64_t));
    int64_t *ukey = (int64_t *)malloc((size_t)(ntok > 0 ? ntok : 1) * sizeof(int64_t));
    int64_t *utok = (int64_t *)malloc((size_t)(ntok > 0 ? ntok : 1) * sizeof(int64_t));
    int64_t *rank_of = (int64_t *)malloc((size_t)(ntok > 0 ? ntok : 1) * sizeof(int64_t));
    uint64_t *keys = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    int64_t *ord = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *sz = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *poff = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    uint64_t *bm = (uint64_t *)malloc((size_t)n * (size_t)W * sizeof(uint64_t));
    if (!all || !ukey || !utok || !rank_of || !keys || !ord || !sz || !poff || !bm) {
        counts[0] = counts[1] = counts[2] = -1;
        free(all); free(ukey); free(utok); free(rank_of); free(keys); free(ord); free(sz);
        free(poff); free(bm);
        return;
    }
    for (int64_t k = 0; k < ntok; k++) all[k] = tok[k];
    qsort(all, (size_t)ntok, sizeof(int64_t), cmp_i64);
    int64_t nu = 0;
    for (int64_t k = 0; k < ntok;) {
        int64_t e = k;
        while (e < ntok && all[e] == all[k]) e++;
        utok[nu] = all[k];                       /* ascending token ids */
        ukey[nu] = ((e - k) << 32) | nu;         /* (count, index into utok) */
        nu++;
        k = e;
    }
    qsort(ukey, (size_t)nu, sizeof(int64_t), cmp_i64);  /* by count, then token id */
    for (int64_t r = 0; r < nu; r++) rank_of[ukey[r] & 0xffffffff] = r;  /* rank per utok index */
    /* size order */
    for (int64_t x = 0; x < n; x++)
        keys[x] = ((uint64_t)(off[x + 1] - off[x]) << 32) | (uint64_t)x;
    qsort(keys, (size_t)n, sizeof(uint64_t), cmp_pair64);
    /* prefixes: the ranks of each set's tokens, sorted, first x - low(x) + 1 of them */
    poff[0] = 0;
    for (int64_t i = 0; i < n; i++) {
        ord[i] = (int64_t)(keys[i] & 0xffffffffu);
        sz[i] = (int64_t)(keys[i] >> 32);
        int64_t low = 1;
        while (low <= sz[i] && !oracle_in_window(sim, low, sz[i], p, q)) low++;
        int64_t len = sz[i] - low + 1;
        if (len < 0) len = 0;
        poff[i + 1] = poff[i] + len;
        oracle_bitmap(tok + off[ord[i]], sz[i], b, method, bm + i * W);
    }
    int64_t *pre = (int64_t *)malloc((size_t)(poff[n] > 0 ? poff[n] : 1) * sizeof(int64_t));
    int64_t *tmp = (int64_t *)malloc((size_t)(ntok > 0 ? ntok : 1) * sizeof(int64_t));
    if (!pre || !tmp) {
        counts[0] = counts[1] = counts[2] = -1;
    } else {
        for (int64_t i = 0; i < n; i++) {
            const int32_t *x = tok + off[ord[i]];
            for (int64_t k = 0; k < sz[i]; k++) {
                /* rank of token x[k]: binary search in the ascending distinct tokens */
                int64_t lo = 0, hi = nu - 1;
                while (lo < hi) {
                    int64_t mid = (lo + hi) / 2;
                    if (utok[mid] < x[k]) lo = mid + 1; else hi = mid;
                }
                tmp[k] = rank_of[lo];
            }
            qsort(tmp, (size_t)sz[i], sizeof(int64_t), cmp_i64);
            for (int64_t k = 0; k < poff[i + 1] - poff[i]; k++) pre[poff[i] + k] = tmp[k];
        }
        int64_t cand = 0, surv = 0, res = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : cand, surv, res)
        for (int64_t i = 0; i < n; i++) {
            for (int64_t j = 0; j < i; j++) {
                if (!oracle_in_window(sim, sz[j], sz[i], p, q)) continue;
                /* do the two sorted prefixes share a rank? */
                int64_t a = poff[i], ae = poff[i + 1], c = poff[j], ce = poff[j + 1];
                int share = 0;
                while (a < ae && c < ce) {
                    if (pre[a] == pre[c]) { share = 1; break; }
                    if (pre[a] < pre[c]) a++; else c++;
                }
                if (!share) continue;
                cand++;
                int64_t h = oracle_hamming(bm + i * W, bm + j * W, b);
                if (!oracle_similar_sim(sim, oracle_upper_bound(sz[i], sz[j], h), sz[i], sz[j], p, q))
                    continue;
                surv++;
                int64_t o = oracle_overlap(tok + off[ord[i]], sz[i], tok + off[ord[j]], sz[j]);
                if (oracle_similar_sim(sim, o, sz[i], sz[j], p, q)) res++;
            }
        }
        counts[0] = cand;
        counts[1] = surv;
        counts[2] = res;
    }
    free(pre); free(tmp);
    free(all); free(ukey); free(utok); free(rank_of); free(keys); free(ord); free(sz); free(poff);
    free(bm);
}

/*
 * RS-join (Section 2.1, Eq. 1 with R and S two collections): every pair
 * (r, s) of R x S is verified; the output is every similar pair as (r, s)
 * with r an id of R and s an id of S, in (r, s) order.  Rows of R are spread
 * over threads and concatenated in row order.  Returns the pair count, or -1
 * on allocation failure (*out_a / *out_b as for oracle_self_join).
 */
int64_t oracle_rs_join(int64_t nr, const int64_t *offr, const int32_t *tokr, int64_t ns,
                       const int64_t *offs, const int32_t *toks, int sim, int64_t p, int64_t q,
                       uint32_t **out_a, uint32_t **out_b)
{
    *out_a = NULL;
    *out_b = NULL;
    if (nr <= 0 || ns <= 0) return 0;
    pairbuf *rows = (pairbuf *)calloc((size_t)nr, sizeof(pairbuf));
    if (!rows) return -1;
    int failed = 0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < nr; r++) {
        const int32_t *xr = tokr + offr[r];
        int64_t lr = offr[r + 1] - offr[r];
        for (int64_t t = 0; t < ns; t++) {
            int64_t lt = offs[t + 1] - offs[t];
            int64_t o = oracle_overlap(xr, lr, toks + offs[t], lt);
            if (oracle_similar_sim(sim, o, lr, lt, p, q))
                if (pb_push(&rows[r], (uint32_t)r, (uint32_t)t)) failed = 1;
        }
    }
    int64_t total = 0;
    for (int64_t r = 0; r < nr; r++) total += rows[r].n;
    uint32_t *A = NULL, *B = NULL;
    if (!failed && total > 0) {
        A = (uint32_t *)malloc((size_t)total * sizeof(uint32_t));
        B = (uint32_t *)malloc((size_t)total * sizeof(uint32_t));
        if (!A || !B) failed = 1;
    }
    int64_t k = 0;
    for (int64_t r = 0; r < nr; r++) {
        if (!failed && rows[r].n) {
            memcpy(A + k, rows[r].a, (size_t)rows[r].n * sizeof(uint32_t));
            memcpy(B + k, rows[r].b, (size_t)rows[r].n * sizeof(uint32_t));
            k += rows[r].n;
        }
        free(rows[r].a);
        free(rows[r].b);
    }
    free(rows);
    if (failed) { free(A); free(B); return -1; }
    *out_a = A;
    *out_b = B;
    return total;
}

/*
 * Counts of an RS-join run as the GPU algorithm runs a self-join: a pair
 * (r, s) is in the window when its sizes, smaller first, pass the length
 * filter of Table 2; a window pair survives the Bitmap Filter when the Eq. 2
 * bound of its bitmaps passes the similarity test, and a survivor is a result
 * when its exact overlap does.  Every pair of R x S is looked at, so no order
 * of the sets is involved.  cutoff as for oracle_filter_counts (on the larger
 * of the two sizes).  Writes window pairs, survivors and results to
 * counts[0..2] (-1 on allocation failure).
 */
void oracle_rs_filter_counts(int64_t nr, const int64_t *offr, const int32_t *tokr, int64_t ns,
                             const int64_t *offs, const int32_t *toks, int sim, int64_t p,
                             int64_t q, int b, int method, int64_t cutoff, int64_t *counts)
{
    counts[0] = counts[1] = counts[2] = 0;
    if (nr <= 0 || ns <= 0) return;
    if (method == OR_COMBINED) method = oracle_combined_method_sim(sim, p, q);
    int W = b / 64;
    uint64_t *bmr = (uint64_t *)malloc((size_t)nr * (size_t)W * sizeof(uint64_t));
    uint64_t *bms = (uint64_t *)malloc((size_t)ns * (size_t)W * sizeof(uint64_t));
    if (!bmr || !bms) {
        counts[0] = counts[1] = counts[2] = -1;
        free(bmr); free(bms);
        return;
    }
    oracle_bitmaps(nr, offr, tokr, b, method, bmr);
    oracle_bitmaps(ns, offs, toks, b, method, bms);
    int64_t win = 0, surv = 0, res = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : win, surv, res)
    for (int64_t r = 0; r < nr; r++) {
        int64_t lr = offr[r + 1] - offr[r];
        for (int64_t t = 0; t < ns; t++) {
            int64_t lt = offs[t + 1] - offs[t];
            int64_t mn = lr < lt ? lr : lt, mx = lr < lt ? lt : lr;
            if (!oracle_in_window(sim, mn, mx, p, q)) continue;
            win++;
            int64_t h = oracle_hamming(bmr + r * W, bms + t * W, b);
            int skip = cutoff > 0 && mx > cutoff;
            if (!skip && !oracle_similar_sim(sim, oracle_upper_bound(lr, lt, h), lr, lt, p, q))
                continue;
            surv++;
            int64_t o = oracle_overlap(tokr + offr[r], lr, toks + offs[t], lt);
            if (oracle_similar_sim(sim, o, lr, lt, p, q)) res++;
        }
    }
    counts[0] = win;
    counts[1] = surv;
    counts[2] = res;
    free(bmr); free(bms);
}

/*
 * The prefix filter (Section 2.2) for an RS-join: tokens are ranked by their
 * frequency over R and S together (rarest first, ties by token id); every set
 * of R and of S keeps its x - low(x) + 1 lowest-ranked tokens as its prefix,
 * low(x) being the smallest partner size inside the length window (the
 * smallest overlap a similar partner can have, whichever collection it is
 * in).  A pair (r, s) of the window is a candidate when the two prefixes share
 * a rank.  counts[0] = candidates, counts[1] = candidates passing Eq. 2 with
 * the b-bit bitmaps of `method`, counts[2] = results among them (-1 on
 * allocation failure).
 */
void oracle_rs_prefix_counts(int64_t nr, const int64_t *offr, const int32_t *tokr, int64_t ns,
                             const int64_t *offs, const int32_t *toks, int sim, int64_t p,
                             int64_t q, int b, int method, int64_t *counts)
{
    counts[0] = counts[1] = counts[2] = 0;
    if (nr <= 0 || ns <= 0) return;
    if (method == OR_COMBINED) method = oracle_combined_method_sim(sim, p, q);
    const int64_t n = nr + ns, tr = offr[nr], ntok = offr[nr] + offs[ns];
    const int W = b / 64;
    /* R and S as one list of sets: set x < nr is r_x, set nr + y is s_y */
    int64_t *off = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    int32_t *tok = (int32_t *)malloc((size_t)(ntok > 0 ? ntok : 1) * sizeof(int32_t));
    int64_t *all = (int64_t *)malloc((size_t)(ntok > 0 ? ntok : 1) * sizeof(int64_t));
    int64_t *ukey = (int64_t *)malloc((size_t)(ntok > 0 ? ntok : 1) * sizeof(int64_t));
    int64_t *utok = (int64_t *)malloc((size_t)(ntok > 0 ? ntok : 1) * sizeof(int64_t));
    int64_t *rank_of = (int64_t *)malloc((size_t)(ntok > 0 ? ntok : 1) * sizeof(int64_t));
    int64_t *poff = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    int64_t *tmp = (int64_t *)malloc((size_t)(ntok > 0 ? ntok : 1) * sizeof(int64_t));
    uint64_t *bm = (uint64_t *)malloc((size_t)n * (size_t)W * sizeof(uint64_t));
    int64_t *pre = NULL;
    int64_t nu = 0;
    if (off && tok && all && ukey && utok && rank_of && poff && tmp && bm) {
        for (int64_t x = 0; x <= nr; x++) off[x] = offr[x];
        for (int64_t y = 1; y <= ns; y++) off[nr + y] = tr + offs[y];
        memcpy(tok, tokr, (size_t)tr * sizeof(int32_t));
        memcpy(tok + tr, toks, (size_t)offs[ns] * sizeof(int32_t));
        /* global token order: distinct tokens with their counts, sorted by (count, token) */
        for (int64_t k = 0; k < ntok; k++) all[k] = tok[k];
        qsort(all, (size_t)ntok, sizeof(int64_t), cmp_i64);
        for (int64_t k = 0; k < ntok;) {
            int64_t e = k;
            while (e < ntok && all[e] == all[k]) e++;
            utok[nu] = all[k];                   /* ascending token ids */
            ukey[nu] = ((e - k) << 32) | nu;     /* (count, index into utok) */
            nu++;
            k = e;
        }
        qsort(ukey, (size_t)nu, sizeof(int64_t), cmp_i64);
        for (int64_t r = 0; r < nu; r++) rank_of[ukey[r] & 0xffffffff] = r;
        /* prefix lengths x - low(x) + 1 and the bitmaps */
        poff[0] = 0;
        for (int64_t x = 0; x < n; x++) {
            const int64_t sx = off[x + 1] - off[x];
            int64_t low = 1;
            while (low <= sx && !oracle_in_window(sim, low, sx, p, q)) low++;
            poff[x + 1] = poff[x] + (sx - low + 1 > 0 ? sx - low + 1 : 0);
            oracle_bitmap(tok + off[x], sx, b, method, bm + x * W);
        }
        pre = (int64_t *)malloc((size_t)(poff[n] > 0 ? poff[n] : 1) * sizeof(int64_t));
    }
    if (!pre) {
        counts[0] = counts[1] = counts[2] = -1;
    } else {
        /* each set's prefix: the ranks of its tokens, sorted, first poff[x+1]-poff[x] */
        for (int64_t x = 0; x < n; x++) {
            const int64_t sx = off[x + 1] - off[x];
            for (int64_t k = 0; k < sx; k++) {
                int64_t lo = 0, hi = nu - 1;   /* the token among the ascending distinct ones */
                while (lo < hi) {
                    int64_t mid = (lo + hi) / 2;
                    if (utok[mid] < tok[off[x] + k]) lo = mid + 1; else hi = mid;
                }
                tmp[k] = rank_of[lo];
            }
            qsort(tmp, (size_t)sx, sizeof(int64_t), cmp_i64);
            for (int64_t k = 0; k < poff[x + 1] - poff[x]; k++) pre[poff[x] + k] = tmp[k];
        }
        int64_t cand = 0, surv = 0, res = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : cand, surv, res)
        for (int64_t r = 0; r < nr; r++) {
            const int64_t lr = off[r + 1] - off[r];
            for (int64_t y = 0; y < ns; y++) {
                const int64_t t = nr + y, lt = off[t + 1] - off[t];
                const int64_t mn = lr < lt ? lr : lt, mx = lr < lt ? lt : lr;
                if (!oracle_in_window(sim, mn, mx, p, q)) continue;
                /* do the two sorted prefixes share a rank? */
                int64_t a = poff[r], ae = poff[r + 1], c = poff[t], ce = poff[t + 1];
                int share = 0;
                while (a < ae && c < ce) {
                    if (pre[a] == pre[c]) { share = 1; break; }
                    if (pre[a] < pre[c]) a++; else c++;
                }
                if (!share) continue;
                cand++;
                int64_t h = oracle_hamming(bm + r * W, bm + t * W, b);
                if (!oracle_similar_sim(sim, oracle_upper_bound(lr, lt, h), lr, lt, p, q)) continue;
                surv++;
                int64_t o = oracle_overlap(tok + off[r], lr, tok + off[t], lt);
                if (oracle_similar_sim(sim, o, lr, lt, p, q)) res++;
            }
        }
        counts[0] = cand;
        counts[1] = surv;
        counts[2] = res;
    }
    free(off); free(tok); free(all); free(ukey); free(utok); free(rank_of); free(poff); free(tmp);
    free(bm); free(pre);
}
