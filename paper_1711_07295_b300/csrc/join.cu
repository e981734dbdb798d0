// join.cu -- host orchestration of the self-join and the C ABI entry points.
//
// bmj_self_join runs the stages of the GPU algorithm (Alg. 6) on one stream:
//   validate -> size sort -> sorted CSR + bitmaps -> window tiles ->
//   Bitmap Filter -> exact verification -> canonical result sort -> output.
// bmj_rs_join runs the same stages on R and S held in one size-sorted array
// (S first): the rows are R's sets, the columns S's inside each row's window.
// The host reads back three small counters (validation flags and maximum
// size; survivor count; result count), which size the next allocations.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "kernels.cuh"
#include "host_util.cuh"
#include "prefix.cuh"

namespace bmj {

// Time of one prefix-candidate slot (expansion, Eq. 2, its share of the
// verification) in window pairs of the Bitmap Filter at W words, measured on a
// B300: about 35 ps per slot against 0.42, 0.65 and 1.15 ps per window pair at
// b = 64, 128, 256 (BMJ_CAND_AUTO takes the prefix filter when
// slots x this < window pairs).
static double slot_cost_in_pairs(int W) {
    return W == 1 ? 80.0 : W == 2 ? 55.0 : W == 4 ? 30.0 : 80.0 / W;
}

static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t launches() { return g_launches.load(std::memory_order_relaxed); }

static std::atomic<int> g_alloc_fault{0};

FaultPlan read_fault_plan() {
    FaultPlan f;
    const char *e = getenv("BMJ_FAULT");
    if (!e) return f;
    if (strncmp(e, "alloc:", 6) == 0) f.alloc_at = atoi(e + 6);
    if (strcmp(e, "timeout") == 0) f.timeout = true;
    if (strcmp(e, "keys") == 0) f.keys = true;
    if (strcmp(e, "serve") == 0) f.serve = true;
    return f;
}

void arm_alloc_fault(int k) { g_alloc_fault.store(k > 0 ? k : 0); }

bool alloc_fault_fires() {
    int v = g_alloc_fault.load();
    while (v > 0) {
        if (g_alloc_fault.compare_exchange_weak(v, v - 1)) return v == 1;
    }
    return false;
}

void retain_pool_memory(int device) {
    static std::mutex mu;
    static bool done[128] = {false};
    std::lock_guard<std::mutex> lk(mu);
    if (device < 0 || device >= 128 || done[device]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    done[device] = true;
}

static int64_t auto_queue_cap(int64_t window) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        free_b = (size_t)8 << 30;
    }
    int64_t budget = (int64_t)(free_b / 4 / sizeof(uint2));
    int64_t cap = window / 128;
    if (cap < ((int64_t)1 << 20)) cap = (int64_t)1 << 20;
    if (cap > budget) cap = budget;
    if (cap > ((int64_t)1 << 32)) cap = (int64_t)1 << 32;
    if (cap < 1) cap = 1;
    return cap;
}

// coll_s == nullptr: the self-join of coll; else the RS-join of R = coll and
// S = coll_s.
static int self_join_impl(const bmj_collection *coll, const bmj_collection *coll_s, int sim,
                          uint32_t p, uint32_t q, const bmj_options &o, bmj_pairs *out,
                          bmj_stats *stats) {
    NvtxRange nv_call(coll_s ? "bmj_rs_join" : "bmj_self_join");
    cudaStream_t s = (cudaStream_t)o.stream;
    const int64_t launches0 = launches();
    const FaultPlan fault = read_fault_plan();
    arm_alloc_fault(fault.alloc_at);
    int dev = 0;
    BMJ_CHECK(cudaGetDevice(&dev));
    retain_pool_memory(dev);
    const int sms = num_sms(dev);
    bmj_stats stl;
    memset(&stl, 0, sizeof(stl));
    const int b = o.b;
    const int W = b / 64;
    int method = o.method == BMJ_COMBINED ? combined_method(sim, p, q) : o.method;
    stl.b = b;
    stl.method = method;
    // cutoff point (Section 3.5): pairs whose larger set exceeds it skip Eq. 2
    uint32_t cut = 0xffffffffu;
    if (o.cutoff > 0) cut = (uint32_t)o.cutoff;
    else if (o.cutoff == BMJ_CUTOFF_AUTO) {
        const int64_t w = cutoff_point(b, method, sim, p, q);
        if (w > 0) cut = (uint32_t)w;
    }
    stl.cutoff = cut == 0xffffffffu ? 0 : (int32_t)cut;

    Events ev;
    int st = ev.init();
    if (st) return st;
    Arena A(s);
    BMJ_CHECK(cudaEventRecord(ev.e[0], s));
    DevColl d;
    const bool rs = coll_s != nullptr;
    st = rs ? stage_two(coll, coll_s, A, s, &d) : stage_collection(coll, A, s, &d);
    if (st) return st;
    const int64_t n = d.n;
    // RS-join: R's sets are ids [0, n_r) of the staged collection and sort after
    // S's, which fill size-order positions [0, n_sc)
    const int64_t n_r = rs ? coll->n_sets : 0, n_sc = rs ? coll_s->n_sets : 0;

    uint32_t *sizes = nullptr, *ids = nullptr;
    int max_size = 0;
    if (n > 0) {
        st = validate(d, o.validate != 0, A, s, &sizes, &ids, &max_size);
        if (st) return st;
    }
    stl.max_set_size = max_size;

    uint64_t *keys_sorted = nullptr;
    int64_t n_res = 0;
    const int nbits = n > 1 ? bit_length((uint64_t)(n - 1)) : 1;
    BMJ_CHECK(cudaEventRecord(ev.e[1], s));
    if (rs ? (n_r > 0 && n_sc > 0) : n >= 2) {
        // ---- size sort (ties by original id) and sorted CSR + bitmaps ----
        uint32_t *ssz = nullptr, *perm = nullptr;
        int64_t *soff = nullptr;
        int32_t *stok = nullptr;
        uint64_t *bm = nullptr;
        st = A.alloc(&ssz, (size_t)n + 4);
        if (!st) st = A.alloc(&perm, (size_t)n);
        if (!st) st = A.alloc(&soff, (size_t)n);
        if (!st) st = A.alloc(&stok, (size_t)d.ntok);
        if (!st) st = A.alloc(&bm, (size_t)(n + 4) * W);  // padded: TMA chunks may read 3 past the end
        if (st) return st;
        // Second, wider bitmaps for the cascade check in verification.
        const int b2 = o.cascade_b == 0 ? (b < 256 ? 256 : 0) : (o.cascade_b > b ? o.cascade_b : 0);
        const int W2 = b2 / 64;
        uint64_t *bm2 = nullptr;
        if (b2) {
            st = A.alloc(&bm2, (size_t)n * W2);
            if (st) return st;
        }
        stl.cascade_b = b2;
        const int sbits = bit_length((uint64_t)max_size);
        if (rs) st = launch_or_bits(sizes, n_r, 1u << sbits, s);  // R after S
        if (!st) st = radix_sort_u32_pairs(sizes, ids, ssz, perm, n, sbits + (rs ? 1 : 0), A, s);
        if (!st && rs) st = launch_and_bits(ssz, n, (1u << sbits) - 1u, s);
        if (st) return st;
        st = launch_widen(ssz, soff, n, s);
        if (!st) st = exclusive_scan_i64(soff, soff, n, nullptr, A, s);
        if (!st) {
            const bool multi = (method == BMJ_XOR || method == BMJ_SET) &&
                               (b == 64 || b == 128 || b == 256) && (b2 == 0 || b2 == 256);
            if (multi) {  // one pass over the tokens for both widths
                st = launch_build_multi(perm, d.off, d.tok, soff, stok, n, method,
                                        b == 64 ? bm : nullptr, b == 128 ? bm : nullptr,
                                        b == 256 ? bm : (b2 == 256 ? bm2 : nullptr), s);
            } else {
                st = launch_gather_build(perm, d.off, d.tok, soff, stok, bm, n, b, method, s);
                if (!st && b2)
                    st = launch_gather_build(perm, d.off, d.tok, nullptr, nullptr, bm2, n, b2,
                                             method, s);
            }
        }
        if (st) return st;

        // ---- thresholds per |x|+|y|, window tiles, window size ----
        const int64_t n_s = 2 * (int64_t)max_size + 1;
        const SimWindow win = sim_window(sim, p, q);
        int32_t *need = nullptr, *lim = nullptr;
        const int tile_rows = filter_tma_tile_rows(W);
        const int chunk_cols = W <= 4 ? 4096 : 2048;
        stl.tile_rows = tile_rows;
        stl.chunk_cols = chunk_cols;
        // rows joined: size-order positions [r0, r1) (all rows unless a band is given)
        const int64_t r0 = rs ? n_sc : (o.row_begin == 0 && o.row_end == 0) ? 0 : o.row_begin;
        const int64_t r1 = rs ? n : (o.row_begin == 0 && o.row_end == 0) ? n : o.row_end;
        if (r0 < 0 || r1 < r0 || r1 > n) return BMJ_ERR_INVALID_ARG;
        const int64_t n_tiles = (r1 - r0 + tile_rows - 1) / tile_rows;
        int32_t *tile_c0 = nullptr, *tile_c1 = nullptr;
        int64_t *tile_off = nullptr;
        // [0] window, [1] queue count, [2] item counter, [3] results, [4] verified,
        // [5] first-level survivors (cascade), [6] [7] the filter's folded-test column
        // steps and those of them that took the full test (b = 128)
        unsigned long long *ctr = nullptr;
        int *err = nullptr;
        st = A.alloc(&need, (size_t)n_s);
        if (!st) st = A.alloc(&lim, (size_t)n_s);
        if (!st) st = A.alloc(&tile_c0, (size_t)(n_tiles > 0 ? n_tiles : 1));
        if (!st) st = A.alloc(&tile_off, (size_t)n_tiles + 1);
        if (!st && rs) st = A.alloc(&tile_c1, (size_t)(n_tiles > 0 ? n_tiles : 1));
        if (!st) st = A.alloc(&ctr, 8);
        if (!st) st = A.alloc(&err, 1);
        if (st) return st;
        BMJ_CHECK(cudaMemsetAsync(ctr, 0, 8 * sizeof(unsigned long long), s));
        BMJ_CHECK(cudaMemsetAsync(err, 0, sizeof(int), s));
        BMJ_CHECK(cudaMemsetAsync(ssz + n, 0, 4 * sizeof(uint32_t), s));
        BMJ_CHECK(cudaMemsetAsync(bm + (size_t)n * W, 0, 4 * W * sizeof(uint64_t), s));
        st = launch_tables(need, lim, n_s, sim, p, q, s);
        if (!st && rs)
            st = launch_rs_tiles(ssz, n_sc, win, tile_rows, chunk_cols, n_tiles, tile_c0, tile_c1,
                                 tile_off, r0, r1, s);
        else if (!st)
            st = launch_tiles(ssz, n, win, tile_rows, chunk_cols, n_tiles, tile_c0, tile_off, s, r0,
                              r1);
        if (!st) st = exclusive_scan_i64(tile_off, tile_off, n_tiles, tile_off + n_tiles, A, s);
        if (!st && rs) st = launch_rs_window_count(ssz, n_sc, win, &ctr[0], r0, r1, s);
        else if (!st) st = launch_window_count(ssz, n, win, &ctr[0], s, r0, r1);
        if (st) return st;
        BMJ_CHECK(cudaEventRecord(ev.e[2], s));
        int64_t hv[2] = {0, 0};
        BMJ_CHECK(cudaMemcpyAsync(&hv[0], ctr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        BMJ_CHECK(cudaMemcpyAsync(&hv[1], tile_off + n_tiles, sizeof(int64_t),
                                  cudaMemcpyDeviceToHost, s));
        BMJ_CHECK(cudaStreamSynchronize(s));
        stl.window_pairs = hv[0];
        const int64_t n_items = hv[1];

        uint64_t *keys = nullptr;
        int64_t res_cap = 0;
        // Appends r result keys from src to the growing result buffer.
        auto append = [&](const uint64_t *src, int64_t r) -> int {
            if (n_res + r > res_cap) {
                const int64_t ncap = std::max(2 * res_cap, n_res + r);
                uint64_t *grown = nullptr;
                int rc = A.alloc(&grown, (size_t)ncap);
                if (rc) return rc;
                if (n_res)
                    BMJ_CHECK(cudaMemcpyAsync(grown, keys, n_res * sizeof(uint64_t),
                                              cudaMemcpyDeviceToDevice, s));
                if (keys) A.free_one(keys);
                keys = grown;
                res_cap = ncap;
            }
            if (r)
                BMJ_CHECK(cudaMemcpyAsync(keys + n_res, src, r * sizeof(uint64_t),
                                          cudaMemcpyDeviceToDevice, s));
            n_res += r;
            return BMJ_OK;
        };

        // ---- candidates from the prefix filter (Section 2.2), if asked for ----
        // The index of every prefix is built once; its candidate slots are then
        // expanded a range at a time into a buffer of fixed size (a quarter of the
        // free memory, or opt.queue_cap slots), and each range's candidates pass
        // Eq. 2 with the join's bitmaps and the merge before the next range.
        bool done = false;
        if (o.candidates == BMJ_CAND_PREFIX || o.candidates == BMJ_CAND_AUTO) {
            Arena PA(s);  // its buffers go once the candidates are verified
            BMJ_CHECK(cudaEventRecord(ev.e[3], s));
            PrefixIndex px;
            nvtxRangePushA("bmj.prefix_index");
            int pst = prefix_index(ssz, soff, stok, n, d.ntok, rs ? n_sc : 0, win, PA, s, &px);
            nvtxRangePop();
            if (pst == BMJ_ERR_OOM) {  // the index itself does not fit: the window instead
                cudaGetLastError();
                PA.release();
                stl.candidates = -1;
            } else if (pst) {
                return pst;
            } else if (o.candidates == BMJ_CAND_AUTO &&
                       (double)px.slots * slot_cost_in_pairs(W) >= (double)stl.window_pairs) {
                // the whole window is cheaper than expanding this many slots
                PA.release();
                stl.candidates = -2;
                stl.candidate_slots = px.slots;
            } else {
                float ms_index = 0.f;
                BMJ_CHECK(cudaEventRecord(ev.e[4], s));
                BMJ_CHECK(cudaEventSynchronize(ev.e[4]));
                ms_index = ev.ms(3, 4);
                size_t free_b = 0, total_b = 0;
                if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = (size_t)8 << 30;
                cudaGetLastError();
                // a range's slots need 8 bytes of candidates and 8 of result keys each
                int64_t chunk = o.queue_cap > 0 ? o.queue_cap
                                                : std::max<int64_t>((int64_t)1 << 20,
                                                                    (int64_t)(free_b / 4 / 16));
                chunk = std::max<int64_t>(1, std::min(chunk, px.slots));
                uint2 *cq = nullptr;
                uint64_t *ckeys = nullptr;
                unsigned long long *ccnt = nullptr;
                st = PA.alloc(&cq, (size_t)chunk);
                if (!st) st = PA.alloc(&ckeys, (size_t)chunk);
                if (!st) st = PA.alloc(&ccnt, 2);  // [0] passed Eq. 2, [1] candidates
                if (st) return st;
                // The Bitmap Filter runs inside the expansion (only survivors are written)
                // where the limit depends on |x|+|y| alone and b is 64, 128 or 256; the
                // survivors then take the cascade check and the merge of the window path.
                // Otherwise every candidate is written and verification applies Eq. 2.
                PrefixTest test;
                const bool fused = sim != BMJ_COSINE && (W == 1 || W == 2 || W == 4);
                if (fused) {
                    test.bm = bm;
                    test.lim = lim;
                    test.W = W;
                }
                st = prefix_records(px, test, PA, s);
                if (st) return st;
                stl.candidates = 0;
                stl.survivors = 0;
                stl.verified = 0;
                stl.filter_passes = 0;
                float ms_expand = 0.f;
                for (int64_t o0 = 0; o0 < px.slots; o0 += chunk) {
                    const int64_t o1 = std::min(px.slots, o0 + chunk);
                    BMJ_CHECK(cudaMemsetAsync(ccnt, 0, 2 * sizeof(unsigned long long), s));
                    BMJ_CHECK(cudaMemsetAsync(&ctr[3], 0, 2 * sizeof(unsigned long long), s));
                    BMJ_CHECK(cudaEventRecord(ev.e[3], s));
                    NvtxRange nv_range("bmj.prefix_range");
                    st = prefix_expand(px, o0, o1, test, cq, &ccnt[0], &ccnt[1], s);
                    if (st) return st;
                    BMJ_CHECK(cudaEventRecord(ev.e[4], s));
                    int64_t hc[2] = {0, 0};  // written pairs, candidates
                    BMJ_CHECK(cudaMemcpyAsync(hc, ccnt, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
                    BMJ_CHECK(cudaStreamSynchronize(s));
                    ms_expand += ev.ms(3, 4);
                    stl.candidates += hc[1];
                    stl.filter_passes++;
                    if (fused) stl.survivors += hc[0];
                    if (hc[0] == 0) continue;
                    // fused: the cascade check (if any) and the merge on the survivors;
                    // otherwise Eq. 2 with the join's bitmaps on every candidate, then the merge
                    BMJ_CHECK(cudaEventRecord(ev.e[5], s));
                    st = fused ? launch_verify(cq, hc[0], soff, stok, ssz, perm, need, lim, bm2, W2,
                                               ckeys, &ctr[3], bm2 ? &ctr[4] : nullptr, nbits, sms,
                                               s, sim, p, q)
                               : launch_verify(cq, hc[0], soff, stok, ssz, perm, need, lim, bm, W,
                                               ckeys, &ctr[3], &ctr[4], nbits, sms, s, sim, p, q);
                    if (st) return st;
                    BMJ_CHECK(cudaEventRecord(ev.e[6], s));
                    int64_t hv2[2] = {0, 0};
                    BMJ_CHECK(cudaMemcpyAsync(hv2, &ctr[3], 2 * sizeof(int64_t),
                                              cudaMemcpyDeviceToHost, s));
                    BMJ_CHECK(cudaStreamSynchronize(s));
                    if (fused) {
                        stl.verified += bm2 ? hv2[1] : hc[0];
                    } else {
                        stl.survivors += hv2[1];
                        stl.verified += hv2[1];
                    }
                    stl.ms_verify += ev.ms(5, 6);
                    st = append(ckeys, hv2[0]);
                    if (st) return st;
                }
                stl.candidate_slots = px.slots;
                stl.ms_filter = ms_index + ms_expand;
                done = true;
            }
        }
        if (!done) {
            // ---- Bitmap Filter + exact verification ----
            // The filter's queue counts every survivor, also past its capacity.  When
            // the first pass over all work items overflows, the filter reruns with
            // exact room if that fits (automatic capacity), else the items run in
            // consecutive ranges whose survivors fit the queue, each verified before
            // the next; no pair is ever dropped.
            const bool user_cap = o.queue_cap > 0;
            int64_t qcap = user_cap ? o.queue_cap : auto_queue_cap(stl.window_pairs);
            uint2 *queue = nullptr;
            st = A.alloc(&queue, (size_t)qcap);
            if (st == BMJ_ERR_OOM && user_cap) {  // a requested capacity that does not fit: the
                cudaGetLastError();                // automatic one, drained in item ranges
                qcap = std::min(qcap, auto_queue_cap(stl.window_pairs));
                st = A.alloc(&queue, (size_t)qcap);
            }
            if (st) return st;
            FilterArgs fa;
            fa.bm = bm;
            fa.ssz = ssz;
            fa.lim = lim;
            fa.n = n;
            fa.row0 = r0;
            fa.row_end = r1;
            fa.p = p;
            fa.sim = sim;
            fa.q = q;
            fa.tile_item_off = tile_off;
            fa.tile_c0 = tile_c0;
            fa.tile_c1 = tile_c1;
            fa.cut = cut;
            fa.n_tiles = n_tiles;
            fa.n_items = n_items;
            fa.tile_rows = tile_rows;
            fa.chunk_cols = chunk_cols;
            fa.queue = queue;
            fa.qcount = &ctr[1];
            fa.qcap = qcap;
            fa.item_counter = &ctr[2];
            fa.steps = &ctr[6];
            if (fault.timeout) {
                fa.fault_skip_copy = 1;
                fa.wait_limit = 1 << 12;
            }
            // Filters work items [lo, hi) into the queue; *count = their survivors.  The
            // folded-test step counts are taken from the first pass (every item once).
            int64_t fold_steps[2] = {0, 0};
            bool fold_read = false;
            auto run_filter = [&](int64_t lo, int64_t hi, int64_t *count) -> int {
                NvtxRange nv("bmj.filter");
                const unsigned long long init[2] = {0ull, (unsigned long long)lo};
                BMJ_CHECK(cudaMemcpyAsync(&ctr[1], init, sizeof(init), cudaMemcpyHostToDevice, s));
                fa.n_items = hi;
                BMJ_CHECK(cudaEventRecord(ev.e[3], s));
                int rc = launch_filter_tma(fa, W, err, sms, s);
                if (rc) return rc;
                BMJ_CHECK(cudaEventRecord(ev.e[4], s));
                int herr = 0;
                BMJ_CHECK(cudaMemcpyAsync(count, &ctr[1], sizeof(int64_t), cudaMemcpyDeviceToHost, s));
                BMJ_CHECK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
                const bool read_steps = !fold_read && (W == 2 || W == 4);
                if (read_steps)
                    BMJ_CHECK(cudaMemcpyAsync(fold_steps, &ctr[6], 2 * sizeof(int64_t),
                                              cudaMemcpyDeviceToHost, s));
                BMJ_CHECK(cudaStreamSynchronize(s));
                if (herr) return BMJ_ERR_TIMEOUT;
                if (read_steps) {
                    fold_read = true;
                    stl.fold_steps = fold_steps[0];
                    stl.fold_full_steps = fold_steps[1];
                }
                stl.filter_passes++;
                stl.ms_filter += ev.ms(3, 4);
                return BMJ_OK;
            };
            // Verifies the m survivors at qptr into out_keys (*n_out results).
            auto run_verify = [&](const uint2 *qptr, int64_t m, uint64_t *out_keys,
                                  int64_t *n_out) -> int {
                NvtxRange nv("bmj.verify");
                BMJ_CHECK(cudaMemsetAsync(&ctr[3], 0, 2 * sizeof(unsigned long long), s));
                BMJ_CHECK(cudaEventRecord(ev.e[5], s));
                int rc = launch_verify(qptr, m, soff, stok, ssz, perm, need, lim, bm2, W2, out_keys,
                                       &ctr[3], bm2 ? &ctr[4] : nullptr, nbits, sms, s, sim, p, q);
                if (rc) return rc;
                BMJ_CHECK(cudaEventRecord(ev.e[6], s));
                int64_t hv2[2] = {0, 0};
                BMJ_CHECK(cudaMemcpyAsync(hv2, &ctr[3], 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
                BMJ_CHECK(cudaStreamSynchronize(s));
                *n_out = hv2[0];
                stl.verified += bm2 ? hv2[1] : m;
                stl.ms_verify += ev.ms(5, 6);
                return BMJ_OK;
            };

            int64_t n_surv = 0;
            st = run_filter(0, n_items, &n_surv);
            if (st) return st;
            stl.survivors = n_surv;
            bool banded = false;
            if (n_surv > qcap) {
                uint2 *exact = nullptr;
                if (!user_cap && A.alloc(&exact, (size_t)n_surv) == BMJ_OK) {
                    A.free_one(queue);
                    queue = exact;
                    qcap = n_surv;
                    fa.queue = queue;
                    fa.qcap = qcap;
                    int64_t again = 0;
                    st = run_filter(0, n_items, &again);
                    if (st) return st;
                } else {
                    banded = true;
                }
            }
            if (!banded && !fault.keys && A.alloc(&keys, (size_t)(n_surv > 0 ? n_surv : 1)) == BMJ_OK) {
                st = run_verify(queue, n_surv, keys, &n_res);
                if (st) return st;
            } else if (!banded) {
                // every survivor is queued but a key buffer as long as the queue does
                // not fit: verify the queue in slices (results <= survivors per slice)
                const int64_t slice = std::max<int64_t>(
                    1, std::min<int64_t>(fault.keys ? (n_surv + 4) / 5 : n_surv, (int64_t)1 << 26));
                uint64_t *bkeys = nullptr;
                st = A.alloc(&bkeys, (size_t)slice);
                if (st) return st;
                for (int64_t at = 0; at < n_surv; at += slice) {
                    int64_t r = 0;
                    st = run_verify(queue + at, std::min(slice, n_surv - at), bkeys, &r);
                    if (!st) st = append(bkeys, r);
                    if (st) return st;
                }
                A.free_one(bkeys);
            } else {
                // Item ranges sized from the measured survivor density; a range that
                // still overflows is split again, and a single item that overflows
                // gets a queue of exactly its size.
                uint64_t *bkeys = nullptr;
                st = A.alloc(&bkeys, (size_t)qcap);
                if (st) return st;
                int64_t lo = 0;
                double density = (double)n_surv / (double)std::max<int64_t>(n_items, 1);
                while (lo < n_items) {
                    int64_t step = (int64_t)(0.8 * (double)qcap / std::max(density, 1e-12));
                    step = std::max<int64_t>(1, std::min(step, n_items - lo));
                    int64_t c = 0;
                    st = run_filter(lo, lo + step, &c);
                    if (st) return st;
                    if (c > qcap) {
                        if (step > 1) {  // too dense here: retry a shorter range
                            density = std::max(density, (double)c / (double)step);
                            continue;
                        }
                        // one work item alone overflows: give the queue its exact size
                        A.free_one(queue);
                        A.free_one(bkeys);
                        qcap = c;
                        st = A.alloc(&queue, (size_t)qcap);
                        if (!st) st = A.alloc(&bkeys, (size_t)qcap);
                        if (st) return st;
                        fa.queue = queue;
                        fa.qcap = qcap;
                        st = run_filter(lo, lo + 1, &c);
                        if (st) return st;
                    }
                    int64_t r = 0;
                    st = run_verify(queue, c, bkeys, &r);
                    if (!st) st = append(bkeys, r);
                    if (st) return st;
                    lo += step;
                    if (c > 0) density = 0.5 * density + 0.5 * (double)c / (double)step;
                }
                A.free_one(bkeys);
            }
            A.free_one(queue);
        }

        // ---- canonical order ----
        if (n_res > 0) {
            NvtxRange nv("bmj.result_sort");
            st = A.alloc(&keys_sorted, (size_t)n_res);
            if (!st) st = radix_sort_u64(keys, keys_sorted, n_res, 2 * nbits, A, s);
            if (st) return st;
        }
    } else {
        BMJ_CHECK(cudaEventRecord(ev.e[2], s));
        BMJ_CHECK(cudaEventRecord(ev.e[5], s));
        BMJ_CHECK(cudaEventRecord(ev.e[6], s));
    }
    stl.results = n_res;

    // ---- output ----
    NvtxRange nv_out("bmj.output");
    bmj_pairs res;
    memset(&res, 0, sizeof(res));
    res.on_device = o.output_on_device ? 1 : 0;
    if (n_res > 0) {
        if (o.output_on_device) {
            if (cudaMalloc(&res.a, n_res * sizeof(uint32_t)) != cudaSuccess ||
                cudaMalloc(&res.b, n_res * sizeof(uint32_t)) != cudaSuccess) {
                cudaGetLastError();
                if (res.a) cudaFree(res.a);
                return BMJ_ERR_OOM;
            }
            st = launch_unpack(keys_sorted, n_res, nbits, res.a, res.b, s, (uint32_t)n_r);
        } else {
            uint32_t *da = nullptr, *db = nullptr;
            st = A.alloc(&da, (size_t)n_res);
            if (!st) st = A.alloc(&db, (size_t)n_res);
            if (!st) st = launch_unpack(keys_sorted, n_res, nbits, da, db, s, (uint32_t)n_r);
            if (!st) {
                // one page-locked block (a, then b) from the reuse pool, so that the
                // copy out runs at full link speed without pinning pages every call
                uint32_t *blk = (uint32_t *)pinned_alloc(2 * (size_t)n_res * sizeof(uint32_t));
                if (blk) {
                    res.a = blk;
                    res.b = blk + n_res;
                    res.host_pinned = 1;
                } else {
                    res.a = (uint32_t *)malloc(n_res * sizeof(uint32_t));
                    res.b = (uint32_t *)malloc(n_res * sizeof(uint32_t));
                    res.host_pinned = 0;
                    if (!res.a || !res.b) st = BMJ_ERR_OOM;
                }
            }
            if (!st) {
                cudaError_t e1 = cudaMemcpyAsync(res.a, da, n_res * sizeof(uint32_t),
                                                 cudaMemcpyDeviceToHost, s);
                cudaError_t e2 = cudaMemcpyAsync(res.b, db, n_res * sizeof(uint32_t),
                                                 cudaMemcpyDeviceToHost, s);
                if (e1 != cudaSuccess || e2 != cudaSuccess) st = status_of(e1 ? e1 : e2);
            }
        }
        if (st) {
            bmj_pairs_free(&res);
            return st;
        }
        res.n = n_res;
    }
    BMJ_CHECK(cudaEventRecord(ev.e[7], s));
    A.release();
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        bmj_pairs_free(&res);
        return status_of(e);
    }
    stl.ms_prepare = ev.ms(0, 2);
    stl.ms_output = ev.ms(6, 7);
    stl.ms_total = ev.ms(0, 7);
    stl.n_launches = (int32_t)(launches() - launches0);
    *out = res;
    if (stats) *stats = stl;
    return BMJ_OK;
}

static int build_bitmaps_impl(const bmj_collection *coll, int b, int method, uint64_t *out,
                              cudaStream_t s) {
    int dev = 0;
    BMJ_CHECK(cudaGetDevice(&dev));
    retain_pool_memory(dev);
    Arena A(s);
    DevColl d;
    int st = stage_collection(coll, A, s, &d);
    if (st) return st;
    if (d.n == 0) return BMJ_OK;
    uint32_t *sizes = nullptr, *ids = nullptr;
    int max_size = 0;
    st = validate(d, true, A, s, &sizes, &ids, &max_size);
    if (st) return st;
    const int W = b / 64;
    uint64_t *dst = out;
    if (!coll->on_device) {
        st = A.alloc(&dst, (size_t)d.n * W);
        if (st) return st;
    }
    st = launch_gather_build(nullptr, d.off, d.tok, nullptr, nullptr, dst, d.n, b, method, s);
    if (st) return st;
    if (!coll->on_device)
        BMJ_CHECK(cudaMemcpyAsync(out, dst, (size_t)d.n * W * sizeof(uint64_t),
                                  cudaMemcpyDeviceToHost, s));
    A.release();
    BMJ_CHECK(cudaStreamSynchronize(s));
    return BMJ_OK;
}

}  // namespace bmj

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

void bmj_default_options(bmj_options *opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->b = 64;
    opt->method = BMJ_XOR;
    opt->output_on_device = 0;
    opt->validate = 1;
    opt->queue_cap = 0;
    opt->stream = nullptr;
    opt->rows_per_thread = 0;
}

const char *bmj_strerror(int status) {
    switch (status) {
        case BMJ_OK: return "ok";
        case BMJ_ERR_INVALID_ARG: return "invalid argument";
        case BMJ_ERR_UNSORTED: return "tokens of a set are not strictly increasing (or offsets are inconsistent)";
        case BMJ_ERR_EMPTY_SET: return "empty set in the collection";
        case BMJ_ERR_NEG_TOKEN: return "negative token id";
        case BMJ_ERR_OOM: return "out of memory";
        case BMJ_ERR_OUTPUT_OVERFLOW: return "output buffer too small";
        case BMJ_ERR_TIMEOUT: return "bounded device wait timed out";
        case BMJ_ERR_CUDA: return "CUDA runtime error";
        case BMJ_ERR_TOO_LARGE: return "too large (n_sets >= 2^31, a set of >= 2^24 tokens, or a probe above the server's limit)";
        case BMJ_PENDING: return "pending: the query has not completed yet";
        default: return "unknown status";
    }
}

static int check_collection(const bmj_collection *c) {
    if (!c) return BMJ_ERR_INVALID_ARG;
    if (c->n_sets < 0) return BMJ_ERR_INVALID_ARG;
    if (c->n_sets > 0x7fffffffLL) return BMJ_ERR_TOO_LARGE;
    if (!c->offsets) return BMJ_ERR_INVALID_ARG;
    if (c->n_sets > 0 && !c->tokens) return BMJ_ERR_INVALID_ARG;
    return BMJ_OK;
}

int bmj_build_bitmaps(const bmj_collection *coll, int b, int method, uint64_t *out,
                      void *stream) {
    int st = check_collection(coll);
    if (st) return st;
    if (!bmj::valid_b(b)) return BMJ_ERR_INVALID_ARG;
    if (method != BMJ_XOR && method != BMJ_SET && method != BMJ_NEXT) return BMJ_ERR_INVALID_ARG;
    if (coll->n_sets > 0 && !out) return BMJ_ERR_INVALID_ARG;
    try {
        st = bmj::build_bitmaps_impl(coll, b, method, out, (cudaStream_t)stream);
    } catch (...) {
        st = BMJ_ERR_OOM;
    }
    cudaGetLastError();
    return st;
}

int bmj_self_join(const bmj_collection *coll, int sim, uint32_t p, uint32_t q,
                  const bmj_options *opt, bmj_pairs *out, bmj_stats *stats) {
    if (!out) return BMJ_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    if (stats) memset(stats, 0, sizeof(*stats));
    int st = check_collection(coll);
    if (st) return st;
    if (!bmj::sim_valid(sim, p, q)) return BMJ_ERR_INVALID_ARG;
    bmj_options o;
    if (opt) o = *opt;
    else bmj_default_options(&o);
    if (!bmj::valid_b(o.b)) return BMJ_ERR_INVALID_ARG;
    if (o.method < BMJ_XOR || o.method > BMJ_COMBINED) return BMJ_ERR_INVALID_ARG;
    if (o.queue_cap < 0) return BMJ_ERR_INVALID_ARG;
    if (o.cascade_b != 0 && o.cascade_b != -1 && !bmj::valid_b(o.cascade_b)) return BMJ_ERR_INVALID_ARG;
    if (o.row_begin < 0 || o.row_end < 0 || o.row_end < o.row_begin) return BMJ_ERR_INVALID_ARG;
    if (o.candidates != BMJ_CAND_WINDOW && o.candidates != BMJ_CAND_PREFIX &&
        o.candidates != BMJ_CAND_AUTO)
        return BMJ_ERR_INVALID_ARG;
    if (o.candidates != BMJ_CAND_WINDOW && (o.row_begin != 0 || o.row_end != 0 || o.cutoff != 0))
        return BMJ_ERR_INVALID_ARG;
    if (o.cutoff < BMJ_CUTOFF_AUTO) return BMJ_ERR_INVALID_ARG;
    if ((o.row_begin != 0 || o.row_end != 0) && o.row_end > coll->n_sets) return BMJ_ERR_INVALID_ARG;
    try {
        st = bmj::self_join_impl(coll, nullptr, sim, p, q, o, out, stats);
    } catch (...) {
        st = BMJ_ERR_OOM;
    }
    bmj::arm_alloc_fault(0);
    if (st) {
        bmj_pairs_free(out);
        cudaGetLastError();
    }
    return st;
}

int bmj_rs_join(const bmj_collection *r, const bmj_collection *s, int sim, uint32_t p, uint32_t q,
                const bmj_options *opt, bmj_pairs *out, bmj_stats *stats) {
    if (!out) return BMJ_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    if (stats) memset(stats, 0, sizeof(*stats));
    int st = check_collection(r);
    if (!st) st = check_collection(s);
    if (st) return st;
    if (r->n_sets + s->n_sets > 0x7fffffffLL) return BMJ_ERR_TOO_LARGE;
    if (!bmj::sim_valid(sim, p, q)) return BMJ_ERR_INVALID_ARG;
    bmj_options o;
    if (opt) o = *opt;
    else bmj_default_options(&o);
    if (!bmj::valid_b(o.b)) return BMJ_ERR_INVALID_ARG;
    if (o.method < BMJ_XOR || o.method > BMJ_COMBINED) return BMJ_ERR_INVALID_ARG;
    if (o.queue_cap < 0) return BMJ_ERR_INVALID_ARG;
    if (o.cascade_b != 0 && o.cascade_b != -1 && !bmj::valid_b(o.cascade_b)) return BMJ_ERR_INVALID_ARG;
    if (o.row_begin != 0 || o.row_end != 0) return BMJ_ERR_INVALID_ARG;
    if (o.candidates != BMJ_CAND_WINDOW && o.candidates != BMJ_CAND_PREFIX &&
        o.candidates != BMJ_CAND_AUTO)
        return BMJ_ERR_INVALID_ARG;
    if (o.cutoff < BMJ_CUTOFF_AUTO) return BMJ_ERR_INVALID_ARG;
    if (o.candidates != BMJ_CAND_WINDOW && o.cutoff != 0) return BMJ_ERR_INVALID_ARG;
    try {
        st = bmj::self_join_impl(r, s, sim, p, q, o, out, stats);
    } catch (...) {
        st = BMJ_ERR_OOM;
    }
    bmj::arm_alloc_fault(0);
    if (st) {
        bmj_pairs_free(out);
        cudaGetLastError();
    }
    return st;
}

void bmj_pairs_free(bmj_pairs *pairs) {
    if (!pairs) return;
    if (pairs->on_device) {
        if (pairs->a) cudaFree(pairs->a);
        if (pairs->b) cudaFree(pairs->b);
    } else if (pairs->host_pinned == 1) {  // one pooled page-locked block holding a and b
        bmj::pinned_release(pairs->a);
    } else {
        free(pairs->a);
        free(pairs->b);
    }
    pairs->host_pinned = 0;
    pairs->a = nullptr;
    pairs->b = nullptr;
    pairs->n = 0;
}

int64_t bmj_kernel_launches(void) { return bmj::launches(); }

}  // extern "C"
