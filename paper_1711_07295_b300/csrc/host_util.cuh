// host_util.cuh -- host-side helpers shared by the join entry points.
#pragma once

#include <cmath>
#include <cstring>
#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "kernels.cuh"

namespace bmj {

inline int num_sms(int device) {
    static std::mutex mu;
    static int cache[128] = {0};
    std::lock_guard<std::mutex> lk(mu);
    if (device >= 0 && device < 128 && cache[device]) return cache[device];
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v <= 0)
        v = 148;
    if (device >= 0 && device < 128) cache[device] = v;
    return v;
}

inline int bit_length(uint64_t v) {
    int b = 0;
    while (v) {
        b++;
        v >>= 1;
    }
    return b;
}

// Alg. 4 with its switch points read on the normalised overlap 2p/(p+q).
inline int combined_method(uint32_t p, uint32_t q) {
    const uint64_t P = p, D = (uint64_t)p + q;
    if (200 * P <= 56 * D) return BMJ_NEXT;
    if (200 * P >= 73 * D) return BMJ_XOR;
    return BMJ_SET;
}

// Alg. 4 for any function: the switch points apply to the normalised overlap of
// two equal-sized sets at the threshold (Jaccard 2p/(p+q) above; Dice and Cosine
// p/q itself); an Overlap threshold counts tokens and is not normalised, so Xor
// (the paper's GPU choice) is kept.
inline int combined_method(int sim, uint32_t p, uint32_t q) {
    if (sim == BMJ_JACCARD) return combined_method(p, q);
    if (sim == BMJ_OVERLAP) return BMJ_XOR;
    const uint64_t P = p, Q = q;
    if (100 * P <= 56 * Q) return BMJ_NEXT;
    if (100 * P >= 73 * Q) return BMJ_XOR;
    return BMJ_SET;
}

// Section 3.5: the expected Eq. 2 bound of two random n-token sets hashed into
// b bits -- Eq. 4 (Set) as n + b r^2 - b r with r = (1 - 1/b)^n, Eq. 5 (Xor)
// with its sum of odd binomial terms in closed form, Eq. 6 (Next).
inline double expected_bound(int b, int method, double n) {
    const double bb = (double)b;
    if (method == BMJ_SET) {
        const double r = pow(1.0 - 1.0 / bb, n);
        return n + bb * r * r - bb * r;
    }
    if (method == BMJ_NEXT) return fmin(n * n / bb, n);
    return n - bb / 4.0 * (1.0 - pow(1.0 - 2.0 / bb, 2.0 * n));
}

// The cutoff point: the largest set size n whose expected normalised bound
// E(b, n)/n is still at most the normalised threshold (Jaccard 2p/(p+q), Dice
// and Cosine p/q), at least 1; 0 when there is none (Overlap, whose threshold
// is not normalised, or a threshold no size reaches below the largest size).
inline int64_t cutoff_point(int b, int method, int sim, uint32_t p, uint32_t q) {
    if (sim == BMJ_OVERLAP) return 0;
    const double u = sim == BMJ_JACCARD ? 2.0 * p / ((double)p + (double)q) : (double)p / (double)q;
    auto above = [&](int64_t n) { return expected_bound(b, method, (double)n) / (double)n > u; };
    int64_t hi = 2;
    while (!above(hi)) {
        if (hi > kMaxSetSize) return 0;
        hi *= 2;
    }
    int64_t lo = 1;  // E/n grows with n: the answer lies in [lo, hi)
    if (above(lo)) return 1;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) / 2;
        if (above(mid)) hi = mid;
        else lo = mid;
    }
    return lo;
}

inline int flags_to_status(int flags) {
    if (flags & kFlagTooLarge) return BMJ_ERR_TOO_LARGE;
    if (flags & kFlagUnsorted) return BMJ_ERR_UNSORTED;
    if (flags & kFlagNegative) return BMJ_ERR_NEG_TOKEN;
    if (flags & kFlagEmpty) return BMJ_ERR_EMPTY_SET;
    return BMJ_OK;
}

inline bool valid_b(int b) { return b >= 64 && b <= 4096 && (b % 64) == 0; }

// A named NVTX range over a host scope (a call or a stage): profilers (ncu
// --nvtx, nsys) see the library's stages; without a tool attached a range
// costs a few nanoseconds.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Device-resident view of a collection (copied in when it is host memory).
struct DevColl {
    const int64_t *off = nullptr;
    const int32_t *tok = nullptr;
    int64_t n = 0;
    int64_t ntok = 0;
};

inline int stage_collection(const bmj_collection *c, Arena &A, cudaStream_t s, DevColl *d) {
    d->n = c->n_sets;
    if (c->on_device) {
        int64_t v = 0;
        BMJ_CHECK(cudaMemcpyAsync(&v, c->offsets + c->n_sets, sizeof(int64_t),
                                  cudaMemcpyDeviceToHost, s));
        BMJ_CHECK(cudaStreamSynchronize(s));
        d->off = c->offsets;
        d->tok = c->tokens;
        d->ntok = v;
        if (v < 0) return BMJ_ERR_UNSORTED;
        return BMJ_OK;
    }
    d->ntok = c->offsets[c->n_sets];
    if (d->ntok < 0) return BMJ_ERR_UNSORTED;
    int64_t *off = nullptr;
    int32_t *tok = nullptr;
    int st = A.alloc(&off, (size_t)(c->n_sets + 1));
    if (!st) st = A.alloc(&tok, (size_t)d->ntok);
    if (st) return st;
    BMJ_CHECK(cudaMemcpyAsync(off, c->offsets, (c->n_sets + 1) * sizeof(int64_t),
                              cudaMemcpyHostToDevice, s));
    if (d->ntok)
        BMJ_CHECK(cudaMemcpyAsync(tok, c->tokens, d->ntok * sizeof(int32_t),
                                  cudaMemcpyHostToDevice, s));
    d->off = off;
    d->tok = tok;
    return BMJ_OK;
}

// The two collections of an RS-join as one device CSR, R's sets first: set x
// of S becomes set n_r + x.  Each input must start at offset 0.
inline int stage_two(const bmj_collection *r, const bmj_collection *c, Arena &A, cudaStream_t s,
                     DevColl *d) {
    int64_t ends[2][2] = {{0, 0}, {0, 0}};  // first and last offset of R and of S
    const bmj_collection *in[2] = {r, c};
    for (int k = 0; k < 2; k++) {
        const bmj_collection *x = in[k];
        if (x->on_device) {
            BMJ_CHECK(cudaMemcpyAsync(&ends[k][0], x->offsets, sizeof(int64_t),
                                      cudaMemcpyDeviceToHost, s));
            BMJ_CHECK(cudaMemcpyAsync(&ends[k][1], x->offsets + x->n_sets, sizeof(int64_t),
                                      cudaMemcpyDeviceToHost, s));
        } else {
            ends[k][0] = x->offsets[0];
            ends[k][1] = x->offsets[x->n_sets];
        }
    }
    BMJ_CHECK(cudaStreamSynchronize(s));
    for (int k = 0; k < 2; k++)
        if (ends[k][0] != 0 || ends[k][1] < 0) return BMJ_ERR_UNSORTED;
    const int64_t nr = r->n_sets, ns = c->n_sets, tr = ends[0][1], ts = ends[1][1];
    d->n = nr + ns;
    d->ntok = tr + ts;
    int64_t *off = nullptr;
    int32_t *tok = nullptr;
    int st = A.alloc(&off, (size_t)(d->n + 1));
    if (!st) st = A.alloc(&tok, (size_t)(d->ntok > 0 ? d->ntok : 1));
    if (st) return st;
    BMJ_CHECK(cudaMemcpyAsync(off, r->offsets, (nr + 1) * sizeof(int64_t),
                              r->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    BMJ_CHECK(cudaMemcpyAsync(off + nr, c->offsets, (ns + 1) * sizeof(int64_t),
                              c->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    st = launch_add_i64(off + nr, ns + 1, tr, s);
    if (st) return st;
    if (tr)
        BMJ_CHECK(cudaMemcpyAsync(tok, r->tokens, tr * sizeof(int32_t),
                                  r->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  s));
    if (ts)
        BMJ_CHECK(cudaMemcpyAsync(tok + tr, c->tokens, ts * sizeof(int32_t),
                                  c->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  s));
    d->off = off;
    d->tok = tok;
    return BMJ_OK;
}

// Validation: returns the status and the maximum set size.
inline int validate(const DevColl &d, bool check_tokens, Arena &A, cudaStream_t s,
                    uint32_t **sizes, uint32_t **ids, int *max_size) {
    int *info = nullptr;
    int st = A.alloc(&info, 2);
    if (!st) st = A.alloc(sizes, (size_t)d.n);
    if (!st) st = A.alloc(ids, (size_t)d.n);
    if (st) return st;
    BMJ_CHECK(cudaMemsetAsync(info, 0, 2 * sizeof(int), s));
    st = launch_validate(d.off, d.tok, d.n, d.ntok, check_tokens ? 1 : 0, *sizes, *ids, info, s);
    if (st) return st;
    int h[2] = {0, 0};
    BMJ_CHECK(cudaMemcpyAsync(h, info, sizeof(h), cudaMemcpyDeviceToHost, s));
    BMJ_CHECK(cudaStreamSynchronize(s));
    *max_size = h[1];
    return flags_to_status(h[0]);
}

struct Events {
    cudaEvent_t e[8];
    int n = 0;
    Events() {
        for (auto &x : e) x = nullptr;
    }
    int init() {
        for (int k = 0; k < 8; k++) BMJ_CHECK(cudaEventCreate(&e[k]));
        n = 8;
        return BMJ_OK;
    }
    ~Events() {
        for (int k = 0; k < n; k++) cudaEventDestroy(e[k]);
    }
    float ms(int a, int b) const {
        float v = 0.f;
        if (cudaEventElapsedTime(&v, e[a], e[b]) != cudaSuccess) {
            cudaGetLastError();
            return 0.f;
        }
        return v;
    }
};

}  // namespace bmj
