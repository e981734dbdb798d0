// verify.cu -- exact verification of the filter's survivors and the canonical
// output (kept apart from the filter kernels in kernels.cu).
//   k_verify         exact overlap of the survivors by merge intersection
//                    (the verification of Alg. 6's host code, moved on the GPU),
//                    after an optional second Eq. 2 test with wider bitmaps
//   k_verify_c256    the same with the 256-bit second test, several survivors
//                    per thread
//   k_unpack         canonical output pairs
#include "kernels.cuh"

namespace bmj {
namespace {
// need / lim of a pair of sizes: the tables indexed by |x|+|y|, or computed for
// Cosine (whose smallest passing overlap depends on |x|*|y|).
struct PairTest {
    const int32_t *need, *lim;
    uint32_t p, q;
};
template <bool kCos>
__device__ __forceinline__ int pair_need(const PairTest &t, uint32_t x, uint32_t y) {
    return kCos ? (int)cosine_need(t.p, t.q, x, y) : t.need[x + y];
}
template <bool kCos>
__device__ __forceinline__ int pair_limit(const PairTest &t, uint32_t x, uint32_t y) {
    return kCos ? (int)((int64_t)x + y - 2 * cosine_need(t.p, t.q, x, y)) : t.lim[x + y];
}
}  // namespace
}  // namespace bmj

// Survivors per thread of the verification with the 256-bit cascade (2 was
// fastest on the 1M-set workload at threshold 1/2: 13.3 ms, against 13.9 ms
// for 1, 16.5 ms for 4 and 17.8 ms for k_verify).
#ifndef BMJ_VERIFY_SPT
#define BMJ_VERIFY_SPT 2
#endif

namespace bmj {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// ----------------------------------------------------------------------------
// Verification: one survivor per thread.  When a second, wider bitmap array is
// given (cascade), the survivor first meets the Eq. 2 bound again with those
// bitmaps -- Theorem 1 holds for any b, so this drops no similar pair -- and
// only pairs that pass it are merged.  The merge of the two sorted token
// arrays stops as soon as the outcome is decided (the overlap reached need[S],
// or the remaining tokens cannot reach it).
template <bool kCos>
__global__ void __launch_bounds__(256)
    k_verify(const uint2 *__restrict__ queue, int64_t n_surv, const int64_t *__restrict__ soff,
             const int32_t *__restrict__ stok, const uint32_t *__restrict__ ssz,
             const uint32_t *__restrict__ perm, const PairTest pt,
             const uint64_t *__restrict__ bm2, int W2,
             uint64_t *__restrict__ keys, unsigned long long *__restrict__ rcount,
             unsigned long long *__restrict__ ccount, int nbits) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    unsigned n_passed = 0;
    for (int64_t base = gw * 32; base < n_surv; base += warps * 32) {
        const int64_t idx = base + lane;
        bool similar = false, passed = false;
        uint64_t key = 0;
        if (idx < n_surv) {
            const uint2 pr = queue[idx];
            const uint32_t si = ssz[pr.x], sj = ssz[pr.y];
            passed = true;
            if (bm2) {
                const uint64_t *a = bm2 + (int64_t)pr.x * W2;
                const uint64_t *c = bm2 + (int64_t)pr.y * W2;
                int h = 0;
                for (int w = 0; w < W2; w++) h += __popcll(a[w] ^ c[w]);
                passed = h <= pair_limit<kCos>(pt, si, sj);
            }
            if (passed) {
                const int nd = pair_need<kCos>(pt, si, sj);
                const int32_t *x = stok + soff[pr.x];
                const int32_t *y = stok + soff[pr.y];
                int a = 0, b = 0, o = 0;
                const int na = (int)si, nb = (int)sj;
                while (a < na && b < nb) {
                    if (o + min(na - a, nb - b) < nd) break;
                    const int32_t xa = x[a], yb = y[b];
                    o += (xa == yb);
                    a += (xa <= yb);
                    b += (yb <= xa);
                    if (o >= nd) break;
                }
                similar = o >= nd;
                if (similar) {
                    const uint64_t u = perm[pr.x], v = perm[pr.y];
                    key = u < v ? ((u << nbits) | v) : ((v << nbits) | u);
                }
            }
        }
        n_passed += passed ? 1u : 0u;
        const unsigned ball = __ballot_sync(kFull, similar);
        if (ball) {
            unsigned long long off = 0;
            if (lane == 0) off = atomicAdd(rcount, (unsigned long long)__popc(ball));
            off = __shfl_sync(kFull, off, 0);
            if (similar) keys[off + __popc(ball & ((1u << lane) - 1u))] = key;
        }
    }
    if (ccount) {  // one atomic per block
        __shared__ unsigned long long block_passed;
        if (threadIdx.x == 0) block_passed = 0;
        __syncthreads();
        const unsigned v = __reduce_add_sync(kFull, n_passed);
        if (lane == 0 && v) atomicAdd(&block_passed, (unsigned long long)v);
        __syncthreads();
        if (threadIdx.x == 0 && block_passed) atomicAdd(ccount, block_passed);
    }
}

// Verification with the 256-bit cascade (the path of every join with b < 256):
// the same test as k_verify, specialised to 32-byte second bitmaps read as two
// 16-byte loads, with SPT survivors per thread whose loads are all issued
// before any of them is used, so that a thread keeps several independent L2
// requests in flight (the kernel is bound by L2 latency, not bandwidth).
template <int SPT, bool kCos>
__global__ void __launch_bounds__(256)
    k_verify_c256(const uint2 *__restrict__ queue, int64_t n_surv, const int64_t *__restrict__ soff,
                  const int32_t *__restrict__ stok, const uint32_t *__restrict__ ssz,
                  const uint32_t *__restrict__ perm, const PairTest pt,
                  const uint4 *__restrict__ bm2,
                  uint64_t *__restrict__ keys, unsigned long long *__restrict__ rcount,
                  unsigned long long *__restrict__ ccount, int nbits) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    unsigned n_passed = 0;
    for (int64_t base = gw * 32 * SPT; base < n_surv; base += warps * 32 * SPT) {
        uint2 pr[SPT];
#pragma unroll
        for (int u = 0; u < SPT; u++) {
            const int64_t idx = base + u * 32 + lane;
            pr[u] = idx < n_surv ? queue[idx] : make_uint2(0u, 0u);  // set 0 exists: n_surv > 0
        }
        uint32_t si[SPT], sj[SPT];
        uint4 x0[SPT], x1[SPT], y0[SPT], y1[SPT];
#pragma unroll
        for (int u = 0; u < SPT; u++) {
            si[u] = ssz[pr[u].x];
            sj[u] = ssz[pr[u].y];
            x0[u] = bm2[2 * (int64_t)pr[u].x];
            x1[u] = bm2[2 * (int64_t)pr[u].x + 1];
            y0[u] = bm2[2 * (int64_t)pr[u].y];
            y1[u] = bm2[2 * (int64_t)pr[u].y + 1];
        }
#pragma unroll
        for (int u = 0; u < SPT; u++) {
            const int64_t idx = base + u * 32 + lane;
            const int h = __popc(x0[u].x ^ y0[u].x) + __popc(x0[u].y ^ y0[u].y) +
                          __popc(x0[u].z ^ y0[u].z) + __popc(x0[u].w ^ y0[u].w) +
                          __popc(x1[u].x ^ y1[u].x) + __popc(x1[u].y ^ y1[u].y) +
                          __popc(x1[u].z ^ y1[u].z) + __popc(x1[u].w ^ y1[u].w);
            const bool passed = idx < n_surv && h <= pair_limit<kCos>(pt, si[u], sj[u]);
            bool similar = false;
            uint64_t key = 0;
            if (passed) {
                const int nd = pair_need<kCos>(pt, si[u], sj[u]);
                const int32_t *x = stok + soff[pr[u].x];
                const int32_t *y = stok + soff[pr[u].y];
                int a = 0, b = 0, o = 0;
                const int na = (int)si[u], nb = (int)sj[u];
                while (a < na && b < nb) {
                    if (o + min(na - a, nb - b) < nd) break;
                    const int32_t xa = x[a], yb = y[b];
                    o += (xa == yb);
                    a += (xa <= yb);
                    b += (yb <= xa);
                    if (o >= nd) break;
                }
                similar = o >= nd;
                if (similar) {
                    const uint64_t v0 = perm[pr[u].x], v1 = perm[pr[u].y];
                    key = v0 < v1 ? ((v0 << nbits) | v1) : ((v1 << nbits) | v0);
                }
            }
            n_passed += passed ? 1u : 0u;
            const unsigned ball = __ballot_sync(kFull, similar);
            if (ball) {
                unsigned long long off = 0;
                if (lane == 0) off = atomicAdd(rcount, (unsigned long long)__popc(ball));
                off = __shfl_sync(kFull, off, 0);
                if (similar) keys[off + __popc(ball & ((1u << lane) - 1u))] = key;
            }
        }
    }
    if (ccount) {  // one atomic per block
        __shared__ unsigned long long block_passed;
        if (threadIdx.x == 0) block_passed = 0;
        __syncthreads();
        const unsigned v = __reduce_add_sync(kFull, n_passed);
        if (lane == 0 && v) atomicAdd(&block_passed, (unsigned long long)v);
        __syncthreads();
        if (threadIdx.x == 0 && block_passed) atomicAdd(ccount, block_passed);
    }
}

__global__ void k_unpack(const uint64_t *__restrict__ keys, int64_t n, int nbits,
                         uint32_t *__restrict__ a, uint32_t *__restrict__ b, uint32_t b_sub) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const uint64_t mask = (nbits >= 64) ? ~0ull : ((1ull << nbits) - 1ull);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t k = keys[i];
        a[i] = (uint32_t)(k >> nbits);
        b[i] = (uint32_t)(k & mask) - b_sub;
    }
}

unsigned grid_for(int64_t n, int threads, int64_t cap) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

}  // namespace

template <bool kCos>
int launch_verify_t(const uint2 *queue, int64_t n_surv, const int64_t *soff, const int32_t *stok,
                    const uint32_t *ssz, const uint32_t *perm, const int32_t *need,
                    const int32_t *lim, const uint64_t *bm2, int W2, uint64_t *keys,
                    unsigned long long *rcount, unsigned long long *ccount, int nbits, int num_sms,
                    cudaStream_t s, uint32_t p, uint32_t q) {
    if (n_surv <= 0) return BMJ_OK;
    const PairTest pt{need, lim, p, q};
#if BMJ_VERIFY_SPT > 0
    if (bm2 && W2 == 4) {
        constexpr int kSpt = BMJ_VERIFY_SPT;
        int per_sm = 0;
        BMJ_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_verify_c256<kSpt, kCos>,
                                                                256, 0));
        if (per_sm < 1) per_sm = 1;
        BMJ_LAUNCH((k_verify_c256<kSpt, kCos>),
                   grid_for(n_surv, 256 * kSpt, (int64_t)num_sms * per_sm), 256, 0, s, queue,
                   n_surv, soff, stok, ssz, perm, pt, reinterpret_cast<const uint4 *>(bm2), keys,
                   rcount, ccount, nbits);
        return BMJ_OK;
    }
#endif
    BMJ_LAUNCH((k_verify<kCos>), grid_for(n_surv, 256, (int64_t)num_sms * 8), 256, 0, s, queue,
               n_surv, soff, stok, ssz, perm, pt, bm2, W2, keys, rcount, ccount, nbits);
    return BMJ_OK;
}

int launch_verify(const uint2 *queue, int64_t n_surv, const int64_t *soff, const int32_t *stok,
                  const uint32_t *ssz, const uint32_t *perm, const int32_t *need,
                  const int32_t *lim, const uint64_t *bm2, int W2, uint64_t *keys,
                  unsigned long long *rcount, unsigned long long *ccount, int nbits, int num_sms,
                  cudaStream_t s, int sim, uint32_t p, uint32_t q) {
    return sim == BMJ_COSINE
               ? launch_verify_t<true>(queue, n_surv, soff, stok, ssz, perm, need, lim, bm2, W2,
                                       keys, rcount, ccount, nbits, num_sms, s, p, q)
               : launch_verify_t<false>(queue, n_surv, soff, stok, ssz, perm, need, lim, bm2, W2,
                                        keys, rcount, ccount, nbits, num_sms, s, p, q);
}

int launch_unpack(const uint64_t *keys, int64_t n, int nbits, uint32_t *a, uint32_t *b,
                  cudaStream_t s, uint32_t b_sub) {
    if (n <= 0) return BMJ_OK;
    BMJ_LAUNCH(k_unpack, grid_for(n, 256, 148 * 32), 256, 0, s, keys, n, nbits, a, b, b_sub);
    return BMJ_OK;
}

}  // namespace bmj
