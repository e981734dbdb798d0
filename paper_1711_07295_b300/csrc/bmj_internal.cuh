// bmj_internal.cuh -- shared declarations of the CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bmj.h"

namespace bmj {

// ---------------------------------------------------------------------------
// Launch accounting and error plumbing
// ---------------------------------------------------------------------------
void count_launch();                 // one kernel launched
int64_t launches();

struct CudaError {
    cudaError_t err;
};

// Returns the BMJ status for a CUDA error (OOM is distinguished).
inline int status_of(cudaError_t e) {
    if (e == cudaSuccess) return BMJ_OK;
    if (e == cudaErrorMemoryAllocation) return BMJ_ERR_OOM;
    return BMJ_ERR_CUDA;
}

#define BMJ_CHECK(call)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return ::bmj::status_of(e_); \
    } while (0)

// Kernel launch with accounting; checks the launch error.
#define BMJ_LAUNCH(kernel, grid, block, smem, stream, ...)              \
    do {                                                                \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);     \
        ::bmj::count_launch();                                          \
        cudaError_t e_ = cudaGetLastError();                            \
        if (e_ != cudaSuccess) return ::bmj::status_of(e_);             \
    } while (0)

// ---------------------------------------------------------------------------
// Host-side fault injection (tests): BMJ_FAULT=alloc:K makes the K-th device
// allocation of a bmj_self_join call fail; BMJ_FAULT=timeout makes one warp of
// the filter skip one copy, so that its bounded wait runs out;
// BMJ_FAULT=keys refuses the result-key buffer as long as the survivor queue,
// so that verification runs over the queue in slices.
// ---------------------------------------------------------------------------
struct FaultPlan {
    int alloc_at = 0;   // 0: none
    bool timeout = false;
    bool keys = false;
    bool serve = false;  // a call on an index fails as a CUDA runtime error would
};
FaultPlan read_fault_plan();      // parses BMJ_FAULT
void arm_alloc_fault(int k);      // the k-th next Arena allocation fails (0 disarms)
bool alloc_fault_fires();         // consumed by Arena::alloc

// ---------------------------------------------------------------------------
// Device arena: stream-ordered allocations released together.
// ---------------------------------------------------------------------------
struct Arena {
    cudaStream_t stream;
    void *ptrs[256];
    int n = 0;
    explicit Arena(cudaStream_t s) : stream(s) {}
    ~Arena() { release(); }
    template <typename T>
    int alloc(T **p, size_t count) {
        *p = nullptr;
        if (count == 0) count = 1;
        if (n >= 256) return BMJ_ERR_OOM;
        if (alloc_fault_fires()) return BMJ_ERR_OOM;
        void *q = nullptr;
        cudaError_t e = cudaMallocAsync(&q, count * sizeof(T), stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return status_of(e);
        }
        ptrs[n++] = q;
        *p = static_cast<T *>(q);
        return BMJ_OK;
    }
    void free_one(void *p) {
        for (int k = 0; k < n; k++)
            if (ptrs[k] == p) {
                cudaFreeAsync(p, stream);
                ptrs[k] = ptrs[--n];
                return;
            }
    }
    void release() {
        for (int k = 0; k < n; k++) cudaFreeAsync(ptrs[k], stream);
        n = 0;
    }
};

// Keeps the stream-ordered pool's memory between calls (set once per device).
void retain_pool_memory(int device);

// Page-locked host blocks reused between calls (host_pool.cu).  pinned_alloc
// returns nullptr when the CUDA driver refuses; pinned_release returns false for a
// pointer that is not a live block of the pool.
void *pinned_alloc(size_t bytes);
bool pinned_release(void *p);

// ---------------------------------------------------------------------------
// Device-wide primitives (scan_sort.cu)
// ---------------------------------------------------------------------------
// Exclusive prefix sum of n values; in and out may alias.  Writes the grand
// total to *total_dev when it is non-null.
int exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total_dev,
                       Arena &arena, cudaStream_t s);
int exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, Arena &arena,
                       cudaStream_t s);

// Stable LSD radix sort by the low `key_bits` bits of 32-bit keys, carrying
// 32-bit values.  Results end in (keys_out, vals_out).
int radix_sort_u32_pairs(const uint32_t *keys_in, const uint32_t *vals_in, uint32_t *keys_out,
                         uint32_t *vals_out, int64_t n, int key_bits, Arena &arena,
                         cudaStream_t s);

// Stable LSD radix sorts of 32-bit and 64-bit keys by their low `key_bits`
// bits rounded up to whole 8-bit digits (keys equal in those bits keep their
// input order).  The sorted keys end in keys_out.
int radix_sort_u32(const uint32_t *keys_in, uint32_t *keys_out, int64_t n, int key_bits,
                   Arena &arena, cudaStream_t s);
int radix_sort_u64(const uint64_t *keys_in, uint64_t *keys_out, int64_t n, int key_bits,
                   Arena &arena, cudaStream_t s);

}  // namespace bmj
