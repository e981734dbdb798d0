// peak.cu -- measured throughput of the 32-bit population count, the unit of
// the Bitmap Filter's roofline (b/32 popcounts per window pair).
//
// Every thread runs eight independent chains v <- popc(v ^ s) + 2v, so that
// the POPC pipe, not latency, bounds the loop; the xor and the shift-add go to
// the ALU pipe, which has four times the POPC rate.  The grid fills every SM.
#include "bmj_internal.cuh"

namespace bmj {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_popc_peak(uint32_t s, int64_t iters, uint32_t *sink) {
    uint32_t v[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) v[k] = (threadIdx.x + blockIdx.x * blockDim.x) * (2 * k + 1) ^ s;
    for (int64_t i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) v[k] = (uint32_t)__popc(v[k] ^ s) + (v[k] << 1);
    }
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < kChains; k++) acc ^= v[k];
    if (acc == s) sink[0] = acc;  // keeps the chains live; practically never taken
}

}  // namespace
}  // namespace bmj

extern "C" int bmj_measure_popc_rate(void *stream, double *popc_per_s) {
    using namespace bmj;
    if (!popc_per_s) return BMJ_ERR_INVALID_ARG;
    *popc_per_s = 0.0;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    BMJ_CHECK(cudaGetDevice(&dev));
    BMJ_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int per_sm = 0;
    BMJ_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_popc_peak, 256, 0));
    if (per_sm < 1) per_sm = 1;
    const unsigned blocks = (unsigned)(sms * per_sm);
    uint32_t *sink = nullptr;
    BMJ_CHECK(cudaMallocAsync(&sink, sizeof(uint32_t), s));
    cudaEvent_t e0, e1;
    BMJ_CHECK(cudaEventCreate(&e0));
    BMJ_CHECK(cudaEventCreate(&e1));
    const int64_t warm = 1 << 12, iters = 1 << 16;
    int rc = BMJ_OK;
    k_popc_peak<<<blocks, 256, 0, s>>>(0x9e3779b9u, warm, sink);
    count_launch();
    cudaEventRecord(e0, s);
    k_popc_peak<<<blocks, 256, 0, s>>>(0x7f4a7c15u, iters, sink);
    count_launch();
    cudaEventRecord(e1, s);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) rc = status_of(e);
    else if (ms > 0.f)
        *popc_per_s = (double)blocks * 256.0 * (double)iters * kChains / ((double)ms * 1e-3);
    cudaFreeAsync(sink, s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    return rc;
}
