// Measurement aid, no counterpart in the paper: the throughput of the count
// kernel's counter operation on this GPU, the second ceiling (beside HBM) of
// the wedge enumeration.  One 1024-thread CTA per SM with 192 KB of shared
// memory, as the count kernel runs; every thread increments 16-bit counters
// packed two per 32-bit word at pseudo-random indexes with a returning
// atomicAdd, as wedge_op does for each wedge.
#include "bfc_internal.cuh"

namespace bfc {
namespace {

constexpr int kBenchCounters = 65536;   // 128 KB of packed 16-bit counters

__global__ void __launch_bounds__(1024, 1) k_smem_atomics(int32_t iters, uint32_t *sink) {
    extern __shared__ __align__(16) uint32_t words[];
    for (int i = threadIdx.x; i < kBenchCounters / 2; i += blockDim.x) words[i] = 0;
    __syncthreads();
    // a 32-bit LCG per thread (Numerical Recipes constants) spreads the
    // indexes over the banks like the ends of a wedge window
    uint32_t x = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 12345u;
    uint32_t acc = 0;
    for (int32_t i = 0; i < iters; ++i) {
        x = x * 1664525u + 1013904223u;
        const uint32_t idx = (x >> 16) & (kBenchCounters - 1);
        const uint32_t sh = (idx & 1u) << 4;
        const uint32_t old = atomicAdd(words + (idx >> 1), 1u << sh);
        acc += (old >> sh) & 0xffffu;
    }
    if (acc == 0xffffffffu) sink[0] = acc;   // keeps the loop; practically never taken
}

}  // namespace
}  // namespace bfc

extern "C" int bfc_bench_smem_atomics(void *stream, int32_t iters, double *increments_per_s,
                                      double *ms_out) {
    bfc::set_last_error("");
    if (iters < 1 || !increments_per_s) {
        bfc::set_last_error("iters must be >= 1 and increments_per_s non-null");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    BFC_CUDA(cudaGetDevice(&dev));
    BFC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    BFC_CUDA(cudaFuncSetAttribute(bfc::k_smem_atomics, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  bfc::kCounterBytes));
    uint32_t *sink = nullptr;
    BFC_CUDA(bfc::pool_alloc(reinterpret_cast<void **>(&sink), 256, s));
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) { bfc::pool_free(sink, s); return bfc::cuda_fail(e, "cudaEventCreate"); }
    // warm-up launch, then the timed one
    bfc::k_smem_atomics<<<sms, 1024, bfc::kCounterBytes, s>>>(iters < 64 ? iters : 64, sink);
    bfc::note_launch();
    cudaEventRecord(e0, s);
    bfc::k_smem_atomics<<<sms, 1024, bfc::kCounterBytes, s>>>(iters, sink);
    bfc::note_launch();
    cudaEventRecord(e1, s);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    bfc::pool_free(sink, s);
    if (e != cudaSuccess) return bfc::cuda_fail(e, "k_smem_atomics");
    *increments_per_s = (double)sms * 1024.0 * (double)iters / (ms * 1e-3);
    if (ms_out) *ms_out = ms;
    return BFC_OK;
}
