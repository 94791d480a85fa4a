// Measurement support (no counterpart in the paper): the FP32 FMA rate this GPU
// sustains, the denominator of an instruction-issue roofline.  Every thread of a
// full-occupancy grid runs NCHAIN independent FMA chains, so the FMA pipe, not
// dependency latency, sets the pace; the rate counted is FMAs only (the few loop
// instructions per 32 FMAs also take issue slots, so the issue peak is slightly
// higher than the FMA rate reported).
#include "volume.cuh"

namespace {

constexpr int CAL_THREADS = 256;
constexpr int NCHAIN = 8;
constexpr int UNROLL = 4;  // NCHAIN * UNROLL = 32 FMAs per loop iteration

__global__ void __launch_bounds__(CAL_THREADS) fma_rate_kernel(float* sink, int iters, float a, float b) {
    float x[NCHAIN];
#pragma unroll
    for (int c = 0; c < NCHAIN; ++c) x[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
#pragma unroll
            for (int c = 0; c < NCHAIN; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < NCHAIN; ++c) s += x[c];
    // the chains start at x >= 0 and a, b > 0 keep them there, so the store never
    // happens (sink may be null); the compiler cannot know that and keeps every FMA
    if (s < 0.f) sink[threadIdx.x] = s;
}

}  // namespace

extern "C" int sc_measure_fp32_rate(int32_t iters, double* lane_fma_per_s, double* ms_out, sc_stream stream) {
    if (iters < 1 || iters > (1 << 24) || !lane_fma_per_s) return SC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0, per_sm = 0;
    SC_CUDA(cudaGetDevice(&dev));
    SC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_rate_kernel, CAL_THREADS, 0));
    if (per_sm < 1) per_sm = 1;
    const int grid = sms * per_sm;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SC_CUDA(cudaEventCreate(&e0));
    SC_CUDA(cudaEventCreate(&e1));
    // warm-up launch, then the timed one
    fma_rate_kernel<<<grid, CAL_THREADS, 0, s>>>(nullptr, iters / 8 + 1, 0.999f, 1e-3f);
    cudaEventRecord(e0, s);
    fma_rate_kernel<<<grid, CAL_THREADS, 0, s>>>(nullptr, iters, 0.999f, 1e-3f);
    cudaEventRecord(e1, s);
    sc::count_launches(2);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    SC_CUDA(e);
    SC_CUDA(cudaGetLastError());
    const double fmas = (double)grid * CAL_THREADS * (double)iters * NCHAIN * UNROLL;
    *lane_fma_per_s = ms > 0.f ? fmas / (ms * 1e-3) : 0.0;
    if (ms_out) *ms_out = ms;
    return SC_OK;
}
