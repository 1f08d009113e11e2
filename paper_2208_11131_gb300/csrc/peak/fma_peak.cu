// FMA-chain throughput probe: the FP32 and FP64 arithmetic peaks that the benchmark reports the
// stage kernels against (the measured peaks cover HBM copy bandwidth and bf16 GEMMs only).
// Plain CUDA; it reads no device setting and changes none.  Built as its own small library
// (libdgxpeak.so), outside the solver's C ABI.
#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;   // independent accumulators per thread (covers the FMA latency)
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(int iters, T a, T b, T *sink)
{
    T acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (s == (T)-1.2345) sink[blockIdx.x] = s;  // never true for the inputs used; keeps the chains live
}

template <typename T>
int run(int iters, int reps, double *tflops)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_chain_kernel<T>, kThreads, 0) != cudaSuccess)
        return 1;
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    T *sink = nullptr;
    if (cudaMalloc(&sink, blocks * sizeof(T)) != cudaSuccess) return 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const T a = (T)0.999999, b = (T)1e-7;
    fma_chain_kernel<T><<<blocks, kThreads>>>(iters / 8, a, b, sink);  // warm-up
    float best = 1e30f;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0);
        fma_chain_kernel<T><<<blocks, kThreads>>>(iters, a, b, sink);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    const int err = cudaGetLastError() != cudaSuccess;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (err) return 1;
    const double flops = 2.0 * (double)blocks * kThreads * kChains * (double)iters;
    *tflops = flops / (best * 1e-3) / 1e12;
    return 0;
}

}  // namespace

// Best-of-reps FMA throughput in TFLOP/s (2 flops per FMA) of one full-device launch of FMA chains:
// fp64 = 0 for single precision, 1 for double.  Returns 0 on success.
extern "C" int dgx_fma_peak(int fp64, int iters, int reps, double *tflops)
{
    if (!tflops || iters < 8 || reps < 1) return 1;
    return fp64 ? run<double>(iters, reps, tflops) : run<float>(iters, reps, tflops);
}
