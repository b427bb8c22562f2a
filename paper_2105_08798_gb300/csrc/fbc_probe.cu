// Peak-rate probes: the FP32 and FP64 fused multiply-add rates of this GPU, measured rather than
// derived from unit counts, for the rooflines of the CUDA-core contraction forms.
//
// Every thread runs eight independent FMA chains (enough to cover the pipes' latency) for a fixed
// number of iterations; the grid is 8 CTAs of 256 threads per SM.  The chains' values are folded
// into one store per thread under a condition the compiler cannot prove false, so no work is
// removed.  The rate counts 2 flops per FMA.

#include <cuda_runtime.h>

#include "fbc_internal.cuh"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_probe_fma(int iters, T seed, T* __restrict__ sink) {
    T a[8];
#pragma unroll
    for (int c = 0; c < 8; c++) a[c] = seed + (T)(threadIdx.x + c);
    const T m = (T)0.999999, d = (T)1e-7;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < 8; c++) a[c] = fma(a[c], m, d);
    }
    T s = (T)0;
#pragma unroll
    for (int c = 0; c < 8; c++) s += a[c];
    if (s == seed) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never true for the seeds used
}

}  // namespace

extern "C" int fbc_measure_fma_peak(int32_t fp64, double* tflops, void* stream) {
    fbc::report_error(FBC_OK, "");
    if (!tflops) return fbc::report_error(FBC_ERR_INVALID_ARG, "tflops is NULL");
    *tflops = 0.0;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, n_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e) return fbc::report_error(FBC_ERR_CUDA, cudaGetErrorString(e));
    const int blocks = 8 * n_sm, threads = 256;
    const int iters = fp64 ? 1 << 12 : 1 << 16;  // about 10 ms and 15 ms of work on this part
    void* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaMalloc(&sink, (size_t)blocks * threads * 8))) return fbc::report_error(FBC_ERR_OOM, "probe sink");
    if (!(e = cudaEventCreate(&e0)) && !(e = cudaEventCreate(&e1))) {
        for (int rep = 0; rep < 2 && !e; rep++) {  // the first launch warms up clocks and caches
            if ((e = cudaEventRecord(e0, st))) break;
            if (fp64)
                k_probe_fma<double><<<blocks, threads, 0, st>>>(iters, 3.0, (double*)sink);
            else
                k_probe_fma<float><<<blocks, threads, 0, st>>>(iters, 3.0f, (float*)sink);
            if ((e = cudaGetLastError())) break;
            if ((e = cudaEventRecord(e1, st))) break;
            if ((e = cudaEventSynchronize(e1))) break;
        }
        float ms = 0.f;
        if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
        if (!e && ms > 0.f) *tflops = 2.0 * 8.0 * (double)iters * blocks * threads / (ms * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return e ? fbc::report_error(FBC_ERR_CUDA, cudaGetErrorString(e)) : FBC_OK;
}
