// measure.cu -- uaamg_measure_fp64_fma: the FP64 fused multiply-add rate of the device, the
// denominator of the roofline of FP64-bound kernels (the subgraph-reshaping pair kernel).
//
// Every thread runs `chains` independent FMA recurrences x = x * a + b for `iters` steps
// (a slightly below one and b small, so the values stay finite and normal); the grid is a
// whole number of resident blocks on every SM.  One chain per thread measures the latency-
// bound rate, eight the throughput of the FP64 pipe.
#include "common.cuh"

namespace uaamg {

template <int C>
__global__ void __launch_bounds__(kThreads) k_fp64_fma(int iters, double a, double b,
                                                       double* sink) {
    double x[C];
#pragma unroll
    for (int c = 0; c < C; c++) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < C; c++) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < C; c++) s += x[c];
    if (s == -1.0) sink[threadIdx.x] = s;  // never true; keeps the chains live
}

template <int C>
static int time_fma(int blocks, int iters, double* seconds) {
    double* sink = nullptr;
    cudaEvent_t e0, e1;
    int st = check_cuda(cudaMalloc(&sink, sizeof(double) * kThreads));
    if (st) return st;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fp64_fma<C><<<blocks, kThreads>>>(16, 0.999999, 1e-7, sink);  // warm-up
    cudaEventRecord(e0);
    k_fp64_fma<C><<<blocks, kThreads>>>(iters, 0.999999, 1e-7, sink);
    cudaEventRecord(e1);
    st = check_cuda(cudaEventSynchronize(e1));
    float ms = 0.f;
    if (st == UAAMG_OK) st = check_cuda(cudaEventElapsedTime(&ms, e0, e1));
    *seconds = ms * 1e-3;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    return st;
}

}  // namespace uaamg

using namespace uaamg;

extern "C" int uaamg_measure_fp64_fma(int32_t chains, double* fma_per_s) {
    if (!fma_per_s || (chains != 1 && chains != 8)) return UAAMG_ERR_INVALID_ARG;
    int dev = 0, sms = 0, per_sm = 0;
    int st = check_cuda(cudaGetDevice(&dev));
    if (st == UAAMG_OK)
        st = check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (st == UAAMG_OK)
        st = check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, chains == 8 ? (const void*)k_fp64_fma<8> : (const void*)k_fp64_fma<1>,
            kThreads, 0));
    if (st) return st;
    const int blocks = (per_sm > 0 ? per_sm : 1) * sms;
    const int iters = 1 << 14;
    double sec = 0.0;
    st = chains == 8 ? time_fma<8>(blocks, iters, &sec) : time_fma<1>(blocks, iters, &sec);
    if (st) return st;
    *fma_per_s = sec > 0.0 ? (double)blocks * kThreads * chains * (double)iters / sec : 0.0;
    return UAAMG_OK;
}
