// Measured FP64 arithmetic throughput of the device (lb_fp64_peak).
//
// The FP64 build of the step is bound by the FP64 pipe, not by HBM, so its
// roofline needs that pipe's throughput.  This file measures it: every
// thread of a grid that fills the GPU runs kChains independent dependency
// chains of one FP64 operation (DFMA, DADD or DMUL) for `iters` rounds, so
// the pipe always has independent work; the count of operations over the
// event-timed duration is the throughput.  The chains' results are summed
// and stored so that the compiler keeps every operation.
#include <cuda_runtime.h>

#include "../../include/lbfe.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <int KIND>
__global__ void __launch_bounds__(kThreads) fp64_chain_kernel(int iters, double seed, double* sink)
{
    double v[kChains];
    const double b = 1.0 + 1e-16 * double(threadIdx.x);  // keeps values finite and distinct
    const double c = 1e-300 * seed;
#pragma unroll
    for (int k = 0; k < kChains; ++k) v[k] = seed + double(k + blockIdx.x);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < kChains; ++k) {
                if (KIND == 0)
                    v[k] = fma(v[k], b, c);
                else if (KIND == 1)
                    v[k] = v[k] + c;
                else
                    v[k] = v[k] * b;
            }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += v[k];
    if (s == 12345.678) sink[blockIdx.x] = s;  // never true; keeps the chains live
}

template <int KIND>
cudaError_t run_chain(int blocks, int iters, double* sink, cudaStream_t s)
{
    fp64_chain_kernel<KIND><<<blocks, kThreads, 0, s>>>(iters, 1.0, sink);
    return cudaGetLastError();
}

}  // namespace

extern "C" int lb_fp64_peak(int kind, void* stream, double* ops_per_s)
{
    if (!ops_per_s || kind < 0 || kind > 2) return LB_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LB_ERR_CUDA;
    const int blocks = sms * 8;  // 8 x 256 threads per SM: every scheduler busy
    const int iters = 256;       // 256 x 16 x 8 operations per thread
    double* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = LB_ERR_CUDA;
    float ms = 0.f;
    auto launch = [&]() {
        return kind == 0 ? run_chain<0>(blocks, iters, sink, s)
                         : (kind == 1 ? run_chain<1>(blocks, iters, sink, s)
                                      : run_chain<2>(blocks, iters, sink, s));
    };
    if (cudaMalloc(&sink, sizeof(double) * blocks) != cudaSuccess) return LB_ERR_CUDA;
    if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess &&
        launch() == cudaSuccess &&  // warm-up
        cudaEventRecord(e0, s) == cudaSuccess) {
        bool ok = true;
        for (int k = 0; k < 5 && ok; ++k) ok = launch() == cudaSuccess;
        if (ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
            cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f) {
            const double ops = 5.0 * blocks * kThreads * double(iters) * 16.0 * kChains;
            *ops_per_s = ops / (double(ms) * 1e-3);
            rc = LB_OK;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return rc;
}
