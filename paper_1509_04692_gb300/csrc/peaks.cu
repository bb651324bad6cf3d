// peaks.cu -- measured instruction-rate peaks of the FP32 and FP64 pipes.
//
// The set kernels are ALU work (FP32 for the certified filter, FP64 for the
// contract's updates and re-checks), so their roofline is the rate at which
// the GPU retires fused multiply-adds.  Instead of multiplying nominal unit
// counts by a nominal clock, this file times a chain of independent fused
// multiply-adds on every SM with CUDA events, at whatever clock the GPU runs
// (the caller samples the clock alongside).
#include <cuda_runtime.h>

#include <vector>

#include "../../include/hpmc.h"

namespace {

constexpr int kAcc = 8;                 // independent accumulators per thread
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;         // 2048 resident threads per SM

template <typename T>
__device__ __forceinline__ T fma_rn(T a, T b, T c);
template <>
__device__ __forceinline__ float fma_rn<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <>
__device__ __forceinline__ double fma_rn<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

// x <- x * m + c per accumulator: x converges to c / (1 - m), so nothing
// overflows or goes subnormal; the sum is stored so nothing is removed.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chain(uint32_t iters, T m, T c, T* out)
{
    T x[kAcc];
#pragma unroll
    for (int k = 0; k < kAcc; ++k) x[k] = (T)(threadIdx.x + k);
    for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kAcc; ++k) x[k] = fma_rn<T>(x[k], m, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kAcc; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int run_chain(uint32_t iters, int reps, double* flops_per_s, double* ms_out)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        (void)cudaGetLastError();
        return HPMC_ERR_CUDA;
    }
    const uint32_t blocks = (uint32_t)sms * kBlocksPerSM;
    T* out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * (size_t)blocks * kThreads) != cudaSuccess) {
        (void)cudaGetLastError();
        return HPMC_ERR_OOM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = 0;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = HPMC_ERR_CUDA;
    cudaStream_t st = nullptr;
    if (!rc && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) rc = HPMC_ERR_CUDA;
    const T m = (T)0.999999, c = (T)1e-6;
    double best = 0.0, best_ms = 0.0;
    if (!rc) {
        k_fma_chain<T><<<blocks, kThreads, 0, st>>>(iters / 8 + 1, m, c, out);      // warm-up
        for (int r = 0; r < reps && !rc; ++r) {
            cudaEventRecord(e0, st);
            k_fma_chain<T><<<blocks, kThreads, 0, st>>>(iters, m, c, out);
            cudaEventRecord(e1, st);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
                !(ms > 0.f)) {
                rc = HPMC_ERR_CUDA;
                break;
            }
            const double flops = 2.0 * kAcc * (double)iters * (double)blocks * kThreads;
            const double rate = flops / (ms * 1e-3);
            if (rate > best) { best = rate; best_ms = ms; }
        }
    }
    if (cudaGetLastError() != cudaSuccess && !rc) rc = HPMC_ERR_CUDA;
    if (st) cudaStreamDestroy(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (rc) return rc;
    *flops_per_s = best;
    if (ms_out) *ms_out = best_ms;
    return 0;
}

}  // namespace

extern "C" int hpmc_measure_fma_peak(int fp64, uint32_t iters, int reps, double* flops_per_s, double* ms)
{
    if (!flops_per_s || iters == 0 || reps < 1 || reps > 1000) return HPMC_ERR_INVALID_ARG;
    return fp64 ? run_chain<double>(iters, reps, flops_per_s, ms) : run_chain<float>(iters, reps, flops_per_s, ms);
}
