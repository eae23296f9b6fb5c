// fd_probe.cu -- measured binary64 arithmetic rate of the current GPU, the
// denominator of the binary64 kernels' roofline (fd_fp64_peak).
//
// A grid of 8 blocks of 256 threads per SM runs eight independent chains of
// dependent binary64 FMAs per thread (enough independent work to keep the FP64
// pipe issuing every cycle), timed with CUDA events on a private stream after
// one untimed launch.  Each FMA counts two flops.
#include <cuda_runtime.h>

#include "../../include/fdgb300.h"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

__global__ void __launch_bounds__(kThreads) k_dfma_loop(double a, double b, double* __restrict__ out) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3 + c;
    for (int i = 0; i < kIters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = __fma_rn(x[c], a, b);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

}  // namespace

extern "C" int fd_fp64_peak(double* flops_per_s, void* scratch, size_t scratch_bytes) {
    if (!flops_per_s || !scratch) return FD_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FD_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return FD_ECUDA;
    const int blocks = sms * kBlocksPerSm;
    if (scratch_bytes < (size_t)blocks * kThreads * sizeof(double)) return FD_EINVAL;
    double* out = static_cast<double*>(scratch);
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    const int reps = 3;
    if (e == cudaSuccess) {
        k_dfma_loop<<<blocks, kThreads, 0, st>>>(1.0000001, 1e-7, out);  // untimed
        e = cudaEventRecord(e0, st);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) {
            k_dfma_loop<<<blocks, kThreads, 0, st>>>(1.0000001, 1e-7, out);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess || ms <= 0.f) return FD_ECUDA;
    const double fmas = (double)blocks * kThreads * kIters * kChains * reps;
    *flops_per_s = 2.0 * fmas / (ms * 1e-3);
    return FD_OK;
}
