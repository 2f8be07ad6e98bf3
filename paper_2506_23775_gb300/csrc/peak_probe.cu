// Arithmetic-pipe throughput probes (measurement instrument for the roofline
// denominators of the ALU-bound sweep kernels; not part of the method).
//
// Each thread runs kChains independent fused multiply-add chains
// x <- x * a + b for `iters` iterations, on every SM (two CTAs of 256 threads
// per SM), so the pipe, not latency, is the limit: the FP64 pipe for
// pp_fp64_fma_rate, the FP32 pipe for pp_fp32_fma_rate.  Two flops per FMA.
// The result is stored only when `sink` is nonzero (never, at run time), so
// the chains cannot be removed.  Times are CUDA events around `reps` launches
// after one warm-up launch.
//
// pp_fp64_mma_rate does the same with chains of the FP64 tensor-core
// instruction mma.sync m8n8k4 (512 flops per warp instruction).
//
// Built as its own library, libpeak.so, with a plain C ABI:
//   int pp_fp64_fma_rate(int device, int reps, double *tflops, double *ms_per_launch)
//   int pp_fp32_fma_rate(int device, int reps, double *tflops, double *ms_per_launch)
//   int pp_fp64_mma_rate(int device, int reps, double *tflops, double *ms_per_launch)
// return 0 on success, otherwise the CUDA error code.
#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T *out, int iters, T a, T b, int sink) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    if (sink) {
        T s = 0;
#pragma unroll
        for (int c = 0; c < kChains; ++c) s += x[c];
        out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    }
}

template <typename T>
int fma_rate(int device, int reps, int iters, double *tflops, double *ms_per_launch) {
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return (int)e;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return (int)e;
    const int grid = 2 * sms;
    T *out = nullptr;
    e = cudaMalloc(&out, sizeof(T) * grid * kThreads);
    if (e != cudaSuccess) return (int)e;
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    const T a = (T)0.999999, b = (T)1e-7;
    k_fma_chains<T><<<grid, kThreads>>>(out, iters, a, b, 0);
    cudaEventRecord(t0);
    for (int r = 0; r < reps; ++r) k_fma_chains<T><<<grid, kThreads>>>(out, iters, a, b, 0);
    cudaEventRecord(t1);
    e = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFree(out);
    if (e != cudaSuccess) return (int)e;
    const double flops = 2.0 * kChains * (double)iters * grid * kThreads * reps;
    *ms_per_launch = ms / reps;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return 0;
}

// FP64 tensor-core rate: independent chains of mma.sync m8n8k4 (D = A B + C,
// f64, 2 * 8 * 8 * 4 = 512 flops per warp instruction) per warp.
__global__ void __launch_bounds__(kThreads) k_dmma_chains(double *out, int iters, double a, double b, int sink) {
    double c[kChains][2];
#pragma unroll
    for (int k = 0; k < kChains; ++k) c[k][0] = c[k][1] = (double)(threadIdx.x + k) * 1e-3;
    const double av = a * (1.0 + 1e-3 * (threadIdx.x & 31)), bv = b;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                         : "+d"(c[k][0]), "+d"(c[k][1])
                         : "d"(av), "d"(bv));
    }
    if (sink) {
        double s = 0;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += c[k][0] + c[k][1];
        out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    }
}

int dmma_rate(int device, int reps, int iters, double *tflops, double *ms_per_launch) {
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return (int)e;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return (int)e;
    const int grid = 2 * sms;
    double *out = nullptr;
    e = cudaMalloc(&out, sizeof(double) * grid * kThreads);
    if (e != cudaSuccess) return (int)e;
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    k_dmma_chains<<<grid, kThreads>>>(out, iters, 1e-3, 1e-3, 0);
    cudaEventRecord(t0);
    for (int r = 0; r < reps; ++r) k_dmma_chains<<<grid, kThreads>>>(out, iters, 1e-3, 1e-3, 0);
    cudaEventRecord(t1);
    e = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFree(out);
    if (e != cudaSuccess) return (int)e;
    const double flops = 512.0 * kChains * (double)iters * grid * (kThreads / 32) * reps;
    *ms_per_launch = ms / reps;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return 0;
}

}  // namespace

extern "C" int pp_fp64_mma_rate(int device, int reps, double *tflops, double *ms_per_launch) {
    return dmma_rate(device, reps, 1 << 12, tflops, ms_per_launch);
}

extern "C" int pp_fp64_fma_rate(int device, int reps, double *tflops, double *ms_per_launch) {
    return fma_rate<double>(device, reps, 1 << 14, tflops, ms_per_launch);
}

extern "C" int pp_fp32_fma_rate(int device, int reps, double *tflops, double *ms_per_launch) {
    return fma_rate<float>(device, reps, 1 << 18, tflops, ms_per_launch);
}
