// Throughput probes of the GPU the library runs on: binary64 and binary32 FMA rates and
// device-memory copy bandwidth.  They give the denominators of the stage kernels' roofline
// (the binary64 stage kernels are bound by the binary64 pipe, the binary32 ones by HBM).
#include "../../include/pf.h"
#include "pf_internal.cuh"

#include <cuda_runtime.h>

namespace {

// 8 independent FMA chains per thread; the result is written so nothing is dead code.
template <typename T>
__global__ void k_fma_chains(T* out, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = (T)(threadIdx.x + c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < 8; ++c) x[c] = x[c] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_copy2(const double2* __restrict__ a, double2* __restrict__ b, long long n) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        b[q] = a[q];
}

template <typename T>
static cudaError_t time_fma(int sms, int iters, double* tflops) {
    const int blocks = sms * 8, threads = 256;
    T* out = nullptr;
    cudaError_t e = cudaMalloc(&out, sizeof(T) * blocks * threads);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma_chains<T><<<blocks, threads>>>(out, 16, (T)1.0000001, (T)1e-9);
    cudaEventRecord(e0);
    k_fma_chains<T><<<blocks, threads>>>(out, iters, (T)1.0000001, (T)1e-9);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    pfgb::count_launch(2);
    *tflops = 2.0 * 8 * (double)iters * blocks * threads / (ms * 1e-3) / 1e12;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return e;
}

}  // namespace

extern "C" pf_status pf_measure_peaks(double* fp64_tflops, double* fp32_tflops, double* copy_gbs) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PF_E_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PF_E_CUDA;
    double v = 0.0;
    if (fp64_tflops) {
        if (time_fma<double>(sms, 4096, &v) != cudaSuccess) return PF_E_CUDA;
        *fp64_tflops = v;
    }
    if (fp32_tflops) {
        if (time_fma<float>(sms, 65536, &v) != cudaSuccess) return PF_E_CUDA;
        *fp32_tflops = v;
    }
    if (copy_gbs) {
        const long long n = 1LL << 27;  // 2 GiB per buffer
        double2 *a = nullptr, *b = nullptr;
        if (cudaMalloc(&a, n * sizeof(double2)) != cudaSuccess) return PF_E_OOM;
        if (cudaMalloc(&b, n * sizeof(double2)) != cudaSuccess) { cudaFree(a); return PF_E_OOM; }
        cudaMemset(a, 0, n * sizeof(double2));
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = 1e30f;
        cudaError_t e = cudaSuccess;
        for (int r = 0; r < 5 && e == cudaSuccess; ++r) {
            cudaEventRecord(e0);
            k_copy2<<<sms * 8, 256>>>(a, b, n);
            cudaEventRecord(e1);
            e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) best = ms;
        }
        pfgb::count_launch(5);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFree(a);
        cudaFree(b);
        if (e != cudaSuccess) return PF_E_CUDA;
        *copy_gbs = 2.0 * n * sizeof(double2) / (best * 1e-3) / 1e9;
    }
    return PF_OK;
}
