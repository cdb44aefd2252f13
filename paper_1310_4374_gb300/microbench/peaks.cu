// Issue-rate microbenchmarks behind the ALU roofline of the pair kernels: FP32 FFMA,
// packed FFMA2 (f32x2), MUFU rsqrt and FP64 DFMA, each as 8 (4 for DFMA) independent
// dependency chains per thread over a grid of 8 CTAs of 256 threads per SM.
// Build and run:  nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 peaks.cu -o peaks && ./peaks
#include <cstdio>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA %s at %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)

__global__ void k_ffma(float* out, int iters, float a, float b) {
    float x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            x0 = fmaf(x0, a, b); x1 = fmaf(x1, a, b); x2 = fmaf(x2, a, b); x3 = fmaf(x3, a, b);
            x4 = fmaf(x4, a, b); x5 = fmaf(x5, a, b); x6 = fmaf(x6, a, b); x7 = fmaf(x7, a, b);
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

__global__ void k_ffma2(float* out, int iters, float a, float b) {
    float2 A = make_float2(a, a), B = make_float2(b, b);
    float2 x0 = make_float2(threadIdx.x, 1), x1 = make_float2(2, 3), x2 = make_float2(4, 5), x3 = make_float2(6, 7);
    float2 x4 = make_float2(8, 9), x5 = make_float2(10, 11), x6 = make_float2(12, 13), x7 = make_float2(14, 15);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            x0 = __ffma2_rn(x0, A, B); x1 = __ffma2_rn(x1, A, B); x2 = __ffma2_rn(x2, A, B); x3 = __ffma2_rn(x3, A, B);
            x4 = __ffma2_rn(x4, A, B); x5 = __ffma2_rn(x5, A, B); x6 = __ffma2_rn(x6, A, B); x7 = __ffma2_rn(x7, A, B);
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0.x + x1.x + x2.x + x3.x + x4.x + x5.x + x6.x + x7.x + x0.y + x7.y;
}

__device__ __forceinline__ float rsq(float x) { float y; asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }

__global__ void k_mufu(float* out, int iters) {
    float x0 = threadIdx.x + 1.f, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            x0 = rsq(x0); x1 = rsq(x1); x2 = rsq(x2); x3 = rsq(x3); x4 = rsq(x4); x5 = rsq(x5); x6 = rsq(x6); x7 = rsq(x7);
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

__global__ void k_dfma(double* out, int iters, double a, double b) {
    double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}


int main() {
    int dev = 0;
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, dev));
    int clk = 0;
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
    printf("device %s SMs %d max clock %d MHz\n", prop.name, prop.multiProcessorCount, clk / 1000);
    const int nsm = prop.multiProcessorCount, threads = 256, blocks = nsm * 8;
    const size_t n = (size_t)blocks * threads;
    float* out;
    double* outd;
    CK(cudaMalloc(&out, n * sizeof(float)));
    CK(cudaMalloc(&outd, n * sizeof(double)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto timeit = [&](auto launch, const char* name, double ops) {
        launch();
        cudaDeviceSynchronize();
        cudaEventRecord(e0);
        for (int r = 0; r < 5; ++r) launch();
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double s = ms / 5 * 1e-3;
        printf("%-18s %8.3f ms  %8.3f T lane-ops/s  %7.2f per SM per clock at %d MHz\n", name, ms / 5,
               ops / s * 1e-12, ops / s / nsm / (clk * 1e3), clk / 1000);
    };
    const int it = 2000;
    timeit([&] { k_ffma<<<blocks, threads>>>(out, it, 0.999f, 0.001f); }, "ffma", (double)n * it * 128);
    timeit([&] { k_ffma2<<<blocks, threads>>>(out, it, 0.999f, 0.001f); }, "ffma2 (per lane)", (double)n * it * 128);
    timeit([&] { k_mufu<<<blocks, threads>>>(out, it); }, "mufu rsqrt", (double)n * it * 32);
    timeit([&] { k_dfma<<<blocks, threads>>>(outd, 200, 0.999, 0.001); }, "dfma", (double)n * 200 * 16);
    CK(cudaGetLastError());
    return 0;
}
