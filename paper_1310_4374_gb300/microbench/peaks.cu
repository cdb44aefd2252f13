// Issue-rate microbenchmarks behind the ALU roofline of the pair kernels: FP32 FFMA,
// packed FFMA2 (f32x2), MUFU rsqrt and FP64 DFMA, each as 8 (4 for DFMA) independent
// dependency chains per thread over a grid of 8 CTAs of 256 threads per SM; then the
// charge kernel's far pair loop alone, with and without its rsqrt.
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

// The far-unit pair loop of the charge kernel without its surroundings: each thread holds
// 4 targets as 2 packed pairs, read from shared memory (so that the compiler cannot share
// work between them), and runs over 128 sources in shared memory (two broadcast float4
// loads per source): 13 float32 lane operations and one rsqrt per pair, every result
// used, at the kernel's occupancy (4 CTAs of 128 threads per SM).  kMufu = false keeps
// every float32 operation and drops the rsqrt (its input is used as is).
template <bool kMufu>
__device__ __forceinline__ void mix_term(const float4* s, int src, const float2 (&nx)[2], const float2 (&ny)[2],
                                         const float2 (&nz)[2], float2 (&qr)[2], float2 (&gx)[2], float2 (&gy)[2],
                                         float2 (&gz)[2]) {
    const float4 A = s[2 * src], B = s[2 * src + 1];
    const float2 sq = make_float2(B.z, B.w);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const float2 ex = __fadd2_rn(make_float2(A.x, A.y), nx[j]);
        const float2 ey = __fadd2_rn(make_float2(A.z, A.w), ny[j]);
        const float2 ez = __fadd2_rn(make_float2(B.x, B.y), nz[j]);
        float2 r2 = __fmul2_rn(ex, ex);
        r2 = __ffma2_rn(ey, ey, r2);
        r2 = __ffma2_rn(ez, ez, r2);
        const float2 ri = kMufu ? make_float2(rsq(r2.x), rsq(r2.y)) : r2;
        qr[j] = __fmul2_rn(sq, ri);
        const float2 w = __fmul2_rn(qr[j], __fmul2_rn(ri, ri));
        gx[j] = __ffma2_rn(ex, w, gx[j]);
        gy[j] = __ffma2_rn(ey, w, gy[j]);
        gz[j] = __ffma2_rn(ez, w, gz[j]);
    }
}

template <bool kMufu>
__global__ void __launch_bounds__(128, 4) k_pairmix(float* out, int iters) {
    __shared__ float4 s[256];
    __shared__ float2 s_t[3][2][128];
    const int tid = threadIdx.x;
    for (int i = tid; i < 256; i += blockDim.x) {
        const float v = 0.001f * (float)(i >> 1);
        s[i] = (i & 1) ? make_float4(v, v, 1.f, -1.f) : make_float4(v, -v, 0.5f * v, -0.5f * v);
    }
    const float t = 1e-4f * (float)tid;
    for (int j = 0; j < 2; ++j) {                  // every target at least 0.7 from every source
        s_t[0][j][tid] = make_float2(-1.f - t, -1.1f - t - j * t);
        s_t[1][j][tid] = make_float2(-1.2f + t, -1.3f - j * t);
        s_t[2][j][tid] = make_float2(-1.4f - t - j * t, -1.5f + t);
    }
    __syncthreads();
    float2 ph[2], pb[2], gx[2], gy[2], gz[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) ph[j] = pb[j] = gx[j] = gy[j] = gz[j] = make_float2(0.f, 0.f);
    for (int it = 0; it < iters; ++it) {
        float2 nx[2], ny[2], nz[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            nx[j] = s_t[0][j][tid];
            ny[j] = s_t[1][j][tid];
            nz[j] = s_t[2][j][tid];
        }
#pragma unroll 2
        for (int src = 0; src < 128; src += 2) {
            float2 q0[2], q1[2];
            mix_term<kMufu>(s, src, nx, ny, nz, q0, gx, gy, gz);
            mix_term<kMufu>(s, src + 1, nx, ny, nz, q1, gx, gy, gz);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                ph[j] = __fadd2_rn(ph[j], q0[j]);
                pb[j] = __fadd2_rn(pb[j], q1[j]);
            }
        }
    }
    // every lane of every sum is used, or the compiler drops the dead halves of the packed
    // instructions (fewer than 13 operations per pair would be timed)
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < 2; ++j)
        acc += ph[j].x + ph[j].y + pb[j].x + pb[j].y + gx[j].x + gx[j].y + gy[j].x + gy[j].y + gz[j].x + gz[j].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
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
    // pair loop: 13 float32 lane operations per pair, 4 targets x 128 sources per thread per iteration
    // (unused dynamic shared memory keeps exactly 4 CTAs on an SM, as in the kernel)
    const int mb = nsm * 4, mit = 100, dyn = 228 * 1024 / 4 - 8 * 1024;
    cudaFuncSetAttribute(k_pairmix<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    cudaFuncSetAttribute(k_pairmix<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    const double mix_ops = (double)mb * 128 * 4 * 128 * mit * 13;
    timeit([&] { k_pairmix<true><<<mb, 128, dyn>>>(out, mit); }, "pair loop", mix_ops);
    timeit([&] { k_pairmix<false><<<mb, 128, dyn>>>(out, mit); }, "pair loop, no rsqrt", mix_ops);
    CK(cudaGetLastError());
    return 0;
}
