// mufu_rates.cu -- issue rates of the special-function (MUFU) instructions the pair kernels use, of FFMA
// (scalar and two-wide) and of DFMA (the FP64 pipe the FP64 direct sum runs on), in thread operations per
// clock per SM.  Eight independent dependency chains per thread, 8 CTAs of 256 threads per SM, CUDA events;
// prints one JSON line.  A measurement tool, not part of the library: the rates are the denominators of the
// pair kernels' rooflines.
//
// Build and run: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o mufu_rates mufu_rates.cu && ./mufu_rates
#include <cstdio>

#include <cuda_runtime.h>

__device__ __forceinline__ float op_rsqrt(float x) {
    float y;
    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float op_ex2(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float op_rcp(float x) {
    float y;
    asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ unsigned long long op_fma2(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
    unsigned long long d;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// MODE 0 rsqrt, 1 ex2 (of a negative argument: the chains stay finite), 2 rcp (alternating with a negation,
// so no pair of steps cancels), 3 FFMA, 4 two-wide FFMA (fma.rn.f32x2: one instruction, two FMAs; the rate
// counts FMAs), 5 DFMA (FP64 fused multiply-add).
template <int MODE>
__global__ void chains(float* out, int iters, float seed) {
    float a[8];
    double dd[8];
    unsigned long long p[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        a[i] = seed + threadIdx.x * 1e-3f + i;
        dd[i] = (double)a[i];
        p[i] = __float_as_uint(a[i]) | ((unsigned long long)__float_as_uint(a[i] + 1.f) << 32);
    }
    const unsigned long long k1 = 0x3f8000d23f8000d2ull, k2 = 0x3f0000003f000000ull;  // (1.000025, ..), (0.5, 0.5)
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (MODE == 0) a[i] = op_rsqrt(a[i]);
            else if (MODE == 1) a[i] = op_ex2(-a[i]);
            else if (MODE == 2) a[i] = op_rcp(a[i] + 1.0f);
            else if (MODE == 3) a[i] = fmaf(a[i], 1.0001f, 0.5f);
            else if (MODE == 4) p[i] = op_fma2(p[i], k1, k2);
            else dd[i] = fma(dd[i], 0.99990000000001, 0.5);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i)
        s += a[i] + __uint_as_float((unsigned)p[i]) + __uint_as_float((unsigned)(p[i] >> 32)) + (float)dd[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // one element per thread: in bounds by construction
}

int main() {
    int dev = 0, sms = 0, clk_khz = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
    const int blocks = sms * 8, threads = 256, iters = 4096;
    float* out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * blocks * threads) != cudaSuccess) return 1;
    constexpr int kModes = 6;
    const char* names[kModes] = {"rsqrt", "ex2", "rcp", "ffma", "ffma_f32x2", "dfma"};
    double rate[kModes] = {0, 0, 0, 0, 0, 0};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int m = 0; m < kModes; ++m) {
        float best = 1e30f;
        // the FP64 pipe is much slower: fewer iterations keep the DFMA launch short
        const int it_m = m == 5 ? iters / 16 : iters;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0);
            switch (m) {
                case 0: chains<0><<<blocks, threads>>>(out, it_m, 1.5f); break;
                case 1: chains<1><<<blocks, threads>>>(out, it_m, 0.1f); break;
                case 2: chains<2><<<blocks, threads>>>(out, it_m, 1.5f); break;
                case 3: chains<3><<<blocks, threads>>>(out, it_m, 0.5f); break;
                case 4: chains<4><<<blocks, threads>>>(out, it_m, 0.5f); break;
                default: chains<5><<<blocks, threads>>>(out, it_m, 0.5f); break;
            }
            cudaEventRecord(e1);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best) best = ms;
        }
        const double ops = (double)blocks * threads * it_m * 8 * (m == 4 ? 2 : 1);
        rate[m] = ops / (best * 1e-3) / sms / (clk_khz * 1e3);
    }
    const cudaError_t err = cudaGetLastError();
    printf("{\"suite\": \"mufu\", \"sms\": %d, \"clock_mhz\": %d, \"unit\": \"thread ops/clk/SM at the nominal clock\"",
           sms, clk_khz / 1000);
    for (int m = 0; m < kModes; ++m) printf(", \"%s\": %.2f", names[m], rate[m]);
    printf(", \"status\": \"%s\"}\n", cudaGetErrorString(err));
    cudaFree(out);
    return err == cudaSuccess ? 0 : 1;
}
