// FP32 throughput probe: independent FFMA chains, the same with packed FFMA2,
// and FFMA interleaved with integer multiplies (Philox-like work); the FFMA
// rate sustained over 1000 back-to-back launches (a quarter second); and the
// XU (special-function unit) rate on independent reciprocal-square-root
// chains.  Prints one JSON line: TFLOP/s (2 flops per fused multiply-add) and
// XU operations per second.  It checks the FP32 roofline denominator used for
// the rollout kernel (152 SMs x 128 lanes x 2 x clock) and shows whether the
// packed form raises it.
#include <cstdio>
#include <cuda_runtime.h>

constexpr int CH = 8;   // independent chains per thread

__global__ void k_ffma(float* out, int iters, float a, float b) {
    float x[CH];
    for (int i = 0; i < CH; ++i) x[i] = threadIdx.x * 1e-3f + i;
    for (int n = 0; n < iters; ++n)
#pragma unroll
        for (int i = 0; i < CH; ++i) x[i] = fmaf(x[i], a, b);
    float s = 0.0f;
    for (int i = 0; i < CH; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_ffma2(float* out, int iters, float a, float b) {
    float2 x[CH];
    for (int i = 0; i < CH; ++i) x[i] = make_float2(threadIdx.x * 1e-3f + i, i * 0.5f);
    const float2 A = make_float2(a, a), B = make_float2(b, b);
    for (int n = 0; n < iters; ++n)
#pragma unroll
        for (int i = 0; i < CH; ++i) x[i] = __ffma2_rn(x[i], A, B);
    float s = 0.0f;
    for (int i = 0; i < CH; ++i) s += x[i].x + x[i].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_mix(float* out, int iters, float a, float b) {
    float x[CH];
    unsigned u[CH];
    for (int i = 0; i < CH; ++i) {
        x[i] = threadIdx.x * 1e-3f + i;
        u[i] = threadIdx.x + i;
    }
    for (int n = 0; n < iters; ++n)
#pragma unroll
        for (int i = 0; i < CH; ++i) {
            x[i] = fmaf(x[i], a, b);
            u[i] = (u[i] ^ 0x9E3779B9u) * 0xD2511F53u;
        }
    float s = 0.0f;
    for (int i = 0; i < CH; ++i) s += x[i] + (float)u[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_xu(float* out, int iters, float a) {
    float x[CH];
    for (int i = 0; i < CH; ++i) x[i] = 1.0f + threadIdx.x * 1e-3f + i;
    for (int n = 0; n < iters; ++n)
#pragma unroll
        for (int i = 0; i < CH; ++i) x[i] = rsqrtf(x[i]) + a;   // one XU op (+ one add) per step
    float s = 0.0f;
    for (int i = 0; i < CH; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int main() {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess) return 1;
    const int blocks = sms * 8, threads = 256, iters = 1 << 14;
    float* out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * blocks * threads) != cudaSuccess) return 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double tf[3] = {0, 0, 0};
    for (int kind = 0; kind < 3; ++kind) {
        for (int rep = 0; rep < 4; ++rep) {   // the last of 4 launches is kept
            cudaEventRecord(e0);
            if (kind == 0) k_ffma<<<blocks, threads>>>(out, iters, 0.999f, 1e-3f);
            if (kind == 1) k_ffma2<<<blocks, threads>>>(out, iters, 0.999f, 1e-3f);
            if (kind == 2) k_mix<<<blocks, threads>>>(out, iters, 0.999f, 1e-3f);
            cudaEventRecord(e1);
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double fmas = (double)blocks * threads * iters * CH * (kind == 1 ? 2 : 1);
            tf[kind] = 2.0 * fmas / (ms * 1e-3) / 1e12;
        }
    }
    // sustained: 1000 launches back to back, one pair of events around them
    const int n_sus = 1000, it_sus = 1 << 12;
    cudaEventRecord(e0);
    for (int rep = 0; rep < n_sus; ++rep) k_ffma<<<blocks, threads>>>(out, it_sus, 0.999f, 1e-3f);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms_sus = 0.0f;
    cudaEventElapsedTime(&ms_sus, e0, e1);
    const double tf_sus = 2.0 * (double)blocks * threads * it_sus * CH * n_sus / (ms_sus * 1e-3) / 1e12;
    // XU: reciprocal square roots per second (the last of 4 launches)
    double xu = 0.0;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0);
        k_xu<<<blocks, threads>>>(out, iters / 4, 1e-3f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        xu = (double)blocks * threads * (iters / 4) * CH / (ms * 1e-3);
    }
    const cudaError_t e = cudaGetLastError();
    std::printf("{\"sms\": %d, \"ffma_tflops\": %.3f, \"ffma2_tflops\": %.3f, "
                "\"ffma_with_imul_tflops\": %.3f, \"ffma_sustained_tflops\": %.3f, "
                "\"sustained_ms\": %.1f, \"xu_rsqrt_per_s\": %.4g, \"status\": \"%s\"}\n",
                sms, tf[0], tf[1], tf[2], tf_sus, ms_sus, xu, cudaGetErrorString(e));
    cudaFree(out);
    return e != cudaSuccess;
}
