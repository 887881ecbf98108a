// peak.cu -- FP32 FMA throughput probe of the current device, used to state
// the ALU roofline the projector kernels are measured against.  Each thread
// runs 16 independent dependent-FMA chains in registers (no memory traffic
// inside the timed loop); the packed variant issues the same lane-FMAs two per
// instruction with __ffma2_rn.
#include <cuda_runtime.h>

#include "../../include/spect.h"

namespace {

constexpr int kChains = 16;
constexpr int kIters = 4096;

__global__ void __launch_bounds__(256) k_ffma(float* out, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_ffma2(float* out, float a, float b)
{
    float2 x[kChains / 2];
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) x[c] = make_float2((float)(threadIdx.x + c) * 1e-3f, (float)c * 1e-3f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains / 2; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) s += x[c].x + x[c].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" spect_status spect_fp32_peak(double* tflops_ffma, double* tflops_ffma2, spect_stream stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SPECT_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SPECT_ECUDA;
    const int blocks = sms * 8, threads = 256;
    float* out = nullptr;
    if (cudaMalloc((void**)&out, sizeof(float) * blocks * threads) != cudaSuccess) return SPECT_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const double flops = 2.0 * kChains * (double)kIters * blocks * threads;
    double best[2] = {0.0, 0.0};
    for (int mode = 0; mode < 2; ++mode) {
        for (int rep = 0; rep < 5; ++rep) {
            cudaEventRecord(e0, st);
            if (mode == 0) k_ffma<<<blocks, threads, 0, st>>>(out, 0.999999f, 1e-6f);
            else k_ffma2<<<blocks, threads, 0, st>>>(out, 0.999999f, 1e-6f);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms > 0.f) {
                const double t = flops / (ms * 1e-3) / 1e12;
                if (t > best[mode]) best[mode] = t;
            }
        }
    }
    cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return SPECT_ECUDA;
    if (tflops_ffma) *tflops_ffma = best[0];
    if (tflops_ffma2) *tflops_ffma2 = best[1];
    return SPECT_OK;
}
