// mp_probe.cu -- device rate probes behind mp_probe_rates(): the float64 FMA
// rate (the roofline of the float64 path) and the hardware float64 -> float32
// conversion rate (which decides whether per-cell conversions may use the
// float64 pipe).  Each probe is a fixed amount of independent work per thread,
// timed with CUDA events.
#include "mp_internal.h"

namespace mp {

namespace {

constexpr int kIters = 4096;

__global__ void k_probe_dfma(double *out, double a, double b)
{
    double x0 = threadIdx.x * 1e-3, x1 = x0 + 1.0, x2 = x0 + 2.0, x3 = x0 + 3.0;
    double x4 = x0 + 4.0, x5 = x0 + 5.0, x6 = x0 + 6.0, x7 = x0 + 7.0;
#pragma unroll 4
    for (int k = 0; k < kIters; ++k) {
        x0 = fma(x0, a, b);
        x1 = fma(x1, a, b);
        x2 = fma(x2, a, b);
        x3 = fma(x3, a, b);
        x4 = fma(x4, a, b);
        x5 = fma(x5, a, b);
        x6 = fma(x6, a, b);
        x7 = fma(x7, a, b);
    }
    const double s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == 1234.5) out[0] = s;  // keeps the work alive
}

__global__ void k_probe_cvt(float *out, double seed)
{
    // inputs walk through distinct bit patterns (64-bit integer steps), so no
    // conversion can be hoisted out of the loop; the integer steps run on the
    // ALU pipe next to the conversions
    long long b0 = __double_as_longlong(seed + threadIdx.x), b1 = b0 + 7919, b2 = b0 + 104729, b3 = b0 + 1299709;
    float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
#pragma unroll 4
    for (int k = 0; k < kIters; ++k) {
        acc0 += __double2float_rn(__longlong_as_double(b0));
        acc1 += __double2float_rn(__longlong_as_double(b1));
        acc2 += __double2float_rn(__longlong_as_double(b2));
        acc3 += __double2float_rn(__longlong_as_double(b3));
        b0 += 4096;
        b1 += 4096;
        b2 += 4096;
        b3 += 4096;
    }
    const float s = acc0 + acc1 + acc2 + acc3;
    if (s == 1234.5f) out[0] = s;
}

}  // namespace

}  // namespace mp

extern "C" MP_API mp_status mp_probe_rates(double *fp64_tflops, double *cvt_f64_f32_per_s)
{
    using namespace mp;
    if (!fp64_tflops || !cvt_f64_f32_per_s) return set_error(MP_ERR_INVALID_ARG, "NULL argument");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return set_error(MP_ERR_CUDA, "no CUDA device");
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double *dout = nullptr;
    if (cudaMalloc(&dout, 16) != cudaSuccess) return set_error(MP_ERR_OOM, "probe buffer");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = sms * 8, threads = 256;
    float ms = 0.f;
    // float64 FMA
    k_probe_dfma<<<blocks, threads>>>(dout, 0.999999, 1e-7);
    cudaEventRecord(e0);
    k_probe_dfma<<<blocks, threads>>>(dout, 0.999999, 1e-7);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    *fp64_tflops = 2.0 * 8.0 * kIters * (double)blocks * threads / (ms * 1e-3) / 1e12;
    // float64 -> float32 conversion
    k_probe_cvt<<<blocks, threads>>>(reinterpret_cast<float *>(dout), 1.25);
    cudaEventRecord(e0);
    k_probe_cvt<<<blocks, threads>>>(reinterpret_cast<float *>(dout), 1.25);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    *cvt_f64_f32_per_s = 4.0 * kIters * (double)blocks * threads / (ms * 1e-3);
    cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(dout);
    if (err != cudaSuccess) return set_error(MP_ERR_CUDA, "probe: %s", cudaGetErrorString(err));
    return MP_OK;
}
