// Arithmetic pipe rates of the current GPU, measured (hzs_pipe_peaks).
//
// The paper has no counterpart: this is the measurement behind the rooflines of
// the ALU-bound kernels (the FP64 Gram-Schmidt, the FP32 error-free arithmetic
// of the mixed-precision Arnoldi), whose peaks are not in any data sheet of the
// part.  Each kernel runs independent dependency chains of one instruction kind
// in every thread of a grid that fills the GPU, long enough (tens of ms) for the
// launch overhead to vanish, and is timed with CUDA events on a private stream.
// Results are written to memory under a run-time condition so that the compiler
// keeps every chain.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace hzs {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma(int iters, float a, float b, float* sink) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma2(int iters, float a, float b, float* sink) {
    unsigned long long x[kChains], A, B;
    asm("mov.b64 %0, {%1, %1};" : "=l"(A) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(B) : "f"(b));
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        const float v = (float)(threadIdx.x + c);
        asm("mov.b64 %0, {%1, %1};" : "=l"(x[c]) : "f"(v));
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(A), "l"(B));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
        s += lo + hi;
    }
    if (s == 12345.678f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_dfma(int iters, double a, double b, float* sink) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678) sink[threadIdx.x] = (float)s;
}

// integer logic and shifts (the ops that split an FP64 word into FP32 pieces):
// a 3-input logic op and a funnel shift per step of each chain
__global__ void __launch_bounds__(kPeakThreads) k_peak_int(int iters, unsigned a, unsigned b, float* sink) {
    unsigned x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 2654435761u + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            unsigned t;
            asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(t) : "r"(x[c]), "r"(a), "r"(b));
            asm volatile("shf.l.wrap.b32 %0, %1, %2, %3;" : "=r"(x[c]) : "r"(t), "r"(x[c]), "r"(b));
        }
    }
    unsigned s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= x[c];
    if (s == 0x12345u) sink[threadIdx.x] = (float)s;
}

// FP64 -> FP32 -> FP64 conversions (two per step of each chain)
__global__ void __launch_bounds__(kPeakThreads) k_peak_f2f(int iters, double a, float* sink) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c) * a;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            float t;
            asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(t) : "d"(x[c]));
            asm volatile("cvt.f64.f32 %0, %1;" : "=d"(x[c]) : "f"(t));
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678) sink[threadIdx.x] = (float)s;
}

// FP32 and FP64 chains interleaved (ratio rf FFMA per DFMA): whether the two pipes overlap
__global__ void __launch_bounds__(kPeakThreads) k_peak_mix(int iters, int rf, float a, float b, double ad, double bd,
                                                           float* sink) {
    float x[kChains];
    double y[2];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c);
    y[0] = threadIdx.x; y[1] = threadIdx.x + 1.0;
    for (int i = 0; i < iters; ++i) {
        y[0] = fma(y[0], ad, bd);
        y[1] = fma(y[1], ad, bd);
        for (int r = 0; r < rf; ++r) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
        }
    }
    float s = (float)(y[0] + y[1]);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) sink[threadIdx.x] = s;
}

}  // namespace hzs

using namespace hzs;

// Times fn (already bound to its arguments) on stream s: one untimed launch, then
// the mean of reps launches; returns ms per launch or a negative value on error.
template <typename F>
static float time_launch(cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, F fn, int reps) {
    fn();
    if (cudaEventRecord(e0, s) != cudaSuccess) return -1.f;
    for (int r = 0; r < reps; ++r) fn();
    if (cudaEventRecord(e1, s) != cudaSuccess) return -1.f;
    if (cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return -1.f;
    return ms / reps;
}

extern "C" hzs_status hzs_pipe_peaks(hzs_pipe_rates* out) {
    if (!out) return HZS_ERR_INVALID_ARG;
    *out = hzs_pipe_rates{};
    int dev = 0, sms = 0, clk_khz = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
        cudaGetLastError();
        return HZS_ERR_CUDA;
    }
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
    cudaGetLastError();
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float* sink = nullptr;
    hzs_status st = HZS_OK;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess || cudaMalloc(&sink, kPeakThreads * sizeof(float)) != cudaSuccess) {
        st = HZS_ERR_CUDA;
    }
    if (st == HZS_OK) {
        const dim3 grid(8 * sms), blk(kPeakThreads);
        const double threads = (double)grid.x * blk.x;
        const int reps = 5;
        const int it32 = 65536, it64 = 1024, itint = 32768, itcvt = 1024, itmix = 2048, rf = 16;
        const float a = 0.999f, b = 1e-3f;
        const double ad = 0.999, bd = 1e-3;
        float ms;
        // every rate is operations per second over the whole GPU (an FMA counts as 2 flops)
        ms = time_launch(s, e0, e1, [&] { k_peak_ffma<<<grid, blk, 0, s>>>(it32, a, b, sink); }, reps);
        out->fp32_tflops = ms > 0 ? 2.0 * threads * it32 * kChains / (ms * 1e-3) / 1e12 : -1;
        ms = time_launch(s, e0, e1, [&] { k_peak_ffma2<<<grid, blk, 0, s>>>(it32 / 2, a, b, sink); }, reps);
        out->fp32x2_tflops = ms > 0 ? 4.0 * threads * (it32 / 2) * kChains / (ms * 1e-3) / 1e12 : -1;
        ms = time_launch(s, e0, e1, [&] { k_peak_dfma<<<grid, blk, 0, s>>>(it64, ad, bd, sink); }, reps);
        out->fp64_tflops = ms > 0 ? 2.0 * threads * it64 * kChains / (ms * 1e-3) / 1e12 : -1;
        ms = time_launch(s, e0, e1, [&] { k_peak_int<<<grid, blk, 0, s>>>(itint, 0x9e3779b9u, 7u, sink); }, reps);
        out->int_tops = ms > 0 ? 2.0 * threads * itint * kChains / (ms * 1e-3) / 1e12 : -1;
        ms = time_launch(s, e0, e1, [&] { k_peak_f2f<<<grid, blk, 0, s>>>(itcvt, 1.0000001, sink); }, reps);
        out->cvt_tops = ms > 0 ? 2.0 * threads * itcvt * kChains / (ms * 1e-3) / 1e12 : -1;
        ms = time_launch(s, e0, e1, [&] { k_peak_mix<<<grid, blk, 0, s>>>(itmix, rf, a, b, ad, bd, sink); }, reps);
        // time of the mixed kernel against the sum of its parts run alone
        if (ms > 0 && out->fp32_tflops > 0 && out->fp64_tflops > 0) {
            const double t32 = 2.0 * threads * itmix * rf * kChains / (out->fp32_tflops * 1e12);
            const double t64 = 2.0 * threads * itmix * 2 / (out->fp64_tflops * 1e12);
            out->mix_overlap = (t32 + t64) / (ms * 1e-3);
        }
        if (cudaGetLastError() != cudaSuccess) st = HZS_ERR_CUDA;
    }
    out->sms = sms;
    out->clock_mhz = clk_khz / 1000.0;
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaGetLastError();
    return st;
}
