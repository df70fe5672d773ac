// Throughput ceilings of the two pipes the encoder-step kernels compute on, measured on the device
// the library runs on: the FP32 FMA pipe (SIMT) and the warp-level TF32 tensor-core MMA
// (mma.sync.m16n8k8), which carries the entropy model's and the synthesis adjoint's products.
// The roofline fractions the benchmark reports divide by these measured figures.
//
// Each kernel keeps many independent dependency chains per warp (8 per thread for the FMA pipe,
// 8 accumulators per warp for the MMA), fills every SM with resident warps and runs long enough
// (several milliseconds) for launch and tail effects to vanish.  The result is stored only when it
// equals a value it cannot take, so the compiler keeps the arithmetic and nothing is written.
#include <cuda_runtime.h>

#include "../../include/coolchic.h"
#include "cc_kernels.h"
#include "cc_mma.cuh"

namespace cc {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kFmaChains = 8, kFmaUnroll = 16;
constexpr int kMmaChains = 8;

__global__ void __launch_bounds__(kPeakThreads) k_peak_fma(float* sink, float never, int trips) {
    float a[kFmaChains];
#pragma unroll
    for (int j = 0; j < kFmaChains; ++j) a[j] = 1.f + 1e-6f * (float)(threadIdx.x + j);
    const float m = 0.9999999f, c = 1e-7f;
    for (int it = 0; it < trips; ++it) {
#pragma unroll
        for (int u = 0; u < kFmaUnroll; ++u)
#pragma unroll
            for (int j = 0; j < kFmaChains; ++j) a[j] = fmaf(a[j], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kFmaChains; ++j) s += a[j];
    if (s == never) sink[0] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_mma(float* sink, float never, int trips) {
    const uint32_t one = __float_as_uint(1.f);
    uint32_t a[4] = {one, one ^ ((threadIdx.x & 1u) << 13), one, one};
    const uint32_t b0 = one, b1 = one ^ ((threadIdx.x & 2u) << 12);
    float d[kMmaChains][4];
#pragma unroll
    for (int j = 0; j < kMmaChains; ++j) d[j][0] = d[j][1] = d[j][2] = d[j][3] = 0.f;
    for (int it = 0; it < trips; ++it) {
#pragma unroll
        for (int j = 0; j < kMmaChains; ++j) mma1(d[j], a, b0, b1);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kMmaChains; ++j) s += d[j][0] + d[j][1] + d[j][2] + d[j][3];
    if (s == never) sink[0] = s;
}

// FLOP of one launch at `trips` loop trips
double peak_flop(int which, int ctas, int trips) {
    const double threads = (double)ctas * kPeakThreads;
    if (which == CC_PEAK_FP32_FMA) return threads * trips * kFmaUnroll * kFmaChains * 2.0;
    return threads / 32.0 * trips * kMmaChains * (2.0 * 16 * 8 * 8);
}

cudaError_t peak_launch(int which, int ctas, int trips, float* sink, cudaStream_t s) {
    if (which == CC_PEAK_FP32_FMA)
        k_peak_fma<<<ctas, kPeakThreads, 0, s>>>(sink, -1.f, trips);
    else
        k_peak_mma<<<ctas, kPeakThreads, 0, s>>>(sink, -1.f, trips);
    return cudaGetLastError();
}

}  // namespace
}  // namespace cc

using namespace cc;

extern "C" int coolchic_measure_peak(int32_t which, float* sink, double* tflops_out, double* ms_out, void* stream) {
    if (which != CC_PEAK_FP32_FMA && which != CC_PEAK_TF32_MMA)
        return set_error(CC_ERR_ARG, "measure_peak: unknown pipe %d", which);
    if (!sink || !tflops_out) return set_error(CC_ERR_ARG, "measure_peak: NULL sink or tflops_out");
    if (const int rc = device_setup_checked()) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int ctas = num_sms() * (2048 / kPeakThreads);  // every SM full of resident warps
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaError_t e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    double best = 0.0, best_ms = 0.0;
    int trips = 256;
    // calibration: grow the trip count until one launch takes at least 2 ms, then time 3 launches
    for (int round = 0; e == cudaSuccess && round < 24; ++round) {
        e = peak_launch(which, ctas, trips, sink, s);  // warm
        if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
        if (e == cudaSuccess) e = peak_launch(which, ctas, trips, sink, s);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (e != cudaSuccess) break;
        if (ms < 2.f && trips < (1 << 24)) {
            trips *= (ms < 0.25f) ? 8 : 2;
            continue;
        }
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
            e = cudaEventRecord(ev[0], s);
            if (e == cudaSuccess) e = peak_launch(which, ctas, trips, sink, s);
            if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
            if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
            if (e == cudaSuccess && ms > 0.f) {
                const double tf = peak_flop(which, ctas, trips) / (ms * 1e-3) / 1e12;
                if (tf > best) {
                    best = tf;
                    best_ms = ms;
                }
            }
        }
        break;
    }
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
    if (e != cudaSuccess) return set_error(CC_ERR_CUDA, "measure_peak: %s", cudaGetErrorString(e));
    *tflops_out = best;
    if (ms_out) *ms_out = best_ms;
    return CC_OK;
}
