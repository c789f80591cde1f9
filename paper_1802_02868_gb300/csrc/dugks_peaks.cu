// dugks_peaks.cu -- arithmetic throughput of the GPU the library runs on, for
// the roofline of the fused step: FP32 FMAs (scalar and the packed two-lane
// form the step uses for its f/g pairs) and FP64 FMAs.
//
// Each thread runs 8 independent FMA chains for `iters` rounds, so that
// neither latency nor issue order limits the rate; a grid of 8 blocks of 256
// threads per SM keeps every scheduler busy.  The result of every chain feeds
// a store that only a value no chain can produce would trigger, so nothing is
// optimised away and nothing is written.  Rates are timed with CUDA events on
// the caller's stream around the second of two identical launches.
#include <cuda_runtime.h>

#include "../../include/dugks.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

__device__ float g_sink_f;
__device__ double g_sink_d;

__global__ void __launch_bounds__(kThreads) k_peak_f32(int iters, float m, float a)
{
    float v[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) v[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) v[k] = __fmaf_rn(v[k], m, a);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += v[k];
    if (s == -1.2345e30f) g_sink_f = s;
}

__global__ void __launch_bounds__(kThreads) k_peak_f32x2(int iters, float m, float a)
{
    float2 v[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) v[k] = make_float2((float)(threadIdx.x + k) * 1e-3f, (float)k * 1e-3f);
    const float2 mm = make_float2(m, m), aa = make_float2(a, a);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) v[k] = __ffma2_rn(v[k], mm, aa);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += v[k].x + v[k].y;
    if (s == -1.2345e30f) g_sink_f = s;
}

__global__ void __launch_bounds__(kThreads) k_peak_f64(int iters, double m, double a)
{
    double v[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) v[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) v[k] = __fma_rn(v[k], m, a);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += v[k];
    if (s == -1.2345e300) g_sink_d = s;
}

// flop of one launch: threads x chains x iterations x 2 (x 2 for the packed form)
template <typename K>
int time_kernel(K launch, cudaStream_t st, double flop, double *tflops)
{
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess) return DUGKS_ERR_CUDA;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return DUGKS_ERR_CUDA;
    }
    int rc = DUGKS_OK;
    launch();   // warm-up (clocks up, module loaded)
    cudaEventRecord(a, st);
    launch();
    cudaEventRecord(b, st);
    float ms = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
        cudaEventElapsedTime(&ms, a, b) != cudaSuccess || ms <= 0.f)
        rc = DUGKS_ERR_CUDA;
    else
        *tflops = flop / (ms * 1e-3) / 1e12;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return rc;
}

}  // namespace

extern "C" int dugks_measure_alu_peaks(int iters_f32, int iters_f64, double *fp32_tflops, double *fp32x2_tflops,
                                       double *fp64_tflops, void *cuda_stream)
{
    if (iters_f32 < 1 || iters_f64 < 1 || !fp32_tflops || !fp32x2_tflops || !fp64_tflops) return DUGKS_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return DUGKS_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int blocks = 8 * sms;
    const double threads = (double)blocks * kThreads;
    int rc = time_kernel([&] { k_peak_f32<<<blocks, kThreads, 0, st>>>(iters_f32, 0.999999f, 1e-7f); }, st,
                         threads * kChains * iters_f32 * 2.0, fp32_tflops);
    if (rc) return rc;
    rc = time_kernel([&] { k_peak_f32x2<<<blocks, kThreads, 0, st>>>(iters_f32 / 2, 0.999999f, 1e-7f); }, st,
                     threads * kChains * (iters_f32 / 2) * 4.0, fp32x2_tflops);
    if (rc) return rc;
    return time_kernel([&] { k_peak_f64<<<blocks, kThreads, 0, st>>>(iters_f64, 0.999999999, 1e-12); }, st,
                       threads * kChains * iters_f64 * 2.0, fp64_tflops);
}
