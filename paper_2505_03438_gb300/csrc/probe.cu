// probe.cu -- throughput probes of the arithmetic pipes the force and update
// kernels use: FP32 fused multiply-add (scalar and packed FP32x2), FP64
// fused multiply-add and the approximate FP32 reciprocal.  Each probe runs
// independent dependency chains in every thread of a grid that fills every
// SM, so the pipe, not latency, sets the rate; it is timed with CUDA events
// after one warm-up launch, and its iteration count is scaled so that the
// timed launch lasts about the requested time.  These are the peaks the
// rooflines of the force (FP32) and update (FP64) kernels are measured
// against.
#include <cstring>
#include <string>

#include "kernels.cuh"
#include "system.h"

namespace ljsel {
namespace {

constexpr int PR_THREADS = 256;
constexpr int PR_CHAINS = 8;

__global__ void __launch_bounds__(PR_THREADS) k_probe_ffma(float *out, int iters, float a, float b) {
    float acc[PR_CHAINS];
#pragma unroll
    for (int k = 0; k < PR_CHAINS; ++k) acc[k] = threadIdx.x * 1e-3f + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PR_CHAINS; ++k) acc[k] = fmaf(acc[k], a, b);
    }
    float sum = 0.f;
#pragma unroll
    for (int k = 0; k < PR_CHAINS; ++k) sum += acc[k];
    if (sum == 1234.5f) out[blockIdx.x] = sum;  // keeps the chains alive
}

__global__ void __launch_bounds__(PR_THREADS) k_probe_ffma2(float *out, int iters, float a, float b) {
    float2 acc[PR_CHAINS];
#pragma unroll
    for (int k = 0; k < PR_CHAINS; ++k) acc[k] = make_float2(threadIdx.x * 1e-3f + k, k - threadIdx.x * 1e-3f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PR_CHAINS; ++k) acc[k] = __ffma2_rn(acc[k], a2, b2);
    }
    float sum = 0.f;
#pragma unroll
    for (int k = 0; k < PR_CHAINS; ++k) sum += acc[k].x + acc[k].y;
    if (sum == 1234.5f) out[blockIdx.x] = sum;
}

__global__ void __launch_bounds__(PR_THREADS) k_probe_dfma(double *out, int iters, double a, double b) {
    double acc[PR_CHAINS];
#pragma unroll
    for (int k = 0; k < PR_CHAINS; ++k) acc[k] = threadIdx.x * 1e-3 + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PR_CHAINS; ++k) acc[k] = fma(acc[k], a, b);
    }
    double sum = 0.0;
#pragma unroll
    for (int k = 0; k < PR_CHAINS; ++k) sum += acc[k];
    if (sum == 1234.5) out[blockIdx.x] = sum;
}

// x -> 1 / x + c stays bounded for c > 0; one MUFU reciprocal and one FP32
// add per step (the add runs on the FMA pipe, eight times wider).
__global__ void __launch_bounds__(PR_THREADS) k_probe_rcp(float *out, int iters, float c) {
    float acc[PR_CHAINS];
#pragma unroll
    for (int k = 0; k < PR_CHAINS; ++k) acc[k] = 1.0f + threadIdx.x * 1e-3f + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PR_CHAINS; ++k) acc[k] = fast_rcp(acc[k]) + c;
    }
    float sum = 0.f;
#pragma unroll
    for (int k = 0; k < PR_CHAINS; ++k) sum += acc[k];
    if (sum == 1234.5f) out[blockIdx.x] = sum;
}

}  // namespace
}  // namespace ljsel

using namespace ljsel;

extern "C" ljsel_status ljsel_measure_peaks(double target_ms, ljsel_peaks *out) {
    set_error("");
    if (!out || !(target_ms > 0) || target_ms > 10000) { set_error("out required, 0 < target_ms <= 10000"); return LJSEL_ERR_ARG; }
    memset(out, 0, sizeof(*out));
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        set_error("no CUDA device");
        return LJSEL_ERR_CUDA;
    }
    const int blocks = nsm * 8;
    const double threads = (double)blocks * PR_THREADS;
    Buf scratch;
    ljsel_status st = scratch.ensure((size_t)blocks * sizeof(double));
    if (st != LJSEL_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto timed = [&](auto launch, int iters, double *ms) -> bool {
        cudaEventRecord(e0, 0);
        launch(iters);
        cudaEventRecord(e1, 0);
        if (cudaEventSynchronize(e1) != cudaSuccess) return false;
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        *ms = t;
        return cudaGetLastError() == cudaSuccess;
    };
    // rate (operations per second) of one probe: a short launch to warm up
    // and calibrate, then one of about target_ms
    auto rate = [&](auto launch, double ops_per_iter_thread, double *res) -> bool {
        double ms = 0;
        int iters = 1024;
        if (!timed(launch, iters, &ms)) return false;
        for (int k = 0; k < 8 && ms < 0.05 * target_ms && iters < (1 << 26); ++k) {
            iters *= 8;
            if (!timed(launch, iters, &ms)) return false;
        }
        const double scale = target_ms / (ms > 1e-3 ? ms : 1e-3);
        const double it = (double)iters * scale;
        iters = (int)(it > 2e9 ? 2e9 : (it < 1024 ? 1024 : it));
        if (!timed(launch, iters, &ms)) return false;
        *res = threads * (double)iters * ops_per_iter_thread / (ms * 1e-3);
        return true;
    };
    float *fo = (float *)scratch.ptr;
    double *dout = (double *)scratch.ptr;
    double r = 0;
    bool ok = true;
    ok = ok && rate([&](int it) { k_probe_ffma<<<blocks, PR_THREADS>>>(fo, it, 0.9999999f, 1e-7f); }, 2.0 * PR_CHAINS, &r);
    out->fp32_tflops = r * 1e-12;
    ok = ok && rate([&](int it) { k_probe_ffma2<<<blocks, PR_THREADS>>>(fo, it, 0.9999999f, 1e-7f); }, 4.0 * PR_CHAINS, &r);
    out->fp32x2_tflops = r * 1e-12;
    ok = ok && rate([&](int it) { k_probe_dfma<<<blocks, PR_THREADS>>>(dout, it, 0.9999999999, 1e-10); }, 2.0 * PR_CHAINS, &r);
    out->fp64_tflops = r * 1e-12;
    ok = ok && rate([&](int it) { k_probe_rcp<<<blocks, PR_THREADS>>>(fo, it, 0.5f); }, 1.0 * PR_CHAINS, &r);
    out->rcp_tops = r * 1e-12;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    scratch.release();
    if (!ok) {
        set_error(std::string("a probe launch failed: ") + cudaGetErrorString(cudaGetLastError()));
        return LJSEL_ERR_CUDA;
    }
    return LJSEL_OK;
}
