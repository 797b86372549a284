// k_peaks.cu -- arithmetic-rate probes for the roofline denominators of the
// ALU-bound kernels (no counterpart in the paper).
//
// Each probe runs independent dependency chains (enough per thread to hide
// the pipe latency) on every SM and counts the operations it issues:
//   0: packed FP32 FMA (FFMA2, 4 flops per lane and instruction),
//   1: MUFU sine (sin.approx.f32, 1 operation per lane),
//   2: FP64 FMA (2 flops per lane).
// The result is operations per second over the timed launch (CUDA events on
// the given stream, after an untimed warm-up launch).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/bem.h"
#include "pair_math.h"

namespace gbem {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;

__global__ void __launch_bounds__(PK_THREADS) peak_ffma2_kernel(int iters, float seed, float* out) {
    f2 a[PK_CHAINS];
    const f2 m = make_float2(0.9999f, 1.0001f), c = make_float2(1e-7f, -1e-7f);
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) a[k] = make_float2(seed + k + threadIdx.x * 1e-3f, seed - k);
    for (int i = 0; i < iters; i++)
#pragma unroll
        for (int u = 0; u < 16; u++)
#pragma unroll
            for (int k = 0; k < PK_CHAINS; k++) a[k] = fma2(a[k], m, c);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) s += a[k].x + a[k].y;
    if (s == 1234.5f) out[0] = s;  // keeps the chains live
}

__global__ void __launch_bounds__(PK_THREADS) peak_mufu_kernel(int iters, float seed, float* out) {
    float a[PK_CHAINS];
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) a[k] = seed + k + threadIdx.x * 1e-3f;
    for (int i = 0; i < iters; i++)
#pragma unroll
        for (int u = 0; u < 16; u++)
#pragma unroll
            for (int k = 0; k < PK_CHAINS; k++) {
                float y;
                asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[k]));
                a[k] = y;
            }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) s += a[k];
    if (s == 1234.5f) out[0] = s;
}

__global__ void __launch_bounds__(PK_THREADS) peak_dfma_kernel(int iters, double seed, float* out) {
    double a[PK_CHAINS];
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) a[k] = seed + k + threadIdx.x * 1e-3;
    for (int i = 0; i < iters; i++)
#pragma unroll
        for (int u = 0; u < 16; u++)
#pragma unroll
            for (int k = 0; k < PK_CHAINS; k++) a[k] = fma(a[k], 0.9999999, 1e-9);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) s += a[k];
    if (s == 1234.5) out[0] = (float)s;
}

}  // namespace gbem

using namespace gbem;

// Rate of probe `which` on the current device: *ops_per_s receives flops/s
// (which 0, 2) or operations/s (which 1).  iters scales the work (each
// thread runs iters x 16 x 8 chained operations); the grid is 16 CTAs of 256
// threads per SM.  Errors: INVALID_ARG, CUDA.
extern "C" int bem_peak_probe(int which, int iters, void* cuda_stream, double* ops_per_s) {
    if (which < 0 || which > 2 || iters < 1 || !ops_per_s) return BEM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return BEM_ERR_CUDA;
    float* sink = nullptr;
    if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess) return BEM_ERR_CUDA;
    const unsigned grid = (unsigned)n_sm * 16;
    auto launch = [&](int it) {
        if (which == 0) peak_ffma2_kernel<<<grid, PK_THREADS, 0, st>>>(it, 1.0f, sink);
        else if (which == 1) peak_mufu_kernel<<<grid, PK_THREADS, 0, st>>>(it, 0.5f, sink);
        else peak_dfma_kernel<<<grid, PK_THREADS, 0, st>>>(it, 1.0, sink);
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = BEM_OK;
    float ms = 0.f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = BEM_ERR_CUDA;
    if (!rc) {
        launch(std::max(1, iters / 8));  // warm-up
        cudaEventRecord(e0, st);
        launch(iters);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f))
            rc = BEM_ERR_CUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (rc) return rc;
    const double per_lane_op = which == 0 ? 4.0 : which == 1 ? 1.0 : 2.0;
    const double ops = (double)grid * PK_THREADS * iters * 16.0 * PK_CHAINS * per_lane_op;
    *ops_per_s = ops / (ms * 1e-3);
    return BEM_OK;
}
