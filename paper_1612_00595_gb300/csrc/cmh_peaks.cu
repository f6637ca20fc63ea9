// Throughput of the two arithmetic units the float32 sweep leans on, measured
// on the device at hand: the special-function unit (MUFU: ex2, lg2, rcp, the
// per-sample logarithm, reciprocal and envelope exponential of the pricing)
// and the float32 FMA pipe.  They are the denominators of the roofline's
// arithmetic terms next to the measured HBM bandwidth.
//
// Each thread runs kChains independent dependency chains so that the pipes,
// not the latency of one chain, set the pace; the grid holds 8 CTAs of 256
// threads per SM.  The values stay bounded (ex2(lg2(y)) returns y, rcp
// toggles between z and 1/z, the FMA chain converges to 1) and are written to
// a device sink only if they take an impossible value, so no work is dropped.
#include <cuda_runtime.h>

#include "chromh.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kCtasPerSm = 8;

static __device__ float g_peak_sink;

__device__ __forceinline__ float ex2a(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2a(float x) {
    float y;
    asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcpa(float x) {
    float y;
    asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 3 MUFU operations per chain and iteration
__global__ void __launch_bounds__(kThreads) mufu_kernel(int iters) {
    float y[kChains], z[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        y[c] = 1.5f + 0.01f * (float)((threadIdx.x + c) & 15);
        z[c] = 1.25f + 0.01f * (float)c;
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            y[c] = ex2a(lg2a(y[c]));
            z[c] = rcpa(z[c]);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += y[c] + z[c];
    if (s == -1.f) g_peak_sink = s;
}

// 2 flops (one FMA) per chain and iteration
__global__ void __launch_bounds__(kThreads) fma_kernel(int iters) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = 0.5f + 0.001f * (float)(threadIdx.x & 7) + 0.01f * (float)c;
    const float b = 0.999f, k = 0.001f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = __fmaf_rn(a[c], b, k);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == -1.f) g_peak_sink = s;
}

// best of `reps` timed launches, in operations per second
template <typename L>
int time_best(L launch, double ops_per_launch, int reps, cudaStream_t st, double* out) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return CMH_ERR_CUDA;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return CMH_ERR_CUDA;
    }
    int rc = CMH_OK;
    double best = 0.0;
    launch();   // warm-up
    for (int r = 0; r < reps && rc == CMH_OK; ++r) {
        cudaEventRecord(a, st);
        launch();
        cudaEventRecord(b, st);
        if (cudaEventSynchronize(b) != cudaSuccess) {
            rc = CMH_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess || ms <= 0.f) {
            rc = CMH_ERR_CUDA;
            break;
        }
        const double v = ops_per_launch / (ms * 1e-3);
        if (v > best) best = v;
    }
    if (cudaGetLastError() != cudaSuccess) rc = CMH_ERR_CUDA;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *out = best;
    return rc;
}

}  // namespace

extern "C" int cmh_measure_alu_peaks(double* mufu_ops_per_s, double* fma_flops_per_s, void* cuda_stream) {
    if (!mufu_ops_per_s || !fma_flops_per_s) return CMH_ERR_ARG;
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CMH_ERR_CUDA;
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm < 1)
        return CMH_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int grid = n_sm * kCtasPerSm;
    const double threads = (double)grid * kThreads;
    const int it_mufu = 2048, it_fma = 8192;
    int rc = time_best([&] { mufu_kernel<<<grid, kThreads, 0, st>>>(it_mufu); },
                       threads * kChains * 3.0 * it_mufu, 3, st, mufu_ops_per_s);
    if (rc) return rc;
    return time_best([&] { fma_kernel<<<grid, kThreads, 0, st>>>(it_fma); },
                     threads * kChains * 2.0 * it_fma, 3, st, fma_flops_per_s);
}
