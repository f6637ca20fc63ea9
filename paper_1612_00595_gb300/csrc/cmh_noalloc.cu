// Gaussian log-likelihood of caller-owned device buffers, computed without
// allocating any device memory.
//
// Who needs this: code that must not call cudaMalloc -- a host application
// whose memory manager owns every byte of the GPU (a caching pool sized up
// front, where a stray cudaMalloc fails or fragments the pool), a monitoring
// hook that runs between someone else's kernels and must not trigger the
// implicit device synchronisation an allocation can cause, or a plugin loaded
// into a process that forbids allocations outside its framework.  Such a
// caller can still hand us device pointers to its signals and variances.
//
// The per-row partial sums live in one file-scope device array that every GPU
// loading this library keeps until the process exits (kMaxRows + 1 doubles,
// 64 KB).  Host code needs its device address, which cudaGetSymbolAddress
// returns; the first call on a device does that lookup and keeps the address.
// The address belongs to the device's context: if that context is destroyed
// and re-created (cudaDeviceReset), the next call sees a new context id and
// looks the address up again.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "chromh.h"

namespace {

constexpr int kMaxRows = 8191;        // rows (stations) one call may sum
constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;

// [kMaxRows] per-row sums, then the total
static __device__ __align__(256) double g_noalloc_scratch[kMaxRows + 1];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {nullptr};
unsigned long long g_scratch_ctx[kMaxDevices] = {0};   // context id the address belongs to

// the driver's cuCtxGetCurrent / cuCtxGetId, reached through the runtime (no
// link against libcuda); null if the driver does not offer them
typedef CUresult (*ctx_current_fn)(CUcontext*);
typedef CUresult (*ctx_id_fn)(CUcontext, unsigned long long*);
ctx_current_fn g_ctx_current = nullptr;
ctx_id_fn g_ctx_id = nullptr;
bool g_ctx_fns_tried = false;

// id of the current context, or 0 if it cannot be had
unsigned long long current_context_id() {
    if (!g_ctx_fns_tried) {
        g_ctx_fns_tried = true;
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            g_ctx_current = (ctx_current_fn)f1;
            g_ctx_id = (ctx_id_fn)f2;
        }
        cudaGetLastError();
    }
    if (!g_ctx_current || !g_ctx_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (g_ctx_current(&c) != CUDA_SUCCESS || !c) return 0;
    if (g_ctx_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

__device__ __forceinline__ double block_sum(double v, double* s_part) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_part[w];
    return t;
}

// one block per row: sum over samples of log N(s; 0, V)
template <bool F32>
__global__ void __launch_bounds__(kThreads) row_loglik(const void* sig, const void* var, long long n_samp,
                                                       long long pitch, double* scratch) {
    __shared__ double s_part[32];
    const double half_log_2pi = 0.91893853320467274178;
    const long long row = blockIdx.x;
    double acc = 0.0;
    for (long long k = threadIdx.x; k < n_samp; k += blockDim.x) {
        if (F32) {
            const float s = ((const float*)sig)[row * pitch + k];
            const float V = ((const float*)var)[row * pitch + k];
            acc += (double)(-0.5f * logf(V) - s * s / (2.f * V)) - half_log_2pi;
        } else {
            const double s = ((const double*)sig)[row * pitch + k];
            const double V = ((const double*)var)[row * pitch + k];
            acc += -half_log_2pi - 0.5 * log(V) - s * s / (2.0 * V);
        }
    }
    const double t = block_sum(acc, s_part);
    if (threadIdx.x == 0) scratch[row] = t;
}

// rows summed in a fixed order into scratch[kMaxRows]
__global__ void __launch_bounds__(1024) sum_rows(double* scratch, int n_rows) {
    __shared__ double s_part[32];
    double acc = 0.0;
    for (int r = threadIdx.x; r < n_rows; r += blockDim.x) acc += scratch[r];
    const double t = block_sum(acc, s_part);
    if (threadIdx.x == 0) scratch[kMaxRows] = t;
}

// device address of the scratch array for the current device: looked up on
// the first call with that device current, again whenever the device's
// context has changed since (a reset), and on every call if the context id
// cannot be read
int scratch_for_current_device(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CMH_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return CMH_ERR_ARG;
    if (cudaSetDevice(dev) != cudaSuccess) return CMH_ERR_CUDA;   // makes the device's context current
    std::lock_guard<std::mutex> lock(g_mu);
    const unsigned long long ctx = current_context_id();
    if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return CMH_ERR_CUDA;
        g_scratch_addr[dev] = (double*)p;
        g_scratch_ctx[dev] = ctx;
    }
    *out = g_scratch_addr[dev];
    return CMH_OK;
}

}  // namespace

extern "C" int cmh_gaussian_loglik_noalloc(const void* signals, const void* variance, int32_t n_rows,
                                           int64_t n_samples, int64_t row_pitch, cmh_dtype dtype, double* out,
                                           void* cuda_stream) {
    if (!out || n_rows < 0 || n_samples < 1 || row_pitch < n_samples || (dtype != CMH_F32 && dtype != CMH_F64))
        return CMH_ERR_ARG;
    if (n_rows > kMaxRows) return CMH_ERR_CAPACITY;
    if (n_rows == 0) {
        *out = 0.0;
        return CMH_OK;
    }
    if (!signals || !variance) return CMH_ERR_ARG;
    double* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (dtype == CMH_F32)
        row_loglik<true><<<n_rows, kThreads, 0, s>>>(signals, variance, n_samples, row_pitch, scratch);
    else
        row_loglik<false><<<n_rows, kThreads, 0, s>>>(signals, variance, n_samples, row_pitch, scratch);
    sum_rows<<<1, 1024, 0, s>>>(scratch, n_rows);
    if (cudaGetLastError() != cudaSuccess) return CMH_ERR_CUDA;
    if (cudaMemcpyAsync(out, scratch + kMaxRows, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return CMH_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CMH_ERR_CUDA;
    return CMH_OK;
}
